"""The C-ABI library loads, exports every entry point that the headers in
include/ declare, and its host-only logic agrees with the oracle.  No device compute
runs here (these tests pass on a machine without a GPU)."""
import ctypes as C
import glob
import math
import os
import re
import subprocess

import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_symbols():
    txt = "\n".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"^RS_API\s+[\w\s\*]*?\b(rs_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("rs_make_lenses", "rs_shoot_map", "rs_magnification", "rs_lens_count",
                 "rs_shoot_tiles", "rs_last_error", "rs_shoot_map_host"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_1406_0559_b300 as rs
    path = rs.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(rs_\w+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    # nothing beyond the declared surface leaks out
    extra = sorted(s for s in exported if s not in declared_symbols())
    assert not extra, extra
    lib = rs.lib()
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_checked_build_exports_the_same_symbols():
    """The bounds-checked build (RS_CHECKED) is the same library with checked
    map writes: it loads without a GPU and exports exactly the declared entry
    points."""
    import paper_1406_0559_b300 as rs
    import paper_1406_0559_b300.build as B
    assert os.path.exists(B.LIB_CHECKED)
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_CHECKED], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(rs_\w+)$", out, flags=re.M))
    assert exported == set(declared_symbols())
    assert rs.checked_library() is not rs.lib()


def test_version_and_no_error():
    import paper_1406_0559_b300 as rs
    assert "sm_103a" in rs.version()


def test_lens_count_matches_oracle_eq3():
    import paper_1406_0559_b300 as rs
    for ks, R, mm in [(0.6, 200.0, 1.0), (0.4, 280.0, 1.0), (0.4, 11.0, 1.0),
                      (0.3, 10.0, 0.5), (0.0, 5.0, 1.0), (1.2, 123.4, 0.3)]:
        assert rs.lens_count(ks, R, mm) == oracle.lens_count(ks, R, mm)
    with pytest.raises(rs.RSError) as e:
        rs.lens_count(-1.0, 10.0)
    assert e.value.code == -1


def test_navg_matches_oracle():
    import paper_1406_0559_b300 as rs
    for j in (W.PARITY, W.GERLUMPH, W.PRECISION, W.PARITY.with_(n1=1000, n2=777, half2=3.3)):
        assert rs.navg(j) == oracle.navg(j)


def test_tile_shapes():
    import paper_1406_0559_b300 as rs
    for prec in (rs.PREC_FP32, rs.PREC_COMPENSATED):
        tx, ty = rs.tile_shape(prec)
        assert tx % 16 == 0 and ty % 16 == 0
        for shape in range(1, 20):
            tx, ty = rs.tile_shape(prec, shape)
            assert tx > 0 and ty > 0
    assert rs.tile_shape(2) == rs.tile_shape(1)          # double-single: default shape
    assert rs.tile_shape(3) == rs.tile_shape(1)          # refined: default shape
    # the refined form's candidates share the default tile; their sums fold
    # every 24 or 48 lenses, within the error bound's 48
    for shape in rs.tune_candidates(rs.PREC_REFINED):
        assert rs.tile_shape(3, shape) == rs.tile_shape(1)
        fold, unroll = rs.shape_sum(3, shape)
        assert fold in (24, 48) and unroll in (2, 4, 8)
    assert rs.shape_sum(3) == (48, 8) and rs.shape_sum(1) == (24, 2)
    assert rs.tune_candidates(rs.PREC_DOUBLE_SINGLE) == [12]
    assert 28 in rs.tune_candidates(rs.PREC_COMPENSATED)
    with pytest.raises(rs.RSError):
        rs.tile_shape(2, 1)
    with pytest.raises(rs.RSError):
        rs.tile_shape(3, 2)
    with pytest.raises(rs.RSError):
        rs.tile_shape(7)
    with pytest.raises(rs.RSError):
        rs.tile_shape(0, 99)


def test_argument_errors_are_caught_before_any_launch():
    import paper_1406_0559_b300 as rs
    L = rs.lib()
    mc = rs.Macro(0.0, 0.3)
    g = rs.RayGrid(0, 0, 1.0, 1.0, 16, 16)
    mp = rs.MapSpec(0, 0, 1.0, 8)
    st = (C.c_int64 * 8)()
    cnt = (C.c_int32 * 64)()
    # negative ray count, zero width, npix too large, bad precision
    bad_g = rs.RayGrid(0, 0, 1.0, 1.0, -1, 16)
    assert L.rs_shoot_map(C.byref(mc), None, 0, C.byref(bad_g), C.byref(mp), None,
                          C.cast(cnt, C.c_void_p), C.cast(st, C.c_void_p), None) == -1
    bad_m = rs.MapSpec(0, 0, 0.0, 8)
    assert L.rs_shoot_map(C.byref(mc), None, 0, C.byref(g), C.byref(bad_m), None,
                          C.cast(cnt, C.c_void_p), C.cast(st, C.c_void_p), None) == -1
    big_m = rs.MapSpec(0, 0, 1.0, 50000)
    assert L.rs_shoot_map(C.byref(mc), None, 0, C.byref(g), C.byref(big_m), None,
                          C.cast(cnt, C.c_void_p), C.cast(st, C.c_void_p), None) == -6
    huge = rs.RayGrid(0, 0, 1.0, 1.0, 1 << 20, 1 << 20)
    assert L.rs_shoot_map(C.byref(mc), None, 0, C.byref(huge), C.byref(mp), None,
                          C.cast(cnt, C.c_void_p), C.cast(st, C.c_void_p), None) == -6
    o = rs.Options(5, 0, 0, 0)
    assert L.rs_shoot_map(C.byref(mc), None, 0, C.byref(g), C.byref(mp), C.byref(o),
                          C.cast(cnt, C.c_void_p), C.cast(st, C.c_void_p), None) == -1
    assert b"precision" in L.rs_last_error()
    # host buffers where device buffers are required: refused, not launched
    assert L.rs_shoot_map(C.byref(mc), None, 0, C.byref(g), C.byref(mp), None,
                          C.cast(cnt, C.c_void_p), C.cast(st, C.c_void_p), None) == -1
    assert L.rs_shoot_map(C.byref(mc), None, 0, None, C.byref(mp), None,
                          C.cast(cnt, C.c_void_p), C.cast(st, C.c_void_p), None) == -1


def test_profile_half_matches_oracle():
    """Kernel extent (host-only in the library) agrees with the oracle's
    definition for every profile family, sample count and pixel size."""
    import paper_1406_0559_b300 as rs
    for kind in W.PROFILE_KINDS:
        for size_cm in (2e14, 5e14, 3e15, 1e16, 5e16):
            for S in (1, 2, 3, 8, 64):
                prof = W.profile_from_cm(kind, size_cm, supersample=S)
                for w in (0.0025, 24 / 4096, 0.01, 2.0 ** -9):
                    assert rs.profile_half(prof, w) == oracle.profile_half(prof, w)
    with pytest.raises(rs.RSError) as e:
        rs.profile_half(W.Profile(type=W.PROFILE_THIN_DISC, r_out=0.1, r_scale=0.01), 0.01)
    assert e.value.code == -1


def test_header_constants_match_the_binding():
    """Precision codes, the refined form's bound constants and the statistics
    layout: include/rs.h and the binding."""
    import re
    import paper_1406_0559_b300 as rs
    h = open(os.path.join(ROOT, "include", "rs.h")).read()
    consts = dict(re.findall(r"#define (RS_PREC_\w+|RS_REFINE_\w+|RS_NSTATS|RS_STAT_\w+)\s+([0-9.]+)", h))
    assert int(consts["RS_PREC_FP32"]) == rs.PREC_FP32
    assert int(consts["RS_PREC_COMPENSATED"]) == rs.PREC_COMPENSATED
    assert int(consts["RS_PREC_DOUBLE_SINGLE"]) == rs.PREC_DOUBLE_SINGLE
    assert int(consts["RS_PREC_REFINED"]) == rs.PREC_REFINED
    assert float(consts["RS_REFINE_K"]) == rs.REFINE_K
    assert float(consts["RS_REFINE_CB"]) == rs.REFINE_CB
    assert float(consts["RS_REFINE_CL"]) == rs.REFINE_CL
    assert int(consts["RS_REFINE_NEAR_CAP"]) == rs.REFINE_NEAR_CAP
    assert int(consts["RS_NSTATS"]) == rs.NSTATS
    for name in ("IN", "OUT", "NONFINITE", "REFINED", "EXACT", "OVERFLOW", "BAND_USE", "MAX_DELTA"):
        assert int(consts["RS_STAT_" + name]) == getattr(rs, "STAT_" + name)
    # the Hoeffding tail the header states for K
    assert 2 * math.exp(-rs.REFINE_K ** 2 / 2) < 5.5e-7


def test_server_config_errors_are_caught_before_any_device_work():
    """rs_server_create checks its whole configuration before it touches the
    device, so every refusal is visible without a GPU."""
    import paper_1406_0559_b300 as rs
    L = rs.lib()
    h = C.c_void_p()

    def cfg(**kw):
        d = dict(hbm_budget=1 << 30, slice_ms=20.0, rate_gint=5000.0, max_active=64,
                 max_queue=16, policy=rs.SCHED_SRPT, precision=rs.PREC_COMPENSATED, shape=0,
                 threaded=0, max_skips=4, inject_alloc_failures=0)
        d.update(kw)
        return rs.ServerConfig(**d)

    assert L.rs_server_create(None, C.byref(h)) == -1
    cases = [({"hbm_budget": 0}, b"hbm_budget"), ({"max_active": 0}, b"max_active"),
             ({"max_active": 129}, b"max_active"), ({"max_queue": 0}, b"max_queue"),
             ({"policy": 7}, b"policy"), ({"precision": 9}, b"precision"),
             ({"shape": 999}, b"shape"),
             ({"precision": rs.PREC_REFINED, "shape": 2}, b"no refined kernels"),
             ({"precision": rs.PREC_DOUBLE_SINGLE, "shape": 2}, b"default shape"),
             ({"shape": 2}, b"batched kernel")]
    for kw, word in cases:
        c = cfg(**kw)
        assert L.rs_server_create(C.byref(c), C.byref(h)) == -1, kw
        assert word in L.rs_last_error(), (kw, L.rs_last_error())
        assert h.value is None


def test_batch_argument_errors_are_caught_before_any_launch():
    """rs_shoot_batch checks every job before its first launch; an empty
    batch is a no-op."""
    import paper_1406_0559_b300 as rs
    L = rs.lib()
    mc = rs.Macro(0.0, 0.3)
    g = rs.RayGrid(0, 0, 1.0, 1.0, 16, 16)
    mp = rs.MapSpec(0, 0, 1.0, 8)
    cnt = (C.c_int32 * 64)()
    st = (C.c_int64 * 8)()
    jobs = (rs.Job * 2)()
    for j in jobs:
        j.macro, j.d_lens, j.n_lens, j.grid, j.map = mc, None, 0, g, mp
        j.d_counts, j.d_stats, j.d_mu = C.cast(cnt, C.c_void_p), C.cast(st, C.c_void_p), None

    def call(n, js, opt=None):
        return L.rs_shoot_batch(js, n, C.byref(opt) if opt is not None else None, None)

    assert call(-1, jobs) == -1 and b"n_jobs" in L.rs_last_error()
    assert call(1, None) == -1 and b"NULL" in L.rs_last_error()
    assert call(0, jobs) == 0
    assert call(1, jobs, rs.Options(9, 0, 0, 0)) == -1 and b"precision" in L.rs_last_error()
    assert call(1, jobs, rs.Options(rs.PREC_REFINED, 0, 2, 0)) == -1
    assert b"no refined kernels" in L.rs_last_error()
    # host buffers where device buffers are required: refused, not launched
    assert call(2, jobs) == -1 and b"d_counts" in L.rs_last_error()
    bad = (rs.Job * 1)()
    bad[0].macro, bad[0].grid, bad[0].map = mc, rs.RayGrid(0, 0, 1.0, 1.0, -1, 16), mp
    assert call(1, bad) == -1 and b"ray counts" in L.rs_last_error()

"""The bounds-checked build (librs_b300_checked.so, RS_CHECKED), the stand-in
for compute-sanitizer on this pool: its shoot kernels check every count-map
and binning-window index before writing, count and skip any out of range.
Small maps of every kernel family (ragged grids, rays far outside the map,
rays on lenses, the window binning shape, the refined form's three passes,
Salpeter masses) run through it: no write is out of range, and every map
equals the normal library's, bit for bit."""
import ctypes as C

import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_1406_0559_b300 as rs
    return rs


def shoot_with(rs, L, job, lens, precision, shape=0):
    counts = torch.empty((job.npix, job.npix), dtype=torch.int32, device="cuda")
    stats = torch.empty(rs.NSTATS, dtype=torch.int64, device="cuda")
    mc, g, mp = rs.structs(job)
    unit = getattr(job, "mass_model", rs.MASS_SALPETER) == rs.MASS_UNIT
    o = rs.options(precision, unit, shape)
    rc = L.rs_shoot_map(C.byref(mc), C.c_void_p(lens.data_ptr()), lens.numel() // 3, C.byref(g),
                        C.byref(mp), C.byref(o), C.c_void_p(counts.data_ptr()),
                        C.c_void_p(stats.data_ptr()), None)
    assert rc == 0, L.rs_last_error()
    torch.cuda.synchronize()
    return counts, stats


CASES = [
    (W.PARITY.with_(n1=1000, n2=777), 1, 0),                      # ragged tiles
    (W.PARITY.with_(n1=1000, n2=777), 3, 0),                      # refined: three passes
    (W.PARITY.with_(n1=1000, n2=777), 0, 0),                      # plain FP32
    (W.PARITY.with_(n1=600, n2=600, half1=40.0, half2=40.0), 1, 27),   # window binning
    (W.scaled(W.PRECISION, ray_scale=16, map_scale=16, lens_scale=50), 3, 0),   # Salpeter
    (W.PARITY.with_(n1=512, n2=512, width=0.5), 3, 0),            # most rays outside the map
]


@pytest.mark.parametrize("job,precision,shape", CASES,
                         ids=["ragged", "refined", "fp32", "window", "salpeter", "outside"])
def test_checked_build_writes_in_range_and_matches(rs, job, precision, shape):
    Lc = rs.checked_library()
    assert rs.checked_violations(Lc)[0] is True          # built with the checks
    assert rs.checked_violations() == (False, 0)         # the normal library has none
    lens = rs.make_lenses(job)
    c, st = rs.shoot_map(job, lens, precision=precision, shape=shape)
    cc, sc = shoot_with(rs, Lc, job, lens, precision, shape)
    built, bad = rs.checked_violations(Lc)
    assert bad == 0
    assert torch.equal(c, cc)
    assert torch.equal(st[:rs.STAT_BAND_USE], sc[:rs.STAT_BAND_USE])

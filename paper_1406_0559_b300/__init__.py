"""B300-native direct inverse ray-shooting (Vernardos & Fluke 2014, Sec. 2.1).

Python binding of the C ABI in ``include/rs.h`` (``librs_b300.so``).  This
module only marshals arguments: PyTorch supplies device memory and streams,
and every step of the computation runs in the library's CUDA kernels.  There
is no CPU fallback: importing this module without the built library, or with
a library built from other sources, raises.

A "job" is any object with the attributes of ``workloads.MapJob``
(kappa_star, kappa_s, gamma, n_lens, lens_radius, mass_model, m_lo, m_hi,
slope, seed, n1, n2, c1, c2, half1, half2, mc1, mc2, width, npix).
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

__all__ = ["RSError", "lens_count", "navg", "make_lenses", "shoot_map", "shoot_tiles",
           "shoot_tiles_band",
           "tile_shape", "magnification", "shoot_map_host", "library_path",
           "PREC_FP32", "PREC_COMPENSATED", "PREC_DOUBLE_SINGLE", "PREC_REFINED", "MASS_UNIT",
           "MASS_SALPETER"]

PREC_FP32 = 0
PREC_COMPENSATED = 1
PREC_DOUBLE_SINGLE = 2
PREC_REFINED = 3        # compensated, rays within their error bound of a pixel edge
                        # redone in double-single
REFINE_K = 5.5          # the refined form's error bound (include/rs.h, RS_REFINE_*)
REFINE_CB = 6.75
REFINE_CL = 60.5
REFINE_NEAR_CAP = 64
NSTATS = 8              # shoot statistics, RS_STAT_* order:
STAT_IN, STAT_OUT, STAT_NONFINITE, STAT_REFINED, STAT_EXACT, STAT_OVERFLOW, STAT_BAND_USE, \
    STAT_MAX_DELTA = range(8)
MASS_UNIT = 0
MASS_SALPETER = 1

RS_OK = 0
STATUS_NAMES = {0: "RS_OK", -1: "RS_EINVAL", -2: "RS_ENOMEM", -3: "RS_ECUDA",
                -4: "RS_ETIMEOUT", -5: "RS_EBUSY", -6: "RS_ERANGE"}


class RSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Macro(C.Structure):
    _fields_ = [("kappa_s", C.c_double), ("gamma", C.c_double)]


class RayGrid(C.Structure):
    _fields_ = [("c1", C.c_double), ("c2", C.c_double), ("half1", C.c_double),
                ("half2", C.c_double), ("n1", C.c_int64), ("n2", C.c_int64)]


class MapSpec(C.Structure):
    _fields_ = [("c1", C.c_double), ("c2", C.c_double), ("width", C.c_double),
                ("npix", C.c_int64)]


class LensField(C.Structure):
    _fields_ = [("kappa_star", C.c_double), ("radius", C.c_double),
                ("mass_model", C.c_int32), ("reserved", C.c_int32),
                ("m_lo", C.c_double), ("m_hi", C.c_double), ("slope", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("unit_mass", C.c_int32),
                ("shape", C.c_int32), ("accumulate", C.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python paper_1406_0559_b300/build.py` "
                          "(there is no CPU fallback)")
    with open(_build.HASH) as fh:
        built = fh.read().strip()
    if built != _build.source_hash():
        raise ImportError(f"{path} was built from other sources: rebuild it with "
                          "`python paper_1406_0559_b300/build.py`")
    _lib = _declare_core(C.CDLL(path))
    return _lib


_lib_checked = None


def checked_library():
    """The bounds-checked build (librs_b300_checked.so, RS_CHECKED): the same
    library whose shoot kernels check every count-map and window index before
    writing; a ctypes handle with the core entry points declared.  Its
    rs_checked_violations reports the out-of-range writes it skipped."""
    global _lib_checked
    if _lib_checked is None:
        _load()                              # the hash check covers both builds
        if not os.path.exists(_build.LIB_CHECKED):
            raise ImportError(f"{_build.LIB_CHECKED} is missing: rebuild with "
                              "`python paper_1406_0559_b300/build.py`")
        _lib_checked = _declare_core(C.CDLL(_build.LIB_CHECKED))
    return _lib_checked


def checked_violations(L=None) -> tuple[bool, int]:
    """(built with RS_CHECKED, out-of-range writes skipped since the last
    call) of the library L (default: the normal one)."""
    n = C.c_int64()
    rc = (L or lib()).rs_checked_violations(C.byref(n))
    if rc < 0:
        _check(rc)
    return rc == 1, n.value


def _declare_core(L):
    P = C.POINTER
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    L.rs_version.restype = C.c_char_p
    L.rs_version.argtypes = []
    L.rs_last_error.restype = C.c_char_p
    L.rs_last_error.argtypes = []
    L.rs_lens_count.argtypes = [dbl, dbl, dbl, P(i64)]
    L.rs_navg.argtypes = [P(RayGrid), P(MapSpec), P(dbl)]
    L.rs_make_lenses.argtypes = [P(LensField), C.c_uint64, vp, i64, vp]
    L.rs_shoot_map.argtypes = [P(Macro), vp, i64, P(RayGrid), P(MapSpec), P(Options), vp, vp, vp]
    L.rs_tile_shape.argtypes = [P(Options), P(i64), P(i64)]
    L.rs_shoot_map_range.argtypes = [P(Macro), vp, i64, P(RayGrid), P(MapSpec), P(Options), i64,
                                     i64, vp, vp, P(i64), vp]
    L.rs_shape_sum.argtypes = [P(Options), P(i32), P(i32)]
    L.rs_shoot_tiles.argtypes = [P(Macro), vp, i64, P(RayGrid), P(MapSpec), P(Options), vp, i64,
                                 vp, vp, vp]
    L.rs_magnification.argtypes = [vp, P(RayGrid), P(MapSpec), vp, vp]
    L.rs_debug_rays.argtypes = [P(Macro), vp, i64, P(RayGrid), P(MapSpec), P(Options), vp, i64,
                                vp, vp, vp]
    L.rs_shoot_tiles_band.argtypes = [P(Macro), vp, i64, P(RayGrid), P(MapSpec), P(Options), vp,
                                      i64, vp, vp, vp]
    L.rs_shoot_map_host.argtypes = [P(Macro), vp, i64, P(RayGrid), P(MapSpec), P(Options), vp, vp,
                                    vp]
    for name in ("rs_lens_count", "rs_navg", "rs_make_lenses", "rs_shoot_map", "rs_tile_shape",
                 "rs_shape_sum", "rs_shoot_map_range", "rs_shoot_tiles", "rs_magnification", "rs_shoot_map_host", "rs_debug_rays",
                 "rs_shoot_tiles_band", "rs_checked_violations"):
        getattr(L, name).restype = C.c_int
    L.rs_checked_violations.argtypes = [P(i64)]
    return L


def lib():
    return _load()


def _check(rc: int):
    if rc != RS_OK:
        raise RSError(rc, lib().rs_last_error().decode())


def version() -> str:
    return lib().rs_version().decode()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def structs(job):
    mc = Macro(job.kappa_s, job.gamma)
    g = RayGrid(job.c1, job.c2, job.half1, job.half2, job.n1, job.n2)
    mp = MapSpec(job.mc1, job.mc2, job.width, job.npix)
    return mc, g, mp


def options(precision: int = PREC_COMPENSATED, unit_mass: bool = False, shape: int = 0,
            accumulate: bool = False) -> Options:
    return Options(precision, int(bool(unit_mass)), shape, int(bool(accumulate)))


# ---------------------------------------------------------------- API -----

def lens_count(kappa_star: float, radius: float, mean_mass: float = 1.0) -> int:
    """Eq. 3 with A = pi R^2."""
    n = C.c_int64()
    _check(lib().rs_lens_count(kappa_star, radius, mean_mass, C.byref(n)))
    return n.value


def navg(job) -> float:
    """Eq. 4 normalisation: rays per pixel without lensing."""
    _, g, mp = structs(job)
    v = C.c_double()
    _check(lib().rs_navg(C.byref(g), C.byref(mp), C.byref(v)))
    return v.value


def job_lens_count(job) -> int:
    return job.n_lens if job.n_lens > 0 else lens_count(job.kappa_star, job.lens_radius)


def make_lenses(job, device="cuda", stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Device lens list (3, N) float64: planes x1, x2, m (seeded)."""
    n = job_lens_count(job)
    if out is None:
        out = torch.empty((3, n), dtype=torch.float64, device=device)
    assert out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == 3 * n
    f = LensField(job.kappa_star, job.lens_radius, job.mass_model, 0, job.m_lo, job.m_hi, job.slope)
    _check(lib().rs_make_lenses(C.byref(f), job.seed, _ptr(out) if n else None, n, _stream(stream)))
    return out


def _lens_args(lenses: torch.Tensor):
    assert lenses.dtype == torch.float64 and lenses.is_contiguous()
    n = lenses.numel() // 3
    return (_ptr(lenses) if n else None), n


def shoot_map(job, lenses: torch.Tensor, precision: int = PREC_COMPENSATED,
              unit_mass: bool | None = None, shape: int = 0, counts: torch.Tensor | None = None,
              stats: torch.Tensor | None = None, accumulate: bool = False, stream=None):
    """Shoot the job's ray grid; returns (counts (npix, npix) int32, stats (NSTATS,)
    int64) on the device, stats in RS_STAT_* order: n_in, n_out, n_nonfinite,
    n_refined (rays the refined form's second pass shot), n_exact (its third,
    FP64 pass), the refined
    form's list overflow, its band use (x 65536) and largest first-pass error
    (2^-32 pixel) on the recomputed rays; 0 where a form has none."""
    if unit_mass is None:
        unit_mass = getattr(job, "mass_model", MASS_SALPETER) == MASS_UNIT
    dev = lenses.device if lenses.is_cuda else torch.device("cuda")
    if counts is None:
        counts = torch.empty((job.npix, job.npix), dtype=torch.int32, device=dev)
    if stats is None:
        stats = torch.empty(NSTATS, dtype=torch.int64, device=dev)
    mc, g, mp = structs(job)
    o = options(precision, unit_mass, shape, accumulate)
    lp, n = _lens_args(lenses)
    _check(lib().rs_shoot_map(C.byref(mc), lp, n, C.byref(g), C.byref(mp), C.byref(o),
                              _ptr(counts), _ptr(stats), _stream(stream)))
    return counts, stats


def tile_shape(precision: int = PREC_COMPENSATED, shape: int = 0) -> tuple[int, int]:
    tx, ty = C.c_int64(), C.c_int64()
    o = options(precision, False, shape)
    _check(lib().rs_tile_shape(C.byref(o), C.byref(tx), C.byref(ty)))
    return tx.value, ty.value


def shoot_map_range(job, lenses: torch.Tensor, counts: torch.Tensor, stats: torch.Tensor,
                    tile0: int, n_tiles: int, precision: int = PREC_COMPENSATED,
                    unit_mass: bool | None = None, shape: int = 0, stream=None) -> int:
    """Shoot the map's ray tiles [tile0, tile0 + n_tiles) and add them to
    counts / stats (device tensors the caller zeroed before the first
    range); returns the map's number of tiles.  Consecutive ranges covering
    every tile give rs_shoot_map's map (checkpoint / resume)."""
    if unit_mass is None:
        unit_mass = getattr(job, "mass_model", MASS_SALPETER) == MASS_UNIT
    assert counts.dtype == torch.int32 and stats.dtype == torch.int64
    mc, g, mp = structs(job)
    o = options(precision, unit_mass, shape)
    lp, n = _lens_args(lenses)
    total = C.c_int64()
    _check(lib().rs_shoot_map_range(C.byref(mc), lp, n, C.byref(g), C.byref(mp), C.byref(o),
                                    tile0, n_tiles, _ptr(counts), _ptr(stats), C.byref(total),
                                    _stream(stream)))
    return total.value


def shape_sum(precision: int = PREC_COMPENSATED, shape: int = 0) -> tuple[int, int]:
    """(lenses per compensated fold, lens groups per unrolled loop body) of
    the kernel rs_shoot_map runs for this precision and shape."""
    f, u = C.c_int32(), C.c_int32()
    o = options(precision, False, shape)
    _check(lib().rs_shape_sum(C.byref(o), C.byref(f), C.byref(u)))
    return f.value, u.value


def shoot_tiles(job, lenses: torch.Tensor, tile_ids: torch.Tensor,
                precision: int = PREC_COMPENSATED, unit_mass: bool | None = None,
                shape: int = 0, stream=None):
    """Per-ray (y, pix) of the map kernel for the listed tiles:
    y (T, ty, tx, 2) float64, pix (T, ty, tx, 2) int32."""
    if unit_mass is None:
        unit_mass = getattr(job, "mass_model", MASS_SALPETER) == MASS_UNIT
    tx, ty = tile_shape(precision, shape)
    tile_ids = tile_ids.to(device=lenses.device if lenses.is_cuda else "cuda",
                           dtype=torch.int64).contiguous()
    T = tile_ids.numel()
    y = torch.empty((T, ty, tx, 2), dtype=torch.float64, device=tile_ids.device)
    pix = torch.empty((T, ty, tx, 2), dtype=torch.int32, device=tile_ids.device)
    mc, g, mp = structs(job)
    o = options(precision, unit_mass, shape)
    lp, n = _lens_args(lenses)
    _check(lib().rs_shoot_tiles(C.byref(mc), lp, n, C.byref(g), C.byref(mp), C.byref(o),
                                _ptr(tile_ids), T, _ptr(y), _ptr(pix), _stream(stream)))
    return y, pix


def shoot_tiles_band(job, lenses: torch.Tensor, tile_ids: torch.Tensor,
                     unit_mass: bool | None = None, shape: int = 0, first_pass: bool = False,
                     stream=None):
    """Per-ray refinement band (pixels) of the refined form's first pass for
    the listed tiles: (T, ty, tx) float32 on the device; with first_pass,
    also that pass's images (T, ty, tx, 2) float64 -- the sum the band bounds
    -- as (band, y_first)."""
    if unit_mass is None:
        unit_mass = getattr(job, "mass_model", MASS_SALPETER) == MASS_UNIT
    tx, ty = tile_shape(PREC_REFINED, shape)
    tile_ids = tile_ids.to(device=lenses.device if lenses.is_cuda else "cuda",
                           dtype=torch.int64).contiguous()
    T = tile_ids.numel()
    band = torch.empty((T, ty, tx), dtype=torch.float32, device=tile_ids.device)
    y1 = torch.empty((T, ty, tx, 2), dtype=torch.float64, device=tile_ids.device) \
        if first_pass else None
    mc, g, mp = structs(job)
    o = options(PREC_REFINED, unit_mass, shape)
    lp, n = _lens_args(lenses)
    _check(lib().rs_shoot_tiles_band(C.byref(mc), lp, n, C.byref(g), C.byref(mp), C.byref(o),
                                     _ptr(tile_ids), T, _ptr(band), _ptr(y1), _stream(stream)))
    return (band, y1) if first_pass else band


def debug_rays(job, lenses: torch.Tensor, ij, precision: int = PREC_COMPENSATED,
               unit_mass: bool | None = None, shape: int = 0, stream=None):
    """Per-ray (y (k, 2) float64, pix (k, 2) int32) numpy arrays of the map
    kernel for the rays ij (k, 2) = (i, j), the oracle's per-ray interface."""
    import numpy as np
    if unit_mass is None:
        unit_mass = getattr(job, "mass_model", MASS_SALPETER) == MASS_UNIT
    ij = np.ascontiguousarray(ij, dtype=np.int64).reshape(-1, 2)
    ids = np.ascontiguousarray(ij[:, 1] * job.n1 + ij[:, 0], dtype=np.int64)
    k = ids.size
    y = np.empty((k, 2), dtype=np.float64)
    pix = np.empty((k, 2), dtype=np.int32)
    mc, g, mp = structs(job)
    o = options(precision, unit_mass, shape)
    lp, n = _lens_args(lenses)
    _check(lib().rs_debug_rays(C.byref(mc), lp, n, C.byref(g), C.byref(mp), C.byref(o),
                               ids.ctypes.data_as(C.c_void_p), k, y.ctypes.data_as(C.c_void_p),
                               pix.ctypes.data_as(C.c_void_p), _stream(stream)))
    return y, pix


def magnification(job, counts: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Eq. 4: mu = counts / N_avg as float32 on the device."""
    assert counts.dtype == torch.int32 and counts.is_contiguous()
    if out is None:
        out = torch.empty(counts.shape, dtype=torch.float32, device=counts.device)
    _, g, mp = structs(job)
    _check(lib().rs_magnification(_ptr(counts), C.byref(g), C.byref(mp), _ptr(out),
                                  _stream(stream)))
    return out


def shoot_map_host(job, lenses_host: torch.Tensor, mu_host: torch.Tensor | None = None,
                   stats_host: torch.Tensor | None = None, precision: int = PREC_COMPENSATED,
                   unit_mass: bool | None = None, shape: int = 0, stream=None):
    """End-to-end map from HOST buffers: host lens list in, host float32
    magnification map and stats out (pinned host memory recommended)."""
    if unit_mass is None:
        unit_mass = getattr(job, "mass_model", MASS_SALPETER) == MASS_UNIT
    assert not lenses_host.is_cuda and lenses_host.dtype == torch.float64
    lenses_host = lenses_host.contiguous()
    if mu_host is None:
        mu_host = torch.empty((job.npix, job.npix), dtype=torch.float32, pin_memory=True)
    if stats_host is None:
        stats_host = torch.empty(NSTATS, dtype=torch.int64, pin_memory=True)
    mc, g, mp = structs(job)
    o = options(precision, unit_mass, shape)
    lp, n = _lens_args(lenses_host)
    _check(lib().rs_shoot_map_host(C.byref(mc), lp, n, C.byref(g), C.byref(mp), C.byref(o),
                                   _ptr(mu_host), _ptr(stats_host), _stream(stream)))
    return mu_host, stats_host


# load eagerly: a missing or stale library is an import error, never a fallback
_load()


# ------------------------------------------------------------ batching -----

class Job(C.Structure):
    _fields_ = [("macro", Macro), ("d_lens", C.c_void_p), ("n_lens", C.c_int64),
                ("grid", RayGrid), ("map", MapSpec), ("d_counts", C.c_void_p),
                ("d_stats", C.c_void_p), ("d_mu", C.c_void_p)]


def _declare_batch(L):
    P = C.POINTER
    L.rs_shoot_batch.argtypes = [P(Job), C.c_int, P(Options), C.c_void_p]
    L.rs_autotune.argtypes = [P(Job), C.c_int, P(Options), P(C.c_int32), P(C.c_float),
                              C.c_int, C.c_void_p]
    L.rs_tune_candidates.argtypes = [C.c_int, P(C.c_int32), C.c_int]
    L.rs_plan_create.argtypes = [P(Job), C.c_int, P(Options), P(C.c_void_p)]
    L.rs_plan_shape.argtypes = [C.c_void_p, P(C.c_int32)]
    L.rs_plan_launch.argtypes = [C.c_void_p, C.c_void_p]
    L.rs_plan_destroy.argtypes = [C.c_void_p]
    for n in ("rs_shoot_batch", "rs_autotune", "rs_tune_candidates", "rs_plan_create",
              "rs_plan_shape", "rs_plan_launch", "rs_plan_destroy"):
        getattr(L, n).restype = C.c_int


_declare_batch(lib())


class MapBuffers:
    """Device buffers of one map of a batch: lens list, counts, stats, mu."""

    def __init__(self, job, lenses: torch.Tensor, with_mu: bool = True):
        dev = lenses.device
        self.job = job
        self.lenses = lenses
        self.counts = torch.empty((job.npix, job.npix), dtype=torch.int32, device=dev)
        self.stats = torch.empty(NSTATS, dtype=torch.int64, device=dev)
        self.mu = torch.empty((job.npix, job.npix), dtype=torch.float32, device=dev) \
            if with_mu else None

    def cjob(self) -> Job:
        mc, g, mp = structs(self.job)
        lp, n = _lens_args(self.lenses)
        return Job(mc, lp, n, g, mp, self.counts.data_ptr(), self.stats.data_ptr(),
                   self.mu.data_ptr() if self.mu is not None else None)


def _jobs_array(bufs):
    arr = (Job * len(bufs))()
    for k, b in enumerate(bufs):
        arr[k] = b.cjob()
    return arr


def shoot_batch(bufs, precision: int = PREC_COMPENSATED, unit_mass: bool = False,
                shape: int = 0, accumulate: bool = False, stream=None):
    """Shoot a list of MapBuffers as persistent batched launches (plus Eq. 4
    for buffers with mu)."""
    arr = _jobs_array(bufs)
    o = options(precision, unit_mass, shape, accumulate)
    _check(lib().rs_shoot_batch(arr, len(bufs), C.byref(o), _stream(stream)))


def tune_candidates(precision: int = PREC_COMPENSATED) -> list[int]:
    """Shapes rs_autotune tries for this precision, the default first."""
    buf = (C.c_int32 * 64)()
    n = lib().rs_tune_candidates(precision, buf, 64)
    if n < 0:
        _check(n)
    return list(buf[:n])


def autotune(bufs, precision: int = PREC_COMPENSATED, unit_mass: bool = False, stream=None):
    """Time the candidate shapes (tune_candidates(precision)) on a sample of
    the batch; returns (best shape, {shape: ms per 1e9 interactions})."""
    arr = _jobs_array(bufs)
    o = options(precision, unit_mass, 0)
    best = C.c_int32()
    cand = tune_candidates(precision)
    ms = (C.c_float * len(cand))()
    _check(lib().rs_autotune(arr, len(bufs), C.byref(o), C.byref(best), ms, len(cand),
                             _stream(stream)))
    return best.value, {s: float(ms[k]) for k, s in enumerate(cand)}


class Plan:
    """A batch captured into a CUDA graph; launch() replays it."""

    def __init__(self, bufs, precision: int = PREC_COMPENSATED, unit_mass: bool = False,
                 shape: int = 0, accumulate: bool = False):
        self.bufs = list(bufs)            # keeps the device buffers alive
        arr = _jobs_array(self.bufs)
        o = options(precision, unit_mass, shape, accumulate)
        h = C.c_void_p()
        _check(lib().rs_plan_create(arr, len(self.bufs), C.byref(o), C.byref(h)))
        self._h = h

    @property
    def shape(self) -> int:
        v = C.c_int32()
        _check(lib().rs_plan_shape(self._h, C.byref(v)))
        return v.value

    def launch(self, stream=None):
        _check(lib().rs_plan_launch(self._h, _stream(stream)))

    def close(self):
        if self._h:
            lib().rs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------- no-allocation map call -----

lib().rs_shoot_map_host_noalloc.argtypes = [C.POINTER(Macro), C.c_void_p, C.c_int64,
                                            C.POINTER(RayGrid), C.POINTER(MapSpec),
                                            C.POINTER(Options), C.c_void_p, C.c_void_p,
                                            C.c_void_p]
lib().rs_shoot_map_host_noalloc.restype = C.c_int


def shoot_map_host_noalloc(job, lenses_host: torch.Tensor, mu_host: torch.Tensor,
                           stats_host: torch.Tensor, precision: int = PREC_COMPENSATED,
                           unit_mass: bool | None = None, shape: int = 0, stream=None):
    """shoot_map_host for callers that cannot allocate device memory: the
    device working set lives in the library's fixed device array (maps up to
    1024^2 pixels, up to 65536 lenses); the caller passes host buffers."""
    if unit_mass is None:
        unit_mass = getattr(job, "mass_model", MASS_SALPETER) == MASS_UNIT
    lenses_host = lenses_host.contiguous()
    mc, g, mp = structs(job)
    o = options(precision, unit_mass, shape)
    lp, n = _lens_args(lenses_host)
    _check(lib().rs_shoot_map_host_noalloc(C.byref(mc), lp, n, C.byref(g), C.byref(mp),
                                           C.byref(o), _ptr(mu_host), _ptr(stats_host),
                                           _stream(stream)))
    return mu_host, stats_host


# --------------------------------------------------------------- serving -----

SCHED_SRPT = 0
SCHED_FIFO = 1
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = 0, 1, 2, 3, 4


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("slice_ms", C.c_double), ("rate_gint", C.c_double),
                ("max_active", C.c_int32), ("max_queue", C.c_int32), ("policy", C.c_int32),
                ("precision", C.c_int32), ("shape", C.c_int32), ("threaded", C.c_int32),
                ("max_skips", C.c_int32), ("inject_alloc_failures", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("macro", Macro), ("field", LensField), ("seed", C.c_uint64),
                ("n_lens", C.c_int64), ("grid", RayGrid), ("map", MapSpec)]


class Result(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("d_mu", C.c_void_p),
                ("d_counts", C.c_void_p), ("stats", C.c_int64 * NSTATS), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("tiles_total", C.c_int64),
                ("tiles_launched", C.c_int64), ("n_lens", C.c_int64)]


class SchedQueued(C.Structure):
    _fields_ = [("bytes", C.c_int64), ("skips", C.c_int32), ("pad_", C.c_int32)]


class SchedItem(C.Structure):
    _fields_ = [("seq", C.c_int64), ("tiles_left", C.c_int64), ("work_per_tile", C.c_double)]


def _declare_serve(L):
    P, vp = C.POINTER, C.c_void_p
    L.rs_server_create.argtypes = [P(ServerConfig), P(vp)]
    L.rs_server_submit.argtypes = [vp, P(Request), P(C.c_int64)]
    L.rs_server_step.argtypes = [vp, P(C.c_int32)]
    L.rs_server_poll.argtypes = [vp, C.c_int64, P(Result)]
    L.rs_server_wait.argtypes = [vp, C.c_int64, C.c_double, P(Result)]
    L.rs_server_cancel.argtypes = [vp, C.c_int64]
    L.rs_server_release.argtypes = [vp, C.c_int64]
    L.rs_server_drain.argtypes = [vp, C.c_double]
    L.rs_server_counters.argtypes = [vp, P(C.c_int64), C.c_int]
    L.rs_server_clock.argtypes = [vp]
    L.rs_server_clock.restype = C.c_double
    L.rs_server_destroy.argtypes = [vp]
    L.rs_server_inject_alloc_failures.argtypes = [vp, C.c_int]
    L.rs_server_inject_alloc_failures.restype = C.c_int
    L.rs_sched_admit.argtypes = [P(SchedQueued), C.c_int, C.c_int64, C.c_int64, C.c_int,
                                 C.c_int, C.c_int, P(C.c_int32)]
    L.rs_sched_plan.argtypes = [P(SchedItem), C.c_int, C.c_double, C.c_int, C.c_int,
                                P(C.c_int64)]
    for n in ("rs_server_create", "rs_server_submit", "rs_server_step", "rs_server_poll",
              "rs_server_wait", "rs_server_cancel", "rs_server_release", "rs_server_drain",
              "rs_server_counters", "rs_server_destroy", "rs_sched_admit", "rs_sched_plan"):
        getattr(L, n).restype = C.c_int


_declare_serve(lib())


def sched_admit(queued, bytes_used, budget, active, max_active, max_skips=4):
    """Host-only admission policy: list of (bytes, skips) -> admit flags."""
    arr = (SchedQueued * len(queued))(*[SchedQueued(b, s, 0) for b, s in queued])
    out = (C.c_int32 * max(1, len(queued)))()
    n = lib().rs_sched_admit(arr, len(queued), bytes_used, budget, active, max_active,
                             max_skips, out)
    if n < 0:
        _check(n)
    return [int(v) for v in out[:len(queued)]]


def sched_plan(items, budget, policy=SCHED_SRPT, max_maps=128):
    """Host-only slice planning: list of (seq, tiles_left, work_per_tile) ->
    tiles granted to each."""
    arr = (SchedItem * len(items))(*[SchedItem(a, b, c) for a, b, c in items])
    out = (C.c_int64 * max(1, len(items)))()
    n = lib().rs_sched_plan(arr, len(items), budget, policy, max_maps, out)
    if n < 0:
        _check(n)
    return [int(v) for v in out[:len(items)]]


def make_request(job) -> Request:
    mc, g, mp = structs(job)
    f = LensField(job.kappa_star, job.lens_radius, job.mass_model, 0, job.m_lo, job.m_hi,
                  job.slope)
    return Request(mc, f, job.seed, job.n_lens, g, mp)


class Server:
    """Continuous-batching map server (C++ runtime in the library)."""

    def __init__(self, hbm_budget=8 << 30, slice_ms=25.0, rate_gint=5000.0, max_active=64,
                 max_queue=4096, policy=SCHED_SRPT, precision=PREC_COMPENSATED, shape=0,
                 threaded=True, max_skips=4, inject_alloc_failures=0):
        cfg = ServerConfig(hbm_budget, slice_ms, rate_gint, max_active, max_queue, policy,
                           precision, shape, int(threaded), max_skips, inject_alloc_failures)
        h = C.c_void_p()
        _check(lib().rs_server_create(C.byref(cfg), C.byref(h)))
        self._h = h

    def submit(self, job) -> int:
        t = C.c_int64()
        r = make_request(job)
        _check(lib().rs_server_submit(self._h, C.byref(r), C.byref(t)))
        return t.value

    def step(self) -> bool:
        p = C.c_int32()
        _check(lib().rs_server_step(self._h, C.byref(p)))
        return bool(p.value)

    def poll(self, ticket) -> Result:
        r = Result()
        _check(lib().rs_server_poll(self._h, ticket, C.byref(r)))
        return r

    def wait(self, ticket, timeout_s=60.0) -> Result:
        r = Result()
        _check(lib().rs_server_wait(self._h, ticket, timeout_s, C.byref(r)))
        return r

    def cancel(self, ticket):
        _check(lib().rs_server_cancel(self._h, ticket))

    def release(self, ticket):
        _check(lib().rs_server_release(self._h, ticket))

    def drain(self, timeout_s=600.0):
        _check(lib().rs_server_drain(self._h, timeout_s))

    def counters(self) -> dict:
        v = (C.c_int64 * 10)()
        _check(lib().rs_server_counters(self._h, v, 10))
        keys = ("slices", "launches", "admitted", "completed", "failed", "cancelled",
                "peak_bytes", "bytes_in_use", "queued", "running")
        return dict(zip(keys, [int(x) for x in v]))

    def clock(self) -> float:
        return lib().rs_server_clock(self._h)

    def inject_alloc_failures(self, k: int):
        """Test hook: the next k admissions fail as if out of device memory."""
        _check(lib().rs_server_inject_alloc_failures(self._h, k))

    @staticmethod
    def map_tensors(res: Result, npix: int):
        """(mu, counts) device tensors viewing a finished request's maps
        (valid until release)."""
        mu = _device_view(res.d_mu, (npix, npix), torch.float32)
        counts = _device_view(res.d_counts, (npix, npix), torch.int32)
        return mu, counts

    def close(self):
        if self._h:
            lib().rs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """Minimal __cuda_array_interface__ holder for a library-owned buffer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def _device_view(ptr, shape, dtype):
    """Zero-copy tensor view of a library-owned device buffer (the library
    keeps ownership: the view is valid until the buffer is released)."""
    typestr = {torch.float32: "<f4", torch.int32: "<i4"}[dtype]
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")


# ------------------------------------------------------------------- MPD -----

lib().rs_mpd.argtypes = [C.c_void_p, C.POINTER(RayGrid), C.POINTER(MapSpec), C.c_void_p,
                         C.c_void_p, C.c_int64, C.c_void_p]
lib().rs_mpd.restype = C.c_int
lib().rs_prob_sums.argtypes = [C.c_void_p, C.c_int64, C.POINTER(RayGrid), C.POINTER(MapSpec),
                               C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
lib().rs_prob_sums.restype = C.c_int


def count_histogram(job, counts: torch.Tensor, n_bins: int = 1 << 20,
                    mu_out: torch.Tensor | None = None, hist: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Exact histogram of the count map (the MPD numerator, Sec. 3.2.1);
    with mu_out, Eq. 4 is written in the same pass."""
    assert counts.dtype == torch.int32 and counts.is_contiguous()
    if hist is None:
        hist = torch.empty(n_bins, dtype=torch.int64, device=counts.device)
    assert hist.dtype == torch.int64 and hist.numel() == n_bins
    _, g, mp = structs(job)
    _check(lib().rs_mpd(_ptr(counts), C.byref(g), C.byref(mp), _ptr(mu_out), _ptr(hist),
                        n_bins, _stream(stream)))
    return hist


def prob_sums(job, hist: torch.Tensor, mu_lim, stream=None):
    """Pixels with mu < mu_lim and mu > mu_lim (device int64 tensors)."""
    lim = [float(v) for v in (mu_lim if hasattr(mu_lim, "__len__") else [mu_lim])]
    arr = (C.c_double * len(lim))(*lim)
    below = torch.empty(len(lim), dtype=torch.int64, device=hist.device)
    above = torch.empty(len(lim), dtype=torch.int64, device=hist.device)
    _, g, mp = structs(job)
    _check(lib().rs_prob_sums(_ptr(hist), hist.numel(), C.byref(g), C.byref(mp), arr, len(lim),
                              _ptr(below), _ptr(above), _stream(stream)))
    return below, above


# ---------------------------------------------------- finite sources -----
# Source profiles binned to map pixels and the convolution of Eq. 6
# (Sec. 2.4), pixelFlux records and value histograms of convolved maps
# (Sec. 3.2.2); C ABI in include/rs_conv.h.

PROFILE_UNIFORM, PROFILE_GAUSSIAN, PROFILE_POWER_LAW, PROFILE_THIN_DISC = 0, 1, 2, 3


class Profile(C.Structure):
    _fields_ = [("type", C.c_int32), ("supersample", C.c_int32), ("r_out", C.c_double),
                ("r_in", C.c_double), ("sigma1", C.c_double), ("sigma2", C.c_double),
                ("r_scale", C.c_double), ("index", C.c_double)]


class PixFlux(C.Structure):
    _fields_ = [("x", C.c_int16), ("y", C.c_int16), ("value", C.c_float)]


def _declare_conv(L):
    P, vp, i64 = C.POINTER, C.c_void_p, C.c_int64
    L.rs_profile_half.argtypes = [P(Profile), C.c_double, P(i64)]
    L.rs_profile_kernel.argtypes = [P(Profile), C.c_double, vp, i64, vp]
    L.rs_conv_create.argtypes = [i64, P(vp)]
    L.rs_conv_destroy.argtypes = [vp]
    L.rs_conv_destroy.restype = None
    L.rs_conv_bytes.argtypes = [vp, P(C.c_size_t)]
    L.rs_conv_set_profile.argtypes = [vp, P(Profile), C.c_double, vp]
    L.rs_conv_set_kernel.argtypes = [vp, vp, i64, vp]
    L.rs_conv_apply_counts.argtypes = [vp, vp, C.c_double, vp, vp]
    L.rs_conv_apply.argtypes = [vp, vp, vp, vp]
    L.rs_conv_load_counts.argtypes = [vp, vp, C.c_double, vp]
    L.rs_conv_load.argtypes = [vp, vp, vp]
    L.rs_conv_apply_loaded.argtypes = [vp, vp, vp]
    L.rs_conv_set_profile_slot.argtypes = [vp, C.c_int, P(Profile), C.c_double, vp]
    L.rs_conv_apply_loaded_slot.argtypes = [vp, C.c_int, vp, vp]
    L.rs_pixel_flux.argtypes = [vp, i64, vp, C.c_uint64, i64, vp, vp]
    L.rs_value_histogram.argtypes = [vp, i64, vp, i64, vp, vp]
    L.rs_conv_fft_kind.argtypes = [vp, P(C.c_int)]
    for n in ("rs_profile_half", "rs_profile_kernel", "rs_conv_create", "rs_conv_bytes",
              "rs_conv_fft_kind",
              "rs_conv_set_profile", "rs_conv_set_kernel", "rs_conv_apply_counts",
              "rs_conv_apply", "rs_conv_load_counts", "rs_conv_load", "rs_conv_apply_loaded",
              "rs_conv_set_profile_slot", "rs_conv_apply_loaded_slot",
              "rs_pixel_flux", "rs_value_histogram"):
        getattr(L, n).restype = C.c_int


_declare_conv(lib())


def _profile(prof) -> Profile:
    return Profile(prof.type, prof.supersample, prof.r_out, prof.r_in, prof.sigma1,
                   prof.sigma2, prof.r_scale, prof.index)


def profile_half(prof, pixel: float) -> int:
    """Half size h of the profile's binned kernel ((2h+1)^2 pixels)."""
    h = C.c_int64()
    _check(lib().rs_profile_half(C.byref(_profile(prof)), pixel, C.byref(h)))
    return h.value


def profile_kernel(prof, pixel: float, device="cuda", stream=None) -> torch.Tensor:
    """The profile binned to pixels of side `pixel`, unit sum, (2h+1, 2h+1)
    float32 on the device (row offset a + h, column offset b + h)."""
    h = profile_half(prof, pixel)
    k = torch.empty((2 * h + 1, 2 * h + 1), dtype=torch.float32, device=device)
    _check(lib().rs_profile_kernel(C.byref(_profile(prof)), pixel, _ptr(k), h, _stream(stream)))
    return k


CONV_FFT_OWN = 1
CONV_FFT_CUFFT = 2


class Convolver:
    """Eq. 6 for npix x npix maps: holds the kernel spectrum, a spectrum
    buffer and the transforms (the library's own for the survey's sizes,
    cuFFT plans otherwise).  One host thread at a time."""

    def __init__(self, npix: int):
        self.npix = int(npix)
        h = C.c_void_p()
        _check(lib().rs_conv_create(self.npix, C.byref(h)))
        self._h = h

    @property
    def nbytes(self) -> int:
        v = C.c_size_t()
        _check(lib().rs_conv_bytes(self._h, C.byref(v)))
        return v.value

    @property
    def fft_kind(self) -> int:
        """CONV_FFT_OWN or CONV_FFT_CUFFT."""
        v = C.c_int()
        _check(lib().rs_conv_fft_kind(self._h, C.byref(v)))
        return v.value

    SLOTS = 16

    def set_profile(self, prof, pixel: float, stream=None, slot: int = 0):
        """Bin the profile and keep its spectrum (in kernel slot `slot`; slot
        0 is the kernel apply / apply_counts use)."""
        _check(lib().rs_conv_set_profile_slot(self._h, slot, C.byref(_profile(prof)), pixel,
                                              _stream(stream)))

    def set_kernel(self, kernel: torch.Tensor, stream=None):
        assert kernel.dtype == torch.float32 and kernel.is_cuda and kernel.is_contiguous()
        h = (kernel.shape[0] - 1) // 2
        assert kernel.shape == (2 * h + 1, 2 * h + 1)
        _check(lib().rs_conv_set_kernel(self._h, _ptr(kernel), h, _stream(stream)))

    def _out(self, like: torch.Tensor, out):
        if out is None:
            out = torch.empty((self.npix, self.npix), dtype=torch.float32, device=like.device)
        assert out.dtype == torch.float32 and out.is_contiguous() and \
            out.numel() == self.npix * self.npix
        return out

    def apply_counts(self, counts: torch.Tensor, scale: float, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
        """scale * counts convolved with the kernel (scale = 1 / N_avg gives
        the convolved magnification map)."""
        assert counts.dtype == torch.int32 and counts.is_contiguous() and \
            counts.numel() == self.npix * self.npix
        out = self._out(counts, out)
        _check(lib().rs_conv_apply_counts(self._h, _ptr(counts), float(scale), _ptr(out),
                                          _stream(stream)))
        return out

    def apply(self, m: torch.Tensor, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
        assert m.dtype == torch.float32 and m.is_contiguous() and m.numel() == self.npix ** 2
        out = self._out(m, out)
        _check(lib().rs_conv_apply(self._h, _ptr(m), _ptr(out), _stream(stream)))
        return out

    def load_counts(self, counts: torch.Tensor, scale: float, stream=None):
        """Keep the spectrum of scale * counts for several kernels."""
        assert counts.dtype == torch.int32 and counts.is_contiguous() and \
            counts.numel() == self.npix * self.npix
        _check(lib().rs_conv_load_counts(self._h, _ptr(counts), float(scale), _stream(stream)))

    def load(self, m: torch.Tensor, stream=None):
        assert m.dtype == torch.float32 and m.is_contiguous() and m.numel() == self.npix ** 2
        _check(lib().rs_conv_load(self._h, _ptr(m), _stream(stream)))

    def apply_loaded(self, out: torch.Tensor | None = None, stream=None,
                     slot: int = 0) -> torch.Tensor:
        """The loaded map convolved with the kernel in slot `slot`."""
        if out is None:
            out = torch.empty((self.npix, self.npix), dtype=torch.float32, device="cuda")
        assert out.dtype == torch.float32 and out.is_contiguous() and \
            out.numel() == self.npix * self.npix
        _check(lib().rs_conv_apply_loaded_slot(self._h, slot, _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().rs_conv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pixel_flux(m: torch.Tensor, k: int = 0, seed: int = 0, xy: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """pixelFlux records (k, 8 bytes as uint8 view) {int16 x, int16 y, float32
    value}; locations from xy (k, 2) int16 or drawn from seed.  Returns a
    (k,) int64 tensor holding the packed records (see unpack_pixel_flux)."""
    npix = m.shape[-1]
    assert m.dtype == torch.float32 and m.is_contiguous() and m.numel() == npix * npix
    if xy is not None:
        assert xy.dtype == torch.int16 and xy.is_contiguous() and xy.shape[-1] == 2
        k = xy.shape[0]
    rec = torch.empty(k, dtype=torch.int64, device=m.device)
    _check(lib().rs_pixel_flux(_ptr(m), npix, _ptr(xy), seed, k, _ptr(rec) if k else None,
                               _stream(stream)))
    return rec


def unpack_pixel_flux(rec: torch.Tensor):
    """(x, y, value) numpy arrays from packed pixelFlux records."""
    import numpy as np
    a = rec.cpu().numpy().view(np.dtype([("x", "<i2"), ("y", "<i2"), ("value", "<f4")]))
    return a["x"].copy(), a["y"].copy(), a["value"].copy()


def value_histogram(v: torch.Tensor, edges, hist: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """hist[b] = values with exactly b edges at or below them (n_edges + 1
    int64 bins on the device; NaN in bin 0)."""
    import numpy as np
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.float32))
    assert v.dtype == torch.float32 and v.is_contiguous()
    if hist is None:
        hist = torch.empty(e.size + 1, dtype=torch.int64, device=v.device)
    _check(lib().rs_value_histogram(_ptr(v) if v.numel() else None, v.numel(),
                                    e.ctypes.data_as(C.c_void_p), e.size, _ptr(hist),
                                    _stream(stream)))
    return hist


# ------------------------------------------- indexed maps and previews -----
# Indexed count maps (App. B) and map previews / colorbar (Sec. 3.2.1,
# Sec. 4.6); C ABI in include/rs_codec.h.

class IndexInfo(C.Structure):
    _fields_ = [("distinct", C.c_int64), ("bits", C.c_int32), ("max_count", C.c_int32),
                ("words", C.c_int64)]


def _declare_codec(L):
    P, vp, i64 = C.POINTER, C.c_void_p, C.c_int64
    L.rs_index_bits.argtypes = [i64]
    L.rs_index_encode.argtypes = [vp, i64, C.c_int, vp, i64, vp, i64, P(IndexInfo), vp]
    L.rs_index_decode.argtypes = [vp, i64, C.c_int, vp, i64, vp, vp]
    L.rs_colorbar_lut.argtypes = [vp, vp, C.c_int, vp]
    L.rs_preview_counts.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
    L.rs_preview_f32.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
    L.rs_colorize.argtypes = [vp, i64, vp, vp, vp]
    for n in ("rs_index_bits", "rs_index_encode", "rs_index_decode", "rs_colorbar_lut",
              "rs_preview_counts", "rs_preview_f32", "rs_colorize"):
        getattr(L, n).restype = C.c_int


_declare_codec(lib())


def index_bits(distinct: int) -> int:
    return int(lib().rs_index_bits(distinct))


def index_encode(counts: torch.Tensor, bits: int = 0, table_cap: int = 1 << 20,
                 stream=None):
    """Indexed map of a device count map: (table (D,) int32, words (W,)
    int32 holding the packed uint32 stream, info dict).  Synchronises."""
    assert counts.dtype == torch.int32 and counts.is_contiguous() and counts.is_cuda
    n = counts.numel()
    cap_t = max(1, min(n, table_cap))
    cap_w = max(1, (n * (bits or 20) + 31) // 32)
    for _ in range(2):
        table = torch.empty(cap_t, dtype=torch.int32, device=counts.device)
        words = torch.empty(cap_w, dtype=torch.int32, device=counts.device)
        info = IndexInfo()
        rc = lib().rs_index_encode(_ptr(counts), n, bits, _ptr(table), cap_t, _ptr(words), cap_w,
                                   C.byref(info), _stream(stream))
        if rc == -6 and info.distinct > 0 and (info.distinct > cap_t or info.words > cap_w) \
                and info.bits >= index_bits(info.distinct):
            cap_t, cap_w = max(cap_t, info.distinct), max(cap_w, info.words)
            continue
        _check(rc)
        break
    d = {"distinct": info.distinct, "bits": info.bits, "max_count": info.max_count,
         "words": info.words}
    return table[:info.distinct], words[:info.words], d


def index_decode(words: torch.Tensor, n: int, bits: int, table: torch.Tensor,
                 out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Counts (n,) int32 from a packed map; -1 where an index is not in the table."""
    assert words.is_contiguous() and table.dtype == torch.int32 and table.is_contiguous()
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=words.device)
    _check(lib().rs_index_decode(_ptr(words), n, bits, _ptr(table), table.numel(), _ptr(out),
                                 _stream(stream)))
    return out


def colorbar_lut(pos, rgb):
    """256 x 3 uint8 colour table (numpy) from colour stops."""
    import numpy as np
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8).reshape(-1, 3)
    lut = np.empty((256, 3), dtype=np.uint8)
    _check(lib().rs_colorbar_lut(pos.ctypes.data_as(C.c_void_p), rgb.ctypes.data_as(C.c_void_p),
                                 pos.size, lut.ctypes.data_as(C.c_void_p)))
    return lut


def preview(m: torch.Tensor, s: int, thresholds, lut=None, stream=None):
    """s x s preview of a device map: (gray (s, s) uint8, rgba (s, s) int32
    holding RGBA8 or None).  int32 count maps take float64 thresholds, float32
    maps float32 thresholds (255, ascending)."""
    import numpy as np
    npix = m.shape[-1]
    assert m.is_contiguous() and m.numel() == npix * npix
    gray = torch.empty((s, s), dtype=torch.uint8, device=m.device)
    rgba = None if lut is None else torch.empty((s, s), dtype=torch.int32, device=m.device)
    lut_np = None if lut is None else np.ascontiguousarray(lut, dtype=np.uint8)
    lp = None if lut_np is None else lut_np.ctypes.data_as(C.c_void_p)
    if m.dtype == torch.int32:
        t = np.ascontiguousarray(thresholds, dtype=np.float64)
        fn = lib().rs_preview_counts
    else:
        assert m.dtype == torch.float32
        t = np.ascontiguousarray(thresholds, dtype=np.float32)
        fn = lib().rs_preview_f32
    assert t.size == 255, "255 thresholds"
    _check(fn(_ptr(m), npix, s, t.ctypes.data_as(C.c_void_p), lp, _ptr(gray), _ptr(rgba),
              _stream(stream)))
    return gray, rgba


def colorize(gray: torch.Tensor, lut, stream=None) -> torch.Tensor:
    """Recolour gray levels with a 256 x 3 table: RGBA8 in int32."""
    import numpy as np
    lut_np = np.ascontiguousarray(lut, dtype=np.uint8)
    out = torch.empty(gray.shape, dtype=torch.int32, device=gray.device)
    _check(lib().rs_colorize(_ptr(gray), gray.numel(), lut_np.ctypes.data_as(C.c_void_p),
                             _ptr(out), _stream(stream)))
    return out


def rgba_bytes(rgba: torch.Tensor):
    """(s, s, 4) uint8 numpy view of RGBA8 pixels."""
    import numpy as np
    a = rgba.cpu().numpy()
    return a.view(np.uint8).reshape(a.shape + (4,))


def write_png(path: str, rgba) -> None:
    """Write an (h, w, 4) uint8 RGBA image as a PNG file (icon.png,
    sample.png), zlib-compressed, no filtering."""
    import struct
    import zlib

    import numpy as np
    img = np.ascontiguousarray(rgba, dtype=np.uint8)
    h, w = img.shape[:2]
    raw = b"".join(b"\x00" + img[r].tobytes() for r in range(h))

    def chunk(tag, data):
        return (struct.pack(">I", len(data)) + tag + data +
                struct.pack(">I", zlib.crc32(tag + data) & 0xffffffff))
    with open(path, "wb") as fh:
        fh.write(b"\x89PNG\r\n\x1a\n")
        fh.write(chunk(b"IHDR", struct.pack(">IIBBBBB", w, h, 8, 6, 0, 0, 0)))
        fh.write(chunk(b"IDAT", zlib.compress(raw, 6)))
        fh.write(chunk(b"IEND", b""))

"""FP64 CPU oracle for direct inverse ray-shooting (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark are the only callers.  The arithmetic lives in
``rs_oracle.c`` (plain FP64, compiled with ``-ffp-contract=off``); this module
only compiles it and marshals numpy arrays.  It imports nothing from the CUDA
package and the CUDA package imports nothing from here.

Paper: Vernardos & Fluke 2014, Sec. 2.1 (Eq. 1 lens equation, Eq. 3 lens
count, Eq. 4 magnification) and Fig. 1 (lenses uniform in a disk, regular
ray grid, map region away from the edges).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_HDR = os.path.join(_HERE, "rs_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
          "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (plain gcc)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        cc = os.environ.get("CC", "gcc")
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run([cc, *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Macro(C.Structure):
    _fields_ = [("kappa_s", C.c_double), ("gamma", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("c1", C.c_double), ("c2", C.c_double), ("h1", C.c_double),
                ("h2", C.c_double), ("n1", C.c_int64), ("n2", C.c_int64)]


class Map(C.Structure):
    _fields_ = [("c1", C.c_double), ("c2", C.c_double), ("width", C.c_double),
                ("npix", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("type", C.c_int32), ("supersample", C.c_int32), ("r_out", C.c_double),
                ("r_in", C.c_double), ("sigma1", C.c_double), ("sigma2", C.c_double),
                ("r_scale", C.c_double), ("index", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_u01.restype = C.c_double
        L.orc_u01.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_lens_count.restype = C.c_int64
        L.orc_lens_count.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_make_lenses.restype = C.c_int
        L.orc_make_lenses.argtypes = [C.c_double, C.c_int, C.c_double, C.c_double,
                                      C.c_double, C.c_int64, C.c_uint64, C.c_void_p]
        L.orc_deflection.restype = None
        L.orc_deflection.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                     C.c_void_p, C.c_void_p]
        L.orc_shoot.restype = C.c_int
        L.orc_shoot.argtypes = [P(Macro), C.c_void_p, C.c_int64, P(Grid), P(Map),
                                C.c_void_p, C.c_void_p, C.c_int]
        L.orc_shoot_rays.restype = C.c_int
        L.orc_shoot_rays.argtypes = [P(Macro), C.c_void_p, C.c_int64, P(Grid), P(Map),
                                     C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_int]
        L.orc_navg.restype = C.c_double
        L.orc_navg.argtypes = [P(Grid), P(Map)]
        L.orc_magnification.restype = None
        L.orc_magnification.argtypes = [C.c_void_p, P(Grid), P(Map), C.c_void_p]
        L.orc_count_histogram.restype = C.c_int
        L.orc_count_histogram.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]
        L.orc_prob_sums.restype = C.c_int
        L.orc_prob_sums.argtypes = [C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_int,
                                    C.c_void_p, C.c_void_p]
        L.orc_profile_half.restype = C.c_int64
        L.orc_profile_half.argtypes = [P(Profile), C.c_double]
        L.orc_profile_kernel.restype = C.c_int
        L.orc_profile_kernel.argtypes = [P(Profile), C.c_double, C.c_int64, C.c_void_p,
                                         P(C.c_double)]
        L.orc_convolve_direct.restype = C.c_int
        L.orc_convolve_direct.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                          C.c_void_p, C.c_int]
        L.orc_convolve_counts_at.restype = C.c_int
        L.orc_convolve_counts_at.argtypes = [C.c_void_p, C.c_double, C.c_int64, C.c_void_p,
                                             C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]
        L.orc_pixel_locations.restype = None
        L.orc_pixel_locations.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_void_p]
        L.orc_value_histogram.restype = C.c_int
        L.orc_value_histogram.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                          C.c_void_p]
        L.orc_index_table.restype = C.c_int64
        L.orc_index_table.argtypes = [C.c_void_p, C.c_int64, C.c_void_p]
        L.orc_index_bits.restype = C.c_int
        L.orc_index_bits.argtypes = [C.c_int64]
        L.orc_index_words.restype = C.c_int64
        L.orc_index_words.argtypes = [C.c_int64, C.c_int]
        L.orc_index_encode.restype = C.c_int
        L.orc_index_encode.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int,
                                       C.c_void_p]
        L.orc_index_decode.restype = C.c_int
        L.orc_index_decode.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64,
                                       C.c_void_p]
        L.orc_colorbar_lut.restype = C.c_int
        L.orc_colorbar_lut.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
        L.orc_sample_gray_counts.restype = C.c_int
        L.orc_sample_gray_counts.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                             C.c_void_p]
        L.orc_sample_gray_f32.restype = C.c_int
        L.orc_sample_gray_f32.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p,
                                          C.c_void_p]
        L.orc_colorize.restype = None
        L.orc_colorize.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _structs(job):
    mc = Macro(job.kappa_s, job.gamma)
    g = Grid(job.c1, job.c2, job.half1, job.half2, job.n1, job.n2)
    mp = Map(job.mc1, job.mc2, job.width, job.npix)
    return mc, g, mp


# --------------------------------------------------------------------------
# public wrappers
# --------------------------------------------------------------------------

def splitmix64(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64(seed, k))


def u01(seed: int, k: int) -> float:
    return float(lib().orc_u01(seed, k))


def lens_count(kappa_star: float, radius: float, mean_mass: float = 1.0) -> int:
    """Eq. 3 with A = pi R^2."""
    return int(lib().orc_lens_count(kappa_star, radius, mean_mass))


def make_lenses(job) -> np.ndarray:
    """Lens planes (3, N): x1, x2, m for a MapJob (N from Eq. 3 if 0)."""
    n = job.n_lens if job.n_lens > 0 else lens_count(job.kappa_star, job.lens_radius)
    out = np.zeros((3, n), dtype=np.float64)
    rc = lib().orc_make_lenses(job.lens_radius, job.mass_model, job.m_lo, job.m_hi,
                               job.slope, n, job.seed, _ptr(out))
    if rc != 0:
        raise ValueError("orc_make_lenses: bad arguments")
    return out


def deflection(lens: np.ndarray, x: np.ndarray):
    """alpha at points x (k, 2) -> (alpha (k, 2), singular (k,))."""
    lens = np.ascontiguousarray(lens, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 2)
    k = x.shape[0]
    alpha = np.empty((k, 2), dtype=np.float64)
    sing = np.empty(k, dtype=np.int32)
    lib().orc_deflection(_ptr(lens), lens.shape[1], _ptr(x), k, _ptr(alpha), _ptr(sing))
    return alpha, sing


def shoot(job, lens: np.ndarray, nthreads: int = 0):
    """Full map: (counts (npix, npix) int32, stats dict)."""
    lens = np.ascontiguousarray(lens, dtype=np.float64).reshape(3, -1)
    mc, g, mp = _structs(job)
    counts = np.empty((job.npix, job.npix), dtype=np.int32)
    stats = np.zeros(3, dtype=np.int64)
    rc = lib().orc_shoot(C.byref(mc), _ptr(lens), lens.shape[1], C.byref(g),
                         C.byref(mp), _ptr(counts), _ptr(stats), nthreads)
    if rc != 0:
        raise ValueError("orc_shoot: bad arguments")
    return counts, {"n_in": int(stats[0]), "n_out": int(stats[1]),
                    "n_singular": int(stats[2])}


def shoot_rays(job, lens: np.ndarray, ij: np.ndarray, nthreads: int = 0):
    """Per-ray y (k, 2), pixel (k, 2) and status (k,) for rays ij (k, 2)."""
    lens = np.ascontiguousarray(lens, dtype=np.float64).reshape(3, -1)
    ij = np.ascontiguousarray(ij, dtype=np.int64).reshape(-1, 2)
    k = ij.shape[0]
    mc, g, mp = _structs(job)
    y = np.empty((k, 2), dtype=np.float64)
    pix = np.empty((k, 2), dtype=np.int64)
    st = np.empty(k, dtype=np.int32)
    rc = lib().orc_shoot_rays(C.byref(mc), _ptr(lens), lens.shape[1], C.byref(g),
                              C.byref(mp), _ptr(ij), k, _ptr(y), _ptr(pix), _ptr(st),
                              nthreads)
    if rc != 0:
        raise ValueError("orc_shoot_rays: bad arguments")
    return y, pix, st


def navg(job) -> float:
    _, g, mp = _structs(job)
    return float(lib().orc_navg(C.byref(g), C.byref(mp)))


def magnification(job, counts: np.ndarray) -> np.ndarray:
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    if counts.size != job.npix * job.npix:
        raise ValueError(f"counts has {counts.size} values, the map {job.npix}^2")
    _, g, mp = _structs(job)
    mu = np.empty(counts.shape, dtype=np.float64)
    lib().orc_magnification(_ptr(counts), C.byref(g), C.byref(mp), _ptr(mu))
    return mu


def count_histogram(counts: np.ndarray, n_bins: int) -> np.ndarray:
    """MPD numerator: pixels per count value (last bin: >= n_bins - 1)."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    hist = np.empty(n_bins, dtype=np.int64)
    if lib().orc_count_histogram(_ptr(counts), counts.size, _ptr(hist), n_bins) != 0:
        raise ValueError("orc_count_histogram: bad arguments")
    return hist


def mpd(counts: np.ndarray, n_bins: int) -> np.ndarray:
    """Magnification probability distribution: frequency of each count value
    divided by the number of pixels (Sec. 3.2.1)."""
    return count_histogram(counts, n_bins) / float(np.asarray(counts).size)


def prob_sums(job, hist: np.ndarray, mu_lim) -> tuple[np.ndarray, np.ndarray]:
    """Pixels with mu < mu_lim and with mu > mu_lim for each mu_lim."""
    hist = np.ascontiguousarray(hist, dtype=np.int64)
    lim = np.ascontiguousarray(np.atleast_1d(mu_lim), dtype=np.float64)
    below = np.empty(lim.size, dtype=np.int64)
    above = np.empty(lim.size, dtype=np.int64)
    rc = lib().orc_prob_sums(_ptr(hist), hist.size, navg(job), _ptr(lim), lim.size,
                             _ptr(below), _ptr(above))
    if rc != 0:
        raise ValueError("orc_prob_sums: bad arguments or threshold in the overflow bin")
    return below, above


def mu_th(kappa: float, gamma: float) -> float:
    """Macro-magnification 1/((1-kappa)^2 - gamma^2) (Sec. 4.4)."""
    return 1.0 / ((1.0 - kappa) ** 2 - gamma ** 2)


# --------------------------------------------------------------------------
# finite source: profiles, Eq. 6, pixelFlux, MPD of a convolved map
# --------------------------------------------------------------------------

def _profile(prof) -> Profile:
    return Profile(prof.type, prof.supersample, prof.r_out, prof.r_in, prof.sigma1,
                   prof.sigma2, prof.r_scale, prof.index)


def profile_half(prof, w: float) -> int:
    h = int(lib().orc_profile_half(C.byref(_profile(prof)), w))
    if h < 0:
        raise ValueError("orc_profile_half: bad profile")
    return h


def profile_kernel(prof, w: float):
    """Source profile binned to map pixels of side w (Sec. 2.4): returns the
    normalised kernel (2h+1, 2h+1), row offset a + h, column b + h, and the
    unnormalised brightness sum over the samples."""
    h = profile_half(prof, w)
    k = np.empty((2 * h + 1, 2 * h + 1), dtype=np.float64)
    raw = C.c_double(0.0)
    if lib().orc_profile_kernel(C.byref(_profile(prof)), w, h, _ptr(k), C.byref(raw)) != 0:
        raise ValueError("orc_profile_kernel: bad arguments")
    return k, float(raw.value)


def convolve_direct(m: np.ndarray, k: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Eq. 6 as a cyclic convolution, summed directly in FP64."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    k = np.ascontiguousarray(k, dtype=np.float64)
    n = m.shape[0]
    h = (k.shape[0] - 1) // 2
    if m.shape != (n, n) or k.shape != (2 * h + 1, 2 * h + 1):
        raise ValueError("square map and odd square kernel expected")
    c = np.empty_like(m)
    if lib().orc_convolve_direct(_ptr(m), n, _ptr(k), h, _ptr(c), nthreads) != 0:
        raise ValueError("orc_convolve_direct: bad arguments (kernel wider than the map?)")
    return c


def convolve_counts_at(counts: np.ndarray, scale: float, k: np.ndarray,
                       qp: np.ndarray) -> np.ndarray:
    """Eq. 6 at the pixels qp (cnt, 2) = (row q, column p) of scale * counts."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    k = np.ascontiguousarray(k, dtype=np.float64)
    qp = np.ascontiguousarray(qp, dtype=np.int64).reshape(-1, 2)
    n = counts.shape[0]
    h = (k.shape[0] - 1) // 2
    out = np.empty(qp.shape[0], dtype=np.float64)
    if lib().orc_convolve_counts_at(_ptr(counts), scale, n, _ptr(k), h, _ptr(qp),
                                    qp.shape[0], _ptr(out)) != 0:
        raise ValueError("orc_convolve_counts_at: bad arguments")
    return out


def convolve_fft(m: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Eq. 6 literally, C = F^-1[F(M) F(K)], with numpy's FP64 FFT: the kernel
    is placed in an n x n image of zeros with its centre on pixel (0, 0)."""
    m = np.asarray(m, dtype=np.float64)
    n = m.shape[0]
    h = (k.shape[0] - 1) // 2
    img = np.zeros((n, n), dtype=np.float64)
    for a in range(-h, h + 1):
        for b in range(-h, h + 1):
            img[a % n, b % n] += k[a + h, b + h]
    return np.real(np.fft.ifft2(np.fft.fft2(m) * np.fft.fft2(img)))


def pixel_locations(seed: int, npix: int, k: int) -> np.ndarray:
    """pixelFlux locations (k, 2) = (x column, y row), int16."""
    if not 1 <= npix <= 32767:
        raise ValueError("pixelFlux locations are int16: npix <= 32767")
    xy = np.empty((k, 2), dtype=np.int16)
    lib().orc_pixel_locations(seed, npix, k, _ptr(xy))
    return xy


def value_histogram(v: np.ndarray, edges: np.ndarray) -> np.ndarray:
    """hist[b] = values with exactly b edges at or below them (float32 values
    and edges; NaN in bin 0)."""
    v = np.ascontiguousarray(v, dtype=np.float32).ravel()
    edges = np.ascontiguousarray(edges, dtype=np.float32)
    hist = np.empty(edges.size + 1, dtype=np.int64)
    if lib().orc_value_histogram(_ptr(v), v.size, _ptr(edges), edges.size, _ptr(hist)) != 0:
        raise ValueError("orc_value_histogram: bad arguments (edges not ascending?)")
    return hist


# --------------------------------------------------------------------------
# indexed maps (App. B) and map previews / colorbar (Sec. 3.2.1, Sec. 4.6)
# --------------------------------------------------------------------------

def index_bits(distinct: int) -> int:
    return int(lib().orc_index_bits(distinct))


def index_words(n: int, bits: int) -> int:
    return int(lib().orc_index_words(n, bits))


def index_encode(counts: np.ndarray, bits: int = 0):
    """(table (D,) int32 ascending distinct counts, words uint32, bits): the
    indexed map at `bits` per pixel (0: the fewest that hold D indices)."""
    counts = np.ascontiguousarray(counts, dtype=np.int32).ravel()
    table = np.empty(max(1, counts.size), dtype=np.int32)
    d = int(lib().orc_index_table(_ptr(counts), counts.size, _ptr(table)))
    if d < 1:
        raise ValueError("orc_index_table: empty map or negative count")
    table = table[:d].copy()
    b = bits or index_bits(d)
    words = np.empty(index_words(counts.size, b), dtype=np.uint32)
    if lib().orc_index_encode(_ptr(counts), counts.size, _ptr(table), d, b, _ptr(words)) != 0:
        raise ValueError("orc_index_encode: bad arguments")
    return table, words, b


def index_decode(words: np.ndarray, n: int, bits: int, table: np.ndarray) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype=np.uint32)
    table = np.ascontiguousarray(table, dtype=np.int32)
    out = np.empty(n, dtype=np.int32)
    if lib().orc_index_decode(_ptr(words), n, bits, _ptr(table), table.size, _ptr(out)) != 0:
        raise ValueError("orc_index_decode: index outside the table or bad arguments")
    return out


def colorbar_lut(pos, rgb) -> np.ndarray:
    """256 x 3 uint8 colour table from stops (positions 0..255, RGB rows)."""
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8).reshape(-1, 3)
    lut = np.empty((256, 3), dtype=np.uint8)
    if lib().orc_colorbar_lut(_ptr(pos), _ptr(rgb), pos.size, _ptr(lut)) != 0:
        raise ValueError("orc_colorbar_lut: stops must run from 0 to 255, non-decreasing")
    return lut


def sample_gray(m: np.ndarray, s: int, thr: np.ndarray) -> np.ndarray:
    """s x s grayscale preview of an int32 count map (float64 thresholds) or
    a float32 map (float32 thresholds): 255 ascending thresholds."""
    n = m.shape[0]
    gray = np.empty((s, s), dtype=np.uint8)
    if m.dtype == np.int32:
        t = np.ascontiguousarray(thr, dtype=np.float64)
        rc = lib().orc_sample_gray_counts(_ptr(np.ascontiguousarray(m)), n, s, _ptr(t),
                                          _ptr(gray))
    else:
        t = np.ascontiguousarray(thr, dtype=np.float32)
        rc = lib().orc_sample_gray_f32(_ptr(np.ascontiguousarray(m, dtype=np.float32)), n, s,
                                       _ptr(t), _ptr(gray))
    if rc != 0 or t.size != 255:
        raise ValueError("sample_gray: bad arguments (255 thresholds expected)")
    return gray


def colorize(gray: np.ndarray, lut: np.ndarray) -> np.ndarray:
    gray = np.ascontiguousarray(gray, dtype=np.uint8)
    lut = np.ascontiguousarray(lut, dtype=np.uint8)
    rgba = np.empty(gray.shape + (4,), dtype=np.uint8)
    lib().orc_colorize(_ptr(gray), gray.size, _ptr(lut), _ptr(rgba))
    return rgba


def index_pack(counts: np.ndarray, table: np.ndarray, bits: int) -> np.ndarray:
    """Indexed map of counts against a given ascending table at `bits`."""
    counts = np.ascontiguousarray(counts, dtype=np.int32).ravel()
    table = np.ascontiguousarray(table, dtype=np.int32)
    words = np.empty(index_words(counts.size, bits), dtype=np.uint32)
    if lib().orc_index_encode(_ptr(counts), counts.size, _ptr(table), table.size, bits,
                              _ptr(words)) != 0:
        raise ValueError("orc_index_encode: a count is not in the table, or too few bits")
    return words

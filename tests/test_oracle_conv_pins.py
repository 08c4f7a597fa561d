"""Pins of the finite-source oracle (Sec. 2.4, Eq. 6; profiles of Sec. 2.5
item 3) against things fixed outside it: exact lattice counts, the closed-form
pixel integrals of a Gaussian, radial integrals by quadrature, scipy's direct
wrap-around convolution, numpy's searchsorted and the SplitMix64 definition.
CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.integrate
import scipy.signal
import scipy.special

import oracle
import workloads as W


def uniform(r_out, S, r_in=0.0):
    return W.Profile(name="u", type=W.PROFILE_UNIFORM, supersample=S, r_out=r_out, r_in=r_in)


def lattice_kernel(r_out, r_in, w, S):
    """Inside-sample counts of a uniform disc with integer arithmetic only:
    sample (u1, u2) (odd offsets, spacing w / 2S) is inside when
    rho_in^2 <= u1^2 + u2^2 < rho_out^2, rho = 2 S r / w (exact rationals
    for dyadic r and w)."""
    ro2 = (2 * S * Fraction(r_out) / Fraction(w)) ** 2
    ri2 = (2 * S * Fraction(r_in) / Fraction(w)) ** 2
    u2min = (S + 1) % 2
    h = 0
    while ((2 * (h + 1) - 1) * S + 1) ** 2 + u2min ** 2 < ro2:
        h += 1
    d = 2 * h + 1
    cnt = np.zeros((d, d), dtype=np.int64)
    for a in range(-h, h + 1):
        for b in range(-h, h + 1):
            c = 0
            for t in range(S):
                for s in range(S):
                    u1 = 2 * (b * S + s) + 1 - S
                    u2 = 2 * (a * S + t) + 1 - S
                    q = u1 * u1 + u2 * u2
                    c += ri2 <= q < ro2
            cnt[a + h, b + h] = c
    return h, cnt


@pytest.mark.parametrize("S", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("r_pix,rin_pix", [(3.5, 0.0), (5.25, 1.5), (2.0, 0.0)])
def test_uniform_disc_is_an_exact_lattice_count(S, r_pix, rin_pix):
    w = 2.0 ** -8                       # dyadic: rho = 2 S r / w is an exact integer
    r_out, r_in = r_pix * w, rin_pix * w
    h_ref, cnt = lattice_kernel(r_out, r_in, w, S)
    prof = uniform(r_out, S, r_in)
    assert oracle.profile_half(prof, w) == h_ref
    k, raw = oracle.profile_kernel(prof, w)
    assert raw == cnt.sum()
    assert np.array_equal(k, cnt / float(cnt.sum()))


def test_uniform_disc_area_converges():
    w = 0.0025
    for r in (0.01, 0.0237, 0.05):
        for S in (4, 16):
            k, raw = oracle.profile_kernel(uniform(r, S), w)
            area = raw * (w / S) ** 2
            # samples off by at most one sample cell along the rim
            bound = 2 * math.pi * r * math.sqrt(2) * (w / S) + 4 * (w / S) ** 2
            assert abs(area - math.pi * r * r) <= bound, (r, S, area)


def test_point_source_is_the_unit_impulse():
    w = 0.01
    for r in (0.001, 0.005):                    # diameter <= pixel side
        k, _ = oracle.profile_kernel(uniform(r, 8), w)
        assert k.shape == (1, 1) and k[0, 0] == 1.0
    # just wider than a pixel but inside the central pixel's samples: 1 x 1
    k, _ = oracle.profile_kernel(uniform(0.0051, 8), w)
    assert k.shape == (1, 1) and k[0, 0] == 1.0
    k, _ = oracle.profile_kernel(uniform(0.0075, 8), w)
    assert k.shape == (3, 3) and abs(k.sum() - 1.0) < 1e-15 and k[1, 1] > k[0, 1] > k[0, 0]


def gauss_cell(lo, hi, sigma):
    return 0.5 * (scipy.special.erf(hi / (math.sqrt(2) * sigma)) -
                  scipy.special.erf(lo / (math.sqrt(2) * sigma)))


@pytest.mark.parametrize("S", [4, 16])
def test_gaussian_matches_erf_pixel_integrals(S):
    w = 0.0025
    s1, s2 = 0.006, 0.0035                       # anisotropic: an axis swap fails
    prof = W.Profile(type=W.PROFILE_GAUSSIAN, supersample=S, r_out=8 * s1, sigma1=s1, sigma2=s2)
    k, _ = oracle.profile_kernel(prof, w)
    h = (k.shape[0] - 1) // 2
    off = (np.arange(-h, h + 1) - 0.5) * w
    g1 = np.array([gauss_cell(o, o + w, s1) for o in off])    # columns, y1
    g2 = np.array([gauss_cell(o, o + w, s2) for o in off])    # rows, y2
    exact = np.outer(g2, g1)
    # composite midpoint rule, step w / S, per axis: |err| <= w (w/S)^2 / 24 max|g''|
    e1 = w * (w / S) ** 2 / 24 / (math.sqrt(2 * math.pi) * s1 ** 3)
    e2 = w * (w / S) ** 2 / 24 / (math.sqrt(2 * math.pi) * s2 ** 3)
    bound = 2 * (e1 + e2) + 1e-12
    assert np.abs(k - exact).max() <= bound
    # sigma1 <-> sigma2 transposes the kernel
    kt, _ = oracle.profile_kernel(prof.with_(sigma1=s2, sigma2=s1), w)
    assert np.allclose(kt, k.T, rtol=0, atol=1e-15)
    # point symmetry of every profile
    assert np.allclose(k, k[::-1, ::-1], rtol=0, atol=1e-15)


def test_power_law_radial_integral():
    w, S = 0.001, 8
    prof = W.Profile(type=W.PROFILE_POWER_LAW, supersample=S, r_out=0.05, r_in=0.004,
                     r_scale=0.01, index=1.5)
    _, raw = oracle.profile_kernel(prof, w)
    p = prof.index
    exact = 2 * math.pi * prof.r_scale ** p * (prof.r_out ** (2 - p) - prof.r_in ** (2 - p)) / (2 - p)
    assert abs(raw * (w / S) ** 2 / exact - 1) < 5e-3


def test_thin_disc_radial_integral():
    w, S = 0.001, 8
    prof = W.Profile(type=W.PROFILE_THIN_DISC, supersample=S, r_out=0.06, r_in=0.002,
                     r_scale=0.01)

    def ring(r):
        xi = (r / prof.r_scale) ** 0.75 * (1 - math.sqrt(prof.r_in / r)) ** -0.25
        return 2 * math.pi * r / math.expm1(xi)

    exact, _ = scipy.integrate.quad(ring, prof.r_in * (1 + 1e-12), prof.r_out, limit=400)
    _, raw = oracle.profile_kernel(prof, w)
    assert abs(raw * (w / S) ** 2 / exact - 1) < 5e-3
    # the brightness vanishes at the inner edge and falls outward beyond r_scale
    k, _ = oracle.profile_kernel(prof, w)
    h = (k.shape[0] - 1) // 2
    assert k[h, h] < k[h, h + 6] and k[h, h + 20] < k[h, h + 6]


def test_bad_profiles_rejected():
    for prof in (W.Profile(type=W.PROFILE_THIN_DISC, r_out=0.1, r_in=0.0, r_scale=0.01),
                 W.Profile(type=W.PROFILE_GAUSSIAN, r_out=0.1, sigma1=0.0),
                 W.Profile(type=7, r_out=0.1), W.Profile(supersample=0),
                 W.Profile(type=W.PROFILE_UNIFORM, r_out=0.1, r_in=0.2)):
        with pytest.raises(ValueError):
            oracle.profile_kernel(prof, 0.01)


def rand_kernel(rng, h):
    k = rng.random((2 * h + 1, 2 * h + 1))      # not symmetric: orientation matters
    return k / k.sum()


@pytest.mark.parametrize("n,h", [(37, 5), (64, 3), (50, 24)])
def test_direct_convolution_matches_scipy_and_fft(n, h):
    rng = np.random.default_rng(n * 100 + h)
    m = rng.random((n, n)) * 100
    k = rand_kernel(rng, h)
    c = oracle.convolve_direct(m, k)
    ref = scipy.signal.convolve2d(m, k, mode="same", boundary="wrap")
    assert np.allclose(c, ref, rtol=1e-13, atol=0)
    assert np.allclose(oracle.convolve_fft(m, k), c, rtol=1e-11, atol=1e-11)
    assert abs(c.sum() - m.sum()) <= 1e-9 * m.sum()          # sum K = 1


def test_impulse_and_shifted_impulse():
    rng = np.random.default_rng(3)
    m = rng.random((40, 40))
    h = 4
    k = np.zeros((2 * h + 1, 2 * h + 1))
    k[h, h] = 1.0
    assert np.array_equal(oracle.convolve_direct(m, k), m)
    k[:] = 0
    k[h + 2, h - 3] = 1.0             # a = +2 rows, b = -3 columns
    assert np.array_equal(oracle.convolve_direct(m, k), np.roll(m, (2, -3), axis=(0, 1)))


def test_counts_at_matches_the_full_map():
    job = W.CONV_SMALL
    counts = W.count_map(job)
    k, _ = oracle.profile_kernel(job.profile, job.pixel)
    scale = 1.0 / 37.5
    full = oracle.convolve_direct(counts * scale, k)
    rng = np.random.default_rng(1)
    qp = np.stack([rng.integers(0, job.npix, 50), rng.integers(0, job.npix, 50)], axis=1)
    at = oracle.convolve_counts_at(counts, scale, k, qp)
    assert np.allclose(at, full[qp[:, 0], qp[:, 1]], rtol=1e-13, atol=0)


def test_kernel_wider_than_map_rejected():
    with pytest.raises(ValueError):
        oracle.convolve_direct(np.ones((8, 8)), np.ones((9, 9)) / 81)


def test_pixel_locations_follow_splitmix64():
    seed, npix, k = 12345, 10000, 2000
    xy = oracle.pixel_locations(seed, npix, k)
    for t in (0, 1, 999, 1999):
        hx = oracle.splitmix64(seed, 2 * t) >> 32
        hy = oracle.splitmix64(seed, 2 * t + 1) >> 32
        assert xy[t, 0] == (hx * npix) >> 32 and xy[t, 1] == (hy * npix) >> 32
    assert xy.min() >= 0 and xy.max() < npix
    # uniform over the map: chi^2 over 10 x 10 cells
    cells = np.histogram2d(xy[:, 0], xy[:, 1], bins=10, range=[[0, npix], [0, npix]])[0]
    chi2 = ((cells - k / 100) ** 2 / (k / 100)).sum()
    assert chi2 < 160                      # 99 dof; p ~ 1e-4
    with pytest.raises(ValueError):
        oracle.pixel_locations(1, 40000, 4)


def test_value_histogram_matches_searchsorted():
    rng = np.random.default_rng(9)
    v = (10 ** rng.uniform(-2, 3, 100000)).astype(np.float32)
    edges = W.log_edges(-1.5, 2.5, 64)
    v[:edges.size] = edges                  # values exactly on edges
    v[edges.size] = np.nan
    v[edges.size + 1] = -1.0
    hist = oracle.value_histogram(v, edges)
    b = np.searchsorted(edges, v, side="right")
    b[np.isnan(v)] = 0
    assert np.array_equal(hist, np.bincount(b, minlength=edges.size + 1))
    assert hist.sum() == v.size
    with pytest.raises(ValueError):
        oracle.value_histogram(v, edges[::-1])

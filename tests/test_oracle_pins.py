"""Pins of the FP64 oracle against things the paper's physics and the
mathematics fix, independently of the oracle's own code.

P1  pure macromodel (no lenses): exact lattice-point counts per pixel
P2  single point lens: Paczynski magnification, circular symmetry, mass scaling
P3  point lens + shear (Chang-Refsdal): image magnifications from the quartic
P4  random field: mean magnification -> 1/|(1-kappa)^2 - gamma^2|
P5  conservation of the ray count, singular rays
P6  mirror symmetry of the map under reflection of the lens field
P7  exact rational arithmetic on tiny inputs
P8  superposition of the deflection
plus the lens-field generator (Eq. 3 count, disk uniformity, Salpeter law)
and the paper's printed geometry/storage numbers (tests/golden).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats as sps

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def job(**kw):
    base = dict(name="pin", kappa_star=0.0, kappa_s=0.0, gamma=0.0, n_lens=0,
                lens_radius=1.0, seed=1)
    base.update(kw)
    return W.MapJob(**base)


def point_lens(m=1.0, x1=0.0, x2=0.0):
    return np.array([[x1], [x2], [m]], dtype=np.float64)


# ---------------------------------------------------------------- P1 -----

def lattice_counts_1d(a: Fraction, c: Fraction, h: Fraction, n: int,
                      y0: Fraction, w: Fraction, npix: int) -> list[int]:
    """Closed-form number of cell-centred rays x_i = c - h + (i+1/2) d,
    d = 2h/n, whose image a*x_i falls in the half-open pixel
    [y0 + p w, y0 + (p+1) w), for each p (exact rational arithmetic)."""
    d = 2 * h / n
    out = []
    for p in range(npix):
        lo, hi = y0 + p * w, y0 + (p + 1) * w
        if a > 0:
            # lo <= a x_i < hi  <=>  A <= i < B
            A = ((lo / a) - (c - h)) / d - Fraction(1, 2)
            B = ((hi / a) - (c - h)) / d - Fraction(1, 2)
            first = max(0, math.ceil(A))
            last = min(n, math.ceil(B))  # exclusive
        else:
            # lo <= a x_i < hi  <=>  hi/a < x_i <= lo/a  <=>  A < i <= B
            A = ((hi / a) - (c - h)) / d - Fraction(1, 2)
            B = ((lo / a) - (c - h)) / d - Fraction(1, 2)
            first = max(0, math.floor(A) + 1)
            last = min(n, math.floor(B) + 1)
        out.append(max(0, last - first))
    return out


@pytest.mark.parametrize("kappa_s,gamma", [(0.25, 0.125), (0.25, 0.25), (0.25, 0.875),
                                           (0.0, 0.0), (1.5, 0.25)])
def test_p1_pure_macro_exact_lattice(kappa_s, gamma):
    # dyadic geometry: every FP64 operation of the oracle is exact
    j = job(kappa_s=kappa_s, gamma=gamma, n1=512, n2=384, c1=0.5, c2=-0.25,
            half1=8.0, half2=6.0, mc1=0.25, mc2=-0.5, width=8.0, npix=64)
    counts, st = oracle.shoot(j, np.zeros((3, 0)))
    a1 = Fraction(1) - Fraction(gamma) - Fraction(kappa_s)
    a2 = Fraction(1) + Fraction(gamma) - Fraction(kappa_s)
    w = Fraction(j.width) / j.npix
    e1 = lattice_counts_1d(a1, Fraction(j.c1), Fraction(j.half1), j.n1,
                           Fraction(j.mc1) - Fraction(j.width) / 2, w, j.npix)
    e2 = lattice_counts_1d(a2, Fraction(j.c2), Fraction(j.half2), j.n2,
                           Fraction(j.mc2) - Fraction(j.width) / 2, w, j.npix)
    expect = np.outer(np.array(e2, dtype=np.int64), np.array(e1, dtype=np.int64))
    assert np.array_equal(counts.astype(np.int64), expect)   # row q <-> y2
    assert st["n_in"] == expect.sum()
    assert st["n_in"] + st["n_out"] + st["n_singular"] == j.n1 * j.n2
    assert st["n_singular"] == 0


def test_p1_map_edges_are_half_open():
    # identity mapping (no lenses, no shear or smooth matter) and dyadic
    # geometry: ray i lands exactly on pixel edge i, so the rays on the
    # lower and left borders are in and those exactly on the upper and right
    # borders are out (pixels are [lo, hi))
    j = job(n1=8, n2=8, half1=1.0, half2=1.0, width=1.75, npix=7)
    counts, st = oracle.shoot(j, np.zeros((3, 0)))
    assert np.array_equal(counts, np.ones((7, 7), dtype=counts.dtype))
    assert (st["n_in"], st["n_out"], st["n_singular"]) == (49, 15, 0)


def test_p1_interior_magnification_is_macro():
    # w / (a d) integer on both axes -> every interior pixel has the same
    # count and mu = 1/|a1 a2| exactly (Eq. 4 with the unlensed N_avg)
    # (rectangular ray cells: d1 = 1/32, d2 = 1/16)
    j = job(kappa_s=0.25, gamma=0.25, n1=512, n2=256, half1=8.0, half2=8.0,
            width=8.0, npix=64)
    counts, _ = oracle.shoot(j, np.zeros((3, 0)))
    mu = oracle.magnification(j, counts)
    assert oracle.navg(j) == 8.0                  # (w/d1)(w/d2) = 4 * 2
    a1, a2 = 0.5, 1.0
    covered = counts > 0
    # pixels whose pre-image is fully inside the ray grid
    assert covered.sum() > 100
    vals = np.unique(mu[covered])
    assert np.all(vals == 1.0 / abs(a1 * a2))


# ---------------------------------------------------------------- P2 -----

def paczynski(u):
    """Total magnification of a point lens for a source at distance u
    (Einstein units): (u^2 + 2) / (u sqrt(u^2 + 4))."""
    return (u * u + 2.0) / (u * np.sqrt(u * u + 4.0))


def pixel_average(fn, j, ngl=8):
    """Gauss-Legendre average of fn(y1, y2) over every map pixel."""
    xg, wg = np.polynomial.legendre.leggauss(ngl)
    w = j.width / j.npix
    y0 = np.array([j.mc1 - j.width / 2, j.mc2 - j.width / 2])
    c = (np.arange(j.npix) + 0.5) * w
    acc = np.zeros((j.npix, j.npix))
    for a, wa in zip(xg, wg):
        for b, wb in zip(xg, wg):
            y1 = y0[0] + c[None, :] + a * w / 2
            y2 = y0[1] + c[:, None] + b * w / 2
            acc += wa * wb * fn(y1, y2)
    return acc / 4.0


@pytest.mark.parametrize("m", [1.0, 4.0])
def test_p2_point_lens_paczynski(m):
    scale = math.sqrt(m)            # Einstein radius of a lens of mass m
    j = job(n1=4096, n2=4096, half1=4.0 * scale, half2=4.0 * scale,
            width=4.0 * scale, npix=32)
    counts, st = oracle.shoot(j, point_lens(m))
    mu = oracle.magnification(j, counts)
    expect = pixel_average(lambda y1, y2: paczynski(np.hypot(y1, y2) / scale), j, ngl=12)
    # the four pixels touching the lens (integrable 1/u peak) are excluded
    mask = np.ones_like(mu, dtype=bool)
    mask[15:17, 15:17] = False
    rel = np.abs(mu - expect) / expect
    assert rel[mask].max() < 0.02
    assert np.abs(mu[mask].mean() / expect[mask].mean() - 1.0) < 2e-3
    # symmetry of a centred point lens on a centred square grid: exact
    assert np.array_equal(counts, counts.T)
    assert np.array_equal(counts, counts[:, ::-1])
    assert np.array_equal(counts, counts[::-1, :])
    assert st["n_singular"] == 0


# ---------------------------------------------------------------- P3 -----

def chang_refsdal_mu(y1, y2, g, tol=1e-9):
    """Total magnification of a point lens (m=1) with shear g for a source
    at (y1, y2), from the images: x1 = y1/(1-g-s), x2 = y2/(1+g-s) with
    s = 1/|x|^2 solving s y1^2 (1+g-s)^2 + s y2^2 (1-g-s)^2
    = (1-g-s)^2 (1+g-s)^2; each image contributes 1/|det A| with
    A = diag(1-g-s, 1+g-s) + 2 s^2 x x^T."""
    y1 = np.asarray(y1, dtype=np.float64).ravel()
    y2 = np.asarray(y2, dtype=np.float64).ravel()
    out = np.empty_like(y1)
    nimg = np.empty(y1.shape, dtype=np.int64)
    P = np.polynomial.polynomial
    for k in range(y1.size):
        a = np.array([1 - g, -1.0])      # (1-g-s) as a poly in s
        b = np.array([1 + g, -1.0])      # (1+g-s)
        s_ = np.array([0.0, 1.0])
        lhs = P.polyadd(P.polymul(s_ * y1[k] ** 2, P.polymul(b, b)),
                        P.polymul(s_ * y2[k] ** 2, P.polymul(a, a)))
        rhs = P.polymul(P.polymul(a, a), P.polymul(b, b))
        poly = P.polysub(lhs, rhs)
        roots = P.polyroots(poly)
        tot = 0.0
        cnt = 0
        for r in roots:
            if abs(r.imag) > 1e-7 * max(1.0, abs(r.real)):
                continue
            s = r.real
            if s <= 0:
                continue
            x1 = y1[k] / (1 - g - s)
            x2 = y2[k] / (1 + g - s)
            r2 = x1 * x1 + x2 * x2
            # keep only true images of the lens equation
            if abs(1.0 / r2 - s) > tol * max(1.0, s):
                continue
            res1 = (1 - g) * x1 - x1 / r2 - y1[k]
            res2 = (1 + g) * x2 - x2 / r2 - y2[k]
            if math.hypot(res1, res2) > 1e-8:
                continue
            A11 = 1 - g - s + 2 * s * s * x1 * x1
            A22 = 1 + g - s + 2 * s * s * x2 * x2
            A12 = 2 * s * s * x1 * x2
            tot += 1.0 / abs(A11 * A22 - A12 * A12)
            cnt += 1
        out[k] = tot
        nimg[k] = cnt
    return out, nimg


def test_p3_chang_refsdal():
    g = 0.3
    j = job(gamma=g, n1=6144, n2=4096, half1=6.0, half2=4.0, width=4.0, npix=32)
    counts, st = oracle.shoot(j, point_lens(1.0))
    mu = oracle.magnification(j, counts)
    w = j.width / j.npix
    xg, wg = np.polynomial.legendre.leggauss(4)
    rng = np.random.default_rng(7)
    # a seeded sample of pixels (the quartic solve is slow in Python)
    picks = [(q, p) for q in range(j.npix) for p in range(j.npix)]
    picks = [picks[t] for t in rng.choice(len(picks), size=80, replace=False)]
    checked = 0
    for q, p in picks:
        y1c = j.mc1 - j.width / 2 + (p + 0.5) * w
        y2c = j.mc2 - j.width / 2 + (q + 0.5) * w
        Y1 = (y1c + xg[None, :] * w / 2) * np.ones((4, 1))
        Y2 = (y2c + xg[:, None] * w / 2) * np.ones((1, 4))
        vals, nimg = chang_refsdal_mu(Y1, Y2, g)
        if len(set(nimg.tolist())) != 1 or vals.max() > 1.3 * vals.min():
            continue  # pixel crosses a caustic or a steep gradient
        avg = float((vals.reshape(4, 4) * np.outer(wg, wg)).sum() / 4.0)
        assert abs(mu[q, p] - avg) / avg < 0.02, (q, p, mu[q, p], avg)
        checked += 1
    assert checked >= 40
    # mirror symmetries of the Chang-Refsdal lens on a centred grid (exact)
    assert np.array_equal(counts, counts[:, ::-1])
    assert np.array_equal(counts, counts[::-1, :])
    # the shear direction: the map is not symmetric under x1 <-> x2
    assert not np.array_equal(counts, counts.T)


def test_p3_far_field_limit():
    # far from the lens the magnification tends to 1/(1-g^2)
    g = 0.3
    vals, nimg = chang_refsdal_mu([60.0, 0.0, 45.0], [0.0, 60.0, 45.0], g)
    assert np.all(nimg == 2)
    assert np.allclose(vals, 1.0 / (1 - g * g), rtol=2e-3)
    # and the oracle's deflection is that of a unit point mass there
    a, _ = oracle.deflection(point_lens(1.0), np.array([[60.0, 0.0]]))
    assert np.allclose(a, [[1.0 / 60.0, 0.0]], rtol=1e-15)


# ---------------------------------------------------------------- P4 -----

@pytest.mark.slow
def test_p4_mean_magnification():
    kstar, ks, g = 0.3, 0.1, 0.2
    kappa = kstar + ks
    mu_th = 1.0 / abs((1 - kappa) ** 2 - g ** 2)
    # ray rectangle = pre-image of the map plus a 4 R_E margin
    h1 = 2.0 / abs(1 - kappa - g) + 4.0
    h2 = 2.0 / abs(1 - kappa + g) + 4.0
    d = 1.0 / 128
    n1 = int(round(2 * h1 / d))
    n2 = int(round(2 * h2 / d))
    means = []
    for seed in range(8):
        j = W.MapJob(name="p4", kappa_star=kstar, kappa_s=ks, gamma=g, n_lens=0,
                     lens_radius=math.sqrt(200 / kstar), seed=100 + seed,
                     n1=n1, n2=n2, half1=n1 * d / 2, half2=n2 * d / 2,
                     width=4.0, npix=64)
        lens = oracle.make_lenses(j)
        assert lens.shape[1] == 200
        counts, st = oracle.shoot(j, lens)
        assert st["n_in"] + st["n_out"] + st["n_singular"] == n1 * n2
        means.append(oracle.magnification(j, counts).mean())
    means = np.array(means)
    sem = means.std(ddof=1) / math.sqrt(len(means))
    assert abs(means.mean() - mu_th) <= 3 * sem + 0.02 * mu_th, (means, mu_th)


# ---------------------------------------------------------------- P5 -----

def test_p5_conservation_and_singular():
    j = W.PARITY.with_(n1=256, n2=256)
    lens = oracle.make_lenses(j)
    counts, st = oracle.shoot(j, lens)
    assert counts.sum() == st["n_in"]
    assert st["n_in"] + st["n_out"] + st["n_singular"] == j.n1 * j.n2
    # a lens placed exactly on the ray (i, j) = (3, 5) of a dyadic grid
    jd = job(n1=64, n2=64, half1=4.0, half2=4.0, width=4.0, npix=16)
    d = 2 * 4.0 / 64
    x1 = -4.0 + 3.5 * d
    x2 = -4.0 + 5.5 * d
    lens = np.array([[x1, 1.0], [x2, -2.0], [1.0, 1.0]])
    counts, st = oracle.shoot(jd, lens)
    assert st["n_singular"] == 1
    assert st["n_in"] + st["n_out"] + 1 == 64 * 64
    y, pix, status = oracle.shoot_rays(jd, lens, np.array([[3, 5], [4, 5]]))
    assert status[0] == 2 and np.all(np.isnan(y[0])) and np.all(pix[0] == -1)
    assert status[1] in (0, 1)


# ---------------------------------------------------------------- P6 -----

def test_p6_mirror_symmetry():
    j = W.PARITY.with_(n1=1024, n2=1024, half1=8.0, half2=8.0)
    lens = oracle.make_lenses(j)
    c0, _ = oracle.shoot(j, lens)
    m2 = lens.copy()
    m2[1] = -m2[1]
    c2, _ = oracle.shoot(j, m2)
    assert np.array_equal(c2, c0[::-1, :])
    m1 = lens.copy()
    m1[0] = -m1[0]
    c1, _ = oracle.shoot(j, m1)
    assert np.array_equal(c1, c0[:, ::-1])


# ---------------------------------------------------------------- P7 -----

def test_p7_exact_rationals_tiny():
    rng = np.random.default_rng(11)
    n = 5
    lens = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n),
                     rng.uniform(0.2, 1.5, n)])
    j = job(kappa_s=0.15, gamma=0.35, n1=16, n2=12, c1=0.1, c2=-0.2,
            half1=2.5, half2=1.9, mc1=0.05, mc2=0.1, width=3.0, npix=24)
    ij = np.array([(i, jj) for jj in range(j.n2) for i in range(j.n1)], dtype=np.int64)
    y, pix, st = oracle.shoot_rays(j, lens, ij)
    F = Fraction
    L = [[F(float(v)) for v in row] for row in lens]
    d1 = F(2) * F(j.half1) / j.n1
    d2 = F(2) * F(j.half2) / j.n2
    w = F(j.width) / j.npix
    y01 = F(j.mc1) - F(j.width) / 2
    y02 = F(j.mc2) - F(j.width) / 2
    for t, (i, jj) in enumerate(ij):
        x1 = F(j.c1) - F(j.half1) + (i + F(1, 2)) * d1
        x2 = F(j.c2) - F(j.half2) + (jj + F(1, 2)) * d2
        a1 = a2 = F(0)
        for k in range(n):
            dx, dy = x1 - L[0][k], x2 - L[1][k]
            r2 = dx * dx + dy * dy
            a1 += L[2][k] * dx / r2
            a2 += L[2][k] * dy / r2
        e1 = (1 - F(j.gamma) - F(j.kappa_s)) * x1 - a1
        e2 = (1 + F(j.gamma) - F(j.kappa_s)) * x2 - a2
        assert abs(float(e1) - y[t, 0]) <= 1e-13 * (1 + abs(float(e1)))
        assert abs(float(e2) - y[t, 1]) <= 1e-13 * (1 + abs(float(e2)))
        u, v = (e1 - y01) / w, (e2 - y02) / w
        inside = 0 <= u < j.npix and 0 <= v < j.npix
        near = min(abs(u - round(u)), abs(v - round(v))) < 1e-9
        if not near:
            assert (st[t] == 0) == inside
            if inside:
                assert pix[t, 0] == math.floor(u) and pix[t, 1] == math.floor(v)


# ---------------------------------------------------------------- P8 -----

def test_p8_superposition_and_massless_lens():
    rng = np.random.default_rng(5)
    A = np.stack([rng.uniform(-5, 5, 40), rng.uniform(-5, 5, 40), rng.uniform(0.1, 1, 40)])
    B = np.stack([rng.uniform(-5, 5, 30), rng.uniform(-5, 5, 30), rng.uniform(0.1, 1, 30)])
    x = rng.uniform(-3, 3, size=(200, 2))
    aA, _ = oracle.deflection(A, x)
    aB, _ = oracle.deflection(B, x)
    aAB, _ = oracle.deflection(np.concatenate([A, B], axis=1), x)
    assert np.allclose(aAB, aA + aB, rtol=1e-12, atol=1e-12)
    # a massless lens changes nothing; doubling every mass doubles alpha
    Z = np.concatenate([A, np.array([[0.3], [0.7], [0.0]])], axis=1)
    aZ, _ = oracle.deflection(Z, x)
    assert np.array_equal(aZ, aA)
    A2 = A.copy()
    A2[2] *= 2
    a2, _ = oracle.deflection(A2, x)
    assert np.allclose(a2, 2 * aA, rtol=1e-14, atol=0)


# ------------------------------------------------------- lens field -----

def test_splitmix64_published_value():
    # first output of SplitMix64 for seed 0, as published with the generator
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    u = np.array([oracle.u01(9, k) for k in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert sps.kstest(u, "uniform").pvalue > 1e-3


def test_lens_count_eq3():
    assert oracle.lens_count(0.6, 200.0) == 24000        # GERLUMPH-scale map
    assert oracle.lens_count(0.4, 280.0) == 31360
    assert oracle.lens_count(0.4, 11.0) == 48
    assert oracle.lens_count(0.3, 10.0, mean_mass=0.5) == 60
    assert oracle.lens_count(0.0, 10.0) == 0


def test_lens_disk_uniform():
    j = job(kappa_star=0.5, lens_radius=50.0, n_lens=20000, seed=21)
    lens = oracle.make_lenses(j)
    r2 = (lens[0] ** 2 + lens[1] ** 2) / 50.0 ** 2
    assert r2.max() < 1.0
    assert sps.kstest(r2, "uniform").pvalue > 1e-3          # P(r<s) = s^2/R^2
    phi = (np.arctan2(lens[1], lens[0]) + np.pi) / (2 * np.pi)
    assert sps.kstest(phi, "uniform").pvalue > 1e-3
    assert np.all(lens[2] == 1.0)
    # seeded: same seed -> same field, other seed -> other field
    assert np.array_equal(lens, oracle.make_lenses(j))
    assert not np.array_equal(lens, oracle.make_lenses(j.with_(seed=22)))


def test_lens_salpeter_masses():
    j = job(kappa_star=0.4, lens_radius=30.0, n_lens=50000, seed=3,
            mass_model=W.MASS_SALPETER, m_lo=0.1, m_hi=1.0, slope=2.35)
    lens = oracle.make_lenses(j)
    m = lens[2]
    assert abs(m.mean() - 1.0) < 1e-12                      # mean-normalised
    # undo the normalisation with the analytic mean of the truncated law
    a, lo, hi = 2.35, 0.1, 1.0
    mean_raw = ((hi ** (2 - a) - lo ** (2 - a)) / (2 - a)) / \
               ((hi ** (1 - a) - lo ** (1 - a)) / (1 - a))
    raw = m * mean_raw
    # the sample mean differs from the analytic mean by sampling noise only
    assert abs(m.max() / m.min() - raw.max() / raw.min()) < 1e-9
    cdf = lambda x: (np.clip(x, lo, hi) ** (1 - a) - lo ** (1 - a)) / (hi ** (1 - a) - lo ** (1 - a))
    # compare the shape: rescale so the sample range matches [lo, hi]
    scaled = m / m.min() * lo
    assert scaled.max() <= hi * (1 + 1e-3)
    assert sps.kstest(scaled, cdf).pvalue > 1e-3
    assert abs(m.mean() * mean_raw / raw.mean() - 1.0) < 1e-12


# ---------------------------------------------------------- golden -----

def test_paper_geometry_and_storage_numbers():
    gold = json.load(open(GOLDEN))
    ps = gold["pixel_span"]
    # pixel width w = W / npix in R_E, times R_E in cm
    w = ps["width_rein"] / ps["npix"]
    assert abs(w * ps["rein_cm"] - ps["pixel_cm"]) < 1e-6 * ps["pixel_cm"]
    mb = gold["map_bytes"]
    nbytes = mb["npix"] ** 2 * mb["bits"] // 8      # int32 counts, row-major
    assert round(nbytes / 2 ** 20) == mb["megabytes"]
    # every published maximum pixel count fits the int32 count buffer
    for k in ("GD0", "GD1", "GD2"):
        assert gold["max_ray_count"][k] < 2 ** 31 - 1


def test_magnification_eq4_navg():
    j = W.PARITY
    # N_avg: rays per pixel without lensing = (w/d1)(w/d2)
    w = j.width / j.npix
    d = 2 * j.half1 / j.n1
    assert abs(oracle.navg(j) - (w / d) ** 2) < 1e-12
    c = np.arange(j.npix * j.npix, dtype=np.int32).reshape(j.npix, j.npix) % 977
    mu = oracle.magnification(j, c)
    assert np.allclose(mu, c / oracle.navg(j), rtol=1e-15, atol=0)


# ------------------------------------------------------------------ MPD -----

def test_mpd_of_the_closed_form_macro_map():
    # the MPD of a pure-macromodel map follows from the exact lattice counts
    j = job(kappa_s=0.25, gamma=0.125, n1=512, n2=384, c1=0.5, c2=-0.25, half1=8.0,
            half2=6.0, mc1=0.25, mc2=-0.5, width=8.0, npix=64)
    counts, _ = oracle.shoot(j, np.zeros((3, 0)))
    a1 = Fraction(1) - Fraction(j.gamma) - Fraction(j.kappa_s)
    a2 = Fraction(1) + Fraction(j.gamma) - Fraction(j.kappa_s)
    w = Fraction(j.width) / j.npix
    e1 = lattice_counts_1d(a1, Fraction(j.c1), Fraction(j.half1), j.n1,
                           Fraction(j.mc1) - Fraction(j.width) / 2, w, j.npix)
    e2 = lattice_counts_1d(a2, Fraction(j.c2), Fraction(j.half2), j.n2,
                           Fraction(j.mc2) - Fraction(j.width) / 2, w, j.npix)
    expect = np.outer(np.array(e2), np.array(e1)).ravel()
    hist = oracle.count_histogram(counts, 200)
    assert np.array_equal(hist, np.bincount(expect, minlength=200))
    mpd = oracle.mpd(counts, 200)
    assert abs(mpd.sum() - 1.0) < 1e-15


def test_mpd_overflow_bin_and_mean():
    rng = np.random.default_rng(3)
    c = rng.integers(0, 5000, size=(77, 91)).astype(np.int32)
    h = oracle.count_histogram(c, 1000)
    assert h.sum() == c.size
    assert h[-1] == (c >= 999).sum()
    assert np.array_equal(h[:-1], np.bincount(c.ravel(), minlength=5000)[:999])
    # the mean magnification from the full histogram equals the map's
    c = rng.integers(0, 5000, size=(91, 91)).astype(np.int32)
    j = W.PARITY.with_(npix=91)
    hf = oracle.count_histogram(c, 5001)
    mean_h = (np.arange(5001) * hf).sum() / c.size / oracle.navg(j)
    assert abs(mean_h - oracle.magnification(j, c).mean()) < 1e-12 * mean_h


def test_prob_sums_closed_form():
    # covered pixels of this macromodel map hold exactly 16 rays (mu = 2):
    # nothing lies above mu = 2, and below it only the partly covered rim
    j = job(kappa_s=0.25, gamma=0.25, n1=512, n2=256, half1=8.0, half2=8.0,
            width=8.0, npix=64)
    counts, _ = oracle.shoot(j, np.zeros((3, 0)))
    hist = oracle.count_histogram(counts, 64)
    below, above = oracle.prob_sums(j, hist, [2.0, 1.0, 3.0])
    n16 = int((counts == 16).sum())
    assert above[0] == 0 and below[0] == counts.size - n16
    assert below[1] == int((counts < 8).sum()) and above[1] == int((counts > 8).sum())
    assert below[2] == counts.size and above[2] == 0
    # mu_th of the macromodel alone: 1/((1-k)^2 - g^2) with kappa = kappa_s
    assert oracle.mu_th(0.25, 0.25) == 2.0
    with pytest.raises(ValueError):
        oracle.prob_sums(j, hist, [10.0])          # threshold in the overflow bin

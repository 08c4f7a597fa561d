"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Each side draws its own lens field from the seed (the generators are
compared separately), so no oracle input ever comes from the CUDA path.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu

PRECS = (0, 1)   # RS_PREC_FP32, RS_PREC_COMPENSATED
ALL_PRECS = (0, 1, 2, 3)   # + RS_PREC_DOUBLE_SINGLE, RS_PREC_REFINED
# flip budget per precision at the parity configuration: the compensated form
# must meet the spec bar; the plain FP32 running sum is reported beside
# it with the bound its rounding analysis gives (a long FP32 sum of ~N terms
# of size |alpha| accumulates ~sqrt(N) ulp(|alpha|) of error).
FLIP_BOUND = {0: 1e-3, 1: PT.FLIP_MAX, 2: PT.FLIP_MAX, 3: PT.FLIP_MAX}


@pytest.fixture(scope="module")
def rs():
    import paper_1406_0559_b300 as rs
    return rs


def np_(t):
    return t.detach().cpu().numpy()


def all_tiles(rs, job, prec, shape=0):
    tx, ty = rs.tile_shape(prec, shape)
    t1 = -(-job.n1 // tx)
    t2 = -(-job.n2 // ty)
    return np.arange(t1 * t2, dtype=np.int64), tx, ty, t1


def per_ray_compare(rs, job, lens_g, lens_o, prec, tile_ids=None, shape=0):
    """Dump the GPU rays of the given tiles (all tiles by default) and
    compare each with the oracle's ray.  Returns (flip fraction, flips,
    rays, gpu pixels (k,2), max |dy|)."""
    ids, tx, ty, t1 = all_tiles(rs, job, prec, shape)
    if tile_ids is not None:
        ids = np.asarray(tile_ids, dtype=np.int64)
    y, pix = rs.shoot_tiles(job, lens_g, torch.from_numpy(ids).cuda(), precision=prec,
                            shape=shape)
    torch.cuda.synchronize()
    ij, valid = PT.gpu_tile_rays(ids, tx, ty, t1, job.n1, job.n2)
    gy = np_(y).reshape(-1, 2)[valid]
    gp = np_(pix).reshape(-1, 2)[valid]
    ij = ij[valid]
    oy, op, ost = oracle.shoot_rays(job, lens_o, ij)
    frac, nflip = PT.flip_fraction(gp, op, ost)
    both = (ost == 0) & (gp[:, 0] >= 0)
    dy = float(np.abs(gy[both] - oy[both]).max()) if both.any() else 0.0
    return frac, nflip, ij.shape[0], gp, dy


# ------------------------------------------------------------ lens field --

@pytest.mark.parametrize("job", [W.PARITY, W.scaled(W.PRECISION, lens_scale=10)],
                         ids=["unit", "salpeter"])
def test_lens_field_matches_oracle(rs, job):
    g = np_(rs.make_lenses(job))
    o = oracle.make_lenses(job)
    assert g.shape == o.shape
    # same counter-based draws; libm and CUDA's sin/cos/sqrt/pow differ by ulps
    assert np.abs(g[:2] - o[:2]).max() <= 1e-14 * job.lens_radius
    assert np.allclose(g[2], o[2], rtol=1e-13, atol=0)
    g2 = np_(rs.make_lenses(job))
    assert np.array_equal(g, g2)                       # deterministic


# ------------------------------------------------------------ pure macro --

@pytest.mark.parametrize("kappa_s,gamma", [(0.25, 0.125), (0.25, 0.875), (1.5, 0.25)])
@pytest.mark.parametrize("prec", PRECS)
def test_pure_macro_bit_exact(rs, kappa_s, gamma, prec):
    # dyadic geometry: FP64 is exact on both sides, so the maps are identical
    j = W.MapJob(name="macro", kappa_star=0.0, kappa_s=kappa_s, gamma=gamma, n_lens=0,
                 lens_radius=1.0, n1=512, n2=384, c1=0.5, c2=-0.25, half1=8.0, half2=6.0,
                 mc1=0.25, mc2=-0.5, width=8.0, npix=64)
    empty = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    c, st = rs.shoot_map(j, empty, precision=prec)
    co, so = oracle.shoot(j, np.zeros((3, 0)))
    assert np.array_equal(np_(c), co)
    s = np_(st)
    assert s[0] == so["n_in"] and s[1] == so["n_out"] and s[2] == 0


@pytest.mark.parametrize("prec", ALL_PRECS)
def test_map_edges_are_half_open(rs, prec):
    # identity mapping on a dyadic grid: every ray lands exactly on a pixel
    # edge; those on the upper and right map borders are out, as in the oracle
    j = W.MapJob(name="edges", kappa_star=0.0, kappa_s=0.0, gamma=0.0, n_lens=0,
                 lens_radius=1.0, n1=8, n2=8, half1=1.0, half2=1.0, width=1.75, npix=7)
    empty = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    c, st = rs.shoot_map(j, empty, precision=prec)
    co, so = oracle.shoot(j, np.zeros((3, 0)))
    assert np.array_equal(np_(c), co) and co.sum() == 49
    s = np_(st)
    assert (s[0], s[1], s[2]) == (so["n_in"], so["n_out"], 0) == (49, 15, 0)


# ------------------------------------------------------ the parity map ----

@pytest.mark.parametrize("prec", ALL_PRECS)
def test_parity_map_against_oracle(rs, prec):
    j = W.PARITY
    lg = rs.make_lenses(j)
    lo = oracle.make_lenses(j)
    c1, s1 = rs.shoot_map(j, lg, precision=prec)
    c2, s2 = rs.shoot_map(j, lg, precision=prec)
    cg, sg = np_(c1), np_(s1)
    assert np.array_equal(cg, np_(c2)) and np.array_equal(sg, np_(s2))   # run to run
    assert sg[0] + sg[1] + sg[2] == j.n1 * j.n2                           # conservation
    assert cg.sum() == sg[0]
    co, so = oracle.shoot(j, lo)
    frac, nflip, nray, gp, dy = per_ray_compare(rs, j, lg, lo, prec)
    assert nray == j.n1 * j.n2
    # the per-ray dump is the same arithmetic as the map, bit for bit
    assert np.array_equal(PT.histogram_pixels(gp, j.npix), cg)
    print(f"\nparity prec={prec}: flips {nflip}/{nray} = {frac:.3e}, max|dy| = {dy:.3e}")
    assert frac <= FLIP_BOUND[prec]
    assert abs(int(sg[0]) - so["n_in"]) <= nflip
    mu_g = np_(rs.magnification(j, c1)).astype(np.float64)
    mu_o = oracle.magnification(j, co)
    l1, npx = PT.rel_l1(mu_g, mu_o, co)
    print(f"parity prec={prec}: rel L1 = {l1:.3e} over {npx} pixels with >= 100 rays")
    if prec >= 1:
        assert npx > 1000
        assert l1 <= PT.L1_MAX


def test_point_lens_against_oracle(rs):
    j = W.MapJob(name="pointlens", kappa_star=0.0, kappa_s=0.0, gamma=0.0, n_lens=1,
                 lens_radius=0.0, n1=2048, n2=2048, half1=4.0, half2=4.0, width=4.0, npix=32)
    lens = np.array([[0.0], [0.0], [1.0]])
    c, st = rs.shoot_map(j, torch.from_numpy(lens).cuda(), precision=1)
    co, so = oracle.shoot(j, lens)
    frac, nflip, nray, gp, dy = per_ray_compare(rs, j, torch.from_numpy(lens).cuda(), lens, 1)
    assert frac <= PT.FLIP_MAX
    l1, npx = PT.rel_l1(np_(rs.magnification(j, c)).astype(np.float64),
                        oracle.magnification(j, co), co)
    assert l1 <= PT.L1_MAX


# ------------------------------------------------- ragged / degenerate ----

@pytest.mark.parametrize("n_lens", [0, 1, 2, 3, 5, 511, 512, 513, 767, 768, 769, 1537])
@pytest.mark.parametrize("prec", ALL_PRECS)
def test_ragged_lens_counts(rs, n_lens, prec):
    # ray grid not a multiple of any tile, lens count around the stage size
    j = W.PARITY.with_(n_lens=n_lens, n1=203, n2=157, npix=37, lens_radius=9.0, seed=17)
    lg = rs.make_lenses(j)
    lo = oracle.make_lenses(j)
    c, st = rs.shoot_map(j, lg, precision=prec)
    s = np_(st)
    assert s[0] + s[1] + s[2] == j.n1 * j.n2 and np_(c).sum() == s[0]
    frac, nflip, nray, gp, dy = per_ray_compare(rs, j, lg, lo, prec)
    assert nray == j.n1 * j.n2
    assert np.array_equal(PT.histogram_pixels(gp, j.npix), np_(c))
    assert nflip <= max(1, int(FLIP_BOUND[prec] * nray))


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5, 8, 9, 12, 27])
def test_every_shape_agrees_with_oracle(rs, shape):
    j = W.PARITY.with_(n1=517, n2=389, npix=64, seed=23)
    lg = rs.make_lenses(j)
    lo = oracle.make_lenses(j)
    for prec in PRECS:
        c, st = rs.shoot_map(j, lg, precision=prec, shape=shape)
        s = np_(st)
        assert s[0] + s[1] + s[2] == j.n1 * j.n2
        frac, nflip, nray, gp, dy = per_ray_compare(rs, j, lg, lo, prec, shape=shape)
        assert np.array_equal(PT.histogram_pixels(gp, j.npix), np_(c))
        assert nflip <= max(1, int(FLIP_BOUND[prec] * nray))


def test_unit_mass_path_equals_general_path(rs):
    j = W.PARITY.with_(n1=300, n2=300)
    lg = rs.make_lenses(j)
    for prec in ALL_PRECS:
        a, sa = rs.shoot_map(j, lg, precision=prec, unit_mass=True)
        b, sb = rs.shoot_map(j, lg, precision=prec, unit_mass=False)
        # counts and statistics agree; the refined form's diagnostics of its
        # second pass (band use, largest error) may differ in the last bits,
        # as the double-single sums of the two paths round apart
        n = rs.STAT_BAND_USE
        assert torch.equal(a, b) and torch.equal(sa[:n], sb[:n])


def test_degenerate_grids(rs):
    lg = rs.make_lenses(W.PARITY)
    # empty ray grid: zero map, zero stats
    j0 = W.PARITY.with_(n1=0, n2=64)
    c, st = rs.shoot_map(j0, lg)
    assert int(c.sum()) == 0 and np_(st).tolist() == [0] * rs.NSTATS
    # single pixel, single ray
    j1 = W.PARITY.with_(n1=1, n2=1, npix=1, width=40.0)
    c, st = rs.shoot_map(j1, lg)
    co, so = oracle.shoot(j1, oracle.make_lenses(j1))
    assert np.array_equal(np_(c), co)


def test_salpeter_small_against_oracle(rs):
    j = W.scaled(W.PRECISION, ray_scale=16, map_scale=16, lens_scale=50)
    lg = rs.make_lenses(j)
    lo = oracle.make_lenses(j)
    for prec in ALL_PRECS:
        frac, nflip, nray, gp, dy = per_ray_compare(rs, j, lg, lo, prec)
        print(f"\nsalpeter small prec={prec}: flips {nflip}/{nray} = {frac:.3e}")
        assert frac <= FLIP_BOUND[prec]


# ----------------------------------------------------------- magnification --

def test_magnification_matches_oracle(rs):
    j = W.PARITY.with_(npix=509)            # odd size: vector body + tail
    rng = np.random.default_rng(99)
    counts = rng.integers(0, 5_000_000, size=(j.npix, j.npix)).astype(np.int32)
    mu_g = np_(rs.magnification(j, torch.from_numpy(counts).cuda())).astype(np.float64)
    mu_o = oracle.magnification(j, counts)
    rel = np.abs(mu_g - mu_o) / np.maximum(mu_o, 1e-300)
    assert rel[counts > 0].max() <= 1.5 * 2.0 ** -23
    assert np.all(mu_g[counts == 0] == 0)


# ----------------------------------------------------------- API behaviour --

def test_host_entry_point_equals_device_path(rs):
    j = W.PARITY
    lg = rs.make_lenses(j)
    c, st = rs.shoot_map(j, lg)
    mu = np_(rs.magnification(j, c))
    mu_h, st_h = rs.shoot_map_host(j, lg.cpu())
    assert np.array_equal(mu_h.numpy(), mu)
    assert np.array_equal(st_h.numpy(), np_(st))


def test_accumulate_and_stream(rs):
    j = W.PARITY.with_(n1=512, n2=512)
    lg = rs.make_lenses(j)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c, st = rs.shoot_map(j, lg)
        rs.shoot_map(j, lg, counts=c, stats=st, accumulate=True)
    s.synchronize()
    c1, st1 = rs.shoot_map(j, lg)
    torch.cuda.synchronize()
    assert torch.equal(c, 2 * c1) and torch.equal(st, 2 * st1)


def test_host_pointer_is_rejected(rs):
    j = W.PARITY.with_(n1=64, n2=64)
    lg = rs.make_lenses(j)
    with pytest.raises(rs.RSError) as e:
        rs.shoot_map(j, lg, counts=torch.zeros((j.npix, j.npix), dtype=torch.int32))
    assert e.value.code == -1 and "device memory" in str(e.value)


# ------------------------------------------------- full-size, sampled -------

@pytest.mark.slow
@pytest.mark.parametrize("prec", [1, 2, 3], ids=["compensated", "double-single", "refined"])
@pytest.mark.parametrize("job", [W.GERLUMPH, W.PRECISION], ids=["gerlumph", "precision"])
def test_full_size_sampled_against_oracle(rs, job, prec):
    """The workloads the benchmark times, in its launch configuration: the
    whole map on the GPU (conservation, determinism), and a seeded sample of
    whole ray tiles compared ray by ray with the oracle."""
    lg = rs.make_lenses(job)
    lo = oracle.make_lenses(job)
    c, st = rs.shoot_map(job, lg, precision=prec)
    s = np_(st)
    assert s[0] + s[1] + s[2] == job.n1 * job.n2
    assert int(c.sum()) == s[0]
    c2, _ = rs.shoot_map(job, lg, precision=prec)
    assert torch.equal(c, c2)
    ids, tx, ty, t1 = all_tiles(rs, job, prec)
    pick = W.sample_tiles(ids.size, 128, seed=job.seed + 1000)
    frac, nflip, nray, gp, dy = per_ray_compare(rs, job, lg, lo, prec, tile_ids=pick)
    print(f"\n{job.name} prec={prec}: flips {nflip}/{nray} = {frac:.3e}, max|dy| = {dy:.3e}")
    if prec >= 2:
        # double-single terms (refined: for every ray near a pixel edge):
        # the spec bar holds at full size
        assert frac <= PT.FLIP_MAX
    else:
        # rounding analysis: FP32 terms (~1e-7 relative each) summed over N
        # lenses leave |dy| ~ 1e-7 sqrt(sum 1/r^2) ~ 2e-7 R_E against
        # 6.1e-3 R_E pixels, i.e. ~5e-5 of rays near a pixel edge
        assert frac <= 2e-4


@pytest.mark.parametrize("npix,width", [(64, 10.0), (256, 10.0), (4096, 10.0)],
                         ids=["window", "window-tight", "global-fallback"])
@pytest.mark.parametrize("prec", PRECS)
def test_window_binning_equals_global_atomics(rs, npix, width, prec):
    """Shape 27 bins each ray tile through a shared-memory window (coarse
    pixels) or falls back to global atomics (fine pixels: the footprint of a
    tile exceeds the window); integer counts must match shape 12 exactly."""
    j = W.PARITY.with_(npix=npix, width=width, n1=1000, n2=777, seed=5)
    lg = rs.make_lenses(j)
    a, sa = rs.shoot_map(j, lg, precision=prec, shape=12)
    b, sb = rs.shoot_map(j, lg, precision=prec, shape=27)
    assert torch.equal(a, b) and torch.equal(sa, sb)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_debug_rays_matches_tiles_and_oracle(rs, prec):
    """rs_debug_rays: arbitrary rays (any order, repeats, grid corners) give
    the tile dump's values bit for bit, and the oracle's pixels."""
    job = W.PARITY
    lens = rs.make_lenses(job)
    rng = np.random.default_rng(21)
    ij = np.stack([rng.integers(0, job.n1, 3000), rng.integers(0, job.n2, 3000)], axis=1)
    ij = np.concatenate([ij, [[0, 0], [job.n1 - 1, job.n2 - 1], [5, 7], [5, 7]]])
    y, pix = rs.debug_rays(job, lens, ij, precision=prec)
    tx, ty = rs.tile_shape(prec, 0)
    t1 = -(-job.n1 // tx)
    tiles = (ij[:, 1] // ty) * t1 + ij[:, 0] // tx
    yt, pt = rs.shoot_tiles(job, lens, torch.from_numpy(tiles), precision=prec)
    k = np.arange(len(ij))
    a, b = ij[:, 0] % tx, ij[:, 1] % ty
    assert np.array_equal(pt.cpu().numpy()[k, b, a], pix)
    assert np.array_equal(yt.cpu().numpy()[k, b, a], y)
    oy, op, ost = oracle.shoot_rays(job, oracle.make_lenses(job), ij)
    frac, _ = PT.flip_fraction(pix, op, ost)
    assert frac <= (1e-5 if prec >= 2 else 2e-3)
    with pytest.raises(rs.RSError):
        rs.debug_rays(job, lens, [[0, job.n2]])


@pytest.mark.parametrize("prec,tol", [(2, 5e-8), (1, 5e-5)], ids=["double-single", "compensated"])
def test_superposition_at_full_size(rs, prec, tol):
    """P8 on the CUDA path at the benchmark's full size, with no oracle: the
    deflection of a lens set is the sum of the deflections of its halves.
    With y = M(x) - alpha (Eq. 1) and the same macromodel term M on every
    call, y_A + y_B - y_AB = M exactly up to the error of the three sums."""
    job = W.GERLUMPH
    lens = rs.make_lenses(job)
    n = lens.shape[1]
    a, b = lens[:, : n // 2].contiguous(), lens[:, n // 2:].contiguous()
    rng = np.random.default_rng(31)
    ij = np.stack([rng.integers(0, job.n1, 4096), rng.integers(0, job.n2, 4096)], axis=1)
    y_ab, _ = rs.debug_rays(job, lens, ij, precision=prec)
    y_a, _ = rs.debug_rays(job, a, ij, precision=prec)
    y_b, _ = rs.debug_rays(job, b, ij, precision=prec)
    d1 = 2 * job.half1 / job.n1
    d2 = 2 * job.half2 / job.n2
    x1 = (job.c1 - job.half1) + (ij[:, 0] + 0.5) * d1
    x2 = (job.c2 - job.half2) + (ij[:, 1] + 0.5) * d2
    m = np.stack([(1 - job.gamma - job.kappa_s) * x1, (1 + job.gamma - job.kappa_s) * x2], axis=1)
    err = np.abs(y_a + y_b - y_ab - m)
    print(f"\nsuperposition prec={prec}: max |y_A + y_B - y_AB - M| = {err.max():.3e}")
    assert np.isfinite(err).all()
    assert err.max() <= tol, err.max()

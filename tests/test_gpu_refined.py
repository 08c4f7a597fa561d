"""RS_PREC_REFINED on the GPU: the compensated map kernel lists the rays whose
image lies within its error bound of a pixel edge, a double-single pass bins
them except those within the double-single sum's own bound of an edge, which
an FP64 pass bins.  Its maps are compared whole with the FP64 oracle's
(small maps), per ray on sampled tiles at the serving and survey scales
(8192^2 with 80,000 lenses; 10000^2 over 25 R_E with a ray spacing off the
2^-12 grid), and with the double-single map (full size).  The bound itself is
checked on every sampled ray: the first pass's error against the oracle lies
inside the ray's band."""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu

REFINED = 3

# the serving maximum (8192^2 maps over 25 R_E, 80,000 lenses, rays 4x the
# side over 60 R_E) and the survey's 10000^2 over 25 R_E resolution with
# 40000^2 rays over 60 R_E (a spacing off the 2^-12 grid: the coherent-rounding
# correction is active)
SERVE_MAX = W.MapJob(name="serve-8192/80k", kappa_star=1.0, kappa_s=0.0, gamma=0.3,
                     n_lens=80000, lens_radius=math.sqrt(80000 / 1.0), seed=11,
                     n1=32768, n2=32768, half1=30.0, half2=30.0, width=25.0, npix=8192)
SERVE_MAX_SALP = SERVE_MAX.with_(name="serve-8192/80k-salpeter", kappa_star=0.77, kappa_s=0.33,
                                 gamma=0.5, lens_radius=math.sqrt(80000 / 0.77),
                                 mass_model=W.MASS_SALPETER, seed=13)
GD_10000 = W.MapJob(name="gd-10000", kappa_star=0.6, kappa_s=0.0, gamma=0.25, n_lens=50000,
                    lens_radius=math.sqrt(50000 / 0.6), seed=12, n1=40000, n2=40000,
                    half1=30.0, half2=30.0, width=25.0, npix=10000)


@pytest.fixture(scope="module")
def rs():
    import paper_1406_0559_b300 as rs
    return rs


def np_(t):
    return t.detach().cpu().numpy()


def check_stats(job, counts, stats):
    assert stats[0] + stats[1] + stats[2] == job.n1 * job.n2      # conservation
    assert counts.sum() == stats[0]


@pytest.mark.parametrize("job", [W.PARITY, W.scaled(W.PRECISION, ray_scale=16, map_scale=16,
                                                    lens_scale=50)],
                         ids=["parity-256", "salpeter-small"])
def test_refined_map_equals_oracle_map(rs, job):
    lg = rs.make_lenses(job)
    c, st = rs.shoot_map(job, lg, precision=REFINED)
    c2, st2 = rs.shoot_map(job, lg, precision=REFINED)
    cg, sg = np_(c), np_(st)
    assert np.array_equal(cg, np_(c2)) and np.array_equal(sg, np_(st2))   # run to run
    check_stats(job, cg, sg)
    co, so = oracle.shoot(job, oracle.make_lenses(job))
    moved = int(np.abs(cg.astype(np.int64) - co).sum())
    cc, _ = rs.shoot_map(job, lg, precision=1)
    moved_comp = int(np.abs(np_(cc).astype(np.int64) - co).sum())
    print(f"\n{job.name}: refined rays {sg[3]} ({sg[3] / max(1, sg[0]):.2%} of in-map), "
          f"|refined - oracle| = {moved}, |compensated - oracle| = {moved_comp}")
    # every ray moved between pixels counts twice in the sum
    assert moved <= 2 * max(1, int(1e-6 * job.n1 * job.n2))
    assert abs(int(sg[0]) - so["n_in"]) <= moved
    assert sg[rs.STAT_REFINED] > 0 and sg[rs.STAT_OVERFLOW] == 0
    # the a-posteriori check: every recomputed ray's first-pass error was
    # inside its band
    assert 0 < sg[rs.STAT_BAND_USE] < 65536
    # every shape the autotuner may pick for the refined form (unrolls of
    # 2-8 lens groups, folds of 24 or 48 lenses) meets the same bar
    for shape in rs.tune_candidates(REFINED)[1:]:
        cs, ss = rs.shoot_map(job, lg, precision=REFINED, shape=shape)
        cs, ss = np_(cs), np_(ss)
        check_stats(job, cs, ss)
        moved_s = int(np.abs(cs.astype(np.int64) - co).sum())
        assert moved_s <= 2 * max(1, int(1e-6 * job.n1 * job.n2)), (shape, moved_s)
        assert ss[rs.STAT_OVERFLOW] == 0 and 0 < ss[rs.STAT_BAND_USE] < 65536, shape


@pytest.mark.parametrize("job", [W.GERLUMPH, W.scaled(W.PRECISION, ray_scale=2)],
                         ids=["gerlumph-4096", "precision-4096/rays8192"])
def test_refined_full_size_equals_double_single(rs, job):
    """At the benchmark's full size the refined map is the double-single map
    (which matches the oracle on every sampled ray), while the compensated
    map differs from it by ~4e-5 of the rays."""
    lg = rs.make_lenses(job)
    cr, sr = rs.shoot_map(job, lg, precision=REFINED)
    cd, sd = rs.shoot_map(job, lg, precision=2)
    cc, sc = rs.shoot_map(job, lg, precision=1)
    r, d, c = np_(cr).astype(np.int64), np_(cd).astype(np.int64), np_(cc).astype(np.int64)
    sr_, sd_ = np_(sr), np_(sd)
    check_stats(job, r, sr_)
    moved = int(np.abs(r - d).sum())
    moved_c = int(np.abs(c - d).sum())
    n = job.n1 * job.n2
    print(f"\n{job.name}: |refined - double-single| = {moved} ({moved / 2 / n:.1e} of rays), "
          f"|compensated - double-single| = {moved_c} ({moved_c / 2 / n:.1e}), "
          f"refined rays {sr_[3]} ({sr_[3] / n:.2%})")
    assert moved / 2 <= 1e-6 * n
    assert abs(int(sr_[0]) - int(sd_[0])) <= moved
    assert moved_c > moved


def test_refined_host_entry_point_equals_device_path(rs):
    j = W.PARITY
    lg = rs.make_lenses(j)
    c, st = rs.shoot_map(j, lg, precision=REFINED)
    mu = np_(rs.magnification(j, c))
    mu_h, st_h = rs.shoot_map_host(j, lg.cpu(), precision=REFINED)
    assert np.array_equal(mu_h.numpy(), mu)
    assert np.array_equal(st_h.numpy(), np_(st))


def test_refined_accumulates_and_handles_degenerate_grids(rs):
    j = W.PARITY.with_(n1=512, n2=512)
    lg = rs.make_lenses(j)
    c, st = rs.shoot_map(j, lg, precision=REFINED)
    rs.shoot_map(j, lg, precision=REFINED, counts=c, stats=st, accumulate=True)
    c1, st1 = rs.shoot_map(j, lg, precision=REFINED)
    torch.cuda.synchronize()
    # counts add; the diagnostics of the second pass are maxima
    n = rs.STAT_BAND_USE
    assert torch.equal(c, 2 * c1) and torch.equal(st[:n], 2 * st1[:n])
    assert torch.equal(st[n:], st1[n:])
    for n1, n2 in [(0, 5), (1, 1), (3, 1000)]:
        jd = W.PARITY.with_(n1=n1, n2=n2)
        cd, sd = rs.shoot_map(jd, lg, precision=REFINED)
        check_stats(jd, np_(cd), np_(sd))
    c0, s0 = rs.shoot_map(j, lg[:, :0].contiguous(), precision=REFINED)   # no lenses
    cz, sz = rs.shoot_map(j, lg[:, :0].contiguous(), precision=2)
    assert torch.equal(c0, cz) and torch.equal(s0[:3], sz[:3])


def test_refined_dump_equals_map(rs):
    """Per-ray dump of the refined path (all tiles) histograms to the map."""
    j = W.PARITY.with_(n1=1000, n2=777)        # ragged tiles
    lg = rs.make_lenses(j)
    c, st = rs.shoot_map(j, lg, precision=REFINED)
    tx, ty = rs.tile_shape(REFINED, 0)
    t1, t2 = -(-j.n1 // tx), -(-j.n2 // ty)
    ids = torch.arange(t1 * t2, dtype=torch.int64, device="cuda")
    y, pix = rs.shoot_tiles(j, lg, ids, precision=REFINED)
    p = np_(pix).reshape(-1, 2)
    inside = p[:, 0] >= 0
    hist = np.zeros((j.npix, j.npix), dtype=np.int64)
    np.add.at(hist, (p[inside, 1], p[inside, 0]), 1)
    assert np.array_equal(hist, np_(c)) and inside.sum() == int(np_(st)[0])
    # the first pass's images: every ray the later passes did not recompute
    # keeps exactly its first-pass image; the recomputed ones (the listed
    # rays near an edge, a small fraction) moved by less than their band
    band, y1 = rs.shoot_tiles_band(j, lg, ids, first_pass=True)
    y, y1, band = np_(y).reshape(-1, 2), np_(y1).reshape(-1, 2), np_(band).reshape(-1)
    fin = np.all(np.isfinite(y), axis=1) & np.all(np.isfinite(y1), axis=1)
    same = np.all(y == y1, axis=1) | ~fin
    assert 0.9 < same.mean() < 1.0
    w = j.width / j.npix
    moved = ~same
    assert np.all(np.abs(y[moved] - y1[moved]).max(axis=1) / w < band[moved])


def test_refined_is_refused_where_it_does_not_apply(rs):
    j = W.PARITY
    lg = rs.make_lenses(j)
    with pytest.raises(rs.RSError):
        rs.shoot_map(j, lg, precision=REFINED, shape=2)
    with pytest.raises(rs.RSError):
        rs.shoot_batch([rs.MapBuffers(j, lg)], precision=REFINED, shape=2)
    with pytest.raises(rs.RSError):
        rs.Server(precision=REFINED, shape=2)


def sampled_compare(rs, job, n_tiles=128, seed=99):
    """Per ray on sampled tiles: the first pass's error (the compensated sum
    the refined form runs, folds of 48 lenses) against the oracle in pixels,
    the ray's band, and the refined form's pixels against the oracle's."""
    lg = rs.make_lenses(job)
    lo = oracle.make_lenses(job)
    tx, ty = rs.tile_shape(REFINED, 0)
    t1, t2 = -(-job.n1 // tx), -(-job.n2 // ty)
    tiles = W.sample_tiles(t1 * t2, n_tiles, seed=seed)
    ids = torch.from_numpy(tiles).cuda()
    _, pr = rs.shoot_tiles(job, lg, ids, precision=REFINED)
    band, yc = rs.shoot_tiles_band(job, lg, ids, first_pass=True)
    ij, valid = PT.gpu_tile_rays(tiles, tx, ty, t1, job.n1, job.n2)
    yo, po, so = oracle.shoot_rays(job, lo, ij[valid])
    yc = np_(yc).reshape(-1, 2)[valid]
    pr = np_(pr).reshape(-1, 2)[valid]
    band = np_(band).reshape(-1)[valid]
    w = job.width / job.npix
    u = (yo - (np.array([job.mc1, job.mc2]) - job.width / 2)) / w
    near = np.all((u > -1) & (u < job.npix + 1), axis=1)
    err = np.abs(yc - yo).max(axis=1) / w
    frac, nflip = PT.flip_fraction(pr, po, so)
    return lg, err[near], band[near], frac, nflip, int(valid.sum())


@pytest.mark.parametrize("job", [W.PARITY, W.GERLUMPH, W.PRECISION, SERVE_MAX, SERVE_MAX_SALP,
                                 GD_10000], ids=lambda j: j.name)
def test_refined_bound_and_flips_on_sampled_tiles(rs, job):
    """The first pass's error lies inside its band on every sampled ray (so a
    ray outside its band cannot change pixel), and the refined form's pixels
    equal the oracle's within the flip bar (expected: all of them)."""
    _, err, band, frac, nflip, n = sampled_compare(rs, job)
    ratio = err / band
    print(f"\n{job.name}: {n} rays, band {band.mean():.2e} px mean, error/band max "
          f"{ratio.max():.3f}, refined flips {nflip}")
    assert np.all(band > 0) and np.all(band <= 1)
    assert ratio.max() < 1.0
    assert frac <= PT.FLIP_MAX


@pytest.mark.parametrize("job", [SERVE_MAX, GD_10000], ids=lambda j: j.name)
def test_refined_full_map_statistics_at_survey_scale(rs, job):
    """Whole maps at the serving maximum and at 10000^2: conservation, no list
    overflow, and the a-posteriori check holds over the recomputed rays."""
    lg = rs.make_lenses(job)
    c, st = rs.shoot_map(job, lg, precision=REFINED)
    s = np_(st)
    total = int(np_(c).astype(np.int64).sum())
    print(f"\n{job.name}: {s.tolist()}; recomputed {s[3] / max(1, s[0]):.3%} of in-map rays, "
          f"FP64 {s[4]}, band use {s[6] / 65536:.3f}")
    assert s[0] + s[1] + s[2] == job.n1 * job.n2 and total == s[0]
    assert s[rs.STAT_OVERFLOW] == 0
    assert 0 < s[rs.STAT_BAND_USE] < 65536
    assert s[rs.STAT_EXACT] > 0


def test_refined_list_overflow_is_reported(rs):
    """A coarse ray grid over a dense lens field: every tile holds more near
    lenses than the list keeps, so every ray near the map is listed, and with
    2^23 rays the list (2^22 rays) overflows.  The overflow is counted, rays
    keep their first-pass pixel, and conservation still holds."""
    job = W.MapJob(name="overflow", kappa_star=2.0, kappa_s=0.0, gamma=0.1, n_lens=200000,
                   lens_radius=math.sqrt(200000 / 2.0), seed=21, n1=8192, n2=1024,
                   half1=409.6, half2=51.2, width=900.0, npix=256)
    lg = rs.make_lenses(job)
    ids = torch.arange(4, dtype=torch.int64, device="cuda") + 3 * 128 + 60   # inside the disk
    band = np_(rs.shoot_tiles_band(job, lg, ids))
    assert np.all(band == 1.0)              # near lenses beyond the list: whole tiles
    c, st = rs.shoot_map(job, lg, precision=REFINED)
    s = np_(st)
    assert s[0] + s[1] + s[2] == job.n1 * job.n2
    assert int(np_(c).astype(np.int64).sum()) == s[0]
    assert s[rs.STAT_OVERFLOW] > 0
    assert s[rs.STAT_REFINED] == 1 << 22


@pytest.mark.parametrize("precision", [1, REFINED], ids=["compensated", "refined"])
def test_map_in_tile_ranges_equals_whole_map(rs, precision):
    """Checkpoint / resume: the map shot as uneven consecutive tile ranges
    (the last one reaching past the end) equals the single call's map, and
    an empty range or a range starting beyond the map changes nothing or is
    refused."""
    j = W.PARITY.with_(n1=1000, n2=777)
    lg = rs.make_lenses(j)
    c, st = rs.shoot_map(j, lg, precision=precision)
    counts = torch.zeros_like(c)
    stats = torch.zeros_like(st)
    total = rs.shoot_map_range(j, lg, counts, stats, 0, 0, precision=precision)
    assert int(counts.sum()) == 0 and total > 10
    t0 = 0
    for n in (1, 5, 3, total):
        rs.shoot_map_range(j, lg, counts, stats, t0, n, precision=precision)
        t0 += n
    assert torch.equal(counts, c)
    assert torch.equal(stats[:rs.STAT_BAND_USE], st[:rs.STAT_BAND_USE])
    with pytest.raises(rs.RSError):
        rs.shoot_map_range(j, lg, counts, stats, total + 1, 1, precision=precision)

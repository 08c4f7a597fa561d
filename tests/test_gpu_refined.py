"""RS_PREC_REFINED on the GPU: the compensated map kernel lists the rays whose
image lies within 2^-9 pixel of a pixel edge, and a double-single pass bins
them.  Its maps are compared whole with the FP64 oracle's (small maps) and
with the double-single map (full size), which the per-ray tests of
test_gpu_parity.py pin to the oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

REFINED = 3


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
    # about 4 x 2^-9 of the in-map rays lie near an edge
    assert 0.3 * 4 * 2.0 ** -9 * sg[0] < sg[3] < 3 * 4 * 2.0 ** -9 * sg[0] + 100


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
    assert torch.equal(c, 2 * c1) and torch.equal(st, 2 * st1)
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


def test_refined_is_refused_where_it_does_not_apply(rs):
    j = W.PARITY
    lg = rs.make_lenses(j)
    with pytest.raises(rs.RSError):
        rs.shoot_map(j, lg, precision=REFINED, shape=2)
    with pytest.raises(rs.RSError):
        rs.shoot_batch([rs.MapBuffers(j, lg)], precision=REFINED, shape=2)
    with pytest.raises(rs.RSError):
        rs.Server(precision=REFINED, shape=2)

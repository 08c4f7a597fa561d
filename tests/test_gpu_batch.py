"""Batching form on the GPU: many uneven maps in persistent launches and CUDA
graphs give exactly the maps of single-map calls (same kernel shape), and
agree with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_1406_0559_b300 as rs
    return rs


def small_batch(n=7, seed=41, unit=True):
    """Uneven maps: lens counts from 0 to a few thousand, ragged ray grids,
    odd and even pixel counts, different macromodels."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(n):
        npix = int(rng.choice([31, 64, 100, 128]))
        nl = int(rng.choice([0, 1, 2, 150, 769, 2000]))
        kstar = float(rng.uniform(0.1, 0.6))
        jobs.append(W.MapJob(name=f"b{k}", kappa_star=kstar, kappa_s=float(rng.uniform(0, 0.3)),
                             gamma=float(rng.uniform(0, 0.5)), n_lens=nl,
                             lens_radius=float(np.sqrt(max(nl, 1) / kstar)),
                             mass_model=W.MASS_UNIT if unit else W.MASS_SALPETER,
                             seed=int(rng.integers(1, 2**40)),
                             n1=int(rng.integers(100, 700)), n2=int(rng.integers(100, 700)),
                             half1=float(rng.uniform(4, 9)), half2=float(rng.uniform(4, 9)),
                             width=float(rng.uniform(3, 8)), npix=npix))
    return jobs


def buffers(rs, jobs):
    return [rs.MapBuffers(j, rs.make_lenses(j)) for j in jobs]


@pytest.mark.parametrize("unit", [True, False], ids=["unit", "salpeter"])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_batch_equals_single_map_calls(rs, unit, prec):
    jobs = small_batch(unit=unit, seed=41 + int(unit))
    bufs = buffers(rs, jobs)
    rs.shoot_batch(bufs, precision=prec, unit_mass=unit, shape=12)
    torch.cuda.synchronize()
    for b in bufs:
        c, st = rs.shoot_map(b.job, b.lenses, precision=prec, unit_mass=unit, shape=12)
        assert torch.equal(b.counts, c), b.job.name
        assert torch.equal(b.stats, st), b.job.name
        s = b.stats.cpu().numpy()
        assert s[0] + s[1] + s[2] == b.job.n1 * b.job.n2
        assert torch.equal(b.mu, rs.magnification(b.job, c))


@pytest.mark.parametrize("shape", [28, 29, 30])
@pytest.mark.parametrize("prec", [1, 3], ids=["compensated", "refined"])
def test_tuning_candidates_batch_equal_single_calls(rs, prec, shape):
    """The unroll / fold candidates: a batch run with one of them equals the
    single-map calls of the same shape, general masses included (their
    single-map kernels exist for unit masses only in the compensated form,
    so the comparison there is unit-mass)."""
    unit = prec == 1
    jobs = small_batch(unit=unit, seed=43)
    bufs = buffers(rs, jobs)
    rs.shoot_batch(bufs, precision=prec, unit_mass=unit, shape=shape)
    torch.cuda.synchronize()
    for b in bufs:
        c, st = rs.shoot_map(b.job, b.lenses, precision=prec, unit_mass=unit, shape=shape)
        assert torch.equal(b.counts, c), (shape, b.job.name)
        assert torch.equal(b.stats[:rs.STAT_BAND_USE], st[:rs.STAT_BAND_USE]), (shape, b.job.name)


@pytest.mark.parametrize("shape", [14, 15, 16])
def test_other_batch_shapes_against_oracle(rs, shape):
    jobs = small_batch(n=5, seed=77)
    bufs = buffers(rs, jobs)
    rs.shoot_batch(bufs, precision=1, unit_mass=True, shape=shape)
    torch.cuda.synchronize()
    for b in bufs:
        co, so = oracle.shoot(b.job, oracle.make_lenses(b.job))
        cg = b.counts.cpu().numpy()
        s = b.stats.cpu().numpy()
        assert s[0] + s[1] + s[2] == b.job.n1 * b.job.n2 and cg.sum() == s[0]
        moved = int(np.abs(cg.astype(np.int64) - co).sum())
        assert moved <= max(2, int(2 * PT.FLIP_MAX * b.job.n1 * b.job.n2)), (b.job.name, moved)


def test_more_maps_than_one_launch(rs):
    jobs = [W.PARITY.with_(name=f"m{k}", n1=64, n2=48, npix=16, n_lens=3 + (k % 5),
                           seed=1000 + k) for k in range(131)]
    bufs = buffers(rs, jobs)
    rs.shoot_batch(bufs, precision=1, unit_mass=True)
    torch.cuda.synchronize()
    for b in bufs[::13]:
        c, st = rs.shoot_map(b.job, b.lenses, precision=1, unit_mass=True, shape=12)
        assert torch.equal(b.counts, c) and torch.equal(b.stats, st)


@pytest.mark.parametrize("prec", [1, 3], ids=["compensated", "refined"])
def test_plan_replays_the_batch(rs, prec):
    jobs = small_batch(n=6, seed=5)
    bufs = buffers(rs, jobs)
    rs.shoot_batch(bufs, precision=prec, unit_mass=True, shape=12)
    torch.cuda.synchronize()
    ref = [(b.counts.clone(), b.stats.clone(), b.mu.clone()) for b in bufs]
    for b in bufs:
        b.counts.fill_(7)
        b.mu.fill_(-1)
    plan = rs.Plan(bufs, precision=prec, unit_mass=True, shape=12)
    assert plan.shape == 12
    for _ in range(2):
        plan.launch()
        torch.cuda.synchronize()
        for b, (c, s, m) in zip(bufs, ref):
            assert torch.equal(b.counts, c) and torch.equal(b.stats, s) and torch.equal(b.mu, m)
    plan.close()


def test_autotune_picks_a_candidate_and_plans_use_it(rs):
    jobs = small_batch(n=4, seed=9)
    bufs = buffers(rs, jobs)
    best, ms = rs.autotune(bufs, precision=1, unit_mass=True)
    assert best in rs.tune_candidates()
    assert all(v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())
    plan = rs.Plan(bufs, precision=1, unit_mass=True)     # shape 0: the tuned one
    assert plan.shape == best
    plan.launch()
    torch.cuda.synchronize()
    for b in bufs:
        c, st = rs.shoot_map(b.job, b.lenses, precision=1, unit_mass=True, shape=best) \
            if best == 12 else (None, None)
        s = b.stats.cpu().numpy()
        assert s[0] + s[1] + s[2] == b.job.n1 * b.job.n2
        if c is not None:
            assert torch.equal(b.counts, c)


def test_autotune_refined_times_its_own_candidates(rs):
    """The refined form's candidates (unroll, fold) are timed on their first
    pass with ray lists; a plan then runs the chosen shape, and its maps equal
    the single-map refined calls of that shape."""
    cand = rs.tune_candidates(3)
    assert cand[0] == 12 and len(cand) >= 3
    jobs = small_batch(n=4, seed=9)
    bufs = buffers(rs, jobs)
    best, ms = rs.autotune(bufs, precision=3, unit_mass=True)
    assert best in cand and set(ms) == set(cand)
    assert all(v > 0 for v in ms.values()) and ms[best] == min(ms.values())
    plan = rs.Plan(bufs, precision=3, unit_mass=True)
    assert plan.shape == best
    plan.launch()
    torch.cuda.synchronize()
    for b in bufs:
        c, st = rs.shoot_map(b.job, b.lenses, precision=3, unit_mass=True, shape=best)
        assert torch.equal(b.counts, c)
        assert torch.equal(b.stats[:rs.STAT_BAND_USE], st[:rs.STAT_BAND_USE])


def test_batch_rejects_bad_jobs(rs):
    jobs = small_batch(n=3, seed=3)
    bufs = buffers(rs, jobs)
    bufs[1].counts = torch.zeros_like(bufs[1].counts, device="cpu")   # host buffer
    with pytest.raises(rs.RSError) as e:
        rs.shoot_batch(bufs)
    assert "job 1" in str(e.value)


@pytest.mark.parametrize("prec", [1, 0, 3])
def test_gpu_filling_maps_take_their_own_launch(rs, prec):
    """A map with at least 8 waves of tiles is launched on its own inside the
    batch (single-map kernel), the small ones share the batched launch: every
    map is still bit-identical to rs_shoot_map, directly and through a plan."""
    big = W.PARITY.with_(name="big", n1=2304, n2=2304, npix=512, n_lens=40, seed=77)
    jobs = [big] + small_batch(n=5, seed=19)
    bufs = buffers(rs, jobs)
    rs.shoot_batch(bufs, precision=prec, unit_mass=True, shape=12)
    torch.cuda.synchronize()
    ref = []
    for b in bufs:
        c, st = rs.shoot_map(b.job, b.lenses, precision=prec, unit_mass=True, shape=12)
        assert torch.equal(b.counts, c) and torch.equal(b.stats, st), b.job.name
        ref.append(c)
    for b in bufs:
        b.counts.fill_(3)
    plan = rs.Plan(bufs, precision=prec, unit_mass=True, shape=12)
    plan.launch()
    torch.cuda.synchronize()
    for b, c in zip(bufs, ref):
        assert torch.equal(b.counts, c), b.job.name
    plan.close()

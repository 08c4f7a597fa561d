"""The seeded synthetic inputs are what the recipe says: the three benchmark
maps' parameters (Sec. 3.1 and Table 3 shapes, Eq. 3 lens counts), the
survey grid of the batching form and the Poisson request stream of the
serving form (ranges, rejection of near-critical points, Eq. 3 disk radii,
determinism)."""
import math

import numpy as np

import workloads as W


def test_benchmark_maps():
    p, g, q = W.PARITY, W.GERLUMPH, W.PRECISION
    # parity: 150 unit lenses in R = 11, 2048^2 rays over 15 R_E, 256^2 map over 10 R_E
    assert (p.n_lens, p.lens_radius, p.mass_model) == (150, 11.0, W.MASS_UNIT)
    assert (p.n1, p.n2, 2 * p.half1, 2 * p.half2, p.npix, p.width) == (2048, 2048, 15, 15, 256, 10)
    # GERLUMPH scale: N = kappa_* R^2 = 0.6 * 200^2 (Eq. 3), 16384^2 rays over
    # 60 R_E, 4096^2 map over 25 R_E
    assert g.n_lens == round(g.kappa_star * g.lens_radius ** 2) == 24000
    assert (g.kappa_s, g.gamma, g.mass_model) == (0.0, 0.3, W.MASS_UNIT)
    assert (g.n1, g.n2, 2 * g.half1, g.npix, g.width) == (16384, 16384, 60, 4096, 25)
    # precision map: 50,000 Salpeter lenses (0.1-1.0, slope 2.35) in R = 280
    assert (q.n_lens, q.lens_radius, q.mass_model) == (50000, 280.0, W.MASS_SALPETER)
    assert (q.m_lo, q.m_hi, q.slope) == (0.1, 1.0, 2.35)
    assert (q.kappa_s, q.gamma, q.npix, q.n1) == (0.4, 0.2, 4096, 16384)
    assert W.GERLUMPH_SMALL.n1 == 2048 and W.GERLUMPH_SMALL.npix == g.npix
    assert len({p.seed, g.seed, q.seed}) == 3


def test_batch_grid_recipe():
    jobs = W.batch_grid()
    assert len(jobs) == 64
    for j in jobs:
        kappa = j.kappa_star + j.kappa_s
        assert 0.1 <= kappa <= 1.2 and 0.0 <= j.gamma <= 1.0
        assert abs((1.0 - kappa) ** 2 - j.gamma ** 2) >= 0.05      # off the critical line
        s = j.kappa_s / kappa
        assert min(abs(s - t) for t in (0.0, 0.3, 0.6, 0.9)) < 1e-12
        assert 500 <= j.n_lens <= 50000
        assert j.npix in (1024, 2048, 4096) and j.n1 == j.n2 == 4 * j.npix
        assert 2 * j.half1 == 60.0 and j.width == 25.0
        # Eq. 3 with unit mean mass: the disk radius gives kappa_* back
        assert math.isclose(j.n_lens / j.lens_radius ** 2, j.kappa_star, rel_tol=1e-12)
    # seeded: the same draw twice, a different one for another seed
    assert [j.seed for j in W.batch_grid()] == [j.seed for j in jobs]
    assert [j.seed for j in W.batch_grid(seed=5)] != [j.seed for j in jobs]
    # N spans the log-uniform range
    n = np.log([j.n_lens for j in jobs])
    assert n.min() < math.log(2000) and n.max() > math.log(12000)


def test_serve_stream_recipe():
    reqs = W.serve_stream(n_req=1000, seed=5, rate_hz=2.0)
    t = np.array([r.arrival_s for r in reqs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    # exponential gaps with mean 1/rate: mean and coefficient of variation
    assert abs(gaps.mean() - 0.5) < 0.05 and abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    for r in reqs:
        j = r.job
        assert 200 <= j.n_lens <= 80000
        assert j.npix in (512, 1024, 2048, 4096, 8192) and j.n1 == 4 * j.npix
    assert [r.rid for r in reqs] == list(range(1000))
    again = W.serve_stream(n_req=1000, seed=5, rate_hz=2.0)
    assert [(r.arrival_s, r.job.seed) for r in again] == [(r.arrival_s, r.job.seed) for r in reqs]


def test_sampling_helpers():
    ids = W.sample_tiles(1000, 256, seed=7)
    assert ids.dtype == np.int64 and len(np.unique(ids)) == 256 and np.all(np.diff(ids) > 0)
    assert ids.min() >= 0 and ids.max() < 1000
    assert np.array_equal(ids, W.sample_tiles(1000, 256, seed=7))
    ij = W.sample_rays(300, 200, 5000, seed=3)
    assert ij.shape == (5000, 2) and ij[:, 0].max() < 300 and ij[:, 1].max() < 200
    assert ij.min() >= 0

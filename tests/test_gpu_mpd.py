"""MPD and probability sums on the GPU against the oracle: bit-exact on the
same count maps (seeded synthetic maps, and a map on which the GPU's
double-single path and the oracle agree ray for ray)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_1406_0559_b300 as rs
    return rs


@pytest.mark.parametrize("shape,hi,n_bins", [((256, 256), 300, 1 << 12), ((509, 509), 20000, 1 << 16),
                                             ((1, 1), 5, 4), ((333, 77), 100000, 50000),
                                             ((4096, 4096), 3000, 1 << 20)])
def test_histogram_bit_exact(rs, shape, hi, n_bins):
    rng = np.random.default_rng(hi)
    # counts concentrated at small values with a long tail, like a map
    c = np.minimum(rng.geometric(1.0 / (hi / 10 + 1), size=shape) - 1, hi).astype(np.int32)
    c.ravel()[:: 97] = hi                      # some large counts
    j = W.PARITY.with_(npix=shape[0]) if shape[0] == shape[1] else None
    job = j if j is not None else W.PARITY.with_(npix=int(np.sqrt(c.size)))
    if c.size != job.npix * job.npix:          # non-square test array: flatten to a square
        side = int(np.ceil(np.sqrt(c.size)))
        pad = np.zeros(side * side, dtype=np.int32)
        pad[:c.size] = c.ravel()
        c = pad.reshape(side, side)
        job = W.PARITY.with_(npix=side)
    h_g = rs.count_histogram(job, torch.from_numpy(c).cuda(), n_bins=n_bins).cpu().numpy()
    h_o = oracle.count_histogram(c, n_bins)
    assert np.array_equal(h_g, h_o)


def test_fused_magnification_and_prob_sums(rs):
    rng = np.random.default_rng(8)
    job = W.GERLUMPH.with_(npix=1024)
    c = rng.poisson(40.0, size=(1024, 1024)).astype(np.int32)
    ct = torch.from_numpy(c).cuda()
    mu = torch.empty_like(ct, dtype=torch.float32)
    hist = rs.count_histogram(job, ct, n_bins=4096, mu_out=mu)
    assert torch.equal(mu, rs.magnification(job, ct))
    navg = oracle.navg(job)
    lims = [0.3 * 40 / navg * navg / navg, 1.0, 40.0 / navg, 3.0]
    b_g, a_g = rs.prob_sums(job, hist, lims)
    b_o, a_o = oracle.prob_sums(job, oracle.count_histogram(c, 4096), lims)
    assert np.array_equal(b_g.cpu().numpy(), b_o) and np.array_equal(a_g.cpu().numpy(), a_o)
    with pytest.raises(rs.RSError):
        rs.prob_sums(job, hist, [1e9])


def test_mpd_of_an_identical_map(rs):
    """The double-single map matches the oracle ray for ray on this job, so
    its MPD and probability sums must equal the oracle's exactly."""
    job = W.PARITY
    lg = rs.make_lenses(job)
    c, st = rs.shoot_map(job, lg, precision=rs.PREC_DOUBLE_SINGLE)
    co, so = oracle.shoot(job, oracle.make_lenses(job))
    assert np.array_equal(c.cpu().numpy(), co)
    hist = rs.count_histogram(job, c, n_bins=1 << 14)
    h_o = oracle.count_histogram(co, 1 << 14)
    assert np.array_equal(hist.cpu().numpy(), h_o)
    mu_th = oracle.mu_th(job.kappa, job.gamma)
    lims = [0.3 * abs(mu_th), 3.0 * abs(mu_th)]
    b_g, a_g = rs.prob_sums(job, hist, lims)
    b_o, a_o = oracle.prob_sums(job, h_o, lims)
    assert np.array_equal(b_g.cpu().numpy(), b_o) and np.array_equal(a_g.cpu().numpy(), a_o)

"""Finite-source convolution on the GPU (Sec. 2.4, Eq. 6) against the FP64
oracle: binned profiles, the convolved map at small sizes element by element
and at the survey's 10000^2 resolution on sampled pixels, pixelFlux records
and value histograms.

Tolerances (derived from the arithmetic, u = 2^-24):
  * kernel pixels: FP32 brightness per sample (a few ulp), FP32 sums of S
    samples per sample row, FP64 across rows, one rounding on store and one
    on normalisation: |dK| <= 2 (S + 8) u K + 1e-6 max K (the last term for
    the thin disc's inner edge, where 1 - sqrt(r_in / r) cancels; there the
    brightness is ~0).
  * convolved map, L2 over the map: the FFT round-off bound (Higham, Accuracy
    and Stability of Numerical Algorithms, Thm. 24.2: log2(N) eta per
    transform, eta = u + gamma_4 (sqrt 2 + u) ~ 6.7 u) for the map transform,
    the kernel transform, the product and the inverse transform, plus the
    kernel's own error (|| dK * M ||_2 <= max_rel(dK) ||M||_2):
      ||dC||_2 <= (4 log2(N) 6.7 u + 2 (S + 8) u + 4 u) ||M||_2,  N = npix^2.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def rs():
    import paper_1406_0559_b300 as rs
    return rs


def kernel_tol(k_orc, S):
    return 2 * (S + 8) * U * np.abs(k_orc) + 1e-6 * np.abs(k_orc).max()


def conv_tol(npix, S):
    return 4 * math.log2(npix * npix) * 6.7 * U + 2 * (S + 8) * U + 4 * U


@pytest.mark.parametrize("kind", W.PROFILE_KINDS)
@pytest.mark.parametrize("S", [1, 4, 8, 64])
@pytest.mark.parametrize("size_cm,w", [(3e15, 0.0025), (1e16, 24 / 4096), (4e14, 0.01)])
def test_profile_kernel_matches_oracle(rs, kind, S, size_cm, w):
    prof = W.profile_from_cm(kind, size_cm, supersample=S)
    k_orc, _ = oracle.profile_kernel(prof, w)
    k = rs.profile_kernel(prof, w).cpu().numpy().astype(np.float64)
    assert k.shape == k_orc.shape
    assert np.all(np.abs(k - k_orc) <= kernel_tol(k_orc, S)), np.abs(k - k_orc).max()
    assert abs(k.sum() - 1.0) < 1e-5


def test_point_source_kernel_is_the_impulse(rs):
    prof = W.profile_from_cm("gaussian", 1e14)            # 0.002 R_E, pixel 0.01
    k = rs.profile_kernel(prof, 0.01).cpu().numpy()
    assert k.shape == (1, 1) and k[0, 0] == 1.0


def small_job(npix, kind, S=8, size_cm=1.2e15, seed=8):
    return W.CONV_SMALL.with_(npix=npix, width=0.0025 * npix, seed=seed,
                              profile=W.profile_from_cm(kind, size_cm, supersample=S))


# own transforms: 96 (rows 48 = 4 4 3), 200, 256, 300 (rows 150 = 2 5 5 3),
# 512 (rows 256 and columns 512: both in the padded shared-memory layout of
# lengths that are multiples of 256; 256 pads its columns only);
# cuFFT: 201, 97 (odd, prime factors above 5)
@pytest.mark.parametrize("npix", [96, 200, 201, 256, 300, 512, 97])
@pytest.mark.parametrize("kind", ["uniform", "gaussian", "thin-disc", "power-law"])
def test_convolution_matches_oracle(rs, npix, kind):
    job = small_job(npix, kind)
    counts = W.count_map(job)
    scale = 1.0 / 37.25
    k_orc, _ = oracle.profile_kernel(job.profile, job.pixel)
    c_orc = oracle.convolve_direct(counts * scale, k_orc)
    conv = rs.Convolver(npix)
    conv.set_profile(job.profile, job.pixel)
    d_counts = torch.from_numpy(counts).cuda()
    c = conv.apply_counts(d_counts, scale).cpu().numpy().astype(np.float64)
    m = counts * scale
    err = np.linalg.norm(c - c_orc) / np.linalg.norm(m)
    assert err <= conv_tol(npix, job.profile.supersample), err
    # the input is left as it was and the total is conserved (sum K = 1)
    assert np.array_equal(d_counts.cpu().numpy(), counts)
    assert abs(c.sum() / m.sum() - 1) < 1e-5
    conv.close()


def test_padded_layout_1024_matches_oracle(rs):
    """1024^2: rows of 512 and columns of 1024 complex values, the padded
    layout in all three passes with two stages of span 1-8 in each."""
    job = small_job(1024, "gaussian", seed=21)
    counts = W.count_map(job)
    k_orc, _ = oracle.profile_kernel(job.profile, job.pixel)
    c_orc = oracle.convolve_direct(counts * 0.02, k_orc)
    conv = rs.Convolver(1024)
    assert conv.fft_kind == rs.CONV_FFT_OWN
    conv.set_profile(job.profile, job.pixel)
    c = conv.apply_counts(torch.from_numpy(counts).cuda(), 0.02).cpu().numpy().astype(np.float64)
    err = np.linalg.norm(c - c_orc) / np.linalg.norm(counts * 0.02)
    assert err <= conv_tol(1024, job.profile.supersample), err
    conv.close()


def test_transform_kind_by_size(rs):
    """The survey's sizes run the library's own FFTs; sizes outside its
    radices (odd, prime factors above 5) or above 10240 run cuFFT."""
    for n, own in [(4096, True), (10000, True), (96, True), (300, True), (1000, True),
                   (97, False), (201, False), (250, False), (333, False), (12000, False)]:
        conv = rs.Convolver(n)
        assert (conv.fft_kind == rs.CONV_FFT_OWN) == own, n
        conv.close()


def test_own_and_cufft_transforms_agree(rs):
    """Maps of 1000^2 (own transforms) and 999^2 (cuFFT) cut from one count
    field both agree with the oracle's direct sum within the FFT bound."""
    job = small_job(1000, "gaussian")
    counts = W.count_map(job)
    k_orc, _ = oracle.profile_kernel(job.profile, job.pixel)
    for n in (1000, 999):
        cj = job.with_(npix=n, width=job.pixel * n)
        cc = counts[:n, :n].copy()
        c_orc = oracle.convolve_direct(cc * 0.01, k_orc)
        conv = rs.Convolver(n)
        conv.set_profile(cj.profile, cj.pixel)
        c = conv.apply_counts(torch.from_numpy(cc).cuda(), 0.01).cpu().numpy().astype(np.float64)
        err = np.linalg.norm(c - c_orc) / np.linalg.norm(cc * 0.01)
        assert err <= conv_tol(n, cj.profile.supersample), (n, err)
        conv.close()


def test_float_input_and_in_place(rs):
    job = small_job(128, "gaussian")
    rng = np.random.default_rng(2)
    m = (10 ** rng.uniform(-1, 2, (128, 128))).astype(np.float32)
    k_orc, _ = oracle.profile_kernel(job.profile, job.pixel)
    c_orc = oracle.convolve_direct(m.astype(np.float64), k_orc)
    conv = rs.Convolver(128)
    conv.set_profile(job.profile, job.pixel)
    d = torch.from_numpy(m).cuda()
    out = conv.apply(d)
    assert torch.equal(d.cpu(), torch.from_numpy(m))           # R2C leaves its input
    c1 = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(c1 - c_orc) / np.linalg.norm(m) <= conv_tol(128, 8)
    conv.apply(d, out=d)                                          # in place
    assert torch.equal(d, out)


def test_caller_kernels_impulse_and_shift(rs):
    n = 64
    rng = np.random.default_rng(4)
    m = rng.random((n, n)).astype(np.float32) * 100
    conv = rs.Convolver(n)
    conv.set_kernel(torch.ones((1, 1), dtype=torch.float32, device="cuda"))
    c = conv.apply(torch.from_numpy(m).cuda()).cpu().numpy()
    tol = conv_tol(n, 1) * np.linalg.norm(m)
    assert np.linalg.norm(c - m) <= tol
    h = 3
    k = torch.zeros((2 * h + 1, 2 * h + 1), dtype=torch.float32, device="cuda")
    k[h + 2, h - 3] = 1.0                              # a = +2 rows, b = -3 columns
    conv.set_kernel(k)
    c = conv.apply(torch.from_numpy(m).cuda()).cpu().numpy()
    assert np.linalg.norm(c - np.roll(m, (2, -3), axis=(0, 1))) <= tol
    # a random, asymmetric kernel against the oracle
    kr = rng.random((9, 9))
    kr /= kr.sum()
    conv.set_kernel(torch.from_numpy(kr.astype(np.float32)).cuda())
    c = conv.apply(torch.from_numpy(m).cuda()).cpu().numpy().astype(np.float64)
    c_orc = oracle.convolve_direct(m.astype(np.float64), kr.astype(np.float32).astype(np.float64))
    assert np.linalg.norm(c - c_orc) / np.linalg.norm(m) <= conv_tol(n, 1)


def test_convolver_errors(rs):
    conv = rs.Convolver(32)
    with pytest.raises(rs.RSError) as e:
        conv.apply(torch.zeros((32, 32), device="cuda"))          # no kernel yet
    assert e.value.code == -1
    with pytest.raises(rs.RSError) as e:                          # kernel wider than map
        conv.set_profile(W.profile_from_cm("uniform", 1e16), 0.0025)
    assert e.value.code == -6
    conv.set_profile(W.profile_from_cm("uniform", 1e15), 0.0025)
    with pytest.raises(rs.RSError) as e:                          # host buffer
        conv.apply(torch.zeros((32, 32)), out=torch.zeros((32, 32), device="cuda"))
    assert e.value.code == -1
    with pytest.raises(rs.RSError):
        rs.Convolver(1)
    assert conv.nbytes >= 2 * 8 * 32 * 17


@pytest.fixture(scope="module")
def gd1(rs):
    """The survey's 10000^2 resolution (Table 3), a 0.2 R_E Gaussian source."""
    job = W.CONV_GD1
    counts = W.count_map(job)
    d_counts = torch.from_numpy(counts).cuda()
    conv = rs.Convolver(job.npix)
    conv.set_profile(job.profile, job.pixel)
    scale = 1.0 / 300.0
    c = conv.apply_counts(d_counts, scale)
    torch.cuda.synchronize()
    yield job, counts, scale, conv, c
    conv.close()


def test_full_size_sampled_pixels(rs, gd1):
    job, counts, scale, conv, c = gd1
    n = job.npix
    rng = np.random.default_rng(11)
    qp = np.concatenate([
        np.stack([rng.integers(0, n, 1500), rng.integers(0, n, 1500)], axis=1),
        # pixels within the kernel's reach of the edges and corners (wrap-around)
        np.array([[0, 0], [0, n - 1], [n - 1, 0], [n - 1, n - 1], [5, n // 2], [n - 3, 17]]),
    ])
    k_orc, _ = oracle.profile_kernel(job.profile, job.pixel)
    ref = oracle.convolve_counts_at(counts, scale, k_orc, qp)
    got = c[torch.from_numpy(qp[:, 0]).cuda(), torch.from_numpy(qp[:, 1]).cuda()]
    got = got.cpu().numpy().astype(np.float64)
    rms_m = scale * math.sqrt(float(np.mean(counts.astype(np.float64) ** 2)))
    tol = conv_tol(n, job.profile.supersample)
    # the L2 bound, estimated on the sample, and a per-pixel cap of 10x it
    assert math.sqrt(np.mean((got - ref) ** 2)) <= tol * rms_m
    assert np.abs(got - ref).max() <= 10 * tol * rms_m
    # total conserved
    total = float(c.double().sum())
    assert abs(total / (scale * counts.sum(dtype=np.int64)) - 1) < 1e-5


def test_gd0_4096_sampled_pixels(rs):
    """The 4096^2 map over 24 R_E (the padded layout at the survey's
    power-of-two size): sampled pixels, wrapped corners included, against the
    oracle's direct sum within the FFT bound; total conserved."""
    job = W.CONV_GD0
    counts = W.count_map(job)
    n = job.npix
    scale = 1.0 / job.mean_count
    conv = rs.Convolver(n)
    assert conv.fft_kind == rs.CONV_FFT_OWN
    conv.set_profile(job.profile, job.pixel)
    c = conv.apply_counts(torch.from_numpy(counts).cuda(), scale)
    rng = np.random.default_rng(13)
    qp = np.concatenate([
        np.stack([rng.integers(0, n, 1500), rng.integers(0, n, 1500)], axis=1),
        np.array([[0, 0], [0, n - 1], [n - 1, 0], [n - 1, n - 1], [2, n // 2], [n - 5, 31]]),
    ])
    k_orc, _ = oracle.profile_kernel(job.profile, job.pixel)
    ref = oracle.convolve_counts_at(counts, scale, k_orc, qp)
    got = c[torch.from_numpy(qp[:, 0]).cuda(), torch.from_numpy(qp[:, 1]).cuda()]
    got = got.cpu().numpy().astype(np.float64)
    rms_m = scale * math.sqrt(float(np.mean(counts.astype(np.float64) ** 2)))
    tol = conv_tol(n, job.profile.supersample)
    assert math.sqrt(np.mean((got - ref) ** 2)) <= tol * rms_m
    assert np.abs(got - ref).max() <= 10 * tol * rms_m
    total = float(c.double().sum())
    assert abs(total / (scale * counts.sum(dtype=np.int64)) - 1) < 1e-5
    conv.close()


def test_pixel_flux_records(rs, gd1):
    job, counts, scale, conv, c = gd1
    rec = rs.pixel_flux(c, k=4000, seed=77)
    x, y, v = rs.unpack_pixel_flux(rec)
    xy = oracle.pixel_locations(77, job.npix, 4000)
    assert np.array_equal(x, xy[:, 0]) and np.array_equal(y, xy[:, 1])
    cv = c.cpu().numpy()
    assert np.array_equal(v, cv[y, x])                  # the map's own values, bit for bit
    # caller-given locations, one outside the map
    loc = torch.tensor([[0, 0], [9999, 9999], [123, 4567], [-1, 5], [10000, 3]],
                       dtype=torch.int16, device="cuda")
    x, y, v = rs.unpack_pixel_flux(rs.pixel_flux(c, xy=loc))
    assert v[0] == cv[0, 0] and v[1] == cv[9999, 9999] and v[2] == cv[4567, 123]
    assert np.isnan(v[3]) and np.isnan(v[4]) and x[3] == -1 and y[4] == 3


@pytest.mark.parametrize("n_bins", [0, 1, 2, 500, 1023, 4094])
def test_value_histogram_bit_exact(rs, n_bins):
    rng = np.random.default_rng(12 + n_bins)
    v = (10 ** rng.normal(0.3, 0.6, 3_000_001)).astype(np.float32)
    edges = W.log_edges(-2, 3, n_bins)
    v[:edges.size] = edges
    v[edges.size] = np.nan
    v[edges.size + 1] = -5
    hist = rs.value_histogram(torch.from_numpy(v).cuda(), edges).cpu().numpy()
    assert np.array_equal(hist, oracle.value_histogram(v, edges))
    # a smooth region: whole warps in one bin
    flat = np.full(1_000_003, edges[edges.size // 2], dtype=np.float32)
    flat[::7] = edges[0]
    hf = rs.value_histogram(torch.from_numpy(flat).cuda(), edges).cpu().numpy()
    assert np.array_equal(hf, oracle.value_histogram(flat, edges))
    # an unaligned start (scalar path)
    hu = rs.value_histogram(torch.from_numpy(v).cuda()[1:], edges).cpu().numpy()
    assert np.array_equal(hu, oracle.value_histogram(v[1:], edges))
    h0 = rs.value_histogram(torch.empty(0, dtype=torch.float32, device="cuda"), edges)
    assert int(h0.sum()) == 0
    if edges.size > 1:
        with pytest.raises(rs.RSError):
            rs.value_histogram(torch.from_numpy(v).cuda(), edges[::-1].copy())
    with pytest.raises(rs.RSError):
        rs.value_histogram(torch.from_numpy(v).cuda(), np.arange(4096, dtype=np.float32))


def test_convolved_mpd_matches_oracle(rs):
    """MPD of a convolved map: the GPU histogram of the GPU map and the
    oracle's histogram of the oracle's map differ only by pixels within the
    per-pixel error bound of a bin edge."""
    job = small_job(256, "gaussian", size_cm=2e15)
    counts = W.count_map(job)
    scale = 1.0 / 300
    k_orc, _ = oracle.profile_kernel(job.profile, job.pixel)
    c_orc = oracle.convolve_direct(counts * scale, k_orc)
    conv = rs.Convolver(256)
    conv.set_profile(job.profile, job.pixel)
    c = conv.apply_counts(torch.from_numpy(counts).cuda(), scale)
    edges = W.log_edges(-0.5, 0.5, 200)
    hg = rs.value_histogram(c.view(-1), edges).cpu().numpy()
    ho = oracle.value_histogram(c_orc.astype(np.float32), edges)
    assert hg.sum() == ho.sum() == 256 * 256
    delta = 10 * conv_tol(256, 8) * scale * math.sqrt(float(np.mean(counts.astype(float) ** 2)))
    e64 = edges.astype(np.float64)
    near = np.abs(c_orc.ravel()[:, None] - e64[None, :]).min(axis=1) <= delta
    assert np.abs(hg - ho).sum() <= 2 * int(near.sum())


def test_value_histogram_signed_zero_infinities_and_dense_edges(rs):
    """Values and edges at -0/+0, infinities, NaN and negative numbers, and
    edges packed closer than the bucket width: bit-exact against the oracle."""
    edges = np.array([-np.inf, -2.5, -1.0, -0.0, 1e-30, 1.0, 1.0000001, 1.0000002, 3.0, np.inf],
                     dtype=np.float32)
    edges = np.unique(edges)          # ascending, -0.0 and +0.0 merged
    v = np.array([-0.0, 0.0, -1.0, -1.0000001, 1.0, 1.0000001, 1.00000012, 2.9999998, 3.0,
                  np.inf, -np.inf, np.nan, 1e-30, -1e-30, 5e-39, -5e-39, 1e38, -1e38] * 37,
                 dtype=np.float32)
    hist = rs.value_histogram(torch.from_numpy(v).cuda(), edges).cpu().numpy()
    assert np.array_equal(hist, oracle.value_histogram(v, edges))
    dense = (1.0 + np.arange(3000, dtype=np.float32) * np.float32(2 ** -23)).astype(np.float32)
    rng = np.random.default_rng(5)
    vd = (1.0 + rng.integers(0, 3100, 200_001).astype(np.float32) * np.float32(2 ** -23))
    vd = vd.astype(np.float32)
    hd = rs.value_histogram(torch.from_numpy(vd).cuda(), dense).cpu().numpy()
    assert np.array_equal(hd, oracle.value_histogram(vd, dense))


@pytest.mark.parametrize("npix,h", [(256, 0), (256, 1), (300, 4), (333, 6), (1000, 6),
                                    (300, 7), (1000, 10)])
def test_direct_and_fft_paths_small_kernels(rs, npix, h):
    """Kernels up to 13^2 are summed directly (no FFT), larger ones go
    through Eq. 6: element by element
    against the oracle, counts and float input, in place included."""
    rng = np.random.default_rng(npix + h)
    k = rng.random((2 * h + 1, 2 * h + 1))            # asymmetric: orientation matters
    k /= k.sum()
    k32 = k.astype(np.float32)
    counts = W.count_map(W.CONV_SMALL.with_(npix=npix, seed=npix + 7 * h))
    scale = 1.0 / 29.5
    conv = rs.Convolver(npix)
    conv.set_kernel(torch.from_numpy(k32).cuda())
    ref = oracle.convolve_direct(counts * scale, k32.astype(np.float64))
    d_counts = torch.from_numpy(counts).cuda()
    c = conv.apply_counts(d_counts, scale).cpu().numpy().astype(np.float64)
    m = counts * scale
    if h <= 6:
        # FP32 sums of (2h+1)^2 positive terms: relative error <= (2h+1)^2 u per pixel
        tol = ((2 * h + 1) ** 2 + 2) * U
        assert np.all(np.abs(c - ref) <= tol * np.abs(ref) + 1e-30), np.abs(c / ref - 1).max()
    else:
        tol = conv_tol(npix, 1) * np.linalg.norm(m)
        assert np.linalg.norm(c - ref) <= tol
    assert np.array_equal(d_counts.cpu().numpy(), counts)
    mf = torch.from_numpy(m.astype(np.float32)).cuda()
    reff = oracle.convolve_direct(m.astype(np.float32).astype(np.float64), k32.astype(np.float64))
    cf = conv.apply(mf)
    if h <= 6:
        assert np.all(np.abs(cf.cpu().numpy() - reff) <= tol * np.abs(reff))
    else:
        assert np.linalg.norm(cf.cpu().numpy() - reff) <= tol
    conv.apply(mf, out=mf)                                      # in place
    assert torch.equal(mf, cf)


def test_direct_path_full_size_sampled(rs, gd1):
    """A small source (0.01 R_E, h = 4) on the 10000^2 map: the direct path,
    sampled pixels including the wrapped corners."""
    job, counts, scale, _, _ = gd1
    prof = W.profile_from_cm("gaussian", 5.0e14)
    conv = rs.Convolver(job.npix)
    conv.set_profile(prof, job.pixel)
    c = conv.apply_counts(torch.from_numpy(counts).cuda(), scale)
    k_orc, _ = oracle.profile_kernel(prof, job.pixel)
    assert k_orc.shape[0] <= 13
    n = job.npix
    rng = np.random.default_rng(12)
    qp = np.concatenate([np.stack([rng.integers(0, n, 2000), rng.integers(0, n, 2000)], axis=1),
                         np.array([[0, 0], [0, n - 1], [n - 1, 0], [n - 1, n - 1], [3, 9998]])])
    ref = oracle.convolve_counts_at(counts, scale, k_orc, qp)
    got = c[torch.from_numpy(qp[:, 0]).cuda(), torch.from_numpy(qp[:, 1]).cuda()]
    got = got.cpu().numpy().astype(np.float64)
    # kernel binning (2(S+8)u relative) plus the direct FP32 sum ((2h+1)^2 u)
    tol = (2 * (prof.supersample + 8) + k_orc.size + 2) * U
    assert np.all(np.abs(got - ref) <= tol * np.abs(ref)), np.abs(got / ref - 1).max()
    conv.close()


def test_loaded_map_with_several_profiles(rs):
    """One map, several source profiles: the loaded spectrum gives the same
    maps bit for bit as convolving from scratch (transform path), across
    kernel changes; a small kernel on a loaded map goes through the
    transforms and matches the oracle."""
    job = small_job(256, "gaussian")
    counts = W.count_map(job)
    d = torch.from_numpy(counts).cuda()
    scale = 1.0 / 41.0
    conv = rs.Convolver(256)
    conv.set_profile(job.profile, job.pixel)
    with pytest.raises(rs.RSError):
        conv.apply_loaded()                                  # nothing loaded yet
    conv.load_counts(d, scale)
    kinds = [("gaussian", 2.5e15), ("uniform", 2.0e15), ("thin-disc", 3.0e15)]
    for kind, size in kinds:
        prof = W.profile_from_cm(kind, size)
        conv.set_profile(prof, job.pixel)
        assert rs.profile_half(prof, job.pixel) > 6          # transform path
        a = conv.apply_loaded().clone()
        conv2 = rs.Convolver(256)
        conv2.set_profile(prof, job.pixel)
        b = conv2.apply_counts(d, scale)
        assert torch.equal(a, b), kind
        conv2.close()
    # a small kernel on the loaded map (transform path) against the oracle
    small = W.profile_from_cm("gaussian", 5e14)
    conv.set_profile(small, job.pixel)
    c = conv.apply_loaded().cpu().numpy().astype(np.float64)
    k_orc, _ = oracle.profile_kernel(small, job.pixel)
    ref = oracle.convolve_direct(counts * scale, k_orc)
    assert np.linalg.norm(c - ref) / np.linalg.norm(counts * scale) <= conv_tol(256, 8)
    # float maps load too; apply_counts discards the loaded spectrum
    conv.load(torch.from_numpy((counts * scale).astype(np.float32)).cuda())
    conv.apply_loaded()
    conv.apply_counts(d, scale)
    with pytest.raises(rs.RSError):
        conv.apply_loaded()
    conv.close()


def test_kernel_slots(rs):
    """Kernel spectra kept in slots give the same maps bit for bit as the
    same profile set as the convolver's kernel; bad slots are refused."""
    job = small_job(256, "gaussian")
    counts = W.count_map(job)
    d = torch.from_numpy(counts).cuda()
    scale = 1.0 / 33.0
    profs = [W.profile_from_cm(k, c) for k, c in [("gaussian", 2.5e15), ("uniform", 2e15),
                                                  ("power-law", 3e15)]]
    conv = rs.Convolver(256)
    for k, p in enumerate(profs):
        conv.set_profile(p, job.pixel, slot=k + 1)
    conv.load_counts(d, scale)
    outs = [conv.apply_loaded(slot=k + 1).clone() for k in range(len(profs))]
    for p, o in zip(profs, outs):
        conv.set_profile(p, job.pixel)            # slot 0, the loaded map survives
        assert torch.equal(conv.apply_loaded(), o)
    with pytest.raises(rs.RSError):
        conv.apply_loaded(slot=9)                 # never set
    with pytest.raises(rs.RSError):
        conv.set_profile(profs[0], job.pixel, slot=16)
    assert conv.nbytes >= (3 + len(profs)) * 8 * 256 * 129
    conv.close()

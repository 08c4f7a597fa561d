"""Indexed count maps (App. B) and map previews / colorbar (Sec. 3.2.1,
Sec. 4.6) on the GPU against the oracle: integer and byte work, bit-exact."""
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


def words_u32(w: torch.Tensor) -> np.ndarray:
    return w.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,hi,seed", [(1, 1, 0), (31, 2, 1), (33, 5, 2), (1000, 7, 3),
                                       (4097, 3000, 4), (100003, 70000, 5), (65536, 1, 6)])
def test_encode_matches_oracle_and_round_trips(rs, n, hi, seed):
    rng = np.random.default_rng(seed)
    counts = rng.integers(0, hi, n).astype(np.int32)
    t_o, w_o, b_o = oracle.index_encode(counts)
    d = torch.from_numpy(counts).cuda()
    table, words, info = rs.index_encode(d)
    assert info["bits"] == b_o and info["distinct"] == t_o.size
    assert info["max_count"] == counts.max() and info["words"] == w_o.size
    assert np.array_equal(table.cpu().numpy(), t_o)
    assert np.array_equal(words_u32(words), w_o)
    back = rs.index_decode(words, n, info["bits"], table)
    assert np.array_equal(back.cpu().numpy(), counts)


@pytest.mark.parametrize("bits", [8, 13, 16, 20, 31, 32])
def test_fixed_widths(rs, bits):
    rng = np.random.default_rng(bits)
    counts = rng.integers(0, 250, 12345).astype(np.int32)
    _, w_o, _ = oracle.index_encode(counts, bits=bits)
    table, words, info = rs.index_encode(torch.from_numpy(counts).cuda(), bits=bits)
    assert info["bits"] == bits and np.array_equal(words_u32(words), w_o)
    assert np.array_equal(rs.index_decode(words, counts.size, bits, table).cpu().numpy(), counts)


def test_gd0_map_round_trip(rs):
    """A 4096^2 count map (GD0 resolution) element by element against the
    oracle; the table grows past its first guess."""
    job = W.CONV_GD0.with_(mean_count=3000.0)
    counts = W.count_map(job, sigma=1.0)
    t_o, w_o, b_o = oracle.index_encode(counts)
    d = torch.from_numpy(counts).cuda()
    table, words, info = rs.index_encode(d, table_cap=1000)
    assert info["distinct"] == t_o.size > 1000 and info["bits"] == b_o
    assert np.array_equal(table.cpu().numpy(), t_o)
    assert np.array_equal(words_u32(words), w_o)
    assert torch.equal(rs.index_decode(words, counts.size, b_o, table).view(job.npix, job.npix), d)


def test_gd1_map_round_trip_and_sampled_groups(rs):
    """The 10000^2 map (GD1-GD3 resolution): exact round trip, the table
    against numpy.unique, sampled 32-pixel groups against the oracle."""
    job = W.CONV_GD1
    counts = W.count_map(job)
    d = torch.from_numpy(counts).cuda()
    table, words, info = rs.index_encode(d)
    uniq = np.unique(counts)
    t = table.cpu().numpy()
    assert np.array_equal(t, uniq)
    b = info["bits"]
    assert b == oracle.index_bits(uniq.size)
    assert info["words"] == oracle.index_words(counts.size, b)
    assert torch.equal(rs.index_decode(words, counts.size, b, table).view_as(d), d)
    flat = counts.ravel()
    w = words_u32(words)
    rng = np.random.default_rng(3)
    for g in np.concatenate([rng.integers(0, flat.size // 32, 200), [flat.size // 32 - 1]]):
        ref = oracle.index_pack(flat[32 * g:32 * g + 32], uniq, b)
        assert np.array_equal(w[g * b:(g + 1) * b], ref), g


def test_codec_errors_and_corrupt_input(rs):
    with pytest.raises(rs.RSError) as e:
        rs.index_encode(torch.tensor([1, -3, 2], dtype=torch.int32, device="cuda"))
    assert e.value.code == -1
    with pytest.raises(rs.RSError) as e:
        rs.index_encode(torch.arange(300, dtype=torch.int32, device="cuda"), bits=8)
    assert e.value.code == -6
    counts = torch.arange(300, dtype=torch.int32, device="cuda")
    table, words, info = rs.index_encode(counts)
    out = rs.index_decode(words, 300, info["bits"], table[:100])     # indices past the table
    o = out.cpu().numpy()
    assert np.array_equal(o[:100], np.arange(100)) and np.all(o[100:] == -1)


def test_colorbar_lut_matches_oracle(rs):
    for pos, rgb in [([0, 255], [[0, 0, 0], [255, 255, 255]]),
                     ([0, 64, 128, 128, 255],
                      [[0, 0, 0], [255, 0, 10], [255, 255, 0], [0, 0, 255], [255, 255, 255]]),
                     ([0, 1, 2, 254, 255], [[9, 8, 7], [200, 1, 3], [5, 5, 5], [0, 0, 0], [1, 2, 3]])]:
        assert np.array_equal(rs.colorbar_lut(pos, rgb), oracle.colorbar_lut(pos, rgb))
    with pytest.raises(rs.RSError):
        rs.colorbar_lut([0, 300, 255], [[0, 0, 0]] * 3)


@pytest.mark.parametrize("s", [1000, 200, 7, 1])
def test_previews_match_oracle(rs, s):
    n = 1000
    rng = np.random.default_rng(s)
    counts = rng.integers(0, 5000, (n, n)).astype(np.int32)
    counts[0, :256] = (np.arange(256) * 10).astype(np.int32)       # on the thresholds
    thr = np.arange(1, 256) * 10.0
    lut = oracle.colorbar_lut([0, 100, 200, 255], [[0, 0, 0], [255, 0, 0], [255, 255, 0],
                                                   [255, 255, 255]])
    gray, rgba = rs.preview(torch.from_numpy(counts).cuda(), s, thr, lut)
    g_o = oracle.sample_gray(counts, s, thr)
    assert np.array_equal(gray.cpu().numpy(), g_o)
    assert np.array_equal(rs.rgba_bytes(rgba), oracle.colorize(g_o, lut))
    mu = (10 ** rng.uniform(-1, 2, (n, n))).astype(np.float32)
    tf = W.log_edges(-1, 2, 254)
    mu[1, :255] = tf
    gray, _ = rs.preview(torch.from_numpy(mu).cuda(), s, tf)
    assert np.array_equal(gray.cpu().numpy(), oracle.sample_gray(mu, s, tf))


def test_colorize_and_png(rs, tmp_path):
    lut = rs.colorbar_lut([0, 255], [[10, 20, 30], [250, 240, 230]])
    gray = torch.arange(256, dtype=torch.uint8, device="cuda").view(16, 16)
    rgba = rs.colorize(gray, lut)
    assert np.array_equal(rs.rgba_bytes(rgba), oracle.colorize(gray.cpu().numpy(), lut))
    p = tmp_path / "icon.png"
    rs.write_png(str(p), rs.rgba_bytes(rgba))
    assert p.read_bytes()[:8] == b"\x89PNG\r\n\x1a\n"


@pytest.mark.parametrize("bits", list(range(1, 33)))
def test_decode_every_width(rs, bits):
    """One decode kernel per bit width: each against the oracle's packing,
    with a ragged last chunk, a table past the shared-memory limit for wide
    codes, and an output buffer that is not 16-byte aligned."""
    rng = np.random.default_rng(200 + bits)
    distinct = min(2 ** bits, 20000 if bits >= 15 else 3000)
    n = max(3 * 1024, distinct) + 37 * bits
    table = np.sort(rng.choice(2 ** 31 - 1, distinct, replace=False)).astype(np.int32)
    counts = table[rng.integers(0, distinct, n)]
    counts[:distinct] = table                       # every entry used
    t_o, w_o, b_o = oracle.index_encode(counts, bits=bits)
    tg, words, info = rs.index_encode(torch.from_numpy(counts).cuda(), bits=bits)
    assert info["bits"] == bits and np.array_equal(words_u32(words), w_o)
    assert np.array_equal(tg.cpu().numpy(), t_o)
    assert np.array_equal(rs.index_decode(words, n, bits, tg).cpu().numpy(), counts)
    buf = torch.full((n + 1,), 7, dtype=torch.int32, device="cuda")
    rs.index_decode(words, n, bits, tg, out=buf[1:])
    b = buf.cpu().numpy()
    assert b[0] == 7 and np.array_equal(b[1:], counts)


@pytest.mark.parametrize("vmax", [16382, 16383, 16384, 16385])
def test_shared_memory_limits(rs, vmax):
    """Both sides of the shared-memory paths: rank table (largest count below
    16384 or not) and decode table (16384 entries or more)."""
    rng = np.random.default_rng(vmax)
    counts = np.concatenate([np.arange(vmax + 1), rng.integers(0, vmax + 1, 50000)]).astype(np.int32)
    rng.shuffle(counts)
    t_o, w_o, b_o = oracle.index_encode(counts)
    tg, words, info = rs.index_encode(torch.from_numpy(counts).cuda())
    assert info["distinct"] == vmax + 1 and info["bits"] == b_o
    assert np.array_equal(words_u32(words), w_o)
    assert np.array_equal(rs.index_decode(words, counts.size, b_o, tg).cpu().numpy(), counts)

"""Comparison helpers for GPU-vs-oracle parity (no method arithmetic here).

Tolerances (the spec bar for this path):
  * total ray counts: conservation exact on each side, GPU run-to-run
    bit-identical;
  * per ray: at most FLIP_MAX of the compared rays in a different pixel
    (or in/out of the map on one side only);
  * per pixel: relative L1 of the magnification <= L1_MAX over pixels where
    the oracle map holds at least 100 rays.
"""
import numpy as np

FLIP_MAX = 1e-5
L1_MAX = 1e-3


def gpu_tile_rays(tile_ids, tx, ty, tiles1, n1, n2):
    """(i, j) of every ray of the listed tiles, in the dump order of
    rs_shoot_tiles (tile-major, then row, then column), plus a validity mask."""
    tile_ids = np.asarray(tile_ids, dtype=np.int64)
    tj, ti = np.divmod(tile_ids, tiles1)
    b, a = np.meshgrid(np.arange(ty), np.arange(tx), indexing="ij")
    i = ti[:, None, None] * tx + a[None]
    j = tj[:, None, None] * ty + b[None]
    ij = np.stack([i.ravel(), j.ravel()], axis=1)
    valid = (ij[:, 0] < n1) & (ij[:, 1] < n2)
    return ij, valid


def flip_fraction(gpu_pix: np.ndarray, orc_pix: np.ndarray, orc_status: np.ndarray):
    """Fraction of rays whose (in/out, p, q) differ.  gpu_pix (k, 2) with -1
    for out; orc_pix (k, 2) and status (0 = in)."""
    g_in = gpu_pix[:, 0] >= 0
    o_in = orc_status == 0
    diff = (g_in != o_in) | (g_in & o_in & np.any(gpu_pix != orc_pix, axis=1))
    return float(diff.mean()) if diff.size else 0.0, int(diff.sum())


def rel_l1(mu_gpu: np.ndarray, mu_orc: np.ndarray, counts_orc: np.ndarray, min_count=100):
    m = counts_orc >= min_count
    if not m.any():
        return 0.0, 0
    return float(np.abs(mu_gpu[m] - mu_orc[m]).sum() / mu_orc[m].sum()), int(m.sum())


def histogram_pixels(pix: np.ndarray, npix: int) -> np.ndarray:
    """Count map from per-ray pixels (rows q, columns p), -1 ignored."""
    ok = pix[:, 0] >= 0
    flat = pix[ok, 1].astype(np.int64) * npix + pix[ok, 0].astype(np.int64)
    return np.bincount(flat, minlength=npix * npix).reshape(npix, npix).astype(np.int32)

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


def window_rays(rs, job, lens, window: int, precisions, margin: int = 2, chunk_tiles: int = 4096):
    """Rays of a full-size map that can land in the central window x window
    pixels: every ray whose image under precisions[0] lies within `margin`
    pixels of the window (first-pass errors are far below a pixel, so no ray
    of the window is missed), from per-ray dumps of all tiles in chunks.
    Returns (ij (k, 2) int64, {precision: pixels (k, 2) int32}, p0) with the
    window's pixels [p0, p0 + window) on both axes."""
    import torch
    p0 = (job.npix - window) // 2
    lo_, hi_ = p0 - margin, p0 + window + margin
    tx, ty = rs.tile_shape(precisions[0], 0)
    t1, t2 = -(-job.n1 // tx), -(-job.n2 // ty)
    ij_all, pix_all = [], {p: [] for p in precisions}
    b, a = torch.meshgrid(torch.arange(ty, device="cuda"), torch.arange(tx, device="cuda"),
                          indexing="ij")
    for c0 in range(0, t1 * t2, chunk_tiles):
        ids = torch.arange(c0, min(t1 * t2, c0 + chunk_tiles), dtype=torch.int64, device="cuda")
        pixs = {}
        for p in precisions:
            _, pix = rs.shoot_tiles(job, lens, ids, precision=p)
            pixs[p] = pix.reshape(-1, 2)
        tj, ti = ids // t1, ids % t1
        i = (ti[:, None, None] * tx + a[None]).reshape(-1)
        j = (tj[:, None, None] * ty + b[None]).reshape(-1)
        q = pixs[precisions[0]]
        # rays outside the map dump -1: keep those too when any precision has
        # them in the window, else by the first precision's pixel
        sel = (i < job.n1) & (j < job.n2)
        inwin = torch.zeros_like(sel)
        for p in precisions:
            pp = pixs[p]
            inwin |= (pp[:, 0] >= lo_) & (pp[:, 0] < hi_) & (pp[:, 1] >= lo_) & (pp[:, 1] < hi_)
        sel &= inwin
        k = sel.nonzero().squeeze(1)
        ij_all.append(torch.stack([i[k], j[k]], 1).cpu())
        for p in precisions:
            pix_all[p].append(pixs[p][k].cpu())
    ij = torch.cat(ij_all).numpy().astype(np.int64)
    return ij, {p: torch.cat(v).numpy() for p, v in pix_all.items()}, p0


def window_compare(gp: np.ndarray, op: np.ndarray, ost: np.ndarray, p0: int, window: int,
                   min_count: int = 100):
    """Flips and per-pixel counts restricted to the window: rays in the window
    on either side whose pixel differs (or that are in it on one side only),
    over the rays the oracle puts in the window; relative L1 of the window's
    counts over pixels where the oracle has >= min_count rays."""
    def in_win(p):
        return (p[:, 0] >= p0) & (p[:, 0] < p0 + window) & (p[:, 1] >= p0) & (p[:, 1] < p0 + window)
    g_in = in_win(gp)
    o_in = (ost == 0) & in_win(op)
    diff = (g_in != o_in) | (g_in & o_in & np.any(gp != op, axis=1))
    n_o = int(o_in.sum())

    def counts(p, m):
        flat = (p[m, 1] - p0).astype(np.int64) * window + (p[m, 0] - p0)
        return np.bincount(flat, minlength=window * window)
    cg, co = counts(gp, g_in), counts(op, o_in)
    m = co >= min_count
    l1 = float(np.abs(cg[m] - co[m]).sum() / co[m].sum()) if m.any() else None
    l1_all = float(np.abs(cg - co).sum() / max(1, co.sum()))
    return {"rays_in_window": n_o, "flips": int(diff.sum()),
            "flip_fraction": float(diff.sum()) / max(1, n_o),
            "pixels_with_min_count": int(m.sum()), "rel_l1_min_count": l1,
            "rel_l1_all_pixels": l1_all, "max_count": int(co.max()) if co.size else 0}

"""The precision workload (kappa = 0.8 split 0.4 / 0.4 into stars and smooth
matter, gamma = 0.2, 50,000 Salpeter lenses, 4096^2 map, 16384^2 rays)
compared with the FP64 oracle on a central pixel window: every ray that can
land in the window is found from full per-ray dumps of the map, and the
oracle shoots those rays.  Plain FP32, compensated and refined maps are
compared ray by ray (flips) and pixel by pixel (relative L1 where the oracle
window holds >= 100 rays).  The benchmark's window mode runs the same
comparison on the 512^2 window."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def test_precision_workload_window_against_oracle():
    import paper_1406_0559_b300 as rs
    job = W.PRECISION
    window = 128
    lens = rs.make_lenses(job)
    precs = (rs.PREC_COMPENSATED, rs.PREC_FP32, rs.PREC_REFINED)
    ij, pix, p0 = PT.window_rays(rs, job, lens, window, precs)
    assert p0 == (4096 - window) // 2 and ij.shape[0] > 100000
    _, op, ost = oracle.shoot_rays(job, oracle.make_lenses(job), ij)
    res = {p: PT.window_compare(pix[p], op, ost, p0, window) for p in precs}
    for p, r in res.items():
        print(f"\nprecision {p}: {r}")
    n = res[rs.PREC_REFINED]["rays_in_window"]
    # refined: rays near an edge decided in double-single, then FP64
    assert res[rs.PREC_REFINED]["flips"] <= max(1, int(PT.FLIP_MAX * n))
    # compensated: its documented floor at 4096^2 (FP32 per-term rounding)
    assert res[rs.PREC_COMPENSATED]["flip_fraction"] <= 2e-4
    assert res[rs.PREC_FP32]["flip_fraction"] <= 2e-2
    # the window's counts (L1 over all pixels: each moved ray counts twice)
    assert res[rs.PREC_REFINED]["rel_l1_all_pixels"] <= 2 * PT.FLIP_MAX
    for p in precs:
        if res[p]["rel_l1_min_count"] is not None and p != rs.PREC_FP32:
            assert res[p]["rel_l1_min_count"] <= PT.L1_MAX

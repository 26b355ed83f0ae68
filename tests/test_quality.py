"""PSNR and SSIM of a completed tensor (Sec. 4), computed by libfctn, against
the oracle's definitions evaluated on the same X."""
import numpy as np
import pytest

from oracle import fctn_oracle as O
from tests.util import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2510_22506_gb300 import fctn
    return fctn


@pytest.mark.parametrize("dims,r,cap,precision", [((30, 30, 10), 3, None, "fp64"), ((48, 40, 9), 4, None, "fp32"),
                                                   ((13, 7, 3, 5), 3, (3, 2), "fp64"), ((37, 29), 5, None, "fp32"),
                                                   ((144, 176, 3, 5), 3, (3, 3), "fp32")])
def test_quality_matches_oracle(F, dims, r, cap, precision):
    d = inputs(None, dims=dims, r=r, p=0.3, idx=46, noise=0.0, cap=cap)
    p = F.make_params(d["dims"], d["R"], precision=precision)
    dt = F.elem_dtype(p)
    h = F.fctn_create(p)
    try:
        F.fctn_set_data(h, np.ascontiguousarray(d["Y"].astype(dt)), d["mask"].astype(np.uint8))
        F.fctn_set_factors(h, [np.ascontiguousarray(a.astype(dt)) for a in d["init"]])
        F.fctn_pam_sweep(h, 5)
        X = np.empty(d["dims"], dtype=dt)
        F.fctn_get_X(h, X)
        truth = np.ascontiguousarray(d["truth"].astype(dt))
        ps, ss = F.fctn_quality(h, truth)
        # the same call with the truth already on the device
        import torch
        tt = torch.from_numpy(truth).cuda()
        ps2, ss2 = F.fctn_quality(h, tt)
    finally:
        F.fctn_destroy(h)
    want_p = O.psnr(X, truth)
    want_s = O.ssim(X, truth)
    assert abs(ps - want_p) <= 1e-9 * abs(want_p), (ps, want_p)
    assert abs(ss - want_s) <= 1e-9, (ss, want_s)
    assert (ps2, ss2) == (ps, ss)


def test_quality_of_truth_itself(F):
    d = inputs(None, dims=(20, 16, 4), r=2, p=1.0, idx=47, noise=0.0, cap=None)
    p = F.make_params(d["dims"], d["R"], precision="fp64")
    h = F.fctn_create(p)
    try:
        F.fctn_set_data(h, np.ascontiguousarray(d["truth"]), np.ones(d["dims"], dtype=np.uint8))
        ps, ss = F.fctn_quality(h, np.ascontiguousarray(d["truth"]))
    finally:
        F.fctn_destroy(h)
    assert ps == pytest.approx(120.0)  # MSE floored at 1e-12
    assert ss == pytest.approx(1.0, abs=1e-12)

"""Tensor-core (tcgen05) TF32 / BF16 paths against the FP32 path and the oracle.

Reduced-precision criterion: the final PSNR against the ground truth stays
within 0.05 dB of the FP64 oracle's for TF32; pure BF16 sweeps on these small
shapes (8 mantissa bits, few terms per product) within 0.1 dB.  The 0.05 dB
acceptance of the mixed path for both precisions on the 256x256x31x8
workload is tests/test_workloads_full.py.  The one-sweep comparison with the
FP32 path isolates the contraction precision (the solve is the same FP32
path with its refinement in all three).
"""
import numpy as np
import pytest

from oracle import fctn_oracle as O
from tests.util import gpu_run, inputs, oracle_run, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2510_22506_gb300 import fctn
    return fctn


@pytest.mark.parametrize("dims,r,cap", [((48, 40, 9), 4, None), ((30, 24, 3, 7), 3, (3, 2)),
                                        ((12, 10, 6, 5), 6, None)])
@pytest.mark.parametrize("precision,tol", [("tf32", 3e-3), ("bf16", 3e-2)])
def test_one_sweep_close_to_fp32(F, dims, r, cap, precision, tol):
    d = inputs(None, dims=dims, r=r, p=0.3, idx=60, noise=0.0, cap=cap, dtype=np.float32)
    a = gpu_run(F, d, 1, precision="fp32")
    b = gpu_run(F, d, 1, precision=precision)
    assert rel(b["X"], a["X"]) <= tol, rel(b["X"], a["X"])


@pytest.mark.parametrize("dims,r,cap,sweeps", [((48, 40, 9), 4, None, 80), ((30, 24, 3, 7), 3, (3, 2), 60)])
@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_final_psnr_within_005_db_of_oracle(F, dims, r, cap, sweeps, precision):
    d = inputs(None, dims=dims, r=r, p=0.3, idx=61, noise=0.0, cap=cap, dtype=np.float32)
    st, _ = oracle_run(d, sweeps)
    g = gpu_run(F, d, sweeps, precision=precision)
    p_or = O.psnr(st.X, d["truth"])
    p_gpu = O.psnr(g["X"], d["truth"])
    print(f"{precision} {dims}: PSNR oracle {p_or:.4f} dB, GPU {p_gpu:.4f} dB, X rel err {rel(g['X'], st.X):.2e}")
    assert abs(p_gpu - p_or) <= (0.05 if precision == "tf32" else 0.1)


def test_tf32_deterministic(F):
    d = inputs(None, dims=(40, 33, 12), r=4, p=0.2, idx=62, noise=0.0, cap=None, dtype=np.float32)
    a = gpu_run(F, d, 4, precision="tf32")
    b = gpu_run(F, d, 4, precision="tf32")
    np.testing.assert_array_equal(a["X"], b["X"])

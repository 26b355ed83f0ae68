"""Full-size parity on the benchmark workloads, against the FP64 oracle.

256 x 256 x 31 x 8 (all FCTN ranks 6, Bernoulli(0.1)): 5 sweeps in the plain
order with reuse (the head-mode association on the GPU, Algorithm 2's pair
reuse in the oracle).  FP32: X and every A_k within 1e-4 (relative Frobenius
error).  TF32 and BF16 (tensor-core contractions): the per-result errors are
printed, and the PSNR against the generated truth stays within 0.05 dB of the
oracle's.

144 x 176 x 3 x 50 (ranks 6, 3 on the size-3 mode, Bernoulli(0.05)):
20 sweeps in the plain order, reuse on (head-mode association) and off
(merged tensors from scratch, Algorithm 1): both within 1e-4 of the oracle.

The oracle sweeps of the first workload take several seconds each on the
host; each oracle run happens once per module.
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


@pytest.fixture(scope="module")
def c4():
    d = inputs("c4", dtype=np.float32)
    st, hist = oracle_run(d, 5, policy="plain")
    return d, st, hist


@pytest.fixture(scope="module")
def c3():
    d = inputs("c3", dtype=np.float32)
    st, hist = oracle_run(d, 20, policy="plain")
    return d, st, hist


def _errors(g, st):
    return [rel(g["X"], st.X)] + [rel(a, b) for a, b in zip(g["factors"], st.factors)]


def test_c4_fp32_within_1e4_of_oracle(F, c4):
    d, st, hist = c4
    g = gpu_run(F, d, 5, precision="fp32", policy="plain")
    errs = _errors(g, st)
    print("256x256x31x8 fp32, 5 sweeps: rel err X, A_1..A_4 =", ["%.2e" % e for e in errs])
    assert all(e <= 1e-4 for e in errs), errs
    assert abs(g["stats"]["objective"] - hist[-1]["objective"]) <= 1e-4 * abs(hist[-1]["objective"])


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_c4_reduced_precision_psnr_within_005_db(F, c4, precision):
    d, st, _ = c4
    g = gpu_run(F, d, 5, precision=precision, policy="plain")
    errs = _errors(g, st)
    p_or, p_gpu = O.psnr(st.X, d["truth"]), O.psnr(g["X"], d["truth"])
    print(f"256x256x31x8 {precision}, 5 sweeps: rel err X, A_1..A_4 =", ["%.2e" % e for e in errs],
          f"PSNR oracle {p_or:.4f} dB, GPU {p_gpu:.4f} dB")
    assert g["stats"]["status"] == 0
    assert abs(p_gpu - p_or) <= 0.05


@pytest.mark.parametrize("reuse", [True, False])
def test_c3_reuse_on_off_within_1e4_of_oracle(F, c3, reuse):
    d, st, _ = c3
    g = gpu_run(F, d, 20, precision="fp32", reuse=reuse, policy="plain")
    errs = _errors(g, st)
    print(f"144x176x3x50 fp32 reuse={reuse}, 20 sweeps: rel err X, A_1..A_4 =", ["%.2e" % e for e in errs])
    assert all(e <= 1e-4 for e in errs), errs

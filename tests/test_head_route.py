"""The head-mode association of a sweep (FP32 / TF32 / BF16 with reuse and
the plain order 1..N) against the FP64 oracle and against the merged-tensor
route of the same sweep order.

The head route evaluates the products of Eq. 5 in another association: the
merged tensor M_1 of every factor but the first serves the first factor's
right-hand side and the reconstruction F of Eq. 10, Z = X_(1)^T A_(1) serves
every other right-hand side, and every Gram M_k M_k^T comes from the Grams of
the factors.  Exact arithmetic gives the oracle's iterates; FP32 stays within
1e-4 (relative Frobenius error per result) after the fixed sweeps.
"""
import numpy as np
import pytest

from tests.util import gpu_run, inputs, oracle_run, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2510_22506_gb300 import fctn
    return fctn


CASES = [
    ((48, 40, 9), 4, None, 10),          # N = 3, ragged against every tile
    ((13, 7, 3, 5), 3, (3, 2), 8),       # N = 4, ragged, capped bonds of the size-3 mode
    ((30, 24, 3, 7), 3, (3, 2), 8),
    ((5, 4, 3, 4, 3), 2, None, 6),       # N = 5
    ((64, 33, 17), 8, None, 6),          # s = 64, several K chunks
    ((24, 20, 9, 8), 6, None, 6),        # N = 4, s = 216: the large eigensolver
]


@pytest.mark.parametrize("solve", ["chol", "eig"])
@pytest.mark.parametrize("dims,r,cap,sweeps", CASES)
def test_head_route_fp32_matches_oracle(F, dims, r, cap, sweeps, solve):
    d = inputs(None, dims=dims, r=r, p=0.3, idx=70, noise=0.0, cap=cap, dtype=np.float32)
    st, hist = oracle_run(d, sweeps, reuse=True, policy="plain")
    g = gpu_run(F, d, sweeps, precision="fp32", reuse=True, policy="plain", solve_method=solve)
    e = rel(g["X"], st.X)
    assert e <= 1e-4, e
    for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
        assert rel(a, b) <= 1e-4, (k, rel(a, b))
    assert abs(g["stats"]["objective"] - hist[-1]["objective"]) <= 1e-4 * abs(hist[-1]["objective"])


@pytest.mark.parametrize("dims,r,cap", [((30, 24, 3, 7), 3, (3, 2)), ((20, 16, 12), 5, None)])
def test_head_route_agrees_with_merged_route(F, dims, r, cap):
    """Same order, reuse on (head route) and off (merged tensors from scratch):
    the two differ only by association."""
    d = inputs(None, dims=dims, r=r, p=0.25, idx=71, noise=0.0, cap=cap, dtype=np.float32)
    a = gpu_run(F, d, 6, precision="fp32", reuse=True, policy="plain")
    b = gpu_run(F, d, 6, precision="fp32", reuse=False, policy="plain")
    assert rel(a["X"], b["X"]) <= 1e-4
    for x, y in zip(a["factors"], b["factors"]):
        assert rel(x, y) <= 1e-4


def test_head_route_graph_and_eager_identical(F):
    """Graph-captured sweeps launch the same kernels as eager ones."""
    d = inputs(None, dims=(30, 24, 3, 7), r=3, p=0.3, idx=72, noise=0.0, cap=(3, 2), dtype=np.float32)
    p = F.make_params(d["dims"], d["R"], precision="fp32", reuse=True, order_policy="plain")
    out = []
    for graphs in (True, False):
        h = F.fctn_create(p)
        try:
            F.fctn_set_graphs(h, graphs)
            F.fctn_set_data(h, np.ascontiguousarray(d["Y"]), np.ascontiguousarray(d["mask"].astype(np.uint8)))
            F.fctn_set_factors(h, [np.ascontiguousarray(a) for a in d["init"]])
            F.fctn_pam_sweep(h, 5)
            X = np.empty(d["dims"], dtype=np.float32)
            F.fctn_get_X(h, X)
            out.append(X)
        finally:
            F.fctn_destroy(h)
    np.testing.assert_array_equal(out[0], out[1])


# ---- tensor-core products (TF32 / BF16) of the head route -----------------
TC_CASES = [((48, 40, 9), 4, None), ((32, 24, 3, 7), 3, (3, 2)), ((24, 20, 9, 8), 6, None),
            ((136, 40, 12), 5, None)]   # I_1 = 136: two row tiles of 128 in X_(1) M_1^T


@pytest.mark.parametrize("dims,r,cap", TC_CASES)
@pytest.mark.parametrize("precision,tol", [("tf32", 3e-3), ("bf16", 3e-2)])
def test_head_route_tensor_core_one_sweep_close_to_fp32(F, dims, r, cap, precision, tol):
    """One sweep: the TMA / tcgen05 products (X_(1) M_1^T, X_(1)^T A_(1),
    M_1^T A_(1)^T with the X update) against the FP32 CUDA-core products."""
    d = inputs(None, dims=dims, r=r, p=0.3, idx=73, noise=0.0, cap=cap, dtype=np.float32)
    a = gpu_run(F, d, 1, precision="fp32", policy="plain")
    b = gpu_run(F, d, 1, precision=precision, policy="plain")
    assert b["stats"]["status"] == 0
    assert rel(b["X"], a["X"]) <= tol, rel(b["X"], a["X"])
    for x, y in zip(b["factors"], a["factors"]):
        assert rel(x, y) <= 10 * tol, rel(x, y)


@pytest.mark.parametrize("dims,r,cap,sweeps", [((48, 40, 9), 4, None, 60), ((32, 24, 3, 7), 3, (3, 2), 50)])
@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_head_route_tensor_core_psnr_within_005_db(F, dims, r, cap, sweeps, precision):
    """Pure tensor-core sweeps (no FP32 finish) on small shapes: TF32 within
    0.05 dB of the oracle's PSNR; BF16 (8 mantissa bits, 4e-3 relative per
    operand, with few terms per product here) within 0.1 dB.  The 0.05 dB bar
    for both on the 256x256x31x8 workload is tests/test_workloads_full.py."""
    from oracle import fctn_oracle as O
    d = inputs(None, dims=dims, r=r, p=0.3, idx=74, noise=0.0, cap=cap, dtype=np.float32)
    st, _ = oracle_run(d, sweeps, policy="plain")
    g = gpu_run(F, d, sweeps, precision=precision, policy="plain")
    p_or, p_gpu = O.psnr(st.X, d["truth"]), O.psnr(g["X"], d["truth"])
    print(f"{precision} {dims}: PSNR oracle {p_or:.4f} GPU {p_gpu:.4f}, X rel err {rel(g['X'], st.X):.2e}")
    assert abs(p_gpu - p_or) <= (0.05 if precision == "tf32" else 0.1)


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_mixed_precision_finishes_in_fp32(F, precision):
    """finish_fp32_at: tensor-core sweeps until rel_change <= 1e-3, FP32 sweeps
    after; fctn_complete then reaches rel_change <= 1e-4 and the completed
    tensor's PSNR matches the plain FP32 run's within 0.05 dB."""
    from oracle import fctn_oracle as O
    d = inputs(None, dims=(48, 40, 9), r=4, p=0.3, idx=75, noise=0.0, cap=None, dtype=np.float32)
    out = {}
    for prec, fin in (("fp32", 0.0), (precision, 1e-3)):
        p = F.make_params(d["dims"], d["R"], precision=prec, order_policy="plain", finish_fp32_at=fin)
        h = F.fctn_create(p)
        try:
            F.fctn_set_data(h, np.ascontiguousarray(d["Y"]), np.ascontiguousarray(d["mask"].astype(np.uint8)))
            F.fctn_set_factors(h, [np.ascontiguousarray(a) for a in d["init"]])
            X = np.empty(d["dims"], dtype=np.float32)
            st = F.fctn_complete(h, 1e-4, 400, X)
        finally:
            F.fctn_destroy(h)
        out[prec] = (st, O.psnr(X, d["truth"]))
    st, ps = out[precision]
    assert st["converged"] and st["rel_change"] <= 1e-4, st
    assert abs(ps - out["fp32"][1]) <= 0.05


# ---- every launch shape the autotuner may pick keeps parity ----------------
@pytest.fixture(scope="module")
def tile_case():
    d = inputs(None, dims=(136, 40, 12), r=5, p=0.3, idx=76, noise=0.0, cap=None, dtype=np.float32)
    st, _ = oracle_run(d, 6, policy="plain")
    return d, st


@pytest.mark.parametrize("code", [0, 1, 2, 4, 6, 8, 16, 24, 32, 64, 96, 128, 136, 160])
@pytest.mark.parametrize("precision", ["fp32", "tf32"])
def test_tile_codes_keep_parity(F, tile_case, code, precision):
    """Tile codes change only launch shapes and summation orders: FP32 stays
    within 1e-4 of the oracle, TF32 within 3e-3 (X) after 6 sweeps."""
    d, st = tile_case
    g = gpu_run(F, d, 6, precision=precision, policy="plain", tile_code=code)
    tol = 1e-4 if precision == "fp32" else 3e-3
    assert g["stats"]["status"] == 0
    assert rel(g["X"], st.X) <= tol, (code, rel(g["X"], st.X))


def test_tile_autotuner_picks_a_candidate(F):
    d = inputs(None, dims=(48, 40, 9), r=4, p=0.3, idx=77, noise=0.0, cap=None, dtype=np.float32)
    p = F.make_params(d["dims"], d["R"], precision="tf32", order_policy="plain")
    best, ms = F.fctn_autotune_tiles(p, np.ascontiguousarray(d["Y"]), d["mask"].astype(np.uint8),
                                     [np.ascontiguousarray(a) for a in d["init"]], sweeps=2)
    assert best in F.TILE_CANDIDATES and set(ms) == set(F.TILE_CANDIDATES)
    assert all(v > 0 for v in ms.values()) and ms[best] == min(ms.values())

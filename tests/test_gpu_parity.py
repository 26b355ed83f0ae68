"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative Frobenius error, per result):
  FP64 path: X and every A_k <= 1e-9 after 20 sweeps (30x30x10, R = 3).
  FP32 path: X and every A_k <= 1e-4 after the fixed sweeps.
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


# ---- the FCTN contraction (FCTN format) ---------------------------------
@pytest.mark.parametrize("dims,r", [((30, 30, 10), 3), ((7, 5, 3, 4), 2), ((9, 11), 4), ((1, 2, 3), 2),
                                    ((4, 3, 2, 3, 2), 2)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_contract_matches_oracle(F, dims, r, precision, tol):
    N = len(dims)
    R = np.full((N, N), r)
    rng = np.random.default_rng(7)
    fs = [rng.standard_normal(O.factor_shape(dims, R, k)) for k in range(N)]
    p = F.make_params(dims, R, precision=precision, reuse=False)
    dt = F.elem_dtype(p)
    fs_c = [np.ascontiguousarray(a.astype(dt)) for a in fs]
    h = F.fctn_create(p)
    try:
        F.fctn_set_factors(h, fs_c)
        out = np.empty(dims, dtype=dt)
        F.fctn_contract(h, out)
        back = []
        for k, shp in enumerate(F.factor_shapes(p)):
            a = np.empty(shp, dtype=dt)
            F.fctn_get_factor(h, k, a)
            back.append(a)
    finally:
        F.fctn_destroy(h)
    ref = O.fctn_full([a.astype(np.float64) for a in fs_c])
    assert rel(out, ref) <= tol
    for a, b in zip(back, fs_c):
        np.testing.assert_array_equal(a, b)


# ---- FP64 path, 30x30x10 R=3, 20 sweeps ---------------------------------
@pytest.mark.parametrize("reuse", [True, False])
@pytest.mark.parametrize("sign", ["psd", "printed"])
def test_fp64_c1_matches_oracle(F, reuse, sign):
    d = inputs("c1")
    st, hist = oracle_run(d, 20, reuse=reuse, sign=sign)
    g = gpu_run(F, d, 20, precision="fp64", reuse=reuse, sign=sign)
    assert rel(g["X"], st.X) <= 1e-9, rel(g["X"], st.X)
    for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
        assert rel(a, b) <= 1e-9, (k, rel(a, b))
    assert g["stats"]["t"] == 20
    assert abs(g["stats"]["rel_change"] - hist[-1]["rel"]) <= 1e-9 * max(1.0, hist[-1]["rel"])
    assert abs(g["stats"]["objective"] - hist[-1]["objective"]) <= 1e-9 * abs(hist[-1]["objective"])


def test_fp64_fourth_order_ragged_alternate_order(F):
    """N = 4 with a ragged shape (no size a multiple of a tile) and pair reuse."""
    d = inputs(None, dims=(13, 7, 3, 5), r=3, p=0.3, idx=40, noise=0.0, cap=(3, 2))
    for reuse in (True, False):
        st, _ = oracle_run(d, 8, reuse=reuse, policy="alternate")
        g = gpu_run(F, d, 8, precision="fp64", reuse=reuse, policy="alternate")
        assert rel(g["X"], st.X) <= 1e-9
        for a, b in zip(g["factors"], st.factors):
            assert rel(a, b) <= 1e-9


@pytest.mark.parametrize("dims,r", [((5, 4, 3, 4, 3), 2), ((3, 4, 2, 3, 2, 3), 2)])
def test_fp64_order_5_and_6_half_reuse(F, dims, r):
    """N >= 5: half-network intermediates (reuse) and the alternating order."""
    d = inputs(None, dims=dims, r=r, p=0.4, idx=49, noise=0.0, cap=None)
    for reuse in (True, False):
        st, _ = oracle_run(d, 6, reuse=reuse, policy="alternate")
        g = gpu_run(F, d, 6, precision="fp64", reuse=reuse, policy="alternate")
        assert rel(g["X"], st.X) <= 1e-9, (reuse, rel(g["X"], st.X))
        for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
            assert rel(a, b) <= 1e-9, (reuse, k, rel(a, b))


def test_fp32_order_5_half_reuse(F):
    d = inputs(None, dims=(9, 8, 6, 7, 5), r=2, p=0.3, idx=50, noise=0.0, cap=None, dtype=np.float32)
    st, _ = oracle_run(d, 8, reuse=True, policy="alternate")
    g = gpu_run(F, d, 8, precision="fp32", reuse=True, policy="alternate")
    assert rel(g["X"], st.X) <= 1e-4, rel(g["X"], st.X)
    for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
        assert rel(a, b) <= 1e-4, (k, rel(a, b))


def test_fp64_second_order(F):
    d = inputs(None, dims=(37, 29), r=5, p=0.4, idx=41, noise=0.0, cap=None)
    st, _ = oracle_run(d, 10)
    g = gpu_run(F, d, 10, precision="fp64")
    assert rel(g["X"], st.X) <= 1e-9
    for a, b in zip(g["factors"], st.factors):
        assert rel(a, b) <= 1e-9


def test_fp64_tiny_modes(F):
    """Modes of size 1 and 2, where the Laplacian stencil entries coincide."""
    d = inputs(None, dims=(1, 2, 9), r=2, p=0.6, idx=42, noise=0.0, cap=None)
    st, _ = oracle_run(d, 6)
    g = gpu_run(F, d, 6, precision="fp64")
    assert rel(g["X"], st.X) <= 1e-9
    for a, b in zip(g["factors"], st.factors):
        assert rel(a, b) <= 1e-9


def test_reuse_on_off_identical_order_fp64(F):
    d = inputs("c1")
    a = gpu_run(F, d, 20, precision="fp64", reuse=True, policy="plain")
    b = gpu_run(F, d, 20, precision="fp64", reuse=False, policy="plain")
    assert rel(a["X"], b["X"]) <= 1e-12


def test_deterministic_bytes(F):
    d = inputs(None, dims=(40, 33, 12), r=4, p=0.2, idx=43, noise=0.0, cap=None)
    a = gpu_run(F, d, 5, precision="fp32")
    b = gpu_run(F, d, 5, precision="fp32")
    np.testing.assert_array_equal(a["X"], b["X"])
    for x, y in zip(a["factors"], b["factors"]):
        np.testing.assert_array_equal(x, y)


def test_singular_system_reported(F):
    d = inputs("c1")
    with pytest.raises(F.FctnError) as ei:
        gpu_run(F, d, 2, precision="fp64", sign="printed", lam=10.0)
    assert ei.value.code == F.FCTN_E_SINGULAR


def test_nothing_observed_is_nonfinite(F):
    d = inputs("c1")
    d["mask"] = np.zeros_like(d["mask"])
    d["Y"] = np.zeros_like(d["Y"])
    with pytest.raises(F.FctnError) as ei:
        gpu_run(F, d, 1, precision="fp64")
    assert ei.value.code == F.FCTN_E_NONFINITE


# ---- the Gram of Eq. 5 from the operand Grams of the pair form -------------
@pytest.mark.parametrize("dims,r,cap,reuse", [((30, 30, 10), 3, None, True), ((30, 30, 10), 3, None, False),
                                              ((13, 7, 3, 5), 3, (3, 2), True), ((13, 7, 3, 5), 3, (3, 2), False),
                                              ((37, 29), 5, None, True), ((2, 9, 1), 2, None, True)])
def test_fp64_factored_gram_matches_oracle(F, dims, r, cap, reuse):
    """FCTN_GRAM_FACTORED: G_k = sum over the contracted pair of (L L^T) o (R R^T) blocks."""
    d = inputs(None, dims=dims, r=r, p=0.3, idx=45, noise=0.0, cap=cap)
    st, _ = oracle_run(d, 8, reuse=reuse)
    g = gpu_run(F, d, 8, precision="fp64", reuse=reuse, gram_mode="factored")
    assert rel(g["X"], st.X) <= 1e-9, rel(g["X"], st.X)
    for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
        assert rel(a, b) <= 1e-9, (k, rel(a, b))


def test_fp32_factored_and_direct_gram(F):
    d = inputs(None, dims=(48, 40, 9), r=4, p=0.2, idx=44, noise=0.0, cap=None, dtype=np.float32)
    st, _ = oracle_run(d, 10)
    for mode in ("factored", "direct"):
        g = gpu_run(F, d, 10, precision="fp32", gram_mode=mode)
        assert rel(g["X"], st.X) <= 1e-4, (mode, rel(g["X"], st.X))
        for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
            assert rel(a, b) <= 1e-4, (mode, k, rel(a, b))


@pytest.mark.parametrize("r", [6, 11, 12, 14])
def test_fp32_eigensolver_sizes(F, r):
    """Gram sizes s = r^2 across the FP32 eigensolver's configurations: 36
    (an odd number of 8 x 8 subproblems, one half warp idle), 121 (the
    largest case with B and V^T on chip, 16 subproblems), 144 and 196 (B on
    chip, rotation blocks recorded and applied to V by many CTAs)."""
    d = inputs(None, dims=(40, 36, 12), r=r, p=0.3, idx=46, noise=0.0, cap=None, dtype=np.float32)
    st, _ = oracle_run(d, 10)
    g = gpu_run(F, d, 10, precision="fp32", solve_method="eig")
    assert rel(g["X"], st.X) <= 1e-4, rel(g["X"], st.X)
    for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
        assert rel(a, b) <= 1e-4, (k, rel(a, b))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_gram_wider_than_a_solve_block(F, precision, tol):
    """s = 17^2 = 289 columns exceed the solve kernels' 256 threads: every
    column group of Q^T R and Q W must be formed (and the eigensolver takes
    its global-memory one-sided form).  P_k >= s for every k, so that the
    Grams have full rank (with rank-deficient Grams and rho = 0.1 the FP32
    Gram's rounding alone moves the solution by ~1e-3)."""
    d = inputs(None, dims=(40, 36, 30), r=17, p=0.4, idx=47, noise=0.0, cap=None,
               dtype=np.float64 if precision == "fp64" else np.float32)
    st, _ = oracle_run(d, 5)
    g = gpu_run(F, d, 5, precision=precision)
    assert rel(g["X"], st.X) <= tol, rel(g["X"], st.X)
    for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
        assert rel(a, b) <= tol, (k, rel(a, b))


def test_fp32_autotuned_launch_shape(F):
    """The autotuner times its candidates and returns one of them; every
    launch shape of the right-hand-side kernel keeps parity with the oracle."""
    d = inputs(None, dims=(48, 40, 9), r=4, p=0.2, idx=44, noise=0.0, cap=None, dtype=np.float32)
    p = F.make_params(d["dims"], d["R"], precision="fp32")
    best, ms = F.fctn_autotune(p, d["Y"], d["mask"].astype(np.uint8), d["init"], candidates=(8, 96, 600), sweeps=2)
    assert best in (8, 96, 600)
    assert all(v > 0 for v in ms.values()), ms
    assert ms[best] == min(ms.values())
    st, _ = oracle_run(d, 10)
    for c in (8, 600):
        g = gpu_run(F, d, 10, precision="fp32", rhs_ctas=c)
        assert rel(g["X"], st.X) <= 1e-4, (c, rel(g["X"], st.X))
        for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
            assert rel(a, b) <= 1e-4, (c, k, rel(a, b))


# ---- FP32 path ------------------------------------------------------------
def test_fp32_small_matches_oracle(F):
    d = inputs(None, dims=(48, 40, 9), r=4, p=0.2, idx=44, noise=0.0, cap=None, dtype=np.float32)
    st, _ = oracle_run(d, 30)
    g = gpu_run(F, d, 30, precision="fp32")
    assert rel(g["X"], st.X) <= 1e-4, rel(g["X"], st.X)
    for k, (a, b) in enumerate(zip(g["factors"], st.factors)):
        assert rel(a, b) <= 1e-4, (k, rel(a, b))


@pytest.mark.slow
def test_fp32_c2_full_size_100_sweeps(F):
    """256x256x31, R = 8, SR 0.1, noise 0.01: plain FP32 vs the FP64 oracle."""
    d = inputs("c2", dtype=np.float32)
    st, _ = oracle_run(d, 100)
    g = gpu_run(F, d, 100, precision="fp32")
    errs = [rel(g["X"], st.X)] + [rel(a, b) for a, b in zip(g["factors"], st.factors)]
    print("c2 fp32 errors X, A_k:", errs)
    assert errs[0] <= 1e-4, errs
    assert all(e <= 1e-4 for e in errs[1:]), errs


def test_graphs_on_off_identical_and_profiler(F):
    d = inputs(None, dims=(40, 36, 7, 5), r=3, p=0.2, idx=45, noise=0.0, cap=(7, 2), dtype=np.float32)
    outs = []
    for graphs in (True, False):
        p = F.make_params(d["dims"], d["R"], precision="fp32", reuse=True, order_policy="alternate")
        h = F.fctn_create(p)
        try:
            F.fctn_set_graphs(h, graphs)
            F.fctn_set_data(h, d["Y"], d["mask"].astype(np.uint8))
            F.fctn_set_factors(h, d["init"])
            F.fctn_pam_sweep(h, 6)
            F.fctn_profile(h, "xupdate")
            F.fctn_pam_sweep(h, 2)
            pr = F.fctn_profile_read(h)
            F.fctn_profile(h, None)
            assert pr["launches"] == 2 and pr["ms"] > 0 and pr["bytes"] > 0
            X = np.empty(d["dims"], dtype=np.float32)
            F.fctn_get_X(h, X)
            outs.append(X)
        finally:
            F.fctn_destroy(h)
    np.testing.assert_array_equal(outs[0], outs[1])


def test_device_pointer_path_and_stream(F):
    torch = pytest.importorskip("torch")
    d = inputs("c1")
    st, _ = oracle_run(d, 5)
    p = F.make_params(d["dims"], d["R"], precision="fp64")
    s = torch.cuda.Stream()
    h = F.fctn_create(p, s)
    try:
        F.fctn_set_data(h, torch.from_numpy(d["Y"]).cuda(), torch.from_numpy(d["mask"].astype(np.uint8)).cuda())
        F.fctn_set_factors(h, [torch.from_numpy(a).cuda() for a in d["init"]])
        F.fctn_pam_sweep(h, 5)
        X = torch.empty(d["dims"], dtype=torch.float64, device="cuda")
        F.fctn_get_X(h, X)
        s.synchronize()
    finally:
        F.fctn_destroy(h)
    assert rel(X.cpu().numpy(), st.X) <= 1e-9


@pytest.mark.parametrize("dims,r,cap", [((30, 30, 10), 3, None), ((13, 7, 3, 5), 3, (3, 2))])
def test_fp64_asymmetric_extrapolation_matches_oracle(F, dims, r, cap):
    """The multi-temporal variant (Sec. 4.3): alpha = beta = 0.5 after every factor update."""
    d = inputs(None, dims=dims, r=r, p=0.3, idx=46, noise=0.0, cap=cap)
    st, _ = oracle_run(d, 15, extrapolation=(0.5, 0.5))
    g = gpu_run(F, d, 15, precision="fp64", extrapolation=(0.5, 0.5))
    assert rel(g["X"], st.X) <= 1e-9, rel(g["X"], st.X)
    for a, b in zip(g["factors"], st.factors):
        assert rel(a, b) <= 1e-9


# ---- the eigensolver's sweep cap is reported, not hidden ------------------
@pytest.mark.parametrize("precision,dims,r", [("fp32", (40, 36, 9), 5), ("fp32", (12, 10, 6, 5), 6),
                                              ("fp64", (30, 30, 10), 3)])
def test_eig_sweep_cap_is_reported(F, precision, dims, r):
    """A cap of one Jacobi sweep on a cold Gram (first PAM sweep, no warm
    start) cannot meet the stop test: every factor reports the cap in
    fctn_stats.eig_capped while the sweep itself still completes (FCTN_OK,
    finite values).  The default cap is not reached on the same inputs."""
    dt = np.float64 if precision == "fp64" else np.float32
    d = inputs(None, dims=dims, r=r, p=0.3, idx=63, noise=0.0, cap=None, dtype=dt)
    g = gpu_run(F, d, 1, precision=precision, eig_max_sweeps=1, solve_method="eig")
    st = g["stats"]
    assert st["status"] == 0
    assert st["eig_capped"] == len(dims), st
    assert st["eig_sweeps"] == 1
    assert np.isfinite(g["X"]).all()
    g2 = gpu_run(F, d, 1, precision=precision, solve_method="eig")
    assert g2["stats"]["eig_capped"] == 0, g2["stats"]
    assert g2["stats"]["eig_sweeps"] > 1

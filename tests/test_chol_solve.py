"""The shifted-Cholesky solve of Eq. 5 (FCTN_SOLVE_CHOL).

In the real eigenbasis Q of the circulant L_k (closed form), Eq. 6 is block
diagonal: row i of W = Q^T A solves W_i (G + (lam mu_i + rho) I) = (Q^T Y)_i,
and the cos / sin columns of one frequency share mu_i.  The CPU test checks
this reading against the oracle's Eq. 8 solve; the GPU tests compare the
Cholesky path with the oracle across the panel counts of the factorization
(s from 4 to 256), single-row groups (I = 1, 2, odd I) and the singular case.
"""
import numpy as np
import pytest

from oracle import fctn_oracle as O
from tests.util import gpu_run, inputs, oracle_run, rel


def _basis(I):
    """Real orthonormal eigenbasis of a symmetric circulant and its frequencies:
    column 0 constant; columns 2j - 1, 2j = cos, sin of frequency j; for even
    I the last column alternates in sign (frequency I / 2)."""
    n = np.arange(I)
    Q = np.empty((I, I))
    freq = np.empty(I, dtype=int)
    Q[:, 0] = 1.0 / np.sqrt(I)
    freq[0] = 0
    for col in range(1, I):
        if I % 2 == 0 and col == I - 1:
            Q[:, col] = (-1.0) ** n / np.sqrt(I)
            freq[col] = I // 2
        else:
            j = (col + 1) // 2
            f = np.cos if col % 2 == 1 else np.sin
            Q[:, col] = np.sqrt(2.0 / I) * f(2 * np.pi * j * n / I)
            freq[col] = j
    return Q, freq


@pytest.mark.parametrize("I", [1, 2, 3, 8, 31, 32])
@pytest.mark.parametrize("sign,lam", [("psd", 0.01), ("psd", 0.4), ("printed", 0.01)])
def test_row_decoupled_shifted_solves_equal_eq8(I, sign, lam):
    rng = np.random.default_rng(100 + I)
    s, delta, rho = 20, 0.5, 0.1
    M = rng.standard_normal((s, 3 * s))
    G = M @ M.T / (3 * s)
    Y = rng.standard_normal((I, s))
    L = O.laplacian(I, delta, sign)
    A8 = O.solve_factor(G, Y, L, lam, rho)
    Q, freq = _basis(I)
    np.testing.assert_allclose(Q.T @ Q, np.eye(I), atol=1e-13)
    sg = -1.0 if sign == "printed" else 1.0
    mu = sg * (2.0 + delta - 2.0 * np.cos(2 * np.pi * freq / I))
    np.testing.assert_allclose(Q.T @ L @ Q, np.diag(mu), atol=1e-12)
    Yt = Q.T @ Y
    W = np.empty_like(Yt)
    groups = {}
    for i in range(I):
        groups.setdefault(freq[i], []).append(i)
    assert len(groups) == I // 2 + 1
    for j, rows in groups.items():
        assert rows == ([0] if j == 0 else [I - 1] if 2 * j == I else [2 * j - 1, 2 * j])
        c = lam * mu[rows[0]] + rho
        Lc = np.linalg.cholesky(G + c * np.eye(s))
        for i in rows:
            z = np.linalg.solve(Lc, Yt[i])
            W[i] = np.linalg.solve(Lc.T, z)
    A = Q @ W
    assert rel(A, A8) <= 1e-12
    # and it solves Eq. 5
    R = A @ G + lam * L @ A + rho * A - Y
    assert np.linalg.norm(R) <= 1e-11 * np.linalg.norm(Y)


@pytest.fixture(scope="module")
def F():
    from paper_2510_22506_gb300 import fctn
    return fctn


CASES = [
    ((48, 40, 9), 4, None),       # s = 16: one panel
    ((40, 36, 12), 6, None),      # s = 36: two panels, ragged
    ((40, 36, 12), 11, None),     # s = 121
    ((40, 36, 30), 14, None),     # s = 196
    ((10, 9, 8, 7), 6, None),     # s = 216: seven panels, every factor
    ((40, 36, 30), 16, None),     # s = 256: eight full panels
    ((1, 2, 3), 2, None),         # I = 1 and 2: single-row groups
    ((13, 7, 3, 5), 3, (3, 2)),   # odd I, unequal ranks
]


@pytest.mark.gpu
@pytest.mark.parametrize("dims,r,cap", CASES)
def test_fp32_cholesky_solve_matches_oracle(F, dims, r, cap):
    d = inputs(None, dims=dims, r=r, p=0.3, idx=72, noise=0.0, cap=cap, dtype=np.float32)
    st, _ = oracle_run(d, 8)
    g = gpu_run(F, d, 8, precision="fp32", solve_method="chol")
    errs = [rel(g["X"], st.X)] + [rel(a, b) for a, b in zip(g["factors"], st.factors)]
    assert g["stats"]["status"] == 0
    assert g["stats"]["eig_sweeps"] == 0
    assert all(e <= 1e-4 for e in errs), errs


@pytest.mark.gpu
@pytest.mark.parametrize("refine", [0, 1, 2])
def test_fp32_cholesky_and_eigen_solves_agree(F, refine):
    """Both solves of Eq. 5 reach the oracle; with refinement they agree
    with each other far below the parity bound."""
    d = inputs(None, dims=(24, 20, 9, 8), r=6, p=0.3, idx=73, noise=0.0, cap=None, dtype=np.float32)
    st, _ = oracle_run(d, 6, policy="plain")
    a = gpu_run(F, d, 6, precision="fp32", policy="plain", solve_method="chol", refine_steps=refine)
    b = gpu_run(F, d, 6, precision="fp32", policy="plain", solve_method="eig", refine_steps=max(refine, 1))
    for g in (a, b):
        assert rel(g["X"], st.X) <= 1e-4
        for x, y in zip(g["factors"], st.factors):
            assert rel(x, y) <= 1e-4
    assert rel(a["X"], b["X"]) <= (1e-4 if refine == 0 else 2e-5)


@pytest.mark.gpu
@pytest.mark.parametrize("method", ["chol", "eig"])
def test_fp32_singular_system_reported(F, method):
    """The printed (negative definite) L_k with a large lam: G + c I is not
    positive definite for some shift, FCTN_E_SINGULAR from either solve."""
    d = inputs("c1", dtype=np.float32)
    with pytest.raises(F.FctnError) as ei:
        gpu_run(F, d, 2, precision="fp32", sign="printed", lam=10.0, solve_method=method)
    assert ei.value.code == F.FCTN_E_SINGULAR

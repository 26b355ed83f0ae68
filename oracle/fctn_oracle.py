"""FP64 CPU oracle for trace-regularized FCTN completion solved by PAM.

TEST INFRASTRUCTURE ONLY.  This module is imported by the test suite, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
product path (the CUDA library and its Python binding) never imports, calls or
links it, and it imports nothing from the product package.

It restates, in plain NumPy float64, what the paper (arXiv 2510.22506,
"Accelerated Tensor Completion via Trace-Regularized Fully-Connected Tensor
Network") computes, step by step and in the paper's order and notation:

* FCTN format (Sec. 1, the element-wise definition of an N-th order FCTN) and
  Property 1 (X_(k) = A_k(k) M_k), Definitions 1-3 (Sec. 2.2).
* The periodically modified negative Laplacian L_k (Sec. 3.1, below Eq. 1).
* Model (1)/(2) objective, the PAM scheme (3), the factor subproblem (4), its
  Sylvester normal equation (5), the eigen-route solution (7)-(9) and the
  closed-form X update (10) (Sec. 3.2).
* Algorithm 1 (PAM-FCTNLR, every merged tensor contracted from scratch) and
  Algorithm 2 (PAM-AFCTNLR, intermediate-tensor reuse and the permuted update
  order) (Sec. 3.2-3.3).
* The per-iteration operation counts of Tables 1 and 2 (Sec. 3.4), as a flop
  counter per cost centre.
* PSNR (Sec. 4).

Readings of passages the paper leaves open:

* Laplacian sign: the printed matrix (diagonal -2-delta, neighbours +1) is
  negative definite, while the text says the term penalises second-order
  variation and the convergence proof needs every diagonal entry of the
  transformed system to be >= rho.  Default ``sign="psd"`` uses the negated
  printed matrix (diagonal 2+delta, neighbours -1); ``sign="printed"`` keeps
  the literal one.  Small modes (I_k <= 2) add the stencil entries that fall
  on the same position.
* X^(1) = Y means X^(1) = P_Omega(Y) (unobserved entries 0).
* The loop of Algorithms 1/2 runs as a do-while: sweep, then test
  ||X^{t+1}-X^t||_F / ||X^t||_F <= tol or t == max_sweeps.
* The "unordered permutation" of Algorithm 2 (its figure is not printed) is
  ``"alternate"``: for N = 4, odd sweeps update (1,2,3,4) and even sweeps
  (3,4,1,2), so each sweep starts with the pair whose shared intermediate
  tensor is still valid (this reproduces the t >= 2 row of Table 1).  For
  N >= 5 the same with the halves (1..N/2) and (N/2+1..N) of the modes,
  whose intermediates are shared (Table 2's general-order reuse, whose
  scheme is not printed).  For N <= 3 the order stays (1..N).
* Eq. (8) is evaluated with the real orthonormal eigenbasis of the symmetric
  circulant L_k (numpy.linalg.eigh) in place of the complex DFT; the solution
  is the same.  The orientation of T is I_k x s_k with
  T_ij = lambda_k Lambda_i + Phi_j + rho.

The unfolding convention is internal: every merged tensor is built with
``numpy.tensordot`` over explicitly named bonds, its rows are the open bonds
r_{k,t} (t != k, ascending t, row-major) and its columns the physical indices
i_t (t != k, ascending t, row-major); A_k(k) and X_(k) use the same orders, so
Property 1 holds with plain matrix products.

Function-level parity status: every function below is pinned by a test in
``tests/test_oracle_pins.py`` except ``psnr`` (no printed value can be
reproduced without the paper's datasets), which is checked only against its
definition on a hand-made case.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ORDER_PLAIN = "plain"
ORDER_ALTERNATE = "alternate"

COST_CENTRES = ("M", "svd", "fft", "matmul", "cwm", "cwd", "X")


# --------------------------------------------------------------------------
# Index bookkeeping (FCTN format, Sec. 1; factor layout of Eq. 1)
# --------------------------------------------------------------------------

def rank(R, a, b):
    """FCTN rank R_{a,b} of the bond between modes a and b (symmetric)."""
    return int(R[min(a, b)][max(a, b)])


def factor_shape(dims, R, k):
    """Shape of A_k: (R_{1,k},...,R_{k-1,k}, I_k, R_{k,k+1},...,R_{k,N})."""
    N = len(dims)
    return tuple(dims[k] if t == k else rank(R, k, t) for t in range(N))


def s_k(dims, R, k):
    """s_k = prod_{t != k} R_{k,t} (Eq. 6)."""
    return int(np.prod([rank(R, k, t) for t in range(len(dims)) if t != k], dtype=np.int64))


def _mode_label(t):
    return ("i", t)


def _bond_label(a, b):
    return ("r", min(a, b), max(a, b))


def _factor_labels(N, k):
    return [_mode_label(k) if t == k else _bond_label(k, t) for t in range(N)]


@dataclass
class FlopCounter:
    """Operation counts per cost centre of Tables 1 and 2.

    "M": contractions that form merged tensors M_k (and shared pair
    intermediates), 2 x (output size) x (contracted size) per contraction.
    "matmul": Gram M_k M_k^T (2 s_k^2 P_k) and right-hand side X_(k) M_k^T
    (2 I_k s_k P_k).  "X": contractions that form FCTN(A) for the X update.
    "svd", "fft", "cwm", "cwd": the conventions of Table 1 per factor update:
    (4/3) s_k^3, 5 (I_k^2 + I_k s_k) log2 I_k, I_k s_k, I_k s_k.
    """
    counts: dict = field(default_factory=lambda: {c: 0.0 for c in COST_CENTRES})

    def add(self, centre, n):
        self.counts[centre] += float(n)


def _contract(x, xl, y, yl, counter=None, centre=None):
    """Contract two labelled tensors over every label they share (Def. 3).

    Returns (z, zl).  Adds 2 * size(z) * prod(shared extents) to ``counter``.
    """
    shared = [l for l in xl if l in yl]
    ax = [xl.index(l) for l in shared]
    ay = [yl.index(l) for l in shared]
    z = np.tensordot(x, y, axes=(ax, ay))
    zl = [l for l in xl if l not in shared] + [l for l in yl if l not in shared]
    if counter is not None:
        csize = int(np.prod([x.shape[a] for a in ax], dtype=np.int64)) if ax else 1
        counter.add(centre, 2 * z.size * csize)
    return z, zl


def _to_order(z, zl, order):
    return np.transpose(z, [zl.index(l) for l in order]), list(order)


def merged_labels(N, k):
    """Canonical axis order of M_k: open bonds r_{k,t}, then modes i_t (t != k)."""
    others = [t for t in range(N) if t != k]
    return [_bond_label(k, t) for t in others] + [_mode_label(t) for t in others]


# --------------------------------------------------------------------------
# FCTN contraction (Sec. 1) and merged tensors (Property 1)
# --------------------------------------------------------------------------

def fctn_full(factors, counter=None, centre="X"):
    """FCTN({A_k}) by contracting the factors in ascending order (Algorithm 1).

    The k-th step adds A_k to the running product; with equal sizes its cost
    is 2 I^K R^{K(N-K)+K-1}, the terms summed in Table 2 ("Computing X").
    """
    N = len(factors)
    cur, cl = factors[0], _factor_labels(N, 0)
    for k in range(1, N):
        cur, cl = _contract(cur, cl, factors[k], _factor_labels(N, k), counter, centre)
    out, _ = _to_order(cur, cl, [_mode_label(t) for t in range(N)])
    return np.ascontiguousarray(out)


def merged_sequential(factors, k, counter=None):
    """M_k = FCTN({A_t}_{t != k}) contracted from scratch in ascending order.

    This is the merged-tensor step of Algorithm 1 (cost term "Computing M_k"
    of Tables 1-2).
    Returns the tensor in canonical order (see ``merged_labels``).
    """
    N = len(factors)
    others = [t for t in range(N) if t != k]
    cur, cl = factors[others[0]], _factor_labels(N, others[0])
    for t in others[1:]:
        cur, cl = _contract(cur, cl, factors[t], _factor_labels(N, t), counter, "M")
    out, _ = _to_order(cur, cl, merged_labels(N, k))
    return np.ascontiguousarray(out)


def pair_of(N, k):
    """For N = 4: the pair (c, d) whose intermediate M_k reuses, and k's partner b.

    M_1, M_2 share the contraction of A_3 and A_4; M_3, M_4 share that of A_1
    and A_2 (Sec. 3.3, the shared intermediates of Figs. 2-3).
    """
    if N != 4:
        raise ValueError("pair sharing is defined for N = 4")
    if k in (0, 1):
        return (2, 3), 1 - k
    return (0, 1), 5 - k


def pair_intermediate(factors, c, d, counter=None):
    """T_cd = A_c x_{R_cd} A_d: the intermediate shared by two merged tensors."""
    N = len(factors)
    return _contract(factors[c], _factor_labels(N, c), factors[d], _factor_labels(N, d), counter, "M")


def merged_from_pair(factors, k, T, Tl, counter=None):
    """M_k = A_b x T_cd over the bonds (b,c), (b,d) (reuse path of Algorithm 2)."""
    N = len(factors)
    _, b = pair_of(N, k)
    cur, cl = _contract(factors[b], _factor_labels(N, b), T, Tl, counter, "M")
    out, _ = _to_order(cur, cl, merged_labels(N, k))
    return np.ascontiguousarray(out)


def halves(N):
    """The two halves of the modes whose intermediates are shared: modes
    0 .. N//2 - 1 and N//2 .. N-1 (for N = 4 the pairs (1,2), (3,4) of Sec. 3.3)."""
    return list(range(N // 2)), list(range(N // 2, N))


def half_of(N, k):
    """For N >= 4: the other half (whose intermediate M_k reuses) and the
    members of k's own half except k.  Generalises pair_of: every M_k of one
    half shares the contraction of the whole other half."""
    if N < 4:
        raise ValueError("half sharing is defined for N >= 4")
    H = halves(N)
    q = 0 if k < N // 2 else 1
    return tuple(H[1 - q]), [t for t in H[q] if t != k]


def half_intermediate(factors, members, counter=None):
    """T_H: the contraction of the factors of a half, in ascending order
    (for two members the pair intermediate T_cd)."""
    if len(members) == 2:
        return pair_intermediate(factors, members[0], members[1], counter)
    N = len(factors)
    cur, cl = factors[members[0]], _factor_labels(N, members[0])
    for t in members[1:]:
        cur, cl = _contract(cur, cl, factors[t], _factor_labels(N, t), counter, "M")
    return cur, cl


def merged_from_half(factors, k, T, Tl, counter=None):
    """M_k = (contraction of k's own half except k) x T_other (reuse path)."""
    N = len(factors)
    _, own = half_of(N, k)
    if len(own) == 1 and N == 4:
        return merged_from_pair(factors, k, T, Tl, counter)
    cur, cl = factors[own[0]], _factor_labels(N, own[0])
    for t in own[1:]:
        cur, cl = _contract(cur, cl, factors[t], _factor_labels(N, t), counter, "M")
    cur, cl = _contract(cur, cl, T, Tl, counter, "M")
    out, _ = _to_order(cur, cl, merged_labels(N, k))
    return np.ascontiguousarray(out)


def merged_matrix(Mt, dims, R, k):
    """GUnfold of M_k into the s_k x P_k matrix M_k (Eq. 4)."""
    return Mt.reshape(s_k(dims, R, k), -1)


def unfold_factor(Ak, k):
    """A_k(k): mode-k unfolding, I_k x s_k, bonds in ascending t order."""
    return np.moveaxis(Ak, k, 0).reshape(Ak.shape[k], -1)


def fold_factor(Ak_mat, dims, R, k):
    """GFold back to A_k (Eq. 9)."""
    shp = factor_shape(dims, R, k)
    rest = [shp[t] for t in range(len(dims)) if t != k]
    return np.ascontiguousarray(np.moveaxis(Ak_mat.reshape([shp[k]] + rest), 0, k))


def unfold_tensor(X, k):
    """X_(k): I_k x P_k, remaining modes in ascending order, row-major."""
    return np.moveaxis(X, k, 0).reshape(X.shape[k], -1)


def fold_tensor(Xk, dims, k):
    rest = [dims[t] for t in range(len(dims)) if t != k]
    return np.ascontiguousarray(np.moveaxis(Xk.reshape([dims[k]] + rest), 0, k))


# --------------------------------------------------------------------------
# Periodically modified negative Laplacian (Sec. 3.1)
# --------------------------------------------------------------------------

def laplacian(I, delta, sign="psd"):
    """Dense I x I circulant L_k built entry by entry from its stencil.

    Printed form: diagonal -2-delta, both cyclic neighbours +1.  ``sign="psd"``
    negates it.  Entries that coincide for I <= 2 are summed.
    """
    if sign == "printed":
        c0, c1 = -2.0 - delta, 1.0
    elif sign == "psd":
        c0, c1 = 2.0 + delta, -1.0
    else:
        raise ValueError(sign)
    L = np.zeros((I, I))
    for i in range(I):
        L[i, i] += c0
        L[i, (i + 1) % I] += c1
        L[i, (i - 1) % I] += c1
    return L


# --------------------------------------------------------------------------
# Factor subproblem (Eqs. 4-9) and X update (Eq. 10)
# --------------------------------------------------------------------------

def gram_rhs(Xk, Mk, Ak_old, rho, dims=None, k=None, counter=None):
    """G = M_k M_k^T and Y = X_(k) M_k^T + rho A_k(k)^(t) (Eqs. 5 and 8)."""
    G = Mk @ Mk.T
    Y = Xk @ Mk.T + rho * Ak_old
    if counter is not None:
        s, P = Mk.shape
        counter.add("matmul", 2 * s * s * P + 2 * Xk.shape[0] * s * P)
    return G, Y


def solve_factor(G, Y, L, lam, rho, counter=None):
    """Solve A G + lam L A + rho A = Y (Eq. 5) by the eigen route (Eqs. 7-8).

    G = C Phi C^T (symmetric eigendecomposition of the Gram), L = Q Lambda Q^T,
    T_ij = lam Lambda_i + Phi_j + rho, A = Q ((Q^T Y C) / T) C^T.
    Raises ValueError if some T_ij <= 0 (the system is then not uniquely
    solvable by this route).
    """
    Phi, C = np.linalg.eigh(G)
    Lam, Q = np.linalg.eigh(L)
    T = lam * Lam[:, None] + Phi[None, :] + rho
    if np.min(T) <= 0:
        raise ValueError("Sylvester system of Eq. (5) is singular or indefinite (min T <= 0)")
    A = Q @ ((Q.T @ Y @ C) / T) @ C.T
    if counter is not None:
        I, s = Y.shape
        counter.add("svd", 4.0 / 3.0 * s ** 3)
        counter.add("fft", 5.0 * (I * I + I * s) * math.log2(max(I, 2)))
        counter.add("cwm", I * s)
        counter.add("cwd", I * s)
    return A


def x_update(F, X_old, mask, rho):
    """Eq. (10): X = P_{Omega^c}((F + rho X^t)/(1+rho)) + P_Omega(Y).

    X_old equals Y on Omega (true from X^(1) = P_Omega(Y) on), so the observed
    entries are taken from X_old.
    """
    return np.where(mask, X_old, (F + rho * X_old) / (1.0 + rho))


def trace_term(factors, Ls, lams):
    """sum_k lam_k/2 tr(A_k(k)^T L_k A_k(k)) (Eq. 1)."""
    tot = 0.0
    for k, A in enumerate(factors):
        Am = unfold_factor(A, k)
        tot += 0.5 * lams[k] * float(np.sum(Am * (Ls[k] @ Am)))
    return tot


def objective(X, factors, Ls, lams):
    """f(A, X) of Eq. (2) for X in D (the indicator is zero there)."""
    F = fctn_full(factors)
    return 0.5 * float(np.sum((X - F) ** 2)) + trace_term(factors, Ls, lams)


def psnr(X, truth):
    """Mean PSNR over the slices spanned by modes 1-2 (Max = 1).

    For N = 3 the mean runs over i_3; for N = 4 over (i_3, i_4).  Slice MSE is
    floored at 1e-12.
    """
    d = (np.asarray(X, dtype=np.float64) - np.asarray(truth, dtype=np.float64)) ** 2
    mse = d.reshape(d.shape[0] * d.shape[1], -1).mean(axis=0)
    return float(np.mean(10.0 * np.log10(1.0 / np.maximum(mse, 1e-12))))


# --------------------------------------------------------------------------
# FCTN-rank growth (Algorithms 1-2 start from all-ones ranks and grow them to
# the maximal FCTN-rank; the schedule below is the reading taken here)
# --------------------------------------------------------------------------
_U64 = np.uint64


def splitmix64(seed, counters):
    """SplitMix64 (Steele, Lea & Flood 2014): output number c + 1 of the
    generator seeded with `seed`, for every counter c (uint64 arithmetic mod 2^64)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _U64(seed) + (c + _U64(1)) * _U64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        z = z ^ (z >> _U64(31))
    return z


def growth_values(seed, k, n, scale):
    """Entries 0..n-1 of factor k's new slices: scale (2u - 1), u = top 53 bits / 2^53."""
    c = (np.uint64(k) << np.uint64(40)) + np.arange(n, dtype=np.uint64)
    u = (splitmix64(seed, c) >> _U64(11)).astype(np.float64) / 2.0 ** 53
    return scale * (2.0 * u - 1.0)


def grow_factors(factors, R_old, R_new, scale, seed):
    """Factors padded from ranks R_old to R_new: old entries kept, new ones from growth_values."""
    N = len(factors)
    out = []
    for k, A in enumerate(factors):
        shape = tuple(A.shape[t] if t == k else int(R_new[min(t, k)][max(t, k)]) for t in range(N))
        new = growth_values(seed, k, int(np.prod(shape)), scale).reshape(shape)
        new[tuple(slice(0, s) for s in A.shape)] = A
        out.append(new)
    return out


def complete_growth(Y, mask, init, R_max, prob_kw, grow_every, scale, seed, tol, max_sweeps, reuse=True,
                    policy=ORDER_ALTERNATE):
    """Completion with rank growth: `init` are factors of rank one on every
    bond; after every `grow_every` sweeps every bond below its maximum grows by
    one, the factors getting new slices from growth_values(seed + e, ...) for
    the e-th growth (e = 0, 1, ...).  Stops when rel <= tol with every bond at
    its maximum, or after max_sweeps sweeps.  Returns (state, history, ranks
    during each sweep)."""
    dims = Y.shape
    N = len(dims)
    R = np.ones((N, N), dtype=int)
    st = init_state(np.asarray(Y, dtype=np.float64), mask, [np.asarray(a, dtype=np.float64) for a in init])
    hist, rank_hist = [], []
    e = 0
    while st.t < max_sweeps:
        prob = Problem(dims=dims, R=R.copy(), **prob_kw)
        h = pam_sweep(st, prob, reuse=reuse, policy=policy)
        hist.append(h)
        rank_hist.append(R.copy())
        at_max = all(R[a][b] >= R_max[a][b] for a in range(N) for b in range(a + 1, N))
        if at_max and h["rel"] <= tol:
            break
        if not at_max and st.t % grow_every == 0:
            R_new = R.copy()
            for a in range(N):
                for b in range(a + 1, N):
                    R_new[a][b] = R_new[b][a] = min(R[a][b] + 1, R_max[a][b])
            st.factors = grow_factors(st.factors, R, R_new, scale, (seed + e) % 2 ** 64)
            st.versions = [v + 1 for v in st.versions]  # every factor changed: cached pairs are stale
            st.cache = {}
            R = R_new
            e += 1
    return st, hist, rank_hist


SSIM_C1 = 0.01 ** 2   # (0.01 L)^2 with dynamic range L = 1 (data in [0, 1])
SSIM_C2 = 0.03 ** 2   # (0.03 L)^2


def ssim(X, truth, c1=SSIM_C1, c2=SSIM_C2):
    """Mean SSIM over the slices spanned by modes 1-2 (Sec. 4, global form).

    Per slice: ((2 nu_T nu_X + c1)(2 omega_TX + c2)) / ((nu_T^2 + nu_X^2 + c1)
    (omega_T^2 + omega_X^2 + c2)) with nu the slice mean, omega_T, omega_X the
    standard deviations and omega_TX the covariance (sample statistics,
    divisor n - 1); the mean runs over the remaining indices as in psnr().
    """
    T = np.asarray(truth, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    n = T.shape[0] * T.shape[1]
    Ts = T.reshape(n, -1)
    Xs = X.reshape(n, -1)
    vals = []
    for t in range(Ts.shape[1]):
        a, b = Ts[:, t], Xs[:, t]
        mu_a, mu_b = a.mean(), b.mean()
        sd_a, sd_b = a.std(ddof=1), b.std(ddof=1)
        cov = np.cov(a, b, ddof=1)[0, 1]
        vals.append(((2 * mu_a * mu_b + c1) * (2 * cov + c2)) /
                    ((mu_a ** 2 + mu_b ** 2 + c1) * (sd_a ** 2 + sd_b ** 2 + c2)))
    return float(np.mean(vals))


# --------------------------------------------------------------------------
# PAM sweeps: Algorithm 1 (reuse off) and Algorithm 2 (reuse on)
# --------------------------------------------------------------------------

@dataclass
class Problem:
    dims: tuple
    R: np.ndarray            # N x N, symmetric; R[a][b] for a < b used
    lam: tuple
    delta: tuple
    rho: float = 0.1
    sign: str = "psd"


@dataclass
class State:
    factors: list
    X: np.ndarray
    mask: np.ndarray
    t: int = 0                       # completed sweeps
    versions: list = None            # bumped whenever A_k changes
    cache: dict = None               # (c, d) -> (T, labels, (ver_c, ver_d))
    counter: FlopCounter = None


def sweep_order(N, t_next, policy):
    """Update order n of sweep number t_next (1-based), Algorithm 2: with the
    alternating order (N >= 4) even sweeps take the second half of the modes
    first, whose shared intermediate (of the first half) is still valid."""
    if policy == ORDER_ALTERNATE and N >= 4 and t_next % 2 == 0:
        h0, h1 = halves(N)
        return h1 + h0
    if policy not in (ORDER_PLAIN, ORDER_ALTERNATE):
        raise ValueError(policy)
    return list(range(N))


def init_state(Y, mask, factors):
    """X^(1) = P_Omega(Y); A_k^(1) given (standard normal draws in the paper)."""
    Y = np.asarray(Y, dtype=np.float64)
    mask = np.asarray(mask, dtype=bool)
    N = Y.ndim
    return State(factors=[np.array(a, dtype=np.float64, copy=True) for a in factors],
                 X=np.where(mask, Y, 0.0), mask=mask, versions=[0] * N, cache={},
                 counter=FlopCounter())


def _merged(state, prob, k, reuse):
    N = len(prob.dims)
    if reuse and N >= 4:
        other, _ = half_of(N, k)
        vers = tuple(state.versions[t] for t in other)
        ent = state.cache.get(other)
        if ent is None or ent[2] != vers:
            T, Tl = half_intermediate(state.factors, list(other), state.counter)
            state.cache[other] = (T, Tl, vers)
        T, Tl, _ = state.cache[other]
        return merged_from_half(state.factors, k, T, Tl, state.counter)
    return merged_sequential(state.factors, k, state.counter)


def extrapolate(A_new, A_old, alpha, beta):
    """Asymmetric extrapolation (Sec. 4.3): A + alpha (A - beta A^(t))."""
    return A_new + alpha * (A_new - beta * A_old)


def pam_sweep(state, prob, reuse=True, policy=ORDER_ALTERNATE, trace_blocks=False, extrapolation=None):
    """One PAM sweep (scheme 3): every A_k in order, then X (Algorithms 1/2).

    ``extrapolation = (alpha, beta)`` replaces every new factor by its
    asymmetric extrapolation right after its update (the multi-temporal HSI
    variant of Sec. 4.3); None is the plain method.

    With ``reuse`` the merged tensors come from cached half intermediates
    (N >= 4; pairs for N = 4) and FCTN(A^{t+1}) for the X update is A_last(last) M'_last, where
    M'_last is the merged tensor of the factor updated last (every other
    factor is already new there).  Without ``reuse`` every merged tensor and
    FCTN(A^{t+1}) are contracted from scratch.

    Returns a dict with rel (= ||X^{t+1}-X^t|| / ||X^t||), objective (Eq. 2
    value after the sweep) and, if ``trace_blocks``, the objective before the
    sweep and after every block with the block's ||Delta||_F^2.
    """
    dims = tuple(prob.dims)
    N = len(dims)
    Ls = [laplacian(dims[k], prob.delta[k], prob.sign) for k in range(N)]
    order = sweep_order(N, state.t + 1, policy)
    blocks = []
    f_prev = objective(state.X, state.factors, Ls, prob.lam) if trace_blocks else None
    last_M = None
    for k in order:
        Mt = _merged(state, prob, k, reuse)
        Mk = merged_matrix(Mt, dims, prob.R, k)
        Xk = unfold_tensor(state.X, k)
        Ak_old = unfold_factor(state.factors[k], k)
        G, Y = gram_rhs(Xk, Mk, Ak_old, prob.rho, counter=state.counter)
        Ak_new = solve_factor(G, Y, Ls[k], prob.lam[k], prob.rho, counter=state.counter)
        if extrapolation is not None:
            Ak_new = extrapolate(Ak_new, Ak_old, extrapolation[0], extrapolation[1])
        state.factors[k] = fold_factor(Ak_new, dims, prob.R, k)
        state.versions[k] += 1
        last_M = (k, Mk)
        if trace_blocks:
            f_new = objective(state.X, state.factors, Ls, prob.lam)
            blocks.append(("A", k, f_prev, f_new, float(np.sum((Ak_new - Ak_old) ** 2))))
            f_prev = f_new
    # X update (Eq. 10)
    if reuse:
        k, Mk = last_M
        Fk = unfold_factor(state.factors[k], k) @ Mk
        state.counter.add("X", 2 * Fk.size * Mk.shape[0])
        F = fold_tensor(Fk, dims, k)
    else:
        F = fctn_full(state.factors, state.counter, "X")
    X_old = state.X
    X_new = x_update(F, X_old, state.mask, prob.rho)
    rel = float(np.linalg.norm(X_new - X_old) / np.linalg.norm(X_old))
    state.X = X_new
    state.t += 1
    trace = 0.0
    for kk in range(N):
        Am = unfold_factor(state.factors[kk], kk)
        trace += 0.5 * prob.lam[kk] * float(np.sum(Am * (Ls[kk] @ Am)))
    obj = 0.5 * float(np.sum((X_new - F) ** 2)) + trace
    out = {"t": state.t, "rel": rel, "objective": obj, "order": order}
    if trace_blocks:
        blocks.append(("X", -1, f_prev, obj, float(np.sum((X_new - X_old) ** 2))))
        out["blocks"] = blocks
    return out


def complete(Y, mask, factors, prob, tol=1e-4, max_sweeps=500, reuse=True,
             policy=ORDER_ALTERNATE, callback=None, extrapolation=None):
    """Run sweeps until rel <= tol or max_sweeps (do-while, Algorithms 1/2).

    ``tol <= 0`` runs exactly ``max_sweeps`` sweeps.
    """
    st = init_state(Y, mask, factors)
    hist = []
    while True:
        info = pam_sweep(st, prob, reuse=reuse, policy=policy, extrapolation=extrapolation)
        hist.append(info)
        if callback is not None:
            callback(st, info)
        if (tol > 0 and info["rel"] <= tol) or st.t >= max_sweeps:
            break
    return st, hist

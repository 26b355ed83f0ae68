"""Seeded synthetic inputs shared by the tests, the oracle runs and the bench.

This module holds random draws and data-recipe steps only (no step of the
completion method): standard-normal factor draws, a circular moving average
along each factor's physical mode, additive noise, min-max scaling,
Bernoulli observation masks and the standard-normal initial factors of
Algorithms 1/2.  The FCTN contraction that turns the drawn factors into a
low-rank tensor is done by the consumer (the oracle in tests, the library's
own contraction in the bench), so that neither side depends on the other.

Seeds follow one recipe for every workload: data = 1000 + i, mask = 2000 + i,
initial factors = 3000 + i (NumPy PCG64), where i is the workload index.
"""
from __future__ import annotations

import numpy as np


def rank_matrix(dims, r, cap_small=None):
    """Symmetric N x N FCTN rank matrix with every R_ab = r.

    ``cap_small`` = (size, cap): every bond touching a mode of that size is
    capped at ``cap`` (e.g. (3, 3) caps the bonds of a colour mode at 3).
    The diagonal is unused and set to 0.
    """
    N = len(dims)
    R = np.zeros((N, N), dtype=np.int64)
    for a in range(N):
        for b in range(N):
            if a == b:
                continue
            v = r
            if cap_small is not None and (dims[a] == cap_small[0] or dims[b] == cap_small[0]):
                v = min(v, cap_small[1])
            R[a, b] = v
    return R


def factor_shape(dims, R, k):
    N = len(dims)
    return tuple(int(dims[k]) if t == k else int(R[min(k, t), max(k, t)]) for t in range(N))


def normal_factors(dims, R, seed):
    """Standard-normal factor draws A_k with the FCTN factor shapes (float64)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(factor_shape(dims, R, k)) for k in range(len(dims))]


def smooth_along(a, axis, taps=5):
    """Circular moving average with ``taps`` equal weights along ``axis``."""
    h = taps // 2
    acc = np.zeros_like(a)
    for o in range(-h, h + 1):
        acc += np.roll(a, o, axis=axis)
    return acc / taps


def smoothed_factors(dims, R, seed):
    """Factors of the ground-truth tensor: N(0,1) draws smoothed along I_k."""
    fs = normal_factors(dims, R, seed)
    return [smooth_along(f, k) for k, f in enumerate(fs)]


def finish_tensor(raw, noise_sigma=0.0, seed=0):
    """Add sigma * N(0,1) noise (seeded), then min-max scale to [0, 1]."""
    x = np.array(raw, dtype=np.float64, copy=True)
    if noise_sigma > 0:
        rng = np.random.default_rng([seed, 7])
        x += noise_sigma * rng.standard_normal(x.shape)
    lo, hi = float(x.min()), float(x.max())
    return (x - lo) / (hi - lo) if hi > lo else np.zeros_like(x)


def bernoulli_mask(dims, p, seed):
    """i.i.d. Bernoulli(p) observation set Omega as a bool array."""
    rng = np.random.default_rng(seed)
    return rng.random(tuple(dims)) < p


def init_factors(dims, R, seed):
    """A_k^(1) with standard-normal entries (Algorithms 1/2, Initialize)."""
    return normal_factors(dims, R, seed)


# Workloads: sizes, ranks, sampling rates and sweep counts.
WORKLOADS = {
    "c1": dict(dims=(30, 30, 10), r=3, cap=None, p=0.3, noise=0.0, sweeps=20, idx=0),
    "c2": dict(dims=(256, 256, 31), r=8, cap=None, p=0.1, noise=0.01, sweeps=100, idx=1),
    "c3": dict(dims=(144, 176, 3, 50), r=6, cap=(3, 3), p=0.05, noise=0.0, sweeps=100, idx=2),
    "c4": dict(dims=(256, 256, 31, 8), r=6, cap=None, p=0.1, noise=0.0, sweeps=500, idx=3),
}

LAMBDA = 0.01
DELTA = 0.5
RHO = 0.1


def workload_inputs(name, contract, dims=None, r=None, p=None, idx=None, noise=None, cap="default"):
    """Return (truth, Y, mask, init, R) for a workload.

    ``contract(factors) -> ndarray`` performs the FCTN contraction of the
    drawn ground-truth factors; it is supplied by the caller.  Overrides of
    dims / r / p / idx build scaled-down variants with the same recipe.
    """
    w = dict(WORKLOADS[name]) if name is not None else {}
    dims = tuple(dims if dims is not None else w["dims"])
    r = r if r is not None else w["r"]
    p = p if p is not None else w["p"]
    idx = idx if idx is not None else w.get("idx", 0)
    noise = noise if noise is not None else w.get("noise", 0.0)
    capv = w.get("cap") if cap == "default" else cap
    R = rank_matrix(dims, r, capv)
    truth = finish_tensor(contract(smoothed_factors(dims, R, 1000 + idx)), noise, 1000 + idx)
    mask = bernoulli_mask(dims, p, 2000 + idx)
    Y = np.where(mask, truth, 0.0)
    init = init_factors(dims, R, 3000 + idx)
    return truth, Y, mask, init, R

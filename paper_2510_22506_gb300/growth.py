"""Completion with FCTN-rank growth through libfctn.

Algorithms 1-2 start from all-ones FCTN ranks and grow them to the maximal
FCTN-rank.  Schedule (this package's rule): after every `grow_every` sweeps,
every bond below its maximum grows by one (fctn_grow_ranks, whose new factor
slices come from the library's SplitMix64 noise with seed + e for the e-th
growth); the run stops when rel_change <= tol with every bond at its maximum,
or after max_sweeps sweeps.  Host bookkeeping only: every sweep and every
re-layout runs in the library.
"""
from __future__ import annotations

import numpy as np

from . import fctn as F


def complete_with_growth(Y, mask, init, R_max, grow_every, scale, seed, tol, max_sweeps, precision="fp32",
                         stream=None, **params):
    """Returns (handle, history); the caller destroys the handle.  `init` are
    the rank-one factors (FCTN shapes) in the compute precision; `params` are
    passed to make_params (lam, delta, rho, reuse, order_policy, ...)."""
    dims = tuple(Y.shape)
    N = len(dims)
    R = np.ones((N, N), dtype=int)
    p = F.make_params(dims, R, precision=precision, **params)
    h = F.fctn_create(p, stream)
    hist = []
    try:
        dt = F.elem_dtype(p)
        F.fctn_set_data(h, np.ascontiguousarray(Y.astype(dt)), np.ascontiguousarray(mask.astype(np.uint8)))
        F.fctn_set_factors(h, [np.ascontiguousarray(np.asarray(a).astype(dt)) for a in init])
        e = 0
        for _ in range(max_sweeps):
            st = F.fctn_pam_sweep(h, 1)
            hist.append(dict(st, ranks=R.copy()))
            at_max = all(R[a][b] >= R_max[a][b] for a in range(N) for b in range(a + 1, N))
            if at_max and st["rel_change"] <= tol:
                break
            if not at_max and st["t"] % grow_every == 0:
                Rn = R.copy()
                for a in range(N):
                    for b in range(a + 1, N):
                        Rn[a][b] = Rn[b][a] = min(R[a][b] + 1, R_max[a][b])
                F.fctn_grow_ranks(h, Rn, scale, (seed + e) % 2 ** 64)
                R = Rn
                e += 1
    except BaseException:
        F.fctn_destroy(h)
        raise
    return h, hist

"""FCTN-rank growth (from all-ones ranks to the maximal FCTN-rank): the
library (fctn_grow_ranks driven by growth.complete_with_growth) against the
oracle's complete_growth with the same inputs and schedule."""
import numpy as np
import pytest

from oracle import fctn_oracle as O
from paper_2510_22506_gb300 import synth
from tests.util import inputs, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2510_22506_gb300 import fctn
    return fctn


def _case(dims, rmax, cap):
    d = inputs(None, dims=dims, r=rmax, p=0.4, idx=48, noise=0.0, cap=cap)
    N = len(dims)
    ones = np.ones((N, N), dtype=int)
    init = synth.init_factors(dims, ones, 3100)
    return d, init


@pytest.mark.parametrize("dims,rmax,cap,precision,tol", [((30, 30, 10), 3, None, "fp64", 1e-9),
                                                        ((13, 7, 3, 5), 3, (3, 2), "fp64", 1e-9),
                                                        ((40, 36, 12), 4, None, "fp32", 1e-4)])
def test_growth_matches_oracle(F, dims, rmax, cap, precision, tol):
    from paper_2510_22506_gb300 import growth
    d, init = _case(dims, rmax, cap)
    R_max = d["R"]
    N = len(dims)
    prob_kw = dict(lam=(0.01,) * N, delta=(0.5,) * N, rho=0.1)
    st, hist, ranks = O.complete_growth(d["Y"].astype(np.float64), d["mask"], init, R_max, prob_kw, grow_every=3,
                                        scale=0.1, seed=123, tol=0.0, max_sweeps=12)
    h, ghist = growth.complete_with_growth(d["Y"], d["mask"], init, R_max, grow_every=3, scale=0.1, seed=123,
                                           tol=0.0, max_sweeps=12, precision=precision)
    try:
        dt = np.float64 if precision == "fp64" else np.float32
        X = np.empty(dims, dtype=dt)
        F.fctn_get_X(h, X)
        facs = []
        for k in range(N):
            a = np.empty(O.factor_shape(dims, R_max, k), dtype=dt)
            F.fctn_get_factor(h, k, a)
            facs.append(a)
    finally:
        F.fctn_destroy(h)
    assert len(ghist) == len(hist) == 12
    for a, b in zip(ghist, ranks):
        np.testing.assert_array_equal(a["ranks"], b)
    assert np.array_equal(np.triu(ranks[-1], 1), np.triu(R_max, 1))  # reached the maximal ranks
    assert rel(X, st.X) <= tol, rel(X, st.X)
    for k, (a, b) in enumerate(zip(facs, st.factors)):
        assert rel(a, b) <= tol, (k, rel(a, b))


def test_growth_rejects_shrinking(F):
    d, init = _case((12, 10, 4), 2, None)
    p = F.make_params(d["dims"], np.full((3, 3), 2), precision="fp64")
    h = F.fctn_create(p)
    try:
        F.fctn_set_data(h, d["Y"], d["mask"].astype(np.uint8))
        F.fctn_set_factors(h, [np.ascontiguousarray(a) for a in
                               synth.init_factors(d["dims"], np.full((3, 3), 2), 3101)])
        with pytest.raises(F.FctnError) as ei:
            F.fctn_grow_ranks(h, np.full((3, 3), 1), 0.1, 1)
        assert ei.value.code == F.FCTN_E_ARG
        F.fctn_pam_sweep(h, 1)  # the handle is still usable
    finally:
        F.fctn_destroy(h)

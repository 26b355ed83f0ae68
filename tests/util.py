"""Helpers shared by the GPU tests: seeded inputs, oracle runs, GPU runs."""
import numpy as np

from oracle import fctn_oracle as O
from paper_2510_22506_gb300 import synth


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def inputs(name=None, dtype=np.float64, **over):
    """Seeded inputs cast to the GPU element type; the oracle gets the same values."""
    truth, Y, mask, init, R = synth.workload_inputs(name, O.fctn_full, **over)
    Yc = Y.astype(dtype)
    initc = [a.astype(dtype) for a in init]
    return dict(truth=truth, Y=Yc, mask=mask, init=initc, R=R, dims=tuple(Y.shape))


def oracle_run(d, sweeps, lam=0.01, delta=0.5, rho=0.1, reuse=True, policy="alternate", sign="psd",
               extrapolation=None):
    N = len(d["dims"])
    prob = O.Problem(dims=d["dims"], R=d["R"], lam=(lam,) * N, delta=(delta,) * N, rho=rho, sign=sign)
    st, hist = O.complete(d["Y"].astype(np.float64), d["mask"], [a.astype(np.float64) for a in d["init"]], prob,
                          tol=0, max_sweeps=sweeps, reuse=reuse, policy=policy, extrapolation=extrapolation)
    return st, hist


def gpu_run(F, d, sweeps, precision="fp64", lam=0.01, delta=0.5, rho=0.1, reuse=True, policy="alternate",
            sign="psd", refine_steps=None, stats_every=None, extrapolation=None, gram_mode="auto", rhs_ctas=0,
            eig_max_sweeps=0, eig_tol=0.0, tile_code=0, solve_method="auto"):
    p = F.make_params(d["dims"], d["R"], lam=lam, delta=delta, rho=rho, precision=precision, reuse=reuse,
                      order_policy=policy, laplacian_sign=sign, refine_steps=refine_steps,
                      extrapolation=extrapolation, gram_mode=gram_mode, rhs_ctas=rhs_ctas,
                      eig_max_sweeps=eig_max_sweeps, eig_tol=eig_tol, tile_code=tile_code,
                      solve_method=solve_method)
    dt = F.elem_dtype(p)
    h = F.fctn_create(p)
    try:
        F.fctn_set_data(h, np.ascontiguousarray(d["Y"].astype(dt)), np.ascontiguousarray(d["mask"].astype(np.uint8)))
        F.fctn_set_factors(h, [np.ascontiguousarray(a.astype(dt)) for a in d["init"]])
        hist = []
        if stats_every:
            done = 0
            while done < sweeps:
                n = min(stats_every, sweeps - done)
                hist.append(F.fctn_pam_sweep(h, n))
                done += n
            st = hist[-1]
        else:
            st = F.fctn_pam_sweep(h, sweeps)
        X = np.empty(d["dims"], dtype=dt)
        F.fctn_get_X(h, X)
        facs = []
        for k, shp in enumerate(F.factor_shapes(p)):
            a = np.empty(shp, dtype=dt)
            F.fctn_get_factor(h, k, a)
            facs.append(a)
        launches = F.fctn_launch_count(h)
    finally:
        F.fctn_destroy(h)
    return dict(X=X, factors=facs, stats=st, hist=hist, launches=launches)

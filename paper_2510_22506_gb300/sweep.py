"""Run PAM sweeps of a named synthetic workload through libfctn.

    python -m paper_2510_22506_gb300.sweep --workload c4 --precision tf32 --sweeps 3 [--time]
        [--order plain|alternate] [--reuse 1] [--tile-code N] [--rhs-ctas N] [--solve auto|eig|chol]

Workloads (seeded, see synth.WORKLOADS): c1 30x30x10, c2 256x256x31,
c3 144x176x3x50, c4 256x256x31x8.  The ground-truth tensor is contracted by
the library itself.  Prints the stop-test values after the sweeps and, with
--time, the device time per sweep (CUDA events on the handle's stream).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import fctn as F
from . import synth


def library_inputs(name):
    w = synth.WORKLOADS[name]
    dims = tuple(w["dims"])
    R = synth.rank_matrix(dims, w["r"], w["cap"])

    def contract(fs):
        p = F.make_params(dims, R, precision="fp64", reuse=False)
        h = F.fctn_create(p)
        try:
            F.fctn_set_factors(h, [np.ascontiguousarray(a) for a in fs])
            out = np.empty(dims, dtype=np.float64)
            F.fctn_contract(h, out)
        finally:
            F.fctn_destroy(h)
        return out

    return synth.workload_inputs(name, contract)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--sweeps", type=int, default=3)
    ap.add_argument("--reuse", type=int, default=1)
    ap.add_argument("--time", action="store_true")
    ap.add_argument("--rhs-ctas", type=int, default=0, help="launch shape of the Gram / RHS kernel (0 = built-in)")
    ap.add_argument("--order", default="plain", choices=["plain", "alternate"])
    ap.add_argument("--tile-code", type=int, default=0, help="launch shapes of the head-mode route (0 = built-in)")
    ap.add_argument("--solve", default="auto", choices=["auto", "eig", "chol"], help="solve of Eq. 5")
    a = ap.parse_args(argv)
    truth, Y, mask, init, R = library_inputs(a.workload)
    p = F.make_params(Y.shape, R, lam=synth.LAMBDA, delta=synth.DELTA, rho=synth.RHO, precision=a.precision,
                      reuse=bool(a.reuse), rhs_ctas=a.rhs_ctas, order_policy=a.order, tile_code=a.tile_code,
                      solve_method=a.solve)
    dt = F.elem_dtype(p)
    out = {"workload": a.workload, "precision": a.precision, "sweeps": a.sweeps}
    if a.time:
        import torch
        st = torch.cuda.Stream()
        h = F.fctn_create(p, st)
    else:
        h = F.fctn_create(p)
    try:
        F.fctn_set_data(h, np.ascontiguousarray(Y.astype(dt)), mask.astype(np.uint8))
        F.fctn_set_factors(h, [np.ascontiguousarray(x.astype(dt)) for x in init])
        if a.time:
            F.fctn_pam_sweep(h, 3, want_stats=False)  # warm-up: graph capture, warm starts
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            F.fctn_pam_sweep(h, a.sweeps, want_stats=False)
            e1.record(st)
            torch.cuda.synchronize()
            out["ms_per_sweep"] = e0.elapsed_time(e1) / max(a.sweeps, 1)
        else:
            F.fctn_pam_sweep(h, a.sweeps, want_stats=False)
        out["stats"] = F.fctn_pam_sweep(h, 0)
        out["launches"] = F.fctn_launch_count(h)
    finally:
        F.fctn_destroy(h)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

"""Serving driver: Poisson arrivals of completion jobs into the libfctn server.

The scheduling itself (admission by device footprint, one CUDA-graph sweep
per job per pass on the job's own stream or, grouped, one graph per shape
class, retirement on the stop test) lives in the library (fctn_server_*).
This module builds a job mix, submits jobs at their arrival times while
stepping the server, and reports throughput, latency percentiles and the
final PSNR of every job; `run_sequential` serves the same arrivals one job at
a time through fctn_complete (first come, first served) for comparison.
"""
from __future__ import annotations

import time

import numpy as np

from . import fctn as F
from . import synth

MIX_SHAPES = [(64, 64, 16), (128, 128, 31), (144, 176, 3, 20), (256, 256, 31)]
MIX_RANKS = [3, 4, 6]
MIX_RATES = [0.05, 0.1, 0.2]


def library_contract(dims, R):
    """FCTN contraction of host factors through the library (FP64)."""
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
    return contract


def mix_jobs(n_jobs, seed=5000, rate=20.0, shapes=MIX_SHAPES, contract=None):
    """Job specs of the serving mix: shape, ranks, sampling rate, Poisson arrival time."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n_jobs)
    arrivals = np.cumsum(gaps) - gaps[0]
    jobs = []
    for i in range(n_jobs):
        dims = tuple(shapes[rng.integers(len(shapes))])
        r = int(MIX_RANKS[rng.integers(len(MIX_RANKS))])
        pr = float(MIX_RATES[rng.integers(len(MIX_RATES))])
        cap = (3, 3) if 3 in dims else None
        R = synth.rank_matrix(dims, r, cap)
        c = contract(dims, R) if contract else library_contract(dims, R)
        truth, Y, mask, init, _ = synth.workload_inputs(None, c, dims=dims, r=r, p=pr, idx=100 + i, noise=0.0,
                                                        cap=cap)
        jobs.append(dict(i=i, dims=dims, r=r, p=pr, R=R, Y=Y, mask=mask, init=init, truth=truth,
                         arrival=float(arrivals[i])))
    return jobs


# mixed precision: tensor-core sweeps until the change falls to this, FP32 sweeps after
FINISH_FP32_AT = 1e-3


def job_params(job, precision, tuner=None):
    p = F.make_params(job["dims"], job["R"], lam=synth.LAMBDA, delta=synth.DELTA, rho=synth.RHO,
                      precision=precision, reuse=True, order_policy="plain",
                      finish_fp32_at=FINISH_FP32_AT if precision in ("tf32", "bf16") else 0.0)
    if tuner is not None:
        p.tile_code = tuner.get(job, p)
    return p


class TuneCache:
    """Tile codes (fctn_params.tile_code: tensor-core or CUDA-core products,
    pipeline depth, K splits) per job class (dims, ranks, precision), chosen
    by libfctn's autotuner (fctn_autotune_tiles) on the first job of the class
    and reused for the rest; `fill` tunes every class of a job list up front,
    as a server would load a stored cache before taking traffic."""

    def __init__(self, sweeps=3, candidates=None):
        self.sweeps, self.candidates, self.table, self.tune_s = sweeps, candidates, {}, 0.0

    @staticmethod
    def key(job, p):
        N = len(job["dims"])
        return (tuple(job["dims"]), tuple(int(job["R"][a][b]) for a in range(N) for b in range(a + 1, N)),
                int(p.precision))

    def get(self, job, p):
        k = self.key(job, p)
        if k not in self.table:
            dt = F.elem_dtype(p)
            t0 = time.perf_counter()
            best, _ = F.fctn_autotune_tiles(p, np.ascontiguousarray(job["Y"].astype(dt)),
                                            job["mask"].astype(np.uint8),
                                            [np.ascontiguousarray(a.astype(dt)) for a in job["init"]],
                                            candidates=self.candidates, sweeps=self.sweeps)
            self.tune_s += time.perf_counter() - t0
            self.table[k] = best
        return self.table[k]

    def fill(self, jobs, precision):
        for j in jobs:
            job_params(j, precision, self)
        return self


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if xs else None


def psnr(X, truth):
    """PSNR of Sec. 4 for the serving report: mean over the slices of modes
    1-2 of 10 log10(1 / MSE) (peak 1, data in [0, 1]), MSE floored at 1e-12."""
    X = np.asarray(X, dtype=np.float64).reshape(truth.shape[0] * truth.shape[1], -1)
    T = np.asarray(truth, dtype=np.float64).reshape(X.shape)
    mse = np.maximum(np.mean((X - T) ** 2, axis=0), 1e-12)
    return float(np.mean(10.0 * np.log10(1.0 / mse)))


def run_mix(jobs, precision="fp32", tol=1e-4, max_sweeps=500, max_jobs=32, mem_budget_bytes=0,
            keep_results=False, poll_sleep=2e-5, arrivals=True, tuner=None, group=True):
    """Submit jobs at their arrival times, step the server until all finish;
    `tuner` (a TuneCache) supplies each job's launch shape; `group` sweeps the
    ready jobs of a shape class as one graph."""
    srv = F.fctn_server_create(max_jobs=max_jobs, mem_budget_bytes=mem_budget_bytes, group=group)
    pending = sorted(jobs, key=lambda j: j["arrival"]) if arrivals else list(jobs)
    ids, t_arr, results, infos = {}, {}, {}, {}
    try:
        t0 = time.perf_counter()
        nxt = 0
        while nxt < len(pending) or ids:
            now = time.perf_counter() - t0
            while nxt < len(pending) and (not arrivals or pending[nxt]["arrival"] <= now):
                j = pending[nxt]
                p = job_params(j, precision, tuner)
                dt = F.elem_dtype(p)
                jid = F.fctn_server_submit(srv, p, j["Y"].astype(dt), j["mask"], [a.astype(dt) for a in j["init"]],
                                           tol, max_sweeps)
                ids[jid] = j["i"]
                t_arr[j["i"]] = t0 + (j["arrival"] if arrivals else 0.0)
                nxt += 1
            F.fctn_server_step(srv)
            done = F.fctn_server_finished(srv)
            tnow = time.perf_counter()
            for jid in done:
                info = F.fctn_server_poll(srv, jid)
                info["t_wall_done"] = tnow
                infos[ids[jid]] = info
            for jid in done:
                i = ids.pop(jid)
                if infos[i]["state"] == F.FCTN_JOB_DONE:
                    j = jobs[i] if jobs[i]["i"] == i else next(x for x in jobs if x["i"] == i)
                    out = np.empty(j["dims"], dtype=F.elem_dtype(job_params(j, precision)))
                    F.fctn_server_result(srv, jid, out)
                    infos[i]["psnr_db"] = psnr(out, j["truth"])
                    if keep_results:
                        results[i] = out
            if not done and poll_sleep:
                time.sleep(poll_sleep)
        t_end = time.perf_counter()
        stats = F.fctn_server_stats(srv)
        gstats = F.fctn_server_group_stats(srv)
    finally:
        F.fctn_server_destroy(srv)
    lat = [infos[i]["t_wall_done"] - t_arr[i] for i in infos]
    ttt = [infos[i]["t_done"] - infos[i]["t_admit"] for i in infos if infos[i]["state"] == F.FCTN_JOB_DONE]
    sweeps = sum(infos[i]["sweeps"] for i in infos)
    first = min(t_arr.values())
    return {"jobs": len(infos), "failed": sum(1 for i in infos if infos[i]["state"] != F.FCTN_JOB_DONE),
            "wall_s": t_end - first, "jobs_per_s": len(infos) / (t_end - first), "sweeps": int(sweeps),
            "sweeps_per_s": sweeps / (t_end - first), "latency_p50_s": _pct(lat, 50), "latency_p99_s": _pct(lat, 99),
            "ttt_p50_s": _pct(ttt, 50), "ttt_p99_s": _pct(ttt, 99), "sweeps_launched": stats["sweeps_launched"],
            "psnr_mean_db": float(np.mean([v["psnr_db"] for v in infos.values() if "psnr_db" in v])),
            **gstats, "infos": infos, "results": results}


def run_sequential(jobs, precision="fp32", tol=1e-4, max_sweeps=500, keep_results=False, arrivals=True):
    """The same jobs one at a time through fctn_complete, first come first
    served: a job starts at its arrival time or when the previous one ends,
    whichever is later; latency = end - arrival, time to tolerance = end -
    start."""
    infos, results = {}, {}
    order = sorted(jobs, key=lambda j: j["arrival"]) if arrivals else list(jobs)
    t0 = time.perf_counter()
    sweeps = 0
    for j in order:
        if arrivals:
            wait = t0 + j["arrival"] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
        p = job_params(j, precision)
        dt = F.elem_dtype(p)
        h = F.fctn_create(p)
        try:
            ts = time.perf_counter()
            F.fctn_set_data(h, np.ascontiguousarray(j["Y"].astype(dt)), j["mask"].astype(np.uint8))
            F.fctn_set_factors(h, [np.ascontiguousarray(a.astype(dt)) for a in j["init"]])
            out = np.empty(j["dims"], dtype=dt)
            st = F.fctn_complete(h, tol, max_sweeps, out)
            te = time.perf_counter()
            infos[j["i"]] = dict(st, wall=te - ts, latency=te - (t0 + (j["arrival"] if arrivals else 0.0)),
                                 psnr_db=psnr(out, j["truth"]))
            sweeps += st["t"]
            if keep_results:
                results[j["i"]] = out
        finally:
            F.fctn_destroy(h)
    wall = time.perf_counter() - t0
    ttt = [v["wall"] for v in infos.values()]
    lat = [v["latency"] for v in infos.values()]
    return {"jobs": len(jobs), "wall_s": wall, "jobs_per_s": len(jobs) / wall, "sweeps": int(sweeps),
            "sweeps_per_s": sweeps / wall, "latency_p50_s": _pct(lat, 50), "latency_p99_s": _pct(lat, 99),
            "ttt_p50_s": _pct(ttt, 50), "ttt_p99_s": _pct(ttt, 99),
            "psnr_mean_db": float(np.mean([v["psnr_db"] for v in infos.values()])),
            "infos": infos, "results": results}

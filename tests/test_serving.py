"""Serving: continuous batching of completion jobs (fctn_server_*).

Each job's result must be the same alone and in the mix (the kernels are
deterministic, so the bytes are identical), admission must respect the
memory budget, and a failing job must not stop the others.
"""
import numpy as np
import pytest

from oracle import fctn_oracle as O
from paper_2510_22506_gb300 import synth

pytestmark = pytest.mark.gpu

SMALL = [(32, 30, 9), (24, 20, 3, 6), (40, 36, 12), (20, 18, 3, 5)]


@pytest.fixture(scope="module")
def mods():
    from paper_2510_22506_gb300 import fctn as F
    from paper_2510_22506_gb300 import serve as S
    return F, S


def _contract(dims, R):
    return O.fctn_full


def test_results_identical_alone_and_in_mix(mods):
    F, S = mods
    jobs = S.mix_jobs(8, seed=7, rate=1000.0, shapes=SMALL, contract=_contract)
    mix = S.run_mix(jobs, precision="fp32", tol=1e-4, max_sweeps=40, max_jobs=3, keep_results=True, arrivals=False)
    alone = S.run_sequential(jobs, precision="fp32", tol=1e-4, max_sweeps=40, keep_results=True, arrivals=False)
    assert mix["failed"] == 0 and mix["jobs"] == len(jobs)
    for j in jobs:
        i = j["i"]
        assert mix["infos"][i]["sweeps"] == alone["infos"][i]["t"]
        np.testing.assert_array_equal(mix["results"][i], alone["results"][i])


@pytest.mark.parametrize("group", [True, False])
def test_grouped_sweeps_identical_alone_and_in_mix(mods, group):
    """Jobs of one shape class sweep as one captured graph (re-launched while
    the members stay, captured anew when one leaves); every result keeps the
    bytes of the job run alone.  Without grouping each job launches its own
    sweep graph."""
    F, S = mods
    jobs = S.mix_jobs(8, seed=17, rate=1000.0, shapes=[(40, 36, 12)], contract=_contract)
    mix = S.run_mix(jobs, precision="fp32", tol=1e-4, max_sweeps=40, max_jobs=8, keep_results=True,
                    arrivals=False, group=group)
    alone = S.run_sequential(jobs, precision="fp32", tol=1e-4, max_sweeps=40, keep_results=True, arrivals=False)
    assert mix["failed"] == 0 and mix["jobs"] == len(jobs)
    if group:
        assert mix["group_launches"] > mix["group_captures"] > 0
    else:
        assert mix["group_launches"] == 0
    for j in jobs:
        i = j["i"]
        assert mix["infos"][i]["sweeps"] == alone["infos"][i]["t"]
        np.testing.assert_array_equal(mix["results"][i], alone["results"][i])


def test_arrivals_are_admitted_while_others_run(mods):
    F, S = mods
    jobs = S.mix_jobs(6, seed=8, rate=400.0, shapes=SMALL, contract=_contract)
    out = S.run_mix(jobs, precision="fp32", tol=1e-4, max_sweeps=60, max_jobs=4)
    assert out["failed"] == 0 and out["jobs"] == 6
    assert out["latency_p99_s"] >= out["latency_p50_s"] > 0


def test_admission_respects_memory_budget(mods):
    F, S = mods
    jobs = S.mix_jobs(5, seed=9, rate=1000.0, shapes=[(40, 36, 12)], contract=_contract)
    fp = max(F.fctn_footprint_bytes(S.job_params(j, "fp32")) for j in jobs)
    srv = F.fctn_server_create(max_jobs=8, mem_budget_bytes=int(fp * 1.5))   # room for one job at a time
    try:
        ids = []
        for j in jobs:
            p = S.job_params(j, "fp32")
            ids.append(F.fctn_server_submit(srv, p, j["Y"].astype(np.float32), j["mask"],
                                            [a.astype(np.float32) for a in j["init"]], 1e-4, 30))
        left = set(ids)
        waited = False
        for _ in range(200000):
            running, queued = F.fctn_server_step(srv)
            assert F.fctn_server_stats(srv)["bytes_in_use"] <= int(fp * 1.5)
            waited |= running >= 1 and queued >= 1
            for jid in list(left):
                if F.fctn_server_poll(srv, jid)["state"] == F.FCTN_JOB_DONE:
                    F.fctn_server_result(srv, jid)
                    left.discard(jid)
            if not left:
                break
        assert not left
        assert waited   # jobs were held back by the memory budget while others ran
    finally:
        F.fctn_server_destroy(srv)


def test_oversized_job_rejected_at_submit(mods):
    F, S = mods
    jobs = S.mix_jobs(1, seed=10, rate=1000.0, shapes=[(40, 36, 12)], contract=_contract)
    srv = F.fctn_server_create(max_jobs=2, mem_budget_bytes=1024)
    try:
        j = jobs[0]
        with pytest.raises(F.FctnError) as ei:
            F.fctn_server_submit(srv, S.job_params(j, "fp32"), j["Y"].astype(np.float32), j["mask"],
                                 [a.astype(np.float32) for a in j["init"]], 1e-4, 10)
        assert ei.value.code == F.FCTN_E_OOM
    finally:
        F.fctn_server_destroy(srv)


def test_failing_job_does_not_stop_the_others(mods):
    F, S = mods
    jobs = S.mix_jobs(3, seed=11, rate=1000.0, shapes=[(32, 30, 9)], contract=_contract)
    srv = F.fctn_server_create(max_jobs=3)
    try:
        ids = []
        for n, j in enumerate(jobs):
            if n == 1:   # printed Laplacian sign with a large lambda: Eq. 5 is not positive definite
                p = F.make_params(j["dims"], j["R"], lam=10.0, precision="fp32", laplacian_sign="printed")
            else:
                p = S.job_params(j, "fp32")
            ids.append(F.fctn_server_submit(srv, p, j["Y"].astype(np.float32), j["mask"],
                                            [a.astype(np.float32) for a in j["init"]], 1e-4, 30))
        states = {}
        for _ in range(200000):
            F.fctn_server_step(srv)
            states = {jid: F.fctn_server_poll(srv, jid) for jid in ids}
            if all(v["state"] in (F.FCTN_JOB_DONE, F.FCTN_JOB_FAILED) for v in states.values()):
                break
        assert states[ids[1]]["state"] == F.FCTN_JOB_FAILED
        assert states[ids[1]]["status"] == F.FCTN_E_SINGULAR
        assert states[ids[0]]["state"] == F.FCTN_JOB_DONE and states[ids[2]]["state"] == F.FCTN_JOB_DONE
    finally:
        F.fctn_server_destroy(srv)


def test_tuning_cache_per_job_class(mods):
    """The per-class tuning cache tunes each (dims, ranks, precision) class
    once, hands every job of a class the same launch shape, and a tuned mix
    still matches each job run alone with that shape."""
    F, S = mods
    jobs = S.mix_jobs(6, seed=9, rate=1000.0, shapes=SMALL[:2], contract=_contract)
    tuner = S.TuneCache(sweeps=1, candidates=(0, 96)).fill(jobs, "fp32")
    classes = {S.TuneCache.key(j, S.job_params(j, "fp32")) for j in jobs}
    assert set(tuner.table) == classes
    assert all(v in (0, 96) for v in tuner.table.values())
    for j in jobs:
        assert S.job_params(j, "fp32", tuner).tile_code == tuner.table[S.TuneCache.key(j, S.job_params(j, "fp32"))]
    mix = S.run_mix(jobs, precision="fp32", tol=1e-4, max_sweeps=30, max_jobs=3, keep_results=True,
                    arrivals=False, tuner=tuner)
    assert mix["failed"] == 0
    for j in jobs:
        p = S.job_params(j, "fp32", tuner)
        dt = F.elem_dtype(p)
        h = F.fctn_create(p)
        try:
            F.fctn_set_data(h, np.ascontiguousarray(j["Y"].astype(dt)), j["mask"].astype(np.uint8))
            F.fctn_set_factors(h, [np.ascontiguousarray(a.astype(dt)) for a in j["init"]])
            out = np.empty(j["dims"], dtype=dt)
            F.fctn_complete(h, 1e-4, 30, out)
        finally:
            F.fctn_destroy(h)
        np.testing.assert_array_equal(mix["results"][j["i"]], out)

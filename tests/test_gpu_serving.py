"""Serving loop: continuous batching of mining jobs, admission by memory."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fb():
    from paper_0905_2203_gb300 import build as b
    b.build()
    from paper_0905_2203_gb300 import binding
    return binding


def _jobs(k, n_lo=2e4, n_hi=3e5, seed=0xFE0005):
    out = []
    for spec in synth.serving_jobs(seed, n_jobs=k, n_lo=n_lo, n_hi=n_hi):
        s, cfg = synth.make_job_stream(spec)
        out.append((s, cfg))
    return out


def _levels(res, max_size):
    return [res.level(0, N) for N in range(1, max_size + 1)]


def test_results_identical_alone_and_in_the_mix(fb):
    """Every job's result through the server (jobs overlapping on the GPU,
    each at its own level) equals its result mined alone, and the oracle."""
    jobs = _jobs(8)
    srv = fb.Server(0, 0, max_jobs=4)
    ids = []
    for s, cfg in jobs:  # submitted back to back: later jobs wait for slots
        ids.append(srv.submit(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], cfg["max_size"]))
    mixed = []
    for jid, (s, cfg) in zip(ids, jobs):
        res, info = srv.wait(jid, 120000)
        assert info["finish_s"] >= info["admit_s"] >= info["submit_s"]
        assert info["n_events"] == s.n
        mixed.append(_levels(res, cfg["max_size"]))
        res.free()
    srv.close()
    ctx = fb.Context(0)
    for k, (s, cfg) in enumerate(jobs):
        st = ctx.load_stream(s.types, s.times, s.n_types)
        res = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
        alone = _levels(res, cfg["max_size"])
        res.free()
        st.free()
        assert mixed[k] == alone, k
        if s.n <= 60000:
            want = oracle.mine_levelwise(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"],
                                         cfg["max_size"])
            for N in range(1, cfg["max_size"] + 1):
                eps, counts = alone[N - 1]
                assert list(zip(eps, counts)) == want[N], (k, N)
    ctx.close()


def test_admission_under_tight_budget_and_concurrent_submitters(fb):
    """A budget that fits about one job at a time still serves every job
    correctly; submissions from several host threads."""
    jobs = _jobs(6, n_lo=3e4, n_hi=1e5, seed=77)
    srv = fb.Server(0, 96 * 1024 * 1024, max_jobs=8)
    ids = [None] * len(jobs)

    def sub(k):
        s, cfg = jobs[k]
        ids[k] = srv.submit(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], cfg["max_size"])

    th = [threading.Thread(target=sub, args=(k,)) for k in range(len(jobs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    ctx = fb.Context(0)
    for k, (s, cfg) in enumerate(jobs):
        res, info = srv.wait(ids[k], 120000)
        got = _levels(res, cfg["max_size"])
        res.free()
        st = ctx.load_stream(s.types, s.times, s.n_types)
        r2 = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
        assert got == _levels(r2, cfg["max_size"])
        r2.free()
        st.free()
    ctx.close()
    srv.close()


def test_server_errors_and_cancellation(fb):
    s, cfg = _jobs(1, n_lo=2e5, n_hi=2e5, seed=5)[0]
    srv = fb.Server(0, 64 * 1024 * 1024, max_jobs=1)
    # a job whose stream alone exceeds the budget can never be admitted
    nb = 12_000_000
    big_t = np.arange(nb, dtype=np.int32)
    big_y = (np.arange(nb) % 60).astype(np.uint16)
    with pytest.raises(fb.FemError) as e:
        srv.submit(big_y, big_t, 60, synth.BINS_4, 100, 4)
    assert e.value.status == fb.FEM_ERR_NOMEM
    with pytest.raises(fb.FemError) as e:
        srv.wait(12345, 10)
    assert e.value.status == fb.FEM_ERR_NOTFOUND
    with pytest.raises(fb.FemError) as e:
        srv.submit(s.types, s.times, s.n_types, [(5, 5)], 10, 3)
    assert e.value.status == fb.FEM_ERR_INVAL
    ids = [srv.submit(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], cfg["max_size"])
           for _ in range(3)]
    # the first finishes; destroying the server cancels the rest without hanging
    res, info = srv.wait(ids[0], 120000)
    res.free()
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 60

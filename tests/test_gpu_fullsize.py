"""Full-size parity in the launch configurations bench.py uses.

C2 (1.07M events, levels 1-6): the whole level-wise result equals the oracle
miner's.  C3 (4M events, 200k candidates of sizes 2-8, one counting call):
every one of the 200k counts equals the oracle's.  C4 (all 256 recordings,
about 2.2e8 events, mined in one call): the level-wise results of 32
recordings, the largest among them, equal the oracle miner's.  C5 (the
1e8-event stress job of the serving workload): level 1 equals the event
frequencies; 2000 random level-2 candidates and 2000 random level-3
candidates count as in the oracle and are reported frequent exactly when the
oracle's count passes the threshold; every reported frequent episode of
levels 2-4 carries the oracle's count.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def fb():
    from paper_0905_2203_gb300 import build as b
    b.build()
    from paper_0905_2203_gb300 import binding
    return binding


def _csr(eps):
    return oracle.to_csr(eps)


def test_c2_full_mining_equals_oracle(fb):
    s, cfg = synth.c2_mid()
    ctx = fb.Context(0)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    res = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
    want = oracle.mine_levelwise(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], cfg["max_size"])
    for N in range(1, cfg["max_size"] + 1):
        eps, counts = res.level(0, N)
        assert list(zip(eps, counts)) == want[N], N
    # the planted chains' 4-node prefixes are found
    found4 = {ep[0] for ep in res.level(0, 4)[0]}
    assert any(tuple(ch["neurons"][:4]) in found4 for ch in s.chains)
    res.free()
    st.free()
    ctx.close()


def test_c3_full_counting_every_candidate(fb):
    s, (offs, ct, lo, hi) = synth.c3_batched()
    assert s.n == 4_000_000 and len(offs) == 200_001
    ctx = fb.Context(0)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    got = ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
    stats = ctx.last_stats()
    assert stats["candidates_counted"] == 200_000
    want, _ = oracle.count_many(s.types, s.times, offs, ct, lo, hi)
    bad = np.nonzero(got != want.astype(np.int64))[0]
    assert bad.size == 0, (bad[:5], got[bad[:5]], want[bad[:5]])
    assert got.max() > 0
    # the same counts through the multi-recording entry point
    got_b = ctx.count_batch([st], fb.Cands(offs, ct, lo, hi), np.zeros(200_000, np.uint32)).astype(np.int64)
    assert np.array_equal(got_b, got)
    st.free()
    ctx.close()


def test_c4_all_recordings_one_call_equals_oracle_on_32(fb):
    recs = synth.c4_recordings()
    assert len(recs) == 256
    ctx = fb.Context(0)
    sts = [ctx.load_stream(s.types, s.times, s.n_types) for s, _ in recs]
    bins = recs[0][1]["bins"]
    max_size = recs[0][1]["max_size"]
    res = ctx.mine_levelwise(sts, bins, [c["threshold"] for _, c in recs], max_size)
    # the largest recording and 31 others in a seeded order
    ns = np.array([s.n for s, _ in recs])
    order = [int(i) for i in np.argsort(synth.Rng(0xC4, 1).uniform(256)) if i != int(np.argmax(ns))]
    pick = [int(np.argmax(ns))] + order[:31]
    assert ns[pick[0]] > 5_000_000
    for r in pick:
        s, cfg = recs[r]
        want = oracle.mine_levelwise(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], max_size)
        for N in range(1, max_size + 1):
            eps, counts = res.level(r, N)
            assert list(zip(eps, counts)) == want[N], (r, N)
    assert sum(len(res.level(r, 3)[0]) for r in pick) > 0
    res.free()
    for st in sts:
        st.free()
    ctx.close()


def test_c5_stress_job_sampled(fb):
    jobs = synth.serving_jobs(stress_n=100_000_000)
    job = jobs[-1]
    assert job["n"] == 100_000_000
    s, cfg = synth.make_job_stream(job)
    assert s.n > 90_000_000
    thr, bins, max_size = cfg["threshold"], cfg["bins"], cfg["max_size"]
    ctx = fb.Context(0)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    res = ctx.mine_levelwise([st], bins, [thr], max_size)
    freq = np.bincount(s.types.astype(np.int64), minlength=s.n_types)
    ftypes = [a for a in range(s.n_types) if freq[a] > thr]
    eps1, c1 = res.level(0, 1)
    assert [e[0][0] for e in eps1] == ftypes and list(c1) == [int(freq[a]) for a in ftypes]
    rng = synth.Rng(0xC5, 1)
    levels = {N: dict(zip(*res.level(0, N))) for N in range(2, max_size + 1)}
    # level 2: random candidates of the oracle's own generator
    cands2 = oracle.generate_candidates([], 2, ftypes, bins)
    pick2 = [cands2[i] for i in np.argsort(rng.uniform(len(cands2)))[:2000]]
    # level 3: random joins of the reported level-2 set (each reported count
    # is itself checked against the oracle below)
    cands3 = oracle.generate_candidates(sorted(levels[2], key=oracle.canonical_key), 3, ftypes, bins)
    pick3 = [cands3[i] for i in np.argsort(rng.uniform(max(len(cands3), 1)))[:2000]] if cands3 else []
    for N, pick in ((2, pick2), (3, pick3)):
        if not pick:
            continue
        offs, ct, lo, hi = _csr(pick)
        want, _ = oracle.count_many(s.types, s.times, offs, ct, lo, hi)
        got = ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
        assert np.array_equal(got, want.astype(np.int64)), N
        for ep, w in zip(pick, want):
            if int(w) > thr:
                assert levels[N].get(ep) == int(w), (N, ep)
            else:
                assert ep not in levels[N], (N, ep)
    # every reported frequent episode of levels 2-4 (at most 1500 per level)
    for N in range(2, min(max_size, 4) + 1):
        eps = sorted(levels[N], key=oracle.canonical_key)
        if not eps:
            continue
        eps = [eps[i] for i in np.argsort(rng.uniform(len(eps)))[:1500]]
        offs, ct, lo, hi = _csr(eps)
        want, _ = oracle.count_many(s.types, s.times, offs, ct, lo, hi)
        assert [levels[N][e] for e in eps] == [int(w) for w in want], N
        assert all(int(w) > thr for w in want)
    assert len(levels[2]) > 0
    res.free()
    st.free()
    ctx.close()

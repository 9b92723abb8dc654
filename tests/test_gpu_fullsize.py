"""Full-size parity in the launch configuration bench.py uses.

C2 (1.07M events, levels 1-6): the whole level-wise result equals the oracle
miner's.  C3 (4M events, 200k candidates of sizes 2-8): every count comes from
one counting call; a random sample of 1500 is recounted by the oracle, and
properties that hold for every candidate are checked on all of them.
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


def test_c2_full_mining_equals_oracle(fb):
    s, cfg = synth.c2_mid()
    ctx = fb.Context(0)
    ctx.set_tuning(autotune=1)
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


def test_c3_full_counting_sampled(fb):
    s, (offs, ct, lo, hi) = synth.c3_batched()
    assert s.n == 4_000_000 and len(offs) == 200_001
    ctx = fb.Context(0)
    ctx.set_tuning(autotune=1)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    got = ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
    stats = ctx.last_stats()
    assert stats["candidates_counted"] == 200_000
    r = synth.Rng(33, 1)
    pick = np.unique(r.integers(0, 199_999, 1500))
    sub_offs = [0]
    st_, sl, sh = [], [], []
    for c in pick:
        a, b = int(offs[c]), int(offs[c + 1])
        st_.extend(ct[a:b]); sl.extend(lo[a - c:b - c - 1]); sh.extend(hi[a - c:b - c - 1])
        sub_offs.append(sub_offs[-1] + b - a)
    want, _ = oracle.count_many(s.types, s.times, np.array(sub_offs), np.array(st_, np.uint16),
                                np.array(sl, np.int32), np.array(sh, np.int32))
    assert np.array_equal(got[pick], want.astype(np.int64))
    # every count is bounded by its rarest type's frequency
    freq = np.bincount(s.types.astype(np.int64), minlength=60)
    minf = np.minimum.reduceat(freq[ct.astype(np.int64)], offs[:-1])
    assert np.all(got <= minf)
    assert got.max() > 0
    # the same counts through the multi-recording entry point
    got_b = ctx.count_batch([st], fb.Cands(offs, ct, lo, hi), np.zeros(200_000, np.uint32)).astype(np.int64)
    assert np.array_equal(got_b, got)
    st.free()
    ctx.close()

"""The timeout path of the tiled kernel's shared-memory pipeline.

Every mbarrier wait of the tiled kernel is bounded.  fem_tuning.wait_polls
shortens the pipeline waits to a few non-blocking polls, so that they run out
while the bulk copies they wait for are still in flight: the kernel then
records the timeout, waits for its own copies with the default limit and
returns, and the call reports FEM_ERR_TIMEOUT.  No fault is involved; the
context must stay usable and the next call with the default limit must give
the oracle's counts.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_short_wait_limit_reports_timeout_and_context_recovers():
    pytest.importorskip("torch")
    from paper_0905_2203_gb300 import build
    build.build()
    from paper_0905_2203_gb300 import binding as fb

    s = synth.bursty_60(0xFE0103, 200_000)
    offs, ct, lo, hi = synth.random_candidates(0xFE0103, 256, 60, 2, 5, synth.BINS_4, s.chains, 0.1)
    ref, _ = oracle.count_many(s.types, s.times, offs, ct, lo, hi)
    ref = ref.astype(np.int64)
    ctx = fb.Context(0)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    cands = fb.Cands(offs, ct, lo, hi)
    ctx.set_tuning(kernel=1, segments=16, wait_polls=1)
    seen = 0
    for _ in range(6):
        try:
            got = ctx.count_episodes(st, cands).astype(np.int64)
        except fb.FemError as e:
            assert e.status == fb.FEM_ERR_TIMEOUT, e
            seen += 1
            continue
        # a call whose waits all succeeded is exact
        assert np.array_equal(got, ref)
    assert seen > 0, "no pipeline wait ran out with a one-poll limit"
    # default limits again: the same context counts exactly
    ctx.set_tuning(kernel=1, segments=16)
    assert np.array_equal(ctx.count_episodes(st, cands).astype(np.int64), ref)
    ctx.reset_tuning()
    assert np.array_equal(ctx.count_episodes(st, cands).astype(np.int64), ref)
    st.free()
    ctx.close()

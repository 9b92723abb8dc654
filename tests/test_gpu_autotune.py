"""Autotuner: timed launch configurations per workload signature, cached."""
import json

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


def test_autotune_exact_cached_and_reused(fb, tmp_path):
    s = synth.bursty_60(0xFE0003, 200_000)
    offs, ct, lo, hi = synth.random_candidates(0xFE0003, 4000, 60, 2, 8, synth.BINS_4, s.chains, 0.05)
    want, _ = oracle.count_many(s.types, s.times, offs, ct, lo, hi)
    path = tmp_path / "tune.json"
    ctx = fb.Context(0)
    ctx.set_autotune_cache(path)
    ctx.set_tuning(autotune=1)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    got = ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi))
    assert np.array_equal(got.astype(np.uint64), want)
    table = json.loads(path.read_text())
    assert len(table) >= 1
    for k, (lanes, tile, mult, kernel) in table.items():
        assert lanes % 32 == 0 and 32 <= lanes <= 256 and tile % 256 == 0 and mult > 0 and kernel in (1, 2, 3)
    # a fresh context picks the cached choices up (no further entries needed)
    ctx2 = fb.Context(0)
    ctx2.set_autotune_cache(path)
    st2 = ctx2.load_stream(s.types, s.times, s.n_types)
    got2 = ctx2.count_episodes(st2, fb.Cands(offs, ct, lo, hi))
    assert np.array_equal(got2.astype(np.uint64), want)
    assert json.loads(path.read_text()) == table
    st.free(); st2.free(); ctx.close(); ctx2.close()


def test_autotune_cache_rejects_malformed_file(fb, tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text('{"n0.r0.c5.e20.m1": [33, 1024, 1.0]}')
    ctx = fb.Context(0)
    with pytest.raises(fb.FemError) as e:
        ctx.set_autotune_cache(bad)
    assert e.value.status == fb.FEM_ERR_INVAL
    ctx.close()

"""The allocation-free counting entry point agrees with fem_count_episodes and
with the oracle.

fem_count_episodes_noalloc is for callers that cannot allocate device memory
when they need a count (allocator callbacks, fully reserved devices,
real-time loops).  It runs on caller-owned device buffers plus the library's
fixed static scratch array.  This file sorts last so that, in a run that stops
at the first failure, every other test has already run; it also passes on its
own in a fresh process.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _lib():
    torch = pytest.importorskip("torch")
    from paper_0905_2203_gb300 import build
    build.build()
    from paper_0905_2203_gb300 import binding as fb
    return torch, fb


def _noalloc(torch, fb, d_types, d_times, offs, ct, lo, hi):
    dev = d_types.device
    out = torch.full((len(offs) - 1,), -1, dtype=torch.int32, device=dev)
    fb.count_episodes_noalloc(d_types, d_times, torch.from_numpy(offs).to(dev),
                              torch.from_numpy(ct.view(np.int16)).to(dev), torch.from_numpy(lo).to(dev),
                              torch.from_numpy(hi).to(dev), out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).astype(np.int64)


def test_noalloc_matches_count_episodes_on_two_calls():
    torch, fb = _lib()
    dev = torch.device("cuda:0")
    ctx = fb.Context(0)
    s, _ = synth.c1_tiny()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    d_types = torch.from_numpy(s.types.view(np.int16)).to(dev)
    d_times = torch.from_numpy(s.times).to(dev)
    # two calls in a row with different candidate sets: the shared scratch
    # array keeps the previous call's contents, which must not leak
    for seed, n_cand, sizes in ((31, 900, (2, 6)), (32, 2500, (2, 4))):
        offs, ct, lo, hi = synth.random_candidates(seed, n_cand, s.n_types, sizes[0], sizes[1],
                                                   [(0, 5), (2, 7), (0, 12)], s.chains, 0.3)
        want = ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
        ref, _ = oracle.count_many(s.types, s.times, offs, ct, lo, hi)
        got = _noalloc(torch, fb, d_types, d_times, offs, ct, lo, hi)
        assert np.array_equal(got, want), seed
        assert np.array_equal(got, ref.astype(np.int64)), seed
        assert want.max() > 0
    st.free()
    ctx.close()


def test_noalloc_rejects_offsets_not_starting_at_zero():
    torch, fb = _lib()
    dev = torch.device("cuda:0")
    s, _ = synth.c1_tiny()
    d_types = torch.from_numpy(s.types.view(np.int16)).to(dev)
    d_times = torch.from_numpy(s.times).to(dev)
    offs, ct, lo, hi = synth.random_candidates(33, 64, s.n_types, 2, 3, [(0, 5)])
    # a slice of a larger set: offs[0] = 2 with buffers sized for offs[-1]
    shifted = offs + 2
    ct2 = np.concatenate([np.zeros(2, np.uint16), ct])
    lo2 = np.concatenate([np.zeros(2, np.int32), lo])
    hi2 = np.concatenate([np.ones(2, np.int32), hi])
    with pytest.raises(fb.FemError) as e:
        _noalloc(torch, fb, d_types, d_times, shifted, ct2, lo2, hi2)
    assert e.value.status == fb.FEM_ERR_INVAL


def test_noalloc_ring_overflow_is_reported():
    """A burst longer than the per-node ring (32 timestamps) inside the lower
    bound of an edge: 40 A events on consecutive ticks and A -(40,100]-> B.
    The call must return FEM_ERR_NOMEM (never a wrong count); the library's
    allocating entry point still counts it exactly."""
    torch, fb = _lib()
    dev = torch.device("cuda:0")
    ty = np.array([0] * 40 + [1] * 5, np.uint16)
    tm = np.array(list(range(40)) + [60, 75, 90, 130, 200], np.int32)
    offs = np.array([0, 2], np.int64)
    ct = np.array([0, 1], np.uint16)
    lo = np.array([40], np.int32)
    hi = np.array([100], np.int32)
    d_types = torch.from_numpy(ty.view(np.int16)).to(dev)
    d_times = torch.from_numpy(tm).to(dev)
    with pytest.raises(fb.FemError) as e:
        _noalloc(torch, fb, d_types, d_times, offs, ct, lo, hi)
    assert e.value.status == fb.FEM_ERR_NOMEM
    ref, _ = oracle.count_many(ty, tm, offs, ct, lo, hi)
    ctx = fb.Context(0)
    st = ctx.load_stream(ty, tm, 2)
    got = ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi)).astype(np.int64)
    assert np.array_equal(got, ref.astype(np.int64)) and got[0] > 0
    st.free()
    ctx.close()
    # the array is shared: a good call right after the refused one is exact
    s, _ = synth.c1_tiny()
    offs, ct, lo, hi = synth.random_candidates(34, 300, s.n_types, 2, 5, [(0, 5), (1, 9)], s.chains, 0.3)
    got = _noalloc(torch, fb, torch.from_numpy(s.types.view(np.int16)).to(dev), torch.from_numpy(s.times).to(dev),
                   offs, ct, lo, hi)
    ref, _ = oracle.count_many(s.types, s.times, offs, ct, lo, hi)
    assert np.array_equal(got, ref.astype(np.int64))

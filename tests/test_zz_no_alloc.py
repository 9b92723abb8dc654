"""The allocation-free counting entry point agrees with fem_count_episodes.

fem_count_episodes_noalloc is for callers that cannot allocate device memory
when they need a count (allocator callbacks, fully reserved devices,
real-time loops).  It runs on caller-owned device buffers plus the library's
fixed static scratch array.  This file sorts last so that, in a run that stops
at the first failure, every other test has already run; it also passes on its
own in a fresh process.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_count_episodes_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_0905_2203_gb300 import build
    build.build()
    from paper_0905_2203_gb300 import binding as fb

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
        out = torch.full((n_cand,), -1, dtype=torch.int32, device=dev)
        fb.count_episodes_noalloc(d_types, d_times, torch.from_numpy(offs).to(dev),
                                  torch.from_numpy(ct.view(np.int16)).to(dev), torch.from_numpy(lo).to(dev),
                                  torch.from_numpy(hi).to(dev), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.array_equal(got, want), seed
        assert want.max() > 0
    st.free()
    ctx.close()

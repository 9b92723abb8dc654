"""The rule behind counting over a growing stream, checked on the CPU.

A session keeps per episode the count and the time of the last end that the
greedy of Algorithm 1 kept, plus the events at or after t_last - S (S = the
largest sum of upper bounds).  Each append recounts only the tail followed by
the new events, takes ends among the new events only, and starts the greedy
from the stored end.  This test runs that rule in plain Python (latest-start
values per end event, then the greedy) on random tiny streams cut into random
chunks, cuts between equal times included, and checks every prefix against
the oracle's state-machine count (O1), and that no end inside the retained
tail could be kept again.  It checks the reading, not the CUDA code (the GPU
tests do that through the C ABI).
"""
import numpy as np
import pytest

import oracle
import synth


def latest_starts(ty, tm, E, lo, hi):
    """L(j) for every event j of type E[-1] (None when no occurrence ends at
    j), by the latest-start recursion over the given events only."""
    n, N = len(ty), len(E)
    L = [tm[j] if ty[j] == E[0] else None for j in range(n)]
    for k in range(1, N):
        nxt = [None] * n
        for j in range(n):
            if ty[j] != E[k]:
                continue
            best = None
            for i in range(n):
                if ty[i] == E[k - 1] and L[i] is not None and lo[k - 1] < tm[j] - tm[i] <= hi[k - 1]:
                    best = L[i] if best is None else max(best, L[i])
            nxt[j] = best
        L = nxt
    return L


def session_counts(ty, tm, E, lo, hi, cuts):
    """Counts after each chunk, by the session rule."""
    span = sum(hi)
    tail_ty, tail_tm = [], []
    count, last_end, out = 0, None, []
    for a, b in zip(cuts[:-1], cuts[1:]):
        buf_ty = tail_ty + [int(x) for x in ty[a:b]]
        buf_tm = tail_tm + [int(x) for x in tm[a:b]]
        n_old = len(tail_ty)
        if len(buf_ty):
            L = latest_starts(buf_ty, buf_tm, E, lo, hi)
            # ends inside the retained tail were decided before: the greedy
            # could not keep any of them again
            assert all(L[j] is None or (last_end is not None and L[j] <= last_end) for j in range(n_old))
            for j in range(n_old, len(buf_ty)):  # buffer is in time order
                if L[j] is not None and (last_end is None or L[j] > last_end):
                    count += 1
                    last_end = buf_tm[j]
            cut = buf_tm[-1] - span
            keep = [i for i in range(len(buf_tm)) if buf_tm[i] >= cut]
            tail_ty = [buf_ty[i] for i in keep]
            tail_tm = [buf_tm[i] for i in keep]
        out.append(count)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_session_rule_equals_prefix_counts(seed):
    r = synth.Rng(0x5E5, seed)
    for trial in range(25):
        n_types = 3
        ty, tm = synth.tiny_random_stream(seed * 100 + trial, 60, n_types, 90, sid=7)
        N = int(r.integers(1, 4, 1)[0])
        E = [int(x) for x in r.integers(0, n_types - 1, N)]
        lo = [int(x) for x in r.integers(0, 3, N - 1)]
        hi = [l + int(x) for l, x in zip(lo, r.integers(1, 8, N - 1))]
        cuts = np.concatenate([[0], np.sort(r.integers(0, len(ty), 5)), [len(ty)]])
        got = session_counts(ty, tm, E, lo, hi, cuts)
        want = [oracle.count_fsm(ty[:b], tm[:b], E, lo, hi) for b in cuts[1:]]
        assert got == want, (seed, trial, E, lo, hi, list(cuts), got, want)

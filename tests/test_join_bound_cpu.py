"""The level-3 join bound as a statement about counts (runs without a GPU).

For a 3-node episode A -(l1,h1]-> B -(l2,h2]-> C, every occurrence passes
through a B event that has an A event inside (l1, h1] before it and a C
event inside (l2, h2] after it, and non-overlapped occurrences use distinct B
events; so the count is at most the number of B events with both.  The
mining graph drops a level-3 candidate when this number is at or below the
threshold.  Here the bound is written out from its definition over the
events (plain loops), and checked against the oracle's exact count: never
below it on random tiny streams with many equal times, equal to it where
every B event is used, and zero where an edge cannot be met.
"""
import numpy as np

import oracle
import synth


def join_ub(ty, tm, E, lo, hi):
    """#{ B events with an A event at distance in (lo[0], hi[0]] before and a
    C event at distance in (lo[1], hi[1]] after }."""
    A, B, C = E
    ta = tm[ty == A]
    tb = tm[ty == B]
    tc = tm[ty == C]
    n = 0
    for t in tb:
        d_before = t - ta
        d_after = tc - t
        if np.any((d_before > lo[0]) & (d_before <= hi[0])) and np.any((d_after > lo[1]) & (d_after <= hi[1])):
            n += 1
    return n


def test_join_bound_never_below_the_count():
    r = synth.Rng(0x3B0, 1)
    seen_tight = 0
    for trial in range(1500):
        n_types = int(r.integers(3, 6, 1)[0])
        n = int(r.integers(5, 120, 1)[0])
        ty, tm = synth.tiny_random_stream(7000 + trial, n, n_types, int(r.integers(n // 3 + 3, 3 * n, 1)[0]))
        ty = ty.astype(np.int64)
        tm = tm.astype(np.int64)
        E = [int(x) for x in r.integers(0, n_types - 1, 3)]
        if len(set(E)) < 3:
            continue
        lo = [int(x) for x in r.integers(0, 4, 2)]
        hi = [lo[k] + int(r.integers(1, 8, 1)[0]) for k in range(2)]
        ub = join_ub(ty, tm, E, lo, hi)
        c = oracle.count_fsm(ty.astype(np.uint16), tm.astype(np.int32), np.array(E, np.uint16),
                             np.array(lo, np.int32), np.array(hi, np.int32))
        assert ub >= c, (trial, E, lo, hi, ub, c)
        seen_tight += ub == c and c > 0
    assert seen_tight > 0


def test_join_bound_tight_on_a_clean_chain_and_zero_on_an_unmet_edge():
    # A at 10k, B at 10k+3, C at 10k+7 for k = 0..19: every B event starts and
    # ends exactly one occurrence, so bound = count = 20
    ty = np.array([0, 1, 2] * 20, np.uint16)
    tm = np.array([t for k in range(20) for t in (10 * k, 10 * k + 3, 10 * k + 7)], np.int32)
    E, lo, hi = [0, 1, 2], [2, 3], [4, 5]
    c = oracle.count_fsm(ty, tm, np.array(E, np.uint16), np.array(lo, np.int32), np.array(hi, np.int32))
    assert join_ub(ty.astype(np.int64), tm.astype(np.int64), E, lo, hi) == c == 20
    # the second edge asks for C more than 4 ticks after B: never met
    lo2, hi2 = [2, 4], [4, 5]
    c2 = oracle.count_fsm(ty, tm, np.array(E, np.uint16), np.array(lo2, np.int32), np.array(hi2, np.int32))
    assert join_ub(ty.astype(np.int64), tm.astype(np.int64), E, lo2, hi2) == c2 == 0

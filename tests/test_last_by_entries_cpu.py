"""The argument behind driving the last node by entries (runs without a GPU).

With L_k(j) the latest start of a partial occurrence of nodes 1..k ending at
event j (L_1(j) = t_j, L_k(j) = max L_{k-1}(i) over i with
lo < t_j - t_i <= hi), the count is Algorithm 1 over the last node's valid
ends: select an end when its latest start is after the previous selected
end.  The ends served by entry i of node N-1 (the newest one older than
t - lo) lie in (T_i + lo, T_{i+1} + lo] and all carry L_i; the claim is that
only the first of them can be selected.  Here both forms are written out
from these definitions in plain loops and checked against the oracle's
count: all valid ends, and one end per entry (the first event after
T_i + lo, kept when it lies before T_{i+1} + lo and within T_i + hi).
"""
import bisect

import numpy as np

import oracle
import synth


def entries(ty, tm, E, lo, hi):
    """(T, L) of the last inner node, in time order (node 0: L = T)."""
    T = [int(t) for t, y in zip(tm, ty) if y == E[0]]
    L = list(T)
    for k in range(1, len(E) - 1):
        nT, nL = [], []
        for t, y in zip(tm, ty):
            if y != E[k]:
                continue
            i = bisect.bisect_left(T, int(t) - lo[k - 1]) - 1  # newest entry with T < t - lo
            if i >= 0 and T[i] >= int(t) - hi[k - 1]:
                nT.append(int(t))
                nL.append(L[i])
        T, L = nT, nL
    return T, L


def greedy(ends):
    prev, n = -1, 0
    for t, l in ends:
        if l > prev:
            n += 1
            prev = t
    return n


def ends_all(ty, tm, E, lo, hi):
    T, L = entries(ty, tm, E, lo, hi)
    out = []
    for t, y in zip(tm, ty):
        if y != E[-1]:
            continue
        i = bisect.bisect_left(T, int(t) - lo[-1]) - 1
        if i >= 0 and T[i] >= int(t) - hi[-1]:
            out.append((int(t), L[i]))
    return out


def ends_first_per_entry(ty, tm, E, lo, hi):
    T, L = entries(ty, tm, E, lo, hi)
    C = [int(t) for t, y in zip(tm, ty) if y == E[-1]]
    out = []
    for i in range(len(T)):
        p = bisect.bisect_right(C, T[i] + lo[-1])  # first event after T_i + lo
        if p == len(C):
            continue
        e = C[p]
        owned = i + 1 >= len(T) or e <= T[i + 1] + lo[-1]
        if owned and e <= T[i] + hi[-1]:
            out.append((e, L[i]))
    return out


def test_first_end_per_entry_gives_the_count():
    r = synth.Rng(0x1E7, 1)
    for trial in range(1500):
        n_types = int(r.integers(2, 6, 1)[0])
        n = int(r.integers(4, 120, 1)[0])
        ty, tm = synth.tiny_random_stream(9000 + trial, n, n_types, int(r.integers(n // 3 + 3, 3 * n, 1)[0]))
        N = int(r.integers(2, 5, 1)[0])
        E = [int(x) for x in r.integers(0, n_types - 1, N)]
        lo = [int(x) for x in r.integers(0, 4, N - 1)]
        hi = [lo[k] + int(r.integers(1, 9, 1)[0]) for k in range(N - 1)]
        want = oracle.count_fsm(ty, tm, np.array(E, np.uint16), np.array(lo, np.int32), np.array(hi, np.int32))
        all_ends = ends_all(ty, tm, E, lo, hi)
        first = ends_first_per_entry(ty, tm, E, lo, hi)
        assert greedy(all_ends) == want, (trial, E, lo, hi)
        assert greedy(first) == want, (trial, E, lo, hi)
        # the first ends are a subset of the valid ends, in time order
        assert set(first) <= set(all_ends)
        assert [t for t, _ in first] == sorted(t for t, _ in first)

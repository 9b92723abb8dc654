"""Coarse-tick upper bound on the non-overlapped count (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product library never does.

Definition (a bound used for pruning, "Temporal Data Mining": a candidate
whose count cannot pass the threshold is dropped without counting; the
paper's own pruning is anti-monotone, this bound is a cheaper
over-approximation of the count).  Cut time into ticks of w units,
tick(t) = floor(t / w).  An edge with interval (lo, hi] between events at t
and t' (lo < t' - t <= hi) joins ticks whose difference lies in
[dlo, dhi] = [floor((lo + 1) / w), floor((hi + w - 1) / w)].  Let T_a be the
set of ticks holding a type-a event, M_1 = T_{E_1} and
M_{k+1} = { u in T_{E_{k+1}} : u - v in [dlo_k, dhi_k] for some v in M_k }.
Then

    ub(alpha, w) = number of type-E_N events whose tick lies in M_N.

Every occurrence maps to a chain of ticks, so every event that ends an
occurrence is counted; non-overlapped occurrences end at distinct events, so
ub >= count.  With w = 1 the ticks are the times and ub is exactly the
number of events that end at least one occurrence.

``mutant`` plants a mistake for the pin tests (0 = none): 1 = upper tick
offset floor(hi / w) (no round-up), 2 = lower tick offset floor(lo / w) + 1,
3 = ticks counted instead of events, 4 = the intermediate nodes' types
ignored (M_{k+1} dilated from M_k without intersecting T_{E_{k+1}} for
k + 1 < N).
"""
from __future__ import annotations

import numpy as np


def tick_offsets(lo: int, hi: int, w: int, mutant: int = 0) -> tuple[int, int]:
    """[dlo, dhi]: the tick differences an edge (lo, hi] can produce."""
    dlo = (lo + 1) // w
    dhi = (hi + w - 1) // w
    if mutant == 1:
        dhi = hi // w
    if mutant == 2:
        dlo = lo // w + 1
    return dlo, dhi


def coarse_ub(types, times, E, lo, hi, w: int, mutant: int = 0) -> int:
    """ub(alpha, w) for one episode alpha = (E, lo, hi) over one stream."""
    types = np.asarray(types, dtype=np.int64)
    times = np.asarray(times, dtype=np.int64)
    assert w >= 1
    N = len(E)
    ticks_of = {}
    for a in set(int(x) for x in E):
        ticks_of[a] = set(int(t) // w for t in times[types == a])
    M = set(ticks_of[int(E[0])])
    for k in range(N - 1):
        dlo, dhi = tick_offsets(int(lo[k]), int(hi[k]), w, mutant)
        reach = set()
        for v in M:
            for d in range(dlo, dhi + 1):
                reach.add(v + d)
        if mutant == 4 and k + 2 < N:
            M = reach
        else:
            M = reach & ticks_of[int(E[k + 1])]
    end_ticks = [int(t) // w for t in times[types == int(E[-1])]]
    if mutant == 3:
        return len(set(u for u in end_ticks if u in M))
    return sum(1 for u in end_ticks if u in M)


def coarse_ub_many(types, times, offs, ctypes_, lo, hi, w: int, mutant: int = 0) -> np.ndarray:
    """coarse_ub of every candidate of a CSR set (edge arrays as in fem_cands)."""
    offs = np.asarray(offs, dtype=np.int64)
    out = np.zeros(len(offs) - 1, dtype=np.int64)
    for c in range(len(offs) - 1):
        o0, o1 = int(offs[c]), int(offs[c + 1])
        e0 = o0 - c
        E = [int(x) for x in ctypes_[o0:o1]]
        out[c] = coarse_ub(types, times, E, lo[e0:e0 + len(E) - 1], hi[e0:e0 + len(E) - 1], w, mutant)
    return out


def default_tick(hi_max: int) -> int:
    """The smallest w whose upper tick offset floor((hi + w - 1) / w) stays
    <= 31 for every hi <= hi_max (that holds exactly when hi <= 31 w)."""
    return max(1, -(-hi_max // 31))

"""Checks that pin the CPU oracle to facts outside itself.

Each check returns a list of failure strings (empty = pass) so that the same
suite serves the plain pin tests and the planted-mistake (mutant) tests.
What pins what:
  * hand-derived golden cases (tests/golden/*.case)          -> O1, O2, O3
  * O3 (enumeration + exhaustive search, the definition)     -> O1, O2
  * closed forms: K separated copies, periodic streams        -> O1, O2
  * exhaustive interval optimum (textbook)                    -> Algorithm 1
  * invariants: 1-node count = frequency, prefix/suffix
    anti-monotonicity, count <= min frequency, widening an
    interval never lowers the count, tie-order invariance     -> O1, O2
"""
import numpy as np

import oracle
import synth
from golden_io import all_cases


def _counters(mutant):
    return {
        "fsm": lambda ty, tm, E, lo, hi: oracle.count_fsm(ty, tm, E, lo, hi, mutant=mutant),
        "dp": lambda ty, tm, E, lo, hi: oracle.count_dp(ty, tm, E, lo, hi, mutant=mutant),
    }


def check_golden(mutant=0):
    fails = []
    for name, ty, tm, (E, lo, hi), expect in all_cases():
        for cname, f in _counters(mutant).items():
            got = f(ty, tm, E, lo, hi)
            if got != expect:
                fails.append(f"{name}: {cname} {got} != {expect}")
        if mutant == 0:
            got = oracle.count_brute(ty, tm, E, lo, hi)
            if got != expect:
                fails.append(f"{name}: brute {got} != {expect}")
    return fails


def random_episode(r, n_types, N, max_lo=3, max_span=5):
    E = r.integers(0, n_types - 1, N).tolist()
    lo = r.integers(0, max_lo, N - 1).tolist()
    hi = [l + int(d) for l, d in zip(lo, r.integers(1, max_span, N - 1))]
    return E, lo, hi


def check_vs_brute(mutant=0, trials=1500, seed=1):
    """O1 and O2 against O3 on many tiny random streams with frequent ties,
    repeated types, zero lower bounds and events at t = 0."""
    fails = []
    r = synth.Rng(seed, 5)
    cnt = _counters(mutant)
    for k in range(trials):
        n_types = int(r.integers(1, 3, 1)[0])
        n = int(r.integers(0, 12, 1)[0])
        ty, tm = synth.tiny_random_stream(seed * 100003 + k, n, n_types, int(r.integers(3, 14, 1)[0]))
        N = int(r.integers(1, 4, 1)[0])
        E, lo, hi = random_episode(r, n_types, N)
        want = oracle.count_brute(ty, tm, E, lo, hi)
        for cname, f in cnt.items():
            got = f(ty, tm, E, lo, hi)
            if got != want:
                fails.append(f"trial {k}: {cname} {got} != brute {want} "
                             f"E={E} lo={lo} hi={hi} ty={ty.tolist()} tm={tm.tolist()}")
                if len(fails) > 5:
                    return fails
    return fails


def check_closed_forms(mutant=0):
    fails = []
    cnt = _counters(mutant)
    # K well-separated clean copies of a 4-node chain in an otherwise empty stream.
    E, lo, hi = [3, 1, 4, 2], [0, 5, 2], [4, 9, 6]
    gaps = [3, 7, 5]
    for K in (0, 1, 7, 40):
        ty, tm = [], []
        for k in range(K):
            t = 1000 * k
            ty.append(E[0]); tm.append(t)
            for g, e in zip(gaps, E[1:]):
                t += g
                ty.append(e); tm.append(t)
        ty = np.array(ty, np.uint16); tm = np.array(tm, np.int32)
        for cname, f in cnt.items():
            got = f(ty, tm, E, lo, hi)
            if got != K:
                fails.append(f"copies K={K}: {cname} {got}")
    # Periodic stream: A at kP, B at kP + d, k = 0..M-1, P > hi.  A -(l,h]-> B
    # occurs once per period iff l < d <= h, and occurrences of different
    # periods are disjoint -> count M or 0.
    P, M = 50, 30
    for d in (1, 4, 5, 6, 9):
        ty = np.array([0, 1] * M, np.uint16)
        tm = np.array([v for k in range(M) for v in (k * P, k * P + d)], np.int32)
        for (l, h) in ((0, 5), (4, 9), (5, 6), (3, 4)):
            want = M if l < d <= h else 0
            for cname, f in cnt.items():
                got = f(ty, tm, [0, 1], [l], [h])
                if got != want:
                    fails.append(f"periodic d={d} ({l},{h}]: {cname} {got} != {want}")
    # Periodic with two B's per period inside the window: still one per period.
    ty = np.array([0, 1, 1] * M, np.uint16)
    tm = np.array([v for k in range(M) for v in (k * P, k * P + 2, k * P + 3)], np.int32)
    for cname, f in cnt.items():
        got = f(ty, tm, [0, 1], [0], [5])
        if got != M:
            fails.append(f"periodic double-B: {cname} {got} != {M}")
    # Dense periodic: A at every even tick, B at every odd tick, (0,1]:
    # occurrence (2k, 2k+1) for every k; disjoint -> one per pair.
    T = 60
    ty = np.array([t % 2 for t in range(T)], np.uint16)
    tm = np.arange(T, dtype=np.int32)
    for cname, f in cnt.items():
        got = f(ty, tm, [0, 1], [0], [1])
        if got != T // 2:
            fails.append(f"dense alternating: {cname} {got} != {T // 2}")
    # Only the first N-1 types present -> 0.
    ty = np.array([0, 1, 2] * 10, np.uint16)
    tm = np.arange(30, dtype=np.int32)
    for cname, f in cnt.items():
        got = f(ty, tm, [0, 1, 2, 3], [0, 0, 0], [9, 9, 9])
        if got != 0:
            fails.append(f"missing last type: {cname} {got}")
    return fails


def check_invariants(mutant=0, trials=150, seed=3):
    fails = []
    r = synth.Rng(seed, 9)
    cnt = _counters(mutant)
    for k in range(trials):
        n_types = int(r.integers(2, 5, 1)[0])
        ty, tm = synth.tiny_random_stream(seed * 7 + k, int(r.integers(20, 200, 1)[0]), n_types,
                                          int(r.integers(20, 300, 1)[0]))
        freq = np.bincount(ty.astype(np.int64), minlength=n_types)
        N = int(r.integers(2, 4, 1)[0])
        E, lo, hi = random_episode(r, n_types, N, max_lo=6, max_span=12)
        for cname, f in cnt.items():
            c = f(ty, tm, E, lo, hi)
            # 1-node count = frequency (distinct (type,time) events)
            for a in range(n_types):
                c1 = f(ty, tm, [a], [], [])
                if c1 != freq[a]:
                    fails.append(f"inv {k}: {cname} 1-node {a} {c1} != freq {freq[a]}")
            cp = f(ty, tm, E[:-1], lo[:-1], hi[:-1])
            cs = f(ty, tm, E[1:], lo[1:], hi[1:])
            if c > cp or c > cs:
                fails.append(f"inv {k}: {cname} count {c} > prefix {cp} or suffix {cs}")
            if c > min(freq[e] for e in E):
                fails.append(f"inv {k}: {cname} count {c} > min frequency")
            # widening every interval (lo -> 0, hi -> hi+3) never lowers the count
            cw = f(ty, tm, E, [0] * len(lo), [h + 3 for h in hi])
            if cw < c:
                fails.append(f"inv {k}: {cname} widened {cw} < {c}")
            # permuting events of equal time leaves the count unchanged
            tie = synth.Rng(seed * 11 + k, 1).uniform(len(tm))
            order = np.lexsort((tie, tm))
            c2 = f(ty[order], tm[order], E, lo, hi)
            if c2 != c:
                fails.append(f"inv {k}: {cname} tie order {c2} != {c}")
        if len(fails) > 5:
            break
    return fails


def check_fsm_vs_dp_medium(mutant=0, trials=40, seed=5):
    """O1 == O2 on medium streams (brute force is out of reach there)."""
    fails = []
    r = synth.Rng(seed, 13)
    for k in range(trials):
        n_types = int(r.integers(2, 6, 1)[0])
        ty, tm = synth.tiny_random_stream(seed * 13 + k, int(r.integers(200, 3000, 1)[0]), n_types,
                                          int(r.integers(300, 3000, 1)[0]))
        N = int(r.integers(2, 5, 1)[0])
        E, lo, hi = random_episode(r, n_types, N, max_lo=8, max_span=15)
        a = oracle.count_fsm(ty, tm, E, lo, hi, mutant=mutant)
        b = oracle.count_dp(ty, tm, E, lo, hi, mutant=mutant)
        if a != b:
            fails.append(f"medium {k}: fsm {a} != dp {b}")
    return fails


def run_all(mutant):
    fails = []
    for chk in (check_golden, check_closed_forms, check_vs_brute, check_invariants,
                check_fsm_vs_dp_medium):
        fails += chk(mutant)
        if fails:
            break
    return fails

"""Pins of the CPU oracle (runs without a GPU)."""
import numpy as np
import pytest

import oracle
import synth
import oracle_pinsuite as ps
from golden_io import all_cases


def test_golden_cases_hand_derived():
    assert len(all_cases()) >= 10
    assert ps.check_golden(0) == []


def test_closed_forms():
    assert ps.check_closed_forms(0) == []


def test_fsm_and_dp_equal_bruteforce_on_tiny_streams():
    assert ps.check_vs_brute(0, trials=3000, seed=1) == []


def test_invariants():
    assert ps.check_invariants(0) == []


def test_fsm_equals_dp_on_medium_streams():
    assert ps.check_fsm_vs_dp_medium(0) == []


def test_algorithm1_greedy_is_optimal_on_random_intervals():
    """Algorithm 1 (sorted by end, select when start > previous end) equals the
    exhaustive largest pairwise non-overlapped subset (interval scheduling)."""
    r = synth.Rng(17, 1)
    for k in range(2000):
        m = int(r.integers(0, 14, 1)[0])
        s = r.integers(-5, 30, m)
        e = s + r.integers(0, 8, m)
        order = np.lexsort((s, e))
        g = oracle.greedy_sorted(s[order], e[order])
        b = oracle.intervals_brute(s, e)
        assert g == b, (s.tolist(), e.tolist(), g, b)


def test_count_many_matches_single_calls_and_threads():
    s, cfg = synth.c1_tiny()
    offs, ct, lo, hi = synth.random_candidates(3, 300, 32, 2, 4, [(0, 5), (2, 7)])
    c1, used1 = oracle.count_many(s.types, s.times, offs, ct, lo, hi, threads=1)
    c4, used4 = oracle.count_many(s.types, s.times, offs, ct, lo, hi, threads=4)
    cdp, _ = oracle.count_many(s.types, s.times, offs, ct, lo, hi, threads=3, method="dp")
    assert used1 == 1 and used4 == 4
    assert np.array_equal(c1, c4) and np.array_equal(c1, cdp)
    for c in range(0, 300, 37):
        o, p = offs[c], offs[c + 1]
        eo = o - c
        assert c1[c] == oracle.count_fsm(s.types, s.times, ct[o:p], lo[eo:eo + p - o - 1],
                                         hi[eo:eo + p - o - 1])


def _all_episodes(n_types, max_size, bins):
    """Every episode with distinct types up to max_size nodes and edges from bins."""
    import itertools
    out = [((a,), (), ()) for a in range(n_types)]
    for N in range(2, max_size + 1):
        for types in itertools.permutations(range(n_types), N):
            for bs in itertools.product(range(len(bins)), repeat=N - 1):
                out.append((types, tuple(bins[b][0] for b in bs), tuple(bins[b][1] for b in bs)))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_levelwise_equals_exhaustive_filter(seed):
    """The level-wise procedure (Apriori join + count > threshold) returns
    exactly the episodes, among ALL distinct-type episodes over the bins, whose
    count exceeds the threshold: anti-monotonicity makes the join complete."""
    r = synth.Rng(seed, 3)
    n_types = 4
    bins = [(0, 3), (2, 6)]
    ty, tm = synth.tiny_random_stream(seed, 160, n_types, 120)
    thr = int(r.integers(3, 8, 1)[0])
    lv = oracle.mine_levelwise(ty, tm, n_types, bins, thr, 4)
    got = set()
    for N in range(1, 5):
        for ep, c in lv[N]:
            got.add((ep, c))
    want = set()
    for ep in _all_episodes(n_types, 4, bins):
        c = oracle.count_fsm(ty, tm, ep[0], ep[1], ep[2])
        if c > thr:
            want.add((ep, c))
    assert got == want
    # canonical order inside each level
    for N in range(1, 5):
        keys = [oracle.canonical_key(ep) for ep, _ in lv[N]]
        assert keys == sorted(keys)


def test_levelwise_recovers_planted_chains_c1():
    """Sanity (not parity): the two planted 4-neuron chains of the tiny
    workload are frequent 4-node episodes."""
    s, cfg = synth.c1_tiny()
    lv = oracle.mine_levelwise(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"],
                               cfg["max_size"])
    found = {ep[0] for ep, _ in lv[4]}
    for ch in s.chains:
        assert tuple(ch["neurons"]) in found

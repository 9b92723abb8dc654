"""Pins for the coarse-tick upper bound of the oracle (no GPU).

The bound's definition is in oracle/coarse_bound.py.  Pins: with w = 1 it is
the number of events that end at least one occurrence (brute force over
event tuples on tiny streams); it never falls below the exact count (the
pinned state-machine counter O1); with one tick covering the whole stream
it is the end type's frequency (or 0 when an earlier node's type is
missing); a hand-worked case; and each planted mistake fails one of these.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import coarse_bound as cb
import synth


def brute_valid_ends(ty, tm, E, lo, hi):
    """Events that end at least one occurrence: every index tuple checked."""
    n, N = len(ty), len(E)
    ends = set()
    for idx in itertools.product(range(n), repeat=N):
        if any(int(ty[idx[k]]) != E[k] for k in range(N)):
            continue
        if all(lo[k] < int(tm[idx[k + 1]]) - int(tm[idx[k]]) <= hi[k] for k in range(N - 1)):
            ends.add(idx[-1])
    return len(ends)


def _random_case(r, n_types, n, t_max):
    ty, tm = synth.tiny_random_stream(int(r.integers(0, 10**6, 1)[0]), n, n_types, t_max)
    N = int(r.integers(1, 4, 1)[0])
    E = [int(x) for x in r.integers(0, n_types - 1, N)]
    lo = [int(x) for x in r.integers(0, 4, N - 1)]
    hi = [l + int(x) for l, x in zip(lo, r.integers(1, 8, N - 1))]
    return ty, tm, E, lo, hi


def pin_w1_is_valid_ends(mutant=0, cases=60):
    r = synth.Rng(0xC0A5, 1)
    bad = []
    for i in range(cases):
        ty, tm, E, lo, hi = _random_case(r, 3, 14, 30)
        if cb.coarse_ub(ty, tm, E, lo, hi, 1, mutant) != brute_valid_ends(ty, tm, E, lo, hi):
            bad.append(i)
    return bad


def pin_bound_above_count(mutant=0, cases=80):
    r = synth.Rng(0xC0A5, 2)
    bad = []
    for i in range(cases):
        ty, tm, E, lo, hi = _random_case(r, 4, 60, 120)
        c = oracle.count_fsm(ty, tm, E, lo, hi)
        for w in (1, 2, 3, 5, 8):
            if cb.coarse_ub(ty, tm, E, lo, hi, w, mutant) < c:
                bad.append((i, w))
    return bad


def pin_one_tick(mutant=0, cases=40):
    r = synth.Rng(0xC0A5, 3)
    bad = []
    for i in range(cases):
        ty, tm, E, lo, hi = _random_case(r, 4, 30, 60)
        w = 10**6
        present = all(np.any(ty == a) for a in E[:-1])
        want = int(np.sum(ty == E[-1])) if present else 0
        if cb.coarse_ub(ty, tm, E, lo, hi, w, mutant) != want:
            bad.append(i)
    return bad


def pin_hand_case(mutant=0):
    # A@0 B@3 A@10 B@14 B@15 B@16 C@20; episode A -> B, interval (0, 5].
    # Fine ticks (w = 1): ends B@3, B@14, B@15 (B@16 is 6 after A@10) -> 3.
    # w = 4: ticks A {0, 2}, B {0, 3, 3, 4}; offsets [floor(1/4), floor(8/4)] =
    # [0, 2]; reach of {0, 2} = {0..4} -> all four B events -> 4.
    # The exact count is 2 (A@0-B@3, A@10-B@14).
    ty = np.array([0, 1, 0, 1, 1, 1, 2], np.uint16)
    tm = np.array([0, 3, 10, 14, 15, 16, 20], np.int32)
    got = (cb.coarse_ub(ty, tm, [0, 1], [0], [5], 1, mutant), cb.coarse_ub(ty, tm, [0, 1], [0], [5], 4, mutant))
    return [] if got == (3, 4) and oracle.count_fsm(ty, tm, [0, 1], [0], [5]) == 2 else [got]


PINS = [pin_w1_is_valid_ends, pin_bound_above_count, pin_one_tick, pin_hand_case]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_pin_holds(pin):
    assert pin() == []


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_pins_catch_planted_mistake(m):
    assert any(pin(m) for pin in PINS), f"mutant {m} survived every pin"


def test_default_tick_keeps_offsets_within_a_word():
    for hi in range(1, 5000, 7):
        w = cb.default_tick(hi)
        assert cb.tick_offsets(0, hi, w)[1] <= 31
        if w > 1:
            assert cb.tick_offsets(0, hi, w - 1)[1] > 31

"""Planted mistakes in the oracle must be caught by the pins.

Each mutant is the oracle compiled with -DORC_MUTANT=k, which plants one
plausible mistake (a tie admitted at the overlap boundary, a closed lower or
open upper bound, no reset after a completion, the garbled completion node,
only the newest list entry examined, pruning by the wrong bound, Algorithm 1's
literal prev_e = 0, a non-strict overlap test).  The mistake lives in the
oracle on the CPU only.
"""
import pytest

import oracle
import oracle_pinsuite as ps

MUTANTS = [1, 2, 3, 4, 5, 6, 7, 8, 9]


@pytest.mark.parametrize("m", MUTANTS)
def test_pins_catch_mutant(m):
    oracle.build(m)
    assert oracle._load(m).orc_mutant_id() == m
    fails = ps.run_all(m)
    assert fails, f"mutant {m} survived every pin"


def test_unmutated_oracle_passes_same_suite():
    assert oracle._load(0).orc_mutant_id() == 0
    assert ps.run_all(0) == []

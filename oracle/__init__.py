"""CPU oracle for exact non-overlapped serial-episode counting.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may
import this package.  The product library never does; the two share no code,
header, table or helper.  Inputs come from ``synth`` (seeded generators that
hold none of the counting arithmetic).

Contents
  build()            compile ``fem_oracle.c`` with gcc (optionally a mutant).
  count_fsm / count_dp / count_brute
                     the three independent counters O1/O2/O3 (see the C file
                     header for the passages each follows).
  greedy_sorted / intervals_brute
                     Algorithm 1 alone and the exhaustive interval optimum.
  count_many         O1 (or O2) over many candidates on a pthread pool.
  mine_levelwise     the level-wise Apriori procedure of section "Temporal
                     Data Mining": level 1 = event frequencies, level N
                     candidates joined from frequent (N-1)-episodes, counted
                     with O1, kept when count > threshold.
  coarse_bound       (submodule, plain Python) the coarse-tick upper bound
                     on the count, written from its definition; pinned in
                     tests/test_oracle_coarse_bound.py.

Parity status: O1, O2 and O3 are pinned against each other, against closed
forms and against invariants (tests/test_oracle_pins.py) and the pins are
shown to catch planted mistakes (tests/test_oracle_mutants.py).  No function
here is "parity unpinned"; the paper prints no counts, so no pin comes from a
printed value (its worked example is internally inconsistent and unused).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem_oracle.c")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

NEG_INF = -(2**63)
_FAIL = 2**64 - 1


def _lib_path(mutant: int) -> str:
    name = "libfem_oracle.so" if mutant == 0 else f"libfem_oracle_m{mutant}.so"
    return os.path.join(_HERE, name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (``-DORC_MUTANT=mutant`` plants a test mistake)."""
    out = _lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
           f"-DORC_MUTANT={mutant}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load(mutant: int = 0) -> ctypes.CDLL:
    with _LOCK:
        if mutant in _LIBS:
            return _LIBS[mutant]
        lib = ctypes.CDLL(build(mutant))
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int
        u64 = ctypes.c_uint64
        lib.orc_count_fsm.argtypes = [P, P, i64, i32, P, P, P]
        lib.orc_count_fsm.restype = u64
        lib.orc_count_dp.argtypes = [P, P, i64, i32, P, P, P]
        lib.orc_count_dp.restype = u64
        lib.orc_count_brute.argtypes = [P, P, i64, i32, P, P, P, i64]
        lib.orc_count_brute.restype = u64
        lib.orc_greedy_sorted.argtypes = [P, P, i64]
        lib.orc_greedy_sorted.restype = u64
        lib.orc_intervals_brute.argtypes = [P, P, i64]
        lib.orc_intervals_brute.restype = u64
        lib.orc_count_many.argtypes = [P, P, i64, i64, P, P, P, P, P, i32, i32]
        lib.orc_count_many.restype = i32
        lib.orc_mutant_id.argtypes = []
        lib.orc_mutant_id.restype = i32
        _LIBS[mutant] = lib
        return lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


def _stream(types, times):
    ty = np.ascontiguousarray(types, dtype=np.uint16)
    tm = np.ascontiguousarray(times, dtype=np.int32)
    assert ty.shape == tm.shape and ty.ndim == 1
    return ty, tm


def _episode(E, lo, hi):
    E = np.ascontiguousarray(E, dtype=np.uint16)
    lo = np.ascontiguousarray(lo if len(lo) else np.zeros(1), dtype=np.int32)
    hi = np.ascontiguousarray(hi if len(hi) else np.zeros(1), dtype=np.int32)
    return E, lo, hi


def _check(v: int) -> int:
    if v == _FAIL:
        raise MemoryError("oracle: allocation failed or input too large")
    return int(v)


def count_fsm(types, times, E, lo, hi, mutant: int = 0) -> int:
    """O1: serial state machine count of episode (E, lo, hi)."""
    ty, tm = _stream(types, times)
    E, lo_a, hi_a = _episode(E, lo, hi)
    lib = _load(mutant)
    return _check(lib.orc_count_fsm(_ptr(ty), _ptr(tm), len(ty), len(E), _ptr(E), _ptr(lo_a), _ptr(hi_a)))


def count_dp(types, times, E, lo, hi, mutant: int = 0) -> int:
    """O2: latest-start dynamic programme + Algorithm 1."""
    ty, tm = _stream(types, times)
    E, lo_a, hi_a = _episode(E, lo, hi)
    lib = _load(mutant)
    return _check(lib.orc_count_dp(_ptr(ty), _ptr(tm), len(ty), len(E), _ptr(E), _ptr(lo_a), _ptr(hi_a)))


def count_brute(types, times, E, lo, hi, max_occ: int = 4096) -> int:
    """O3: all occurrences + exhaustive largest non-overlapped subset."""
    ty, tm = _stream(types, times)
    E, lo_a, hi_a = _episode(E, lo, hi)
    lib = _load(0)
    return _check(lib.orc_count_brute(_ptr(ty), _ptr(tm), len(ty), len(E), _ptr(E), _ptr(lo_a),
                                      _ptr(hi_a), max_occ))


def greedy_sorted(s, e) -> int:
    """Algorithm 1 over intervals already sorted by end."""
    s = np.ascontiguousarray(s, dtype=np.int64)
    e = np.ascontiguousarray(e, dtype=np.int64)
    return _check(_load(0).orc_greedy_sorted(_ptr(s), _ptr(e), len(s)))


def intervals_brute(s, e) -> int:
    """Exhaustive largest pairwise non-overlapped subset of closed intervals."""
    s = np.ascontiguousarray(s, dtype=np.int64)
    e = np.ascontiguousarray(e, dtype=np.int64)
    return _check(_load(0).orc_intervals_brute(_ptr(s), _ptr(e), len(s)))


def count_many(types, times, offs, ctypes_, lo, hi, threads: int = 0, method: str = "fsm",
               mutant: int = 0):
    """Count every candidate of a CSR set (offs[n_cand+1], node types, edge
    lo/hi) with O1 (``method="fsm"``) or O2 (``"dp"``).  Returns
    (counts uint64[n_cand], threads_used)."""
    ty, tm = _stream(types, times)
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    ct = np.ascontiguousarray(ctypes_, dtype=np.uint16)
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    n_cand = len(offs) - 1
    counts = np.zeros(max(n_cand, 1), dtype=np.uint64)
    if threads <= 0:
        threads = len(os.sched_getaffinity(0))
    if n_cand == 0:
        return counts[:0], threads
    if lo.size == 0:
        lo = np.zeros(1, np.int32)
        hi = np.zeros(1, np.int32)
    used = _load(mutant).orc_count_many(_ptr(ty), _ptr(tm), len(ty), n_cand, _ptr(offs), _ptr(ct),
                                        _ptr(lo), _ptr(hi), _ptr(counts), threads,
                                        1 if method == "dp" else 0)
    if used < 1:
        raise MemoryError("oracle: thread pool allocation failed")
    if np.any(counts[:n_cand] == np.uint64(_FAIL)):
        raise MemoryError("oracle: allocation failed")
    return counts[:n_cand], used


# --------------------------------------------------------------------------
# Level-wise mining (section "Temporal Data Mining": candidates of size N are
# generated from frequent (N-1)-episodes, counted in one pass, and kept when
# their count is greater than the threshold).
#
# An episode is a tuple (types, lo, hi) of python tuples.  Readings of what
# the paper leaves open: candidates use distinct types; level 2 pairs every ordered pair
# of distinct frequent types with every interval bin; level N >= 3 joins
# alpha and beta of size N-1 when alpha minus its first node equals beta minus
# its last node (types and intervals), giving alpha followed by beta's last
# node and last edge; count > threshold is kept (strict).

def canonical_key(ep):
    """Interleaved order (E1, lo1, hi1, E2, ..., lo_{N-1}, hi_{N-1}, EN)."""
    types, lo, hi = ep
    key = []
    for k in range(len(types)):
        key.append(types[k])
        if k < len(lo):
            key.append(lo[k])
            key.append(hi[k])
    return (len(types), tuple(key))


def to_csr(episodes):
    """List of (types, lo, hi) -> (offs int64, types uint16, lo int32, hi int32)."""
    offs = [0]
    t, l, h = [], [], []
    for types, lo, hi in episodes:
        t.extend(types)
        l.extend(lo)
        h.extend(hi)
        offs.append(len(t))
    return (np.array(offs, np.int64), np.array(t, np.uint16), np.array(l, np.int32),
            np.array(h, np.int32))


def generate_candidates(frequent, level, frequent_types, bins):
    """Candidates of size `level` from the frequent episodes of size level-1."""
    out = []
    if level == 2:
        for a in frequent_types:
            for (blo, bhi) in bins:
                for b in frequent_types:
                    if a != b:
                        out.append(((a, b), (blo,), (bhi,)))
        return out
    for alpha in frequent:
        at, al, ah = alpha
        for beta in frequent:
            bt, bl, bh = beta
            if at[1:] != bt[:-1] or al[1:] != bl[:-1] or ah[1:] != bh[:-1]:
                continue
            if bt[-1] in at:
                continue
            out.append((at + (bt[-1],), al + (bl[-1],), ah + (bh[-1],)))
    return out


def mine_levelwise(types, times, n_types, bins, threshold, max_size, threads: int = 0):
    """Returns a list indexed by level (1..max_size) of lists of
    (episode, count) in canonical order; entry 0 is unused."""
    ty, tm = _stream(types, times)
    bins = sorted((int(a), int(b)) for a, b in bins)
    freq = np.bincount(ty.astype(np.int64), minlength=n_types)[:n_types]
    levels = [[] for _ in range(max_size + 1)]
    ftypes = [a for a in range(n_types) if freq[a] > threshold]
    levels[1] = [(((a,), (), ()), int(freq[a])) for a in ftypes]
    frequent = [ep for ep, _ in levels[1]]
    for N in range(2, max_size + 1):
        cands = generate_candidates(frequent, N, ftypes, bins)
        if not cands:
            break
        offs, ct, lo, hi = to_csr(cands)
        counts, _ = count_many(ty, tm, offs, ct, lo, hi, threads=threads)
        kept = [(ep, int(c)) for ep, c in zip(cands, counts) if int(c) > threshold]
        kept.sort(key=lambda ec: canonical_key(ec[0]))
        levels[N] = kept
        frequent = [ep for ep, _ in kept]
        if not frequent:
            break
    return levels

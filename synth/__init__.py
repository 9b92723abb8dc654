"""Seeded synthetic spike-train streams and candidate sets.

This module holds no counting arithmetic: it only draws inputs.  Both the
CPU oracle and the CUDA library are fed from here, so neither side generates
inputs for the other.

Random numbers come from splitmix64 evaluated on a counter (a counter-based
generator: value k of stream s is splitmix64(seed_mix(s) + k)), so a draw does
not depend on earlier draws and the integer outputs are identical on every
machine.  Exponential and log-normal draws go through numpy's libm; after
quantisation to integer ticks a last-ulp difference between machines could in
principle move one event by one tick, which only matters for files stored on
one machine and read on another (none are).

The workloads model the paper's spike-train data (section "Test datasets":
non-homogeneous Poisson neurons with embedded chains of firing neurons):
  * every neuron fires as a Poisson process at its own rate, optionally
    multiplied inside network bursts;
  * an embedded chain (n_0 -> n_1 -> ...) makes every spike of n_0 trigger
    n_1 with probability p after a delay, and every triggered spike of n_k
    trigger n_{k+1} in the same way;
  * times are quantised to integer ticks, (type, tick) duplicates are removed
    (a refractory period of one tick), and events are sorted by (time, type).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK53 = float(2**-53)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied to x + golden (Steele, Lea, Flood 2014)."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + _GOLDEN).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based stream: draw k of stream (seed, sid) = splitmix64(base + k)."""

    def __init__(self, seed: int, sid: int = 0):
        base = splitmix64(np.array([(seed * 0x100000001B3 + sid) & (2**64 - 1)], np.uint64))[0]
        self.base = np.uint64(base)
        self.k = 0

    def bits(self, n: int) -> np.ndarray:
        idx = np.arange(self.k, self.k + n, dtype=np.uint64)
        self.k += n
        with np.errstate(over="ignore"):
            return splitmix64(idx + self.base)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1)."""
        return (self.bits(n) >> np.uint64(11)).astype(np.float64) * _MASK53

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers uniform in [lo, hi] (inclusive), by multiply-shift."""
        span = hi - lo + 1
        u = self.uniform(n)
        return (lo + np.minimum(np.floor(u * span), span - 1)).astype(np.int64)

    def exponential(self, n: int) -> np.ndarray:
        return -np.log1p(-self.uniform(n))

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclasses.dataclass
class Stream:
    types: np.ndarray  # uint16[n]
    times: np.ndarray  # int32[n] (ticks)
    n_types: int
    tick_s: float
    chains: list       # list of (neuron list, per-edge delay description)
    meta: dict

    @property
    def n(self) -> int:
        return int(self.types.shape[0])


def _poisson_times(rng: Rng, rate_hz: float, duration_s: float) -> np.ndarray:
    """Homogeneous Poisson spike times in [0, duration)."""
    if rate_hz <= 0:
        return np.zeros(0)
    expect = rate_hz * duration_s
    out = []
    t0 = 0.0
    while True:
        m = int(expect * 1.1 + 10 * math.sqrt(expect) + 16)
        gaps = rng.exponential(m) / rate_hz
        ts = t0 + np.cumsum(gaps)
        out.append(ts[ts < duration_s])
        if ts[-1] >= duration_s:
            break
        t0 = ts[-1]
    return np.concatenate(out)


def _burst_mask_times(rng: Rng, duration_s: float, gap_lo: float, gap_hi: float,
                      len_lo: float, len_hi: float):
    """Network burst windows [s, e): gaps U(gap_lo, gap_hi), lengths U(len_lo, len_hi)."""
    starts, ends = [], []
    t = 0.0
    while True:
        t += gap_lo + (gap_hi - gap_lo) * rng.uniform(1)[0]
        if t >= duration_s:
            break
        ln = len_lo + (len_hi - len_lo) * rng.uniform(1)[0]
        starts.append(t)
        ends.append(min(t + ln, duration_s))
        t += ln
    return np.array(starts), np.array(ends)


def _in_windows(ts: np.ndarray, starts: np.ndarray, ends: np.ndarray) -> np.ndarray:
    if len(starts) == 0:
        return np.zeros(ts.shape, bool)
    k = np.searchsorted(starts, ts, side="right") - 1
    ok = k >= 0
    res = np.zeros(ts.shape, bool)
    res[ok] = ts[ok] < ends[k[ok]]
    return res


def _sorted_unique(key: np.ndarray) -> np.ndarray:
    """Sorted distinct values (np.unique's result, by a plain sort and a
    neighbour comparison, which stays fast on tens of millions of keys)."""
    key = np.sort(key)
    if key.size:
        keep = np.empty(key.size, bool)
        keep[0] = True
        np.not_equal(key[1:], key[:-1], out=keep[1:])
        key = key[keep]
    return key


def _finish(types_list, times_list, tick_s: float, n_types: int, chains, meta) -> Stream:
    ty = np.concatenate(types_list).astype(np.int64) if types_list else np.zeros(0, np.int64)
    ts = np.concatenate(times_list) if times_list else np.zeros(0)
    ticks = np.floor(ts / tick_s).astype(np.int64)
    keep = ticks >= 0
    ty, ticks = ty[keep], ticks[keep]
    if ticks.size and ticks.max() >= 2**31 - 1:
        raise ValueError("stream span overflows int32 ticks")
    key = ticks * 65536 + ty
    key = _sorted_unique(key)  # sorts by (time, type) and drops (type, tick) duplicates
    times = (key // 65536).astype(np.int32)
    types = (key % 65536).astype(np.uint16)
    return Stream(types, times, n_types, tick_s, chains, meta)


def spike_train(seed: int, n_neurons: int, rates_hz, duration_s: float, tick_s: float,
                chains=(), bursts=None) -> Stream:
    """General generator.

    rates_hz: per-neuron base rate.  chains: list of dicts
    {"neurons": [...], "p": follow prob, "delays_s": [(lo, hi) per edge]} with
    each edge delay uniform in [lo, hi] seconds, or {"delays_ticks": [[...]]}
    for a uniform choice among integer tick delays.  bursts: None or dict
    {"gap": (lo, hi) s, "len": (lo, hi) s, "gain": factor}.
    """
    rng = Rng(seed, 1)
    types_list, times_list = [], []
    starts = ends = np.zeros(0)
    gain = 1.0
    if bursts:
        starts, ends = _burst_mask_times(Rng(seed, 2), duration_s, *bursts["gap"], *bursts["len"])
        gain = float(bursts["gain"])
    for a in range(n_neurons):
        r = float(rates_hz[a])
        if gain > 1.0:
            # thinning: candidate spikes at gain*r, kept with prob 1 outside bursts 1/gain
            cand = _poisson_times(rng, r * gain, duration_s)
            inb = _in_windows(cand, starts, ends)
            u = rng.uniform(cand.size)
            ts = cand[inb | (u < 1.0 / gain)]
        else:
            ts = _poisson_times(rng, r, duration_s)
        types_list.append(np.full(ts.size, a, np.int64))
        times_list.append(ts)
    chain_meta = []
    for ci, ch in enumerate(chains):
        crng = Rng(seed, 1000 + ci)
        neurons = list(ch["neurons"])
        src = times_list[neurons[0]]
        cur = src
        for e in range(len(neurons) - 1):
            follow = crng.uniform(cur.size) < ch["p"]
            cur = cur[follow]
            if "delays_ticks" in ch:
                opts = np.array(ch["delays_ticks"][e], np.int64)
                pick = crng.integers(0, len(opts) - 1, cur.size)
                d = opts[pick] * tick_s
                # land the follower inside the intended tick after quantisation
                cur = (np.floor(cur / tick_s) + 0.5) * tick_s + d
            else:
                dlo, dhi = ch["delays_s"][e]
                cur = cur + dlo + (dhi - dlo) * crng.uniform(cur.size)
            cur = cur[cur < duration_s]
            types_list.append(np.full(cur.size, neurons[e + 1], np.int64))
            times_list.append(cur)
        chain_meta.append(ch)
    meta = {"seed": seed, "duration_s": duration_s, "n_neurons": n_neurons}
    return _finish(types_list, times_list, tick_s, n_neurons, chain_meta, meta)


# --------------------------------------------------------------------------
# The five workload families (seed for family i = 0xFE0000 + i).

def c1_tiny(seed: int = 0xFE0001) -> tuple[Stream, dict]:
    """32 neurons at 5 Hz for 30 s, 1 ms ticks, two 4-neuron chains (follow
    prob 0.8, delays of 3, 4 or 5 ms), bin (0,5] ms, threshold 50, sizes <= 4."""
    rng = Rng(seed, 7)
    perm = np.argsort(rng.uniform(32))
    chains = [
        {"neurons": [int(x) for x in perm[0:4]], "p": 0.8, "delays_ticks": [[3, 4, 5]] * 3},
        {"neurons": [int(x) for x in perm[4:8]], "p": 0.8, "delays_ticks": [[3, 4, 5]] * 3},
    ]
    s = spike_train(seed, 32, np.full(32, 5.0), 30.0, 1e-3, chains)
    return s, {"bins": [(0, 5)], "threshold": 50, "max_size": 4}


def c2_mid(seed: int = 0xFE0002, duration_s: float = 1000.0) -> tuple[Stream, dict]:
    """128 neurons, log-normal rates clipped to [2, 20] Hz, 1 us ticks, six
    chains of 4-6 neurons (follow prob 0.9, each edge delay a bin centre
    +- 1 ms), bins {(0,5], (5,10], (10,15], (15,20]} ms, threshold 0.25% of n,
    sizes <= 6.  The stated 300 s cannot reach ~1M events at 2-20 Hz, so the
    duration is stretched (default 1000 s, ~1M events)."""
    rng = Rng(seed, 7)
    rates = np.clip(np.exp(math.log(6.0) + 0.6 * rng.normal(128)), 2.0, 20.0)
    perm = np.argsort(rng.uniform(128))
    centres = [2.5e-3, 7.5e-3, 12.5e-3, 17.5e-3]
    chains, pos = [], 0
    for c in range(6):
        ln = int(rng.integers(4, 6, 1)[0])
        neurons = [int(x) for x in perm[pos:pos + ln]]
        pos += ln
        bins = rng.integers(0, 3, ln - 1)
        delays = [(centres[b] - 1e-3, centres[b] + 1e-3) for b in bins]
        chains.append({"neurons": neurons, "p": 0.9, "delays_s": delays})
    s = spike_train(seed, 128, rates, duration_s, 1e-6, chains)
    bins = [(0, 5000), (5000, 10000), (10000, 15000), (15000, 20000)]
    thr = int(0.0025 * s.n)
    return s, {"bins": bins, "threshold": thr, "max_size": 6}


def bursty_60(seed: int, target_n: int, tick_s: float = 1e-5, n_chains: int = 3,
              rate_hz: float = 20.0) -> Stream:
    """60 types at a base rate, network bursts every U(2,10) s lasting
    U(100,300) ms at 10x, plus embedded chains; duration chosen for ~target_n."""
    rng = Rng(seed, 7)
    per_s = 60 * rate_hz * (1.0 + 9.0 * 0.2 / 6.2)
    duration = target_n / per_s
    perm = np.argsort(rng.uniform(60))
    centres = [2.5e-3, 7.5e-3, 12.5e-3, 17.5e-3]
    chains, pos = [], 0
    for c in range(n_chains):
        ln = int(rng.integers(4, 6, 1)[0])
        neurons = [int(x) for x in perm[pos:pos + ln]]
        pos += ln
        bins = rng.integers(0, 3, ln - 1)
        chains.append({"neurons": neurons, "p": 0.9,
                       "delays_s": [(centres[b] - 1e-3, centres[b] + 1e-3) for b in bins]})
    return spike_train(seed, 60, np.full(60, rate_hz), duration, tick_s, chains,
                       bursts={"gap": (2.0, 10.0), "len": (0.1, 0.3), "gain": 10.0})


BINS_4 = [(0, 500), (500, 1000), (1000, 1500), (1500, 2000)]  # ms bins in 10 us ticks


def random_candidates(seed: int, n_cand: int, n_types: int, size_lo: int, size_hi: int,
                      bins, planted=(), planted_frac: float = 0.0):
    """CSR candidate set: sizes uniform in [size_lo, size_hi], distinct random
    types, each edge a bin chosen uniformly; a fraction are contiguous
    sub-episodes of the planted chains (padded with random distinct types when
    the chain is shorter than the drawn size)."""
    rng = Rng(seed, 11)
    sizes = rng.integers(size_lo, size_hi, n_cand)
    offs = np.zeros(n_cand + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    total = int(offs[-1])
    bins = np.asarray(list(bins), np.int64).reshape(-1, 2)
    # distinct random types per candidate: the first N of a random permutation
    order = np.argsort(rng.uniform(n_cand * n_types).reshape(n_cand, n_types), axis=1)
    nmax = int(sizes.max()) if n_cand else 0
    seq = order[:, :max(nmax, 1)].copy()
    planted = [list(ch["neurons"]) for ch in planted if len(ch["neurons"]) >= 2]
    if planted and planted_frac > 0:
        u = rng.uniform(n_cand)
        pick = rng.integers(0, len(planted) - 1, n_cand)
        start_u = rng.uniform(n_cand)
        for c in np.nonzero(u < planted_frac)[0]:
            ch = planted[int(pick[c])]
            N = int(sizes[c])
            N2 = min(N, len(ch))
            st = int(np.floor(start_u[c] * (len(ch) - N2 + 1)))
            head = ch[st:st + N2]
            rest = [int(x) for x in order[c] if int(x) not in head][: N - N2]
            seq[c, :N] = head + rest
    col = np.arange(max(nmax, 1))[None, :]
    types = seq[col < sizes[:, None]].astype(np.uint16)
    n_edges = total - n_cand
    pickb = rng.integers(0, len(bins) - 1, n_edges)
    lo = bins[pickb, 0].astype(np.int32)
    hi = bins[pickb, 1].astype(np.int32)
    return offs, types, lo, hi


def c3_batched(seed: int = 0xFE0003, n_events: int = 4_000_000, n_cand: int = 200_000):
    """One bursty 60-type stream (10 us ticks) and 200k candidates of sizes
    2-8 with edges drawn from the 4-bin set; 5% planted-chain sub-episodes."""
    s = bursty_60(seed, int(n_events * 1.05))
    # generated until n events: keep the time-ordered prefix of exactly n_events
    s.types, s.times = s.types[:n_events].copy(), s.times[:n_events].copy()
    offs, types, lo, hi = random_candidates(seed, n_cand, 60, 2, 8, BINS_4, s.chains, 0.05)
    return s, (offs, types, lo, hi)


def c4_lengths(seed: int = 0xFE0004, n_rec: int = 256, n_lo: float = 1e4, n_hi: float = 5e6) -> np.ndarray:
    """The event counts of the many-recordings set (log-uniform in [n_lo, n_hi])."""
    u = Rng(seed, 7).uniform(n_rec)
    return np.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * u).astype(np.int64)


def c4_recordings(seed: int = 0xFE0004, n_rec: int = 256, n_lo: float = 1e4, n_hi: float = 5e6, which=None):
    """n_rec 60-channel recordings, lengths log-uniform in [n_lo, n_hi], base
    rates 5-20 Hz, 10 us ticks, three chains of 4-6 neurons each; threshold
    per recording max(20, 0.25% n_r); bins the 4-bin set; sizes <= 6.
    `which` (optional) lists the recordings to draw (each is drawn from its
    own seed, so a subset equals the same entries of the whole set)."""
    ns = c4_lengths(seed, n_rec, n_lo, n_hi)
    out = []
    for r in (range(n_rec) if which is None else which):
        rr = Rng(seed * 1315423911 + r, 3)
        rates = 5.0 + 15.0 * rr.uniform(60)
        per_s = float(rates.sum())
        dur = float(ns[r]) / per_s
        perm = np.argsort(rr.uniform(60))
        centres = [2.5e-3, 7.5e-3, 12.5e-3, 17.5e-3]
        chains, pos = [], 0
        for c in range(3):
            ln = int(rr.integers(4, 6, 1)[0])
            neurons = [int(x) for x in perm[pos:pos + ln]]
            pos += ln
            bb = rr.integers(0, 3, ln - 1)
            chains.append({"neurons": neurons, "p": 0.9,
                           "delays_s": [(centres[b] - 1e-3, centres[b] + 1e-3) for b in bb]})
        s = spike_train(seed * 7919 + r, 60, rates, dur, 1e-5, chains)
        thr = max(20, int(0.0025 * s.n))
        out.append((s, {"bins": BINS_4, "threshold": thr, "max_size": 6}))
    return out


def serving_jobs(seed: int = 0xFE0005, n_jobs: int = 200, n_lo: float = 5e4, n_hi: float = 2e7,
                 stress_n: int = 0):
    """Job descriptions for the serving workload: n log-uniform in [n_lo, n_hi],
    types U{60..256}, threshold U(0.1%, 1%) of n, max size U{4..8}, ~20-30 Hz
    per type, 10 us ticks.  Streams are drawn lazily by make_job_stream()."""
    rng = Rng(seed, 7)
    jobs = []
    for j in range(n_jobs):
        u = rng.uniform(5)
        n = int(math.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * u[0]))
        nt = 60 + int(u[1] * 197)
        thr_frac = 0.001 + 0.009 * u[2]
        max_size = 4 + int(u[3] * 5)
        jobs.append({"seed": seed * 31 + j, "n": n, "n_types": min(nt, 256),
                     "thr_frac": thr_frac, "max_size": min(max_size, 8)})
    if stress_n:
        # the stress job: 256 types (each about 0.39% of the events) at the
        # low end of the threshold range, so that every type is frequent and
        # level 2 counts (or bounds) all 261,120 ordered pairs x bins over
        # the whole stream; the planted chains carry the deeper levels
        jobs.append({"seed": seed * 31 + 99991, "n": int(stress_n), "n_types": 256,
                     "thr_frac": 0.001, "max_size": 6})
    return jobs


def make_job_stream(job: dict) -> tuple[Stream, dict]:
    rr = Rng(job["seed"], 3)
    nt = job["n_types"]
    rates = 20.0 + 10.0 * rr.uniform(nt)
    dur = job["n"] / float(rates.sum())
    perm = np.argsort(rr.uniform(nt))
    centres = [2.5e-3, 7.5e-3, 12.5e-3, 17.5e-3]
    chains, pos = [], 0
    for c in range(3):
        ln = int(rr.integers(4, 6, 1)[0])
        neurons = [int(x) for x in perm[pos:pos + ln]]
        pos += ln
        bb = rr.integers(0, 3, ln - 1)
        chains.append({"neurons": neurons, "p": 0.9,
                       "delays_s": [(centres[b] - 1e-3, centres[b] + 1e-3) for b in bb]})
    s = spike_train(job["seed"], nt, rates, dur, 1e-5, chains)
    return s, {"bins": BINS_4, "threshold": int(job["thr_frac"] * s.n), "max_size": job["max_size"]}


def tiny_random_stream(rng_seed: int, n: int, n_types: int, t_max: int, sid: int = 0):
    """Small random stream for pins: n draws of (type, time) with times in
    [0, t_max], duplicates (type, time) removed, sorted by (time, then a random
    tie order).  Ties in time are frequent on purpose."""
    r = Rng(rng_seed, 100 + sid)
    ty = r.integers(0, n_types - 1, n)
    tm = r.integers(0, t_max, n)
    key = _sorted_unique(tm * 65536 + ty)
    tm = key // 65536
    ty = key % 65536
    # random order among equal times (Definition 1 allows any order of ties)
    tie = r.uniform(key.size)
    order = np.lexsort((tie, tm))
    return ty[order].astype(np.uint16), tm[order].astype(np.int32)

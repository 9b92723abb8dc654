"""Benchmark: level-wise frequent-episode mining on GB300.

One step = one full level-wise mining pass (levels 1..6: candidate
generation, upper-bound pre-pass, exact counting, threshold) over the
many-recordings workload: 256 synthetic 60-channel spike-train recordings of
log-uniform lengths 1e4..5e6 events (about 2.2e8 events in all, 10 us ticks,
three embedded chains each, bins {(0,5],(5,10],(10,15],(15,20]} ms, threshold
max(20, 0.25% of n) per recording), every recording mined in the same call.

Metric: episode-events counted per second = sum over every exactly counted
(candidate, recording) pair of the recording's event count, divided by the
step time.  Candidates that the level-2 pre-pass proves infrequent are not
counted and are reported apart (`pruned`).  `value` times the step with the
streams already resident in HBM; `e2e` times the same step through the C ABI
from pinned host buffers (stream upload, mining, result download inside the
timed region).

Beside the headline: the plain per-level GPU path on a sample of recordings
(and the library on the same sample), the mid-size single recording mining
pass, the 200k-candidate batched counting call, the serving workload (Poisson
job arrivals, 200 jobs plus one 1e8-event stress job), and the CPU oracle.

Multi-GPU: the path does not shard (replicas only); with N ranks each rank
mines its own replica and value = all ranks' episode-events / max rank time.

`--impl reference` times the CPU oracle (plain serial counter, all host
cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "episode-events counted/s (level-wise mining pass, exact)"
UNIT = "episode-events/s"
HEADLINE_PREPASS = 2  # fem_tuning.prepass of the headline step: the level-2 pair bound only
C4_DESC = ("batched multi-recording mining: 256 synthetic 60-channel recordings, lengths log-uniform "
           "1e4-5e6 events, 10 us ticks, levels 1-6, threshold max(20, 0.25% n)")
TRACK_SRC = os.path.join(ROOT, "paper_0905_2203_gb300", "csrc", "fem_track.cu")
COUNTERS = os.path.join(ROOT, "profiles", "track_counters.json")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.rows = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up (driver queries) must not overlap the timed
            # steps: wait for its first sample before the caller starts timing.
            t_end = time.time() + 15.0
            while not self.rows and self.proc.poll() is None and time.time() < t_end:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def aggregate_over_ranks(local_ms: float, local_units: float, world: int, device=None):
    """Replica aggregation: every rank did `local_units` episode-events in
    `local_ms`; the job's time is the slowest rank's, and its throughput is
    all ranks' work over that time.  Uses the process group of the caller
    (NCCL on GPUs, gloo in the CPU tests)."""
    if world <= 1:
        return local_ms, local_units / (local_ms / 1e3)
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms, local_units], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    t_max = float(mx[0].item())
    return t_max, float(sm[1].item()) / (t_max / 1e3)


def track_counters():
    """ncu counters of the local-tracking count kernel (DRAM bytes and issue
    activity of one launch, from the committed profile summary), or None once
    the kernel source has changed since they were taken."""
    try:
        d = json.load(open(COUNTERS))
        sha = hashlib.sha256(open(TRACK_SRC, "rb").read()).hexdigest()[:16]
        return d if d.get("kernel_sha16") == sha else None
    except Exception:
        return None


# ---------------------------------------------------------------------------
# Workload pieces

def c4_workload(n_rec: int = 256):
    """The first n_rec of the 256 recordings (all by default)."""
    return synth.c4_recordings(which=range(n_rec))


def plain_sample(recs, max_events: int = 3_000_000):
    """Indices of the recordings the plain per-level path is timed on: every
    16th recording in length order (a spread of lengths), kept while their
    events add up to at most max_events."""
    order = np.argsort([s.n for s, _ in recs])
    pick, tot = [], 0
    for i in order[::16]:
        if tot + recs[i][0].n > max_events:
            break
        pick.append(int(i))
        tot += recs[i][0].n
    return sorted(pick)


def sample_recordings(seed: int, k: int = 4):
    """k of the 256 recordings in a seeded order (drawn alone)."""
    return synth.c4_recordings(which=_sample_idx(seed, k))


def _sample_idx(seed: int, k: int = 4):
    return [int(i) for i in np.argsort(synth.Rng(seed, 3).uniform(256))[:k]]


def oracle_sample(recs, seconds: float, threads: int, seed: int = 0):
    """A bounded oracle sample of the many-recordings workload: level-2
    candidates (ordered pairs of frequent types x bins) of the given
    recordings, counted with the serial state machine; grown until it is
    about `seconds` of work on `threads` threads.  Returns (one-call
    function, description, episode-events per call)."""
    import oracle
    rng = synth.Rng(seed, 5)
    jobs = []
    for s, cfg in recs:
        freq = np.bincount(s.types.astype(np.int64), minlength=s.n_types)
        ftypes = [a for a in range(s.n_types) if freq[a] > cfg["threshold"]]
        cands = oracle.generate_candidates([], 2, ftypes, cfg["bins"])
        pick = np.argsort(rng.uniform(len(cands)))
        jobs.append((s, cands, pick))

    def make(m):
        parts = []
        for s, cands, pick in jobs:
            k = min(len(cands), m)
            parts.append((s, oracle.to_csr([cands[j] for j in pick[:k]]), k))
        return parts

    def run(parts):
        used = 0
        for s, (offs, ct, lo, hi), _ in parts:
            _, used = oracle.count_many(s.types, s.times, offs, ct, lo, hi, threads=threads)
        return used

    m = 4 * threads
    parts = make(m)
    t0 = time.perf_counter()
    run(parts)
    dt = time.perf_counter() - t0
    m = int(max(m, m * seconds / max(dt, 1e-3)))
    parts = make(m)
    ee = float(sum(k * s.n for s, _, k in parts))
    desc = (f"level-2 candidates (ordered pairs of frequent types x 4 bins) of {len(parts)} recordings of the "
            f"256 ({', '.join(str(s.n) for s, _, _ in parts)} events), up to {m} random candidates each, "
            f"{int(sum(k for _, _, k in parts))} candidates per call")
    return (lambda: run(parts)), desc, ee


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The CPU oracle on a bounded sample of the headline workload (level-2
    candidates of a few of the 256 recordings, about 5 s per step on all host
    cores), on the same metric and unit as the GPU arm."""
    if rank != 0:
        return
    recs = sample_recordings(0xBE)
    threads = len(os.sched_getaffinity(0))
    call, desc, ee = oracle_sample(recs, args.ref_seconds, threads)
    for _ in range(min(args.warmup, 1)):
        call()
    times, used = [], threads
    for _ in range(args.steps):
        t0 = time.perf_counter()
        used = call()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    v = ee * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": C4_DESC + f" ({args.c4_recs} recordings)",
                   "sample": "oracle on a bounded sample per step"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc,
                         "cpu_model": cpu_model()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(recs):
    """The oracle as it stands on the machine's host cores: a bounded sample of the
    headline workload on all cores and on one core, plus one whole mining pass
    of the mid-size recording (oracle.mine_levelwise)."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    call, desc, ee = oracle_sample([recs[i] for i in _sample_idx(0xBF)], 10.0, threads)
    t0 = time.perf_counter()
    used = call()
    dt = time.perf_counter() - t0
    call1, desc1, ee1 = oracle_sample([recs[i] for i in _sample_idx(0xC0)], 4.0, 1)
    t1 = time.perf_counter()
    call1()
    dt1 = time.perf_counter() - t1
    s, cfg = synth.c2_mid()
    t2 = time.perf_counter()
    oracle.mine_levelwise(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], cfg["max_size"],
                          threads=threads)
    dt2 = time.perf_counter() - t2
    return {"value": ee / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": desc + f", {dt:.1f} s", "cpu_model": cpu_model(),
            "single_core": {"value": ee1 / dt1, "unit": UNIT, "cores": 1, "sample": desc1 + f", {dt1:.1f} s"},
            "c2_mining_pass_s": dt2,
            "c2_mining_pass": f"oracle.mine_levelwise of the mid-size recording (n={s.n}, levels 1-6) on "
                              f"{threads} threads"}


def c2_leg(ctx, tstream, flush, steps: int):
    """Mid-size single recording (128 neurons, ~1.07M events, 1 us ticks):
    one mining pass (levels 1-6, one captured graph) per step."""
    import torch
    s, cfg = synth.c2_mid()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    stt = []
    for _ in range(3):
        r = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
        r.free()
    ms = 0.0
    for k in range(steps):
        flush.fill_(k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(tstream)
        r = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
        b.record(tstream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        stt.append(r.stats())
        r.free()
    st.free()
    ee = sum(x["counted_episode_events"] for x in stt)
    return {"workload": f"plain level-wise mining, mid: 128 neurons, lognormal 2-20 Hz, 1 us ticks (n={s.n}, "
                        f"levels 1-6, threshold {cfg['threshold']})",
            "value": ee / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "pruned_per_step": float(np.mean([x["candidates_pruned"] for x in stt])),
            "counted_per_step": float(np.mean([x["candidates_counted"] for x in stt])),
            "graph": bool(stt[-1]["graph_tails"])}


def c3_leg(ctx, tstream, flush, steps: int = 3):
    """Batched counting: one 4M-event bursty 60-type stream and 200k
    candidates (sizes 2-8, 4-bin intervals), one count_episodes call per
    step, stream resident; every candidate is counted over the whole
    stream, so episode-events = 200k x 4M per call."""
    import torch
    from paper_0905_2203_gb300 import binding as fb
    s, (offs, ct, lo, hi) = synth.c3_batched()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    cands = fb.Cands(offs, ct, lo, hi)
    ctx.count_episodes(st, cands)  # warm-up: builds per-type lists and densities
    ms, rel, kms, sp = 0.0, 0.0, 0.0, 0
    for k in range(steps):
        flush.fill_(k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(tstream)
        ctx.count_episodes(st, cands)
        b.record(tstream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        S = ctx.last_stats()
        rel += S["relevant_events"]
        kms += S["count_kernel_ms"]
        sp += S["sparse_launches"]
    st.free()
    n_c = len(offs) - 1
    return {"workload": f"one bursty 60-type stream, n={s.n}, {n_c} candidates sizes 2-8, 4 bins",
            "value": n_c * s.n * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "relevant_events_per_s": rel / (kms / 1e3) if kms else None,
            "count_launches_per_step": sp / steps}


def _level_arrays(res, n_recs: int, max_size: int):
    out = []
    for r in range(n_recs):
        for N in range(1, max_size + 1):
            out.append(res.level(r, N))  # (episodes, counts), canonical order
    return out


def _same_levels(a, b) -> bool:
    return len(a) == len(b) and all(x[0] == y[0] and x[1] == y[1] for x, y in zip(a, b))


def _lat_summary(lat_s, ee, span_s):
    lat = np.asarray(lat_s) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "episode_events_per_s": float(ee / span_s) if span_s > 0 else None}


def serving_leg(n_jobs: int = 200, stress_n: int = 100_000_000, load: float = 0.7, seed: int = 0xFE0005,
                plain_jobs: int = 12, plain_cap: int = 500_000):
    """Serving: the job list (n log-uniform in [5e4, 2e7], 60-256 types, max
    size 4-8, threshold 0.1-1% of n) plus the stress job.  Arrivals are
    Poisson (seeded) at `load` x the served path's measured capacity.  Arms,
    on the same arrival times:
      served      -- the serving loop (admission by device memory, streams and
                     candidates resident, ready levels of all admitted jobs
                     counted together), live; latency = result ready - submit;
      ours_fifo   -- the library's mine_levelwise, one job at a time, each
                     job's measured service time queued first-in first-out;
      plain_fifo  -- the plain per-level GPU path, the same way, on the first
                     `plain_jobs` jobs of at most `plain_cap` events (the plain
                     path needs hours for the whole list), against ours_fifo
                     on the same jobs.
    Every job's frequent episodes and counts must agree across arms."""
    import torch
    from paper_0905_2203_gb300 import binding as fb
    jobs = [j for j in synth.serving_jobs(seed, n_jobs=n_jobs, stress_n=stress_n)]
    data = [synth.make_job_stream(j) for j in jobs]
    K = len(jobs)
    srv = fb.Server(0, 0, 16)

    def submit(i):
        s, cfg = data[i]
        return srv.submit(s.types, s.times, s.n_types, cfg["bins"], cfg["threshold"], cfg["max_size"])

    def collect(ids, idx):
        lat, ee, arrays, sub, fin = [], 0.0, [], [], []
        for i, jid in zip(idx, ids):
            res, info = srv.wait(jid)
            lat.append(info["finish_s"] - info["submit_s"])
            sub.append(info["submit_s"])
            fin.append(info["finish_s"])
            ee += res.stats()["counted_episode_events"]
            arrays.append(_level_arrays(res, 1, data[i][1]["max_size"]))
            res.free()
        return lat, ee, arrays, min(sub), max(fin)

    # warm-up (kernel loading, first allocations), then capacity: all at once
    collect([submit(0)], [0])
    _, ee_all, _, t_a, t_b = collect([submit(i) for i in range(K)], list(range(K)))
    capacity = K / max(t_b - t_a, 1e-9)
    lam = load * capacity
    u = synth.Rng(seed, 11).uniform(K)
    arrive = np.cumsum(-np.log1p(-u) / lam)
    t0 = time.perf_counter()
    ids = []
    for i in range(K):
        d = t0 + arrive[i] - time.perf_counter()
        if d > 0:
            time.sleep(d)
        ids.append(submit(i))
    lat_srv, ee_srv, arr_srv, t_a, t_b = collect(ids, list(range(K)))
    srv.close()

    def service(plain: bool, idx):
        ctx = fb.Context(0)
        if plain:
            ctx.set_tuning(plain_path=1)
        svc, arrays, ee = [], [], []
        for i in [idx[0]] + list(idx):  # the first one twice: warm-up
            s, cfg = data[i]
            torch.cuda.synchronize()
            t = time.perf_counter()
            st = ctx.load_stream(s.types, s.times, s.n_types)
            res = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
            a = _level_arrays(res, 1, cfg["max_size"])
            e = res.stats()["counted_episode_events"]
            res.free()
            st.free()
            svc.append(time.perf_counter() - t)
            arrays.append(a)
            ee.append(e)
        ctx.close()
        return svc[1:], arrays[1:], ee[1:]

    def fifo(svc, arr):
        end, lat = 0.0, []
        for a, sv in zip(arr, svc):
            start = max(a, end)
            end = start + sv
            lat.append(end - a)
        return lat, end - arr[0]

    svc_o, arr_o, ee_o = service(False, list(range(K)))
    lat_o, span_o = fifo(svc_o, arrive)
    small = [i for i in range(K) if jobs[i]["n"] <= plain_cap][:plain_jobs]
    svc_p, arr_p, ee_p = service(True, small)
    sub_arrive = np.cumsum(-np.log1p(-synth.Rng(seed, 12).uniform(len(small))) / lam)
    lat_p, span_p = fifo(svc_p, sub_arrive)
    svc_os = [svc_o[i] for i in small]
    lat_os, span_os = fifo(svc_os, sub_arrive)
    parity = all(_same_levels(a, b) for a, b in zip(arr_srv, arr_o))
    parity = parity and all(_same_levels(arr_o[i], b) for i, b in zip(small, arr_p))
    n_ev = int(sum(d[0].n for d in data))
    return {
        "workload": f"serving: {K - (1 if stress_n else 0)} jobs of the job list"
                    + (f" plus the {stress_n}-event stress job" if stress_n else "")
                    + f", {n_ev} events, 60-256 types, max size 4-8, 10 us ticks",
        "arrivals": f"Poisson, {lam:.2f} jobs/s = {load} x served capacity ({capacity:.2f} jobs/s)",
        "served": _lat_summary(lat_srv, ee_srv, t_b - t_a),
        "ours_fifo": dict(_lat_summary(lat_o, sum(ee_o), span_o), service_ms_mean=1e3 * float(np.mean(svc_o))),
        "plain_sample": {
            "jobs": f"the first {len(small)} jobs of at most {plain_cap} events, own Poisson arrivals at the "
                    f"same rate",
            "plain_fifo": dict(_lat_summary(lat_p, sum(ee_p), span_p), service_ms_mean=1e3 * float(np.mean(svc_p))),
            "ours_fifo": dict(_lat_summary(lat_os, sum(ee_o[i] for i in small), span_os),
                              service_ms_mean=1e3 * float(np.mean(svc_os))),
        },
        "stress_job_ms": {"served": 1e3 * lat_srv[-1], "ours_service": 1e3 * svc_o[-1]} if stress_n else None,
        "parity_across_arms": bool(parity),
        "note": "p99 over the jobs (interpolated); FIFO arms queued on the same arrivals",
    }


def run_case(name: str):
    """Small fixed invocations used for ncu captures (no timing line):
    c4_mining      -- one mining call of the first 32 recordings of the
                      many-recordings set (after one warm-up call);
    c3_mid         -- one count of 20k episodes (sizes 2-8) over a 1M-event
                      bursty stream (after one warm-up call);
    c3_mid_sparse  -- the same count with the per-thread sparse kernel forced
                      (fem_tuning.kernel = 2);
    c3_mid_tiled   -- the same count with the tiled TMA / ballot kernel forced
                      (fem_tuning.kernel = 1);
    c2_mining      -- one default C2 mining pass (after one warm-up call)."""
    import torch
    from paper_0905_2203_gb300 import binding as fb
    ctx = fb.Context(0)
    sts = []
    if name == "c4_mining":
        recs = c4_workload(32)
        sts = [ctx.load_stream(s.types, s.times, s.n_types) for s, _ in recs]
        for _ in range(2):
            res = ctx.mine_levelwise(sts, recs[0][1]["bins"], [c["threshold"] for _, c in recs], 6)
            stats = res.stats()
            res.free()
    elif name == "c4_mid_mining":
        # the 12 recordings of 200k-600k events: the level structure of the
        # whole set at a device footprint small enough for a full profile
        ns = synth.c4_lengths()
        pick = [int(i) for i in np.nonzero((ns >= 200_000) & (ns <= 600_000))[0][:12]]
        recs = synth.c4_recordings(which=pick)
        sts = [ctx.load_stream(s.types, s.times, s.n_types) for s, _ in recs]
        for _ in range(2):
            res = ctx.mine_levelwise(sts, recs[0][1]["bins"], [c["threshold"] for _, c in recs], 6)
            stats = res.stats()
            res.free()
    elif name == "c2_mining":
        s, cfg = synth.c2_mid()
        sts = [ctx.load_stream(s.types, s.times, s.n_types)]
        for _ in range(2):
            res = ctx.mine_levelwise(sts, cfg["bins"], [cfg["threshold"]], cfg["max_size"])
            stats = res.stats()
            res.free()
    elif name in ("c3_mid", "c3_mid_sparse", "c3_mid_tiled"):
        s = synth.bursty_60(0xFE0003, 1_000_000)
        offs, ct, lo, hi = synth.random_candidates(0xFE0003, 20000, 60, 2, 8, synth.BINS_4, s.chains, 0.05)
        sts = [ctx.load_stream(s.types, s.times, s.n_types)]
        if name == "c3_mid_sparse":
            ctx.set_tuning(kernel=2)
        elif name == "c3_mid_tiled":
            ctx.set_tuning(kernel=1)
        for _ in range(2):
            ctx.count_episodes(sts[0], fb.Cands(offs, ct, lo, hi))
        stats = ctx.last_stats()
    else:
        raise SystemExit(f"unknown case {name}")
    print(json.dumps({"case": name, "stats": stats}))
    torch.cuda.synchronize()
    for st in sts:
        st.free()
    ctx.close()


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_0905_2203_gb300 import binding as fb

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    recs = c4_workload(args.c4_recs)
    bins = recs[0][1]["bins"]
    thr = [c["threshold"] for _, c in recs]
    max_size = recs[0][1]["max_size"]
    n_tot = int(sum(s.n for s, _ in recs))
    tstream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(tstream)
    ctx = fb.Context(local_rank, 0, tstream.cuda_stream)
    sts = [ctx.load_stream(s.types, s.times, s.n_types) for s, _ in recs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > L2 (129 MB)
    # The headline step times the exact-count pass with the level-2 pair bound
    # as its only pre-pass (prepass = 2), so every level-3 candidate is
    # counted; the library's default adds the level-3 join bound, which
    # prunes nearly all of them before the count: that configuration is the
    # mining_default leg (same workload, same results, fewer counted pairs).
    ctx.set_tuning(prepass=HEADLINE_PREPASS)

    def step():
        res = ctx.mine_levelwise(sts, bins, thr, max_size)
        stt = res.stats()
        res.free()
        return stt

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            flush.fill_(k)  # evict from L2 between timed steps (untimed)
            ev[k][0].record(tstream)
            stats.append(step())
            ev[k][1].record(tstream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ee_counted = sum(x["counted_episode_events"] for x in stats)
    ee_all = sum(x["episode_events"] for x in stats)
    rel = sum(x["relevant_events"] for x in stats)
    cnt_ms = sum(x["count_kernel_ms"] for x in stats)
    launches = sum(x["kernel_launches"] for x in stats)
    t_max, value = aggregate_over_ranks(ms, ee_counted, world, dev)

    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "value": value, "ms_per_step": t_max / args.steps,
                              "count_kernel_ms_per_step": cnt_ms / args.steps, "gpu_launches": int(launches),
                              "graph": bool(stats[-1]["graph_tails"])}))
        ctx.close()
        return

    # --- the same step with the library's default pre-passes (level-3 join
    # bound on): mining latency, and the same results as the headline step
    res = ctx.mine_levelwise(sts, bins, thr, max_size)
    ref_levels = _level_arrays(res, len(sts), max_size)
    res.free()
    ctx.reset_tuning()
    for _ in range(max(args.warmup, 2)):
        step()
    torch.cuda.synchronize()
    d_ms, d_stats = 0.0, []
    d_steps = max(3, min(args.steps, 10))
    for k in range(d_steps):
        flush.fill_(k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(tstream)
        d_stats.append(step())
        b.record(tstream)
        torch.cuda.synchronize()
        d_ms += a.elapsed_time(b)
    res = ctx.mine_levelwise(sts, bins, thr, max_size)
    same_default = _same_levels(ref_levels, _level_arrays(res, len(sts), max_size))
    res.free()
    del ref_levels
    mining_default = {
        "workload": "the headline step with the library defaults (level-2 pair bound and level-3 join bound)",
        "ms_per_step": d_ms / d_steps,
        "value": float(np.mean([x["counted_episode_events"] for x in d_stats])) / (d_ms / d_steps / 1e3),
        "unit": UNIT, "count_kernel_ms_per_step": float(np.mean([x["count_kernel_ms"] for x in d_stats])),
        "candidates_counted_per_step": float(np.mean([x["candidates_counted"] for x in d_stats])),
        "candidates_pruned_per_step": float(np.mean([x["candidates_pruned"] for x in d_stats])),
        "same_results_as_headline": bool(same_default), "timing": "CUDA events per step, L2 flushed between steps"}
    ctx.set_tuning(prepass=HEADLINE_PREPASS)

    # --- end to end through the C ABI from pinned host buffers
    pins = [(torch.from_numpy(s.types.view(np.int16)).pin_memory(), torch.from_numpy(s.times).pin_memory())
            for s, _ in recs]
    e2e_steps = max(1, min(args.steps, 3))
    e2e_ms, e2e_ee, d2h = 0.0, 0.0, 0
    for k in range(e2e_steps + 1):  # the first run warms the new streams' tables and graph
        flush.fill_(k)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(tstream)
        sts2 = [ctx.load_stream(tp.numpy().view(np.uint16), mp.numpy(), s.n_types)
                for (tp, mp), (s, _) in zip(pins, recs)]
        res = ctx.mine_levelwise(sts2, bins, thr, max_size)
        out_bytes = 0
        for r in range(len(sts2)):
            for N in range(1, max_size + 1):
                arrs = res.level_arrays(r, N)
                out_bytes += sum(x.nbytes for x in arrs)
        ee_k = res.stats()["counted_episode_events"]
        res.free()
        for st2 in sts2:
            st2.free()
        b.record(tstream)
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms += a.elapsed_time(b)
            e2e_ee += ee_k
            d2h = out_bytes
    del pins
    e2e_value = e2e_ee * world / (e2e_ms / 1e3)

    # --- plain per-level GPU path (comparison) on a sample of recordings, and
    # the library on the same sample
    pick = plain_sample(recs)
    sub = [sts[i] for i in pick]
    sub_thr = [thr[i] for i in pick]

    def sub_step(plain: bool):
        ctx.set_tuning(plain_path=1 if plain else 0, prepass=HEADLINE_PREPASS)
        try:
            res = ctx.mine_levelwise(sub, bins, sub_thr, max_size)
            a = _level_arrays(res, len(sub), max_size)
            e = res.stats()["counted_episode_events"]
            res.free()
        finally:
            ctx.reset_tuning()
        return a, e

    sub_step(False)
    torch.cuda.synchronize()
    t = time.perf_counter()
    a_o, e_o = sub_step(False)
    torch.cuda.synchronize()
    t_o = time.perf_counter() - t
    sub_step(True)  # warm-up of the plain path's tables
    torch.cuda.synchronize()
    t = time.perf_counter()
    a_p, e_p = sub_step(True)
    torch.cuda.synchronize()
    t_p = time.perf_counter() - t
    plain = {"recordings": f"{len(pick)} of the 256 (every 16th in length order, "
                           f"{int(sum(recs[i][0].n for i in pick))} events)",
             "value": e_p / t_p, "unit": UNIT, "ms_per_step": 1e3 * t_p,
             "ours_same_sample": {"value": e_o / t_o, "ms_per_step": 1e3 * t_o},
             "speedup": (e_o / t_o) / (e_p / t_p) if e_p else None,
             "parity": _same_levels(a_o, a_p), "timing": "host wall clock around a synchronised call"}

    c2 = None if args.no_legs else c2_leg(ctx, tstream, flush, max(3, min(args.steps, 20)))
    c3 = None if args.no_legs else c3_leg(ctx, tstream, flush)
    for st in sts:
        st.free()
    serving = None if (args.no_legs or args.no_serving) else serving_leg()
    if rank != 0:
        ctx.close()
        return
    peaks = _peaks()
    clocks = clk.summary()
    # roofline of the dominant kernel (the local-tracking count kernel): its
    # algorithmic work is one update per relevant (episode, event) pair
    # (events whose type is one of the episode's node types); peak = one
    # lane-instruction per lane per cycle: SMs x 4 schedulers x 32 lanes x clock
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_alu = props.multi_processor_count * 128 * sm_max * 1e6
    achieved = rel / (cnt_ms / 1e3) if cnt_ms > 0 else 0.0
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    counters = track_counters()
    pruned = float(np.mean([x["candidates_pruned"] for x in stats]))
    counted = float(np.mean([x["candidates_counted"] for x in stats]))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": C4_DESC + f" ({len(recs)} recordings)", "events": n_tot,
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs ({6 * n_tot / 1e9:.2f} GB of streams) larger than L2; a 256 MB buffer is also "
                         f"written between timed steps",
                   "candidates_counted_per_step": counted, "levels": float(np.mean([x["levels"] for x in stats])),
                   "numerator": "episode-events of exactly counted (candidate, recording) pairs",
                   "pre_pass": "level-2 pair bound only (fem_tuning.prepass = 2); the library default also "
                               "runs the level-3 join bound: see mining_default"},
        "pruned": {"value": (ee_all - ee_counted) * world / (t_max / 1e3), "unit": "episode-events/s pruned",
                   "candidates_per_step": pruned,
                   "note": "level-2 candidates resolved by the upper-bound pre-pass (never counted)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_alu,
                     "unit": "relevant episode-events/s", "frac": achieved / peak_alu,
                     "traffic": counters.get("dram_bytes_per_launch") if counters else None,
                     "issue_active": counters.get("issue_active_pct") if counters else None,
                     "note": "peak = SMs x 128 lanes x sm_max_mhz (one lane-op per relevant episode-event); "
                             "achieved over the count kernels' device time (CUDA events inside the graph); "
                             "traffic and issue_active from the committed ncu summary of the count kernel"},
        "hbm": {"achieved_gbs": counters.get("dram_gbs") if counters else None, "peak_gbs": hbm_peak,
                "frac": counters["dram_gbs"] / hbm_peak if counters and counters.get("dram_gbs") else None,
                "note": "DRAM read+write bytes of one count-kernel launch over its duration (ncu, committed "
                        "summary; null when the kernel has changed since)"},
        "count_kernel_ms_per_step": cnt_ms / args.steps,
        "relevant_events_per_step": rel / args.steps,
        "plain_gpu": plain,
        "mining_default": mining_default,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(6 * n_tot),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms / e2e_steps},
        "gpu_launches": int(launches),
        "graph": bool(stats[-1]["graph_tails"]),
        "c2_mining_pass": c2,
        "c3_batched_counting": c3,
        "serving": serving,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(recs)
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--c4-recs", type=int, default=256, help="recordings of the headline workload (256 = all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=5.0,
                    help="--impl reference: seconds of oracle work per step (on all host cores)")
    ap.add_argument("--no-legs", action="store_true", help="skip the mid-size, batched-counting and serving legs")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--quick", action="store_true", help="time the headline step only (for profiling)")
    ap.add_argument("--case", default=None,
                    help="run one small fixed invocation for profiling (c4_mining, c4_mid_mining, c3_mid, c3_mid_sparse, "
                         "c3_mid_tiled, c2_mining)")
    args = ap.parse_args()
    if args.case:
        run_case(args.case)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

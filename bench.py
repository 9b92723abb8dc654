"""Benchmark: level-wise frequent-episode mining on GB300.

One step = one full level-wise mining pass (levels 1..6: candidate
generation, exact counting, threshold) over the mid-size spike-train workload
(128 neurons, log-normal 2-20 Hz, 1 us ticks, ~1.07M events, six embedded
chains, bins {(0,5],(5,10],(10,15],(15,20]} ms, threshold 0.25% of n).

Metric: episode-events counted per second = sum over every counted
(candidate, recording) of the recording's event count, divided by the step
time.  `value` times the step with the stream already resident in HBM;
`e2e` times the same step through the C ABI from host buffers (stream upload,
mining, result download inside the timed region).

Multi-GPU: the path does not shard (replicas only); with N ranks each rank
mines its own replica and value = all ranks' episode-events / max rank time.

`--impl reference` times the CPU oracle (plain serial counter, all host
cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


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


def workload(name: str):
    if name == "c2":
        s, cfg = synth.c2_mid()
        return s, cfg, "plain level-wise mining, mid: 128 neurons, lognormal 2-20 Hz, 1 us ticks"
    if name == "c1":
        s, cfg = synth.c1_tiny()
        return s, cfg, "plain level-wise mining, tiny: 32 neurons, 5 Hz, 30 s, 1 ms ticks"
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    """CPU oracle on a bounded sample: level-2 candidates of the workload
    counted with the serial state machine on all host cores."""
    if rank != 0:
        return
    import oracle
    s, cfg, desc = workload(args.workload)
    freq = np.bincount(s.types.astype(np.int64), minlength=s.n_types)
    ftypes = [a for a in range(s.n_types) if freq[a] > cfg["threshold"]]
    cands = oracle.generate_candidates([], 2, ftypes, cfg["bins"])
    rng = synth.Rng(0xBE, 1)
    threads = len(os.sched_getaffinity(0))
    # calibrate the sample size to ~1.5 s of CPU work per step
    pick = np.argsort(rng.uniform(len(cands)))
    m = min(len(cands), 64 * threads)
    offs, ct, lo, hi = oracle.to_csr([cands[i] for i in pick[:m]])
    t0 = time.perf_counter()
    oracle.count_many(s.types, s.times, offs, ct, lo, hi, threads=threads)
    dt = time.perf_counter() - t0
    m2 = int(min(len(cands), max(m, m * 1.5 / max(dt, 1e-3))))
    offs, ct, lo, hi = oracle.to_csr([cands[i] for i in pick[:m2]])
    for _ in range(args.warmup if args.warmup < 2 else 1):
        oracle.count_many(s.types, s.times, offs[: min(len(offs), 33)], ct, lo, hi, threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, used = oracle.count_many(s.types, s.times, offs, ct, lo, hi, threads=threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    ee = float(m2) * s.n * args.steps
    v = ee / total
    sample = (f"{m2} of {len(cands)} level-2 candidates (random) over the full {s.n}-event stream "
              f"per step; serial state-machine counter, one candidate per task")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": desc + f" (n={s.n})", "levels": "2 (sample)", "l2": "stream 6.4 MB fits L2"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(s, cfg):
    """Bounded oracle timing (~10-20 s of CPU work) for the cpu_baseline key."""
    import oracle
    freq = np.bincount(s.types.astype(np.int64), minlength=s.n_types)
    ftypes = [a for a in range(s.n_types) if freq[a] > cfg["threshold"]]
    cands = oracle.generate_candidates([], 2, ftypes, cfg["bins"])
    rng = synth.Rng(0xBE, 2)
    pick = np.argsort(rng.uniform(len(cands)))
    threads = len(os.sched_getaffinity(0))
    m = min(len(cands), 32 * threads)
    offs, ct, lo, hi = oracle.to_csr([cands[i] for i in pick[:m]])
    t0 = time.perf_counter()
    oracle.count_many(s.types, s.times, offs, ct, lo, hi, threads=threads)
    dt = time.perf_counter() - t0
    m2 = int(min(len(cands), max(m, m * 10.0 / max(dt, 1e-3))))
    offs, ct, lo, hi = oracle.to_csr([cands[i] for i in pick[:m2]])
    t0 = time.perf_counter()
    _, used = oracle.count_many(s.types, s.times, offs, ct, lo, hi, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": m2 * s.n / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{m2} of {len(cands)} level-2 candidates over the full {s.n}-event stream, "
                      f"serial state-machine counter on {used} threads, {dt:.1f} s"}


def c3_leg(ctx, tstream, flush, steps: int = 2):
    """Batched counting: one 4M-event bursty 60-type stream and 200k
    candidates (sizes 2-8, 4-bin intervals), one count_episodes call per
    step, stream resident; episode-events/s over all 200k x 4M pairs."""
    import torch
    from paper_0905_2203_gb300 import binding as fb
    s, (offs, ct, lo, hi) = synth.c3_batched()
    st = ctx.load_stream(s.types, s.times, s.n_types)
    cands = fb.Cands(offs, ct, lo, hi)
    ctx.set_tuning()  # default kernel choice, no autotuning trials here
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
    ctx.set_tuning(autotune=1)
    n_c = len(offs) - 1
    return {"workload": f"one bursty 60-type stream, n={s.n}, {n_c} candidates sizes 2-8, 4 bins",
            "value": n_c * s.n * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "relevant_events_per_s": rel / (kms / 1e3) if kms else None,
            "sparse_launches_per_step": sp / steps}


def run_case(name: str):
    """Small fixed invocations used for ncu captures (no timing line):
    c2_level2_tiled -- one C2 mining pass with the pre-pass off and the tiled
                       kernel forced (level 2 counts all 55k candidates);
    c3_mid_sparse   -- one count of 20k episodes (sizes 2-8) over a 1M-event
                       bursty stream with the sparse kernel forced;
    c2_mining       -- one default C2 mining pass."""
    import torch
    from paper_0905_2203_gb300 import binding as fb
    ctx = fb.Context(0)
    if name in ("c2_level2_tiled", "c2_mining"):
        s, cfg = synth.c2_mid()
        st = ctx.load_stream(s.types, s.times, s.n_types)
        if name == "c2_level2_tiled":
            ctx.set_tuning(prepass=-1, kernel=1)
        res = ctx.mine_levelwise([st], cfg["bins"], [cfg["threshold"]], cfg["max_size"])
        print(json.dumps({"case": name, "stats": res.stats()}))
        res.free()
    elif name == "c3_mid_sparse":
        s = synth.bursty_60(0xFE0003, 1_000_000)
        offs, ct, lo, hi = synth.random_candidates(0xFE0003, 20000, 60, 2, 8, synth.BINS_4, s.chains, 0.05)
        st = ctx.load_stream(s.types, s.times, s.n_types)
        ctx.set_tuning(kernel=2)
        ctx.count_episodes(st, fb.Cands(offs, ct, lo, hi))
        print(json.dumps({"case": name, "stats": ctx.last_stats()}))
    else:
        raise SystemExit(f"unknown case {name}")
    torch.cuda.synchronize()
    st.free()
    ctx.close()


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_0905_2203_gb300 import binding as fb

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    s, cfg, desc = workload(args.workload)
    tstream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(tstream)
    ctx = fb.Context(local_rank, 0, tstream.cuda_stream)
    st = ctx.load_stream(s.types, s.times, s.n_types)
    # autotuner on: its timing trials run during the warm-up steps
    ctx.set_tuning(autotune=1)
    bins, thr, max_size = cfg["bins"], cfg["threshold"], cfg["max_size"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > L2 (129 MB)

    def step():
        res = ctx.mine_levelwise([st], bins, [thr], max_size)
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
            flush.fill_(k)  # evict the stream from L2 between timed steps (untimed)
            ev[k][0].record(tstream)
            stats.append(step())
            ev[k][1].record(tstream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ee = sum(x["episode_events"] for x in stats)
    ee_counted = sum(x["counted_episode_events"] for x in stats)
    pruned = float(np.mean([x["candidates_pruned"] for x in stats]))
    rel = sum(x["relevant_events"] for x in stats)
    cnt_ms = sum(x["count_kernel_ms"] for x in stats)
    launches = sum(x["kernel_launches"] for x in stats)
    t_max, value = aggregate_over_ranks(ms, ee, world, dev)

    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "value": ee * world / (t_max / 1e3), "ms_per_step": t_max / args.steps,
                              "count_kernel_ms_per_step": cnt_ms / args.steps, "gpu_launches": int(launches)}))
        st.free()
        ctx.close()
        return

    sparse_launches = sum(x["sparse_launches"] for x in stats)
    graph_tails = sum(x["graph_tails"] for x in stats)

    # --- plain per-level GPU path (comparison): same step, one thread per episode
    ctx.set_tuning(plain_path=1)
    step()
    torch.cuda.synchronize()
    pe = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    pst = []
    p_steps = max(1, min(args.steps, 3))
    flush.fill_(7)
    pe[0].record(tstream)
    for _ in range(p_steps):
        pst.append(step())
    pe[1].record(tstream)
    torch.cuda.synchronize()
    p_ms = pe[0].elapsed_time(pe[1])
    ctx.set_tuning(autotune=1)
    plain_value = sum(x["episode_events"] for x in pst) / (p_ms / 1e3)

    # --- end to end through the C ABI from host buffers
    types_pin = torch.from_numpy(s.types.view(np.int16)).pin_memory()
    times_pin = torch.from_numpy(s.times).pin_memory()
    e2e_ms = 0.0
    e2e_ee = 0.0
    d2h = 0
    for k in range(max(1, min(args.steps, 5))):
        flush.fill_(k)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(tstream)
        st2 = ctx.load_stream(types_pin.numpy().view(np.uint16), times_pin.numpy(), s.n_types)
        res = ctx.mine_levelwise([st2], bins, [thr], max_size)
        out_bytes = 0
        for N in range(1, max_size + 1):
            eps, counts = res.level(0, N)
            out_bytes += len(counts) * (4 + 2 * N + 8 * max(N - 1, 0) + 8)
        e2e_ee += res.stats()["episode_events"]
        res.free()
        st2.free()
        b.record(tstream)
        torch.cuda.synchronize()
        e2e_ms += a.elapsed_time(b)
        d2h = out_bytes
    e2e_steps = max(1, min(args.steps, 5))
    e2e_value = e2e_ee * world / (e2e_ms / 1e3)

    c3 = None if args.no_c3 else c3_leg(ctx, tstream, flush)
    if rank != 0:
        return
    peaks = _peaks()
    clocks = clk.summary()
    # roofline of the dominant kernel (the tiled exact-count kernel): its
    # algorithmic work is one state update per relevant (episode, event) pair
    # (events whose type is one of the episode's node types); peak = one
    # lane-instruction per lane per cycle: SMs x 4 schedulers x 32 lanes x clock.
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_alu = props.multi_processor_count * 128 * sm_max * 1e6
    achieved = rel / (cnt_ms / 1e3) if cnt_ms > 0 else 0.0
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # algorithmic bytes of the count kernels per step: the stream read once per
    # level pass (6 B/event) + candidate CSR (~22 B/candidate) + counts (4 B)
    levels = np.mean([x["levels"] for x in stats])
    cand = np.mean([x["candidates_counted"] + x["candidates_pruned"] for x in stats])
    alg_bytes = (levels - 1) * 6 * s.n + cand * 26
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": desc + f" (n={s.n}, levels 1-{max_size}, threshold {thr})",
                   "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written between timed steps (stream 6.4 MB < L2)",
                   "candidates_per_step": float(cand), "levels": float(levels),
                   "numerator": "every generated candidate x n (resolved by the exact count or, at level 2, "
                                "by the upper-bound pre-pass)",
                   "pruned_by_prepass_per_step": pruned},
        "counted_exact": {"value": ee_counted * world / (t_max / 1e3), "unit": UNIT,
                          "note": "episode-events resolved by the exact counting kernels only"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_alu,
                     "unit": "relevant episode-events/s", "frac": achieved / peak_alu,
                     "traffic": None,
                     "note": "peak = SMs x 128 lanes x sm_max_mhz (one lane-op per relevant episode-event)"},
        "hbm": {"achieved_gbs": alg_bytes / (cnt_ms / 1e3 / args.steps) / 1e9 if cnt_ms else None,
                "peak_gbs": hbm_peak,
                "frac": (alg_bytes / (cnt_ms / 1e3 / args.steps) / 1e9) / hbm_peak if cnt_ms else None},
        "count_kernel_ms_per_step": cnt_ms / args.steps,
        "plain_gpu": {"value": plain_value, "unit": UNIT, "ms_per_step": p_ms / p_steps,
                      "speedup_of_tiled": value / world / plain_value if plain_value else None},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(6 * s.n),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms / e2e_steps},
        "gpu_launches": int(launches),
        "kernels": {"sparse_launches_per_step": sparse_launches / args.steps,
                    "graph_tail_steps": graph_tails},
        "c3_batched_counting": c3,
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(s, cfg)
    print(json.dumps(line), flush=True)
    st.free()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c3", action="store_true", help="skip the batched-counting (C3) leg")
    ap.add_argument("--quick", action="store_true",
                    help="time the tiled path only (no plain-path, e2e or CPU legs); for profiling")
    ap.add_argument("--case", default=None,
                    help="run one small fixed invocation for profiling (c2_level2_tiled, c3_mid_sparse, c2_mining)")
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

#!/usr/bin/env python3
"""Throughput of the GPA stall-blame path on GB300.

A step is one pass of the whole path over one batch: zero the counters,
aggregate the batch's packed PC samples (Sec. 2.1), reaching definitions and
backward slicing, pruning and Eq. 1 apportioning (Sec. 4), roll-up,
optimizer matching and estimators (Sec. 5). The default workload is the
batched uneven one: 2,000 synthetic SASS-like functions of 50-20,000
instructions (log-uniform) and 5e8 packed samples (4 GB, larger than L2, so
no L2 flush is needed between steps).

  value  blamed PC samples/s with samples and program resident in HBM
  e2e    the same through the C ABI from pinned host memory: host->device copy
         of the samples inside the timed region, advice copied back to the host
The default run also records, at one GPU, the serving workload (p50/p99
ingest-to-advice latency) and the large stress kernel (one function of 200,000
instructions, 1e9 samples streamed from pinned host memory every step).
Prints one JSON line on rank 0. Under torchrun every rank processes its own
batch (seeded by rank) on its own GPU with no data-path collective (weak scaling).
`--impl reference` times the CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "blamed PC samples/s & analysed instrs/s (batched vs plain); p99 advise latency"
UNIT = "samples/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpa", choices=["gpa", "reference"])
    ap.add_argument("--workload", default="batched", choices=["plain", "rodinia", "batched", "large"])
    ap.add_argument("--samples", type=int, default=0, help="override the workload's sample count")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-functions", type=int, default=250, help="functions in the CPU-baseline sample")
    ap.add_argument("--cpu-samples", type=int, default=8_000_000, help="sample cap of the CPU-baseline sample")
    ap.add_argument("--hist-variant", type=int, default=None, help="aggregation kernel variant (gpa_options)")
    ap.add_argument("--options", default="", help="gpa_options fields as JSON, e.g. '{\"search_slots\": 1216}'")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the library's default schedule without tuning it on the workload first")
    ap.add_argument("--serving", action="store_true", help="run the serving workload instead")
    ap.add_argument("--sessions", type=int, default=200, help="serving: sessions")
    ap.add_argument("--serving-sessions", type=int, default=100,
                    help="sessions of the serving record in the default run (0 to skip)")
    ap.add_argument("--large-samples", type=int, default=1_000_000_000,
                    help="samples of the large stress kernel's record in the default run, streamed from "
                         "pinned host memory (0 to skip)")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=8, help="serving: concurrent sessions")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serving: device-memory admission budget")
    ap.add_argument("--plain-workload", default="rodinia",
                    help="workload of the batched-vs-plain comparison ('' to skip)")
    ap.add_argument("--functions", type=int, default=0, help="keep only the first N functions (profiling runs)")
    ap.add_argument("--search-slots", type=int, default=0, help="third-tier search warps (0 = library default)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel: str):
    """Per-launch DRAM bytes of `kernel` from profiles/traffic.json, or None if the
    kernel source changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
        return rec if h == rec["source_sha"] else None
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    v = [x.strip() for x in line.split(",")]
                    if len(v) >= 8 and v[0].replace(".", "").isdigit():
                        rows.append(v)
        except Exception:
            pass
        finally:
            if self.path:
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[0]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][1]), "reasons": reasons,
                "power_w_max": max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit()),
                "samples": len(rows)}


def make_workload(name: str, seed: int, n_override: int = 0, functions: int = 0):
    """The workload's program (with a call table: a tenth of the functions are device
    functions called from other functions, for Function Inlining) and sample count.
    Returns (generator handle for the samples, program arrays, samples)."""
    ps, ns, kz = synth.workload(name, seed=seed)
    if functions:
        ps = ps[:functions]
    P = synth.make_program(ps, kz, kseed=seed)
    return P, synth.add_calls(P, 0.1, seed=seed), (n_override or ns)


def cpu_sample(P, n_total: int, k_funcs: int, seed: int, cap: int):
    """The oracle's bounded sample: functions 0..k_funcs-1 with the samples of their
    launch runs, in stream order, up to `cap` samples (regenerated run by run from
    the counter-based stream, so they are the very samples the GPU counts)."""
    starts, kern = P.launch_runs(n_total, seed=seed)
    parts, got = [], 0
    for r in np.flatnonzero(kern < k_funcs):
        take = min(int(starts[r + 1] - starts[r]), cap - got)
        if take <= 0:
            break
        parts.append(P.samples(take, seed=seed, n0=int(starts[r]), total=n_total))
        got += take
    sub = np.concatenate(parts) if parts else np.zeros(0, np.uint64)
    return sub, got


def reduce_max(x: float, world: int) -> float:
    """The largest x over the ranks (x itself at one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(n_per_rank: int, ms: float, world: int) -> float:
    """Whole-job samples/s: every rank processed n_per_rank in ms (the slowest rank's time)."""
    return world * n_per_rank / (ms / 1e3)


def plain_vs_batched(gpa, workload: str, seed: int, dev, stream, reps: int = 3) -> dict:
    """Samples/s of one batched program over all functions of `workload` against one
    program per function (the plain form), each fed its own launch runs; same GPU,
    same samples, eager steps (reset, ingest, blame, advise kept on the device)."""
    import torch
    P, arrays, n = make_workload(workload, seed, 0, 0)
    s = P.samples(n, seed=seed)
    ctx = gpa.Context(synth.default_arch())
    try:
        progs, inputs = [ctx.load_program(arrays)], [torch.from_numpy(s.view(np.int64)).to(dev)]
        plain, plain_in = [], []
        for f in range(P.n_functions):
            plain.append(ctx.load_program(synth.subprogram(arrays, f, f + 1)))
            plain_in.append(torch.from_numpy(synth.rebase_samples(s, f, f + 1).view(np.int64)).to(dev))

        def run(ps, xs):
            for p_, x in zip(ps, xs):
                p_.reset(stream)
                if x.numel():
                    p_.ingest(x, stream=stream)
                p_.blame(stream)
                p_.advise(fetch=False, stream=stream)

        out = {}
        for name, ps, xs in (("batched", progs, inputs), ("plain", plain, plain_in)):
            run(ps, xs)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                run(ps, xs)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            out[name] = {"value": n / (ms / 1e3), "ms_per_step": ms}
            for p_ in ps:
                st, _ = p_.status(stream)
                if st != 0:
                    raise SystemExit(f"device status {st} in the {name} form")
        return {"workload": workload, "functions": P.n_functions, "samples": n, "unit": UNIT,
                "batched": out["batched"], "plain": out["plain"],
                "speedup": out["batched"]["value"] / out["plain"]["value"]}
    finally:
        ctx.close()


def serving_measure(a, gpa, dev, n_sessions: int) -> dict:
    """Serving workload: Poisson session arrivals (mean a.rate per second) through the
    continuous-batching server, p50/p99 ingest-to-advice latency and samples/s, against
    the same sessions one at a time."""
    import torch
    from paper_2009_04061_gb300.serving import Server, Session, latency_summary, one_at_a_time, serve
    arch = synth.default_arch()
    specs = synth.serving_sessions(n_sessions, seed=a.seed, rate_per_s=a.rate)
    sessions, keep = [], []
    for i, d in enumerate(specs):
        P = synth.make_program(d["params"], 1.0, d["seed"])
        host = torch.empty(d["n_samples"], dtype=torch.int64).pin_memory()
        P.samples(d["n_samples"], seed=d["seed"], out=host.numpy().view(np.uint64))
        keep.append(host)
        sessions.append(Session(i, P.arrays, host.numpy().view(np.uint64)))
    arrivals = [d["t_arrival"] for d in specs]
    budget = int(a.budget_gb * (1 << 30))
    opts = json.loads(a.options) if a.options else None
    srv = Server(arch, slots=a.slots, budget_bytes=budget, options=opts)
    try:
        # warm each slot (lazy staging buffers, first-launch costs) with a small session
        small = min(range(len(sessions)), key=lambda i: sessions[i].samples.size)
        serve(srv, [sessions[small]] * a.slots, [0.0] * a.slots)
        torch.cuda.synchronize(dev)
        with Clocks(torch.cuda.current_device()) as clk:
            res = serve(srv, sessions, arrivals)
    finally:
        srv.close()
    mix = latency_summary(res)
    t_seq, res1 = one_at_a_time(arch, sessions, options=opts)
    seq = latency_summary(res1)
    n = sum(s.samples.size for s in sessions)
    return {
        "value": mix["samples_per_s"], "unit": UNIT, "span_s": mix["span_s"],
        "config": {"workload": "serving", "sessions": len(sessions), "rate_per_s": a.rate, "slots": a.slots,
                   "budget_gb": a.budget_gb, "samples": n, "options": opts,
                   "instructions": int(sum(int(s.program["n_instr"]) for s in sessions))},
        "latency_ms": {"p50": mix["p50_ms"], "p99": mix["p99_ms"], "mean": mix["mean_ms"], "max": mix["max_ms"]},
        "one_at_a_time": {"value": n / t_seq, "unit": UNIT, "seconds": t_seq,
                          "latency_ms_without_queueing": {"p50": seq["p50_ms"], "p99": seq["p99_ms"]}},
        "speedup_vs_one_at_a_time": mix["samples_per_s"] / (n / t_seq),
        "clocks": clk.summary(),
    }


def serving_bench(a, gpa, dev):
    """The serving workload alone; prints one JSON line."""
    r = serving_measure(a, gpa, dev, a.sessions)
    print(json.dumps({
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": r["span_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": r["config"],
        "latency_ms": r["latency_ms"], "one_at_a_time": r["one_at_a_time"],
        "speedup_vs_one_at_a_time": r["speedup_vs_one_at_a_time"], "clocks": r["clocks"],
    }), flush=True)


def pinned_h2d_gbs(host, dev, nbytes: int = 1 << 31) -> float:
    """Best of three plain copies of `nbytes` from pinned host memory to the device (GB/s)."""
    import torch
    m = min(host.numel(), nbytes // 8)
    src = host[:m]
    dst = torch.empty(m, dtype=torch.int64, device=dev)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize(dev)
        best = max(best, 8 * m / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del dst
    return best


def large_measure(a, gpa, dev, steps: int = 3) -> dict:
    """The large stress kernel (one function of 200,000 instructions) at its full
    sample count, streamed from pinned host memory through the C ABI every step
    (the aggregation kernel reads the pinned buffer over the host link): the
    step time (ingest, blame, advice copied out), the cold first step, and the
    ingest rate against a plain pinned host-to-device copy."""
    import torch
    P, arrays, n = make_workload("large", a.seed, a.large_samples)
    t0 = time.perf_counter()
    host = torch.empty(n, dtype=torch.int64).pin_memory()
    P.samples(n, seed=a.seed, out=host.numpy().view(np.uint64))
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    with gpa.Context(synth.default_arch()) as ctx:
        prog = ctx.load_program(arrays)
        bufs = prog.advice_buffers(pinned=True)
        try:
            def step():
                prog.reset(stream)
                prog.ingest_host(host, stream=stream)
                prog.blame(stream)
                return prog.advise(fetch=True, stream=stream, out=bufs)  # synchronizes the stream

            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            step()
            cold_ms = (time.perf_counter() - t0) * 1e3
            step()
            st, info = prog.status(stream)
            if st != 0:
                raise SystemExit(f"large workload: device status {st}: {info}")
            cnt, bad = prog.counts(stream)
            assert int(cnt.sum()) + bad == n, "large workload: counts do not add up"
            times = []
            for _ in range(steps):
                t0 = time.perf_counter()
                adv = step()
                times.append((time.perf_counter() - t0) * 1e3)
            d2h = sum(v.nbytes for v in adv.values())
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            prog.reset(stream)
            e[0].record(stream)
            prog.ingest_host(host, stream=stream)
            e[1].record(stream)
            prog.blame(stream)
            e[2].record(stream)
            torch.cuda.synchronize(dev)
            ingest_ms, blame_ms = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        finally:
            prog.unload()
    h2d = pinned_h2d_gbs(host, dev)
    ms = statistics.median(times)
    ingest_gbs = 8 * n / (ingest_ms / 1e3) / 1e9
    return {"workload": "large", "functions": P.n_functions, "instructions": P.n_instr, "blocks": P.n_blocks,
            "samples": n, "sample_bytes": 8 * n, "source": "pinned host memory, read over the host link each step",
            "ms_per_step": ms, "samples_per_s": n / (ms / 1e3), "cold_first_step_ms": cold_ms,
            "ingest_ms": ingest_ms, "blame_ms": blame_ms, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": d2h,
            "host_link": {"ingest_gbs": ingest_gbs, "pinned_h2d_gbs": h2d, "frac": ingest_gbs / h2d},
            "general_searches": info["general_searches"], "largest_search_nodes": info["max_nodes"],
            "generate_s": gen_s}


def e2e_overlapped(gpa, arrays, host, opts, stats, sm, dev, reps: int) -> float:
    """Seconds per step end to end with consecutive steps overlapped, as a user feeding
    a stream of batches would run them: two contexts, each with the program loaded, its
    own stream, pinned advice arrays and host thread; step k runs on pair k % 2, so one
    step's ingest over the host link runs beside the other's blame. Every step copies its
    own samples from pinned host memory and reads its own advice back inside the timed
    region, through the same calls as the sequential measurement."""
    import threading
    import torch
    arch = synth.default_arch()
    pairs, errors = [], []
    try:
        for _ in range(2):
            c = gpa.Context(arch, opts or None)
            p = c.load_program(arrays)
            p.set_launch_stats(stats, sm)
            pairs.append((c, p, torch.cuda.Stream(dev), p.advice_buffers(pinned=True)))

        def run(i, k):
            try:
                torch.cuda.set_device(dev)  # the current device is per host thread
                _, p, st, b = pairs[i]
                for _ in range(k):
                    p.reset(st)
                    p.ingest_host(host, stream=st)
                    p.blame(st)
                    p.advise(fetch=True, stream=st, out=b)  # synchronizes st
            except Exception as e:  # noqa: BLE001 (re-raised below)
                errors.append(e)

        for i in range(2):
            run(i, 2)  # warm-up: kernels loaded, search tiers known
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        threads = [threading.Thread(target=run, args=(i, reps)) for i in range(2)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        te = (time.perf_counter() - t0) / (2 * reps)
        if errors:
            raise errors[0]
        for _, p, st, _ in pairs:
            code, info = p.status(st)
            if code != 0:
                raise SystemExit(f"overlapped end to end: device status {code}: {info}")
        return te
    finally:
        for c, p, _, _ in pairs:
            p.unload()
            c.close()


def run_oracle_once(P, sub, k_funcs, threads: int = 1):
    """Seconds the oracle takes for the bounded sample: the histogram of `sub` and
    the analysis of functions 0..k_funcs-1, on a program cut to those functions.
    With threads > 1 the samples are counted in `threads` slices and the functions
    analyzed one per task on a pool of host threads (the oracle's C++ runs outside
    the interpreter lock), and the slice counts summed: the same results."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    arch = synth.default_arch()
    Q = synth.subprogram(P, 0, k_funcs)
    t0 = time.perf_counter()
    if threads <= 1:
        cnt, _ = oracle.histogram(Q, sub)
        oracle.analyze(Q, arch, cnt, 0, k_funcs)
        return time.perf_counter() - t0
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda x: oracle.histogram(Q, x)[0], np.array_split(sub, threads)))
        cnt = parts[0]
        for c in parts[1:]:
            cnt += c
        sizes = np.diff(np.asarray(Q["func_instr_off"]))
        order = np.argsort(-sizes, kind="stable")          # largest functions first
        list(ex.map(lambda f: oracle.analyze(Q, arch, cnt, int(f), int(f) + 1), order))
    return time.perf_counter() - t0


def host_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def reference_arm(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    P, arrays, n = make_workload(a.workload, a.seed, a.samples)
    threads = host_threads()
    k_funcs = min(P.n_functions, max(1, a.cpu_functions // 4))
    sub, m = cpu_sample(P, n, k_funcs, a.seed, max(1, a.cpu_samples // 4))
    for _ in range(a.warmup):
        run_oracle_once(arrays, sub, k_funcs, threads)
    ts = [run_oracle_once(arrays, sub, k_funcs, threads) for _ in range(a.steps)]
    t = statistics.mean(ts)
    v = sub.size / t
    instr = int(P.func_instr_off[k_funcs])
    sample = (f"functions 0..{k_funcs - 1} of the {a.workload} workload ({instr} instructions) with the "
              f"first {sub.size} samples of their launch runs; oracle over functions on {threads} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": a.workload, "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        return reference_arm(a)
    import torch
    import torch.distributed as dist

    import paper_2009_04061_gb300 as gpa

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if a.serving:
        if rank == 0:
            serving_bench(a, gpa, dev)
        if world > 1:
            dist.destroy_process_group()
        return

    P, arrays, n = make_workload(a.workload, a.seed + rank, a.samples, a.functions)
    host = torch.empty(n, dtype=torch.int64).pin_memory()
    P.samples(n, seed=a.seed + rank, out=host.numpy().view(np.uint64))
    d = host.to(dev, non_blocking=False)
    opts = {"search_slots": a.search_slots} if a.search_slots else {}
    if a.hist_variant is not None:
        opts["hist_variant"] = a.hist_variant
    if a.options:
        opts.update(json.loads(a.options))
    tuned = None
    if not a.no_autotune and not a.options and a.hist_variant is None and not a.search_slots:
        from paper_2009_04061_gb300 import autotune
        stream0 = torch.cuda.current_stream(dev)
        with gpa.Context(synth.default_arch(), opts or None) as c0:
            fixed_ms = autotune.time_step(c0, arrays, d, stream0)
        best, table = autotune.tune(synth.default_arch(), arrays, d, stream0)
        tuned = {"fixed_ms_per_step": fixed_ms, "tuned_ms_per_step": next(t for o, t in table if o == best),
                 "options": best, "candidates_tried": len(table),
                 "searched": {name: list(values) for name, values in autotune.DIMENSIONS}}
        opts = best
    torch.cuda.synchronize(dev)
    t_load = time.perf_counter()
    ctx = gpa.Context(synth.default_arch(), opts or None)
    prog = ctx.load_program(arrays)
    torch.cuda.synchronize(dev)
    load_ms = (time.perf_counter() - t_load) * 1e3
    # Seeded launch statistics of the workload's kernels on this GPU's SM model:
    # the advice step also runs the parallel optimizers (Table 2, Eqs. 6-10).
    lstats = synth.launch_stats(P.n_functions, a.seed)
    sm_model = gpa.gpa_sm_model_of_device(torch.cuda.current_device())
    prog.set_launch_stats(lstats, sm_model)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        prog.reset(stream)
        if ev:
            ev[0].record(stream)
        prog.ingest(d, stream=stream)
        if ev:
            ev[1].record(stream)
        prog.blame(stream)
        if ev:
            ev[2].record(stream)
        prog.advise(fetch=False, stream=stream)
        if ev:
            ev[3].record(stream)

    # The cold step: the first one of the freshly loaded program (kernels load on
    # first use, and no search knows its tier yet), as a profile analysed once sees it.
    cold = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize(dev)
    t_cold = time.perf_counter()
    step(cold)
    torch.cuda.synchronize(dev)
    cold_wall_ms = (time.perf_counter() - t_cold) * 1e3
    cold_step = {"ms": cold[0].elapsed_time(cold[3]), "wall_ms": cold_wall_ms,
                 "blame_ms": cold[1].elapsed_time(cold[2]), "load_ms": load_ms}
    for _ in range(a.warmup):
        step()
    st, info = prog.status(stream)
    if st != 0:
        raise SystemExit(f"device status {st} after warm-up: {info}; search overflow bits "
                         f"{prog.search_profile(stream)['overflow_bits']:#x}")
    cnt, bad = prog.counts(stream)
    assert int(cnt.sum()) + bad == n, "counts do not add up to the samples ingested"

    # Eager steps: the phase split and the aggregation kernel's launch time
    # (the roofline's denominator), from events around each call.
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(a.steps)]
    for k in range(a.steps):
        step(evs[k])
    torch.cuda.synchronize(dev)
    phase = {
        "ingest_ms": statistics.mean(e[0].elapsed_time(e[1]) for e in evs),
        "blame_ms": statistics.mean(e[1].elapsed_time(e[2]) for e in evs),
        "advise_ms": statistics.mean(e[2].elapsed_time(e[3]) for e in evs),
    }
    eager_ms = statistics.mean(e[0].elapsed_time(e[3]) for e in evs)

    # The timed steps: the whole step captured once as a CUDA graph, one graph
    # launch per step.
    prog.capture_step(d)
    prog.launch_step(stream)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = ctx.launches()
    with Clocks(local) as clk:
        start.record(stream)
        for k in range(a.steps):
            prog.launch_step(stream)
        end.record(stream)
        torch.cuda.synchronize(dev)
    launches = ctx.launches() - l0
    ms = start.elapsed_time(end) / a.steps
    st, info = prog.status(stream)
    if st != 0:
        raise SystemExit(f"device status {st} after the timed steps: {info}")
    ms = reduce_max(ms, world)
    if world > 1:
        dist.barrier()
    clocks = clk.summary()
    value = weak_value(n, ms, world)
    instr_per_s = world * P.n_instr / (ms / 1e3)

    # Roofline of the aggregation kernel: 8 algorithmic bytes per sample over
    # its launch time in the eager steps above (the reset memset runs before
    # the first event).
    hbm_peak, peak_kind = load_peaks()
    t_hist = phase["ingest_ms"] / 1e3
    achieved = 8.0 * n / t_hist / 1e9
    kname = "k_histogram_runs" if not opts.get("hist_variant") else "k_histogram"
    tr = traffic_record(kname)
    roofline = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": f"{peak_kind} (copy bandwidth)",
                "traffic": (tr["dram_bytes_per_sample"] * n) if tr else None,
                "algorithmic_bytes": 8 * n, "launch_ms": t_hist * 1e3}

    # End to end through the C ABI from pinned host memory.
    e2e = None
    if not a.no_e2e:
        bufs = prog.advice_buffers(pinned=True)  # the advice lands in the same pinned arrays every step
        for _ in range(2):
            prog.reset(stream)
            prog.ingest_host(host, stream=stream)
            prog.blame(stream)
            adv = prog.advise(fetch=True, stream=stream, out=bufs)
        d2h = sum(v.nbytes for v in adv.values())
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        reps = max(1, min(a.steps, 5))
        for _ in range(reps):
            prog.reset(stream)
            prog.ingest_host(host, stream=stream)
            prog.blame(stream)
            adv = prog.advise(fetch=True, stream=stream, out=bufs)  # synchronizes the stream
        te = (time.perf_counter() - t0) / reps
        te = reduce_max(te, world)
        # The host link: ingest from pinned host memory alone (CUDA events) against a
        # plain pinned host-to-device copy.
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        prog.reset(stream)
        e0.record(stream)
        prog.ingest_host(host, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ingest_gbs = 8 * n / (e0.elapsed_time(e1) / 1e3) / 1e9
        h2d = pinned_h2d_gbs(host, dev)
        to = reduce_max(e2e_overlapped(gpa, arrays, host, opts, lstats, sm_model, dev, reps), world)
        e2e = {"value": weak_value(n, to * 1e3, world), "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": d2h,
               "ms_per_step": to * 1e3,
               "schedule": "consecutive steps overlapped: two contexts, steps alternating on two streams and host "
                           "threads; each step copies its samples in and its advice out inside the timed region",
               "sequential": {"value": weak_value(n, te * 1e3, world), "ms_per_step": te * 1e3},
               "host_link": {"ingest_gbs": ingest_gbs, "pinned_h2d_gbs": h2d, "frac": ingest_gbs / h2d}}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline and a.workload == "large":
        cpu = {"unavailable": "the oracle's analysis of the one 200,000-instruction function does not finish in "
                              "a bounded sample (its searches take hours on the host); see the batched workload"}
    elif rank == 0 and world == 1 and not a.no_cpu_baseline:
        k_funcs = min(P.n_functions, a.cpu_functions)
        sub, m = cpu_sample(P, n, k_funcs, a.seed, a.cpu_samples)
        threads = host_threads()
        t_all = run_oracle_once(arrays, sub, k_funcs, threads)
        t_one = run_oracle_once(arrays, sub, k_funcs, 1)
        sample = (f"functions 0..{k_funcs - 1} ({int(P.func_instr_off[k_funcs])} instructions) with the first "
                  f"{sub.size} samples of their launch runs")
        cpu = {"value": sub.size / t_all, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{sample}; {t_all:.1f} s on {threads} host threads (functions in parallel)",
               "single_core": {"value": sub.size / t_one, "unit": UNIT, "cores": 1, "seconds": t_one}}

    # Single dependency coverage (Sec. 6) of this workload, before and after pruning.
    # Its searches have no latency bound, so on a very large function they can
    # outgrow the largest arena; the diagnostic then says so.
    try:
        nodes, single_before, single_after = prog.coverage(stream)
        coverage = {"stalled_uses": nodes, "before_pruning": single_before / max(nodes, 1),
                    "after_pruning": single_after / max(nodes, 1)}
    except gpa.GpaError as e:
        coverage = {"unavailable": str(e)}
    adv = prog.get_advice(stream)
    parallel = {"block_increase_matched": int(adv["par_match"][:, 0].sum()),
                "thread_increase_matched": int(adv["par_match"][:, 1].sum()),
                "largest_speedup": float(adv["par_speedup"].max())}

    bvp = None
    if rank == 0 and world == 1 and a.plain_workload:
        bvp = plain_vs_batched(gpa, a.plain_workload, a.seed, dev, stream)
    serving = None
    if rank == 0 and world == 1 and a.serving_sessions > 0:
        prog.unload()
        ctx.close()
        prog = ctx = None
        del d
        torch.cuda.empty_cache()
        serving = serving_measure(a, gpa, dev, a.serving_sessions)
    large = None
    if rank == 0 and world == 1 and a.large_samples > 0 and a.workload != "large":
        if prog is not None:
            prog.unload()
            ctx.close()
            prog = ctx = None
            del d
            torch.cuda.empty_cache()
        large = large_measure(a, gpa, dev)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int64", "data": "synthetic",
            "config": {"workload": a.workload, "functions": P.n_functions, "instructions": P.n_instr,
                       "blocks": P.n_blocks, "loops": P.n_loops, "samples_per_gpu": n,
                       "call_sites": int(arrays["call_site"].size),
                       "device_functions": int(np.unique(arrays["call_callee"]).size),
                       "sample_bytes_per_gpu": 8 * n, "l2": "inputs (samples) larger than L2, no flush",
                       "parallelism": f"replicas x{world}, no collective on the data path"},
            "analysed_instrs_per_s": instr_per_s, "phases_ms": phase, "eager_ms_per_step": eager_ms,
            "cuda_graph": True,
            "general_searches": info["general_searches"], "search_tiers": [
                info["general_searches"], info["tier2_searches"], info["tier3_searches"]],
            "largest_search_nodes": info["max_nodes"], "gpu_launches": launches,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "batched_vs_plain": bvp, "autotune": tuned, "options": opts, "dependency_coverage": coverage,
            "parallel_optimizers": parallel, "cold_first_step": cold_step, "serving": serving,
            "large_stress_kernel": large,
        }
        print(json.dumps(line), flush=True)
    if prog is not None:
        prog.unload()
        ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

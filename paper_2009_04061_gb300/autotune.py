"""Schedule autotuner: times steps (reset, ingest, blame, advice) of a program
under candidate context options and keeps the fastest.

The options it searches are the launch schedules of the path, one dimension
at a time (a coordinate search from the library defaults, each dimension
tried with the best values found so far for the others):

- aggregation: the kernel variant (the per-segment window kernel, or a
  grid-strided hash kernel of one of three CTA shapes and hash sizes);
- aggregation tile chunk: tiles of 8,192 samples an SM claims at a time (the
  window kernel's scheduling grain);
- reaching-definitions schedule: a CTA per function staged in shared memory
  (launched by size class) against the windowed kernel, a lane per basic block
  in windows of 32 blocks, for every function;
- search tiers: the node capacity of the first tier's shared-memory arenas, the
  first tier's warps per SM, and the number of global-memory search warps per SM.

A dimension's values are compared by the time of the phase it schedules
(ingest for the aggregation options, blame for the others). Every candidate
computes the same results; only the time differs.
"""
from __future__ import annotations

from . import gpa

# Candidate values per dimension (the first is the library default) and the
# phase of the step the dimension schedules, by whose time it is judged.
DIMENSIONS = [
    ("hist_variant", (0, 1, 2, 3)),
    ("hist_chunk", (24, 8, 16, 32, 48)),
    ("reach_schedule", (0, 1)),
    ("small_search_nodes", (64, 128, 32)),
    ("small_search_warps", (24, 16, 20)),
    ("search_slots_per_sm", (0, 12, 16)),
]
PHASE = {"hist_variant": "ingest", "hist_chunk": "ingest", "reach_schedule": "blame", "small_search_nodes": "blame",
         "small_search_warps": "blame", "search_slots_per_sm": "blame"}


def _options(point: dict, sms: int) -> dict:
    o = {k: v for k, v in point.items() if k != "search_slots_per_sm"}
    if point.get("search_slots_per_sm"):
        o["search_slots"] = point["search_slots_per_sm"] * sms
    if o.get("hist_variant", 0) != 0:
        o.pop("hist_chunk", None)  # the chunk only schedules the window kernel
    return o


def time_phases(ctx, arrays, dev_samples, stream, reps: int = 3) -> dict:
    """Milliseconds per step of the program on this context, and of its ingest, blame
    and advise phases (CUDA events around each call, mean of `reps` eager steps after
    one untimed step)."""
    import torch
    prog = ctx.load_program(arrays)
    try:
        def step(ev=None):
            prog.reset(stream)
            if ev:
                ev[0].record(stream)
            prog.ingest(dev_samples, stream=stream)
            if ev:
                ev[1].record(stream)
            prog.blame(stream)
            if ev:
                ev[2].record(stream)
            prog.advise(fetch=False, stream=stream)
            if ev:
                ev[3].record(stream)
        step()
        st, info = prog.status(stream)
        if st != 0:
            raise RuntimeError(f"device status {st}: {info}")
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
        for e in evs:
            step(e)
        evs[-1][3].synchronize()
        mean = lambda a, b: sum(e[a].elapsed_time(e[b]) for e in evs) / reps  # noqa: E731
        return {"step": mean(0, 3), "ingest": mean(0, 1), "blame": mean(1, 2), "advise": mean(2, 3)}
    finally:
        prog.unload()


def time_step(ctx, arrays, dev_samples, stream, reps: int = 3) -> float:
    """Milliseconds per step (reset, ingest, blame, advise) of the program on this context."""
    return time_phases(ctx, arrays, dev_samples, stream, reps)["step"]


def tune(arch, arrays, dev_samples, stream=None, dims=None, reps: int = 3) -> tuple[dict, list[tuple[dict, float]]]:
    """Returns (best options, [(options, ms per step)] for every candidate timed).
    dims: a list of (name, values) to search (default DIMENSIONS); the first value of
    each dimension is the starting point, and a dimension's values are compared by
    the time of the phase it schedules (PHASE; the whole step for others)."""
    import torch
    stream = stream or torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    dims = dims or DIMENSIONS
    table: list[tuple[dict, float]] = []
    seen: dict[tuple, dict] = {}

    def run(point):
        opts = _options(point, sms)
        key = tuple(sorted(opts.items()))
        if key not in seen:
            with gpa.Context(arch, opts) as c:
                seen[key] = time_phases(c, arrays, dev_samples, stream, reps)
            table.append((opts, seen[key]["step"]))
        return seen[key]

    point = {name: values[0] for name, values in dims}
    best = run(point)
    for name, values in dims:
        if name == "hist_chunk" and point.get("hist_variant", 0) != 0:
            continue
        phase = PHASE.get(name, "step")
        for v in values[1:]:
            trial = dict(point, **{name: v})
            t = run(trial)
            if t[phase] < best[phase]:
                best, point = t, trial
    return _options(point, sms), table

"""Schedule autotuner: times whole steps (reset, ingest, blame, advice) of a
program under candidate context options and keeps the fastest.

The options it searches are the launch schedules of the path: the
aggregation kernel's variant (hash size, CTA shape, CTAs per SM), the node
capacities of the search tiers (which searches run with several warps per CTA
in shared memory, alone in a larger shared-memory arena, or in global
memory) and the number of global-memory search warps. Every candidate
computes the same results; only the time differs.
"""
from __future__ import annotations

import itertools

from . import gpa

DEFAULT = {}


def candidates(sms: int) -> list[dict]:
    out = []
    for hv, small, mid, slots in itertools.product((0, 1, 2, 3), (64, 128), (128, 512), (4, 21)):
        out.append(dict(hist_variant=hv, small_search_nodes=small, mid_search_nodes=mid, search_slots=slots * sms))
    return out


def time_step(ctx, arrays, dev_samples, stream, reps: int = 2) -> float:
    """Milliseconds per step of the program on this context (one untimed step first)."""
    import torch
    prog = ctx.load_program(arrays)
    try:
        def step():
            prog.reset(stream)
            prog.ingest(dev_samples, stream=stream)
            prog.blame(stream)
            prog.advise(fetch=False, stream=stream)
        step()
        st, info = prog.status(stream)
        if st != 0:
            raise RuntimeError(f"device status {st}: {info}")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            step()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps
    finally:
        prog.unload()


def tune(arch, arrays, dev_samples, stream=None, cands: list[dict] | None = None, reps: int = 2,
         prune: int = 2) -> tuple[dict, list[tuple[dict, float]]]:
    """Returns (best options, [(options, ms)] for every candidate tried).

    Coordinate search: the aggregation variant first (search options at their
    defaults), then the search options with the best variant; `prune` keeps
    that many aggregation variants for the second round."""
    import torch
    stream = stream or torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    cands = cands or candidates(sms)
    table: list[tuple[dict, float]] = []

    def run(opts):
        with gpa.Context(arch, opts) as c:
            ms = time_step(c, arrays, dev_samples, stream, reps)
        table.append((opts, ms))
        return ms

    variants = sorted({c["hist_variant"] for c in cands})
    first = sorted(((run({"hist_variant": v}), v) for v in variants))[:prune]
    best_v = [v for _, v in first]
    for c in cands:
        if c["hist_variant"] in best_v:
            run(c)
    best = min(table, key=lambda t: t[1])[0]
    return best, table

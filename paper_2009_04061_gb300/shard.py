"""Sharding one batch over several GPUs: function ownership plus one exchange
of counts.

Step (a) is a sum over samples, so the counts of disjoint chunks of a sample
stream add up to the counts of the whole stream (Sec. 2.1); steps (b)-(d) work
on each function alone (Sec. 3: every launch context is analyzed separately).
A batch therefore shards as:

1. ownership: every function gets one owner rank, by a size-balanced longest
   processing time first (LPT) assignment of the functions' instruction counts;
2. every rank aggregates an even chunk of the sample stream over the whole
   program (counters of every function);
3. one exchange: the owner of each function receives the sum over the ranks
   of that function's count rows (a reduce of each owner's rows to it);
4. every owner runs blame and advice on a program of the functions it owns,
   with the exchanged counts (gpa_set_counts); nothing else is exchanged.

The results are those of the unsharded batch, function by function. The
module is host logic around the C ABI (the counts never leave the devices
except through torch.distributed).
"""
from __future__ import annotations

import numpy as np

N_CNT = 24  # counters per instruction: 12 classes x latency flag


def function_costs(arrays) -> np.ndarray:
    """Instructions per function: the size the assignment balances."""
    a = arrays.arrays if hasattr(arrays, "arrays") else arrays
    return np.diff(np.asarray(a["func_instr_off"], dtype=np.int64))


def lpt_owners(costs, world: int) -> np.ndarray:
    """Owner rank of every function: functions in order of decreasing cost (ties:
    lower function first), each to the rank with the least cost so far (ties: lower
    rank). The most loaded rank holds at most 4/3 of the optimum plus one function."""
    if world < 1:
        raise ValueError("world must be at least 1")
    costs = np.asarray(costs, dtype=np.int64)
    owner = np.zeros(costs.size, np.int32)
    load = np.zeros(world, np.int64)
    for f in np.argsort(-costs, kind="stable"):
        r = int(np.argmin(load))
        owner[f] = r
        load[r] += costs[f]
    return owner


def sample_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank's even chunk of an n-sample stream."""
    return n * rank // world, n * (rank + 1) // world


def _ranges(starts, lens) -> np.ndarray:
    """The concatenation of [starts[k], starts[k] + lens[k]) over k."""
    starts, lens = np.asarray(starts, dtype=np.int64), np.asarray(lens, dtype=np.int64)
    tot = int(lens.sum())
    if tot == 0:
        return np.zeros(0, np.int64)
    before = np.concatenate([[0], np.cumsum(lens)[:-1]])
    return np.repeat(starts - before, lens) + np.arange(tot, dtype=np.int64)


def instr_rows(arrays, funcs) -> np.ndarray:
    """Global instruction indices of the functions `funcs` (ascending), in order."""
    a = arrays.arrays if hasattr(arrays, "arrays") else arrays
    fio = np.asarray(a["func_instr_off"], dtype=np.int64)
    funcs = np.asarray(funcs, dtype=np.int64)
    return _ranges(fio[funcs], fio[funcs + 1] - fio[funcs])


def select_functions(arrays, funcs) -> tuple[dict, dict]:
    """The program made of the functions `funcs` (ascending) alone, in the layout of
    gpa_program_desc, and the maps back to the whole program: instr[k] / block[k] /
    loop[k] = the global index of the selection's k-th instruction / block / loop,
    func[k] its function. Line ids stay global (n_lines unchanged). A call whose
    site or callee is selected is kept, the other end -1 when not selected."""
    a = arrays.arrays if hasattr(arrays, "arrays") else arrays
    funcs = np.asarray(sorted(int(f) for f in funcs), dtype=np.int64)
    fio, fbo, flo = (np.asarray(a[k], dtype=np.int64) for k in ("func_instr_off", "func_block_off", "func_loop_off"))
    bio, so, do, uo = (np.asarray(a[k], dtype=np.int64) for k in ("block_instr_off", "succ_off", "def_off", "use_off"))
    succ, bl, lp, lh = (np.asarray(a[k], dtype=np.int64) for k in ("succ", "block_loop", "loop_parent", "loop_header"))
    instr = instr_rows(a, funcs)
    blocks = _ranges(fbo[funcs], fbo[funcs + 1] - fbo[funcs])
    loops = _ranges(flo[funcs], flo[funcs + 1] - flo[funcs])
    new_instr = np.full(int(fio[-1]), -1, np.int64)
    new_instr[instr] = np.arange(instr.size)
    new_block = np.full(int(fbo[-1]), -1, np.int64)
    new_block[blocks] = np.arange(blocks.size)
    new_loop = np.full(max(int(flo[-1]), 1), -1, np.int64)
    new_loop[loops] = np.arange(loops.size)
    new_func = np.full(fio.size - 1, -1, np.int64)
    new_func[funcs] = np.arange(funcs.size)

    def offsets(sizes):
        return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)

    def remap_loops(x):
        x = np.asarray(x, dtype=np.int64)
        return np.where(x >= 0, new_loop[np.maximum(x, 0)], -1).astype(np.int32)

    def csr(off, vals, rows):
        cnt = off[rows + 1] - off[rows]
        return offsets(cnt), np.asarray(vals)[_ranges(off[rows], cnt)]

    succ_off, succ_new = csr(so, succ, blocks)
    def_off, def_res = csr(do, np.asarray(a["def_res"]), instr)
    use_off, use_res = csr(uo, np.asarray(a["use_res"]), instr)
    # Calls with a selected site or callee; the other end, when not selected, becomes
    # -1 (a call out of or into the selection), so call sites and device functions
    # keep their status.
    cs = np.asarray(a.get("call_site", np.zeros(0, np.int32)), dtype=np.int64)
    cc = np.asarray(a.get("call_callee", np.zeros(0, np.int32)), dtype=np.int64)
    ns = np.where(cs >= 0, new_instr[np.maximum(cs, 0)], -1)
    nc = np.where(cc >= 0, new_func[np.maximum(cc, 0)], -1)
    keep = (ns >= 0) | (nc >= 0)
    order = np.argsort(ns[keep], kind="stable")
    ns, nc = ns[keep][order], nc[keep][order]
    sub = dict(
        n_functions=int(funcs.size), n_instr=int(instr.size), n_blocks=int(blocks.size), n_loops=int(loops.size),
        n_lines=int(a["n_lines"]),
        func_instr_off=offsets(fio[funcs + 1] - fio[funcs]), func_block_off=offsets(fbo[funcs + 1] - fbo[funcs]),
        func_loop_off=offsets(flo[funcs + 1] - flo[funcs]),
        block_instr_off=offsets(bio[blocks + 1] - bio[blocks]),
        succ_off=succ_off, succ=new_block[succ_new].astype(np.int32),
        opclass=np.asarray(a["opclass"])[instr].copy(), guard=np.asarray(a["guard"])[instr].copy(),
        iflags=np.asarray(a["iflags"])[instr].copy(), line=np.asarray(a["line"])[instr].astype(np.int32),
        def_off=def_off, def_res=def_res.astype(np.uint16), use_off=use_off, use_res=use_res.astype(np.uint16),
        block_loop=remap_loops(bl[blocks]), loop_parent=remap_loops(lp[loops]),
        loop_header=new_block[lh[loops]].astype(np.int32),
        call_site=ns.astype(np.int32), call_callee=nc.astype(np.int32),
    )
    return sub, dict(instr=instr, block=blocks, loop=loops, func=funcs)


def exchange_counts(partial, owners, arrays, rank: int, world: int, group=None):
    """The one exchange. partial: this rank's counters of the whole program (a 64-bit
    torch tensor of n_instr * 24, on any device); returns the sum over the ranks of
    the rows of the functions `rank` owns (in the order of select_functions), a
    tensor on partial's device. Each owner's rows are reduced to it (a reduce-scatter
    by owner; counts are added as 64-bit integers, which wrap like the counters)."""
    import torch
    rows = partial.view(-1, N_CNT)
    if rows.dtype == torch.uint64:
        rows = rows.view(torch.int64)
    mine = None
    for d in range(world):
        idx = torch.as_tensor(instr_rows(arrays, np.flatnonzero(np.asarray(owners) == d)), device=rows.device)
        buf = rows.index_select(0, idx).contiguous()
        if world > 1:
            import torch.distributed as dist
            dist.reduce(buf, dst=d, op=dist.ReduceOp.SUM, group=group)
        if d == rank:
            mine = buf
    return mine.view(-1)


class ShardedStep:
    """One rank of a sharded batch on its own GPU: the whole program for aggregating
    this rank's chunk of the samples, and the program of the functions this rank
    owns for blame and advice. step() runs reset, ingest, copy of the counters,
    the exchange, set, blame and advice (left on the device)."""

    def __init__(self, ctx, arrays, rank: int, world: int, group=None):
        import torch
        a = arrays.arrays if hasattr(arrays, "arrays") else arrays
        self.arrays, self.rank, self.world, self.group = a, rank, world, group
        self.owners = lpt_owners(function_costs(a), world)
        self.funcs = np.flatnonzero(self.owners == rank)
        self.full = ctx.load_program(a)
        self.sub_arrays, self.maps = select_functions(a, self.funcs)
        self.mine = ctx.load_program(self.sub_arrays) if self.funcs.size else None
        self.partial = torch.empty(int(a["n_instr"]) * N_CNT, dtype=torch.int64, device="cuda")

    def step(self, dev_chunk, stream=None):
        self.full.reset(stream)
        if dev_chunk.numel():
            self.full.ingest(dev_chunk, stream=stream)
        self.full.copy_counts(self.partial, stream)
        if stream is not None:
            stream.synchronize()
        owned = exchange_counts(self.partial, self.owners, self.arrays, self.rank, self.world, self.group)
        if self.mine is not None:
            self.mine.set_counts(owned, 0, stream)
            self.mine.blame(stream)
            self.mine.advise(fetch=False, stream=stream)
        return owned

    def close(self):
        if self.mine is not None:
            self.mine.unload()
        self.full.unload()

"""Hand-built tiny programs in the flat array format of the synthetic-input
module, for the paper's worked examples (Fig. 1, 3, 4) and edge cases."""
import numpy as np

import synth


def res(name: str) -> int:
    """'R5' -> 5, 'P3' -> 258, 'B2' -> 264."""
    k, v = name[0], int(name[1:])
    return {"R": synth.R_BASE, "P": synth.P_BASE, "B": synth.B_BASE}[k] + v


def guard_lit(g) -> int:
    if g is None:
        return 0
    if g.startswith("!"):
        return 8 + int(g[2:])
    return 1 + int(g[1:])


def I(op, defs=(), uses=(), guard=None, wb=None, rb=None, wait=(), line=0, flags=0):
    """One instruction: `defs`/`uses` register names, guard 'P0' or '!P0',
    wb/rb write/read barrier index set, wait = barrier indices waited on."""
    d = [res(x) for x in defs]
    if wb is not None:
        d.append((synth.B_BASE + wb) | (synth.KIND_WRITE << 12))
    if rb is not None:
        d.append((synth.B_BASE + rb) | (synth.KIND_READ << 12))
    u = [res(x) for x in uses]
    if guard is not None:
        u.append(res("P" + guard.lstrip("!")[1:]))
    u += [synth.B_BASE + k for k in wait]
    return dict(op=synth.OP[op], guard=guard_lit(guard), defs=d, uses=u, line=line, flags=flags)


def program(functions, calls=()):
    """functions: list of (blocks, succ, loops); blocks = list of instruction
    lists, succ = list of successor lists (local block ids), loops = list of
    (header, body_blocks, parent_loop_local_or_-1). calls: (global instruction
    index of a call site, called function) pairs."""
    a = {k: [] for k in ("block_instr_off", "succ_off", "succ", "opclass", "guard", "iflags", "line",
                         "def_off", "def_res", "use_off", "use_res", "block_loop", "loop_parent",
                         "loop_header", "func_instr_off", "func_block_off", "func_loop_off", "func_line_off")}
    ni = nb = nl = 0
    a["block_instr_off"].append(0); a["succ_off"].append(0); a["def_off"].append(0); a["use_off"].append(0)
    a["func_instr_off"].append(0); a["func_block_off"].append(0); a["func_loop_off"].append(0)
    a["func_line_off"].append(0)
    max_line = 0
    for blocks, succ, loops in functions:
        for b, ins in enumerate(blocks):
            for x in ins:
                a["opclass"].append(x["op"]); a["guard"].append(x["guard"]); a["iflags"].append(x["flags"])
                a["line"].append(x["line"]); max_line = max(max_line, x["line"])
                a["def_res"] += x["defs"]; a["use_res"] += x["uses"]
                a["def_off"].append(len(a["def_res"])); a["use_off"].append(len(a["use_res"]))
            ni += len(ins)
            a["block_instr_off"].append(ni)
            a["succ"] += [nb + s for s in succ[b]]
            a["succ_off"].append(len(a["succ"]))
        # innermost loop per block: the loop with the smallest body containing it
        for b in range(len(blocks)):
            best, size = -1, 10**9
            for l, (h, body, par) in enumerate(loops):
                if b in body and len(body) < size:
                    best, size = l, len(body)
            a["block_loop"].append(-1 if best < 0 else nl + best)
        for (h, body, par) in loops:
            a["loop_header"].append(nb + h)
            a["loop_parent"].append(-1 if par < 0 else nl + par)
        nb += len(blocks); nl += len(loops)
        a["func_instr_off"].append(ni); a["func_block_off"].append(nb); a["func_loop_off"].append(nl)
        a["func_line_off"].append(max_line + 1)
    dt = dict(opclass=np.uint8, guard=np.uint8, iflags=np.uint8, def_res=np.uint16, use_res=np.uint16)
    out = {k: np.array(v, dtype=dt.get(k, np.int32)) for k, v in a.items()}
    out.update(n_functions=len(functions), n_instr=ni, n_blocks=nb, n_loops=nl, n_lines=max_line + 1)
    calls = sorted(calls)
    out.update(call_site=np.array([c[0] for c in calls], dtype=np.int32),
               call_callee=np.array([c[1] for c in calls], dtype=np.int32))
    return out


def sample(kernel, pc, cls, lat, sm=0):
    return np.uint64((kernel << 48) | (pc << 24) | (cls << 20) | (lat << 19) | (sm << 11))


def counts(n_instr, entries):
    """Dense count array [n_instr, 12, 2] from {(pc, class, lat): n}."""
    c = np.zeros((n_instr, 12, 2), dtype=np.uint64)
    for (pc, cls, lat), v in entries.items():
        c[pc, cls, lat] = v
    return c

"""Brute-force path enumeration on tiny CFGs: an independent restatement of
the source-path semantics, used to pin the oracle.

It shares nothing with the oracle's state-graph search: it enumerates every
simple instruction-level path that ends at the use, applies the paper's
predicate-coverage condition to each path as a whole (Sec. 4: a def i is an
immediate source of use j through resource r if the union of the guard
predicates of the defs of r strictly between i and j does not contain j's
guard, where Pi and !Pi together make "_"), and takes back edges from the loop
nest input rather than from dominators.

Why simple paths suffice: removing a cycle from a walk only drops defs from
the union, and every cycle of a reducible CFG holds a back edge, so the
shortest path, the fewest back edges K, the longest path with exactly K back
edges and "k lies on every path" are all decided by simple paths.
"""
import numpy as np

import synth

ALL = "_"


def lits_add(S, g):
    if g == 0:
        return S | {ALL}
    name = f"P{g - 1}" if g <= 7 else f"!P{g - 8}"
    S = S | {name}
    for i in range(7):
        if f"P{i}" in S and f"!P{i}" in S:
            S = S | {ALL}
    return S


def lits_contains(S, g):
    if ALL in S:
        return True
    if g == 0:
        return False
    name = f"P{g - 1}" if g <= 7 else f"!P{g - 8}"
    return name in S


class Fn:
    def __init__(self, prog, f):
        a = prog.arrays if hasattr(prog, "arrays") else prog
        self.a = a
        self.i0, self.i1 = int(a["func_instr_off"][f]), int(a["func_instr_off"][f + 1])
        self.b0, self.b1 = int(a["func_block_off"][f]), int(a["func_block_off"][f + 1])
        bio = a["block_instr_off"]
        self.block_of = {}
        for b in range(self.b0, self.b1):
            for x in range(int(bio[b]), int(bio[b + 1])):
                self.block_of[x] = b

        def loops_of(b):
            out, q = [], int(a["block_loop"][b])
            while q >= 0:
                out.append(q)
                q = int(a["loop_parent"][q])
            return out

        # edge u -> v is a back edge iff v heads a loop that contains u
        self.preds = {x: [] for x in range(self.i0, self.i1)}
        self.succs = {x: [] for x in range(self.i0, self.i1)}
        for b in range(self.b0, self.b1):
            first, last = int(bio[b]), int(bio[b + 1]) - 1
            for x in range(first, last):
                self.preds[x + 1].append((x, 0))
                self.succs[x].append(x + 1)
            for e in range(int(a["succ_off"][b]), int(a["succ_off"][b + 1])):
                v = int(a["succ"][e])
                bk = int(any(int(a["loop_header"][q]) == v for q in loops_of(b)))
                self.preds[int(bio[v])].append((last, bk))
                self.succs[last].append(int(bio[v]))

    def defs(self, x):
        a = self.a
        return [int(a["def_res"][e]) & 0x1FF for e in range(int(a["def_off"][x]), int(a["def_off"][x + 1]))]

    def uses(self, x):
        a = self.a
        return [int(a["use_res"][e]) & 0x1FF for e in range(int(a["use_off"][x]), int(a["use_off"][x + 1]))]

    def guard(self, x):
        return int(self.a["guard"][x])


def sources(F: Fn, j: int, r: int, limit: int = 2_000_000):
    """{i: dict(dmin, K, dlong, dom)} for global use j and resource r."""
    gj = F.guard(j)
    found = {}  # i -> list of (length, backs, frozenset(internal nodes))
    steps = [0]

    def dfs(x, visited, length, backs, S):
        steps[0] += 1
        if steps[0] > limit:
            raise RuntimeError("path enumeration limit")
        for y, bk in F.preds[x]:
            L, B = length + 1, backs + bk
            S2 = S
            if r in F.defs(y):
                if y == j or y not in visited:
                    if not lits_contains(S, gj):
                        found.setdefault(y, []).append((L, B, frozenset(visited - {j})))
                S2 = lits_add(S, F.guard(y))
            if lits_contains(S2, gj) or y == j or y in visited:
                continue
            dfs(y, visited | {y}, L, B, S2)

    dfs(j, {j}, 0, 0, frozenset())
    out = {}
    for i, paths in found.items():
        K = min(p[1] for p in paths)
        cand = [k for k in range(F.i0, F.i1) if k not in (i, j) and F.guard(k) == 0 and r in F.uses(k)]
        dom = any(all(k in p[2] for p in paths) for k in cand)
        out[i] = dict(dmin=min(p[0] for p in paths), K=K, dlong=max(p[0] for p in paths if p[1] == K), dom=dom)
    return out


def reaching(F: Fn):
    """Brute-force RIN/ROUT projections: for each def site, walk forward at
    instruction level until an unguarded def of the same resource."""
    a = F.a
    bio = a["block_instr_off"]
    nb = F.b1 - F.b0
    rin = np.zeros((nb, 9), np.uint32)
    rout = np.zeros((nb, 9), np.uint32)
    for x in range(F.i0, F.i1):
        for r in F.defs(x):
            before = set()
            st = list(F.succs[x])
            while st:
                y = st.pop()
                if y in before:
                    continue
                before.add(y)
                killed = (y != x) and (r in F.defs(y)) and F.guard(y) == 0
                if not killed:
                    st.extend(F.succs[y])

            def after(y):
                return y == x or (y in before and not ((r in F.defs(y)) and F.guard(y) == 0))

            for b in range(F.b0, F.b1):
                first, last = int(bio[b]), int(bio[b + 1]) - 1
                if first in before:
                    rin[b - F.b0, r >> 5] |= np.uint32(1 << (r & 31))
                if after(last):
                    rout[b - F.b0, r >> 5] |= np.uint32(1 << (r & 31))
    return rin, rout


def tiny_program(seed: int, n_instr: int = 30, n_loops: int = 2, guard_pct: int = 35, n_regs: int = 8):
    return synth.make_program([dict(n_instr=n_instr, n_loops=n_loops, max_depth=2, n_regs=n_regs,
                                    guard_pct=guard_pct, seed=seed)])

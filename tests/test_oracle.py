"""Pins of the CPU oracle against things other than itself: the paper's worked
examples (tests/golden), brute-force path enumeration on tiny CFGs, closed
forms of Eq. 1/2/4/5, Theorem 1, and invariants. No GPU."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from bruteforce import Fn, reaching as bf_reaching, sources as bf_sources, tiny_program
from progbuild import I, counts, program, res, sample

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ARCH = synth.default_arch()
LAT = dict(zip(synth.OPS, ARCH[0]))
C_EXEC, C_MEM, C_SYNC, C_CONST = 2, 3, 5, 6


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def one_block(ins):
    return program([([ins], [[]], [])])


# ---------------------------------------------------------------- Sec. 2.1, Fig. 1
def test_fig1_sampling_ratios():
    g = gold("fig1_sampling.json")
    prog = one_block([I("IADD", ["R1"], ["R2", "R3"]), I("EXIT")])
    ss = []
    for s in g["samples"]:
        # stall samples carry a stall reason; the one sample without one is SELECTED
        cls = (C_MEM if s["latency"] else 9) if s["stall"] else 0
        ss.append(sample(0, 0, cls, s["latency"]))
    cnt, bad = oracle.histogram(prog, np.array(ss, dtype=np.uint64))
    assert bad == 0
    R = oracle.analyze(prog, ARCH, cnt)
    T, A, L, issued = (int(x) for x in R["totals"][0])
    e = g["expect"]
    assert (T, A, L) == (e["total"], e["active"], e["latency"])
    assert T - issued == e["stall_samples"]
    assert L / T == e["stall_ratio"] and A / T == e["active_ratio"]


def test_histogram_exact_and_invalid():
    prog = program([([[I("IADD", ["R1"], ["R2"]), I("IADD", ["R3"], ["R1"])]], [[]], []),
                    ([[I("MOV", ["R1"], ["R2"])]], [[]], [])])
    ss = [sample(0, 0, 0, 0)] * 3 + [sample(0, 1, 2, 1)] * 2 + [sample(1, 0, 11, 0)]
    bad = [sample(2, 0, 0, 0),            # unknown kernel
           sample(1, 1, 0, 0),            # pc past the function
           sample(0, 0, 12, 0),           # class out of range
           sample(0, 0, 0, 1),            # SELECTED with the latency flag
           sample(0, 0, 3, 0) | np.uint64(5)]  # reserved bits set
    cnt, nbad = oracle.histogram(prog, np.array(ss + bad, dtype=np.uint64))
    assert nbad == len(bad)
    assert cnt[0, 0, 0] == 3 and cnt[1, 2, 1] == 2 and cnt[2, 11, 0] == 1
    assert int(cnt.sum()) == len(ss)


def test_histogram_generated_conserves():
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps, kz)
    s = P.samples(200_000, invalid_ppm=20_000)
    cnt, bad = oracle.histogram(P, s)
    assert int(cnt.sum()) + bad == s.size
    assert 0 < bad < s.size // 10
    k = (s >> np.uint64(48)).astype(np.int64)
    ok = k < P.n_functions
    # per-kernel totals equal the number of valid samples of that kernel
    tot = np.add.reduceat(cnt.reshape(P.n_instr, -1).sum(1), P.func_instr_off[:-1])
    assert int(tot.sum()) <= int(ok.sum())


# ---------------------------------------------------------------- Sec. 4, Fig. 3
def test_fig3_barrier_dependency():
    gold("fig3_barrier.json")
    prog = one_block([I("LDG", ["R0"], ["R2", "R3"], wb=0), I("IADD", ["R5"], ["R6", "R7"]),
                      I("BRA", [], [], wait=[0])])
    cnt = counts(3, {(0, 0, 0): 5, (2, C_MEM, 0): 40, (2, C_MEM, 1): 60})
    R = oracle.analyze(prog, ARCH, cnt)
    b = R["blame"]
    assert b[0, C_MEM, 0] == 40 and b[0, C_MEM, 1] == 60
    assert b[2, C_MEM].sum() == 0
    e = R["edges"]
    assert list(e["i"]) == [0] and list(e["j"]) == [2]
    assert e["flags"][0] & 2 and not e["flags"][0] & 4      # through a barrier, not a register


# ---------------------------------------------------------------- Sec. 4, Fig. 4
def fig4(use_guard=None, mov_between=False):
    ins = [I("ISETP", ["P0"], ["R10", "R11"]), I("ISETP", ["P1"], ["R10", "R12"]),
           I("MOV", ["R20"], ["R21"]), I("MOV", ["R22"], ["R21"]),
           I("LDC", ["R0"], [], guard="!P0"),
           I("IMAD", ["R0"], ["R4", "R5", "R6"], guard="P1"),
           I("MOV", ["R0"] if mov_between else ["R23"], ["R21"]),
           I("LDG", ["R0"], ["R2", "R3"], guard="P0"),
           I("MOV", ["R24"], ["R21"]), I("MOV", ["R25"], ["R21"]),
           I("IADD", ["R1"], ["R0", "R7"], guard=use_guard)]
    return one_block(ins)


def test_fig4a_predicate_coverage():
    g = gold("fig4_blamer.json")
    src = {s["i"]: s for s in oracle.search(fig4(), 10, res("R0"))}
    assert sorted(src) == [4, 5, 7]                           # LDC, IMAD, LDG
    assert {4: "LDC", 7: "LDG"}.keys() <= src.keys()
    assert set(g["expect"]["sources_unpredicated_use"]) == {"LDG", "LDC"}
    assert [src[i]["dmin"] for i in (7, 5, 4)] == [3, 5, 6]
    # an unguarded def between them ends the search there
    src = {s["i"] for s in oracle.search(fig4(mov_between=True), 10, res("R0"))}
    assert src == {6, 7}
    # a use guarded by P0 is covered by the @P0 def alone
    src = {s["i"] for s in oracle.search(fig4(use_guard="P0"), 10, res("R0"))}
    assert src == {7}


def test_fig4cd_opcode_pruning_and_equal_shares():
    prog = fig4()
    cnt = counts(11, {(7, 0, 0): 10, (4, 0, 0): 20, (5, 0, 0): 7, (10, C_MEM, 0): 100, (10, C_EXEC, 1): 9})
    R = oracle.analyze(prog, ARCH, cnt)
    b = R["blame"]
    # memory stalls: IMAD pruned by opcode; LDC (2x issue, 2x path) and LDG get equal shares
    assert b[5, C_MEM].sum() == 0
    assert b[7, C_MEM, 0] == 50 and b[4, C_MEM, 0] == 50
    assert gold("fig4_blamer.json")["expect"]["ldc_over_ldg_share"] == b[4, C_MEM, 0] / b[7, C_MEM, 0]
    # execution stalls: no opcode rule, all three sources share them
    assert int(b[[4, 5, 7], C_EXEC, 1].sum()) == 9 and b[5, C_EXEC, 1] > 0


# ---------------------------------------------------------------- pruning rules
def test_dominator_pruning_straight_line():
    prog = one_block([I("LDG", ["R0"], ["R2", "R3"], wb=0), I("IADD", ["R1"], ["R0", "R5"], wait=[0]),
                      I("FFMA", ["R3"], ["R0", "R6", "R7"])])
    s = oracle.search(prog, 2, res("R0"))
    assert len(s) == 1 and s[0]["i"] == 0 and s[0]["dom"]       # IADD reads R0 on the only path
    cnt = counts(3, {(2, C_MEM, 0): 30, (1, C_MEM, 1): 12, (0, 0, 0): 1})
    R = oracle.analyze(prog, ARCH, cnt)
    assert R["blame"][2, C_MEM, 0] == 30                         # no surviving source: stays
    assert R["blame"][0, C_MEM, 1] == 12                         # IADD's stalls go to the LDG


def diamond(extra_use_in_entry):
    b0 = [I("LDG", ["R0"], ["R2", "R3"])]
    if extra_use_in_entry:
        b0.append(I("IADD", ["R9"], ["R0", "R5"]))
    b0 += [I("ISETP", ["P0"], ["R5", "R6"]), I("BRA", [], [], guard="P0")]
    b1 = [I("IADD", ["R1"], ["R0", "R5"])]
    b2 = [I("FFMA", ["R3"], ["R0", "R6", "R7"]), I("EXIT")]
    return program([([b0, b1, b2], [[1, 2], [2], []], [])])


def test_dominator_pruning_needs_every_path():
    p = diamond(False)
    j = int(p["block_instr_off"][2])
    s = oracle.search(p, j, res("R0"))
    assert [(x["i"], x["dom"]) for x in s] == [(0, False)]      # the B0->B2 path avoids the IADD
    assert s[0]["dmin"] == 3 and s[0]["dlong"] == 4
    p = diamond(True)
    j = int(p["block_instr_off"][2])
    s = oracle.search(p, j, res("R0"))
    assert [(x["i"], x["dom"]) for x in s] == [(0, True)]       # now an unguarded reader is on both


@pytest.mark.parametrize("pad,blamed", [(3, True), (4, True), (5, False)])
def test_latency_pruning(pad, blamed):
    ins = [I("IMAD", ["R0"], ["R1", "R2", "R3"])] + [I("MOV", ["R9"], ["R8"])] * pad + \
          [I("IADD", ["R4"], ["R0", "R5"])]
    prog = one_block(ins)
    j = len(ins) - 1
    cnt = counts(len(ins), {(j, C_EXEC, 0): 10, (0, 0, 0): 3})
    R = oracle.analyze(prog, ARCH, cnt)
    assert pad + 1 <= LAT["IMAD"] or not blamed
    assert (R["blame"][0, C_EXEC, 0] == 10) == blamed
    assert (R["blame"][j, C_EXEC, 0] == 10) == (not blamed)


def test_loop_carried_longest_path():
    # B0 entry; B1 loop (body: use of R0, then later def of R0); B2 exit.
    b0 = [I("MOV", ["R0"], ["R1"])]
    b1 = [I("IADD", ["R2"], ["R0", "R3"]), I("MOV", ["R7"], ["R8"]), I("MOV", ["R0"], ["R2"]),
          I("ISETP", ["P0"], ["R2", "R3"]), I("BRA", [], [], guard="P0")]
    b2 = [I("EXIT")]
    p = program([([b0, b1, b2], [[1], [2, 1], []], [(1, [1], -1)])])
    s = {x["i"]: x for x in oracle.search(p, 1, res("R0"))}
    assert sorted(s) == [0, 3]
    assert (s[0]["dmin"], s[0]["K"], s[0]["dlong"]) == (1, 0, 1)
    assert (s[3]["dmin"], s[3]["K"], s[3]["dlong"]) == (3, 1, 3)   # def -> ISETP -> BRA -> back edge -> use


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(40))
def test_sources_match_bruteforce(seed):
    P = tiny_program(seed, n_instr=22 + seed % 15, n_loops=seed % 3, guard_pct=20 + 5 * (seed % 6))
    assert oracle.check_loops(P, 0) == 0
    F = Fn(P, 0)
    n = 0
    for j in range(P.n_instr):
        for r in sorted(set(F.uses(j))):
            want = bf_sources(F, j, r)
            got = {s["i"]: dict(dmin=s["dmin"], K=s["K"], dlong=s["dlong"], dom=s["dom"])
                   for s in oracle.search(P, j, r)}
            assert got == want, (seed, j, r)
            n += len(want)
    assert n > 0


@pytest.mark.parametrize("seed", range(12))
def test_reaching_match_bruteforce(seed):
    P = tiny_program(100 + seed, n_instr=40, n_loops=1 + seed % 2, guard_pct=30)
    rin, rout = oracle.reaching(P)
    bin_, bout = bf_reaching(Fn(P, 0))
    assert (rin == bin_).all() and (rout == bout).all()


def test_generated_loops_are_natural_loops():
    for name in ("plain", "rodinia"):
        ps, _, kz = synth.workload(name)
        P = synth.make_program(ps, kz)
        assert all(oracle.check_loops(P, f) == 0 for f in range(P.n_functions))
    ps = synth.batched_params(40, np.random.default_rng(1), 1)
    P = synth.make_program(ps)
    assert all(oracle.check_loops(P, f) == 0 for f in range(P.n_functions))


# ---------------------------------------------------------------- Eq. 1
def _apportion_prog(dists, issues, S):
    """One use with len(dists) unguarded-reader-free sources at the given distances."""
    n = max(dists) + 1
    ins = [I("MOV", ["R30"], ["R31"]) for _ in range(n)]
    srcs = []
    for t, d in enumerate(dists):
        ins[n - 1 - d] = I("LDG", [f"R{t}"], ["R20", "R21"])
        srcs.append(n - 1 - d)
    ins[n - 1] = I("FFMA", ["R29"], [f"R{t}" for t in range(len(dists))])
    ent = {(x, 0, 0): v for x, v in zip(srcs, issues) if v}
    ent[(n - 1, C_MEM, 0)] = S
    return one_block(ins), counts(n, ent), srcs


def test_eq1_largest_remainder_rule():
    # equal weights: floor(7/3) = 2 each, the leftover unit goes to the lowest def index
    prog, cnt, srcs = _apportion_prog([1, 2, 3], [4, 8, 12], 7)   # issue/dist = 4 for all three
    R = oracle.analyze(prog, ARCH, cnt)
    sh = {x: int(R["blame"][x, C_MEM, 0]) for x in srcs}
    assert sorted(sh.values()) == [2, 2, 3] and sh[min(srcs)] == 3
    # proportional case: weights 10/2 : 60/4 = 1:3 split 100 as 25:75
    prog, cnt, srcs = _apportion_prog([2, 4], [10, 60], 100)
    R = oracle.analyze(prog, ARCH, cnt)
    assert [int(R["blame"][x, C_MEM, 0]) for x in srcs] == [25, 75]
    # no issued samples anywhere: weight by 1 / longest path (2:1)
    prog, cnt, srcs = _apportion_prog([1, 2], [0, 0], 30)
    R = oracle.analyze(prog, ARCH, cnt)
    assert [int(R["blame"][x, C_MEM, 0]) for x in srcs] == [20, 10]


# ---------------------------------------------------------------- Sec. 5
def test_eq2_eq4_closed_forms():
    ins = [I("LDG", ["R0"], ["R2", "R3"]), I("MOV", ["R9"], ["R8"]), I("FFMA", ["R1"], ["R0", "R5", "R6"])]
    prog = one_block(ins)
    cnt = counts(3, {(0, 0, 0): 20, (1, 1, 0): 15, (1, 1, 1): 10, (2, C_MEM, 1): 40, (2, 9, 0): 15})
    R = oracle.analyze(prog, ARCH, cnt)
    T, A, L, _ = (int(x) for x in R["totals"][0])
    assert (T, A, L) == (100, 50, 50)
    sp = R["speedup"][0]
    assert sp[2] == 100 / (100 - 25)                         # Function Split, Eq. 2: INST_FETCH
    assert sp[7] == 100 / (100 - min(50, 40))                # Code Reordering, Eq. 4
    assert R["M"][0][7] == 40
    assert list(R["rank"][0][:2]) == [7, 2]
    hot = R["hot"][0][7][0]
    assert list(hot[[0, 1, 4, 5]]) == [0, 2, 2, 40]          # def pc, use pc, distance, samples


def test_theorem1_latency_hiding_bound():
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps[:8], kz)
    for seed in range(3):
        cnt, _ = oracle.histogram(P, P.samples(300_000, seed=seed))
        R = oracle.analyze(P, ARCH, cnt)
        assert (R["speedup"][:, 6] <= 2.0).all() and (R["speedup"][:, 7] <= 2.0).all()
        assert (R["loop_S"] <= 2.0).all()
        T = R["totals"][:, 0].astype(float)
        A = R["totals"][:, 1].astype(float)
        M = R["M"][:, 7].astype(float)
        ok = T > 0
        assert np.array_equal(R["speedup"][ok, 7], T[ok] / (T[ok] - np.minimum(A[ok], M[ok])))


def test_eq5_scope_nesting():
    # loop scopes: A of an outer loop includes the inner loop's active samples
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps[:6], kz)
    cnt, _ = oracle.histogram(P, P.samples(300_000, seed=4))
    R = oracle.analyze(P, ARCH, cnt)
    par = P.loop_parent
    for l in range(P.n_loops):
        if par[l] >= 0:
            assert R["loop_A"][par[l]] >= R["loop_A"][l]
            assert R["loop_ML"][par[l]] >= R["loop_ML"][l]


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("name,nfun,ns", [("plain", 1, 100_000), ("rodinia", 20, 400_000)])
def test_blame_invariants(name, nfun, ns):
    ps, _, kz = synth.workload(name)
    P = synth.make_program(ps[:nfun], kz)
    cnt, _ = oracle.histogram(P, P.samples(ns))
    R = oracle.analyze(P, ARCH, cnt)
    # conservation per (class, latency flag)
    assert np.array_equal(R["blame"].sum(0), cnt.sum(0))
    e = R["edges"]
    assert len(e["j"]) > 0
    for t in range(len(e["j"])):
        i, j = int(e["i"][t]), int(e["j"][t])
        di = {int(x) & 0x1FF for x in P.def_res[P.def_off[i]:P.def_off[i + 1]]}
        uj = {int(x) & 0x1FF for x in P.use_res[P.use_off[j]:P.use_off[j + 1]]}
        assert di & uj                                        # the blamed def writes what j reads
        assert e["dmin"][t] <= ARCH[0][P.opclass[i]]          # latency rule holds on survivors
        assert 1 <= e["dmin"][t] <= e["dlong"][t]
    # edge shares add up to the blame moved off each use
    sh = e["share"].sum(0)
    assert int(sh.sum()) <= int(cnt[:, [2, 3, 5, 6], :].sum())
    # sorted by (use, def)
    key = e["j"].astype(np.int64) * (1 << 32) + e["i"]
    assert (np.diff(key) > 0).all()


# ---------------------------------------------------------------- Sec. 6, single dependency coverage
def _keeps(flags, cls, op):
    if cls in (3, 6):
        return bool(flags[op] & 1)      # memory dependencies: memory instructions only
    if cls == 5:
        return bool(flags[op] & 2)      # synchronization: barriers only
    return True


def _bf_coverage(P, arch, cnt):
    """Coverage from the brute-force sources: nodes are the stalled uses; a node is
    single if every resource it reads has at most one source (before pruning) or at most
    one source that survives rules 2, 3 and 1 for one of its stalled classes (after)."""
    lat, flags = arch
    F = Fn(P, 0)
    c3 = np.asarray(cnt).reshape(-1, 12, 2)
    nodes = before = after = 0
    for j in range(P.n_instr):
        stalled = [c for c in (2, 3, 5, 6) if c3[j, c].sum() > 0]
        if not stalled:
            continue
        nodes += 1
        most_all = most_kept = 0
        for r in sorted(set(F.uses(j))):
            src = bf_sources(F, j, r)
            kept = sum(1 for i, d in src.items()
                       if not d["dom"] and d["dmin"] <= lat[F.a["opclass"][i]]
                       and any(_keeps(flags, c, F.a["opclass"][i]) for c in stalled))
            most_all, most_kept = max(most_all, len(src)), max(most_kept, kept)
        before += most_all <= 1
        after += most_kept <= 1
    return nodes, before, after


@pytest.mark.parametrize("seed", range(12))
def test_coverage_matches_bruteforce(seed):
    P = tiny_program(300 + seed, n_instr=24 + seed % 12, n_loops=seed % 3, guard_pct=25 + 5 * (seed % 5))
    arch = synth.default_arch()
    cnt, _ = oracle.histogram(P, P.samples(30_000, seed=seed))
    got = oracle.coverage(P, arch, cnt)
    assert got == _bf_coverage(P, arch, cnt)
    assert got[0] > 0 and got[1] <= got[2] <= got[0]


def test_coverage_diamond_opcode_rule():
    """Two defs of R1 reach the use: not single before pruning. With memory stalls only,
    the IMAD cannot cause them (rule 1) and the node becomes single; with execution
    stalls as well, both stay."""
    b0 = [I("ISETP", ["P0"], ["R5", "R6"]), I("BRA", [], [], guard="P0")]
    b1 = [I("LDG", ["R1"], ["R2", "R3"])]
    b2 = [I("IMAD", ["R1"], ["R5", "R6", "R7"])]
    b3 = [I("IADD", ["R4"], ["R1", "R5"]), I("EXIT")]
    p = program([([b0, b1, b2, b3], [[1, 2], [3], [3], []], [])])
    j = int(p["block_instr_off"][3])
    arch = synth.default_arch()
    mem = counts(len(p["opclass"]), {(j, 3, 0): 50})
    assert oracle.coverage(p, arch, mem) == (1, 0, 1)
    both = counts(len(p["opclass"]), {(j, 3, 0): 50, (j, 2, 1): 7})
    assert oracle.coverage(p, arch, both) == (1, 0, 0)


# ---------------------------------------------------------------- parallel optimizers (Table 2, Eqs. 6-10)
GB_SM = dict(n_sms=152, schedulers_per_sm=4, max_warps_per_sm=64, max_blocks_per_sm=32, regs_per_sm=65536,
             reg_alloc_unit=256, smem_per_sm=233472, smem_alloc_unit=128, smem_reserved_per_block=1024)
SMALL_SM = dict(GB_SM, n_sms=4)


def _par(sm, blocks, threads, regs, smem, T, issued):
    st = dict(blocks=[blocks], threads_per_block=[threads], regs_per_thread=[regs], smem_per_block=[smem])
    tot = np.array([[T, 0, 0, issued]], dtype=np.uint64)
    return oracle.parallel(st, sm, tot)


def test_occupancy_worked_cases():
    """Blocks per SM by hand: 256 threads, 64 registers, 48 KB -> registers allow
    4 x floor(16384 / 2048) = 32 warps = 4 blocks, shared memory floor(233472 /
    50176) = 4 blocks (the tie reports registers); 32 threads with 96 registers ->
    4 x floor(16384 / 3072) = 20 warps (20 blocks); 32 threads, 32 registers, no
    shared memory -> the 32-block cap binds; 1,024 threads -> 2 blocks by warp slots."""
    from oracle.parallel import occupancy
    o = occupancy(256, 64, 48 * 1024, GB_SM)
    assert (o["blocks_per_sm"], o["limit"], o["limits"][2]) == (4, 1, 4)
    o = occupancy(32, 96, 0, GB_SM)
    assert (o["blocks_per_sm"], o["limit"], o["warps_by_regs"]) == (20, 1, 20)
    o = occupancy(32, 32, 0, GB_SM)
    assert (o["blocks_per_sm"], o["limit"]) == (32, 3)
    o = occupancy(1024, 0, 0, GB_SM)
    assert (o["blocks_per_sm"], o["limit"]) == (2, 0)
    o = occupancy(64, 32, 200 * 1024, GB_SM)   # one 201 KB block fits
    assert (o["blocks_per_sm"], o["limit"]) == (1, 2)


def test_block_increase_closed_form():
    """2 blocks of 8 warps on 4 SMs: W = 8 / 4 = 2 warps per scheduler, W_new = 2 * 2 / 4 = 1;
    Eq. 10 gives (W / W_new) * (1 - (1-R)) / (1 - (1-R)^2) = 2 / (2 - R)."""
    for R, T in [(0.5, 1000), (0.25, 4000), (0.1, 10)]:
        r = _par(SMALL_SM, 2, 256, 32, 0, T, int(R * T))
        assert r["par_match"][0].tolist() == [1, 0]
        assert math.isclose(r["par_speedup"][0, 0], 2 / (2 - R), rel_tol=1e-14)
        assert r["par_warps"][0, 0].tolist() == [2.0, 1.0]


def test_thread_increase_closed_form():
    """1-warp blocks capped at 32 per SM (W = 8), the grid large enough: merging them
    lets all 64 warp slots fill (W_new = 16) and C_W = 1, so S = (1 - (1-R)^16) /
    (1 - (1-R)^8) = 1 + (1-R)^8."""
    for R in (0.5, 0.2, 0.05):
        r = _par(SMALL_SM, 4 * 32 * 2, 32, 32, 0, 10 ** 6, int(R * 10 ** 6))
        assert r["par_match"][0].tolist() == [0, 1] and r["par_limit"][0] == 3
        assert r["par_warps"][0, 1].tolist() == [8.0, 16.0]
        assert math.isclose(r["par_speedup"][0, 1], 1 + (1 - R) ** 8, rel_tol=1e-14)
    # the grid caps W_new: 4 SMs x 40 one-warp blocks give 40 warps per SM (W_new = 10)
    r = _par(SMALL_SM, 4 * 40, 32, 32, 0, 1000, 500)
    assert r["par_warps"][0, 1].tolist() == [8.0, 10.0]
    assert math.isclose(r["par_speedup"][0, 1], (1 - 0.5 ** 10) / (1 - 0.5 ** 8), rel_tol=1e-14)


def test_parallel_unmatched_and_degenerate():
    """Grid of exactly one block per SM, or a limit other than the block cap: no match,
    speedup 1.0. No issued samples: matched, speedup 1.0. No statistics: limit -1."""
    r = _par(SMALL_SM, 4, 256, 32, 0, 1000, 100)
    assert r["par_match"][0].tolist() == [0, 0] and r["par_speedup"][0].tolist() == [1.0, 1.0]
    r = _par(SMALL_SM, 4 * 32 * 2, 64, 32, 0, 1000, 100)   # 32 blocks x 2 warps = 64: tie, warp slots reported
    assert r["par_limit"][0] == 0 and r["par_match"][0].tolist() == [0, 0]
    r = _par(SMALL_SM, 3 * 32, 32, 32, 0, 1000, 100)       # grid gives an SM 24 blocks, below the cap
    assert r["par_limit"][0] == 3 and r["par_match"][0].tolist() == [0, 0]
    r = _par(SMALL_SM, 2, 256, 32, 0, 1000, 0)
    assert r["par_match"][0].tolist() == [1, 0] and r["par_speedup"][0].tolist() == [1.0, 1.0]
    none = oracle.parallel(None, SMALL_SM, np.zeros((3, 4), np.uint64))
    assert none["par_limit"].tolist() == [-1, -1, -1] and np.all(none["par_speedup"] == 1.0)


# ---------------------------------------------------------------- Sec. 2.3, the two motivating examples
def _loop_program(body):
    """entry block, one single-block loop `body` (header and latch), exit block."""
    entry = [I("MOV", ["R10"], ["R11"])]
    return program([([entry, body, [I("EXIT")]], [[1], [1, 2], []], [(1, [1], -1)])])


def test_motivating_conversion_chain_strength_reduction():
    """Sec. 2.3, first example: execution-dependency stalls on an FMA that consumes a
    type conversion inside a hot loop are blamed on the conversion, so Strength
    Reduction (conversions are flagged long-latency arithmetic) matches them, ranks
    first, and points at the conversion -> FMA pair."""
    body = [I("LDS", ["R2"], ["R10"]), I("F2F", ["R4"], ["R2"]), I("FFMA", ["R5"], ["R4", "R6", "R7"]),
            I("STS", [], ["R10", "R5"]), I("IADD", ["R10"], ["R10", "R12"]), I("ISETP", ["P0"], ["R10", "R13"]),
            I("BRA", [], [], guard="P0")]
    prog = _loop_program(body)
    ffma, f2f = 3, 2                                  # global instruction indices (entry block has one)
    cnt = counts(9, {(ffma, C_EXEC, 1): 60, (ffma, C_EXEC, 0): 20, (f2f, 0, 0): 10, (1, 0, 0): 10,
                     (4, 0, 0): 10, (6, 9, 0): 5})
    R = oracle.analyze(prog, ARCH, cnt)
    T, A, L, _ = (int(x) for x in R["totals"][0])
    assert (T, L) == (115, 60)
    assert R["blame"][f2f, C_EXEC].tolist() == [20, 60] and R["blame"][ffma, C_EXEC].sum() == 0
    assert R["M"][0][1] == 80 and R["speedup"][0][1] == 115 / (115 - 80)    # Eq. 2
    assert R["rank"][0][0] == 1                                             # Strength Reduction first
    assert list(R["hot"][0][1][0][[0, 1, 4, 5]]) == [f2f, ffma, 1, 80]      # def, use, distance, samples


def test_motivating_short_load_use_in_synchronized_loop():
    """Sec. 2.3, second example: a global load whose value is consumed by the next
    instruction in a loop that also synchronizes. The use's memory-dependency latency
    samples are blamed on the load at distance 1: Code Reordering and Loop Unrolling
    (def and use share the loop) match them (Eq. 4), and the barrier's sync stalls
    match Warp Balance (Eq. 2)."""
    body = [I("LDG", ["R0"], ["R2", "R3"]), I("ISETP", ["P0"], ["R0", "R4"]), I("BAR"),
            I("IADD", ["R10"], ["R10", "R12"]), I("ISETP", ["P1"], ["R10", "R13"]), I("BRA", [], [], guard="P1")]
    prog = _loop_program(body)
    ldg, use, bar = 1, 2, 3
    cnt = counts(8, {(use, C_MEM, 1): 50, (use, C_MEM, 0): 10, (bar, C_SYNC, 1): 20, (bar, C_SYNC, 0): 10,
                     (ldg, 0, 0): 15, (4, 0, 0): 15})
    R = oracle.analyze(prog, ARCH, cnt)
    T, A, L, _ = (int(x) for x in R["totals"][0])
    assert (T, A, L) == (120, 50, 70)
    assert R["blame"][ldg, C_MEM].tolist() == [10, 50]
    M, sp = R["M"][0], R["speedup"][0]
    assert M[6] == M[7] == 50 and M[4] == 30
    assert sp[6] == sp[7] == 120 / (120 - min(50, 50)) and sp[4] == 120 / (120 - 30)
    assert list(R["rank"][0][:3]) == [6, 7, 4]        # equal speedups: the lower id first
    assert list(R["hot"][0][7][0][[0, 1, 4, 5]]) == [ldg, use, 1, 50]


def test_counts_independent_of_order_and_chunking():
    """Sec. 2.1: the counters are a multiset statistic of the samples. A permuted
    stream gives the same counts, and chunks counted apart add up to the whole
    stream's counts (invalid samples included); the analysis follows the counts."""
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps[:6], kz)
    s = P.samples(200_000, invalid_ppm=5000, seed=8)
    cnt, bad = oracle.histogram(P, s)
    perm = np.random.default_rng(8).permutation(s.size)
    cnt_p, bad_p = oracle.histogram(P, s[perm])
    assert np.array_equal(cnt, cnt_p) and bad == bad_p
    parts = [oracle.histogram(P, c) for c in np.array_split(s[perm], [1, 70_001, 150_000])]
    assert np.array_equal(sum(p[0] for p in parts), cnt) and sum(p[1] for p in parts) == bad
    R, Rp = oracle.analyze(P, ARCH, cnt), oracle.analyze(P, ARCH, cnt_p)
    assert np.array_equal(R["blame"], Rp["blame"]) and np.array_equal(R["rank"], Rp["rank"])


# ---------------------------------------------------------------- hand-worked pins of single oracle functions
def war_case(dst, uses=("R6", "R7"), kind="rb"):
    st = I("STG", [], ["R2", "R3", "R4"], **{kind: 1})
    prog = one_block([st, I("MOV", ["R9"], ["R8"]), I("IADD", [dst], list(uses), wait=[1])])
    return prog, {(0, 0, 0): 5, (2, C_EXEC, 0): 10, (2, C_EXEC, 1): 40}


def test_write_after_read_flag():
    """Sec. 4, Fig. 6: an execution-dependency edge is write-after-read when its
    resource is a read barrier set by a variable-latency instruction i and the
    stalled instruction j overwrites a register that i reads. Here a store reads R4
    and sets read barrier B1; the next writer of R4 waits on B1. Flags: bit 1 (2) =
    through a barrier, bit 0 (1) = write-after-read. The flag needs all three: a
    read barrier (not a write barrier), j writing (not merely reading) a register
    that i reads, and i of variable latency."""
    def run(dst, uses=("R6", "R7"), kind="rb", arch=ARCH):
        prog, ent = war_case(dst, uses, kind)
        R = oracle.analyze(prog, arch, counts(3, ent))
        e = R["edges"]
        assert list(e["i"]) == [0] and list(e["j"]) == [2]
        assert R["blame"][0, C_EXEC].tolist() == [10, 40] and R["blame"][2, C_EXEC].sum() == 0
        return int(e["flags"][0])
    assert run("R4") == 2 | 1                      # j overwrites R4, which the store reads
    assert run("R9") == 2                          # j writes another register
    assert run("R9", uses=("R4", "R7")) == 2       # j only reads R4: no write after read
    assert run("R4", kind="wb") == 2               # write barrier: a read-after-write wait
    lat, fl = ARCH
    fl = fl.copy()
    fl[synth.OP["STG"]] &= ~np.uint32(synth.F_VARLAT)
    assert run("R4", arch=(lat, fl)) == 2          # fixed-latency i: no barrier to wait for


def register_reuse_case():
    ins = [I("LDL", ["R0"], ["R1"]), I("LDG", ["R4"], ["R2", "R3"]), I("MOV", ["R9"], ["R8"]),
           I("FFMA", ["R5"], ["R0", "R4", "R6"])]
    return one_block(ins), {(0, 0, 0): 30, (1, 0, 0): 20, (2, 0, 0): 10, (3, C_MEM, 0): 30, (3, C_MEM, 1): 60,
                            (3, C_EXEC, 1): 8}


def test_register_reuse_local_memory_blame():
    """Table 2 Register Reuse: memory-dependency stalls blamed on local-memory
    instructions. The FFMA reads R0 from an LDL (3 instructions up) and R4 from an
    LDG (2 up). Issue/longest path is 30/3 = 20/2 for both, so Eq. 1 splits evenly:
    memory stalls 30 active + 60 latency -> 15 + 30 to each load, execution stalls
    8 (latency) -> 4 + 4. Register Reuse takes only the LDL's memory shares: M = 45,
    Eq. 2 gives T / (T - M) = 158 / 113. Code Reordering takes execution latency
    samples and global-memory latency samples: 4 + 4 + 30 = 38, min(A = 90, 38)."""
    prog, ent = register_reuse_case()
    R = oracle.analyze(prog, ARCH, counts(4, ent))
    assert R["blame"][0, C_MEM].tolist() == [15, 30] and R["blame"][1, C_MEM].tolist() == [15, 30]
    assert R["blame"][0, C_EXEC].tolist() == [0, 4] and R["blame"][1, C_EXEC].tolist() == [0, 4]
    T, A, L, _ = (int(x) for x in R["totals"][0])
    assert (T, A, L) == (158, 90, 68)
    assert R["M"][0][0] == 45 and R["speedup"][0][0] == 158 / 113
    assert R["M"][0][7] == 38 and R["speedup"][0][7] == 158 / 120
    assert R["n_hot"][0][0] == 1 and list(R["hot"][0][0][0][[0, 1, 4, 5]]) == [0, 3, 3, 45]


def transaction_case():
    ins = [I("LDG", ["R0"], ["R2", "R3"]), I("LDS", ["R4"], ["R5"]), I("STG", [], ["R2", "R3", "R0"]), I("EXIT")]
    return one_block(ins), {(0, 8, 0): 7, (0, 8, 1): 5, (1, 8, 1): 9, (2, 8, 0): 4, (0, 0, 0): 10, (3, 9, 0): 5}


def test_memory_transaction_reduction_global_only():
    """Table 2 Memory Transaction Reduction: memory-throttle samples at global-memory
    instructions. Throttling at the LDG (7 + 5) and the STG (4) counts, at the LDS (9)
    it does not: M = 16 of T = 40, Eq. 2 = 40 / 24; hotspots are the instructions
    themselves (def = use, distance 0), the larger first."""
    prog, ent = transaction_case()
    R = oracle.analyze(prog, ARCH, counts(4, ent))
    assert int(R["totals"][0][0]) == 40
    assert R["M"][0][5] == 16 and R["speedup"][0][5] == 40 / 24
    assert R["n_hot"][0][5] == 2
    assert R["hot"][0][5][0].tolist() == [0, 0, 0, 0, 0, 12] and R["hot"][0][5][1].tolist() == [2, 2, 0, 0, 0, 4]


def fast_math_case():
    ins = [I("MOV", ["R1"], ["R2"]), I("MUFU", ["R3"], ["R1"], flags=1), I("FFMA", ["R4"], ["R3", "R5", "R6"], flags=1),
           I("FFMA", ["R7"], ["R4", "R5", "R6"])]
    return one_block(ins), {(0, 0, 0): 5, (1, 0, 0): 20, (1, C_EXEC, 1): 6, (1, 7, 0): 3, (1, 1, 1): 2,
                            (2, C_EXEC, 0): 4, (3, C_EXEC, 1): 10}


def test_fast_math_stalls_at_math_library_instructions():
    """Table 2 Fast Math: stall samples observed at instructions of a math-library
    routine (iflags bit 0). The flagged MUFU has 20 issued samples (not stalls) and
    6 + 3 + 2 stalls of three reasons; the flagged FFMA after it 4; the unflagged
    FFMA's 10 do not count. The stalls are taken where they were sampled, before
    blame moves dependency stalls to their sources: M = 15 of T = 50, Eq. 2 = 50 / 35.
    (Counted after blame it would be 9 + 10 = 19.)"""
    prog, ent = fast_math_case()
    R = oracle.analyze(prog, ARCH, counts(4, ent))
    assert int(R["totals"][0][0]) == 50
    assert R["M"][0][3] == 15 and R["speedup"][0][3] == 50 / 35
    assert R["hot"][0][3][0].tolist() == [1, 1, 0, 0, 0, 11] and R["hot"][0][3][1].tolist() == [2, 2, 0, 0, 0, 4]


def _nest_program():
    """Entry B0; outer loop B1..B3 (header B1, latch B3); inner single-block loop B2
    inside it; exit B4."""
    b0 = [I("LDG", ["R0"], ["R2", "R3"])]                                          # 0
    b1 = [I("LDG", ["R4"], ["R2", "R3"]), I("MOV", ["R9"], ["R8"])]                # 1, 2
    b2 = [I("IADD", ["R5"], ["R4", "R6"]), I("LDG", ["R10"], ["R2", "R3"]),         # 3, 4
          I("FFMA", ["R11"], ["R10", "R0", "R6"]), I("ISETP", ["P0"], ["R5", "R6"]),  # 5, 6
          I("BRA", [], [], guard="P0")]                                             # 7
    b3 = [I("IMAD", ["R12"], ["R5", "R6"]), I("IADD", ["R13"], ["R12", "R6"]),      # 8, 9
          I("ISETP", ["P1"], ["R13", "R6"]), I("BRA", [], [], guard="P1")]           # 10, 11
    b4 = [I("EXIT")]                                                                # 12
    return program([([b0, b1, b2, b3, b4], [[1], [2], [2, 3], [1, 4], []], [(1, [1, 2, 3], -1), (2, [2], 0)])])


def nest_case():
    return _nest_program(), {(0, 0, 0): 10, (1, 0, 0): 10, (4, 0, 0): 10, (8, 0, 0): 10,
                             (3, C_MEM, 1): 40, (5, C_MEM, 1): 30, (9, C_EXEC, 1): 12, (9, C_EXEC, 0): 3,
                             (6, 9, 0): 7, (2, 9, 0): 5, (12, 9, 0): 4, (0, 9, 0): 2}


def test_eq5_two_level_loop_nest_by_hand():
    """Eq. 5 scopes on a two-level nest, every term by hand. Edges with latency
    samples: LDG@1 -> IADD@3 (memory, 40; innermost common loop: outer), LDG@4 ->
    FFMA@5 (memory 25 after Eq. 1 gives it 5:1 against LDG@0: issue 10 over paths
    1 and 5), LDG@0 -> FFMA@5 (memory 5; the def is outside every loop) and
    IMAD@8 -> IADD@9 (execution, 12; outer). A of a loop sums the active samples of
    its body with nested loops: inner = 10 + 7 = 17, outer = 10 + 5 + 17 + 10 + 3 =
    45. M^L of a loop sums edges whose innermost common loop is nested in it: inner
    = 25, outer = 40 + 25 + 12 = 77. T = 143, so S_inner = 143 / (143 - 17) and
    S_outer = 143 / (143 - 45). At function scope Loop Unrolling has M^L = 77 and
    Code Reordering 82 (the edge from outside the loops too), both bounded by A = 61
    in Eq. 4."""
    prog, ent = nest_case()
    R = oracle.analyze(prog, ARCH, counts(13, ent))
    assert R["blame"][4, C_MEM, 1] == 25 and R["blame"][0, C_MEM, 1] == 5 and R["blame"][1, C_MEM, 1] == 40
    T, A, L, _ = (int(x) for x in R["totals"][0])
    assert (T, A, L) == (143, 61, 82)
    assert R["loop_A"].tolist() == [45, 17]
    assert R["loop_ML"].tolist() == [77, 25]
    assert R["loop_S"].tolist() == [143 / 98, 143 / 126]
    assert R["M"][0][6] == 77 and R["M"][0][7] == 82
    assert R["speedup"][0][6] == 143 / 82 and R["speedup"][0][7] == 143 / 82


def lines_case():
    ins = [I("LDG", ["R0"], ["R2", "R3"], line=5), I("MOV", ["R9"], ["R8"], line=5),
           I("FFMA", ["R1"], ["R0", "R6", "R7"], line=7), I("EXIT", line=7)]
    return one_block(ins), {(0, 0, 0): 10, (1, 1, 0): 6, (1, 1, 1): 4, (2, C_MEM, 0): 20, (2, C_MEM, 1): 30,
                            (2, 9, 0): 5, (3, 0, 0): 3}


def test_line_rollup_after_blame():
    """Lines sum the stall samples (every reason but SELECTED) that blame leaves on
    their instructions, and the latency part of them. Line 5 holds the LDG, which
    takes the FFMA's memory stalls (20 + 30), and a MOV with instruction-fetch
    stalls (6 + 4): 60 samples, 34 latency. Line 7 keeps the FFMA's own
    not-selected samples (5, active) and the EXIT's issued samples do not count."""
    prog, ent = lines_case()
    R = oracle.analyze(prog, ARCH, counts(4, ent))
    assert R["line_stall"].tolist() == [0, 0, 0, 0, 0, 60, 0, 5]
    assert R["line_lat"].tolist() == [0, 0, 0, 0, 0, 34, 0, 0]


def test_edges_of_selected_uses_equal_full_analysis():
    """The oracle's per-use entry (used where the whole analysis is too slow) gives,
    for any set of uses, exactly the rows of the full analysis's edge list."""
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps[:5], kz)
    cnt, _ = oracle.histogram(P, P.samples(200_000, seed=3))
    R = oracle.analyze(P, ARCH, cnt)["edges"]
    uses = np.unique(R["j"])
    pick = np.random.default_rng(3).choice(uses, size=len(uses) // 3, replace=False)
    pick = np.concatenate([pick, [0, P.n_instr - 1]])          # unstalled uses add nothing
    got = oracle.edges_of_uses(P, ARCH, cnt, pick)
    keep = np.isin(R["j"], pick)
    for k in ("j", "i", "dmin", "dlong", "flags", "share"):
        assert np.array_equal(got[k], R[k][keep]), k
    assert len(got["j"]) > 0


def inlining_case(with_calls=True):
    """f0 calls device function f1 at instruction 2; f2 is unrelated."""
    f0 = [I("LDG", ["R0"], ["R2", "R3"]), I("MOV", ["R1"], ["R4"]), I("CALL", ["R5"], ["R0"]),
          I("FFMA", ["R6"], ["R5", "R7", "R8"]), I("EXIT")]
    f1 = [I("IADD", ["R1"], ["R2", "R3"]), I("FFMA", ["R4"], ["R1", "R5", "R6"]), I("EXIT")]
    f2 = [I("LDG", ["R0"], ["R2", "R3"]), I("FFMA", ["R1"], ["R0", "R4", "R5"]), I("EXIT")]
    prog = program([([f0], [[]], []), ([f1], [[]], []), ([f2], [[]], [])], calls=[(2, 1)] if with_calls else [])
    ent = {(0, 0, 0): 10, (1, 0, 0): 5, (2, C_MEM, 1): 20, (2, 9, 1): 5, (2, 9, 0): 3, (3, C_EXEC, 1): 7,
           (5, 0, 0): 4, (6, C_EXEC, 1): 12, (6, C_EXEC, 0): 6, (7, 1, 1): 2,
           (8, 0, 0): 3, (9, C_MEM, 1): 9}
    return prog, ent


def test_function_inlining_device_functions_and_call_sites():
    """Table 2 Function Inlining, a latency-hiding optimizer (Eq. 4): the latency
    stall samples sampled in device functions and at their call sites. f0 (T = 50,
    A = 18) has 20 memory + 5 not-selected latency samples at its call instruction
    (the 3 active ones and the FFMA's 7 after the call do not count): M^L = 25,
    S = 50 / (50 - min(18, 25)) = 50 / 32. f1 is the device function (T = 24, A =
    10): its latency stalls 12 + 2, S = 24 / (24 - 10). f2 takes no part: M = 0,
    S = 1. The call-site stalls count where they were sampled (blame moves the
    memory stall to the load). Without the call table nothing matches."""
    prog, ent = inlining_case()
    R = oracle.analyze(prog, ARCH, counts(11, ent))
    assert R["blame"][0, C_MEM, 1] == 20                          # the call's memory stall goes to the load
    assert [list(map(int, t[:2])) for t in R["totals"]] == [[50, 18], [24, 10], [12, 3]]
    assert R["M"][:, 8].tolist() == [25, 14, 0]
    assert R["speedup"][:, 8].tolist() == [50 / 32, 24 / 14, 1.0]
    assert R["hot"][0][8][0].tolist() == [2, 2, 0, 0, 0, 25]
    assert R["hot"][1][8][:2].tolist() == [[1, 1, 0, 0, 0, 12], [2, 2, 0, 0, 0, 2]]
    assert R["n_hot"][:, 8].tolist() == [1, 2, 0]
    # in f1 the FFMA's execution latency stalls are blamed on the IADD one up, so Code
    # Reordering also has M^L = 12 and the same 24 / 14: equal speedups rank the lower id first
    assert R["speedup"][1][7] == 24 / 14 and R["rank"][1][:2].tolist() == [7, 8]
    prog, ent = inlining_case(with_calls=False)
    R = oracle.analyze(prog, ARCH, counts(11, ent))
    assert R["M"][:, 8].tolist() == [0, 0, 0] and R["speedup"][:, 8].tolist() == [1.0, 1.0, 1.0]


def test_add_calls_keeps_dataflow():
    """The generator's call tables turn MOVs into CALLs: ascending distinct sites in
    functions other than their callee, the same defs and uses, and the oracle's
    edges change only through the call's latency."""
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps[:8], kz)
    a = synth.add_calls(P, 0.25, seed=1)
    cs, cc = a["call_site"], a["call_callee"]
    assert cs.size > 0 and np.all(np.diff(cs) > 0)
    fio = P.func_instr_off
    for x, d in zip(cs, cc):
        assert not (fio[d] <= x < fio[d + 1])
        assert a["opclass"][x] == synth.OP["CALL"] and P.opclass[x] == synth.OP["MOV"]
    assert np.array_equal(np.delete(a["opclass"], cs), np.delete(P.opclass, cs))
    sub = synth.subprogram(a, 0, 8)
    assert np.array_equal(sub["call_site"], cs) and np.array_equal(sub["call_callee"], cc)

"""CUDA path (through the C ABI) against the CPU oracle, element by element:
counts, reaching masks, merged edges with their distances and shares, blame,
and advice. Bit-exact for every integer; FP64 speedups within 1e-12 relative."""
import numpy as np
import pytest

import oracle
import synth
from bruteforce import tiny_program
from parity import ARCH, RTOL, assert_advice_equal, assert_edges_equal, assert_full_parity, gpu_run, oracle_run
from progbuild import I, counts, program

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2009_04061_gb300 as g
    c = g.Context(ARCH)
    yield c
    c.close()


def dev(samples):
    import torch
    return torch.from_numpy(np.ascontiguousarray(samples).view(np.int64)).cuda()


def test_paper_examples_blame(ctx):
    import test_oracle as T
    for prog, cnt_entries in [
        (T.fig4(), {(7, 0, 0): 10, (4, 0, 0): 20, (5, 0, 0): 7, (10, 3, 0): 100, (10, 2, 1): 9}),
        (T.one_block([I("LDG", ["R0"], ["R2", "R3"], wb=0), I("IADD", ["R5"], ["R6", "R7"]),
                      I("BRA", [], [], wait=[0])]), {(0, 0, 0): 5, (2, 3, 0): 40, (2, 3, 1): 60}),
        (T.diamond(False), {(0, 0, 0): 3, (5, 3, 1): 30, (3, 2, 0): 4}),
        (T.diamond(True), {(0, 0, 0): 3, (6, 3, 1): 30, (4, 2, 0): 4}),
    ]:
        ss = []
        for (pc, c, l), v in cnt_entries.items():
            ss += [(0 << 48) | (pc << 24) | (c << 20) | (l << 19)] * v
        s = np.array(ss, dtype=np.uint64)
        g = gpu_run(ctx, prog, dev(s))
        R = oracle_run(prog, s)
        assert_full_parity(g, R)


def _samples_of(entries):
    ss = []
    for (pc, c, l), v in entries.items():
        ss += [(pc << 24) | (c << 20) | (l << 19)] * v
    return np.array(ss, dtype=np.uint64)


def test_hand_worked_pins(ctx):
    """The oracle's hand-worked cases (write-after-read, Register Reuse, Memory
    Transaction Reduction, Fast Math, the two-level Eq. 5 nest, line roll-up) through
    the CUDA path: every output equals the oracle's, and the hand-derived values hold."""
    import test_oracle as T
    cases = [T.war_case("R4"), T.war_case("R9"), T.war_case("R9", uses=("R4", "R7")), T.war_case("R4", kind="wb"),
             T.register_reuse_case(), T.transaction_case(), T.fast_math_case(), T.nest_case(), T.lines_case()]
    got = []
    for prog, ent in cases:
        s = _samples_of(ent)
        g = gpu_run(ctx, prog, dev(s))
        assert_full_parity(g, oracle_run(prog, s))
        got.append(g)
    assert [int(g["edges"]["flags"][0]) for g in got[:4]] == [3, 2, 2, 2]
    assert got[4]["advice"]["matched"][0][0] == 45 and got[5]["advice"]["matched"][0][5] == 16
    assert got[6]["advice"]["matched"][0][3] == 15
    assert got[7]["advice"]["loop_active"].tolist() == [45, 17] and got[7]["advice"]["loop_matched"].tolist() == [77, 25]
    assert got[8]["advice"]["line_stall"].tolist() == [0, 0, 0, 0, 0, 60, 0, 5]


def test_function_inlining(ctx):
    """Function Inlining from the call table (Table 2): the hand-worked three-function
    case and a generated program whose MOVs partly became calls; everything equals the
    oracle, and call tables that break the format are refused."""
    import test_oracle as T
    import paper_2009_04061_gb300 as g
    prog, ent = T.inlining_case()
    fio, ss = prog["func_instr_off"], []
    for (x, c, l), v in ent.items():       # global instruction index -> (kernel, pc)
        k = int(np.searchsorted(fio, x, side="right")) - 1
        ss += [(k << 48) | ((x - int(fio[k])) << 24) | (c << 20) | (l << 19)] * v
    s = np.array(ss, dtype=np.uint64)
    gr = gpu_run(ctx, prog, dev(s))
    R = oracle_run(prog, s)
    assert_full_parity(gr, R)
    assert gr["advice"]["matched"][:, 8].tolist() == [25, 14, 0]
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps, kz)
    a = synth.add_calls(P, 0.2, seed=3)
    s = P.samples(2_000_000, seed=3)
    gr = gpu_run(ctx, a, dev(s))
    R = oracle_run(a, s)
    assert_full_parity(gr, R)
    assert (gr["advice"]["matched"][:, 8] > 0).sum() >= 4
    bad = [dict(a, call_site=a["call_site"][::-1].copy(), call_callee=a["call_callee"][::-1].copy()),
           dict(a, call_site=np.array([a["n_instr"]], np.int32), call_callee=np.array([0], np.int32)),
           dict(a, call_site=np.array([0], np.int32), call_callee=np.array([a["n_functions"]], np.int32))]
    for b in bad:
        with pytest.raises(g.GpaError) as e:
            ctx.load_program(b)
        assert e.value.status == -2


@pytest.mark.parametrize("seed", range(16))
def test_tiny_guarded_programs(ctx, seed):
    P = tiny_program(seed, n_instr=25 + seed, n_loops=seed % 3, guard_pct=20 + 3 * seed)
    s = P.samples(20_000, seed=seed)
    g = gpu_run(ctx, P, dev(s))
    assert_full_parity(g, oracle_run(P, s))


def test_plain_workload(ctx):
    ps, ns, kz = synth.workload("plain")
    P = synth.make_program(ps, kz)
    s = P.samples(ns)
    g = gpu_run(ctx, P, dev(s))
    assert_full_parity(g, oracle_run(P, s))


def test_rodinia_workload_with_invalid_and_ragged_tail(ctx):
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps, kz)
    s = P.samples(2_000_003, invalid_ppm=3000)      # odd count: scalar tail
    g = gpu_run(ctx, P, dev(s))
    R = oracle_run(P, s)
    assert R["invalid"] > 0
    assert_full_parity(g, R)


def test_misaligned_start_and_edge_sizes(ctx):
    ps, _, kz = synth.workload("plain")
    P = synth.make_program(ps, kz)
    s = P.samples(10_001)
    d = dev(s)
    for lo, hi in [(1, 10_001), (1, 2), (0, 1), (3, 4), (0, 0)]:
        g = gpu_run(ctx, P, d[lo:hi])
        cnt, bad = oracle.histogram(P, s[lo:hi])
        assert np.array_equal(g["counts"], cnt) and g["invalid"] == bad


def test_all_invalid_samples(ctx):
    ps, _, kz = synth.workload("plain")
    P = synth.make_program(ps, kz)
    bad = np.array([(5 << 48), (0 << 48) | (300 << 24), (0 << 48) | (13 << 20), (1 << 19), 7], dtype=np.uint64)
    g = gpu_run(ctx, P, dev(np.tile(bad, 1000)))
    assert g["invalid"] == 5000 and int(g["counts"].sum()) == 0
    assert int(g["blame"].sum()) == 0 and g["status"] == 0


def test_batched_subset_of_uneven_functions(ctx):
    rng = np.random.default_rng(5)
    ps = synth.batched_params(60, rng, 5)
    P = synth.make_program(ps, 1.0)
    s = P.samples(6_000_000, seed=5)
    g = gpu_run(ctx, P, dev(s))
    assert_full_parity(g, oracle_run(P, s))


def test_host_ingest_pinned_and_pageable(ctx):
    """Host samples: pinned memory read by the aggregation kernel over the host link
    (also from an interior pointer that is not 16-byte aligned), pageable memory
    through the staging buffers; all give the oracle's counts and the device path's blame."""
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps, kz)
    s = P.samples(1_000_001, invalid_ppm=1000, seed=3)
    import torch
    g2 = gpu_run(ctx, P, dev(s))
    cnt, bad = oracle.histogram(P, s)
    assert np.array_equal(g2["counts"], cnt) and g2["invalid"] == bad
    h = torch.from_numpy(s.view(np.int64)).pin_memory()
    for host, (c, b) in [(h, (cnt, bad)), (h[1:], oracle.histogram(P, s[1:])), (s.copy(), (cnt, bad))]:
        g1 = gpu_run(ctx, P, None, host=host)
        assert np.array_equal(g1["counts"], c) and g1["invalid"] == b
    g1 = gpu_run(ctx, P, None, host=h)
    assert np.array_equal(g1["blame"], g2["blame"])


def test_plain_per_function_equals_batched(ctx):
    """Each function loaded alone gives the same results as in the batched program."""
    rng = np.random.default_rng(9)
    ps = synth.batched_params(12, rng, 9)
    P = synth.make_program(ps, 1.0)
    s = P.samples(2_000_000, seed=9)
    gb = gpu_run(ctx, P, dev(s))
    k = (s >> np.uint64(48)).astype(np.int64)
    for f in range(P.n_functions):
        Pf = synth.make_program([ps[f]], 1.0)
        sf = s[k == f] & ~np.uint64(0xFFFF << 48)
        gf = gpu_run(ctx, Pf, dev(sf))
        i0, i1 = P.func_instr_off[f], P.func_instr_off[f + 1]
        assert np.array_equal(gf["blame"], gb["blame"][i0:i1])
        assert np.array_equal(gf["advice"]["speedup"][0], gb["advice"]["speedup"][f])
        # pcs, distance and samples of every hotspot (line ids are offset per program)
        assert np.array_equal(gf["advice"]["hot"][0][..., [0, 1, 4, 5]], gb["advice"]["hot"][f][..., [0, 1, 4, 5]])


def _unnatural_loop_program():
    """A loop whose listed body holds an exit block that cannot reach the latch
    (not a natural loop): carrying the latch's def back to the header takes a
    sweep of the fixpoint that the seeded single sweep of natural loops skips."""
    b0 = [I("MOV", ["R1"], ["R2"])]
    b1 = [I("IADD", ["R3"], ["R1", "R4"])]
    b2 = [I("MOV", ["R1"], ["R5"]), I("ISETP", ["P0"], ["R3", "R6"]), I("BRA", [], [], guard="P0")]
    b3 = [I("FFMA", ["R7"], ["R1", "R3", "R5"]), I("EXIT")]
    return program([([b0, b1, b2, b3], [[1], [2], [1, 3], []], [(1, [1, 2, 3], -1)])])


def test_fixpoint_sweep_limit_reports_not_converged():
    """The sweep limit applies to functions whose loop bodies are not natural loops
    (the others take one sweep that is exact): one sweep leaves such a function
    unconverged and reports it, while the natural plain workload converges within the
    same limit. Without the limit both equal the oracle's fixpoint."""
    import paper_2009_04061_gb300 as g
    odd = _unnatural_loop_program()
    s_odd = np.array([(3 << 24) | (2 << 20)] * 20 + [(1 << 24) | (2 << 20) | (1 << 19)] * 7, dtype=np.uint64)
    ps, ns, kz = synth.workload("plain")
    P = synth.make_program(ps, kz)
    with g.Context(ARCH, dict(max_fixpoint_sweeps=1)) as c:
        assert gpu_run(c, odd, dev(s_odd))["status"] == -4
        r = gpu_run(c, P, dev(P.samples(1000)))
        assert r["status"] == 0 and r["info"]["sweeps"] == 1
    with g.Context(ARCH) as c:
        r = gpu_run(c, odd, dev(s_odd))
        assert r["status"] == 0 and r["info"]["sweeps"] == 2
        assert_full_parity(r, oracle_run(odd, s_odd))


def test_invalid_program_rejected(ctx):
    import paper_2009_04061_gb300 as g
    bad = program([([[I("IADD", ["R1"], ["R2"])], [I("EXIT")]], [[1], [0]], [])])  # back edge without a loop
    with pytest.raises(g.GpaError) as e:
        ctx.load_program(bad)
    assert e.value.status == -2


def test_small_search_slots_overflow_to_large_tier():
    """Tiny first- and second-tier arenas force general searches through all three tiers
    (shared memory, larger shared memory, global memory); results stay exact."""
    import paper_2009_04061_gb300 as g
    with g.Context(ARCH, dict(small_search_nodes=4, mid_search_nodes=16, search_slots=64)) as c:
        rng = np.random.default_rng(11)
        P = synth.make_program(synth.batched_params(20, rng, 11), 1.0)
        s = P.samples(1_000_000, seed=11)
        r = gpu_run(c, P, dev(s))
        assert r["info"]["general_searches"] > 0 and r["info"]["max_nodes"] > 4
        assert_full_parity(r, oracle_run(P, s))


def test_first_tier_warp_counts_agree():
    """The first tier's warps per SM only change how many searches run at once:
    12, 16 and 24 warps (and 128-node arenas at 12) give the oracle's results, and a
    count that is not a multiple of 4 or above 32 is refused."""
    import paper_2009_04061_gb300 as g
    rng = np.random.default_rng(19)
    P = synth.make_program(synth.batched_params(24, rng, 19), 1.0)
    s = P.samples(1_000_000, seed=19)
    R = oracle_run(P, s)
    for opts in (dict(small_search_warps=12), dict(small_search_warps=16),
                 dict(small_search_warps=24, small_search_nodes=32), dict(small_search_nodes=128, small_search_warps=12)):
        with g.Context(ARCH, opts) as c:
            r = gpu_run(c, P, dev(s))
            assert r["info"]["general_searches"] > 0
            assert_full_parity(r, R)
    for bad in (6, 36, -4):
        with pytest.raises(g.GpaError):
            g.Context(ARCH, dict(small_search_warps=bad))


def test_advice_into_reused_pinned_buffers(ctx):
    """Advice copied into one set of pinned host arrays, step after step, equals advice
    copied into fresh arrays."""
    rng = np.random.default_rng(23)
    P = synth.make_program(synth.batched_params(12, rng, 23), 1.0)
    s = P.samples(500_000, seed=23)
    d = dev(s)
    prog = ctx.load_program(P)
    try:
        bufs = prog.advice_buffers(pinned=True)
        for _ in range(2):
            prog.reset()
            prog.ingest(d)
            prog.blame()
            got = prog.advise(fetch=True, out=bufs)
            ref = prog.get_advice()
            assert set(got) == set(ref)
            for k in ref:
                assert np.array_equal(got[k], ref[k], equal_nan=True), k
            bufs["speedup"][...] = 0.0  # the next step overwrites every entry
    finally:
        prog.unload()


def test_tier_hints_on_repeated_steps():
    """Searches that outgrew a tier are queued straight for the bigger one on later
    steps of the same program; every step gives the oracle's results."""
    import paper_2009_04061_gb300 as g
    with g.Context(ARCH, dict(small_search_nodes=4, mid_search_nodes=16, max_search_nodes=64, search_slots=64)) as c:
        rng = np.random.default_rng(13)
        P = synth.make_program(synth.batched_params(16, rng, 13), 1.0)
        s = P.samples(1_000_000, seed=13)
        R = oracle_run(P, s)
        prog = c.load_program(P)
        try:
            d = dev(s)
            tiers = []
            for step in range(3):
                prog.reset()
                prog.ingest(d)
                prog.blame()
                adv = prog.advise(fetch=True)
                st, info = prog.status()
                cnt, bad = prog.counts()
                r = dict(status=st, info=info, counts=cnt, invalid=bad, rin=prog.reaching()[0],
                         rout=prog.reaching()[1], blame=prog.blame_counts(), edges=prog.edges(), advice=adv)
                assert_full_parity(r, R)
                tiers.append((info["tier2_searches"], info["tier3_searches"]))
            # the first step found the big searches by overflow; later steps queue them directly
            assert tiers[0][0] > 0 and tiers[1] == tiers[2]
        finally:
            prog.unload()


def test_large_and_fourth_tier_hints_on_repeated_steps():
    """Later steps start the third-tier searches that were large (here: 8 nodes or more)
    before the others, beside the first two tiers, and send the searches that outgrew
    the third tier straight to the program's own fourth tier; eager steps and CUDA-graph
    launches of the same program give the oracle's results every time."""
    import paper_2009_04061_gb300 as g
    opts = dict(small_search_nodes=4, mid_search_nodes=8, max_search_nodes=32, search_slots=32,
                large_search_nodes=8)
    with g.Context(ARCH, opts) as c:
        rng = np.random.default_rng(12)
        P = synth.make_program(synth.batched_params(12, rng, 12), 1.0)
        s = P.samples(1_000_000, seed=12)
        R = oracle_run(P, s)
        prog = c.load_program(P)
        d = dev(s)

        def results(adv):
            st, info = prog.status()
            cnt, bad = prog.counts()
            rin, rout = prog.reaching()
            return dict(status=st, info=info, counts=cnt, invalid=bad, rin=rin, rout=rout,
                        blame=prog.blame_counts(), edges=prog.edges(), advice=adv)
        try:
            infos = []
            for step in range(3):
                prog.reset()
                prog.ingest(d)
                prog.blame()
                r = results(prog.advise(fetch=True))
                assert_full_parity(r, R)
                infos.append(r["info"])
            assert infos[0]["max_nodes"] > 32 and infos[0]["tier3_searches"] > 0
            assert infos[1]["tier3_searches"] == infos[2]["tier3_searches"]
            prog.capture_step(d)
            for _ in range(2):
                prog.launch_step()
            assert_full_parity(results(prog.get_advice()), R)
        finally:
            prog.unload()


def test_search_of_thousands_of_nodes(ctx):
    """One 20,034-instruction function of the batched workload whose largest search
    (a global-memory search) has more than 4,096 nodes; results equal the oracle's."""
    ps, _, _ = synth.workload("batched")
    P = synth.make_program([ps[1544]], 1.0)
    s = P.samples(2_000_000, seed=3)
    g = gpu_run(ctx, P, dev(s))
    assert g["status"] == 0 and g["info"]["max_nodes"] > 4096, g["info"]
    assert_full_parity(g, oracle_run(P, s))


def test_parallel_optimizers_match_oracle(ctx):
    """Parallel optimizers (Table 2, Eqs. 6-10) from launch statistics: generated ones
    plus launches made to match each rule, on this device's SM model and on a 4-SM
    model. Match flags and binding limits equal the oracle's exactly, warps and
    speedups within 1e-12; clearing the statistics resets the outputs."""
    import paper_2009_04061_gb300 as g
    import torch
    rng = np.random.default_rng(31)
    P = synth.make_program(synth.batched_params(40, rng, 31), 1.0)
    s = P.samples(2_000_000, seed=31)
    R = oracle_run(P, s)
    st = synth.launch_stats(40, seed=31)
    st["blocks"][:5] = [10 ** 5, 3, 10 ** 5, 7, 500]
    st["threads_per_block"][:5] = [32, 256, 16, 1024, 32]
    st["regs_per_thread"][:5] = [32, 64, 0, 40, 24]
    st["smem_per_block"][:5] = [0, 48 * 1024, 0, 200 * 1024, 0]
    dev_sm = g.gpa_sm_model_of_device(torch.cuda.current_device())
    small_sm = dict(dev_sm, n_sms=4)
    prog = ctx.load_program(P)
    try:
        d = dev(s)
        prog.reset()
        prog.ingest(d)
        prog.blame()
        for sm in (dev_sm, small_sm):
            prog.set_launch_stats(st, sm)
            adv = prog.advise(fetch=True)
            exp = oracle.parallel(st, sm, R["totals"])
            assert np.array_equal(adv["totals"], R["totals"])
            assert np.array_equal(adv["par_match"], exp["par_match"]), sm
            assert np.array_equal(adv["par_limit"], exp["par_limit"]), sm
            assert np.allclose(adv["par_speedup"], exp["par_speedup"], rtol=RTOL, atol=0), sm
            assert np.allclose(adv["par_warps"], exp["par_warps"], rtol=RTOL, atol=0), sm
            assert exp["par_match"][:, 0].sum() > 0 and exp["par_match"][:, 1].sum() > 0
        prog.set_launch_stats(None)
        adv = prog.advise(fetch=True)
        assert np.all(adv["par_limit"] == -1) and np.all(adv["par_speedup"] == 1.0) and not adv["par_match"].any()
        # out-of-range statistics or a missing SM model are refused and change nothing
        for k, bad in [("threads_per_block", 0), ("threads_per_block", 1025), ("regs_per_thread", 256),
                       ("blocks", 0), ("smem_per_block", -1)]:
            st_bad = {key: v.copy() for key, v in st.items()}
            st_bad[k][7] = bad
            with pytest.raises(g.GpaError):
                prog.set_launch_stats(st_bad, dev_sm)
        with pytest.raises(g.GpaError):
            prog.set_launch_stats(st, dict(dev_sm, n_sms=0))
        assert np.all(prog.advise(fetch=True)["par_limit"] == -1)
        assert dev_sm["n_sms"] == torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    finally:
        prog.unload()


def test_use_with_many_sources(ctx):
    """A use with 70 surviving sources (past the thread-per-use arrays) is merged and
    apportioned by the shared-memory path, bit for bit like the oracle."""
    import test_oracle as T
    body = [I("ISETP", ["P0"], ["R9"]), I("ISETP", ["P1"], ["R9"])]
    body += [I("LDG", ["R1"], ["R2", "R3"], guard="P0") for _ in range(70)]
    body += [I("IADD", ["R4"], ["R1", "R5"], guard="P1")]
    prog = T.one_block(body)
    j = len(body) - 1
    ss = [(j << 24) | (3 << 20)] * 1000 + [(j << 24) | (3 << 20) | (1 << 19)] * 777
    ss += [((2 + k) << 24) for k in range(70) for _ in range(k + 1)]   # issued samples of the loads
    s = np.array(ss, dtype=np.uint64)
    g = gpu_run(ctx, prog, dev(s))
    R = oracle_run(prog, s)
    assert len(R["edges"]["j"]) == 70
    assert_full_parity(g, R)


def test_fourth_tier_program_arena():
    """A third tier of 32 nodes sends the larger searches on to the program's own
    fourth tier (sized from its largest function); results stay exact."""
    import paper_2009_04061_gb300 as g
    with g.Context(ARCH, dict(small_search_nodes=4, mid_search_nodes=8, max_search_nodes=32, search_slots=32)) as c:
        rng = np.random.default_rng(12)
        P = synth.make_program(synth.batched_params(12, rng, 12), 1.0)
        s = P.samples(1_000_000, seed=12)
        r = gpu_run(c, P, dev(s))
        assert r["status"] == 0 and r["info"]["max_nodes"] > 32
        assert_full_parity(r, oracle_run(P, s))


def test_full_batched_workload_sampled_functions(ctx):
    """The bench's workload at full size (2,000 functions, 5e8 samples): invariants over the
    whole program, and a stratified sample of functions (every 10th by size, plus the sizes
    nearest 60, 400, 1,500, 5,000 and 20,000 instructions: about 205, so every search tier's
    size range is met) against the oracle element by element: counts, RIN/ROUT, blame,
    edges with shares, and advice."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    ps, n, kz = synth.workload("batched")
    P = synth.make_program(ps, kz)
    host = torch.empty(n, dtype=torch.int64)
    s = P.samples(n, out=host.numpy().view(np.uint64))
    g = gpu_run(ctx, P, host.cuda())
    assert g["status"] == 0, g["info"]
    assert int(g["counts"].sum()) + g["invalid"] == n
    assert np.array_equal(g["blame"].sum(0), g["counts"].sum(0))          # conservation per class and flag
    sizes = np.diff(P.func_instr_off)
    by_size = np.argsort(sizes, kind="stable")
    picks = {int(np.argmin(np.abs(sizes - t))) for t in (60, 400, 1500, 5000, 20000)}
    picks |= {int(f) for f in by_size[::10]}
    picks = sorted(picks)
    # The oracle's histogram of the picked functions' samples (every sample of a picked
    # function is in the subset, so its counters are complete), in slices on host threads.
    keep = np.zeros(P.n_functions + 1, bool)  # the last entry: kernel ids past the program
    keep[picks] = True
    kid = np.minimum(s >> np.uint64(48), np.uint64(P.n_functions)).astype(np.int64)
    sub = s[keep[kid]]
    del kid
    with ThreadPoolExecutor(8) as ex:
        parts = list(ex.map(lambda x: oracle.histogram(P, x)[0], np.array_split(sub, 4)))
        cnt = parts[0]
        for c in parts[1:]:
            cnt += c
        del parts
        results = list(ex.map(lambda f: (oracle.analyze(P, ARCH, cnt, f, f + 1), oracle.reaching(P, f, f + 1)), picks))
    for f, (R, (rin, rout)) in zip(picks, results):
        i0, i1 = int(P.func_instr_off[f]), int(P.func_instr_off[f + 1])
        b0, b1 = int(P.func_block_off[f]), int(P.func_block_off[f + 1])
        l0, l1 = int(P.func_loop_off[f]), int(P.func_loop_off[f + 1])
        assert np.array_equal(g["counts"][i0:i1], cnt[i0:i1]), f
        assert np.array_equal(g["rin"][b0:b1], rin) and np.array_equal(g["rout"][b0:b1], rout), f
        assert np.array_equal(g["blame"][i0:i1], R["blame"]), f
        assert_edges_equal(g["edges"], R["edges"], i0, i1)
        assert_advice_equal(dict(g["advice"]), R, f, f + 1, l0, l1)


def test_graph_step_matches_eager(ctx):
    """The CUDA-graph step (reset, ingest, blame, advise) gives the eager step's results, launch after launch."""
    ps, ns, kz = synth.workload("rodinia", 1)
    P = synth.make_program(ps, kz, 1)
    s = dev(P.samples(ns, seed=1))
    eager = gpu_run(ctx, P, s)
    graph = gpu_run(ctx, P, s, graph_launches=3)
    assert graph["status"] == 0
    for k in ("counts", "invalid", "rin", "rout", "blame"):
        assert np.array_equal(np.asarray(eager[k]), np.asarray(graph[k])), k
    assert_edges_equal(graph["edges"], eager["edges"])
    for k in eager["advice"]:
        assert np.array_equal(eager["advice"][k], graph["advice"][k]), k


def test_histogram_variants_agree():
    """Every aggregation variant the autotuner may pick gives the oracle's counts."""
    import paper_2009_04061_gb300 as g
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps, kz)
    s = P.samples(3_000_001, invalid_ppm=2000, seed=4)
    cnt, bad = oracle.histogram(P, s)
    d = dev(s)
    for v in (0, 1, 2, 3):
        with g.Context(ARCH, dict(hist_variant=v)) as c:
            r = gpu_run(c, P, d, advise=False)
            assert np.array_equal(r["counts"], cnt) and r["invalid"] == bad, v
            for lo, hi in [(1, 3_000_001), (0, 1), (5, 4101), (3, 3)]:  # unaligned, tiny, one tile, empty
                r = gpu_run(c, P, d[lo:hi], advise=False)
                c2, b2 = oracle.histogram(P, s[lo:hi])
                assert np.array_equal(r["counts"], c2) and r["invalid"] == b2, (v, lo, hi)
    # one hot counter far past 2^16
    hot = np.full(1_000_003, s[0], dtype=np.uint64)
    ch, bh = oracle.histogram(P, hot)
    with g.Context(ARCH, dict(hist_variant=0)) as c:
        r = gpu_run(c, P, dev(hot), advise=False)
        assert np.array_equal(r["counts"], ch) and r["invalid"] == bh
    # a stream with interleaved kernels (every tile straddles many kernels)
    si = P.samples(1_000_000, seed=6, order="interleaved")
    ci, bi = oracle.histogram(P, si)
    with g.Context(ARCH, dict(hist_variant=0)) as c:
        r = gpu_run(c, P, dev(si), advise=False)
        assert np.array_equal(r["counts"], ci) and r["invalid"] == bi


def test_histogram_partial_window():
    """Kernels larger than the aggregation window (2,078 instructions): samples
    inside the window placed for the run, samples outside it, hot counters in
    both far past 65,536, and malformed samples of the windowed kernel."""
    # (n_instr, n_loops, seed) of the generator; the two middle functions come out
    # at exactly 2,078 and 2,079 instructions, the window's size and one more
    shapes = [(500, 1, 40), (2051, 5, 75), (2053, 5, 75), (5000, 12, 43), (12000, 30, 44), (20000, 50, 45)]
    ps = [dict(n_instr=n, n_loops=nl, max_depth=5, n_regs=128, zipf_s=1.1, seed=sd) for n, nl, sd in shapes]
    P = synth.make_program(ps, 1.0, 3)
    n_instr = np.diff(P.func_instr_off)
    assert list(n_instr[1:3]) == [2078, 2079]
    s = P.samples(3_000_001, invalid_ppm=2000, seed=7)
    cnt, bad = oracle.histogram(P, s)
    with g_context() as c:
        r = gpu_run(c, P, dev(s), advise=False)
        assert np.array_equal(r["counts"], cnt) and r["invalid"] == bad

        def pack(k, pc, cls, lat, low=0):
            return np.uint64((k << 48) | (pc << 24) | (cls << 20) | (lat << 19) | low)
        k = 5  # about 20,000 instructions
        a, b = pack(k, 100, 2, 1), pack(k, 15000, 3, 0)
        crafted = np.empty(400_006, dtype=np.uint64)
        crafted[0::2], crafted[1::2] = a, b
        junk = [pack(k, 101, 12, 0), pack(k, 102, 0, 1), pack(k, 103, 2, 0, low=1 << 3),
                pack(k, int(n_instr[k]), 2, 0), pack(k, 3000, 15, 1), pack(6, 0, 0, 0)]
        crafted[1000:1000 + len(junk)] = junk
        crafted[300_000:300_000 + len(junk)] = junk
        ch, bh = oracle.histogram(P, crafted)
        assert bh == 2 * len(junk)
        r = gpu_run(c, P, dev(crafted), advise=False)
        assert np.array_equal(r["counts"], ch) and r["invalid"] == bh


def g_context(**opts):
    import paper_2009_04061_gb300 as g
    return g.Context(ARCH, dict(hist_variant=0, **opts))


def test_autotune_picks_a_timed_candidate():
    import torch
    from paper_2009_04061_gb300 import autotune
    ps, ns, kz = synth.workload("plain")
    P = synth.make_program(ps, kz)
    d = dev(P.samples(ns))
    dims = [("hist_variant", (0, 1)), ("hist_chunk", (24, 8)), ("reach_schedule", (0, 1)),
            ("search_slots_per_sm", (0, 4))]
    best, table = autotune.tune(ARCH, P.arrays, d, torch.cuda.current_stream(), dims=dims, reps=1)
    assert best in [t[0] for t in table] and all(ms > 0 for _, ms in table)
    assert 4 <= len(table) <= 5                       # one pass: the start and each other value once


def test_reach_schedules_agree(ctx):
    """The fixpoint's two schedules (a warp per function staged in shared memory, and the
    windowed kernel with a lane per basic block for every function) give the oracle's
    RIN/ROUT and everything after them, on programs of every size class."""
    import paper_2009_04061_gb300 as g
    rng = np.random.default_rng(17)
    P = synth.make_program(synth.batched_params(30, rng, 17), 1.0)
    s = P.samples(1_000_000, seed=17)
    R = oracle_run(P, s)
    for sched in (0, 1):
        with g.Context(ARCH, dict(reach_schedule=sched)) as c:
            assert_full_parity(gpu_run(c, P, dev(s)), R)
    with pytest.raises(g.GpaError):
        g.Context(ARCH, dict(reach_schedule=2))


@pytest.mark.parametrize("which", ["rodinia", "tiny", "batched_subset"])
def test_dependency_coverage(ctx, which):
    """Single dependency coverage (Sec. 6) from the unbounded GPU searches equals the
    oracle's; blame and edges of the program are left as they were."""
    if which == "rodinia":
        ps, ns, kz = synth.workload("rodinia")
        P = synth.make_program(ps, kz)
        s = P.samples(2_000_000, seed=21)
    elif which == "tiny":
        P = tiny_program(21, n_instr=36, n_loops=2, guard_pct=40)
        s = P.samples(30_000, seed=21)
    else:
        P = synth.make_program(synth.batched_params(24, np.random.default_rng(21), 21), 1.0)
        s = P.samples(2_000_000, seed=21)
    cnt, _ = oracle.histogram(P, s)
    want = oracle.coverage(P, ARCH, cnt)
    prog = ctx.load_program(P)
    try:
        prog.reset()
        prog.ingest(dev(s))
        prog.blame()
        e1, b1 = prog.edges(), prog.blame_counts()
        got = prog.coverage()
        assert got == want
        assert got[0] > 0 and got[1] <= got[2]
        assert np.array_equal(prog.blame_counts(), b1)
        e2 = prog.edges()
        for k in e1:
            assert np.array_equal(e1[k], e2[k]), k
    finally:
        prog.unload()


@pytest.mark.parametrize("which", ["tiny", "guarded", "rodinia"])
def test_unpruned_edge_export(ctx, which):
    """The exported dependency graph before pruning equals the oracle's search, source by
    source, for every stalled use and resource (the dominator rule evaluated for all)."""
    if which == "rodinia":
        ps, ns, kz = synth.workload("rodinia")
        P = synth.make_program(ps[:6], kz)
        s = P.samples(400_000, seed=22)
    else:
        P = tiny_program(22 if which == "tiny" else 23, n_instr=40, n_loops=2,
                         guard_pct=20 if which == "tiny" else 45)
        s = P.samples(40_000, seed=22)
    cnt, _ = oracle.histogram(P, s)
    prog = ctx.load_program(P)
    try:
        prog.reset()
        prog.ingest(dev(s))
        prog.blame()
        x = prog.unpruned_edges()
    finally:
        prog.unload()
    c3 = cnt.reshape(-1, 12, 2)
    want = []
    uo, ur = P.use_off, P.use_res
    for j in range(P.n_instr):
        if c3[j, [2, 3, 5, 6]].sum() == 0:
            continue
        for r in sorted(set(int(v) & 0x1FF for v in ur[uo[j]:uo[j + 1]])):
            for src in oracle.search(P, j, r):
                want.append((j, r, src["i"], src["dmin"], src["K"], src["dlong"], int(src["dom"])))
    want.sort()
    got = sorted(zip(*(x[k].tolist() for k in ("use", "res", "def", "dmin", "K", "dlong", "dom"))))
    assert len(want) > 0
    assert got == want

"""The device side of a sharded batch on one GPU. Two ranks run one after the
other (their one exchange is the sum of their count rows on the device: one GPU
has no peer to reduce with): each counts its chunk of the samples over the
whole program, copies the counters out (gpa_copy_counts), and each owner loads
its functions' summed rows into its own program (gpa_set_counts) and runs blame
and advice. Every result equals the unsharded run and the oracle."""
import numpy as np
import pytest

import oracle
import synth
from paper_2009_04061_gb300 import shard
from parity import ARCH, assert_advice_equal, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def test_two_owners_on_one_gpu_equal_the_whole_batch():
    import torch
    import paper_2009_04061_gb300 as g
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps, kz)
    a = synth.add_calls(P, 0.3, seed=2)
    n, world = 2_000_001, 2
    s = P.samples(n, seed=6)
    owners = shard.lpt_owners(shard.function_costs(a), world)
    with g.Context(ARCH) as ctx:
        whole = gpu_run(ctx, a, _dev(s))
        R = oracle_run(a, s)
        assert np.array_equal(whole["blame"], R["blame"])
        full = ctx.load_program(a)
        partials = []
        for r in range(world):
            lo, hi = shard.sample_range(n, r, world)
            full.reset()
            full.ingest(_dev(s[lo:hi]))
            t = torch.empty(a["n_instr"] * 24, dtype=torch.int64, device="cuda")
            full.copy_counts(t)
            partials.append(t)
        full.unload()
        assert np.array_equal(sum(p.cpu() for p in partials).numpy().view(np.uint64).reshape(-1, 12, 2),
                              whole["counts"])
        for r in range(world):
            funcs = np.flatnonzero(owners == r)
            sub, m = shard.select_functions(a, funcs)
            idx = torch.as_tensor(m["instr"]).cuda()
            owned = sum(p.view(-1, 24).index_select(0, idx) for p in partials).reshape(-1).contiguous()
            prog = ctx.load_program(sub)
            try:
                prog.set_counts(owned, 0)
                prog.blame()
                adv = prog.advise()
                st, info = prog.status()
                assert st == 0, info
                cnt, bad = prog.counts()
                assert bad == 0 and np.array_equal(cnt.reshape(-1, 24), whole["counts"].reshape(-1, 24)[m["instr"]])
                assert np.array_equal(prog.blame_counts().reshape(-1, 24), whole["blame"].reshape(-1, 24)[m["instr"]])
                e = prog.edges()
                keep = np.isin(whole["edges"]["j"], m["instr"])
                assert np.array_equal(m["instr"][e["j"]], whole["edges"]["j"][keep])
                assert np.array_equal(m["instr"][e["i"]], whole["edges"]["i"][keep])
                assert np.array_equal(e["share"], whole["edges"]["share"][keep])
                for k in ("totals", "matched", "speedup", "rank", "n_hot", "hot"):
                    assert np.array_equal(adv[k], whole["advice"][k][funcs]), k
                assert np.array_equal(adv["loop_speedup"], whole["advice"]["loop_speedup"][m["loop"]])
            finally:
                prog.unload()
        # one rank (no exchange): the sharded step's own path equals the whole batch
        step = shard.ShardedStep(ctx, a, 0, 1)
        try:
            owned = step.step(_dev(s))
            assert np.array_equal(owned.cpu().numpy().view(np.uint64).reshape(-1, 12, 2), whole["counts"])
            adv = step.mine.get_advice()
            assert_advice_equal(adv, R)
        finally:
            step.close()


def test_set_counts_refuses_bad_buffers():
    import torch
    import paper_2009_04061_gb300 as g
    ps, _, kz = synth.workload("plain")
    P = synth.make_program(ps, kz)
    with g.Context(ARCH) as ctx:
        prog = ctx.load_program(P)
        try:
            for bad in (np.zeros(P.n_instr * 24, np.int64), torch.zeros(P.n_instr * 24 - 1, dtype=torch.int64,
                                                                        device="cuda"),
                        torch.zeros(P.n_instr * 24, dtype=torch.int32, device="cuda")):
                with pytest.raises(ValueError):
                    prog.set_counts(bad)
                with pytest.raises(ValueError):
                    prog.copy_counts(bad)
            lib = g.library()
            assert lib.gpa_set_counts(ctx.handle, prog.pid, None, 0, None) == -1
            assert lib.gpa_copy_counts(ctx.handle, prog.pid, None, None) == -1
        finally:
            prog.unload()

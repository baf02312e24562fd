"""Sharding one batch over ranks (function ownership + one exchange of counts),
on CPU ranks over gloo: each rank counts its even chunk of the samples with the
oracle, the owners receive their functions' summed count rows in the one
exchange, analyze the functions they own, and the merged results equal the
oracle's analysis of the whole batch. Also the planner's own properties."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2009_04061_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARCH = synth.default_arch()
N_SAMPLES = 400_000


def _program():
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps, kz)
    return P, synth.add_calls(P, 0.3, seed=2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P, a = _program()
    owners = shard.lpt_owners(shard.function_costs(a), world)
    lo, hi = shard.sample_range(N_SAMPLES, rank, world)
    chunk = P.samples(hi - lo, seed=5, n0=lo, total=N_SAMPLES)
    partial, _ = oracle.histogram(a, chunk)                   # this rank's counts of the whole program
    owned = shard.exchange_counts(torch.from_numpy(partial.reshape(-1).view(np.int64)), owners, a, rank, world)
    funcs = np.flatnonzero(owners == rank)
    sub, maps = shard.select_functions(a, funcs)
    R = oracle.analyze(sub, ARCH, owned.numpy().view(np.uint64))
    e = R["edges"]
    res = dict(funcs=funcs, instr=maps["instr"], loop=maps["loop"], blame=R["blame"].reshape(-1, 24),
               ej=maps["instr"][e["j"]], ei=maps["instr"][e["i"]], share=e["share"], dmin=e["dmin"],
               speedup=R["speedup"], M=R["M"], rank=R["rank"], hot=R["hot"], totals=R["totals"],
               loop_A=R["loop_A"], loop_S=R["loop_S"], line_stall=R["line_stall"])
    got = [None] * world
    dist.all_gather_object(got, res)
    if rank == 0:
        out["parts"] = got
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sharded_batch_equals_oracle():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        parts = out["parts"]
    P, a = _program()
    cnt, _ = oracle.histogram(a, P.samples(N_SAMPLES, seed=5))
    R = oracle.analyze(a, ARCH, cnt)
    seen = np.zeros(P.n_functions, int)
    blame = np.zeros((P.n_instr, 24), np.uint64)
    edges = []
    line_stall = np.zeros_like(R["line_stall"])
    for p in parts:
        seen[p["funcs"]] += 1
        blame[p["instr"]] = p["blame"]
        for k in ("speedup", "M", "rank", "totals"):
            assert np.array_equal(p[k], R[k][p["funcs"]]), k
        assert np.array_equal(p["hot"], R["hot"][p["funcs"]])
        assert np.array_equal(p["loop_A"], R["loop_A"][p["loop"]]) and np.array_equal(p["loop_S"], R["loop_S"][p["loop"]])
        edges += list(zip(p["ej"], p["ei"], p["dmin"], map(tuple, p["share"].reshape(-1, 8))))
        line_stall += p["line_stall"]
    assert (seen == 1).all()                                   # every function has exactly one owner
    assert np.array_equal(blame, R["blame"].reshape(-1, 24))
    e = R["edges"]
    want = list(zip(e["j"], e["i"], e["dmin"], map(tuple, e["share"].reshape(-1, 8))))
    assert sorted(edges) == sorted(want)
    assert np.array_equal(line_stall, R["line_stall"])
    assert len(parts[0]["funcs"]) > 0 and len(parts[1]["funcs"]) > 0


def test_lpt_owners_balance_and_determinism():
    """LPT by hand: costs 7, 5, 4, 3, 3 on two ranks go 7 -> 0, 5 -> 1, 4 -> 1, 3 -> 0, 3 -> 1
    (loads 10 and 12); and on the batched workload's sizes the most loaded of 8 ranks
    stays within 4/3 of the mean plus one function."""
    assert shard.lpt_owners([7, 5, 4, 3, 3], 2).tolist() == [0, 1, 1, 0, 1]
    assert shard.lpt_owners([1, 1, 1], 1).tolist() == [0, 0, 0]
    ps, _, _ = synth.workload("batched")
    costs = np.array([p["n_instr"] for p in ps])
    for world in (2, 3, 8):
        own = shard.lpt_owners(costs, world)
        load = np.bincount(own, weights=costs, minlength=world)
        assert load.max() <= 4 / 3 * costs.sum() / world + costs.max()
        assert np.array_equal(own, shard.lpt_owners(costs, world))
    with pytest.raises(ValueError):
        shard.lpt_owners([1], 0)


def test_sample_ranges_cover_the_stream():
    for n, world in ((10, 3), (0, 2), (7, 8), (1_000_003, 4)):
        r = [shard.sample_range(n, k, world) for k in range(world)]
        assert r[0][0] == 0 and r[-1][1] == n and all(r[k][1] == r[k + 1][0] for k in range(world - 1))
        assert max(h - l for l, h in r) - min(h - l for l, h in r) <= 1


def test_selected_functions_analyze_like_the_whole():
    """Any selection of functions, cut out with its call relations kept (calls to and
    from functions outside it become -1), gives the oracle the whole program's results
    for those functions; the loop nests are the natural loops."""
    P, a = _program()
    cnt, _ = oracle.histogram(a, P.samples(300_000, seed=1))
    R = oracle.analyze(a, ARCH, cnt)
    for funcs in ([0], [3, 7, 11], list(range(0, 20, 2)), list(range(20))):
        sub, m = shard.select_functions(a, funcs)
        assert all(oracle.check_loops(sub, f) == 0 for f in range(sub["n_functions"]))
        Rs = oracle.analyze(sub, ARCH, cnt.reshape(-1, 24)[m["instr"]])
        assert np.array_equal(Rs["blame"].reshape(-1, 24), R["blame"].reshape(-1, 24)[m["instr"]])
        for k in ("speedup", "M", "rank", "hot", "totals"):
            assert np.array_equal(Rs[k], R[k][m["func"]]), (funcs, k)
        assert np.array_equal(Rs["loop_S"], R["loop_S"][m["loop"]])

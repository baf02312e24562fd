"""Serving: sessions admitted while others run on the device give the same
results as each session run alone and as the oracle on that session
(bit-exact counts, edges and blame; advice bit-exact, speedups within 1e-12)."""
import numpy as np
import pytest

import synth
from parity import ARCH, assert_advice_equal, assert_edges_equal, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _sessions(n, seed=0):
    from paper_2009_04061_gb300.serving import Session
    import torch
    out = []
    for s, d in enumerate(synth.serving_sessions(n, seed=seed, max_functions=12)):
        P = synth.make_program(d["params"], 1.0, d["seed"])
        ns = min(d["n_samples"], 400_000)
        host = torch.empty(ns, dtype=torch.int64).pin_memory()
        P.samples(ns, seed=d["seed"], out=host.numpy().view(np.uint64))
        out.append((P, Session(s, P.arrays, host.numpy().view(np.uint64))))
    return out


def test_sessions_same_alone_and_in_the_mix():
    import paper_2009_04061_gb300 as g
    from paper_2009_04061_gb300.serving import Server, serve
    import torch
    items = _sessions(7)
    srv = Server(ARCH, slots=3, budget_bytes=8 << 30, keep_results=True)
    try:
        res = serve(srv, [s for _, s in items], [0.0] * len(items))
    finally:
        srv.close()
    assert sorted(r.sid for r in res) == list(range(len(items)))
    # the slots overlapped: some session was admitted before another finished
    spans = sorted((r.t_admit, r.t_done) for r in res)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    ctx = g.Context(ARCH)
    try:
        for r in res:
            P, s = items[r.sid]
            alone = gpu_run(ctx, P, torch.from_numpy(s.samples.view(np.int64)).cuda())
            assert np.array_equal(alone["counts"], r.counts)
            assert np.array_equal(alone["blame"], r.blame)
            for k in alone["advice"]:
                assert np.array_equal(alone["advice"][k], r.advice[k]), (r.sid, k)
            # and the oracle on the same session
            R = oracle_run(P, s.samples)
            assert np.array_equal(r.counts, R["counts"]), r.sid
            assert_edges_equal(r.edges, R["edges"])
            assert np.array_equal(r.blame, R["blame"]), r.sid
            assert_advice_equal(r.advice, R)
            assert np.array_equal(r.advice["line_stall"], R["line_stall"])
            assert np.array_equal(r.advice["line_latency"], R["line_lat"])
    finally:
        ctx.close()


def test_budget_limits_admission():
    """At every admission the programs in flight fit the budget, and the
    largest session alone fills it."""
    from paper_2009_04061_gb300.serving import Server, serve
    items = _sessions(4, seed=1)
    probe = Server(ARCH, slots=1, budget_bytes=1 << 40)
    need = max(probe.slots[0].ctx.footprint(s.program) for _, s in items)
    probe.close()
    srv = Server(ARCH, slots=4, budget_bytes=need)
    try:
        res = serve(srv, [s for _, s in items], [0.0] * len(items))
    finally:
        srv.close()
    assert len(res) == len(items)
    for r in res:
        held = sum(q.device_bytes for q in res if q.t_admit <= r.t_admit < q.t_done)
        assert held <= need
    big = max(res, key=lambda q: q.device_bytes)
    assert not any(q is not big and q.t_admit < big.t_done and big.t_admit < q.t_done for q in res)


def test_footprint_equals_loaded_bytes():
    import paper_2009_04061_gb300 as g
    ctx = g.Context(ARCH)
    try:
        for P, s in _sessions(3, seed=2):
            f = ctx.footprint(s.program)
            prog = ctx.load_program(s.program)
            assert prog.device_bytes() == f > 0
            prog.unload()
    finally:
        ctx.close()

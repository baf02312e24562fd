"""The large-kernel stress workload against the oracle, in the parts the oracle
can finish: one function of 200,000 instructions (28,280 blocks, 40 loops
nested up to 4 deep, 255 registers, 30% global loads) and the first
64M-sample chunk of its 1e9-sample stream, ingested from pinned host memory.

- counts: the oracle's histogram of the whole chunk, element by element;
- reaching definitions: RIN/ROUT of every block (a function this large runs
  the windowed global-memory fixpoint) against the oracle's worklist;
- edges: for a seeded sample of stalled uses plus the uses of the largest
  searches, every surviving edge with its distances, flags and Eq. 1 shares
  against the oracle's analysis of those uses;
- blame: conserved per stall class and latency flag over the whole function.
The oracle runs on host threads while the GPU works."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import synth
from parity import ARCH, assert_edges_equal

pytestmark = pytest.mark.gpu

CHUNK = 1 << 26
N_PICK = 96


def test_large_kernel_chunk_against_oracle():
    import torch
    import paper_2009_04061_gb300 as g
    ps, n_total, kz = synth.workload("large")
    P = synth.make_program(ps, kz)
    host = torch.empty(CHUNK, dtype=torch.int64).pin_memory()
    s = P.samples(CHUNK, total=n_total, out=host.numpy().view(np.uint64))
    pool = ThreadPoolExecutor(16)
    f_hist = pool.submit(oracle.histogram, P, s)
    f_reach = pool.submit(oracle.reaching, P)
    try:
        with g.Context(ARCH) as ctx:
            prog = ctx.load_program(P)
            try:
                prog.reset()
                prog.ingest_host(host)
                prog.blame()
                adv = prog.advise()
                st, info = prog.status()
                assert st == 0, info
                cnt, bad = prog.counts()
                rin, rout = prog.reaching()
                blame = prog.blame_counts()
                edges = prog.edges()
            finally:
                prog.unload()
        ocnt, obad = f_hist.result()
        assert bad == obad and np.array_equal(cnt, ocnt)
        assert int(cnt.sum()) + bad == CHUNK
        assert np.array_equal(blame.sum(0), cnt.sum(0))            # conservation per class and flag
        T = int(cnt.sum())
        assert int(adv["totals"][0][0]) == T and int(adv["totals"][0][1]) == int(cnt[:, :, 0].sum())
        # a seeded sample of the stalled uses, and the use of the largest search
        stalled = np.flatnonzero(ocnt[:, [2, 3, 5, 6]].sum((1, 2)) > 0)
        pick = np.random.default_rng(4).choice(stalled, N_PICK, replace=False)
        print(f"largest search: use {info['largest_use']} resource {info['largest_resource']} "
              f"nodes {info['max_nodes']}")
        pick = np.unique(pick)
        parts = [x for x in np.array_split(pick, 16) if x.size]
        want = list(pool.map(lambda u: oracle.edges_of_uses(P, ARCH, ocnt, u), parts))
        oe = {k: np.concatenate([w[k] for w in want]) for k in want[0]}
        keep = np.isin(edges["j"], pick)
        ge = {k: v[keep] for k, v in edges.items()}
        assert len(oe["j"]) > 0
        assert_edges_equal(ge, oe)
        orin, orout = f_reach.result()
        assert np.array_equal(rin, orin) and np.array_equal(rout, orout)
    finally:
        pool.shutdown(wait=True, cancel_futures=True)

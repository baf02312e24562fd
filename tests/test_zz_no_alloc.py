"""The allocation-free scan (gpa_exclusive_scan_noalloc) against the scan the
library runs inside gpa_blame, whose result shows in gpa_get_edges: edges are
stored by use, so the first edge of each use sits at the exclusive prefix sum
of the per-use edge counts. Some callers cannot call cudaMalloc (inside
another framework's memory pool, in a profiler callback); this entry point
keeps its scratch in a fixed static device array instead. Collected last so a
failure here cannot hide the other tests."""
import numpy as np
import pytest

import synth
from parity import ARCH

pytestmark = pytest.mark.gpu


def _edge_offsets_from_library():
    import torch
    import paper_2009_04061_gb300 as g
    ps, _, kz = synth.workload("rodinia")
    P = synth.make_program(ps, kz)
    s = P.samples(1_000_000, seed=2)
    with g.Context(ARCH) as c:
        prog = c.load_program(P)
        prog.ingest(torch.from_numpy(s.view(np.int64)).cuda())
        prog.blame()
        e = prog.edges()
        prog.unload()
    counts = np.bincount(e["j"], minlength=P.n_instr).astype(np.int32)
    first = np.searchsorted(e["j"], np.arange(P.n_instr), side="left").astype(np.int32)
    return counts, first, len(e["j"])


def test_noalloc_scan_matches_library_scan_twice():
    import torch
    import paper_2009_04061_gb300 as g
    counts, first, total = _edge_offsets_from_library()
    assert total > 0
    out_total = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):  # two calls in a row share the static scratch
        buf = torch.from_numpy(counts.copy()).cuda()
        g.gpa_exclusive_scan_noalloc(buf, out_total)
        torch.cuda.synchronize()
        assert np.array_equal(buf.cpu().numpy(), first)
        assert int(out_total.item()) == total


def test_noalloc_scan_sizes_and_limit():
    import torch
    import paper_2009_04061_gb300 as g
    rng = np.random.default_rng(0)
    t = torch.zeros(1, dtype=torch.int32, device="cuda")
    for n in (0, 1, 4095, 4096, 4097, 3 * 4096 + 17, 1 << 20):
        x = rng.integers(0, 50, n).astype(np.int32)
        d = torch.from_numpy(x).cuda()
        g.gpa_exclusive_scan_noalloc(d, t)
        torch.cuda.synchronize()
        want = np.concatenate([[0], np.cumsum(x)[:-1]]).astype(np.int32) if n else x
        assert np.array_equal(d.cpu().numpy(), want) and int(t.item()) == int(x.sum())
    # the library's own limit, called through the C ABI directly: refused before any launch
    lib = g.library()
    assert lib.gpa_exclusive_scan_noalloc(g.gpa._p(t), (1 << 24) + 1, g.gpa._p(t), None) == -5
    assert lib.gpa_exclusive_scan_noalloc(g.gpa._p(t), -1, g.gpa._p(t), None) == -1


def test_noalloc_scan_binding_refuses_bad_arguments():
    """The binding checks what the C ABI cannot: a host array, another dtype, a
    non-contiguous view, an empty total, or n past the tensor's elements never reach
    the library (they would be read and written on the device as int32 data)."""
    import torch
    import paper_2009_04061_gb300 as g
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    tot = torch.zeros(1, dtype=torch.int32, device="cuda")
    bad = [(np.zeros(64, np.int32), tot, None), (buf.to(torch.int64), tot, None), (buf, tot.to(torch.int64), None),
           (buf.cpu(), tot, None), (buf[::2], tot, None), (buf, tot[:0], None), (buf, tot, 65), (buf, tot, -1)]
    for b, t, n in bad:
        with pytest.raises(ValueError):
            g.gpa_exclusive_scan_noalloc(b, t, n=n)
    g.gpa_exclusive_scan_noalloc(buf, tot, n=64)

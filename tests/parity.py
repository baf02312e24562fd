"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs, and compare element by element."""
import numpy as np

import oracle
import synth

ARCH = synth.default_arch()
# FP64 speedups are ratios of integers computed in one correctly rounded
# division on both sides; anything beyond 1e-12 relative is a real mismatch.
RTOL = 1e-12


def gpu_run(ctx, prog, samples_dev, stream=None, host=None, advise=True, graph_launches=0):
    """Load, ingest (device tensor, or host array if `host`), blame, advise; returns a dict of results.
    With graph_launches > 0 the step is captured as a CUDA graph and launched that many times instead."""
    P = ctx.load_program(prog)
    try:
        if graph_launches:
            P.capture_step(samples_dev)
            for _ in range(graph_launches):
                P.launch_step(stream)
            adv = P.get_advice(stream)
        else:
            P.reset(stream)
            if host is not None:
                P.ingest_host(host, stream=stream)
            elif samples_dev is not None and samples_dev.numel():
                P.ingest(samples_dev, stream=stream)
            P.blame(stream)
            adv = P.advise(fetch=True, stream=stream) if advise else None
        st, info = P.status(stream)
        cnt, bad = P.counts(stream)
        rin, rout = P.reaching(stream)
        out = dict(status=st, info=info, counts=cnt, invalid=bad, rin=rin, rout=rout, blame=P.blame_counts(stream),
                   edges=P.edges(stream), advice=adv)
    finally:
        P.unload()
    return out


def oracle_run(prog, samples, f_lo=0, f_hi=None, counts=None):
    cnt, bad = (counts, None) if counts is not None else oracle.histogram(prog, samples)
    R = oracle.analyze(prog, ARCH, cnt, f_lo, f_hi)
    rin, rout = oracle.reaching(prog, f_lo, f_hi)
    R.update(counts=cnt, invalid=bad, rin=rin, rout=rout)
    return R


def assert_edges_equal(ge, oe, j_lo=None, j_hi=None):
    if j_lo is not None:
        m = (ge["j"] >= j_lo) & (ge["j"] < j_hi)
        ge = {k: v[m] for k, v in ge.items()}
    for k in ("j", "i", "dmin", "dlong", "flags"):
        assert np.array_equal(ge[k], oe[k]), (k, _first_diff(ge, oe))
    assert np.array_equal(ge["share"], oe["share"]), _first_diff(ge, oe)


def _first_diff(ge, oe):
    n = min(len(ge["j"]), len(oe["j"]))
    for t in range(n):
        a = tuple(int(ge[k][t]) for k in ("j", "i", "dmin", "dlong", "flags"))
        b = tuple(int(oe[k][t]) for k in ("j", "i", "dmin", "dlong", "flags"))
        if a != b or not np.array_equal(ge["share"][t], oe["share"][t]):
            return dict(t=t, gpu=a, oracle=b, gshare=ge["share"][t].tolist(), oshare=oe["share"][t].tolist())
    return dict(n_gpu=len(ge["j"]), n_oracle=len(oe["j"]))


def assert_advice_equal(ga, R, f_lo=0, f_hi=None, l_lo=0, l_hi=None):
    f_hi = ga["totals"].shape[0] if f_hi is None else f_hi
    sl = slice(f_lo, f_hi)
    assert np.array_equal(ga["totals"][sl], R["totals"])
    assert np.array_equal(ga["matched"][sl], R["M"])
    assert np.allclose(ga["speedup"][sl], R["speedup"], rtol=RTOL, atol=0)
    assert np.array_equal(ga["rank"][sl], R["rank"])
    assert np.array_equal(ga["n_hot"][sl], R["n_hot"])
    assert np.array_equal(ga["hot"][sl], R["hot"])
    l_hi = ga["loop_active"].size if l_hi is None else l_hi
    assert np.array_equal(ga["loop_active"][l_lo:l_hi], R["loop_A"])
    assert np.array_equal(ga["loop_matched"][l_lo:l_hi], R["loop_ML"])
    assert np.allclose(ga["loop_speedup"][l_lo:l_hi], R["loop_S"], rtol=RTOL, atol=0)


def assert_full_parity(g, R, samples_n=None):
    assert g["status"] == 0, g
    assert np.array_equal(g["counts"], R["counts"])
    if R.get("invalid") is not None:
        assert g["invalid"] == R["invalid"]
    assert np.array_equal(g["rin"], R["rin"]) and np.array_equal(g["rout"], R["rout"])
    assert_edges_equal(g["edges"], R["edges"])
    assert np.array_equal(g["blame"], R["blame"])
    assert_advice_equal(g["advice"], R)
    assert np.array_equal(g["advice"]["line_stall"], R["line_stall"])
    assert np.array_equal(g["advice"]["line_latency"], R["line_lat"])

"""The seeded input generator: counter-based slices and launch-ordered streams.

The generator holds none of the analysis arithmetic; these tests pin the
properties the parity tests and the benchmark rely on."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def prog():
    params, _, kz = synth.workload("rodinia", 0)
    return synth.make_program(params, kz, 0)


def kernels_of(s):
    return (s >> np.uint64(48)).astype(np.int64)


@pytest.mark.parametrize("order", ["launch", "interleaved"])
def test_slices_regenerate_the_stream(prog, order):
    n = 300_001
    full = prog.samples(n, seed=3, order=order)
    a = prog.samples(123_457, seed=3, total=n, order=order)
    b = prog.samples(n - 123_457, seed=3, n0=123_457, total=n, order=order)
    assert np.array_equal(full, np.concatenate([a, b]))


def test_launch_runs_are_kernel_contiguous(prog):
    n = 1_000_000
    starts, kern = prog.launch_runs(n, seed=1)
    assert starts[0] == 0 and starts[-1] == n and np.all(np.diff(starts) > 0)
    s = prog.samples(n, seed=1)
    k = kernels_of(s)
    for r in range(len(kern)):
        assert np.all(k[starts[r]:starts[r + 1]] == kern[r])
    # each kernel gets 1-8 launches, and its share follows the kernel weights
    per = np.bincount(kern, minlength=prog.n_functions)
    assert per.max() <= 8 and per.min() >= 1


def test_launch_shares_match_interleaved_in_expectation(prog):
    n = 2_000_000
    a = np.bincount(kernels_of(prog.samples(n, seed=2)), minlength=prog.n_functions) / n
    b = np.bincount(kernels_of(prog.samples(n, seed=2, order="interleaved")), minlength=prog.n_functions) / n
    assert np.abs(a - b).max() < 0.01


def test_single_kernel_orders_agree():
    params, ns, kz = synth.workload("plain", 0)
    P = synth.make_program(params, kz, 0)
    assert np.array_equal(P.samples(ns), P.samples(ns, order="interleaved"))


def test_subprogram_matches_the_batch():
    """A function cut out of a batch (indices rebased) with its own samples
    gives the oracle the same blame and edges as inside the batch."""
    import oracle
    params, ns, kz = synth.workload("rodinia", 0)
    P = synth.make_program(params, kz, 0)
    s = P.samples(ns // 4)
    arch = synth.default_arch()
    cnt, _ = oracle.histogram(P, s)
    for f in (0, 7):
        R = oracle.analyze(P, arch, cnt, f, f + 1)
        sub = synth.subprogram(P.arrays, f, f + 1)
        c_f, bad = oracle.histogram(sub, synth.rebase_samples(s, f, f + 1))
        assert bad == 0
        R_f = oracle.analyze(sub, arch, c_f)
        i0 = int(P.func_instr_off[f])
        assert np.array_equal(R["blame"], R_f["blame"])
        assert np.array_equal(R["edges"]["j"] - i0, R_f["edges"]["j"])
        assert np.array_equal(R["edges"]["i"] - i0, R_f["edges"]["i"])
        assert np.array_equal(R["edges"]["share"], R_f["edges"]["share"])
        assert np.array_equal(R["speedup"], R_f["speedup"])


def test_launch_stats_seeded_and_in_range():
    """Launch statistics are a pure function of (count, seed), stay within the ABI's
    ranges, and include grids smaller than a GPU and launches where the per-SM block
    cap binds (both parallel optimizers can match)."""
    a, b = synth.launch_stats(500, seed=3), synth.launch_stats(500, seed=3)
    c = synth.launch_stats(500, seed=4)
    assert all(np.array_equal(a[k], b[k]) for k in a)
    assert any(not np.array_equal(a[k], c[k]) for k in a)
    assert a["blocks"].min() >= 1 and a["blocks"].max() <= 2 ** 17
    assert a["threads_per_block"].min() >= 1 and a["threads_per_block"].max() <= 1024
    assert a["regs_per_thread"].min() >= 0 and a["regs_per_thread"].max() <= 255
    assert a["smem_per_block"].min() >= 0
    assert (a["blocks"] < 152).mean() > 0.2 and (a["threads_per_block"] <= 32).mean() > 0.1

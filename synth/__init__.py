"""Seeded synthetic inputs for the GPA stall-blame path.

Programs are SASS-like control-flow graphs whose instructions carry the
fields of Table 1 that matter for dependency analysis (opcode class, guard
predicate, destination and source operands, write/read barrier and wait mask;
Sec. 2.2) and packed PC samples shaped like Sec. 2.1's sampling model. The
generator itself is C++ (synth.cpp, built into libgpa_synth.so beside this
file). This module holds no analysis arithmetic: it is the one input module
that both the CPU oracle and the CUDA path are fed from.

Data format shared by everything downstream (all arrays global over the
program's functions, functions laid out one after another):

* resources: 0..254 = R0..R254, 255..261 = P0..P6, 262..267 = B0..B5.
* def entries (uint16): resource | kind << 12, kind 1 = write barrier,
  2 = read barrier (only for B resources), 0 otherwise.
* guard literal (uint8): 0 = none ("_"), 1+i = Pi, 8+i = !Pi.
* blocks are numbered so that every edge u->v with v > u is a forward edge
  and every edge with v <= u goes to the header of a loop containing u.
* packed sample (uint64): kernel 16b | pc 24b | class 4b | latency 1b |
  sm 8b | 11 reserved zero bits (most significant first).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgpa_synth.so")

# ---------------------------------------------------------------- constants
N_RES = 268
R_BASE, P_BASE, B_BASE = 0, 255, 262
KIND_WRITE, KIND_READ = 1, 2

OPS = ["IADD", "IMAD", "FFMA", "ISETP", "MOV", "BRA", "BAR", "MEMBAR", "LDG", "STG",
       "LDS", "STS", "LDL", "STL", "LDC", "ATOM", "F2F", "MUFU", "DFMA", "EXIT", "CALL"]
OP = {n: i for i, n in enumerate(OPS)}

# Stall reasons (modelled on the public CUPTI PC-sampling reason list, Sec. 4).
CLASSES = ["SELECTED", "INST_FETCH", "EXEC_DEPENDENCY", "MEMORY_DEPENDENCY", "TEXTURE",
           "SYNC", "CONSTANT_MEMORY_DEPENDENCY", "PIPE_BUSY", "MEMORY_THROTTLE",
           "NOT_SELECTED", "OTHER", "SLEEPING"]
N_CLASSES = 12

# Opcode-class property bits of the architecture table.
F_MEM, F_SYNC, F_GLOBAL, F_LOCAL, F_CONST, F_SHARED, F_LONG_ARITH, F_VARLAT = (
    1, 2, 4, 8, 16, 32, 64, 128)


def default_arch():
    """Latency (instructions) and property bits per opcode class.

    The paper prints no latency values (Sec. 4, "Instruction latency based
    pruning" takes microbenchmarked fixed latencies and upper bounds for
    variable-latency memory operations); these are stand-ins of that shape. A
    call's results are ready when the callee returns: the same upper bound as
    a global load.
    """
    lat = {"IADD": 4, "IMAD": 5, "FFMA": 4, "ISETP": 4, "MOV": 2, "BRA": 0, "BAR": 32,
           "MEMBAR": 32, "LDG": 1024, "STG": 1024, "LDS": 32, "STS": 32, "LDL": 1024,
           "STL": 1024, "LDC": 64, "ATOM": 1024, "F2F": 16, "MUFU": 16, "DFMA": 8, "EXIT": 0,
           "CALL": 1024}
    flags = {"BAR": F_SYNC, "MEMBAR": F_SYNC,
             "LDG": F_MEM | F_GLOBAL | F_VARLAT, "STG": F_MEM | F_GLOBAL | F_VARLAT,
             "ATOM": F_MEM | F_GLOBAL | F_VARLAT,
             "LDL": F_MEM | F_LOCAL | F_VARLAT, "STL": F_MEM | F_LOCAL | F_VARLAT,
             "LDC": F_MEM | F_CONST | F_VARLAT,
             "LDS": F_SHARED | F_VARLAT, "STS": F_SHARED | F_VARLAT,
             "F2F": F_LONG_ARITH | F_VARLAT, "MUFU": F_LONG_ARITH | F_VARLAT}
    latency = np.array([lat[o] for o in OPS], dtype=np.int32)
    fl = np.array([flags.get(o, 0) for o in OPS], dtype=np.uint32)
    return latency, fl


# ---------------------------------------------------------------- library
def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "synth.cpp")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", _LIB_PATH, src,
                               "-lpthread"])
    return _LIB_PATH


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_program_new.restype = ctypes.c_void_p
        lib.synth_program_new.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_double,
                                          ctypes.c_uint64, ctypes.c_int32]
        lib.synth_program_free.argtypes = [ctypes.c_void_p]
        lib.synth_program_sizes.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_program_copy.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 19
        lib.synth_samples.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_int32]
        lib.synth_launch_runs.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64]
        lib.synth_launch_runs.restype = ctypes.c_int64
        _lib = lib
    return _lib


class _FnParams(ctypes.Structure):
    _fields_ = [("n_instr", ctypes.c_int32), ("n_loops", ctypes.c_int32), ("max_depth", ctypes.c_int32),
                ("n_regs", ctypes.c_int32), ("ldg_pct", ctypes.c_int32), ("tmpl", ctypes.c_int32),
                ("guard_pct", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("zipf_s", ctypes.c_double), ("seed", ctypes.c_uint64)]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Program:
    """A generated program: flat arrays plus the generator handle for sampling."""
    arrays: dict
    handle: object = field(repr=False, default=None)

    def __getattr__(self, k):
        a = self.__dict__.get("arrays")
        if a is not None and k in a:
            return a[k]
        raise AttributeError(k)

    @property
    def n_functions(self):
        return int(self.arrays["n_functions"])

    @property
    def n_instr(self):
        return int(self.arrays["n_instr"])

    @property
    def n_blocks(self):
        return int(self.arrays["n_blocks"])

    @property
    def n_loops(self):
        return int(self.arrays["n_loops"])

    def samples(self, n: int, seed: int = 0, n0: int = 0, invalid_ppm: int = 0, threads: int = 0,
                out: np.ndarray | None = None, total: int | None = None, order: str = "launch") -> np.ndarray:
        """Packed samples [n0, n0+n) of the stream `seed` (counter based).

        order "launch": the stream of `total` samples (default n0 + n) is a
        sequence of kernel-launch runs, each holding one kernel's samples, as a
        profiler that serializes kernels delivers them; see launch_runs().
        order "interleaved": every sample draws its kernel independently.
        """
        if out is None:
            out = np.empty(n, dtype=np.uint64)
        assert out.dtype == np.uint64 and out.size >= n and out.flags.c_contiguous
        tot = n0 + n if total is None else int(total)
        assert tot >= n0 + n, "slice beyond the end of the stream"
        if threads <= 0:
            threads = os.cpu_count() or 1
        if n:
            _L().synth_samples(self.handle, ctypes.c_uint64(seed), n0, n, _ptr(out), invalid_ppm, threads, tot,
                               {"interleaved": 0, "launch": 1}[order])
        return out

    def launch_runs(self, total: int, seed: int = 0):
        """(starts[n_runs + 1], kernels[n_runs]) of the launch-ordered stream of `total` samples."""
        nr = _L().synth_launch_runs(self.handle, ctypes.c_uint64(seed), total, None, None, 0)
        starts = np.zeros(nr + 1, np.int64)
        kernels = np.zeros(max(nr, 1), np.int32)[:nr]
        _L().synth_launch_runs(self.handle, ctypes.c_uint64(seed), total, _ptr(starts), _ptr(kernels), nr)
        return starts, kernels

    def __del__(self):
        h = self.__dict__.get("handle")
        if h and _lib is not None:
            _lib.synth_program_free(h)
            self.__dict__["handle"] = None


def make_program(params: list[dict], kernel_zipf_s: float = 1.0, kseed: int = 0, threads: int = 0) -> Program:
    """Generate one program of len(params) functions.

    Each dict: n_instr, n_loops, max_depth, n_regs, ldg_pct (0 = default mix),
    tmpl (1 = the fixed 200-instruction/12-block layout), guard_pct (percent of
    guarded instructions, default 10), zipf_s, seed.
    """
    nf = len(params)
    arr = (_FnParams * nf)()
    for i, p in enumerate(params):
        arr[i] = _FnParams(int(p["n_instr"]), int(p.get("n_loops", 0)), int(p.get("max_depth", 1)),
                           int(p.get("n_regs", 64)), int(p.get("ldg_pct", 0)), int(p.get("tmpl", 0)),
                           int(p.get("guard_pct", 10)), 0, float(p.get("zipf_s", 1.1)), int(p["seed"]) & (2**64 - 1))
    lib = _L()
    h = lib.synth_program_new(nf, ctypes.cast(arr, ctypes.c_void_p), kernel_zipf_s, ctypes.c_uint64(kseed),
                              threads or (os.cpu_count() or 1))
    sz = np.zeros(8, dtype=np.int64)
    lib.synth_program_sizes(h, _ptr(sz))
    nf_, ni, nb, nl, ne, nd, nu, nlines = (int(x) for x in sz)
    a = dict(
        func_instr_off=np.empty(nf + 1, np.int32), func_block_off=np.empty(nf + 1, np.int32),
        func_loop_off=np.empty(nf + 1, np.int32), func_line_off=np.empty(nf + 1, np.int32),
        block_instr_off=np.empty(nb + 1, np.int32), succ_off=np.empty(nb + 1, np.int32),
        succ=np.empty(max(ne, 1), np.int32)[:ne],
        opclass=np.empty(ni, np.uint8), guard=np.empty(ni, np.uint8), iflags=np.empty(ni, np.uint8),
        prof=np.empty(ni, np.uint8), line=np.empty(ni, np.int32),
        def_off=np.empty(ni + 1, np.int32), def_res=np.empty(max(nd, 1), np.uint16)[:nd],
        use_off=np.empty(ni + 1, np.int32), use_res=np.empty(max(nu, 1), np.uint16)[:nu],
        block_loop=np.empty(nb, np.int32), loop_parent=np.empty(max(nl, 1), np.int32)[:nl],
        loop_header=np.empty(max(nl, 1), np.int32)[:nl],
    )
    order = ["func_instr_off", "func_block_off", "func_loop_off", "func_line_off", "block_instr_off",
             "succ_off", "succ", "opclass", "guard", "iflags", "prof", "line", "def_off", "def_res",
             "use_off", "use_res", "block_loop", "loop_parent", "loop_header"]
    lib.synth_program_copy(h, *[_ptr(a[k]) for k in order])
    a.update(n_functions=nf_, n_instr=ni, n_blocks=nb, n_loops=nl, n_lines=nlines)
    return Program(a, h)


# ---------------------------------------------------------------- workloads
def _loguniform_int(rng, lo, hi, n):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n)).astype(np.int64)


def workload(name: str, seed: int = 0):
    """Function parameter lists and sample counts of the five workloads.

    plain      one function, 200 instructions in 12 blocks (one loop, one
               if/else), R0-R63; 1e5 samples, Zipf(1.1) hotness, x32 per loop level.
    rodinia    20 functions of 100-2,000 instructions (log-uniform), 1-4 nested
               loops, up to 128 registers; 1e7 samples over Zipf(1.0) kernel weights.
    batched    2,000 functions of 50-20,000 instructions (log-uniform), loop depth
               up to 5, up to 255 registers; 5e8 samples (4 GB).
    large      one function of 200,000 instructions, 40 loops nested up to 4,
               255 registers, 30% global loads; 1e9 samples in 64M-sample chunks.
    serving    sessions of 1-500 functions drawn as in `batched` with 1e5-1e7
               samples each (see `serving_sessions`).
    Returns (params, n_samples, kernel_zipf_s).
    """
    rng = np.random.default_rng(seed + 7919)
    if name == "plain":
        return [dict(n_instr=200, n_loops=1, max_depth=1, n_regs=64, tmpl=1, zipf_s=1.1, seed=seed)], 10**5, 1.0
    if name == "rodinia":
        sizes = _loguniform_int(rng, 100, 2000, 20)
        ps = []
        for f in range(20):
            nl = int(rng.integers(1, 5))
            ps.append(dict(n_instr=int(sizes[f]), n_loops=nl, max_depth=nl, n_regs=int(rng.integers(32, 129)),
                           zipf_s=1.1, seed=seed * 1000003 + f))
        return ps, 10**7, 1.0
    if name == "batched":
        return batched_params(2000, rng, seed), 5 * 10**8, 1.0
    if name == "large":
        return [dict(n_instr=200_000, n_loops=40, max_depth=4, n_regs=255, ldg_pct=30, zipf_s=1.1,
                     seed=seed)], 10**9, 1.0
    raise KeyError(name)


def batched_params(nf: int, rng, seed: int, base: int = 0):
    sizes = _loguniform_int(rng, 50, 20000, nf)
    ps = []
    for f in range(nf):
        n = int(sizes[f])
        nl = int(min(64, max(0, round(n / 400 + rng.uniform(-0.5, 1.5)))))
        ps.append(dict(n_instr=n, n_loops=nl, max_depth=5, n_regs=int(rng.integers(64, 256)), zipf_s=1.1,
                       seed=(seed * 1000003 + base + f) & (2**63 - 1)))
    return ps


def serving_sessions(n_sessions: int, seed: int = 0, rate_per_s: float = 200.0, max_functions: int = 500):
    """Session list for the serving workload: Poisson arrivals (seeded
    exponential gaps), log-uniform 1..max_functions functions and 1e5..1e7
    samples per session. Returns a list of dicts (t_arrival, params, n_samples, seed)."""
    rng = np.random.default_rng(seed + 104729)
    t = 0.0
    out = []
    for s in range(n_sessions):
        t += float(rng.exponential(1.0 / rate_per_s))
        nf = int(_loguniform_int(rng, 1, max_functions + 1, 1)[0])
        nf = max(1, min(max_functions, nf))
        ns = int(_loguniform_int(rng, 10**5, 10**7, 1)[0])
        out.append(dict(t_arrival=t, params=batched_params(nf, rng, seed, base=s * 1000), n_samples=ns,
                        seed=seed * 7777 + s))
    return out


# ---------------------------------------------------------------- launch statistics
def launch_stats(n_functions: int, seed: int = 0) -> dict:
    """Seeded launch statistics, one kernel launch per function (the inputs of
    the parallel optimizers): blocks log-uniform over 1..2^17 (some grids
    smaller than the GPU), threads per block from small (16, 32: the per-SM
    block cap binds) to 1,024, registers per thread 16..255, shared memory per
    block 0 for half of the kernels, else up to 96 KB."""
    rng = np.random.default_rng(seed + 15485863)
    blocks = np.maximum(1, _loguniform_int(rng, 1, 2 ** 17 + 1, n_functions))
    threads = rng.choice(np.array([16, 32, 32, 64, 96, 128, 192, 256, 256, 512, 640, 1024]), n_functions)
    regs = rng.integers(16, 256, n_functions)
    smem = np.where(rng.random(n_functions) < 0.5, 0, rng.integers(1, 96 * 1024 + 1, n_functions))
    return dict(blocks=blocks.astype(np.int64), threads_per_block=threads.astype(np.int32),
                regs_per_thread=regs.astype(np.int32), smem_per_block=smem.astype(np.int32))


# ---------------------------------------------------------------- slicing
def subprogram(arrays: dict, f_lo: int, f_hi: int) -> dict:
    """The arrays of functions [f_lo, f_hi) as a program of their own (all
    instruction, block, loop and line indices rebased to start at 0)."""
    a = arrays.arrays if hasattr(arrays, "arrays") else arrays
    fi, fb, fl, fn = (np.asarray(a[k]) for k in ("func_instr_off", "func_block_off", "func_loop_off",
                                                  "func_line_off"))
    i0, i1, b0, b1 = int(fi[f_lo]), int(fi[f_hi]), int(fb[f_lo]), int(fb[f_hi])
    l0, l1, n0, n1 = int(fl[f_lo]), int(fl[f_hi]), int(fn[f_lo]), int(fn[f_hi])
    so, do, uo = (np.asarray(a[k]) for k in ("succ_off", "def_off", "use_off"))
    s0, s1, d0, d1, u0, u1 = int(so[b0]), int(so[b1]), int(do[i0]), int(do[i1]), int(uo[i0]), int(uo[i1])

    def loops(x):
        x = np.asarray(x).astype(np.int32)
        return np.where(x >= 0, x - l0, -1).astype(np.int32)

    out = dict(
        func_instr_off=(fi[f_lo:f_hi + 1] - i0).astype(np.int32),
        func_block_off=(fb[f_lo:f_hi + 1] - b0).astype(np.int32),
        func_loop_off=(fl[f_lo:f_hi + 1] - l0).astype(np.int32),
        func_line_off=(fn[f_lo:f_hi + 1] - n0).astype(np.int32),
        block_instr_off=(np.asarray(a["block_instr_off"])[b0:b1 + 1] - i0).astype(np.int32),
        succ_off=(so[b0:b1 + 1] - s0).astype(np.int32),
        succ=(np.asarray(a["succ"])[s0:s1] - b0).astype(np.int32),
        def_off=(do[i0:i1 + 1] - d0).astype(np.int32), def_res=np.asarray(a["def_res"])[d0:d1].copy(),
        use_off=(uo[i0:i1 + 1] - u0).astype(np.int32), use_res=np.asarray(a["use_res"])[u0:u1].copy(),
        line=(np.asarray(a["line"])[i0:i1] - n0).astype(np.int32),
        block_loop=loops(np.asarray(a["block_loop"])[b0:b1]),
        loop_parent=loops(np.asarray(a["loop_parent"])[l0:l1]),
        loop_header=(np.asarray(a["loop_header"])[l0:l1] - b0).astype(np.int32),
        n_functions=f_hi - f_lo, n_instr=i1 - i0, n_blocks=b1 - b0, n_loops=l1 - l0, n_lines=n1 - n0,
    )
    for k in ("opclass", "guard", "iflags", "prof"):
        out[k] = np.asarray(a[k])[i0:i1].copy()
    # calls whose site and callee both lie in the range (a function whose callers
    # are all outside it is no longer a device function of the slice)
    cs, cc = np.asarray(a.get("call_site", [])), np.asarray(a.get("call_callee", []))
    keep = (cs >= i0) & (cs < i1) & (cc >= f_lo) & (cc < f_hi)
    out["call_site"] = (cs[keep] - i0).astype(np.int32)
    out["call_callee"] = (cc[keep] - f_lo).astype(np.int32)
    return out


def rebase_samples(samples: np.ndarray, f_lo: int, f_hi: int) -> np.ndarray:
    """The samples of kernels [f_lo, f_hi), their kernel field shifted down by f_lo."""
    s = np.asarray(samples, dtype=np.uint64)
    k = s >> np.uint64(48)
    keep = (k >= np.uint64(f_lo)) & (k < np.uint64(f_hi))
    return (s[keep] - (np.uint64(f_lo) << np.uint64(48))).astype(np.uint64)


# ---------------------------------------------------------------- calls (Function Inlining)
def add_calls(arrays, device_frac: float = 0.1, seed: int = 0, max_sites: int = 3) -> dict:
    """A copy of the program's arrays with a call table: a seeded `device_frac` of
    the functions become device functions, each called from 1..max_sites call
    sites in other functions. A call site is a MOV (one register in, one out)
    turned into a CALL: argument and result pass through those registers, so the
    dataflow is unchanged and only the opcode class (its latency) differs.
    Returns the arrays with call_site (ascending) and call_callee added."""
    a = dict(arrays.arrays if hasattr(arrays, "arrays") else arrays)
    nf = int(a["n_functions"])
    fio = np.asarray(a["func_instr_off"], dtype=np.int64)
    op = np.asarray(a["opclass"]).copy()
    rng = np.random.default_rng(seed + 2654435761)
    sites, callees = [], []
    if nf >= 2:
        n_dev = max(1, int(round(device_frac * nf)))
        devs = rng.choice(nf, size=min(n_dev, nf - 1), replace=False)
        movs = np.flatnonzero(op == OP["MOV"])
        taken = set()
        for d in devs:
            cands = movs[(movs < fio[d]) | (movs >= fio[d + 1])]
            cands = np.array([x for x in cands if int(x) not in taken], dtype=np.int64)
            if cands.size == 0:
                continue
            k = int(rng.integers(1, max_sites + 1))
            for x in rng.choice(cands, size=min(k, cands.size), replace=False):
                taken.add(int(x))
                sites.append(int(x))
                callees.append(int(d))
    order = np.argsort(np.asarray(sites, dtype=np.int64), kind="stable")
    cs = np.asarray(sites, dtype=np.int32)[order]
    cc = np.asarray(callees, dtype=np.int32)[order]
    op[cs] = OP["CALL"]
    a.update(opclass=op, call_site=cs, call_callee=cc)
    return a

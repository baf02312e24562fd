"""CPU oracle for the GPA stall-blame path — TEST INFRASTRUCTURE ONLY.

A thin ctypes binding over gpa_oracle.cpp (built into libgpa_oracle.so beside
this file), the plain, slow, literal restatement of the method that the CUDA
path is checked against. Only tests/, the package smoke check and bench.py's
CPU-baseline and reference legs may import this module; the product never
does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .parallel import parallel  # noqa: E402,F401  (Table 2 parallel optimizers, Eqs. 6-10)

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "libgpa_oracle.so")
N_OPT = 9
OPT_NAMES = ["REG_REUSE", "STRENGTH_RED", "FUNC_SPLIT", "FAST_MATH", "WARP_BALANCE", "MEM_TXN_RED",
             "LOOP_UNROLL", "CODE_REORDER", "FUNC_INLINE"]


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "gpa_oracle.cpp")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", _LIB, src])
    return _LIB


class _OProg(ctypes.Structure):
    _fields_ = [("nf", ctypes.c_int32), ("ni", ctypes.c_int32), ("nb", ctypes.c_int32), ("nl", ctypes.c_int32),
                ("n_lines", ctypes.c_int32)] + [(k, ctypes.c_void_p) for k in (
                    "func_instr_off", "func_block_off", "func_loop_off", "block_instr_off", "succ_off", "succ",
                    "opclass", "guard", "iflags", "line", "def_off", "def_res", "use_off", "use_res",
                    "block_loop", "loop_parent", "loop_header")] + [
                    ("n_calls", ctypes.c_int32), ("call_site", ctypes.c_void_p), ("call_callee", ctypes.c_void_p)]


class _OArch(ctypes.Structure):
    _fields_ = [("n_op", ctypes.c_int32), ("latency", ctypes.c_void_p), ("flags", ctypes.c_void_p)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.oracle_histogram.argtypes = [vp, vp, i64, vp, vp]
        lib.oracle_reaching.argtypes = [vp, i32, i32, vp, vp]
        lib.oracle_search.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, vp]
        lib.oracle_coverage.argtypes = [vp, vp, vp, i32, i32, vp]
        lib.oracle_check_loops.argtypes = [vp, i32]
        lib.oracle_analyze.argtypes = [vp, vp, vp, i32, i32]
        lib.oracle_analyze.restype = vp
        lib.oracle_edges_of_uses.argtypes = [vp, vp, vp, i32, vp]
        lib.oracle_edges_of_uses.restype = vp
        lib.oracle_n_edges.argtypes = [vp]
        lib.oracle_n_edges.restype = i64
        lib.oracle_get_edges.argtypes = [vp] * 7
        lib.oracle_get_blame.argtypes = [vp, vp]
        lib.oracle_get_advice.argtypes = [vp] * 12
        lib.oracle_free.argtypes = [vp]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Bound:
    """Keeps the arrays alive while the C struct points at them."""

    def __init__(self, prog: dict, arch=None):
        keep = {}

        def arr(k, dt):
            a = np.ascontiguousarray(prog.get(k, np.zeros(0, dt)), dtype=dt)
            if a.size == 0:
                a = np.zeros(1, dtype=dt)
            keep[k] = a
            return _p(a)

        self.s = _OProg(int(prog["n_functions"]), int(prog["n_instr"]), int(prog["n_blocks"]), int(prog["n_loops"]),
                        int(prog["n_lines"]),
                        arr("func_instr_off", np.int32), arr("func_block_off", np.int32),
                        arr("func_loop_off", np.int32), arr("block_instr_off", np.int32),
                        arr("succ_off", np.int32), arr("succ", np.int32), arr("opclass", np.uint8),
                        arr("guard", np.uint8), arr("iflags", np.uint8), arr("line", np.int32),
                        arr("def_off", np.int32), arr("def_res", np.uint16), arr("use_off", np.int32),
                        arr("use_res", np.uint16), arr("block_loop", np.int32), arr("loop_parent", np.int32),
                        arr("loop_header", np.int32), int(np.asarray(prog.get("call_site", [])).size),
                        arr("call_site", np.int32), arr("call_callee", np.int32))
        if arch is not None:
            lat = np.ascontiguousarray(arch[0], dtype=np.int32)
            fl = np.ascontiguousarray(arch[1], dtype=np.uint32)
            keep["lat"], keep["fl"] = lat, fl
            self.a = _OArch(lat.size, _p(lat), _p(fl))
        self.keep = keep

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _arrays(prog):
    return prog.arrays if hasattr(prog, "arrays") else prog


def histogram(prog, samples: np.ndarray):
    """Dense counts cnt[n_instr, 12, 2] (uint64) and the invalid-sample count."""
    prog = _arrays(prog)
    b = _Bound(prog)
    s = np.ascontiguousarray(samples, dtype=np.uint64)
    cnt = np.zeros(int(prog["n_instr"]) * 24, dtype=np.uint64)
    bad = np.zeros(1, dtype=np.uint64)
    _L().oracle_histogram(b.ref, _p(s) if s.size else None, s.size, _p(cnt), _p(bad))
    return cnt.reshape(-1, 12, 2), int(bad[0])


def reaching(prog, f_lo: int = 0, f_hi: int | None = None):
    """RIN, ROUT resource projections (uint32[n_blocks_in_range, 9])."""
    prog = _arrays(prog)
    f_hi = int(prog["n_functions"]) if f_hi is None else f_hi
    b = _Bound(prog)
    nb = int(prog["func_block_off"][f_hi] - prog["func_block_off"][f_lo])
    rin = np.zeros(nb * 9, dtype=np.uint32)
    rout = np.zeros(nb * 9, dtype=np.uint32)
    _L().oracle_reaching(b.ref, f_lo, f_hi, _p(rin), _p(rout))
    return rin.reshape(-1, 9), rout.reshape(-1, 9)


def coverage(prog, arch, cnt: np.ndarray, f_lo: int = 0, f_hi: int | None = None) -> tuple[int, int, int]:
    """Single dependency coverage (Sec. 6): (stalled uses, single-dependency uses before
    pruning, after pruning) over functions [f_lo, f_hi)."""
    prog = _arrays(prog)
    f_hi = int(prog["n_functions"]) if f_hi is None else f_hi
    b = _Bound(prog, arch)
    c = np.ascontiguousarray(cnt, dtype=np.uint64).reshape(-1)
    out = np.zeros(3, np.int64)
    _L().oracle_coverage(b.ref, ctypes.byref(b.a), _p(c), f_lo, f_hi, _p(out))
    return int(out[0]), int(out[1]), int(out[2])


def search(prog, j: int, r: int):
    """Immediate sources of global use j through resource r:
    list of dicts (i, dmin, K, dlong, dom) sorted by i."""
    prog = _arrays(prog)
    b = _Bound(prog)
    cap = 4096
    out = [np.zeros(cap, np.int32) for _ in range(4)] + [np.zeros(cap, np.uint8)]
    n = _L().oracle_search(b.ref, j, r, cap, *[_p(a) for a in out])
    assert n <= cap
    return [dict(i=int(out[0][t]), dmin=int(out[1][t]), K=int(out[2][t]), dlong=int(out[3][t]),
                 dom=bool(out[4][t])) for t in range(n)]


def check_loops(prog, f: int) -> int:
    prog = _arrays(prog)
    b = _Bound(prog)
    return int(_L().oracle_check_loops(b.ref, f))


def _read_edges(lib, h):
    ne = int(lib.oracle_n_edges(h))
    m = max(ne, 1)
    ej, ei, dmin, dlong = (np.zeros(m, np.int32) for _ in range(4))
    fl = np.zeros(m, np.uint32)
    share = np.zeros(m * 8, np.uint64)
    lib.oracle_get_edges(h, _p(ej), _p(ei), _p(dmin), _p(dlong), _p(fl), _p(share))
    return dict(j=ej[:ne], i=ei[:ne], dmin=dmin[:ne], dlong=dlong[:ne], flags=fl[:ne],
                share=share[:ne * 8].reshape(ne, 4, 2))


def edges_of_uses(prog, arch, cnt: np.ndarray, uses) -> dict:
    """Surviving merged edges with their Eq. 1 shares of the given uses only (global
    instruction indices): the rows of analyze()'s edges whose use is listed."""
    prog = _arrays(prog)
    b = _Bound(prog, arch)
    c = np.ascontiguousarray(cnt, dtype=np.uint64).reshape(-1)
    u = np.ascontiguousarray(np.unique(np.asarray(uses, dtype=np.int64)), dtype=np.int32)
    lib = _L()
    h = lib.oracle_edges_of_uses(b.ref, ctypes.byref(b.a), _p(c), int(u.size), _p(u) if u.size else None)
    try:
        return _read_edges(lib, h)
    finally:
        lib.oracle_free(h)


def analyze(prog, arch, cnt: np.ndarray, f_lo: int = 0, f_hi: int | None = None) -> dict:
    """Blame, surviving merged edges and advice for functions [f_lo, f_hi)."""
    prog = _arrays(prog)
    nf = int(prog["n_functions"])
    f_hi = nf if f_hi is None else f_hi
    b = _Bound(prog, arch)
    c = np.ascontiguousarray(cnt, dtype=np.uint64).reshape(-1)
    lib = _L()
    h = lib.oracle_analyze(b.ref, ctypes.byref(b.a), _p(c), f_lo, f_hi)
    try:
        edges = _read_edges(lib, h)
        i_lo, i_hi = int(prog["func_instr_off"][f_lo]), int(prog["func_instr_off"][f_hi])
        blame = np.zeros((i_hi - i_lo) * 24, np.uint64)
        lib.oracle_get_blame(h, _p(blame))
        nfr = f_hi - f_lo
        l_lo, l_hi = int(prog["func_loop_off"][f_lo]), int(prog["func_loop_off"][f_hi])
        nlines = int(prog["n_lines"])
        tot = np.zeros(nfr * 4, np.uint64)
        M = np.zeros(nfr * N_OPT, np.uint64)
        sp = np.zeros(nfr * N_OPT, np.float64)
        rank = np.zeros(nfr * N_OPT, np.int32)
        nhot = np.zeros(nfr * N_OPT, np.int32)
        hot = np.zeros(nfr * N_OPT * 5 * 6, np.int64)
        lA = np.zeros(max(l_hi - l_lo, 1), np.uint64)
        lML = np.zeros(max(l_hi - l_lo, 1), np.uint64)
        lS = np.zeros(max(l_hi - l_lo, 1), np.float64)
        ls = np.zeros(max(nlines, 1), np.uint64)
        ll = np.zeros(max(nlines, 1), np.uint64)
        lib.oracle_get_advice(h, _p(tot), _p(M), _p(sp), _p(rank), _p(nhot), _p(hot), _p(lA), _p(lML), _p(lS),
                              _p(ls), _p(ll))
    finally:
        lib.oracle_free(h)
    return dict(
        edges=edges,
        blame=blame.reshape(-1, 12, 2),
        totals=tot.reshape(nfr, 4), M=M.reshape(nfr, N_OPT), speedup=sp.reshape(nfr, N_OPT),
        rank=rank.reshape(nfr, N_OPT), n_hot=nhot.reshape(nfr, N_OPT), hot=hot.reshape(nfr, N_OPT, 5, 6),
        loop_A=lA[:l_hi - l_lo], loop_ML=lML[:l_hi - l_lo], loop_S=lS[:l_hi - l_lo],
        line_stall=ls[:nlines], line_lat=ll[:nlines],
    )

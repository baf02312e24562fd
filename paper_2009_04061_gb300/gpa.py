"""ctypes binding of libgpa.so (include/gpa.h), argument marshalling only.

Every step of the stall-blame path runs in the library's CUDA kernels; this
module converts numpy arrays and torch tensors into the pointers and sizes
the C ABI takes. Functions keep the C names (gpa_create, gpa_load_program,
gpa_ingest_samples, gpa_blame, gpa_advise, ...); Context and Program wrap
them for convenience. Importing fails loudly when libgpa.so is missing.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpa.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gpa.h")

GPA_OK = 0
STATUS = {0: "GPA_OK", -1: "GPA_ERR_INVALID_ARG", -2: "GPA_ERR_INVALID_PROGRAM", -3: "GPA_ERR_CUDA",
          -4: "GPA_ERR_NOT_CONVERGED", -5: "GPA_ERR_CAPACITY", -6: "GPA_ERR_TIMEOUT", -7: "GPA_ERR_NO_PROGRAM",
          -8: "GPA_ERR_OOM"}
NUM_OPT = 9
OPT_NAMES = ["REGISTER_REUSE", "STRENGTH_REDUCTION", "FUNCTION_SPLIT", "FAST_MATH", "WARP_BALANCE",
             "MEMORY_TRANSACTION_REDUCTION", "LOOP_UNROLLING", "CODE_REORDERING", "FUNCTION_INLINING"]


class GpaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class gpa_arch_desc(ctypes.Structure):
    _fields_ = [("n_opclasses", ctypes.c_int32), ("latency", ctypes.c_void_p), ("flags", ctypes.c_void_p)]


class gpa_options(ctypes.Structure):
    _fields_ = [("max_fixpoint_sweeps", ctypes.c_int32), ("max_search_nodes", ctypes.c_int32),
                ("search_slots", ctypes.c_int32), ("max_sources_per_use", ctypes.c_int32),
                ("small_search_nodes", ctypes.c_int32), ("mid_search_nodes", ctypes.c_int32),
                ("hist_variant", ctypes.c_int32), ("large_search_nodes", ctypes.c_int32),
                ("hist_chunk", ctypes.c_int32), ("reach_schedule", ctypes.c_int32),
                ("small_search_warps", ctypes.c_int32)]


_PROG_ARRAYS = ["func_instr_off", "func_block_off", "func_loop_off", "block_instr_off", "succ_off", "succ",
                "opclass", "guard", "iflags", "line", "def_off", "def_res", "use_off", "use_res", "block_loop",
                "loop_parent", "loop_header"]
_PROG_DTYPES = dict(opclass=np.uint8, guard=np.uint8, iflags=np.uint8, def_res=np.uint16, use_res=np.uint16)


class gpa_program_desc(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("n_functions", "n_instr", "n_blocks", "n_loops", "n_lines", "n_succ",
                                             "n_def", "n_use")] + [(k, ctypes.c_void_p) for k in _PROG_ARRAYS] + [
                   ("n_calls", ctypes.c_int32), ("call_site", ctypes.c_void_p), ("call_callee", ctypes.c_void_p)]


_ADV = ["totals", "matched", "speedup", "rank", "n_hot", "hot", "loop_active", "loop_matched", "loop_speedup",
        "line_stall", "line_latency", "par_match", "par_speedup", "par_warps", "par_limit"]


class gpa_advice(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in _ADV]


# One function's launch statistics (gpa_launch_stats) as a numpy record.
LAUNCH_DTYPE = np.dtype([("blocks", np.int64), ("threads_per_block", np.int32), ("regs_per_thread", np.int32),
                         ("smem_per_block", np.int32), ("reserved", np.int32)])
_SM_FIELDS = ["n_sms", "schedulers_per_sm", "max_warps_per_sm", "max_blocks_per_sm", "regs_per_sm", "reg_alloc_unit",
              "smem_per_sm", "smem_alloc_unit", "smem_reserved_per_block"]


class gpa_sm_model(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in _SM_FIELDS]


_lib = None


def library() -> ctypes.CDLL:
    """Loads libgpa.so; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgpa.so not built ({LIB_PATH}); run paper_2009_04061_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "gpa_status_string": ([i32], ctypes.c_char_p),
        "gpa_arch_default": ([vp], i32),
        "gpa_create": ([vp, vp, vp], i32),
        "gpa_destroy": ([vp], i32),
        "gpa_load_program": ([vp, vp, vp], i32),
        "gpa_unload_program": ([vp, u32], i32),
        "gpa_reset_counts": ([vp, u32, vp], i32),
        "gpa_ingest_samples": ([vp, u32, vp, ctypes.c_size_t, vp], i32),
        "gpa_ingest_host_samples": ([vp, u32, vp, ctypes.c_size_t, vp], i32),
        "gpa_blame": ([vp, u32, vp], i32),
        "gpa_advise": ([vp, u32, vp, vp], i32),
        "gpa_sync_status": ([vp, u32, vp, vp], i32),
        "gpa_get_counts": ([vp, u32, vp, vp, vp], i32),
        "gpa_get_search_profile": ([vp, u32, vp, vp], i32),
        "gpa_step_capture": ([vp, u32, vp, ctypes.c_size_t], i32),
        "gpa_program_footprint": ([vp, vp, vp], i32),
        "gpa_program_bytes": ([vp, u32, vp], i32),
        "gpa_unload_program_async": ([vp, u32, vp], i32),
        "gpa_dependency_coverage": ([vp, u32, vp, vp], i32),
        "gpa_export_unpruned_edges": ([vp, u32, vp, vp], i32),
        "gpa_get_unpruned_edges": ([vp, u32, vp, vp, vp, vp, vp, vp, vp, vp], i32),
        "gpa_step_launch": ([vp, u32, vp], i32),
        "gpa_get_reaching": ([vp, u32, vp, vp, vp], i32),
        "gpa_get_blame": ([vp, u32, vp, vp], i32),
        "gpa_get_edges": ([vp, u32, vp, i64, vp, vp, vp, vp, vp, vp, vp], i32),
        "gpa_get_advice": ([vp, u32, vp, vp], i32),
        "gpa_set_launch_stats": ([vp, u32, vp, vp], i32),
        "gpa_sm_model_of_device": ([ctypes.c_int, vp], i32),
        "gpa_launch_count": ([vp], i64),
        "gpa_exclusive_scan_noalloc": ([vp, i64, vp, vp], i32),
        "gpa_copy_counts": ([vp, u32, vp, vp], i32),
        "gpa_set_counts": ([vp, u32, vp, ctypes.c_uint64, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the entry points declared in include/gpa.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?![\s/*#])[\w\s\*]+?\b(gpa_\w+)\s*\(", text, flags=re.M)))


def _p(a) -> ctypes.c_void_p:
    if a is None:
        return ctypes.c_void_p(0)
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(st: int, what: str):
    if st != GPA_OK:
        raise GpaError(st, what)


# ---------------------------------------------------------------- C-named wrappers
def gpa_arch_default():
    a = gpa_arch_desc()
    _check(library().gpa_arch_default(ctypes.byref(a)), "gpa_arch_default")
    n = a.n_opclasses
    lat = np.ctypeslib.as_array(ctypes.cast(a.latency, ctypes.POINTER(ctypes.c_int32)), (n,)).copy()
    fl = np.ctypeslib.as_array(ctypes.cast(a.flags, ctypes.POINTER(ctypes.c_uint32)), (n,)).copy()
    return lat, fl


def gpa_create(arch=None, options: dict | None = None):
    lat, fl = arch if arch is not None else gpa_arch_default()
    lat = np.ascontiguousarray(lat, dtype=np.int32)
    fl = np.ascontiguousarray(fl, dtype=np.uint32)
    a = gpa_arch_desc(lat.size, _p(lat), _p(fl))
    o = gpa_options()
    for k, v in (options or {}).items():
        setattr(o, k, int(v))
    ctx = ctypes.c_void_p()
    _check(library().gpa_create(ctypes.byref(a), ctypes.byref(o), ctypes.byref(ctx)), "gpa_create")
    return ctx


def gpa_destroy(ctx):
    _check(library().gpa_destroy(ctx), "gpa_destroy")


def program_desc(arrays: dict):
    """gpa_program_desc over host arrays (kept alive in the returned tuple). The call
    table (call_site, call_callee) is optional."""
    keep = {}
    for k in _PROG_ARRAYS + ["call_site", "call_callee"]:
        a = np.ascontiguousarray(arrays.get(k, np.zeros(0, np.int32)), dtype=_PROG_DTYPES.get(k, np.int32))
        keep[k] = a if a.size else np.zeros(1, dtype=a.dtype)
    n_calls = int(np.asarray(arrays.get("call_site", np.zeros(0))).size)
    d = gpa_program_desc(int(arrays["n_functions"]), int(arrays["n_instr"]), int(arrays["n_blocks"]),
                         int(arrays["n_loops"]), int(arrays["n_lines"]), int(np.asarray(arrays["succ"]).size),
                         int(np.asarray(arrays["def_res"]).size), int(np.asarray(arrays["use_res"]).size),
                         *[_p(keep[k]) for k in _PROG_ARRAYS], n_calls, _p(keep["call_site"]),
                         _p(keep["call_callee"]))
    return d, keep


def gpa_load_program(ctx, arrays: dict) -> int:
    d, keep = program_desc(arrays)
    pid = ctypes.c_uint32()
    st = library().gpa_load_program(ctx, ctypes.byref(d), ctypes.byref(pid))
    del keep
    _check(st, "gpa_load_program")
    return pid.value


def gpa_program_footprint(ctx, arrays: dict) -> int:
    """Device bytes a load of `arrays` would request (nothing is allocated)."""
    d, keep = program_desc(arrays)
    b = ctypes.c_int64()
    st = library().gpa_program_footprint(ctx, ctypes.byref(d), ctypes.byref(b))
    del keep
    _check(st, "gpa_program_footprint")
    return b.value


def gpa_program_bytes(ctx, pid) -> int:
    b = ctypes.c_int64()
    _check(library().gpa_program_bytes(ctx, pid, ctypes.byref(b)), "gpa_program_bytes")
    return b.value


def gpa_unload_program_async(ctx, pid, stream=None):
    _check(library().gpa_unload_program_async(ctx, pid, _stream(stream)), "gpa_unload_program_async")


def gpa_unload_program(ctx, pid):
    _check(library().gpa_unload_program(ctx, pid), "gpa_unload_program")


def gpa_reset_counts(ctx, pid, stream=None):
    _check(library().gpa_reset_counts(ctx, pid, _stream(stream)), "gpa_reset_counts")


def gpa_ingest_samples(ctx, pid, dev_samples, n: int | None = None, stream=None):
    """dev_samples: a CUDA tensor of 64-bit samples (or a raw device pointer with n)."""
    if n is None:
        n = dev_samples.numel()
    _check(library().gpa_ingest_samples(ctx, pid, _p(dev_samples), n, _stream(stream)), "gpa_ingest_samples")


def gpa_ingest_host_samples(ctx, pid, host_samples, n: int | None = None, stream=None):
    if n is None:
        n = host_samples.numel() if hasattr(host_samples, "numel") else host_samples.size
    _check(library().gpa_ingest_host_samples(ctx, pid, _p(host_samples), n, _stream(stream)),
           "gpa_ingest_host_samples")


def _dev_u64(t, n: int, what: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype not in (torch.int64, torch.uint64) \
            or not t.is_contiguous() or t.numel() < n:
        raise ValueError(f"{what} must be a contiguous 64-bit CUDA tensor of at least {n} elements")


def gpa_copy_counts(ctx, pid, dev_dst, n_instr: int, stream=None):
    """Copies the program's counters into dev_dst (a 64-bit CUDA tensor of n_instr * 24 elements)."""
    _dev_u64(dev_dst, n_instr * 24, "dev_dst")
    _check(library().gpa_copy_counts(ctx, pid, _p(dev_dst), _stream(stream)), "gpa_copy_counts")


def gpa_set_counts(ctx, pid, dev_counts, n_instr: int, invalid: int = 0, stream=None):
    """Replaces the program's counters with dev_counts (a 64-bit CUDA tensor of n_instr * 24 elements)."""
    _dev_u64(dev_counts, n_instr * 24, "dev_counts")
    _check(library().gpa_set_counts(ctx, pid, _p(dev_counts), int(invalid), _stream(stream)), "gpa_set_counts")


def gpa_blame(ctx, pid, stream=None):
    _check(library().gpa_blame(ctx, pid, _stream(stream)), "gpa_blame")


def advice_buffers(shape, pinned: bool = False) -> dict:
    """Host arrays for one program's advice, shape = (n_functions, n_loops, n_lines),
    to pass as `out` to gpa_advise / gpa_get_advice on every step instead of new
    arrays each call. pinned: page-locked host memory (torch), which the device
    writes at the host link's rate; fresh pageable arrays are paged in during the
    copy."""
    b = _advice_buffers(shape)
    if not pinned:
        return b
    import torch
    out = {}
    for k, v in b.items():
        t = torch.empty(v.nbytes, dtype=torch.uint8).pin_memory()
        out[k] = t.numpy().view(v.dtype).reshape(v.shape)  # the array's base keeps the tensor alive
        out[k][...] = 0
    return out


def _advice_buffers(shape):
    nf, nl, nlines = shape
    return dict(totals=np.zeros((nf, 4), np.uint64), matched=np.zeros((nf, NUM_OPT), np.uint64),
                speedup=np.zeros((nf, NUM_OPT), np.float64), rank=np.zeros((nf, NUM_OPT), np.int32),
                n_hot=np.zeros((nf, NUM_OPT), np.int32), hot=np.zeros((nf, NUM_OPT, 5, 6), np.int64),
                loop_active=np.zeros(max(nl, 1), np.uint64), loop_matched=np.zeros(max(nl, 1), np.uint64),
                loop_speedup=np.zeros(max(nl, 1), np.float64), line_stall=np.zeros(max(nlines, 1), np.uint64),
                line_latency=np.zeros(max(nlines, 1), np.uint64), par_match=np.zeros((nf, 2), np.int32),
                par_speedup=np.zeros((nf, 2), np.float64), par_warps=np.zeros((nf, 2, 2), np.float64),
                par_limit=np.zeros(nf, np.int32))


def _trim(b, shape):
    nf, nl, nlines = shape
    b = dict(b)
    for k in ("loop_active", "loop_matched", "loop_speedup"):
        b[k] = b[k][:nl]
    for k in ("line_stall", "line_latency"):
        b[k] = b[k][:nlines]
    return b


def _advice_out(shape, out):
    """`out` (from advice_buffers) checked against shape, or new arrays."""
    ref = _advice_buffers(shape)
    if out is None:
        return ref
    for k in _ADV:
        a = out.get(k)
        if not isinstance(a, np.ndarray) or a.dtype != ref[k].dtype or a.shape != ref[k].shape or \
                not a.flags.c_contiguous or not a.flags.writeable:
            raise ValueError(f"advice buffer {k!r}: expected a writable contiguous {ref[k].dtype} array "
                             f"of shape {ref[k].shape}")
    return out


def gpa_advise(ctx, pid, shape=None, stream=None, out=None):
    """shape = (n_functions, n_loops, n_lines) to fetch results, or None to keep them on
    the device; out: arrays from advice_buffers(shape) to fill (else new ones)."""
    if shape is None:
        _check(library().gpa_advise(ctx, pid, None, _stream(stream)), "gpa_advise")
        return None
    b = _advice_out(shape, out)
    adv = gpa_advice(*[_p(b[k]) for k in _ADV])
    _check(library().gpa_advise(ctx, pid, ctypes.byref(adv), _stream(stream)), "gpa_advise")
    return _trim(b, shape)


def gpa_set_launch_stats(ctx, pid, stats, sm: dict | None = None):
    """stats: LAUNCH_DTYPE records (or a dict of equal-length arrays), one per
    function, or None to clear; sm: the gpa_sm_model fields as a dict."""
    if stats is None:
        _check(library().gpa_set_launch_stats(ctx, pid, None, None), "gpa_set_launch_stats")
        return
    if isinstance(stats, dict):
        rec = np.zeros(len(stats["blocks"]), LAUNCH_DTYPE)
        for k in ("blocks", "threads_per_block", "regs_per_thread", "smem_per_block"):
            rec[k] = stats[k]
        stats = rec
    stats = np.ascontiguousarray(stats, dtype=LAUNCH_DTYPE)
    m = gpa_sm_model(*[int(sm[k]) for k in _SM_FIELDS])
    _check(library().gpa_set_launch_stats(ctx, pid, _p(stats), ctypes.byref(m)), "gpa_set_launch_stats")


def gpa_sm_model_of_device(device: int = 0) -> dict:
    m = gpa_sm_model()
    _check(library().gpa_sm_model_of_device(device, ctypes.byref(m)), "gpa_sm_model_of_device")
    return {k: int(getattr(m, k)) for k in _SM_FIELDS}


def gpa_get_advice(ctx, pid, shape, stream=None, out=None):
    b = _advice_out(shape, out)
    adv = gpa_advice(*[_p(b[k]) for k in _ADV])
    _check(library().gpa_get_advice(ctx, pid, ctypes.byref(adv), _stream(stream)), "gpa_get_advice")
    return _trim(b, shape)


def gpa_sync_status(ctx, pid, stream=None):
    info = np.zeros(8, np.int64)
    st = library().gpa_sync_status(ctx, pid, _stream(stream), _p(info))
    return st, dict(invalid=int(info[0]), general_searches=int(info[1]), max_nodes=int(info[2]),
                    sweeps=int(info[3]), tier2_searches=int(info[4]), tier3_searches=int(info[5]),
                    largest_use=int(info[6]), largest_resource=int(info[7]))


def gpa_dependency_coverage(ctx, pid, stream=None) -> tuple[int, int, int]:
    """(stalled uses, single dependency uses before pruning, after pruning)."""
    out = np.zeros(3, np.int64)
    _check(library().gpa_dependency_coverage(ctx, pid, _stream(stream), _p(out)), "gpa_dependency_coverage")
    return int(out[0]), int(out[1]), int(out[2])


def gpa_unpruned_edges(ctx, pid, stream=None) -> dict:
    """Every immediate source before pruning: use, def, res, dmin, K, dlong, dom (ordered)."""
    n = ctypes.c_int64()
    _check(library().gpa_export_unpruned_edges(ctx, pid, _stream(stream), ctypes.byref(n)),
           "gpa_export_unpruned_edges")
    m = max(n.value, 1)
    out = {k: np.zeros(m, np.int32) for k in ("use", "def", "res", "dmin", "K", "dlong")}
    out["dom"] = np.zeros(m, np.uint8)
    _check(library().gpa_get_unpruned_edges(ctx, pid, *[_p(out[k]) for k in ("use", "def", "res", "dmin", "K",
                                                                              "dlong", "dom")], _stream(stream)),
           "gpa_get_unpruned_edges")
    return {k: v[:n.value] for k, v in out.items()}


def gpa_step_capture(ctx, pid, dev_samples, n: int | None = None):
    """Capture reset + ingest + blame + advise of the program into a CUDA graph."""
    if n is None:
        n = dev_samples.numel()
    _check(library().gpa_step_capture(ctx, pid, _p(dev_samples) if n else None, n), "gpa_step_capture")


def gpa_step_launch(ctx, pid, stream=None):
    _check(library().gpa_step_launch(ctx, pid, _stream(stream)), "gpa_step_launch")


def gpa_get_search_profile(ctx, pid, stream=None) -> np.ndarray:
    """Search diagnostics (zeros unless built with -DGPA_PHASE_TIMING): per-tier phase
    cycles, shape (3, 6); searches by log2 of their node count (16); searches past the bound."""
    out = np.zeros(59, np.uint64)
    _check(library().gpa_get_search_profile(ctx, pid, _p(out), _stream(stream)), "gpa_get_search_profile")
    return dict(phases=out[:18].reshape(3, 6), sizes=out[18:34], pass_b=int(out[34]),
                slowest=dict(cycles=int(out[35]) >> 20, nodes=int(out[35]) & 0xFFFFF, rule2_runs=int(out[36]),
                             phase_cycles=[int(x) for x in out[37:42]]),
                size_cycles=out[42:58], overflow_bits=int(out[58]))


def gpa_get_counts(ctx, pid, n_instr: int, stream=None):
    c = np.zeros(n_instr * 24, np.uint64)
    bad = np.zeros(1, np.uint64)
    _check(library().gpa_get_counts(ctx, pid, _p(c), _p(bad), _stream(stream)), "gpa_get_counts")
    return c.reshape(n_instr, 12, 2), int(bad[0])


def gpa_get_reaching(ctx, pid, n_blocks: int, stream=None):
    rin = np.zeros(n_blocks * 9, np.uint32)
    rout = np.zeros(n_blocks * 9, np.uint32)
    _check(library().gpa_get_reaching(ctx, pid, _p(rin), _p(rout), _stream(stream)), "gpa_get_reaching")
    return rin.reshape(-1, 9), rout.reshape(-1, 9)


def gpa_get_blame(ctx, pid, n_instr: int, stream=None):
    b = np.zeros(n_instr * 24, np.uint64)
    _check(library().gpa_get_blame(ctx, pid, _p(b), _stream(stream)), "gpa_get_blame")
    return b.reshape(n_instr, 12, 2)


def gpa_get_edges(ctx, pid, stream=None):
    n = ctypes.c_int64()
    lib = library()
    _check(lib.gpa_get_edges(ctx, pid, ctypes.byref(n), 0, None, None, None, None, None, None, _stream(stream)),
           "gpa_get_edges")
    m = n.value
    a = dict(j=np.zeros(max(m, 1), np.int32), i=np.zeros(max(m, 1), np.int32), dmin=np.zeros(max(m, 1), np.int32),
             dlong=np.zeros(max(m, 1), np.int32), flags=np.zeros(max(m, 1), np.uint32),
             share=np.zeros(max(m, 1) * 8, np.uint64))
    _check(lib.gpa_get_edges(ctx, pid, ctypes.byref(n), m, _p(a["j"]), _p(a["i"]), _p(a["dmin"]), _p(a["dlong"]),
                             _p(a["flags"]), _p(a["share"]), _stream(stream)), "gpa_get_edges")
    out = {k: v[:m] for k, v in a.items() if k != "share"}
    out["share"] = a["share"][:m * 8].reshape(m, 4, 2)
    return out


def gpa_launch_count(ctx) -> int:
    return int(library().gpa_launch_count(ctx))


def gpa_exclusive_scan_noalloc(dev_buf, dev_total, n: int | None = None, stream=None):
    """In-place exclusive scan of the first n values (default: all) of a contiguous int32
    CUDA tensor on the current device; the total goes to dev_total[0] (int32, same device).
    Allocates no device memory (fixed static scratch, see include/gpa.h). Raises ValueError
    for anything else, before the library sees a pointer: a host array or a tensor of
    another dtype or device would be read and written on the device as if it were this."""
    import torch
    for name, t in (("dev_buf", dev_buf), ("dev_total", dev_total)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int32:
            raise ValueError(f"{name} must be an int32 CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on {t.device}, not on the current device")
    if not dev_buf.is_contiguous():
        raise ValueError("dev_buf must be contiguous")
    if dev_total.numel() < 1:
        raise ValueError("dev_total must hold at least one element")
    if n is None:
        n = dev_buf.numel()
    if not 0 <= int(n) <= dev_buf.numel():
        raise ValueError(f"n = {n} outside 0..{dev_buf.numel()} (the elements of dev_buf)")
    _check(library().gpa_exclusive_scan_noalloc(_p(dev_buf), n, _p(dev_total), _stream(stream)),
           "gpa_exclusive_scan_noalloc")


# ---------------------------------------------------------------- convenience objects
class Context:
    def __init__(self, arch=None, options: dict | None = None):
        self.handle = gpa_create(arch, options)

    def load_program(self, arrays) -> "Program":
        a = arrays.arrays if hasattr(arrays, "arrays") else arrays
        return Program(self, gpa_load_program(self.handle, a), a)

    def launches(self) -> int:
        return gpa_launch_count(self.handle)

    def footprint(self, arrays) -> int:
        a = arrays.arrays if hasattr(arrays, "arrays") else arrays
        return gpa_program_footprint(self.handle, a)

    def close(self):
        if self.handle:
            gpa_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Program:
    def __init__(self, ctx: Context, pid: int, arrays: dict):
        self.ctx, self.pid = ctx, pid
        self.n_instr, self.n_blocks = int(arrays["n_instr"]), int(arrays["n_blocks"])
        self.shape = (int(arrays["n_functions"]), int(arrays["n_loops"]), int(arrays["n_lines"]))

    @property
    def h(self):
        return self.ctx.handle

    def reset(self, stream=None):
        gpa_reset_counts(self.h, self.pid, stream)

    def ingest(self, dev_samples, n=None, stream=None):
        gpa_ingest_samples(self.h, self.pid, dev_samples, n, stream)

    def ingest_host(self, host_samples, n=None, stream=None):
        gpa_ingest_host_samples(self.h, self.pid, host_samples, n, stream)

    def set_launch_stats(self, stats, sm: dict | None = None):
        gpa_set_launch_stats(self.h, self.pid, stats, sm)

    def copy_counts(self, dev_dst, stream=None):
        gpa_copy_counts(self.h, self.pid, dev_dst, self.n_instr, stream)

    def set_counts(self, dev_counts, invalid: int = 0, stream=None):
        gpa_set_counts(self.h, self.pid, dev_counts, self.n_instr, invalid, stream)

    def blame(self, stream=None):
        gpa_blame(self.h, self.pid, stream)

    def advise(self, fetch: bool = True, stream=None, out=None):
        return gpa_advise(self.h, self.pid, self.shape if fetch else None, stream, out)

    def advice_buffers(self, pinned: bool = False) -> dict:
        return advice_buffers(self.shape, pinned)

    def status(self, stream=None):
        return gpa_sync_status(self.h, self.pid, stream)

    def counts(self, stream=None):
        return gpa_get_counts(self.h, self.pid, self.n_instr, stream)

    def coverage(self, stream=None):
        return gpa_dependency_coverage(self.h, self.pid, stream)

    def unpruned_edges(self, stream=None):
        return gpa_unpruned_edges(self.h, self.pid, stream)

    def device_bytes(self) -> int:
        return gpa_program_bytes(self.h, self.pid)

    def capture_step(self, dev_samples, n=None):
        gpa_step_capture(self.h, self.pid, dev_samples, n)

    def launch_step(self, stream=None):
        gpa_step_launch(self.h, self.pid, stream)

    def get_advice(self, stream=None, out=None):
        return gpa_get_advice(self.h, self.pid, self.shape, stream, out)

    def search_profile(self, stream=None):
        return gpa_get_search_profile(self.h, self.pid, stream)

    def reaching(self, stream=None):
        return gpa_get_reaching(self.h, self.pid, self.n_blocks, stream)

    def blame_counts(self, stream=None):
        return gpa_get_blame(self.h, self.pid, self.n_instr, stream)

    def edges(self, stream=None):
        return gpa_get_edges(self.h, self.pid, stream)

    def advice(self, stream=None):
        return gpa_get_advice(self.h, self.pid, self.shape, stream)

    def unload(self):
        gpa_unload_program(self.h, self.pid)

    def unload_async(self, stream=None):
        """Free in stream order after the work queued on `stream` (no host wait)."""
        gpa_unload_program_async(self.h, self.pid, stream)

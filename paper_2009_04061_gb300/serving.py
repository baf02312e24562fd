"""Continuous-batching analysis server over the C ABI.

Profiling sessions (a program and its packed samples) arrive over time. A
session is admitted as soon as a slot is free and the device-memory budget
has room for its program: a slot is a context of its own (own search scratch,
own sample staging) with its own CUDA stream and its own host thread, so
admitted sessions run side by side on the device and their host work (the
program's validation and upload, the advice copy-out) runs side by side on
the host cores, while later sessions queue. For each admitted session the
slot's thread loads the program and queues ingest (from pinned host memory)
-> blame -> advice on the slot's stream, waits for it, copies the advice out
and frees the program in stream order. A session's device footprint (for the
budget) is computed when it is submitted, on a small pool of host threads.

Latency is ingest-to-advice: from a session's arrival (its submission) to
its advice being on the host.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import gpa


@dataclass
class Session:
    sid: int
    program: dict                 # program arrays (the gpa_program_desc fields)
    samples: np.ndarray           # packed uint64 samples, host memory (pinned for overlap)
    t_arrival: float = 0.0        # seconds on the server's clock
    need: object = field(default=None, repr=False)  # future of its device footprint (bytes)


@dataclass
class Result:
    sid: int
    advice: dict
    n_samples: int
    t_arrival: float
    t_admit: float
    t_done: float
    device_bytes: int
    counts: np.ndarray | None = None
    blame: np.ndarray | None = None
    edges: dict | None = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class _Slot:
    ctx: object
    stream: object
    jobs: object = None            # queue of (session, t_admit, bytes) for the slot's thread
    busy: bool = False
    thread: object = field(default=None, repr=False)


class Server:
    """slots: concurrent sessions; budget_bytes: device memory the admitted
    sessions' programs may hold together; keep_results: also return counts,
    blame and edges (for checking results against the session run alone and
    against the oracle)."""

    def __init__(self, arch, slots: int = 4, budget_bytes: int = 64 << 30, options: dict | None = None,
                 keep_results: bool = False):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device()
        if options is None:
            # Slots run side by side: four global-memory search warps per SM each
            # (about 2.6 GB of search scratch per slot) instead of a whole GPU's worth.
            sms = torch.cuda.get_device_properties(self.device).multi_processor_count
            options = {"search_slots": 4 * sms}
        self.slots = [_Slot(gpa.Context(arch, options), torch.cuda.Stream()) for _ in range(slots)]
        self.budget = int(budget_bytes)
        self.used = 0
        self.pending: collections.deque[Session] = collections.deque()
        self.keep_results = keep_results
        self.t0 = time.perf_counter()
        self._done: queue.Queue = queue.Queue()
        self._sizer = ThreadPoolExecutor(4)
        for k, sl in enumerate(self.slots):
            sl.jobs = queue.Queue()
            sl.thread = threading.Thread(target=self._work, args=(k,), daemon=True)
            sl.thread.start()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, s: Session, t_arrival: float | None = None):
        s.t_arrival = self.now() if t_arrival is None else t_arrival
        if s.need is None:
            s.need = self._sizer.submit(self.slots[0].ctx.footprint, s.program)
        self.pending.append(s)

    def busy(self) -> int:
        return sum(1 for sl in self.slots if sl.busy)

    def _work(self, k: int):
        """The slot's thread: run the sessions handed to it one after another."""
        self._torch.cuda.set_device(self.device)
        sl = self.slots[k]
        while True:
            job = sl.jobs.get()
            if job is None:
                return
            s, t_admit, nbytes = job
            try:
                r = self._run(sl, s, t_admit, nbytes)
            except BaseException as e:  # handed to the polling thread, which raises it
                r = e
            self._done.put((k, r))

    def _run(self, sl: _Slot, s: Session, t_admit: float, nbytes: int) -> Result:
        st = sl.stream
        prog = sl.ctx.load_program(s.program)  # raises (nothing loaded) on a malformed program
        try:
            prog.reset(st)
            if s.samples.size:
                prog.ingest_host(s.samples, stream=st)
            prog.blame(st)
            prog.advise(fetch=False, stream=st)
            code, info = prog.status(st)  # waits for the slot's stream
            if code != 0:
                raise RuntimeError(f"session {s.sid}: device status {code} ({info})")
            adv = prog.get_advice(st)
            counts = blame = edges = None
            if self.keep_results:
                counts, _ = prog.counts(st)
                blame = prog.blame_counts(st)
                edges = prog.edges(st)
            return Result(s.sid, adv, int(s.samples.size), s.t_arrival, t_admit, self.now(), nbytes, counts, blame,
                          edges)
        finally:
            prog.unload_async(st)

    def poll(self) -> list[Result]:
        """Collect finished sessions, then admit waiting ones (in arrival order)
        while a slot is free and the budget allows."""
        done = []
        while True:
            try:
                k, r = self._done.get_nowait()
            except queue.Empty:
                break
            self.slots[k].busy = False
            if isinstance(r, BaseException):
                raise r
            self.used -= r.device_bytes
            done.append(r)
        while self.pending:
            free = [sl for sl in self.slots if not sl.busy]
            if not free:
                break
            s = self.pending[0]
            if not s.need.done():
                break
            need = s.need.result()
            if need > self.budget:
                raise ValueError(f"session {s.sid} needs {need} bytes, more than the whole budget")
            if self.used + need > self.budget:
                break
            self.pending.popleft()
            self.used += need
            free[0].busy = True
            free[0].jobs.put((s, self.now(), need))
        return done

    def close(self):
        while self.busy():
            self.poll()
            time.sleep(1e-4)
        for sl in self.slots:
            sl.jobs.put(None)
        for sl in self.slots:
            sl.thread.join()
            sl.stream.synchronize()
            sl.ctx.close()
        self._sizer.shutdown(wait=True)


def serve(server: Server, sessions: list[Session], arrivals: list[float], idle_sleep: float = 1e-4) -> list[Result]:
    """Replays `sessions` arriving at `arrivals` (seconds from now) through the
    server and returns their results in completion order."""
    order = np.argsort(np.asarray(arrivals), kind="stable")
    start = server.now()
    out: list[Result] = []
    k = 0
    while len(out) < len(sessions):
        t = server.now() - start
        while k < len(order) and arrivals[order[k]] <= t:
            i = order[k]
            server.submit(sessions[i], start + arrivals[i])
            k += 1
        got = server.poll()
        out += got
        if not got:
            time.sleep(idle_sleep)
    return out


def one_at_a_time(arch, sessions: list[Session], options: dict | None = None) -> tuple[float, list[Result]]:
    """The same sessions run back to back on one context and stream, each
    waiting for the previous one; returns (seconds, results)."""
    srv = Server(arch, slots=1, budget_bytes=1 << 62, options=options)
    try:
        t0 = time.perf_counter()
        out = []
        for s in sessions:
            srv.submit(s)
            while True:
                got = srv.poll()
                if got:
                    out += got
                    break
                time.sleep(1e-4)
        return time.perf_counter() - t0, out
    finally:
        srv.close()


def latency_summary(results: list[Result]) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    span = max(r.t_done for r in results) - min(r.t_arrival for r in results)
    n = sum(r.n_samples for r in results)
    return {"sessions": len(results), "samples": n, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "samples_per_s": n / span, "span_s": span}

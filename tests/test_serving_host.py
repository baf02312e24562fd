"""The serving record's host arithmetic (no device): ingest-to-advice latency
percentiles and throughput over the span from the first arrival to the last answer."""
import numpy as np
import pytest

from paper_2009_04061_gb300.serving import Result, latency_summary


def _result(sid, t_arrival, t_done, n):
    return Result(sid=sid, advice={}, n_samples=n, t_arrival=t_arrival, t_admit=t_arrival,
                  t_done=t_done, device_bytes=0)


def test_latency_summary_by_hand():
    # latencies 10, 20, ..., 100 ms; the first arrives at t = 1.0 s, the last answer at 1.5 s
    rs = [_result(i, 1.0 + 0.04 * i, 1.0 + 0.04 * i + 0.01 * (i + 1), 1000 * (i + 1)) for i in range(10)]
    m = latency_summary(rs)
    assert m["sessions"] == 10 and m["samples"] == 55_000
    assert m["span_s"] == pytest.approx(1.46 - 1.0)                  # last t_done = 1.36 + 0.10
    assert m["samples_per_s"] == pytest.approx(55_000 / 0.46)
    assert m["p50_ms"] == pytest.approx(55.0)                        # midway between 50 and 60 ms
    assert m["p99_ms"] == pytest.approx(np.percentile(np.arange(10, 101, 10), 99))
    assert m["mean_ms"] == pytest.approx(55.0) and m["max_ms"] == pytest.approx(100.0)


def test_latency_is_arrival_to_answer():
    r = _result(0, 2.5, 2.75, 1)
    assert r.latency == pytest.approx(0.25)                           # queueing included

"""The open-loop load generator of the query server (serving.py), on the CPU:
its seeded schedule, and its bookkeeping against a stand-in server."""
import threading

import numpy as np

from paper_2509_01654_gb300 import serving, synth


def test_request_plan_is_poisson_and_log_uniform():
    arrivals, sizes = serving.request_plan(20_000, 40.0, 1, 4096, seed=5)
    again = serving.request_plan(20_000, 40.0, 1, 4096, seed=5)
    assert np.array_equal(arrivals, again[0]) and np.array_equal(sizes, again[1])
    gaps = np.diff(np.concatenate([[0.0], arrivals]))
    assert np.all(gaps >= 0)
    assert abs(gaps.mean() * 40.0 - 1.0) < 0.03              # exponential gaps of mean 1/rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05       # coefficient of variation 1
    assert sizes.min() >= 1 and sizes.max() <= 4096
    # log-uniform on [1, 4096]: about half the requests at or below sqrt(4096) = 64 words
    assert abs(np.mean(sizes <= 64) - 0.5) < 0.03


class FakeServer:
    """Records each request and answers it at once with server-style timings."""

    def __init__(self):
        self.requests = []
        self.lock = threading.Lock()
        self.t = 0.0

    def submit(self, codes, qoff):
        assert qoff[0] == 0 and np.all(np.diff(qoff.astype(np.int64)) >= 0) and qoff[-1] == codes.size
        with self.lock:
            self.requests.append(qoff.size - 1)
            return len(self.requests) - 1

    def wait(self, rid):
        n = self.requests[rid]
        info = {"submit_s": 1.0 * rid, "done_s": 1.0 * rid + 1e-3 * n, "batch_requests": 1,
                "inflight_at_start": 0}
        return None, None, info


def test_run_load_bookkeeping():
    pool = synth.serving_queries(5000, seed=9)
    srv = FakeServer()
    out = serving.run_load(srv, pool, n_requests=60, rate_hz=1e6, max_batch=512, seed=3)
    _, sizes = serving.request_plan(60, 1e6, 1, 512, 3)
    assert srv.requests == sizes.tolist()
    assert out["requests"] == 60 and out["queries"] == int(sizes.sum())
    lat = 1e-3 * sizes * 1e3  # the stand-in's latency is n ms
    assert abs(out["p50_ms"] - np.percentile(lat, 50)) < 1e-9
    assert abs(out["p99_ms"] - np.percentile(lat, 99)) < 1e-9
    assert out["max_inflight_seen"] == 1 and out["mean_requests_per_batch"] == 1.0

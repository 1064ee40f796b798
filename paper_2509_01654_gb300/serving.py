"""Open-loop load generator for the query server (nw_server_*).

Requests arrive as a Poisson process; each carries a batch of query words whose
size is log-uniform on [min_batch, max_batch]; query words come from the
seeded query generator (lengths uniform on [1, 30], the dictionary's alphabet
and code law).  A submitter thread issues requests at their arrival times and
the caller's thread collects them; latencies are the server's own
submit-to-results times.  Returns p50/p99 latency and throughput.
"""
from __future__ import annotations

import math
import threading
import time

import numpy as np

from . import nw, synth


def request_plan(n_requests: int, rate_hz: float, min_batch: int, max_batch: int, seed: int):
    """(arrival offsets in s, batch sizes) of a seeded open-loop schedule."""
    u = synth.uniform01(seed, synth.STREAM_MISC, 2 * n_requests)
    gaps = -np.log1p(-u[:n_requests]) / rate_hz
    arrivals = np.cumsum(gaps)
    lo, hi = math.log(min_batch), math.log(max_batch + 1)
    sizes = np.minimum(max_batch, np.floor(np.exp(lo + u[n_requests:] * (hi - lo)))).astype(np.int64)
    return arrivals, np.maximum(sizes, 1)


def run_load(server: "nw.Server", pool: "synth.WordList", n_requests: int = 200, rate_hz: float = 50.0,
             min_batch: int = 1, max_batch: int = 4096, seed: int = 5):
    arrivals, sizes = request_plan(n_requests, rate_hz, min_batch, max_batch, seed)
    starts = np.zeros(n_requests, dtype=np.int64)
    starts[1:] = np.cumsum(sizes)[:-1] % max(1, pool.n - max_batch)
    offs = pool.offsets.astype(np.int64)
    ids = [None] * n_requests
    ready = threading.Semaphore(0)

    def submitter():
        t0 = time.perf_counter()
        for r in range(n_requests):
            delay = arrivals[r] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            a, b = int(starts[r]), int(starts[r] + sizes[r])
            codes = pool.codes[offs[a]:offs[b]]
            qoff = (offs[a:b + 1] - offs[a]).astype(np.uint32)
            ids[r] = server.submit(codes, qoff)
            ready.release()

    th = threading.Thread(target=submitter)
    th.start()
    infos = []
    for r in range(n_requests):
        ready.acquire()
        _, _, info = server.wait(ids[r])
        infos.append(info)
    th.join()
    lat = np.array([i["done_s"] - i["submit_s"] for i in infos]) * 1e3
    t_first = min(i["submit_s"] for i in infos)
    t_last = max(i["done_s"] for i in infos)
    nq = int(sizes.sum())
    return {
        "requests": n_requests,
        "queries": nq,
        "offered_rate_hz": rate_hz,
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()),
        "queries_per_s": nq / (t_last - t_first),
        "mean_requests_per_batch": float(np.mean([i["batch_requests"] for i in infos])),
        "max_inflight_seen": int(max(i["inflight_at_start"] for i in infos)) + 1,
    }

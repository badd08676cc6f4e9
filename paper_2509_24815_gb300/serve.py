"""Serving runs: Poisson arrival traces replayed through the continuous-
batching server (seismic_server_*), with latency percentiles and throughput.
The server and its admission control are native (csrc/serve.cu); this module
only builds traces and summarises them."""
from __future__ import annotations

import numpy as np

from . import Server, SearchParams, search_params


def poisson_arrivals(n: int, rate_qps: float, seed: int = 3) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_qps, size=n))


def k_mix(n: int, ks=(10, 100), probs=(0.9, 0.1), seed: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed + 1)
    return rng.choice(np.asarray(ks, dtype=np.uint32), size=n, p=np.asarray(probs, dtype=np.float64))


def run_trace(index, queries, rate_qps: float, ks=(10, 100), probs=(0.9, 0.1), search: SearchParams | None = None,
              max_batch=256, streams=4, seed=3, server: Server | None = None):
    """Replays `queries` (host CSR) arriving as a Poisson process; returns the
    results and a summary (p50/p99/mean latency in ms, achieved QPS)."""
    n = queries.n_rows
    arr = poisson_arrivals(n, rate_qps, seed)
    kq = k_mix(n, ks, probs, seed)
    srv = server or Server(index, search if search is not None else search_params(), max_batch=max_batch,
                           streams=streams)
    ids, sc, lat, wall = srv.replay(queries, arr, kq)
    lat_ms = lat / 1e3
    summary = {"offered_qps": rate_qps, "achieved_qps": n / wall, "p50_ms": float(np.percentile(lat_ms, 50)),
               "p99_ms": float(np.percentile(lat_ms, 99)), "mean_ms": float(lat_ms.mean()), "queries": n,
               "k_mix": {int(k): float(p) for k, p in zip(ks, probs)}, **srv.settings}
    return ids, sc, kq, summary

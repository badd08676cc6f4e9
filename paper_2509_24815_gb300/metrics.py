"""accuracy@k (Definition "ann-accuracy", Section 2) and the algorithmic byte
count of a search, from the library's own outputs and work counters."""
from __future__ import annotations

import numpy as np

from . import NONE_ID, STATS


def recall_at_k(ids, scores, gt_scores, k: int = 10, rel_tol: float = 1e-5) -> np.ndarray:
    """|S cap S'| / k per query, tie-aware: a returned id counts when its score
    reaches the exact k-th score minus rel_tol * |k-th| (fp32 scores, so
    rel_tol covers their rounding).  Returned ids are distinct by construction."""
    ids = np.asarray(ids)[:, :k].astype(np.uint32)
    sc = np.asarray(scores, dtype=np.float64)[:, :k]
    kth = np.asarray(gt_scores, dtype=np.float64)[:, k - 1]
    thr = kth - rel_tol * np.abs(kth)
    hit = (ids != NONE_ID) & (sc >= thr[:, None])
    return hit.sum(axis=1) / k


def algorithmic_bytes(stats: np.ndarray, k: int, quantized: bool, kappa: int = 0, fp16: bool = False,
                      knn_bits: int = 32) -> np.ndarray:
    """Bytes the method must move per query under this library's layout
    (no padding, no sector rounding):
      query in: 8 (indptr pair) + 6 per entry (u16 term + f32 value)
      per list: 8 (block range) + 4 per summary-directory word read (a
        presence word per query term, a column's bounds when present)
      per scored block: 8 (m, size) when quantised
      per summary column entry: 2 (block) + 1 (code) quantised, 2 + 4 fp32
      per evaluated block: 8 (member range) + 4 per member id
      per scored document: 8 (row descriptor) + per nonzero 2 (term) + 4
        (fp32 value) or 2 (fp16 value)
      kappa expansion: knn_bits / 8 per neighbour id read (bit-packed) + rows as above
      out: 8 per result."""
    s = {n: stats[:, i].astype(np.float64) for i, n in enumerate(STATS)}
    per_nnz = 4 if fp16 else 6
    b = 8 + 6 * s["query_nnz"]
    b += 8 * s["lists"] + 4 * s["dir_lookups"]
    b += (8 * s["blocks_scored"]) if quantized else 0
    b += (3 if quantized else 6) * s["summary_entries"]
    b += 8 * s["blocks_evaluated"] + 4 * s["block_docs"]
    b += 8 * s["docs"] + per_nnz * s["doc_nnz"]
    if kappa:
        b += knn_bits / 8 * kappa * k + 8 * s["knn_docs"] + per_nnz * s["knn_nnz"]
    b += 8 * k
    return b


def queue_occupancy(stats: np.ndarray, slots: int) -> dict:
    """Load balance of one persistent launch from the per-query device
    timestamps: `busy` = the fraction of slot-time (slots = resident CTAs or
    warps) spent inside queries between the first start and the last end, and
    `tail_ms` = the time from the last query's start (the queue is empty) to
    the last end, during which slots fall idle one by one.  1 - busy bounds
    what a finer-grained work queue (splitting queries across CTAs) could win."""
    t0 = stats[:, STATS.index("t_start_ns")].astype(np.float64)
    t1 = stats[:, STATS.index("t_end_ns")].astype(np.float64)
    span = float(t1.max() - t0.min())
    busy = float((t1 - t0).sum()) / (slots * span) if span > 0 else 1.0
    per_q = (t1 - t0) / 1e6
    return {"busy": busy, "span_ms": span / 1e6, "tail_ms": float(t1.max() - t0.max()) / 1e6,
            "query_ms_p50": float(np.percentile(per_q, 50)), "query_ms_p99": float(np.percentile(per_q, 99)),
            "query_ms_max": float(per_q.max()), "slots": int(slots)}

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


def algorithmic_bytes(stats: np.ndarray, k: int, quantized: bool, kappa: int = 0) -> np.ndarray:
    """Bytes the method must move per query under this library's layout
    (no padding, no sector rounding):
      query in: 8 (indptr pair) + 6 per entry (u16 term + f32 value)
      per list: 8 (block range) + 4 per directory entry read (2 per query term)
      per scored block: 8 (m, size) when quantised
      per summary column entry: 2 (block) + 1 (code) quantised, 2 + 4 fp32
      per evaluated block: 8 (member range) + 4 per member id
      per scored document: 8 (row range) + 6 per nonzero
      kappa expansion: 4 per neighbour id read + rows as above
      out: 8 per result."""
    s = {n: stats[:, i].astype(np.float64) for i, n in enumerate(STATS)}
    b = 8 + 6 * s["query_nnz"]
    b += 8 * s["lists"] + 4 * s["dir_lookups"]
    b += (8 * s["blocks_scored"]) if quantized else 0
    b += (3 if quantized else 6) * s["summary_entries"]
    b += 8 * s["blocks_evaluated"] + 4 * s["block_docs"]
    b += 8 * s["docs"] + 6 * s["doc_nnz"]
    if kappa:
        b += 4 * kappa * k + 8 * s["knn_docs"] + 6 * s["knn_nnz"]
    b += 8 * k
    return b

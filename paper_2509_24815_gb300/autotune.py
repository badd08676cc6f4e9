"""Launch-configuration autotuner for batched search.

The result of a search depends only on (k, cut, heap_factor, hf_mode, alpha_q,
kappa expansion) and on `wave` (blocks of a wave pass the skip test against
the heap at the wave's start); the kernel shape, the lane-group width and the
warps per CTA change only the speed.  The tuner times each candidate launch
configuration on the caller's batch with CUDA events on one stream, keeps those
whose recall (judged by the caller's function) stays at or above a floor, and
returns the fastest.  Winners are cached in a JSON file keyed by the index,
the batch and the device, so a serving process tunes once.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import DeviceCSR, search_params, seismic_info, seismic_search

# (shape, group, cta_warps, wave, L2 row prefetch): shape 1 = one CTA per query
# (group 1: chunk-flattened scoring, else lane groups of that width), 2 = one
# warp per query
DEFAULT_CANDIDATES = tuple(
    [(1, 1, 8, v, pf) for v in (4, 8, 16, 32) for pf in (False, True)] +
    [(1, 1, 16, v, pf) for v in (8, 16) for pf in (False, True)] +
    [(1, 8, 8, v, pf) for v in (4, 16) for pf in (False, True)] +
    [(1, 16, 8, 16, True), (1, 8, 4, 16, True)] +
    [(2, g, 4, 1, pf) for g in (4, 8) for pf in (False, True)])


def signature(index, queries: DeviceCSR, base: dict) -> str:
    import torch
    info = seismic_info(index)
    dev = torch.cuda.get_device_name(queries.vals.device)
    keys = ("k", "cut", "heap_factor", "hf_mode", "alpha_q", "use_knn", "learned")
    b = ",".join(f"{k}={base.get(k)}" for k in keys)
    return (f"{dev}|docs={info['n_docs']}|nnz={info['nnz']}|blocks={info['n_blocks']}|kappa={info['kappa']}|"
            f"nq={queries.n_rows}|qnnz={queries.vals.numel()}|{b}")


def autotune(index, queries: DeviceCSR, base: dict, recall_fn=None, min_recall: float | None = None,
             candidates=DEFAULT_CANDIDATES, reps: int = 3, stream=None, cache: str | None = None, log=None):
    """Returns (best, table).  `base` holds the search parameters that fix the
    result (k, cut, heap_factor, ...); `recall_fn(ids, scores) -> float` judges
    a candidate's output when `min_recall` is given.  `best` is a dict of
    search_params keyword arguments (base + the chosen launch configuration)."""
    import torch
    sig = signature(index, queries, base)
    if cache and os.path.exists(cache):
        with open(cache) as f:
            hit = json.load(f).get(sig)
        if hit:
            return dict(base, **hit["launch"]), hit["table"]
    st = stream or torch.cuda.Stream()
    nq, k = queries.n_rows, base.get("k", 10)
    ids = torch.empty((nq, k), dtype=torch.int32, device=queries.vals.device)
    sc = torch.empty((nq, k), dtype=torch.float32, device=queries.vals.device)
    table = []
    for shape, g, w, v, pf in candidates:
        if shape == 2 and k > 128:
            continue
        launch = dict(shape=shape, group=g, cta_warps=w, wave=v, persistent=True, no_prefetch=not pf)
        p = search_params(max_query_nnz=queries.max_row_nnz, **dict(base, **launch))
        try:
            seismic_search(index, queries, p, ids_out=ids, scores_out=sc, stream=st)
            st.synchronize()
        except RuntimeError as e:  # a configuration the index or batch does not fit (shared memory)
            table.append(dict(launch, error=str(e)))
            continue
        rec = None
        if recall_fn is not None:
            rec = float(recall_fn(ids, sc))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        with torch.cuda.stream(st):
            for i in range(reps):
                ev[2 * i].record(st)
                seismic_search(index, queries, p, ids_out=ids, scores_out=sc, stream=st)
                ev[2 * i + 1].record(st)
        st.synchronize()
        ms = float(np.median([ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(reps)]))
        table.append(dict(launch, ms=ms, qps=nq / ms * 1e3, recall=rec))
        if log:
            log(f"  autotune shape={shape} group={g:2d} warps={w:2d} wave={v:2d} prefetch={int(pf)}: {ms:7.2f} ms"
                + (f"  recall {rec:.4f}" if rec is not None else ""))
    ok = [t for t in table if "ms" in t and (min_recall is None or t["recall"] is None or t["recall"] >= min_recall)]
    if not ok:
        raise RuntimeError("autotune: no launch configuration ran and met the recall floor")
    top = min(ok, key=lambda t: t["ms"])
    launch = {x: top[x] for x in ("shape", "group", "cta_warps", "wave", "persistent", "no_prefetch")}
    if cache:
        data = {}
        if os.path.exists(cache):
            with open(cache) as f:
                data = json.load(f)
        data[sig] = {"launch": launch, "table": table}
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, cache)
    return dict(base, **launch), table

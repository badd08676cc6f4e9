"""Learned per-query search parameters (not in the paper, which tunes alpha_q
or cut and heap_factor globally, Section 5.3).

Labels come from the method itself: every training query is searched at each
(cut, heap_factor) of a grid, its recall@10 is judged against the exact top-10
(brute force on the device), and its label is the cheapest grid point (fewest
bytes read, from the search's work counters) whose recall reaches the target.
The MLP (64 -> 128 -> 64 -> 2, ReLU, bf16 activations) is trained on the GPU by
the library's own forward/backward/Adam kernels and installed in the index;
``learned=1`` searches then run the feature and MLP kernels ahead of the
search, with the fixed parameters as the fallback for non-finite outputs.
"""
from __future__ import annotations

import numpy as np

from . import (MLP_PARAMS, DeviceCSR, STATS, search_params, seismic_query_features, seismic_search,
               seismic_search_exact, seismic_set_mlp, seismic_mlp_train_step, seismic_mlp_forward)
from .metrics import algorithmic_bytes, recall_at_k

GRID_CUT = (3, 4, 5, 6, 8, 10, 12, 15, 20, 25, 30)
GRID_HF = (0.5, 0.6, 0.7, 0.8, 0.9, 1.0)
CUT_LO, CUT_SPAN = 3.0, 27.0
HF_LO, HF_SPAN = 0.5, 0.5


def init_weights(seed: int = 0) -> np.ndarray:
    """He-initialised weights, packed W1, b1, W2, b2, W3, b3; the last layer is
    zeroed so the untrained network predicts the middle of both ranges."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((128, 64)) * np.sqrt(2.0 / 64)
    w2 = rng.standard_normal((64, 128)) * np.sqrt(2.0 / 128)
    parts = [w1.ravel(), np.zeros(128), w2.ravel(), np.zeros(64), np.zeros(2 * 64), np.zeros(2)]
    return np.concatenate(parts).astype(np.float32)


def label_queries(index, queries: DeviceCSR, k: int = 10, target: float = 0.9, quantized: bool = True,
                  grid_cut=GRID_CUT, grid_hf=GRID_HF, base_params: dict | None = None):
    """Per-query (cut, heap_factor) labels: the grid point with the fewest
    algorithmic bytes whose recall@k reaches `target`; queries that never reach
    it take their highest-recall point.  Returns (cut, hf, table) where table
    holds every grid point's per-query recall and bytes."""
    base = dict(base_params or {})
    _, gt = seismic_search_exact(index, queries, k)
    gt = gt.cpu().numpy()
    nq = queries.n_rows
    best_bytes = np.full(nq, np.inf)
    best_rec = np.full(nq, -1.0)
    cut = np.full(nq, grid_cut[len(grid_cut) // 2], dtype=np.int64)
    hf = np.full(nq, 0.8)
    table = []
    for c in grid_cut:
        for h in grid_hf:
            ids, sc, st = seismic_search(index, queries, search_params(k=k, cut=c, heap_factor=h,
                                                                      max_query_nnz=queries.max_row_nnz,
                                                                      **base), stats=True)
            rec = recall_at_k(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), gt, k)
            by = algorithmic_bytes(st, k, quantized)
            table.append((c, h, rec, by))
            ok = rec >= target
            better = ok & ((best_rec < target) | (by < best_bytes))
            fallback = (~ok) & (best_rec < target) & (rec > best_rec)
            upd = better | fallback
            cut[upd], hf[upd] = c, h
            best_bytes[upd] = by[upd]
            best_rec[upd] = rec[upd]
    return cut, hf, table


def lagrangian_labels(table, target: float, margin: float = 0.01):
    """Per-query labels that meet the target on average with the least work:
    each query takes the grid point maximising recall - mu * bytes, and mu is
    the largest value (bisection) whose mean recall still reaches
    target + margin.  Returns (cut, hf, mean recall, mean bytes)."""
    cuts = np.array([c for c, _, _, _ in table], dtype=np.int64)
    hfs = np.array([h for _, h, _, _ in table], dtype=np.float64)
    rec = np.stack([r for _, _, r, _ in table], axis=1)   # [nq, G]
    by = np.stack([b for _, _, _, b in table], axis=1)    # [nq, G]
    want = min(target + margin, float(rec.max(axis=1).mean()))

    def choose(mu):
        g = np.argmax(rec - mu * by, axis=1)
        return g, float(rec[np.arange(len(g)), g].mean())

    lo, hi = 0.0, 1.0 / max(float(by.min()), 1.0)  # mu = hi: recall is worth less than one byte
    while choose(hi)[1] >= want and hi < 1e3:
        hi *= 2.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if choose(mid)[1] >= want:
            lo = mid
        else:
            hi = mid
    g, r = choose(lo)
    return cuts[g], hfs[g], r, float(by[np.arange(len(g)), g].mean())


def standardize(features: np.ndarray):
    """Per-feature mean and spread of the training features (spread 1 where a
    feature is constant); the features differ in scale by two orders of
    magnitude (values near 1, their L1 norm up to ~200)."""
    f = np.asarray(features, dtype=np.float64)
    mu, sd = f.mean(axis=0), f.std(axis=0)
    sd[sd < 1e-6] = 1.0
    return mu, sd


def fold_input_scaling(weights: np.ndarray, mu: np.ndarray, sd: np.ndarray) -> np.ndarray:
    """Weights trained on (x - mu) / sd, rewritten to take x itself:
    W1 <- W1 / sd (per input column), b1 <- b1 - (W1 / sd) mu.  The installed
    network and the inference kernels then see raw features."""
    w = np.array(weights, dtype=np.float64, copy=True)
    n1 = 128 * 64
    w1 = w[:n1].reshape(128, 64) / sd[None, :]
    w[:n1] = w1.ravel()
    w[n1:n1 + 128] = w[n1:n1 + 128] - w1 @ mu
    return w.astype(np.float32)


def targets_from_labels(cut, hf) -> np.ndarray:
    t0 = (np.asarray(cut, dtype=np.float64) - CUT_LO) / CUT_SPAN
    t1 = (np.asarray(hf, dtype=np.float64) - HF_LO) / HF_SPAN
    return np.clip(np.stack([t0, t1], axis=1), 0.0, 1.0).astype(np.float32)


def train(features: np.ndarray, targets: np.ndarray, steps: int = 3000, lr: float = 2e-3, batch: int = 4096,
          seed: int = 0, weights: np.ndarray | None = None, log_every: int = 0):
    """Adam on the device with the library's MLP kernels; returns the weights
    (host float32) and the loss trace."""
    import torch
    dev = "cuda"
    rng = np.random.default_rng(seed)
    # feature scaling is part of the data, not the network: keep raw features
    f_all = torch.from_numpy(np.ascontiguousarray(features, dtype=np.float32)).to(dev)
    t_all = torch.from_numpy(np.ascontiguousarray(targets, dtype=np.float32)).to(dev)
    w = torch.from_numpy(weights if weights is not None else init_weights(seed)).to(dev)
    g = torch.zeros_like(w)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    loss = torch.zeros(1, device=dev)
    n = f_all.shape[0]
    trace = []
    for step in range(1, steps + 1):
        if batch < n:
            idx = torch.from_numpy(rng.choice(n, size=batch, replace=False)).to(dev)
            f, t = f_all.index_select(0, idx).contiguous(), t_all.index_select(0, idx).contiguous()
        else:
            f, t = f_all, t_all
        seismic_mlp_train_step(w, g, m, v, f, t, lr, step, loss)
        if log_every and step % log_every == 0:
            trace.append((step, float(loss.item())))
    torch.cuda.synchronize()
    trace.append((steps, float(loss.item())))
    return w.cpu().numpy(), trace


def predict(weights: np.ndarray, features: np.ndarray):
    """(cut, heap_factor) the device MLP predicts (same mapping as the search)."""
    import torch
    w = torch.from_numpy(np.ascontiguousarray(weights, dtype=np.float32)).cuda()
    f = torch.from_numpy(np.ascontiguousarray(features, dtype=np.float32)).cuda()
    out = torch.empty((f.shape[0], 2), device="cuda")
    seismic_mlp_forward(w, f, out)
    o = out.cpu().numpy().astype(np.float64)
    s = 1.0 / (1.0 + np.exp(-o))
    cut = np.clip(np.rint(CUT_LO + CUT_SPAN * s[:, 0]), 3, 30).astype(np.int64)
    hf = HF_LO + HF_SPAN * s[:, 1]
    return cut, hf


def calibrate(index, weights: np.ndarray, queries: DeviceCSR, gt_scores, k: int, target: float,
              quantized: bool, base_params=None, margin: float = 0.005, max_shift: float = 12.0, iters: int = 12):
    """Shifts the output biases (logit units) so that the learned form's mean
    recall on held-out training queries reaches `target + margin`: the cut
    output's bias up by `shift` and the heap_factor output's bias down by the
    same amount (both raise recall: more lists, less skipping); the smallest
    such shift in [0, max_shift] (the least work), found by bisection.  When
    even the largest shift stays below target + margin (the collection's
    recall ceiling is near the target), the goal drops to target + 0.002, or to
    the target itself.
    Returns (weights, shift, recall)."""
    base = dict(base_params or {})
    b3 = MLP_PARAMS - 2
    goal = target + margin

    def run(shift):
        w = weights.copy()
        w[b3] += np.float32(shift)
        w[b3 + 1] -= np.float32(shift)
        seismic_set_mlp(index, w)
        ids, sc = seismic_search(index, queries, search_params(k=k, cut=10, heap_factor=0.8, learned=True,
                                                               max_query_nnz=queries.max_row_nnz, **base))
        return w, float(recall_at_k(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), gt_scores, k).mean())

    w0, r0 = run(0.0)
    if r0 >= goal:
        return w0, 0.0, r0
    whi, rhi = run(max_shift)
    if rhi < goal:
        # the ceiling is close to the target: the largest reachable of a small
        # margin above it and the target itself
        goal = target + 0.002 if rhi >= target + 0.002 else target
        if r0 >= goal:
            return w0, 0.0, r0
        if rhi < goal:
            return whi, max_shift, rhi
    lo, hi, best = 0.0, max_shift, (whi, max_shift, rhi)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        w, r = run(mid)
        if r >= goal:
            hi, best = mid, (w, mid, r)
        else:
            lo = mid
    return best


def fit(index, train_queries: DeviceCSR, host_train_queries, k: int = 10, target: float = 0.9,
        quantized: bool = True, steps: int = 3000, lr: float = 2e-3, seed: int = 0, base_params=None,
        val_frac: float = 0.2, grid_cut=GRID_CUT, grid_hf=GRID_HF, max_shift: float = 12.0,
        standardize_features: bool = False, table=None):
    """Labels (trade-off form), features, training on the first part of the
    training queries, calibration on the rest; installs the network.  With
    `standardize_features` the network trains on standardized features and
    their mean and spread are folded into its first layer afterwards.
    `table`, the grid runs of an earlier call on the same queries, skips the
    labelling runs."""
    if table is None:
        _, _, table = label_queries(index, train_queries, k, target, quantized, grid_cut=grid_cut, grid_hf=grid_hf,
                                    base_params=base_params)
    cut, hf, lab_rec, lab_bytes = lagrangian_labels(table, target)
    feats = seismic_query_features(index, host_train_queries)
    n = host_train_queries.n_rows
    ntr = max(1, int(n * (1.0 - val_frac)))
    tgt = targets_from_labels(cut[:ntr], hf[:ntr])
    if standardize_features:
        mu, sd = standardize(feats[:ntr])
        w, trace = train(((feats[:ntr] - mu) / sd).astype(np.float32), tgt, steps=steps, lr=lr, seed=seed)
        w = fold_input_scaling(w, mu, sd)
    else:
        w, trace = train(feats[:ntr], tgt, steps=steps, lr=lr, seed=seed)
    val_host = host_train_queries.slice(ntr, n)
    val = DeviceCSR.from_host(val_host)
    _, gt_val = seismic_search_exact(index, val, k)
    w, shift, val_rec = calibrate(index, w, val, gt_val.cpu().numpy(), k, target, quantized, base_params,
                                  max_shift=max_shift)
    seismic_set_mlp(index, w)
    return dict(weights=w, trace=trace, label_cut=cut, label_hf=hf, label_recall=lab_rec, label_bytes=lab_bytes,
                table=table, features=feats, calib_shift=shift, val_recall=val_rec)

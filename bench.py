#!/usr/bin/env python
"""Benchmark of batched Seismic search on GB300: QPS at recall@10 >= 0.9.

A step is one pass of the whole query path (list selection, summary scoring,
block ordering, skipping, forward-index scoring, top-k, kappa-NN expansion
where the workload has a graph) over the batch of synthetic queries, with the
index and the queries resident in HBM.  The operating point is the fastest
(cut, heap_factor) of the workload's grid whose mean recall@10 against the
exact top-10 (computed on the device by brute force) is >= 0.9; when no point
of the configured grid reaches it, larger cuts are added (and said so).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3] [--impl reference]

Default workload: 8.8M documents (about 1.06B nonzeros), kappa = 10, 10k
queries.  Prints one JSON line.  Under torchrun each rank holds a full replica
and searches the full batch (the path does not shard); `value` is all ranks'
queries over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID_HF = (0.6, 0.7, 0.8, 0.9)
WORKLOADS = {
    # the tiny configuration: fp32 summaries, fixed (cut, heap_factor)
    "c1": dict(desc="Seismic 100k docs, vocab 30522, lambda=2000, beta=100, alpha=0.4, fp32 summaries, "
                    "1k queries (lognormal nnz), k=10", n_docs=100_000, n_q=1000, uneven=False, lam=2000,
               beta=100, alpha=0.4, quant=False, cuts=(10,), hfs=(0.8,), kappa=0, cpu_sample=1000, ref_point=(10, 0.8)),
    # the batched configuration: 1M documents, the configured sweep
    "c2": dict(desc="Seismic 1M docs, vocab 30522, lambda=6000, beta=400, alpha=0.4, u8 summaries, "
                    "10k queries (uniform nnz 10-150), k=10, grid cut {5,10,20} x hf {0.6..0.9}",
               n_docs=1_000_000, n_q=10_000, uneven=True, lam=6000, beta=400, alpha=0.4, quant=True,
               cuts=(5, 10, 20), hfs=GRID_HF, kappa=0, cpu_sample=200, n_train=20_000,
               serve_rates=(5_000, 50_000, 100_000, 200_000), ref_point=(5, 0.9)),
    # the c2 shape at 300k documents and 2k queries: small enough for multi-pass ncu captures
    "c2s": dict(desc="Seismic 300k docs, vocab 30522, lambda=6000, beta=400, alpha=0.4, u8 summaries, "
                     "2k queries (uniform nnz 10-150), k=10, cut=5, heap_factor=0.9", n_docs=300_000, n_q=2000,
                uneven=True, lam=6000, beta=400, alpha=0.4, quant=True, cuts=(5,), hfs=(0.9,), kappa=0,
                cpu_sample=100, n_train=4000, serve_rates=(20_000, 200_000), ref_point=(5, 0.9)),
    # the full-scale shape (the headline): kappa-NN graph, learned parameters and serving on it
    "c3": dict(desc="Seismic 8.8M docs (~1.06B nnz), vocab 30522, lambda=6000, beta=400, alpha=0.4, u8 summaries, "
                    "kappa=10, 10k queries (uniform nnz 10-150), k=10", n_docs=8_800_000, n_q=10_000, uneven=True,
               lam=6000, beta=400, alpha=0.4, quant=True, cuts=(5, 10, 20), hfs=GRID_HF, extra_cuts=(30, 40),
               kappa=10, graph=dict(cut=10, heap_factor=0.9, refine=1), cpu_sample=100, n_train=200_000,
               label_cuts=(5, 10, 15, 20, 25, 30), label_hfs=(0.6, 0.7, 0.8, 0.9, 1.0),
               fine_cuts=(10, 15, 20, 25, 30), serve_rates=(5_000, 25_000, 50_000, 100_000), compact=True,
               ref_point=(30, 0.9)),
}
DEFAULT_WORKLOAD = "c3"
RECALL_TARGET = 0.9
K = 10
METRIC = "QPS at recall@10>=0.9 (batched Seismic search, fixed parameters)"
# DRAM traffic of k_search per byte it executes (read + write), from one ncu capture of the current
# kernel on the 300k-document workload (fp32 rows, wave 8), keyed by the L2 row prefetch (which
# brings whole rows in); used to estimate a full launch's traffic from its executed bytes.  A form
# without a capture of the current kernel reports null.
TRAFFIC_PER_EXEC_BYTE = {False: (14.940076544e9 + 0.615757056e9) / 24.652337535e9,
                         True: (19.571495424e9 + 0.855928576e9) / 24.652337535e9}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev, self.proc, self.lines = dev, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0=None, t1=None):
        """Summary of the samples taken in [t0, t1] (all samples if none fall there)."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for ts, ln in self.lines if t0 is not None and t0 <= ts <= t1]
        for ln in (inside or [ln for _, ln in self.lines]):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value over all ranks (the slowest rank's time); x itself
    when there is one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_qps(world: int, queries_per_rank: int, ms_slowest: float) -> float:
    """Whole-job throughput: every rank searches its own full batch (replicas),
    so the job answers world x queries_per_rank queries in the slowest rank's time."""
    return world * queries_per_rank / ms_slowest * 1e3


def make_data(w, seed=0):
    import synth
    t = time.time()
    docs = synth.docs(w["n_docs"], seed=seed)
    queries = synth.queries(w["n_q"], seed=seed, uneven=w["uneven"])
    log(f"data: {docs.n_rows} docs / {docs.nnz} nnz, {queries.n_rows} queries in {time.time() - t:.1f}s")
    return docs, queries


def sample_rows(w, queries):
    """The query sample the oracle runs on (parity and CPU baseline): seeded, spread over the batch."""
    rng = np.random.default_rng(7)
    n = min(w["cpu_sample"], queries.n_rows)
    return np.sort(rng.choice(queries.n_rows, n, replace=False))


def oracle_on_sample(w, docs, queries, cut, threads):
    """The oracle's index lists that a cut-limited search of the sample
    traverses (built untimed), with the sample itself."""
    import oracle
    qs = sample_rows(w, queries)
    sub = queries.take(qs)
    t = time.time()
    terms = oracle.query_list_terms(sub, cut)
    ox = oracle.Index(docs, w["lam"], w["beta"], w["alpha"], w["quant"], seed=0, threads=threads, terms=terms)
    log(f"oracle: lists for {len(terms)} terms built in {time.time() - t:.1f}s")
    return qs, sub, ox


def cpu_baseline(w, ox, sub, cut, hf, threads, knn=None, steps=1):
    """The oracle, as it stands, on the host cores: sequential Seismic search
    (one query per thread) over a bounded sample of the workload's queries."""
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        ox.search(sub, K, cut=cut, heap_factor=float(np.float32(hf)), knn=knn, threads=threads)
        times.append(time.perf_counter() - t0)
    qps = sub.n_rows / float(np.median(times))
    # the paper's protocol: one thread, mean time per query (a smaller sample)
    n1 = max(1, min(sub.n_rows, 20))
    t0 = time.perf_counter()
    ox.search(sub.slice(0, n1), K, cut=cut, heap_factor=float(np.float32(hf)), knn=knn, threads=1)
    us1 = (time.perf_counter() - t0) / n1 * 1e6
    stage = "with the kappa-NN expansion over the library's graph (input data, built untimed)" if knn is not None \
        else "without the kappa-NN stage"
    return {"value": qps, "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": f"{sub.n_rows} of the workload's queries (seeded sample), cut={cut}, heap_factor={hf}, "
                      f"{stage}, one query per thread; lists built untimed", "times_s": times,
            "single_thread_us_per_query": us1, "single_thread_sample": n1}


def sample_parity(w, sz, ix, docs, sub, qs, ox, gt_ids, gt_sc, ids, sc, cut, hf, knn_graph, n_nodes=100):
    """Full-size parity on sampled outputs, against the oracle: the device's
    exact top-10 (the recall judge) and the timed configuration's returned
    scores on the sample, the oracle's recall beside the device's at the same
    parameters (same graph), and the kappa-NN graph on a sample of nodes."""
    import oracle
    t = time.time()
    ei, es = oracle.exact_topk(docs, sub, K)
    gi = gt_ids[qs].view(np.uint32)
    gs = gt_sc[qs].astype(np.float64)
    qi = np.repeat(np.arange(len(qs), dtype=np.uint64), K)
    ex = oracle.pair_dots(docs, sub, qi, gi.reshape(-1)).reshape(gi.shape)
    rel_exact = float(np.max(np.abs(gs - ex) / np.maximum(np.abs(ex), 1e-30)))
    same = gi == ei
    tie_ok = bool(np.all(same | (np.abs(ex - es) <= 2e-5 * np.abs(es))))
    ri = ids[qs].view(np.uint32)
    valid = ri != oracle.NONE_ID
    rs = oracle.pair_dots(docs, sub, qi[valid.reshape(-1)], ri[valid])
    rel_search = float(np.max(np.abs(sc[qs][valid] - rs) / np.maximum(np.abs(rs), 1e-30), initial=0.0))
    ref = ox.search(sub, K, cut=cut, heap_factor=float(np.float32(hf)), knn=knn_graph)
    r_or = float(oracle.recall_at_k(docs, sub, ref["ids"], es, K).mean())
    r_gpu = float(oracle.recall_at_k(docs, sub, ri, es, K).mean())
    out = {"queries": int(len(qs)), "exact_ids_equal": float(same.mean()), "exact_ties_only": tie_ok,
           "exact_max_rel_err": rel_exact, "search_scores_max_rel_err": rel_search,
           "recall_oracle": r_or, "recall_gpu": r_gpu, "cut": cut, "heap_factor": hf}
    if w["kappa"]:
        rng = np.random.default_rng(8)
        nodes = np.sort(rng.choice(docs.n_rows, min(n_nodes, docs.n_rows), replace=False))
        ni, _ = oracle.exact_topk(docs, docs.take(nodes), w["kappa"] + 1)
        g = knn_graph[nodes]
        rec = []
        for r, row in enumerate(ni):
            truth = [x for x in row if x != nodes[r]][: w["kappa"]]
            rec.append(len(set(truth) & set(g[r].tolist())) / w["kappa"])
        out["knn_nodes"] = int(len(nodes))
        out["knn_graph_exact_fraction"] = float(np.mean(rec))
        out["knn_self_loops"] = int(np.sum(g == nodes[:, None]))
    out["seconds"] = time.time() - t
    log(f"sample parity: {out}")
    return out


def graph_exactness(sz, ix, docs, kappa, n_nodes=1000):
    """Fraction of the exact neighbours (device brute force) the graph holds on sampled nodes."""
    rng = np.random.default_rng(5)
    nodes = np.sort(rng.choice(docs.n_rows, min(n_nodes, docs.n_rows), replace=False))
    ni, _ = sz.seismic_search_exact(ix, docs.take(nodes), kappa + 1)
    g = sz.seismic_get_knn(ix)[nodes]
    rec = [len(set([x for x in row if x != nodes[r]][:kappa]) & set(g[r].tolist())) / kappa
           for r, row in enumerate(ni)]
    return float(np.mean(rec))


def learned_eval(args, w, sz, ix, dq, gt_sc, stream, time_runs, launch):
    """Trains the per-query parameter MLP on separate synthetic training
    queries (labels from the method's own runs), then measures the learned form
    on the benchmark's queries against the fixed form at equal recall."""
    import torch
    import synth
    from paper_2509_24815_gb300 import learn, metrics
    t = time.time()
    tq = synth.queries(w["n_train"], seed=0, uneven=w["uneven"], stream=synth.TRAIN_STREAM)
    dtq = sz.DeviceCSR.from_host(tq)
    base = dict(launch, use_knn=bool(w["kappa"]))
    kw = {}
    if "label_cuts" in w:
        kw = dict(grid_cut=w["label_cuts"], grid_hf=w["label_hfs"])
    res = learn.fit(ix, dtq, tq, k=K, target=args.learn_target, quantized=w["quant"], steps=3000, base_params=base,
                    **kw)
    t_fit = time.time() - t
    log(f"learned: labels + training on {tq.n_rows} queries in {t_fit:.1f}s, final loss {res['trace'][-1][1]:.4f}, "
        f"calibration shift {res['calib_shift']:.2f}")
    del dtq

    def measure(**kw_):
        p = sz.search_params(k=K, max_query_nnz=dq.max_row_nnz, **base, **kw_)
        ids, sc = sz.seismic_search(ix, dq, p)
        torch.cuda.synchronize()
        rec = float(metrics.recall_at_k(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), gt_sc, K).mean())
        for _ in range(2):
            sz.seismic_search(ix, dq, p, stream=stream)
        ms = float(np.median(time_runs(p, max(3, min(args.steps, 5)))))
        return dict(recall=rec, ms=ms, qps=dq.n_rows / ms * 1e3)

    lr = measure(cut=10, heap_factor=0.8, learned=True)
    fine = []
    for cut in w.get("fine_cuts", (3, 4, 5, 6, 8, 10)):
        for hf in (0.6, 0.7, 0.8, 0.9, 1.0):
            fine.append(dict(cut=cut, heap_factor=hf, **measure(cut=cut, heap_factor=hf)))
    at = [f for f in fine if f["recall"] >= lr["recall"] - 1e-9]
    ref = max(at, key=lambda f: f["qps"]) if at else max(fine, key=lambda f: f["recall"])
    # the fixed form's recall/QPS frontier, interpolated linearly at the learned recall
    front = sorted(fine, key=lambda f: f["recall"])
    front = [f for i, f in enumerate(front) if all(g["qps"] < f["qps"] for g in front[i + 1:])]
    interp = None
    for f0, f1 in zip(front, front[1:]):
        if f0["recall"] <= lr["recall"] <= f1["recall"]:
            t = (lr["recall"] - f0["recall"]) / max(f1["recall"] - f0["recall"], 1e-12)
            interp = f0["qps"] + t * (f1["qps"] - f0["qps"])
    log(f"learned: recall {lr['recall']:.4f} at {lr['qps']:,.0f} q/s; best fixed at >= that recall: "
        f"cut={ref['cut']} hf={ref['heap_factor']} recall {ref['recall']:.4f} at {ref['qps']:,.0f} q/s; "
        f"fixed frontier at that recall: {interp if interp is None else round(interp)} q/s")
    return {"value": lr["qps"], "unit": "queries/s", "recall@10": lr["recall"], "ms_per_step": lr["ms"],
            "fixed_at_equal_recall": ref, "qps_gain_vs_fixed": lr["qps"] / ref["qps"],
            "fixed_frontier_qps_at_learned_recall": interp,
            "qps_gain_vs_fixed_frontier": (lr["qps"] / interp) if interp else None,
            "train_queries": int(tq.n_rows * 0.8), "calibration_queries": tq.n_rows - int(tq.n_rows * 0.8),
            "evaluated_on": f"the benchmark's {dq.n_rows} queries (a stream disjoint from the training queries)",
            "label_grid": {"cut": list(kw.get("grid_cut", learn.GRID_CUT)), "hf": list(kw.get("grid_hf", learn.GRID_HF))},
            "label_target_recall": args.learn_target, "fit_seconds": t_fit,
            "final_loss": res["trace"][-1][1], "label_mean_recall": res["label_recall"],
            "label_mean_bytes_per_query": res["label_bytes"],
            "label_grid_bytes_per_query": {f"cut={c} hf={h}": float(np.mean(b)) for c, h, _, b in res["table"]},
            "label_grid_recall": {f"cut={c} hf={h}": float(np.mean(r)) for c, h, r, _ in res["table"]},
            "calibration_shift": res["calib_shift"], "validation_recall": res["val_recall"],
            "fixed_fine_grid": fine}


def serving_eval(args, w, sz, ix, best, learned, launch):
    """Poisson arrivals replayed through the continuous-batching server:
    p50/p99 latency (arrival to results on the host) and achieved QPS per
    offered rate, with recall@10 of the served k=10 requests."""
    import synth
    from paper_2509_24815_gb300 import metrics, serve
    sp = sz.search_params(cut=best["cut"], heap_factor=best["heap_factor"], learned=learned,
                          use_knn=bool(w["kappa"]), **launch)
    srv = sz.Server(ix, sp, max_batch=1024, streams=16, max_query_nnz=160)
    out = []
    for rate in w["serve_rates"]:
        n = int(min(20_000, max(2_000, rate * 2.0)))
        q = synth.queries(n, seed=0, uneven=True, stream=synth.SERVE_STREAM)
        ids, sc, kq, summ = serve.run_trace(ix, q, rate, search=sp, server=srv)
        gi, gs = sz.seismic_search_exact(ix, q, K)
        m10 = kq == 10
        rec = metrics.recall_at_k(ids[m10][:, :K], sc[m10][:, :K], gs[m10], K).mean() if m10.any() else None
        summ["recall@10_k10_requests"] = float(rec) if rec is not None else None
        out.append(summ)
        log(f"serving {rate:>9,.0f} q/s offered: achieved {summ['achieved_qps']:,.0f} q/s, "
            f"p50 {summ['p50_ms']:.3f} ms, p99 {summ['p99_ms']:.3f} ms, recall@10 {summ['recall@10_k10_requests']:.4f}")
    srv.close()
    return {"params": ("learned (fixed fallback)" if learned else "fixed") + (", kappa-NN expansion" if w["kappa"] else ""),
            "rates": out}


def compact_eval(args, w, sz, docs, dq, gt32, graph, point, launch, stream, time_runs_ix):
    """The 16-bit forward-value form (Section 5.4's setup) at the operating
    point: an index of the fp16-rounded collection with the same graph, its
    bytes per query, QPS, and recall against both the rounded collection's and
    the fp32 collection's exact top-10."""
    import torch
    from paper_2509_24815_gb300 import metrics
    t = time.time()
    ix16 = sz.seismic_build(docs, lambda_=w["lam"], beta=w["beta"], alpha=w["alpha"], quantize_u8=w["quant"], seed=0,
                            keep_full_lists=True, values_fp16=True)
    torch.cuda.synchronize()
    t_build = time.time() - t
    _, gt16 = sz.seismic_search_exact(ix16, dq, K)
    gt16 = gt16.cpu().numpy()
    if graph is not None:
        sz.seismic_set_knn(ix16, graph)
    info = sz.seismic_info(ix16)
    p = sz.search_params(k=K, cut=point["cut"], heap_factor=point["heap_factor"], use_knn=bool(w["kappa"]),
                         max_query_nnz=dq.max_row_nnz, **launch)
    ids, sc, st = sz.seismic_search(ix16, dq, p, stats=True)
    torch.cuda.synchronize()
    i_ = ids.cpu().numpy().view(np.uint32)
    s_ = sc.cpu().numpy()
    r16 = float(metrics.recall_at_k(i_, s_, gt16, K).mean())
    r32 = float(metrics.recall_at_k(i_, s_, gt32, K).mean())
    for _ in range(2):
        sz.seismic_search(ix16, dq, p, stream=stream)
    ms = float(np.median(time_runs_ix(ix16, p, max(3, min(args.steps, 10)))))
    by = float(metrics.algorithmic_bytes(st, K, w["quant"], w["kappa"], fp16=True, knn_bits=info["knn_bits"]).mean())
    ix16.close()
    out = {"values": "fp16", "build_s": t_build, "device_gib": info["device_bytes"] / 2**30,
           "qps": dq.n_rows / ms * 1e3, "ms_per_step": ms, "recall@10_vs_rounded_collection": r16,
           "recall@10_vs_fp32_collection": r32, "bytes_per_query": by, "cut": point["cut"],
           "heap_factor": point["heap_factor"]}
    log(f"fp16 rows: {out}")
    return out


def run_reference(args, w):
    """The reference arm: the oracle timed on the host cores, at the workload's
    declared operating point, on a bounded sample of its queries."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    docs, queries = make_data(w)
    cut, hf = w["ref_point"]
    threads = os.cpu_count() or 1
    qs, sub, ox = oracle_on_sample(w, docs, queries, cut, threads)
    cb = cpu_baseline(w, ox, sub, cut, hf, threads, steps=max(1, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"],
            "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.median(cb["times_s"])), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "cut": cut, "heap_factor": hf, "k": K,
                       "queries_per_step": queries.n_rows, "sample_per_step": int(sub.n_rows)},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--group", type=int, default=1, help="1: chunk-flattened scoring, 8/16/32: lane groups")
    ap.add_argument("--cta-warps", type=int, default=0)
    ap.add_argument("--wave", type=int, default=16)
    ap.add_argument("--persistent", type=int, default=1)
    ap.add_argument("--shape", type=int, default=1, help="1 (or 0): CTA per query, 2: warp per query")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-compact", action="store_true", help="skip the fp16 forward-value form")
    ap.add_argument("--no-parity", action="store_true", help="skip the sampled oracle parity")
    ap.add_argument("--learn-target", type=float, default=0.9)
    ap.add_argument("--prefetch", type=int, default=0, help="TMA L2 prefetch of the wave's rows (when not autotuned)")
    ap.add_argument("--autotune", type=int, default=1, help="tune the launch configuration at the operating point")
    ap.add_argument("--graph", type=int, default=1, help="time the step as a CUDA graph replay")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    import paper_2509_24815_gb300 as sz
    from paper_2509_24815_gb300 import autotune, metrics

    t_all = time.time()
    os.environ.setdefault("SEISMIC_BUILD_TRACE", "1")  # the index build's phase times go to the log
    docs, queries = make_data(w)
    t = time.time()
    ix = sz.seismic_build(docs, lambda_=w["lam"], beta=w["beta"], alpha=w["alpha"], quantize_u8=w["quant"], seed=0,
                          keep_full_lists=True)
    torch.cuda.synchronize()
    t_build = time.time() - t
    info = sz.seismic_info(ix)
    log(f"build {t_build:.1f}s; index {info['device_bytes'] / 2**30:.2f} GiB on device, "
        f"{info['n_blocks']} blocks, {info['n_summary_entries']} summary entries")
    dq = sz.DeviceCSR.from_host(queries)
    t = time.time()
    gt_ids, gt_sc = sz.seismic_search_exact(ix, dq, K)
    torch.cuda.synchronize()
    gt_ids, gt_sc = gt_ids.cpu().numpy(), gt_sc.cpu().numpy()
    log(f"exact top-{K} (device brute force) in {time.time() - t:.1f}s")
    graph_rep, knn_graph = None, None
    if w["kappa"]:
        gcfg = w["graph"]
        t = time.time()
        sz.seismic_build_knn(ix, w["kappa"], sz.search_params(k=w["kappa"] + 1, cut=gcfg["cut"],
                                                              heap_factor=gcfg["heap_factor"], shape=1, group=1,
                                                              wave=16, persistent=True))
        torch.cuda.synchronize()
        graph_rep = {"search": {"cut": gcfg["cut"], "heap_factor": gcfg["heap_factor"]},
                     "stages": [{"stage": "search", "s": time.time() - t, "exact_fraction": graph_exactness(
                         sz, ix, docs, w["kappa"])}]}
        for r in range(gcfg["refine"]):
            t = time.time()
            sz.seismic_refine_knn(ix, 1)
            torch.cuda.synchronize()
            graph_rep["stages"].append({"stage": f"refine {r + 1}", "s": time.time() - t,
                                        "exact_fraction": graph_exactness(sz, ix, docs, w["kappa"])})
        graph_rep["bits_per_id"] = sz.seismic_info(ix)["knn_bits"]
        graph_rep["bytes"] = sz.seismic_info(ix)["knn_bytes"]
        knn_graph = sz.seismic_get_knn(ix)
        log(f"kappa-NN graph: {graph_rep}")

    stream = torch.cuda.Stream()
    ids = torch.empty((dq.n_rows, K), dtype=torch.int32, device="cuda")
    sc = torch.empty((dq.n_rows, K), dtype=torch.float32, device="cuda")

    def params(cut, hf, **kw):
        base = dict(k=K, cut=cut, heap_factor=hf, use_knn=bool(w["kappa"]), wave=args.wave, group=args.group,
                    cta_warps=args.cta_warps, persistent=bool(args.persistent), max_query_nnz=dq.max_row_nnz,
                    shape=args.shape, no_prefetch=not args.prefetch)
        base.update(kw)
        return sz.search_params(**base)

    def run(p, index=None):
        sz.seismic_search(index or ix, dq, p, ids_out=ids, scores_out=sc, stream=stream)

    def time_runs(p, n, fn=None, index=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n)]
        with torch.cuda.stream(stream):
            for i in range(n):
                ev[2 * i].record(stream)
                if fn is None:
                    run(p, index)
                else:
                    fn()
                ev[2 * i + 1].record(stream)
        stream.synchronize()
        return [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(n)]

    def recall_now():
        return float(metrics.recall_at_k(ids.cpu().numpy().view(np.uint32), sc.cpu().numpy(), gt_sc, K).mean())

    # operating point: the fastest grid point reaching the recall target
    grid = []

    def sweep(cuts):
        for cut in cuts:
            for hf in w["hfs"]:
                p = params(cut, hf)
                run(p)
                stream.synchronize()
                rec = recall_now()
                ms = float(np.median(time_runs(p, 2)))
                grid.append(dict(cut=cut, heap_factor=hf, recall=rec, ms=ms, qps=dq.n_rows / ms * 1e3))
                log(f"  cut={cut:2d} hf={hf:.1f}: recall@10 {rec:.4f}  {ms:7.2f} ms  {grid[-1]['qps']:,.0f} q/s")

    sweep(w["cuts"])
    extended = None
    if not any(g["recall"] >= RECALL_TARGET for g in grid) and w.get("extra_cuts"):
        extended = list(w["extra_cuts"])
        log(f"no configured grid point reaches recall {RECALL_TARGET}: adding cuts {extended}")
        sweep(extended)
    ok = [g for g in grid if g["recall"] >= RECALL_TARGET]
    best = max(ok, key=lambda g: g["qps"]) if ok else max(grid, key=lambda g: g["recall"])
    launch = dict(shape=args.shape, group=args.group, cta_warps=args.cta_warps, wave=args.wave,
                  persistent=bool(args.persistent), no_prefetch=not args.prefetch)
    p = params(best["cut"], best["heap_factor"])
    tuned = None
    if args.autotune:
        # launch configuration (kernel shape, lane group, warps, wave, prefetch) at the operating point
        base = dict(k=K, cut=best["cut"], heap_factor=best["heap_factor"], use_knn=bool(w["kappa"]))
        floor = min(RECALL_TARGET, best["recall"])

        def rec_fn(i, s):
            return metrics.recall_at_k(i.cpu().numpy().view(np.uint32), s.cpu().numpy(), gt_sc, K).mean()
        kw, table = autotune.autotune(ix, dq, base, recall_fn=rec_fn, min_recall=floor, stream=stream, log=log)
        launch = {x: kw[x] for x in launch}
        p = sz.search_params(max_query_nnz=dq.max_row_nnz, **dict(base, **launch))
        run(p)
        stream.synchronize()
        best["recall"] = recall_now()
        tuned = {"chosen": launch, "candidates": len(table),
                 "table": [{x: t.get(x) for x in ("shape", "group", "cta_warps", "wave", "no_prefetch", "ms",
                                                   "recall")} for t in table]}
        log(f"autotune: {launch}, recall@10 {best['recall']:.4f}")

    # the method's bytes: the work counters of the sequential visiting order (wave 1) at the operating
    # point; the kernel's executed bytes: the same counters at the timed wave
    kbits = info["knn_bits"] if not w["kappa"] else sz.seismic_info(ix)["knn_bits"]
    p1 = sz.search_params(max_query_nnz=dq.max_row_nnz, **dict(k=K, cut=best["cut"], heap_factor=best["heap_factor"],
                                                              use_knn=bool(w["kappa"]), **dict(launch, wave=1)))
    _, _, st1 = sz.seismic_search(ix, dq, p1, stats=True)
    alg_bytes = float(metrics.algorithmic_bytes(st1, K, w["quant"], w["kappa"], knn_bits=kbits).sum())
    _, _, stw = sz.seismic_search(ix, dq, p, stats=True)
    exec_bytes = float(metrics.algorithmic_bytes(stw, K, w["quant"], w["kappa"], knn_bits=kbits).sum())
    slots = 152 * 5 if launch["shape"] != 2 else 152 * 16
    occupancy = metrics.queue_occupancy(stw, slots)
    log(f"bytes per launch: method (wave 1) {alg_bytes / 1e9:.2f} GB, executed (wave {launch['wave']}) "
        f"{exec_bytes / 1e9:.2f} GB; queue occupancy {occupancy}")

    for _ in range(args.warmup):
        run(p)
    stream.synchronize()
    step, graph_note = (lambda: run(p)), "direct launches"
    if args.graph:
        # the whole step (queue reset, work-queue order, search, expansion) as one CUDA graph
        g = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
                run(p)
            stream.synchronize()
            step, graph_note = g.replay, "CUDA graph replay"
            for _ in range(args.warmup):
                with torch.cuda.stream(stream):
                    step()
            stream.synchronize()
        except Exception as e:  # capture unsupported here: direct launches of the same kernels
            graph_note = f"direct launches (graph capture failed: {e})"
            log(graph_note)
    # the clock sampler starts (and finishes initialising) before the warm-up
    # steps, so it never competes with the timed launches
    clocks = Clocks(local)
    clocks.start()
    time.sleep(1.0)
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            step()
    stream.synchronize()
    barrier()
    torch.cuda.synchronize()
    t_timed = time.time()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly the timed launches
    per = time_runs(p, args.steps, step)  # events bracket each step on its stream
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop(t_timed, time.time())
    ms_step = max_over_ranks(float(np.mean(per)), dist, "cuda")
    qps = job_qps(world, dq.n_rows, ms_step)

    # end to end through the public call with host buffers (pinned), copies inside the timed region
    pin = {f: torch.from_numpy(np.ascontiguousarray(getattr(queries, f))).pin_memory()
           for f in ("indptr", "terms", "vals")}
    hq = type(queries)(pin["indptr"].numpy(), pin["terms"].numpy(), pin["vals"].numpy(), queries.dim)
    hid = torch.empty((queries.n_rows, K), dtype=torch.int32).pin_memory()
    hsc = torch.empty((queries.n_rows, K), dtype=torch.float32).pin_memory()
    pe = sz.search_params(k=K, cut=best["cut"], heap_factor=best["heap_factor"], use_knn=bool(w["kappa"]), **launch)
    for _ in range(2):
        sz.seismic_search(ix, hq, pe, ids_out=hid, scores_out=hsc, stream=stream)
    e2e_t = []
    for _ in range(max(3, args.steps)):
        t0 = time.perf_counter()
        sz.seismic_search(ix, hq, pe, ids_out=hid, scores_out=hsc, stream=stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_qps = job_qps(world, queries.n_rows, 1e3 * max_over_ranks(float(np.median(e2e_t)), dist, "cuda"))
    h2d = queries.indptr.nbytes + queries.terms.nbytes + queries.vals.nbytes
    d2h = hid.numel() * 4 + hsc.numel() * 4

    # kernels per step: the search, plus the work-queue order (keys, sort) ahead of a persistent launch
    launches_per_step = 1 + (2 if (launch["persistent"] or launch["shape"] == 2) and dq.n_rows > 1 else 0)
    peak, peak_kind = peaks()
    sec = float(np.mean(per)) * 1e-3
    achieved = alg_bytes / sec / 1e9  # this rank's kernel, per launch
    ratio = TRAFFIC_PER_EXEC_BYTE.get(not launch["no_prefetch"]) if launch["shape"] != 2 else None
    traffic = ratio * exec_bytes if ratio else None
    line = {
        "metric": METRIC,
        "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["desc"], "cut": best["cut"], "heap_factor": best["heap_factor"],
                   "recall@10": best["recall"], "queries_per_step": dq.n_rows, "k": K,
                   "l2": "index resident in HBM, larger than L2 (no flush)", **launch,
                   "launch": graph_note, "parallelism": f"replicas x{world}",
                   "grid_extended_with_cuts": extended},
        "grid": grid,
        "autotune": tuned,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_kind, "kernel": "k_search",
                     "alg_bytes_per_launch": alg_bytes, "alg_bytes_basis": "work counters of the sequential "
                     "visiting order (wave 1) at the operating point",
                     "executed_bytes_per_launch": exec_bytes, "executed_frac": exec_bytes / sec / 1e9 / peak,
                     "traffic_basis": ("ncu DRAM bytes per executed byte on the 300k-document workload (same "
                                       "prefetch setting), scaled by this launch's executed bytes") if traffic else None,
                     "traffic_over_alg": (traffic / alg_bytes) if traffic else None},
        "queue_occupancy": occupancy,
        "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": args.steps * launches_per_step,
        "clocks": clk,
        "index": {**{k: info[k] for k in ("n_docs", "nnz", "n_postings", "n_blocks", "n_summary_entries",
                                          "device_bytes")}, "build_s": t_build},
        "knn_graph": graph_rep,
    }
    run(p)
    stream.synchronize()
    ids_h, sc_h = ids.cpu().numpy(), sc.cpu().numpy()
    threads = os.cpu_count() or 1
    ox = sub = qs = None
    if rank == 0 and world == 1 and not (args.no_parity and args.no_cpu_baseline):
        qs, sub, ox = oracle_on_sample(w, docs, queries, best["cut"], threads)
    if ox is not None and not args.no_parity:
        line["parity_sample"] = sample_parity(w, sz, ix, docs, sub, qs, ox, gt_ids, gt_sc, ids_h, sc_h, best["cut"],
                                              best["heap_factor"], knn_graph)
    if ox is not None and not args.no_cpu_baseline:
        cb = cpu_baseline(w, ox, sub, best["cut"], best["heap_factor"], threads, knn=knn_graph)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                   "single_thread_us_per_query", "single_thread_sample")}
    del ox
    extras = world == 1  # the scaling runs report the timed throughput only
    if extras and not args.no_compact and w.get("compact"):
        line["compact"] = compact_eval(args, w, sz, docs, dq, gt_sc, knn_graph, best, launch, stream,
                                       lambda index, p_, n: time_runs(p_, n, index=index))
    if extras and not args.no_learned and w.get("n_train"):
        line["learned"] = learned_eval(args, w, sz, ix, dq, gt_sc, stream, time_runs, launch)
    if extras and not args.no_serve and w.get("serve_rates"):
        line["serving"] = serving_eval(args, w, sz, ix, best, bool(line.get("learned")), launch)
    line["bench_seconds"] = time.time() - t_all
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

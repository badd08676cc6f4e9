"""ORACLE -- test infrastructure only.

Plain fp64 CPU statement of the Seismic method (arXiv 2509.24815), in
``oracle.c``: exact top-k (Definition SMIPS), alpha-MSS (Section 3.2), the
indexing algorithm (Section 4.4), the exact kappa-NN graph (Eq. knn-graph) and
the query-processing algorithm (Section 4.5).  Only ``tests/``, the smoke check
and the benchmark's CPU-baseline leg may import this package.  It shares no
code with the GPU library; its inputs come from ``synth`` only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None
NONE_ID = 0xFFFFFFFF
STAT_NAMES = ("lists", "blocks_scored", "blocks_evaluated", "blocks_skipped", "docs", "doc_nnz",
              "knn_docs", "summary_entries")


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` (plain C, fp64, no contraction of multiply-adds)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, u64, u32, dbl, ci = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_double, ctypes.c_int)
            lib.or_exact_topk.argtypes = [vp, vp, vp, u64, u32, vp, vp, vp, u64, u32, ci, vp, vp]
            lib.or_alpha_mss.argtypes = [vp, vp, u32, dbl, vp]
            lib.or_alpha_mss.restype = u32
            lib.or_splitmix64.argtypes = [vp]
            lib.or_splitmix64.restype = u64
            lib.or_build.argtypes = [vp, vp, vp, u64, u32, u32, dbl, u32, dbl, dbl, ci, u64, ci]
            lib.or_build.restype = vp
            lib.or_build_masked.argtypes = [vp, vp, vp, u64, u32, u32, dbl, u32, dbl, dbl, ci, u64, ci, vp]
            lib.or_build_masked.restype = vp
            lib.or_free.argtypes = [vp]
            lib.or_list_sizes.argtypes = [vp, u32, vp]
            lib.or_list_get.argtypes = [vp, u32] + [vp] * 13
            lib.or_knn_exact.argtypes = [vp, vp, vp, u64, u32, u32, ci, vp]
            lib.or_knn_refine.argtypes = [vp, vp, vp, u64, u32, vp, u32, ci, vp]
            lib.or_search.argtypes = [vp, vp, vp, vp, u64, vp, vp, vp, u64, u32, u32, dbl, dbl, ci, ci,
                                      vp, u32, ci, vp, vp, vp, vp]
            lib.or_block_scores.argtypes = [vp, vp, vp, u32, u32, vp]
            lib.or_pair_dots.argtypes = [vp, vp, vp, u64, u32, vp, vp, vp, u64, vp, vp, u64, vp]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _csr_args(m):
    ip = np.ascontiguousarray(m.indptr, dtype=np.uint64)
    t = np.ascontiguousarray(m.terms, dtype=np.uint16)
    v = np.ascontiguousarray(m.vals, dtype=np.float32)
    return (ip, t, v)


def _threads(threads):
    return threads if threads else (os.cpu_count() or 1)


def exact_topk(docs, queries, k: int, threads: int | None = None):
    """Definition SMIPS: the k best documents by (<q,u> desc, id asc), fp64."""
    lib = _load()
    d_ = _csr_args(docs)
    q_ = _csr_args(queries)
    nq = queries.n_rows
    ids = np.empty((nq, k), dtype=np.uint32)
    sc = np.empty((nq, k), dtype=np.float64)
    lib.or_exact_topk(_p(d_[0]), _p(d_[1]), _p(d_[2]), docs.n_rows, docs.dim, _p(q_[0]), _p(q_[1]),
                      _p(q_[2]), nq, k, _threads(threads), _p(ids), _p(sc))
    return ids, sc


def alpha_mss(terms, vals, alpha: float):
    """Definition alpha-MSS: returns (kept count, entry order by |v| desc, term asc)."""
    lib = _load()
    t = np.ascontiguousarray(terms, dtype=np.uint16)
    v = np.ascontiguousarray(vals, dtype=np.float32)
    order = np.empty(len(t), dtype=np.uint32)
    keep = lib.or_alpha_mss(_p(t), _p(v), len(t), float(alpha), _p(order))
    return int(keep), order


def splitmix64(state: int, n: int):
    lib = _load()
    st = np.array([state], dtype=np.uint64)
    return [int(lib.or_splitmix64(_p(st))) for _ in range(n)]


class Index:
    """Handle on an oracle index (Algorithm "Indexing with Seismic")."""

    def __init__(self, docs, lam, beta, alpha, quantize, seed, lambda_frac=0.0, beta_frac=0.0,
                 threads=None, terms=None):
        """``terms``: build only these lists (enough for queries whose traversed
        lists are among them); None builds every list."""
        lib = _load()
        self._keep = _csr_args(docs)
        self.docs = docs
        self.dim = docs.dim
        self.quantize = bool(quantize)
        mask = None
        if terms is not None:
            mask = np.zeros(docs.dim, dtype=np.uint8)
            mask[np.asarray(terms, dtype=np.int64)] = 1
        self._h = lib.or_build_masked(_p(self._keep[0]), _p(self._keep[1]), _p(self._keep[2]), docs.n_rows,
                                      docs.dim, int(lam), float(lambda_frac), int(beta), float(beta_frac),
                                      float(alpha), int(bool(quantize)), int(seed), _threads(threads), _p(mask))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_free(self._h)
            self._h = None

    def list(self, t: int) -> dict:
        """All arrays of list t: postings, centroids, assignment, blocks, summaries."""
        lib = _load()
        sz = np.zeros(4, dtype=np.uint32)
        lib.or_list_sizes(self._h, t, _p(sz))
        n, nc, nb, ns = (int(x) for x in sz)
        out = dict(doc=np.empty(n, np.uint32), val=np.empty(n, np.float32), cent=np.empty(nc, np.uint32),
                   assign=np.empty(n, np.uint32), bcent=np.empty(nb, np.uint32),
                   bptr=np.zeros(nb + 1, np.uint32), bmem=np.empty(n, np.uint32),
                   sptr=np.zeros(nb + 1, np.uint32), sterm=np.empty(ns, np.uint16),
                   sval=np.empty(ns, np.float32), scode=np.empty(ns, np.uint8), qm=np.empty(nb, np.float32),
                   qsz=np.empty(nb, np.float32))
        keys = ("doc", "val", "cent", "assign", "bcent", "bptr", "bmem", "sptr", "sterm", "sval", "scode",
                "qm", "qsz")
        lib.or_list_get(self._h, t, *[_p(out[k_]) for k_ in keys])
        return out

    def block_scores(self, qterms, qvals, t: int):
        """r_b = <q, S_b> for every block of list t (fp64, dequantised summaries)."""
        lib = _load()
        qt = np.ascontiguousarray(qterms, dtype=np.uint16)
        qv = np.ascontiguousarray(qvals, dtype=np.float32)
        nb = len(self.list(t)["bcent"])
        out = np.empty(nb, dtype=np.float64)
        lib.or_block_scores(self._h, _p(qt), _p(qv), len(qt), t, _p(out))
        return out

    def search(self, queries, k, cut=10, heap_factor=0.8, hf_mode=0, exhaustive=False, alpha_q=0.0,
               knn=None, threads=None, want_phase1=False):
        """Algorithm "Query processing with Seismic" (one query at a time, fp64)."""
        lib = _load()
        q_ = _csr_args(queries)
        nq = queries.n_rows
        ids = np.empty((nq, k), dtype=np.uint32)
        sc = np.empty((nq, k), dtype=np.float64)
        st = np.zeros((nq, len(STAT_NAMES)), dtype=np.uint64)
        ph = np.empty((nq, k), dtype=np.uint32) if want_phase1 else None
        kappa = 0
        kn = None
        if knn is not None:
            kn = np.ascontiguousarray(knn, dtype=np.uint32)
            kappa = kn.shape[1]
        lib.or_search(self._h, _p(self._keep[0]), _p(self._keep[1]), _p(self._keep[2]), self.docs.n_rows,
                      _p(q_[0]), _p(q_[1]), _p(q_[2]), nq, k, cut, float(alpha_q), float(heap_factor),
                      hf_mode, int(bool(exhaustive)), _p(kn), kappa, _threads(threads), _p(ids), _p(sc),
                      _p(st), _p(ph))
        res = dict(ids=ids, scores=sc, stats=st)
        if want_phase1:
            res["phase1"] = ph
        return res


def knn_exact(docs, kappa: int, threads=None):
    """Eq. knn-graph, exactly: N(u) = the kappa best v != u by (<u,v> desc, id asc)."""
    lib = _load()
    d_ = _csr_args(docs)
    out = np.empty((docs.n_rows, kappa), dtype=np.uint32)
    lib.or_knn_exact(_p(d_[0]), _p(d_[1]), _p(d_[2]), docs.n_rows, docs.dim, kappa, _threads(threads),
                     _p(out))
    return out


def knn_refine(docs, knn, threads=None):
    """One neighbour-of-neighbour pass: the new N(u) is the kappa best v != u of
    N(u) u N(N(u)) by (<u,v> desc, id asc), fp64 (the expansion step of query
    processing applied to the graph itself)."""
    lib = _load()
    d_ = _csr_args(docs)
    kn = np.ascontiguousarray(knn, dtype=np.uint32)
    out = np.empty_like(kn)
    lib.or_knn_refine(_p(d_[0]), _p(d_[1]), _p(d_[2]), docs.n_rows, docs.dim, _p(kn), kn.shape[1],
                      _threads(threads), _p(out))
    return out


def pair_dots(docs, queries, qidx, didx):
    """fp64 <q_i, u_j> for (qidx[n], didx[n]) pairs; ids past the collection score -inf."""
    lib = _load()
    d_ = _csr_args(docs)
    q_ = _csr_args(queries)
    qi = np.ascontiguousarray(qidx, dtype=np.uint64)
    di = np.ascontiguousarray(didx, dtype=np.uint32)
    out = np.empty(len(qi), dtype=np.float64)
    lib.or_pair_dots(_p(d_[0]), _p(d_[1]), _p(d_[2]), docs.n_rows, docs.dim, _p(q_[0]), _p(q_[1]),
                     _p(q_[2]), queries.n_rows, _p(qi), _p(di), len(qi), _p(out))
    return out


def query_list_terms(queries, cut):
    """The terms whose lists a cut-limited search traverses, per query (value desc, term asc)."""
    out = set()
    for i in range(queries.n_rows):
        t, v = queries.row(i)
        nz = v != 0
        t, v = t[nz], v[nz]
        o = np.lexsort((t, -v))[:cut]
        out.update(int(x) for x in t[o])
    return sorted(out)


def recall_at_k(docs, queries, ids, exact_scores, k: int, rel_tol: float = 1e-6):
    """accuracy@k (Definition ann-accuracy), tie-aware: a returned id is a hit when
    its exact score reaches the exact k-th score minus rel_tol*|k-th|; ids are
    counted once.  Returns the per-query recall."""
    ids = np.asarray(ids)[:, :k]
    nq = ids.shape[0]
    qidx = np.repeat(np.arange(nq, dtype=np.uint64), k)
    flat = ids.reshape(-1).astype(np.uint32)
    s = pair_dots(docs, queries, qidx, flat).reshape(nq, k)
    kth = np.asarray(exact_scores)[:, k - 1]
    thr = kth - rel_tol * np.abs(kth)
    hit = (s >= thr[:, None]) & (ids != NONE_ID)
    out = np.empty(nq)
    for i in range(nq):
        seen = set()
        c = 0
        for j in range(k):
            if hit[i, j] and int(ids[i, j]) not in seen:
                seen.add(int(ids[i, j]))
                c += 1
        out[i] = c / k
    return out

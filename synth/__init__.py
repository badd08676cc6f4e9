"""Seeded synthetic SPLADE-shaped collections and query sets.

The paper evaluates on SPLADE embeddings of MS MARCO (8.8M passages, about
119 nonzeros per passage and 43 per query over a ~30k-term WordPiece
vocabulary, Section 5.1.1-5.1.2).  Those embeddings are not available here;
this module draws stand-ins with the same shape from a latent-topic model
(see ``synth.c``).  It holds none of the search method's arithmetic and is
the only code shared by the oracle and the GPU library's tests/benchmarks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None

VOCAB = 30522


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``_synth.so`` (gcc, portable flags)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u64, u32, dbl, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p
            lib.synth_topics.argtypes = [u64, u32, u32, dbl, vp, vp]
            lib.synth_topics.restype = None
            lib.synth_rows.argtypes = [u64, u64, u64, u32, u32, dbl, dbl, ctypes.c_int, dbl, dbl,
                                       u32, u32, vp, vp, ctypes.c_int, vp, vp, vp, vp]
            lib.synth_rows.restype = None
            _lib = lib
    return _lib


@dataclass
class CSR:
    """Row-major sparse matrix: row i holds terms[indptr[i]:indptr[i+1]] (ascending) and vals."""
    indptr: np.ndarray  # uint64 [n+1]
    terms: np.ndarray   # uint16 [nnz]
    vals: np.ndarray    # float32 [nnz]
    dim: int

    @property
    def n_rows(self) -> int:
        return len(self.indptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def row(self, i):
        a, b = int(self.indptr[i]), int(self.indptr[i + 1])
        return self.terms[a:b], self.vals[a:b]

    def slice(self, lo: int, hi: int) -> "CSR":
        a, b = int(self.indptr[lo]), int(self.indptr[hi])
        return CSR((self.indptr[lo:hi + 1] - self.indptr[lo]).astype(np.uint64),
                   self.terms[a:b].copy(), self.vals[a:b].copy(), self.dim)

    def take(self, rows) -> "CSR":
        rows = np.asarray(rows, dtype=np.int64)
        lens = (self.indptr[rows + 1] - self.indptr[rows]).astype(np.uint64)
        indptr = np.zeros(len(rows) + 1, dtype=np.uint64)
        np.cumsum(lens, out=indptr[1:])
        terms = np.empty(int(indptr[-1]), dtype=np.uint16)
        vals = np.empty(int(indptr[-1]), dtype=np.float32)
        for j, r in enumerate(rows):
            a, b = int(self.indptr[r]), int(self.indptr[r + 1])
            terms[int(indptr[j]):int(indptr[j + 1])] = self.terms[a:b]
            vals[int(indptr[j]):int(indptr[j + 1])] = self.vals[a:b]
        return CSR(indptr, terms, vals, self.dim)

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n_rows, self.dim), dtype=np.float64)
        rows = np.repeat(np.arange(self.n_rows), np.diff(self.indptr.astype(np.int64)))
        out[rows, self.terms.astype(np.int64)] = self.vals
        return out


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def topics(seed: int, d: int = VOCAB, K: int = 64, zipf_s: float = 1.0):
    lib = _load()
    perm = np.empty((K, d), dtype=np.uint16)
    cdf = np.empty(d, dtype=np.float64)
    lib.synth_topics(seed, d, K, zipf_s, _ptr(perm), _ptr(cdf))
    return perm, cdf


def generate(n: int, *, seed: int, stream: int, d: int = VOCAB, K: int = 64, zipf_s: float = 1.0,
             dirichlet: float = 0.1, nnz: tuple = ("lognormal", 120.0, 40.0), nnz_clip=(10, 400),
             threads: int | None = None) -> CSR:
    """Draw ``n`` rows.  ``nnz`` is ("lognormal", mean, sd) in linear space or ("uniform", lo, hi)."""
    if d > 65536:
        raise ValueError("term ids are u16")
    lib = _load()
    perm, cdf = topics(seed, d, K, zipf_s)
    mode = 0 if nnz[0] == "lognormal" else 1
    a, b = float(nnz[1]), float(nnz[2])
    lo, hi = int(nnz_clip[0]), int(nnz_clip[1])
    if mode == 1:
        lo, hi = int(nnz[1]), int(nnz[2])
    threads = threads or min(64, os.cpu_count() or 1)
    counts = np.empty(n, dtype=np.uint64)
    lib.synth_rows(seed, stream, n, d, K, zipf_s, dirichlet, mode, a, b, lo, hi, _ptr(perm), _ptr(cdf),
                   threads, None, _ptr(counts), None, None)
    indptr = np.zeros(n + 1, dtype=np.uint64)
    np.cumsum(counts, out=indptr[1:])
    terms = np.empty(int(indptr[-1]), dtype=np.uint16)
    vals = np.empty(int(indptr[-1]), dtype=np.float32)
    lib.synth_rows(seed, stream, n, d, K, zipf_s, dirichlet, mode, a, b, lo, hi, _ptr(perm), _ptr(cdf),
                   threads, _ptr(indptr), None, _ptr(terms), _ptr(vals))
    return CSR(indptr, terms, vals, d)


# Streams: documents and each query set draw from disjoint streams of one seed
# (one seed fixes the topic model they all share): the evaluation queries,
# training queries for the parameter model, a held-out set, serving arrivals.
DOC_STREAM, QUERY_STREAM, TRAIN_STREAM, HELDOUT_STREAM, SERVE_STREAM = 1, 2, 3, 4, 5


def docs(n: int, seed: int = 0, d: int = VOCAB, **kw) -> CSR:
    """Passages: nnz ~ round(lognormal(mean 120, sd 40)) clipped to [10, 400]."""
    return generate(n, seed=seed, stream=DOC_STREAM, d=d, nnz=("lognormal", 120.0, 40.0),
                    nnz_clip=(10, 400), **kw)


def queries(n: int, seed: int = 0, d: int = VOCAB, uneven: bool = False, stream: int = QUERY_STREAM,
            **kw) -> CSR:
    """Queries: nnz ~ lognormal(mean 40, sd 15) clipped to [10, 150], or uniform 10..150 (uneven)."""
    if uneven:
        return generate(n, seed=seed, stream=stream, d=d, nnz=("uniform", 10, 150), **kw)
    return generate(n, seed=seed, stream=stream, d=d, nnz=("lognormal", 40.0, 15.0),
                    nnz_clip=(10, 150), **kw)

"""Python binding of ``libseismic.so``, the GB300 (sm_103a) implementation of
Seismic (arXiv 2509.24815).  Argument marshalling only: every step of index
search runs in the library's CUDA kernels.  There is no CPU fallback: importing
this package without a built library raises.

Names mirror the C ABI in ``include/seismic.h``.  Host inputs are numpy arrays;
device inputs are torch CUDA tensors (``DeviceCSR``), in which case results
stay on the device.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libseismic.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(nvcc, sm_103a).  The search path has no CPU fallback.")
_lib = ctypes.CDLL(LIB_PATH)

NONE_ID = 0xFFFFFFFF
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUDGET, EIO = 0, -1, -2, -3, -4, -5, -6
STATS = ("lists", "blocks_scored", "blocks_evaluated", "blocks_skipped", "docs", "doc_nnz", "knn_docs",
         "summary_entries", "knn_nnz", "dir_lookups", "block_docs", "query_nnz", "t_start_ns", "t_end_ns")
EXPORTS = ("list_ptr", "list_doc", "blk_ptr", "bdoc_ptr", "bdoc", "blk_m", "blk_size", "sum_ptr", "sum_term",
           "sum_val", "sum_code", "cent", "sbm", "scptr", "scol_blk", "scol_code", "scol_val")
_EXPORT_DT = dict(list_ptr=np.uint32, list_doc=np.uint32, blk_ptr=np.uint32, bdoc_ptr=np.uint32, bdoc=np.uint32,
                  blk_m=np.float32, blk_size=np.float32, sum_ptr=np.uint32, sum_term=np.uint16,
                  sum_val=np.float32, sum_code=np.uint8, cent=np.uint32, sbm=np.uint32, scptr=np.uint32,
                  scol_blk=np.uint16, scol_code=np.uint8, scol_val=np.float32)
MLP_IN, MLP_PARAMS = 64, 128 * 64 + 128 + 64 * 128 + 64 + 2 * 64 + 2


class SeismicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"seismic error {code}: {msg}")
        self.code = code


class _CSR(ctypes.Structure):
    _fields_ = [("indptr", ctypes.c_void_p), ("terms", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("n_rows", ctypes.c_uint64), ("dim", ctypes.c_uint32), ("on_device", ctypes.c_int32)]


class BuildParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_uint32), ("beta", ctypes.c_uint32), ("alpha", ctypes.c_double),
                ("quantize_u8", ctypes.c_int32), ("seed", ctypes.c_uint64), ("lambda_frac", ctypes.c_double),
                ("beta_frac", ctypes.c_double), ("keep_full_lists", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("keep_block_summaries", ctypes.c_int32), ("values_fp16", ctypes.c_int32)]


class SearchParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("cut", ctypes.c_uint32), ("heap_factor", ctypes.c_float),
                ("hf_mode", ctypes.c_int32), ("exhaustive", ctypes.c_int32), ("alpha_q", ctypes.c_float),
                ("use_knn", ctypes.c_int32), ("learned", ctypes.c_int32), ("wave", ctypes.c_uint32),
                ("group", ctypes.c_uint32), ("cta_warps", ctypes.c_uint32), ("persistent", ctypes.c_uint32),
                ("max_query_nnz", ctypes.c_uint32), ("hash_slots", ctypes.c_uint32), ("shape", ctypes.c_uint32),
                ("no_prefetch", ctypes.c_int32), ("order", ctypes.c_uint32)]


class IndexInfo(ctypes.Structure):
    _fields_ = [("n_docs", ctypes.c_uint64), ("nnz", ctypes.c_uint64), ("n_postings", ctypes.c_uint64),
                ("n_blocks", ctypes.c_uint64), ("n_summary_entries", ctypes.c_uint64), ("dim", ctypes.c_uint32),
                ("kappa", ctypes.c_uint32), ("quantize_u8", ctypes.c_int32), ("has_full_lists", ctypes.c_int32),
                ("has_mlp", ctypes.c_int32), ("device_bytes", ctypes.c_uint64), ("values_fp16", ctypes.c_int32),
                ("knn_bits", ctypes.c_uint32), ("knn_bytes", ctypes.c_uint64)]


class ServerParams(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("streams", ctypes.c_uint32), ("max_query_nnz", ctypes.c_uint32),
                ("slot_budget", ctypes.c_uint32)]


_vp, _u64, _u32, _i32, _f32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_float
_P = ctypes.POINTER
_SIGS = {
    "seismic_build": ([_P(_CSR), _P(BuildParams), _P(_vp)], ctypes.c_int),
    "seismic_search": ([_vp, _P(_CSR), _P(SearchParams), _vp, _vp, _i32, _vp, _vp], ctypes.c_int),
    "seismic_search_exact": ([_vp, _P(_CSR), _u32, _vp, _vp, _i32, _vp], ctypes.c_int),
    "seismic_set_knn": ([_vp, _vp, _u64, _u32, _i32], ctypes.c_int),
    "seismic_build_knn": ([_vp, _u32, _P(SearchParams)], ctypes.c_int),
    "seismic_get_knn": ([_vp, _vp, _u64], ctypes.c_int),
    "seismic_refine_knn": ([_vp, _u32, _P(SearchParams)], ctypes.c_int),
    "seismic_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "seismic_load": ([ctypes.c_char_p, _P(_vp)], ctypes.c_int),
    "seismic_info": ([_vp, _P(IndexInfo)], ctypes.c_int),
    "seismic_export": ([_vp, _i32, _vp, _u64, _P(_u64)], ctypes.c_int),
    "seismic_set_mlp": ([_vp, _vp, _u64], ctypes.c_int),
    "seismic_query_features": ([_vp, _P(_CSR), _vp, _i32, _vp], ctypes.c_int),
    "seismic_mlp_forward": ([_vp, _vp, _u64, _vp, _vp], ctypes.c_int),
    "seismic_mlp_train_step": ([_vp, _vp, _vp, _vp, _vp, _vp, _u64, _f32, _u32, _vp, _vp], ctypes.c_int),
    "seismic_search_noalloc": ([_vp, _P(_CSR), _P(SearchParams), _vp, _vp, _vp], ctypes.c_int),
    "seismic_server_create": ([_vp, _P(SearchParams), _P(ServerParams), _P(_vp)], ctypes.c_int),
    "seismic_server_submit": ([_vp, _vp, _vp, _u32, _u32, _P(_u64)], ctypes.c_int),
    "seismic_server_progress": ([_vp, _P(_u32)], ctypes.c_int),
    "seismic_server_result": ([_vp, _u64, _vp, _vp, _P(ctypes.c_double), _P(_i32)], ctypes.c_int),
    "seismic_server_replay": ([_vp, _P(_CSR), _vp, _vp, _u32, _vp, _vp, _vp, _P(ctypes.c_double)], ctypes.c_int),
    "seismic_server_destroy": ([_vp], None),
    "seismic_free": ([_vp], None),
    "seismic_last_error": ([], ctypes.c_char_p),
    "seismic_version": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def _check(rc):
    if rc != OK:
        raise SeismicError(rc, _lib.seismic_last_error().decode(errors="replace"))


def seismic_last_error() -> str:
    return _lib.seismic_last_error().decode(errors="replace")


def seismic_version() -> str:
    return _lib.seismic_version().decode()


@dataclass
class DeviceCSR:
    """A CSR matrix in device memory (torch CUDA tensors): indptr int64 [n+1],
    terms int16 (u16 bits) [nnz], vals float32 [nnz]."""
    indptr: "object"
    terms: "object"
    vals: "object"
    dim: int
    max_row_nnz: int = 0

    @property
    def n_rows(self):
        return int(self.indptr.shape[0]) - 1

    @staticmethod
    def from_host(csr, device="cuda"):
        import torch
        ip = torch.from_numpy(np.ascontiguousarray(csr.indptr, dtype=np.uint64).view(np.int64)).to(device)
        t = torch.from_numpy(np.ascontiguousarray(csr.terms, dtype=np.uint16).view(np.int16)).to(device)
        v = torch.from_numpy(np.ascontiguousarray(csr.vals, dtype=np.float32)).to(device)
        lens = np.diff(np.asarray(csr.indptr, dtype=np.int64))
        return DeviceCSR(ip, t, v, csr.dim, int(lens.max()) if len(lens) else 0)


def _csr_struct(m):
    """(struct, keepalive) for a host CSR (numpy fields) or a DeviceCSR."""
    if isinstance(m, DeviceCSR):
        s = _CSR(m.indptr.data_ptr(), m.terms.data_ptr(), m.vals.data_ptr(), m.n_rows, m.dim, 1)
        return s, (m,)
    ip = np.ascontiguousarray(m.indptr, dtype=np.uint64)
    t = np.ascontiguousarray(m.terms, dtype=np.uint16)
    v = np.ascontiguousarray(m.vals, dtype=np.float32)
    s = _CSR(ip.ctypes.data, t.ctypes.data, v.ctypes.data, len(ip) - 1, int(m.dim), 0)
    return s, (ip, t, v)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Index:
    """Owns a ``seismic_index*``; freed with the object."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h and self._h.value:
            _lib.seismic_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return seismic_info(self)


def seismic_build(docs, lambda_=2000, beta=100, alpha=0.4, quantize_u8=False, seed=0, lambda_frac=0.0,
                  beta_frac=0.0, keep_full_lists=False, threads=0, keep_block_summaries=False,
                  values_fp16=False) -> Index:
    """Algorithm "Indexing with Seismic" on the current CUDA device."""
    s, keep = _csr_struct(docs)
    p = BuildParams(int(lambda_), int(beta), float(alpha), int(bool(quantize_u8)), int(seed), float(lambda_frac),
                    float(beta_frac), int(bool(keep_full_lists)), int(threads), int(bool(keep_block_summaries)),
                    int(bool(values_fp16)))
    h = ctypes.c_void_p()
    _check(_lib.seismic_build(ctypes.byref(s), ctypes.byref(p), ctypes.byref(h)))
    return Index(h.value)


def search_params(k=10, cut=10, heap_factor=0.8, hf_mode=0, exhaustive=False, alpha_q=0.0, use_knn=False,
                  learned=False, wave=1, group=0, cta_warps=0, persistent=False, max_query_nnz=0,
                  hash_slots=0, shape=0, no_prefetch=False, order=0) -> SearchParams:
    return SearchParams(int(k), int(cut), float(heap_factor), int(hf_mode), int(bool(exhaustive)), float(alpha_q),
                        int(bool(use_knn)), int(bool(learned)), int(wave), int(group), int(cta_warps),
                        int(bool(persistent)), int(max_query_nnz), int(hash_slots), int(shape),
                        int(bool(no_prefetch)), int(order))


def seismic_search(index: Index, queries, params: SearchParams | None = None, *, ids_out=None, scores_out=None,
                   stream=None, stats=False, **kw):
    """Algorithm "Query processing with Seismic" for a batch.  Host queries ->
    numpy (ids uint32, scores float32); DeviceCSR -> torch CUDA tensors (or the
    given ``ids_out``/``scores_out``).  ``stats=True`` also returns the
    per-query work counters (uint64 [nq, len(STATS)])."""
    # a copy: the caller's struct is never written (a bound filled here would go stale on a larger batch)
    p = SearchParams.from_buffer_copy(params) if params is not None else search_params(**kw)
    if isinstance(queries, DeviceCSR) and not p.max_query_nnz and queries.max_row_nnz:
        p.max_query_nnz = queries.max_row_nnz
    s, keep = _csr_struct(queries)
    nq, k = s.n_rows, p.k
    st = np.zeros((nq, len(STATS)), dtype=np.uint64) if stats else None
    if isinstance(queries, DeviceCSR):
        import torch
        dev = queries.vals.device
        ids = ids_out if ids_out is not None else torch.empty((nq, k), dtype=torch.int32, device=dev)
        sc = scores_out if scores_out is not None else torch.empty((nq, k), dtype=torch.float32, device=dev)
        rc = _lib.seismic_search(index.handle, ctypes.byref(s), ctypes.byref(p), ids.data_ptr(), sc.data_ptr(), 1,
                                 _stream_ptr(stream), st.ctypes.data if stats else None)
    else:
        ids = ids_out if ids_out is not None else np.empty((nq, k), dtype=np.uint32)
        sc = scores_out if scores_out is not None else np.empty((nq, k), dtype=np.float32)
        rc = _lib.seismic_search(index.handle, ctypes.byref(s), ctypes.byref(p), _host_ptr(ids), _host_ptr(sc), 0,
                                 _stream_ptr(stream), st.ctypes.data if stats else None)
    _check(rc)
    return (ids, sc, st) if stats else (ids, sc)


def _host_ptr(a):
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # pinned torch CPU tensor


def seismic_search_exact(index: Index, queries, k=10, *, stream=None):
    """Exact top-k by brute force on the device (needs keep_full_lists)."""
    s, keep = _csr_struct(queries)
    nq = s.n_rows
    if isinstance(queries, DeviceCSR):
        import torch
        dev = queries.vals.device
        ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
        sc = torch.empty((nq, k), dtype=torch.float32, device=dev)
        _check(_lib.seismic_search_exact(index.handle, ctypes.byref(s), k, ids.data_ptr(), sc.data_ptr(), 1,
                                         _stream_ptr(stream)))
    else:
        ids = np.empty((nq, k), dtype=np.uint32)
        sc = np.empty((nq, k), dtype=np.float32)
        _check(_lib.seismic_search_exact(index.handle, ctypes.byref(s), k, ids.ctypes.data, sc.ctypes.data, 0,
                                         _stream_ptr(stream)))
    return ids, sc


def seismic_set_knn(index: Index, nbrs: np.ndarray):
    nbrs = np.ascontiguousarray(nbrs, dtype=np.uint32)
    _check(_lib.seismic_set_knn(index.handle, nbrs.ctypes.data, nbrs.shape[0], nbrs.shape[1], 0))


def seismic_build_knn(index: Index, kappa: int, params: SearchParams | None = None, exact=False):
    """kappa-NN graph: exact (needs keep_full_lists) or by Seismic search."""
    if exact:
        _check(_lib.seismic_build_knn(index.handle, kappa, None))
    else:
        p = params if params is not None else search_params()
        _check(_lib.seismic_build_knn(index.handle, kappa, ctypes.byref(p)))


def seismic_refine_knn(index: Index, rounds: int = 1, params: SearchParams | None = None):
    """Neighbour-of-neighbour passes over the installed graph: each row becomes
    the kappa best of the document's list and its neighbours' lists."""
    _check(_lib.seismic_refine_knn(index.handle, int(rounds), ctypes.byref(params) if params is not None else None))


def seismic_get_knn(index: Index) -> np.ndarray:
    inf = seismic_info(index)
    out = np.empty((inf["n_docs"], inf["kappa"]), dtype=np.uint32)
    _check(_lib.seismic_get_knn(index.handle, out.ctypes.data, out.size))
    return out


def seismic_save(index: Index, path: str):
    _check(_lib.seismic_save(index.handle, path.encode()))


def seismic_load(path: str) -> Index:
    h = ctypes.c_void_p()
    _check(_lib.seismic_load(path.encode(), ctypes.byref(h)))
    return Index(h.value)


def seismic_info(index: Index) -> dict:
    inf = IndexInfo()
    _check(_lib.seismic_info(index.handle, ctypes.byref(inf)))
    return {f: getattr(inf, f) for f, _ in IndexInfo._fields_}


def seismic_export(index: Index, what: str) -> np.ndarray:
    wid = EXPORTS.index(what)
    need = ctypes.c_uint64()
    _check(_lib.seismic_export(index.handle, wid, None, 0, ctypes.byref(need)))
    dt = _EXPORT_DT[what]
    out = np.empty(need.value // np.dtype(dt).itemsize, dtype=dt)
    if need.value:
        _check(_lib.seismic_export(index.handle, wid, out.ctypes.data, need.value, ctypes.byref(need)))
    return out


def seismic_set_mlp(index: Index, weights: np.ndarray):
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(_lib.seismic_set_mlp(index.handle, w.ctypes.data, w.size))


def seismic_query_features(index: Index, queries) -> np.ndarray:
    s, keep = _csr_struct(queries)
    out = np.empty((s.n_rows, MLP_IN), dtype=np.float32)
    _check(_lib.seismic_query_features(index.handle, ctypes.byref(s), out.ctypes.data, 0, None))
    return out


def seismic_mlp_forward(weights, features, out, stream=None):
    """Device buffers (torch CUDA float32): weights [MLP_PARAMS], features [n, 64] -> out [n, 2]."""
    _check(_lib.seismic_mlp_forward(weights.data_ptr(), features.data_ptr(), features.shape[0], out.data_ptr(),
                                    _stream_ptr(stream)))


def seismic_mlp_train_step(weights, grads, adam_m, adam_v, features, targets, lr, step, loss_out, stream=None):
    """One Adam step on device buffers; loss_out (1 float) gets the loss before the step."""
    _check(_lib.seismic_mlp_train_step(weights.data_ptr(), grads.data_ptr(), adam_m.data_ptr(), adam_v.data_ptr(),
                                       features.data_ptr(), targets.data_ptr(), features.shape[0], float(lr),
                                       int(step), loss_out.data_ptr(), _stream_ptr(stream)))


def seismic_search_noalloc(index: Index, queries: DeviceCSR, params: SearchParams, ids_out, scores_out,
                           stream=None):
    """Search with no memory allocation (device queries and outputs, torch CUDA
    tensors); work memory is the library's fixed device array.  Enqueued on
    ``stream`` without waiting; calls that overlap on the GPU race."""
    p = SearchParams.from_buffer_copy(params)  # the caller's struct is never written
    if not p.max_query_nnz:
        p.max_query_nnz = queries.max_row_nnz
    s, keep = _csr_struct(queries)
    _check(_lib.seismic_search_noalloc(index.handle, ctypes.byref(s), ctypes.byref(p), ids_out.data_ptr(),
                                       scores_out.data_ptr(), _stream_ptr(stream)))


class Server:
    """Continuous-batching server over an index (seismic_server_*)."""

    def __init__(self, index: Index, search: SearchParams | None = None, max_batch=256, streams=4,
                 max_query_nnz=1024, slot_budget=0):
        self.index = index  # kept alive for the server's lifetime
        self.settings = dict(max_batch=max_batch, streams=streams, max_query_nnz=max_query_nnz,
                             slot_budget=slot_budget)
        sp = search if search is not None else search_params()
        pp = ServerParams(int(max_batch), int(streams), int(max_query_nnz), int(slot_budget))
        h = ctypes.c_void_p()
        _check(_lib.seismic_server_create(index.handle, ctypes.byref(sp), ctypes.byref(pp), ctypes.byref(h)))
        self._h = h

    def close(self):
        if self._h and self._h.value:
            _lib.seismic_server_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, terms, vals, k=10) -> int:
        t = np.ascontiguousarray(terms, dtype=np.uint16)
        v = np.ascontiguousarray(vals, dtype=np.float32)
        tk = ctypes.c_uint64()
        _check(_lib.seismic_server_submit(self._h, t.ctypes.data, v.ctypes.data, len(t), int(k), ctypes.byref(tk)))
        return tk.value

    def progress(self) -> int:
        n = ctypes.c_uint32()
        _check(_lib.seismic_server_progress(self._h, ctypes.byref(n)))
        return n.value

    def result(self, ticket: int, k: int):
        """(ids, scores, latency_us) once done, else None."""
        ids = np.empty(k, dtype=np.uint32)
        sc = np.empty(k, dtype=np.float32)
        lat = ctypes.c_double()
        done = ctypes.c_int32()
        _check(_lib.seismic_server_result(self._h, ticket, ids.ctypes.data, sc.ctypes.data, ctypes.byref(lat),
                                          ctypes.byref(done)))
        return (ids, sc, lat.value) if done.value else None

    def replay(self, queries, arrival_s, k_per_query):
        """Replays an arrival trace; returns (ids, scores, latency_us, wall_s)."""
        s, keep = _csr_struct(queries)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        ks = np.ascontiguousarray(k_per_query, dtype=np.uint32)
        kst = int(ks.max()) if len(ks) else 1
        n = len(arr)
        ids = np.empty((n, kst), dtype=np.uint32)
        sc = np.empty((n, kst), dtype=np.float32)
        lat = np.empty(n, dtype=np.float64)
        wall = ctypes.c_double()
        _check(_lib.seismic_server_replay(self._h, ctypes.byref(s), arr.ctypes.data, ks.ctypes.data, kst,
                                          ids.ctypes.data, sc.ctypes.data, lat.ctypes.data, ctypes.byref(wall)))
        return ids, sc, lat, wall.value


def seismic_free(index: Index):
    index.close()

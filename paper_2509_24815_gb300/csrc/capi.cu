// The C ABI (include/seismic.h): argument checks, staging of host buffers,
// kernel dispatch, graph install, persistence and inspection.
#include <cuda_fp16.h>

#include <cstdio>
#include <memory>
#include <new>

#include "search_impl.h"

namespace seismic {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }
int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return SEISMIC_ECUDA;
}

int build_index(const seismic_csr *docs, const seismic_build_params *bp, seismic_index **out);

namespace {

__global__ void k_max_row_nnz(const uint64_t *indptr, uint64_t n, uint32_t *out) {
  uint32_t m = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    { const uint64_t len = indptr[i + 1] - indptr[i]; m = max(m, len > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)len); }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// A flat CSR view of forward-index rows [r0, r0 + n): every padded row entry
// is kept (the padding has value 0, which every reader ignores).  ip[0..n]
// (8 entries per chunk, prefix-summed) is given.
__global__ void k_fwd_to_csr(const unsigned long long *frow, const uint8_t *data, int fp16, uint64_t r0, uint64_t n,
                             const uint64_t *ip, uint16_t *terms, float *vals) {
  for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const unsigned long long row = frow[r0 + i];
    const uint32_t nch = (uint32_t)(row >> 32);
    const uint8_t *rec = data + (size_t)(uint32_t)row * kUnitBytes;
    const uint64_t o = ip[i];
    for (uint32_t j = threadIdx.x; j < 8 * nch; j += blockDim.x) {
      const uint32_t c = j / 8, e = j % 8;
      if (fp16) {
        terms[o + j] = reinterpret_cast<const uint16_t *>(rec + (size_t)kUnitBytes * c)[e];
        vals[o + j] = __half2float(reinterpret_cast<const __half *>(rec + (size_t)kUnitBytes * c + 16)[e]);
      } else {
        terms[o + j] = reinterpret_cast<const uint16_t *>(rec)[j];
        vals[o + j] = reinterpret_cast<const float *>(rec + (size_t)kUnitBytes * ((nch + 1) / 2))[j];
      }
    }
  }
}

// Bits per stored kappa-NN id: the smallest b with 2^b > n_docs, which is the
// paper's floor(log2(n_docs - 1)) + 1 (Section 4.3) except when n_docs is a
// power of two, where one more bit leaves the all-ones code free for a
// missing neighbour.
uint32_t knn_bits_for(uint64_t n) {
  uint32_t b = 1;
  while (b < 32 && (1ull << b) <= n) b++;
  return b;
}

// Work-queue order of a persistent search: queries sorted by their largest
// term (the first list they traverse), so queries that read the same lists,
// blocks and rows run at the same time and share them through L2.  With
// longest_first, queries that traverse more lists (min(nonzeros, cut), the
// per-query cut when learned) come first and the largest term orders each
// such class, so the queue ends on its cheapest queries.  Results do not
// depend on the order.
__global__ void k_order_keys(const uint64_t *ip, const uint16_t *t, const float *v, uint32_t nq,
                             unsigned long long *keys, int longest_first, uint32_t cut, const uint32_t *q_cut) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  float bv = -INFINITY;
  uint32_t bt = 0xFFFFu, nz = 0;
  for (uint64_t p = ip[q]; p < ip[q + 1]; p++) {
    const float x = v[p];
    const uint32_t tt = t[p];
    nz += x != 0.0f;
    if (x != 0.0f && (x > bv || (x == bv && tt < bt))) { bv = x; bt = tt; }
  }
  unsigned long long key = ((unsigned long long)bt << 32) | q;
  if (longest_first) {
    const uint32_t lists = min(nz, q_cut ? q_cut[q] : cut);
    key |= (unsigned long long)(0xFFFFu - min(lists, 0xFFFFu)) << 48;
  }
  keys[q] = key;
}

constexpr uint32_t kOrderChunk = 8192;

__global__ void __launch_bounds__(1024) k_order_sort(const unsigned long long *keys, uint32_t nq, uint32_t *perm) {
  extern __shared__ unsigned long long sk[];
  const uint32_t c0 = blockIdx.x * kOrderChunk, n = min(kOrderChunk, nq - c0);
  uint32_t P2 = 1;
  while (P2 < n) P2 <<= 1;
  for (uint32_t i = threadIdx.x; i < P2; i += blockDim.x) sk[i] = i < n ? keys[c0 + i] : ~0ull;
  __syncthreads();
  for (uint32_t k2 = 2; k2 <= P2; k2 <<= 1)
    for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P2; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long x = sk[i], y = sk[ixj];
          if ((x > y) == ((i & k2) == 0)) { sk[i] = y; sk[ixj] = x; }
        }
      }
      __syncthreads();
    }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) perm[c0 + i] = (uint32_t)(sk[i] & 0xFFFFFFFFu);
}

int sm_count(int dev) {
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

struct Staged {
  const uint64_t *ip = nullptr;
  const uint16_t *t = nullptr;
  const float *v = nullptr;
  uint32_t maxnnz = 0;
};

// Puts the queries on the device (copying host ones into the workspace) and
// finds the largest row.
int stage_queries(seismic_index *ix, Workspace *w, const seismic_csr *q, uint32_t bound, cudaStream_t st,
                  Staged &out) {
  if (!q->on_device) {
    int rc = validate_host_csr(q, "queries", ix->dim);
    if (rc) return rc;
    uint64_t nnz = q->indptr[q->n_rows], mx = 0;
    for (uint64_t i = 0; i < q->n_rows; i++) mx = std::max<uint64_t>(mx, q->indptr[i + 1] - q->indptr[i]);
    size_t b_ip = (q->n_rows + 1) * 8, b_t = ((nnz * 2 + 15) / 16) * 16, b_v = nnz * 4;
    if ((rc = w->q.ensure(b_ip + b_t + b_v + 64))) return rc;
    uint8_t *base = w->q.as<uint8_t>();
    SZ_CUDA(cudaMemcpyAsync(base, q->indptr, b_ip, cudaMemcpyHostToDevice, st));
    if (nnz) {
      SZ_CUDA(cudaMemcpyAsync(base + b_ip, q->terms, nnz * 2, cudaMemcpyHostToDevice, st));
      SZ_CUDA(cudaMemcpyAsync(base + b_ip + b_t, q->vals, nnz * 4, cudaMemcpyHostToDevice, st));
    }
    out.ip = reinterpret_cast<const uint64_t *>(base);
    out.t = reinterpret_cast<const uint16_t *>(base + b_ip);
    out.v = reinterpret_cast<const float *>(base + b_ip + b_t);
    out.maxnnz = (uint32_t)std::min<uint64_t>(mx, 0xFFFFFFFFull);
    return SEISMIC_OK;
  }
  if (q->dim != ix->dim) return fail(SEISMIC_EINVAL, "queries: dim differs from the index");
  out.ip = q->indptr;
  out.t = q->terms;
  out.v = q->vals;
  if (bound) {
    out.maxnnz = bound;
    return SEISMIC_OK;
  }
  int rc = w->queue.ensure(64);
  if (rc) return rc;
  uint32_t *m = w->queue.as<uint32_t>() + 4;
  SZ_CUDA(cudaMemsetAsync(m, 0, 4, st));
  k_max_row_nnz<<<std::max<uint64_t>(1, std::min<uint64_t>(1024, (q->n_rows + 255) / 256)), 256, 0, st>>>(q->indptr, q->n_rows, m);
  SZ_CUDA(cudaGetLastError());
  uint32_t h = 0;
  SZ_CUDA(cudaMemcpyAsync(&h, m, 4, cudaMemcpyDeviceToHost, st));
  SZ_CUDA(cudaStreamSynchronize(st));
  out.maxnnz = h;
  return SEISMIC_OK;
}

int check_params(const seismic_index *ix, const seismic_search_params *p) {
  if (!p) return fail(SEISMIC_EINVAL, "NULL search params");
  if (p->k == 0 || p->k > kMaxK) return fail(SEISMIC_EINVAL, "k must be in 1..1024");
  if (p->alpha_q <= 0.0f && p->cut == 0 && !p->learned) return fail(SEISMIC_EINVAL, "cut must be >= 1");
  if (p->alpha_q > 1.0f) return fail(SEISMIC_EINVAL, "alpha_q must be <= 1");
  if (!p->exhaustive && !(p->heap_factor > 0.0f) ) return fail(SEISMIC_EINVAL, "heap_factor must be > 0");
  if (p->hf_mode != 0 && p->hf_mode != 1) return fail(SEISMIC_EINVAL, "hf_mode must be 0 or 1");
  if (p->use_knn && ix->kappa == 0) return fail(SEISMIC_EINVAL, "use_knn: the index has no kappa-NN graph");
  if (p->learned && !ix->has_mlp) return fail(SEISMIC_EINVAL, "learned: the index has no MLP");
  if (p->shape > 2) return fail(SEISMIC_EINVAL, "shape must be 0 (auto), 1 (CTA per query) or 2 (warp per query)");
  const bool ws = p->shape == 2;
  uint32_t g = p->group ? p->group : (ws ? 8 : 1), w = p->cta_warps ? p->cta_warps : 8;
  if (!(g == 8 || g == 16 || g == 32 || (ws && g == 4) || (!ws && g == 1)))
    return fail(SEISMIC_EINVAL, "group must be 8/16/32 (4 also for the warp shape, 1 for the CTA shape)");
  const uint32_t ww = p->cta_warps ? p->cta_warps : 4;
  if (ws ? !(ww == 1 || ww == 2 || ww == 4) : !(w == 4 || w == 8 || w == 16))
    return fail(SEISMIC_EINVAL, "cta_warps must be 1/2/4 (warp shape) or 4/8/16 (CTA shape)");
  uint32_t hs = p->hash_slots ? p->hash_slots : 2048;
  if (hs & (hs - 1)) return fail(SEISMIC_EINVAL, "hash_slots must be a power of two");
  return SEISMIC_OK;
}

}  // namespace

int search_ws(seismic_index *ix, Workspace *w, const seismic_csr *queries, const seismic_search_params *p,
              uint32_t *ids_out, float *scores_out, int32_t out_on_device, void *stream, uint64_t *stats,
              const uint32_t *seed) {
  if (!ix || !queries || !w) return fail(SEISMIC_EINVAL, "NULL index/queries");
  int rc = check_params(ix, p);
  if (rc) return rc;
  if (!ids_out || !scores_out) return fail(SEISMIC_EINVAL, "NULL outputs");
  if (queries->n_rows == 0) return SEISMIC_OK;
  if (queries->n_rows > 0x7FFFFFFFull) return fail(SEISMIC_EINVAL, "too many queries in one call");
  SZ_CUDA(cudaSetDevice(ix->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t nq = (uint32_t)queries->n_rows, k = p->k;
  Staged q;
  if ((rc = stage_queries(ix, w, queries, p->max_query_nnz, st, q))) return rc;
  uint32_t *d_ids = ids_out;
  float *d_sc = scores_out;
  if (!out_on_device) {
    if ((rc = w->out.ensure((size_t)nq * k * 8))) return rc;
    d_ids = w->out.as<uint32_t>();
    d_sc = reinterpret_cast<float *>(d_ids + (size_t)nq * k);
  }
  if ((rc = w->queue.ensure(64))) return rc;
  SZ_CUDA(cudaMemsetAsync(w->queue.p, 0, 16, st));
  unsigned long long *d_stats = nullptr;
  if (stats) {
    if ((rc = w->stats.ensure((size_t)nq * SEISMIC_STATS_N * 8))) return rc;
    d_stats = w->stats.as<unsigned long long>();
  }
  SearchArgs a{};
  a.fwd_row = ix->fwd_row.as<unsigned long long>();
  a.fwd_data = ix->fwd_data.as<uint8_t>();
  a.fp16 = ix->bp.values_fp16 ? 1 : 0;
  a.fwd_nnz = ix->fwd_nnz.as<uint16_t>();
  a.blk_ptr = ix->blk_ptr.as<uint32_t>();
  a.bdoc_ptr = ix->bdoc_ptr.as<uint32_t>();
  a.bdoc = ix->bdoc.as<uint32_t>();
  a.bdoc_row = ix->bdoc_row.as<unsigned long long>();
  a.blk_m = ix->blk_m.as<float>();
  a.blk_size = ix->blk_size.as<float>();
  a.sbm = ix->sbm.as<uint2>();
  a.scptr = ix->scptr.as<uint32_t>();
  a.scol_blk = ix->scol_blk.as<uint16_t>();
  a.scol_code = ix->scol_code.as<uint8_t>();
  a.scol_val = ix->scol_val.as<float>();
  a.knn = ix->knn.as<uint32_t>();
  a.kappa = ix->kappa;
  a.knn_bits = ix->knn_bits;
  a.dim = ix->dim;
  a.quant = ix->bp.quantize_u8 ? 1 : 0;
  a.q_indptr = q.ip;
  a.q_terms = q.t;
  a.q_vals = q.v;
  a.nq = nq;
  a.k = k;
  a.cut = p->cut;
  a.hf = p->heap_factor;
  a.hf_mode = p->hf_mode;
  a.exhaustive = p->exhaustive ? 1 : 0;
  a.use_knn = p->use_knn ? 1 : 0;
  a.alpha_q = p->alpha_q > 0.0f ? p->alpha_q : 0.0f;
  a.wave = p->wave ? p->wave : 1;
  a.ids = d_ids;
  a.scores = d_sc;
  a.stats = d_stats;
  a.seed = seed;
  if (seed && (p->shape == 2 || !p->use_knn || p->k != ix->kappa + 1))
    return fail(SEISMIC_EINVAL, "graph refinement runs the CTA shape with the expansion and k = kappa + 1");
  a.queue = w->queue.as<uint32_t>();
  a.persistent = p->persistent ? 1 : 0;
  a.W = (ix->dim + 31) / 32;
  a.QN = std::max<uint32_t>(4, (q.maxnnz + 3) & ~3u);
  a.BMAX = std::max<uint32_t>(1, ix->max_blocks_per_list);
  a.BPOW2 = 1;
  while (a.BPOW2 < a.BMAX) a.BPOW2 <<= 1;
  a.HS = p->hash_slots ? p->hash_slots : 2048;
  a.CAND = 256;
  if (p->learned) {
    // (cut, heap_factor) per query from the MLP, fused ahead of the search
    size_t need = (size_t)nq * (SEISMIC_MLP_IN * 4 + 8);
    if ((rc = w->params.ensure(need))) return rc;
    float *feat = w->params.as<float>();
    uint32_t *qc = reinterpret_cast<uint32_t *>(feat + (size_t)nq * SEISMIC_MLP_IN);
    float *qh = reinterpret_cast<float *>(qc + nq);
    if ((rc = launch_features(q.ip, q.t, q.v, nq, ix->list_ptr.as<uint32_t>(), ix->blk_ptr.as<uint32_t>(), ix->dim,
                              feat, st)))
      return rc;
    if ((rc = launch_mlp_params(ix->mlp.as<float>(), feat, nq, p->cut ? p->cut : 10,
                                p->heap_factor > 0.0f ? p->heap_factor : 0.8f, qc, qh, st)))
      return rc;
    a.q_cut = qc;
    a.q_hf = qh;
    a.QN = std::max<uint32_t>(a.QN, 32);
  }
  // defaults: one CTA per query with chunk-flattened scoring (the measured fastest)
  const uint32_t nw = p->cta_warps ? p->cta_warps : 8, group = p->group ? p->group : (p->shape == 2 ? 8 : 1);
  a.sum_absmax = ix->sum_absmax;
  a.prefetch = p->no_prefetch ? 0u : 256u;
  const bool warp_shape0 = p->shape == 2;
  if ((p->order == 0 || p->order == 2) && nq > 1 && (a.persistent || warp_shape0)) {
    if ((rc = w->perm.ensure((size_t)nq * 12))) return rc;
    unsigned long long *keys = w->perm.as<unsigned long long>();
    uint32_t *perm = reinterpret_cast<uint32_t *>(keys + nq);
    k_order_keys<<<(nq + 255) / 256, 256, 0, st>>>(q.ip, q.t, q.v, nq, keys, p->order == 2 ? 1 : 0,
                                                     p->alpha_q > 0.0f ? 0xFFFFu : p->cut, a.q_cut);
    SZ_CUDA(cudaGetLastError());
    static std::atomic<uint64_t> attr{0};
    if ((rc = set_smem_limit_once(attr, (const void *)k_order_sort, kOrderChunk * 8))) return rc;
    k_order_sort<<<(nq + kOrderChunk - 1) / kOrderChunk, 1024, kOrderChunk * 8, st>>>(keys, nq, perm);
    SZ_CUDA(cudaGetLastError());
    a.perm = perm;
  }
  // shape: one CTA per query (default) or one warp per query
  const bool warp_shape = p->shape == 2;
  if (warp_shape) {
    if (k > 128) return fail(SEISMIC_EINVAL, "the warp-per-query shape needs k <= 128");
    const uint32_t wpb = p->cta_warps ? p->cta_warps : 4;
    size_t wbytes = search_layout_warp(a);
    size_t smem = wbytes * wpb;
    if (smem > 200 * 1024)
      return fail(SEISMIC_EBUDGET, "search: shared memory per CTA (" + std::to_string(smem) + " B) exceeds 200 KB");
    int blocks = 1;
    if ((rc = search_occupancy_warp(group, k, smem, wpb, &blocks))) return rc;
    uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((nq + wpb - 1) / wpb,
                                                                     (uint64_t)std::max(1, blocks) * sm_count(ix->device)));
    a.seen_words = (uint32_t)(((ix->n_docs + 31) / 32 + 3) & ~3ull);
    if ((rc = w->seen.ensure((size_t)grid * wpb * a.seen_words * 4))) return rc;
    a.seen_bm = w->seen.as<uint32_t>();
    a.persistent = 1;
    if ((rc = launch_search_warp(a, group, smem, grid, wpb, st))) return rc;
  } else {
  a.flat = group == 1 ? 1u : 0u;
  size_t smem = search_layout(a, nw);
  if (smem > 200 * 1024)
    return fail(SEISMIC_EBUDGET, "search: shared memory per query (" + std::to_string(smem) +
                                     " B) exceeds 200 KB; lower hash_slots or the query size");
  uint32_t grid = nq;
  if (a.persistent) {
    // persistent CTAs keep a seen bitmap of the collection each, in global
    // memory (cleared per query), so deduplication never overflows
    a.HS = 16;
    smem = search_layout(a, nw);
    int blocks = 1;
    if ((rc = search_occupancy(group, nw, smem, &blocks))) return rc;
    grid = (uint32_t)std::min<uint64_t>(nq, (uint64_t)std::max(1, blocks) * sm_count(ix->device));
    a.seen_words = (uint32_t)(((ix->n_docs + 31) / 32 + 3) & ~3ull);
    if ((rc = w->seen.ensure((size_t)grid * a.seen_words * 4))) return rc;
    a.seen_bm = w->seen.as<uint32_t>();
  }
  if ((rc = launch_search(a, group, nw, smem, grid, st))) return rc;
  }
  if (!out_on_device) {
    SZ_CUDA(cudaMemcpyAsync(ids_out, d_ids, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
    SZ_CUDA(cudaMemcpyAsync(scores_out, d_sc, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
  }
  if (stats) SZ_CUDA(cudaMemcpyAsync(stats, d_stats, (size_t)nq * SEISMIC_STATS_N * 8, cudaMemcpyDeviceToHost, st));
  if (!out_on_device || stats || !queries->on_device) {
    uint32_t err = 0;
    SZ_CUDA(cudaMemcpyAsync(&err, w->queue.as<uint32_t>() + 1, 4, cudaMemcpyDeviceToHost, st));
    SZ_CUDA(cudaStreamSynchronize(st));
    if (err) return fail(SEISMIC_EINVAL, "queries: a query exceeded max_query_nnz or held a term >= dim");
  }
  return SEISMIC_OK;
}

int search_impl(seismic_index *ix, const seismic_csr *queries, const seismic_search_params *p, uint32_t *ids_out,
                float *scores_out, int32_t out_on_device, void *stream, uint64_t *stats) {
  if (!ix) return fail(SEISMIC_EINVAL, "NULL index");
  return search_ws(ix, &ix->ws, queries, p, ids_out, scores_out, out_on_device, stream, stats);
}

int exact_impl(seismic_index *ix, const seismic_csr *queries, uint32_t k, uint32_t *ids_out, float *scores_out,
               int32_t out_on_device, void *stream) {
  if (!ix || !queries || !ids_out || !scores_out) return fail(SEISMIC_EINVAL, "NULL argument");
  if (!ix->has_full) return fail(SEISMIC_EINVAL, "exact search needs an index built with keep_full_lists = 1");
  if (k == 0 || k > kExactMaxK) return fail(SEISMIC_EINVAL, "k must be in 1..1024");
  if (queries->n_rows == 0) return SEISMIC_OK;
  SZ_CUDA(cudaSetDevice(ix->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t nq = (uint32_t)queries->n_rows;
  Staged q;
  Workspace *w = &ix->ws;
  int rc = stage_queries(ix, w, queries, 1, st, q);
  if (rc) return rc;
  uint32_t *d_ids = ids_out;
  float *d_sc = scores_out;
  if (!out_on_device) {
    if ((rc = w->out.ensure((size_t)nq * k * 8))) return rc;
    d_ids = w->out.as<uint32_t>();
    d_sc = reinterpret_cast<float *>(d_ids + (size_t)nq * k);
  }
  uint32_t grid = (uint32_t)std::min<uint64_t>(nq, 2ull * sm_count(ix->device));
  size_t accb = (size_t)grid * ix->n_docs * 4;
  if ((rc = ix->ws_exact.ensure(accb))) return rc;
  SZ_CUDA(cudaMemsetAsync(ix->ws_exact.p, 0, accb, st));
  ExactArgs a{};
  a.full_ptr = ix->full_ptr.as<uint32_t>();
  a.full_doc = ix->full_doc.as<uint32_t>();
  a.full_val = ix->full_val.as<float>();
  a.n_docs = (uint32_t)ix->n_docs;
  a.q_indptr = q.ip;
  a.q_terms = q.t;
  a.q_vals = q.v;
  a.nq = nq;
  a.k = k;
  a.acc = ix->ws_exact.as<float>();
  a.ids = d_ids;
  a.scores = d_sc;
  if ((rc = launch_exact(a, grid, st))) return rc;
  if (!out_on_device) {
    SZ_CUDA(cudaMemcpyAsync(ids_out, d_ids, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
    SZ_CUDA(cudaMemcpyAsync(scores_out, d_sc, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
    SZ_CUDA(cudaStreamSynchronize(st));
  }
  return SEISMIC_OK;
}

int set_knn_impl(seismic_index *ix, const uint32_t *nbrs, uint64_t n, uint32_t kappa, int on_device) {
  if (!ix || (!nbrs && kappa)) return fail(SEISMIC_EINVAL, "NULL argument");
  if (n != ix->n_docs) return fail(SEISMIC_EINVAL, "knn: n_docs differs from the index");
  if (kappa == 0) {
    ix->knn.release();
    ix->kappa = 0;
    return SEISMIC_OK;
  }
  SZ_CUDA(cudaSetDevice(ix->device));
  std::vector<uint32_t> h;
  const uint32_t *src = nbrs;
  if (on_device) {
    h.resize(n * kappa);
    SZ_CUDA(cudaMemcpy(h.data(), nbrs, n * kappa * 4, cudaMemcpyDeviceToHost));
    src = h.data();
  }
  for (uint64_t i = 0; i < n * kappa; i++)
    if (src[i] != SEISMIC_NONE_ID && src[i] >= n) return fail(SEISMIC_EINVAL, "knn: neighbour id out of range");
  // pack the ids back to back, `bits` each, low bits first
  const uint32_t bits = knn_bits_for(n);
  const uint64_t none = (1ull << bits) - 1ull, entries = n * kappa;
  std::vector<uint32_t> words((entries * bits + 31) / 32 + 1, 0u);
  for (uint64_t e = 0; e < entries; e++) {
    const uint64_t v = src[e] == SEISMIC_NONE_ID ? none : (uint64_t)src[e];
    const uint64_t b = e * bits;
    const uint64_t w = b >> 5, sh = b & 31;
    words[w] |= (uint32_t)(v << sh);
    if (sh + bits > 32) words[w + 1] |= (uint32_t)(v >> (32 - sh));
  }
  if (int rc = upload(ix->knn, words)) return rc;
  ix->kappa = kappa;
  ix->knn_bits = bits;
  return SEISMIC_OK;
}

// kappa-NN graph of the collection itself: exact (params NULL, needs the
// unpruned lists) or with Seismic search as the paper builds it.  Each
// document is a query; the top kappa+1 minus the document itself remain.
int build_knn_impl(seismic_index *ix, uint32_t kappa, const seismic_search_params *p) {
  if (!ix || kappa == 0) return fail(SEISMIC_EINVAL, "kappa must be >= 1");
  if (kappa + 1 > kMaxK) return fail(SEISMIC_EINVAL, "kappa too large");
  if (!p && !ix->has_full) return fail(SEISMIC_EINVAL, "exact kappa-NN needs keep_full_lists = 1");
  SZ_CUDA(cudaSetDevice(ix->device));
  const uint64_t N = ix->n_docs;
  const uint32_t kk = kappa + 1;
  const uint64_t batch = 1u << 16;
  std::vector<uint32_t> graph(N * kappa, SEISMIC_NONE_ID);
  DevBuf ip, tt, vv, ids, sc;
  std::vector<uint64_t> frow(N), hip(batch + 1);
  SZ_CUDA(cudaMemcpy(frow.data(), ix->fwd_row.p, N * 8, cudaMemcpyDeviceToHost));
  int rc;
  if ((rc = ids.alloc(batch * kk * 4)) || (rc = sc.alloc(batch * kk * 4)) || (rc = ip.alloc((batch + 1) * 8)))
    return rc;
  std::vector<uint32_t> hid(batch * kk);
  seismic_search_params sp{};
  if (p) {
    sp = *p;
    sp.k = kk;
    sp.use_knn = 0;
    sp.learned = 0;
    sp.max_query_nnz = 0;
  }
  for (uint64_t r0 = 0; r0 < N; r0 += batch) {
    const uint64_t n = std::min(batch, N - r0);
    uint32_t mx = 0;
    hip[0] = 0;
    for (uint64_t i = 0; i < n; i++) {
      const uint32_t e = 8u * (uint32_t)(frow[r0 + i] >> 32);
      hip[i + 1] = hip[i] + e;
      mx = std::max(mx, e);
    }
    const uint64_t ent = hip[n];
    if ((rc = tt.ensure(ent * 2 + 16)) || (rc = vv.ensure(ent * 4 + 16))) return rc;
    SZ_CUDA(cudaMemcpy(ip.p, hip.data(), (n + 1) * 8, cudaMemcpyHostToDevice));
    k_fwd_to_csr<<<(unsigned)std::min<uint64_t>(n, 65535), 64>>>(ix->fwd_row.as<unsigned long long>(),
                                                                 ix->fwd_data.as<uint8_t>(), ix->bp.values_fp16, r0, n,
                                                                 ip.as<uint64_t>(), tt.as<uint16_t>(), vv.as<float>());
    SZ_CUDA(cudaGetLastError());
    seismic_csr qc{ip.as<uint64_t>(), tt.as<uint16_t>(), vv.as<float>(), n, ix->dim, 1};
    if (p) {
      sp.max_query_nnz = mx;
      rc = search_impl(ix, &qc, &sp, ids.as<uint32_t>(), sc.as<float>(), 1, nullptr, nullptr);
    } else {
      rc = exact_impl(ix, &qc, kk, ids.as<uint32_t>(), sc.as<float>(), 1, nullptr);
    }
    if (rc) return rc;
    SZ_CUDA(cudaMemcpy(hid.data(), ids.p, n * kk * 4, cudaMemcpyDeviceToHost));
    for (uint64_t i = 0; i < n; i++) {
      uint32_t self = (uint32_t)(r0 + i), o = 0;
      for (uint32_t j = 0; j < kk && o < kappa; j++) {
        uint32_t v = hid[i * kk + j];
        if (v == self) continue;
        graph[(r0 + i) * kappa + o++] = v;
      }
    }
  }
  return set_knn_impl(ix, graph.data(), N, kappa, 0);
}

// Neighbour-of-neighbour passes over the installed graph (not a step of the
// paper, whose Section 4.3 builds the graph approximately with the method
// itself; this applies the method's expansion step to the graph): in each
// round every document u is scored against its own list and its neighbours'
// lists, and keeps the kappa best of them other than itself.  A round reads
// only the graph from before it.
int refine_knn_impl(seismic_index *ix, uint32_t rounds, const seismic_search_params *p) {
  if (!ix) return fail(SEISMIC_EINVAL, "NULL index");
  if (!ix->kappa) return fail(SEISMIC_EINVAL, "refine: the index has no kappa-NN graph");
  if (ix->kappa + 1 > kMaxK) return fail(SEISMIC_EINVAL, "kappa too large");
  SZ_CUDA(cudaSetDevice(ix->device));
  const uint64_t N = ix->n_docs, batch = 1u << 16;
  const uint32_t kappa = ix->kappa, kk = kappa + 1;
  std::vector<uint64_t> frow(N), hip(batch + 1);
  SZ_CUDA(cudaMemcpy(frow.data(), ix->fwd_row.p, N * 8, cudaMemcpyDeviceToHost));
  DevBuf ip, tt, vv, ids, sc, seeds;
  int rc;
  if ((rc = ids.alloc(batch * kk * 4)) || (rc = sc.alloc(batch * kk * 4)) || (rc = ip.alloc((batch + 1) * 8)) ||
      (rc = seeds.alloc(batch * 4)))
    return rc;
  std::vector<uint32_t> hid(batch * kk), hseed(batch);
  seismic_search_params sp{};
  if (p) sp = *p;
  sp.k = kk;
  sp.cut = 1;
  sp.heap_factor = 1.0f;
  sp.use_knn = 1;
  sp.learned = 0;
  sp.exhaustive = 0;
  sp.alpha_q = 0.0f;
  sp.shape = 1;
  sp.persistent = 1;
  for (uint32_t round = 0; round < rounds; round++) {
    std::vector<uint32_t> graph(N * kappa, SEISMIC_NONE_ID);
    for (uint64_t r0 = 0; r0 < N; r0 += batch) {
      const uint64_t n = std::min(batch, N - r0);
      uint32_t mx = 0;
      hip[0] = 0;
      for (uint64_t i = 0; i < n; i++) {
        const uint32_t e = 8u * (uint32_t)(frow[r0 + i] >> 32);
        hip[i + 1] = hip[i] + e;
        mx = std::max(mx, e);
        hseed[i] = (uint32_t)(r0 + i);
      }
      if ((rc = tt.ensure(hip[n] * 2 + 16)) || (rc = vv.ensure(hip[n] * 4 + 16))) return rc;
      SZ_CUDA(cudaMemcpy(ip.p, hip.data(), (n + 1) * 8, cudaMemcpyHostToDevice));
      SZ_CUDA(cudaMemcpy(seeds.p, hseed.data(), n * 4, cudaMemcpyHostToDevice));
      k_fwd_to_csr<<<(unsigned)std::min<uint64_t>(n, 65535), 64>>>(ix->fwd_row.as<unsigned long long>(),
                                                                   ix->fwd_data.as<uint8_t>(), ix->bp.values_fp16, r0,
                                                                   n, ip.as<uint64_t>(), tt.as<uint16_t>(),
                                                                   vv.as<float>());
      SZ_CUDA(cudaGetLastError());
      seismic_csr qc{ip.as<uint64_t>(), tt.as<uint16_t>(), vv.as<float>(), n, ix->dim, 1};
      sp.max_query_nnz = mx;
      if ((rc = search_ws(ix, &ix->ws, &qc, &sp, ids.as<uint32_t>(), sc.as<float>(), 1, nullptr, nullptr,
                          seeds.as<uint32_t>())))
        return rc;
      SZ_CUDA(cudaMemcpy(hid.data(), ids.p, n * kk * 4, cudaMemcpyDeviceToHost));
      for (uint64_t i = 0; i < n; i++) {
        const uint32_t self = (uint32_t)(r0 + i);
        uint32_t o = 0;
        for (uint32_t j = 0; j < kk && o < kappa; j++) {
          const uint32_t v = hid[i * kk + j];
          if (v == self) continue;
          graph[(r0 + i) * kappa + o++] = v;
        }
      }
    }
    if ((rc = set_knn_impl(ix, graph.data(), N, kappa, 0))) return rc;
  }
  return SEISMIC_OK;
}

// ---------------------------------------------------------------- persistence
namespace {
constexpr char kMagic[8] = {'S', 'E', 'I', 'S', 'M', 'I', 'C', '1'};
constexpr uint32_t kVersion = 3;

struct FileHead {
  char magic[8];
  uint32_t version, dim;
  uint64_t n_docs, nnz, n_postings, n_blocks, n_sum;
  uint32_t max_blocks_per_list, max_block_docs, kappa, has_full, has_mlp, quant, knn_bits;
  float sum_absmax;
  seismic_build_params bp;
};

DevBuf *file_bufs(seismic_index *ix, int i) {
  DevBuf *b[] = {&ix->fwd_row, &ix->fwd_data, &ix->fwd_nnz, &ix->list_ptr, &ix->list_doc, &ix->cent, &ix->blk_ptr,
                 &ix->bdoc_ptr, &ix->bdoc, &ix->bdoc_row, &ix->blk_m, &ix->blk_size, &ix->sum_ptr, &ix->sum_term, &ix->sum_val,
                 &ix->sum_code, &ix->sbm, &ix->scptr, &ix->scol_blk, &ix->scol_code, &ix->scol_val, &ix->full_ptr,
                 &ix->full_doc, &ix->full_val, &ix->knn, &ix->mlp};
  return i < (int)(sizeof(b) / sizeof(b[0])) ? b[i] : nullptr;
}
}  // namespace

int save_impl(const seismic_index *cix, const char *path) {
  if (!cix || !path) return fail(SEISMIC_EINVAL, "NULL argument");
  seismic_index *ix = const_cast<seismic_index *>(cix);
  SZ_CUDA(cudaSetDevice(ix->device));
  std::unique_ptr<FILE, int (*)(FILE *)> f(std::fopen(path, "wb"), std::fclose);
  if (!f) return fail(SEISMIC_EIO, std::string("cannot open ") + path);
  FileHead h{};
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.dim = ix->dim;
  h.n_docs = ix->n_docs;
  h.nnz = ix->nnz;
  h.n_postings = ix->n_postings;
  h.n_blocks = ix->n_blocks;
  h.n_sum = ix->n_sum;
  h.max_blocks_per_list = ix->max_blocks_per_list;
  h.max_block_docs = ix->max_block_docs;
  h.kappa = ix->kappa;
  h.knn_bits = ix->knn_bits;
  h.has_full = ix->has_full;
  h.has_mlp = ix->has_mlp;
  h.quant = ix->bp.quantize_u8;
  h.sum_absmax = ix->sum_absmax;
  h.bp = ix->bp;
  if (std::fwrite(&h, sizeof(h), 1, f.get()) != 1) return fail(SEISMIC_EIO, "write failed");
  std::vector<uint8_t> tmp;
  for (int i = 0;; i++) {
    DevBuf *b = file_bufs(ix, i);
    if (!b) break;
    uint64_t n = b->p ? b->bytes : 0;
    if (std::fwrite(&n, 8, 1, f.get()) != 1) return fail(SEISMIC_EIO, "write failed");
    if (!n) continue;
    tmp.resize(n);
    SZ_CUDA(cudaMemcpy(tmp.data(), b->p, n, cudaMemcpyDeviceToHost));
    if (std::fwrite(tmp.data(), 1, n, f.get()) != n) return fail(SEISMIC_EIO, "write failed");
  }
  return SEISMIC_OK;
}

int load_impl(const char *path, seismic_index **out) {
  if (!path || !out) return fail(SEISMIC_EINVAL, "NULL argument");
  std::unique_ptr<FILE, int (*)(FILE *)> f(std::fopen(path, "rb"), std::fclose);
  if (!f) return fail(SEISMIC_EIO, std::string("cannot open ") + path);
  FileHead h{};
  if (std::fread(&h, sizeof(h), 1, f.get()) != 1 || std::memcmp(h.magic, kMagic, 8) || h.version != kVersion)
    return fail(SEISMIC_EIO, "not a seismic index file of this version");
  std::unique_ptr<seismic_index> ix(new seismic_index());
  SZ_CUDA(cudaGetDevice(&ix->device));
  ix->dim = h.dim;
  ix->n_docs = h.n_docs;
  ix->nnz = h.nnz;
  ix->n_postings = h.n_postings;
  ix->n_blocks = h.n_blocks;
  ix->n_sum = h.n_sum;
  ix->max_blocks_per_list = h.max_blocks_per_list;
  ix->max_block_docs = h.max_block_docs;
  ix->kappa = h.kappa;
  ix->knn_bits = h.knn_bits;
  ix->has_full = h.has_full;
  ix->has_mlp = h.has_mlp;
  ix->bp = h.bp;
  ix->sum_absmax = h.sum_absmax;
  std::vector<uint8_t> tmp;
  for (int i = 0;; i++) {
    DevBuf *b = file_bufs(ix.get(), i);
    if (!b) break;
    uint64_t n = 0;
    if (std::fread(&n, 8, 1, f.get()) != 1) return fail(SEISMIC_EIO, "truncated index file");
    if (!n) continue;
    tmp.resize(n);
    if (std::fread(tmp.data(), 1, n, f.get()) != n) return fail(SEISMIC_EIO, "truncated index file");
    int rc = b->alloc(n);
    if (rc) return rc;
    SZ_CUDA(cudaMemcpy(b->p, tmp.data(), n, cudaMemcpyHostToDevice));
  }
  *out = ix.release();
  return SEISMIC_OK;
}

int export_impl(const seismic_index *ix, int32_t what, void *dst, uint64_t cap, uint64_t *needed) {
  if (!ix) return fail(SEISMIC_EINVAL, "NULL index");
  const DevBuf *b = nullptr;
  uint64_t n = 0;
  switch (what) {
    case SEISMIC_X_LIST_PTR: b = &ix->list_ptr; n = (ix->dim + 1ull) * 4; break;
    case SEISMIC_X_LIST_DOC: b = &ix->list_doc; n = ix->n_postings * 4; break;
    case SEISMIC_X_BLK_PTR: b = &ix->blk_ptr; n = (ix->dim + 1ull) * 4; break;
    case SEISMIC_X_BDOC_PTR: b = &ix->bdoc_ptr; n = (ix->n_blocks + 1) * 4; break;
    case SEISMIC_X_BDOC: b = &ix->bdoc; n = ix->n_postings * 4; break;
    case SEISMIC_X_BLK_M: b = &ix->blk_m; n = ix->n_blocks * 4; break;
    case SEISMIC_X_BLK_SIZE: b = &ix->blk_size; n = ix->n_blocks * 4; break;
    case SEISMIC_X_SUM_PTR: b = &ix->sum_ptr; n = (ix->n_blocks + 1) * 4; break;
    case SEISMIC_X_SUM_TERM: b = &ix->sum_term; n = ix->n_sum * 2; break;
    case SEISMIC_X_SUM_VAL: b = &ix->sum_val; n = ix->n_sum * 4; break;
    case SEISMIC_X_SUM_CODE: b = &ix->sum_code; n = ix->bp.quantize_u8 ? ix->n_sum : 0; break;
    case SEISMIC_X_CENT: b = &ix->cent; n = ix->n_postings * 4; break;
    case SEISMIC_X_SBM: b = &ix->sbm; n = b->p ? b->bytes : 0; break;
    case SEISMIC_X_SCPTR: b = &ix->scptr; n = b->p ? b->bytes : 0; break;
    case SEISMIC_X_SCOL_BLK: b = &ix->scol_blk; n = b->p ? b->bytes : 0; break;
    case SEISMIC_X_SCOL_CODE: b = &ix->scol_code; n = b->p ? b->bytes : 0; break;
    case SEISMIC_X_SCOL_VAL: b = &ix->scol_val; n = b->p ? b->bytes : 0; break;
    default: return fail(SEISMIC_EINVAL, "unknown export id");
  }
  if (n && !b->p) return fail(SEISMIC_EINVAL, "array not kept: build with keep_block_summaries = 1");
  if (needed) *needed = n;
  if (!dst || cap < n || n == 0) return SEISMIC_OK;
  SZ_CUDA(cudaSetDevice(ix->device));
  SZ_CUDA(cudaMemcpy(dst, b->p, n, cudaMemcpyDeviceToHost));
  return SEISMIC_OK;
}

}  // namespace seismic

using namespace seismic;

#define SZ_GUARD(expr)                                        \
  try {                                                       \
    return (expr);                                            \
  } catch (const std::bad_alloc &) {                          \
    return fail(SEISMIC_ENOMEM, "host allocation failed");    \
  } catch (const std::exception &e) {                         \
    return fail(SEISMIC_EINVAL, e.what());                    \
  }

extern "C" {

int seismic_build(const seismic_csr *docs, const seismic_build_params *params, seismic_index **out) {
  SZ_GUARD(build_index(docs, params, out));
}

int seismic_search(seismic_index *index, const seismic_csr *queries, const seismic_search_params *params,
                   uint32_t *ids_out, float *scores_out, int32_t out_on_device, void *stream, uint64_t *stats) {
  SZ_GUARD(search_impl(index, queries, params, ids_out, scores_out, out_on_device, stream, stats));
}

int seismic_search_exact(seismic_index *index, const seismic_csr *queries, uint32_t k, uint32_t *ids_out,
                         float *scores_out, int32_t out_on_device, void *stream) {
  SZ_GUARD(exact_impl(index, queries, k, ids_out, scores_out, out_on_device, stream));
}

int seismic_set_knn(seismic_index *index, const uint32_t *nbrs, uint64_t n_docs, uint32_t kappa, int32_t on_device) {
  SZ_GUARD(set_knn_impl(index, nbrs, n_docs, kappa, on_device));
}

int seismic_build_knn(seismic_index *index, uint32_t kappa, const seismic_search_params *params) {
  SZ_GUARD(build_knn_impl(index, kappa, params));
}

int seismic_refine_knn(seismic_index *index, uint32_t rounds, const seismic_search_params *params) {
  SZ_GUARD(refine_knn_impl(index, rounds, params));
}

int seismic_get_knn(const seismic_index *index, uint32_t *nbrs, uint64_t cap_entries) {
  if (!index || !nbrs) return fail(SEISMIC_EINVAL, "NULL argument");
  if (!index->kappa) return fail(SEISMIC_EINVAL, "the index has no kappa-NN graph");
  const uint64_t n = index->n_docs * index->kappa, bits = index->knn_bits, none = (1ull << bits) - 1ull;
  if (cap_entries < n) return fail(SEISMIC_EINVAL, "buffer too small");
  std::vector<uint32_t> words(index->knn.bytes / 4);
  SZ_CUDA(cudaSetDevice(index->device));
  SZ_CUDA(cudaMemcpy(words.data(), index->knn.p, words.size() * 4, cudaMemcpyDeviceToHost));
  for (uint64_t e = 0; e < n; e++) {
    const uint64_t b = e * bits, w = b >> 5, sh = b & 31;
    uint64_t x = words[w];
    if (sh + bits > 32) x |= (uint64_t)words[w + 1] << 32;
    const uint64_t v = (x >> sh) & none;
    nbrs[e] = v == none ? SEISMIC_NONE_ID : (uint32_t)v;
  }
  return SEISMIC_OK;
}

int seismic_save(const seismic_index *index, const char *path) { SZ_GUARD(save_impl(index, path)); }

int seismic_load(const char *path, seismic_index **out) { SZ_GUARD(load_impl(path, out)); }

int seismic_info(const seismic_index *ix, seismic_index_info *out) {
  if (!ix || !out) return fail(SEISMIC_EINVAL, "NULL argument");
  out->n_docs = ix->n_docs;
  out->nnz = ix->nnz;
  out->n_postings = ix->n_postings;
  out->n_blocks = ix->n_blocks;
  out->n_summary_entries = ix->n_sum;
  out->dim = ix->dim;
  out->kappa = ix->kappa;
  out->quantize_u8 = ix->bp.quantize_u8;
  out->has_full_lists = ix->has_full;
  out->has_mlp = ix->has_mlp;
  out->device_bytes = device_bytes(ix);
  out->values_fp16 = ix->bp.values_fp16;
  out->knn_bits = ix->knn_bits;
  out->knn_bytes = ix->kappa ? ix->knn.bytes : 0;
  return SEISMIC_OK;
}

int seismic_export(const seismic_index *index, int32_t what, void *dst, uint64_t cap_bytes, uint64_t *needed_bytes) {
  SZ_GUARD(export_impl(index, what, dst, cap_bytes, needed_bytes));
}

void seismic_free(seismic_index *index) {
  if (!index) return;
  cudaSetDevice(index->device);
  delete index;
}

const char *seismic_last_error(void) { return g_err.c_str(); }

const char *seismic_version(void) { return "seismic-gb300 1.0 (sm_103a)"; }

}  // extern "C"

// Index construction: Algorithm "Indexing with Seismic" (Section 4.4).
//
// Host (threads): validation, forward-index layout, full posting lists,
// centroid sampling and blocks.
// Device: the posting lists pruned to their top-lambda values (prune.cu; Set
// alpha-MSS, fixed-lambda form of Table 4, or the proportional form of
// Definition "Set alpha-MSS"); the shallow k-means assignment (Section 4.1.2):
// every list member against every centroid of its list; then (summary.cu) the
// max summaries (Eq. "summary") with their alpha-MSS and 8-bit quantisation
// (Section 4.1.3), and the term-major summary layout the search reads.
#include <cuda_fp16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>

#include "seismic_impl.h"

namespace seismic {

namespace {

struct HostCsr {
  std::vector<uint64_t> ip;
  std::vector<uint16_t> t;
  std::vector<float> v;
  uint64_t n = 0;
  uint32_t d = 0;
};

// Copies `m` to host (if needed), validates it and drops explicit zeros.
// With fp16 = 1 every value is first rounded to the nearest fp16 (ties to
// even): the index then stores, and search scores, that rounded collection
// (the 16-bit value setup of Section 5.4); a value that rounds to 0 is
// dropped like an explicit zero, one beyond the fp16 range is refused.
int fetch_docs(const seismic_csr *m, HostCsr &h, int fp16) {
  if (!m || !m->indptr || m->n_rows == 0) return fail(SEISMIC_EINVAL, "documents: empty or NULL CSR");
  if (m->dim == 0 || m->dim > 65535) return fail(SEISMIC_EINVAL, "documents: dim must be in 1..65535");
  if (m->n_rows >= 0xFFFFFFFFull) return fail(SEISMIC_EINVAL, "documents: more than 2^32-2 rows");
  std::vector<uint64_t> ip(m->n_rows + 1);
  const uint64_t *ipp = m->indptr;
  const uint16_t *tp = m->terms;
  const float *vp = m->vals;
  std::vector<uint16_t> tbuf;
  std::vector<float> vbuf;
  if (m->on_device) {
    SZ_CUDA(cudaMemcpy(ip.data(), m->indptr, ip.size() * 8, cudaMemcpyDeviceToHost));
    uint64_t nnz = ip.back();
    tbuf.resize(nnz);
    vbuf.resize(nnz);
    if (nnz) {
      SZ_CUDA(cudaMemcpy(tbuf.data(), m->terms, nnz * 2, cudaMemcpyDeviceToHost));
      SZ_CUDA(cudaMemcpy(vbuf.data(), m->vals, nnz * 4, cudaMemcpyDeviceToHost));
    }
    ipp = ip.data();
    tp = tbuf.data();
    vp = vbuf.data();
  }
  seismic_csr hc = *m;
  hc.indptr = ipp;
  hc.terms = tp;
  hc.vals = vp;
  hc.on_device = 0;
  int rc = validate_host_csr(&hc, "documents", m->dim);
  if (rc) return rc;
  h.n = m->n_rows;
  h.d = m->dim;
  h.ip.assign(h.n + 1, 0);
  auto value = [&](uint64_t p) { return fp16 ? __half2float(__float2half_rn(vp[p])) : vp[p]; };
  if (fp16)
    for (uint64_t p = 0; p < ipp[h.n]; p++)
      if (std::isinf(value(p)))
        return fail(SEISMIC_EINVAL, "documents: a value exceeds the fp16 range (|v| > 65504)");
  uint64_t nnz = 0;
  for (uint64_t i = 0; i < h.n; i++) {
    uint64_t c = 0;
    for (uint64_t p = ipp[i]; p < ipp[i + 1]; p++) c += value(p) != 0.0f;
    if (c > kMaxRowNnzBuild)
      return fail(SEISMIC_EINVAL, "documents: a row has more than " + std::to_string(kMaxRowNnzBuild) +
                                      " nonzeros");
    nnz += c;
    h.ip[i + 1] = nnz;
  }
  h.t.resize(nnz);
  h.v.resize(nnz);
  for (uint64_t i = 0, o = 0; i < h.n; i++)
    for (uint64_t p = ipp[i]; p < ipp[i + 1]; p++) {
      const float v = value(p);
      if (v != 0.0f) {
        h.t[o] = tp[p];
        h.v[o] = v;
        o++;
      }
    }
  return SEISMIC_OK;
}

// Phase timings of a build, printed to stderr when SEISMIC_BUILD_TRACE=1.
struct PhaseTimer {
  bool on = std::getenv("SEISMIC_BUILD_TRACE") && std::getenv("SEISMIC_BUILD_TRACE")[0] == '1';
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  void mark(const char *what) {
    if (!on) return;
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "seismic build: %-28s %8.2f s\n", what, std::chrono::duration<double>(now - t).count());
    t = now;
  }
};

uint64_t splitmix64_next(uint64_t &state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ------------------------------------------------------------------ clustering kernel
// One CTA per list.  Centroids are taken in chunks whose nonzeros fit in
// shared memory; a chunk is turned into a small inverted index (term ->
// (centroid, value)) addressed through a bitmap + popcount rank over the
// vocabulary.  Each thread then scores one list member against the whole
// chunk: it walks the member's terms in ascending order and, for each term the
// chunk holds, adds the exact fp64 product into its per-centroid fp64
// accumulators.  Each accumulator thus receives the nonzero products of the
// two vectors' common terms in ascending term order: the same fp64 sum as a
// sequential merge of the two sorted rows.  Argmax ties keep the lower
// centroid index.
constexpr int kAsgThreads = 128;
constexpr int kAsgCC = 48;        // centroids per chunk (cluster index fits in u8); 2 CTAs per SM
constexpr int kAsgMaxEnt = 8192;  // nonzeros per chunk (= kMaxRowNnzBuild bound below)
static_assert(kMaxRowNnzBuild <= kAsgMaxEnt, "a centroid row must fit one chunk");
static_assert((size_t)kAsgCC * kAsgThreads * 8 >= (size_t)(kAsgMaxEnt + 1) * 4, "the cursors share the accumulators");

__device__ __forceinline__ void asg_scan_rank(const uint32_t *bits, uint16_t *rank, uint32_t W, uint32_t *wtmp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kAsgThreads / 32;
  uint32_t per = (W + kAsgThreads - 1) / kAsgThreads, lo = min(W, tid * per), hi = min(W, lo + per);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; i++) s += __popc(bits[i]);
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < nw ? wtmp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < nw) wtmp[lane] = v;
  }
  __syncthreads();
  uint32_t base = (warp ? wtmp[warp - 1] : 0) + x - s;
  for (uint32_t i = lo; i < hi; i++) {
    rank[i] = (uint16_t)base;
    base += __popc(bits[i]);
  }
  __syncthreads();
}

// exclusive scan of cnt[0..n) into off[0..n] (u16) and cnt (cursor copy)
__device__ __forceinline__ void asg_scan_counts(uint32_t *cnt, uint16_t *off, uint32_t n, uint32_t *wtmp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kAsgThreads / 32;
  uint32_t per = (n + kAsgThreads - 1) / kAsgThreads, lo = min(n, tid * per), hi = min(n, lo + per);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; i++) s += cnt[i];
  uint32_t x = s;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < nw ? wtmp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < nw) wtmp[lane] = v;
  }
  __syncthreads();
  uint32_t base = (warp ? wtmp[warp - 1] : 0) + x - s;
  for (uint32_t i = lo; i < hi; i++) {
    uint32_t c = cnt[i];
    off[i] = (uint16_t)base;
    cnt[i] = base;
    base += c;
  }
  if (tid == kAsgThreads - 1) off[n] = (uint16_t)wtmp[nw - 1];
  __syncthreads();
}

__global__ void __launch_bounds__(kAsgThreads) k_assign(
    const uint32_t *__restrict__ work, uint32_t n_work, const uint32_t *__restrict__ list_ptr,
    const uint32_t *__restrict__ list_doc, const uint32_t *__restrict__ cent_ptr,
    const uint32_t *__restrict__ cent_doc, const uint64_t *__restrict__ indptr,
    const uint16_t *__restrict__ terms, const float *__restrict__ vals, uint32_t dim,
    const unsigned long long *__restrict__ fwd_row, const uint8_t *__restrict__ fwd, int fp16,
    double *__restrict__ best, uint32_t *__restrict__ assign) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t W = (dim + 31) / 32;
  double *acc = reinterpret_cast<double *>(smem);                    // kAsgCC * kAsgThreads
  // the chunk's per-term counts and cursors (kAsgMaxEnt + 1) live in the
  // accumulators' space: they are dead once the chunk's index is built
  uint32_t *ccur = reinterpret_cast<uint32_t *>(smem);
  float *ent_w = reinterpret_cast<float *>(acc + kAsgCC * kAsgThreads);  // kAsgMaxEnt
  uint32_t *cbits = reinterpret_cast<uint32_t *>(ent_w + kAsgMaxEnt);    // W
  uint16_t *coff = reinterpret_cast<uint16_t *>(cbits + W);               // kAsgMaxEnt + 1
  uint16_t *crank = coff + (kAsgMaxEnt + 1);                              // W
  uint8_t *ent_c = reinterpret_cast<uint8_t *>(crank + W);                // kAsgMaxEnt
  __shared__ uint32_t wtmp[32];
  const int tid = threadIdx.x;

  for (uint32_t wi = blockIdx.x; wi < n_work; wi += gridDim.x) {
    const uint32_t t = work[wi];
    const uint32_t lp0 = list_ptr[t], n = list_ptr[t + 1] - lp0;
    const uint32_t cp0 = cent_ptr[t], nb = cent_ptr[t + 1] - cp0;
    uint32_t c0 = 0;
    while (c0 < nb) {
      uint32_t c1 = c0, ent = 0;
      while (c1 < nb && c1 - c0 < (uint32_t)kAsgCC) {
        uint32_t cd = cent_doc[cp0 + c1];
        uint32_t len = (uint32_t)(indptr[cd + 1] - indptr[cd]);
        if (c1 > c0 && ent + len > (uint32_t)kAsgMaxEnt) break;
        ent += len;
        c1++;
      }
      for (uint32_t i = tid; i < W; i += kAsgThreads) cbits[i] = 0;
      __syncthreads();
      for (uint32_t c = c0; c < c1; c++) {
        uint32_t cd = cent_doc[cp0 + c];
        for (uint64_t p = indptr[cd] + tid; p < indptr[cd + 1]; p += kAsgThreads) {
          uint16_t s = terms[p];
          atomicOr(&cbits[s >> 5], 1u << (s & 31));
        }
      }
      __syncthreads();
      asg_scan_rank(cbits, crank, W, wtmp);
      const uint32_t ndist = (W ? crank[W - 1] + __popc(cbits[W - 1]) : 0);
      for (uint32_t i = tid; i <= ndist; i += kAsgThreads) ccur[i] = 0;
      __syncthreads();
      for (uint32_t c = c0; c < c1; c++) {
        uint32_t cd = cent_doc[cp0 + c];
        for (uint64_t p = indptr[cd] + tid; p < indptr[cd + 1]; p += kAsgThreads) {
          uint16_t s = terms[p];
          uint32_t w = cbits[s >> 5];
          uint32_t idx = crank[s >> 5] + __popc(w & ((1u << (s & 31)) - 1u));
          atomicAdd(&ccur[idx], 1u);
        }
      }
      __syncthreads();
      asg_scan_counts(ccur, coff, ndist, wtmp);
      for (uint32_t c = c0; c < c1; c++) {
        uint32_t cd = cent_doc[cp0 + c];
        for (uint64_t p = indptr[cd] + tid; p < indptr[cd + 1]; p += kAsgThreads) {
          uint16_t s = terms[p];
          uint32_t w = cbits[s >> 5];
          uint32_t idx = crank[s >> 5] + __popc(w & ((1u << (s & 31)) - 1u));
          uint32_t pos = atomicAdd(&ccur[idx], 1u);
          ent_c[pos] = (uint8_t)(c - c0);
          ent_w[pos] = vals[p];
        }
      }
      __syncthreads();
      const uint32_t ncc = c1 - c0;
      double *a = acc + tid;
      for (uint32_t i = tid; i < n; i += kAsgThreads) {
        const uint32_t j = list_doc[lp0 + i];
        for (uint32_t cc = 0; cc < ncc; cc++) a[cc * kAsgThreads] = 0.0;
        // the member's terms in ascending order, 8 per 16-byte load from its
        // forward-index record; a value is read only where the chunk holds the term
        const unsigned long long row = fwd_row[j];
        const uint8_t *rec = fwd + (size_t)(uint32_t)row * kUnitBytes;
        const uint32_t nch = (uint32_t)(row >> 32), nnz = (uint32_t)(indptr[j + 1] - indptr[j]);
        for (uint32_t o = 0; o < nch; o++) {
          const uint4 tq = *reinterpret_cast<const uint4 *>(rec + (size_t)o * (fp16 ? kUnitBytes : 16u));
          const uint32_t tw[4] = {tq.x, tq.y, tq.z, tq.w};
#pragma unroll
          for (uint32_t e8 = 0; e8 < kChunk; e8++) {
            if (o * kChunk + e8 >= nnz) break;  // the padding after the row's last entry
            const uint32_t s = (e8 & 1) ? (tw[e8 >> 1] >> 16) : (tw[e8 >> 1] & 0xFFFFu);
            const uint32_t w = cbits[s >> 5];
            const uint32_t bit = 1u << (s & 31);
            if (!(w & bit)) continue;
            const uint32_t idx = crank[s >> 5] + __popc(w & (bit - 1u));
            double u;
            if (fp16) {
              u = (double)__half2float(*reinterpret_cast<const __half *>(rec + (size_t)o * kUnitBytes + 16 + 2 * e8));
            } else {
              u = (double)*reinterpret_cast<const float *>(rec + (size_t)kUnitBytes * ((nch + 1) / 2 + o) + 4 * e8);
            }
            for (uint32_t e = coff[idx]; e < coff[idx + 1]; e++)
              a[(uint32_t)ent_c[e] * kAsgThreads] = __dadd_rn(a[(uint32_t)ent_c[e] * kAsgThreads],
                                                                __dmul_rn(u, (double)ent_w[e]));
          }
        }
        double bv;
        uint32_t bc, cc0;
        if (c0 == 0) {
          bv = a[0];
          bc = 0;
          cc0 = 1;
        } else {
          bv = best[lp0 + i];
          bc = assign[lp0 + i];
          cc0 = 0;
        }
        for (uint32_t cc = cc0; cc < ncc; cc++) {
          double v = a[cc * kAsgThreads];
          if (v > bv) {
            bv = v;
            bc = c0 + cc;
          }
        }
        best[lp0 + i] = bv;
        assign[lp0 + i] = bc;
      }
      __syncthreads();
      c0 = c1;
    }
  }
}

size_t asg_smem_bytes(uint32_t dim) {
  uint32_t W = (dim + 31) / 32;
  return (size_t)kAsgCC * kAsgThreads * 8 + (size_t)kAsgMaxEnt * 4 + W * 4 + (size_t)(kAsgMaxEnt + 1) * 2 + W * 2 +
         kAsgMaxEnt + 16;
}

}  // namespace

int validate_host_csr(const seismic_csr *m, const char *what, uint32_t dim_expect) {
  std::string w(what);
  if (!m || !m->indptr) return fail(SEISMIC_EINVAL, w + ": NULL CSR");
  if (m->dim != dim_expect) return fail(SEISMIC_EINVAL, w + ": dim differs from the index");
  if (m->indptr[0] != 0) return fail(SEISMIC_EINVAL, w + ": indptr[0] != 0");
  uint64_t nnz = m->indptr[m->n_rows];
  if (nnz && (!m->terms || !m->vals)) return fail(SEISMIC_EINVAL, w + ": NULL terms/vals");
  for (uint64_t i = 0; i < m->n_rows; i++) {
    if (m->indptr[i + 1] < m->indptr[i]) return fail(SEISMIC_EINVAL, w + ": indptr decreases at row " + std::to_string(i));
    for (uint64_t p = m->indptr[i]; p < m->indptr[i + 1]; p++) {
      if (m->terms[p] >= m->dim) return fail(SEISMIC_EINVAL, w + ": term id >= dim in row " + std::to_string(i));
      if (p > m->indptr[i] && m->terms[p] <= m->terms[p - 1])
        return fail(SEISMIC_EINVAL, w + ": terms not strictly increasing in row " + std::to_string(i));
      if (!std::isfinite(m->vals[p])) return fail(SEISMIC_EINVAL, w + ": non-finite value in row " + std::to_string(i));
    }
  }
  return SEISMIC_OK;
}

uint64_t device_bytes(const seismic_index *ix) {
  const DevBuf *b[] = {&ix->fwd_row, &ix->fwd_data, &ix->fwd_nnz, &ix->list_ptr, &ix->list_doc, &ix->cent,
                       &ix->blk_ptr, &ix->bdoc_ptr, &ix->bdoc, &ix->bdoc_row, &ix->blk_m, &ix->blk_size, &ix->sum_ptr,
                       &ix->sum_term, &ix->sum_val, &ix->sum_code, &ix->sbm, &ix->scptr, &ix->scol_blk,
                       &ix->scol_code, &ix->scol_val, &ix->full_ptr, &ix->full_doc, &ix->full_val, &ix->knn, &ix->mlp};
  uint64_t s = 0;
  for (auto *x : b) s += x->bytes;
  return s;
}

int build_index(const seismic_csr *docs, const seismic_build_params *bp, seismic_index **out) {
  if (!bp || !out) return fail(SEISMIC_EINVAL, "NULL params/out");
  if (!(bp->alpha > 0.0 && bp->alpha <= 1.0)) return fail(SEISMIC_EINVAL, "alpha must be in (0, 1]");
  if (bp->beta == 0 && !(bp->beta_frac > 0.0)) return fail(SEISMIC_EINVAL, "beta must be >= 1");
  if (bp->lambda_frac < 0.0 || bp->lambda_frac > 1.0 || bp->beta_frac < 0.0 || bp->beta_frac > 1.0)
    return fail(SEISMIC_EINVAL, "lambda_frac / beta_frac must be in [0, 1]");
  if (bp->values_fp16 != 0 && bp->values_fp16 != 1) return fail(SEISMIC_EINVAL, "values_fp16 must be 0 or 1");
  const int fp16 = bp->values_fp16;
  PhaseTimer timer;
  HostCsr D;
  int rc = fetch_docs(docs, D, fp16);
  if (rc) return rc;
  const int T = hw_threads(bp->threads);
  const uint32_t d = D.d;
  std::unique_ptr<seismic_index> ix(new seismic_index());
  SZ_CUDA(cudaGetDevice(&ix->device));
  ix->dim = d;
  ix->n_docs = D.n;
  ix->nnz = D.ip.back();
  ix->bp = *bp;

  timer.mark("input");
  // ---- forward index: rows of 8-entry chunks in sector-aligned records
  std::vector<uint64_t> frow(D.n);  // first unit | chunks << 32
  {
    std::vector<uint16_t> rnnz(D.n);
    uint64_t units = 0;
    for (uint64_t i = 0; i < D.n; i++) {
      const uint64_t n = D.ip[i + 1] - D.ip[i];
      const uint32_t nch = (uint32_t)((n + kChunk - 1) / kChunk);
      rnnz[i] = (uint16_t)n;
      frow[i] = units | ((uint64_t)nch << 32);
      units += row_units(nch, fp16);
      if (units > 0xFFFFFFFFull) return fail(SEISMIC_EINVAL, "forward index exceeds 2^32 32-byte units");
    }
    std::vector<uint8_t> data((size_t)units * kUnitBytes, 0);
    parallel_ranges((int64_t)D.n, T, 4096, [&](int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; i++) {
        const uint64_t n = D.ip[i + 1] - D.ip[i];
        const uint32_t nch = (uint32_t)(frow[i] >> 32);
        uint8_t *rec = data.data() + (size_t)(uint32_t)frow[i] * kUnitBytes;
        for (uint64_t p = 0; p < n; p++) {
          const uint64_t o = p / kChunk, e = p % kChunk;
          const uint16_t t = D.t[D.ip[i] + p];
          const float v = D.v[D.ip[i] + p];
          if (fp16) {
            std::memcpy(rec + o * kUnitBytes + 2 * e, &t, 2);
            const __half hv = __float2half_rn(v);  // exact: v is already an fp16 value
            std::memcpy(rec + o * kUnitBytes + 16 + 2 * e, &hv, 2);
          } else {
            std::memcpy(rec + 2 * p, &t, 2);
            std::memcpy(rec + (size_t)kUnitBytes * ((nch + 1) / 2) + 4 * p, &v, 4);
          }
        }
      }
    });
    if ((rc = upload(ix->fwd_row, frow)) || (rc = upload(ix->fwd_data, data)) || (rc = upload(ix->fwd_nnz, rnnz)))
      return rc;
  }

  timer.mark("forward index");
  // ---- full inverted lists (ascending doc ids)
  std::vector<uint64_t> fptr(d + 1, 0);
  std::vector<uint32_t> fdoc(ix->nnz);
  std::vector<float> fval(ix->nnz);
  {
    // a counting sort in parallel: each worker counts, then places, the
    // postings of its own contiguous range of documents; a term's postings from
    // earlier ranges come first, so every list is in ascending document order
    const uint64_t parts = std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)T, D.n));
    std::vector<std::vector<uint64_t>> hist(parts, std::vector<uint64_t>(d, 0));
    auto range = [&](uint64_t r, uint64_t &lo, uint64_t &hi) {
      lo = D.n * r / parts;
      hi = D.n * (r + 1) / parts;
    };
    parallel_for((int64_t)parts, T, [&](int64_t r, int) {
      uint64_t lo, hi;
      range((uint64_t)r, lo, hi);
      for (uint64_t p = D.ip[lo]; p < D.ip[hi]; p++) hist[r][D.t[p]]++;
    });
    uint64_t run = 0;
    for (uint32_t t = 0; t < d; t++) {
      fptr[t] = run;
      for (uint64_t r = 0; r < parts; r++) {
        const uint64_t c = hist[r][t];
        hist[r][t] = run;  // this range's first slot in list t
        run += c;
      }
    }
    fptr[d] = run;
    parallel_for((int64_t)parts, T, [&](int64_t r, int) {
      uint64_t lo, hi;
      range((uint64_t)r, lo, hi);
      std::vector<uint64_t> &cur = hist[r];
      for (uint64_t i = lo; i < hi; i++)
        for (uint64_t p = D.ip[i]; p < D.ip[i + 1]; p++) {
          const uint64_t o = cur[D.t[p]]++;
          fdoc[o] = (uint32_t)i;
          fval[o] = D.v[p];
        }
    });
  }
  if (bp->keep_full_lists) {
    if (ix->nnz > 0xFFFFFFFFull) return fail(SEISMIC_EINVAL, "keep_full_lists: more than 2^32 nonzeros");
    std::vector<uint32_t> fp32(fptr.begin(), fptr.end());
    if ((rc = upload(ix->full_ptr, fp32)) || (rc = upload(ix->full_doc, fdoc)) || (rc = upload(ix->full_val, fval)))
      return rc;
    ix->has_full = 1;
  }

  timer.mark("full lists");
  // ---- pruned lists: top-lambda_t postings by (value desc, doc asc)
  std::vector<uint32_t> lptr(d + 1, 0);
  for (uint32_t t = 0; t < d; t++) {
    uint64_t full = fptr[t + 1] - fptr[t];
    uint64_t lam;
    if (bp->lambda_frac > 0.0) lam = (uint64_t)std::ceil(bp->lambda_frac * (double)full);
    else lam = bp->lambda ? bp->lambda : full;
    if (lam > full) lam = full;
    if ((uint64_t)lptr[t] + lam > 0xFFFFFFFFull) return fail(SEISMIC_EINVAL, "more than 2^32 postings");
    lptr[t + 1] = lptr[t] + (uint32_t)lam;
  }
  const uint64_t npost = lptr[d];
  ix->n_postings = npost;
  std::vector<uint32_t> ldoc(npost);
  {
    // on the device: each list's top-lambda_t by (value desc, doc asc), from the full lists
    DevBuf d_fptr, d_fdoc, d_fval, d_lptr, d_ldoc;
    const uint32_t *gdoc = ix->full_doc.as<uint32_t>();
    const float *gval = ix->full_val.as<float>();
    if ((rc = upload(d_fptr, fptr)) || (rc = upload(d_lptr, lptr)) || (rc = d_ldoc.alloc(npost * 4))) return rc;
    if (!ix->has_full) {
      if ((rc = upload(d_fdoc, fdoc)) || (rc = upload(d_fval, fval))) return rc;
      gdoc = d_fdoc.as<uint32_t>();
      gval = d_fval.as<float>();
    }
    uint32_t cap = 0;
    if ((rc = launch_prune(d_fptr.as<uint64_t>(), gdoc, gval, d_lptr.as<uint32_t>(), d, d_ldoc.as<uint32_t>(), &cap,
                           0)))
      return rc;
    SZ_CUDA(cudaDeviceSynchronize());
    if (npost) SZ_CUDA(cudaMemcpy(ldoc.data(), d_ldoc.p, npost * 4, cudaMemcpyDeviceToHost));
    // lists whose lambda_t exceeds what the device sorts in shared memory: on host threads
    parallel_for(d, T, [&](int64_t t, int) {
      const uint64_t a = fptr[t], n = fptr[t + 1] - a, lam = lptr[t + 1] - lptr[t];
      if (lam <= cap) return;
      std::vector<uint32_t> idx(n);
      for (uint64_t i = 0; i < n; i++) idx[i] = (uint32_t)i;
      auto cmp = [&](uint32_t x, uint32_t y) {
        float vx = fval[a + x], vy = fval[a + y];
        if (vx != vy) return vx > vy;
        return fdoc[a + x] < fdoc[a + y];
      };
      if (lam < n) std::partial_sort(idx.begin(), idx.begin() + lam, idx.end(), cmp);
      else std::sort(idx.begin(), idx.end(), cmp);
      for (uint64_t i = 0; i < lam; i++) ldoc[lptr[t] + i] = fdoc[a + idx[i]];
    });
  }
  std::vector<uint64_t>().swap(fptr);
  std::vector<uint32_t>().swap(fdoc);
  std::vector<float>().swap(fval);

  timer.mark("pruned lists");
  // ---- centroids: partial Fisher-Yates per list, splitmix64(seed ^ t*golden)
  std::vector<uint32_t> cptr2(d + 1, 0);
  for (uint32_t t = 0; t < d; t++) {
    uint32_t n = lptr[t + 1] - lptr[t];
    uint32_t nb = 0;
    if (n) {
      nb = bp->beta_frac > 0.0 ? (uint32_t)std::ceil(bp->beta_frac * (double)n) : bp->beta;
      nb = std::max(1u, std::min(nb, n));
    }
    cptr2[t + 1] = cptr2[t] + nb;
  }
  std::vector<uint32_t> cdoc(cptr2[d]);
  parallel_for(d, T, [&](int64_t t, int) {
    uint32_t n = lptr[t + 1] - lptr[t], nb = cptr2[t + 1] - cptr2[t];
    if (!nb) return;
    std::vector<uint32_t> pos(n);
    for (uint32_t i = 0; i < n; i++) pos[i] = i;
    uint64_t st = bp->seed ^ ((uint64_t)t * 0x9E3779B97F4A7C15ull);
    for (uint32_t i = 0; i < nb; i++) {
      uint32_t j = i + (uint32_t)(splitmix64_next(st) % (uint64_t)(n - i));
      std::swap(pos[i], pos[j]);
      cdoc[cptr2[t] + i] = ldoc[lptr[t] + pos[i]];
    }
  });

  timer.mark("centroids");
  // ---- clustering on the device
  std::vector<uint32_t> assign(npost);
  DevBuf d_ip, d_t, d_v;  // the collection on the device: clustering, then the summaries
  {
    std::vector<uint32_t> work;
    for (uint32_t t = 0; t < d; t++)
      if (lptr[t + 1] > lptr[t]) work.push_back(t);
    DevBuf d_work, d_lptr, d_ldoc, d_cptr, d_cdoc, d_best, d_asg;
    if ((rc = upload(d_work, work)) || (rc = upload(d_lptr, lptr)) || (rc = upload(d_ldoc, ldoc)) ||
        (rc = upload(d_cptr, cptr2)) || (rc = upload(d_cdoc, cdoc)) || (rc = upload(d_ip, D.ip)) ||
        (rc = upload(d_t, D.t)) || (rc = upload(d_v, D.v)) || (rc = d_best.alloc(npost * 8)) ||
        (rc = d_asg.alloc(npost * 4)))
      return rc;
    size_t smem = asg_smem_bytes(d);
    SZ_CUDA(cudaFuncSetAttribute(k_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 1;
    SZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device));
    uint32_t grid = (uint32_t)std::min<size_t>(work.size(), (size_t)sms * 8);
    if (grid) {
      k_assign<<<grid, kAsgThreads, smem>>>(d_work.as<uint32_t>(), (uint32_t)work.size(), d_lptr.as<uint32_t>(),
                                            d_ldoc.as<uint32_t>(), d_cptr.as<uint32_t>(), d_cdoc.as<uint32_t>(),
                                            d_ip.as<uint64_t>(), d_t.as<uint16_t>(), d_v.as<float>(), d,
                                            ix->fwd_row.as<unsigned long long>(), ix->fwd_data.as<uint8_t>(), fp16,
                                            d_best.as<double>(), d_asg.as<uint32_t>());
      SZ_CUDA(cudaGetLastError());
      SZ_CUDA(cudaDeviceSynchronize());
    }
    if (npost) SZ_CUDA(cudaMemcpy(assign.data(), d_asg.p, npost * 4, cudaMemcpyDeviceToHost));
  }

  timer.mark("clustering (device)");
  // ---- blocks (non-empty clusters in centroid order; members ascending)
  std::vector<uint32_t> nblk_of(d, 0);
  parallel_for(d, T, [&](int64_t t, int) {
    uint32_t nb = cptr2[t + 1] - cptr2[t];
    if (!nb) return;
    std::vector<uint8_t> used(nb, 0);
    for (uint32_t p = lptr[t]; p < lptr[t + 1]; p++) used[assign[p]] = 1;
    uint32_t c = 0;
    for (uint8_t u : used) c += u;
    nblk_of[t] = c;
  });
  std::vector<uint32_t> bptr(d + 1, 0);
  for (uint32_t t = 0; t < d; t++) bptr[t + 1] = bptr[t] + nblk_of[t];
  const uint32_t nblk = bptr[d];
  ix->n_blocks = nblk;
  std::vector<uint32_t> bdptr(nblk + 1, 0), bdoc(npost);
  parallel_for(d, T, [&](int64_t t, int) {
    uint32_t nb = cptr2[t + 1] - cptr2[t];
    if (!nb) return;
    std::vector<uint32_t> cnt(nb, 0), start(nb, 0);
    for (uint32_t p = lptr[t]; p < lptr[t + 1]; p++) cnt[assign[p]]++;
    uint32_t g = bptr[t], off = lptr[t];  // members of list t occupy [lptr[t], lptr[t+1])
    for (uint32_t c = 0; c < nb; c++) {
      if (!cnt[c]) continue;
      bdptr[g] = off;  // written per block; the last entry is set below
      start[c] = off;
      off += cnt[c];
      g++;
    }
    for (uint32_t p = lptr[t]; p < lptr[t + 1]; p++) bdoc[start[assign[p]]++] = ldoc[p];
    g = bptr[t];
    for (uint32_t c = 0; c < nb; c++) {
      if (!cnt[c]) continue;
      std::sort(bdoc.begin() + bdptr[g], bdoc.begin() + bdptr[g] + cnt[c]);
      g++;
    }
  });
  bdptr[nblk] = (uint32_t)npost;
  uint32_t maxbd = 0, maxnb = 0;
  for (uint32_t g = 0; g < nblk; g++) maxbd = std::max(maxbd, bdptr[g + 1] - bdptr[g]);
  for (uint32_t t = 0; t < d; t++) maxnb = std::max(maxnb, nblk_of[t]);
  ix->max_block_docs = maxbd;
  ix->max_blocks_per_list = maxnb;
  std::vector<uint32_t>().swap(cdoc);

  timer.mark("blocks");
  // ---- summaries (max vector, alpha-MSS, u8) and their term-major layout, on the device
  const int quant = bp->quantize_u8 ? 1 : 0;
  const bool keep_bm = bp->keep_block_summaries != 0;  // the block-major copies are kept only for export
  const uint32_t W = (d + 31) / 32;
  if (ix->max_blocks_per_list > 65535) return fail(SEISMIC_EINVAL, "more than 65535 blocks in a list");
  if ((rc = upload(ix->list_ptr, lptr)) || (rc = upload(ix->list_doc, ldoc)) || (rc = upload(ix->cent, assign)) ||
      (rc = upload(ix->blk_ptr, bptr)) || (rc = upload(ix->bdoc_ptr, bdptr)) || (rc = upload(ix->bdoc, bdoc)))
    return rc;
  {
    int sms = 1, occ = 1;
    SZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device));
    if ((rc = sum_occupancy(W, &occ))) return rc;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(nblk, (uint64_t)sms * occ));
    uint32_t gstride = 1;
    while (gstride < d) gstride <<= 1;
    DevBuf d_keep, d_thr, d_babs, d_gphi, d_gkeys;
    if ((rc = ix->blk_m.alloc((size_t)nblk * 4)) || (rc = ix->blk_size.alloc((size_t)nblk * 4)) ||
        (rc = d_keep.alloc((size_t)nblk * 4)) || (rc = d_thr.alloc((size_t)nblk * 8)) ||
        (rc = d_babs.alloc((size_t)nblk * 8)) || (rc = d_gphi.alloc((size_t)grid * gstride * 4)) ||
        (rc = d_gkeys.alloc((size_t)grid * gstride * 8)))
      return rc;
    SumArgs sa{};
    sa.ip = d_ip.as<uint64_t>();
    sa.t = d_t.as<uint16_t>();
    sa.v = d_v.as<float>();
    sa.bdptr = ix->bdoc_ptr.as<uint32_t>();
    sa.bdoc = ix->bdoc.as<uint32_t>();
    sa.nblk = nblk;
    sa.W = W;
    sa.alpha = bp->alpha;
    sa.quant = quant;
    sa.keep = d_keep.as<uint32_t>();
    sa.thr = d_thr.as<unsigned long long>();
    sa.bm = ix->blk_m.as<float>();
    sa.bsz = ix->blk_size.as<float>();
    sa.babs = d_babs.as<double>();
    sa.gphi = d_gphi.as<uint32_t>();
    sa.gkeys = d_gkeys.as<unsigned long long>();
    sa.gstride = gstride;
    if ((rc = launch_sum_pass(sa, 1, grid, 0))) return rc;
    SZ_CUDA(cudaDeviceSynchronize());
    std::vector<uint32_t> keep(nblk), sptr(nblk + 1, 0);
    std::vector<double> babs(nblk);
    if (nblk) {
      SZ_CUDA(cudaMemcpy(keep.data(), d_keep.p, (size_t)nblk * 4, cudaMemcpyDeviceToHost));
      SZ_CUDA(cudaMemcpy(babs.data(), d_babs.p, (size_t)nblk * 8, cudaMemcpyDeviceToHost));
    }
    uint64_t acc = 0;
    double mx = 0.0;  // bound on |summary value| as the search reconstructs it (m + code * size)
    for (uint64_t g = 0; g < nblk; g++) {
      sptr[g] = (uint32_t)acc;
      acc += keep[g];
      if (acc > 0xFFFFFFFFull) return fail(SEISMIC_EINVAL, "more than 2^32 summary entries");
      mx = std::max(mx, babs[g]);
    }
    sptr[nblk] = (uint32_t)acc;
    ix->n_sum = acc;
    ix->sum_absmax = (float)(mx * 1.001 + 1e-30);
    const uint64_t nsum = acc;
    timer.mark("summaries: max, alpha-MSS, u8 (device)");
    if ((rc = upload(ix->sum_ptr, sptr)) || (rc = ix->sum_term.alloc(nsum * 2)) ||
        ((!quant || keep_bm) && (rc = ix->sum_val.alloc(nsum * 4))) || (quant && (rc = ix->sum_code.alloc(nsum))))
      return rc;
    sa.sptr = ix->sum_ptr.as<uint32_t>();
    sa.sterm = ix->sum_term.as<uint16_t>();
    sa.sval = ix->sum_val.p ? ix->sum_val.as<float>() : nullptr;
    sa.scode = ix->sum_code.as<uint8_t>();
    if ((rc = launch_sum_pass(sa, 2, grid, 0))) return rc;
    // the term-major columns of each list, behind the presence-bitmap directory
    DevBuf d_ncols, d_cbase, d_cur;
    if ((rc = ix->sbm.alloc((size_t)d * W * 8)) || (rc = d_ncols.alloc((size_t)d * 4))) return rc;
    ColArgs ca{};
    ca.dim = d;
    ca.W = W;
    ca.blk_ptr = ix->blk_ptr.as<uint32_t>();
    ca.sptr = ix->sum_ptr.as<uint32_t>();
    ca.sterm = ix->sum_term.as<uint16_t>();
    ca.sval = sa.sval;
    ca.scode = sa.scode;
    ca.quant = quant;
    ca.sbm = ix->sbm.as<uint2>();
    ca.ncols = d_ncols.as<uint32_t>();
    const uint32_t cgrid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(d, (uint64_t)sms * 8));
    if ((rc = launch_cols_pass(ca, 1, cgrid, 0))) return rc;
    std::vector<uint32_t> ncols(d), cbase(d);
    SZ_CUDA(cudaMemcpy(ncols.data(), d_ncols.p, (size_t)d * 4, cudaMemcpyDeviceToHost));
    uint64_t cacc = 0;
    for (uint32_t t = 0; t < d; t++) {
      cbase[t] = (uint32_t)cacc;
      cacc += ncols[t] + 1ull;  // the list's columns and its sentinel
      if (cacc > 0xFFFFFFFFull) return fail(SEISMIC_EINVAL, "more than 2^32 summary columns");
    }
    if ((rc = upload(d_cbase, cbase)) || (rc = ix->scptr.alloc(cacc * 4)) || (rc = d_cur.alloc(cacc * 4)) ||
        (rc = ix->scol_blk.alloc(nsum * 2)) || (quant && (rc = ix->scol_code.alloc(nsum))) ||
        (!quant && (rc = ix->scol_val.alloc(nsum * 4))))
      return rc;
    ca.cbase = d_cbase.as<uint32_t>();
    ca.scptr = ix->scptr.as<uint32_t>();
    ca.cur = d_cur.as<uint32_t>();
    ca.cblk = ix->scol_blk.as<uint16_t>();
    ca.ccode = ix->scol_code.as<uint8_t>();
    ca.cval = ix->scol_val.as<float>();
    if ((rc = launch_cols_pass(ca, 2, cgrid, 0))) return rc;
    SZ_CUDA(cudaDeviceSynchronize());
    if (!keep_bm) {
      ix->sum_ptr.release();
      ix->sum_term.release();
      ix->sum_val.release();
      ix->sum_code.release();
    }
  }
  d_ip.release();
  d_t.release();
  d_v.release();
  timer.mark("summary layout (device)");
  {  // each member's forward row (first unit, chunk count) beside its id: one dependent load fewer
    std::vector<uint64_t> brow(npost);
    parallel_ranges((int64_t)npost, T, 1 << 16, [&](int64_t p0, int64_t p1) {
      for (int64_t p = p0; p < p1; p++) brow[p] = frow[bdoc[p]];
    });
    if ((rc = upload(ix->bdoc_row, brow))) return rc;
  }
  SZ_CUDA(cudaDeviceSynchronize());
  timer.mark("member rows");
  *out = ix.release();
  return SEISMIC_OK;
}

}  // namespace seismic

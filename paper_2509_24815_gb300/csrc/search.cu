// Query processing: Algorithm "Query processing with Seismic" (Section 4.5),
// one CTA per query.
//
//  H0  the query is held in shared memory as a vocabulary bitmap plus a
//      popcount rank per 32-term word and its values in term order: a lookup
//      is one 4-byte shared load when the term is absent (the common case)
//      and two more when present.  About 8 KB per query instead of a 122 KB
//      dense vector, so several queries share an SM.
//  H1  list terms: the top-`cut` query terms by (value desc, term asc), or
//      the alpha_q-MSS of q (Section 3.2 applied to the query).
//  H2  r_b = <q, S_b> for every block of the list with the full query.  The
//      summaries are stored term-major per list (a column per term, blocks
//      ascending), so only the query's columns are read; each warp owns a
//      partial-score array and the partials are added in warp order, which
//      makes r_b deterministic.
//  H3  blocks are ordered by (r desc, block asc) with a bitonic sort.
//  H4  a block is skipped iff the top-k is full and r < hf * theta (or
//      r < theta / hf); r is non-increasing and theta non-decreasing along
//      the order, so the first skipped block ends the list.
//  H5  forward rows: groups of G lanes score one document each; a row is a
//      record of 8-entry chunks (16 B of terms then 32 B of values per chunk),
//      read with 16-byte vector loads.  Each document is scored at most once
//      per query (a bounded shared-memory hash set; on overflow a document may
//      be scored again, which changes no result).
//  H6  top-k by (score desc, id asc): candidates that beat the k-th score are
//      collected per wave and merged by rank.
//  H7  kappa-NN expansion of the top-k after the lists (S fixed first).
//
// Waves: with wave = 1 every block is evaluated before the next skip test,
// which is exactly the sequential order of the algorithm (the final heap
// after a block does not depend on the order of its documents).
#include <algorithm>

#include "search_impl.h"

namespace seismic {

namespace {

__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
  return __uint_as_float(u);
}

__device__ __forceinline__ bool better(float s1, uint32_t i1, float s2, uint32_t i2) {
  return s1 > s2 || (s1 == s2 && i1 < i2);
}

__device__ __forceinline__ float qlookup(const uint32_t *__restrict__ qbits, const uint16_t *__restrict__ qrank,
                                         const float *__restrict__ qval, uint32_t t) {
  const uint32_t w = qbits[t >> 5];
  const uint32_t bit = 1u << (t & 31);
  if (!(w & bit)) return 0.0f;
  return qval[qrank[t >> 5] + __popc(w & (bit - 1u))];
}

// 16-byte read-only loads that do not allocate in L1: rows are touched once
// per query, reuse across queries happens in L2.
__device__ __forceinline__ uint4 ldg_na(const void *p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

template <int G>
__device__ __forceinline__ float doc_dot(const uint8_t *__restrict__ fwd, const uint32_t *__restrict__ cptr,
                                         uint32_t d, int gl, uint32_t gmask, const uint32_t *__restrict__ qbits,
                                         const uint16_t *__restrict__ qrank, const float *__restrict__ qval) {
  const uint32_t c0 = __ldg(cptr + d), nch = __ldg(cptr + d + 1) - c0;
  const uint8_t *rec = fwd + (size_t)c0 * 48;
  const uint8_t *vrec = rec + 16 * (size_t)nch;
  float acc = 0.0f;
  uint32_t c = gl;
#pragma unroll 1
  for (; c + G < nch; c += 2 * G) {  // two chunks in flight per lane
    uint4 t0 = ldg_na(rec + 16 * (size_t)c);
    uint4 a0 = ldg_na(vrec + 32 * (size_t)c);
    uint4 b0 = ldg_na(vrec + 32 * (size_t)c + 16);
    uint4 t1 = ldg_na(rec + 16 * (size_t)(c + G));
    uint4 a1 = ldg_na(vrec + 32 * (size_t)(c + G));
    uint4 b1 = ldg_na(vrec + 32 * (size_t)(c + G) + 16);
    const uint32_t tw0[4] = {t0.x, t0.y, t0.z, t0.w};
    const uint32_t va0[8] = {a0.x, a0.y, a0.z, a0.w, b0.x, b0.y, b0.z, b0.w};
    const uint32_t tw1[4] = {t1.x, t1.y, t1.z, t1.w};
    const uint32_t va1[8] = {a1.x, a1.y, a1.z, a1.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int e = 0; e < 4; e++) {
      acc = fmaf(qlookup(qbits, qrank, qval, tw0[e] & 0xFFFFu), __uint_as_float(va0[2 * e]), acc);
      acc = fmaf(qlookup(qbits, qrank, qval, tw0[e] >> 16), __uint_as_float(va0[2 * e + 1]), acc);
    }
#pragma unroll
    for (int e = 0; e < 4; e++) {
      acc = fmaf(qlookup(qbits, qrank, qval, tw1[e] & 0xFFFFu), __uint_as_float(va1[2 * e]), acc);
      acc = fmaf(qlookup(qbits, qrank, qval, tw1[e] >> 16), __uint_as_float(va1[2 * e + 1]), acc);
    }
  }
  if (c < nch) {
    uint4 t0 = ldg_na(rec + 16 * (size_t)c);
    uint4 a0 = ldg_na(vrec + 32 * (size_t)c);
    uint4 b0 = ldg_na(vrec + 32 * (size_t)c + 16);
    const uint32_t tw0[4] = {t0.x, t0.y, t0.z, t0.w};
    const uint32_t va0[8] = {a0.x, a0.y, a0.z, a0.w, b0.x, b0.y, b0.z, b0.w};
#pragma unroll
    for (int e = 0; e < 4; e++) {
      acc = fmaf(qlookup(qbits, qrank, qval, tw0[e] & 0xFFFFu), __uint_as_float(va0[2 * e]), acc);
      acc = fmaf(qlookup(qbits, qrank, qval, tw0[e] >> 16), __uint_as_float(va0[2 * e + 1]), acc);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gmask, acc, o, G);
  return acc;
}

// Insert d into the per-query seen set; true when d was not there before
// (or the set is too crowded to tell, in which case d is scored again).
__device__ __forceinline__ bool seen_insert(uint32_t *tab, uint32_t hs_mask, uint32_t d, uint32_t *full) {
  const uint32_t key = d + 1u;
  uint32_t h = (d * 0x9E3779B1u) & hs_mask;
#pragma unroll 1
  for (int p = 0; p < 16; p++) {
    uint32_t old = atomicCAS(&tab[h], 0u, key);
    if (old == 0u) return true;
    if (old == key) return false;
    h = (h + 1u) & hs_mask;
  }
  *full = 1u;
  return true;
}

template <int NT>
__device__ uint32_t block_rank_scan(const uint32_t *bits, uint16_t *rank, uint32_t W, uint32_t *wtmp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = NT / 32;
  const uint32_t per = (W + NT - 1) / NT, lo = min(W, tid * per), hi = min(W, lo + per);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; i++) s += __popc(bits[i]);
  uint32_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < nw ? wtmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < nw) wtmp[lane] = v;
  }
  __syncthreads();
  uint32_t base = (warp ? wtmp[warp - 1] : 0) + x - s;
  for (uint32_t i = lo; i < hi; i++) {
    rank[i] = (uint16_t)min(base, 65535u);
    base += __popc(bits[i]);
  }
  const uint32_t total = wtmp[nw - 1];
  __syncthreads();
  return total;
}

struct Smem {
  uint32_t *qbits;
  uint16_t *qrank;
  float *qval;
  uint16_t *qterm;
  uint16_t *cutT;
  float *aq;
  float *part;
  unsigned long long *keys;
  uint32_t *clo, *chi;
  uint32_t *hash;
  uint32_t *seen;  // this CTA's global bitmap, or NULL
  float *tk_s, *tmp_s, *cand_s;
  uint32_t *tk_id, *tmp_id, *cand_id;
  uint8_t *cand_ok;
};

struct Shared {
  uint32_t q, nzq, ncut, count, ncand, nvalid, hash_full, bad;
  float hf;
  uint32_t cut;
  uint32_t wtmp[32];
  unsigned long long st[SEISMIC_STATS_N];
};

template <int NT>
__device__ void merge_candidates(const SearchArgs &a, Smem &s, Shared &sh) {
  const int tid = threadIdx.x;
  const uint32_t m = sh.ncand, cnt = sh.count, k = a.k;
  if (m == 0) return;  // uniform: every thread read the same ncand after the barrier
  const bool dupcheck = sh.hash_full != 0u;
  for (uint32_t i = tid; i < m; i += NT) {
    const uint32_t id = s.cand_id[i];
    uint8_t ok = 1;
    for (uint32_t j = 0; j < cnt; j++)
      if (s.tk_id[j] == id) { ok = 0; break; }
    if (ok && dupcheck)
      for (uint32_t j = 0; j < i; j++)
        if (s.cand_id[j] == id) { ok = 0; break; }
    s.cand_ok[i] = ok;
    if (ok) atomicAdd(&sh.nvalid, 1u);
  }
  __syncthreads();
  for (uint32_t i = tid; i < m; i += NT) {
    if (!s.cand_ok[i]) continue;
    const float sc = s.cand_s[i];
    const uint32_t id = s.cand_id[i];
    uint32_t lo = 0, hi = cnt;  // topk entries better than (sc, id)
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (better(s.tk_s[mid], s.tk_id[mid], sc, id)) lo = mid + 1; else hi = mid;
    }
    uint32_t r = lo;
    for (uint32_t j = 0; j < m; j++)
      if (s.cand_ok[j] && better(s.cand_s[j], s.cand_id[j], sc, id)) r++;
    if (r < k) { s.tmp_s[r] = sc; s.tmp_id[r] = id; }
  }
  for (uint32_t i = tid; i < cnt; i += NT) {
    const float sc = s.tk_s[i];
    const uint32_t id = s.tk_id[i];
    uint32_t r = i;
    for (uint32_t j = 0; j < m; j++)
      if (s.cand_ok[j] && better(s.cand_s[j], s.cand_id[j], sc, id)) r++;
    if (r < k) { s.tmp_s[r] = sc; s.tmp_id[r] = id; }
  }
  __syncthreads();
  const uint32_t nc = min(k, cnt + sh.nvalid);
  for (uint32_t i = tid; i < nc; i += NT) { s.tk_s[i] = s.tmp_s[i]; s.tk_id[i] = s.tmp_id[i]; }
  __syncthreads();
  if (tid == 0) { sh.count = nc; sh.ncand = 0; sh.nvalid = 0; }
  __syncthreads();
}

// Scores up to CAND documents drawn from a source functor, then merges.
template <int G, int NT, class Src>
__device__ void eval_wave(const SearchArgs &a, Smem &s, Shared &sh, uint32_t n, Src src, int knn_stage) {
  constexpr int NG = NT / G;
  const int tid = threadIdx.x, grp = tid / G, gl = tid % G;
  const uint32_t lane = tid & 31;
  const uint32_t gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(uint32_t)(G - 1)));
  const bool full = sh.count == a.k;
  const float th = full ? s.tk_s[a.k - 1] : -INFINITY;
  const uint32_t thid = full ? s.tk_id[a.k - 1] : 0u;
  for (uint32_t i = grp; i < n; i += NG) {
    const uint32_t d = src(i);
    if (d == SEISMIC_NONE_ID) continue;
    uint32_t fresh = 0;
    if (gl == 0) {
      if (s.seen) {
        const uint32_t bit = 1u << (d & 31);
        fresh = (atomicOr(s.seen + (d >> 5), bit) & bit) ? 0u : 1u;
      } else {
        fresh = seen_insert(s.hash, a.HS - 1u, d, &sh.hash_full) ? 1u : 0u;
      }
    }
    fresh = __shfl_sync(gmask, fresh, 0, G);
    if (!fresh) continue;
    const float p = doc_dot<G>(a.fwd_data, a.fwd_cptr, d, gl, gmask, s.qbits, s.qrank, s.qval);
    if (gl == 0) {
      if (a.stats) {
        atomicAdd(&sh.st[knn_stage ? SEISMIC_ST_KNN_DOCS : SEISMIC_ST_DOCS], 1ull);
        atomicAdd(&sh.st[knn_stage ? SEISMIC_ST_KNN_NNZ : SEISMIC_ST_DOC_NNZ], (unsigned long long)a.fwd_nnz[d]);
      }
      if (!full || better(p, d, th, thid)) {
        uint32_t pos = atomicAdd(&sh.ncand, 1u);
        s.cand_s[pos] = p;
        s.cand_id[pos] = d;
      }
    }
  }
  __syncthreads();
  merge_candidates<NT>(a, s, sh);
}

template <int NT>
__device__ void bitonic_sort_u64(unsigned long long *keys, uint32_t P2) {
  const int tid = threadIdx.x;
  for (uint32_t k2 = 2; k2 <= P2; k2 <<= 1)
    for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < P2; i += NT) {
        uint32_t ixj = i ^ j;
        if (ixj > i) {
          unsigned long long x = keys[i], y = keys[ixj];
          bool up = (i & k2) == 0;
          if ((x > y) == up) { keys[i] = y; keys[ixj] = x; }
        }
      }
      __syncthreads();
    }
}

template <int G, int NW>
__global__ void __launch_bounds__(NW * 32) k_search(const SearchArgs a) {
  constexpr int NT = NW * 32;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ Shared sh;
  Smem s;
  s.qbits = reinterpret_cast<uint32_t *>(sm + a.off_qbits);
  s.qrank = reinterpret_cast<uint16_t *>(sm + a.off_qrank);
  s.qval = reinterpret_cast<float *>(sm + a.off_qval);
  s.qterm = reinterpret_cast<uint16_t *>(sm + a.off_qterm);
  s.cutT = reinterpret_cast<uint16_t *>(sm + a.off_cut);
  s.aq = reinterpret_cast<float *>(sm + a.off_aq);
  s.part = reinterpret_cast<float *>(sm + a.off_part);
  s.keys = reinterpret_cast<unsigned long long *>(sm + a.off_keys);
  s.clo = reinterpret_cast<uint32_t *>(sm + a.off_clo);
  s.chi = reinterpret_cast<uint32_t *>(sm + a.off_chi);
  s.hash = reinterpret_cast<uint32_t *>(sm + a.off_hash);
  s.tk_s = reinterpret_cast<float *>(sm + a.off_tk_s);
  s.tk_id = reinterpret_cast<uint32_t *>(sm + a.off_tk_id);
  s.tmp_s = reinterpret_cast<float *>(sm + a.off_tmp_s);
  s.tmp_id = reinterpret_cast<uint32_t *>(sm + a.off_tmp_id);
  s.cand_s = reinterpret_cast<float *>(sm + a.off_cand_s);
  s.cand_id = reinterpret_cast<uint32_t *>(sm + a.off_cand_id);
  s.cand_ok = reinterpret_cast<uint8_t *>(sm + a.off_cand_ok);
  s.seen = a.seen_bm ? a.seen_bm + (size_t)blockIdx.x * a.seen_words : nullptr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  bool first = true;

  for (;;) {
    if (tid == 0) {
      if (a.persistent) sh.q = atomicAdd(a.queue, 1u);
      else sh.q = first ? blockIdx.x : a.nq;
    }
    first = false;
    __syncthreads();
    const uint32_t q = sh.q;
    if (q >= a.nq) break;

    // ---------------------------------------------------------- H0: ingest
    const uint64_t qb = a.q_indptr[q], qe = a.q_indptr[q + 1];
    const uint32_t nnz = (uint32_t)(qe - qb);
    for (uint32_t i = tid; i < a.W; i += NT) s.qbits[i] = 0u;
    if (s.seen) {  // seen_words is a multiple of 4 and the slot is 16-byte aligned
      uint4 *z = reinterpret_cast<uint4 *>(s.seen);
      for (uint32_t i = tid; i < a.seen_words / 4; i += NT) z[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      for (uint32_t i = tid; i < a.HS; i += NT) s.hash[i] = 0u;
    }
    if (tid < SEISMIC_STATS_N) sh.st[tid] = 0ull;
    if (tid == 0) {
      sh.count = 0; sh.ncand = 0; sh.nvalid = 0; sh.hash_full = 0; sh.bad = 0;
      sh.cut = a.cut;
      sh.hf = a.hf;
      if (a.q_cut) {  // learned per-query parameters (already validated by their producer)
        sh.cut = a.q_cut[q];
        sh.hf = a.q_hf[q];
      }
    }
    __syncthreads();
    for (uint32_t i = tid; i < nnz; i += NT) {
      const float v = a.q_vals[qb + i];
      if (v != 0.0f) {
        const uint32_t t = a.q_terms[qb + i];
        if (t < a.dim) atomicOr(&s.qbits[t >> 5], 1u << (t & 31));
        else sh.bad = 1u;
      }
    }
    __syncthreads();
    const uint32_t nzq = block_rank_scan<NT>(s.qbits, s.qrank, a.W, sh.wtmp);
    if (nzq > a.QN || sh.bad) {  // more nonzeros than the launch was sized for, or a bad term
      if (tid == 0) atomicOr(a.queue + 1, 1u);
      for (uint32_t i = tid; i < a.k; i += NT) {
        a.ids[(size_t)q * a.k + i] = SEISMIC_NONE_ID;
        a.scores[(size_t)q * a.k + i] = -INFINITY;
      }
      __syncthreads();
      if (!a.persistent) break;
      continue;
    }
    for (uint32_t i = tid; i < nnz; i += NT) {
      const float v = a.q_vals[qb + i];
      if (v != 0.0f) {
        const uint32_t t = a.q_terms[qb + i];
        const uint32_t w = s.qbits[t >> 5];
        const uint32_t pos = s.qrank[t >> 5] + __popc(w & ((1u << (t & 31)) - 1u));
        s.qval[pos] = v;
        s.qterm[pos] = (uint16_t)t;
      }
    }
    __syncthreads();

    // ---------------------------------------------------------- H1: list terms
    if (a.alpha_q > 0.0f) {
      for (uint32_t i = tid; i < nzq; i += NT) {
        const float av = fabsf(s.qval[i]);
        const uint32_t t = s.qterm[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < nzq; j++) {
          const float aj = fabsf(s.qval[j]);
          r += (aj > av || (aj == av && s.qterm[j] < t)) ? 1u : 0u;
        }
        s.aq[r] = av;
        s.cutT[r] = (uint16_t)t;
      }
      __syncthreads();
      if (tid == 0) {  // alpha_q-MSS: fp64 prefix mass in sketch order
        double tot = 0.0;
        for (uint32_t i = 0; i < nzq; i++) tot += (double)s.aq[i];
        const double target = (double)a.alpha_q * tot;
        double c = 0.0;
        uint32_t keep = nzq;
        for (uint32_t i = 0; i < nzq; i++) {
          c += (double)s.aq[i];
          if (c >= target) { keep = i + 1; break; }
        }
        sh.ncut = keep;
      }
    } else {
      const uint32_t cut = sh.cut;
      for (uint32_t i = tid; i < nzq; i += NT) {
        const float v = s.qval[i];
        const uint32_t t = s.qterm[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < nzq; j++) {
          const float vj = s.qval[j];
          r += (vj > v || (vj == v && s.qterm[j] < t)) ? 1u : 0u;
        }
        if (r < cut) s.cutT[r] = (uint16_t)t;
      }
      if (tid == 0) sh.ncut = min(cut, nzq);
    }
    __syncthreads();
    const uint32_t ncut = sh.ncut;
    const float hf = sh.hf;
    if (a.stats && tid == 0) sh.st[SEISMIC_ST_QUERY_NNZ] = nnz;

    // ---------------------------------------------------------- lists
    for (uint32_t li = 0; li < ncut; li++) {
      const uint32_t t = s.cutT[li];
      const uint32_t g0 = a.blk_ptr[t], nb = a.blk_ptr[t + 1] - g0;
      if (a.stats && tid == 0) sh.st[SEISMIC_ST_LISTS]++;
      if (nb == 0) continue;
      if (a.exhaustive) {
        const uint32_t d0 = a.bdoc_ptr[g0], d1 = a.bdoc_ptr[g0 + nb];
        if (a.stats && tid == 0) {
          sh.st[SEISMIC_ST_BLOCKS_EVALUATED] += nb;
          sh.st[SEISMIC_ST_BLOCK_DOCS] += d1 - d0;
        }
        for (uint32_t c0 = d0; c0 < d1; c0 += a.CAND) {
          const uint32_t n = min(a.CAND, d1 - c0);
          const uint32_t *src = a.bdoc + c0;
          eval_wave<G, NT>(a, s, sh, n, [src](uint32_t i) { return __ldg(src + i); }, 0);
        }
        continue;
      }
      // ---- H2: summary scores of every block of the list
      const size_t dbase = (size_t)t * (a.dim + 1u);
      for (uint32_t i = tid; i < nzq; i += NT) {
        const uint32_t sterm = s.qterm[i];
        s.clo[i] = __ldg(a.sdir + dbase + sterm);
        s.chi[i] = __ldg(a.sdir + dbase + sterm + 1);
      }
      for (uint32_t i = tid; i < NW * a.BMAX; i += NT) s.part[i] = 0.0f;
      __syncthreads();
      {
        float *pw = s.part + warp * a.BMAX;
        const float *bm = a.blk_m + g0;
        const float *bs = a.blk_size + g0;
        uint32_t ent = 0;
        for (uint32_t i = warp; i < nzq; i += NW) {
          const uint32_t lo = s.clo[i], hi = s.chi[i];
          const float qv = s.qval[i];
          ent += hi - lo;
          for (uint32_t e = lo + lane; e < hi; e += 32) {
            const uint32_t b = __ldg(a.scol_blk + e);
            float sv;
            if (a.quant) sv = fmaf((float)__ldg(a.scol_code + e), __ldg(bs + b), __ldg(bm + b));
            else sv = __ldg(a.scol_val + e);
            pw[b] = fmaf(qv, sv, pw[b]);
          }
          __syncwarp();
        }
        if (a.stats && lane == 0) atomicAdd(&sh.st[SEISMIC_ST_SUMMARY_ENTRIES], (unsigned long long)ent);
      }
      __syncthreads();
      uint32_t P2 = 1;
      while (P2 < nb) P2 <<= 1;
      for (uint32_t b = tid; b < P2; b += NT) {
        if (b < nb) {
          float r = 0.0f;
          for (int w = 0; w < NW; w++) r += s.part[w * a.BMAX + b];
          s.keys[b] = ((unsigned long long)(~f2ord(r)) << 32) | b;
        } else {
          s.keys[b] = ~0ull;
        }
      }
      if (a.stats && tid == 0) {
        sh.st[SEISMIC_ST_BLOCKS_SCORED] += nb;
        sh.st[SEISMIC_ST_DIR_LOOKUPS] += 2ull * nzq;
      }
      __syncthreads();
      // ---- H3: order blocks by (r desc, block asc)
      bitonic_sort_u64<NT>(s.keys, P2);
      // ---- H4/H5/H6: visit blocks in order, waves of a.wave blocks
      uint32_t bi = 0;
      while (bi < nb) {
        // skip test at the head of the wave (uniform: shared state after a barrier)
        if (sh.count == a.k) {
          const float theta = s.tk_s[a.k - 1];
          const float thr = a.hf_mode == 0 ? hf * theta : theta / hf;
          const float r = ord2f(~(uint32_t)(s.keys[bi] >> 32));
          if (r < thr) {
            if (a.stats && tid == 0) sh.st[SEISMIC_ST_BLOCKS_SKIPPED] += nb - bi;
            break;
          }
        }
        if (a.wave <= 1) {
          const uint32_t b = (uint32_t)(s.keys[bi] & 0xFFFFFFFFu);
          const uint32_t d0 = a.bdoc_ptr[g0 + b], d1 = a.bdoc_ptr[g0 + b + 1];
          if (a.stats && tid == 0) {
            sh.st[SEISMIC_ST_BLOCKS_EVALUATED]++;
            sh.st[SEISMIC_ST_BLOCK_DOCS] += d1 - d0;
          }
          for (uint32_t c0 = d0; c0 < d1; c0 += a.CAND) {
            const uint32_t n = min(a.CAND, d1 - c0);
            const uint32_t *src = a.bdoc + c0;
            eval_wave<G, NT>(a, s, sh, n, [src](uint32_t i) { return __ldg(src + i); }, 0);
          }
          bi++;
        } else {
          // a wave: the next blocks whose score passes the test against the
          // threshold at the wave's start, up to a.wave blocks / CAND documents
          uint32_t be = bi, ndocs = 0;
          const bool fullk = sh.count == a.k;
          const float theta = fullk ? s.tk_s[a.k - 1] : -INFINITY;
          const float thr = a.hf_mode == 0 ? hf * theta : theta / hf;
          while (be < nb && be - bi < a.wave) {
            const uint32_t b = (uint32_t)(s.keys[be] & 0xFFFFFFFFu);
            const float r = ord2f(~(uint32_t)(s.keys[be] >> 32));
            if (fullk && r < thr) break;
            const uint32_t nd = a.bdoc_ptr[g0 + b + 1] - a.bdoc_ptr[g0 + b];
            if (be > bi && ndocs + nd > a.CAND) break;
            ndocs += nd;
            be++;
          }
          if (ndocs > a.CAND) {  // one oversized block: evaluate it alone, in pieces
            const uint32_t b = (uint32_t)(s.keys[bi] & 0xFFFFFFFFu);
            const uint32_t d0 = a.bdoc_ptr[g0 + b], d1 = a.bdoc_ptr[g0 + b + 1];
            for (uint32_t c0 = d0; c0 < d1; c0 += a.CAND) {
              const uint32_t n = min(a.CAND, d1 - c0);
              const uint32_t *src = a.bdoc + c0;
              eval_wave<G, NT>(a, s, sh, n, [src](uint32_t i) { return __ldg(src + i); }, 0);
            }
          } else {
            // per-document source over the wave's blocks (walk the block list)
            const unsigned long long *keys = s.keys;
            const uint32_t *bdp = a.bdoc_ptr + g0;
            const uint32_t *bd = a.bdoc;
            const uint32_t b0 = bi, nbw = be - bi;
            eval_wave<G, NT>(a, s, sh, ndocs,
                             [keys, bdp, bd, b0, nbw](uint32_t i) {
                               for (uint32_t w = 0; w < nbw; w++) {
                                 const uint32_t b = (uint32_t)(keys[b0 + w] & 0xFFFFFFFFu);
                                 const uint32_t lo = __ldg(bdp + b), n = __ldg(bdp + b + 1) - lo;
                                 if (i < n) return __ldg(bd + lo + i);
                                 i -= n;
                               }
                               return SEISMIC_NONE_ID;
                             },
                             0);
          }
          if (a.stats && tid == 0) {
            sh.st[SEISMIC_ST_BLOCKS_EVALUATED] += be - bi;
            sh.st[SEISMIC_ST_BLOCK_DOCS] += ndocs;
          }
          bi = be;
        }
      }
      __syncthreads();
    }

    // ---------------------------------------------------------- H7: kappa-NN expansion
    if (a.use_knn && a.kappa > 0 && sh.count > 0) {
      const uint32_t ns = sh.count;
      for (uint32_t i = tid; i < ns; i += NT) s.tmp_id[i] = s.tk_id[i];  // S, fixed before expanding
      __syncthreads();
      // tmp_id is rewritten by merges: keep S in the candidate-id area's tail? use clo (>= k entries)
      for (uint32_t i = tid; i < ns; i += NT) s.clo[i] = s.tmp_id[i];
      __syncthreads();
      const uint32_t total = ns * a.kappa;
      const uint32_t *S = s.clo;
      const uint32_t *knn = a.knn;
      const uint32_t kappa = a.kappa;
      for (uint32_t c0 = 0; c0 < total; c0 += a.CAND) {
        const uint32_t n = min(a.CAND, total - c0);
        eval_wave<G, NT>(a, s, sh, n,
                         [S, knn, kappa, c0](uint32_t i) {
                           const uint32_t x = c0 + i;
                           return __ldg(knn + (size_t)S[x / kappa] * kappa + (x % kappa));
                         },
                         1);
      }
    }

    // ---------------------------------------------------------- output
    for (uint32_t i = tid; i < a.k; i += NT) {
      const bool ok = i < sh.count;
      a.ids[(size_t)q * a.k + i] = ok ? s.tk_id[i] : SEISMIC_NONE_ID;
      a.scores[(size_t)q * a.k + i] = ok ? s.tk_s[i] : -INFINITY;
    }
    if (a.stats && tid < SEISMIC_STATS_N) a.stats[(size_t)q * SEISMIC_STATS_N + tid] = sh.st[tid];
    __syncthreads();
    if (!a.persistent) break;
  }
}

template <int G, int NW>
int launch_t(const SearchArgs &a, size_t smem, uint32_t grid, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    SZ_CUDA(cudaFuncSetAttribute(k_search<G, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    configured = true;
  }
  k_search<G, NW><<<grid, NW * 32, smem, st>>>(a);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

template <int G, int NW>
int occupancy_t(size_t smem, int *blocks) {
  SZ_CUDA(cudaFuncSetAttribute(k_search<G, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  SZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_search<G, NW>, NW * 32, smem));
  return SEISMIC_OK;
}

}  // namespace

static inline uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }

size_t search_layout(SearchArgs &a, uint32_t nw) {
  uint32_t o = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t r = o;
    o = al16(o + bytes);
    return r;
  };
  a.off_qbits = take(a.W * 4);
  a.off_qrank = take(a.W * 2);
  a.off_qval = take(a.QN * 4);
  a.off_qterm = take(a.QN * 2);
  a.off_cut = take(a.QN * 2);
  a.off_aq = take(a.alpha_q > 0.0f ? a.QN * 4 : 4);
  a.off_part = take(a.exhaustive ? 4 : nw * a.BMAX * 4);
  a.off_keys = take(a.exhaustive ? 8 : a.BPOW2 * 8);
  const uint32_t nclo = std::max(a.QN, a.k);  // clo also holds S during the expansion
  a.off_clo = take(nclo * 4);
  a.off_chi = take(a.QN * 4);
  a.off_hash = take(a.HS * 4);
  a.off_tk_s = take(a.k * 4);
  a.off_tk_id = take(a.k * 4);
  a.off_tmp_s = take(a.k * 4);
  a.off_tmp_id = take(a.k * 4);
  a.off_cand_s = take(a.CAND * 4);
  a.off_cand_id = take(a.CAND * 4);
  a.off_cand_ok = take(a.CAND);
  return o;
}

int launch_search(const SearchArgs &a, uint32_t group, uint32_t nw, size_t smem, uint32_t grid, cudaStream_t st) {
#define SZ_CASE(G_, NW_) \
  if (group == G_ && nw == NW_) return launch_t<G_, NW_>(a, smem, grid, st);
  SZ_CASE(8, 4) SZ_CASE(8, 8) SZ_CASE(8, 16)
  SZ_CASE(16, 4) SZ_CASE(16, 8) SZ_CASE(16, 16)
  SZ_CASE(32, 4) SZ_CASE(32, 8) SZ_CASE(32, 16)
#undef SZ_CASE
  return fail(SEISMIC_EINVAL, "group must be 8/16/32 and cta_warps 4/8/16");
}

int search_occupancy(uint32_t group, uint32_t nw, size_t smem, int *blocks) {
#define SZ_CASE(G_, NW_) \
  if (group == G_ && nw == NW_) return occupancy_t<G_, NW_>(smem, blocks);
  SZ_CASE(8, 4) SZ_CASE(8, 8) SZ_CASE(8, 16)
  SZ_CASE(16, 4) SZ_CASE(16, 8) SZ_CASE(16, 16)
  SZ_CASE(32, 4) SZ_CASE(32, 8) SZ_CASE(32, 16)
#undef SZ_CASE
  return fail(SEISMIC_EINVAL, "group must be 8/16/32 and cta_warps 4/8/16");
}

}  // namespace seismic

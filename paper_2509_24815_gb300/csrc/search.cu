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
//      record of 8-entry chunks read with 16-byte vector loads.  At the start
//      of a wave every row of the wave is prefetched into L2 with one TMA bulk
//      prefetch per document, and the member lists of the next wave's blocks
//      too, so the groups' sequential row reads hit L2.  Each document is
//      scored at most once per query (a global bitmap per persistent CTA, or
//      a bounded shared-memory hash set).
//  H6  top-k by (score desc, id asc): candidates that beat the k-th score are
//      collected per wave and merged by rank.
//  H7  kappa-NN expansion of the top-k after the lists (S fixed first).
//
// Waves: with wave = 1 every block is evaluated before the next skip test,
// which is exactly the sequential order of the algorithm (the final heap
// after a block does not depend on the order of its documents).  With wave =
// W the next W blocks that pass the test against the threshold at the wave's
// start are evaluated together (batch-synchronous).
#include <algorithm>

#include "search_common.cuh"

namespace seismic {

namespace {

using namespace dev;

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

// The query's shared-memory arrays.  Each is addressed from the dynamic
// shared-memory base and its offset in the launch arguments (constant bank)
// when used, so no pointer to them stays live in a register.
extern __shared__ __align__(16) unsigned char g_sm[];

struct Smem {
  const SearchArgs &a;
  uint32_t *seen;  // this CTA's global bitmap, or NULL
  __device__ __forceinline__ uint32_t *qbits() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_qbits); }
  __device__ __forceinline__ uint16_t *qrank() const { return reinterpret_cast<uint16_t *>(g_sm + a.off_qrank); }
  __device__ __forceinline__ float *qval() const { return reinterpret_cast<float *>(g_sm + a.off_qval); }
  __device__ __forceinline__ uint16_t *qterm() const { return reinterpret_cast<uint16_t *>(g_sm + a.off_qterm); }
  __device__ __forceinline__ uint16_t *cutT() const { return reinterpret_cast<uint16_t *>(g_sm + a.off_cut); }
  __device__ __forceinline__ float *aq() const { return reinterpret_cast<float *>(g_sm + a.off_aq); }
  __device__ __forceinline__ float *part() const { return reinterpret_cast<float *>(g_sm + a.off_part); }
  __device__ __forceinline__ unsigned long long *keys() const { return reinterpret_cast<unsigned long long *>(g_sm + a.off_keys); }
  __device__ __forceinline__ uint32_t *clo() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_clo); }
  __device__ __forceinline__ uint32_t *chi() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_chi); }
  __device__ __forceinline__ uint32_t *hash() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_hash); }
  __device__ __forceinline__ float *tk_s() const { return reinterpret_cast<float *>(g_sm + a.off_tk_s); }
  __device__ __forceinline__ float *tmp_s() const { return reinterpret_cast<float *>(g_sm + a.off_tmp_s); }
  __device__ __forceinline__ float *cand_s() const { return reinterpret_cast<float *>(g_sm + a.off_cand_s); }
  __device__ __forceinline__ uint32_t *tk_id() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_tk_id); }
  __device__ __forceinline__ uint32_t *tmp_id() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_tmp_id); }
  __device__ __forceinline__ uint32_t *cand_id() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_cand_id); }
  __device__ __forceinline__ uint8_t *cand_ok() const { return reinterpret_cast<uint8_t *>(g_sm + a.off_cand_ok); }
  __device__ __forceinline__ uint32_t *bptr() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_bptr); }
  __device__ __forceinline__ uint32_t *fdoc() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_fdoc); }
  __device__ __forceinline__ uint32_t *fc0() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_fc0); }
  __device__ __forceinline__ uint32_t *fpre() const { return reinterpret_cast<uint32_t *>(g_sm + a.off_fpre); }
  __device__ __forceinline__ uint8_t *cmap() const { return reinterpret_cast<uint8_t *>(g_sm + a.off_cmap); }
};

struct Shared {
  uint32_t q, nzq, ncut, count, ncand, nvalid, hash_full, bad;
  float hf;
  uint32_t cut;
  uint32_t wtmp[32];
  unsigned long long st[SEISMIC_STATS_N];
};

// The members of the wave's blocks keys[0 .. nw) (sorted positions) of the
// current list, as one run: member i is found by walking the blocks' sizes in
// shared memory, so forming a wave needs no barrier.
struct WaveBlocks {
  const unsigned long long *keys;
  const uint32_t *bptr;
  uint32_t nw;
  const uint32_t *ids;
  const unsigned long long *rows;
  __device__ __forceinline__ uint32_t at(uint32_t i) const {
    uint32_t b = (uint32_t)(keys[0] & 0xFFFFFFFFu), lo = bptr[b], nd = bptr[b + 1] - lo;
    for (uint32_t w = 1; w < nw && i >= nd; w++) {
      i -= nd;
      b = (uint32_t)(keys[w] & 0xFFFFFFFFu);
      lo = bptr[b];
      nd = bptr[b + 1] - lo;
    }
    return lo + i;
  }
  __device__ __forceinline__ uint32_t id(uint32_t i) const { return __ldg(ids + at(i)); }
  __device__ __forceinline__ unsigned long long row(uint32_t i, uint32_t) const { return __ldg(rows + at(i)); }
  __device__ __forceinline__ void fetch(uint32_t i, uint32_t &d, unsigned long long &r) const {
    const uint32_t m = at(i);
    d = __ldg(ids + m);
    r = __ldg(rows + m);
  }
};

template <int NT>
__device__ void merge_candidates(const SearchArgs &a, Smem &s, Shared &sh) {
  const int tid = threadIdx.x;
  const uint32_t m = sh.ncand, cnt = sh.count, k = a.k;
  if (m == 0) return;  // uniform: every thread read the same ncand after the barrier
  // With the global seen bitmap a document becomes fresh once per query, so no
  // candidate repeats a heap entry or another candidate.  The bounded hash set
  // may score a document again when it is crowded: there repeats are dropped.
  const bool check = s.seen == nullptr;
  uint32_t nvalid = m;
  if (check) {
    const bool dupcheck = sh.hash_full != 0u;
    for (uint32_t i = tid; i < m; i += NT) {
      const uint32_t id = s.cand_id()[i];
      uint8_t ok = 1;
      for (uint32_t j = 0; j < cnt; j++)
        if (s.tk_id()[j] == id) { ok = 0; break; }
      if (ok && dupcheck)
        for (uint32_t j = 0; j < i; j++)
          if (s.cand_id()[j] == id) { ok = 0; break; }
      s.cand_ok()[i] = ok;
      if (ok) atomicAdd(&sh.nvalid, 1u);
    }
    __syncthreads();
    nvalid = sh.nvalid;
  }
  for (uint32_t i = tid; i < m; i += NT) {
    if (check && !s.cand_ok()[i]) continue;
    const float sc = s.cand_s()[i];
    const uint32_t id = s.cand_id()[i];
    uint32_t lo = 0, hi = cnt;  // topk entries better than (sc, id)
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (better(s.tk_s()[mid], s.tk_id()[mid], sc, id)) lo = mid + 1; else hi = mid;
    }
    uint32_t r = lo;
    for (uint32_t j = 0; j < m; j++)
      if ((!check || s.cand_ok()[j]) && better(s.cand_s()[j], s.cand_id()[j], sc, id)) r++;
    if (r < k) { s.tmp_s()[r] = sc; s.tmp_id()[r] = id; }
  }
  for (uint32_t i = tid; i < cnt; i += NT) {
    const float sc = s.tk_s()[i];
    const uint32_t id = s.tk_id()[i];
    uint32_t r = i;
    for (uint32_t j = 0; j < m; j++)
      if ((!check || s.cand_ok()[j]) && better(s.cand_s()[j], s.cand_id()[j], sc, id)) r++;
    if (r < k) { s.tmp_s()[r] = sc; s.tmp_id()[r] = id; }
  }
  __syncthreads();
  // nc comes from registers, so thread 0 may reset the counters in this phase
  const uint32_t nc = min(k, cnt + nvalid);
  for (uint32_t i = tid; i < nc; i += NT) { s.tk_s()[i] = s.tmp_s()[i]; s.tk_id()[i] = s.tmp_id()[i]; }
  if (tid == 0) { sh.count = nc; sh.ncand = 0; sh.nvalid = 0; }
  __syncthreads();
}

// Scores up to CAND documents of a source, then merges the candidates.
template <int G, int NT, class Src>
__device__ void eval_wave(const SearchArgs &a, Smem &s, Shared &sh, uint32_t n, const Src &src, int knn_stage) {
  constexpr int NG = NT / G;
  const int tid = threadIdx.x, grp = tid / G, gl = tid % G;
  const uint32_t lane = tid & 31;
  const uint32_t gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(uint32_t)(G - 1)));
  const bool full = sh.count == a.k;
  const float th = full ? s.tk_s()[a.k - 1] : -INFINITY;
  const uint32_t thid = full ? s.tk_id()[a.k - 1] : 0u;
  if (a.prefetch && n > (uint32_t)NG) {  // every row of the wave into L2, one bulk prefetch each
    for (uint32_t i = tid; i < n; i += NT) {
      uint32_t d;
      unsigned long long row;
      src.fetch(i, d, row);
      if (d != SEISMIC_NONE_ID) prefetch_row(a.fwd_data, row, a.fp16);
    }
  }
  // Software pipeline per lane group: the next document's (id, row) are loaded
  // while the current one is scored, and the seen-bitmap test is issued with
  // the row's loads and read after the dot (a seen document's score is dropped).
  uint32_t dn = SEISMIC_NONE_ID;
  unsigned long long rn = 0ull;
  if ((uint32_t)grp < n) src.fetch(grp, dn, rn);
  for (uint32_t i = grp; i < n; i += NG) {
    const uint32_t d = dn;
    const unsigned long long row = rn;
    if (i + NG < n) src.fetch(i + NG, dn, rn);
    if (d == SEISMIC_NONE_ID) continue;
    uint32_t old = 0u, fresh = 0u;
    const uint32_t bit = 1u << (d & 31);
    if (gl == 0) {
      if (s.seen) old = atomicOr(s.seen + (d >> 5), bit);
      else fresh = seen_insert(s.hash(), a.HS - 1u, d, &sh.hash_full) ? 1u : 0u;
    }
    const float p = row_dot<G>(a.fwd_data, row, a.fp16, gl, gmask, s.qbits(), s.qrank(), s.qval());
    if (s.seen) fresh = (old & bit) ? 0u : 1u;
    fresh = __shfl_sync(gmask, fresh, 0, G);
    if (!fresh) continue;
    if (gl == 0) {
      if (a.stats) {
        atomicAdd(&sh.st[knn_stage ? SEISMIC_ST_KNN_DOCS : SEISMIC_ST_DOCS], 1ull);
        atomicAdd(&sh.st[knn_stage ? SEISMIC_ST_KNN_NNZ : SEISMIC_ST_DOC_NNZ], (unsigned long long)a.fwd_nnz[d]);
      }
      if (!full || better(p, d, th, thid)) {
        uint32_t pos = atomicAdd(&sh.ncand, 1u);
        s.cand_s()[pos] = p;
        s.cand_id()[pos] = d;
      }
    }
  }
  __syncthreads();
  merge_candidates<NT>(a, s, sh);
}

// v[0..n) -> exclusive prefix sums, v[n] = the total.  Thread t takes a
// contiguous range of ceil(n / NT) elements; warps scan their threads' sums
// with shuffles and every thread adds the totals of the warps before it, so
// the scan costs two barriers.  Every thread must call it (after a barrier
// that published v).  When map is given and the total is at most cap, also
// writes map[v[i] .. v[i+1]) = i (the owner of each unit, i < 256).
template <int NT>
__device__ uint32_t block_exclusive_scan(uint32_t *v, uint32_t n, uint32_t *wtmp, uint8_t *map = nullptr,
                                         uint32_t cap = 0) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = NT / 32;
  const uint32_t per = (n + NT - 1) / NT, lo = min(n, tid * per), hi = min(n, lo + per);
  uint32_t sum = 0;
  for (uint32_t i = lo; i < hi; i++) sum += v[i];
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtmp[warp] = x;
  __syncthreads();
  uint32_t before = 0, total = 0;
#pragma unroll
  for (int w = 0; w < nw; w++) {
    const uint32_t t = wtmp[w];
    before += w < warp ? t : 0u;
    total += t;
  }
  uint32_t run = before + x - sum;
  const bool fill = map != nullptr && total <= cap;
  for (uint32_t i = lo; i < hi; i++) {
    const uint32_t c = v[i];
    v[i] = run;
    if (fill)
      for (uint32_t u = 0; u < c; u++) map[run + u] = (uint8_t)i;
    run += c;
  }
  if (tid == 0) v[n] = total;
  __syncthreads();
  return total;
}

// Group 1: the wave's documents are deduplicated first (one thread each),
// then their rows' chunks are laid end to end and scored by all threads of
// the CTA, U chunks in flight per thread, each chunk's products with query
// terms added in entry order; a document's score is the sum of its chunks'
// partials in chunk order (deterministic, independent of the launch shape).
// Work per thread is balanced whatever the row lengths; seen documents cost
// no row reads.  fp32 rows: a chunk's values (one 32-byte sector) are read
// only where a term is in the query (4-byte read-only loads; most chunks of a
// row miss).  fp16 rows: a chunk is one sector, terms and values read together.
template <int NT, bool FP16, class Src>
__device__ __forceinline__ void eval_wave_flat(const SearchArgs &a, Smem &s, Shared &sh, uint32_t n, const Src &src,
                                               int knn_stage) {
  constexpr int U = 2;
  const int tid = threadIdx.x;
  const bool full = sh.count == a.k;
  const float th = full ? s.tk_s()[a.k - 1] : -INFINITY;
  const uint32_t thid = full ? s.tk_id()[a.k - 1] : 0u;
  float *cpart = s.part();  // the block-score partials are dead while documents are scored
  for (uint32_t i = tid; i < n; i += NT) {
    uint32_t d;
    unsigned long long row;
    src.fetch(i, d, row);
    uint32_t keep = SEISMIC_NONE_ID, nch = 0;
    if (d != SEISMIC_NONE_ID) {
      bool fresh;
      if (s.seen) {
        const uint32_t bit = 1u << (d & 31);
        fresh = !(atomicOr(s.seen + (d >> 5), bit) & bit);
      } else {
        fresh = seen_insert(s.hash(), a.HS - 1u, d, &sh.hash_full);
      }
      if (fresh) {
        keep = d;
        nch = (uint32_t)(row >> 32);
        if (a.prefetch) prefetch_row(a.fwd_data, row, a.fp16);
        if (a.stats) {
          atomicAdd(&sh.st[knn_stage ? SEISMIC_ST_KNN_DOCS : SEISMIC_ST_DOCS], 1ull);
          atomicAdd(&sh.st[knn_stage ? SEISMIC_ST_KNN_NNZ : SEISMIC_ST_DOC_NNZ], (unsigned long long)a.fwd_nnz[d]);
        }
      }
    }
    s.fdoc()[i] = keep;
    s.fc0()[i] = (uint32_t)row;
    s.fpre()[i] = nch;
  }
  __syncthreads();
  // the chunk map of a wave that fits one pass is written by the scan itself
  const uint32_t all = block_exclusive_scan<NT>(s.fpre(), n, sh.wtmp, s.cmap(), a.CAPC);
  const uint32_t *qb = s.qbits();
  const uint16_t *qr = s.qrank();
  const float *qv = s.qval();
  uint32_t i0 = 0;
  while (i0 < n) {
    // a pass: the documents from i0 whose chunks fit in CAPC (one always does)
    const uint32_t base = s.fpre()[i0];
    uint32_t lo = i0 + 1, hi = n;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (s.fpre()[mid] - base <= a.CAPC) lo = mid; else hi = mid - 1;
    }
    const uint32_t i1 = lo, total = s.fpre()[i1] - base;
    if (all > a.CAPC) {  // several passes: map this one
      for (uint32_t i = i0 + tid; i < i1; i += NT) {
        const uint32_t e = s.fpre()[i + 1] - base;
        for (uint32_t c = s.fpre()[i] - base; c < e; c++) s.cmap()[c] = (uint8_t)i;  // i < CAND <= 256
      }
      __syncthreads();
    }
#pragma unroll 1
    for (uint32_t j = tid; j < total; j += NT * U) {
      // a row holds its chunks' terms (16 B each), then their values (32 B each):
      // the terms are read first and a value only where the term is in the query
      uint4 t[U], vh[U];
      const float *vp[U];
#pragma unroll
      for (int u = 0; u < U; u++) {  // past the end: the last chunk again (unconditional loads stay in registers)
        const uint32_t jj = min(j + u * NT, total - 1u);
        {
          const uint32_t i = s.cmap()[jj], p0 = s.fpre()[i];
          const uint32_t nch = s.fpre()[i + 1] - p0, o = base + jj - p0;
          const uint8_t *rec = a.fwd_data + (size_t)s.fc0()[i] * kUnitBytes;
          vp[u] = reinterpret_cast<const float *>(chunk_vals(rec, nch, o, FP16));
          if (FP16) {
            ldg_na_v8(chunk_terms(rec, o, true), t[u], vh[u]);  // the chunk's sector: terms, then halves
          } else {
            t[u] = ldg_na(chunk_terms(rec, o, false));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const uint32_t jj = j + u * NT;
        if (jj < total) {
          const uint32_t tw[4] = {t[u].x, t[u].y, t[u].z, t[u].w};
          const uint32_t hw[4] = {vh[u].x, vh[u].y, vh[u].z, vh[u].w};
          float acc = 0.0f;
#pragma unroll
          for (int e = 0; e < 8; e++) {  // absent terms (most) cost one shared load and no value read
            const uint32_t tt = (e & 1) ? (tw[e >> 1] >> 16) : (tw[e >> 1] & 0xFFFFu);
            const uint32_t w = qb[tt >> 5], sh5 = tt & 31u;
            if ((w >> sh5) & 1u) {
              float v;
              if (FP16) v = __half2float(__ushort_as_half((unsigned short)((e & 1) ? (hw[e >> 1] >> 16) : (hw[e >> 1] & 0xFFFFu))));
              else v = __ldg(vp[u] + e);
              acc = fmaf(qv[qr[tt >> 5] + __popc(w & ((1u << sh5) - 1u))], v, acc);
            }
          }
          cpart[jj] = acc;
        }
      }
    }
    __syncthreads();
    for (uint32_t i = i0 + tid; i < i1; i += NT) {
      const uint32_t d = s.fdoc()[i];
      if (d == SEISMIC_NONE_ID) continue;
      const uint32_t e = s.fpre()[i + 1] - base;
      float p = 0.0f;
      for (uint32_t c = s.fpre()[i] - base; c < e; c++) p += cpart[c];
      if (!full || better(p, d, th, thid)) {
        const uint32_t pos = atomicAdd(&sh.ncand, 1u);
        s.cand_s()[pos] = p;
        s.cand_id()[pos] = d;
      }
    }
    __syncthreads();
    i0 = i1;
  }
  merge_candidates<NT>(a, s, sh);
}

template <int G, int NT, class Src>
__device__ __forceinline__ void eval(const SearchArgs &a, Smem &s, Shared &sh, uint32_t n, const Src &src,
                                     int knn_stage) {
  if constexpr (G == 1) {
    if (a.fp16) eval_wave_flat<NT, true>(a, s, sh, n, src, knn_stage);
    else eval_wave_flat<NT, false>(a, s, sh, n, src, knn_stage);
  } else {
    eval_wave<G, NT>(a, s, sh, n, src, knn_stage);
  }
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

// 5 CTAs of 256 threads per SM (48 registers).  A 40-register build for 6
// CTAs per SM spilled little but measured 3-7 % slower at waves >= 4.
template <int G, int NW>
__global__ void __launch_bounds__(NW * 32, 1280 / (NW * 32))
    k_search(const __grid_constant__ SearchArgs a) {
  constexpr int NT = NW * 32;
  __shared__ Shared sh;
  Smem s{a, a.seen_bm ? a.seen_bm + (size_t)blockIdx.x * a.seen_words : nullptr};
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  bool first = true;

  for (;;) {
    if (tid == 0) {
      if (a.persistent) {
        const uint32_t slot = atomicAdd(a.queue, 1u);
        sh.q = (a.perm && slot < a.nq) ? a.perm[slot] : slot;
      }
      else sh.q = first ? blockIdx.x : a.nq;
    }
    first = false;
    __syncthreads();
    const uint32_t q = sh.q;
    if (q >= a.nq) break;

    // ---------------------------------------------------------- H0: ingest
    const uint64_t qb = a.q_indptr[q], qe = a.q_indptr[q + 1];
    const uint32_t nnz = (uint32_t)(qe - qb);
    for (uint32_t i = tid; i < a.W; i += NT) s.qbits()[i] = 0u;
    if (s.seen) {  // seen_words is a multiple of 4 and the slot is 16-byte aligned
      uint4 *z = reinterpret_cast<uint4 *>(s.seen);
      for (uint32_t i = tid; i < a.seen_words / 4; i += NT) z[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
      for (uint32_t i = tid; i < a.HS; i += NT) s.hash()[i] = 0u;
    }
    if (tid < SEISMIC_STATS_N) sh.st[tid] = tid == SEISMIC_ST_T_START && a.stats ? globaltimer_ns() : 0ull;
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
        if (t < a.dim) atomicOr(&s.qbits()[t >> 5], 1u << (t & 31));
        else sh.bad = 1u;
      }
    }
    __syncthreads();
    const uint32_t nzq = block_rank_scan<NT>(s.qbits(), s.qrank(), a.W, sh.wtmp);
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
        const uint32_t w = s.qbits()[t >> 5];
        const uint32_t pos = s.qrank()[t >> 5] + __popc(w & ((1u << (t & 31)) - 1u));
        s.qval()[pos] = v;
        s.qterm()[pos] = (uint16_t)t;
      }
    }
    __syncthreads();

    // ---------------------------------------------------------- H1: list terms
    if (a.alpha_q > 0.0f) {
      for (uint32_t i = tid; i < nzq; i += NT) {
        const float av = fabsf(s.qval()[i]);
        const uint32_t t = s.qterm()[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < nzq; j++) {
          const float aj = fabsf(s.qval()[j]);
          r += (aj > av || (aj == av && s.qterm()[j] < t)) ? 1u : 0u;
        }
        s.aq()[r] = av;
        s.cutT()[r] = (uint16_t)t;
      }
      __syncthreads();
      if (tid == 0) {  // alpha_q-MSS: fp64 prefix mass in sketch order
        double tot = 0.0;
        for (uint32_t i = 0; i < nzq; i++) tot += (double)s.aq()[i];
        const double target = (double)a.alpha_q * tot;
        double c = 0.0;
        uint32_t keep = nzq;
        for (uint32_t i = 0; i < nzq; i++) {
          c += (double)s.aq()[i];
          if (c >= target) { keep = i + 1; break; }
        }
        sh.ncut = keep;
      }
    } else {
      const uint32_t cut = sh.cut;
      for (uint32_t i = tid; i < nzq; i += NT) {
        const float v = s.qval()[i];
        const uint32_t t = s.qterm()[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < nzq; j++) {
          const float vj = s.qval()[j];
          r += (vj > v || (vj == v && s.qterm()[j] < t)) ? 1u : 0u;
        }
        if (r < cut) s.cutT()[r] = (uint16_t)t;
      }
      if (tid == 0) sh.ncut = min(cut, nzq);
    }
    __syncthreads();
    const uint32_t ncut = a.seed ? 0u : sh.ncut;  // graph refinement: no lists
    const float hf = sh.hf;
    if (a.stats && tid == 0) sh.st[SEISMIC_ST_QUERY_NNZ] = nnz;

    // ---------------------------------------------------------- lists
    for (uint32_t li = 0; li < ncut; li++) {
      const uint32_t t = s.cutT()[li];
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
          const MemberSrc src{a.bdoc + c0, a.bdoc_row + c0};
          eval<G, NT>(a, s, sh, n, src, 0);
        }
        continue;
      }
      // ---- H2: summary scores of every block of the list
      {
        uint32_t words = 0;
        for (uint32_t i = tid; i < nzq; i += NT)
          words += summary_column(a.sbm, a.scptr, a.W, t, s.qterm()[i], s.clo() + i, s.chi() + i);
        if (a.stats && words) atomicAdd(&sh.st[SEISMIC_ST_DIR_LOOKUPS], (unsigned long long)words);
      }
      for (uint32_t i = tid; i < NW * a.BMAX; i += NT) s.part()[i] = 0.0f;
      for (uint32_t b = tid; b <= nb; b += NT) s.bptr()[b] = __ldg(a.bdoc_ptr + g0 + b);  // block member ranges
      __syncthreads();
      {
        float *pw = s.part() + warp * a.BMAX;
        const float *bm = a.blk_m + g0;
        const float *bs = a.blk_size + g0;
        uint32_t ent = 0;
        for (uint32_t i = warp; i < nzq; i += NW) {
          const uint32_t lo = s.clo()[i], hi = s.chi()[i];
          const float qv = s.qval()[i];
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
          for (int w = 0; w < NW; w++) r += s.part()[w * a.BMAX + b];
          s.keys()[b] = ((unsigned long long)(~f2ord(r)) << 32) | b;
        } else {
          s.keys()[b] = ~0ull;
        }
      }
      if (a.stats && tid == 0) sh.st[SEISMIC_ST_BLOCKS_SCORED] += nb;
      __syncthreads();
      // ---- H3: order blocks by (r desc, block asc)
      bitonic_sort_u64<NT>(s.keys(), P2);
      // ---- H4/H5/H6: visit blocks in order, waves of a.wave blocks
      const uint32_t W = min(a.wave, kMaxWave);
      uint32_t bi = 0;
      while (bi < nb) {
        // skip test at the head of the wave (uniform: shared state after a barrier)
        const bool fullk = sh.count == a.k;
        const float theta = fullk ? s.tk_s()[a.k - 1] : -INFINITY;
        const float thr = a.hf_mode == 0 ? hf * theta : theta / hf;
        if (fullk && ord2f(~(uint32_t)(s.keys()[bi] >> 32)) < thr) {
          if (a.stats && tid == 0) sh.st[SEISMIC_ST_BLOCKS_SKIPPED] += nb - bi;
          break;
        }
        // the wave: the next blocks that pass the test against theta now, up to
        // W blocks and CAND documents (a larger block goes alone, in pieces)
        uint32_t be = bi, ndocs = 0;
        while (be < nb && be - bi < W) {
          const uint32_t b = (uint32_t)(s.keys()[be] & 0xFFFFFFFFu);
          if (be > bi && fullk && ord2f(~(uint32_t)(s.keys()[be] >> 32)) < thr) break;
          const uint32_t nd = s.bptr()[b + 1] - s.bptr()[b];
          if (be > bi && ndocs + nd > a.CAND) break;
          ndocs += nd;
          be++;
        }
        if (a.prefetch && tid < W && be + tid < nb) {  // member lists of the next wave's blocks
          const uint32_t b = (uint32_t)(s.keys()[be + tid] & 0xFFFFFFFFu);
          const uint32_t e0 = s.bptr()[b], e1 = s.bptr()[b + 1];
          prefetch_l2(a.bdoc + e0, 4 * (e1 - e0));
          prefetch_l2(a.bdoc_row + e0, 8 * (e1 - e0));
        }
        if (a.stats && tid == 0) {
          sh.st[SEISMIC_ST_BLOCKS_EVALUATED] += be - bi;
          sh.st[SEISMIC_ST_BLOCK_DOCS] += ndocs;
        }
        if (be - bi == 1) {
          const uint32_t b = (uint32_t)(s.keys()[bi] & 0xFFFFFFFFu);
          const uint32_t d0 = s.bptr()[b], d1 = s.bptr()[b + 1];
          for (uint32_t c0 = d0; c0 < d1; c0 += a.CAND) {
            const MemberSrc src{a.bdoc + c0, a.bdoc_row + c0};
            eval<G, NT>(a, s, sh, min(a.CAND, d1 - c0), src, 0);
          }
        } else {
          const WaveBlocks src{s.keys() + bi, s.bptr(), be - bi, a.bdoc, a.bdoc_row};
          eval<G, NT>(a, s, sh, ndocs, src, 0);
        }
        bi = be;
      }
      __syncthreads();
    }

    // graph refinement: the heap starts from the document and its neighbours
    if (a.seed) {
      const SeedSrc src{a.seed[q], a.knn, a.fwd_row, a.kappa, a.knn_bits};
      eval<G, NT>(a, s, sh, 1 + a.kappa, src, 0);
    }

    // ---------------------------------------------------------- H7: kappa-NN expansion
    if (a.use_knn && a.kappa > 0 && sh.count > 0) {
      const uint32_t ns = sh.count;
      for (uint32_t i = tid; i < ns; i += NT) s.clo()[i] = s.tk_id()[i];  // S, fixed before expanding
      __syncthreads();
      const uint32_t total = ns * a.kappa;
      for (uint32_t c0 = 0; c0 < total; c0 += a.CAND) {
        const uint32_t n = min(a.CAND, total - c0);
        const GraphSrc src{s.clo(), a.knn, a.fwd_row, a.kappa, a.knn_bits};
        // positions c0 .. c0 + n of the neighbour list of S
        struct Shifted {
          GraphSrc g;
          uint32_t c0;
          __device__ uint32_t id(uint32_t i) const { return g.id(c0 + i); }
          __device__ unsigned long long row(uint32_t i, uint32_t d) const { return g.row(c0 + i, d); }
          __device__ void fetch(uint32_t i, uint32_t &d, unsigned long long &r) const { g.fetch(c0 + i, d, r); }
        } sh_src{src, c0};
        eval<G, NT>(a, s, sh, n, sh_src, 1);
      }
    }

    // ---------------------------------------------------------- output
    for (uint32_t i = tid; i < a.k; i += NT) {
      const bool ok = i < sh.count;
      a.ids[(size_t)q * a.k + i] = ok ? s.tk_id()[i] : SEISMIC_NONE_ID;
      a.scores[(size_t)q * a.k + i] = ok ? s.tk_s()[i] : -INFINITY;
    }
    if (a.stats && tid == SEISMIC_ST_T_END) sh.st[tid] = globaltimer_ns();
    if (a.stats && tid < SEISMIC_STATS_N) a.stats[(size_t)q * SEISMIC_STATS_N + tid] = sh.st[tid];
    __syncthreads();
    if (!a.persistent) break;
  }
}

template <int G, int NW>
int launch_t(const SearchArgs &a, size_t smem, uint32_t grid, cudaStream_t st) {
  static std::atomic<uint64_t> configured{0};
  int rc = set_smem_limit_once(configured, (const void *)k_search<G, NW>, 200 * 1024);
  if (rc) return rc;
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
  a.off_bptr = take(a.exhaustive ? 4 : (a.BMAX + 1) * 4);
  a.CAPC = 0;
  if (a.flat) {
    // chunk partials reuse the block-score partials; at least 2048 chunks,
    // more than any row holds (kMaxRowNnzBuild / kChunk)
    a.CAPC = std::max<uint32_t>(2048u, (a.exhaustive ? 0u : nw * a.BMAX));
    if (a.exhaustive || nw * a.BMAX < a.CAPC) {
      a.off_part = take(a.CAPC * 4);  // the earlier part region is too small: a fresh one
    }
    a.off_fdoc = take(a.CAND * 4);
    a.off_fc0 = take(a.CAND * 4);
    a.off_fpre = take((a.CAND + 1) * 4);
    a.off_cmap = take(a.CAPC);
  }
  return o;
}

int launch_search(const SearchArgs &a, uint32_t group, uint32_t nw, size_t smem, uint32_t grid, cudaStream_t st) {
#define SZ_CASE(G_, NW_) \
  if (group == G_ && nw == NW_) return launch_t<G_, NW_>(a, smem, grid, st);
  SZ_CASE(1, 4) SZ_CASE(1, 8) SZ_CASE(1, 16)
  SZ_CASE(8, 4) SZ_CASE(8, 8) SZ_CASE(8, 16)
  SZ_CASE(16, 4) SZ_CASE(16, 8) SZ_CASE(16, 16)
  SZ_CASE(32, 4) SZ_CASE(32, 8) SZ_CASE(32, 16)
#undef SZ_CASE
  return fail(SEISMIC_EINVAL, "group must be 1/8/16/32 and cta_warps 4/8/16");
}

int search_occupancy(uint32_t group, uint32_t nw, size_t smem, int *blocks) {
#define SZ_CASE(G_, NW_) \
  if (group == G_ && nw == NW_) return occupancy_t<G_, NW_>(smem, blocks);
  SZ_CASE(1, 4) SZ_CASE(1, 8) SZ_CASE(1, 16)
  SZ_CASE(8, 4) SZ_CASE(8, 8) SZ_CASE(8, 16)
  SZ_CASE(16, 4) SZ_CASE(16, 8) SZ_CASE(16, 16)
  SZ_CASE(32, 4) SZ_CASE(32, 8) SZ_CASE(32, 16)
#undef SZ_CASE
  return fail(SEISMIC_EINVAL, "group must be 1/8/16/32 and cta_warps 4/8/16");
}

}  // namespace seismic

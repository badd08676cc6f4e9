// Query processing, one warp per query: Algorithm "Query processing with
// Seismic" (Section 4.5) with no CTA-wide barrier anywhere.
//
// A CTA holds several independent warps; each warp pulls query ids from a
// device counter and owns a slice of shared memory (the query as a bitmap +
// popcount rank + values, the block scores of the current list) and a seen
// bitmap of the collection in global memory.
//
//  H2  summary scores: every lane streams the list's column entries for the
//      query's terms (one flat index over the columns), multiplies in fp64 and
//      adds the product, rounded to a fixed-point int64 whose scale comes from
//      a bound on |r| (sum |q_i| times the index's largest summary value), with
//      shared-memory 64-bit atomics.  Integer addition is associative, so r_b
//      does not depend on the order the lanes run in.
//  H3  blocks ordered by (r desc, block asc): warp bitonic sort in shared memory.
//  H4  the skip test before each block, exactly as the sequential algorithm.
//  H5  groups of G lanes score one document each (32 / G documents at a
//      time); rows are read as 16-byte vectors.
//  H6  the top-k lives in registers, element e = r * 32 + lane: an offer is
//      placed by ballot (count of better elements) and shifted in with
//      shuffles; theta is the k-th element.  Every offered (score, id) is
//      inserted at once, so the heap after a block is the algorithm's.
//  H7  the kappa-NN expansion of the top-k (S fixed first).
#include <algorithm>

#include "search_common.cuh"

namespace seismic {

namespace {

using namespace dev;

// Top-k in registers: element e = r * 32 + lane, best first.
template <int R>
struct TopK {
  float s[R];
  uint32_t id[R];
  uint32_t count;
  float th;       // k-th score once full
  uint32_t thid;  // k-th id once full

  __device__ void init() {
#pragma unroll
    for (int r = 0; r < R; r++) { s[r] = -INFINITY; id[r] = SEISMIC_NONE_ID; }
    count = 0;
    th = -INFINITY;
    thid = SEISMIC_NONE_ID;
  }
  __device__ __forceinline__ bool admits(float p, uint32_t d, uint32_t k) const {
    return count < k || better(p, d, th, thid);
  }
  // warp-uniform call: (p, d) admitted
  __device__ void insert(float p, uint32_t d, uint32_t k, int lane) {
    uint32_t pos = 0;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint32_t e = r * 32 + lane;
      const bool b = e < count && better(s[r], id[r], p, d);
      pos += __popc(__ballot_sync(0xffffffffu, b));
    }
#pragma unroll
    for (int r = R - 1; r >= 0; r--) {
      float ps = __shfl_up_sync(0xffffffffu, s[r], 1);
      uint32_t pi = __shfl_up_sync(0xffffffffu, id[r], 1);
      float cs = -INFINITY;
      uint32_t ci = SEISMIC_NONE_ID;
      if (r > 0) {
        cs = __shfl_sync(0xffffffffu, s[r > 0 ? r - 1 : 0], 31);
        ci = __shfl_sync(0xffffffffu, id[r > 0 ? r - 1 : 0], 31);
      }
      if (lane == 0) { ps = cs; pi = ci; }
      const uint32_t e = r * 32 + lane;
      if (e > pos) { s[r] = ps; id[r] = pi; }
      else if (e == pos) { s[r] = p; id[r] = d; }
    }
    count = min(k, count + 1);
    if (count == k) {
      const uint32_t e = k - 1;
      float ts = -INFINITY;
      uint32_t ti = SEISMIC_NONE_ID;
#pragma unroll
      for (int r = 0; r < R; r++) {
        float xs = __shfl_sync(0xffffffffu, s[r], e & 31);
        uint32_t xi = __shfl_sync(0xffffffffu, id[r], e & 31);
        if ((e >> 5) == (uint32_t)r) { ts = xs; ti = xi; }
      }
      th = ts;
      thid = ti;
    }
  }
};

struct WarpSmem {
  uint32_t *qbits;
  uint16_t *qrank;
  float *qval;
  uint16_t *qterm;
  uint16_t *cutT;
  float *aq;
  unsigned long long *rk;  // fixed-point r, then sort keys
  uint32_t *clo;
  uint32_t *cofs;
};

struct WarpCounters {
  unsigned long long v[SEISMIC_STATS_N];
};

// Scores documents 0..n of src (n uniform over the warp), offering each new
// one to the top-k.  The seen-bitmap test is issued together with the row's
// loads; a document already seen is scored and dropped.
template <int G, int R, class Src>
__device__ void eval_docs(const SearchArgs &a, const WarpSmem &s, uint32_t *seen, TopK<R> &tk, uint32_t n, Src src,
                          int lane, WarpCounters &st, int knn_stage) {
  constexpr int NG = 32 / G;
  const int grp = lane / G, gl = lane % G;
  const uint32_t gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  // the next round's (id, row) are loaded while this round is scored
  uint32_t dn = SEISMIC_NONE_ID;
  unsigned long long rn = 0ull;
  if ((uint32_t)grp < n) {
    dn = src.id(grp);
    rn = src.row(grp, dn);
  }
  for (uint32_t base = 0; base < n; base += NG) {
    const uint32_t i = base + grp;
    uint32_t d = SEISMIC_NONE_ID, old = 0u, bit = 0u;
    unsigned long long row = 0ull;
    if (i < n) {
      d = dn;
      row = rn;
      if (i + NG < n) {
        dn = src.id(i + NG);
        rn = src.row(i + NG, dn);
      }
      if (d != SEISMIC_NONE_ID) {
        bit = 1u << (d & 31);
        if (gl == 0) old = atomicOr(seen + (d >> 5), bit);
      }
    }
    float p = -INFINITY;
    if (d != SEISMIC_NONE_ID)
      p = row_dot<G>(a.fwd_data, row, a.fp16, gl, gmask, s.qbits, s.qrank, s.qval);
    uint32_t fresh = (d != SEISMIC_NONE_ID && !(old & bit)) ? 1u : 0u;
    fresh = __shfl_sync(0xffffffffu, fresh, grp * G);
    if (fresh && a.stats && gl == 0) {
      st.v[knn_stage ? SEISMIC_ST_KNN_DOCS : SEISMIC_ST_DOCS]++;
      st.v[knn_stage ? SEISMIC_ST_KNN_NNZ : SEISMIC_ST_DOC_NNZ] += a.fwd_nnz[d];
    }
#pragma unroll
    for (int g = 0; g < NG; g++) {
      const uint32_t fg = __shfl_sync(0xffffffffu, fresh, g * G);
      if (!fg) continue;
      const float pg = __shfl_sync(0xffffffffu, p, g * G);
      const uint32_t dg = __shfl_sync(0xffffffffu, d, g * G);
      if (tk.admits(pg, dg, a.k)) tk.insert(pg, dg, a.k, lane);
    }
  }
}

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t x, int lane, uint32_t *total) {
  uint32_t v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  *total = __shfl_sync(0xffffffffu, v, 31);
  return v - x;
}

template <int G, int R>
__global__ void __launch_bounds__(128, 5) k_search_warp(const SearchArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *wb = sm + (size_t)warp * a.warp_bytes;
  WarpSmem s;
  s.qbits = reinterpret_cast<uint32_t *>(wb + a.off_qbits);
  s.qrank = reinterpret_cast<uint16_t *>(wb + a.off_qrank);
  s.qval = reinterpret_cast<float *>(wb + a.off_qval);
  s.qterm = reinterpret_cast<uint16_t *>(wb + a.off_qterm);
  s.cutT = reinterpret_cast<uint16_t *>(wb + a.off_cut);
  s.aq = reinterpret_cast<float *>(wb + a.off_aq);
  s.rk = reinterpret_cast<unsigned long long *>(wb + a.off_keys);
  s.clo = reinterpret_cast<uint32_t *>(wb + a.off_clo);
  s.cofs = reinterpret_cast<uint32_t *>(wb + a.off_chi);
  const size_t wid = (size_t)blockIdx.x * (blockDim.x >> 5) + warp;
  uint32_t *seen = a.seen_bm + wid * a.seen_words;
  const uint32_t W = a.W;

  for (;;) {
    uint32_t q = 0;
    if (lane == 0) {
      const uint32_t slot = atomicAdd(a.queue, 1u);
      q = (a.perm && slot < a.nq) ? a.perm[slot] : slot;
    }
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= a.nq) break;
    WarpCounters st;
    if (a.stats)
      for (int i = 0; i < SEISMIC_STATS_N; i++) st.v[i] = 0ull;
      if (a.stats && lane == 0) st.v[SEISMIC_ST_T_START] = globaltimer_ns();  // lanes' partials are summed

    // ---------------------------------------------------------- H0
    const uint64_t qb = a.q_indptr[q], qe = a.q_indptr[q + 1];
    const uint32_t nnz = (uint32_t)(qe - qb);
    for (uint32_t i = lane; i < W; i += 32) s.qbits[i] = 0u;
    {
      uint4 *z = reinterpret_cast<uint4 *>(seen);
      for (uint32_t i = lane; i < a.seen_words / 4; i += 32) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncwarp();
    uint32_t bad = 0;
    float l1 = 0.0f;
    for (uint32_t i = lane; i < nnz; i += 32) {
      const float v = a.q_vals[qb + i];
      if (v != 0.0f) {
        const uint32_t t = a.q_terms[qb + i];
        if (t < a.dim) { atomicOr(&s.qbits[t >> 5], 1u << (t & 31)); l1 += fabsf(v); }
        else bad = 1;
      }
    }
    __syncwarp();
    {
      const uint32_t per = (W + 31) / 32, lo = min(W, lane * per), hi = min(W, lo + per);
      uint32_t c = 0;
      for (uint32_t i = lo; i < hi; i++) c += __popc(s.qbits[i]);
      uint32_t total;
      uint32_t base = warp_excl_scan(c, lane, &total);
      for (uint32_t i = lo; i < hi; i++) {
        s.qrank[i] = (uint16_t)min(base, 65535u);
        base += __popc(s.qbits[i]);
      }
      bad = __any_sync(0xffffffffu, bad) ? 1u : 0u;
      if (total > a.QN || bad) {
        if (lane == 0) atomicOr(a.queue + 1, 1u);
        for (uint32_t i = lane; i < a.k; i += 32) {
          a.ids[(size_t)q * a.k + i] = SEISMIC_NONE_ID;
          a.scores[(size_t)q * a.k + i] = -INFINITY;
        }
        __syncwarp();
        continue;
      }
      __syncwarp();
      for (uint32_t i = lane; i < nnz; i += 32) {
        const float v = a.q_vals[qb + i];
        if (v != 0.0f) {
          const uint32_t t = a.q_terms[qb + i];
          const uint32_t w = s.qbits[t >> 5];
          const uint32_t pos = s.qrank[t >> 5] + __popc(w & ((1u << (t & 31)) - 1u));
          s.qval[pos] = v;
          s.qterm[pos] = (uint16_t)t;
        }
      }
      __syncwarp();
      const uint32_t nzq = total;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, o);

      // ------------------------------------------------------ H1
      uint32_t cut = a.cut;
      float hf = a.hf;
      if (a.q_cut) { cut = a.q_cut[q]; hf = a.q_hf[q]; }
      uint32_t ncut;
      if (a.alpha_q > 0.0f) {
        for (uint32_t i = lane; i < nzq; i += 32) {
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
        __syncwarp();
        uint32_t keep = nzq;
        if (lane == 0) {  // alpha_q-MSS: fp64 prefix mass in sketch order
          double tot = 0.0;
          for (uint32_t i = 0; i < nzq; i++) tot += (double)s.aq[i];
          const double target = (double)a.alpha_q * tot;
          double c2 = 0.0;
          for (uint32_t i = 0; i < nzq; i++) {
            c2 += (double)s.aq[i];
            if (c2 >= target) { keep = i + 1; break; }
          }
        }
        ncut = __shfl_sync(0xffffffffu, keep, 0);
      } else {
        for (uint32_t i = lane; i < nzq; i += 32) {
          const float v = s.qval[i];
          const uint32_t t = s.qterm[i];
          uint32_t r = 0;
          for (uint32_t j = 0; j < nzq; j++) {
            const float vj = s.qval[j];
            r += (vj > v || (vj == v && s.qterm[j] < t)) ? 1u : 0u;
          }
          if (r < cut) s.cutT[r] = (uint16_t)t;
        }
        ncut = min(cut, nzq);
      }
      __syncwarp();
      if (a.stats && lane == 0) st.v[SEISMIC_ST_QUERY_NNZ] = nnz;
      // fixed-point scale for the summary scores: |r| < 2^61
      const double bound = (double)l1 * 1.0001 * (double)a.sum_absmax + 1e-30;
      const double scale = ldexp(1.0, 61 - ilogb(bound) - 1);

      TopK<R> tk;
      tk.init();
      // ------------------------------------------------------ lists
      for (uint32_t li = 0; li < ncut; li++) {
        const uint32_t t = s.cutT[li];
        const uint32_t g0 = __ldg(a.blk_ptr + t), nb = __ldg(a.blk_ptr + t + 1) - g0;
        if (a.stats && lane == 0) st.v[SEISMIC_ST_LISTS]++;
        if (nb == 0) continue;
        if (a.exhaustive) {
          const uint32_t d0 = __ldg(a.bdoc_ptr + g0), d1 = __ldg(a.bdoc_ptr + g0 + nb);
          if (a.stats && lane == 0) {
            st.v[SEISMIC_ST_BLOCKS_EVALUATED] += nb;
            st.v[SEISMIC_ST_BLOCK_DOCS] += d1 - d0;
          }
          const MemberSrc src{a.bdoc + d0, a.bdoc_row + d0};
          eval_docs<G, R>(a, s, seen, tk, d1 - d0, src, lane, st, 0);
          continue;
        }
        // ---- H2: column ranges, flat offsets, fixed-point scores
        uint32_t carry = 0, dir_words = 0;
        for (uint32_t i0 = 0; i0 < nzq; i0 += 32) {
          const uint32_t i = i0 + lane;
          uint32_t lo = 0, len = 0;
          if (i < nzq) {
            uint32_t hi;
            dir_words += summary_column(a.sbm, a.scptr, a.W, t, s.qterm[i], &lo, &hi);
            len = hi - lo;
            s.clo[i] = lo;
          }
          uint32_t tot;
          const uint32_t ex = warp_excl_scan(len, lane, &tot);
          if (i < nzq) s.cofs[i] = carry + ex;
          carry += tot;
        }
        const uint32_t T = carry;
        dir_words = __reduce_add_sync(0xffffffffu, dir_words);
        if (lane == 0) s.cofs[nzq] = T;
        for (uint32_t b = lane; b < nb; b += 32) s.rk[b] = 0ull;
        __syncwarp();
        {
          const float *bm = a.blk_m + g0;
          const float *bsz = a.blk_size + g0;
          uint32_t c = 0;
          for (uint32_t j = lane; j < T; j += 32) {
            while (s.cofs[c + 1] <= j) c++;
            const uint32_t e = s.clo[c] + (j - s.cofs[c]);
            const uint32_t b = __ldg(a.scol_blk + e);
            double sv;
            if (a.quant) sv = (double)fmaf((float)__ldg(a.scol_code + e), __ldg(bsz + b), __ldg(bm + b));
            else sv = (double)__ldg(a.scol_val + e);
            const long long fx = __double2ll_rn((double)s.qval[c] * sv * scale);
            atomicAdd(s.rk + b, (unsigned long long)fx);
          }
        }
        __syncwarp();
        uint32_t P2 = 1;
        while (P2 < nb) P2 <<= 1;
        for (uint32_t b = lane; b < P2; b += 32) {
          if (b < nb) {
            const float r = (float)((double)(long long)s.rk[b] / scale);
            s.rk[b] = ((unsigned long long)(~f2ord(r)) << 32) | b;
          } else {
            s.rk[b] = ~0ull;
          }
        }
        __syncwarp();
        if (a.stats && lane == 0) {
          st.v[SEISMIC_ST_BLOCKS_SCORED] += nb;
          st.v[SEISMIC_ST_DIR_LOOKUPS] += dir_words;
          st.v[SEISMIC_ST_SUMMARY_ENTRIES] += T;
        }
        // ---- H3: warp bitonic sort
        for (uint32_t k2 = 2; k2 <= P2; k2 <<= 1)
          for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
            for (uint32_t i = lane; i < P2; i += 32) {
              const uint32_t ixj = i ^ j;
              if (ixj > i) {
                const unsigned long long x = s.rk[i], y = s.rk[ixj];
                const bool up = (i & k2) == 0;
                if ((x > y) == up) { s.rk[i] = y; s.rk[ixj] = x; }
              }
            }
            __syncwarp();
          }
        // ---- H4-H6: visit blocks.  While block bi is scored, the member
        // lists of block bi+2 and the rows of block bi+1 are prefetched into L2
        // (speculatively: a skip ends the list, wasting at most two blocks).
        const uint32_t pf = a.prefetch;
        auto members_l2 = [&](uint32_t bj) {
          if (!pf || bj >= nb || lane != 0) return;
          const uint32_t bb = (uint32_t)(s.rk[bj] & 0xFFFFFFFFu);
          const uint32_t e0 = __ldg(a.bdoc_ptr + g0 + bb), e1 = __ldg(a.bdoc_ptr + g0 + bb + 1);
          prefetch_l2(a.bdoc + e0, 4 * (e1 - e0));
          prefetch_l2(a.bdoc_row + e0, 8 * (e1 - e0));
        };
        auto rows_l2 = [&](uint32_t bj) {
          if (!pf || bj >= nb) return;
          const uint32_t bb = (uint32_t)(s.rk[bj] & 0xFFFFFFFFu);
          const uint32_t e0 = __ldg(a.bdoc_ptr + g0 + bb), e1 = min(__ldg(a.bdoc_ptr + g0 + bb + 1), e0 + pf);
          for (uint32_t e = e0 + lane; e < e1; e += 32) {
            const unsigned long long row = __ldg(a.bdoc_row + e);
            prefetch_row(a.fwd_data, row, a.fp16);
          }
        };
        members_l2(0);
        members_l2(1);
        rows_l2(0);
        for (uint32_t bi = 0; bi < nb; bi++) {
          const unsigned long long key = s.rk[bi];
          if (tk.count == a.k) {
            const float r = ord2f(~(uint32_t)(key >> 32));
            const float thr = a.hf_mode == 0 ? hf * tk.th : tk.th / hf;
            if (r < thr) {
              if (a.stats && lane == 0) st.v[SEISMIC_ST_BLOCKS_SKIPPED] += nb - bi;
              break;
            }
          }
          const uint32_t b = (uint32_t)(key & 0xFFFFFFFFu);
          const uint32_t d0 = __ldg(a.bdoc_ptr + g0 + b), d1 = __ldg(a.bdoc_ptr + g0 + b + 1);
          if (a.stats && lane == 0) {
            st.v[SEISMIC_ST_BLOCKS_EVALUATED]++;
            st.v[SEISMIC_ST_BLOCK_DOCS] += d1 - d0;
          }
          members_l2(bi + 2);
          rows_l2(bi + 1);
          const MemberSrc src{a.bdoc + d0, a.bdoc_row + d0};
          eval_docs<G, R>(a, s, seen, tk, d1 - d0, src, lane, st, 0);
        }
        __syncwarp();
      }
      // ------------------------------------------------------ H7
      if (a.use_knn && a.kappa > 0 && tk.count > 0) {
        const uint32_t ns = tk.count;
        uint32_t *S = s.clo;  // column starts are free now; S is fixed before expanding
#pragma unroll
        for (int r = 0; r < R; r++) {
          const uint32_t e = r * 32 + lane;
          if (e < ns) S[e] = tk.id[r];
        }
        __syncwarp();
        const GraphSrc src{S, a.knn, a.fwd_row, a.kappa, a.knn_bits};
        eval_docs<G, R>(a, s, seen, tk, ns * a.kappa, src, lane, st, 1);
      }
      // ------------------------------------------------------ output
#pragma unroll
      for (int r = 0; r < R; r++) {
        const uint32_t e = r * 32 + lane;
        if (e < a.k) {
          const bool ok = e < tk.count;
          a.ids[(size_t)q * a.k + e] = ok ? tk.id[r] : SEISMIC_NONE_ID;
          a.scores[(size_t)q * a.k + e] = ok ? tk.s[r] : -INFINITY;
        }
      }
      if (a.stats) {
        if (lane == 0) st.v[SEISMIC_ST_T_END] = globaltimer_ns();
        for (int i = 0; i < SEISMIC_STATS_N; i++) {
          unsigned long long v = st.v[i];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) a.stats[(size_t)q * SEISMIC_STATS_N + i] = v;
        }
      }
      __syncwarp();
    }
  }
}

template <int G, int R>
int launch_w(const SearchArgs &a, size_t smem, uint32_t grid, uint32_t wpb, cudaStream_t st) {
  static std::atomic<uint64_t> configured{0};
  int rc = set_smem_limit_once(configured, (const void *)k_search_warp<G, R>, 200 * 1024);
  if (rc) return rc;
  k_search_warp<G, R><<<grid, wpb * 32, smem, st>>>(a);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

template <int G, int R>
int occ_w(size_t smem, uint32_t wpb, int *blocks) {
  SZ_CUDA(cudaFuncSetAttribute(k_search_warp<G, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  SZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_search_warp<G, R>, wpb * 32, smem));
  return SEISMIC_OK;
}

}  // namespace

static inline uint32_t al16w(uint32_t x) { return (x + 15u) & ~15u; }

size_t search_layout_warp(SearchArgs &a) {
  uint32_t o = 0;
  auto take = [&](uint32_t bytes) {
    uint32_t r = o;
    o = al16w(o + bytes);
    return r;
  };
  a.off_qbits = take(a.W * 4);
  a.off_qrank = take(a.W * 2);
  a.off_qval = take(a.QN * 4);
  a.off_qterm = take(a.QN * 2);
  a.off_cut = take(a.QN * 2);
  a.off_aq = take(a.alpha_q > 0.0f ? a.QN * 4 : 4);
  a.off_keys = take(a.exhaustive ? 8 : a.BPOW2 * 8);
  a.off_clo = take(std::max(a.QN, a.k) * 4);
  a.off_chi = take((a.QN + 1) * 4);
  a.warp_bytes = o;
  return o;
}

int launch_search_warp(const SearchArgs &a, uint32_t group, size_t smem, uint32_t grid, uint32_t wpb,
                       cudaStream_t st) {
  const uint32_t R = (a.k + 31) / 32;
#define SZ_CASE(G_, R_) \
  if (group == G_ && R <= R_) return launch_w<G_, R_>(a, smem, grid, wpb, st);
  SZ_CASE(4, 1) SZ_CASE(4, 2) SZ_CASE(4, 4)
  SZ_CASE(8, 1) SZ_CASE(8, 2) SZ_CASE(8, 4)
  SZ_CASE(16, 1) SZ_CASE(16, 2) SZ_CASE(16, 4)
  SZ_CASE(32, 1) SZ_CASE(32, 2) SZ_CASE(32, 4)
#undef SZ_CASE
  return fail(SEISMIC_EINVAL, "warp search: group must be 4/8/16/32 and k <= 128");
}

int search_occupancy_warp(uint32_t group, uint32_t k, size_t smem, uint32_t wpb, int *blocks) {
  const uint32_t R = (k + 31) / 32;
#define SZ_CASE(G_, R_) \
  if (group == G_ && R <= R_) return occ_w<G_, R_>(smem, wpb, blocks);
  SZ_CASE(4, 1) SZ_CASE(4, 2) SZ_CASE(4, 4)
  SZ_CASE(8, 1) SZ_CASE(8, 2) SZ_CASE(8, 4)
  SZ_CASE(16, 1) SZ_CASE(16, 2) SZ_CASE(16, 4)
  SZ_CASE(32, 1) SZ_CASE(32, 2) SZ_CASE(32, 4)
#undef SZ_CASE
  return fail(SEISMIC_EINVAL, "warp search: group must be 4/8/16/32 and k <= 128");
}

}  // namespace seismic

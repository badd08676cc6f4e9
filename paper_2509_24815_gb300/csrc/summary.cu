// Block summaries and their term-major layout on the device: the summary
// part of Algorithm "Indexing with Seismic" (Section 4.4) -- the coordinate
// max of a block's members (Eq. "summary", Section 4.1.3), its alpha-mass
// subvector sketch (Definition "alpha-mass subvector sketch", Section 3.2)
// and the 8-bit scalar quantisation of Section 4.1.3 -- followed by the
// term-major column layout the search reads.
//
// Every result is bit-identical to a sequential computation in the reading
// the oracle takes:
//  - phi_i = max over the members holding term i; a member without the term
//    contributes 0, so a negative maximum over a strict subset becomes 0;
//  - the nonzero coordinates are ordered by (|phi| desc, term asc) (a
//    bitonic sort of 64-bit keys, unique because terms are), the total mass
//    and the prefix masses are added in fp64 in that order by one thread (the
//    same operations in the same order), and the smallest prefix reaching
//    alpha * total is kept;
//  - m = min and M = max of the kept values, size = fp32((M - m) / 256) in
//    fp64, code = min(255, floor((v - m) / size)) in fp64 (0 when size = 0).
//
// Pass 1 (k_sum_select) computes per block the kept count, the key of the
// last kept coordinate, (m, size) and its contribution to the bound on
// |summary value|; the host turns the counts into offsets; pass 2
// (k_sum_write) recomputes the max vector and writes the kept coordinates in
// term order (block-major).  k_cols_count / k_cols_fill then build, per list,
// the presence bitmap directory and the columns (blocks ascending within a
// column) by a stable counting sort over the list's blocks in order.
#include "seismic_impl.h"

namespace seismic {

namespace {

constexpr int kSumThreads = 256;
constexpr uint32_t kSumCap = 4096;  // distinct terms of a block held in shared memory (power of two)

__device__ __forceinline__ uint32_t f2ord(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// (|phi| desc, term asc) as an ascending 64-bit key: the complemented bits of
// |phi| (a non-negative float orders like its bits), then the term
__device__ __forceinline__ unsigned long long sum_key(float phi, uint32_t term) {
  return ((unsigned long long)(0xFFFFFFFFu - __float_as_uint(fabsf(phi))) << 16) | term;
}
__device__ __forceinline__ double key_mass(unsigned long long key) {
  return (double)__uint_as_float(0xFFFFFFFFu - (uint32_t)(key >> 16));
}

// Contiguous range of W words for thread tid (the slots of a word range are
// contiguous and in term order).
__device__ __forceinline__ void word_range(uint32_t W, uint32_t &lo, uint32_t &hi) {
  const uint32_t per = (W + kSumThreads - 1) / kSumThreads;
  lo = min(W, threadIdx.x * per);
  hi = min(W, lo + per);
}

// Exclusive scan of one value per thread; returns this thread's offset and
// writes the total to *total (valid for every thread on return).
__device__ uint32_t cta_scan(uint32_t x, uint32_t *wtmp, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int nw = kSumThreads / 32;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();  // wtmp may still be read by a previous call
  if (lane == 31) wtmp[warp] = inc;
  __syncthreads();
  uint32_t before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < nw; w++) {
    const uint32_t t = wtmp[w];
    before += w < warp ? t : 0u;
    tot += t;
  }
  *total = tot;
  return before + inc - x;
}

// The popcount rank of each bitmap word (slot of its first set bit); returns
// the number of set bits.  Ends with a barrier.
__device__ uint32_t rank_words(const uint32_t *bits, uint32_t *rank, uint32_t W, uint32_t *wtmp) {
  uint32_t lo, hi, s = 0, total;
  word_range(W, lo, hi);
  for (uint32_t i = lo; i < hi; i++) s += __popc(bits[i]);
  uint32_t base = cta_scan(s, wtmp, &total);
  for (uint32_t i = lo; i < hi; i++) {
    rank[i] = base;
    base += __popc(bits[i]);
  }
  __syncthreads();
  return total;
}

__device__ __forceinline__ uint32_t slot_of(const uint32_t *bits, const uint32_t *rank, uint32_t s) {
  const uint32_t w = s >> 5;
  return rank[w] + __popc(bits[w] & ((1u << (s & 31)) - 1u));
}

// Ascending bitonic sort of keys[0 .. P2) (P2 a power of two); every thread calls it.
__device__ void bitonic_u64(unsigned long long *keys, uint32_t P2) {
  for (uint32_t k2 = 2; k2 <= P2; k2 <<= 1)
    for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P2; i += kSumThreads) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long x = keys[i], y = keys[ixj];
          if ((x > y) == ((i & k2) == 0)) {
            keys[i] = y;
            keys[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
}

struct SumShared {
  uint32_t wtmp[kSumThreads / 32];
  uint32_t ne, nz, keep, lo, hi;
  unsigned long long thr;
};

// The block's max vector: bits/rank over its distinct terms (slot = rank in
// term order) and phi[slot] = the summary value of that term as float bits.
// phi and keys point to shared memory when the block has at most kSumCap
// distinct terms, else to this CTA's global scratch; keys is used here for the
// members-per-slot counts.  Returns the number of distinct terms.
__device__ uint32_t block_max(const SumArgs &a, uint64_t g, uint32_t *bits, uint32_t *rank, SumShared &sh,
                              uint32_t *sphi, unsigned long long *skeys, uint32_t *&phi,
                              unsigned long long *&keys) {
  constexpr int NW = kSumThreads / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t m0 = a.bdptr[g], m1 = a.bdptr[g + 1], bs = m1 - m0;
  for (uint32_t i = threadIdx.x; i < a.W; i += kSumThreads) bits[i] = 0u;
  __syncthreads();
  for (uint32_t m = m0 + warp; m < m1; m += NW) {
    const uint32_t j = a.bdoc[m];
    const uint64_t p1 = a.ip[j + 1];
    for (uint64_t p = a.ip[j] + lane; p < p1; p += 32) {
      const uint32_t s = a.t[p];
      atomicOr(&bits[s >> 5], 1u << (s & 31));
    }
  }
  __syncthreads();
  const uint32_t ne = rank_words(bits, rank, a.W, sh.wtmp);
  if (ne <= kSumCap) {
    phi = sphi;
    keys = skeys;
  } else {
    phi = a.gphi + (size_t)blockIdx.x * a.gstride;
    keys = a.gkeys + (size_t)blockIdx.x * a.gstride;
  }
  uint32_t *cnt = reinterpret_cast<uint32_t *>(keys);
  for (uint32_t i = threadIdx.x; i < ne; i += kSumThreads) {
    phi[i] = 0u;  // below the order code of every float
    cnt[i] = 0u;
  }
  __syncthreads();
  for (uint32_t m = m0 + warp; m < m1; m += NW) {
    const uint32_t j = a.bdoc[m];
    const uint64_t p1 = a.ip[j + 1];
    for (uint64_t p = a.ip[j] + lane; p < p1; p += 32) {
      const uint32_t slot = slot_of(bits, rank, a.t[p]);
      atomicMax(&phi[slot], f2ord(a.v[p]));
      atomicAdd(&cnt[slot], 1u);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < ne; i += kSumThreads) {
    float f = ord2f(phi[i]);
    if (cnt[i] < bs && f < 0.0f) f = 0.0f;  // the members without the term contribute 0
    phi[i] = __float_as_uint(f);
  }
  __syncthreads();
  return ne;
}

__device__ __forceinline__ void sum_smem(const SumArgs &a, unsigned char *sm, uint32_t *&bits, uint32_t *&rank,
                                         uint32_t *&sphi, unsigned long long *&skeys) {
  bits = reinterpret_cast<uint32_t *>(sm);
  rank = bits + a.W;
  sphi = rank + a.W;  // 2W + kSumCap words: a multiple of 2, so the keys are 8-byte aligned
  skeys = reinterpret_cast<unsigned long long *>(sphi + kSumCap);
}

// Pass 1: per block, the alpha-MSS size, the key of its last coordinate, (m, size)
// and the block's bound on |summary value| as the search reconstructs it.
__global__ void __launch_bounds__(kSumThreads) k_sum_select(const SumArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ SumShared sh;
  uint32_t *bits, *rank, *sphi;
  unsigned long long *skeys;
  sum_smem(a, sm, bits, rank, sphi, skeys);
  for (uint64_t g = blockIdx.x; g < a.nblk; g += gridDim.x) {
    uint32_t *phi;
    unsigned long long *keys;
    const uint32_t ne = block_max(a, g, bits, rank, sh, sphi, skeys, phi, keys);
    // the keys of the nonzero coordinates; zero ones and the padding sort last
    uint32_t lo, hi, nzl = 0;
    word_range(a.W, lo, hi);
    for (uint32_t w = lo; w < hi; w++) {
      uint32_t word = bits[w], r = rank[w];
      while (word) {
        const uint32_t b = __ffs(word) - 1;
        word &= word - 1u;
        const float f = __uint_as_float(phi[r]);
        keys[r++] = f != 0.0f ? sum_key(f, w * 32 + b) : ~0ull;
        nzl += f != 0.0f ? 1u : 0u;
      }
    }
    uint32_t P2 = 1;
    while (P2 < ne) P2 <<= 1;
    for (uint32_t i = ne + threadIdx.x; i < P2; i += kSumThreads) keys[i] = ~0ull;
    uint32_t nz;
    cta_scan(nzl, sh.wtmp, &nz);  // its barriers publish the keys
    bitonic_u64(keys, P2);
    if (threadIdx.x == 0) {
      // the mass in fp64, added in the sketch's order; the smallest prefix reaching alpha * total
      double total = 0.0;
      for (uint32_t i = 0; i < nz; i++) total += key_mass(keys[i]);
      const double target = a.alpha * total;
      double c = 0.0;
      uint32_t keep = nz;
      for (uint32_t i = 0; i < nz; i++) {
        c += key_mass(keys[i]);
        if (c >= target) {
          keep = i + 1;
          break;
        }
      }
      sh.keep = keep;
      sh.thr = keep ? keys[keep - 1] : 0ull;
      sh.lo = 0xFFFFFFFFu;
      sh.hi = 0u;
    }
    __syncthreads();
    const uint32_t keep = sh.keep;
    for (uint32_t i = threadIdx.x; i < keep; i += kSumThreads) {
      const uint32_t o = f2ord(__uint_as_float(phi[slot_of(bits, rank, (uint32_t)(keys[i] & 0xFFFFu))]));
      atomicMin(&sh.lo, o);
      atomicMax(&sh.hi, o);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const float vlo = keep ? ord2f(sh.lo) : 0.0f, vhi = keep ? ord2f(sh.hi) : 0.0f;
      const float size = (float)(((double)vhi - (double)vlo) / 256.0);
      a.keep[g] = keep;
      a.thr[g] = sh.thr;
      a.bm[g] = vlo;
      a.bsz[g] = size;
      a.babs[g] = a.quant ? fabs((double)vlo) + 256.0 * (double)size : (keep ? key_mass(keys[0]) : 0.0);
    }
    __syncthreads();
  }
}

// Pass 2: the kept coordinates of each block, in term order, at sptr[g]:
// term, value (when sval is given) and 8-bit code (quantised indexes).
__global__ void __launch_bounds__(kSumThreads) k_sum_write(const SumArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ SumShared sh;
  uint32_t *bits, *rank, *sphi;
  unsigned long long *skeys;
  sum_smem(a, sm, bits, rank, sphi, skeys);
  for (uint64_t g = blockIdx.x; g < a.nblk; g += gridDim.x) {
    uint32_t *phi;
    unsigned long long *keys;
    block_max(a, g, bits, rank, sh, sphi, skeys, phi, keys);
    const uint32_t keep = a.keep[g];
    const unsigned long long thr = a.thr[g];
    const float m = a.bm[g], size = a.bsz[g];
    uint32_t lo, hi, n = 0;
    word_range(a.W, lo, hi);
    for (uint32_t w = lo; w < hi; w++) {
      uint32_t word = bits[w], r = rank[w];
      while (word) {
        const uint32_t b = __ffs(word) - 1;
        word &= word - 1u;
        const float f = __uint_as_float(phi[r++]);
        n += (keep && f != 0.0f && sum_key(f, w * 32 + b) <= thr) ? 1u : 0u;
      }
    }
    uint32_t total;
    uint32_t o = a.sptr[g] + cta_scan(n, sh.wtmp, &total);
    const uint32_t oend = a.sptr[g + 1];  // == o + n: the count of pass 1 (the same max vector, the same keys)
    for (uint32_t w = lo; w < hi; w++) {
      uint32_t word = bits[w], r = rank[w];
      while (word) {
        const uint32_t b = __ffs(word) - 1, s = w * 32 + b;
        word &= word - 1u;
        const float f = __uint_as_float(phi[r++]);
        if (!(keep && f != 0.0f && sum_key(f, s) <= thr) || o >= oend) continue;
        a.sterm[o] = (uint16_t)s;
        if (a.sval) a.sval[o] = f;
        if (a.quant) {
          double q = size > 0.0f ? floor(((double)f - (double)m) / (double)size) : 0.0;
          q = fmin(255.0, fmax(0.0, q));
          a.scode[o] = (uint8_t)q;
        }
        o++;
      }
    }
    __syncthreads();
  }
}

// The presence bitmap of each list's summary terms (the directory's bits)
// and its number of columns.
__global__ void __launch_bounds__(kSumThreads) k_cols_count(const ColArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint32_t wtmp[kSumThreads / 32];
  uint32_t *bits = reinterpret_cast<uint32_t *>(sm);
  for (uint32_t t = blockIdx.x; t < a.dim; t += gridDim.x) {
    for (uint32_t i = threadIdx.x; i < a.W; i += kSumThreads) bits[i] = 0u;
    __syncthreads();
    const uint32_t e0 = a.sptr[a.blk_ptr[t]], e1 = a.sptr[a.blk_ptr[t + 1]];
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += kSumThreads) {
      const uint32_t s = a.sterm[e];
      atomicOr(&bits[s >> 5], 1u << (s & 31));
    }
    __syncthreads();
    uint32_t n = 0;
    for (uint32_t i = threadIdx.x; i < a.W; i += kSumThreads) {
      a.sbm[(size_t)t * a.W + i] = make_uint2(bits[i], 0u);
      n += __popc(bits[i]);
    }
    uint32_t total;
    cta_scan(n, wtmp, &total);
    if (threadIdx.x == 0) a.ncols[t] = total;
    __syncthreads();
  }
}

// The columns of each list: column c of list t (its c-th summary term in
// ascending order) holds the list's blocks whose summary has that term, in
// ascending block order, at scptr[cbase[t] + c] .. scptr[cbase[t] + c + 1);
// the list's entries keep their block-major range [sptr[first block],
// sptr[last block + 1]) and its pointers end with a sentinel.  Entries are
// placed block by block (a block's terms are distinct, so its entries take
// distinct cursors), which makes the counting sort stable.
__global__ void __launch_bounds__(kSumThreads) k_cols_fill(const ColArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint32_t wtmp[kSumThreads / 32];
  uint32_t *bits = reinterpret_cast<uint32_t *>(sm), *rank = bits + a.W;
  for (uint32_t t = blockIdx.x; t < a.dim; t += gridDim.x) {
    const uint2 *dir = a.sbm + (size_t)t * a.W;
    for (uint32_t i = threadIdx.x; i < a.W; i += kSumThreads) bits[i] = dir[i].x;
    __syncthreads();
    const uint32_t ncols = rank_words(bits, rank, a.W, wtmp), cb = a.cbase[t];
    for (uint32_t i = threadIdx.x; i < a.W; i += kSumThreads) a.sbm[(size_t)t * a.W + i].y = cb + rank[i];
    const uint32_t g0 = a.blk_ptr[t], g1 = a.blk_ptr[t + 1], e0 = a.sptr[g0], e1 = a.sptr[g1];
    uint32_t *cnt = a.scptr + cb;
    for (uint32_t c = threadIdx.x; c < ncols; c += kSumThreads) cnt[c] = 0u;
    __syncthreads();
    for (uint32_t e = e0 + threadIdx.x; e < e1; e += kSumThreads) atomicAdd(&cnt[slot_of(bits, rank, a.sterm[e])], 1u);
    __syncthreads();
    // column starts: an exclusive scan of the counts (contiguous ranges per thread), from e0
    const uint32_t per = (ncols + kSumThreads - 1) / kSumThreads, lo = min(ncols, threadIdx.x * per),
                   hi = min(ncols, lo + per);
    uint32_t sum = 0, total;
    for (uint32_t c = lo; c < hi; c++) sum += __ldcg(cnt + c);
    uint32_t run = e0 + cta_scan(sum, wtmp, &total);
    for (uint32_t c = lo; c < hi; c++) {
      const uint32_t n = __ldcg(cnt + c);
      cnt[c] = run;
      a.cur[cb + c] = run;
      run += n;
    }
    if (threadIdx.x == 0) cnt[ncols] = e1;  // the list's sentinel
    __syncthreads();
    for (uint32_t g = g0; g < g1; g++) {
      const uint32_t b0 = a.sptr[g], b1 = a.sptr[g + 1];
      for (uint32_t e = b0 + threadIdx.x; e < b1; e += kSumThreads) {
        uint32_t *cp = a.cur + cb + slot_of(bits, rank, a.sterm[e]);
        const uint32_t o = __ldcg(cp);
        *cp = o + 1u;
        a.cblk[o] = (uint16_t)(g - g0);
        if (a.quant) a.ccode[o] = a.scode[e];
        else a.cval[o] = a.sval[e];
      }
      __syncthreads();
    }
  }
}

size_t sum_smem_bytes(uint32_t W) { return (size_t)(2 * W + kSumCap) * 4 + (size_t)kSumCap * 8; }

}  // namespace

int sum_occupancy(uint32_t W, int *blocks) {
  const size_t smem = sum_smem_bytes(W);
  SZ_CUDA(cudaFuncSetAttribute(k_sum_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  SZ_CUDA(cudaFuncSetAttribute(k_sum_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int b1 = 1, b2 = 1;
  SZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_sum_select, kSumThreads, smem));
  SZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_sum_write, kSumThreads, smem));
  *blocks = std::max(1, std::min(b1, b2));
  return SEISMIC_OK;
}

int launch_sum_pass(const SumArgs &a, int pass, uint32_t grid, cudaStream_t st) {
  if (!grid || !a.nblk) return SEISMIC_OK;
  const size_t smem = sum_smem_bytes(a.W);
  if (pass == 1) k_sum_select<<<grid, kSumThreads, smem, st>>>(a);
  else k_sum_write<<<grid, kSumThreads, smem, st>>>(a);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

int launch_cols_pass(const ColArgs &a, int pass, uint32_t grid, cudaStream_t st) {
  if (!grid || !a.dim) return SEISMIC_OK;
  if (pass == 1) k_cols_count<<<grid, kSumThreads, (size_t)a.W * 4, st>>>(a);
  else k_cols_fill<<<grid, kSumThreads, (size_t)a.W * 8, st>>>(a);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

}  // namespace seismic

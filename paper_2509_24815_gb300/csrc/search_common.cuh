// Device helpers shared by the two search kernels (CTA per query, warp per query).
#pragma once

#include <cuda_fp16.h>

#include "search_impl.h"

namespace seismic {
namespace dev {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// float <-> order-preserving u32
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
  return __uint_as_float(u);
}

// the result order: score descending, then id ascending
__device__ __forceinline__ bool better(float s1, uint32_t i1, float s2, uint32_t i2) {
  return s1 > s2 || (s1 == s2 && i1 < i2);
}

// q[t] from the shared-memory query: bitmap word, popcount rank, values in term order
__device__ __forceinline__ float qlookup(const uint32_t *__restrict__ qbits, const uint16_t *__restrict__ qrank,
                                         const float *__restrict__ qval, uint32_t t) {
  const uint32_t w = qbits[t >> 5];
  const uint32_t bit = 1u << (t & 31);
  if (!(w & bit)) return 0.0f;
  return qval[qrank[t >> 5] + __popc(w & (bit - 1u))];
}

// 16-byte read-only load that does not allocate in L1 (rows are read once per
// query; reuse across queries is in L2)
__device__ __forceinline__ uint4 ldg_na(const void *p) {
  uint4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "l"(p));
  return r;
}

// 32-byte read-only load (one DRAM sector) that does not allocate in L1; p is
// 32-byte aligned
__device__ __forceinline__ void ldg_na_v8(const void *p, uint4 &lo, uint4 &hi) {
  asm volatile("ld.global.nc.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
               : "l"(p));
}

// TMA bulk prefetch of [p, p + bytes) into L2 (no registers, no completion):
// p is rounded down and the end up to 16-byte boundaries; device allocations
// carry 256 bytes of slack, so the rounded range stays inside them.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), lo = a & ~(uintptr_t)15;
  const uint32_t n = (uint32_t)(((a + bytes + 15) & ~(uintptr_t)15) - lo);
  if (n) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(n) : "memory");
}

// Forward rows (see the layout in seismic_impl.h): a row descriptor is its
// first 32-byte unit | its chunk count << 32.
__device__ __forceinline__ const uint8_t *row_base(const uint8_t *fwd, unsigned long long row) {
  return fwd + (size_t)(uint32_t)row * kUnitBytes;
}
// chunk o's 16 bytes of terms, and the address of its values
__device__ __forceinline__ const uint8_t *chunk_terms(const uint8_t *rec, uint32_t o, int fp16) {
  return rec + (fp16 ? kUnitBytes : 16u) * (size_t)o;
}
__device__ __forceinline__ const uint8_t *chunk_vals(const uint8_t *rec, uint32_t nch, uint32_t o, int fp16) {
  return fp16 ? rec + (size_t)kUnitBytes * o + 16 : rec + (size_t)kUnitBytes * ((nch + 1) / 2 + o);
}

// Adds q[t_e] * v_e over one chunk's 8 entries to acc (in entry order):
// tw = the chunk's terms, v = its values as 8 fp32 or 8 fp16 in 4 words.
__device__ __forceinline__ float chunk_dot(const uint32_t tw[4], const uint32_t vv[8], int fp16,
                                           const uint32_t *__restrict__ qbits, const uint16_t *__restrict__ qrank,
                                           const float *__restrict__ qval, float acc) {
#pragma unroll
  for (int e = 0; e < 8; e++) {
    const uint32_t t = (e & 1) ? (tw[e >> 1] >> 16) : (tw[e >> 1] & 0xFFFFu);
    float v;
    if (fp16) v = __half2float(__ushort_as_half((unsigned short)((e & 1) ? (vv[e >> 1] >> 16) : (vv[e >> 1] & 0xFFFFu))));
    else v = __uint_as_float(vv[e]);
    acc = fmaf(qlookup(qbits, qrank, qval, t), v, acc);
  }
  return acc;
}

// <q, row> for a forward-index row of nch 8-entry chunks.  G lanes cooperate:
// lane gl takes chunks gl, gl + G, ... and keeps U of them in flight; it adds
// its products in chunk order and the G partial sums are combined by a fixed
// butterfly, so the result depends on G only.
template <int G>
__device__ __forceinline__ float row_dot(const uint8_t *__restrict__ fwd, unsigned long long row, int fp16, int gl,
                                         uint32_t gmask, const uint32_t *__restrict__ qbits,
                                         const uint16_t *__restrict__ qrank, const float *__restrict__ qval) {
  constexpr int U = G >= 16 ? 2 : 16 / G;
  const uint8_t *rec = row_base(fwd, row);
  const uint32_t nch = (uint32_t)(row >> 32);
  float acc = 0.0f;
#pragma unroll 1
  for (uint32_t c = gl; c < nch; c += U * G) {
    uint4 t[U], va[U], vb[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint32_t cc = c + u * G;
      t[u] = make_uint4(0u, 0u, 0u, 0u);
      va[u] = t[u];
      vb[u] = t[u];
      if (cc < nch) {
        t[u] = ldg_na(chunk_terms(rec, cc, fp16));
        const uint8_t *vp = chunk_vals(rec, nch, cc, fp16);
        va[u] = ldg_na(vp);
        if (!fp16) vb[u] = ldg_na(vp + 16);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (c + u * G >= nch) break;
      const uint32_t tw[4] = {t[u].x, t[u].y, t[u].z, t[u].w};
      const uint32_t vv[8] = {va[u].x, va[u].y, va[u].z, va[u].w, vb[u].x, vb[u].y, vb[u].z, vb[u].w};
      acc = chunk_dot(tw, vv, fp16, qbits, qrank, qval, acc);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gmask, acc, o, G);
  return acc;
}

__device__ __forceinline__ void prefetch_row(const uint8_t *fwd, unsigned long long row, int fp16) {
  prefetch_l2(row_base(fwd, row), kUnitBytes * row_units((uint32_t)(row >> 32), fp16));
}

// The summary column of term s in list t: [*lo, *hi) in the scol_* arrays
// (empty when the list's summaries never hold s).  Returns the 4-byte words
// read (2 for the presence word, 2 more for a column's bounds).
__device__ __forceinline__ uint32_t summary_column(const uint2 *__restrict__ sbm, const uint32_t *__restrict__ scptr,
                                                   uint32_t W, uint32_t t, uint32_t s, uint32_t *lo, uint32_t *hi) {
  const uint2 e = __ldg(sbm + (size_t)t * W + (s >> 5));
  const uint32_t bit = 1u << (s & 31);
  if (!(e.x & bit)) {
    *lo = 0;
    *hi = 0;
    return 2;
  }
  const uint32_t c = e.y + __popc(e.x & (bit - 1u));
  *lo = __ldg(scptr + c);
  *hi = __ldg(scptr + c + 1);
  return 4;
}

// Entry e of the bit-packed kappa-NN graph (bits per id; all ones = missing).
__device__ __forceinline__ uint32_t knn_entry(const uint32_t *__restrict__ words, uint32_t bits, uint64_t e) {
  const uint64_t b = e * bits;
  const uint32_t w = (uint32_t)(b >> 5), sh = (uint32_t)(b & 31);
  uint64_t x = __ldg(words + w);
  if (sh + bits > 32) x |= (uint64_t)__ldg(words + w + 1) << 32;
  const uint32_t v = (uint32_t)(x >> sh) & (uint32_t)((1ull << bits) - 1ull);
  return v == (uint32_t)((1ull << bits) - 1ull) ? SEISMIC_NONE_ID : v;
}

// Document sources: id(i), and row(i, id) = first chunk | chunks << 32.
// fetch(i, d, row) reads both with independent loads.
struct MemberSrc {  // a contiguous range of block members (ids and rows side by side)
  const uint32_t *ids;
  const unsigned long long *rows;
  __device__ __forceinline__ uint32_t id(uint32_t i) const { return __ldg(ids + i); }
  __device__ __forceinline__ unsigned long long row(uint32_t i, uint32_t) const { return __ldg(rows + i); }
  __device__ __forceinline__ void fetch(uint32_t i, uint32_t &d, unsigned long long &r) const {
    d = __ldg(ids + i);
    r = __ldg(rows + i);
  }
};

struct GraphSrc {  // the kappa-NN neighbours of the ids in S
  const uint32_t *S, *knn;
  const unsigned long long *frow;
  uint32_t kappa, bits;
  __device__ __forceinline__ uint32_t id(uint32_t x) const {
    return knn_entry(knn, bits, (uint64_t)S[x / kappa] * kappa + (x % kappa));
  }
  __device__ __forceinline__ unsigned long long row(uint32_t, uint32_t d) const {
    return d == SEISMIC_NONE_ID ? 0ull : __ldg(frow + d);
  }
  __device__ __forceinline__ void fetch(uint32_t x, uint32_t &d, unsigned long long &r) const {
    d = id(x);
    r = row(x, d);
  }
};

struct SeedSrc {  // a document, then its kappa-NN neighbours
  uint32_t doc;
  const uint32_t *knn;
  const unsigned long long *frow;
  uint32_t kappa, bits;
  __device__ __forceinline__ uint32_t id(uint32_t i) const {
    return i == 0 ? doc : knn_entry(knn, bits, (uint64_t)doc * kappa + (i - 1));
  }
  __device__ __forceinline__ unsigned long long row(uint32_t, uint32_t d) const {
    return d == SEISMIC_NONE_ID ? 0ull : __ldg(frow + d);
  }
  __device__ __forceinline__ void fetch(uint32_t i, uint32_t &d, unsigned long long &r) const {
    d = id(i);
    r = row(i, d);
  }
};

}  // namespace dev
}  // namespace seismic

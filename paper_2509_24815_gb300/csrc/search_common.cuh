// Device helpers shared by the two search kernels (CTA per query, warp per query).
#pragma once

#include "search_impl.h"

namespace seismic {
namespace dev {

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

// TMA bulk prefetch of [p, p + bytes) into L2 (no registers, no completion):
// p is rounded down and the end up to 16-byte boundaries; device allocations
// carry 256 bytes of slack, so the rounded range stays inside them.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), lo = a & ~(uintptr_t)15;
  const uint32_t n = (uint32_t)(((a + bytes + 15) & ~(uintptr_t)15) - lo);
  if (n) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(n) : "memory");
}

// <q, row> for a forward-index row of nch 8-entry chunks starting at chunk c0
// (16 B of terms, then 32 B of values per chunk).  G lanes cooperate: lane gl
// takes chunks gl, gl + G, ... and keeps U of them in flight; it adds its
// products in chunk order and the G partial sums are combined by a fixed
// butterfly, so the result depends on G only.
template <int G>
__device__ __forceinline__ float row_dot(const uint8_t *__restrict__ fwd, uint32_t c0, uint32_t nch, int gl,
                                         uint32_t gmask, const uint32_t *__restrict__ qbits,
                                         const uint16_t *__restrict__ qrank, const float *__restrict__ qval) {
  constexpr int U = G >= 16 ? 2 : 16 / G;
  const uint8_t *rec = fwd + (size_t)c0 * 48;
  const uint8_t *vrec = rec + 16 * (size_t)nch;
  float acc = 0.0f;
#pragma unroll 1
  for (uint32_t c = gl; c < nch; c += U * G) {
    uint4 t[U], va[U], vb[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const uint32_t cc = c + u * G;
      if (cc < nch) {
        t[u] = ldg_na(rec + 16 * (size_t)cc);
        va[u] = ldg_na(vrec + 32 * (size_t)cc);
        vb[u] = ldg_na(vrec + 32 * (size_t)cc + 16);
      } else {
        t[u] = make_uint4(0u, 0u, 0u, 0u);
        va[u] = t[u];
        vb[u] = t[u];
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (c + u * G >= nch) break;
      const uint32_t tw[4] = {t[u].x, t[u].y, t[u].z, t[u].w};
      const uint32_t vv[8] = {va[u].x, va[u].y, va[u].z, va[u].w, vb[u].x, vb[u].y, vb[u].z, vb[u].w};
#pragma unroll
      for (int e = 0; e < 4; e++) {
        acc = fmaf(qlookup(qbits, qrank, qval, tw[e] & 0xFFFFu), __uint_as_float(vv[2 * e]), acc);
        acc = fmaf(qlookup(qbits, qrank, qval, tw[e] >> 16), __uint_as_float(vv[2 * e + 1]), acc);
      }
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(gmask, acc, o, G);
  return acc;
}

__device__ __forceinline__ void prefetch_row(const uint8_t *fwd, unsigned long long row) {
  prefetch_l2(fwd + (size_t)(uint32_t)row * 48, 48u * (uint32_t)(row >> 32));
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
  const uint32_t *S, *knn, *cptr;
  uint32_t kappa;
  __device__ __forceinline__ uint32_t id(uint32_t x) const {
    return __ldg(knn + (size_t)S[x / kappa] * kappa + (x % kappa));
  }
  __device__ __forceinline__ unsigned long long row(uint32_t, uint32_t d) const {
    if (d == SEISMIC_NONE_ID) return 0ull;
    const uint32_t c0 = __ldg(cptr + d);
    return (unsigned long long)c0 | ((unsigned long long)(__ldg(cptr + d + 1) - c0) << 32);
  }
  __device__ __forceinline__ void fetch(uint32_t x, uint32_t &d, unsigned long long &r) const {
    d = id(x);
    r = row(x, d);
  }
};

}  // namespace dev
}  // namespace seismic

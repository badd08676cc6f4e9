// Exact top-k (Definition "SMIPS", Section 2) on the device: the recall
// judge, and the exact kappa-NN graph (Eq. "knn-graph") for small
// collections.
//
// One CTA per query.  Scores accumulate term-at-a-time over the unpruned
// lists into a per-CTA fp32 array of n_docs entries (zero between queries),
// in ascending query-term order with a barrier between terms, so every sum is
// deterministic.  Candidates are then offered once each: an atomic exchange
// replaces a touched document's score by a marker, so a document in several
// lists is offered by whichever list reaches it first.  Offers that beat the
// current k-th (score desc, id asc) go to a shared buffer that is merged with
// the top-k by a bitonic sort of packed keys whenever it could overflow.
// Documents that share no term with the query score 0 and are offered in
// ascending id order while they can still enter.
#include "search_impl.h"

namespace seismic {

namespace {

constexpr int kExNT = 256;
constexpr uint32_t kExCB = 4096;  // sort area: buffer + top-k
constexpr uint32_t kExFlush = 2048;
constexpr uint32_t kMark = 0xFFFFFFFFu;  // NaN bit pattern: "already offered"

__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
  return __uint_as_float(u);
}
// ascending key order = (score desc, id asc)
__device__ __forceinline__ unsigned long long mkkey(float s, uint32_t id) {
  return ((unsigned long long)(~f2ord(s)) << 32) | id;
}

struct ExShared {
  uint32_t cbn, count;
  unsigned long long theta;
};

__device__ void ex_merge(unsigned long long *cb, unsigned long long *tk, ExShared &sh, uint32_t k) {
  const int tid = threadIdx.x;
  const uint32_t cbn = sh.cbn, cnt = sh.count, n = cbn + cnt;
  for (uint32_t i = tid; i < cnt; i += kExNT) cb[cbn + i] = tk[i];
  uint32_t P2 = 1;
  while (P2 < n) P2 <<= 1;
  for (uint32_t i = n + tid; i < P2; i += kExNT) cb[i] = ~0ull;
  __syncthreads();
  for (uint32_t k2 = 2; k2 <= P2; k2 <<= 1)
    for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < P2; i += kExNT) {
        uint32_t ixj = i ^ j;
        if (ixj > i) {
          unsigned long long x = cb[i], y = cb[ixj];
          bool up = (i & k2) == 0;
          if ((x > y) == up) { cb[i] = y; cb[ixj] = x; }
        }
      }
      __syncthreads();
    }
  const uint32_t nc = min(k, n);
  for (uint32_t i = tid; i < nc; i += kExNT) tk[i] = cb[i];
  __syncthreads();
  if (tid == 0) {
    sh.count = nc;
    sh.cbn = 0;
    sh.theta = nc == k ? tk[k - 1] : ~0ull;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kExNT) k_exact(const ExactArgs a) {
  __shared__ unsigned long long cb[kExCB];
  __shared__ unsigned long long tk[kExactMaxK];
  __shared__ ExShared sh;
  const int tid = threadIdx.x;
  float *acc = a.acc + (size_t)blockIdx.x * a.n_docs;
  uint32_t *accb = reinterpret_cast<uint32_t *>(acc);
  for (uint32_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
    const uint64_t qb = a.q_indptr[q], qe = a.q_indptr[q + 1];
    if (tid == 0) { sh.cbn = 0; sh.count = 0; sh.theta = ~0ull; }
    // pass 1: accumulate
    for (uint64_t e = qb; e < qe; e++) {
      const float v = a.q_vals[e];
      if (v == 0.0f) continue;
      const uint32_t t = a.q_terms[e];
      const uint32_t p0 = a.full_ptr[t], p1 = a.full_ptr[t + 1];
      for (uint32_t p = p0 + tid; p < p1; p += kExNT) {
        const uint32_t d = a.full_doc[p];
        acc[d] = fmaf(v, a.full_val[p], acc[d]);
      }
      __syncthreads();
    }
    __syncthreads();
    // pass 2: offer every touched document once
    for (uint64_t e = qb; e < qe; e++) {
      if (a.q_vals[e] == 0.0f) continue;
      const uint32_t t = a.q_terms[e];
      const uint32_t p0 = a.full_ptr[t], p1 = a.full_ptr[t + 1];
      for (uint32_t base = p0; base < p1; base += kExNT) {
        const uint32_t p = base + tid;
        if (p < p1) {
          const uint32_t d = a.full_doc[p];
          const uint32_t x = atomicExch(&accb[d], kMark);
          if (x != kMark) {
            const unsigned long long key = mkkey(__uint_as_float(x), d);
            if (sh.count < a.k || key < sh.theta) cb[atomicAdd(&sh.cbn, 1u)] = key;
          }
        }
        __syncthreads();
        if (sh.cbn > kExFlush - kExNT) ex_merge(cb, tk, sh, a.k);
      }
    }
    // untouched documents score 0: offer them by ascending id while they can enter
    for (uint32_t base = 0; base < a.n_docs; base += kExNT) {
      if (sh.count == a.k && mkkey(0.0f, base) > sh.theta) break;
      const uint32_t d = base + tid;
      if (d < a.n_docs && accb[d] != kMark) {
        const unsigned long long key = mkkey(0.0f, d);
        if (sh.count < a.k || key < sh.theta) cb[atomicAdd(&sh.cbn, 1u)] = key;
      }
      __syncthreads();
      if (sh.cbn > kExFlush - kExNT) ex_merge(cb, tk, sh, a.k);
    }
    __syncthreads();
    if (sh.cbn > 0) ex_merge(cb, tk, sh, a.k);
    // pass 3: restore zeros
    for (uint64_t e = qb; e < qe; e++) {
      if (a.q_vals[e] == 0.0f) continue;
      const uint32_t t = a.q_terms[e];
      for (uint32_t p = a.full_ptr[t] + tid; p < a.full_ptr[t + 1]; p += kExNT) acc[a.full_doc[p]] = 0.0f;
    }
    for (uint32_t i = tid; i < a.k; i += kExNT) {
      const bool ok = i < sh.count;
      a.ids[(size_t)q * a.k + i] = ok ? (uint32_t)(tk[i] & 0xFFFFFFFFu) : SEISMIC_NONE_ID;
      a.scores[(size_t)q * a.k + i] = ok ? ord2f(~(uint32_t)(tk[i] >> 32)) : -INFINITY;
    }
    __syncthreads();
  }
}

}  // namespace

int launch_exact(const ExactArgs &a, uint32_t grid, cudaStream_t st) {
  if (a.k == 0 || a.k > kExactMaxK) return fail(SEISMIC_EINVAL, "exact search: k must be in 1..1024");
  k_exact<<<grid, kExNT, 0, st>>>(a);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

}  // namespace seismic

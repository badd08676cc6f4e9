// Posting-list pruning on the device: each list L_t keeps its top-lambda_t
// postings by (value desc, doc asc) (the fixed-lambda form of Table 4 or the
// proportional Set alpha-MSS, Definition "Set alpha-MSS", Section 3.2; the
// tie-break is the oracle's reading), stored in that order.
//
// One CTA per list.  A posting is the 64-bit key (~order(value) << 32 | doc),
// which ascends in exactly that order and is unique within a list.  A list of
// at most kPruneCap postings is sorted whole in shared memory; a longer one
// first finds its lambda-th smallest key by an MSB-first radix select (eight
// 8-bit digits, each a histogram over the postings still matching the digits
// chosen so far), then gathers the lambda keys up to it and sorts them.  Lists
// whose lambda_t exceeds kPruneCap are left to the host (launch_prune reports
// the cap).
#include "seismic_impl.h"

namespace seismic {

namespace {

constexpr int kPruneThreads = 512;
constexpr uint32_t kPruneCap = 8192;  // keys a list sorts in shared memory (power of two)

__device__ __forceinline__ unsigned long long post_key(float v, uint32_t doc) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // ascends with v
  return ((unsigned long long)~ord << 32) | doc;
}

__device__ void bitonic_keys(unsigned long long *keys, uint32_t P2) {
  for (uint32_t k2 = 2; k2 <= P2; k2 <<= 1)
    for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < P2; i += kPruneThreads) {
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

__global__ void __launch_bounds__(kPruneThreads) k_prune(const uint64_t *__restrict__ fptr,
                                                         const uint32_t *__restrict__ fdoc,
                                                         const float *__restrict__ fval,
                                                         const uint32_t *__restrict__ lptr, uint32_t dim,
                                                         uint32_t *__restrict__ ldoc) {
  extern __shared__ __align__(16) unsigned long long keys[];  // kPruneCap
  __shared__ uint32_t hist[256];
  __shared__ uint32_t s_cnt, s_need;
  __shared__ unsigned long long s_prefix;
  const uint32_t tid = threadIdx.x;
  for (uint32_t t = blockIdx.x; t < dim; t += gridDim.x) {
    const uint64_t a = fptr[t], n = fptr[t + 1] - a;
    const uint32_t l0 = lptr[t], lam = lptr[t + 1] - l0;
    if (lam == 0 || lam > kPruneCap) continue;  // uniform over the CTA
    uint32_t m;
    if (n <= kPruneCap) {
      for (uint32_t i = tid; i < (uint32_t)n; i += kPruneThreads) keys[i] = post_key(fval[a + i], fdoc[a + i]);
      m = (uint32_t)n;
    } else {
      // the lam-th smallest key, one 8-bit digit per pass from the top
      unsigned long long prefix = 0ull;
      uint32_t need = lam;
      for (int shift = 56; shift >= 0; shift -= 8) {
        const unsigned long long hi = shift == 56 ? 0ull : (~0ull << (shift + 8));  // the digits chosen so far
        for (uint32_t i = tid; i < 256; i += kPruneThreads) hist[i] = 0u;
        __syncthreads();
        for (uint64_t i = tid; i < n; i += kPruneThreads) {
          const unsigned long long key = post_key(fval[a + i], fdoc[a + i]);
          if ((key & hi) == prefix) atomicAdd(&hist[(uint32_t)(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid == 0) {
          uint32_t before = 0, dgt = 255;
          for (uint32_t dd = 0; dd < 256; dd++) {
            if (before + hist[dd] >= need) {
              dgt = dd;
              break;
            }
            before += hist[dd];
          }
          s_prefix = prefix | ((unsigned long long)dgt << shift);
          s_need = need - before;
        }
        __syncthreads();
        prefix = s_prefix;
        need = s_need;
        __syncthreads();  // s_prefix and s_need are rewritten by the next pass
      }
      // exactly lam keys are <= the lam-th smallest (keys are unique)
      if (tid == 0) s_cnt = 0u;
      __syncthreads();
      for (uint64_t i = tid; i < n; i += kPruneThreads) {
        const unsigned long long key = post_key(fval[a + i], fdoc[a + i]);
        if (key <= prefix) {
          const uint32_t pos = atomicAdd(&s_cnt, 1u);
          if (pos < kPruneCap) keys[pos] = key;
        }
      }
      __syncthreads();
      m = min(s_cnt, kPruneCap);
    }
    uint32_t P2 = 1;
    while (P2 < m) P2 <<= 1;
    for (uint32_t i = m + tid; i < P2; i += kPruneThreads) keys[i] = ~0ull;
    __syncthreads();
    bitonic_keys(keys, P2);
    for (uint32_t i = tid; i < lam; i += kPruneThreads) ldoc[l0 + i] = (uint32_t)keys[i];
    __syncthreads();
  }
}

}  // namespace

int launch_prune(const uint64_t *fptr, const uint32_t *fdoc, const float *fval, const uint32_t *lptr, uint32_t dim,
                 uint32_t *ldoc, uint32_t *cap, cudaStream_t st) {
  *cap = kPruneCap;
  if (!dim) return SEISMIC_OK;
  const size_t smem = (size_t)kPruneCap * 8;
  static std::atomic<uint64_t> configured{0};
  int rc = set_smem_limit_once(configured, (const void *)k_prune, (int)smem);
  if (rc) return rc;
  int sms = 1, occ = 1, dev = 0;
  SZ_CUDA(cudaGetDevice(&dev));
  SZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_prune, kPruneThreads, smem));
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(dim, (uint64_t)sms * std::max(1, occ)));
  k_prune<<<grid, kPruneThreads, smem, st>>>(fptr, fdoc, fval, lptr, dim, ldoc);
  SZ_CUDA(cudaGetLastError());
  return SEISMIC_OK;
}

}  // namespace seismic

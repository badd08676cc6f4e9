// Internal declarations of the Seismic GB300 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <functional>
#include <string>
#include <thread>
#include <vector>

#include "../../include/seismic.h"

namespace seismic {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define SZ_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Sets a kernel's dynamic shared-memory limit once per device (function
// attributes belong to the device's context); safe from several host threads,
// since setting it twice is harmless.
inline int set_smem_limit_once(std::atomic<uint64_t> &done, const void *func, int bytes) {
  int dev = 0;
  SZ_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return SEISMIC_OK;
  SZ_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_release);
  return SEISMIC_OK;
}

// ---------------------------------------------------------------- threads
inline int hw_threads(int want) {
  int n = (int)std::thread::hardware_concurrency();
  if (n <= 0) n = 1;
  return want > 0 ? want : n;
}

// Runs fn(i, tid) for i in [0, n) on `threads` workers pulling from a counter.
inline void parallel_for(int64_t n, int threads, const std::function<void(int64_t, int)> &fn) {
  if (threads <= 1 || n < 2) {
    for (int64_t i = 0; i < n; i++) fn(i, 0);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < threads; t++)
    th.emplace_back([&, t] {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        fn(i, t);
      }
    });
  for (auto &x : th) x.join();
}

// Runs fn(lo, hi) over [0, n) in ranges of `grain` items, on `threads`
// workers: for loops whose items are too small to be handed out one by one.
inline void parallel_ranges(int64_t n, int threads, int64_t grain,
                            const std::function<void(int64_t, int64_t)> &fn) {
  const int64_t parts = (n + grain - 1) / grain;
  parallel_for(parts, threads, [&](int64_t r, int) { fn(r * grain, std::min(n, (r + 1) * grain)); });
}

// ---------------------------------------------------------------- device memory
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  int alloc(size_t n) {  // SEISMIC_OK or SEISMIC_ENOMEM; contents undefined
    release();
    // 256 bytes of slack: readers may round a range out to 16-byte boundaries
    // (bulk L2 prefetches), which must stay inside the allocation
    cudaError_t e = cudaMalloc(&p, n + 256);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return fail(SEISMIC_ENOMEM, std::string("cudaMalloc of ") + std::to_string(n) + " bytes failed");
    }
    bytes = n;
    return SEISMIC_OK;
  }
  int ensure(size_t n) { return n <= bytes && p ? SEISMIC_OK : alloc(n); }
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

template <class T> int upload(DevBuf &b, const std::vector<T> &v) {
  int rc = b.alloc(v.size() * sizeof(T));
  if (rc) return rc;
  if (!v.empty()) SZ_CUDA(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SEISMIC_OK;
}

// Forward-index layout.  Each row is padded to a multiple of 8 entries (c
// chunks; padding entries are (term 0, value 0), which add 0) and stored as a
// record that starts on a 32-byte DRAM sector and fills whole sectors
// ("units").  A row is addressed by its first unit and its chunk count.
//   fp32 values: the 8c u16 terms (16c bytes, padded to a multiple of 32),
//     then the 8c fp32 values, chunk o's 8 values in the 32-byte unit
//     ceil(c/2) + o, so the values of one chunk are one sector;
//     units per row = ceil(c/2) + c.
//   fp16 values: chunk o is unit o, its 8 u16 terms then its 8 fp16 values;
//     units per row = c.
constexpr uint32_t kChunk = 8;
constexpr uint32_t kUnitBytes = 32;
__host__ __device__ inline uint32_t row_units(uint32_t nch, int fp16) { return fp16 ? nch : (nch + 1) / 2 + nch; }

// Limits checked on the host before any device work.
constexpr uint32_t kMaxRowNnzBuild = 8192;  // clustering stages a centroid chunk in shared memory
constexpr uint32_t kMaxK = 1024;

// Device memory one search call works in: one per concurrent stream.
struct Workspace {
  DevBuf q;       // staged host queries
  DevBuf out;     // staged outputs
  DevBuf stats;   // per-query work counters
  DevBuf queue;   // persistent work counter, error word, scratch words
  DevBuf params;  // learned mode: features and per-query (cut, heap_factor)
  DevBuf seen;    // per-CTA (or per-warp) seen bitmaps
  DevBuf perm;    // work-queue order keys and permutation
};

}  // namespace seismic

struct seismic_index {
  int device = 0;
  uint32_t dim = 0;
  uint64_t n_docs = 0, nnz = 0, n_postings = 0, n_blocks = 0, n_sum = 0;
  seismic_build_params bp{};
  uint32_t max_blocks_per_list = 0;
  uint32_t max_block_docs = 0;
  float sum_absmax = 0.0f;  // >= every |summary value| as the search dequantises it

  // forward index
  seismic::DevBuf fwd_row;   // u64[n_docs]: first 32-byte unit | chunks << 32
  seismic::DevBuf fwd_data;  // the row records
  seismic::DevBuf fwd_nnz;   // u16[n_docs] true nonzeros per row (work counters only)

  // pruned lists, blocks
  seismic::DevBuf list_ptr;  // u32[dim+1]
  seismic::DevBuf list_doc;  // u32[n_postings]
  seismic::DevBuf cent;      // u32[n_postings] cluster index per list position
  seismic::DevBuf blk_ptr;   // u32[dim+1]
  seismic::DevBuf bdoc_ptr;  // u32[n_blocks+1]
  seismic::DevBuf bdoc;      // u32[n_postings]
  seismic::DevBuf bdoc_row;  // u64[n_postings]: member's forward row, first unit | chunks << 32
  seismic::DevBuf blk_m;     // f32[n_blocks]
  seismic::DevBuf blk_size;  // f32[n_blocks]

  // summaries, block-major (export / save)
  seismic::DevBuf sum_ptr;   // u32[n_blocks+1]
  seismic::DevBuf sum_term;  // u16[n_sum]
  seismic::DevBuf sum_val;   // f32[n_sum]
  seismic::DevBuf sum_code;  // u8[n_sum]

  // summaries, term-major per list (search)
  // summary directory: list t's column of term s exists iff bit s & 31 of
  // sbm[t * W + s / 32].x is set (W = ceil(dim / 32)); its index is
  // sbm[...].y + popcount of the lower bits of that word, and its entries are
  // scol_*[scptr[index] .. scptr[index + 1]).  Each list's column pointers end
  // with a sentinel, so memory is dim * W * 8 bytes + 4 per column.
  seismic::DevBuf sbm;       // uint2[dim * W]: presence bits, first column index of the word
  seismic::DevBuf scptr;     // u32[columns + dim]
  seismic::DevBuf scol_blk;  // u16[n_sum] local block index
  seismic::DevBuf scol_code; // u8[n_sum]
  seismic::DevBuf scol_val;  // f32[n_sum] (fp32 summaries)

  // unpruned lists for exact search
  int has_full = 0;
  seismic::DevBuf full_ptr;  // u32[dim+1]
  seismic::DevBuf full_doc;  // u32[nnz]
  seismic::DevBuf full_val;  // f32[nnz]

  // kappa-NN graph, ids bit-packed: entry e (= doc * kappa + slot) holds
  // knn_bits bits starting at bit e * knn_bits of the u32 word array (low bits
  // first); the all-ones code is a missing neighbour
  uint32_t kappa = 0;
  uint32_t knn_bits = 0;
  seismic::DevBuf knn;

  // MLP
  int has_mlp = 0;
  seismic::DevBuf mlp;       // f32[SEISMIC_MLP_PARAMS]

  // the default search workspace (grown on demand); concurrent searches on
  // other streams bring their own
  seismic::Workspace ws;
  seismic::DevBuf ws_exact;  // exact-search accumulators
};

namespace seismic {
// Block summaries on the device (summary.cu).
struct SumArgs {
  const uint64_t *ip;  // the collection: CSR rows (terms ascending, no zeros)
  const uint16_t *t;
  const float *v;
  const uint32_t *bdptr;  // u32[nblk + 1]: members of block g
  const uint32_t *bdoc;
  uint64_t nblk;
  uint32_t W;  // ceil(dim / 32)
  double alpha;
  int quant;
  // pass 1 outputs: kept entries, key of the last kept one, (m, size), bound on |value|
  uint32_t *keep;
  unsigned long long *thr;
  float *bm, *bsz;
  double *babs;
  // pass 2 outputs, block-major at sptr[g] (sval may be NULL)
  const uint32_t *sptr;
  uint16_t *sterm;
  float *sval;
  uint8_t *scode;
  // scratch for blocks with more distinct terms than shared memory holds:
  // gstride phi words and keys per CTA of the launch
  uint32_t *gphi;
  unsigned long long *gkeys;
  uint32_t gstride;
};
struct ColArgs {
  uint32_t dim, W;
  const uint32_t *blk_ptr, *sptr;
  const uint16_t *sterm;
  const float *sval;
  const uint8_t *scode;
  int quant;
  uint2 *sbm;             // uint2[dim * W]: presence bits, first column index of the word
  uint32_t *ncols;        // u32[dim]: columns of list t (count pass)
  const uint32_t *cbase;  // u32[dim]: first column of list t (fill pass)
  uint32_t *scptr, *cur;  // column pointers (+ one sentinel per list), cursors
  uint16_t *cblk;
  uint8_t *ccode;
  float *cval;
};
// Pruned lists (prune.cu): ldoc[lptr[t] ..] = list t's top (lptr[t+1] - lptr[t])
// postings by (value desc, doc asc), for every list whose count is at most *cap
// (set by the call); the others are left for the host.
int launch_prune(const uint64_t *fptr, const uint32_t *fdoc, const float *fval, const uint32_t *lptr, uint32_t dim,
                 uint32_t *ldoc, uint32_t *cap, cudaStream_t st);
// grid: CTAs of the launch (the scratch holds gstride entries for each)
int launch_sum_pass(const SumArgs &a, int pass, uint32_t grid, cudaStream_t st);
int launch_cols_pass(const ColArgs &a, int pass, uint32_t grid, cudaStream_t st);
int sum_occupancy(uint32_t W, int *blocks);

uint64_t device_bytes(const seismic_index *ix);
int validate_host_csr(const seismic_csr *m, const char *what, uint32_t dim_expect);
}  // namespace seismic

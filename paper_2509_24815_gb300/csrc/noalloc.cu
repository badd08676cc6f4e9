// seismic_search_noalloc: query processing that allocates no memory.
//
// Some callers cannot allocate device memory while they run queries: a
// serving process whose memory pool is fixed at start-up, a caller that keeps
// cudaMalloc (which can synchronise the device) off its latency path, or a
// runtime that forbids allocation once its own arenas are set.  This entry
// point serves them.  The only working memory the search needs beyond the
// caller's inputs and outputs -- the work-queue counter, an error word and one
// "seen" bitmap of the collection per persistent CTA -- lives in the fixed
// array below, which every GPU that loads the library holds until exit.
#include <mutex>

#include "search_impl.h"

namespace seismic {
namespace {

constexpr size_t kNoAllocBytes = 32ull << 20;  // 32 MiB
constexpr size_t kNoAllocHeader = 256;         // queue counter, error word
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// In host code `g_noalloc_scratch` names a host-side stand-in, not device
// memory: the device address is looked up once per device, with that device
// current, and passed to the kernel.
std::mutex g_noalloc_mu;
void *g_noalloc_addr[128] = {};

int noalloc_scratch(int dev, void **out) {
  if (dev < 0 || dev >= 128) return fail(SEISMIC_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return SEISMIC_OK;
}

}  // namespace
}  // namespace seismic

using namespace seismic;

extern "C" int seismic_search_noalloc(seismic_index *ix, const seismic_csr *queries, const seismic_search_params *p,
                                      uint32_t *ids_out, float *scores_out, void *stream) {
  if (!ix || !queries || !p || !ids_out || !scores_out) return fail(SEISMIC_EINVAL, "NULL argument");
  if (!queries->on_device) return fail(SEISMIC_EINVAL, "noalloc search: queries must be on the device");
  if (queries->dim != ix->dim) return fail(SEISMIC_EINVAL, "queries: dim differs from the index");
  if (p->max_query_nnz == 0) return fail(SEISMIC_EINVAL, "noalloc search: max_query_nnz must be given");
  if (p->k == 0 || p->k > kMaxK) return fail(SEISMIC_EINVAL, "k must be in 1..1024");
  if (p->learned) return fail(SEISMIC_EINVAL, "noalloc search: learned parameters need a features buffer");
  if (p->alpha_q <= 0.0f && p->cut == 0) return fail(SEISMIC_EINVAL, "cut must be >= 1");
  if (p->alpha_q > 1.0f) return fail(SEISMIC_EINVAL, "alpha_q must be <= 1");
  if (!p->exhaustive && !(p->heap_factor > 0.0f)) return fail(SEISMIC_EINVAL, "heap_factor must be > 0");
  if (p->hf_mode != 0 && p->hf_mode != 1) return fail(SEISMIC_EINVAL, "hf_mode must be 0 or 1");
  if (p->use_knn && ix->kappa == 0) return fail(SEISMIC_EINVAL, "use_knn: the index has no kappa-NN graph");
  if (p->shape == 2) return fail(SEISMIC_EINVAL, "noalloc search: only the CTA-per-query shape (0 or 1)");
  if (p->shape > 2) return fail(SEISMIC_EINVAL, "shape must be 0 (auto), 1 (CTA per query) or 2 (warp per query)");
  const uint32_t group = p->group ? p->group : 1, nw = p->cta_warps ? p->cta_warps : 8;
  if (!(group == 1 || group == 8 || group == 16 || group == 32) || !(nw == 4 || nw == 8 || nw == 16))
    return fail(SEISMIC_EINVAL, "noalloc search: group must be 1/8/16/32 and cta_warps 4/8/16");
  if (queries->n_rows == 0) return SEISMIC_OK;
  if (queries->n_rows > 0x7FFFFFFFull) return fail(SEISMIC_EINVAL, "too many queries in one call");
  const uint64_t words = ((ix->n_docs + 31) / 32 + 3) & ~3ull;
  const uint64_t per_cta = words * 4;
  const uint64_t cap_ctas = (kNoAllocBytes - kNoAllocHeader) / per_cta;
  if (cap_ctas == 0)
    return fail(SEISMIC_EBUDGET, "noalloc search: the collection needs a " + std::to_string(per_cta) +
                                     "-byte seen bitmap; the fixed scratch holds " +
                                     std::to_string(kNoAllocBytes - kNoAllocHeader));
  SZ_CUDA(cudaSetDevice(ix->device));
  void *scratch = nullptr;
  int rc = noalloc_scratch(ix->device, &scratch);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t nq = (uint32_t)queries->n_rows;
  uint32_t *queue = reinterpret_cast<uint32_t *>(scratch);
  SZ_CUDA(cudaMemsetAsync(queue, 0, 16, st));

  SearchArgs a{};
  a.fwd_row = ix->fwd_row.as<unsigned long long>();
  a.fwd_data = ix->fwd_data.as<uint8_t>();
  a.fp16 = ix->bp.values_fp16 ? 1 : 0;
  a.fwd_nnz = ix->fwd_nnz.as<uint16_t>();
  a.blk_ptr = ix->blk_ptr.as<uint32_t>();
  a.bdoc_ptr = ix->bdoc_ptr.as<uint32_t>();
  a.bdoc = ix->bdoc.as<uint32_t>();
  a.bdoc_row = ix->bdoc_row.as<unsigned long long>();
  a.blk_m = ix->blk_m.as<float>();
  a.blk_size = ix->blk_size.as<float>();
  a.sbm = ix->sbm.as<uint2>();
  a.scptr = ix->scptr.as<uint32_t>();
  a.scol_blk = ix->scol_blk.as<uint16_t>();
  a.scol_code = ix->scol_code.as<uint8_t>();
  a.scol_val = ix->scol_val.as<float>();
  a.knn = ix->knn.as<uint32_t>();
  a.kappa = ix->kappa;
  a.knn_bits = ix->knn_bits;
  a.dim = ix->dim;
  a.quant = ix->bp.quantize_u8 ? 1 : 0;
  a.q_indptr = queries->indptr;
  a.q_terms = queries->terms;
  a.q_vals = queries->vals;
  a.nq = nq;
  a.k = p->k;
  a.cut = p->cut;
  a.hf = p->heap_factor;
  a.hf_mode = p->hf_mode;
  a.exhaustive = p->exhaustive ? 1 : 0;
  a.use_knn = p->use_knn ? 1 : 0;
  a.alpha_q = p->alpha_q > 0.0f ? p->alpha_q : 0.0f;
  a.wave = p->wave ? p->wave : 1;
  a.ids = ids_out;
  a.scores = scores_out;
  a.stats = nullptr;
  a.queue = queue;
  a.persistent = 1;
  a.W = (ix->dim + 31) / 32;
  a.QN = std::max<uint32_t>(4, (p->max_query_nnz + 3) & ~3u);
  a.BMAX = std::max<uint32_t>(1, ix->max_blocks_per_list);
  a.BPOW2 = 1;
  while (a.BPOW2 < a.BMAX) a.BPOW2 <<= 1;
  a.HS = 16;
  a.CAND = 256;
  a.sum_absmax = ix->sum_absmax;
  a.prefetch = p->no_prefetch ? 0u : 256u;
  a.perm = nullptr;
  a.flat = group == 1 ? 1u : 0u;
  const size_t smem = search_layout(a, nw);
  if (smem > 200 * 1024) return fail(SEISMIC_EBUDGET, "search: shared memory per query exceeds 200 KB");
  int blocks = 1;
  if ((rc = search_occupancy(group, nw, smem, &blocks))) return rc;
  int sms = 1;
  SZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device));
  uint64_t grid = std::min<uint64_t>(nq, (uint64_t)std::max(1, blocks) * sms);
  grid = std::min<uint64_t>(grid, cap_ctas);
  a.seen_words = (uint32_t)words;
  a.seen_bm = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(scratch) + kNoAllocHeader);
  return launch_search(a, group, nw, smem, (uint32_t)grid, st);
}

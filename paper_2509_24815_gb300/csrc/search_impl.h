// Launch arguments of the search kernels (internal).
#pragma once

#include "seismic_impl.h"

namespace seismic {

struct SearchArgs {
  // index
  const unsigned long long *fwd_row;  // per document: first 32-byte unit | chunks << 32
  const uint8_t *fwd_data;
  int fp16;                           // forward values are fp16 (unit per chunk) rather than fp32
  const uint16_t *fwd_nnz;
  const uint32_t *blk_ptr;
  const uint32_t *bdoc_ptr;
  const uint32_t *bdoc;
  const unsigned long long *bdoc_row;  // member's forward row: first chunk | chunks << 32
  const float *blk_m;
  const float *blk_size;
  const uint2 *sbm;       // summary directory: presence bits + column base per 32-term word of a list
  const uint32_t *scptr;  // column pointers into scol_*
  const uint16_t *scol_blk;
  const uint8_t *scol_code;
  const float *scol_val;
  const uint32_t *knn;    // bit-packed ids, knn_bits each
  uint32_t kappa, knn_bits;
  uint32_t dim;
  int quant;
  // queries: CSR rows
  const uint64_t *q_indptr;
  const uint16_t *q_terms;
  const float *q_vals;
  uint32_t nq;
  // parameters
  uint32_t k, cut;
  float hf;
  int hf_mode, exhaustive, use_knn;
  float alpha_q;
  uint32_t wave;
  const uint32_t *q_cut;  // learned per-query parameters, or NULL
  const float *q_hf;
  // outputs
  uint32_t *ids;
  float *scores;
  unsigned long long *stats;
  uint32_t *queue;  // [0] next query (persistent), [1] error bits
  int persistent;
  // seen set in global memory: one bitmap of seen_words words per CTA of a
  // persistent launch (NULL: the bounded shared-memory hash set instead)
  uint32_t *seen_bm;
  uint32_t seen_words;
  // warp-per-query kernel: shared-memory bytes per warp, and an upper bound
  // on |summary value| (fixes the fixed-point scale of the summary scores)
  uint32_t warp_bytes;
  float sum_absmax;
  uint32_t prefetch;  // rows of the next block prefetched into L2 (at most this many; 0 = off)
  const uint32_t *perm;  // persistent launches pull queries in this order (NULL: 0, 1, 2, ...)
  // graph refinement (CTA kernel): query q is document seed[q]; its lists are
  // not traversed, the heap is seeded with the document and its graph row, and
  // the kappa-NN expansion follows (NULL: ordinary search)
  const uint32_t *seed;
  // CTA kernel, group 1: documents are scored chunk by chunk by all threads
  // of the CTA (a wave's chunks laid end to end, then summed per document)
  uint32_t flat;
  // shared-memory layout
  uint32_t W, QN, BMAX, BPOW2, HS, CAND, CAPC;
  uint32_t off_qbits, off_qrank, off_qval, off_qterm, off_cut, off_aq, off_part, off_keys, off_clo, off_chi,
      off_hash, off_tk_s, off_tk_id, off_tmp_s, off_tmp_id, off_cand_s, off_cand_id, off_cand_ok,
      off_fdoc, off_fc0, off_fpre, off_cmap, off_bptr;
};

constexpr uint32_t kMaxWave = 64;  // blocks per wave (CTA kernel)
size_t search_layout(SearchArgs &a, uint32_t nw);
int launch_search(const SearchArgs &a, uint32_t group, uint32_t nw, size_t smem, uint32_t grid, cudaStream_t st);
int search_occupancy(uint32_t group, uint32_t nw, size_t smem, int *blocks);
size_t search_layout_warp(SearchArgs &a);
int launch_search_warp(const SearchArgs &a, uint32_t group, size_t smem, uint32_t grid, uint32_t wpb,
                       cudaStream_t st);
// One search call on a workspace (the C ABI's seismic_search, the server's
// streams); `seed` selects the graph-refinement mode above.
int search_ws(seismic_index *ix, Workspace *w, const seismic_csr *queries, const seismic_search_params *p,
              uint32_t *ids_out, float *scores_out, int32_t out_on_device, void *stream, uint64_t *stats,
              const uint32_t *seed = nullptr);
int search_occupancy_warp(uint32_t group, uint32_t k, size_t smem, uint32_t wpb, int *blocks);

struct ExactArgs {
  const uint32_t *full_ptr;
  const uint32_t *full_doc;
  const float *full_val;
  uint32_t n_docs;
  const uint64_t *q_indptr;
  const uint16_t *q_terms;
  const float *q_vals;
  uint32_t nq;
  uint32_t k;
  float *acc;  // gridDim.x * n_docs floats, all zero between queries
  uint32_t *ids;
  float *scores;
};
int launch_exact(const ExactArgs &a, uint32_t grid, cudaStream_t st);
constexpr uint32_t kExactMaxK = 1024;

// MLP and features
int launch_features(const uint64_t *q_indptr, const uint16_t *q_terms, const float *q_vals, uint32_t nq,
                    const uint32_t *list_ptr, const uint32_t *blk_ptr, uint32_t dim, float *feat, cudaStream_t st);
int launch_mlp_params(const float *w, const float *feat, uint32_t n, uint32_t cut_fallback, float hf_fallback,
                      uint32_t *q_cut, float *q_hf, cudaStream_t st);

}  // namespace seismic

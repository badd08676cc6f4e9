/*
 * seismic.h -- C ABI of a GB300 (sm_103a) implementation of Seismic, the
 * sparse maximum-inner-product search method of "Efficient Sketching and
 * Nearest Neighbor Search Algorithms for Sparse Vector Sets"
 * (arXiv 2509.24815).
 *
 * Problem (Definition "SMIPS", Section 2): for a collection S of sparse
 * vectors and a query q, return argmax^(k)_{u in S} <q, u>.  Seismic answers
 * it approximately with an inverted index whose lists are pruned (Set
 * alpha-MSS, Section 3.3), split into clustered blocks with sketched max
 * summaries (Section 4.1), a forward index (Section 4.2) and an optional
 * kappa-NN graph (Section 4.3); queries run Algorithm "Query processing with
 * Seismic" (Section 4.5).
 *
 * Conventions for every call:
 *   - Return value: SEISMIC_OK (0) or a negative SEISMIC_E* code.  On error
 *     seismic_last_error() gives a message (per calling thread) and no output
 *     buffer is guaranteed to hold anything meaningful.
 *   - Sparse inputs are CSR: row i holds terms[indptr[i] .. indptr[i+1]) and
 *     the matching vals.  Terms are strictly increasing within a row and
 *     < dim <= 65535; values are finite fp32.  An explicit 0.0 is not an
 *     entry of a sparse vector: build and search ignore it.
 *   - Results are ordered by (score desc, id asc).  A query with fewer than k
 *     candidates is padded with id SEISMIC_NONE_ID and score -INFINITY.
 *   - Host inputs are validated before any device work.  Device-resident
 *     inputs (on_device = 1) are trusted: the caller guarantees the format.
 *   - The library never keeps a pointer to a caller buffer after a call
 *     returns, and never frees one.
 *   - Scores are fp32, accumulated on the device in fp32.
 */
#ifndef SEISMIC_H
#define SEISMIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEISMIC_OK 0
#define SEISMIC_EINVAL (-1)   /* bad argument or malformed input */
#define SEISMIC_ENOMEM (-2)   /* host or device allocation failed */
#define SEISMIC_ECUDA (-3)    /* a CUDA runtime call failed */
#define SEISMIC_ETIMEOUT (-4) /* a bounded device-side wait gave up */
#define SEISMIC_EBUDGET (-5)  /* request larger than a configured budget */
#define SEISMIC_EIO (-6)      /* file missing, unreadable or of another format */

#define SEISMIC_NONE_ID 0xFFFFFFFFu

typedef struct seismic_index seismic_index; /* opaque; owns all its host and device memory */

/* A caller-owned, read-only CSR matrix (documents or queries). */
typedef struct {
  const uint64_t *indptr; /* n_rows + 1 offsets, indptr[0] = 0 */
  const uint16_t *terms;  /* indptr[n_rows] term ids */
  const float *vals;      /* indptr[n_rows] values */
  uint64_t n_rows;
  uint32_t dim;           /* vocabulary size d, <= 65535 */
  int32_t on_device;      /* 1: the three arrays are device pointers */
} seismic_csr;

/* Index construction (Algorithm "Indexing with Seismic", Section 4.4). */
typedef struct {
  uint32_t lambda;       /* keep the top-lambda postings of each list by value (Table 4's fixed
                            lambda); 0 keeps every posting */
  uint32_t beta;         /* clusters (blocks) per list: min(beta, |list|) (Section 4.1.2) */
  double alpha;          /* mass fraction of each block summary's alpha-MSS (the paper's gamma,
                            Section 4.1.3), in (0, 1] */
  int32_t quantize_u8;   /* 1: summary values as 8-bit codes with per-block (m, size) */
  uint64_t seed;         /* seed of the centroid sampling */
  double lambda_frac;    /* > 0: proportional Set alpha-MSS, lambda_t = ceil(lambda_frac * |L_t|)
                            (Definition "Set alpha-MSS"); overrides lambda */
  double beta_frac;      /* > 0: ceil(beta_frac * |list|) clusters per list; overrides beta */
  int32_t keep_full_lists; /* 1: also keep the unpruned lists for seismic_search_exact */
  int32_t threads;       /* host threads used by the build; 0 = all */
  int32_t keep_block_summaries; /* 1: also keep the block-major summary arrays (SEISMIC_X_SUM_*);
                                   search reads only the term-major copy */
  int32_t values_fp16;   /* 1: 16-bit forward values (the 16-bit setup of Section 5.4): every
                            document value is rounded to the nearest fp16 (ties to even) on
                            input, and the whole index -- lists, blocks, summaries, exact search --
                            is built from that rounded collection, so results equal those of an
                            fp32 index of the rounded values.  Rows shrink from 6 to 4 bytes per
                            entry.  A value beyond the fp16 range (|v| > 65504) is EINVAL; one that
                            rounds to 0 is dropped like an explicit zero */
} seismic_build_params;

/* Query processing (Algorithm "Query processing with Seismic", Section 4.5). */
typedef struct {
  uint32_t k;            /* results per query, 1..1024 */
  uint32_t cut;          /* traverse the lists of the query's top-`cut` terms by value */
  float heap_factor;     /* skip a block iff the top-k is full and r < heap_factor * theta
                            (hf_mode 0, the prose of Section 4.5) or r < theta / heap_factor
                            (hf_mode 1, the algorithm listing); theta = current k-th score */
  int32_t hf_mode;
  int32_t exhaustive;    /* 1: visit every block of the traversed lists (no skipping) */
  float alpha_q;         /* > 0: traverse the lists of the query's alpha_q-MSS instead of `cut` */
  int32_t use_knn;       /* 1: expand the top-k with the kappa-NN graph (needs a graph) */
  int32_t learned;       /* 1: per-query (cut, heap_factor) from the index's MLP; non-finite
                            predictions fall back to (cut, heap_factor) above */
  uint32_t wave;         /* blocks evaluated per threshold update; 1 (default) keeps the
                            sequential visiting order of the algorithm exactly */
  uint32_t group;        /* how documents are scored.  CTA shape: 1 = every thread of the CTA
                            takes row chunks of the whole wave (chunk-flattened; seen documents
                            are dropped before their rows are read), 8/16/32 = lane groups of
                            that width score one row each.  Warp shape: 4/8/16/32 lanes per
                            row.  0 = 1 on the CTA shape, 8 on the warp shape.  Scores differ
                            only in fp32 summation order */
  uint32_t cta_warps;    /* warps per CTA: 4, 8 or 16; 0 = 8 */
  uint32_t persistent;   /* 1: one persistent launch that pulls queries from a device queue */
  uint32_t max_query_nnz; /* device queries: an upper bound on any query's nonzeros, which sizes
                            shared memory; 0 = measure it (one device synchronisation, so not
                            inside stream capture).  Ignored for host queries. */
  uint32_t hash_slots;   /* per-query seen-set slots (power of two); 0 = 2048.  A full set only
                            costs repeated work, never a different result */
  uint32_t shape;        /* 0 or 1: one CTA per query (any k, any wave; the measured fastest);
                            2: one warp per query (k <= 128, wave 1, persistent, cta_warps
                            independent warps per CTA: 1/2/4, 0 = 4).  Both keep the
                            algorithm's sequential order at wave 1 */
  int32_t no_prefetch;   /* 1 turns off the L2 bulk prefetch of upcoming member lists and rows
                            (a speed knob; results are the same) */
  uint32_t order;        /* persistent launches: 0 (default) runs queries grouped by their
                            largest term, so queries reading the same lists share L2; 1 runs
                            them in input order; 2 runs the queries that traverse the most
                            lists first, grouped by largest term within each count, so the
                            queue ends on its cheapest queries.  Results do not depend on it */
} seismic_search_params;

/* Per-query work counters written by seismic_search when `stats` is non-NULL:
 * uint64_t stats[n_queries][SEISMIC_STATS_N].  The last two are device
 * timestamps (the GPU's global nanosecond timer), not counts: when the query's
 * CTA (or warp) took it up and when it wrote its results. */
enum {
  SEISMIC_ST_LISTS = 0,          /* posting lists traversed */
  SEISMIC_ST_BLOCKS_SCORED,      /* blocks whose summary was scored */
  SEISMIC_ST_BLOCKS_EVALUATED,   /* blocks whose documents were evaluated */
  SEISMIC_ST_BLOCKS_SKIPPED,     /* blocks skipped by the heap_factor test */
  SEISMIC_ST_DOCS,               /* forward rows scored in the list traversal */
  SEISMIC_ST_DOC_NNZ,            /* nonzeros of those rows */
  SEISMIC_ST_KNN_DOCS,           /* forward rows scored by the kappa-NN expansion */
  SEISMIC_ST_SUMMARY_ENTRIES,    /* summary column entries read */
  SEISMIC_ST_KNN_NNZ,            /* nonzeros of the expansion's rows */
  SEISMIC_ST_DIR_LOOKUPS,        /* summary directory entries read */
  SEISMIC_ST_BLOCK_DOCS,         /* block member ids read */
  SEISMIC_ST_QUERY_NNZ,          /* query entries read */
  SEISMIC_ST_T_START,            /* ns: the query was taken up */
  SEISMIC_ST_T_END,              /* ns: its results were written */
  SEISMIC_STATS_N
};

/* Facts about an index. */
typedef struct {
  uint64_t n_docs, nnz, n_postings, n_blocks, n_summary_entries;
  uint32_t dim, kappa;
  int32_t quantize_u8, has_full_lists, has_mlp;
  uint64_t device_bytes;  /* device memory held by the index */
  int32_t values_fp16;    /* the forward values are 16-bit */
  uint32_t knn_bits;      /* bits per stored kappa-NN id: floor(log2(n_docs - 1)) + 1 (Section 4.3),
                             one more when n_docs is a power of two (the missing-neighbour code) */
  uint64_t knn_bytes;     /* device bytes of the packed graph */
} seismic_index_info;

/* Builds an index from `docs` (host or device CSR) on the current CUDA
 * device.  The document ids of the index are the row numbers of `docs`.
 * Rows may hold at most 8192 nonzeros (the clustering kernel stages centroid
 * rows in shared memory).  Errors: EINVAL (bad params / malformed CSR / a
 * limit exceeded), ENOMEM, ECUDA.  *out is set only on success; free it with
 * seismic_free. */
int seismic_build(const seismic_csr *docs, const seismic_build_params *params, seismic_index **out);

/* Searches a batch of queries.  ids_out[n_queries * k], scores_out[n_queries
 * * k] are caller-owned, on the device when out_on_device = 1, else on the
 * host.  `stream` is a cudaStream_t (NULL = the legacy default stream); with
 * device inputs and outputs the call only enqueues work on it and returns
 * (the caller synchronises); otherwise it returns after the results are on
 * the host.  `stats` (host, may be NULL) receives SEISMIC_STATS_N counters
 * per query and forces a synchronisation.  Errors: EINVAL (bad params,
 * queries whose dim differs from the index, malformed host CSR), ENOMEM,
 * ECUDA, ETIMEOUT (the persistent kernel's bounded queue wait). */
int seismic_search(seismic_index *index, const seismic_csr *queries, const seismic_search_params *params,
                   uint32_t *ids_out, float *scores_out, int32_t out_on_device, void *stream,
                   uint64_t *stats);

/* Exact top-k (Definition SMIPS) by term-at-a-time accumulation over the
 * unpruned lists; needs an index built with keep_full_lists = 1.  Scores are
 * fp32 sums in ascending query-term order.  Documents sharing no term with a
 * query score 0 and fill the result in ascending id order.  Used as the
 * recall judge.  Same buffer and stream rules as seismic_search. */
int seismic_search_exact(seismic_index *index, const seismic_csr *queries, uint32_t k, uint32_t *ids_out,
                         float *scores_out, int32_t out_on_device, void *stream);

/* Installs a kappa-NN graph (Eq. "knn-graph", Section 4.3): nbrs[n_docs *
 * kappa] row-major, SEISMIC_NONE_ID for missing neighbours; host or device.
 * The index stores each id in floor(log2(n_docs - 1)) + 1 bits, the cost the
 * paper gives for the graph (Section 4.3), packed back to back (one bit more
 * when n_docs is a power of two, to leave a code for a missing neighbour).
 * Replaces any previous graph.  Errors: EINVAL (size mismatch, id out of
 * range), ENOMEM, ECUDA. */
int seismic_set_knn(seismic_index *index, const uint32_t *nbrs, uint64_t n_docs, uint32_t kappa,
                    int32_t on_device);

/* Builds the kappa-NN graph approximately, as the paper does (Section 5.3:
 * each document is searched with Seismic itself, without the graph), using
 * `params` for those searches and k = kappa + 1 (the document itself is
 * removed).  Synchronous. */
int seismic_build_knn(seismic_index *index, uint32_t kappa, const seismic_search_params *params);

/* Improves the installed graph by `rounds` neighbour-of-neighbour passes (not
 * a step of the paper: its Section 4.3 builds the graph approximately with
 * Seismic itself, and a pass applies Seismic's expansion step -- the union of
 * the neighbour lists of a set -- to the graph): in a round every document u
 * is scored exactly against the documents of N(u) and of N(v) for v in N(u),
 * and N(u) becomes the kappa best of them other than u, by (score desc, id
 * asc).  A round reads only the graph from before it, so a row never gets
 * worse and the exact graph is a fixed point.  `params` (may be NULL) only
 * chooses the launch configuration (group, cta_warps, no_prefetch); the rest
 * is fixed.  Synchronous.  Errors: EINVAL (no graph), ENOMEM, ECUDA. */
int seismic_refine_knn(seismic_index *index, uint32_t rounds, const seismic_search_params *params);

/* Copies the graph to the host, unpacked: nbrs[n_docs * kappa]. */
int seismic_get_knn(const seismic_index *index, uint32_t *nbrs, uint64_t cap_entries);

/* Versioned little-endian file of the whole index (and graph and MLP).
 * Errors: EIO, ENOMEM, ECUDA. */
int seismic_save(const seismic_index *index, const char *path);
int seismic_load(const char *path, seismic_index **out);

int seismic_info(const seismic_index *index, seismic_index_info *out);

/* Copies one internal array to host memory for inspection (tests, tools):
 * `what` is a SEISMIC_X_* id.  If dst is NULL or cap_bytes is too small,
 * only *needed_bytes is written.  Errors: EINVAL (unknown id). */
enum {
  SEISMIC_X_LIST_PTR = 0,   /* uint32[dim+1]: postings of term t, after pruning */
  SEISMIC_X_LIST_DOC,       /* uint32[n_postings]: by (value desc, doc asc) per list */
  SEISMIC_X_BLK_PTR,        /* uint32[dim+1]: blocks of list t */
  SEISMIC_X_BDOC_PTR,       /* uint32[n_blocks+1]: member ids of block g */
  SEISMIC_X_BDOC,           /* uint32[n_postings]: members, ascending per block */
  SEISMIC_X_BLK_M,          /* float[n_blocks]: quantisation minimum m */
  SEISMIC_X_BLK_SIZE,       /* float[n_blocks]: quantisation sub-interval size */
  SEISMIC_X_SUM_PTR,        /* uint32[n_blocks+1]: block-major summary entries (SUM_* need
                               keep_block_summaries = 1) */
  SEISMIC_X_SUM_TERM,       /* uint16[n_summary_entries]: ascending per block */
  SEISMIC_X_SUM_VAL,        /* float[n_summary_entries]: max-summary values */
  SEISMIC_X_SUM_CODE,       /* uint8[n_summary_entries]: 8-bit codes */
  SEISMIC_X_CENT,           /* uint32[n_postings]: per list position, assigned cluster index */
  /* the term-major summaries the search reads (always kept) */
  SEISMIC_X_SBM,            /* uint32[dim * W * 2], W = ceil(dim / 32): per list t and 32-term word w,
                               the presence bits of t's summary terms, then the index of the word's
                               first column */
  SEISMIC_X_SCPTR,          /* uint32[columns + dim]: column pointers into SCOL_*; each list's
                               pointers end with a sentinel */
  SEISMIC_X_SCOL_BLK,       /* uint16[n_summary_entries]: block (index within its list), ascending
                               within a column */
  SEISMIC_X_SCOL_CODE,      /* uint8[n_summary_entries]: 8-bit codes (quantised indexes) */
  SEISMIC_X_SCOL_VAL,       /* float[n_summary_entries]: values (fp32 summaries) */
  SEISMIC_X_N
};
int seismic_export(const seismic_index *index, int32_t what, void *dst, uint64_t cap_bytes,
                   uint64_t *needed_bytes);

/* Per-query parameter model (not in the paper): an MLP 64 -> 128 -> 64 -> 2
 * with fp32 weights and bf16 activations that maps query features to
 * (cut, heap_factor) = (clamp(round(3 + 27 * sigmoid(o0)), 3, 30),
 * 0.5 + 0.5 * sigmoid(o1)).  Weights: W1[128][64], b1[128], W2[64][128],
 * b2[64], W3[2][64], b3[2], packed in that order (SEISMIC_MLP_PARAMS floats). */
#define SEISMIC_MLP_IN 64
#define SEISMIC_MLP_H1 128
#define SEISMIC_MLP_H2 64
#define SEISMIC_MLP_PARAMS (128 * 64 + 128 + 64 * 128 + 64 + 2 * 64 + 2)
int seismic_set_mlp(seismic_index *index, const float *weights, uint64_t n_floats);

/* Query features for the MLP, fp32 [n_queries][64]: log(1 + nnz(q)); the 16
 * largest query values (descending, 0-padded); log(1 + |pruned list|) of
 * those 16 terms; log(1 + blocks) of those terms; the query's L1 and L2
 * norms; 13 zeros.  `features` is caller-owned (device when on_device = 1).
 * Synchronous. */
int seismic_query_features(seismic_index *index, const seismic_csr *queries, float *features,
                           int32_t on_device, void *stream);

/* MLP forward pass on device buffers: weights[SEISMIC_MLP_PARAMS],
 * features[n][64] -> out[n][2] raw outputs (o0, o1); ReLU hidden layers,
 * activations rounded to bf16.  Enqueued on `stream`. */
int seismic_mlp_forward(const float *weights, const float *features, uint64_t n, float *out, void *stream);

/* One Adam step of the MLP on device buffers: loss = mean over rows of
 * (sigmoid(o0) - t0)^2 + (sigmoid(o1) - t1)^2 with targets t[n][2] in [0, 1].
 * weights, grads, m, v hold SEISMIC_MLP_PARAMS floats each; loss_out (device,
 * 1 float) receives the mean loss before the step.  grads receives the
 * gradient.  `step` is the 1-based Adam step number. */
int seismic_mlp_train_step(float *weights, float *grads, float *adam_m, float *adam_v,
                           const float *features, const float *targets, uint64_t n, float lr,
                           uint32_t step, float *loss_out, void *stream);

/* Continuous-batching server (not in the paper, whose queries run one at a
 * time on one CPU thread).  Requests queue on the host; progress() reaps
 * finished batches and admits waiting requests as soon as a stream and device
 * slots are free, so requests that arrive while others run start without
 * waiting for them, and their work overlaps on the GPU.  Each stream has its
 * own workspace and pinned staging buffers; the index is shared read-only, so
 * a request's result is the same alone and in the mix. */
typedef struct seismic_server seismic_server;
typedef struct {
  uint32_t max_batch;     /* requests per launch; 0 = 256 */
  uint32_t streams;       /* batches in flight at once (1..64); 0 = 4 */
  uint32_t max_query_nnz; /* admission: longer requests are refused; 0 = 1024 */
  uint32_t slot_budget;   /* admission: requests on the device at once; 0 = what the search kernel's
                             shared memory per query (query, block scores, a 100-entry heap) lets
                             stay resident: CTAs per SM x SMs */
} seismic_server_params;

/* Creates a server over `index` (which must outlive it).  `search` fixes the
 * search parameters (its k is replaced per request); every stream's workspace
 * is sized by one warm-up batch, so serving does not allocate device memory.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int seismic_server_create(seismic_index *index, const seismic_search_params *search,
                          const seismic_server_params *params, seismic_server **out);
/* Queues one host query (ascending terms) for top-k; `ticket` identifies it.
 * The arrival time is now.  Errors: EINVAL (malformed, too long). */
int seismic_server_submit(seismic_server *srv, const uint16_t *terms, const float *vals, uint32_t nnz, uint32_t k,
                          uint64_t *ticket);
/* Non-blocking: reaps finished batches, launches admitted ones.  `completed`
 * (may be NULL) receives how many requests finished in this call. */
int seismic_server_progress(seismic_server *srv, uint32_t *completed);
/* If the request is done (*done = 1): copies its k ids/scores (caller-owned
 * host buffers, may be NULL), its arrival-to-completion latency in
 * microseconds, and forgets it.  Otherwise *done = 0.  EINVAL: unknown ticket. */
int seismic_server_result(seismic_server *srv, uint64_t ticket, uint32_t *ids, float *scores, double *latency_us,
                          int32_t *done);
/* Replays an arrival trace in a tight host loop: query i (host CSR row i)
 * arrives arrival_s[i] seconds after the start (non-decreasing) asking for
 * top-k_per_query[i]; results go to ids_out/scores_out[n * k_stride] (rows
 * padded past their k), latencies to latency_us[n] (from the scheduled
 * arrival), the elapsed time to *wall_s (may be NULL). */
int seismic_server_replay(seismic_server *srv, const seismic_csr *queries, const double *arrival_s,
                          const uint32_t *k_per_query, uint32_t k_stride, uint32_t *ids_out, float *scores_out,
                          double *latency_us, double *wall_s);
void seismic_server_destroy(seismic_server *srv);

/* Query processing that allocates no memory (this entry point has no
 * counterpart in the paper; it is for callers that cannot allocate device
 * memory while they serve queries: a process whose memory pool is fixed at
 * start-up, or one that keeps cudaMalloc's device synchronisation off its
 * latency path).  It runs the same CTA-per-query persistent kernel as
 * seismic_search with the same results, and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   - queries, ids_out and scores_out must be device buffers; params must set
 *     max_query_nnz.  Not available here: stats, learned parameters, the
 *     warp-per-query shape (shape = 2 is refused with EINVAL), work-queue
 *     ordering (`order` is ignored: queries run in input order, with the same
 *     results) and `hash_slots` (ignored: the seen set is the bitmap in the
 *     fixed array).
 *   - Working memory is one fixed 32 MiB device array inside the library,
 *     held by every GPU that loads it until the process exits: a 256-byte
 *     header (queue counter, error word, cleared on `stream` at each call)
 *     and one seen bitmap of ceil(n_docs / 32) words per persistent CTA.  The
 *     number of CTAs is capped by what fits; an index whose single bitmap does
 *     not fit (more than about 268 million documents) gets SEISMIC_EBUDGET.
 *   - The first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress, with that device current) and caches it: make
 *     that first call before any stream capture.
 *   - Every call shares the array and enqueues its work on `stream` without
 *     waiting: calls that overlap on the GPU (other streams, other threads,
 *     other indexes on the same device) race on it.  Serialise them.
 *   - A malformed device query (more nonzeros than max_query_nnz) yields a
 *     padded row, as in seismic_search's device path.
 * Errors: EINVAL (arguments), EBUDGET (collection too large for the fixed
 * array), ECUDA. */
int seismic_search_noalloc(seismic_index *index, const seismic_csr *queries, const seismic_search_params *params,
                           uint32_t *ids_out, float *scores_out, void *stream);

void seismic_free(seismic_index *index);
const char *seismic_last_error(void);
const char *seismic_version(void);

#ifdef __cplusplus
}
#endif
#endif

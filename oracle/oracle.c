/*
 * ORACLE -- test infrastructure only.  A plain, slow, fp64 CPU statement of
 * what the Seismic method computes, written from the paper
 * (arXiv 2509.24815, "Efficient Sketching and Nearest Neighbor Search
 * Algorithms for Sparse Vector Sets").  Only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code with
 * the GPU library.
 *
 * Contents (each cites the passage it follows):
 *   or_exact_topk   -- Definition "SMIPS" (Section 2): argmax^(k) <q,u>.
 *   or_alpha_mss    -- Definition "alpha-mass subvector sketch" (Section 3.2).
 *   or_build        -- Algorithm "Indexing with Seismic" (Section 4.4):
 *                      Set alpha-MSS lists (Def. "Set alpha-MSS", Section 3.3,
 *                      fixed-lambda form of Table 4), shallow k-means blocking
 *                      (Section 4.1.2), max summaries (Eq. "summary"),
 *                      gamma-MSS of the summary and 8-bit scalar quantisation
 *                      (Section 4.1.3).
 *   or_knn_exact    -- Eq. "knn-graph" (Section 4.3), computed exactly.
 *   or_knn_refine   -- one neighbour-of-neighbour pass over a graph: the
 *                      expansion step of Section 4.5 applied to N(u) itself.
 *   or_search       -- Algorithm "Query processing with Seismic" (Section 4.5).
 *
 * Readings where the paper is silent or inconsistent (all listed in the
 * design notes):
 *   - total order on results: score descending, then id ascending; the heap
 *     admits (p, d) iff it is not full or (p, d) beats the current k-th;
 *   - lists keep min(lambda, |L_t|) entries by (value desc, doc asc);
 *   - nb = min(beta, |L'_t|) centroids, drawn by a partial Fisher-Yates
 *     shuffle driven by splitmix64 seeded with seed ^ (t * 0x9E3779B97F4A7C15);
 *     assignment by argmax of the fp64 inner product of full vectors, summed
 *     in ascending term order, ties to the lower centroid index; empty
 *     clusters dropped; members ascending;
 *   - alpha-MSS order: |value| desc, term asc; prefix mass in fp64;
 *   - quantisation: m = min, size = fp32((max - m) / 256),
 *     code = min(255, floor((v - m) / size)), v^ = m + code * size;
 *   - skip test: |H| = k and r < hf * theta (prose of Section 4.5); the
 *     algorithm listing's r < theta / hf is hf_mode 1;
 *   - each document is evaluated at most once per query (a seen set);
 *   - lists are traversed in query-value order (desc, term asc).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NONE_ID 0xFFFFFFFFu

typedef struct {
  const uint64_t *indptr;
  const uint16_t *terms;
  const float *vals;
  uint64_t n;
  uint32_t d;
} csr_t;

/* ------------------------------------------------------------------ */
/* parallel for over [0, n) with a shared counter                       */
typedef struct {
  void (*fn)(void *, int64_t, int);
  void *ctx;
  int64_t n, next;
  int tid_next;
} pf_t;

static void *pf_worker(void *arg) {
  pf_t *p = (pf_t *)arg;
  int tid = __atomic_fetch_add(&p->tid_next, 1, __ATOMIC_SEQ_CST);
  for (;;) {
    int64_t i = __atomic_fetch_add(&p->next, 1, __ATOMIC_SEQ_CST);
    if (i >= p->n) break;
    p->fn(p->ctx, i, tid);
  }
  return NULL;
}

static void pfor(int64_t n, int threads, void (*fn)(void *, int64_t, int), void *ctx) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  pf_t p = {fn, ctx, n, 0, 0};
  pthread_t th[256];
  for (int i = 0; i < threads; i++) pthread_create(&th[i], NULL, pf_worker, &p);
  for (int i = 0; i < threads; i++) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------ */
/* top-k under the total order (score desc, id asc)                      */
typedef struct {
  double s;
  uint32_t id;
} ent_t;

static int better(double s1, uint32_t i1, double s2, uint32_t i2) {
  return s1 > s2 || (s1 == s2 && i1 < i2);
}

typedef struct {
  ent_t *e; /* e[0] best ... e[n-1] worst = the heap minimum */
  uint32_t n, k;
} topk_t;

/* The heap of the paper: insert when not full or when (s, id) beats the
 * minimum; when it would hold k+1 entries, drop the minimum. */
static void offer(topk_t *h, double s, uint32_t id) {
  if (h->k == 0) return;
  if (h->n == h->k) {
    if (!better(s, id, h->e[h->n - 1].s, h->e[h->n - 1].id)) return;
    h->n--;
  }
  uint32_t i = h->n;
  while (i > 0 && better(s, id, h->e[i - 1].s, h->e[i - 1].id)) { h->e[i] = h->e[i - 1]; i--; }
  h->e[i].s = s;
  h->e[i].id = id;
  h->n++;
}

static void emit(const topk_t *h, uint32_t *ids, double *scores) {
  for (uint32_t i = 0; i < h->k; i++) {
    if (i < h->n) { ids[i] = h->e[i].id; scores[i] = h->e[i].s; }
    else { ids[i] = NONE_ID; scores[i] = -INFINITY; }
  }
}

/* ------------------------------------------------------------------ */
/* full inverted lists: for term t, (doc, value) in ascending doc order  */
typedef struct {
  uint64_t *ptr; /* d + 1 */
  uint32_t *doc;
  float *val;
} inv_t;

static void transpose(const csr_t *D, inv_t *L) {
  uint64_t nnz = D->indptr[D->n];
  L->ptr = (uint64_t *)calloc((size_t)D->d + 1, sizeof(uint64_t));
  L->doc = (uint32_t *)malloc(sizeof(uint32_t) * (nnz ? nnz : 1));
  L->val = (float *)malloc(sizeof(float) * (nnz ? nnz : 1));
  for (uint64_t i = 0; i < nnz; i++) L->ptr[D->terms[i] + 1]++;
  for (uint32_t t = 0; t < D->d; t++) L->ptr[t + 1] += L->ptr[t];
  uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)D->d + 1));
  memcpy(cur, L->ptr, sizeof(uint64_t) * ((size_t)D->d + 1));
  for (uint64_t j = 0; j < D->n; j++)
    for (uint64_t p = D->indptr[j]; p < D->indptr[j + 1]; p++) {
      uint64_t o = cur[D->terms[p]]++;
      L->doc[o] = (uint32_t)j;
      L->val[o] = D->vals[p];
    }
  free(cur);
}

static void inv_free(inv_t *L) { free(L->ptr); free(L->doc); free(L->val); }

/* ------------------------------------------------------------------ */
/* Exact top-k (Definition SMIPS).  Scores are fp64 sums of the exact fp64
 * products of the fp32 inputs, accumulated term-at-a-time in ascending
 * query-term order.  Every document is a candidate: one that shares no term
 * with q scores exactly 0. */
typedef struct {
  const csr_t *D, *Q;
  const inv_t *L;
  uint32_t k;
  uint32_t *ids;
  double *scores;
  double **acc;
  uint32_t **stamp;
  ent_t **heap;
} ex_ctx;

static void exact_one(void *vc, int64_t qi, int tid) {
  ex_ctx *c = (ex_ctx *)vc;
  const csr_t *Q = c->Q;
  double *acc = c->acc[tid];
  uint32_t *st = c->stamp[tid];
  uint32_t mark = (uint32_t)qi + 1;
  topk_t h = {c->heap[tid], 0, c->k};
  for (uint64_t p = Q->indptr[qi]; p < Q->indptr[qi + 1]; p++) {
    uint16_t t = Q->terms[p];
    double qv = (double)Q->vals[p];
    for (uint64_t e = c->L->ptr[t]; e < c->L->ptr[t + 1]; e++) {
      uint32_t dd = c->L->doc[e];
      if (st[dd] != mark) { st[dd] = mark; acc[dd] = 0.0; }
      acc[dd] += qv * (double)c->L->val[e];
    }
  }
  for (uint64_t p = Q->indptr[qi]; p < Q->indptr[qi + 1]; p++) {
    uint16_t t = Q->terms[p];
    for (uint64_t e = c->L->ptr[t]; e < c->L->ptr[t + 1]; e++) {
      uint32_t dd = c->L->doc[e];
      if (st[dd] == mark) { offer(&h, acc[dd], dd); st[dd] = mark ^ 0x80000000u; }
    }
  }
  /* untouched documents score 0: ascending ids while they can still enter */
  for (uint64_t dd = 0; dd < c->D->n; dd++) {
    if (h.n == h.k && !better(0.0, (uint32_t)dd, h.e[h.n - 1].s, h.e[h.n - 1].id)) break;
    if (st[dd] != (mark ^ 0x80000000u)) offer(&h, 0.0, (uint32_t)dd);
  }
  emit(&h, c->ids + (uint64_t)qi * c->k, c->scores + (uint64_t)qi * c->k);
}

static csr_t mk(const uint64_t *ip, const uint16_t *t, const float *v, uint64_t n, uint32_t d) {
  csr_t c = {ip, t, v, n, d};
  return c;
}

int or_exact_topk(const uint64_t *dip, const uint16_t *dt, const float *dv, uint64_t nd, uint32_t d,
                  const uint64_t *qip, const uint16_t *qt, const float *qv, uint64_t nq, uint32_t k,
                  int threads, uint32_t *ids, double *scores) {
  csr_t D = mk(dip, dt, dv, nd, d), Q = mk(qip, qt, qv, nq, d);
  inv_t L;
  transpose(&D, &L);
  if (threads < 1) threads = 1;
  ex_ctx c = {&D, &Q, &L, k, ids, scores, NULL, NULL, NULL};
  c.acc = (double **)calloc(threads, sizeof(double *));
  c.stamp = (uint32_t **)calloc(threads, sizeof(uint32_t *));
  c.heap = (ent_t **)calloc(threads, sizeof(ent_t *));
  for (int i = 0; i < threads; i++) {
    c.acc[i] = (double *)malloc(sizeof(double) * (nd ? nd : 1));
    c.stamp[i] = (uint32_t *)calloc(nd ? nd : 1, sizeof(uint32_t));
    c.heap[i] = (ent_t *)malloc(sizeof(ent_t) * (k + 1));
  }
  pfor((int64_t)nq, threads, exact_one, &c);
  for (int i = 0; i < threads; i++) { free(c.acc[i]); free(c.stamp[i]); free(c.heap[i]); }
  free(c.acc); free(c.stamp); free(c.heap);
  inv_free(&L);
  return 0;
}

/* ------------------------------------------------------------------ */
/* alpha-mass subvector sketch (Definition alpha-MSS): order the entries by
 * |value| descending (ties: term ascending), keep the shortest prefix whose
 * fp64 mass reaches alpha * ||u||_1, where ||u||_1 is that same sum taken in
 * the same order.  Returns the number kept; `order` receives entry indices in
 * sketch order. */
typedef struct {
  float a;
  uint16_t t;
  uint32_t i;
} mss_t;

static int mss_cmp(const void *x, const void *y) {
  const mss_t *p = (const mss_t *)x, *q = (const mss_t *)y;
  if (p->a > q->a) return -1;
  if (p->a < q->a) return 1;
  return (p->t > q->t) - (p->t < q->t);
}

static uint32_t alpha_mss(const uint16_t *terms, const float *vals, uint32_t n, double alpha,
                          mss_t *buf) {
  for (uint32_t i = 0; i < n; i++) { buf[i].a = fabsf(vals[i]); buf[i].t = terms[i]; buf[i].i = i; }
  qsort(buf, n, sizeof(mss_t), mss_cmp);
  double total = 0.0;
  for (uint32_t i = 0; i < n; i++) total += (double)buf[i].a;
  double target = alpha * total, c = 0.0;
  for (uint32_t i = 0; i < n; i++) {
    c += (double)buf[i].a;
    if (c >= target) return i + 1;
  }
  return n;
}

uint32_t or_alpha_mss(const uint16_t *terms, const float *vals, uint32_t n, double alpha,
                      uint32_t *order_out) {
  mss_t *buf = (mss_t *)malloc(sizeof(mss_t) * (n ? n : 1));
  uint32_t keep = alpha_mss(terms, vals, n, alpha, buf);
  for (uint32_t i = 0; i < n; i++) order_out[i] = buf[i].i;
  free(buf);
  return keep;
}

/* ------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea, Flood 2014; Vigna's public-domain C statement) */
static uint64_t splitmix64_next(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t or_splitmix64(uint64_t *state) { return splitmix64_next(state); }

/* ------------------------------------------------------------------ */
/* Index (Algorithm "Indexing with Seismic").                             */
typedef struct {
  /* list t: pruned postings in (value desc, doc asc) order */
  uint32_t n; /* |L'_t| */
  uint32_t *doc;
  float *val;
  uint32_t ncent;    /* nb */
  uint32_t *cent;    /* centroid docs, c = 0..nb-1 */
  uint32_t *assign;  /* per list position: centroid index */
  uint32_t nblk;     /* non-empty clusters */
  uint32_t *bcent;   /* per block: centroid index */
  uint32_t *bptr;    /* nblk + 1 */
  uint32_t *bmem;    /* members, ascending within a block */
  uint32_t *sptr;    /* nblk + 1: kept summary entries */
  uint16_t *sterm;   /* ascending within a block */
  float *sval;       /* the max-summary value phi_i */
  uint8_t *scode;
  float *qm, *qsz;   /* per block */
} olist_t;

typedef struct {
  uint32_t d;
  uint64_t n;
  int quantize;
  olist_t *lists; /* d */
} or_index;

typedef struct {
  const csr_t *D;
  const inv_t *L;
  or_index *X;
  const uint8_t *mask; /* NULL: every list; else build list t only where mask[t] */
  uint32_t lambda, beta;
  double lambda_frac, beta_frac, alpha;
  uint64_t seed;
  double **dense;
  float **mx;
  uint32_t **cnt;
  uint16_t **touched;
  mss_t **mss;
} bd_ctx;

typedef struct {
  float v;
  uint32_t doc;
} post_t;

static int post_cmp(const void *x, const void *y) {
  const post_t *a = (const post_t *)x, *b = (const post_t *)y;
  if (a->v > b->v) return -1;
  if (a->v < b->v) return 1;
  return (a->doc > b->doc) - (a->doc < b->doc);
}

static int u32_cmp(const void *x, const void *y) {
  uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
  return (a > b) - (a < b);
}

static int u16_cmp_by_term(const void *x, const void *y) {
  const mss_t *a = (const mss_t *)x, *b = (const mss_t *)y;
  return (a->t > b->t) - (a->t < b->t);
}

static void build_list(void *vc, int64_t ti, int tid) {
  bd_ctx *c = (bd_ctx *)vc;
  const csr_t *D = c->D;
  uint32_t t = (uint32_t)ti;
  olist_t *o = &c->X->lists[t];
  memset(o, 0, sizeof(*o));
  if (c->mask && !c->mask[t]) return;
  uint64_t a = c->L->ptr[t], b = c->L->ptr[t + 1];
  uint32_t full = (uint32_t)(b - a);
  if (full == 0) return;

  /* Set alpha-MSS, column-wise: keep the lambda_t largest values. */
  post_t *pp = (post_t *)malloc(sizeof(post_t) * full);
  for (uint32_t i = 0; i < full; i++) { pp[i].v = c->L->val[a + i]; pp[i].doc = c->L->doc[a + i]; }
  qsort(pp, full, sizeof(post_t), post_cmp);
  uint32_t lam;
  if (c->lambda_frac > 0.0) lam = (uint32_t)ceil(c->lambda_frac * (double)full);
  else lam = c->lambda ? c->lambda : full;
  if (lam > full) lam = full;
  o->n = lam;
  o->doc = (uint32_t *)malloc(sizeof(uint32_t) * lam);
  o->val = (float *)malloc(sizeof(float) * lam);
  for (uint32_t i = 0; i < lam; i++) { o->doc[i] = pp[i].doc; o->val[i] = pp[i].v; }
  free(pp);
  uint32_t n = lam;
  if (n == 0) return;

  /* Shallow k-means: nb centroids sampled uniformly without replacement. */
  uint32_t nb;
  if (c->beta_frac > 0.0) nb = (uint32_t)ceil(c->beta_frac * (double)n);
  else nb = c->beta;
  if (nb > n) nb = n;
  if (nb < 1) nb = 1;
  uint32_t *pos = (uint32_t *)malloc(sizeof(uint32_t) * n);
  for (uint32_t i = 0; i < n; i++) pos[i] = i;
  uint64_t st = c->seed ^ ((uint64_t)t * 0x9E3779B97F4A7C15ULL);
  for (uint32_t i = 0; i < nb; i++) {
    uint32_t j = i + (uint32_t)(splitmix64_next(&st) % (uint64_t)(n - i));
    uint32_t tmp = pos[i]; pos[i] = pos[j]; pos[j] = tmp;
  }
  o->ncent = nb;
  o->cent = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  for (uint32_t i = 0; i < nb; i++) o->cent[i] = o->doc[pos[i]];
  free(pos);

  /* Assign each list member to argmax_c <u_j, mu_c> over the full vectors.
   * The centroid is scattered into a dense fp64 vector; the dot then runs
   * over the document's terms in ascending order, so it adds exactly the
   * nonzero products of the two vectors' common terms in ascending term
   * order (the other products are zeros and leave the sum unchanged). */
  double *dense = c->dense[tid];
  double *best = (double *)malloc(sizeof(double) * n);
  o->assign = (uint32_t *)malloc(sizeof(uint32_t) * n);
  for (uint32_t ci = 0; ci < nb; ci++) {
    uint32_t cd = o->cent[ci];
    for (uint64_t p = D->indptr[cd]; p < D->indptr[cd + 1]; p++) dense[D->terms[p]] = (double)D->vals[p];
    for (uint32_t i = 0; i < n; i++) {
      uint32_t j = o->doc[i];
      double s = 0.0;
      for (uint64_t p = D->indptr[j]; p < D->indptr[j + 1]; p++) s += dense[D->terms[p]] * (double)D->vals[p];
      if (ci == 0 || s > best[i]) { best[i] = s; o->assign[i] = ci; }
    }
    for (uint64_t p = D->indptr[cd]; p < D->indptr[cd + 1]; p++) dense[D->terms[p]] = 0.0;
  }
  free(best);

  /* Blocks: one per non-empty cluster, in centroid order; members ascending. */
  uint32_t *csize = (uint32_t *)calloc(nb, sizeof(uint32_t));
  for (uint32_t i = 0; i < n; i++) csize[o->assign[i]]++;
  uint32_t nblk = 0;
  for (uint32_t ci = 0; ci < nb; ci++) nblk += csize[ci] > 0;
  o->nblk = nblk;
  o->bcent = (uint32_t *)malloc(sizeof(uint32_t) * nblk);
  o->bptr = (uint32_t *)malloc(sizeof(uint32_t) * (nblk + 1));
  o->bmem = (uint32_t *)malloc(sizeof(uint32_t) * n);
  uint32_t *bstart = (uint32_t *)malloc(sizeof(uint32_t) * nb);
  uint32_t bi = 0, off = 0;
  for (uint32_t ci = 0; ci < nb; ci++) {
    if (!csize[ci]) continue;
    o->bcent[bi] = ci;
    o->bptr[bi] = off;
    bstart[ci] = off;
    off += csize[ci];
    bi++;
  }
  o->bptr[nblk] = off;
  for (uint32_t i = 0; i < n; i++) o->bmem[bstart[o->assign[i]]++] = o->doc[i];
  for (uint32_t b2 = 0; b2 < nblk; b2++)
    qsort(o->bmem + o->bptr[b2], o->bptr[b2 + 1] - o->bptr[b2], sizeof(uint32_t), u32_cmp);
  free(bstart);
  free(csize);

  /* Summaries: phi(B)_i = max over members of u_i (absent coordinates are 0),
   * then the alpha-MSS of phi, then optional 8-bit scalar quantisation. */
  float *mx = c->mx[tid];
  uint32_t *cnt = c->cnt[tid];
  uint16_t *touched = c->touched[tid];
  mss_t *ms = c->mss[tid];
  uint32_t cap = 1024, used = 0;
  o->sptr = (uint32_t *)malloc(sizeof(uint32_t) * (nblk + 1));
  o->sterm = (uint16_t *)malloc(sizeof(uint16_t) * cap);
  o->sval = (float *)malloc(sizeof(float) * cap);
  o->scode = (uint8_t *)malloc(cap);
  o->qm = (float *)malloc(sizeof(float) * nblk);
  o->qsz = (float *)malloc(sizeof(float) * nblk);
  uint16_t *et = (uint16_t *)malloc(sizeof(uint16_t) * D->d);
  float *ev = (float *)malloc(sizeof(float) * D->d);
  for (uint32_t b2 = 0; b2 < nblk; b2++) {
    uint32_t bs = o->bptr[b2 + 1] - o->bptr[b2], nt = 0;
    for (uint32_t m = o->bptr[b2]; m < o->bptr[b2 + 1]; m++) {
      uint32_t j = o->bmem[m];
      for (uint64_t p = D->indptr[j]; p < D->indptr[j + 1]; p++) {
        uint16_t tt = D->terms[p];
        float v = D->vals[p];
        if (cnt[tt] == 0) { touched[nt++] = tt; mx[tt] = v; }
        else if (v > mx[tt]) mx[tt] = v;
        cnt[tt]++;
      }
    }
    uint32_t ne = 0;
    for (uint32_t i = 0; i < nt; i++) {
      uint16_t tt = touched[i];
      float phi = mx[tt];
      if (cnt[tt] < bs && phi < 0.0f) phi = 0.0f;
      cnt[tt] = 0;
      if (phi != 0.0f) { et[ne] = tt; ev[ne] = phi; ne++; }
    }
    uint32_t keep = alpha_mss(et, ev, ne, c->alpha, ms);
    qsort(ms, keep, sizeof(mss_t), u16_cmp_by_term);
    if (used + keep > cap) {
      while (used + keep > cap) cap *= 2;
      o->sterm = (uint16_t *)realloc(o->sterm, sizeof(uint16_t) * cap);
      o->sval = (float *)realloc(o->sval, sizeof(float) * cap);
      o->scode = (uint8_t *)realloc(o->scode, cap);
    }
    o->sptr[b2] = used;
    float lo = INFINITY, hi = -INFINITY;
    for (uint32_t i = 0; i < keep; i++) {
      float v = ev[ms[i].i];
      o->sterm[used + i] = ms[i].t;
      o->sval[used + i] = v;
      if (v < lo) lo = v;
      if (v > hi) hi = v;
    }
    if (keep == 0) { lo = 0.0f; hi = 0.0f; }
    float size = (float)(((double)hi - (double)lo) / 256.0);
    o->qm[b2] = lo;
    o->qsz[b2] = size;
    for (uint32_t i = 0; i < keep; i++) {
      double q = size > 0.0f ? floor(((double)o->sval[used + i] - (double)lo) / (double)size) : 0.0;
      if (q > 255.0) q = 255.0;
      if (q < 0.0) q = 0.0;
      o->scode[used + i] = (uint8_t)q;
    }
    used += keep;
  }
  o->sptr[nblk] = used;
  free(et);
  free(ev);
}

/* Builds the index; with a non-NULL term_mask only the lists of the marked
 * terms are built (the others stay empty), which is enough to run queries
 * whose traversed lists are all marked. */
or_index *or_build_masked(const uint64_t *dip, const uint16_t *dt, const float *dv, uint64_t nd, uint32_t d,
                          uint32_t lambda, double lambda_frac, uint32_t beta, double beta_frac, double alpha,
                          int quantize, uint64_t seed, int threads, const uint8_t *term_mask) {
  csr_t D = mk(dip, dt, dv, nd, d);
  inv_t L;
  transpose(&D, &L);
  or_index *X = (or_index *)calloc(1, sizeof(or_index));
  X->d = d;
  X->n = nd;
  X->quantize = quantize;
  X->lists = (olist_t *)calloc(d, sizeof(olist_t));
  if (threads < 1) threads = 1;
  bd_ctx c = {&D, &L, X, term_mask, lambda, beta, lambda_frac, beta_frac, alpha, seed,
              NULL, NULL, NULL, NULL, NULL};
  c.dense = (double **)calloc(threads, sizeof(void *));
  c.mx = (float **)calloc(threads, sizeof(void *));
  c.cnt = (uint32_t **)calloc(threads, sizeof(void *));
  c.touched = (uint16_t **)calloc(threads, sizeof(void *));
  c.mss = (mss_t **)calloc(threads, sizeof(void *));
  for (int i = 0; i < threads; i++) {
    c.dense[i] = (double *)calloc(d, sizeof(double));
    c.mx[i] = (float *)calloc(d, sizeof(float));
    c.cnt[i] = (uint32_t *)calloc(d, sizeof(uint32_t));
    c.touched[i] = (uint16_t *)calloc(d, sizeof(uint16_t));
    c.mss[i] = (mss_t *)calloc(d, sizeof(mss_t));
  }
  pfor((int64_t)d, threads, build_list, &c);
  for (int i = 0; i < threads; i++) {
    free(c.dense[i]); free(c.mx[i]); free(c.cnt[i]); free(c.touched[i]); free(c.mss[i]);
  }
  free(c.dense); free(c.mx); free(c.cnt); free(c.touched); free(c.mss);
  inv_free(&L);
  return X;
}

or_index *or_build(const uint64_t *dip, const uint16_t *dt, const float *dv, uint64_t nd, uint32_t d,
                   uint32_t lambda, double lambda_frac, uint32_t beta, double beta_frac, double alpha,
                   int quantize, uint64_t seed, int threads) {
  return or_build_masked(dip, dt, dv, nd, d, lambda, lambda_frac, beta, beta_frac, alpha, quantize, seed,
                         threads, NULL);
}

void or_free(or_index *X) {
  if (!X) return;
  for (uint32_t t = 0; t < X->d; t++) {
    olist_t *o = &X->lists[t];
    free(o->doc); free(o->val); free(o->cent); free(o->assign); free(o->bcent); free(o->bptr);
    free(o->bmem); free(o->sptr); free(o->sterm); free(o->sval); free(o->scode); free(o->qm);
    free(o->qsz);
  }
  free(X->lists);
  free(X);
}

/* Accessors for the tests: list t's arrays and sizes. */
void or_list_sizes(const or_index *X, uint32_t t, uint32_t *out /* n, ncent, nblk, nsum */) {
  const olist_t *o = &X->lists[t];
  out[0] = o->n;
  out[1] = o->ncent;
  out[2] = o->nblk;
  out[3] = o->nblk ? o->sptr[o->nblk] : 0;
}

void or_list_get(const or_index *X, uint32_t t, uint32_t *doc, float *val, uint32_t *cent,
                 uint32_t *assign, uint32_t *bcent, uint32_t *bptr, uint32_t *bmem, uint32_t *sptr,
                 uint16_t *sterm, float *sval, uint8_t *scode, float *qm, float *qsz) {
  const olist_t *o = &X->lists[t];
  uint32_t ns = o->nblk ? o->sptr[o->nblk] : 0;
  if (doc && o->n) memcpy(doc, o->doc, 4 * (size_t)o->n);
  if (val && o->n) memcpy(val, o->val, 4 * (size_t)o->n);
  if (cent && o->ncent) memcpy(cent, o->cent, 4 * (size_t)o->ncent);
  if (assign && o->n) memcpy(assign, o->assign, 4 * (size_t)o->n);
  if (bcent && o->nblk) memcpy(bcent, o->bcent, 4 * (size_t)o->nblk);
  if (bptr && o->nblk) memcpy(bptr, o->bptr, 4 * ((size_t)o->nblk + 1));
  if (bmem && o->n) memcpy(bmem, o->bmem, 4 * (size_t)o->n);
  if (sptr && o->nblk) memcpy(sptr, o->sptr, 4 * ((size_t)o->nblk + 1));
  if (sterm && ns) memcpy(sterm, o->sterm, 2 * (size_t)ns);
  if (sval && ns) memcpy(sval, o->sval, 4 * (size_t)ns);
  if (scode && ns) memcpy(scode, o->scode, (size_t)ns);
  if (qm && o->nblk) memcpy(qm, o->qm, 4 * (size_t)o->nblk);
  if (qsz && o->nblk) memcpy(qsz, o->qsz, 4 * (size_t)o->nblk);
}

/* ------------------------------------------------------------------ */
/* kappa-NN graph, exactly (Eq. knn-graph): N(u) = the kappa best v != u by
 * (<u,v> desc, id asc) over the whole collection; fp64 term-at-a-time. */
typedef struct {
  const csr_t *D;
  const inv_t *L;
  uint32_t kappa;
  uint32_t *out;
  double **acc;
  uint32_t **stamp;
  ent_t **heap;
} kn_ctx;

static void knn_one(void *vc, int64_t ui, int tid) {
  kn_ctx *c = (kn_ctx *)vc;
  const csr_t *D = c->D;
  double *acc = c->acc[tid];
  uint32_t *st = c->stamp[tid];
  uint32_t mark = (uint32_t)ui + 1;
  topk_t h = {c->heap[tid], 0, c->kappa};
  for (uint64_t p = D->indptr[ui]; p < D->indptr[ui + 1]; p++) {
    uint16_t t = D->terms[p];
    double uv = (double)D->vals[p];
    for (uint64_t e = c->L->ptr[t]; e < c->L->ptr[t + 1]; e++) {
      uint32_t dd = c->L->doc[e];
      if (st[dd] != mark) { st[dd] = mark; acc[dd] = 0.0; }
      acc[dd] += uv * (double)c->L->val[e];
    }
  }
  for (uint64_t p = D->indptr[ui]; p < D->indptr[ui + 1]; p++) {
    uint16_t t = D->terms[p];
    for (uint64_t e = c->L->ptr[t]; e < c->L->ptr[t + 1]; e++) {
      uint32_t dd = c->L->doc[e];
      if (st[dd] == mark) {
        if (dd != (uint32_t)ui) offer(&h, acc[dd], dd);
        st[dd] = mark ^ 0x80000000u;
      }
    }
  }
  for (uint64_t dd = 0; dd < D->n; dd++) {
    if (h.n == h.k && !better(0.0, (uint32_t)dd, h.e[h.n - 1].s, h.e[h.n - 1].id)) break;
    if (dd != (uint64_t)ui && st[dd] != (mark ^ 0x80000000u)) offer(&h, 0.0, (uint32_t)dd);
  }
  for (uint32_t i = 0; i < c->kappa; i++) c->out[(uint64_t)ui * c->kappa + i] = i < h.n ? h.e[i].id : NONE_ID;
}

int or_knn_exact(const uint64_t *dip, const uint16_t *dt, const float *dv, uint64_t nd, uint32_t d,
                 uint32_t kappa, int threads, uint32_t *out) {
  csr_t D = mk(dip, dt, dv, nd, d);
  inv_t L;
  transpose(&D, &L);
  if (threads < 1) threads = 1;
  kn_ctx c = {&D, &L, kappa, out, NULL, NULL, NULL};
  c.acc = (double **)calloc(threads, sizeof(void *));
  c.stamp = (uint32_t **)calloc(threads, sizeof(void *));
  c.heap = (ent_t **)calloc(threads, sizeof(void *));
  for (int i = 0; i < threads; i++) {
    c.acc[i] = (double *)malloc(sizeof(double) * (nd ? nd : 1));
    c.stamp[i] = (uint32_t *)calloc(nd ? nd : 1, sizeof(uint32_t));
    c.heap[i] = (ent_t *)malloc(sizeof(ent_t) * (kappa + 1));
  }
  pfor((int64_t)nd, threads, knn_one, &c);
  for (int i = 0; i < threads; i++) { free(c.acc[i]); free(c.stamp[i]); free(c.heap[i]); }
  free(c.acc); free(c.stamp); free(c.heap);
  inv_free(&L);
  return 0;
}

/* ------------------------------------------------------------------ */
/* One neighbour-of-neighbour pass over a kappa-NN graph (not a step of the
 * paper; its Section 4.3 builds N(u) approximately with the method itself,
 * and this pass applies that method's expansion step -- candidates are the
 * union of the neighbour lists of a set, Algorithm "Query processing with
 * Seismic" -- to the graph): for every u, the candidates are
 * C(u) = (N(u) u N(N(u))) \ {u}, missing entries dropped, and the new N(u)
 * is the kappa best of C(u) by (<u,v> desc, id asc) in fp64, padded with
 * NONE_ID.  Reads `in` only, writes `out` (they must not overlap). */
typedef struct {
  const csr_t *D;
  const uint32_t *in;
  uint32_t kappa;
  uint32_t *out;
  double **qd;
  uint32_t **stamp;
  ent_t **heap;
} rf_ctx;

static void refine_one(void *vc, int64_t ui, int tid) {
  rf_ctx *c = (rf_ctx *)vc;
  const csr_t *D = c->D;
  double *qd = c->qd[tid];
  uint32_t *st = c->stamp[tid];
  const uint32_t mark = (uint32_t)ui + 1, K = c->kappa;
  topk_t h = {c->heap[tid], 0, K};
  for (uint64_t p = D->indptr[ui]; p < D->indptr[ui + 1]; p++) qd[D->terms[p]] = (double)D->vals[p];
  st[ui] = mark; /* u itself is never a candidate */
  for (uint32_t i = 0; i <= K; i++) {
    /* i = 0: u's own list; i >= 1: the list of its (i-1)-th neighbour */
    uint32_t src = (uint32_t)ui;
    if (i > 0) {
      src = c->in[(uint64_t)ui * K + (i - 1)];
      if (src == NONE_ID) continue;
    }
    for (uint32_t e = 0; e < K; e++) {
      uint32_t v = c->in[(uint64_t)src * K + e];
      if (v == NONE_ID || st[v] == mark) continue;
      st[v] = mark;
      double s = 0.0;
      for (uint64_t p = D->indptr[v]; p < D->indptr[v + 1]; p++) s += qd[D->terms[p]] * (double)D->vals[p];
      offer(&h, s, v);
    }
  }
  for (uint64_t p = D->indptr[ui]; p < D->indptr[ui + 1]; p++) qd[D->terms[p]] = 0.0;
  for (uint32_t j = 0; j < K; j++) c->out[(uint64_t)ui * K + j] = j < h.n ? h.e[j].id : NONE_ID;
}

int or_knn_refine(const uint64_t *dip, const uint16_t *dt, const float *dv, uint64_t nd, uint32_t d,
                  const uint32_t *in, uint32_t kappa, int threads, uint32_t *out) {
  csr_t D = mk(dip, dt, dv, nd, d);
  if (threads < 1) threads = 1;
  rf_ctx c = {&D, in, kappa, out, NULL, NULL, NULL};
  c.qd = (double **)calloc(threads, sizeof(void *));
  c.stamp = (uint32_t **)calloc(threads, sizeof(void *));
  c.heap = (ent_t **)calloc(threads, sizeof(void *));
  for (int i = 0; i < threads; i++) {
    c.qd[i] = (double *)calloc(d ? d : 1, sizeof(double));
    c.stamp[i] = (uint32_t *)calloc(nd ? nd : 1, sizeof(uint32_t));
    c.heap[i] = (ent_t *)malloc(sizeof(ent_t) * (kappa + 1));
  }
  pfor((int64_t)nd, threads, refine_one, &c);
  for (int i = 0; i < threads; i++) { free(c.qd[i]); free(c.stamp[i]); free(c.heap[i]); }
  free(c.qd); free(c.stamp); free(c.heap);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Query processing (Algorithm "Query processing with Seismic").          */
enum { ST_LISTS, ST_BLOCKS_SCORED, ST_BLOCKS_EVAL, ST_BLOCKS_SKIPPED, ST_DOCS, ST_DOC_NNZ,
       ST_KNN_DOCS, ST_SUMMARY_ENTRIES, ST_N };

typedef struct {
  const or_index *X;
  const csr_t *D, *Q;
  uint32_t k, cut;
  double alpha_q, hf;
  int hf_mode, exhaustive;
  const uint32_t *knn;
  uint32_t kappa;
  uint32_t *ids;
  double *scores;
  uint64_t *stats;
  uint32_t *phase1_ids;
  double **qd;
  uint32_t **seen;
  ent_t **heap;
  mss_t **ord;
  double **r;
  uint32_t **bord;
} se_ctx;

typedef struct {
  double r;
  uint32_t b;
} rb_t;

static int rb_cmp(const void *x, const void *y) {
  const rb_t *a = (const rb_t *)x, *b = (const rb_t *)y;
  if (a->r > b->r) return -1;
  if (a->r < b->r) return 1;
  return (a->b > b->b) - (a->b < b->b);
}

typedef struct {
  float v;
  uint16_t t;
} qt_t;

static int qt_cmp(const void *x, const void *y) {
  const qt_t *a = (const qt_t *)x, *b = (const qt_t *)y;
  if (a->v > b->v) return -1;
  if (a->v < b->v) return 1;
  return (a->t > b->t) - (a->t < b->t);
}

/* <q, S_b>: the block's sketched summary, dequantised as m + code * size
 * when the index is quantised; fp64, ascending term order. */
static double summary_score(const or_index *X, const olist_t *o, uint32_t b, const double *qd) {
  double r = 0.0;
  for (uint32_t e = o->sptr[b]; e < o->sptr[b + 1]; e++) {
    double sv = X->quantize ? (double)o->qm[b] + (double)o->scode[e] * (double)o->qsz[b]
                            : (double)o->sval[e];
    r += qd[o->sterm[e]] * sv;
  }
  return r;
}

/* r_b for every block of list t against one query (terms/vals, nq entries). */
void or_block_scores(const or_index *X, const uint16_t *qt, const float *qv, uint32_t nq, uint32_t t,
                     double *out) {
  double *qd = (double *)calloc(X->d, sizeof(double));
  for (uint32_t i = 0; i < nq; i++) qd[qt[i]] = (double)qv[i];
  const olist_t *o = &X->lists[t];
  for (uint32_t b = 0; b < o->nblk; b++) out[b] = summary_score(X, o, b, qd);
  free(qd);
}

/* <q, u_d> in fp64 over the document's terms in ascending order */
static double doc_dot(const csr_t *D, const double *qd, uint32_t dd) {
  double s = 0.0;
  for (uint64_t p = D->indptr[dd]; p < D->indptr[dd + 1]; p++) s += qd[D->terms[p]] * (double)D->vals[p];
  return s;
}

static void search_one(void *vc, int64_t qi, int tid) {
  se_ctx *c = (se_ctx *)vc;
  const csr_t *Q = c->Q, *D = c->D;
  const or_index *X = c->X;
  double *qd = c->qd[tid];
  uint32_t *seen = c->seen[tid];
  uint32_t mark = (uint32_t)qi + 1;
  uint64_t *stt = c->stats ? c->stats + (uint64_t)qi * ST_N : NULL;
  uint64_t s_local[ST_N];
  memset(s_local, 0, sizeof(s_local));
  topk_t h = {c->heap[tid], 0, c->k};

  /* explicit zeros are not entries of a sparse vector */
  uint32_t nq = 0;
  qt_t *qe = (qt_t *)malloc(sizeof(qt_t) * (Q->indptr[qi + 1] - Q->indptr[qi] + 1));
  for (uint64_t p = Q->indptr[qi]; p < Q->indptr[qi + 1]; p++) {
    if (Q->vals[p] == 0.0f) continue;
    qd[Q->terms[p]] = (double)Q->vals[p];
    qe[nq].v = Q->vals[p];
    qe[nq].t = Q->terms[p];
    nq++;
  }
  /* the query's list terms: the top `cut` by value, or its alpha_q-MSS */
  uint32_t ncut;
  uint16_t *T = (uint16_t *)malloc(sizeof(uint16_t) * (nq + 1));
  if (c->alpha_q > 0.0) {
    uint16_t *tt = (uint16_t *)malloc(sizeof(uint16_t) * (nq + 1));
    float *vv = (float *)malloc(sizeof(float) * (nq + 1));
    for (uint32_t i = 0; i < nq; i++) { tt[i] = qe[i].t; vv[i] = qe[i].v; }
    mss_t *ms = c->ord[tid];
    ncut = alpha_mss(tt, vv, nq, c->alpha_q, ms);
    for (uint32_t i = 0; i < ncut; i++) T[i] = ms[i].t;
    free(tt);
    free(vv);
  } else {
    qsort(qe, nq, sizeof(qt_t), qt_cmp);
    ncut = c->cut < nq ? c->cut : nq;
    for (uint32_t i = 0; i < ncut; i++) T[i] = qe[i].t;
  }

  rb_t *rb = (rb_t *)c->r[tid];
  for (uint32_t li = 0; li < ncut; li++) {
    const olist_t *o = &X->lists[T[li]];
    s_local[ST_LISTS]++;
    if (o->nblk == 0) continue;
    /* r_j = <q, S_j> for every block of the list, with the full query */
    for (uint32_t b = 0; b < o->nblk; b++) {
      rb[b].r = 0.0;
      rb[b].b = b;
      if (!c->exhaustive) {
        rb[b].r = summary_score(X, o, b, qd);
        s_local[ST_BLOCKS_SCORED]++;
        s_local[ST_SUMMARY_ENTRIES] += o->sptr[b + 1] - o->sptr[b];
      }
    }
    if (!c->exhaustive) qsort(rb, o->nblk, sizeof(rb_t), rb_cmp);
    for (uint32_t bi = 0; bi < o->nblk; bi++) {
      uint32_t b = rb[bi].b;
      if (!c->exhaustive && h.n == h.k) {
        double theta = h.e[h.n - 1].s;
        int skip = c->hf_mode == 0 ? (rb[bi].r < c->hf * theta) : (rb[bi].r < theta / c->hf);
        if (skip) { s_local[ST_BLOCKS_SKIPPED]++; continue; }
      }
      s_local[ST_BLOCKS_EVAL]++;
      for (uint32_t m = o->bptr[b]; m < o->bptr[b + 1]; m++) {
        uint32_t dd = o->bmem[m];
        if (seen[dd] == mark) continue;
        seen[dd] = mark;
        double p = doc_dot(D, qd, dd);
        s_local[ST_DOCS]++;
        s_local[ST_DOC_NNZ] += D->indptr[dd + 1] - D->indptr[dd];
        offer(&h, p, dd);
      }
    }
  }
  if (c->phase1_ids) {
    for (uint32_t i = 0; i < c->k; i++) c->phase1_ids[(uint64_t)qi * c->k + i] = i < h.n ? h.e[i].id : NONE_ID;
  }
  /* kappa-NN expansion of the heap's members (S fixed before expanding) */
  if (c->knn && c->kappa > 0 && h.n > 0) {
    uint32_t ns = h.n;
    uint32_t *S = (uint32_t *)malloc(sizeof(uint32_t) * ns);
    for (uint32_t i = 0; i < ns; i++) S[i] = h.e[i].id;
    for (uint32_t i = 0; i < ns; i++) {
      for (uint32_t e = 0; e < c->kappa; e++) {
        uint32_t v = c->knn[(uint64_t)S[i] * c->kappa + e];
        if (v == NONE_ID || seen[v] == mark) continue;
        seen[v] = mark;
        double p = doc_dot(D, qd, v);
        s_local[ST_KNN_DOCS]++;
        offer(&h, p, v);
      }
    }
    free(S);
  }
  emit(&h, c->ids + (uint64_t)qi * c->k, c->scores + (uint64_t)qi * c->k);
  for (uint64_t p = Q->indptr[qi]; p < Q->indptr[qi + 1]; p++) qd[Q->terms[p]] = 0.0;
  if (stt) memcpy(stt, s_local, sizeof(s_local));
  free(qe);
  free(T);
}

int or_search(const or_index *X, const uint64_t *dip, const uint16_t *dt, const float *dv, uint64_t nd,
              const uint64_t *qip, const uint16_t *qt, const float *qv, uint64_t nq, uint32_t k,
              uint32_t cut, double alpha_q, double hf, int hf_mode, int exhaustive,
              const uint32_t *knn, uint32_t kappa, int threads, uint32_t *ids, double *scores,
              uint64_t *stats, uint32_t *phase1_ids) {
  csr_t D = mk(dip, dt, dv, nd, X->d), Q = mk(qip, qt, qv, nq, X->d);
  if (threads < 1) threads = 1;
  uint32_t maxblk = 1;
  for (uint32_t t = 0; t < X->d; t++) if (X->lists[t].nblk > maxblk) maxblk = X->lists[t].nblk;
  se_ctx c = {X, &D, &Q, k, cut, alpha_q, hf, hf_mode, exhaustive, knn, kappa, ids, scores, stats,
              phase1_ids, NULL, NULL, NULL, NULL, NULL, NULL};
  c.qd = (double **)calloc(threads, sizeof(void *));
  c.seen = (uint32_t **)calloc(threads, sizeof(void *));
  c.heap = (ent_t **)calloc(threads, sizeof(void *));
  c.ord = (mss_t **)calloc(threads, sizeof(void *));
  c.r = (double **)calloc(threads, sizeof(void *));
  for (int i = 0; i < threads; i++) {
    c.qd[i] = (double *)calloc(X->d, sizeof(double));
    c.seen[i] = (uint32_t *)calloc(nd ? nd : 1, sizeof(uint32_t));
    c.heap[i] = (ent_t *)malloc(sizeof(ent_t) * (k + 1));
    c.ord[i] = (mss_t *)malloc(sizeof(mss_t) * (X->d + 1));
    c.r[i] = (double *)malloc(sizeof(rb_t) * maxblk);
  }
  pfor((int64_t)nq, threads, search_one, &c);
  for (int i = 0; i < threads; i++) { free(c.qd[i]); free(c.seen[i]); free(c.heap[i]); free(c.ord[i]); free(c.r[i]); }
  free(c.qd); free(c.seen); free(c.heap); free(c.ord); free(c.r);
  return 0;
}

/* ------------------------------------------------------------------ */
/* <q_i, u_j> in fp64 for listed (query, doc) pairs; used to score a
 * returned id for accuracy@k (Definition ann-accuracy). */
int or_pair_dots(const uint64_t *dip, const uint16_t *dt, const float *dv, uint64_t nd, uint32_t d,
                 const uint64_t *qip, const uint16_t *qt, const float *qv, uint64_t nq,
                 const uint64_t *qidx, const uint32_t *didx, uint64_t npairs, double *out) {
  (void)nq;
  double *qd = (double *)calloc(d, sizeof(double));
  uint64_t cur = (uint64_t)-1;
  for (uint64_t i = 0; i < npairs; i++) {
    uint64_t q = qidx[i];
    if (q != cur) {
      if (cur != (uint64_t)-1)
        for (uint64_t p = qip[cur]; p < qip[cur + 1]; p++) qd[qt[p]] = 0.0;
      for (uint64_t p = qip[q]; p < qip[q + 1]; p++) qd[qt[p]] = (double)qv[p];
      cur = q;
    }
    uint32_t j = didx[i];
    if (j >= nd) { out[i] = -INFINITY; continue; }
    double s = 0.0;
    for (uint64_t p = dip[j]; p < dip[j + 1]; p++) s += qd[dt[p]] * (double)dv[p];
    out[i] = s;
  }
  free(qd);
  return 0;
}

/*
 * Seeded synthetic generator of SPLADE-shaped sparse vectors.
 *
 * Shape targets: the SPLADE embeddings of MS MARCO (Section 5.1.2: about
 * 119 nonzeros per passage, 43 per query, a WordPiece vocabulary of about
 * 30,000 terms).  The real embeddings are not available, so every collection
 * is drawn from this latent-topic model instead:
 *
 *   - K topics, each a Zipf(s) distribution over its own random permutation
 *     of the vocabulary [0, d);
 *   - per row: a topic mixture theta ~ Dirichlet(a * 1_K), a target nnz,
 *     then distinct terms drawn by z ~ theta, rank ~ Zipf, term = perm_z[rank]
 *     (repeats rejected) until nnz distinct terms are held;
 *   - value = |N(0,1)| * (1 + exp(-rank/20)) in fp32 (rank 0-based), never 0.
 *
 * This file holds no part of the search method: it only draws inputs.  Both
 * the oracle and the GPU library consume its output.
 *
 * Randomness: every row draws from its own xoshiro256** stream seeded through
 * splitmix64 from (seed, stream, row), so the output does not depend on the
 * thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } xo_t;

static uint64_t sm64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xo_t *r) {
  uint64_t *s = r->s;
  uint64_t res = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return res;
}

static void xo_seed(xo_t *r, uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t x = seed ^ 0x5EED5EED5EED5EEDULL;
  x = sm64(&x) ^ (stream * 0xD1B54A32D192ED03ULL);
  x = sm64(&x) ^ (idx * 0x8CB92BA72F3D8DD7ULL);
  for (int i = 0; i < 4; i++) r->s[i] = sm64(&x);
}

/* uniform in the open interval (0, 1) */
static double uo(xo_t *r) { return ((double)(xo_next(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

static double normal(xo_t *r) {
  for (;;) { /* Marsaglia polar method */
    double u = 2.0 * uo(r) - 1.0, v = 2.0 * uo(r) - 1.0;
    double s = u * u + v * v;
    if (s > 0.0 && s < 1.0) return u * sqrt(-2.0 * log(s) / s);
  }
}

static double gamma_ge1(xo_t *r, double a) { /* Marsaglia-Tsang, a >= 1 */
  double dd = a - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * dd);
  for (;;) {
    double x = normal(r), v = 1.0 + c * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    double u = uo(r);
    if (log(u) < 0.5 * x * x + dd - dd * v + dd * log(v)) return dd * v;
  }
}

static double gamma_draw(xo_t *r, double a) {
  if (a >= 1.0) return gamma_ge1(r, a);
  return gamma_ge1(r, a + 1.0) * pow(uo(r), 1.0 / a);
}

typedef struct {
  uint32_t d, K;
  double zipf_s, dir_a;
  int nnz_mode; /* 0: lognormal(mean, sd) in linear space; 1: uniform integer */
  double nnz_a, nnz_b;
  uint32_t nnz_lo, nnz_hi;
  uint64_t seed, stream;
  const uint16_t *perm; /* K x d */
  const double *cdf;    /* d */
} cfg_t;

static uint32_t draw_nnz(const cfg_t *c, xo_t *r) {
  double n;
  if (c->nnz_mode == 0) {
    double m = c->nnz_a, s = c->nnz_b;
    double sig2 = log(1.0 + (s * s) / (m * m));
    double mu = log(m) - 0.5 * sig2;
    n = floor(exp(mu + sqrt(sig2) * normal(r)) + 0.5);
  } else {
    uint64_t span = (uint64_t)(c->nnz_hi - c->nnz_lo) + 1;
    n = (double)(c->nnz_lo + xo_next(r) % span);
  }
  if (n < c->nnz_lo) n = c->nnz_lo;
  if (n > c->nnz_hi) n = c->nnz_hi;
  if (n > c->d) n = c->d;
  return (uint32_t)n;
}

static uint32_t zipf_rank(const cfg_t *c, xo_t *r) {
  double u = uo(r);
  uint32_t lo = 0, hi = c->d - 1;
  while (lo < hi) { /* first rank whose cumulative mass reaches u */
    uint32_t mid = lo + (hi - lo) / 2;
    if (c->cdf[mid] >= u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

static void sort_row(uint16_t *t, float *v, uint32_t n) {
  for (uint32_t i = 1; i < n; i++) { /* insertion sort: rows are short */
    uint16_t tk = t[i];
    float vk = v[i];
    uint32_t j = i;
    while (j > 0 && t[j - 1] > tk) { t[j] = t[j - 1]; v[j] = v[j - 1]; j--; }
    t[j] = tk;
    v[j] = vk;
  }
}

/* Draws row `row` into (terms, vals); `mark` is a per-thread stamp array of d. */
static void draw_row(const cfg_t *c, uint64_t row, uint16_t *terms, float *vals, uint32_t *mark,
                     uint32_t stamp, double *theta) {
  xo_t r;
  xo_seed(&r, c->seed, c->stream, row);
  uint32_t nnz = draw_nnz(c, &r);
  double tot = 0.0;
  for (uint32_t z = 0; z < c->K; z++) { theta[z] = gamma_draw(&r, c->dir_a); tot += theta[z]; }
  if (!(tot > 0.0)) { for (uint32_t z = 0; z < c->K; z++) theta[z] = 1.0; tot = c->K; }
  double acc = 0.0;
  for (uint32_t z = 0; z < c->K; z++) { acc += theta[z] / tot; theta[z] = acc; }
  uint32_t have = 0;
  while (have < nnz) {
    double u = uo(&r);
    uint32_t z = 0;
    while (z + 1 < c->K && theta[z] < u) z++;
    uint32_t rank = zipf_rank(c, &r);
    uint16_t t = c->perm[(uint64_t)z * c->d + rank];
    if (mark[t] == stamp) continue;
    mark[t] = stamp;
    double x;
    do { x = fabs(normal(&r)); } while (x == 0.0);
    float v = (float)(x * (1.0 + exp(-(double)rank / 20.0)));
    if (v == 0.0f) v = 1.17549435e-38f;
    terms[have] = t;
    vals[have] = v;
    have++;
  }
  sort_row(terms, vals, nnz);
}

typedef struct {
  const cfg_t *c;
  uint64_t r0, r1;
  const uint64_t *indptr; /* NULL: count pass */
  uint64_t *counts;
  uint16_t *terms;
  float *vals;
} job_t;

static void *worker(void *arg) {
  job_t *j = (job_t *)arg;
  const cfg_t *c = j->c;
  if (!j->indptr) {
    for (uint64_t row = j->r0; row < j->r1; row++) {
      xo_t r;
      xo_seed(&r, c->seed, c->stream, row);
      j->counts[row] = draw_nnz(c, &r);
    }
    return NULL;
  }
  uint32_t *mark = (uint32_t *)calloc(c->d, sizeof(uint32_t));
  double *theta = (double *)malloc(sizeof(double) * c->K);
  uint32_t stamp = 0;
  for (uint64_t row = j->r0; row < j->r1; row++) {
    if (++stamp == 0) { memset(mark, 0, sizeof(uint32_t) * c->d); stamp = 1; }
    uint64_t o = j->indptr[row];
    draw_row(c, row, j->terms + o, j->vals + o, mark, stamp, theta);
  }
  free(mark);
  free(theta);
  return NULL;
}

static void run(const cfg_t *c, uint64_t n, int threads, const uint64_t *indptr, uint64_t *counts,
                uint16_t *terms, float *vals) {
  if (threads < 1) threads = 1;
  if ((uint64_t)threads > n) threads = n ? (int)n : 1;
  pthread_t th[256];
  job_t jb[256];
  if (threads > 256) threads = 256;
  for (int i = 0; i < threads; i++) {
    jb[i] = (job_t){c, n * i / threads, n * (i + 1) / threads, indptr, counts, terms, vals};
    pthread_create(&th[i], NULL, worker, &jb[i]);
  }
  for (int i = 0; i < threads; i++) pthread_join(th[i], NULL);
}

/* Topic permutations (K x d, u16) and the Zipf cumulative table (d, fp64). */
void synth_topics(uint64_t seed, uint32_t d, uint32_t K, double zipf_s, uint16_t *perm, double *cdf) {
  for (uint32_t z = 0; z < K; z++) {
    xo_t r;
    xo_seed(&r, seed, 0x70F1C5ULL, z);
    uint16_t *p = perm + (uint64_t)z * d;
    for (uint32_t i = 0; i < d; i++) p[i] = (uint16_t)i;
    for (uint32_t i = d - 1; i > 0; i--) {
      uint32_t j = (uint32_t)(xo_next(&r) % (uint64_t)(i + 1));
      uint16_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
  }
  double h = 0.0;
  for (uint32_t i = 0; i < d; i++) h += 1.0 / pow((double)(i + 1), zipf_s);
  double acc = 0.0;
  for (uint32_t i = 0; i < d; i++) { acc += 1.0 / pow((double)(i + 1), zipf_s) / h; cdf[i] = acc; }
  cdf[d - 1] = 1.0;
}

/* Pass 1: nnz of every row (counts[n]).  Pass 2: fill terms/vals at indptr. */
void synth_rows(uint64_t seed, uint64_t stream, uint64_t n, uint32_t d, uint32_t K, double zipf_s,
                double dir_a, int nnz_mode, double nnz_a, double nnz_b, uint32_t nnz_lo,
                uint32_t nnz_hi, const uint16_t *perm, const double *cdf, int threads,
                const uint64_t *indptr, uint64_t *counts, uint16_t *terms, float *vals) {
  cfg_t c = {d, K, zipf_s, dir_a, nnz_mode, nnz_a, nnz_b, nnz_lo, nnz_hi, seed, stream, perm, cdf};
  run(&c, n, threads, indptr, counts, terms, vals);
}

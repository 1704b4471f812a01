/*
 * Seeded synthetic graph generators (R-MAT, Erdos-Renyi G(n,m), 2-D grid with
 * random edge deletion) and source sampling.
 *
 * This module only prepares inputs: it builds a symmetric, simple (no
 * self-loops, no duplicate neighbours), row-sorted int32 CSR.  It contains no
 * part of the BFS method and is shared by the CPU oracle tests and by the CUDA
 * path's tests and benchmark.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014) expands a seed into the
 * state of xoshiro256** (Blackman, Vigna 2018).  Only integer arithmetic is
 * used, so a given seed yields byte-identical graphs on x86-64 and AArch64.
 * Probabilities arrive as integer thresholds computed by the caller.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  uint64_t s[4];
} gg_rng;

static uint64_t splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static void rng_seed(gg_rng *r, uint64_t seed, uint64_t stream) {
  uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ull);
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(gg_rng *r) {
  uint64_t *s = r->s;
  const uint64_t result = rotl(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return result;
}

/* Uniform integer in [0, bound), bound > 0: Lemire's multiply-shift with
 * rejection (unbiased). */
static inline uint64_t rng_below(gg_rng *r, uint64_t bound) {
  uint64_t x = rng_next(r);
  __uint128_t m = (__uint128_t)x * bound;
  uint64_t lo = (uint64_t)m;
  if (lo < bound) {
    uint64_t t = (0 - bound) % bound;
    while (lo < t) {
      x = rng_next(r);
      m = (__uint128_t)x * bound;
      lo = (uint64_t)m;
    }
  }
  return (uint64_t)(m >> 64);
}

/* ------------------------------------------------------------------------ */
/* Edge list -> symmetric simple CSR                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t n;
  int64_t nnz;
  int32_t *row_ptr; /* n + 1 */
  int32_t *col_idx; /* nnz */
} gg_csr;

void gg_free(gg_csr *g) {
  if (!g) return;
  free(g->row_ptr);
  free(g->col_idx);
  free(g);
}

/* Stable LSD radix sort of 64-bit keys by their low `bits` bits, 11 bits per
 * pass, each pass a parallel counting sort (per-thread histograms over
 * contiguous slices, so the result does not depend on the thread count). */
static int radix_sort_u64(uint64_t *key, int64_t m, int bits) {
  enum { RB = 11, NB = 1 << 11 };
  if (m <= 1) return 0;
  uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m);
  if (!tmp) return -1;
  int nt = 1;
#ifdef _OPENMP
  nt = omp_get_max_threads();
#endif
  int64_t *hist = (int64_t *)malloc(sizeof(int64_t) * (size_t)NB * (size_t)nt);
  if (!hist) { free(tmp); return -1; }
  uint64_t *src = key, *dst = tmp;
  for (int shift = 0; shift < bits; shift += RB) {
    memset(hist, 0, sizeof(int64_t) * (size_t)NB * (size_t)nt);
#pragma omp parallel num_threads(nt)
    {
      int t = 0;
#ifdef _OPENMP
      t = omp_get_thread_num();
#endif
      int64_t lo = m * t / nt, hi = m * (t + 1) / nt;
      int64_t *h = hist + (size_t)t * NB;
      for (int64_t i = lo; i < hi; ++i) h[(src[i] >> shift) & (NB - 1)]++;
#pragma omp barrier
#pragma omp single
      {
        int64_t run = 0;
        for (int d = 0; d < NB; ++d)
          for (int u = 0; u < nt; ++u) {
            int64_t c = hist[(size_t)u * NB + d];
            hist[(size_t)u * NB + d] = run;
            run += c;
          }
      }
      for (int64_t i = lo; i < hi; ++i) dst[h[(src[i] >> shift) & (NB - 1)]++] = src[i];
    }
    uint64_t *s = src; src = dst; dst = s;
  }
  if (src != key) memcpy(key, src, sizeof(uint64_t) * (size_t)m);
  free(tmp);
  free(hist);
  return 0;
}

/* Build the CSR of the symmetric closure of the m undirected pairs (a[i],
 * b[i]): both directions are inserted, self-loops dropped, then the (row,
 * column) keys are radix-sorted and duplicates removed, giving rows sorted
 * ascending without repeats.  Returns NULL on allocation failure. */
static gg_csr *build_symmetric_csr(int32_t n, int64_t m, const int32_t *a, const int32_t *b) {
  int64_t cap = 2 * m;
  uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cap ? cap : 1));
  gg_csr *g = (gg_csr *)calloc(1, sizeof(gg_csr));
  if (!key || !g) { free(key); gg_free(g); return NULL; }
  int64_t e = 0;
  for (int64_t i = 0; i < m; ++i) {
    uint64_t u = (uint32_t)a[i], v = (uint32_t)b[i];
    if (u == v) continue;
    key[e++] = (u << 32) | v;
    key[e++] = (v << 32) | u;
  }
  int vb = 1;
  while (vb < 31 && ((int64_t)1 << vb) < n) ++vb;
  /* sort by column (low vb bits) then by row (bits 32..32+vb) */
  for (int64_t i = 0; i < e; ++i) key[i] = (key[i] >> 32) << vb | (key[i] & 0xFFFFFFFFull);
  if (radix_sort_u64(key, e, 2 * vb) != 0) { free(key); gg_free(g); return NULL; }
  g->n = n;
  g->row_ptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  g->col_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(e ? e : 1));
  if (!g->row_ptr || !g->col_idx) { free(key); gg_free(g); return NULL; }
  const uint64_t cmask = ((uint64_t)1 << vb) - 1;
  int64_t w = 0;
  int32_t row = 0;
  g->row_ptr[0] = 0;
  for (int64_t i = 0; i < e; ++i) {
    if (i > 0 && key[i] == key[i - 1]) continue;
    int32_t r = (int32_t)(key[i] >> vb);
    while (row < r) g->row_ptr[++row] = (int32_t)w;
    g->col_idx[w++] = (int32_t)(key[i] & cmask);
  }
  while (row < n) g->row_ptr[++row] = (int32_t)w;
  g->nnz = w;
  free(key);
  return g;
}

/* ------------------------------------------------------------------------ */
/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004) as used by Graph500             */
/* ------------------------------------------------------------------------ */

/* nsamples edge samples on 2^scale vertices.  Each of the `scale` bits picks
 * a quadrant: u<ta -> (0,0); u<tab -> (0,1); u<tabc -> (1,0); else (1,1), with
 * u a uniform 32-bit draw and ta, tab, tabc the cumulative thresholds of
 * A, A+B, A+B+C scaled by 2^32.  Vertex ids are then relabelled by a seeded
 * uniform random permutation when relabel != 0.  Samples are drawn from
 * independent streams of 2^16 samples each, so the result does not depend on
 * how the work is split. */
gg_csr *gg_rmat(int32_t scale, int64_t nsamples, uint32_t ta, uint32_t tab, uint32_t tabc,
                uint64_t seed, int32_t relabel) {
  if (scale < 1 || scale > 30 || nsamples < 0) return NULL;
  int32_t n = (int32_t)1 << scale;
  int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsamples ? nsamples : 1));
  int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nsamples ? nsamples : 1));
  int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!a || !b || !perm) { free(a); free(b); free(perm); return NULL; }
  const int64_t block = 1 << 16;
  const int64_t nblocks = (nsamples + block - 1) / block;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t bi = 0; bi < nblocks; ++bi) {
    const int64_t base = bi * block;
    gg_rng r;
    rng_seed(&r, seed, 1 + (uint64_t)(base / block));
    int64_t end = base + block < nsamples ? base + block : nsamples;
    for (int64_t i = base; i < end; ++i) {
      uint32_t u = 0, v = 0;
      uint64_t bits = 0;
      int have = 0;
      for (int k = 0; k < scale; ++k) {
        if (!have) { bits = rng_next(&r); have = 2; }
        uint32_t x = (uint32_t)bits;
        bits >>= 32;
        --have;
        uint32_t ub = 0, vb = 0;
        if (x < ta) { ub = 0; vb = 0; }
        else if (x < tab) { ub = 0; vb = 1; }
        else if (x < tabc) { ub = 1; vb = 0; }
        else { ub = 1; vb = 1; }
        u = (u << 1) | ub;
        v = (v << 1) | vb;
      }
      a[i] = (int32_t)u;
      b[i] = (int32_t)v;
    }
  }
  if (relabel) {
    gg_rng r;
    rng_seed(&r, seed, 0);
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
      int32_t j = (int32_t)rng_below(&r, (uint64_t)i + 1);
      int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nsamples; ++i) { a[i] = perm[a[i]]; b[i] = perm[b[i]]; }
  }
  gg_csr *g = build_symmetric_csr(n, nsamples, a, b);
  free(a); free(b); free(perm);
  return g;
}

/* ------------------------------------------------------------------------ */
/* Erdos-Renyi G(n, m): m distinct undirected non-loop edges                 */
/* ------------------------------------------------------------------------ */

/* Draw pairs (u, v) uniformly, skip loops and pairs already drawn (open-
 * addressing hash set of the canonical key min*n+max), until m distinct
 * undirected edges are collected. */
gg_csr *gg_er(int32_t n, int64_t m, uint64_t seed) {
  if (n < 2 || m < 0) return NULL;
  int64_t maxm = (int64_t)n * (n - 1) / 2;
  if (m > maxm) return NULL;
  uint64_t cap = 1;
  while (cap < (uint64_t)(2 * m + 16)) cap <<= 1;
  uint64_t *tab = (uint64_t *)malloc(sizeof(uint64_t) * cap);
  int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
  int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
  if (!tab || !a || !b) { free(tab); free(a); free(b); return NULL; }
  memset(tab, 0xFF, sizeof(uint64_t) * cap);
  gg_rng r;
  rng_seed(&r, seed, 7);
  int64_t got = 0;
  while (got < m) {
    uint32_t u = (uint32_t)rng_below(&r, (uint64_t)n);
    uint32_t v = (uint32_t)rng_below(&r, (uint64_t)n);
    if (u == v) continue;
    uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
    uint64_t key = lo * (uint64_t)n + hi;
    uint64_t h = (key * 0x9E3779B97F4A7C15ull) & (cap - 1);
    int dup = 0;
    while (tab[h] != ~0ull) {
      if (tab[h] == key) { dup = 1; break; }
      h = (h + 1) & (cap - 1);
    }
    if (dup) continue;
    tab[h] = key;
    a[got] = (int32_t)lo;
    b[got] = (int32_t)hi;
    ++got;
  }
  gg_csr *g = build_symmetric_csr(n, m, a, b);
  free(tab); free(a); free(b);
  return g;
}

/* ------------------------------------------------------------------------ */
/* rows x cols 4-neighbour grid, each undirected edge deleted independently */
/* with probability del_thresh / 2^64                                        */
/* ------------------------------------------------------------------------ */

/* Vertex id = r*cols + c.  Edges are visited in the order (r, c, right-edge,
 * down-edge) and each consumes one 64-bit draw; it is deleted when the draw is
 * below del_thresh.  Rows of the CSR are emitted already sorted (up, left,
 * right, down). */
gg_csr *gg_grid(int32_t rows, int32_t cols, uint64_t del_thresh, uint64_t seed) {
  if (rows < 1 || cols < 1 || (int64_t)rows * cols > 0x7FFFFFFF) return NULL;
  int64_t n = (int64_t)rows * cols;
  uint8_t *keep_r = (uint8_t *)malloc((size_t)n);
  uint8_t *keep_d = (uint8_t *)malloc((size_t)n);
  gg_csr *g = (gg_csr *)calloc(1, sizeof(gg_csr));
  if (!keep_r || !keep_d || !g) { free(keep_r); free(keep_d); free(g); return NULL; }
  gg_rng rg;
  rng_seed(&rg, seed, 11);
  for (int32_t r = 0; r < rows; ++r)
    for (int32_t c = 0; c < cols; ++c) {
      int64_t x = (int64_t)r * cols + c;
      keep_r[x] = 0;
      keep_d[x] = 0;
      if (c + 1 < cols) keep_r[x] = rng_next(&rg) >= del_thresh;
      if (r + 1 < rows) keep_d[x] = rng_next(&rg) >= del_thresh;
    }
  g->n = (int32_t)n;
  g->row_ptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
  int64_t nnz = 0;
  for (int64_t x = 0; x < n; ++x) {
    int32_t r = (int32_t)(x / cols), c = (int32_t)(x % cols);
    nnz += (r > 0 && keep_d[x - cols]) + (c > 0 && keep_r[x - 1]) + keep_r[x] + keep_d[x];
  }
  g->col_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
  if (!g->row_ptr || !g->col_idx) { free(keep_r); free(keep_d); gg_free(g); return NULL; }
  int64_t w = 0;
  for (int64_t x = 0; x < n; ++x) {
    int32_t r = (int32_t)(x / cols), c = (int32_t)(x % cols);
    g->row_ptr[x] = (int32_t)w;
    if (r > 0 && keep_d[x - cols]) g->col_idx[w++] = (int32_t)(x - cols);
    if (c > 0 && keep_r[x - 1]) g->col_idx[w++] = (int32_t)(x - 1);
    if (keep_r[x]) g->col_idx[w++] = (int32_t)(x + 1);
    if (keep_d[x]) g->col_idx[w++] = (int32_t)(x + cols);
  }
  g->row_ptr[n] = (int32_t)w;
  g->nnz = w;
  free(keep_r); free(keep_d);
  return g;
}

/* Symmetric simple CSR from a caller-given undirected edge list (used by tests
 * to build small named graphs). */
gg_csr *gg_from_edges(int32_t n, int64_t m, const int32_t *a, const int32_t *b) {
  if (n < 1 || m < 0) return NULL;
  for (int64_t i = 0; i < m; ++i)
    if (a[i] < 0 || a[i] >= n || b[i] < 0 || b[i] >= n) return NULL;
  return build_symmetric_csr(n, m, a, b);
}

/* k distinct sources, uniformly among vertices with at least one neighbour,
 * by rejection.  Returns the number written (< k only if fewer such vertices
 * exist). */
int32_t gg_sample_sources(int32_t n, const int32_t *row_ptr, int32_t k, uint64_t seed, int32_t *out) {
  int32_t avail = 0;
  for (int32_t v = 0; v < n; ++v) avail += row_ptr[v + 1] > row_ptr[v];
  if (k > avail) k = avail;
  uint8_t *taken = (uint8_t *)calloc((size_t)n, 1);
  if (!taken) return -1;
  gg_rng r;
  rng_seed(&r, seed, 3);
  int32_t got = 0;
  while (got < k) {
    int32_t v = (int32_t)rng_below(&r, (uint64_t)n);
    if (taken[v] || row_ptr[v + 1] == row_ptr[v]) continue;
    taken[v] = 1;
    out[got++] = v;
  }
  free(taken);
  return got;
}

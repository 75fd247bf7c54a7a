/*
 * Seeded synthetic graph generators for the EIC shortest-path workloads.
 *
 * This module holds no shortest-path arithmetic. It only produces edge lists
 * (raw tuples that may contain self-loops and duplicates), edge weights, and
 * source vertices. Both the CUDA path and the CPU oracle consume its output.
 *
 * Randomness is counter based: every draw is SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
 * evaluated at state  base(seed, stream) + (i + 1) * GAMMA,  so draw i of a
 * stream does not depend on the order in which draws are made. Parallel
 * generation therefore produces byte-identical output for any thread count.
 *
 * Workload shapes follow the paper's evaluation graphs (Section 4.2): a
 * uniform random graph (Urand-like), an RMAT/Kronecker graph (Graph500 /
 * GAPBS Kron-like, a,b,c,d = 0.57,0.19,0.19,0.05), and a perturbed grid that
 * stands in for the Road graph. Weights are integers; the paper's real-valued
 * weights in (0,1] are replaced by uniform integers (or a clamped log-normal
 * for the heavy-tailed variant, or the paper's power and pivot variants of
 * Eq. 7-8), and the weight of an undirected pair is a hash of the pair, so
 * duplicates and both directions always agree.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ull

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t base = gg_mix(seed * GG_GAMMA + 0x632BE59BD9B4E019ull) ^ gg_mix((stream + 1) * 0xD1B54A32D192ED03ull);
  return gg_mix(base + (i + 1) * GG_GAMMA);
}

/* uniform integer in [0, range) from the high 32 bits of r (range <= 2^32) */
static inline uint32_t gg_below(uint64_t r, uint64_t range) { return (uint32_t)(((r >> 32) * range) >> 32); }

/* uniform double in [0, 1) with 53 random bits */
static inline double gg_unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* ---------------------------------------------------------------- threads */

typedef void (*gg_range_fn)(void* ctx, uint64_t lo, uint64_t hi);
typedef struct {
  gg_range_fn fn;
  void* ctx;
  uint64_t lo, hi;
} gg_job;

static void* gg_run(void* p) {
  gg_job* j = (gg_job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void gg_parallel(uint64_t count, int nthreads, gg_range_fn fn, void* ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((uint64_t)nthreads > count / 65536 + 1) nthreads = (int)(count / 65536 + 1);
  if (nthreads == 1) {
    fn(ctx, 0, count);
    return;
  }
  pthread_t th[256];
  gg_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = count * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].hi = count * (uint64_t)(t + 1) / (uint64_t)nthreads;
    pthread_create(&th[t], NULL, gg_run, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------ uniform (Urand) */

/* Exactly m distinct undirected pairs {u,v}, u != v, endpoints uniform in
 * [0,n), drawn in order and rejected when they repeat or form a loop.
 * Returns 0, or -1 when m is not achievable / memory fails. */
int gg_uniform(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
  if (n < 2) return m == 0 ? 0 : -1;
  if (m > (uint64_t)n * (uint64_t)(n - 1) / 2) return -1;
  uint64_t cap = 16;
  while (cap < 2 * m + 16) cap <<= 1;
  uint64_t* table = (uint64_t*)malloc(cap * sizeof(uint64_t));
  if (!table) return -1;
  memset(table, 0xFF, cap * sizeof(uint64_t));
  uint64_t got = 0, i = 0;
  while (got < m) {
    uint64_t r = gg_rand(seed, 0, i++);
    uint32_t u = gg_below(r, n);
    uint32_t v = gg_below(r << 32, n);
    if (u == v) continue;
    uint64_t key = u < v ? ((uint64_t)u << 32) | v : ((uint64_t)v << 32) | u;
    uint64_t h = gg_mix(key) & (cap - 1);
    int dup = 0;
    while (table[h] != ~0ull) {
      if (table[h] == key) {
        dup = 1;
        break;
      }
      h = (h + 1) & (cap - 1);
    }
    if (dup) continue;
    table[h] = key;
    src[got] = u;
    dst[got] = v;
    ++got;
  }
  free(table);
  return 0;
}

/* ------------------------------------------------------------ RMAT/Kron */

typedef struct {
  int scale;
  uint64_t seed;
  uint32_t A, AB, ABC; /* cumulative quadrant probabilities in 2^-32 units */
  const uint32_t* perm;
  uint32_t* src;
  uint32_t* dst;
} gg_rmat_ctx;

static void gg_rmat_range(void* p, uint64_t lo, uint64_t hi) {
  gg_rmat_ctx* c = (gg_rmat_ctx*)p;
  const uint64_t draws = (uint64_t)(c->scale + 1) / 2;
  for (uint64_t e = lo; e < hi; ++e) {
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (int l = 0; l < c->scale; ++l) {
      uint32_t x;
      if ((l & 1) == 0) {
        r = gg_rand(c->seed, 2, e * draws + (uint64_t)(l >> 1));
        x = (uint32_t)(r >> 32);
      } else {
        x = (uint32_t)r;
      }
      uint32_t ub, vb;
      if (x < c->A) {
        ub = 0; vb = 0;
      } else if (x < c->AB) {
        ub = 0; vb = 1;
      } else if (x < c->ABC) {
        ub = 1; vb = 0;
      } else {
        ub = 1; vb = 1;
      }
      u = (u << 1) | ub;
      v = (v << 1) | vb;
    }
    if (c->perm) {
      u = c->perm[u];
      v = c->perm[v];
    }
    c->src[e] = u;
    c->dst[e] = v;
  }
}

/* Random permutation of [0, n) by Fisher-Yates with counter-based draws. */
int gg_permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
  for (uint32_t i = 0; i < n; ++i) perm[i] = i;
  for (uint32_t i = n; i > 1; --i) {
    uint32_t j = gg_below(gg_rand(seed, 3, i - 1), i);
    uint32_t t = perm[i - 1];
    perm[i - 1] = perm[j];
    perm[j] = t;
  }
  return 0;
}

/* nedges raw RMAT tuples on 2^scale vertices (self-loops and duplicates kept,
 * no noise), vertex ids optionally relabelled by a seeded permutation. */
int gg_rmat(int scale, uint64_t nedges, double a, double b, double c, uint64_t seed, int permute, uint32_t* src,
            uint32_t* dst, int nthreads) {
  if (scale < 1 || scale > 31) return -1;
  uint32_t n = 1u << scale;
  uint32_t* perm = NULL;
  if (permute) {
    perm = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!perm) return -1;
    gg_permutation(n, seed, perm);
  }
  gg_rmat_ctx ctx;
  ctx.scale = scale;
  ctx.seed = seed;
  ctx.A = (uint32_t)(a * 4294967296.0);
  ctx.AB = (uint32_t)((a + b) * 4294967296.0);
  ctx.ABC = (uint32_t)((a + b + c) * 4294967296.0);
  ctx.perm = perm;
  ctx.src = src;
  ctx.dst = dst;
  gg_parallel(nedges, nthreads, gg_rmat_range, &ctx);
  free(perm);
  return 0;
}

/* ------------------------------------------------------------- grid/Road */

/* side x side grid, 4-neighbour edges each deleted with probability p_del,
 * plus llround(diag_frac * |grid edges|) diagonal shortcuts from uniform
 * random cells to a uniform random in-range diagonal neighbour. Vertex id of
 * cell (r, c) is r*side + c. Writes at most cap tuples; *out_count gets the
 * number written. Returns -1 if cap is too small. */
int gg_grid(uint32_t side, double p_del, double diag_frac, uint64_t seed, uint32_t* src, uint32_t* dst, uint64_t cap,
            uint64_t* out_count) {
  uint64_t S = side;
  uint64_t nh = S * (S - 1); /* horizontal edges */
  uint64_t ne = 2 * nh;
  uint64_t k = 0;
  for (uint64_t idx = 0; idx < ne; ++idx) {
    if (gg_unit(gg_rand(seed, 4, idx)) < p_del) continue;
    uint64_t a, b;
    if (idx < nh) {
      uint64_t r = idx / (S - 1), c = idx % (S - 1);
      a = r * S + c;
      b = a + 1;
    } else {
      uint64_t j = idx - nh;
      uint64_t r = j / S, c = j % S;
      a = r * S + c;
      b = a + S;
    }
    if (k >= cap) return -1;
    src[k] = (uint32_t)a;
    dst[k] = (uint32_t)b;
    ++k;
  }
  uint64_t nd = (uint64_t)llround(diag_frac * (double)ne);
  static const int dr[4] = {-1, -1, 1, 1};
  static const int dc[4] = {-1, 1, -1, 1};
  for (uint64_t j = 0; j < nd; ++j) {
    uint64_t cell = (uint64_t)(((unsigned __int128)gg_rand(seed, 5, j) * (S * S)) >> 64);
    int64_t r = (int64_t)(cell / S), c = (int64_t)(cell % S);
    int opts[4], no = 0;
    for (int q = 0; q < 4; ++q) {
      int64_t rr = r + dr[q], cc = c + dc[q];
      if (rr >= 0 && rr < (int64_t)S && cc >= 0 && cc < (int64_t)S) opts[no++] = q;
    }
    if (no == 0) continue;
    int q = opts[gg_below(gg_rand(seed, 6, j), (uint64_t)no)];
    if (k >= cap) return -1;
    src[k] = (uint32_t)cell;
    dst[k] = (uint32_t)((uint64_t)(r + dr[q]) * S + (uint64_t)(c + dc[q]));
    ++k;
  }
  *out_count = k;
  return 0;
}

/* ------------------------------------------------------------- weights */

typedef struct {
  const uint32_t* src;
  const uint32_t* dst;
  uint32_t* w;
  uint64_t seed;
  uint32_t wmin, wmax;
  double mu, sigma;
  int kind;  /* 0 uniform, 1 log-normal, 2 discretize(x, power), 3 converge(x, pivot) */
  uint32_t power;
  double pivot;
} gg_w_ctx;

/* The benchmark graphs' weight x, uniform in (0,1], per unordered pair. */
static inline double gg_unit_weight(uint64_t seed, uint64_t key) { return 1.0 - gg_unit(gg_rand(seed, 10, key)); }

/* Eq. 7: discretize(x, y) = 1 + x (2^y - 2), rounded to the nearest integer
 * (halves up): the 2^y - 1 integers 1 .. 2^y - 1 for x in (0, 1]. */
static inline uint32_t gg_discretize(double x, uint32_t y) {
  const double span = (double)((1ull << y) - 2);
  uint64_t q = (uint64_t)floor(x * span + 0.5);
  if (q > (1ull << y) - 2) q = (1ull << y) - 2;
  return (uint32_t)(1 + q);
}

/* Eq. 8: converge(x, y), a bell-shaped weight in [0, 1] with its peak and
 * median at the pivot y. */
static inline double gg_converge(double x, double y) {
  const double t = (1.0 - 2.0 * x) * (1.0 - 2.0 * x);
  return x <= 0.5 ? y - y * t : y + (1.0 - y) * t;
}

static inline uint64_t gg_pair_key(uint32_t u, uint32_t v) {
  return u < v ? ((uint64_t)u << 32) | v : ((uint64_t)v << 32) | u;
}

static void gg_w_range(void* p, uint64_t lo, uint64_t hi) {
  gg_w_ctx* c = (gg_w_ctx*)p;
  uint64_t range = (uint64_t)c->wmax - c->wmin + 1;
  for (uint64_t e = lo; e < hi; ++e) {
    uint64_t key = gg_pair_key(c->src[e], c->dst[e]);
    if (c->kind == 0) {
      c->w[e] = c->wmin + gg_below(gg_rand(c->seed, 7, key), range);
    } else if (c->kind == 2) {
      c->w[e] = gg_discretize(gg_unit_weight(c->seed, key), c->power);
    } else if (c->kind == 3) {  /* the real weight quantised to 1..65535 by discretize(., 16) */
      c->w[e] = gg_discretize(gg_converge(gg_unit_weight(c->seed, key), c->pivot), 16);
    } else {
      double u1 = gg_unit(gg_rand(c->seed, 8, key));
      double u2 = gg_unit(gg_rand(c->seed, 9, key));
      double z = sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586 * u2);
      double x = exp(c->mu + c->sigma * z);
      long long q = llround(x);
      if (x > 4.0e18) q = (long long)c->wmax;
      if (q < (long long)c->wmin) q = c->wmin;
      if (q > (long long)c->wmax) q = c->wmax;
      c->w[e] = (uint32_t)q;
    }
  }
}

/* Integer weight uniform in [wmin, wmax], a function of the unordered pair. */
void gg_weights_uniform(uint64_t ne, const uint32_t* src, const uint32_t* dst, uint64_t seed, uint32_t wmin,
                        uint32_t wmax, uint32_t* w, int nthreads) {
  gg_w_ctx c = {src, dst, w, seed, wmin, wmax, 0.0, 0.0, 0, 0, 0.0};
  gg_parallel(ne, nthreads, gg_w_range, &c);
}

/* clamp(llround(exp(mu + sigma*Z)), wmin, wmax), Z standard normal by the
 * Box-Muller transform, a function of the unordered pair. */
void gg_weights_lognormal(uint64_t ne, const uint32_t* src, const uint32_t* dst, uint64_t seed, double mu,
                          double sigma, uint32_t wmin, uint32_t wmax, uint32_t* w, int nthreads) {
  gg_w_ctx c = {src, dst, w, seed, wmin, wmax, mu, sigma, 1, 0, 0.0};
  gg_parallel(ne, nthreads, gg_w_range, &c);
}

/* The paper's power variants (Section 4.2): discretize(x, power) of Eq. 7,
 * rounded, with x uniform in (0,1] per unordered pair; power in 1..31. */
void gg_weights_discretize(uint64_t ne, const uint32_t* src, const uint32_t* dst, uint64_t seed, uint32_t power,
                           uint32_t* w, int nthreads) {
  gg_w_ctx c = {src, dst, w, seed, 1, 0, 0.0, 0.0, 2, power, 0.0};
  gg_parallel(ne, nthreads, gg_w_range, &c);
}

/* The paper's pivot variants (Section 4.2): converge(x, pivot) of Eq. 8 with x
 * uniform in (0,1] per unordered pair, then discretize(., 16) to integers
 * 1..65535 (the path takes integer weights). */
void gg_weights_converge(uint64_t ne, const uint32_t* src, const uint32_t* dst, uint64_t seed, double pivot,
                         uint32_t* w, int nthreads) {
  gg_w_ctx c = {src, dst, w, seed, 1, 0, 0.0, 0.0, 3, 0, pivot};
  gg_parallel(ne, nthreads, gg_w_range, &c);
}

/* Eq. 7 and Eq. 8 on single values (for tests of the transforms). */
uint32_t gg_discretize_value(double x, uint32_t power) { return gg_discretize(x, power); }
double gg_converge_value(double x, double pivot) { return gg_converge(x, pivot); }

/* ------------------------------------------------------------- sources */

static uint32_t gg_find(uint32_t* parent, uint32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

/* count sources, each uniform over the eligible vertices, drawn in order with
 * rejection (repeats allowed across draws only if count exceeds the pool).
 * mode 0: vertices with at least one non-loop edge; mode 1: vertices of the
 * largest connected component (ties: the component of the smallest root id).
 * Returns the number of eligible vertices, or -1 on failure. */
int64_t gg_pick_sources(uint32_t n, uint64_t ne, const uint32_t* src, const uint32_t* dst, uint32_t count,
                        uint64_t seed, int mode, uint32_t* out) {
  uint8_t* ok = (uint8_t*)calloc(n ? n : 1, 1);
  if (!ok) return -1;
  int64_t pool = 0;
  if (mode == 0) {
    for (uint64_t e = 0; e < ne; ++e) {
      if (src[e] != dst[e]) {
        ok[src[e]] = 1;
        ok[dst[e]] = 1;
      }
    }
  } else {
    uint32_t* parent = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    uint32_t* size = (uint32_t*)calloc(n ? n : 1, sizeof(uint32_t));
    if (!parent || !size) {
      free(ok); free(parent); free(size);
      return -1;
    }
    for (uint32_t i = 0; i < n; ++i) parent[i] = i;
    for (uint64_t e = 0; e < ne; ++e) {
      uint32_t a = gg_find(parent, src[e]), b = gg_find(parent, dst[e]);
      if (a != b) {
        if (a < b) parent[b] = a;
        else parent[a] = b;
      }
    }
    uint32_t best = 0, bestsz = 0;
    for (uint32_t i = 0; i < n; ++i) size[gg_find(parent, i)]++;
    for (uint32_t i = 0; i < n; ++i)
      if (size[i] > bestsz) {
        bestsz = size[i];
        best = i;
      }
    for (uint32_t i = 0; i < n; ++i) ok[i] = gg_find(parent, i) == best && bestsz > 1;
    free(parent);
    free(size);
  }
  for (uint32_t i = 0; i < n; ++i) pool += ok[i];
  if (pool == 0) {
    free(ok);
    return 0;
  }
  uint64_t i = 0;
  for (uint32_t k = 0; k < count;) {
    uint32_t x = gg_below(gg_rand(seed, 10, i++), n);
    if (ok[x]) out[k++] = x;
  }
  free(ok);
  return pool;
}

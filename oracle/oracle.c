/*
 * CPU oracle for the EIC shortest-path method (Yu, Wang, Luo, "A Heuristic
 * Algorithm for Shortest Path Search", arXiv 2506.19349).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * execute this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it. It shares no code with the CUDA path.
 *
 * Contents, each written from the paper's definitions:
 *   - its own CSR builder (symmetrise, drop self-loops, keep the minimum weight
 *     of duplicate pairs, rows sorted by (weight, neighbour));
 *   - the problem's plain definition dist[v] = lsp(s, v) (Section 2): binary
 *     heap Dijkstra with lazy deletion, Bellman-Ford and Floyd-Warshall
 *     (the two classical algorithms of Section 2.2) for tiny inputs, and an
 *     invariant checker that certifies a distance array;
 *   - the statistics of Section 3: maxW via the RtoW quantile table
 *     (Section 4.1), highD, sumD, the dynamic-stepping gap (Eq. 1-3) and the
 *     traversal-optimisation threshold computeST (Function 2, Eq. 4-6 with the
 *     clamping of Section 3.2, candidate grid of Section 4.1);
 *   - a sequential restatement of Algorithm 1 with Function 1, emitting the
 *     per-step trace <lb, ub, st> and the paper's counters (Section 4).
 *
 * Floating point: fp64, built with -ffp-contract=off so results are the same
 * on every host architecture.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_INF32 0xFFFFFFFFu
#define OG_INF_T ((int64_t)1 << 62)

/* --------------------------------------------------------------- graph */

typedef struct {
  uint32_t n;
  uint64_t nnz;   /* directed entries = 2m */
  uint64_t* row;  /* n + 1 */
  uint32_t* nbr;  /* nnz, rows sorted by (w, nbr) */
  uint32_t* w;    /* nnz */
  uint32_t maxw;  /* maxW(G,1) */
  uint32_t minw;
  uint32_t maxdeg;
} og_graph;

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

typedef struct {
  uint64_t* rp_raw;
  uint64_t* keys; /* (nbr << 32) | w */
  uint32_t* deg;
  uint32_t n;
  volatile uint64_t next; /* dynamic row chunk counter */
  int phase;              /* 0: sort by (nbr,w) + dedup; 1: sort by (w,nbr) */
} og_build_ctx;

static void* og_build_worker(void* p) {
  og_build_ctx* c = (og_build_ctx*)p;
  for (;;) {
    uint64_t lo = __atomic_fetch_add(&c->next, 4096, __ATOMIC_RELAXED);
    if (lo >= c->n) break;
    uint64_t hi = lo + 4096 < c->n ? lo + 4096 : c->n;
    for (uint64_t u = lo; u < hi; ++u) {
      uint64_t b = c->rp_raw[u], e = b + (c->phase == 0 ? (c->rp_raw[u + 1] - b) : c->deg[u]);
      uint64_t len = e - b;
      if (c->phase == 0) {
        qsort(c->keys + b, len, sizeof(uint64_t), cmp_u64);
        /* keep the first (minimum weight) entry of each neighbour */
        uint64_t k = 0;
        for (uint64_t i = 0; i < len; ++i) {
          if (k > 0 && (c->keys[b + k - 1] >> 32) == (c->keys[b + i] >> 32)) continue;
          c->keys[b + k++] = c->keys[b + i];
        }
        c->deg[u] = (uint32_t)k;
      } else {
        for (uint64_t i = b; i < e; ++i) c->keys[i] = (c->keys[i] << 32) | (c->keys[i] >> 32);
        qsort(c->keys + b, len, sizeof(uint64_t), cmp_u64);
      }
    }
  }
  return NULL;
}

static void og_build_run(og_build_ctx* c, int nthreads) {
  c->next = 0;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 128) nthreads = 128;
  pthread_t th[128];
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, og_build_worker, c);
  og_build_worker(c);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

void og_free(og_graph* g) {
  if (!g) return;
  free(g->row);
  free(g->nbr);
  free(g->w);
  free(g);
}

/* Build the undirected CSR from ne raw tuples (src[e], dst[e], w[e]).
 * Self-loops are dropped; a pair given several times keeps its smallest
 * weight; every pair appears in both rows. *err: 0 ok, 1 bad argument
 * (endpoint >= n, weight 0), 2 out of memory. */
og_graph* og_build(uint32_t n, uint64_t ne, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                   int nthreads, int* err) {
  *err = 0;
  for (uint64_t e = 0; e < ne; ++e) {
    if (src[e] >= n || dst[e] >= n || w[e] == 0) {
      *err = 1;
      return NULL;
    }
  }
  og_graph* g = (og_graph*)calloc(1, sizeof(og_graph));
  uint64_t* rp_raw = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  uint32_t* deg = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
  if (!g || !rp_raw || !deg) goto oom;
  g->n = n;
  for (uint64_t e = 0; e < ne; ++e) {
    if (src[e] == dst[e]) continue;
    rp_raw[src[e] + 1]++;
    rp_raw[dst[e] + 1]++;
  }
  for (uint32_t u = 0; u < n; ++u) rp_raw[u + 1] += rp_raw[u];
  uint64_t* keys = (uint64_t*)malloc((size_t)(rp_raw[n] ? rp_raw[n] : 1) * sizeof(uint64_t));
  uint64_t* cur = (uint64_t*)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
  if (!keys || !cur) {
    free(keys);
    free(cur);
    goto oom;
  }
  memcpy(cur, rp_raw, (size_t)n * sizeof(uint64_t));
  for (uint64_t e = 0; e < ne; ++e) {
    uint32_t a = src[e], b = dst[e];
    if (a == b) continue;
    keys[cur[a]++] = ((uint64_t)b << 32) | w[e];
    keys[cur[b]++] = ((uint64_t)a << 32) | w[e];
  }
  free(cur);
  og_build_ctx ctx;
  ctx.rp_raw = rp_raw;
  ctx.keys = keys;
  ctx.deg = deg;
  ctx.n = n;
  ctx.phase = 0;
  og_build_run(&ctx, nthreads);
  ctx.phase = 1;
  og_build_run(&ctx, nthreads);
  g->row = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!g->row) {
    free(keys);
    goto oom;
  }
  g->row[0] = 0;
  for (uint32_t u = 0; u < n; ++u) g->row[u + 1] = g->row[u] + deg[u];
  g->nnz = g->row[n];
  g->nbr = (uint32_t*)malloc((size_t)(g->nnz ? g->nnz : 1) * sizeof(uint32_t));
  g->w = (uint32_t*)malloc((size_t)(g->nnz ? g->nnz : 1) * sizeof(uint32_t));
  if (!g->nbr || !g->w) {
    free(keys);
    goto oom;
  }
  g->maxw = 0;
  g->minw = OG_INF32;
  g->maxdeg = 0;
  for (uint32_t u = 0; u < n; ++u) {
    uint64_t b = rp_raw[u];
    if (deg[u] > g->maxdeg) g->maxdeg = deg[u];
    for (uint32_t i = 0; i < deg[u]; ++i) {
      uint64_t k = keys[b + i]; /* (w << 32) | nbr */
      uint64_t o = g->row[u] + i;
      g->w[o] = (uint32_t)(k >> 32);
      g->nbr[o] = (uint32_t)k;
      if (g->w[o] > g->maxw) g->maxw = g->w[o];
      if (g->w[o] < g->minw) g->minw = g->w[o];
    }
  }
  if (g->nnz == 0) g->minw = 0;
  free(keys);
  free(rp_raw);
  free(deg);
  return g;
oom:
  *err = 2;
  free(rp_raw);
  free(deg);
  og_free(g);
  return NULL;
}

uint32_t og_n(const og_graph* g) { return g->n; }
uint64_t og_nnz(const og_graph* g) { return g->nnz; }
uint32_t og_maxw(const og_graph* g) { return g->maxw; }
uint32_t og_maxdeg(const og_graph* g) { return g->maxdeg; }

void og_export(const og_graph* g, uint64_t* row, uint32_t* nbr, uint32_t* w) {
  memcpy(row, g->row, ((size_t)g->n + 1) * sizeof(uint64_t));
  memcpy(nbr, g->nbr, (size_t)g->nnz * sizeof(uint32_t));
  memcpy(w, g->w, (size_t)g->nnz * sizeof(uint32_t));
}

static inline uint32_t og_deg(const og_graph* g, uint32_t u) { return (uint32_t)(g->row[u + 1] - g->row[u]); }

/* Distances are reported as uint32 with +inf = 0xFFFFFFFF. The arithmetic is
 * exact in 64 bits; a result counts as overflowing when the largest finite
 * shortest distance plus maxW(G,1) reaches 0xFFFFFFFF, the range in which the
 * termination test of Algorithm 1 (max finite dist + maxW(G,1) < lb) can no
 * longer be evaluated in 32 bits. */
static int og_overflowed(const og_graph* g, const uint64_t* d64) {
  uint64_t mx = 0;
  int any = 0;
  for (uint32_t v = 0; v < g->n; ++v)
    if (d64[v] != UINT64_MAX) {
      any = 1;
      if (d64[v] > mx) mx = d64[v];
    }
  return any && mx + g->maxw >= OG_INF32;
}

static void og_to32(uint32_t n, const uint64_t* d64, uint32_t* dist) {
  for (uint32_t v = 0; v < n; ++v) dist[v] = d64[v] >= OG_INF32 ? OG_INF32 : (uint32_t)d64[v];
}

/* ------------------------------------------------------------ Dijkstra */

typedef struct {
  uint64_t d;
  uint32_t v;
} og_item;

typedef struct {
  og_item* a;
  uint64_t size, cap;
} og_heap;

static int og_heap_push(og_heap* h, uint64_t d, uint32_t v) {
  if (h->size == h->cap) {
    uint64_t nc = h->cap ? 2 * h->cap : 1024;
    og_item* na = (og_item*)realloc(h->a, (size_t)nc * sizeof(og_item));
    if (!na) return -1;
    h->a = na;
    h->cap = nc;
  }
  uint64_t i = h->size++;
  while (i > 0) {
    uint64_t p = (i - 1) / 2;
    if (h->a[p].d <= d) break;
    h->a[i] = h->a[p];
    i = p;
  }
  h->a[i].d = d;
  h->a[i].v = v;
  return 0;
}

static og_item og_heap_pop(og_heap* h) {
  og_item top = h->a[0];
  og_item last = h->a[--h->size];
  uint64_t i = 0;
  for (;;) {
    uint64_t l = 2 * i + 1;
    if (l >= h->size) break;
    uint64_t c = (l + 1 < h->size && h->a[l + 1].d < h->a[l].d) ? l + 1 : l;
    if (h->a[c].d >= last.d) break;
    h->a[i] = h->a[c];
    i = c;
  }
  if (h->size > 0) h->a[i] = last;
  return top;
}

/* dist[v] = lsp(s, v) by Dijkstra's algorithm with a binary heap and lazy
 * deletion. Returns 0, 3 on overflow (see og_overflowed), 1 bad source,
 * 2 out of memory. */
int og_dijkstra(const og_graph* g, uint32_t s, uint32_t* dist) {
  if (s >= g->n) return 1;
  uint64_t* d = (uint64_t*)malloc((size_t)g->n * sizeof(uint64_t));
  if (!d) return 2;
  for (uint32_t v = 0; v < g->n; ++v) d[v] = UINT64_MAX;
  og_heap h = {NULL, 0, 0};
  d[s] = 0;
  int rc = og_heap_push(&h, 0, s);
  while (rc == 0 && h.size > 0) {
    og_item it = og_heap_pop(&h);
    if (it.d > d[it.v]) continue;
    for (uint64_t i = g->row[it.v]; i < g->row[it.v + 1]; ++i) {
      uint64_t nd = it.d + g->w[i];
      uint32_t v = g->nbr[i];
      if (nd < d[v]) {
        d[v] = nd;
        if (og_heap_push(&h, nd, v)) {
          rc = 2;
          break;
        }
      }
    }
  }
  free(h.a);
  if (rc == 0) {
    og_to32(g->n, d, dist);
    if (og_overflowed(g, d)) rc = 3;
  }
  free(d);
  return rc;
}

typedef struct {
  const og_graph* g;
  const uint32_t* sources;
  uint32_t* dists;
  int* rcs;
  uint32_t k;
  volatile uint32_t next;
} og_many_ctx;

static void* og_many_worker(void* p) {
  og_many_ctx* c = (og_many_ctx*)p;
  for (;;) {
    uint32_t i = __atomic_fetch_add(&c->next, 1, __ATOMIC_RELAXED);
    if (i >= c->k) break;
    c->rcs[i] = og_dijkstra(c->g, c->sources[i], c->dists + (uint64_t)i * c->g->n);
  }
  return NULL;
}

/* k independent single-threaded Dijkstra runs, one source per thread. */
void og_dijkstra_many(const og_graph* g, uint32_t k, const uint32_t* sources, uint32_t* dists, int* rcs,
                      int nthreads) {
  og_many_ctx c = {g, sources, dists, rcs, k, 0};
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 128) nthreads = 128;
  pthread_t th[128];
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, og_many_worker, &c);
  og_many_worker(&c);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------- brute force on tiny inputs */

/* Bellman-Ford over the raw tuple list (both directions, loops ignored,
 * duplicates relaxed individually), n-1 passes. Independent of og_build. */
int og_bellman_ford(uint32_t n, uint64_t ne, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                    uint32_t s, uint32_t* dist) {
  if (s >= n) return 1;
  uint64_t* d = (uint64_t*)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
  if (!d) return 2;
  uint32_t maxw = 0;
  for (uint32_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
  d[s] = 0;
  for (uint64_t e = 0; e < ne; ++e)
    if (src[e] != dst[e] && w[e] > maxw) maxw = w[e];
  for (uint32_t it = 0; it + 1 < n; ++it) {
    int changed = 0;
    for (uint64_t e = 0; e < ne; ++e) {
      uint32_t a = src[e], b = dst[e];
      if (a == b) continue;
      if (d[a] != UINT64_MAX && d[a] + w[e] < d[b]) {
        d[b] = d[a] + w[e];
        changed = 1;
      }
      if (d[b] != UINT64_MAX && d[b] + w[e] < d[a]) {
        d[a] = d[b] + w[e];
        changed = 1;
      }
    }
    if (!changed) break;
  }
  og_to32(n, d, dist);
  uint64_t mx = 0;
  int any = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (d[v] != UINT64_MAX) {
      any = 1;
      if (d[v] > mx) mx = d[v];
    }
  free(d);
  return any && mx + maxw >= OG_INF32 ? 3 : 0;
}

/* Floyd-Warshall all pairs from the raw tuple list; writes row s. n <= 512. */
int og_floyd_warshall(uint32_t n, uint64_t ne, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                      uint32_t s, uint32_t* dist) {
  if (s >= n || n > 512) return 1;
  uint64_t* m = (uint64_t*)malloc((size_t)n * n * sizeof(uint64_t));
  if (!m) return 2;
  for (uint64_t i = 0; i < (uint64_t)n * n; ++i) m[i] = UINT64_MAX;
  for (uint32_t i = 0; i < n; ++i) m[(uint64_t)i * n + i] = 0;
  for (uint64_t e = 0; e < ne; ++e) {
    uint32_t a = src[e], b = dst[e];
    if (a == b) continue;
    if (w[e] < m[(uint64_t)a * n + b]) m[(uint64_t)a * n + b] = m[(uint64_t)b * n + a] = w[e];
  }
  for (uint32_t k = 0; k < n; ++k)
    for (uint32_t i = 0; i < n; ++i) {
      uint64_t ik = m[(uint64_t)i * n + k];
      if (ik == UINT64_MAX) continue;
      for (uint32_t j = 0; j < n; ++j) {
        uint64_t kj = m[(uint64_t)k * n + j];
        if (kj != UINT64_MAX && ik + kj < m[(uint64_t)i * n + j]) m[(uint64_t)i * n + j] = ik + kj;
      }
    }
  og_to32(n, m + (uint64_t)s * n, dist);
  free(m);
  return 0;
}

/* --------------------------------------------------- invariant checker */

/* Certifies dist as the shortest distances from s (positive weights):
 *   1: dist[s] != 0
 *   2: some entry (u,v,w) with dist[u] finite has dist[v] > dist[u] + w
 *   3: some finite v != s has no tight entry dist[u] + w == dist[v]
 *   4: finite/infinite disagrees with reachability from s (BFS)
 * Together 1-3 force dist[v] = lsp(s, v): 2 gives dist <= lsp along every
 * shortest path, 3 gives a path of length dist[v] by following tight entries
 * down strictly decreasing distances to s. Returns 0 if all hold, else the
 * first failing code, with the offending vertex in *bad. */
int og_check(const og_graph* g, uint32_t s, const uint32_t* dist, uint32_t* bad) {
  *bad = 0;
  if (s >= g->n) return 5;
  if (dist[s] != 0) {
    *bad = s;
    return 1;
  }
  for (uint32_t u = 0; u < g->n; ++u) {
    if (dist[u] == OG_INF32) continue;
    int tight = (u == s);
    for (uint64_t i = g->row[u]; i < g->row[u + 1]; ++i) {
      uint32_t v = g->nbr[i];
      uint64_t cand = (uint64_t)dist[u] + g->w[i];
      if ((uint64_t)dist[v] > cand) {
        *bad = v;
        return 2;
      }
      if (dist[v] != OG_INF32 && (uint64_t)dist[v] + g->w[i] == dist[u]) tight = 1;
    }
    if (!tight) {
      *bad = u;
      return 3;
    }
  }
  uint8_t* seen = (uint8_t*)calloc(g->n, 1);
  uint32_t* q = (uint32_t*)malloc((size_t)g->n * sizeof(uint32_t));
  if (!seen || !q) {
    free(seen);
    free(q);
    return 6;
  }
  uint64_t qh = 0, qt = 0;
  q[qt++] = s;
  seen[s] = 1;
  while (qh < qt) {
    uint32_t u = q[qh++];
    for (uint64_t i = g->row[u]; i < g->row[u + 1]; ++i)
      if (!seen[g->nbr[i]]) {
        seen[g->nbr[i]] = 1;
        q[qt++] = g->nbr[i];
      }
  }
  int rc = 0;
  for (uint32_t v = 0; v < g->n; ++v)
    if ((dist[v] != OG_INF32) != (seen[v] != 0)) {
      *bad = v;
      rc = 4;
      break;
    }
  free(seen);
  free(q);
  return rc;
}

/* parent[v]: the smallest-id u with dist[u] + w(u,v) == dist[v]; parent[s] =
 * s; 0xFFFFFFFF where v is unreachable (the paper's -1, Section 2). */
void og_parent(const og_graph* g, uint32_t s, const uint32_t* dist, uint32_t* parent) {
  for (uint32_t v = 0; v < g->n; ++v) {
    parent[v] = OG_INF32;
    if (v == s) {
      parent[v] = s;
      continue;
    }
    if (dist[v] == OG_INF32) continue;
    for (uint64_t i = g->row[v]; i < g->row[v + 1]; ++i) {
      uint32_t u = g->nbr[i];
      if (dist[u] != OG_INF32 && (uint64_t)dist[u] + g->w[i] == dist[v] && u < parent[v]) parent[v] = u;
    }
  }
}

/* ------------------------------------------------------------ statistics */

/* RtoW[i] = maxW(G, i/(R-1)) over the m undirected edge weights (Section 4.1).
 * maxW(G, ratio) is the smallest weight W with P(w <= W) >= ratio, i.e. the
 * ceil(ratio*m)-th smallest weight (the smallest one when ratio = 0). */
int og_rtow_from_weights(uint64_t m, const uint32_t* weights, uint32_t R, uint32_t* rtow) {
  if (m == 0 || R < 2) return 1;
  uint64_t* s = (uint64_t*)malloc((size_t)m * sizeof(uint64_t));
  if (!s) return 2;
  for (uint64_t i = 0; i < m; ++i) s[i] = weights[i];
  qsort(s, m, sizeof(uint64_t), cmp_u64);
  for (uint32_t i = 0; i < R; ++i) {
    uint64_t rank = ((uint64_t)i * m + (R - 2)) / (R - 1); /* ceil(i*m/(R-1)) */
    rtow[i] = (uint32_t)s[rank ? rank - 1 : 0];
  }
  free(s);
  return 0;
}

/* RtoW of the graph: the weight of each undirected edge counted once. */
int og_rtow(const og_graph* g, uint32_t R, uint32_t* rtow) {
  uint64_t m = g->nnz / 2, k = 0;
  uint32_t* ws = (uint32_t*)malloc((size_t)(m ? m : 1) * sizeof(uint32_t));
  if (!ws) return 2;
  for (uint32_t u = 0; u < g->n; ++u)
    for (uint64_t i = g->row[u]; i < g->row[u + 1]; ++i)
      if (u < g->nbr[i]) ws[k++] = g->w[i];
  int rc = og_rtow_from_weights(m, ws, R, rtow);
  free(ws);
  return rc;
}

/* highD over a degree multiset given as a histogram cnt[0..maxdeg] (Section 3:
 * the threshold t splitting the set into degrees < t and >= t with the
 * smallest difference of total degree). Candidates are the degree values
 * present (degree 0 contributes nothing and is never a candidate); ties keep
 * the smaller t; 0 when the total degree is 0. */
uint64_t og_highd_hist(uint64_t maxdeg, const uint64_t* cnt) {
  uint64_t total = 0;
  for (uint64_t t = 1; t <= maxdeg; ++t) total += cnt[t] * t;
  if (total == 0) return 0;
  uint64_t best_t = 0, low = 0;
  uint64_t best_diff = UINT64_MAX;
  for (uint64_t t = 1; t <= maxdeg; ++t) {
    if (cnt[t] == 0) continue;
    uint64_t high = total - low;
    uint64_t diff = high > low ? high - low : low - high;
    if (diff < best_diff) {
      best_diff = diff;
      best_t = t;
    }
    low += cnt[t] * t;
  }
  return best_t;
}

/* highD of an explicit degree list. */
uint64_t og_highd_list(uint64_t k, const uint32_t* degs) {
  uint64_t mx = 0;
  for (uint64_t i = 0; i < k; ++i)
    if (degs[i] > mx) mx = degs[i];
  uint64_t* cnt = (uint64_t*)calloc(mx + 1, sizeof(uint64_t));
  if (!cnt) return 0;
  for (uint64_t i = 0; i < k; ++i) cnt[degs[i]]++;
  uint64_t r = og_highd_hist(mx, cnt);
  free(cnt);
  return r;
}

/* Eq. 1-3: gap(x) from sumD(x), highD(x), the total degree 2|E| and RtoW.
 *   prob  = min(beta, max(sumD, 2|E| - sumD) / (2|E|))           (Eq. 1)
 *   ratio = 1 - (1 - prob)^(1 / (prob * highD))                  (Eq. 2)
 *   gap   = maxW(G,1) if highD <= alpha, else maxW(G, ratio)     (Eq. 3)
 * maxW(G, ratio) is read from RtoW at index floor(ratio * (R - 1)); Eq. 2 is
 * evaluated as -expm1(log1p(-prob) / (prob * highD)). *idx_out receives the
 * RtoW index used (R-1 for the highD <= alpha branch). */
int64_t og_gap(uint64_t sumd, uint64_t highd, uint64_t two_m, uint32_t alpha, double beta, uint32_t R,
               const uint32_t* rtow, uint32_t* idx_out, double* ratio_out) {
  if (highd <= alpha || two_m == 0) {
    if (idx_out) *idx_out = R - 1;
    if (ratio_out) *ratio_out = 1.0;
    return rtow[R - 1];
  }
  uint64_t big = sumd > two_m - sumd ? sumd : two_m - sumd;
  double frac = (double)big / (double)two_m;
  double prob = frac < beta ? frac : beta;
  double ratio = -expm1(log1p(-prob) / (prob * (double)highd));
  double pos = ratio * (double)(R - 1);
  uint32_t idx = pos <= 0.0 ? 0 : (pos >= (double)(R - 1) ? R - 1 : (uint32_t)floor(pos));
  if (idx_out) *idx_out = idx;
  if (ratio_out) *ratio_out = ratio;
  return rtow[idx];
}

/* Profit of candidate x for the pair <lb, y> (Section 3.2): with
 *   x' = max(x, lb - maxW), ub0 = min(y, lb + maxW), ub1 = min(y, x' + maxW)
 *   D  = sumD(x') - sumD(lb)
 *   pushed = (ub0 - lb) * D / maxW                     (Eq. 4 at <x', lb, ub0>)
 *   pulled = (ub1 - x') * sumD(lb) / maxW              (Eq. 5 at <x', lb, ub1>)
 *   long   = pulled * D / (2|E|)                       (Eq. 6 at <x', lb, ub1>)
 *   profit = pushed - long - pulled
 * Each operation is one IEEE double operation in the order written. */
double og_profit(int64_t x, int64_t lb, int64_t y, uint64_t dsum, uint64_t sumd_lb, uint32_t maxw,
                 uint64_t two_m) {
  int64_t xc = x > lb - (int64_t)maxw ? x : lb - (int64_t)maxw;
  int64_t ub0 = y < lb + (int64_t)maxw ? y : lb + (int64_t)maxw;
  int64_t ub1 = y < xc + (int64_t)maxw ? y : xc + (int64_t)maxw;
  double pushed = ((double)(ub0 - lb) * (double)dsum) / (double)maxw;
  double pulled = ((double)(ub1 - xc) * (double)sumd_lb) / (double)maxw;
  double lng = (pulled * (double)dsum) / (double)two_m;
  return (pushed - lng) - pulled;
}

/* ------------------------------------------------- sequential Algorithm 1 */

typedef struct {
  uint32_t alpha;
  double beta;
  uint32_t ratio_num;
  uint32_t st_num;
} og_params;

typedef struct {
  int64_t lb, ub, st;  /* thresholds the step ran with (step 1: final ub) */
  int64_t gap_lb;      /* gap(lb) by Eq. 3 */
  uint64_t sumd_lb;    /* sumD(lb) */
  uint64_t highd_lb;   /* highD(lb) */
  uint64_t rounds;     /* relaxation rounds (synchronisations) */
  uint64_t settled;    /* vertices whose distance falls in [lb, ub) */
  uint64_t push_set;   /* |{x: lb0 <= dist[x] <= st}| at step start */
  uint64_t pull_set;   /* |{x: dist[x] > lb}| scanned by the pull, 0 without pull */
  uint64_t push_trav;  /* selected entries relaxed in push (all rounds) */
  uint64_t pull_trav;  /* candidate entries examined by the pull */
  uint64_t frontier;   /* sum over rounds of |Paths| */
  uint64_t improved;   /* successful relaxations (dist decreased) */
} og_step;

typedef struct {
  uint64_t steps, rounds, frontier, traversed, push_trav, pull_trav, improved;
  int64_t st0, st1;
} og_totals;

/* first index i in [b, e) of the weight-sorted row with w[i] >= t */
static uint64_t og_lower(const og_graph* g, uint64_t b, uint64_t e, int64_t t) {
  if (t <= 0) return b;
  while (b < e) {
    uint64_t mid = b + (e - b) / 2;
    if ((int64_t)g->w[mid] < t) b = mid + 1;
    else e = mid;
  }
  return b;
}

static inline int64_t og_d(uint32_t x) { return x == OG_INF32 ? OG_INF_T : (int64_t)x; }

/* sumD(x) and the unsettled degree histogram for highD(x): VS(x) is the set
 * of vertices with dist >= x, +inf included (at a step boundary every vertex
 * with lsp < x is final and every other one has dist >= lsp >= x). */
static void og_vs_stats(const og_graph* g, const uint32_t* dist, int64_t x, uint64_t* cnt, uint64_t* sumd,
                        uint64_t* highd) {
  memset(cnt, 0, ((size_t)g->maxdeg + 1) * sizeof(uint64_t));
  uint64_t s = 0;
  for (uint32_t v = 0; v < g->n; ++v)
    if (og_d(dist[v]) >= x) {
      uint32_t dg = og_deg(g, v);
      cnt[dg]++;
      s += dg;
    }
  *sumd = s;
  *highd = og_highd_hist(g->maxdeg, cnt);
}

/* Function 2, computeST(lb, ub): the selection threshold for the next pair
 * <ub, ub + gap(ub)>. Candidates are the grid x_k = st0 + floor(k (st1 - st0)
 * / ST_NUM), k = 0..ST_NUM, with x_k < ub (Section 4.1); the first maximum
 * with positive profit wins, else ub. */
static int64_t og_compute_st(const og_graph* g, const uint32_t* dist, int64_t ub, uint64_t sumd_ub, int64_t gap_lb,
                             int64_t gap_ub, int64_t st0, int64_t st1, uint32_t st_num, int64_t* sort_buf_d,
                             uint64_t* sort_buf_deg) {
  uint64_t two_m = g->nnz, m = g->nnz / 2;
  int64_t maxw = g->maxw;
  if (sumd_ub >= m || gap_lb == maxw) return ub;
  if (gap_ub == maxw) return ub - maxw;
  int64_t y = ub + gap_ub;
  /* D(x') = sum of degrees over x' <= dist < ub: settled vertices sorted by
   * distance with suffix sums, looked up by binary search */
  uint64_t k = 0;
  for (uint32_t v = 0; v < g->n; ++v)
    if (og_d(dist[v]) < ub) sort_buf_deg[k++] = ((uint64_t)dist[v] << 32) | og_deg(g, v);
  qsort(sort_buf_deg, k, sizeof(uint64_t), cmp_u64);
  /* suffix sums of degree by ascending distance */
  for (uint64_t i = 0; i < k; ++i) sort_buf_d[i] = (int64_t)(sort_buf_deg[i] >> 32);
  uint64_t* suf = (uint64_t*)malloc((size_t)(k + 1) * sizeof(uint64_t));
  suf[k] = 0;
  for (uint64_t i = k; i > 0; --i) suf[i - 1] = suf[i] + (sort_buf_deg[i - 1] & 0xFFFFFFFFull);
  int64_t st = ub;
  double best = 0.0;
  for (uint32_t j = 0; j <= st_num; ++j) {
    int64_t x = st0 + (int64_t)(((uint64_t)j * (uint64_t)(st1 - st0)) / st_num);
    if (x >= ub) continue;
    int64_t xc = x > ub - maxw ? x : ub - maxw;
    uint64_t lo = 0, hi = k; /* first settled with dist >= xc */
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (sort_buf_d[mid] < xc) lo = mid + 1;
      else hi = mid;
    }
    uint64_t dsum = suf[lo];
    double p = og_profit(x, ub, y, dsum, sumd_ub, (uint32_t)maxw, two_m);
    if (best < p) {
      best = p;
      st = x;
    }
  }
  free(suf);
  return st;
}

/* Sequential restatement of Algorithm 1 (with Function 1 and Function 2).
 * Readings where the text is silent or ambiguous:
 *   - the dynamic ub of Algorithm 1 applies to the first step only (the
 *     "first step" of Section 3.3); a later step starting at lb = 0 uses
 *     ub = lb + gap(lb);
 *   - highD(0) for the first step is taken over all vertices;
 *   - VS(x) includes unreachable vertices; sumD, highD at a step boundary use
 *     {dist >= x};
 *   - Function 2's candidate set is the ST_NUM grid of Section 4.1 between
 *     st0 (the first step's final ub) and st1 (the first scheduling threshold
 *     with sumD <= |E|), with the clamped estimates of Section 3.2.
 * Frontiers are processed in insertion order reading the latest distance.
 * Returns 0, 1 bad source, 2 out of memory, 3 overflow. trace may be NULL;
 * at most trace_cap rows are written and the step count is returned in
 * totals->steps. */
int og_eic(const og_graph* g, uint32_t s, const og_params* prm, uint32_t* dist, og_step* trace, uint64_t trace_cap,
           og_totals* totals) {
  if (s >= g->n) return 1;
  uint32_t n = g->n;
  uint64_t two_m = g->nnz, m = g->nnz / 2;
  int64_t maxw = g->maxw;
  uint32_t R = prm->ratio_num;
  memset(totals, 0, sizeof(*totals));
  totals->st0 = -1;
  totals->st1 = -1;
  for (uint32_t v = 0; v < n; ++v) dist[v] = OG_INF32;
  dist[s] = 0;
  if (two_m == 0) {
    totals->steps = 0;
    return 0;
  }
  uint32_t* rtow = (uint32_t*)malloc((size_t)R * sizeof(uint32_t));
  uint64_t* cnt = (uint64_t*)malloc(((size_t)g->maxdeg + 1) * sizeof(uint64_t));
  uint32_t* fr = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* nx = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint8_t* inx = (uint8_t*)calloc(n, 1);
  int64_t* sbd = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  uint64_t* sbg = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  int rc = 0;
  if (!rtow || !cnt || !fr || !nx || !inx || !sbd || !sbg) {
    rc = 2;
    goto done;
  }
  og_rtow(g, R, rtow);

  uint64_t sumd_lb, highd_lb;
  og_vs_stats(g, dist, 0, cnt, &sumd_lb, &highd_lb); /* VS(0) = V */
  uint64_t highd0 = highd_lb;
  int64_t gap_lb = og_gap(sumd_lb, highd_lb, two_m, prm->alpha, prm->beta, R, rtow, NULL, NULL);
  int64_t lb = 0, ub = OG_INF_T, st = 0;
  int64_t st0 = -1, st1 = -1;
  uint64_t step = 0;
  for (;;) {
    ++step;
    int first = (step == 1);
    og_step row;
    memset(&row, 0, sizeof(row));
    row.lb = lb;
    row.st = st;
    row.gap_lb = gap_lb;
    row.sumd_lb = sumd_lb;
    row.highd_lb = highd_lb;

    /* Function 1: initFrontiers(st, lb, ub) */
    int64_t lb0 = lb - maxw > 0 ? lb - maxw : 0;
    uint64_t nf = 0;
    for (uint32_t x = 0; x < n; ++x) {
      int64_t dx = og_d(dist[x]);
      if (dx >= lb0 && dx <= st && dx < OG_INF_T) {
        fr[nf++] = x;
        inx[x] = 1;
      }
    }
    row.push_set = nf;
    if (st != lb) {
      for (uint32_t u = 0; u < n; ++u) {
        if (og_d(dist[u]) <= lb) continue;
        row.pull_set++;
        uint64_t b = g->row[u], e = og_lower(g, g->row[u], g->row[u + 1], ub - st);
        row.pull_trav += e - b;
        for (uint64_t i = b; i < e; ++i) {
          int64_t dv = og_d(dist[g->nbr[i]]);
          if (dv >= st && dv < lb && dv + (int64_t)g->w[i] < ub && dv + (int64_t)g->w[i] < og_d(dist[u])) {
            dist[u] = (uint32_t)(dv + g->w[i]);
            row.improved++;
          }
        }
      }
    }
    for (uint32_t x = 0; x < n; ++x) {
      int64_t dx = og_d(dist[x]);
      if (dx >= lb && dx < ub && !inx[x]) {
        fr[nf++] = x;
        inx[x] = 1;
      }
    }
    for (uint64_t i = 0; i < nf; ++i) inx[fr[i]] = 0;

    /* rounds of edge relaxations */
    while (nf > 0) {
      row.rounds++;
      uint64_t nn = 0;
      for (uint64_t i = 0; i < nf; ++i) {
        uint32_t u = fr[i];
        if (dist[u] > 0 && og_deg(g, u) == 1) continue; /* Paths excludes leaves */
        row.frontier++;
        int64_t d = dist[u];
        uint64_t b = og_lower(g, g->row[u], g->row[u + 1], lb - d);
        uint64_t e = og_lower(g, b, g->row[u + 1], ub - d);
        row.push_trav += e - b;
        for (uint64_t k = b; k < e; ++k) {
          uint32_t v = g->nbr[k];
          int64_t nd = d + (int64_t)g->w[k];
          if (nd >= OG_INF32) continue; /* beyond 32-bit range: reported below */
          if (nd < og_d(dist[v])) {
            dist[v] = (uint32_t)nd;
            row.improved++;
            if (!inx[v]) {
              inx[v] = 1;
              nx[nn++] = v;
            }
          }
        }
      }
      for (uint64_t i = 0; i < nn; ++i) inx[nx[i]] = 0;
      if (first) {
        int64_t best = OG_INF_T;
        for (uint32_t x = 0; x < n; ++x)
          if (og_deg(g, x) >= highd0 && og_d(dist[x]) < best) best = og_d(dist[x]);
        ub = best;
      }
      uint32_t* t = fr;
      fr = nx;
      nx = t;
      nf = nn;
    }

    row.ub = ub;
    /* max{dist[x] < +inf}: the settled part (dist < ub, final) and whether any
     * finite tentative distance >= ub remains (only the first step leaves
     * such values, since later windows create distances below ub) */
    int64_t maxfin = -1;
    int unsettled_finite = 0;
    for (uint32_t x = 0; x < n; ++x) {
      int64_t dx = og_d(dist[x]);
      if (dx >= lb && dx < ub) row.settled++;
      if (dx < ub && dx > maxfin) maxfin = dx;
      if (dx >= ub && dx < OG_INF_T) unsettled_finite = 1;
    }
    if (first) st0 = ub;
    totals->rounds += row.rounds;
    totals->frontier += row.frontier;
    totals->push_trav += row.push_trav;
    totals->pull_trav += row.pull_trav;
    totals->improved += row.improved;
    if (trace && step <= trace_cap) trace[step - 1] = row;

    if (maxfin + maxw >= (int64_t)OG_INF32) {
      rc = 3;
      break;
    }
    if (!unsettled_finite && maxfin + maxw < ub) break; /* termination with lb := ub */

    /* step boundary: <st, lb, ub> <- <computeST(lb, ub), ub, ub + gap(ub)> */
    uint64_t sumd_ub, highd_ub;
    og_vs_stats(g, dist, ub, cnt, &sumd_ub, &highd_ub);
    int64_t gap_ub = og_gap(sumd_ub, highd_ub, two_m, prm->alpha, prm->beta, R, rtow, NULL, NULL);
    if (st1 < 0 && sumd_ub <= m) st1 = ub;
    int64_t st_next = og_compute_st(g, dist, ub, sumd_ub, gap_lb, gap_ub, st0, st1, prm->st_num, sbd, sbg);
    st = st_next;
    lb = ub;
    ub = ub + gap_ub;
    sumd_lb = sumd_ub;
    highd_lb = highd_ub;
    gap_lb = gap_ub;
  }
  totals->steps = step;
  totals->traversed = totals->push_trav + totals->pull_trav;
  totals->st0 = st0;
  totals->st1 = st1;
done:
  free(rtow);
  free(cnt);
  free(fr);
  free(nx);
  free(inx);
  free(sbd);
  free(sbg);
  return rc;
}

/* sumD(x), highD(x) of a final distance array: the statistics of the set
 * {v : lsp(s, v) >= x}, for checking a trace against exact distances. */
void og_stats_at(const og_graph* g, const uint32_t* dist, int64_t x, uint64_t* sumd, uint64_t* highd) {
  uint64_t* cnt = (uint64_t*)malloc(((size_t)g->maxdeg + 1) * sizeof(uint64_t));
  og_vs_stats(g, dist, x, cnt, sumd, highd);
  free(cnt);
}

/* Sum of degrees over {v : x <= lsp(s, v) < y}. */
uint64_t og_degree_between(const og_graph* g, const uint32_t* dist, int64_t x, int64_t y) {
  uint64_t s = 0;
  for (uint32_t v = 0; v < g->n; ++v) {
    int64_t d = og_d(dist[v]);
    if (d >= x && d < y) s += og_deg(g, v);
  }
  return s;
}

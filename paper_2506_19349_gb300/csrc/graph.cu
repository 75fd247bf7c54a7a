// Device CSR builder and graph object (preprocessing of Section 4.1: every
// vertex's incident edges sorted in weight order, and the edge-weight
// distribution quantised into RtoW[RATIO_NUM]).
//
// Pipeline, all on the device:
//   1. validate tuples, drop self-loops, pack each pair as (min, max) keys;
//   2. radix-sort the keys, keep the smallest weight of each distinct pair;
//   3. degrees -> row offsets (exclusive scan);
//   4. emit both directions of every pair in pair order (which lists each
//      row's neighbours in ascending order) and stably radix-sort by
//      (row, weight): rows end up sorted by (weight, neighbour);
//   5. RtoW from the sorted undirected weights; distinct-degree tables and
//      highD(0) for the step statistics; the list of non-isolated vertices.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "graph.h"
#include "radix.cuh"
#include "stats.cuh"

using namespace eic;

namespace {

constexpr int kThreads = 256;

inline int grid_for(uint64_t n, int threads = kThreads) {
  uint64_t b = (n + threads - 1) / threads;
  if (b > 65535ull * 32) b = 65535ull * 32;
  return (int)(b ? b : 1);
}

inline int bits_for(uint64_t x) {  // bits needed to represent values 0..x
  int b = 0;
  while (b < 64 && (x >> b) != 0) ++b;
  return b;
}

__global__ void k_canon(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                        const uint32_t* __restrict__ w, uint64_t T, uint32_t n, int vbits, uint64_t* keys,
                        uint32_t* vals, uint32_t* count, int* err) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
       i - threadIdx.x < T; i += stride) {
    bool valid = i < T;
    uint32_t a = 0, b = 0, ww = 0;
    if (valid) {
      a = src[i];
      b = dst[i];
      ww = w[i];
      if (a >= n || b >= n || ww == 0) {
        atomicExch(err, 1);
        valid = false;
      }
    }
    bool keep = valid && a != b;
    uint32_t slot = warp_append(keep, count);
    if (keep) {
      uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
      keys[slot] = ((uint64_t)lo << vbits) | hi;
      vals[slot] = ww;
    }
  }
}

__global__ void k_heads(const uint64_t* __restrict__ keys, uint64_t K, uint32_t* flags) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// One thread per distinct pair: minimum weight over its run of duplicates.
__global__ void k_dedup(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                        const uint32_t* __restrict__ flags, const uint64_t* __restrict__ pos, uint64_t K,
                        uint64_t* ukeys, uint32_t* uw) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
    if (!flags[i]) continue;
    uint64_t k = keys[i];
    uint32_t best = vals[i];
    for (uint64_t j = i + 1; j < K && keys[j] == k; ++j) best = vals[j] < best ? vals[j] : best;
    ukeys[pos[i]] = k;
    uw[pos[i]] = best;
  }
}

__global__ void k_degrees(const uint64_t* __restrict__ ukeys, const uint32_t* __restrict__ uw, uint64_t m, int vbits,
                          uint32_t* deg, uint32_t* wmax, uint32_t* wmin) {
  uint32_t lmax = 0, lmin = 0xFFFFFFFFu;
  const uint64_t vmask = (1ull << vbits) - 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = ukeys[i];
    atomicAdd(&deg[k >> vbits], 1u);
    atomicAdd(&deg[k & vmask], 1u);
    uint32_t x = uw[i];
    lmax = x > lmax ? x : lmax;
    lmin = x < lmin ? x : lmin;
  }
  for (int o = 16; o > 0; o >>= 1) {
    lmax = max(lmax, __shfl_xor_sync(EIC_FULL_MASK, lmax, o));
    lmin = min(lmin, __shfl_xor_sync(EIC_FULL_MASK, lmin, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(wmax, lmax);
    atomicMin(wmin, lmin);
  }
}

// Both directions of pair i at positions 2i, 2i+1 in internal ids; sort key (row, weight).
__global__ void k_emit(const uint64_t* __restrict__ ukeys, const uint32_t* __restrict__ uw, uint64_t m, int vbits,
                       const uint32_t* __restrict__ orig2int, int wbits, uint64_t* keys, uint32_t* vals) {
  const uint64_t vmask = (1ull << vbits) - 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = ukeys[i];
    uint32_t a = orig2int[k >> vbits], b = orig2int[k & vmask], w = uw[i];
    keys[2 * i] = ((uint64_t)a << wbits) | w;
    vals[2 * i] = b;
    keys[2 * i + 1] = ((uint64_t)b << wbits) | w;
    vals[2 * i + 1] = a;
  }
}

// key of non-isolated vertex v: (maxdeg - deg(v), v), at its compacted position
__global__ void k_relabel_keys(const uint32_t* __restrict__ deg, const uint32_t* __restrict__ flags,
                               const uint64_t* __restrict__ pos, uint32_t n, uint32_t maxdeg, int vbits,
                               uint64_t* keys) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    if (flags[v]) keys[pos[v]] = ((uint64_t)(maxdeg - deg[v]) << vbits) | v;
}

__global__ void k_relabel_maps(const uint64_t* __restrict__ keys, uint32_t ni, int vbits, uint32_t* int2orig,
                               uint32_t* orig2int) {
  const uint64_t vmask = (1ull << vbits) - 1;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)(keys[i] & vmask);
    int2orig[i] = v;
    orig2int[v] = i;
  }
}

__global__ void k_gather_u32(const uint32_t* __restrict__ src, const uint32_t* __restrict__ idx, uint32_t cnt,
                             uint32_t* out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) out[i] = src[idx[i]];
}

// nz[i] = {i, smallest weight of row i, row begin, row end} for every internal vertex
__global__ void k_nz_fill(const uint32_t* __restrict__ row, const uint2* __restrict__ adj, uint32_t ni, uint4* nz) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x)
    nz[i] = make_uint4(i, adj[row[i]].y, row[i], row[i + 1]);
}

__global__ void k_pack_adj(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t E,
                           int wbits, uint2* adj) {
  const uint64_t wmask = wbits >= 64 ? ~0ull : ((1ull << wbits) - 1);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < E; i += (uint64_t)gridDim.x * blockDim.x)
    adj[i] = make_uint2(vals[i], (uint32_t)(keys[i] & wmask));
}

__global__ void k_weights_to_keys(const uint32_t* __restrict__ uw, uint64_t m, uint64_t* keys) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    keys[i] = uw[i];
}

// RtoW[i] = the ceil(i m / (R-1))-th smallest weight (the smallest for i = 0).
__global__ void k_rtow(const uint64_t* __restrict__ sorted_w, uint64_t m, uint32_t* rtow) {
  const uint32_t R = EIC_RATIO_NUM;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) {
    uint64_t rank = ((uint64_t)i * m + (R - 2)) / (R - 1);
    rtow[i] = (uint32_t)sorted_w[rank ? rank - 1 : 0];
  }
}

__global__ void k_max_u32(const uint32_t* __restrict__ a, uint64_t n, uint32_t* out) {
  uint32_t lmax = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    lmax = a[i] > lmax ? a[i] : lmax;
  for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(EIC_FULL_MASK, lmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, lmax);
}

// Degree histogram; degrees below 1024 are counted in shared memory first.
__global__ void k_deg_hist(const uint32_t* __restrict__ deg, uint32_t n, uint32_t* hist) {
  __shared__ uint32_t s_h[1024];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_h[i] = 0;
  __syncthreads();
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t d = deg[v];
    if (d < 1024)
      atomicAdd(&s_h[d], 1u);
    else
      atomicAdd(&hist[d], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 1024; i += blockDim.x)
    if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

__global__ void k_flag_present(const uint32_t* __restrict__ hist, uint32_t len, uint32_t* flags) {
  for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < len; d += gridDim.x * blockDim.x)
    flags[d] = (d >= 1 && hist[d] > 0) ? 1u : 0u;
}

__global__ void k_degree_tables(const uint32_t* __restrict__ hist, const uint32_t* __restrict__ flags,
                                const uint64_t* __restrict__ pos, uint32_t len, uint32_t* dvals, uint32_t* dcnt0,
                                uint32_t* drank) {
  for (uint32_t d = blockIdx.x * blockDim.x + threadIdx.x; d < len; d += gridDim.x * blockDim.x) {
    if (flags[d]) {
      uint32_t r = (uint32_t)pos[d];
      dvals[r] = d;
      dcnt0[r] = hist[d];
      drank[d] = r;
    } else {
      drank[d] = 0xFFFFFFFFu;
    }
  }
}

__global__ void k_highd0(const uint32_t* dcnt0, const uint32_t* dvals, uint32_t D, uint32_t* out) {
  uint32_t h = block_highd(dcnt0, dvals, D);
  if (threadIdx.x == 0) *out = h;
}

__global__ void k_narrow(const uint64_t* __restrict__ in, uint64_t n, uint32_t* out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)in[i];
}

__global__ void k_nz_keys(const uint4* __restrict__ nz, uint32_t cnt, int vbits, uint64_t* keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    keys[i] = ((uint64_t)nz[i].y << vbits) | nz[i].x;
}

__global__ void k_nz_from_keys(const uint64_t* __restrict__ keys, uint32_t cnt, int vbits,
                               const uint32_t* __restrict__ row, uint4* nz) {
  const uint64_t vmask = (1ull << vbits) - 1;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)(keys[i] & vmask);
    nz[i] = make_uint4(v, (uint32_t)(keys[i] >> vbits), row[v], row[v + 1]);
  }
}

// lt[t] = number of entries of the weight-sorted nz with smallest weight < t, t < len
__global__ void k_nz_lt(const uint4* __restrict__ nz, uint32_t cnt, uint32_t len, uint32_t* lt) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= cnt; i += gridDim.x * blockDim.x) {
    const uint32_t lo = i == 0 ? 0 : nz[i - 1].y + 1;           // first t with entry i-1 counted
    const uint32_t hi = i == cnt ? len - 1 : nz[i].y;           // last t before entry i counts
    for (uint32_t t = lo; t <= hi && t < len; ++t) lt[t] = i;
  }
}

__global__ void k_flag_nonzero(const uint32_t* __restrict__ deg, uint32_t n, uint32_t* flags) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
    flags[v] = deg[v] ? 1u : 0u;
}

// Temporary device allocations released on every exit path.
struct Temps {
  void* p[24];
  int k = 0;
  ~Temps() {
    for (int i = 0; i < k; ++i) cudaFree(p[i]);
  }
  template <typename T>
  int alloc(T** out, uint64_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc((void**)out, count * sizeof(T)) != cudaSuccess) {
      (void)cudaGetLastError();
      return EIC_ENOMEM;
    }
    p[k++] = *out;
    return EIC_OK;
  }
  void release(void* q) {
    for (int i = 0; i < k; ++i)
      if (p[i] == q) {
        cudaFree(q);
        p[i] = p[--k];
        return;
      }
  }
};

#define TRY(x)                   \
  do {                           \
    int rc_ = (x);               \
    if (rc_ != EIC_OK) return rc_; \
  } while (0)

template <typename T>
int galloc(eic_graph* g, T** out, uint64_t count) {
  *out = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)out, count * sizeof(T)) != cudaSuccess) {
    (void)cudaGetLastError();
    return EIC_ENOMEM;
  }
  g->bytes += count * sizeof(T);
  return EIC_OK;
}

void graph_free_arrays(eic_graph* g) {
  cudaFree(g->row);
  cudaFree(g->adj);
  cudaFree(g->drank);
  cudaFree(g->dvals);
  cudaFree(g->dcnt0);
  cudaFree(g->dfirst);
  cudaFree(g->dhint);
  cudaFree(g->rtow);
  cudaFree(g->nz);
  cudaFree(g->nz_lt);
  cudaFree(g->orig2int);
  cudaFree(g->int2orig);
}

int build(eic_graph* g, const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t T, uint32_t n,
          int on_device, cudaStream_t st) {
  Temps tmp;
  const uint32_t *dsrc = src, *ddst = dst, *dw = w;
  if (!on_device && T > 0) {
    uint32_t *a, *b, *c;
    TRY(tmp.alloc(&a, T));
    TRY(tmp.alloc(&b, T));
    TRY(tmp.alloc(&c, T));
    EIC_CUDA_TRY(cudaMemcpyAsync(a, src, T * 4, cudaMemcpyHostToDevice, st));
    EIC_CUDA_TRY(cudaMemcpyAsync(b, dst, T * 4, cudaMemcpyHostToDevice, st));
    EIC_CUDA_TRY(cudaMemcpyAsync(c, w, T * 4, cudaMemcpyHostToDevice, st));
    dsrc = a;
    ddst = b;
    dw = c;
  }
  const int vbits = bits_for(n > 1 ? n - 1 : 1);
  uint32_t* small;  // [0] pair count, [1] wmax, [2] wmin, [3] maxdeg, [4] highd0
  int* err;
  uint64_t* scan_scratch;
  uint32_t* hist_scratch;
  TRY(tmp.alloc(&small, 8));
  TRY(tmp.alloc(&err, 1));
  TRY(tmp.alloc(&scan_scratch, kScanBlocksMax + 1));
  TRY(tmp.alloc(&hist_scratch, (uint64_t)kRadixDigits * kSortBlocksMax));
  uint32_t init_small[8] = {0, 0, 0xFFFFFFFFu, 0, 0, 0, 0, 0};
  EIC_CUDA_TRY(cudaMemcpyAsync(small, init_small, sizeof(init_small), cudaMemcpyHostToDevice, st));
  EIC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));

  // 1. canonical pair keys (min, max) with their weights, self-loops dropped
  uint64_t* k0;
  uint32_t* v0;
  TRY(tmp.alloc(&k0, T));
  TRY(tmp.alloc(&v0, T));
  if (T > 0) k_canon<<<grid_for(T), kThreads, 0, st>>>(dsrc, ddst, dw, T, n, vbits, k0, v0, small, err);
  EIC_CUDA_TRY(cudaGetLastError());
  uint32_t hs[8];
  int herr = 0;
  EIC_CUDA_TRY(cudaMemcpyAsync(hs, small, sizeof(hs), cudaMemcpyDeviceToHost, st));
  EIC_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  EIC_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr) return EIC_EINVAL;
  if (!on_device && T > 0) {
    tmp.release((void*)dsrc);
    tmp.release((void*)ddst);
    tmp.release((void*)dw);
  }
  const uint64_t K = hs[0];

  // 2. sort the pair keys; each distinct pair keeps its smallest weight
  uint64_t m = 0;
  uint64_t* ukeys;
  uint32_t* uw;
  {
    uint64_t* k1;
    uint32_t* v1;
    TRY(tmp.alloc(&k1, K));
    TRY(tmp.alloc(&v1, K));
    bool alt = false;
    TRY(radix_sort(k0, v0, k1, v1, K, 2 * vbits, hist_scratch, st, &alt));
    uint64_t* sk = alt ? k1 : k0;
    uint32_t* sv = alt ? v1 : v0;
    uint32_t* flags = alt ? v0 : v1;
    uint64_t* pos;
    TRY(tmp.alloc(&pos, K + 1));
    if (K > 0) {
      k_heads<<<grid_for(K), kThreads, 0, st>>>(sk, K, flags);
      TRY(exclusive_scan<uint32_t>(flags, K, pos, scan_scratch, st));
      EIC_CUDA_TRY(cudaMemcpyAsync(&m, pos + K, 8, cudaMemcpyDeviceToHost, st));
      EIC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    TRY(tmp.alloc(&ukeys, m));
    TRY(tmp.alloc(&uw, m));
    if (K > 0) k_dedup<<<grid_for(K), kThreads, 0, st>>>(sk, sv, flags, pos, K, ukeys, uw);
    EIC_CUDA_TRY(cudaGetLastError());
    EIC_CUDA_TRY(cudaStreamSynchronize(st));
    tmp.release(pos);
    tmp.release(k1);
    tmp.release(v1);
    tmp.release(k0);
    tmp.release(v0);
  }
  const uint64_t E = 2 * m;

  // 3. degrees in original ids, weight range
  uint32_t* deg;
  TRY(tmp.alloc(&deg, (uint64_t)n + 1));
  EIC_CUDA_TRY(cudaMemsetAsync(deg, 0, ((uint64_t)n + 1) * 4, st));
  if (m > 0) k_degrees<<<grid_for(m), kThreads, 0, st>>>(ukeys, uw, m, vbits, deg, small + 1, small + 2);
  k_max_u32<<<grid_for(n), kThreads, 0, st>>>(deg, n, small + 3);
  EIC_CUDA_TRY(cudaGetLastError());
  EIC_CUDA_TRY(cudaMemcpyAsync(hs, small, sizeof(hs), cudaMemcpyDeviceToHost, st));
  EIC_CUDA_TRY(cudaStreamSynchronize(st));
  const uint32_t maxw = m ? hs[1] : 0, minw = m ? hs[2] : 0;
  const uint32_t maxdeg = hs[3];
  const int wbits = bits_for(maxw);

  // 3b. internal ids: the non-isolated vertices ordered by (degree descending,
  // original id), so that the most-touched vertices share cache lines
  uint32_t ni = 0;
  TRY(galloc(g, &g->orig2int, n));
  EIC_CUDA_TRY(cudaMemsetAsync(g->orig2int, 0xFF, (uint64_t)n * 4, st));
  {
    uint32_t* flags;
    uint64_t* pos;
    TRY(tmp.alloc(&flags, n));
    TRY(tmp.alloc(&pos, (uint64_t)n + 1));
    k_flag_nonzero<<<grid_for(n), kThreads, 0, st>>>(deg, n, flags);
    TRY(exclusive_scan<uint32_t>(flags, n, pos, scan_scratch, st));
    uint64_t c = 0;
    EIC_CUDA_TRY(cudaMemcpyAsync(&c, pos + n, 8, cudaMemcpyDeviceToHost, st));
    EIC_CUDA_TRY(cudaStreamSynchronize(st));
    ni = (uint32_t)c;
    TRY(galloc(g, &g->int2orig, ni));
    uint64_t *rk0, *rk1;
    TRY(tmp.alloc(&rk0, ni));
    TRY(tmp.alloc(&rk1, ni));
    const int dbits = bits_for(maxdeg);
    k_relabel_keys<<<grid_for(n), kThreads, 0, st>>>(deg, flags, pos, n, maxdeg, vbits, rk0);
    bool alt = false;
    TRY(radix_sort(rk0, nullptr, rk1, nullptr, ni, dbits + vbits, hist_scratch, st, &alt));
    k_relabel_maps<<<grid_for(ni), kThreads, 0, st>>>(alt ? rk1 : rk0, ni, vbits, g->int2orig, g->orig2int);
    EIC_CUDA_TRY(cudaGetLastError());
    EIC_CUDA_TRY(cudaStreamSynchronize(st));
    tmp.release(rk0);
    tmp.release(rk1);
    tmp.release(flags);
    tmp.release(pos);
  }
  const int ibits = bits_for(ni > 1 ? ni - 1 : 1);
  TRY(galloc(g, &g->row, (uint64_t)ni + 1));
  {
    uint32_t* deg_int;
    uint64_t* row64;
    TRY(tmp.alloc(&deg_int, (uint64_t)ni + 1));
    TRY(tmp.alloc(&row64, (uint64_t)ni + 1));
    k_gather_u32<<<grid_for(ni), kThreads, 0, st>>>(deg, g->int2orig, ni, deg_int);
    TRY(exclusive_scan<uint32_t>(deg_int, ni, row64, scan_scratch, st));
    k_narrow<<<grid_for((uint64_t)ni + 1), kThreads, 0, st>>>(row64, (uint64_t)ni + 1, g->row);
    EIC_CUDA_TRY(cudaGetLastError());
    EIC_CUDA_TRY(cudaStreamSynchronize(st));
    tmp.release(row64);
    tmp.release(deg_int);
  }

  // 4. both directions in internal ids, stable sort by (row, weight): rows in weight order
  TRY(galloc(g, &g->adj, E + 2));  // two spare entries: a 16-byte pair load starting at the last entry stays inside
  if (E > 0) {
    uint64_t *ek0, *ek1;
    uint32_t *ev0, *ev1;
    TRY(tmp.alloc(&ek0, E));
    TRY(tmp.alloc(&ev0, E));
    TRY(tmp.alloc(&ek1, E));
    TRY(tmp.alloc(&ev1, E));
    k_emit<<<grid_for(m), kThreads, 0, st>>>(ukeys, uw, m, vbits, g->orig2int, wbits, ek0, ev0);
    bool alt = false;
    TRY(radix_sort(ek0, ev0, ek1, ev1, E, ibits + wbits, hist_scratch, st, &alt));
    k_pack_adj<<<grid_for(E), kThreads, 0, st>>>(alt ? ek1 : ek0, alt ? ev1 : ev0, E, wbits, g->adj);
    EIC_CUDA_TRY(cudaGetLastError());
    EIC_CUDA_TRY(cudaStreamSynchronize(st));
    tmp.release(ek0);
    tmp.release(ev0);
    tmp.release(ek1);
    tmp.release(ev1);
  }

  // 5a. RtoW from the sorted undirected weights
  TRY(galloc(g, &g->rtow, EIC_RATIO_NUM));
  if (m > 0) {
    uint64_t *wk0, *wk1;
    TRY(tmp.alloc(&wk0, m));
    TRY(tmp.alloc(&wk1, m));
    k_weights_to_keys<<<grid_for(m), kThreads, 0, st>>>(uw, m, wk0);
    bool alt = false;
    TRY(radix_sort(wk0, nullptr, wk1, nullptr, m, wbits, hist_scratch, st, &alt));
    k_rtow<<<(EIC_RATIO_NUM + kThreads - 1) / kThreads, kThreads, 0, st>>>(alt ? wk1 : wk0, m, g->rtow);
    EIC_CUDA_TRY(cudaGetLastError());
    EIC_CUDA_TRY(cudaStreamSynchronize(st));
    tmp.release(wk0);
    tmp.release(wk1);
  } else {
    EIC_CUDA_TRY(cudaMemsetAsync(g->rtow, 0, EIC_RATIO_NUM * 4, st));
  }
  tmp.release(ukeys);
  tmp.release(uw);

  // 5b. distinct-degree tables and highD(0)
  const uint32_t hlen = maxdeg + 1;
  uint32_t D = 0, nlong = 0;
  {
    uint32_t *dh, *flags;
    uint64_t* pos;
    TRY(tmp.alloc(&dh, hlen));
    TRY(tmp.alloc(&flags, hlen));
    TRY(tmp.alloc(&pos, (uint64_t)hlen + 1));
    EIC_CUDA_TRY(cudaMemsetAsync(dh, 0, (uint64_t)hlen * 4, st));
    k_deg_hist<<<grid_for(n), kThreads, 0, st>>>(deg, n, dh);
    k_flag_present<<<grid_for(hlen), kThreads, 0, st>>>(dh, hlen, flags);
    TRY(exclusive_scan<uint32_t>(flags, hlen, pos, scan_scratch, st));
    uint64_t dd = 0;
    EIC_CUDA_TRY(cudaMemcpyAsync(&dd, pos + hlen, 8, cudaMemcpyDeviceToHost, st));
    EIC_CUDA_TRY(cudaStreamSynchronize(st));
    D = (uint32_t)dd;
    TRY(galloc(g, &g->dvals, D));
    TRY(galloc(g, &g->dcnt0, D));
    TRY(galloc(g, &g->drank, hlen));
    k_degree_tables<<<grid_for(hlen), kThreads, 0, st>>>(dh, flags, pos, hlen, g->dvals, g->dcnt0, g->drank);
    k_highd0<<<1, 1024, 0, st>>>(g->dcnt0, g->dvals, D, small + 4);
    EIC_CUDA_TRY(cudaGetLastError());
    // dfirst[r]: the first internal id of degree dvals[r] (ids by degree descending)
    TRY(galloc(g, &g->dfirst, D));
    if (D) {
      std::vector<uint32_t> cnt(D), first(D), vals(D);
      EIC_CUDA_TRY(cudaMemcpyAsync(cnt.data(), g->dcnt0, (uint64_t)D * 4, cudaMemcpyDeviceToHost, st));
      EIC_CUDA_TRY(cudaMemcpyAsync(vals.data(), g->dvals, (uint64_t)D * 4, cudaMemcpyDeviceToHost, st));
      EIC_CUDA_TRY(cudaStreamSynchronize(st));
      uint64_t acc = 0;
      for (uint32_t r = D; r-- > 0;) {
        first[r] = (uint32_t)acc;
        acc += cnt[r];
        if (vals[r] > kCursorMin) nlong = (uint32_t)acc;  // ids [0, acc) have degree >= vals[r]
      }
      EIC_CUDA_TRY(cudaMemcpyAsync(g->dfirst, first.data(), (uint64_t)D * 4, cudaMemcpyHostToDevice, st));
      EIC_CUDA_TRY(cudaStreamSynchronize(st));
    }
    // dhint[b]: the ranks of ids 4096 b + 4095 and 4096 b (the range a rank search in block b needs)
    const uint64_t nblk = (uint64_t)ni / 4096 + 1;
    TRY(galloc(g, &g->dhint, nblk));
    if (D) {
      std::vector<uint32_t> first(D);
      EIC_CUDA_TRY(cudaMemcpyAsync(first.data(), g->dfirst, (uint64_t)D * 4, cudaMemcpyDeviceToHost, st));
      EIC_CUDA_TRY(cudaStreamSynchronize(st));
      auto rank_of = [&](uint64_t x) -> uint32_t {  // the smallest r with first[r] <= x
        uint32_t lo = 0, hi = D - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi) / 2;
          if (first[mid] <= x)
            hi = mid;
          else
            lo = mid + 1;
        }
        return lo;
      };
      std::vector<uint2> hint(nblk);
      for (uint64_t b = 0; b < nblk; ++b) {
        const uint64_t x0 = b * 4096, x1 = std::min<uint64_t>(x0 + 4095, ni ? ni - 1 : 0);
        hint[b] = make_uint2(rank_of(x1), rank_of(std::min<uint64_t>(x0, x1)));
      }
      EIC_CUDA_TRY(cudaMemcpyAsync(g->dhint, hint.data(), nblk * sizeof(uint2), cudaMemcpyHostToDevice, st));
      EIC_CUDA_TRY(cudaStreamSynchronize(st));
    }
  }

  // 5c. every internal vertex with its smallest weight, ordered by (smallest
  // weight, id): the vertices a pull can touch (smallest weight below a bound)
  // form a prefix, located with nz_lt
  uint32_t nz_lt_len = 0;
  {
    TRY(galloc(g, &g->nz, ni));
    k_nz_fill<<<grid_for(ni), kThreads, 0, st>>>(g->row, g->adj, ni, g->nz);
    EIC_CUDA_TRY(cudaGetLastError());
    if (ni > 1) {
      uint64_t *kk0, *kk1;
      TRY(tmp.alloc(&kk0, ni));
      TRY(tmp.alloc(&kk1, ni));
      k_nz_keys<<<grid_for(ni), kThreads, 0, st>>>(g->nz, ni, ibits, kk0);
      bool alt = false;
      TRY(radix_sort(kk0, nullptr, kk1, nullptr, ni, ibits + wbits, hist_scratch, st, &alt));
      k_nz_from_keys<<<grid_for(ni), kThreads, 0, st>>>(alt ? kk1 : kk0, ni, ibits, g->row, g->nz);
      EIC_CUDA_TRY(cudaGetLastError());
      EIC_CUDA_TRY(cudaStreamSynchronize(st));
      tmp.release(kk0);
      tmp.release(kk1);
    }
    nz_lt_len = (maxw < 65535u ? maxw + 1 : 65536u) + 1;
    TRY(galloc(g, &g->nz_lt, nz_lt_len));
    k_nz_lt<<<grid_for((uint64_t)ni + 1), kThreads, 0, st>>>(g->nz, ni, nz_lt_len, g->nz_lt);
    EIC_CUDA_TRY(cudaGetLastError());
  }
  EIC_CUDA_TRY(cudaMemcpyAsync(hs, small, sizeof(hs), cudaMemcpyDeviceToHost, st));
  EIC_CUDA_TRY(cudaStreamSynchronize(st));

  DevGraph& dg = g->dg;
  dg.n = n;
  dg.ni = ni;
  dg.orig2int = g->orig2int;
  dg.int2orig = g->int2orig;
  dg.two_m = E;
  dg.m = m;
  dg.row = g->row;
  dg.adj = g->adj;
  dg.drank = g->drank;
  dg.dvals = g->dvals;
  dg.dcnt0 = g->dcnt0;
  dg.dfirst = g->dfirst;
  dg.dhint = g->dhint;
  dg.nlong = nlong;
  dg.D = D;
  dg.rtow = g->rtow;
  dg.nz = g->nz;
  dg.nz_count = ni;
  dg.nz_lt = g->nz_lt;
  dg.nz_lt_len = nz_lt_len;
  dg.maxw = maxw;
  dg.minw = minw;
  dg.max_deg = maxdeg;
  dg.highd0 = hs[4];
  return EIC_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

int eic_params_default(eic_params* p) {
  if (!p) return EIC_EINVAL;
  memset(p, 0, sizeof(*p));
  p->alpha = 3;
  p->beta = 0.9;
  p->st_num = 1024;
  return EIC_OK;
}

const char* eic_strerror(int status) {
  switch (status) {
    case EIC_OK: return "ok";
    case EIC_EINVAL: return "invalid argument";
    case EIC_ENOMEM: return "out of memory or capacity";
    case EIC_ECUDA: return "CUDA runtime error";
    case EIC_EOVERFLOW: return "distance overflow (max distance + max weight >= 2^32-1)";
    case EIC_ETIMEOUT: return "device wait timed out";
    case EIC_EBUSY: return "busy";
    case EIC_ESIZE: return "graph exceeds the limits of the allocation-free entry point";
    case EIC_EABORT: return "not run: every block group of the batch stopped at an earlier error";
    default: return "unknown status";
  }
}

int eic_version(void) { return 100; }

int eic_graph_create(const uint32_t* src, const uint32_t* dst, const uint32_t* w, uint64_t num_tuples,
                     uint32_t num_vertices, int ptrs_on_device, void* stream, eic_graph** out) {
  if (!out) return EIC_EINVAL;
  *out = nullptr;
  if (num_vertices == 0 || num_vertices >= 0xFFFFFFFFu) return EIC_EINVAL;
  if (num_tuples > 0 && (!src || !dst || !w)) return EIC_EINVAL;
  if (num_tuples >= (1ull << 31)) return EIC_EINVAL;
  eic_graph* g = new (std::nothrow) eic_graph();
  if (!g) return EIC_ENOMEM;
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete g;
    return EIC_ECUDA;
  }
  int rc = build(g, src, dst, w, num_tuples, num_vertices, ptrs_on_device, (cudaStream_t)stream);
  if (rc != EIC_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    (void)cudaGetLastError();
    graph_free_arrays(g);
    delete g;
    return rc;
  }
  *out = g;
  return EIC_OK;
}

int eic_graph_info(const eic_graph* g, uint32_t* n, uint64_t* m, uint32_t* max_deg, uint32_t* max_w,
                   uint32_t* min_w, uint32_t* highd0) {
  if (!g) return EIC_EINVAL;
  if (n) *n = g->dg.n;
  if (m) *m = g->dg.m;
  if (max_deg) *max_deg = g->dg.max_deg;
  if (max_w) *max_w = g->dg.maxw;
  if (min_w) *min_w = g->dg.minw;
  if (highd0) *highd0 = g->dg.highd0;
  return EIC_OK;
}

int eic_graph_export(const eic_graph* g, uint64_t* row_ptr, uint32_t* nbr, uint32_t* w, uint32_t* rtow) {
  if (!g) return EIC_EINVAL;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(g->device);
  int rc = EIC_OK;
  const uint64_t n = g->dg.n, ni = g->dg.ni, E = g->dg.two_m;
  uint32_t* o2i = (uint32_t*)malloc((n ? n : 1) * 4);
  uint32_t* i2o = (uint32_t*)malloc((ni ? ni : 1) * 4);
  uint32_t* row = (uint32_t*)malloc((ni + 1) * 4);
  uint2* adj = (nbr || w) ? (uint2*)malloc((E ? E : 1) * sizeof(uint2)) : nullptr;
  if (!o2i || !i2o || !row || ((nbr || w) && !adj)) rc = EIC_ENOMEM;
  if (rc == EIC_OK && (cudaMemcpy(o2i, g->orig2int, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                       cudaMemcpy(i2o, g->int2orig, ni * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                       cudaMemcpy(row, g->row, (ni + 1) * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                       (adj && E && cudaMemcpy(adj, g->adj, E * sizeof(uint2), cudaMemcpyDeviceToHost) != cudaSuccess)))
    rc = EIC_ECUDA;
  if (rc == EIC_OK) {
    // rows in original vertex order, each sorted by (weight, original neighbour)
    uint64_t off = 0;
    std::vector<uint64_t> tmpk;
    for (uint64_t u = 0; u < n; ++u) {
      if (row_ptr) row_ptr[u] = off;
      const uint32_t i = o2i[u];
      if (i == 0xFFFFFFFFu) continue;
      const uint32_t b = row[i], e = row[i + 1];
      if (adj) {
        tmpk.resize(e - b);
        for (uint32_t k = b; k < e; ++k) tmpk[k - b] = ((uint64_t)adj[k].y << 32) | i2o[adj[k].x];
        std::sort(tmpk.begin(), tmpk.end());
        for (uint32_t k = 0; k < e - b; ++k) {
          if (nbr) nbr[off + k] = (uint32_t)tmpk[k];
          if (w) w[off + k] = (uint32_t)(tmpk[k] >> 32);
        }
      }
      off += e - b;
    }
    if (row_ptr) row_ptr[n] = off;
  }
  if (rtow && rc == EIC_OK && cudaMemcpy(rtow, g->rtow, EIC_RATIO_NUM * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = EIC_ECUDA;
  free(o2i);
  free(i2o);
  free(row);
  free(adj);
  (void)cudaGetLastError();
  cudaSetDevice(dev);
  return rc;
}

int eic_graph_export_internal(const eic_graph* g, uint32_t* ni, uint32_t* int2orig, uint32_t* row, uint32_t* nbr,
                              uint32_t* w) {
  if (!g) return EIC_EINVAL;
  if (ni) *ni = g->dg.ni;
  if (!int2orig && !row && !nbr && !w) return EIC_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(g->device);
  int rc = EIC_OK;
  const uint64_t n_int = g->dg.ni, E = g->dg.two_m;
  if (int2orig && n_int && cudaMemcpy(int2orig, g->int2orig, n_int * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = EIC_ECUDA;
  if (rc == EIC_OK && row && cudaMemcpy(row, g->row, (n_int + 1) * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = EIC_ECUDA;
  if (rc == EIC_OK && (nbr || w) && E) {
    uint2* adj = (uint2*)malloc(E * sizeof(uint2));
    if (!adj) {
      rc = EIC_ENOMEM;
    } else if (cudaMemcpy(adj, g->adj, E * sizeof(uint2), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = EIC_ECUDA;
    } else {
      for (uint64_t k = 0; k < E; ++k) {
        if (nbr) nbr[k] = adj[k].x;
        if (w) w[k] = adj[k].y;
      }
    }
    free(adj);
  }
  (void)cudaGetLastError();
  cudaSetDevice(dev);
  return rc;
}

int eic_graph_memory(const eic_graph* g, uint64_t* graph_bytes, uint64_t* workspace_bytes) {
  if (!g) return EIC_EINVAL;
  if (graph_bytes) *graph_bytes = g->bytes;
  if (workspace_bytes) *workspace_bytes = g->ws.bytes;
  return EIC_OK;
}

int eic_graph_destroy(eic_graph* g) {
  if (!g) return EIC_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  eic_ws_free(&g->ws);
  graph_free_arrays(g);
  (void)cudaGetLastError();
  cudaSetDevice(dev);
  delete g;
  return EIC_OK;
}

}  // extern "C"

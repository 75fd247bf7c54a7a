// Shared definitions of libeic's CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/eic.h"

#define EIC_INF_T (((int64_t)1) << 62)
#define EIC_FULL_MASK 0xFFFFFFFFu

#define EIC_CUDA_TRY(expr)                     \
  do {                                         \
    cudaError_t e_ = (expr);                   \
    if (e_ != cudaSuccess) {                   \
      (void)cudaGetLastError();                \
      return e_ == cudaErrorMemoryAllocation   \
                 ? EIC_ENOMEM                  \
                 : EIC_ECUDA;                  \
    }                                          \
  } while (0)

// Read-only view of a device-resident graph (preprocessing of Section 4.1).
// Vertices have internal ids 0..ni-1: the non-isolated vertices ordered by
// (degree descending, original id); orig2int/int2orig translate.
constexpr uint32_t kCursorMin = 16;  // rows longer than this keep a window cursor

struct DevGraph {
  uint32_t n;             // vertices in the caller's numbering
  uint32_t ni;            // internal vertices (degree >= 1)
  const uint32_t* orig2int;  // [n] internal id, or 0xFFFFFFFF for an isolated vertex
  const uint32_t* int2orig;  // [ni]
  uint64_t two_m;         // directed entries, sum of degrees
  uint64_t m;             // undirected edges
  const uint32_t* row;    // [ni + 1] row offsets (2m < 2^32)
  const uint2* adj;       // [two_m] {neighbour, weight}, rows sorted by (weight, neighbour)
  const uint32_t* drank;  // [max_deg + 1] degree -> rank among distinct degrees (present ones)
  const uint32_t* dvals;  // [D] distinct degrees >= 1, ascending
  const uint32_t* dcnt0;  // [D] number of vertices with degree dvals[r]
  const uint32_t* dfirst;  // [D] first internal id of degree dvals[r] (decreasing in r: ids run by degree descending)
  const uint2* dhint;      // [ni / 4096 + 1] {rank of the block's last id, rank of its first id} per 4096 ids
  uint32_t D;
  const uint32_t* rtow;   // [EIC_RATIO_NUM] maxW(G, i / (RATIO_NUM - 1))
  const uint4* nz;        // [nz_count = ni] {internal id, smallest row weight, row begin, row end}, by (weight, id)
  uint32_t nz_count;
  const uint32_t* nz_lt;  // [nz_lt_len] nz_lt[t] = number of nz entries with smallest weight < t
  uint32_t nz_lt_len;
  uint32_t maxw, minw, max_deg, highd0;
  uint32_t nlong;         // internal vertices of degree > kCursorMin: ids [0, nlong), the rows with a window cursor
};

// Rank (index into dvals) of internal vertex x's degree: internal ids run by
// degree descending, so it is the smallest r with dfirst[r] <= x. A search in
// a small table that stays in L1, narrowed to the ranks of x's block of 4096
// ids, in place of a random row[x], row[x + 1].
__device__ __forceinline__ uint32_t degree_rank(const DevGraph& G, uint32_t x) {
  const uint2 h = __ldg(&G.dhint[x >> 12]);  // the ranks in x's block of 4096 ids: one rank in most blocks
  uint32_t lo = h.x, hi = h.y;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(&G.dfirst[mid]) <= x)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// ------------------------------------------------------------ warp helpers

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(EIC_FULL_MASK, x, o);
    if ((int)lane_id() >= o) x += y;
  }
  return x;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(EIC_FULL_MASK, x, o);
  return x;
}

// Warp-aggregated append of `item` for each lane with want != 0 to
// list[*counter ...]; returns the slot or UINT32_MAX. All lanes must call.
__device__ __forceinline__ uint32_t warp_append(bool want, uint32_t* counter) {
  uint32_t mask = __ballot_sync(EIC_FULL_MASK, want);
  if (mask == 0) return UINT32_MAX;
  uint32_t leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
  base = __shfl_sync(EIC_FULL_MASK, base, leader);
  return want ? base + __popc(mask & ((1u << lane_id()) - 1u)) : UINT32_MAX;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(const volatile int*)p; }

// Release/acquire primitives of the barrier (gpu scope).
__device__ __forceinline__ uint32_t atom_add_acq_rel_u32(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------- bounded grid barrier

struct GridBarrier {
  uint32_t count;
  uint32_t gen;
  unsigned long long arrived;  // arrivals since the query started (single-query launches)
};

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Software barrier over nblocks co-resident (cooperatively launched) blocks:
// the whole grid, or one block group of it. Every wait is bounded: after
// max_spin polls the block records EIC_ETIMEOUT in *status and all blocks
// leave at their next barrier. Returns false when the blocks must stop (one
// of them reported an error).
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, uint32_t* gen_local, uint32_t nblocks, uint64_t max_spin,
                                             int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t g = *gen_local;
    // the arrival releases the block's writes (ordered before it by the block
    // barrier) and, for the last block, acquires everyone else's; the new
    // generation is published with a release after the count is reset
    const uint32_t arrived = atom_add_acq_rel_u32(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      bar->count = 0;
      st_release_u32(&bar->gen, g + 1);
    } else {
      uint64_t spins = 0;
      while (ld_acquire_u32(&bar->gen) == g) {
        if (ld_volatile_int(status) != 0) break;
        if (++spins > max_spin) {
          atomicCAS(status, 0, EIC_ETIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    *gen_local = g + 1;
    s_ok = ld_volatile_int(status) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// The same barrier for a launch that runs one query. The arrival count only
// grows while the query runs (its initialisation zeroes it), so a block
// arrives with one release add that returns nothing and waits, with acquire
// loads, until the count reaches its own next multiple of nblocks: no block
// has to see the last arrival and publish a new generation. ticket: the
// block's barriers passed so far times nblocks.
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned long long* ticket, uint32_t nblocks,
                                             uint64_t max_spin, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long target = *ticket + nblocks;
    red_release_add_u64(&bar->arrived, 1ull);
    uint64_t spins = 0;
    while (ld_acquire_gpu_u64(&bar->arrived) < target) {
      if (ld_volatile_int(status) != 0) break;
      if (++spins > max_spin) {
        atomicCAS(status, 0, EIC_ETIMEOUT);
        break;
      }
      __nanosleep(64);
    }
    *ticket = target;
    s_ok = ld_volatile_int(status) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

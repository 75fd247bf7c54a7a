// Device sort and scan primitives used by the CSR builder.
//
// LSD radix sort of (uint64 key, uint32 value) pairs, 8 bits per pass, in the
// reduce-then-scan form: a fixed grid of blocks each owns one contiguous
// slice of the input; pass = per-slice digit histogram -> one exclusive scan
// of the digit-major histogram -> stable scatter of each slice in order.
// Stability inside a slice comes from ranking 512-element rounds in order,
// warps in order inside a round and lanes in order inside a warp.
#pragma once

#include "common.cuh"

namespace eic {

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortBlocksMax = 1024;
constexpr int kRadixDigits = 256;

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) { return (uint32_t)(k >> shift) & 0xFFu; }

__global__ void __launch_bounds__(kSortThreads) k_radix_count(const uint64_t* __restrict__ keys, uint64_t n,
                                                              uint64_t per_block, int shift, uint32_t* hist) {
  __shared__ uint32_t s_h[kSortWarps][kRadixDigits];
  for (int i = threadIdx.x; i < kSortWarps * kRadixDigits; i += blockDim.x) (&s_h[0][0])[i] = 0;
  __syncthreads();
  uint64_t lo = (uint64_t)blockIdx.x * per_block;
  uint64_t hi = lo + per_block < n ? lo + per_block : n;
  uint32_t w = threadIdx.x >> 5;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) atomicAdd(&s_h[w][digit_of(keys[i], shift)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadixDigits; d += blockDim.x) {
    uint32_t s = 0;
    for (int j = 0; j < kSortWarps; ++j) s += s_h[j][d];
    hist[(uint64_t)d * gridDim.x + blockIdx.x] = s;
  }
}

// Exclusive scan of `count` uint32 in place with one block (count <= 2^20).
__global__ void __launch_bounds__(1024) k_scan_small_u32(uint32_t* data, uint32_t count) {
  __shared__ uint32_t s_part[1024];
  uint32_t per = (count + blockDim.x - 1) / blockDim.x;
  uint32_t lo = threadIdx.x * per, hi = lo + per < count ? lo + per : count;
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; ++i) s += data[i];
  s_part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {
    uint32_t v = threadIdx.x >= (uint32_t)o ? s_part[threadIdx.x - o] : 0;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = s_part[threadIdx.x] - s;
  for (uint32_t i = lo; i < hi; ++i) {
    uint32_t x = data[i];
    data[i] = run;
    run += x;
  }
}

template <bool kHasVals>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t* __restrict__ keys,
                                                                const uint32_t* __restrict__ vals, uint64_t n,
                                                                uint64_t per_block, int shift,
                                                                const uint32_t* __restrict__ hist,
                                                                uint64_t* __restrict__ keys_out,
                                                                uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t s_run[kRadixDigits];               // running global offset per digit
  __shared__ uint32_t s_wcnt[kSortWarps][kRadixDigits];  // this round: count per warp and digit
  for (int d = threadIdx.x; d < kRadixDigits; d += blockDim.x) s_run[d] = hist[(uint64_t)d * gridDim.x + blockIdx.x];
  uint64_t lo = (uint64_t)blockIdx.x * per_block;
  uint64_t hi = lo + per_block < n ? lo + per_block : n;
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  for (uint64_t base = lo; base < hi; base += blockDim.x) {
    for (int i = threadIdx.x; i < kSortWarps * kRadixDigits; i += blockDim.x) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    uint64_t idx = base + threadIdx.x;
    bool valid = idx < hi;
    uint64_t k = valid ? keys[idx] : 0;
    uint32_t v = (kHasVals && valid) ? vals[idx] : 0;
    uint32_t d = valid ? digit_of(k, shift) : kRadixDigits;  // invalid lanes get their own group
    uint32_t peers = __match_any_sync(EIC_FULL_MASK, d);
    uint32_t rank_in_warp = __popc(peers & lt);
    if (valid && rank_in_warp == 0) s_wcnt[w][d] = __popc(peers);
    __syncthreads();
    // per digit: exclusive prefix across warps, advance the running offset
    for (int dd = threadIdx.x; dd < kRadixDigits; dd += blockDim.x) {
      uint32_t run = s_run[dd];
      for (int j = 0; j < kSortWarps; ++j) {
        uint32_t c = s_wcnt[j][dd];
        s_wcnt[j][dd] = run;
        run += c;
      }
      s_run[dd] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = s_wcnt[w][d] + rank_in_warp;
      keys_out[pos] = k;
      if (kHasVals) vals_out[pos] = v;
    }
    __syncthreads();
  }
}

struct SortPlan {
  int blocks;
  uint64_t per_block;
};

inline SortPlan sort_plan(uint64_t n) {
  SortPlan p;
  uint64_t tiles = (n + kSortThreads - 1) / kSortThreads;
  p.blocks = (int)(tiles < (uint64_t)kSortBlocksMax ? (tiles ? tiles : 1) : kSortBlocksMax);
  uint64_t per = (n + p.blocks - 1) / p.blocks;
  p.per_block = ((per + kSortThreads - 1) / kSortThreads) * kSortThreads;
  if (p.per_block == 0) p.per_block = kSortThreads;
  return p;
}

// Sort keys[0..n) (and vals when non-NULL) by bits [0, bits) of the key.
// Ping-pongs between the two buffers; *in_alt tells which one holds the
// result. hist_scratch must hold 256 * kSortBlocksMax uint32.
inline int radix_sort(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, uint64_t n, int bits,
                      uint32_t* hist_scratch, cudaStream_t st, bool* in_alt) {
  *in_alt = false;
  if (n <= 1 || bits <= 0) return EIC_OK;
  SortPlan p = sort_plan(n);
  uint64_t* kin = keys;
  uint32_t* vin = vals;
  uint64_t* kout = keys_alt;
  uint32_t* vout = vals_alt;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_count<<<p.blocks, kSortThreads, 0, st>>>(kin, n, p.per_block, shift, hist_scratch);
    k_scan_small_u32<<<1, 1024, 0, st>>>(hist_scratch, (uint32_t)(kRadixDigits * p.blocks));
    if (vals)
      k_radix_scatter<true><<<p.blocks, kSortThreads, 0, st>>>(kin, vin, n, p.per_block, shift, hist_scratch, kout,
                                                               vout);
    else
      k_radix_scatter<false><<<p.blocks, kSortThreads, 0, st>>>(kin, nullptr, n, p.per_block, shift, hist_scratch,
                                                                kout, nullptr);
    EIC_CUDA_TRY(cudaGetLastError());
    uint64_t* tk = kin;
    kin = kout;
    kout = tk;
    uint32_t* tv = vin;
    vin = vout;
    vout = tv;
    *in_alt = !*in_alt;
  }
  return EIC_OK;
}

// ------------------------------------------------------------------- scans

constexpr int kScanThreads = 1024;
constexpr int kScanBlocksMax = 1024;

template <typename TIn>
__global__ void __launch_bounds__(kScanThreads) k_block_sums(const TIn* __restrict__ in, uint64_t n, uint64_t per,
                                                             uint64_t* sums) {
  __shared__ uint64_t s_w[32];
  uint64_t lo = (uint64_t)blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  uint64_t s = 0;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += (uint64_t)in[i];
  s = warp_sum_u64(s);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t t = threadIdx.x < blockDim.x / 32 ? s_w[threadIdx.x] : 0;
    t = warp_sum_u64(t);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
  }
}

__global__ void k_scan_sums(uint64_t* sums, int count, uint64_t* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    uint64_t run = 0;
    for (int i = 0; i < count; ++i) {
      uint64_t x = sums[i];
      sums[i] = run;
      run += x;
    }
    *total = run;
  }
}

// out[i] = sum(in[0..i)) for i in [0, n], out[n] = total.
template <typename TIn>
__global__ void __launch_bounds__(kScanThreads) k_block_scan(const TIn* __restrict__ in, uint64_t n, uint64_t per,
                                                             const uint64_t* __restrict__ offs,
                                                             uint64_t* __restrict__ out) {
  __shared__ uint64_t s_w[32];
  __shared__ uint64_t s_carry;
  uint64_t lo = (uint64_t)blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  if (threadIdx.x == 0) s_carry = offs[blockIdx.x];
  __syncthreads();
  for (uint64_t base = lo; base < hi; base += blockDim.x) {
    uint64_t i = base + threadIdx.x;
    uint64_t x = i < hi ? (uint64_t)in[i] : 0;
    uint64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(EIC_FULL_MASK, incl, o);
      if ((int)(threadIdx.x & 31) >= o) incl += y;
    }
    if ((threadIdx.x & 31) == 31) s_w[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint64_t t = threadIdx.x < blockDim.x / 32 ? s_w[threadIdx.x] : 0;
      uint64_t ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(EIC_FULL_MASK, ti, o);
        if ((int)threadIdx.x >= o) ti += y;
      }
      s_w[threadIdx.x] = ti - t;
    }
    __syncthreads();
    uint64_t carry = s_carry;
    if (i < hi) out[i] = carry + s_w[threadIdx.x >> 5] + incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = carry + s_w[threadIdx.x >> 5] + incl;
    __syncthreads();
  }
}

// out[0..n] exclusive prefix sums of in[0..n); out[n] = total. scratch holds
// kScanBlocksMax + 1 uint64.
template <typename TIn>
inline int exclusive_scan(const TIn* in, uint64_t n, uint64_t* out, uint64_t* scratch, cudaStream_t st) {
  int blocks = (int)((n + kScanThreads - 1) / kScanThreads);
  if (blocks > kScanBlocksMax) blocks = kScanBlocksMax;
  if (blocks < 1) blocks = 1;
  uint64_t per = (n + blocks - 1) / blocks;
  if (per == 0) per = 1;
  k_block_sums<TIn><<<blocks, kScanThreads, 0, st>>>(in, n, per, scratch);
  k_scan_sums<<<1, 32, 0, st>>>(scratch, blocks, out + n);
  k_block_scan<TIn><<<blocks, kScanThreads, 0, st>>>(in, n, per, scratch, out);
  EIC_CUDA_TRY(cudaGetLastError());
  return EIC_OK;
}

}  // namespace eic

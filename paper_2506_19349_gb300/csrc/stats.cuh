// Step statistics of Section 3: highD (degree-weighted split), the
// dynamic-stepping gap of Eq. 1-3 and the traversal-optimisation profit of
// Eq. 4-6 with the clamping of Section 3.2.
#pragma once

#include "common.cuh"

namespace eic {

// highD over a degree multiset given per distinct degree: cnt[r] vertices of
// degree dvals[r] (ascending, >= 1). The threshold t splits the set into
// degrees < t and >= t with the smallest difference of total degree; t ranges
// over the degrees present, ties keep the smaller t, and an empty (zero total
// degree) set gives 0. Called by all threads of one block; every thread gets
// the result. Uses at most 1024 threads.
static __device__ uint32_t block_highd(const uint32_t* cnt, const uint32_t* dvals, uint32_t D) {
  __shared__ uint64_t s_part[1024];
  __shared__ uint64_t s_bdiff[32];
  __shared__ uint32_t s_brank[32];
  __shared__ uint64_t s_total;
  const uint32_t nt = blockDim.x < 1024 ? blockDim.x : 1024;
  const uint32_t t = threadIdx.x;
  uint32_t per = (D + nt - 1) / nt;
  uint32_t lo = t < nt ? t * per : D, hi = lo + per < D ? lo + per : D;
  if (lo > D) lo = D;
  uint64_t sum = 0;
  for (uint32_t r = lo; r < hi; ++r) sum += (uint64_t)__ldcg(&cnt[r]) * dvals[r];
  if (t < nt) s_part[t] = sum;
  __syncthreads();
  // inclusive scan of s_part over nt entries (Hillis-Steele)
  for (uint32_t o = 1; o < nt; o <<= 1) {
    uint64_t v = (t < nt && t >= o) ? s_part[t - o] : 0;
    __syncthreads();
    if (t < nt) s_part[t] += v;
    __syncthreads();
  }
  if (t == 0) s_total = s_part[nt - 1];
  __syncthreads();
  const uint64_t total = s_total;
  uint64_t low = (t < nt) ? s_part[t] - sum : 0;
  uint64_t bdiff = UINT64_MAX;
  uint32_t brank = UINT32_MAX;
  for (uint32_t r = lo; r < hi; ++r) {
    uint32_t c = __ldcg(&cnt[r]);
    if (c == 0) continue;
    uint64_t high = total - low;
    uint64_t diff = high > low ? high - low : low - high;
    if (diff < bdiff) {
      bdiff = diff;
      brank = r;
    }
    low += (uint64_t)c * dvals[r];
  }
  // block arg-min on (diff, rank)
  for (int o = 16; o > 0; o >>= 1) {
    uint64_t od = __shfl_down_sync(EIC_FULL_MASK, bdiff, o);
    uint32_t orr = __shfl_down_sync(EIC_FULL_MASK, brank, o);
    if (od < bdiff || (od == bdiff && orr < brank)) {
      bdiff = od;
      brank = orr;
    }
  }
  if ((t & 31) == 0) {
    s_bdiff[t >> 5] = bdiff;
    s_brank[t >> 5] = brank;
  }
  __syncthreads();
  if (t < 32) {
    uint32_t nw = (blockDim.x + 31) / 32;
    bdiff = t < nw ? s_bdiff[t] : UINT64_MAX;
    brank = t < nw ? s_brank[t] : UINT32_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      uint64_t od = __shfl_down_sync(EIC_FULL_MASK, bdiff, o);
      uint32_t orr = __shfl_down_sync(EIC_FULL_MASK, brank, o);
      if (od < bdiff || (od == bdiff && orr < brank)) {
        bdiff = od;
        brank = orr;
      }
    }
    if (t == 0) s_brank[0] = brank;
  }
  __syncthreads();
  uint32_t res = (total == 0 || s_brank[0] == UINT32_MAX) ? 0u : dvals[s_brank[0]];
  __syncthreads();
  return res;
}

// The same for D <= 32 * kWarpHighdPer distinct degrees by one warp (no block
// barriers): lane l holds a contiguous run of ranks, a shuffle scan gives each
// run's starting total, and a shuffle arg-min picks the rank (ties: smaller
// rank). Called by the 32 lanes of one warp; every lane gets the result.
constexpr uint32_t kWarpHighdPer = 32;
static __device__ uint32_t warp_highd(const uint32_t* cnt, const uint32_t* dvals, uint32_t D) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t per = (D + 31) / 32;
  const uint32_t lo = min(D, lane * per), hi = min(D, lo + per);
  uint64_t sum = 0;
  for (uint32_t r = lo; r < hi; ++r) sum += (uint64_t)__ldcg(&cnt[r]) * dvals[r];
  uint64_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(EIC_FULL_MASK, incl, o);
    if ((int)lane >= o) incl += y;
  }
  const uint64_t total = __shfl_sync(EIC_FULL_MASK, incl, 31);
  uint64_t low = incl - sum;
  uint64_t bdiff = UINT64_MAX;
  uint32_t brank = UINT32_MAX;
  for (uint32_t r = lo; r < hi; ++r) {
    const uint32_t c = __ldcg(&cnt[r]);
    if (c == 0) continue;
    const uint64_t high = total - low;
    const uint64_t diff = high > low ? high - low : low - high;
    if (diff < bdiff) {
      bdiff = diff;
      brank = r;
    }
    low += (uint64_t)c * dvals[r];
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t od = __shfl_xor_sync(EIC_FULL_MASK, bdiff, o);
    const uint32_t orr = __shfl_xor_sync(EIC_FULL_MASK, brank, o);
    if (od < bdiff || (od == bdiff && orr < brank)) {
      bdiff = od;
      brank = orr;
    }
  }
  return (total == 0 || brank == UINT32_MAX) ? 0u : dvals[brank];
}

// Eq. 1-3. maxW(G, ratio) is read from RtoW at index floor(ratio * (R - 1));
// Eq. 2 is evaluated as -expm1(log1p(-prob) / (prob * highD)). Every
// operation is an explicitly rounded IEEE double operation (no contraction).
__device__ __forceinline__ int64_t dev_gap(uint64_t sumd, uint64_t highd, uint64_t two_m, uint32_t alpha,
                                           double beta, const uint32_t* rtow) {
  const uint32_t R = EIC_RATIO_NUM;
  if (highd <= alpha || two_m == 0) return (int64_t)rtow[R - 1];
  uint64_t big = sumd > two_m - sumd ? sumd : two_m - sumd;
  double frac = __ddiv_rn((double)big, (double)two_m);
  double prob = frac < beta ? frac : beta;
  double ratio = -expm1(__ddiv_rn(log1p(-prob), __dmul_rn(prob, (double)highd)));
  double pos = __dmul_rn(ratio, (double)(R - 1));
  uint32_t idx = pos <= 0.0 ? 0u : (pos >= (double)(R - 1) ? R - 1 : (uint32_t)floor(pos));
  return (int64_t)rtow[idx];
}

// Profit of candidate x for the next pair <lb, y> (Section 3.2):
//   x' = max(x, lb - maxW), ub0 = min(y, lb + maxW), ub1 = min(y, x' + maxW),
//   dsum = sumD(x') - sumD(lb),
//   pushed = (ub0 - lb) dsum / maxW, pulled = (ub1 - x') sumD(lb) / maxW,
//   long = pulled dsum / 2|E|,  profit = pushed - long - pulled.
__device__ __forceinline__ double dev_profit(int64_t x, int64_t lb, int64_t y, uint64_t dsum, uint64_t sumd_lb,
                                             uint32_t maxw, uint64_t two_m) {
  int64_t xc = x > lb - (int64_t)maxw ? x : lb - (int64_t)maxw;
  int64_t ub0 = y < lb + (int64_t)maxw ? y : lb + (int64_t)maxw;
  int64_t ub1 = y < xc + (int64_t)maxw ? y : xc + (int64_t)maxw;
  double pushed = __ddiv_rn(__dmul_rn((double)(ub0 - lb), (double)dsum), (double)maxw);
  double pulled = __ddiv_rn(__dmul_rn((double)(ub1 - xc), (double)sumd_lb), (double)maxw);
  double lng = __ddiv_rn(__dmul_rn(pulled, (double)dsum), (double)two_m);
  return __dsub_rn(__dsub_rn(pushed, lng), pulled);
}

}  // namespace eic

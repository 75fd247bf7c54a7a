// Single-source query by Algorithm 1 of the EIC method: steps with
// scheduling pairs <lb, ub> (dynamic stepping, Eq. 1-3), a selection
// threshold st per step (traversal optimisation, Function 2) and rounds of
// window-filtered edge relaxations (Function 1 and the inner loop of
// Algorithm 1), as one persistent cooperative kernel on sm_103a.
//
// Device layout per query (workspace, reused across queries of one graph):
//   dist[n]      caller's buffer, u32, +inf = 0xFFFFFFFF, updated by atomicMin
//   stamp[n]     round id of the last frontier insertion (the SAP of Algorithm 1)
//   q[2][n]      frontier queues, one per round parity
//   settled[n]   vertices in settling order; step k owns [step_off[k], step_off[k+1])
//   touched[n]   first-step insertions (the first step's ub shrinks, so its
//                tentative distances >= the final ub are reset to +inf)
//   ul[2][n]     compacted unsettled lists for the pull of Function 1
//   hist[D]      unsettled vertices per distinct degree (for highD)
//   ring[R]      degree sums of settled vertices by distance mod R (for the
//                sumD differences of Function 2's candidates)
//   heavy[]      long windows spread over the whole grid
//
// Phases (one grid barrier each): a round over the frontier (the first round
// of a step also runs Function 1's push set and pull), an optional heavy
// phase, and per step one statistics pass whose last block evaluates
// Eq. 1-3 and Function 2 and publishes the next <st, lb, ub>.
#include <stdlib.h>
#include <string.h>

#include "graph.h"
#include "stats.cuh"

using namespace eic;

namespace {

constexpr uint32_t kModePush = 0;     // frontier vertex: relax its window
constexpr uint32_t kModePushSet = 1;  // settled vertex of Function 1's push set
constexpr uint32_t kModePull = 2;     // unsettled vertex pulling over its light prefix
constexpr int kMaxWarps = 32;
constexpr int kShRanks = 1024;
constexpr int kShRing = 2048;
constexpr uint64_t kMask40 = (1ull << 40) - 1;
constexpr uint32_t kHeavyChunk = 256;

struct KArgs {
  DevGraph G;
  uint32_t* dist;
  uint32_t* stamp;
  uint32_t* q0;
  uint32_t* q1;
  uint32_t* settled;
  uint32_t* touched;
  uint32_t* ul0;
  uint32_t* ul1;
  uint32_t* hist;
  unsigned long long* ring;
  HeavyItem* heavy;
  int64_t* step_ub;
  uint32_t* step_off;
  eic_step* trace;
  Ctl* ctl;
  int* status_out;
  uint32_t s;
  uint32_t alpha;
  double beta;
  uint32_t st_num;
  uint32_t gap_shift;
  uint32_t heavy_min;
  uint64_t max_spin;
  uint32_t flags;
  uint32_t ring_mask, ring_shift;
  uint32_t heavy_cap, step_cap, trace_cap;
};

struct WarpScr {
  unsigned long long beg[32];
  uint32_t excl[32];
  uint32_t u[32];
  uint32_t d[32];
  uint32_t best[32];
  uint32_t mode[32];
};

struct S2Scr {
  uint32_t hist[kShRanks];
  unsigned long long ring[kShRing];
};

struct S3Scr {
  unsigned long long part[1024];
  double bp[32];
  uint32_t bk[32];
};

union PhaseScr {
  WarpScr w[kMaxWarps];
  S2Scr s2;
  S3Scr s3;
};

// Control values every block holds between barriers.
struct Local {
  int64_t lb, ub, st, lb0;
  uint32_t step, rid, qsel, cur_cnt, rin;
  uint32_t push_beg, push_end, pull_on, pull_src, pull_cnt, extra_s, step_off_cur, ul_out;
};

struct Counters {
  unsigned long long frontier, trav, pulls, improved, heavy;
};

template <typename T>
__device__ __forceinline__ T vload(const T* p) {
  return *(const volatile T*)p;
}

__device__ __forceinline__ int64_t d64(uint32_t d) { return d == EIC_INF ? EIC_INF_T : (int64_t)d; }

// first index in [b, e) of the weight-sorted row with weight >= t
__device__ __forceinline__ uint64_t lower_bound_w(const uint2* __restrict__ adj, uint64_t b, uint64_t e, int64_t t) {
  if (t <= 1) return b;  // weights are >= 1
  while (b < e) {
    uint64_t mid = b + ((e - b) >> 1);
    if ((int64_t)__ldg(&adj[mid].y) < t)
      b = mid + 1;
    else
      e = mid;
  }
  return b;
}

struct RoundCtx {
  int64_t lb, ub, ub_eff, st, lb0;
  uint32_t rid;
  bool step1;
  uint32_t* qout;
  uint32_t* qcnt_out;
  uint32_t* first_list;
  uint32_t* first_cnt;
  uint32_t* ul_out;
  uint32_t* ulcnt_out;
  unsigned long long* heavy_ctr;
};

// Successful relaxation of v to nd (old = previous distance): SAP into the
// next frontier, first insertion into the settled (or first-step) list, and
// in the first step the running min over high-degree vertices that becomes
// ub (Algorithm 1). Warp-collective: every lane calls it.
__device__ __forceinline__ void on_success(const KArgs& A, const RoundCtx& R, bool ok, uint32_t v, uint32_t nd,
                                           uint32_t old, Counters& C) {
  bool sap = ok && (atomicExch(&A.stamp[v], R.rid) != R.rid);
  uint32_t slot = warp_append(sap, R.qcnt_out);
  if (sap) __stcg(&R.qout[slot], v);
  bool first = ok && old == EIC_INF;
  uint32_t slot2 = warp_append(first, R.first_cnt);
  if (first) __stcg(&R.first_list[slot2], v);
  if (R.step1 && ok) {
    uint64_t dg = __ldg(&A.G.row[v + 1]) - __ldg(&A.G.row[v]);
    if (dg >= A.G.highd0) atomicMin(&A.ctl->ub_cand, nd);
  }
  C.improved += ok ? 1 : 0;
}

// One warp, up to 32 items: windows by binary search in the weight-sorted
// rows, long windows handed to the heavy list, the rest relaxed cooperatively
// over the concatenation of the warp's windows.
__device__ void process_items(const KArgs& A, const RoundCtx& R, WarpScr& S, const Local& L, uint32_t base,
                              uint32_t nitems, bool round1, const uint32_t* qin, const uint32_t* pull_list,
                              Counters& C) {
  const uint32_t lane = lane_id();
  const uint32_t i = base + lane;
  const bool valid = i < nitems;
  uint32_t mode = kModePush, u = 0;
  if (valid) {
    if (!round1) {
      u = __ldcg(&qin[i]);
    } else {
      uint32_t np = L.push_end - L.push_beg;
      if (i < np) {
        u = __ldcg(&A.settled[L.push_beg + i]);
        mode = kModePushSet;
      } else if (i < np + L.pull_cnt) {
        u = __ldcg(&pull_list[i - np]);
        mode = kModePull;
      } else {
        u = A.s;
      }
    }
  }
  uint32_t d = valid ? __ldcg(&A.dist[u]) : EIC_INF;
  uint64_t b = 0, e = 0;
  bool keep_ul = false, counted = false;
  if (valid) {
    const uint64_t rb = __ldg(&A.G.row[u]), re = __ldg(&A.G.row[u + 1]);
    if (mode == kModePull) {
      int64_t dd = d64(d);
      if (dd >= R.lb) {
        keep_ul = true;
        if (dd > R.lb) {
          b = rb;
          e = lower_bound_w(A.G.adj, rb, re, R.ub - R.st);
        }
      }
    } else {
      bool skip = d == EIC_INF || (mode == kModePushSet && ((int64_t)d < R.lb0 || (int64_t)d > R.st)) ||
                  (d > 0 && re - rb == 1);  // Paths excludes leaves (Algorithm 1)
      if (!skip) {
        counted = true;
        int64_t hi = R.ub_eff - (int64_t)d;
        if (hi > 0) {
          b = lower_bound_w(A.G.adj, rb, re, R.lb - (int64_t)d);
          e = lower_bound_w(A.G.adj, b, re, hi);
        }
      }
    }
  }
  C.frontier += counted ? 1 : 0;
  uint32_t us = warp_append(keep_ul, R.ulcnt_out);
  if (keep_ul) __stcg(&R.ul_out[us], u);
  uint64_t len = e - b;
  if (mode == kModePull) C.pulls += len;
  C.trav += len;
  if (len > A.heavy_min) {
    unsigned long long old = atomicAdd(R.heavy_ctr, (1ull << 40) | len);
    uint32_t idx = (uint32_t)(old >> 40);
    HeavyItem h;
    h.beg = b;
    h.prefix = old & kMask40;
    h.u = u;
    h.d = d;
    h.mode = mode == kModePull ? kModePull : kModePush;
    h.pad = 0;
    A.heavy[idx] = h;  // capacity covers 2m / heavy_min items per round
    C.heavy += 1;
    len = 0;
  }
  const uint32_t len32 = (uint32_t)len;
  const uint32_t incl = warp_incl_scan(len32);
  const uint32_t total = __shfl_sync(EIC_FULL_MASK, incl, 31);
  S.beg[lane] = b;
  S.excl[lane] = incl - len32;
  S.u[lane] = u;
  S.d[lane] = d;
  S.mode[lane] = mode;
  S.best[lane] = EIC_INF;
  __syncwarp();
  for (uint32_t g0 = 0; g0 < total; g0 += 32) {
    const uint32_t g = g0 + lane;
    const bool act = g < total;
    bool ok = false;
    uint32_t v = 0, nd = 0, old = 0;
    if (act) {
      uint32_t lo = 0, hi = 31;
      while (lo < hi) {  // last lane whose window starts at or before g
        uint32_t mid = (lo + hi + 1) >> 1;
        if (S.excl[mid] <= g)
          lo = mid;
        else
          hi = mid - 1;
      }
      const uint2 ent = __ldg(&A.G.adj[S.beg[lo] + (g - S.excl[lo])]);
      v = ent.x;
      const uint32_t dv = __ldcg(&A.dist[v]);
      if (S.mode[lo] != kModePull) {
        nd = S.d[lo] + ent.y;  // inside [lb, min(ub, 2^32-1)) by the window bounds
        if (nd < dv) {
          old = atomicMin(&A.dist[v], nd);
          ok = nd < old;
        }
      } else if (dv != EIC_INF) {
        const int64_t dvv = dv;
        if (dvv >= R.st && dvv < R.lb && dvv + ent.y < R.ub) atomicMin(&S.best[lo], (uint32_t)(dvv + ent.y));
      }
    }
    on_success(A, R, ok, v, nd, old, C);
  }
  __syncwarp();
  bool pok = false;
  uint32_t pold = 0;
  const uint32_t pbest = S.best[lane];
  if (valid && mode == kModePull && pbest < d) {
    pold = atomicMin(&A.dist[u], pbest);
    pok = pbest < pold;
  }
  on_success(A, R, pok, u, pbest, pold, C);
  __syncwarp();
}

// Heavy windows of this round, 256 entries per warp task over the grid.
__device__ void heavy_phase(const KArgs& A, const RoundCtx& R, unsigned long long packed, Counters& C) {
  const uint32_t cnt = (uint32_t)(packed >> 40);
  const uint64_t total = packed & kMask40;
  const uint32_t lane = lane_id();
  const uint32_t wpb = blockDim.x >> 5;
  const uint64_t nwarps = (uint64_t)gridDim.x * wpb;
  const uint64_t nch = (total + kHeavyChunk - 1) / kHeavyChunk;
  for (uint64_t c = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5); c < nch; c += nwarps) {
    const uint64_t e0 = c * kHeavyChunk, e1 = e0 + kHeavyChunk < total ? e0 + kHeavyChunk : total;
    uint32_t j = 0;
    if (lane == 0) {
      uint32_t lo = 0, hi = cnt - 1;
      while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (__ldcg(&A.heavy[mid].prefix) <= e0)
          lo = mid;
        else
          hi = mid - 1;
      }
      j = lo;
    }
    j = __shfl_sync(EIC_FULL_MASK, j, 0);
    for (uint64_t g0 = e0; g0 < e1; g0 += 32) {
      const uint64_t g = g0 + lane;
      const bool act = g < e1;
      bool ok = false;
      uint32_t v = 0, nd = 0, old = 0;
      if (act) {
        uint32_t jj = j;
        while (jj + 1 < cnt && __ldcg(&A.heavy[jj + 1].prefix) <= g) ++jj;
        const uint64_t hb = __ldcg(&A.heavy[jj].beg), hp = __ldcg(&A.heavy[jj].prefix);
        const uint32_t hu = __ldcg(&A.heavy[jj].u), hd = __ldcg(&A.heavy[jj].d), hm = __ldcg(&A.heavy[jj].mode);
        const uint2 ent = __ldg(&A.G.adj[hb + (g - hp)]);
        const uint32_t dv = __ldcg(&A.dist[ent.x]);
        if (hm != kModePull) {
          v = ent.x;
          nd = hd + ent.y;
          if (nd < dv) {
            old = atomicMin(&A.dist[v], nd);
            ok = nd < old;
          }
        } else if (dv != EIC_INF) {
          const int64_t dvv = dv;
          if (dvv >= R.st && dvv < R.lb && dvv + ent.y < R.ub) {
            v = hu;
            nd = (uint32_t)(dvv + ent.y);
            old = atomicMin(&A.dist[v], nd);
            ok = nd < old;
          }
        }
      }
      on_success(A, R, ok, v, nd, old, C);
    }
  }
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long x, unsigned long long* sh) {
  x = warp_sum_u64(x);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  unsigned long long t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
    t = warp_sum_u64(t);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// Function 2 for the boundary <lb, ub> -> next pair <ub, ub + gap(ub)>, run by
// one whole block. Candidates x_k = st0 + floor(k (st1 - st0) / ST_NUM) < ub;
// D(x') = sumD(x') - sumD(ub) from the ring of settled degree sums.
__device__ int64_t block_compute_st(const KArgs& A, S3Scr& S, int64_t ub, uint64_t sumd_ub, int64_t gap_lb,
                                    int64_t gap_ub_raw, int64_t y, int64_t st0, int64_t st1) {
  const int64_t maxw = A.G.maxw;
  if (sumd_ub >= A.G.m || gap_lb == maxw) return ub;
  if (gap_ub_raw == maxw) return ub - maxw;
  const uint32_t t = threadIdx.x, nt = blockDim.x;
  const int64_t wl = ub - maxw > 0 ? ub - maxw : 0;
  const uint32_t sh = A.ring_shift;
  const uint64_t sl = (uint64_t)wl >> sh, su = (uint64_t)(ub - 1) >> sh;
  const uint64_t L = su - sl + 1;  // ring slots covering [wl, ub)
  const uint64_t cs = (L + nt - 1) / nt;
  unsigned long long mine = 0;
  for (uint64_t q = sl + t * cs; q < sl + (t + 1) * cs && q <= su; ++q) mine += __ldcg(&A.ring[q & A.ring_mask]);
  S.part[t] = mine;
  __syncthreads();
  // suffix sums: part[t] <- sum over chunks after t
  for (uint32_t o = 1; o < nt; o <<= 1) {
    unsigned long long v = t + o < nt ? S.part[t + o] : 0;
    __syncthreads();
    S.part[t] += v;
    __syncthreads();
  }
  double best = 0.0;
  uint32_t bk = 0xFFFFFFFFu;
  for (uint32_t k = t; k <= A.st_num; k += nt) {
    const int64_t x = st0 + (int64_t)(((uint64_t)k * (uint64_t)(st1 - st0)) / A.st_num);
    if (x >= ub) continue;
    const int64_t xc = x > ub - maxw ? x : ub - maxw;
    const uint64_t q0 = (uint64_t)xc >> sh;
    const uint64_t c = (q0 - sl) / cs;
    unsigned long long dsum = c + 1 < nt ? S.part[c + 1] : 0;
    for (uint64_t q = q0; q < sl + (c + 1) * cs && q <= su; ++q) dsum += __ldcg(&A.ring[q & A.ring_mask]);
    const double p = dev_profit(x, ub, y, dsum, sumd_ub, A.G.maxw, A.G.two_m);
    if (p > best) {
      best = p;
      bk = k;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_down_sync(EIC_FULL_MASK, best, o);
    uint32_t ok = __shfl_down_sync(EIC_FULL_MASK, bk, o);
    if (ob > best || (ob == best && ok < bk)) {
      best = ob;
      bk = ok;
    }
  }
  __syncthreads();
  if ((t & 31) == 0) {
    S.bp[t >> 5] = best;
    S.bk[t >> 5] = bk;
  }
  __syncthreads();
  if (t < 32) {
    best = t < (nt >> 5) ? S.bp[t] : 0.0;
    bk = t < (nt >> 5) ? S.bk[t] : 0xFFFFFFFFu;
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(EIC_FULL_MASK, best, o);
      uint32_t ok = __shfl_down_sync(EIC_FULL_MASK, bk, o);
      if (ob > best || (ob == best && ok < bk)) {
        best = ob;
        bk = ok;
      }
    }
    if (t == 0) S.bk[0] = bk;
  }
  __syncthreads();
  const uint32_t k = S.bk[0];
  __syncthreads();
  if (k == 0xFFFFFFFFu) return ub;
  return st0 + (int64_t)(((uint64_t)k * (uint64_t)(st1 - st0)) / A.st_num);
}

// Step boundary, executed by the last block to finish the statistics pass:
// sumD(ub), highD(ub), gap(ub) (Eq. 1-3), termination (Algorithm 1),
// computeST (Function 2) and the push/pull sets of the next step's
// Function 1. Publishes the new control values before the grid barrier.
__device__ void step_boundary(const KArgs& A, PhaseScr& P, const Local& L, uint32_t rounds_in_step) {
  Ctl* c = A.ctl;
  __shared__ int64_t sh_i[8];
  __shared__ uint64_t sh_u[4];
  __shared__ uint32_t sh_flag[2];
  const DevGraph& G = A.G;
  const int64_t lb = L.lb, ub = L.ub;
  const uint32_t k = L.step;
  if (threadIdx.x == 0) {
    const uint64_t settled_now = vload(&c->settled_cnt);
    const uint64_t acc = vload(&c->acc_deg);
    const uint64_t sumd_ub = vload(&c->sumd_lb) - acc;
    sh_u[0] = sumd_ub;
    sh_u[1] = settled_now;
    int64_t maxs = vload(&c->max_settled);
    if (vload(&c->acc_any)) {
      int64_t am = (int64_t)vload(&c->acc_maxd);
      maxs = am > maxs ? am : maxs;
    }
    c->max_settled = maxs;
    sh_i[0] = maxs;
    // step table and trace row of step k
    A.step_ub[k] = ub;
    if (k <= A.trace_cap && A.trace) {
      eic_step r;
      r.lb = lb;
      r.ub = ub;
      r.st = L.st;
      r.gap_lb = vload(&c->gap_lb);
      r.sumd_lb = vload(&c->sumd_lb);
      r.highd_lb = vload(&c->highd_lb);
      r.rounds = rounds_in_step;
      r.settled = settled_now - L.step_off_cur;
      A.trace[k - 1] = r;
    }
    c->trace_len = k;
    // termination / overflow (Algorithm 1): max{finite dist} + maxW(G,1) < lb
    uint32_t done = 0;
    if (maxs + (int64_t)G.maxw >= (int64_t)EIC_INF) {
      atomicCAS(&c->status, 0, EIC_EOVERFLOW);
      done = 1;
    } else if (maxs + (int64_t)G.maxw < ub) {
      done = 1;
    } else if (k + 1 >= A.step_cap) {
      atomicCAS(&c->status, 0, EIC_ENOMEM);
      done = 1;
    }
    sh_flag[0] = done;
  }
  __syncthreads();
  const uint64_t sumd_ub = sh_u[0];
  const uint32_t highd_ub = block_highd(A.hist, G.dvals, G.D);
  if (sh_flag[0]) {
    if (threadIdx.x == 0) {
      c->done = 1;
      __threadfence();
    }
    __syncthreads();
    return;
  }
  int64_t gap_raw = 0, width = 0, st0 = 0, st1 = 0, gap_lb = 0;
  if (threadIdx.x == 0) {
    gap_raw = dev_gap(sumd_ub, highd_ub, G.two_m, A.alpha, A.beta, G.rtow);
    width = gap_raw << A.gap_shift;
    st0 = k == 1 ? ub : vload(&c->st0);
    st1 = vload(&c->st1);
    if (st1 < 0 && sumd_ub <= G.m) st1 = ub;
    c->st0 = st0;
    c->st1 = st1;
    gap_lb = vload(&c->gap_lb);
    sh_i[1] = gap_raw;
    sh_i[2] = width;
    sh_i[3] = st0;
    sh_i[4] = st1;
    sh_i[5] = gap_lb;
  }
  __syncthreads();
  gap_raw = sh_i[1];
  width = sh_i[2];
  st0 = sh_i[3];
  st1 = sh_i[4];
  gap_lb = sh_i[5];
  const int64_t nlb = ub, nub = ub + width;
  int64_t nst = (A.flags & EIC_FLAG_NO_PULL)
                    ? nlb
                    : block_compute_st(A, P.s3, ub, sumd_ub, gap_lb, gap_raw, nub, st0, st1);
  // zero the ring slots the next step's statistics will fill: [max(nlb, nub - maxW), nub)
  {
    const int64_t zl = nub - (int64_t)G.maxw > nlb ? nub - (int64_t)G.maxw : nlb;
    const uint64_t ql = (uint64_t)zl >> A.ring_shift, qu = (uint64_t)(nub - 1) >> A.ring_shift;
    for (uint64_t q = ql + threadIdx.x; q <= qu; q += blockDim.x) __stcg(&A.ring[q & A.ring_mask], 0ull);
  }
  if (threadIdx.x == 0) {
    const uint32_t settled_now = (uint32_t)sh_u[1];
    A.step_off[k + 1] = settled_now;
    uint32_t scnt = settled_now;
    uint32_t extra = 0;
    if (k == 1 && ub == 0) {  // the source itself was not settled by the first step
      A.settled[scnt++] = A.s;
      extra = 1;
    }
    // Function 1's push set {lb0 <= dist <= st} from the settled steps
    const int64_t lb0 = nlb - (int64_t)G.maxw > 0 ? nlb - (int64_t)G.maxw : 0;
    uint32_t pb = 0, pe = 0;
    if (nst >= lb0) {
      uint32_t lo = 1, hi = k + 1;  // first step j with ub_j > lb0
      while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (A.step_ub[mid] > lb0)
          hi = mid;
        else
          lo = mid + 1;
      }
      const uint32_t j0 = lo;
      lo = 1;
      hi = k;  // last step j with lb_j <= nst (lb_1 = 0, lb_j = ub_{j-1})
      while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (A.step_ub[mid - 1] <= nst)
          lo = mid;
        else
          hi = mid - 1;
      }
      const uint32_t j1 = lo;
      if (j0 <= j1) {
        pb = A.step_off[j0];
        pe = A.step_off[j1 + 1];
      }
    }
    // Function 1's pull over the unsettled vertices when st < lb
    uint32_t pull_on = nst < nlb ? 1u : 0u, pull_src = 0, pull_cnt = 0, ul_out = 0;
    uint32_t ul_valid = vload(&c->ul_valid), ul_sel = vload(&c->ul_sel);
    if (L.pull_on) {  // the step just finished pulled into ul[L.ul_out]
      ul_valid = 1;
      ul_sel = L.ul_out;
    }
    if (pull_on) {
      if (ul_valid) {
        pull_src = 1 + ul_sel;
        pull_cnt = vload(&c->ulcnt[ul_sel]);
        ul_out = ul_sel ^ 1u;
      } else {
        pull_src = 0;
        pull_cnt = G.nz_count;
        ul_out = 0;
      }
      c->ulcnt[ul_out] = 0;
    }
    c->ul_valid = ul_valid;
    c->ul_sel = ul_sel;
    c->settled_cnt = scnt;
    c->lb = nlb;
    c->ub = nub;
    c->st = nst;
    c->lb0 = lb0;
    c->step = k + 1;
    c->push_beg = pb;
    c->push_end = pe;
    c->pull_on = pull_on;
    c->pull_src = pull_src;
    c->pull_cnt = pull_cnt;
    c->extra_s = extra;
    c->step_off_cur = settled_now;
    c->ul_out = ul_out;
    c->sumd_lb = sumd_ub;
    c->highd_lb = highd_ub;
    c->gap_lb = gap_raw;
    c->acc_deg = 0;
    c->acc_maxd = 0;
    c->acc_any = 0;
    c->s2_done = 0;
    c->done = 0;
    __threadfence();
  }
  __syncthreads();
}

__device__ void read_ctl(const Ctl* c, Local& L) {
  L.lb = vload(&c->lb);
  L.ub = vload(&c->ub);
  L.st = vload(&c->st);
  L.lb0 = vload(&c->lb0);
  L.step = vload(&c->step);
  L.push_beg = vload(&c->push_beg);
  L.push_end = vload(&c->push_end);
  L.pull_on = vload(&c->pull_on);
  L.pull_src = vload(&c->pull_src);
  L.pull_cnt = vload(&c->pull_cnt);
  L.extra_s = vload(&c->extra_s);
  L.step_off_cur = vload(&c->step_off_cur);
  L.ul_out = vload(&c->ul_out);
}

__global__ void __launch_bounds__(1024) k_eic(KArgs A) {
  __shared__ PhaseScr P;
  __shared__ unsigned long long sh_red[32];
  __shared__ uint32_t sh_last;
  Ctl* c = A.ctl;
  uint32_t gen = vload(&c->bar.gen);
  Local L;
  read_ctl(c, L);
  L.rid = vload(&c->round_base);
  L.qsel = 0;
  L.cur_cnt = 1;  // the first round's frontier is {s}
  Counters C = {0, 0, 0, 0, 0};
  const uint32_t warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const uint32_t gwarp = blockIdx.x * wpb + warp, nwarps = gridDim.x * wpb;
  bool alive = true;
  uint32_t total_rounds = 0;
  constexpr uint32_t kMaxRounds = 1u << 22;  // every block counts the same rounds and stops together
  while (alive) {
    // ------------------------------------------------ rounds of one step
    uint32_t rin = 0;
    for (;;) {
      ++L.rid;
      if (++total_rounds > kMaxRounds) {
        if (threadIdx.x == 0) atomicCAS(&c->status, 0, EIC_ETIMEOUT);
        alive = false;
        break;
      }
      const bool round1 = (L.step >= 2 && rin == 0);
      // counters of round rid+1 were last read two barriers ago: clear them now
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->qcnt[(L.rid + 1) % 3] = 0;
        c->heavy_packed[(L.rid + 1) % 3] = 0;
      }
      RoundCtx R;
      R.lb = L.lb;
      R.ub = L.ub;
      R.ub_eff = L.ub < (int64_t)EIC_INF ? L.ub : (int64_t)EIC_INF;
      R.st = L.st;
      R.lb0 = L.lb0;
      R.rid = L.rid;
      R.step1 = L.step == 1;
      R.qout = L.qsel ? A.q0 : A.q1;
      R.qcnt_out = &c->qcnt[L.rid % 3];
      R.first_list = R.step1 ? A.touched : A.settled;
      R.first_cnt = R.step1 ? &c->touched_cnt : &c->settled_cnt;
      R.ul_out = L.ul_out ? A.ul1 : A.ul0;
      R.ulcnt_out = &c->ulcnt[L.ul_out];
      R.heavy_ctr = &c->heavy_packed[L.rid % 3];
      const uint32_t* qin = L.qsel ? A.q1 : A.q0;
      const uint32_t* pull_list = L.pull_src == 0 ? A.G.nz : (L.pull_src == 1 ? A.ul0 : A.ul1);
      uint32_t nitems;
      if (round1)
        nitems = (L.push_end - L.push_beg) + (L.pull_on ? L.pull_cnt : 0) + L.extra_s;
      else
        nitems = L.cur_cnt;
      for (uint32_t base = gwarp * 32; base < nitems; base += nwarps * 32)
        process_items(A, R, P.w[warp], L, base, nitems, round1, qin, pull_list, C);
      if (!grid_barrier(&c->bar, &gen, A.max_spin, &c->status)) {
        alive = false;
        break;
      }
      const unsigned long long hp = vload(&c->heavy_packed[L.rid % 3]);
      if (hp != 0) {
        heavy_phase(A, R, hp, C);
        if (!grid_barrier(&c->bar, &gen, A.max_spin, &c->status)) {
          alive = false;
          break;
        }
      }
      if (R.step1) {
        const uint32_t uc = vload(&c->ub_cand);
        if (uc != EIC_INF && (int64_t)uc < L.ub) L.ub = uc;
      }
      L.cur_cnt = vload(&c->qcnt[L.rid % 3]);
      L.qsel ^= 1u;
      ++rin;
      if (L.cur_cnt == 0) break;
    }
    if (!alive) break;
    // ------------------------------------------------ statistics pass (S2)
    {
      S2Scr& S = P.s2;
      for (int r = threadIdx.x; r < kShRanks; r += blockDim.x) S.hist[r] = 0;
      const int64_t wlo = L.ub - (int64_t)A.G.maxw > L.lb ? L.ub - (int64_t)A.G.maxw : L.lb;
      const bool ring_sh = A.ring_shift == 0 && L.ub < EIC_INF_T && (L.ub - wlo) <= kShRing;
      if (ring_sh)
        for (int r = threadIdx.x; r < kShRing; r += blockDim.x) S.ring[r] = 0;
      __syncthreads();
      const bool step1 = L.step == 1;
      const uint32_t* list = step1 ? A.touched : A.settled;
      const uint32_t lbeg = step1 ? 0 : L.step_off_cur;
      const uint32_t lend = step1 ? vload(&c->touched_cnt) : vload(&c->settled_cnt);
      unsigned long long bdeg = 0;
      uint32_t bmax = 0, bany = 0;
      const uint32_t nthreads = gridDim.x * blockDim.x;
      for (uint32_t base = lbeg + blockIdx.x * blockDim.x; base < lend; base += nthreads) {
        const uint32_t idx = base + threadIdx.x;
        bool take = false;
        uint32_t x = 0, d = 0;
        if (idx < lend) {
          x = __ldcg(&list[idx]);
          d = __ldcg(&A.dist[x]);
          take = true;
          if (step1 && d64(d) >= L.ub) {  // first step: keep only what is final
            if (x != A.s) __stcg(&A.dist[x], EIC_INF);
            take = false;
          }
        }
        if (step1) {
          uint32_t slot = warp_append(take, &c->settled_cnt);
          if (take) __stcg(&A.settled[slot], x);
        }
        if (take) {
          const uint32_t dg = (uint32_t)(__ldg(&A.G.row[x + 1]) - __ldg(&A.G.row[x]));
          if (dg > 0) {  // degree-0 vertices (an isolated source) carry no rank
            const uint32_t r = __ldg(&A.G.drank[dg]);
            if (r < (uint32_t)kShRanks)
              atomicAdd(&S.hist[r], 1u);
            else
              atomicSub(&A.hist[r], 1u);
          }
          bdeg += dg;
          bmax = d > bmax ? d : bmax;
          bany = 1;
          if ((int64_t)d >= wlo) {
            if (ring_sh)
              atomicAdd(&S.ring[d - wlo], (unsigned long long)dg);
            else
              atomicAdd(&A.ring[((uint64_t)d >> A.ring_shift) & A.ring_mask], (unsigned long long)dg);
          }
        }
      }
      __syncthreads();
      for (int r = threadIdx.x; r < kShRanks; r += blockDim.x)
        if (S.hist[r]) atomicSub(&A.hist[r], S.hist[r]);
      if (ring_sh)
        for (int r = threadIdx.x; r < kShRing && r < L.ub - wlo; r += blockDim.x)
          if (S.ring[r]) atomicAdd(&A.ring[((uint64_t)(wlo + r)) & A.ring_mask], S.ring[r]);
      const unsigned long long tdeg = block_sum_u64(bdeg, sh_red);
      for (int o = 16; o > 0; o >>= 1) {
        bmax = max(bmax, __shfl_xor_sync(EIC_FULL_MASK, bmax, o));
        bany |= __shfl_xor_sync(EIC_FULL_MASK, bany, o);
      }
      if ((threadIdx.x & 31) == 0 && bany) {
        atomicMax(&c->acc_maxd, bmax);
        atomicOr(&c->acc_any, 1u);
      }
      const unsigned long long f = block_sum_u64(C.frontier, sh_red);
      const unsigned long long tr = block_sum_u64(C.trav, sh_red);
      const unsigned long long pl = block_sum_u64(C.pulls, sh_red);
      const unsigned long long im = block_sum_u64(C.improved, sh_red);
      const unsigned long long hv = block_sum_u64(C.heavy, sh_red);
      C = {0, 0, 0, 0, 0};
      if (threadIdx.x == 0) {
        if (tdeg) atomicAdd(&c->acc_deg, tdeg);
        atomicAdd(&c->cnt_frontier, f);
        atomicAdd(&c->cnt_trav, tr);
        atomicAdd(&c->cnt_pulls, pl);
        atomicAdd(&c->cnt_improved, im);
        atomicAdd(&c->cnt_heavy, hv);
        __threadfence();
        sh_last = atomicAdd(&c->s2_done, 1u) == gridDim.x - 1 ? 1u : 0u;
      }
      __syncthreads();
      if (sh_last) {
        __threadfence();
        if (threadIdx.x == 0) c->cnt_rounds += rin;
        step_boundary(A, P, L, rin);
      }
    }
    if (!grid_barrier(&c->bar, &gen, A.max_spin, &c->status)) break;
    if (vload(&c->done)) break;
    read_ctl(c, L);
    L.cur_cnt = 0;
  }
  // the next query's stamp ids start above every id any block used
  if (threadIdx.x == 0) atomicMax(&c->round_base, L.rid);
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.status_out) *A.status_out = vload(&c->status);
}

__global__ void k_init(KArgs A) {
  Ctl* c = A.ctl;
  const DevGraph& G = A.G;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < G.D; r += gridDim.x * blockDim.x) A.hist[r] = G.dcnt0[r];
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r <= A.ring_mask; r += gridDim.x * blockDim.x) A.ring[r] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.dist[A.s] = 0;
    A.q0[0] = A.s;
    A.touched[0] = A.s;
    A.step_off[1] = 0;
    A.step_ub[0] = 0;
    const uint64_t dgs = G.row[A.s + 1] - G.row[A.s];
    c->lb = 0;
    c->ub = EIC_INF_T;
    c->st = 0;
    c->lb0 = 0;
    c->step = 1;
    c->done = 0;
    c->push_beg = c->push_end = 0;
    c->pull_on = c->pull_src = c->pull_cnt = c->extra_s = 0;
    c->step_off_cur = 0;
    c->ul_out = 0;
    c->st0 = -1;
    c->st1 = -1;
    c->sumd_lb = G.two_m;
    c->highd_lb = G.highd0;
    c->gap_lb = dev_gap(G.two_m, G.highd0, G.two_m, A.alpha, A.beta, G.rtow);
    c->max_settled = -1;
    c->ul_sel = 0;
    c->ul_valid = 0;
    c->rounds_in_step = 0;
    c->trace_len = 0;
    c->qcnt[0] = c->qcnt[1] = c->qcnt[2] = 0;
    c->settled_cnt = 0;
    c->touched_cnt = 1;
    c->ulcnt[0] = c->ulcnt[1] = 0;
    c->ub_cand = (G.highd0 > 0 && dgs >= G.highd0) ? 0u : EIC_INF;
    c->heavy_packed[0] = c->heavy_packed[1] = c->heavy_packed[2] = 0;
    c->s2_done = 0;
    c->acc_maxd = 0;
    c->acc_deg = 0;
    c->acc_any = 0;
    c->cnt_rounds = c->cnt_frontier = c->cnt_trav = c->cnt_pulls = c->cnt_improved = c->cnt_heavy = 0;
    c->bar.count = 0;
    c->status = 0;
  }
}

// parent[v] = smallest-id u with dist[u] + w(u, v) == dist[v]; one warp per vertex.
__global__ void k_parent(DevGraph G, const uint32_t* __restrict__ dist, uint32_t s, uint32_t* parent) {
  const uint32_t lane = lane_id();
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t v = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < G.n; v += nw) {
    const uint32_t dv = dist[v];
    uint32_t best = EIC_INF;
    if (v != s && dv != EIC_INF) {
      const uint64_t rb = G.row[v], re = G.row[v + 1];
      for (uint64_t i = rb + lane; i < re; i += 32) {
        const uint2 ent = G.adj[i];
        if (ent.y > dv) break;
        const uint32_t du = dist[ent.x];
        if (du != EIC_INF && (uint64_t)du + ent.y == dv && ent.x < best) best = ent.x;
      }
      for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(EIC_FULL_MASK, best, o));
    }
    if (lane == 0) parent[v] = v == s ? s : best;
  }
}

}  // namespace

// ------------------------------------------------------------------ host

namespace {

constexpr uint32_t kStepCap = 1u << 20;     // steps per query
constexpr uint32_t kTraceCap = 1u << 16;    // trace rows kept on the device
constexpr uint32_t kHeavyMinFloor = 256;    // smallest accepted heavy_min
constexpr uint32_t kDefaultHeavyMin = 2048;
constexpr int kDefaultBlock = 512;
constexpr uint32_t kDefaultSpinLog2 = 22;

template <typename T>
int walloc(Workspace* ws, T** p, uint64_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    (void)cudaGetLastError();
    return EIC_ENOMEM;
  }
  ws->bytes += count * sizeof(T);
  return EIC_OK;
}

int resolve_params(const eic_params* in, eic_params* out) {
  if (in) {
    *out = *in;
  } else {
    eic_params_default(out);
  }
  if (!(out->beta > 0.0 && out->beta < 1.0)) return EIC_EINVAL;
  if (out->st_num == 0) return EIC_EINVAL;
  if (out->gap_shift > 16) return EIC_EINVAL;
  if (out->block_threads != 0 &&
      (out->block_threads % 32 != 0 || out->block_threads < 128 || out->block_threads > 1024))
    return EIC_EINVAL;
  if (out->heavy_min == 0) out->heavy_min = kDefaultHeavyMin;
  if (out->heavy_min < kHeavyMinFloor) return EIC_EINVAL;
  if (out->max_spin_log2 == 0) out->max_spin_log2 = kDefaultSpinLog2;
  if (out->max_spin_log2 > 40) return EIC_EINVAL;
  return EIC_OK;
}

struct DeviceGuard {
  int prev = 0;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    (void)cudaGetLastError();
  }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

int launch_shape(Workspace* ws, int block) {
  if (ws->grid && ws->block == block) return EIC_OK;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  EIC_CUDA_TRY(cudaGetDevice(&dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return EIC_ECUDA;
  EIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eic, block, 0));
  if (per_sm < 1) return EIC_ECUDA;
  ws->grid = sms * per_sm;
  ws->block = block;
  return EIC_OK;
}

KArgs make_args(eic_graph* g, uint32_t s, uint32_t* dist, const eic_params& p, int* status_out) {
  Workspace& w = g->ws;
  KArgs A;
  A.G = g->dg;
  A.dist = dist;
  A.stamp = w.stamp;
  A.q0 = w.q[0];
  A.q1 = w.q[1];
  A.settled = w.settled;
  A.touched = w.touched;
  A.ul0 = w.ul[0];
  A.ul1 = w.ul[1];
  A.hist = w.hist;
  A.ring = w.ring;
  A.heavy = w.heavy;
  A.step_ub = w.step_ub;
  A.step_off = w.step_off;
  A.trace = w.trace;
  A.ctl = w.ctl;
  A.status_out = status_out;
  A.s = s;
  A.alpha = p.alpha;
  A.beta = p.beta;
  A.st_num = p.st_num;
  A.gap_shift = p.gap_shift;
  A.heavy_min = p.heavy_min;
  A.max_spin = 1ull << p.max_spin_log2;
  A.flags = p.flags;
  A.ring_mask = (1u << w.ring_bits) - 1u;
  A.ring_shift = w.ring_shift;
  A.heavy_cap = w.heavy_cap;
  A.step_cap = w.step_cap;
  A.trace_cap = kTraceCap;
  return A;
}

// Enqueue one query: dist <- +inf, init, persistent kernel, optional parent.
int enqueue_query(eic_graph* g, uint32_t s, uint32_t* dist, uint32_t* parent, const eic_params& p, int* status_out,
                  cudaStream_t st) {
  Workspace& w = g->ws;
  const int block = p.block_threads ? (int)p.block_threads : kDefaultBlock;
  int rc = launch_shape(&w, block);
  if (rc) return rc;
  if (w.host_round_base > (1u << 30)) {  // keep stamp ids far from wrapping
    EIC_CUDA_TRY(cudaMemsetAsync(w.stamp, 0, (uint64_t)w.n * 4, st));
    EIC_CUDA_TRY(cudaMemsetAsync(&w.ctl->round_base, 0, 4, st));
    w.host_round_base = 0;
  }
  EIC_CUDA_TRY(cudaMemsetAsync(dist, 0xFF, (uint64_t)g->dg.n * 4, st));
  KArgs A = make_args(g, s, dist, p, status_out);
  k_init<<<64, 256, 0, st>>>(A);
  EIC_CUDA_TRY(cudaGetLastError());
  void* args[] = {&A};
  EIC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_eic, dim3(w.grid), dim3(block), args, 0, st));
  if (parent) {
    k_parent<<<1024, 256, 0, st>>>(g->dg, dist, s, parent);
    EIC_CUDA_TRY(cudaGetLastError());
  }
  return EIC_OK;
}

int trivial_query(eic_graph* g, uint32_t s, uint32_t* dist, uint32_t* parent, cudaStream_t st) {
  const uint64_t n = g->dg.n;
  EIC_CUDA_TRY(cudaMemsetAsync(dist, 0xFF, n * 4, st));
  EIC_CUDA_TRY(cudaMemsetAsync(dist + s, 0, 4, st));
  if (parent) {
    EIC_CUDA_TRY(cudaMemsetAsync(parent, 0xFF, n * 4, st));
    EIC_CUDA_TRY(cudaMemcpyAsync(parent + s, &s, 4, cudaMemcpyHostToDevice, st));
  }
  EIC_CUDA_TRY(cudaStreamSynchronize(st));
  return EIC_OK;
}

}  // namespace

void eic_ws_free(Workspace* w) {
  cudaFree(w->stamp);
  cudaFree(w->q[0]);
  cudaFree(w->q[1]);
  cudaFree(w->settled);
  cudaFree(w->touched);
  cudaFree(w->ul[0]);
  cudaFree(w->ul[1]);
  cudaFree(w->hist);
  cudaFree(w->ring);
  cudaFree(w->heavy);
  cudaFree(w->step_ub);
  cudaFree(w->step_off);
  cudaFree(w->trace);
  cudaFree(w->ctl);
  if (w->ctl_host) cudaFreeHost(w->ctl_host);
  *w = Workspace();
}

int eic_ws_ensure(eic_graph* g, int) {
  Workspace* w = &g->ws;
  if (w->ctl) return EIC_OK;
  const DevGraph& G = g->dg;
  const uint64_t n = G.n;
  int rc = EIC_OK;
  uint32_t maxw = G.maxw ? G.maxw : 1;
  uint32_t bits = 0;
  while (bits < 32 && (1ull << bits) <= maxw) ++bits;  // 2^bits > maxW
  w->ring_bits = bits < 20 ? bits : 20;
  w->ring_shift = bits > 20 ? bits - 20 : 0;
  w->heavy_cap = (uint32_t)(G.two_m / kHeavyMinFloor + 2);
  w->step_cap = kStepCap;
  w->n = G.n;
  if ((rc = walloc(w, &w->stamp, n)) || (rc = walloc(w, &w->q[0], n)) || (rc = walloc(w, &w->q[1], n)) ||
      (rc = walloc(w, &w->settled, n + 2)) || (rc = walloc(w, &w->touched, n + 1)) ||
      (rc = walloc(w, &w->ul[0], (uint64_t)G.nz_count + 1)) || (rc = walloc(w, &w->ul[1], (uint64_t)G.nz_count + 1)) ||
      (rc = walloc(w, &w->hist, (uint64_t)G.D + 1)) || (rc = walloc(w, &w->ring, 1ull << w->ring_bits)) ||
      (rc = walloc(w, &w->heavy, w->heavy_cap)) || (rc = walloc(w, &w->step_ub, (uint64_t)kStepCap + 2)) ||
      (rc = walloc(w, &w->step_off, (uint64_t)kStepCap + 2)) || (rc = walloc(w, &w->trace, kTraceCap)) ||
      (rc = walloc(w, &w->ctl, 1))) {
    eic_ws_free(w);
    return rc;
  }
  if (cudaMallocHost((void**)&w->ctl_host, sizeof(Ctl)) != cudaSuccess) {
    (void)cudaGetLastError();
    eic_ws_free(w);
    return EIC_ENOMEM;
  }
  if (cudaMemset(w->stamp, 0, n * 4) != cudaSuccess || cudaMemset(w->ctl, 0, sizeof(Ctl)) != cudaSuccess) {
    (void)cudaGetLastError();
    eic_ws_free(w);
    return EIC_ECUDA;
  }
  return EIC_OK;
}

extern "C" {

int eic_sssp(const eic_graph* gc, uint32_t source, uint32_t* dist, uint32_t* parent, const eic_params* params,
             eic_stats* stats, void* stream) {
  eic_graph* g = const_cast<eic_graph*>(gc);
  if (!g || !dist) return EIC_EINVAL;
  if (source >= g->dg.n) return EIC_EINVAL;
  eic_params p;
  int rc = resolve_params(params, &p);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g->mu);
  DeviceGuard dg(g->device);
  if (!dg.ok) return EIC_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  eic_step* trace = stats ? stats->trace : nullptr;
  const uint64_t trace_cap = stats ? stats->trace_cap : 0;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->trace = trace;
    stats->trace_cap = trace_cap;
  }
  if (g->dg.two_m == 0) return trivial_query(g, source, dist, parent, st);
  if ((rc = eic_ws_ensure(g, 0))) return rc;
  if ((rc = enqueue_query(g, source, dist, parent, p, nullptr, st))) {
    cudaStreamSynchronize(st);
    (void)cudaGetLastError();
    return rc;
  }
  Workspace& w = g->ws;
  EIC_CUDA_TRY(cudaMemcpyAsync(w.ctl_host, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  EIC_CUDA_TRY(cudaStreamSynchronize(st));
  const Ctl& h = *w.ctl_host;
  w.host_round_base = h.round_base;
  if (stats) {
    stats->steps = h.trace_len;
    stats->rounds = h.cnt_rounds;
    stats->frontier = h.cnt_frontier;
    stats->traversed = h.cnt_trav;
    stats->pulls = h.cnt_pulls;
    stats->improved = h.cnt_improved;
    stats->heavy = h.cnt_heavy;
    stats->trace_len = h.trace_len;
    if (trace && trace_cap) {
      uint64_t rows = h.trace_len < trace_cap ? h.trace_len : trace_cap;
      if (rows > kTraceCap) rows = kTraceCap;
      if (rows) EIC_CUDA_TRY(cudaMemcpy(trace, w.trace, rows * sizeof(eic_step), cudaMemcpyDeviceToHost));
    }
  }
  return h.status;
}

int eic_sssp_batch(const eic_graph* const* graphs, const uint32_t* sources, uint32_t num_queries,
                   uint32_t* const* dists, const eic_params* params, int* statuses, void* stream) {
  if (num_queries == 0) return EIC_OK;
  if (!graphs || !sources || !dists) return EIC_EINVAL;
  eic_params p;
  int rc = resolve_params(params, &p);
  if (rc) return rc;
  for (uint32_t i = 0; i < num_queries; ++i) {
    if (!graphs[i] || !dists[i] || sources[i] >= graphs[i]->dg.n) {
      if (statuses)
        for (uint32_t j = 0; j < num_queries; ++j) statuses[j] = EIC_EINVAL;
      return EIC_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* dstat = nullptr;
  int* hstat = nullptr;
  if (cudaMalloc((void**)&dstat, num_queries * sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&hstat, num_queries * sizeof(int)) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(dstat);
    return EIC_ENOMEM;
  }
  cudaMemsetAsync(dstat, 0, num_queries * sizeof(int), st);
  int first_err = EIC_OK;
  for (uint32_t i = 0; i < num_queries && first_err == EIC_OK; ++i) {
    eic_graph* g = const_cast<eic_graph*>(graphs[i]);
    std::lock_guard<std::mutex> lock(g->mu);
    DeviceGuard dg(g->device);
    if (g->dg.two_m == 0) {
      if ((rc = trivial_query(g, sources[i], dists[i], nullptr, st))) first_err = rc;
      continue;
    }
    if ((rc = eic_ws_ensure(g, 0)) || (rc = enqueue_query(g, sources[i], dists[i], nullptr, p, dstat + i, st)))
      first_err = rc;
  }
  if (cudaMemcpyAsync(hstat, dstat, num_queries * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    if (first_err == EIC_OK) first_err = EIC_ECUDA;
  }
  for (uint32_t i = 0; i < num_queries; ++i) {
    int s_i = first_err != EIC_OK ? first_err : hstat[i];
    if (statuses) statuses[i] = s_i;
    if (first_err == EIC_OK && s_i != EIC_OK) first_err = s_i;
  }
  for (uint32_t i = 0; i < num_queries; ++i) {  // refresh stamp-id bases
    eic_graph* g = const_cast<eic_graph*>(graphs[i]);
    if (g->ws.ctl && g->ws.ctl_host) {
      DeviceGuard dg(g->device);
      if (cudaMemcpy(&g->ws.host_round_base, &g->ws.ctl->round_base, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        (void)cudaGetLastError();
    }
  }
  cudaFree(dstat);
  cudaFreeHost(hstat);
  return first_err;
}

}  // extern "C"

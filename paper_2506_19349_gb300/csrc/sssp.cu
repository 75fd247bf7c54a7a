// Single-source query by Algorithm 1 of the EIC method: steps with
// scheduling pairs <lb, ub> (dynamic stepping, Eq. 1-3), a selection
// threshold st per step (traversal optimisation, Function 2) and rounds of
// window-filtered edge relaxations (Function 1 and the inner loop of
// Algorithm 1), as one persistent cooperative kernel on sm_103a.
//
// Device layout per query (workspace, reused across queries of one graph):
//   dist[ni]     distances in internal ids (non-isolated vertices by degree,
//                densest first), u32, +inf = 0xFFFFFFFF, updated by atomicMin;
//                copied to the caller's buffer in the original numbering at the end
//   fbits[2][n/32]  frontier bitmaps by round parity: the SAP of Algorithm 1 inserts
//                a vertex into the next frontier only if its bit was clear
//   cursor[n]    where the last window relaxed from a vertex ended (offset in its row)
//   q[2][n]      frontier queues, one per round parity
//   sid/sd/scur  settled list in settling order (vertex, final distance, window
//                cursor); step k owns [step_off[k], step_off[k+1])
//   touched[n]   first-step insertions (the first step's ub shrinks, so its
//                tentative distances >= the final ub are reset to +inf)
//   sbits[n/32]  settled bitmap: the pull set of Function 1 is the unsettled part of
//                a prefix of the non-isolated vertices ordered by smallest row weight
//   hist[D]      unsettled vertices per distinct degree (for highD)
//   ring[R]      degree sums of settled vertices by distance mod R (for the
//                sumD differences of Function 2's candidates, while maxW < 2^20;
//                wider weights sum them exactly from the settled list)
//   tasks[]      windows longer than heavy_min, cut into 64-entry tasks for the grid
//
// Phases (one grid barrier each): a round (the first round of a step runs
// Function 1's push set and pull), an optional task phase, and per step one
// statistics pass after which block 0 evaluates Eq. 1-3 and Function 2 and
// publishes the next <st, lb, ub>. In a round each warp takes 32 items at a
// time (warp-strided, its next items' records loaded ahead); each lane finds
// its item's window in the weight-sorted row, and the warp relaxes the
// concatenation of its lanes' windows, windows longer than heavy_min becoming
// 64-entry tasks for the task phase. A pull set of at least half the vertices
// is swept in vertex order over the unsettled vertices only, compacted from
// the settled bitmap 512 vertices at a time.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "graph.h"
#include "pool.h"
#include "serve.h"
#include "stats.cuh"

using namespace eic;

namespace {

constexpr uint32_t kModePush = 0;     // frontier or push-set vertex: relax its window
constexpr uint32_t kModePull = 2;     // unsettled vertex pulling over its light prefix
constexpr uint32_t kKindNone = 0, kKindVertex = 1, kKindPush = 2, kKindPull = 3;  // a lane's item in a round
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kShRanks = 1024;
constexpr int kShRing = 2048;
constexpr int64_t kRingNarrow = 16;  // statistics windows up to this width aggregate ring updates per warp

struct KArgs {
  DevGraph G;
  uint32_t* dist;  // internal ids
  uint32_t* out;   // caller's buffer, original ids
  uint32_t* fbits;  // two bitmaps of fwords words
  uint32_t fwords;
  uint32_t* cursor;
  uint32_t* q0;
  uint32_t* q1;
  uint32_t* sid;
  uint32_t* sd;
  uint32_t* scur;
  uint32_t* touched;
  uint32_t* sbits;  // settled bitmap
  uint32_t* hist;
  unsigned long long* ring;
  Task* tasks;
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
  uint32_t task_cap, step_cap, trace_cap;
  unsigned long long* timeline;  // NULL unless the caller asked for it
  uint32_t timeline_cap;
  uint32_t nb;  // blocks working on this query: the grid, or one block group of a batch
  uint32_t fuse;  // fused rounds for this query (kernels that decide per query)
};

// Index of the block within the blocks that work on its query.
__device__ __forceinline__ uint32_t qblock(const KArgs& A) { return blockIdx.x % A.nb; }

constexpr uint32_t kMaxBlock = 512;
constexpr uint32_t kMaxWarps = kMaxBlock / 32;
constexpr uint32_t kTaskLen = 64;     // adjacency entries per grid task
// Round-phase shapes (pull prefix entries a lane answers itself, window
// entries a lane relaxes at a time), per kernel: more of each is faster while
// registers last; the batch and serving kernels hold more state.
constexpr uint32_t kPullFastSingle = 8, kRelaxIlpSingle = 2;  // k_eic
constexpr uint32_t kPullFastGroup = 4, kRelaxIlpGroup = 1;    // k_eic_batch, k_eic_serve
constexpr uint32_t kSweepNum = 1, kSweepDen = 2;  // sweep the pull set when it holds >= 1/2 of the vertices
constexpr uint32_t kSweepChunk = 16;  // settled-bitmap words a warp takes at a time in a sweep (<= 32)
constexpr uint32_t kStageT = 1024;    // tasks staged per block
constexpr uint32_t kWarpStage = 256;  // next-frontier / settled-list appends staged per warp

struct WarpScr {  // one warp's small windows
  uint32_t beg[32];
  uint32_t excl[32];
  uint32_t val[32];  // source distance (push) or best candidate (pull)
  uint32_t u[32];
  uint32_t mode[32];
};

struct RoundScr {
  WarpScr w[kMaxWarps];
};

// Appends gathered in shared memory. Next-frontier and settled-list entries
// are staged per warp and written by the warp with one global atomic per
// kWarpStage entries (no block synchronisation); tasks are staged per block
// and written at the end of a phase.
struct Stage {
  uint32_t tn, tbase;
  Task tbuf[kStageT];
  uint32_t wq[kMaxWarps][kWarpStage];
  uint32_t wf[kMaxWarps][kWarpStage];
};

// One warp's append stage for one list. n is warp-uniform.
struct WarpList {
  uint32_t* buf;    // shared memory, kWarpStage entries
  uint32_t n;       // entries held
  uint32_t* gcnt;   // the list's global count
  uint32_t* glist;  // the list
};

__device__ __forceinline__ void warp_flush(WarpList& W) {
  if (W.n == 0) return;
  uint32_t base = 0;
  if (lane_id() == 0) base = atomicAdd(W.gcnt, W.n);
  base = __shfl_sync(EIC_FULL_MASK, base, 0);
  __syncwarp();
  for (uint32_t k = lane_id(); k < W.n; k += 32) __stcg(&W.glist[base + k], W.buf[k]);
  __syncwarp();
  W.n = 0;
}

// Warp-collective append of v for the lanes with want.
__device__ __forceinline__ void warp_push(WarpList& W, bool want, uint32_t v) {
  const uint32_t mask = __ballot_sync(EIC_FULL_MASK, want);
  if (mask == 0) return;
  const uint32_t cnt = __popc(mask);
  if (W.n + cnt > kWarpStage) warp_flush(W);
  if (want) W.buf[W.n + __popc(mask & ((1u << lane_id()) - 1u))] = v;
  __syncwarp();
  W.n += cnt;
}

struct S2Scr {
  uint32_t hist[kShRanks];
  unsigned long long ring[kShRing];
};

constexpr uint32_t kGapPar = 256;   // distinct degrees up to which the boundary evaluates Eq. 1-3 for each
constexpr uint32_t kStBins = 1920;  // Function 2 candidate bins held in shared memory (ST_NUM + 2 at most)

struct S3Scr {
  unsigned long long part[kMaxBlock];
  unsigned long long bp[32];  // per warp: the best profit's key (see block_argmax)
  uint32_t bk[32];
  unsigned long long bins[kStBins];
};

union PhaseScr {
  RoundScr r;
  S2Scr s2;
  S3Scr s3;
};

// Control values every block holds between barriers.
struct Local {
  int64_t lb, ub, st, lb0;
  uint32_t step, rid, qsel, cur_cnt, s_int;
  uint32_t push_beg, push_end, pull_on, pull_cnt, pull_sweep, extra_s, step_off_cur, done;
};

// State of the step controller, kept in block 0's shared memory across steps.
struct BState {
  int64_t st0, st1, gap_lb, max_settled;
  uint64_t sumd_lb, highd_lb;
  uint32_t j0;
};

struct Counters {  // one thread's counts over the query (added to the 64-bit totals at its end)
  uint32_t frontier, trav, pulls, improved, heavy, pitems;
};

__device__ __forceinline__ void tl_mark(const KArgs& A, uint32_t kind, uint32_t rid) {
  if (!A.timeline) return;
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  uint32_t i = atomicAdd(&A.ctl->tl_len, 1u);
  if (i < A.timeline_cap) {
    A.timeline[2 * i] = t;
    A.timeline[2 * i + 1] = ((unsigned long long)kind << 32) | rid;
  }
}

constexpr uint32_t kFlagBlockTimeline = 1u << 30;  // diagnostic: per-block phase marks

// per-block mark: kind 6 item phase done, 7 task phase done (tag has the block id)
__device__ __forceinline__ void tl_block(const KArgs& A, uint32_t kind, uint32_t rid) {
  if (!A.timeline || !(A.flags & kFlagBlockTimeline) || threadIdx.x != 0) return;
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  uint32_t i = atomicAdd(&A.ctl->tl_len, 1u);
  if (i < A.timeline_cap) {
    A.timeline[2 * i] = t;
    A.timeline[2 * i + 1] = ((unsigned long long)kind << 32) | ((unsigned long long)qblock(A) << 48) | rid;
  }
}

// position of the k-th (from 0) set bit of m; m has more than k set bits
__device__ __forceinline__ uint32_t kth_set_bit(uint32_t m, uint32_t k) {
  uint32_t p = 0;
#pragma unroll
  for (uint32_t half = 16; half >= 1; half >>= 1) {
    const uint32_t low = (uint32_t)__popc(m & ((1u << (p + half)) - 1u));  // set bits below p + half
    if (low <= k) p += half;
  }
  return p;
}

__device__ __forceinline__ int64_t d64(uint32_t d) { return d == EIC_INF ? EIC_INF_T : (int64_t)d; }

// Streaming reads (adjacency entries, the pull list) carry an L2 evict-first
// policy, so that the per-vertex arrays (dist, row offsets, bitmaps, cursors)
// stay in L2 while the adjacency streams past.
__device__ __forceinline__ uint64_t stream_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint2 ld_stream(const uint2* p) {
  uint2 v;
  asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(stream_policy()));
  return v;
}

__device__ __forceinline__ uint32_t ld_stream_w(const uint2* p) {
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(&p->y), "l"(stream_policy()));
  return v;
}

// The same for lists written earlier in the kernel (frontier queue, settled
// list, tasks): L2 only (no L1 copy that another block's write could leave
// stale), evict-first.
__device__ __forceinline__ uint32_t ld_list(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.cg.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(stream_policy()));
  return v;
}

__device__ __forceinline__ uint2 ld_list2(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p), "l"(stream_policy()));
  return v;
}

__device__ __forceinline__ uint4 ld_list4(const void* p) {
  uint4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(stream_policy()));
  return v;
}

__device__ __forceinline__ uint4 ld_stream4(const uint4* p) {
  uint4 v;
  asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(stream_policy()));
  return v;
}

// first index in [b, e) of the weight-sorted row with weight >= t
__device__ __forceinline__ uint32_t lower_bound_w(const uint2* __restrict__ adj, uint32_t b, uint32_t e, int64_t t) {
  if (t <= 1) return b;  // weights are >= 1
  while (b < e) {
    uint32_t mid = b + ((e - b) >> 1);
    if ((int64_t)ld_stream_w(&adj[mid]) < t)
      b = mid + 1;
    else
      e = mid;
  }
  return b;
}

// The same, given that every entry before p has weight < t: exponential
// probes forward from p, then a binary search in the last interval. Costs
// O(log distance), and a short window costs one or two probes of one sector.
__device__ __forceinline__ uint32_t gallop_w(const uint2* __restrict__ adj, uint32_t p, uint32_t e, int64_t t) {
  if (t <= 1 || p >= e) return p;
  if ((int64_t)ld_stream_w(&adj[p]) >= t) return p;
  uint32_t lo = p;  // weight at lo < t
  uint32_t hi;
  uint64_t step = 1;
  for (;;) {
    const uint64_t h = (uint64_t)lo + step;
    if (h >= e) {
      hi = e;
      break;
    }
    if ((int64_t)ld_stream_w(&adj[h]) >= t) {
      hi = (uint32_t)h;
      break;
    }
    lo = (uint32_t)h;
    step <<= 1;
  }
  return lower_bound_w(adj, lo + 1, hi, t);
}

struct RoundCtx {
  int64_t lb, ub, ub_eff, st, lb0;
  uint32_t rid;
  uint32_t* fbits;  // this round's insertion bitmap
  bool step1;
  uint32_t* qout;
  uint32_t* qcnt_out;
  uint32_t* first_list;
  uint32_t* first_cnt;
  uint32_t* tcnt;
  uint32_t* work;
};

// Flush the block's task stage to the global list (block-uniform call).
__device__ __forceinline__ void stage_flush(Stage& T, const RoundCtx& R, Task* tasks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t tn = min(T.tn, kStageT);
    T.tn = tn;
    T.tbase = tn ? atomicAdd(R.tcnt, tn) : 0;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < T.tn; i += blockDim.x) tasks[T.tbase + i] = T.tbuf[i];
  __syncthreads();
  if (threadIdx.x == 0) T.tn = 0;
}

// Cut the window [b, b + len) of vertex u into kTaskLen-entry tasks, staged in
// the block (or written straight to the global list when the stage is full).
__device__ __forceinline__ void emit_tasks(const KArgs& A, const RoundCtx& R, Stage& T, uint32_t b, uint32_t len,
                                           uint32_t u, uint32_t d) {
  const uint32_t nt = (len + kTaskLen - 1) / kTaskLen;
  const uint32_t pos = atomicAdd(&T.tn, nt);
  const uint32_t in_stage = pos < kStageT ? min(nt, kStageT - pos) : 0;
  // the rest goes straight to the global list; capacity covers 2m / 16 tasks per round
  const uint32_t gpos = nt > in_stage ? atomicAdd(R.tcnt, nt - in_stage) : 0;
  for (uint32_t k = 0; k < nt; ++k) {
    Task t;
    t.beg = b + k * kTaskLen;
    t.len = min(kTaskLen, len - k * kTaskLen);
    t.u = u;
    t.d = d;
    if (k < in_stage)
      T.tbuf[pos + k] = t;
    else
      A.tasks[gpos + (k - in_stage)] = t;
  }
}

// Successful relaxation of v to nd (old = previous distance): SAP into the
// next frontier, first insertion into the settled (or first-step) list, and
// in the first step the running min over high-degree vertices that becomes
// ub (Algorithm 1). Warp-collective: every lane calls it; the appends go
// through the warp's stages.
// Sets v's bit in the round's insertion bitmap; true when this call set it.
__device__ __forceinline__ bool claim_bit(const RoundCtx& R, uint32_t v) {
  const uint32_t bit = 1u << (v & 31);
  return !(atomicOr(&R.fbits[v >> 5], bit) & bit);
}

// After a relaxation: v into the next frontier when sap (its insertion bit was
// set by this lane), into the first-reached list when it had no distance, and
// the first step's ub candidate when v's degree is at least highD(0).
__device__ __forceinline__ void on_claimed(const KArgs& A, const RoundCtx& R, bool ok, bool sap, uint32_t v,
                                           uint32_t nd, uint32_t old, Counters& C, WarpList& Q, WarpList& F) {
  const bool first = ok && old == EIC_INF;
  warp_push(Q, sap, v);
  warp_push(F, first, v);
  if (R.step1 && ok) {
    const uint32_t dg = __ldg(&A.G.row[v + 1]) - __ldg(&A.G.row[v]);
    if (dg >= A.G.highd0) atomicMin(&A.ctl->ub_cand, nd);
  }
  C.improved += ok ? 1 : 0;
}

__device__ __forceinline__ void on_success(const KArgs& A, const RoundCtx& R, bool ok, uint32_t v, uint32_t nd,
                                           uint32_t old, Counters& C, WarpList& Q, WarpList& F) {
  bool sap = false;
  if (ok) {
    const uint32_t bit = 1u << (v & 31);
    sap = !(atomicOr(&R.fbits[v >> 5], bit) & bit);
  }
  const bool first = ok && old == EIC_INF;
  warp_push(Q, sap, v);
  warp_push(F, first, v);
  if (R.step1 && ok) {
    const uint32_t dg = __ldg(&A.G.row[v + 1]) - __ldg(&A.G.row[v]);
    if (dg >= A.G.highd0) atomicMin(&A.ctl->ub_cand, nd);
  }
  C.improved += ok ? 1 : 0;
}

// One round over nitems items. Items are frontier vertices (queue qin), or in
// a step's first round Function 1's push set (a settled-list range), its pull
// set and, once, the source. The pull set is a prefix of the weight-ordered
// non-isolated vertices (listed), or, when that prefix holds at least half of
// them, every unsettled vertex (swept in vertex order). Warp by warp without
// block synchronisation, each lane finds its item's window in the
// weight-sorted row; windows up to heavy_min entries are relaxed by the warp
// over their concatenation, kRelaxIlp entries per lane at a time, longer ones
// become grid tasks. A pull reads the prefix of its vertex's row with weight
// < ub - st: its first kPullFast entries in the lane, the rest by the warp.
// Next-frontier and settled-list appends are staged per warp in shared
// memory; tasks per block.
template <uint32_t kPullFast, uint32_t kRelaxIlp>
__device__ void round_phase(const KArgs& A, const RoundCtx& R, const Local& L, RoundScr& S, Stage& T,
                            uint32_t nitems, bool round1, const uint32_t* qin, Counters& C) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x, lane = lane_id(), warp = tid >> 5;
  const uint32_t np = round1 ? L.push_end - L.push_beg : 0;
  const bool sweep = round1 && L.pull_sweep;  // the pull set is every unsettled vertex, swept below
  const uint32_t npp = np + (sweep ? 0u : L.pull_cnt);
  const uint32_t nlisted = sweep ? nitems - L.pull_cnt : nitems;  // items of the listed part
  const uint32_t gwarp = qblock(A) * (nt >> 5) + warp, nwarps = A.nb * (nt >> 5);
  const int64_t pull_bound = R.ub - R.st;
  WarpScr& W = S.w[warp];
  WarpList Qw = {T.wq[warp], 0u, R.qcnt_out, R.qout};
  WarpList Fw = {T.wf[warp], 0u, R.first_cnt, R.first_list};
  // An item's record: {vertex, dist, row begin, row end} for a frontier
  // vertex or the source, {dist, row begin, row end, cursor} for the push set
  // (from the settled list), the nz entry for a listed pull. Records are loaded one
  // warp iteration ahead, a frontier vertex's queue entry two ahead.
  // (the push set's settled-list vertices come in the same way, two ahead)
  auto fetch_id = [&](uint32_t ii) -> uint32_t {
    if (ii >= nlisted) return 0u;
    if (!round1) return ld_list(&qin[ii]);
    return ii < np ? ld_list(&A.sid[L.push_beg + ii]) : 0u;
  };
  auto fetch = [&](uint32_t ii, uint32_t id) -> uint4 {
    if (ii >= nlisted) return make_uint4(0u, 0u, 0u, 0u);
    if (!round1 || ii >= npp) {  // frontier vertex (or the source, once)
      const uint32_t u = round1 ? L.s_int : id;
      return make_uint4(u, __ldcg(&A.dist[u]), __ldg(&A.G.row[u]), __ldg(&A.G.row[u + 1]));
    }
    if (ii < np)
      return make_uint4(ld_list(&A.sd[L.push_beg + ii]), __ldg(&A.G.row[id]), __ldg(&A.G.row[id + 1]),
                        ld_list(&A.scur[L.push_beg + ii]));
    return ld_stream4(&A.G.nz[ii - np]);
  };
  // one warp iteration: each lane's item (kind kKindNone: no item)
  auto step_items = [&](const uint4 rec, const uint32_t i, const uint32_t kind) {
    uint32_t u = 0, val = EIC_INF, b = 0, len = 0, mode = kModePush;
    uint32_t pfast = EIC_INF;       // best pull candidate of the lane's vertex
    uint32_t du = EIC_INF;          // the pulled vertex's distance when its pull started
    bool plong = false;             // its prefix is longer than kPullFast entries
    if (kind != kKindNone) {
      if (kind == kKindVertex) {  // frontier vertex (or the source, once)
        u = rec.x;
        const uint32_t d = rec.y, rb = rec.z, re = rec.w;
        val = d;
        if (d != EIC_INF && !(d > 0 && re - rb == 1)) {  // Paths excludes leaves (Algorithm 1)
          C.frontier += 1;
          const int64_t hi = R.ub_eff - (int64_t)d;
          if (hi > 0) {
            b = lower_bound_w(A.G.adj, rb, re, R.lb - (int64_t)d);
            const uint32_t e = gallop_w(A.G.adj, b, re, hi);
            if (re - rb > kCursorMin) __stcg(&A.cursor[u], e - rb);
            len = e - b;
          }
        }
      } else if (kind == kKindPush) {  // push set: settled, lb0 <= dist <= st (all from the settled list)
        const uint32_t idx = L.push_beg + i;
        const uint32_t d = rec.x;
        val = d;
        if ((int64_t)d >= R.lb0 && (int64_t)d <= R.st) {
          const uint32_t rb = rec.y, re = rec.z;
          if (!(d > 0 && re - rb == 1)) {
            C.frontier += 1;
            const uint32_t cur = rec.w;
            // windows of consecutive steps are contiguous: resume at the cursor
            b = cur == kNone ? lower_bound_w(A.G.adj, rb, re, R.lb - (int64_t)d)
                             : gallop_w(A.G.adj, rb + cur, re, R.lb - (int64_t)d);
            const uint32_t e = gallop_w(A.G.adj, b, re, R.ub_eff - (int64_t)d);
            __stcg(&A.scur[idx], e - rb);
            len = e - b;
          }
        }
      } else {  // pull set: unsettled, smallest weight < ub - st (Function 1)
        const uint4 z = rec;  // {vertex, lightest weight or settled word, row begin, row end}
        u = z.x;
        mode = kModePull;
        const uint32_t bits = L.pull_sweep ? z.y : __ldcg(&A.sbits[u >> 5]);
        if (!((bits >> (u & 31)) & 1u)) {  // unsettled: its row's first kPullFast entries, together
          const uint32_t rl = z.w - z.z;
          du = __ldcg(&A.dist[u]);
          uint2 ent[kPullFast];
  #pragma unroll
          for (uint32_t k = 0; k < kPullFast; ++k)
            ent[k] = k < rl ? ld_stream(&A.G.adj[z.z + k]) : make_uint2(0u, EIC_INF);
          uint32_t c = 0;  // the prefix with w < ub - st (rows are weight-sorted)
  #pragma unroll
          for (uint32_t k = 0; k < kPullFast; ++k) c += (k < rl && (int64_t)ent[k].y < pull_bound) ? 1u : 0u;
          C.pitems += c > 0 ? 1 : 0;  // in the pull set iff its lightest edge is below the bound
          plong = c == kPullFast && rl > kPullFast;  // the prefix goes on: the warp scans the rest
          {  // the loaded part of the prefix, answered in the lane
            uint32_t dv[kPullFast];
  #pragma unroll
            for (uint32_t k = 0; k < kPullFast; ++k) dv[k] = k < c ? __ldcg(&A.dist[ent[k].x]) : EIC_INF;
  #pragma unroll
            for (uint32_t k = 0; k < kPullFast; ++k) {
              if (k >= c) continue;
              C.trav += 1;
              C.pulls += 1;
              const int64_t dvv = dv[k];
              if (dv[k] != EIC_INF && dvv >= R.st && dvv < R.lb && dvv + ent[k].y < R.ub)
                pfast = min(pfast, (uint32_t)(dvv + ent[k].y));
            }
          }
          if (plong) {  // the prefix goes on past the lane's entries: find its end, then the rest
                        // is a window like a push window (the warp's concatenation, or grid tasks)
            b = z.z + kPullFast;
            const uint32_t e = pull_bound > (int64_t)A.G.maxw ? z.w : gallop_w(A.G.adj, b, z.w, pull_bound);
            len = e - b;
          }
        }
      }
    }
    if (len > A.heavy_min) {
      emit_tasks(A, R, T, b, len, u, mode == kModePull ? kNone : val);
      C.heavy += (len + kTaskLen - 1) / kTaskLen;
      len = 0;
    }
    const uint32_t incl = warp_incl_scan(len);
    const uint32_t total = __shfl_sync(EIC_FULL_MASK, incl, 31);
    W.beg[lane] = b;
    W.excl[lane] = incl - len;
    W.val[lane] = mode == kModePull ? pfast : val;
    W.u[lane] = u;
    W.mode[lane] = mode;
    __syncwarp();
    // the concatenated windows, kRelaxIlp entries per lane at a time (their
    // loads in flight together)
    for (uint32_t g0 = 0; g0 < total; g0 += 32 * kRelaxIlp) {
      uint32_t own[kRelaxIlp], dv[kRelaxIlp], nd[kRelaxIlp], old[kRelaxIlp];
      uint2 ent[kRelaxIlp];
      bool act[kRelaxIlp], push[kRelaxIlp], ok[kRelaxIlp], sap[kRelaxIlp];
#pragma unroll
      for (uint32_t h = 0; h < kRelaxIlp; ++h) {
        const uint32_t g = g0 + h * 32 + lane;
        act[h] = g < total;
        own[h] = 0;
        ent[h] = make_uint2(0u, 0u);
        if (act[h]) {
          uint32_t lo = 0, hi = 31;
          while (lo < hi) {  // last lane whose window starts at or before g
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (W.excl[mid] <= g)
              lo = mid;
            else
              hi = mid - 1;
          }
          own[h] = lo;
          ent[h] = ld_stream(&A.G.adj[W.beg[lo] + (g - W.excl[lo])]);
        }
      }
#pragma unroll
      for (uint32_t h = 0; h < kRelaxIlp; ++h) {
        push[h] = act[h] && W.mode[own[h]] != kModePull;
        // a pull entry is a request answered by a settled v with st <= dist[v] < lb
        act[h] = push[h] || (act[h] && (int64_t)ent[h].y < pull_bound);
        dv[h] = act[h] ? __ldcg(&A.dist[ent[h].x]) : EIC_INF;
      }
#pragma unroll
      for (uint32_t h = 0; h < kRelaxIlp; ++h) {
        ok[h] = false;
        sap[h] = false;
        nd[h] = 0;
        old[h] = 0;
        if (push[h]) {
          C.trav += 1;
          nd[h] = W.val[own[h]] + ent[h].y;  // inside [lb, min(ub, 2^32-1)) by the window bounds
          if (nd[h] < dv[h]) {
            // The insertion bit is claimed together with the atomicMin, not
            // after it. Should the atomicMin find a value <= nd, another
            // relaxation lowered dist[v] in this round after the read above
            // (distances only fall, and the round sees every earlier round's
            // writes), so v is in the next frontier either way and whichever
            // lane set the bit queues it.
            old[h] = atomicMin(&A.dist[ent[h].x], nd[h]);
            sap[h] = claim_bit(R, ent[h].x);
            ok[h] = nd[h] < old[h];
          }
        } else if (act[h]) {
          C.trav += 1;
          C.pulls += 1;
          const int64_t dvv = dv[h];
          if (dv[h] != EIC_INF && dvv >= R.st && dvv < R.lb && dvv + ent[h].y < R.ub)
            atomicMin(&W.val[own[h]], (uint32_t)(dvv + ent[h].y));
        }
      }
#pragma unroll
      for (uint32_t h = 0; h < kRelaxIlp; ++h) on_claimed(A, R, ok[h], sap[h], ent[h].x, nd[h], old[h], C, Qw, Fw);
    }
    __syncwarp();
    bool pok = false, psap = false;
    uint32_t pold = 0;
    const uint32_t pbest = W.val[lane];
    if (mode == kModePull && pbest < du) {  // du was read in this round: the insertion bit is
                                            // claimed with the atomicMin, as for pushes
      pold = atomicMin(&A.dist[u], pbest);
      psap = claim_bit(R, u);
      pok = pbest < pold;
    }
    on_claimed(A, R, pok, psap, u, pbest, pold, C, Qw, Fw);
    __syncwarp();
  };
  const uint32_t stride = nwarps * 32;
  uint4 pre = fetch(gwarp * 32 + lane, fetch_id(gwarp * 32 + lane));
  uint32_t idn = fetch_id(gwarp * 32 + stride + lane);
  for (uint32_t base = gwarp * 32; base < nlisted; base += stride) {
    const uint32_t i = base + lane;
    const uint4 rec = pre;
    pre = fetch(base + stride + lane, idn);
    idn = fetch_id(base + 2 * stride + lane);
    step_items(rec, i, i >= nlisted ? kKindNone : (!round1 || i >= npp) ? kKindVertex : i < np ? kKindPush : kKindPull);
  }
  if (sweep) {
    // Function 1's pull set swept in vertex order, compacted: a warp takes
    // kSweepChunk settled-bitmap words (32 vertices each) at a time and hands
    // its lanes only the unsettled vertices, 32 per iteration, the next
    // batch's row bounds loaded while the current one runs
    const uint32_t ni = A.G.ni, nwords = (ni + 31) >> 5, nchunks = (nwords + kSweepChunk - 1) / kSweepChunk;
    uint32_t ch = gwarp, m = 0, off = 0, tot = 0, r0 = 0, wn = ~0u;
    auto word_at = [&](uint32_t c) -> uint32_t {
      const uint32_t wi = c * kSweepChunk + lane;
      return c < nchunks && lane < kSweepChunk && wi < nwords ? __ldcg(&A.sbits[wi]) : ~0u;
    };
    auto open_chunk = [&](uint32_t word) {  // this lane's unsettled mask, its exclusive rank, the chunk total
      const uint32_t wi = ch * kSweepChunk + lane;
      uint32_t mm = lane < kSweepChunk && wi < nwords ? ~word : 0u;
      if (wi == nwords - 1 && (ni & 31u)) mm &= (1u << (ni & 31u)) - 1u;
      m = mm;
      const uint32_t c = __popc(mm), inc = warp_incl_scan(c);
      off = inc - c;
      tot = __shfl_sync(EIC_FULL_MASK, inc, 31);
      r0 = 0;
    };
    if (ch < nchunks) {
      open_chunk(word_at(ch));
      wn = word_at(ch + nwarps);
    }
    auto next_batch = [&](bool& ok) -> uint4 {
      while (r0 >= tot && ch < nchunks) {  // warp-uniform: skip to the next chunk with unsettled vertices
        ch += nwarps;
        if (ch >= nchunks) break;
        open_chunk(wn);
        wn = word_at(ch + nwarps);
      }
      ok = false;
      if (ch >= nchunks) return make_uint4(0u, 0u, 0u, 0u);
      const uint32_t r = r0 + lane;
      r0 += 32;
      uint32_t l = 0;  // the last word whose exclusive rank is <= r
#pragma unroll
      for (uint32_t h = 16; h > 0; h >>= 1) {
        const uint32_t o = __shfl_sync(EIC_FULL_MASK, off, l + h);
        if (o <= r) l += h;
      }
      const uint32_t ml = __shfl_sync(EIC_FULL_MASK, m, l), ol = __shfl_sync(EIC_FULL_MASK, off, l);
      if (r >= tot) return make_uint4(0u, 0u, 0u, 0u);
      ok = true;
      const uint32_t v = ((ch * kSweepChunk + l) << 5) + kth_set_bit(ml, r - ol);
      return make_uint4(v, 0u, __ldg(&A.G.row[v]), __ldg(&A.G.row[v + 1]));  // {vertex, settled word 0, row}
    };
    bool okc = false;
    uint4 cur = next_batch(okc);
    while (__any_sync(EIC_FULL_MASK, okc)) {
      bool okn = false;
      const uint4 nx = next_batch(okn);
      step_items(cur, 0u, okc ? kKindPull : kKindNone);
      cur = nx;
      okc = okn;
    }
  }
  warp_flush(Qw);
  warp_flush(Fw);
  tl_block(A, 6, R.rid);
  stage_flush(T, R, A.tasks);
}

// The round's tasks, one warp per task of at most 64 entries.
// With kAhead, a warp loads its next task while it runs the current one and
// relaxes a push task's two entries per lane with their loads in flight
// together (the single-query kernel's shape).
template <bool kAhead>
__device__ void task_phase(const KArgs& A, const RoundCtx& R, uint32_t ntasks, Stage& T, Counters& C) {
  const uint32_t lane = lane_id();
  const uint32_t wpb = blockDim.x >> 5;
  const uint32_t nwarps = A.nb * wpb;
  WarpList Qw = {T.wq[threadIdx.x >> 5], 0u, R.qcnt_out, R.qout};
  WarpList Fw = {T.wf[threadIdx.x >> 5], 0u, R.first_cnt, R.first_list};
  const int64_t pull_bound = R.ub - R.st;
  const uint32_t t0 = qblock(A) * wpb + (threadIdx.x >> 5);
  uint4 tnext = make_uint4(0u, 0u, 0u, 0u);
  if constexpr (kAhead) {
    if (t0 < ntasks) tnext = ld_list4(&A.tasks[t0]);
  }
  for (uint32_t t = t0; t < ntasks; t += nwarps) {
    uint4 tv;
    if constexpr (kAhead) {
      tv = tnext;
      if (t + nwarps < ntasks) tnext = ld_list4(&A.tasks[t + nwarps]);
    } else {
      tv = ld_list4(&A.tasks[t]);
    }
    const Task tk = {tv.x, tv.y, tv.z, tv.w};
    if (kAhead && tk.d != kNone) {  // push, both entries' loads in flight together
      uint2 ent[2];
      uint32_t dv[2], nd[2], old[2];
      bool act[2], ok[2], sap[2];
      if (!(tk.beg & 1u)) {  // the task starts on a 16-byte boundary: a lane loads its two entries as one pair
        const uint32_t j = 2 * lane;
        uint4 pr = make_uint4(0u, 0u, 0u, 0u);
        if (j < tk.len) pr = ld_stream4(reinterpret_cast<const uint4*>(A.G.adj + tk.beg + j));  // (2 spare entries)
        act[0] = j < tk.len;
        act[1] = j + 1 < tk.len;
        ent[0] = make_uint2(pr.x, pr.y);
        ent[1] = act[1] ? make_uint2(pr.z, pr.w) : make_uint2(0u, 0u);
      } else {
#pragma unroll
        for (uint32_t h = 0; h < 2; ++h) {
          act[h] = lane + 32 * h < tk.len;
          ent[h] = act[h] ? ld_stream(&A.G.adj[tk.beg + lane + 32 * h]) : make_uint2(0u, 0u);
        }
      }
#pragma unroll
      for (uint32_t h = 0; h < 2; ++h) dv[h] = act[h] ? __ldcg(&A.dist[ent[h].x]) : 0u;
#pragma unroll
      for (uint32_t h = 0; h < 2; ++h) {
        ok[h] = false;
        sap[h] = false;
        old[h] = 0;
        nd[h] = tk.d + ent[h].y;
        if (act[h]) {
          C.trav += 1;
          if (nd[h] < dv[h]) {  // the insertion bit claimed together with the atomicMin, as in the rounds
            old[h] = atomicMin(&A.dist[ent[h].x], nd[h]);
            sap[h] = claim_bit(R, ent[h].x);
            ok[h] = nd[h] < old[h];
          }
        }
      }
#pragma unroll
      for (uint32_t h = 0; h < 2; ++h) on_claimed(A, R, ok[h], sap[h], ent[h].x, nd[h], old[h], C, Qw, Fw);
    } else if (tk.d != kNone) {  // push
#pragma unroll
      for (uint32_t h = 0; h < 2; ++h) {
        const uint32_t j = lane + 32 * h;
        bool ok = false;
        uint32_t v = 0, nd = 0, old = 0;
        if (j < tk.len) {
          const uint2 ent = ld_stream(&A.G.adj[tk.beg + j]);
          v = ent.x;
          nd = tk.d + ent.y;
          C.trav += 1;
          const uint32_t dv = __ldcg(&A.dist[v]);
          if (nd < dv) {
            old = atomicMin(&A.dist[v], nd);
            ok = nd < old;
          }
        }
        on_success(A, R, ok, v, nd, old, C, Qw, Fw);
      }
    } else {  // pull request over a row segment
      uint32_t best = EIC_INF;
#pragma unroll
      for (uint32_t h = 0; h < 2; ++h) {
        const uint32_t j = lane + 32 * h;
        if (j < tk.len) {
          const uint2 ent = ld_stream(&A.G.adj[tk.beg + j]);
          if ((int64_t)ent.y < pull_bound) {
            C.trav += 1;
            C.pulls += 1;
            const uint32_t dv = __ldcg(&A.dist[ent.x]);
            const int64_t dvv = dv;
            if (dv != EIC_INF && dvv >= R.st && dvv < R.lb && dvv + ent.y < R.ub)
              best = min(best, (uint32_t)(dvv + ent.y));
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(EIC_FULL_MASK, best, o));
      bool ok = false;
      uint32_t old = 0;
      if (lane == 0 && best != EIC_INF) {
        old = atomicMin(&A.dist[tk.u], best);
        ok = best < old;
      }
      on_success(A, R, ok, tk.u, best, old, C, Qw, Fw);
    }
  }
  warp_flush(Qw);
  warp_flush(Fw);
  tl_block(A, 7, R.rid);
  stage_flush(T, R, A.tasks);
}

// The first candidate index with the largest positive profit over the block
// (ties: the smaller index), or 0xFFFFFFFF when no profit is positive. The
// reduction compares integer keys: a positive double's bit pattern orders as
// the double does, and a profit <= 0 gets key 0 (this GPU's double-precision
// units are few, and a block of double compares queues on them).
__device__ __forceinline__ uint32_t block_argmax(S3Scr& S, double best, uint32_t bk) {
  const uint32_t t = threadIdx.x, nt = blockDim.x;
  unsigned long long key = best > 0.0 ? (unsigned long long)__double_as_longlong(best) : 0ull;
  if (!key) bk = 0xFFFFFFFFu;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ok = __shfl_down_sync(EIC_FULL_MASK, key, o);
    const uint32_t okk = __shfl_down_sync(EIC_FULL_MASK, bk, o);
    if (ok > key || (ok == key && okk < bk)) {
      key = ok;
      bk = okk;
    }
  }
  __syncthreads();
  if ((t & 31) == 0) {
    S.bp[t >> 5] = key;
    S.bk[t >> 5] = bk;
  }
  __syncthreads();
  if (t < 32) {
    key = t < (nt >> 5) ? S.bp[t] : 0ull;
    bk = t < (nt >> 5) ? S.bk[t] : 0xFFFFFFFFu;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_down_sync(EIC_FULL_MASK, key, o);
      const uint32_t okk = __shfl_down_sync(EIC_FULL_MASK, bk, o);
      if (ok > key || (ok == key && okk < bk)) {
        key = ok;
        bk = okk;
      }
    }
    if (t == 0) S.bk[0] = key ? bk : 0xFFFFFFFFu;
  }
  __syncthreads();
  const uint32_t k = S.bk[0];
  __syncthreads();
  return k;
}

// The candidate grid x_k = st0 + floor(k span / ST_NUM) (Section 4.1): a
// shift when ST_NUM is a power of two (the paper's 1024), else a division.
__device__ __forceinline__ int64_t st_candidate(uint32_t k, uint64_t span, uint32_t st_num, uint32_t sh, int64_t st0) {
  const uint64_t q = (uint64_t)k * span;
  return st0 + (int64_t)(sh < 32 ? q >> sh : q / st_num);
}


// Function 2 for weights of 2^20 and above (one block), with D(x') summed
// exactly from the settled list: over the entries of the steps
// j (from j0 to step) that end above wl, the vertex at distance d >= wl adds
// its degree to bin 1 + k_d, k_d the last candidate k with x_k <= d (-1 if
// none); after a suffix sum, D(x_k) is bin 1 + k for x_k >= wl and bin 0 for a
// candidate clamped to wl. The bins are in shared memory, or in the ring
// (2^20 slots, unused for such weights) when ST_NUM is large.
__device__ __forceinline__ int64_t block_st_exact(const KArgs& A, S3Scr& S, int64_t ub, uint64_t sumd_ub,
                                                  int64_t gap_lb, int64_t gap_ub_raw, int64_t y, int64_t st0,
                                                  int64_t st1, uint32_t j0, uint32_t step, uint32_t send) {
  __shared__ uint32_t s_beg;
  const uint32_t t = threadIdx.x, nt = blockDim.x;
  const int64_t maxw = A.G.maxw;
  if (sumd_ub >= A.G.m || gap_lb == maxw) return ub;
  if (gap_ub_raw == maxw) return ub - maxw;
  const int64_t wl = ub - maxw > 0 ? ub - maxw : 0;
  const uint64_t nbins = (uint64_t)A.st_num + 2;
  const bool sh = nbins <= kStBins;
  unsigned long long* bins = sh ? S.bins : A.ring;
  for (uint64_t q = t; q < nbins; q += nt) bins[q] = 0ull;
  if (t == 0) {
    uint32_t j = j0;
    while (j <= step && __ldcg(&A.step_ub[j]) <= wl) ++j;
    s_beg = j <= step ? __ldcg(&A.step_off[j]) : send;
  }
  __syncthreads();
  const uint64_t span = (uint64_t)(st1 - st0);
  for (uint32_t i = s_beg + t; i < send; i += nt) {
    const int64_t d = ld_list(&A.sd[i]);
    if (d < wl) continue;
    const uint32_t dg = __ldg(&A.G.dvals[degree_rank(A.G, ld_list(&A.sid[i]))]);
    uint64_t cnt;  // how many x_k are <= d: the k with k (st1 - st0) < (d - st0 + 1) ST_NUM
    if (d < st0)
      cnt = 0;
    else if (span == 0)
      cnt = nbins - 1;
    else
      cnt = min(((uint64_t)(d - st0 + 1) * A.st_num + span - 1) / span, nbins - 1);
    atomicAdd(&bins[cnt], (unsigned long long)dg);
  }
  __syncthreads();
  // suffix sums: chunk totals, a scan over the chunks, then within the chunks
  const uint64_t cs = (nbins + nt - 1) / nt;
  const uint64_t q0 = t * cs, q1 = min(nbins, q0 + cs);
  unsigned long long mine = 0;
  for (uint64_t q = q0; q < q1; ++q) mine += sh ? bins[q] : __ldcg(&bins[q]);
  S.part[t] = mine;
  __syncthreads();
  for (uint32_t o = 1; o < nt; o <<= 1) {
    unsigned long long v = t + o < nt ? S.part[t + o] : 0;
    __syncthreads();
    S.part[t] += v;
    __syncthreads();
  }
  unsigned long long acc = t + 1 < nt ? S.part[t + 1] : 0;
  for (uint64_t q = q1; q > q0; --q) {
    acc += sh ? bins[q - 1] : __ldcg(&bins[q - 1]);
    if (sh)
      bins[q - 1] = acc;
    else
      __stcg(&bins[q - 1], acc);
  }
  __syncthreads();
  double best = 0.0;
  uint32_t bk = 0xFFFFFFFFu;
  const uint32_t gsh = (A.st_num & (A.st_num - 1)) == 0 ? __ffs(A.st_num) - 1 : 32u;
  for (uint32_t k = t; k <= A.st_num; k += nt) {
    const int64_t x = st_candidate(k, span, A.st_num, gsh, st0);
    if (x >= ub) continue;
    const uint64_t q = x >= wl ? (uint64_t)k + 1 : 0;
    const unsigned long long dsum = sh ? bins[q] : __ldcg(&bins[q]);
    const double p = dev_profit(x, ub, y, dsum, sumd_ub, A.G.maxw, A.G.two_m);
    if (p > best) {
      best = p;
      bk = k;
    }
  }
  const uint32_t k = block_argmax(S, best, bk);
  if (k == 0xFFFFFFFFu) return ub;
  return st_candidate(k, span, A.st_num, gsh, st0);
}

// The same out of line, for the batch and serving kernels: inlined there it
// costs their query loop registers (and their speed), while the single-query
// kernel is not affected either way.
__device__ __noinline__ int64_t block_st_exact_call(const KArgs& A, S3Scr& S, int64_t ub, uint64_t sumd_ub,
                                                    int64_t gap_lb, int64_t gap_ub_raw, int64_t y, int64_t st0,
                                                    int64_t st1, uint32_t j0, uint32_t step, uint32_t send) {
  return block_st_exact(A, S, ub, sumd_ub, gap_lb, gap_ub_raw, y, st0, st1, j0, step, send);
}

// A fused round: the FUSED local iterations of Section 4.1 (bucket fusion),
// for graphs in which no window is longer than heavy_min (every degree <=
// heavy_min, so there are no grid tasks), in every round of a step after the
// first (and its first round too when the step has no pull). Each warp takes
// up to 32 of the round's frontier vertices (or of the push set, whose windows
// start at their cursors) and relaxes their windows; every vertex it improves
// goes into the warp's local queue (shared
// memory, kWarpStage entries) and is relaxed by the same warp in its next
// wave, with the distance it has then, until the local queue is empty. The
// warps advance independently, with no grid barrier between waves: the round
// replaces the step's remaining rounds. A vertex improved by two warps is
// relaxed by both, and the smaller distance wins (within a step any order of
// the relaxations is exact). What a full local queue cannot take goes to the
// next round's queue through the round's SAP bitmap, as in a plain round.
// A wave is one chain of dependent loads (the vertex record, its row, the
// neighbours' distances, the atomicMin) where a plain round adds a grid
// barrier and the next round's item fetch.
__device__ void fused_round(const KArgs& A, const RoundCtx& R, const Local& L, RoundScr& S, Stage& T,
                            uint32_t nitems, bool round1, const uint32_t* qin, Counters& C) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t gwarp = qblock(A) * (blockDim.x >> 5) + warp;
  WarpScr& W = S.w[warp];
  uint32_t* lq = T.wq[warp];  // the local queue: a ring of kWarpStage vertex ids
  uint32_t lh = 0, lt = 0;    // its head and tail (warp-uniform)
  WarpList Fw = {T.wf[warp], 0u, R.first_cnt, R.first_list};
  const uint32_t i0 = gwarp * 32;
  // a step's first round (no pull): the warp's first wave is its share of the
  // push set (and the source, once); later rounds: of the round's queue
  const uint32_t np = round1 ? L.push_end - L.push_beg : 0;
  uint32_t nseed = round1 && i0 < nitems ? min(32u, nitems - i0) : 0u;
  if (!round1 && i0 < nitems) {
    if (i0 + lane < nitems) lq[lane] = ld_list(&qin[i0 + lane]);
    lt = min(32u, nitems - i0);
  }
  __syncwarp();
  while (nseed || lh != lt) {
    uint32_t d = EIC_INF, b = 0, len = 0;
    bool vertex = false;  // a frontier vertex (or the source): its window starts at its row
    uint32_t u = 0;
    if (nseed) {
      const uint32_t i = i0 + lane;
      if (lane < nseed && i < np) {  // push set entry: settled, lb0 <= dist <= st (Function 1)
        const uint32_t idx = L.push_beg + i;
        d = ld_list(&A.sd[idx]);
        const uint32_t x = ld_list(&A.sid[idx]);
        const uint2 rr = make_uint2(__ldg(&A.G.row[x]), __ldg(&A.G.row[x + 1]));
        if ((int64_t)d >= R.lb0 && (int64_t)d <= R.st && !(d > 0 && rr.y - rr.x == 1)) {
          C.frontier += 1;
          const uint32_t cur = ld_list(&A.scur[idx]);
          b = cur == kNone ? lower_bound_w(A.G.adj, rr.x, rr.y, R.lb - (int64_t)d)
                           : gallop_w(A.G.adj, rr.x + cur, rr.y, R.lb - (int64_t)d);
          const uint32_t e = gallop_w(A.G.adj, b, rr.y, R.ub_eff - (int64_t)d);
          __stcg(&A.scur[idx], e - rr.x);
          len = e - b;
        }
      } else if (lane < nseed) {  // the source, once
        u = L.s_int;
        vertex = true;
      }
      nseed = 0;
    } else {
      const uint32_t k = min(32u, lt - lh);
      if (lane < k) {
        u = lq[(lh + lane) & (kWarpStage - 1)];
        vertex = true;
      }
      __syncwarp();
      lh += k;
    }
    if (vertex) {
      d = __ldcg(&A.dist[u]);
      const uint32_t rb = __ldg(&A.G.row[u]), re = __ldg(&A.G.row[u + 1]);
      // d >= lb: the window is the row's prefix with weight < ub - d; rows are
      // short, so the whole row is read and filtered (a search only for rows
      // that keep a cursor)
      if (d != EIC_INF && !(d > 0 && re - rb == 1)) {  // Paths excludes leaves (Algorithm 1)
        C.frontier += 1;
        const int64_t hi = R.ub_eff - (int64_t)d;
        if (hi > 0) {
          b = rb;
          len = re - rb;
          if (re - rb > kCursorMin) {
            const uint32_t e = gallop_w(A.G.adj, rb, re, hi);
            __stcg(&A.cursor[u], e - rb);
            len = e - rb;
          }
        }
      }
    }
    const uint32_t incl = warp_incl_scan(len);
    const uint32_t total = __shfl_sync(EIC_FULL_MASK, incl, 31);
    W.beg[lane] = b;
    W.excl[lane] = incl - len;
    W.val[lane] = d;
    __syncwarp();
    for (uint32_t g0 = 0; g0 < total; g0 += 32) {
      const uint32_t g = g0 + lane;
      bool ok = false, first = false;
      uint32_t v = 0;
      if (g < total) {
        uint32_t lo = 0, hi = 31;
        while (lo < hi) {  // the last lane whose window starts at or before g
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (W.excl[mid] <= g)
            lo = mid;
          else
            hi = mid - 1;
        }
        const uint2 ent = ld_stream(&A.G.adj[W.beg[lo] + (g - W.excl[lo])]);
        const uint32_t du = W.val[lo];
        v = ent.x;
        if ((int64_t)ent.y < R.ub_eff - (int64_t)du) {
          C.trav += 1;
          const uint32_t nd = du + ent.y;  // < min(ub, 2^32 - 1) by the window
          if (nd < __ldcg(&A.dist[v])) {
            const uint32_t old = atomicMin(&A.dist[v], nd);
            ok = nd < old;
            first = ok && old == EIC_INF;
          }
        }
      }
      C.improved += ok ? 1 : 0;
      // into the local queue while it has room, else into the next round's queue (SAP)
      const uint32_t m = __ballot_sync(EIC_FULL_MASK, ok);
      const uint32_t cnt = __popc(m);
      if (cnt && cnt <= kWarpStage - (lt - lh)) {
        if (ok) lq[(lt + __popc(m & ((1u << lane) - 1u))) & (kWarpStage - 1)] = v;
        lt += cnt;
      } else if (cnt) {
        bool sap = false;
        if (ok) {
          const uint32_t bit = 1u << (v & 31);
          sap = !(atomicOr(&R.fbits[v >> 5], bit) & bit);
        }
        const uint32_t slot = warp_append(sap, R.qcnt_out);
        if (sap) __stcg(&R.qout[slot], v);
      }
      warp_push(Fw, first, v);
      __syncwarp();
    }
  }
  warp_flush(Fw);
  tl_block(A, 6, R.rid);
}

// Function 2 for the boundary <lb, ub> -> next pair <ub, ub + gap(ub)>, run by
// one whole block. Candidates x_k = st0 + floor(k (st1 - st0) / ST_NUM) < ub;
// D(x') = sumD(x') - sumD(ub), the degree sum of the settled vertices with
// x' <= dist < ub, x' = max(x, ub - maxW), read from the ring of settled
// degree sums (one slot per distance: maxW < 2^20; wider weights go through
// block_st_exact).
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
  for (uint32_t o = 1; o < nt; o <<= 1) {  // suffix sums over chunks
    unsigned long long v = t + o < nt ? S.part[t + o] : 0;
    __syncthreads();
    S.part[t] += v;
    __syncthreads();
  }
  double best = 0.0;
  uint32_t bk = 0xFFFFFFFFu;
  const uint64_t span = (uint64_t)(st1 - st0);
  const uint32_t gsh = (A.st_num & (A.st_num - 1)) == 0 ? __ffs(A.st_num) - 1 : 32u;
  for (uint32_t k = t; k <= A.st_num; k += nt) {
    const int64_t x = st_candidate(k, span, A.st_num, gsh, st0);
    if (x >= ub) continue;
    const int64_t xc = x > ub - maxw ? x : ub - maxw;
    if (k > 0) {  // the profit depends on x' only: the first candidate of each x' decides the argmax
      const int64_t xp = st_candidate(k - 1, span, A.st_num, gsh, st0);
      if ((xp > ub - maxw ? xp : ub - maxw) == xc) continue;
    }
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
  const uint32_t k = block_argmax(S, best, bk);
  if (k == 0xFFFFFFFFu) return ub;
  return st_candidate(k, span, A.st_num, gsh, st0);
}

// Step boundary, executed by block 0 once every block finished the
// statistics pass: sumD(ub), highD(ub), gap(ub) (Eq. 1-3), termination
// (Algorithm 1), computeST (Function 2) and the push/pull sets of the next
// step's Function 1. Publishes the new control values before the grid barrier.
template <bool kExactInline, bool kParGap>
__device__ void step_boundary(const KArgs& A, PhaseScr& P, BState& B, const Local& L, uint32_t rounds_in_step) {
  Ctl* c = A.ctl;
  __shared__ int64_t sh_i[8];
  __shared__ uint64_t sh_u[4];
  __shared__ uint32_t sh_flag[2];
  __shared__ int64_t sh_gap[kGapPar];
  const DevGraph& G = A.G;
  const int64_t lb = L.lb, ub = L.ub;
  const uint32_t k = L.step;
  if (threadIdx.x == 0) {
    const uint32_t settled_now = __ldcg(&c->settled_cnt);
    const unsigned long long acc = __ldcg(&c->acc_deg);
    const uint32_t acc_maxd1 = __ldcg(&c->acc_maxd1);
    const uint64_t sumd_ub = B.sumd_lb - acc;
    sh_u[0] = sumd_ub;
    sh_u[1] = settled_now;
    if (acc_maxd1 && (int64_t)(acc_maxd1 - 1) > B.max_settled) B.max_settled = acc_maxd1 - 1;
    const int64_t maxs = B.max_settled;
    A.step_ub[k] = ub;
    if (k <= A.trace_cap && A.trace) {
      eic_step r;
      r.lb = lb;
      r.ub = ub;
      r.st = L.st;
      r.gap_lb = B.gap_lb;
      r.sumd_lb = B.sumd_lb;
      r.highd_lb = B.highd_lb;
      r.rounds = rounds_in_step;
      r.settled = settled_now - L.step_off_cur;
      r.flags = (L.pull_on ? EIC_STEP_PULL : 0u) | (L.pull_on && L.pull_sweep ? EIC_STEP_SWEPT : 0u);
      r.reserved = 0;
      A.trace[k - 1] = r;
    }
    c->trace_len = k;
    c->cnt_rounds += rounds_in_step;
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
  uint32_t highd_ub;
  // With few distinct degrees (road-like graphs: the fused kernel), Eq. 1-3 is
  // evaluated for every value highD can take (each distinct degree) by the
  // other warps while warp 0 finds highD: the double-precision chain of Eq. 2
  // is long on this GPU, and it then runs beside highD instead of after it.
  const bool gap_par = kParGap && G.D <= kGapPar && blockDim.x >= 32 + G.D;
  if (gap_par && threadIdx.x >= 32 && threadIdx.x < 32 + G.D)
    sh_gap[threadIdx.x - 32] = dev_gap(sumd_ub, G.dvals[threadIdx.x - 32], G.two_m, A.alpha, A.beta, G.rtow);
  if (G.D <= 32 * kWarpHighdPer) {  // one warp, no block barriers
    if (threadIdx.x < 32) {
      const uint32_t h = warp_highd(A.hist, G.dvals, G.D);
      if (threadIdx.x == 0) sh_flag[1] = h;
    }
    __syncthreads();
    highd_ub = sh_flag[1];
  } else {
    highd_ub = block_highd(A.hist, G.dvals, G.D);
  }
  if (sh_flag[0]) {
    if (threadIdx.x == 0) {
      c->done = 1;
      c->s2_done = 0;  // published by the grid barrier's release
    }
    __syncthreads();
    return;
  }
  if (threadIdx.x == 0) {
    // highD is a distinct degree (its rank from drank) or 0 (empty set: gap maxW(G, 1))
    const int64_t gap_raw = gap_par && highd_ub > 0 ? sh_gap[__ldg(&G.drank[highd_ub])]
                                                    : dev_gap(sumd_ub, highd_ub, G.two_m, A.alpha, A.beta, G.rtow);
    if (k == 1) B.st0 = ub;
    if (B.st1 < 0 && sumd_ub <= G.m) B.st1 = ub;
    sh_i[1] = gap_raw;
    sh_i[2] = gap_raw << A.gap_shift;
  }
  __syncthreads();
  const int64_t gap_raw = sh_i[1], width = sh_i[2];
  const int64_t nlb = ub, nub = ub + width;
  const int64_t nst = (A.flags & EIC_FLAG_NO_PULL) ? nlb
                      : A.ring_shift == 0
                          ? block_compute_st(A, P.s3, ub, sumd_ub, B.gap_lb, gap_raw, nub, B.st0, B.st1)
                          : kExactInline ? block_st_exact(A, P.s3, ub, sumd_ub, B.gap_lb, gap_raw, nub, B.st0, B.st1,
                                                          B.j0, k, (uint32_t)sh_u[1])
                                         : block_st_exact_call(A, P.s3, ub, sumd_ub, B.gap_lb, gap_raw, nub, B.st0,
                                                               B.st1, B.j0, k, (uint32_t)sh_u[1]);
  if (A.ring_shift == 0) {  // zero the ring slots the next statistics pass fills: [max(nlb, nub - maxW), nub)
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
      A.sid[scnt] = L.s_int;
      A.sd[scnt] = 0;
      A.scur[scnt] = kNone;
      ++scnt;
      extra = 1;
    }
    // Function 1's push set {lb0 <= dist <= st}: the settled steps j with
    // ub_j > lb0 (j0, moving forward only) and lb_j <= st (j1, from the back)
    const int64_t lb0 = nlb - (int64_t)G.maxw > 0 ? nlb - (int64_t)G.maxw : 0;
    uint32_t pb = 0, pe = 0;
    while (B.j0 <= k && __ldcg(&A.step_ub[B.j0]) <= lb0) ++B.j0;
    if (nst >= lb0) {
      uint32_t j1 = k;
      int64_t lbj = lb;  // lb_k
      while (j1 >= 1 && lbj > nst) {
        --j1;
        lbj = j1 >= 2 ? __ldcg(&A.step_ub[j1 - 1]) : 0;
      }
      if (B.j0 <= j1 && j1 >= 1) {
        pb = __ldcg(&A.step_off[B.j0]);
        pe = j1 == k ? settled_now : __ldcg(&A.step_off[j1 + 1]);
      }
    }
    // Function 1's pull: unsettled vertices with an edge lighter than ub - st,
    // a prefix of the weight-ordered non-isolated vertices
    const uint32_t pull_on = nst < nlb ? 1u : 0u;
    uint32_t pull_cnt = 0;
    if (pull_on) {
      const int64_t bound = nub - nst;  // smallest weight < bound
      if (bound >= (int64_t)G.nz_lt_len) {
        if ((uint64_t)bound > G.maxw) {
          pull_cnt = G.nz_count;
        } else {
          uint32_t lo = 0, hi = G.nz_count;
          while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if ((int64_t)__ldg(&G.nz[mid].y) < bound)
              lo = mid + 1;
            else
              hi = mid;
          }
          pull_cnt = lo;
        }
      } else if (bound > 0) {
        pull_cnt = __ldg(&G.nz_lt[bound]);
      }
    }
    c->settled_cnt = scnt;
    c->lb = nlb;
    c->ub = nub;
    c->st = nst;
    c->lb0 = lb0;
    c->step = k + 1;
    c->push_beg = pb;
    c->push_end = pe;
    c->pull_on = pull_on;
    // a pull set of most vertices is swept in vertex order: rows are read in
    // address order across the grid (the weight-ordered list would make one
    // pass per weight value), and what the round inserts comes out in
    // vertex order, which the next round and the statistics pass read
    const uint32_t sweep = pull_on && (uint64_t)pull_cnt * kSweepDen >= (uint64_t)G.ni * kSweepNum ? 1u : 0u;
    c->pull_sweep = sweep;
    c->pull_cnt = sweep ? G.ni : pull_cnt;
    c->extra_s = extra;
    c->step_off_cur = settled_now;
    B.sumd_lb = sumd_ub;
    B.highd_lb = highd_ub;
    B.gap_lb = gap_raw;
    c->acc_deg = 0;
    c->acc_maxd1 = 0;
    c->s2_done = 0;
    c->done = 0;  // the control values are published by the grid barrier's release
  }
  __syncthreads();
}

// All threads: control values published before the last barrier (one thread
// loads them from L2, the block shares them).
__device__ void read_ctl(const Ctl* c, Local& L) {
  __shared__ Local sL;
  if (threadIdx.x == 0) {
    sL.lb = __ldcg(&c->lb);
    sL.ub = __ldcg(&c->ub);
    sL.st = __ldcg(&c->st);
    sL.lb0 = __ldcg(&c->lb0);
    sL.step = __ldcg(&c->step);
    sL.push_beg = __ldcg(&c->push_beg);
    sL.push_end = __ldcg(&c->push_end);
    sL.pull_on = __ldcg(&c->pull_on);
    sL.pull_cnt = __ldcg(&c->pull_cnt);
    sL.pull_sweep = __ldcg(&c->pull_sweep);
    sL.extra_s = __ldcg(&c->extra_s);
    sL.step_off_cur = __ldcg(&c->step_off_cur);
    sL.done = __ldcg(&c->done);
    sL.s_int = __ldcg(&c->s_int);
  }
  __syncthreads();
  const uint32_t rid = L.rid, qsel = L.qsel;
  L = sL;
  L.rid = rid;
  L.qsel = qsel;
  L.cur_cnt = 0;
  __syncthreads();
}

// Block sum of several counters; thread 0 receives the totals.
template <int K>
__device__ __forceinline__ void block_sums(unsigned long long (&v)[K], unsigned long long (*sh)[K]) {
#pragma unroll
  for (int j = 0; j < K; ++j) v[j] = warp_sum_u64(v[j]);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int j = 0; j < K; ++j) sh[threadIdx.x >> 5][j] = v[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (uint32_t w = 1; w < (blockDim.x >> 5); ++w)
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] += sh[w][j];
  }
  __syncthreads();
}

// Shared-memory scratch of one block in the query loop.
struct QueryShared {
  PhaseScr P;
  Stage T;
  BState B;
  unsigned long long red[32][7];
  unsigned long long snap[4];
  uint32_t last;
};

// The query loop of Algorithm 1 run by the A.nb blocks of one query: rounds
// of a step (item phase, task phase), statistics pass, step boundary, until
// termination. gen is the block's copy of the barrier generation (uint32_t),
// or its arrival ticket in a launch that runs this one query only (64-bit).
// kFuse: 0 no fused rounds, 1 fused rounds, 2 as A.fuse says (per query).
template <uint32_t kPullFast, uint32_t kRelaxIlp, uint32_t kFuse = 0, class Gen = uint32_t>
__device__ void run_query(const KArgs& A, QueryShared& Q, Gen& gen) {
  PhaseScr& P = Q.P;
  Stage& T = Q.T;
  BState& B = Q.B;
  auto& sh_red = Q.red;
  auto& sh_snap = Q.snap;
  uint32_t& sh_last = Q.last;
  Ctl* c = A.ctl;
  const uint32_t qb = qblock(A);
  Local L;
  L.rid = 0;
  L.qsel = 0;
  read_ctl(c, L);
  L.cur_cnt = 1;  // the first round's frontier is {s}
  Counters C = {0, 0, 0, 0, 0, 0};
  if (threadIdx.x == 0) {
    T.tn = 0;
    B.st0 = -1;
    B.st1 = -1;
    B.gap_lb = __ldcg(&c->gap_lb);
    B.max_settled = -1;
    B.sumd_lb = A.G.two_m;
    B.highd_lb = A.G.highd0;
    B.j0 = 1;
  }
  if (qb == 0 && threadIdx.x == 0) tl_mark(A, 0, L.rid);
  bool alive = !L.done;  // an isolated source has nothing to relax
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
      if (qb == 0 && threadIdx.x == 0) {
        c->qcnt[(L.rid + 1) % 3] = 0;
        c->tcnt[(L.rid + 1) % 3] = 0;
        c->work[(L.rid + 1) % 3] = 0;
      }
      {  // the other bitmap served round rid-1 and is next used in round rid+1: clear it now
        uint32_t* other = A.fbits + ((L.rid + 1) & 1u) * A.fwords;
        for (uint32_t wi = qb * blockDim.x + threadIdx.x; wi < A.fwords; wi += A.nb * blockDim.x)
          __stcg(&other[wi], 0u);
      }
      RoundCtx R;
      R.fbits = A.fbits + (L.rid & 1u) * A.fwords;
      R.lb = L.lb;
      R.ub = L.ub;
      R.ub_eff = L.ub < (int64_t)EIC_INF ? L.ub : (int64_t)EIC_INF;
      R.st = L.st;
      R.lb0 = L.lb0;
      R.rid = L.rid;
      R.step1 = L.step == 1;
      R.qout = L.qsel ? A.q0 : A.q1;
      R.qcnt_out = &c->qcnt[L.rid % 3];
      R.first_list = R.step1 ? A.touched : A.sid;
      R.first_cnt = R.step1 ? &c->touched_cnt : &c->settled_cnt;
      R.tcnt = &c->tcnt[L.rid % 3];
      R.work = &c->work[L.rid % 3];
      const uint32_t* qin = L.qsel ? A.q1 : A.q0;
      Local LL = L;
      if (!L.pull_on) LL.pull_cnt = 0;
      const uint32_t nitems = round1 ? (LL.push_end - LL.push_beg) + LL.pull_cnt + LL.extra_s : L.cur_cnt;
      if (qb == 0 && threadIdx.x == 0) tl_mark(A, 8, nitems);  // diagnostic: the round's items
      if ((kFuse == 1 || (kFuse == 2 && A.fuse)) && !R.step1 && (!round1 || !LL.pull_on) &&
          nitems <= 32u * A.nb * (blockDim.x >> 5))
        fused_round(A, R, LL, P.r, T, nitems, round1, qin, C);
      else
        round_phase<kPullFast, kRelaxIlp>(A, R, LL, P.r, T, nitems, round1, qin, C);
      if (!grid_barrier(&c->bar, &gen, A.nb, A.max_spin, &c->status)) {
        alive = false;
        break;
      }
      if (threadIdx.x == 0) {
        sh_snap[0] = __ldcg(&c->tcnt[L.rid % 3]);
        sh_snap[1] = __ldcg(&c->qcnt[L.rid % 3]);
        sh_snap[2] = __ldcg(&c->ub_cand);
        if (qb == 0) tl_mark(A, 1, L.rid);
      }
      __syncthreads();
      const unsigned long long hp = sh_snap[0];
      L.cur_cnt = (uint32_t)sh_snap[1];
      uint32_t uc = (uint32_t)sh_snap[2];
      __syncthreads();
      if (hp != 0) {
        if (qb == 0 && threadIdx.x == 0) tl_mark(A, 9, (uint32_t)hp);  // diagnostic: the round's tasks
        task_phase<(kRelaxIlp >= 2)>(A, R, (uint32_t)hp, T, C);
        if (!grid_barrier(&c->bar, &gen, A.nb, A.max_spin, &c->status)) {
          alive = false;
          break;
        }
        if (qb == 0 && threadIdx.x == 0) tl_mark(A, 2, L.rid);
        if (threadIdx.x == 0) {
          sh_snap[1] = __ldcg(&c->qcnt[L.rid % 3]);
          sh_snap[2] = __ldcg(&c->ub_cand);
        }
        __syncthreads();
        L.cur_cnt = (uint32_t)sh_snap[1];
        uc = (uint32_t)sh_snap[2];
        __syncthreads();
      }
      if (R.step1 && uc != EIC_INF && (int64_t)uc < L.ub) L.ub = uc;
      L.qsel ^= 1u;
      ++rin;
      if (L.cur_cnt == 0) break;
    }
    if (!alive) break;
    // ------------------------------------------------ statistics pass
    {
      S2Scr& S = P.s2;
      const bool step1 = L.step == 1;
      const uint32_t* list = step1 ? A.touched : A.sid;
      const uint32_t lbeg = step1 ? 0 : L.step_off_cur;
      if (threadIdx.x == 0) sh_snap[3] = step1 ? __ldcg(&c->touched_cnt) : __ldcg(&c->settled_cnt);
      __syncthreads();
      const uint32_t lend = (uint32_t)sh_snap[3];
      const bool has = lbeg + qb * blockDim.x < lend;  // this block has settled vertices to count
      const int64_t wlo = L.ub - (int64_t)A.G.maxw > L.lb ? L.ub - (int64_t)A.G.maxw : L.lb;
      const bool ring_sh = A.ring_shift == 0 && L.ub < EIC_INF_T && (L.ub - wlo) <= kShRing;
      const bool ring_narrow = ring_sh && (L.ub - wlo) <= kRingNarrow && A.G.max_deg < (1u << 27);  // (in shared memory)
      if (has) {
        for (int r = threadIdx.x; r < kShRanks; r += blockDim.x) S.hist[r] = 0;
        if (ring_sh)
          for (int r = threadIdx.x; r < kShRing; r += blockDim.x) S.ring[r] = 0;
      }
      __syncthreads();
      unsigned long long bdeg = 0;
      uint32_t bmax = 0, bany = 0;
      const uint32_t nthreads = A.nb * blockDim.x;
      uint32_t xnext = 0;  // the single-query shape loads the next list entry one iteration ahead
      if constexpr (kRelaxIlp >= 2) {
        if (lbeg + qb * blockDim.x + threadIdx.x < lend) xnext = ld_list(&list[lbeg + qb * blockDim.x + threadIdx.x]);
      }
      for (uint32_t base = lbeg + qb * blockDim.x; base < lend; base += nthreads) {
        const uint32_t idx = base + threadIdx.x;
        bool take = false;
        uint32_t x = 0, d = 0, r = EIC_INF, dg = 0, cx = kNone;
        uint32_t xcur = 0;
        if constexpr (kRelaxIlp >= 2) {
          xcur = xnext;
          if (idx + nthreads < lend) xnext = ld_list(&list[idx + nthreads]);
        }
        if (idx < lend) {
          if constexpr (kRelaxIlp >= 2)
            x = xcur;
          else
            x = ld_list(&list[idx]);
          d = __ldcg(&A.dist[x]);
          cx = x < A.G.nlong ? __ldcg(&A.cursor[x]) : kNone;  // (a long row by its id: loaded with dist)
          r = degree_rank(A.G, x);  // (the degree from the id: no random row read)
          dg = __ldg(&A.G.dvals[r]);
          take = true;
          if (step1 && d64(d) >= L.ub) {  // first step: keep only what is final
            if (x != L.s_int) __stcg(&A.dist[x], EIC_INF);
            take = false;
          }
        }
        if (step1) {
          const uint32_t slot = warp_append(take, &c->settled_cnt);
          if (take) {
            __stcg(&A.sid[slot], x);
            __stcg(&A.sd[slot], d);
            __stcg(&A.scur[slot], kNone);  // the first step's windows used a larger ub
          }
        }
        if (take) {
          atomicOr(&A.sbits[x >> 5], 1u << (x & 31));
          if (!step1) {
            __stcg(&A.sd[idx], d);
            __stcg(&A.scur[idx], cx);
          }
          bdeg += dg;
          bmax = d > bmax ? d : bmax;
          bany = 1;
        }
        // degree histogram (internal vertices all have degree >= 1)
        if (!take) r = EIC_INF;
        if (r < (uint32_t)kShRanks)
          atomicAdd(&S.hist[r], 1u);
        else if (r != EIC_INF)
          atomicSub(&A.hist[r], 1u);
        // D(x) ring: in a narrow window the step's settled vertices share few
        // distances; then one atomic per distinct slot in the warp, with the
        // group's degree sum (32-bit while 32 degrees cannot overflow it)
        const bool rk = take && (int64_t)d >= wlo && A.ring_shift == 0;  // (wide weights: Function 2 sums exactly)
        const uint32_t slot = rk ? (ring_sh ? (uint32_t)(d - wlo) : (uint32_t)(((uint64_t)d >> A.ring_shift) & A.ring_mask))
                                 : EIC_INF;
        if (ring_narrow) {
          const uint32_t rg = __match_any_sync(EIC_FULL_MASK, slot);
          const uint32_t sum = __reduce_add_sync(rg, rk ? dg : 0u);
          if (rk && lane_id() == (uint32_t)__ffs(rg) - 1) atomicAdd(&S.ring[slot], (unsigned long long)sum);
        } else if (rk) {
          if (ring_sh)
            atomicAdd(&S.ring[slot], (unsigned long long)dg);
          else
            atomicAdd(&A.ring[slot], (unsigned long long)dg);
        }
      }
      __syncthreads();
      if (has) {
        for (int r = threadIdx.x; r < kShRanks; r += blockDim.x)
          if (S.hist[r]) atomicSub(&A.hist[r], S.hist[r]);
        if (ring_sh)
          for (int r = threadIdx.x; r < kShRing && r < L.ub - wlo; r += blockDim.x)
            if (S.ring[r]) atomicAdd(&A.ring[((uint64_t)(wlo + r)) & A.ring_mask], S.ring[r]);
      }
      // block totals: degree sum and 1 + the largest distance (0: none), one atomic each
      unsigned long long v[2] = {bdeg, bany ? (unsigned long long)bmax + 1 : 0ull};
      v[0] = warp_sum_u64(v[0]);
      for (int o = 16; o > 0; o >>= 1) v[1] = max(v[1], __shfl_xor_sync(EIC_FULL_MASK, v[1], o));
      if ((threadIdx.x & 31) == 0) {
        sh_red[threadIdx.x >> 5][0] = v[0];
        sh_red[threadIdx.x >> 5][1] = v[1];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (uint32_t w = 1; w < (blockDim.x >> 5); ++w) {
          v[0] += sh_red[w][0];
          v[1] = max(v[1], sh_red[w][1]);
        }
        if (v[0]) atomicAdd(&c->acc_deg, v[0]);
        if (v[1]) atomicMax(&c->acc_maxd1, (uint32_t)v[1]);
        atom_add_acq_rel_u32(&c->s2_done, 1u);  // releases the block's statistics
      }
      if (qb == 0) {  // block 0 waits (bounded) for every block's statistics
        if (threadIdx.x == 0) {
          uint64_t spins = 0;
          sh_last = 1;
          while (ld_acquire_u32(&c->s2_done) < A.nb) {
            if (ld_volatile_int(&c->status) != 0 || ++spins > A.max_spin) {
              atomicCAS(&c->status, 0, EIC_ETIMEOUT);
              sh_last = 0;
              break;
            }
          }
          tl_mark(A, 4, L.rid);
        }
        __syncthreads();
        if (sh_last) step_boundary<(kRelaxIlp >= 2), kFuse == 1>(A, P, B, L, rin);  // (the single-query shape inlines)
        if (threadIdx.x == 0) tl_mark(A, 5, L.rid);
      }
    }
    if (!grid_barrier(&c->bar, &gen, A.nb, A.max_spin, &c->status)) break;
    if (qb == 0 && threadIdx.x == 0) tl_mark(A, 3, L.rid);
    read_ctl(c, L);
    if (L.done) break;
  }
  {  // the query's counters, once per block
    unsigned long long v[7] = {C.frontier, C.trav, C.pulls, C.improved, C.heavy, C.pitems, 0ull};
    block_sums<7>(v, sh_red);
    if (threadIdx.x == 0) {
      atomicAdd(&c->cnt_frontier, v[0]);
      atomicAdd(&c->cnt_trav, v[1]);
      atomicAdd(&c->cnt_pulls, v[2]);
      atomicAdd(&c->cnt_improved, v[3]);
      atomicAdd(&c->cnt_heavy, v[4]);
      atomicAdd(&c->cnt_pitems, v[5]);
    }
  }
  if (qb == 0 && threadIdx.x == 0 && A.status_out) *A.status_out = ld_volatile_int(&c->status);
}

__global__ void __launch_bounds__(kMaxBlock, 2) k_eic(KArgs A) {
  __shared__ QueryShared Q;
  unsigned long long ticket = 0;  // (k_init zeroed the arrival count)
  run_query<kPullFastSingle, kRelaxIlpSingle>(A, Q, ticket);
}

// The same query with fused rounds (bucket fusion), for graphs whose every
// degree is at most heavy_min: road-like graphs, whose steps take many small
// rounds.
__global__ void __launch_bounds__(kMaxBlock, 2) k_eic_fused(KArgs A) {
  __shared__ QueryShared Q;
  unsigned long long ticket = 0;  // (k_init zeroed the arrival count)
  run_query<kPullFastSingle, kRelaxIlpSingle, 1>(A, Q, ticket);
}

// Control block of a new query (one thread): the source's distance, the
// first round's frontier {s}, step 1 = <0, +inf> with st = 0, and gap(0).
__device__ void ctl_init(const KArgs& A) {
  Ctl* c = A.ctl;
  const DevGraph& G = A.G;
  const uint32_t si = G.orig2int[A.s];
  c->s_int = si;
  uint32_t dgs = 0;
  if (si != EIC_INF) {
    A.dist[si] = 0;
    A.q0[0] = si;
    A.touched[0] = si;
    dgs = G.row[si + 1] - G.row[si];
  }
  A.step_off[1] = 0;
  A.step_ub[0] = 0;
  c->lb = 0;
  c->ub = EIC_INF_T;
  c->st = 0;
  c->lb0 = 0;
  c->step = 1;
  c->done = si == EIC_INF ? 1u : 0u;
  c->push_beg = c->push_end = 0;
  c->pull_on = c->pull_cnt = c->extra_s = 0;
  c->pull_sweep = 0;
  c->step_off_cur = 0;
  c->st0 = -1;
  c->st1 = -1;
  c->sumd_lb = G.two_m;
  c->highd_lb = G.highd0;
  c->gap_lb = dev_gap(G.two_m, G.highd0, G.two_m, A.alpha, A.beta, G.rtow);
  c->max_settled = -1;
  c->rounds_in_step = 0;
  c->trace_len = 0;
  c->tl_len = 0;
  c->qcnt[0] = c->qcnt[1] = c->qcnt[2] = 0;
  c->work[0] = c->work[1] = c->work[2] = 0;
  c->settled_cnt = 0;
  c->touched_cnt = 1;
  c->ub_cand = (G.highd0 > 0 && dgs >= G.highd0) ? 0u : EIC_INF;
  c->tcnt[0] = c->tcnt[1] = c->tcnt[2] = 0;
  c->s2_done = 0;
  c->acc_maxd1 = 0;
  c->acc_deg = 0;
  c->cnt_rounds = c->cnt_frontier = c->cnt_trav = c->cnt_pulls = c->cnt_improved = c->cnt_heavy = 0;
  c->cnt_pitems = 0;
}

__global__ void k_init(KArgs A) {
  const DevGraph& G = A.G;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < G.D; r += gridDim.x * blockDim.x) A.hist[r] = G.dcnt0[r];
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r <= A.ring_mask; r += gridDim.x * blockDim.x) A.ring[r] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl_init(A);
    A.ctl->bar.count = 0;
    A.ctl->bar.arrived = 0;
    A.ctl->status = 0;
  }
}

// Distances in the caller's numbering: out[u] = dist[orig2int[u]], +inf for
// isolated vertices, 0 for the source.
// Each thread has kOutIlp independent gathers in flight.
constexpr uint32_t kOutIlp = 4;
__global__ void k_output(DevGraph G, const uint32_t* __restrict__ idist, uint32_t s, uint32_t* out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t u0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u0 < G.n; u0 += kOutIlp * stride) {
    uint32_t i[kOutIlp], d[kOutIlp];
#pragma unroll
    for (uint32_t k = 0; k < kOutIlp; ++k) {
      const uint64_t u = u0 + k * stride;
      i[k] = u < G.n ? __ldg(&G.orig2int[u]) : EIC_INF;
    }
#pragma unroll
    for (uint32_t k = 0; k < kOutIlp; ++k) d[k] = i[k] == EIC_INF ? EIC_INF : __ldcg(&idist[i[k]]);
#pragma unroll
    for (uint32_t k = 0; k < kOutIlp; ++k) {
      const uint64_t u = u0 + k * stride;
      if (u < G.n) out[u] = u == s ? 0u : d[k];
    }
  }
}

// parent[v] = smallest original id u with dist[u] + w(u, v) == dist[v] (one
// warp per vertex); parent[s] = s, +inf where unreachable.
__global__ void k_parent(DevGraph G, const uint32_t* __restrict__ idist, uint32_t s, uint32_t* parent) {
  const uint32_t lane = lane_id();
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t v = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < G.n; v += nw) {
    const uint32_t vi = G.orig2int[v];
    const uint32_t dv = vi == EIC_INF ? EIC_INF : idist[vi];
    uint32_t best = EIC_INF;
    if (v != s && dv != EIC_INF) {
      const uint32_t rb = G.row[vi], re = G.row[vi + 1];
      for (uint32_t i = rb + lane; i < re; i += 32) {
        const uint2 ent = G.adj[i];
        if (ent.y > dv) break;
        const uint32_t du = idist[ent.x];
        if (du != EIC_INF && (uint64_t)du + ent.y == dv) {
          const uint32_t uo = G.int2orig[ent.x];
          best = uo < best ? uo : best;
        }
      }
      for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(EIC_FULL_MASK, best, o));
    }
    if (lane == 0) parent[v] = v == s ? s : best;
  }
}

// ------------------------------------------------------------- batched queries

struct BatchArgs {
  const BatchQuery* q;    // [nq], in the order groups claim them
  const BatchSlot* slot;  // [gridDim.x / nb]
  int* status;            // [nq]; a query no group finished keeps EIC_EABORT
  uint32_t* queue;        // next unclaimed query
  uint32_t nq, nb;        // queries; blocks per group
  uint32_t alpha;
  double beta;
  uint32_t st_num, gap_shift, heavy_min, flags, step_cap;
  uint64_t max_spin;
};

// The query's scratch at its starting values (what the single-query path
// does with memsets and k_init), by the group's blocks.
__device__ bool query_setup(const KArgs& A, uint32_t& gen) {
  const DevGraph& G = A.G;
  const uint32_t stride = A.nb * blockDim.x, t0 = qblock(A) * blockDim.x + threadIdx.x;
  for (uint32_t i = t0; i < G.ni; i += stride) __stcg(&A.dist[i], EIC_INF);
  for (uint32_t i = t0; i < 2 * A.fwords; i += stride) __stcg(&A.fbits[i], 0u);
  for (uint32_t i = t0; i < A.fwords; i += stride) __stcg(&A.sbits[i], 0u);
  for (uint32_t r = t0; r < G.D; r += stride) __stcg(&A.hist[r], __ldg(&G.dcnt0[r]));
  for (uint32_t r = t0; r <= A.ring_mask; r += stride) __stcg(&A.ring[r], 0ull);
  if (!grid_barrier(&A.ctl->bar, &gen, A.nb, A.max_spin, &A.ctl->status)) return false;
  if (qblock(A) == 0 && threadIdx.x == 0) ctl_init(A);
  return grid_barrier(&A.ctl->bar, &gen, A.nb, A.max_spin, &A.ctl->status);
}

// Distances in the caller's numbering (as k_output), by the group's blocks.
__device__ void query_output(const KArgs& A) {
  const DevGraph& G = A.G;
  const uint64_t stride = (uint64_t)A.nb * blockDim.x;
  for (uint64_t u = (uint64_t)qblock(A) * blockDim.x + threadIdx.x; u < G.n; u += stride) {
    const uint32_t i = __ldg(&G.orig2int[u]);
    A.out[u] = u == A.s ? 0u : (i == EIC_INF ? EIC_INF : __ldcg(&A.dist[i]));
  }
}

// Many queries in one cooperative launch. The grid is cut into groups of nb
// blocks; each group claims the next query from a device counter, runs it
// with its own scratch and a barrier over its nb blocks, writes the output,
// and claims again. A group stops at its first query with a non-OK status
// (its barrier state is then unreliable); the other groups carry on.
__global__ void __launch_bounds__(kMaxBlock, 2) k_eic_batch(BatchArgs P) {
  __shared__ QueryShared Q;
  __shared__ KArgs sA;
  __shared__ uint32_t sh_qi;
  const uint32_t grp = blockIdx.x / P.nb, qb = blockIdx.x % P.nb;
  const BatchSlot& W = P.slot[grp];
  Ctl* c = W.ctl;
  uint32_t gen = __ldcg(&c->bar.gen);
  uint32_t qi = 0xFFFFFFFFu;
  for (;;) {
    if (qb == 0 && threadIdx.x == 0) c->next_q = ld_volatile_int(&c->status) == 0 ? atomicAdd(P.queue, 1u) : P.nq;
    if (!grid_barrier(&c->bar, &gen, P.nb, P.max_spin, &c->status)) break;
    if (threadIdx.x == 0) sh_qi = __ldcg(&c->next_q);
    __syncthreads();
    qi = sh_qi;
    if (qi >= P.nq) break;
    if (threadIdx.x == 0) {
      const BatchQuery& bq = P.q[qi];
      sA.G = bq.G;
      sA.dist = W.idist;
      sA.out = bq.out;
      sA.fbits = W.fbits;
      sA.fwords = bq.G.ni / 32 + 2;
      sA.cursor = W.cursor;
      sA.q0 = W.q0;
      sA.q1 = W.q1;
      sA.sid = W.sid;
      sA.sd = W.sd;
      sA.scur = W.scur;
      sA.touched = W.touched;
      sA.sbits = W.sbits;
      sA.hist = W.hist;
      sA.ring = W.ring;
      sA.tasks = W.tasks;
      sA.step_ub = W.step_ub;
      sA.step_off = W.step_off;
      sA.trace = nullptr;
      sA.ctl = c;
      sA.status_out = &P.status[qi];
      sA.s = bq.s;
      sA.alpha = P.alpha;
      sA.beta = P.beta;
      sA.st_num = P.st_num;
      sA.gap_shift = bq.gap_shift;
      sA.heavy_min = bq.heavy_min;
      sA.max_spin = P.max_spin;
      sA.flags = P.flags;
      sA.ring_mask = bq.ring_mask;
      sA.ring_shift = bq.ring_shift;
      sA.task_cap = bq.task_cap;
      sA.step_cap = P.step_cap;
      sA.trace_cap = 0;
      sA.timeline = nullptr;
      sA.timeline_cap = 0;
      sA.nb = P.nb;
      sA.fuse = bq.fuse;
    }
    __syncthreads();
    if (!query_setup(sA, gen)) break;
    run_query<kPullFastGroup, kRelaxIlpGroup, 2>(sA, Q, gen);
    __syncthreads();
    if (ld_volatile_int(&c->status) != 0) break;
    query_output(sA);
  }
  // the query a group stopped in reports the group's status
  if (qb == 0 && threadIdx.x == 0 && qi < P.nq) {
    const int st = ld_volatile_int(&c->status);
    if (st != 0) P.status[qi] = st;
  }
}

// Starting state of every group's barrier and status, of the work queue and
// of the per-query statuses (EIC_EABORT until a group finishes the query).
__global__ void k_batch_prep(BatchArgs P, uint32_t groups) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < groups) {
    P.slot[g].ctl->bar.count = 0;
    P.slot[g].ctl->status = 0;
  }
  if (g < P.nq) P.status[g] = EIC_EABORT;
  if (g == 0) *P.queue = 0;
}

// ------------------------------------------------------------- serving kernel

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_sys_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_sys_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kNoTicket = ~0ull;      // the group leaves
constexpr unsigned long long kRetry = ~0ull - 1;      // nothing yet: the group waits again

// Continuous batching: the grid is cut into groups of nb blocks; each group's
// first thread claims the next admitted request from the ring, the group runs
// it with its own scratch, writes the result into the request's buffer and
// publishes the completion, then claims again. A first thread with nothing to
// claim waits at most poll_ns at a time (its group then passes its barrier
// and waits again, so no barrier wait comes near its bound). After idle_ns
// without work, once no group runs a request, a group registers as idle; when
// every group is registered they all leave together (the host relaunches the
// kernel when work arrives). They also leave when the host sets stop, and,
// in a launch with fewer groups than the server has, once widen_at admitted
// requests wait unclaimed (each after its current request; the host then
// relaunches with more groups). A group stops at its first failing request
// (whose completion carries the error) and counts as idle from then on.
__global__ void __launch_bounds__(kMaxBlock, 2) k_eic_serve(ServeArgs P) {
  __shared__ QueryShared Q;
  __shared__ KArgs sA;
  __shared__ unsigned long long sh_t;
  const uint32_t grp = blockIdx.x / P.nb, qb = blockIdx.x % P.nb;
  const BatchSlot& W = P.slot[grp];
  Ctl* c = W.ctl;
  unsigned long long* claim = &P.claim[0];
  unsigned long long* finished = &P.claim[1];
  unsigned long long* idle_groups = &P.claim[2];
  unsigned long long* leave = &P.claim[3];
  uint32_t gen = __ldcg(&c->bar.gen);
  unsigned long long mine = kNoTicket;  // first thread: the request it claimed last
  bool reported = true;                 // first thread: that request's completion is published
  bool registered = false;              // first thread: this group counts as idle
  for (;;) {
    if (qb == 0 && threadIdx.x == 0) {
      unsigned long long got = kRetry;
      if (ld_volatile_int(&c->status) != 0) got = kNoTicket;
      const unsigned long long t0 = globaltimer_ns();
      while (got == kRetry) {  // bounded: poll_ns per pass
        if (*(volatile uint32_t*)&P.ring->stop || atomicAdd(leave, 0ull) != 0) {
          got = kNoTicket;
          break;
        }
        const unsigned long long head = ld_acquire_sys_u64(&P.ring->head);
        const unsigned long long cur = atomicAdd(claim, 0ull);
        if (P.widen_at && cur < head && head - cur >= P.widen_at) {  // a backlog: make room for more groups
          atomicExch(leave, 1ull);
          got = kNoTicket;
          break;
        }
        if (cur < head) {
          if (atomicCAS(claim, cur, cur + 1) == cur) {
            got = cur;
            if (registered) {
              atomicAdd(idle_groups, ~0ull);  // minus one
              registered = false;
            }
          }
          continue;
        }
        const unsigned long long waited = globaltimer_ns() - t0;
        if (!registered && waited > P.idle_ns && atomicAdd(finished, 0ull) == cur) {
          atomicAdd(idle_groups, 1ull);
          registered = true;
        }
        if (registered && atomicAdd(idle_groups, 0ull) >= P.groups) {
          atomicExch(leave, 1ull);
          got = kNoTicket;
          break;
        }
        if (waited > P.poll_ns) break;  // kRetry
        __nanosleep(256);
      }
      c->next_ticket = got;
      if (got != kNoTicket && got != kRetry) {
        mine = got;
        reported = false;
      }
    }
    if (!grid_barrier(&c->bar, &gen, P.nb, P.max_spin, &c->status)) break;
    if (threadIdx.x == 0) sh_t = __ldcg(&c->next_ticket);
    __syncthreads();
    const unsigned long long t = sh_t;
    if (t == kNoTicket) break;
    if (t == kRetry) continue;
    const uint32_t e = (uint32_t)(t & (P.cap - 1));
    if (threadIdx.x == 0) {  // the entry was published before head (host release, leader acquire)
      const ServeRequest* rq = &P.req[e];
      const uint32_t gi = ld_relaxed_sys_u32(&rq->graph);
      const uint32_t src = ld_relaxed_sys_u32(&rq->source);
      uint32_t* out = (uint32_t*)ld_relaxed_sys_u64((const unsigned long long*)&rq->out);
      const BatchQuery& bq = P.graphs[gi < P.num_graphs ? gi : 0];  // the host admits valid ids only
      sA.G = bq.G;
      sA.dist = W.idist;
      sA.out = out;
      sA.fbits = W.fbits;
      sA.fwords = bq.G.ni / 32 + 2;
      sA.cursor = W.cursor;
      sA.q0 = W.q0;
      sA.q1 = W.q1;
      sA.sid = W.sid;
      sA.sd = W.sd;
      sA.scur = W.scur;
      sA.touched = W.touched;
      sA.sbits = W.sbits;
      sA.hist = W.hist;
      sA.ring = W.ring;
      sA.tasks = W.tasks;
      sA.step_ub = W.step_ub;
      sA.step_off = W.step_off;
      sA.trace = nullptr;
      sA.ctl = c;
      sA.status_out = nullptr;
      sA.s = src;
      sA.alpha = P.alpha;
      sA.beta = P.beta;
      sA.st_num = P.st_num;
      sA.gap_shift = bq.gap_shift;
      sA.heavy_min = bq.heavy_min;
      sA.max_spin = P.max_spin;
      sA.flags = P.flags;
      sA.ring_mask = bq.ring_mask;
      sA.ring_shift = bq.ring_shift;
      sA.task_cap = bq.task_cap;
      sA.step_cap = P.step_cap;
      sA.trace_cap = 0;
      sA.timeline = nullptr;
      sA.timeline_cap = 0;
      sA.nb = P.nb;
      sA.fuse = bq.fuse;
    }
    __syncthreads();
    if (!query_setup(sA, gen)) break;
    run_query<kPullFastGroup, kRelaxIlpGroup, 2>(sA, Q, gen);
    __syncthreads();
    if (ld_volatile_int(&c->status) != 0) break;
    query_output(sA);
    // every block's part of the result is written before the group reports
    if (!grid_barrier(&c->bar, &gen, P.nb, P.max_spin, &c->status)) break;
    if (qb == 0 && threadIdx.x == 0) {
      __threadfence_system();
      P.done[e].status = EIC_OK;
      st_release_sys_u64(&P.done[e].ticket_plus1, t + 1);
      atomicAdd(finished, 1ull);
      reported = true;
    }
  }
  if (qb == 0 && threadIdx.x == 0) {
    if (!reported) {  // a request the group claimed and stopped in reports the group's error
      const unsigned long long t = mine;
      const uint32_t e = (uint32_t)(t & (P.cap - 1));
      const int st = ld_volatile_int(&c->status);
      __threadfence_system();
      P.done[e].status = st != 0 ? st : EIC_ETIMEOUT;
      st_release_sys_u64(&P.done[e].ticket_plus1, t + 1);
      atomicAdd(finished, 1ull);
    }
    // a group that stopped early counts as idle, so the others can leave
    if (!registered && atomicAdd(leave, 0ull) == 0) atomicAdd(idle_groups, 1ull);
  }
}

// Starting state of every group's barrier and status, and of the idle vote.
__global__ void k_serve_prep(const BatchSlot* slot, uint32_t groups, unsigned long long* claim) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < groups) {
    slot[g].ctl->bar.count = 0;
    slot[g].ctl->status = 0;
  }
  if (g == 0) {
    claim[2] = 0;
    claim[3] = 0;
  }
}

}  // namespace

// ------------------------------------------------------------------ host

namespace {

constexpr uint32_t kStepCap = 1u << 20;     // steps per query
constexpr uint32_t kTraceCap = 1u << 16;    // trace rows kept on the device
constexpr uint32_t kTimelineCap = 1u << 16; // diagnostic timeline events
constexpr uint32_t kHeavyMinCeil = 4096;
constexpr uint32_t kDefaultHeavyMin = 32;
constexpr int kDefaultBlock = 512;
constexpr uint32_t kDefaultSpinLog2 = 22;
constexpr uint32_t kStNumMax = 1u << 16;  // Function 2's candidate bins fit the 2^20-slot ring of wide weights

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
  if (out->st_num == 0 || out->st_num > kStNumMax) return EIC_EINVAL;
  if (out->gap_shift > 16) return EIC_EINVAL;
  if (out->block_threads != 0 &&
      (out->block_threads % 32 != 0 || out->block_threads < 128 || out->block_threads > kMaxBlock))
    return EIC_EINVAL;
  if (out->heavy_min == 0) out->heavy_min = kDefaultHeavyMin;
  if (out->heavy_min < kHeavyMinFloor || out->heavy_min > kHeavyMinCeil) return EIC_EINVAL;
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

// The cooperative grid of the query kernel (k_eic, or k_eic_fused), cached
// per workspace for the block size last used.
int launch_shape(Workspace* ws, int block, bool fused) {
  int& grid = fused ? ws->grid_fused : ws->grid;
  int& cached = fused ? ws->block_fused : ws->block;
  if (grid && cached == block) return EIC_OK;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  EIC_CUDA_TRY(cudaGetDevice(&dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return EIC_ECUDA;
  EIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused ? k_eic_fused : k_eic, block, 0));
  if (per_sm < 1) return EIC_ECUDA;
  grid = sms * per_sm;
  cached = block;
  return EIC_OK;
}

// Fused rounds (bucket fusion) apply to graphs whose every degree is at most
// heavy_min, unless the caller turns them off.
bool use_fused(const eic_graph* g, const eic_params& p) { return fuse_ok(g->dg, p.heavy_min, p.flags); }

KArgs make_args(eic_graph* g, uint32_t s, uint32_t* dist, const eic_params& p, int* status_out, int grid) {
  Workspace& w = g->ws;
  KArgs A;
  A.G = g->dg;
  A.dist = w.idist;
  A.out = dist;
  A.fbits = w.fbits;
  A.fwords = (uint32_t)(g->dg.ni / 32 + 2);
  A.cursor = w.cursor;
  A.q0 = w.q[0];
  A.q1 = w.q[1];
  A.sid = w.sid;
  A.sd = w.sd;
  A.scur = w.scur;
  A.touched = w.touched;
  A.sbits = w.sbits;
  A.hist = w.hist;
  A.ring = w.ring;
  A.tasks = w.tasks;
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
  A.task_cap = w.task_cap;
  A.step_cap = w.step_cap;
  A.trace_cap = kTraceCap;
  A.timeline = nullptr;
  A.timeline_cap = 0;
  A.nb = (uint32_t)grid;
  A.fuse = 0;  // (the single-query kernels fix it: k_eic_fused or k_eic)
  return A;
}

// Enqueue one query: dist <- +inf, init, persistent kernel, optional parent.
int enqueue_query(eic_graph* g, uint32_t s, uint32_t* dist, uint32_t* parent, const eic_params& p, int* status_out,
                  cudaStream_t st, bool timeline = false, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr) {
  Workspace& w = g->ws;
  const int block = p.block_threads ? (int)p.block_threads : kDefaultBlock;
  const bool fused = use_fused(g, p);
  int rc = launch_shape(&w, block, fused);
  if (rc) return rc;
  const int grid = fused ? w.grid_fused : w.grid;
  EIC_CUDA_TRY(cudaMemsetAsync(w.idist, 0xFF, (uint64_t)g->dg.ni * 4, st));
  EIC_CUDA_TRY(cudaMemsetAsync(w.sbits, 0, ((uint64_t)g->dg.ni / 32 + 2) * 4, st));
  EIC_CUDA_TRY(cudaMemsetAsync(w.fbits, 0, 2 * ((uint64_t)g->dg.ni / 32 + 2) * 4, st));
  KArgs A = make_args(g, s, dist, p, status_out, grid);
  if (timeline) {
    A.timeline = w.timeline;
    A.timeline_cap = kTimelineCap;
  }
  k_init<<<64, 256, 0, st>>>(A);
  EIC_CUDA_TRY(cudaGetLastError());
  void* args[] = {&A};
  if (ev0) EIC_CUDA_TRY(cudaEventRecord(ev0, st));
  EIC_CUDA_TRY(cudaLaunchCooperativeKernel(fused ? (const void*)k_eic_fused : (const void*)k_eic, dim3(grid),
                                           dim3(block), args, 0, st));
  if (ev1) EIC_CUDA_TRY(cudaEventRecord(ev1, st));
  k_output<<<4 * grid, 256, 0, st>>>(g->dg, w.idist, s, dist);
  EIC_CUDA_TRY(cudaGetLastError());
  if (parent) {
    k_parent<<<1024, 256, 0, st>>>(g->dg, w.idist, s, parent);
    EIC_CUDA_TRY(cudaGetLastError());
  }
  return EIC_OK;
}

// A graph without edges: only the source is reachable (its own parent).
__global__ void k_trivial(uint32_t n, uint32_t s, uint32_t* dist, uint32_t* parent) {
  for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < n; u += (uint64_t)gridDim.x * blockDim.x) {
    dist[u] = u == s ? 0u : EIC_INF;
    if (parent) parent[u] = u == s ? s : EIC_INF;
  }
}

int trivial_query(eic_graph* g, uint32_t s, uint32_t* dist, uint32_t* parent, cudaStream_t st) {
  k_trivial<<<256, 256, 0, st>>>(g->dg.n, s, dist, parent);
  EIC_CUDA_TRY(cudaGetLastError());
  EIC_CUDA_TRY(cudaStreamSynchronize(st));
  return EIC_OK;
}

// The device's address of an output array of the graph's GPU: its device
// memory, managed memory, or page-locked host memory mapped for the device
// (written across the host link). Anything else is rejected before launch.
int output_view(int dev, uint32_t* p, uint32_t** out) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return EIC_EINVAL;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice:
      if (a.device != dev) return EIC_EINVAL;
      *out = p;
      return EIC_OK;
    case cudaMemoryTypeManaged:
      *out = p;
      return EIC_OK;
    case cudaMemoryTypeHost:
      if (!a.devicePointer) return EIC_EINVAL;
      *out = (uint32_t*)a.devicePointer;
      return EIC_OK;
    default:
      return EIC_EINVAL;
  }
}

}  // namespace

void eic_ws_free(Workspace* w) {
  cudaFree(w->idist);
  cudaFree(w->fbits);
  cudaFree(w->q[0]);
  cudaFree(w->q[1]);
  cudaFree(w->sid);
  cudaFree(w->sd);
  cudaFree(w->scur);
  cudaFree(w->cursor);
  cudaFree(w->touched);
  cudaFree(w->sbits);
  cudaFree(w->hist);
  cudaFree(w->ring);
  cudaFree(w->tasks);
  cudaFree(w->step_ub);
  cudaFree(w->step_off);
  cudaFree(w->trace);
  cudaFree(w->timeline);
  cudaFree(w->ctl);
  if (w->ctl_host) cudaFreeHost(w->ctl_host);
  if (w->ev[0]) cudaEventDestroy(w->ev[0]);
  if (w->ev[1]) cudaEventDestroy(w->ev[1]);
  *w = Workspace();
}

int eic_ws_ensure(eic_graph* g, int) {
  Workspace* w = &g->ws;
  if (w->ctl) return EIC_OK;
  const DevGraph& G = g->dg;
  const uint64_t n = G.ni;  // per-vertex arrays cover the internal (non-isolated) vertices
  int rc = EIC_OK;
  uint32_t maxw = G.maxw ? G.maxw : 1;
  uint32_t bits = 0;
  while (bits < 32 && (1ull << bits) <= maxw) ++bits;  // 2^bits > maxW
  w->ring_bits = bits < 20 ? bits : 20;
  w->ring_shift = bits > 20 ? bits - 20 : 0;  // nonzero: Function 2 sums exactly, the ring holds its bins
  // a window longer than heavy_min >= 16 yields ceil(len / 64) <= len / 16 tasks,
  // and the windows of one round belong to distinct vertices
  w->task_cap = (uint32_t)(G.two_m / kHeavyMinFloor + 2);
  w->step_cap = kStepCap;
  w->n = G.ni;
  if ((rc = walloc(w, &w->idist, n)) || (rc = walloc(w, &w->fbits, 2 * (n / 32 + 2))) || (rc = walloc(w, &w->q[0], n)) || (rc = walloc(w, &w->q[1], n)) ||
      (rc = walloc(w, &w->sid, n + 2)) || (rc = walloc(w, &w->sd, n + 2)) ||
      (rc = walloc(w, &w->scur, n + 2)) || (rc = walloc(w, &w->cursor, n)) || (rc = walloc(w, &w->touched, n + 1)) || (rc = walloc(w, &w->sbits, n / 32 + 2)) ||
      (rc = walloc(w, &w->hist, (uint64_t)G.D + 1)) || (rc = walloc(w, &w->ring, 1ull << w->ring_bits)) ||
      (rc = walloc(w, &w->tasks, w->task_cap)) || (rc = walloc(w, &w->step_ub, (uint64_t)kStepCap + 2)) ||
      (rc = walloc(w, &w->step_off, (uint64_t)kStepCap + 2)) || (rc = walloc(w, &w->trace, kTraceCap)) || (rc = walloc(w, &w->timeline, 2ull * kTimelineCap)) ||
      (rc = walloc(w, &w->ctl, 1))) {
    eic_ws_free(w);
    return rc;
  }
  if (cudaMallocHost((void**)&w->ctl_host, sizeof(Ctl)) != cudaSuccess) {
    (void)cudaGetLastError();
    eic_ws_free(w);
    return EIC_ENOMEM;
  }
  if (cudaMemset(w->ctl, 0, sizeof(Ctl)) != cudaSuccess) {
    (void)cudaGetLastError();
    eic_ws_free(w);
    return EIC_ECUDA;
  }
  return EIC_OK;
}

namespace {
constexpr int kMaxDevices = 64;
}  // namespace

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
  if ((rc = output_view(g->device, dist, &dist)) || (parent && (rc = output_view(g->device, parent, &parent))))
    return rc;
  eic_step* trace = stats ? stats->trace : nullptr;
  const uint64_t trace_cap = stats ? stats->trace_cap : 0;
  uint64_t* tl = stats ? stats->timeline : nullptr;
  const uint64_t tl_cap = stats ? stats->timeline_cap : 0;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->trace = trace;
    stats->trace_cap = trace_cap;
    stats->timeline = tl;
    stats->timeline_cap = tl_cap;
  }
  if (g->dg.two_m == 0) return trivial_query(g, source, dist, parent, st);
  if ((rc = eic_ws_ensure(g, 0))) return rc;
  Workspace& w = g->ws;
  if (stats && !w.ev[0]) {
    if (cudaEventCreate(&w.ev[0]) != cudaSuccess || cudaEventCreate(&w.ev[1]) != cudaSuccess) {
      (void)cudaGetLastError();
      return EIC_ECUDA;
    }
  }
  if ((rc = enqueue_query(g, source, dist, parent, p, nullptr, st, tl && tl_cap, stats ? w.ev[0] : nullptr,
                          stats ? w.ev[1] : nullptr))) {
    cudaStreamSynchronize(st);
    (void)cudaGetLastError();
    return rc;
  }
  EIC_CUDA_TRY(cudaMemcpyAsync(w.ctl_host, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  EIC_CUDA_TRY(cudaStreamSynchronize(st));
  const Ctl& h = *w.ctl_host;
  if (stats) {
    stats->steps = h.trace_len;
    stats->rounds = h.cnt_rounds;
    stats->frontier = h.cnt_frontier;
    stats->traversed = h.cnt_trav;
    stats->pulls = h.cnt_pulls;
    stats->improved = h.cnt_improved;
    stats->heavy = h.cnt_heavy;
    stats->pull_items = h.cnt_pitems;
    stats->trace_len = h.trace_len;
    float kms = 0.f;
    if (cudaEventElapsedTime(&kms, w.ev[0], w.ev[1]) == cudaSuccess) stats->kernel_ms = kms;
    (void)cudaGetLastError();
    if (trace && trace_cap) {
      uint64_t rows = h.trace_len < trace_cap ? h.trace_len : trace_cap;
      if (rows > kTraceCap) rows = kTraceCap;
      if (rows) EIC_CUDA_TRY(cudaMemcpy(trace, w.trace, rows * sizeof(eic_step), cudaMemcpyDeviceToHost));
    }
    if (tl && tl_cap) {
      uint64_t ev = h.tl_len < tl_cap ? h.tl_len : tl_cap;
      if (ev > kTimelineCap) ev = kTimelineCap;
      stats->timeline_len = h.tl_len;
      if (ev) EIC_CUDA_TRY(cudaMemcpy(tl, w.timeline, ev * 16, cudaMemcpyDeviceToHost));
    }
  }
  return h.status;
}

}  // extern "C"

// ------------------------------------------------------------ batch host side

namespace {

int batch_grid(int block, uint32_t* grid) {
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  EIC_CUDA_TRY(cudaGetDevice(&dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return EIC_ECUDA;
  EIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eic_batch, block, 0));
  if (per_sm < 1) return EIC_ECUDA;
  *grid = (uint32_t)(sms * per_sm);
  return EIC_OK;
}

SlotPool g_pool[kMaxDevices];  // scratch reused by eic_sssp_batch, per device
std::mutex g_pool_mu;

}  // namespace

// A prepared batch: the query table in claim order (largest graphs first),
// the trivial queries (graphs without edges), the launch configuration and,
// once run, the CUDA graph that replays it.
struct eic_batch {
  int device = 0;
  uint32_t nq = 0;
  eic_params p{};
  std::vector<uint32_t> order;  // claim position -> caller's query index
  std::vector<const eic_graph*> qgraph;  // claim position -> graph, source, output
  std::vector<uint32_t> qsource;
  std::vector<uint32_t*> qdist;
  std::vector<BatchQuery> hq;
  struct Trivial {
    uint32_t* dist;
    uint32_t n, s, index;
  };
  std::vector<Trivial> trivial;
  SlotCaps caps;
  uint32_t groups = 0, nb = 0, block = 0, grid_max = 0;
  SlotPool own;
  SlotPool* pool = &own;
  BatchQuery* d_q = nullptr;
  int* d_status = nullptr;
  int* h_status = nullptr;
  uint32_t* d_queue = nullptr;
  bool use_graph = true;
  cudaGraphExec_t exec = nullptr;
  double tuned_ms = 0.0;
};

namespace {

// Largest group count whose scratch fits in the share of free memory.
uint32_t groups_that_fit(eic_batch* b, uint32_t want) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    (void)cudaGetLastError();
    return want;
  }
  const uint64_t per = slot_layout(b->caps).bytes;
  const uint64_t held = b->pool->base ? (uint64_t)b->pool->count * b->pool->slot_bytes : 0;
  const uint64_t avail = (uint64_t)((double)(fr + held) * kBatchMemFrac);
  const uint64_t fit = per ? avail / per : want;
  return (uint32_t)(fit < want ? fit : want);
}

// groups -> blocks per group for the current block shape; nb_force (when
// nonzero) fixes the blocks per group instead, and the groups then fill at
// most the co-resident grid.
int batch_configure(eic_batch* b, uint32_t groups, uint32_t block, uint32_t nb_force = 0) {
  uint32_t gmax = 0;
  int rc = batch_grid((int)block, &gmax);
  if (rc) return rc;
  if (nb_force) {
    if (nb_force > gmax) nb_force = gmax;
    if (groups == 0 || groups > gmax / nb_force) groups = gmax / nb_force;
  }
  const uint32_t nrun = (uint32_t)b->hq.size();
  if (groups == 0) {  // library choice: about 8 blocks per group, more for graphs above 2^27 entries
    const uint64_t per = b->caps.two_m >> 24;
    const uint32_t nb = per < 8 ? 8 : (per > gmax ? gmax : (uint32_t)per);
    groups = gmax / nb;
  }
  if (groups > nrun) groups = nrun ? nrun : 1;
  if (groups > gmax) groups = gmax;
  groups = groups_that_fit(b, groups);
  if (groups == 0) return EIC_ENOMEM;
  if ((rc = b->pool->ensure(b->caps, groups))) return rc;
  if (b->exec && (b->groups != groups || b->block != block)) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->groups = groups;
  b->block = block;
  b->grid_max = gmax;
  b->nb = nb_force ? nb_force : gmax / groups;
  return EIC_OK;
}

// The host query table to the device (per-query parameters changed).
int batch_upload(eic_batch* b) {
  if (b->hq.empty()) return EIC_OK;
  EIC_CUDA_TRY(cudaMemcpy(b->d_q, b->hq.data(), b->hq.size() * sizeof(BatchQuery), cudaMemcpyHostToDevice));
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return EIC_OK;
}

BatchArgs batch_args(const eic_batch* b) {
  BatchArgs P;
  P.q = b->d_q;
  P.slot = b->pool->d_slots;
  P.status = b->d_status;
  P.queue = b->d_queue;
  P.nq = (uint32_t)b->hq.size();
  P.nb = b->nb;
  P.alpha = b->p.alpha;
  P.beta = b->p.beta;
  P.st_num = b->p.st_num;
  P.gap_shift = b->p.gap_shift;
  P.heavy_min = b->p.heavy_min;
  P.flags = b->p.flags;
  P.step_cap = kBatchStepCap;
  P.max_spin = 1ull << b->p.max_spin_log2;
  return P;
}

int batch_enqueue(eic_batch* b, cudaStream_t st) {
  if (!b->hq.empty()) {
    BatchArgs P = batch_args(b);
    const uint32_t nrun = P.nq, cover = b->groups > nrun ? b->groups : nrun;
    k_batch_prep<<<(cover + 255) / 256, 256, 0, st>>>(P, b->groups);
    EIC_CUDA_TRY(cudaGetLastError());
    void* args[] = {&P};
    EIC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_eic_batch, dim3(b->groups * b->nb), dim3(b->block), args,
                                             0, st));
  }
  for (const auto& t : b->trivial) {  // no edges: only the source is reachable
    EIC_CUDA_TRY(cudaMemsetAsync(t.dist, 0xFF, (uint64_t)t.n * 4, st));
    EIC_CUDA_TRY(cudaMemsetAsync(t.dist + t.s, 0, 4, st));
  }
  return EIC_OK;
}

void batch_free(eic_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->own.release();
  cudaFree(b->d_q);
  cudaFree(b->d_status);
  cudaFree(b->d_queue);
  if (b->h_status) cudaFreeHost(b->h_status);
  delete b;
}

int batch_create(const eic_graph* const* graphs, const uint32_t* sources, uint32_t nq, uint32_t* const* dists,
                 const eic_params* params, SlotPool* shared_pool, eic_batch** out) {
  *out = nullptr;
  if (nq == 0 || !graphs || !sources || !dists) return EIC_EINVAL;
  eic_params p;
  int rc = resolve_params(params, &p);
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return EIC_ECUDA;
  }
  for (uint32_t i = 0; i < nq; ++i)
    if (!graphs[i] || !dists[i] || sources[i] >= graphs[i]->dg.n || graphs[i]->device != dev) return EIC_EINVAL;
  eic_batch* b = new eic_batch();
  b->device = dev;
  b->nq = nq;
  b->p = p;
  if (shared_pool) b->pool = shared_pool;
  std::vector<uint32_t> idx;
  for (uint32_t i = 0; i < nq; ++i) {
    const DevGraph& G = graphs[i]->dg;
    if (G.two_m == 0) {
      b->trivial.push_back({dists[i], G.n, sources[i], i});
      continue;
    }
    idx.push_back(i);
  }
  // largest graphs are claimed first (longest-processing-time order)
  std::stable_sort(idx.begin(), idx.end(),
                   [&](uint32_t a, uint32_t c) { return graphs[a]->dg.two_m > graphs[c]->dg.two_m; });
  for (uint32_t i : idx) {
    const DevGraph& G = graphs[i]->dg;
    BatchQuery q;
    q.G = G;
    q.out = dists[i];
    q.s = sources[i];
    uint32_t shift = 0;
    const uint32_t bits = ring_layout(G.maxw, &shift);
    q.ring_mask = (1u << bits) - 1u;
    q.ring_shift = shift;
    q.task_cap = (uint32_t)(G.two_m / kHeavyMinFloor + 2);
    q.gap_shift = p.gap_shift;
    q.heavy_min = p.heavy_min;
    q.fuse = fuse_ok(G, p.heavy_min, p.flags) ? 1u : 0u;
    b->hq.push_back(q);
    b->order.push_back(i);
    b->qgraph.push_back(graphs[i]);
    b->qsource.push_back(sources[i]);
    b->qdist.push_back(dists[i]);
    SlotCaps& c = b->caps;
    c.ni = G.ni > c.ni ? G.ni : c.ni;
    c.two_m = G.two_m > c.two_m ? G.two_m : c.two_m;
    c.D = G.D > c.D ? G.D : c.D;
    c.ring_bits = bits > c.ring_bits ? bits : c.ring_bits;
  }
  const uint64_t nrun = b->hq.size();
  if (nrun) {
    if (cudaMalloc((void**)&b->d_q, nrun * sizeof(BatchQuery)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_status, nrun * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_queue, sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_status, nrun * sizeof(int)) != cudaSuccess) {
      (void)cudaGetLastError();
      batch_free(b);
      return EIC_ENOMEM;
    }
    if (cudaMemcpy(b->d_q, b->hq.data(), nrun * sizeof(BatchQuery), cudaMemcpyHostToDevice) != cudaSuccess) {
      (void)cudaGetLastError();
      batch_free(b);
      return EIC_ECUDA;
    }
    const uint32_t block = p.block_threads ? p.block_threads : (uint32_t)kDefaultBlock;
    if ((rc = batch_configure(b, p.batch_groups, block))) {
      batch_free(b);
      return rc;
    }
  }
  *out = b;
  return EIC_OK;
}

int batch_run(eic_batch* b, cudaStream_t st) {
  if (b->use_graph && !b->exec) {  // capture the launch sequence once, replay it afterwards
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const int rc = batch_enqueue(b, cs);
      ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && rc == EIC_OK && graph &&
           cudaGraphInstantiate(&b->exec, graph, 0) == cudaSuccess;
    }
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    if (!ok) {  // capture unavailable: launch directly from now on
      (void)cudaGetLastError();
      b->exec = nullptr;
      b->use_graph = false;
    }
  }
  if (b->exec) {
    EIC_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    return EIC_OK;
  }
  return batch_enqueue(b, st);
}

int batch_wait(eic_batch* b, cudaStream_t st, int* statuses) {
  const uint64_t nrun = b->hq.size();
  if (nrun) EIC_CUDA_TRY(cudaMemcpyAsync(b->h_status, b->d_status, nrun * sizeof(int), cudaMemcpyDeviceToHost, st));
  EIC_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int> all(b->nq, EIC_OK);
  for (uint64_t k = 0; k < nrun; ++k) all[b->order[k]] = b->h_status[k];
  int first = EIC_OK;
  for (uint32_t i = 0; i < b->nq; ++i) {
    if (statuses) statuses[i] = all[i];
    if (first == EIC_OK) first = all[i];
  }
  return first;
}

// Device time of one whole batch run (ms), or a negative value on error.
double batch_time(eic_batch* b, cudaStream_t st) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    (void)cudaGetLastError();
    return -1.0;
  }
  double ms = -1.0;
  float t = 0.f;
  if (cudaEventRecord(e0, st) == cudaSuccess && batch_enqueue(b, st) == EIC_OK &&
      cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
      cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && batch_wait(b, st, nullptr) == EIC_OK)
    ms = t;
  (void)cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

}  // namespace

extern "C" {

int eic_sssp_batch(const eic_graph* const* graphs, const uint32_t* sources, uint32_t num_queries,
                   uint32_t* const* dists, const eic_params* params, int* statuses, void* stream) {
  if (num_queries == 0) return EIC_OK;
  if (!graphs || !sources || !dists) return EIC_EINVAL;
  if (!graphs[0]) return EIC_EINVAL;
  DeviceGuard guard(graphs[0]->device);
  if (!guard.ok || graphs[0]->device < 0 || graphs[0]->device >= kMaxDevices) return EIC_ECUDA;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  eic_batch* b = nullptr;
  int rc = batch_create(graphs, sources, num_queries, dists, params, &g_pool[graphs[0]->device], &b);
  if (rc) {
    if (statuses)
      for (uint32_t i = 0; i < num_queries; ++i) statuses[i] = rc;
    return rc;
  }
  b->use_graph = false;  // one-shot: launch directly
  cudaStream_t st = (cudaStream_t)stream;
  rc = batch_enqueue(b, st);
  if (rc == EIC_OK) {
    rc = batch_wait(b, st, statuses);
  } else {
    cudaStreamSynchronize(st);
    (void)cudaGetLastError();
    if (statuses)
      for (uint32_t i = 0; i < num_queries; ++i) statuses[i] = rc;
  }
  batch_free(b);
  return rc;
}

int eic_batch_create(const eic_graph* const* graphs, const uint32_t* sources, uint32_t num_queries,
                     uint32_t* const* dists, const eic_params* params, eic_batch** out) {
  if (!out) return EIC_EINVAL;
  *out = nullptr;
  if (!graphs || !graphs[0]) return EIC_EINVAL;
  DeviceGuard guard(graphs[0]->device);
  if (!guard.ok) return EIC_ECUDA;
  return batch_create(graphs, sources, num_queries, dists, params, nullptr, out);
}

int eic_batch_run(eic_batch* b, void* stream) {
  if (!b) return EIC_EINVAL;
  DeviceGuard guard(b->device);
  if (!guard.ok) return EIC_ECUDA;
  return batch_run(b, (cudaStream_t)stream);
}

int eic_batch_wait(eic_batch* b, void* stream, int* statuses) {
  if (!b) return EIC_EINVAL;
  DeviceGuard guard(b->device);
  if (!guard.ok) return EIC_ECUDA;
  return batch_wait(b, (cudaStream_t)stream, statuses);
}

int eic_batch_tune(eic_batch* b, void* stream, eic_batch_config* best) {
  if (!b) return EIC_EINVAL;
  DeviceGuard guard(b->device);
  if (!guard.ok) return EIC_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  if (!b->hq.empty()) {
    const uint32_t nrun = (uint32_t)b->hq.size();
    int rc = EIC_OK;
    uint32_t best_g = b->groups, best_block = b->block, best_hm = b->p.heavy_min;
    double best_ms = 1e300;
    // one configuration: a warm-up run, then a timed one when the warm-up was
    // within 2x of the best so far
    auto trial = [&](uint32_t g, uint32_t block, uint32_t hm, double* ms_out) -> int {
      for (auto& q : b->hq) {
        q.heavy_min = hm;
        q.fuse = fuse_ok(q.G, hm, b->p.flags) ? 1u : 0u;
      }
      b->p.heavy_min = hm;
      int r = batch_upload(b);
      if (r) return r;
      if ((r = batch_configure(b, g, block))) return r;
      double ms = batch_time(b, st);
      if (ms < 0) return EIC_ECUDA;
      if (ms < 2.0 * best_ms) {
        const double ms2 = batch_time(b, st);
        if (ms2 < 0) return EIC_ECUDA;
        ms = ms2 < ms ? ms2 : ms;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best_g = b->groups;
        best_block = b->block;
        best_hm = hm;
      }
      if (ms_out) *ms_out = ms;
      return EIC_OK;
    };
    uint32_t gmax = 0;
    if ((rc = batch_grid((int)b->block, &gmax))) return rc;
    // pass 1: group counts (divisors of the grid and powers of two), from the
    // most groups down, until two in a row are 20% slower than the best
    std::vector<uint32_t> cand;
    for (uint32_t g = gmax; g >= 1; --g)
      if (g <= nrun && (gmax % g == 0 || (g & (g - 1)) == 0)) cand.push_back(g);
    uint32_t worse = 0;
    for (uint32_t g : cand) {
      double ms = 0;
      if ((rc = trial(g, b->block, best_hm, &ms))) return rc;
      worse = ms > 1.2 * best_ms ? worse + 1 : 0;
      if (worse >= 2) break;
    }
    // pass 2: each graph's step-width scaling (exact for every value), timed on
    // a sub-batch of that graph's queries at the chosen blocks per group:
    // gap_shift + 1, + 2, ... while it helps by 2% (up to 8)
    if ((rc = batch_configure(b, best_g, best_block))) return rc;
    const uint32_t nb = b->nb;
    std::vector<const eic_graph*> seen;
    for (uint32_t k = 0; k < nrun; ++k) {
      const eic_graph* g = b->qgraph[k];
      if (std::find(seen.begin(), seen.end(), g) != seen.end()) continue;
      seen.push_back(g);
      std::vector<uint32_t> pos;
      for (uint32_t j = 0; j < nrun; ++j)
        if (b->qgraph[j] == g) pos.push_back(j);
      std::vector<const eic_graph*> sg(pos.size(), g);
      std::vector<uint32_t> ss;
      std::vector<uint32_t*> sd;
      for (uint32_t j : pos) {
        ss.push_back(b->qsource[j]);
        sd.push_back(b->qdist[j]);
      }
      eic_batch* sub = nullptr;
      if ((rc = batch_create(sg.data(), ss.data(), (uint32_t)pos.size(), sd.data(), &b->p, nullptr, &sub)))
        return rc;
      rc = batch_configure(sub, (uint32_t)pos.size(), best_block, nb);
      uint32_t gs_best = b->hq[k].gap_shift;
      double t_best = -1.0;
      for (uint32_t gs = gs_best; rc == EIC_OK && gs <= 8; ++gs) {
        for (auto& q : sub->hq) q.gap_shift = gs;
        if ((rc = batch_upload(sub))) break;
        double t = batch_time(sub, st);
        const double t2 = batch_time(sub, st);
        if (t < 0 || t2 < 0) {
          rc = EIC_ECUDA;
          break;
        }
        t = t2 < t ? t2 : t;
        if (t_best < 0 || t < 0.98 * t_best) {
          t_best = t;
          gs_best = gs;
        } else {
          break;
        }
      }
      batch_free(sub);
      if (rc) return rc;
      for (uint32_t j : pos) b->hq[j].gap_shift = gs_best;
    }
    best_ms = 1e300;
    if ((rc = trial(best_g, best_block, best_hm, nullptr))) return rc;
    // pass 3 at the best group count: the window-class threshold, then a
    // 256-thread block
    const uint32_t hm0 = best_hm;
    for (uint32_t hm : {64u, 256u})
      if ((rc = trial(best_g, best_block, hm, nullptr))) return rc;
    if ((rc = trial(best_g, 256, best_hm, nullptr))) return rc;
    (void)hm0;
    // keep the winner; the scratch shrinks to its group count
    for (auto& q : b->hq) {
      q.heavy_min = best_hm;
      q.fuse = fuse_ok(q.G, best_hm, b->p.flags) ? 1u : 0u;
    }
    b->p.heavy_min = best_hm;
    if ((rc = batch_upload(b))) return rc;
    if (b->pool == &b->own && b->own.count > best_g) b->own.release();
    if ((rc = batch_configure(b, best_g, best_block))) return rc;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    b->tuned_ms = best_ms;
  }
  return best ? eic_batch_info(b, best) : EIC_OK;
}

int eic_batch_info(const eic_batch* b, eic_batch_config* out) {
  if (!b || !out) return EIC_EINVAL;
  memset(out, 0, sizeof(*out));
  out->groups = b->groups;
  out->blocks_per_group = b->nb;
  out->block_threads = b->block;
  out->cuda_graph = b->exec ? 1u : 0u;
  out->gap_shift = b->p.gap_shift;
  for (const auto& q : b->hq) out->gap_shift = q.gap_shift > out->gap_shift ? q.gap_shift : out->gap_shift;
  out->heavy_min = b->p.heavy_min;
  out->queries = b->nq;
  out->scratch_bytes = (uint64_t)b->pool->count * b->pool->slot_bytes;
  out->tuned_ms = b->tuned_ms;
  return EIC_OK;
}

int eic_batch_gap_shifts(const eic_batch* b, uint32_t* gap_shifts) {
  if (!b || !gap_shifts) return EIC_EINVAL;
  for (uint32_t i = 0; i < b->nq; ++i) gap_shifts[i] = b->p.gap_shift;  // graphs without edges keep the batch's
  for (size_t k = 0; k < b->hq.size(); ++k) gap_shifts[b->order[k]] = b->hq[k].gap_shift;
  return EIC_OK;
}

int eic_batch_destroy(eic_batch* b) {
  if (!b) return EIC_OK;
  DeviceGuard guard(b->device);
  batch_free(b);
  return EIC_OK;
}

}  // extern "C"


// ------------------------------------------------ allocation-free entry point
//
// The query scratch of eic_sssp_noalloc: one file-scope device array carved
// into the workspace arrays of a graph with at most kNaN vertices, kNaE
// adjacency entries, weights below 2^16 and kNaD distinct degrees. Every GPU
// that loads the library holds it until the process exits.
namespace {

constexpr uint64_t kNaN = EIC_NOALLOC_MAX_VERTICES;
constexpr uint64_t kNaE = EIC_NOALLOC_MAX_ENTRIES;
constexpr uint64_t kNaD = EIC_NOALLOC_MAX_DEGREES;
constexpr uint64_t kNaS = EIC_NOALLOC_MAX_STEPS;
constexpr uint32_t kNaRingBits = 16;  // 2^16 > EIC_NOALLOC_MAX_WEIGHT
constexpr uint64_t kNaTasks = kNaE / kHeavyMinFloor + 2;

constexpr uint64_t na_align(uint64_t x) { return (x + 255) & ~255ull; }
constexpr uint64_t kNaIdist = 0;
constexpr uint64_t kNaFbits = kNaIdist + na_align(kNaN * 4);
constexpr uint64_t kNaCursor = kNaFbits + na_align(2 * (kNaN / 32 + 2) * 4);
constexpr uint64_t kNaQ0 = kNaCursor + na_align(kNaN * 4);
constexpr uint64_t kNaQ1 = kNaQ0 + na_align(kNaN * 4);
constexpr uint64_t kNaSid = kNaQ1 + na_align(kNaN * 4);
constexpr uint64_t kNaSd = kNaSid + na_align((kNaN + 2) * 4);
constexpr uint64_t kNaScur = kNaSd + na_align((kNaN + 2) * 4);
constexpr uint64_t kNaTouched = kNaScur + na_align((kNaN + 2) * 4);
constexpr uint64_t kNaSbits = kNaTouched + na_align((kNaN + 1) * 4);
constexpr uint64_t kNaHist = kNaSbits + na_align((kNaN / 32 + 2) * 4);
constexpr uint64_t kNaRing = kNaHist + na_align(kNaD * 4);
constexpr uint64_t kNaTaskOff = kNaRing + na_align((1ull << kNaRingBits) * 8);
constexpr uint64_t kNaStepUb = kNaTaskOff + na_align(kNaTasks * sizeof(Task));
constexpr uint64_t kNaStepOff = kNaStepUb + na_align((kNaS + 2) * 8);
constexpr uint64_t kNaCtl = kNaStepOff + na_align((kNaS + 2) * 4);
constexpr uint64_t kNaBytes = kNaCtl + na_align(sizeof(Ctl));
static_assert(kNaBytes > 13000000 && kNaBytes < 14000000, "the header states the scratch size as about 13.4 MB");

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

struct NaDevice {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_na_scratch on this device
  int grid = 0;
};
NaDevice g_na[kMaxDevices];
std::mutex g_na_mu;

// Once per device, with that device current: the scratch's device address
// (the symbol's host-side name is not a device pointer), a cleared control
// block, and the cooperative grid shape.
int na_setup(NaDevice& d, cudaStream_t st) {
  void* ptr = nullptr;
  EIC_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_na_scratch));
  if (!ptr) return EIC_ECUDA;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  EIC_CUDA_TRY(cudaGetDevice(&dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return EIC_ECUDA;
  EIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eic, kDefaultBlock, 0));
  if (per_sm < 1) return EIC_ECUDA;
  unsigned char* base = (unsigned char*)ptr;
  EIC_CUDA_TRY(cudaMemsetAsync(base + kNaCtl, 0, sizeof(Ctl), st));
  EIC_CUDA_TRY(cudaStreamSynchronize(st));
  d.base = base;
  d.grid = sms * per_sm;
  d.ready = true;
  return EIC_OK;
}

}  // namespace

extern "C" int eic_sssp_noalloc(const eic_graph* gc, uint32_t source, uint32_t* dist, void* stream) {
  if (!gc || !dist) return EIC_EINVAL;
  const DevGraph& G = gc->dg;
  if (source >= G.n) return EIC_EINVAL;
  if (G.n > kNaN || G.two_m > kNaE || G.maxw > EIC_NOALLOC_MAX_WEIGHT || G.D > kNaD) return EIC_ESIZE;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_na_mu);
  DeviceGuard guard(gc->device);
  if (!guard.ok || gc->device < 0 || gc->device >= kMaxDevices) return EIC_ECUDA;
  NaDevice& nd = g_na[gc->device];
  int rc;
  if (!nd.ready && (rc = na_setup(nd, st))) return rc;
  if (G.two_m == 0) {  // no edges: only the source is reachable
    EIC_CUDA_TRY(cudaMemsetAsync(dist, 0xFF, (uint64_t)G.n * 4, st));
    EIC_CUDA_TRY(cudaMemsetAsync(dist + source, 0, 4, st));
    EIC_CUDA_TRY(cudaStreamSynchronize(st));
    return EIC_OK;
  }
  unsigned char* b = nd.base;
  Ctl* ctl = (Ctl*)(b + kNaCtl);
  KArgs A;
  A.G = G;
  A.dist = (uint32_t*)(b + kNaIdist);
  A.out = dist;
  A.fbits = (uint32_t*)(b + kNaFbits);
  A.fwords = (uint32_t)(G.ni / 32 + 2);
  A.cursor = (uint32_t*)(b + kNaCursor);
  A.q0 = (uint32_t*)(b + kNaQ0);
  A.q1 = (uint32_t*)(b + kNaQ1);
  A.sid = (uint32_t*)(b + kNaSid);
  A.sd = (uint32_t*)(b + kNaSd);
  A.scur = (uint32_t*)(b + kNaScur);
  A.touched = (uint32_t*)(b + kNaTouched);
  A.sbits = (uint32_t*)(b + kNaSbits);
  A.hist = (uint32_t*)(b + kNaHist);
  A.ring = (unsigned long long*)(b + kNaRing);
  A.tasks = (Task*)(b + kNaTaskOff);
  A.step_ub = (int64_t*)(b + kNaStepUb);
  A.step_off = (uint32_t*)(b + kNaStepOff);
  A.trace = nullptr;
  A.ctl = ctl;
  A.status_out = nullptr;
  A.s = source;
  A.alpha = 3;
  A.beta = 0.9;
  A.st_num = 1024;
  A.gap_shift = 0;
  A.heavy_min = kDefaultHeavyMin;
  A.max_spin = 1ull << kDefaultSpinLog2;
  A.flags = 0;
  A.ring_mask = (1u << kNaRingBits) - 1u;
  A.ring_shift = 0;
  A.task_cap = (uint32_t)kNaTasks;
  A.step_cap = (uint32_t)kNaS;
  A.trace_cap = 0;
  A.timeline = nullptr;
  A.timeline_cap = 0;
  A.nb = (uint32_t)nd.grid;
  A.fuse = 0;
  // Once anything is enqueued, every return waits for the stream first: the
  // next call may reuse the scratch only when this call's work has finished.
  auto enqueue = [&]() -> int {
    EIC_CUDA_TRY(cudaMemsetAsync(A.dist, 0xFF, (uint64_t)G.ni * 4, st));
    EIC_CUDA_TRY(cudaMemsetAsync(A.sbits, 0, ((uint64_t)G.ni / 32 + 2) * 4, st));
    EIC_CUDA_TRY(cudaMemsetAsync(A.fbits, 0, 2 * ((uint64_t)G.ni / 32 + 2) * 4, st));
    k_init<<<64, 256, 0, st>>>(A);
    EIC_CUDA_TRY(cudaGetLastError());
    void* args[] = {&A};
    EIC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_eic, dim3(nd.grid), dim3(kDefaultBlock), args, 0, st));
    k_output<<<4 * nd.grid, 256, 0, st>>>(G, A.dist, source, dist);
    EIC_CUDA_TRY(cudaGetLastError());
    return EIC_OK;
  };
  int status = 0;
  rc = enqueue();
  if (rc == EIC_OK && cudaMemcpyAsync(&status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = EIC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == EIC_OK) rc = EIC_ECUDA;
  (void)cudaGetLastError();
  if (rc) return rc;
  return status;
}

// ------------------------------------------------------------ serving launch

int eic_serve_grid(int block, uint32_t* grid) {
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  EIC_CUDA_TRY(cudaGetDevice(&dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  EIC_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return EIC_ECUDA;
  EIC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eic_serve, block, 0));
  if (per_sm < 1) return EIC_ECUDA;
  *grid = (uint32_t)(sms * per_sm);
  return EIC_OK;
}

int eic_serve_launch(const ServeArgs& args, uint32_t groups, uint32_t block, cudaStream_t stream) {
  k_serve_prep<<<(groups + 255) / 256, 256, 0, stream>>>(args.slot, groups, args.claim);
  EIC_CUDA_TRY(cudaGetLastError());
  ServeArgs a = args;
  void* kargs[] = {&a};
  EIC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_eic_serve, dim3(groups * args.nb), dim3(block), kargs, 0,
                                           stream));
  return EIC_OK;
}

int eic_tune_step_width(const eic_graph* g, uint32_t source, uint32_t copies, uint32_t nb, const eic_params& p,
                        uint32_t from, cudaStream_t stream, uint32_t* best_shift, double* best_ms) {
  if (!g || copies == 0 || source >= g->dg.n) return EIC_EINVAL;
  *best_shift = from;
  *best_ms = 0.0;
  if (g->dg.two_m == 0) return EIC_OK;
  uint32_t* buf = nullptr;
  const uint64_t n = g->dg.n;
  if (cudaMalloc((void**)&buf, n * 4 * copies) != cudaSuccess) {
    (void)cudaGetLastError();
    return EIC_ENOMEM;
  }
  std::vector<const eic_graph*> gs(copies, g);
  std::vector<uint32_t> ss(copies, source);
  std::vector<uint32_t*> ds;
  for (uint32_t k = 0; k < copies; ++k) ds.push_back(buf + n * k);
  eic_batch* b = nullptr;
  int rc = batch_create(gs.data(), ss.data(), copies, ds.data(), &p, nullptr, &b);
  if (rc == EIC_OK) rc = batch_configure(b, copies, p.block_threads ? p.block_threads : kDefaultBlock, nb);
  double t_best = -1.0;
  for (uint32_t shift = from; rc == EIC_OK && shift <= 8; ++shift) {
    for (auto& q : b->hq) q.gap_shift = shift;
    if ((rc = batch_upload(b))) break;
    double t = batch_time(b, stream);
    const double t2 = batch_time(b, stream);
    if (t < 0 || t2 < 0) {
      rc = EIC_ECUDA;
      break;
    }
    t = t2 < t ? t2 : t;
    if (t_best < 0 || t < 0.98 * t_best) {
      t_best = t;
      *best_shift = shift;
    } else {
      break;
    }
  }
  if (b) batch_free(b);
  cudaFree(buf);
  *best_ms = t_best;
  return rc;
}

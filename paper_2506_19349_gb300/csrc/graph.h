// Host-side definitions of the graph object and the query workspace.
#pragma once

#include <mutex>

#include "common.cuh"

// Smallest accepted heavy_min: a window longer than it yields at most len / 16
// tasks, which bounds every task list at 2m / 16 entries.
constexpr uint32_t kHeavyMinFloor = 16;

// A window of at most kTaskLen adjacency entries relaxed by one warp in a
// round's task phase.
struct Task {
  uint32_t beg;  // first adjacency index
  uint32_t len;  // entries, <= 64
  uint32_t u;    // the vertex whose row is read
  uint32_t d;    // its distance (push); 0xFFFFFFFF marks a pull request
};

// Control block shared by the blocks of the persistent kernel.
struct Ctl {
  // published by the step-boundary block, read by every block after a barrier
  int64_t lb, ub, st, lb0;
  uint32_t step, done;
  uint32_t s_int;  // internal id of the source (0xFFFFFFFF: isolated source)
  uint32_t push_beg, push_end;  // settled-list range pushed in the step's first round
  uint32_t pull_on, pull_cnt, extra_s;
  uint32_t pull_sweep;  // the pull set is swept in vertex order (pull_cnt = all vertices; the round takes the unsettled ones)
  uint32_t step_off_cur;  // settled-list offset where the current step's vertices start
  // private to the step-boundary block
  int64_t st0, st1, gap_lb;
  uint64_t sumd_lb, highd_lb;
  int64_t max_settled;
  uint32_t rounds_in_step;
  uint32_t trace_len;
  uint32_t tl_len;  // diagnostic timeline events recorded
  // appended with atomics during phases
  uint32_t qcnt[3];
  uint32_t work[3];  // dynamic chunk counters, by round id mod 3
  uint32_t settled_cnt;
  uint32_t touched_cnt;
  uint32_t ub_cand;
  uint32_t tcnt[3];  // tasks of the round, by round id mod 3
  uint32_t s2_done;
  uint32_t next_q;  // batch: the query the group's first block claimed
  unsigned long long next_ticket;  // serving: the request the group's first block claimed
  uint32_t acc_maxd1;  // 1 + the largest distance settled in the step (0: none)
  unsigned long long acc_deg;
  unsigned long long cnt_rounds, cnt_frontier, cnt_trav, cnt_pulls, cnt_improved, cnt_heavy, cnt_pitems;
  GridBarrier bar;
  int status;
};

// One query of a batch: graph, caller's output buffer, source, and the
// graph-dependent layout of the statistics ring and task list.
struct BatchQuery {
  DevGraph G;
  uint32_t* out;
  uint32_t s;
  uint32_t ring_mask, ring_shift, task_cap;
  uint32_t gap_shift, heavy_min;  // step-width scaling and window-class threshold for this query's graph
  uint32_t fuse;                  // 1: fused rounds (every degree of the graph <= heavy_min)
};

// Fused rounds (bucket fusion) apply to a graph whose every degree is at most
// heavy_min (no window becomes a grid task), unless the caller turns them off.
inline bool fuse_ok(const DevGraph& G, uint32_t heavy_min, uint32_t flags) {
  return G.max_deg <= heavy_min && !(flags & EIC_FLAG_NO_FUSE);
}

// Scratch of one block group, reused by every query the group runs.
struct BatchSlot {
  uint32_t* idist;
  uint32_t* fbits;
  uint32_t* cursor;
  uint32_t* q0;
  uint32_t* q1;
  uint32_t* sid;
  uint32_t* sd;
  uint32_t* scur;
  uint32_t* touched;
  uint32_t* sbits;
  uint32_t* hist;
  unsigned long long* ring;
  Task* tasks;
  int64_t* step_ub;
  uint32_t* step_off;
  Ctl* ctl;
};

struct Workspace {
  uint32_t n = 0;
  uint32_t* idist = nullptr;  // distances in internal ids
  uint32_t* fbits = nullptr;  // two frontier-insertion bitmaps
  uint32_t* q[2] = {nullptr, nullptr};
  uint32_t* sid = nullptr;   // settled list: vertex
  uint32_t* sd = nullptr;    // settled list: final distance
  uint32_t* scur = nullptr;  // settled list: window cursor (offset in the row)
  uint32_t* cursor = nullptr;
  uint32_t* touched = nullptr;
  uint32_t* sbits = nullptr;  // settled bitmap
  uint32_t* hist = nullptr;
  unsigned long long* ring = nullptr;
  Task* tasks = nullptr;
  int64_t* step_ub = nullptr;
  uint32_t* step_off = nullptr;
  eic_step* trace = nullptr;
  unsigned long long* timeline = nullptr;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;  // pinned mirror for status readback
  cudaEvent_t ev[2] = {nullptr, nullptr};  // around the query kernel, when statistics are asked for
  uint32_t ring_bits = 0, ring_shift = 0;
  uint32_t task_cap = 0, step_cap = 0;
  uint64_t bytes = 0;
  int grid = 0, block = 0;  // cached cooperative launch shape of k_eic
  int grid_fused = 0, block_fused = 0;  // and of k_eic_fused
};

struct eic_graph {
  int device = 0;
  DevGraph dg{};
  uint32_t* row = nullptr;
  uint2* adj = nullptr;
  uint32_t* drank = nullptr;
  uint32_t* dvals = nullptr;
  uint32_t* dcnt0 = nullptr;
  uint32_t* dfirst = nullptr;
  uint2* dhint = nullptr;
  uint32_t* rtow = nullptr;
  uint4* nz = nullptr;
  uint32_t* nz_lt = nullptr;
  uint32_t* orig2int = nullptr;
  uint32_t* int2orig = nullptr;
  uint64_t bytes = 0;
  Workspace ws;
  std::mutex mu;
};

int eic_ws_ensure(eic_graph* g, int block_threads);
void eic_ws_free(Workspace* ws);

// Host-side definitions of the graph object and the query workspace.
#pragma once

#include <mutex>

#include "common.cuh"

struct HeavyItem {
  uint64_t beg;     // first adjacency index of the window
  uint64_t prefix;  // entries of all earlier heavy items in this round
  uint32_t u;       // vertex whose row is read
  uint32_t d;       // its distance (push) or current distance (pull)
  uint32_t mode;    // 0 push, 2 pull
  uint32_t pad;
};

// Control block shared by the blocks of the persistent kernel.
struct Ctl {
  // published by the step-boundary block, read by every block after a barrier
  int64_t lb, ub, st, lb0;
  uint32_t step, done;
  uint32_t push_beg, push_end;  // settled-list range pushed in round 1
  uint32_t pull_on, pull_src, pull_cnt, extra_s;
  uint32_t step_off_cur;  // settled-list offset where the current step's vertices start
  uint32_t ul_out;        // unsettled list written by this step's pull (0 or 1)
  // private to the step-boundary block
  int64_t st0, st1, gap_lb;
  uint64_t sumd_lb, highd_lb;
  int64_t max_settled;
  uint32_t ul_sel, ul_valid;
  uint32_t rounds_in_step;
  uint32_t trace_len;
  // appended with atomics during phases
  uint32_t qcnt[3];
  uint32_t settled_cnt;
  uint32_t touched_cnt;
  uint32_t ulcnt[2];
  uint32_t ub_cand;
  unsigned long long heavy_packed[3];  // (items << 40) | entries, by round id mod 3
  uint32_t s2_done;
  uint32_t acc_maxd;
  unsigned long long acc_deg;
  uint32_t acc_any;
  uint32_t round_base;  // stamp id of the last round of the previous query
  unsigned long long cnt_rounds, cnt_frontier, cnt_trav, cnt_pulls, cnt_improved, cnt_heavy;
  GridBarrier bar;
  int status;
};

struct Workspace {
  uint32_t n = 0;
  uint32_t* stamp = nullptr;
  uint32_t* q[2] = {nullptr, nullptr};
  uint32_t* settled = nullptr;
  uint32_t* touched = nullptr;
  uint32_t* ul[2] = {nullptr, nullptr};
  uint32_t* hist = nullptr;
  unsigned long long* ring = nullptr;
  HeavyItem* heavy = nullptr;
  int64_t* step_ub = nullptr;
  uint32_t* step_off = nullptr;
  eic_step* trace = nullptr;
  Ctl* ctl = nullptr;
  Ctl* ctl_host = nullptr;  // pinned mirror for status readback
  uint32_t ring_bits = 0, ring_shift = 0;
  uint32_t heavy_cap = 0, step_cap = 0;
  uint64_t bytes = 0;
  uint32_t host_round_base = 0;
  int grid = 0, block = 0;  // cached cooperative launch shape
};

struct eic_graph {
  int device = 0;
  DevGraph dg{};
  uint64_t* row = nullptr;
  uint2* adj = nullptr;
  uint32_t* drank = nullptr;
  uint32_t* dvals = nullptr;
  uint32_t* dcnt0 = nullptr;
  uint32_t* rtow = nullptr;
  uint32_t* nz = nullptr;
  uint64_t bytes = 0;
  Workspace ws;
  std::mutex mu;
};

int eic_ws_ensure(eic_graph* g, int block_threads);
void eic_ws_free(Workspace* ws);

// Scratch of block groups (batches and the server): capacities, the layout
// of one group's arrays, and a pool of groups in one device allocation.
#pragma once

#include <vector>

#include "graph.h"

constexpr uint32_t kBatchStepCap = 1u << 17;  // steps per query of a batch
constexpr double kBatchMemFrac = 0.8;         // share of free device memory the scratch may take

// Capacities one block group's scratch must cover.
struct SlotCaps {
  uint64_t ni = 0, two_m = 0;
  uint32_t D = 0, ring_bits = 0;
  bool covers(const SlotCaps& o) const {
    return ni >= o.ni && two_m >= o.two_m && D >= o.D && ring_bits >= o.ring_bits;
  }
};

// Byte offsets of one group's arrays inside its slot (256-byte aligned).
struct SlotLayout {
  uint64_t idist, fbits, cursor, q0, q1, sid, sd, scur, touched, sbits, hist, ring, tasks, step_ub, step_off,
      ctl, bytes;
};

inline SlotLayout slot_layout(const SlotCaps& c) {
  SlotLayout L;
  uint64_t o = 0;
  auto take = [&o](uint64_t bytes) {
    const uint64_t at = o;
    o += (bytes + 255) & ~255ull;
    return at;
  };
  const uint64_t n = c.ni, words = n / 32 + 2;
  L.idist = take(n * 4);
  L.fbits = take(2 * words * 4);
  L.cursor = take(n * 4);
  L.q0 = take(n * 4);
  L.q1 = take(n * 4);
  L.sid = take((n + 2) * 4);
  L.sd = take((n + 2) * 4);
  L.scur = take((n + 2) * 4);
  L.touched = take((n + 1) * 4);
  L.sbits = take(words * 4);
  L.hist = take(((uint64_t)c.D + 1) * 4);
  L.ring = take((1ull << c.ring_bits) * 8);
  L.tasks = take((c.two_m / kHeavyMinFloor + 2) * sizeof(Task));
  L.step_ub = take(((uint64_t)kBatchStepCap + 2) * 8);
  L.step_off = take(((uint64_t)kBatchStepCap + 2) * 4);
  L.ctl = take(sizeof(Ctl));
  L.bytes = o;
  return L;
}

// Scratch of `count` block groups in one device allocation.
struct SlotPool {
  unsigned char* base = nullptr;
  BatchSlot* d_slots = nullptr;
  SlotCaps caps;
  uint32_t count = 0;
  uint64_t slot_bytes = 0;

  void release() {
    cudaFree(base);
    cudaFree(d_slots);
    base = nullptr;
    d_slots = nullptr;
    caps = SlotCaps();
    count = 0;
    slot_bytes = 0;
  }

  int ensure(const SlotCaps& need, uint32_t groups) {
    if (base && count >= groups && caps.covers(need)) return EIC_OK;
    release();
    const SlotLayout L = slot_layout(need);
    if (cudaMalloc((void**)&base, L.bytes * groups) != cudaSuccess ||
        cudaMalloc((void**)&d_slots, sizeof(BatchSlot) * groups) != cudaSuccess) {
      (void)cudaGetLastError();
      release();
      return EIC_ENOMEM;
    }
    std::vector<BatchSlot> h(groups);
    for (uint32_t g = 0; g < groups; ++g) {
      unsigned char* b = base + (uint64_t)g * L.bytes;
      BatchSlot& s = h[g];
      s.idist = (uint32_t*)(b + L.idist);
      s.fbits = (uint32_t*)(b + L.fbits);
      s.cursor = (uint32_t*)(b + L.cursor);
      s.q0 = (uint32_t*)(b + L.q0);
      s.q1 = (uint32_t*)(b + L.q1);
      s.sid = (uint32_t*)(b + L.sid);
      s.sd = (uint32_t*)(b + L.sd);
      s.scur = (uint32_t*)(b + L.scur);
      s.touched = (uint32_t*)(b + L.touched);
      s.sbits = (uint32_t*)(b + L.sbits);
      s.hist = (uint32_t*)(b + L.hist);
      s.ring = (unsigned long long*)(b + L.ring);
      s.tasks = (Task*)(b + L.tasks);
      s.step_ub = (int64_t*)(b + L.step_ub);
      s.step_off = (uint32_t*)(b + L.step_off);
      s.ctl = (Ctl*)(b + L.ctl);
      if (cudaMemset(s.ctl, 0, sizeof(Ctl)) != cudaSuccess) {
        (void)cudaGetLastError();
        release();
        return EIC_ECUDA;
      }
    }
    if (cudaMemcpy(d_slots, h.data(), sizeof(BatchSlot) * groups, cudaMemcpyHostToDevice) != cudaSuccess) {
      (void)cudaGetLastError();
      release();
      return EIC_ECUDA;
    }
    caps = need;
    count = groups;
    slot_bytes = L.bytes;
    return EIC_OK;
  }
};

// Ring of settled degree sums for Function 2: 2^bits slots, one per distance
// while maxW < 2^20; wider weights get *shift > 0 and 2^20 slots, which then
// hold Function 2's candidate bins (summed exactly from the settled list).
inline uint32_t ring_layout(uint32_t maxw, uint32_t* shift) {
  const uint32_t m = maxw ? maxw : 1;
  uint32_t bits = 0;
  while (bits < 32 && (1ull << bits) <= m) ++bits;  // 2^bits > maxW
  *shift = bits > 20 ? bits - 20 : 0;
  return bits < 20 ? bits : 20;
}

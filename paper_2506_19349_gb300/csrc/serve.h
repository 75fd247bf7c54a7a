// The serving path's shared definitions: the request ring in mapped pinned
// host memory (written by the host runtime, read by the serving kernel), the
// completion records (written by the kernel, read by the host), and the
// kernel's launch interface.
#pragma once

#include "graph.h"

// One admitted request, written by the host before it publishes `head`.
struct ServeRequest {
  unsigned long long ticket;
  uint32_t* out;  // device buffer of n uint32 for the result (caller's ids)
  uint32_t graph;
  uint32_t source;
};

// One completion record, written by the group that ran the request: ticket +
// 1 (release, system scope) after the status and after the result is visible.
struct ServeDone {
  unsigned long long ticket_plus1;
  int status;
  uint32_t pad;
};

// Mapped host memory shared by the host runtime and the kernel. Request k
// (k = 0, 1, ...) occupies ring entry k % cap; the host reuses an entry only
// after its previous request completed.
struct ServeRing {
  unsigned long long head;  // requests admitted so far (host, release)
  uint32_t stop;            // host asks every group to leave
  uint32_t cap;             // entries, a power of two
  // followed by ServeRequest req[cap] and ServeDone done[cap]
};

inline ServeRequest* serve_requests(ServeRing* r) { return (ServeRequest*)(r + 1); }
inline ServeDone* serve_done(ServeRing* r) { return (ServeDone*)(serve_requests(r) + r->cap); }

struct ServeArgs {
  ServeRing* ring;                // device view of the mapped ring
  ServeRequest* req;              // device view of its request entries
  ServeDone* done;                // device view of its completion records
  unsigned long long* claim;      // device: [0] next request to claim, [1] requests finished,
                                  // [2] groups registered idle, [3] nonzero: every group leaves
  const BatchQuery* graphs;       // [num_graphs] resident graphs (out and s unused)
  const BatchSlot* slot;          // [groups]
  uint32_t num_graphs, cap, nb;   // graphs; ring entries; blocks per group
  uint32_t groups;
  uint32_t alpha;
  double beta;
  uint32_t st_num, gap_shift, heavy_min, flags, step_cap;
  uint64_t max_spin;              // group-barrier bound (polls)
  uint64_t idle_ns;               // a group registers idle after this long without a request once
                                  // no group runs one; all leave together once all are registered
  uint64_t poll_ns;               // longest single wait of a group's first thread before the group
                                  // passes its barrier and waits again (keeps barrier waits short)
  uint64_t widen_at;              // 0, or: once this many admitted requests wait unclaimed, every group
                                  // leaves after its current request (the host relaunches more groups)
};

// Launch the serving kernel: `groups` groups of args.nb blocks of `block`
// threads, cooperatively, on stream. Returns an EIC_* status.
int eic_serve_launch(const ServeArgs& args, uint32_t groups, uint32_t block, cudaStream_t stream);

// Co-resident blocks of the serving kernel at this block size.
int eic_serve_grid(int block, uint32_t* grid);

// The step-width scaling (gap_shift, from `from` upwards while it helps by 2%,
// up to 8) that runs (g, source) fastest in a group of nb blocks: `copies`
// copies run at once, one per group, and each setting is timed twice on
// stream (the faster kept). *best_ms receives that setting's time.
int eic_tune_step_width(const eic_graph* g, uint32_t source, uint32_t copies, uint32_t nb, const eic_params& p,
                        uint32_t from, cudaStream_t stream, uint32_t* best_shift, double* best_ms);

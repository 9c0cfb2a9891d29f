// Host interface of the persistent batched kernel (blcoc_batched.cu).
#pragma once
#include "blcoc_common.cuh"

namespace blcoc {

// One system of a persistent batch (device-resident array, written by the host).
struct PersSys {
  PassArgs a;       // CSR, blocks, p x p factors, partial-sum slots, control block
  double* stage1;   // first-stage reduction slices
  double* hist;     // residual history
  int pp;           // compile-time width the system runs at (1, 2, 4, 8 or 16)
  int vg[3];        // virtual grid of pass 1 (cocr A / cocg 1), the SpMM, pass 2 (cocr C /
                    // cocg 2): the grids of a single solve, so the reduction order and the
                    // results are those of blcoc_solve
};

// One slot of the ring of work items.  `seq` = ticket the slot holds (published when it
// equals the ticket), `freed` = the next ticket the slot may take (its reader has copied it).
struct QItem {
  unsigned long long seq;
  unsigned long long freed;
  int sys, stage, item, pad;
};

// Scheduler state: tickets taken and published, systems still running, error flag (set by
// a wait that ran out of time).
struct SchedState {
  unsigned long long head;
  unsigned long long tail;
  int active;
  int err;
  int pad[2];
};

// Per system: current stage and its items not yet done.
struct SysRun {
  int stage;
  int remaining;
};

constexpr int PERSISTENT_PMAX = 16;

// Stages of one iteration and items of a stage (host copy of the device rule).
int persistent_stage_count(int method);
// Dynamic shared memory for a batch of one method whose widest system has pmax columns.
size_t persistent_smem(int pmax, int method);
// Resident CTAs per SM at that shared-memory size (also sets the kernel's smem limit).
cudaError_t persistent_ctas_per_sm(size_t smem, int* out);
// Launch the batch: `grid` CTAs take items from the ring until no system runs; every wait
// gives up after timeout_ns (SchedState::err).  The ring, the scheduler state and the
// per-system counters must be initialised (one item per running system: its first
// alpha' stage).
cudaError_t launch_persistent(const PersSys* sys, int method, SchedState* sch, QItem* ring, unsigned cap,
                              SysRun* run, long long timeout_ns, int grid, size_t smem, cudaStream_t s);

}  // namespace blcoc

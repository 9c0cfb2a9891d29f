// Persistent batched solver: every iteration of every system of a batch (independent
// systems of uneven n and p <= 16, one rq method) in ONE kernel launch that runs until no
// system is left running.
//
// Dataflow scheduling.  An iteration of Algorithm 2 or 3 is a chain of stages per system:
//
//   bl_cocr_rq:  alpha' | pass A | reduce | QR | SpMM | reduce | beta' | pass C | reduce
//   bl_cocg_rq:  alpha' | pass 1 | reduce | QR + beta' | pass 2 | SpMM | reduce
//
// A row pass of system s has vg_s items (the virtual CTAs of the launch a single solve of
// s makes, each with its share of 32-row chunks), a reduction 16 (first-stage slices), a
// p x p stage one.  The items wait in one ring of tickets (the systems' work queues,
// merged).  Every CTA loops: take the next ticket, wait until it is published, run its
// item, count it done; the CTA that completes the last item of a stage publishes the
// items of the system's next stage.  The systems thus advance independently: a p x p
// stage of one system overlaps the row passes of the others and an idle CTA takes
// whatever is ready.  A p x p stage that leaves its system stopped (converged at the top
// of an iteration, iteration limit, breakdown) publishes nothing - the system's
// convergence mask - and the kernel ends when no system runs.
//
// * The arithmetic of every item is that of the single-system kernels (the same device
//   functions, the same partial slots, the same reduction order), so each system's
//   iterates are bitwise those of a separate blcoc_solve, whatever the grid size.
// * Items read what other CTAs wrote for earlier stages of the same launch, so this
//   translation unit compiles the shared device code with coherent (L2) loads.
// * A ring slot is reused only after its reader has copied it (the ring holds more than
//   twice the items that can be in flight).  Every wait has a time limit; a wait that
//   runs out sets the scheduler's error flag, every CTA then returns, and the host
//   reports BLCOC_ERR_TIMEOUT.
#include <type_traits>

#define BLCOC_COHERENT_LOADS 1
#define BLCOC_SMALL_LD 16
#include "blcoc_rowpass.cuh"
#include "blcoc_small_dev.cuh"
#include "blcoc_batched.h"

namespace blcoc {

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One row pass of one system, as virtual CTA vb of a G-CTA launch.
template <int PP>
__device__ __noinline__ void row_pass(int kind, const PassArgs& a, int vb, int G) {
  switch (kind) {
    case K_COCR_A: d_cocr_passA<PP, double, false>(a, vb, G); break;
    case K_SPMM_GRAM: d_spmm_gram<PP, double, false>(a, vb, G); break;
    case K_COCR_C: d_cocr_passC<PP, double, false>(a, vb, G); break;
    case K_COCG_1: d_cocg_pass1<PP, double>(a, vb, G); break;
    case K_COCG_2: d_cocg_pass2<PP, double>(a, vb, G); break;
    default: break;
  }
}

// Item `vb` of row pass `which` (0 pass 1, 1 SpMM, 2 pass 2) of one system: virtual CTA
// vb of a launch of vg = y.vg[which] CTAs, exactly as in a single solve.
__device__ void row_item(const PersSys& y, int which, int kind, int tri_mult, int flag, bool gather_s, int vb) {
  PassArgs a = y.a;
  const int vg = y.vg[which];
  a.ne = tri_mult * tri_count(a.p);
  a.flag = flag;
  a.grid = vg;
  if (gather_s) a.W = a.S;
  switch (y.pp) {
    case 1: row_pass<1>(kind, a, vb, vg); break;
    case 2: row_pass<2>(kind, a, vb, vg); break;
    case 4: row_pass<4>(kind, a, vb, vg); break;
    case 8: row_pass<8>(kind, a, vb, vg); break;
    default: row_pass<16>(kind, a, vb, vg); break;
  }
}

// Item `sl` of the first-stage reduction after row pass `which`: slice sl of its vg
// partial slots, summed in the order of k_reduce_stage1.
__device__ void reduce_item(const PersSys& y, int which, int tri_mult, int sl) {
  const int ncomp = 2 * tri_mult * tri_count(y.a.p);
  const int nparts = y.vg[which];
  const double* part = reinterpret_cast<const double*>(y.a.partials);
  const int q0 = (int)((int64_t)sl * nparts / RED_SPLIT), q1 = (int)((int64_t)(sl + 1) * nparts / RED_SPLIT);
  for (int c = threadIdx.x; c < ncomp; c += blockDim.x) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};   // a[g]: q = q0 + g, q0 + g + 4, ... in turn
    for (int q = q0; q < q1; ++q) a[(q - q0) & 3] += __ldcg(part + (int64_t)q * ncomp + c);
    const double a0 = a[0], a1 = a[1], a2 = a[2], a3 = a[3];
    y.stage1[(int64_t)sl * ncomp + c] = (a0 + a1) + (a2 + a3);
  }
}

// ---------------------------------------------------------------------------- stages
// bl_cocr_rq (method 1): 0 alpha' | 1 pass A | 2 reduce | 3 QR | 4 SpMM | 5 reduce | 6 beta' |
//                        7 pass C | 8 reduce
// bl_cocg_rq (method 0): 0 alpha' | 1 pass 1 | 2 reduce | 3 QR + beta' | 4 pass 2 | 5 SpMM |
//                        6 reduce
__host__ __device__ __forceinline__ int stage_count(int method) { return method == 1 ? 9 : 7; }
__device__ __forceinline__ bool stage_is_small(int method, int st) {
  return method == 1 ? (st == 0 || st == 3 || st == 6) : (st == 0 || st == 3);
}
__device__ __forceinline__ int stage_items(const PersSys& y, int method, int st) {
  if (stage_is_small(method, st)) return (method == 1 && st == 0) ? 2 : 1;   // cocr alpha': + the elimination of H_m
  if (method == 1) return st == 1 ? y.vg[0] : st == 4 ? y.vg[1] : st == 7 ? y.vg[2] : RED_SPLIT;
  return st == 1 ? y.vg[0] : st == 4 ? y.vg[2] : st == 5 ? y.vg[1] : RED_SPLIT;
}

__device__ void run_item(SmallShared& S, const PersSys& y, int method, int st, int item) {
  const int p = y.a.p, E = tri_count(p);
  double2* mats = const_cast<double2*>(y.a.mats);
  if (method == 1) {
    switch (st) {
      case 0:   // item 0: the alpha' step; item 1: the elimination of H_m for the beta' step
        if (item == 0) d_small_alpha(S, p, y.stage1, 2 * E, mats, y.a.ctrl, y.hist, 0, nullptr);
        else d_small_hfactor(S, p, mats, y.a.ctrl);
        break;
      case 1: row_item(y, 0, K_COCR_A, 1, 0, false, item); break;        // W = Q - U alpha', W^H W
      case 2: reduce_item(y, 0, 1, item); break;
      case 3: d_small_chol(S, p, 1, y.stage1, 2 * E, mats, y.a.ctrl, 0, nullptr); break;
      case 4: row_item(y, 1, K_SPMM_GRAM, 1, 1, false, item); break;     // V = A W T, W^T A W
      case 5: reduce_item(y, 1, 1, item); break;
      case 6: d_small_cocr_beta(S, p, y.stage1, 2 * E, mats, y.a.ctrl, nullptr, 0, p); break;
      case 7: row_item(y, 2, K_COCR_C, 1, 0, false, item); break;        // Q, X, S, U, U^T U
      default: reduce_item(y, 2, 1, item); break;
    }
  } else {
    switch (st) {
      case 0: d_small_alpha(S, p, y.stage1, 2 * E, mats, y.a.ctrl, y.hist, 0, nullptr); break;
      case 1: row_item(y, 0, K_COCG_1, 2, 0, false, item); break;        // W, X, W^H W, W^T W
      case 2: reduce_item(y, 0, 2, item); break;
      case 3: d_small_chol(S, p, 0, y.stage1, 4 * E, mats, y.a.ctrl, 0, nullptr); break;
      case 4: row_item(y, 2, K_COCG_2, 0, 0, false, item); break;        // Q, S
      case 5: row_item(y, 1, K_SPMM_GRAM, 1, 0, true, item); break;      // A S, S^T A S
      default: reduce_item(y, 1, 1, item); break;
    }
  }
}

// ---------------------------------------------------------------------------- queue
// Take the next ticket and wait for its item.  Returns 0 when no system runs any more or a
// wait ran out of time (then SchedState::err is set).
__device__ int take_item(SchedState* sch, QItem* ring, unsigned cap, long long timeout_ns, int* out) {
  const unsigned long long t = atomicAdd(&sch->head, 1ull);
  QItem* q = ring + (t % cap);
  volatile unsigned long long* seq = &q->seq;
  volatile int* err = &sch->err;
  volatile int* active = &sch->active;
  const long long t0 = global_ns();
  unsigned nap = 32;
  while (*seq != t) {
    if (*err || *active == 0) return 0;
    if (global_ns() - t0 > timeout_ns) {
      atomicExch(&sch->err, 1);
      return 0;
    }
    __nanosleep(nap);
    if (nap < 1024) nap *= 2;
  }
  __threadfence();
  const volatile QItem* vq = q;
  out[0] = vq->sys;
  out[1] = vq->stage;
  out[2] = vq->item;
  __threadfence();
  *reinterpret_cast<volatile unsigned long long*>(&q->freed) = t + cap;   // slot may take ticket t + cap
  return 1;
}

// Publish ticket t: wait until the slot's previous item has been copied by its reader.
__device__ bool put_item(SchedState* sch, QItem* ring, unsigned cap, long long timeout_ns, unsigned long long t,
                         int sys, int stage, int item) {
  QItem* q = ring + (t % cap);
  volatile unsigned long long* freed = &q->freed;
  const long long t0 = global_ns();
  while (*freed != t) {
    if (*reinterpret_cast<volatile int*>(&sch->err)) return false;
    if (global_ns() - t0 > timeout_ns) {
      atomicExch(&sch->err, 1);
      return false;
    }
    __nanosleep(64);
  }
  q->sys = sys;
  q->stage = stage;
  q->item = item;
  __threadfence();
  *reinterpret_cast<volatile unsigned long long*>(&q->seq) = t;
  return true;
}

__global__ void __launch_bounds__(NWARP * 32, 3)
    k_batched_persistent(const PersSys* __restrict__ sys, int method, SchedState* sch, QItem* ring, unsigned cap,
                         SysRun* run, long long timeout_ns) {
  extern __shared__ __align__(16) unsigned char pers_raw[];
  SmallShared& S = *reinterpret_cast<SmallShared*>(pers_raw);
  __shared__ int s_cmd[4];
  __shared__ unsigned long long s_t0;
  for (;;) {
    if (threadIdx.x == 0) s_cmd[3] = take_item(sch, ring, cap, timeout_ns, s_cmd);
    __syncthreads();
    if (!s_cmd[3]) return;
    const int s = s_cmd[0], st = s_cmd[1], item = s_cmd[2];
    const PersSys& y = sys[s];
    run_item(S, y, method, st, item);
    __syncthreads();
    if (threadIdx.x == 0) {
      int publish = 0;
      __threadfence();   // this item's results before its count
      if (atomicSub(&run[s].remaining, 1) == 1) {   // last item of the stage
        if (stage_is_small(method, st) && __ldcg(&y.a.ctrl->done)) {
          atomicSub(&sch->active, 1);                 // the system stopped: publish nothing
        } else {
          const int nxt = st + 1 == stage_count(method) ? 0 : st + 1;
          const int cnt = stage_items(y, method, nxt);
          run[s].stage = nxt;
          atomicExch(&run[s].remaining, cnt);
          __threadfence();
          s_t0 = atomicAdd(&sch->tail, (unsigned long long)cnt);
          s_cmd[1] = nxt;
          s_cmd[2] = cnt;
          publish = 1;
        }
      }
      s_cmd[3] = publish;
    }
    __syncthreads();
    if (s_cmd[3]) {
      const int nxt = s_cmd[1], cnt = s_cmd[2];
      for (int k = threadIdx.x; k < cnt; k += blockDim.x)
        if (!put_item(sch, ring, cap, timeout_ns, s_t0 + (unsigned long long)k, s, nxt, k)) break;
    }
    __syncthreads();   // s_cmd and s_t0 are reused by the next item
  }
}

int persistent_stage_count(int method) { return stage_count(method); }

size_t persistent_smem(int pmax, int method) {
  int PP = 1;
  while (PP < pmax) PP *= 2;
  size_t m = sizeof(SmallShared);
  auto up = [&](size_t v) { m = v > m ? v : m; };
  auto kinds = [&](auto pp) {
    constexpr int W = decltype(pp)::value;
    if (method == 1) {
      up(pass_smem<W, double>(K_COCR_A));
      up(pass_smem<W, double>(K_SPMM_GRAM));
      up(pass_smem<W, double>(K_COCR_C));
    } else {
      up(pass_smem<W, double>(K_COCG_1));
      up(pass_smem<W, double>(K_COCG_2));
      up(pass_smem<W, double>(K_SPMM_GRAM));
    }
  };
  switch (PP) {
    case 1: kinds(std::integral_constant<int, 1>{}); break;
    case 2: kinds(std::integral_constant<int, 2>{}); break;
    case 4: kinds(std::integral_constant<int, 4>{}); break;
    case 8: kinds(std::integral_constant<int, 8>{}); break;
    default: kinds(std::integral_constant<int, 16>{}); break;
  }
  return m;
}

cudaError_t persistent_ctas_per_sm(size_t smem, int* out) {
  cudaError_t e = cudaFuncSetAttribute(k_batched_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_batched_persistent, NWARP * 32, smem);
}

cudaError_t launch_persistent(const PersSys* sys, int method, SchedState* sch, QItem* ring, unsigned cap,
                              SysRun* run, long long timeout_ns, int grid, size_t smem, cudaStream_t s) {
  k_batched_persistent<<<grid, NWARP * 32, smem, s>>>(sys, method, sch, ring, cap, run, timeout_ns);
  return cudaGetLastError();
}

}  // namespace blcoc

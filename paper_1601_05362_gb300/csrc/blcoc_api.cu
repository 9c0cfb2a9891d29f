// C ABI of libblcoc.so and the host-side solve loop (see include/blcoc.h).
//
// One solve = a setup sequence (residual, QR, first products) followed by batches of
// iterations queued on an internal stream, optionally replayed as a CUDA graph.  The
// host never waits inside an iteration: the convergence test, the iteration limit and
// breakdown are decided on the device (control block), every kernel of an iteration
// returns at once after the decision, and the host reads the control block once per
// batch of `poll` iterations.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/blcoc.h"
#include "blcoc_common.cuh"
#include "blcoc_ozaki.cuh"
#include "blcoc_small.h"
#include "blcoc_batched.h"

using namespace blcoc;

namespace {

thread_local std::string g_create_error;

}  // namespace

void blcoc::set_global_error(const char* msg) { g_create_error = msg; }

namespace {

const KernelSet* kernels_for(int p, int* PP, bool f32 = false) {
  if (p <= 1) { *PP = 1; return f32 ? &kernel_set<1, float>() : &kernel_set<1, double>(); }
  if (p <= 2) { *PP = 2; return f32 ? &kernel_set<2, float>() : &kernel_set<2, double>(); }
  if (p <= 4) { *PP = 4; return f32 ? &kernel_set<4, float>() : &kernel_set<4, double>(); }
  if (p <= 8) { *PP = 8; return f32 ? &kernel_set<8, float>() : &kernel_set<8, double>(); }
  if (p <= 16) { *PP = 16; return f32 ? &kernel_set<16, float>() : &kernel_set<16, double>(); }
  *PP = 32;
  return f32 ? &kernel_set<32, float>() : &kernel_set<32, double>();
}

// Kernel set whose p x p block updates run on the tensor cores (block widths 8, 16, 32).
const KernelSet* tc_kernels(int PP) {
  if (PP == 8) return &kernel_set_tc<8>();
  if (PP == 16) return &kernel_set_tc<16>();
  return &kernel_set_tc<32>();
}

__global__ void k_vals_to_c64(const double2* __restrict__ v, float2* __restrict__ o, int64_t nnz) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = make_float2((float)v[i].x, (float)v[i].y);
}

// Names of the timed kernel kinds (index = PassKind of blcoc_rowpass.cuh).
const char* const kKindNames[] = {"resid",       "spmm_gram",   "spmm_plain",  "cocr_passA",  "cocr_passC",
                                  "cocg_pass1",  "cocg_pass2",  "reduce",      "small_setup", "small_H0",
                                  "small_alpha", "small_chol",  "small_beta",  "small_trr",   "small_setup_inner",
                                  "small_chol2", "small_chol2_setup", "qr2"};
constexpr int kNumKinds = 18;
constexpr int kKindReduce = 7, kKindSmall0 = 8;   // small kernel kind = kKindSmall0 + SmallKind
constexpr int kKindQR2 = 17;

struct Timer {
  int kind;
  int iter;   // iteration index within the batch
  cudaEvent_t e0, e1;
};

// NVTX range for profilers (a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// What decides the kernel sequence of a captured batch of iterations: compared field by
// field, so a new option cannot make two different sequences look alike.
struct GraphKey {
  int method = -1;   // blcoc_method of the iteration (the inner rq method for mixed solves)
  int mixed = 0;     // complex64 inner iteration of the mixed-precision refinement
  int uexpl = 0;     // U = A S by a second sparse product
  int plain = 0;     // plain block method (tau = T = xi = I)
  int tc = 0;        // tensor-core block updates
  int qr2 = 0;       // CholQR2
  int split = 0;     // SpMM row bundle
  int qr_fb = 0;     // shifted-CholQR3 fallback passes present
  bool operator==(const GraphKey& o) const {
    return method == o.method && mixed == o.mixed && uexpl == o.uexpl && plain == o.plain && tc == o.tc &&
           qr2 == o.qr2 && split == o.split && qr_fb == o.qr_fb;
  }
};

struct Graph {
  cudaGraphExec_t exec = nullptr;
  GraphKey key;
  int p = -1, batch = 0, timing = 0;
  const void* X = nullptr;
  int64_t gen = -1;
  int launches = 0;
  std::vector<Timer> timers;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    p = -1;
    timers.clear();
  }
};

}  // namespace

struct blcoc_ctx {
  int dev = 0;
  int num_sms = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  int64_t n = 0, nnz = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  double2* va = nullptr;
  float2* vaf = nullptr;      // complex64 values, made on the first mixed-precision solve
  // workspace
  int p_cap = 0;
  int64_t gen = 0;
  double2 *W = nullptr, *S = nullptr, *U = nullptr, *V = nullptr, *Q = nullptr;
  // staging copies of host-memory B and X; st_cap = the columns they hold (independent of
  // p_cap, which device-pointer solves also raise)
  double2 *Bst = nullptr, *Xst = nullptr;
  int st_cap = 0;
  double2* mats = nullptr;
  double2* partials = nullptr;
  size_t partials_cap = 0;   // double2 entries
  double* stage1 = nullptr;
  size_t stage1_cap = 0;     // doubles
  // complex64 workspace of the mixed-precision form (W, S, U, V, Q, D)
  int p_cap32 = 0;
  float2* w32[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* hist = nullptr;
  int hist_cap = 0;
  Ctrl* ctrl = nullptr;
  Ctrl* h_ctrl = nullptr;    // pinned
  int* flags = nullptr;
  // options
  int use_graph = 1;
  int poll = 16;
  int timing = 0;
  int inner_tol_exp = -5;     // mixed precision: inner tolerance 10^inner_tol_exp
  int inner_maxit = 0;        // mixed precision: per inner solve (0 = remaining budget)
  int outer_maxit = 40;
  int outer_iters = 0;
  int fp64_tc = 0;            // cocr, p <= 16: p x p applies on the tensor cores by exact slicing
  uint2* ozbuf = nullptr;     // their factor fragments
  int u_explicit = 0;         // cocr: U_{m+1} = A S_{m+1} by SpMM instead of V + U beta'
  int u_explicit_mixed = 1;   // the same for the complex64 inner solves
  int qr_passes = 1;          // 2: CholQR2 (one re-orthogonalising pass after every Cholesky QR)
  int qr_fallback = 1;        // rq methods, qr_passes = 1: shifted-CholQR3 fallback when a Cholesky QR fails
  int spmm_split = 1;         // SpMM row bundle (1, 2, 4); 0: timed sweep, cached per (n, nnz/row, p)
  // option graph_conditional: captured iterations hold the QR fallback's launches in a
  // conditional graph node (reset to 0 if the runtime refuses one: they are then captured
  // as plain launches that return at once).  Off by default: Nsight Compute does not profile
  // the kernel nodes of a graph that can hold conditional nodes.
  int cond_ok = 0;
  cudaStream_t sbody = nullptr;   // captures the conditional node's body
  int stat_spmm_split = 0;    // row bundle of the last solve
  int persistent_timeout_ms = 10000;   // persistent batch: limit of one wait of the kernel
  int persistent_stall = 0;   // persistent batch, test hook: no first work item is published
  int stat_persistent_graph = -1;   // last persistent batch: 1 graph replays, 0 direct launches
  Graph graph;
  // kernel timing: event pool and per-kind totals of the last solve
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  double kt_ms[kNumKinds] = {0};
  int64_t kt_n[kNumKinds] = {0};
  // results of the last solve
  int iters = 0;
  double relres = 0.0, trr = 0.0;
  std::vector<double> hist_h;
  std::vector<double> xi_h;
  int64_t stat_launches = 0, stat_replays = 0;
  std::string err;
};

namespace {

blcoc_status cuda_fail(blcoc_ctx* h, cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  if (h) h->err = buf;
  else g_create_error = buf;
  return e == cudaErrorMemoryAllocation ? BLCOC_ERR_OOM : BLCOC_ERR_CUDA;
}

#define CK(h, call)                                             \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
  } while (0)

blcoc_status invalid(blcoc_ctx* h, const char* msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return BLCOC_ERR_INVALID_ARG;
}

// Partial entries per CTA for any pass: max over kinds (resid: 2 triangles + norms).
int max_ne(int p) { return 2 * tri_count(p) + 1; }

void free_ws32(blcoc_ctx* h) {
  for (float2*& b : h->w32) {
    if (b) cudaFree(b);
    b = nullptr;
  }
  h->p_cap32 = 0;
}

void free_ws(blcoc_ctx* h) {
  double2* blocks[] = {h->W, h->S, h->U, h->V, h->Q, h->mats, h->partials};
  for (double2* b : blocks)
    if (b) cudaFree(b);
  if (h->stage1) cudaFree(h->stage1);
  h->W = h->S = h->U = h->V = h->Q = h->mats = h->partials = nullptr;
  h->stage1 = nullptr;
  h->p_cap = 0;
  h->partials_cap = h->stage1_cap = 0;
}

blcoc_status ensure_ws32(blcoc_ctx* h, int p) {
  if (!h->vaf) {
    CK(h, cudaMalloc(&h->vaf, h->nnz * sizeof(float2)));
    k_vals_to_c64<<<h->num_sms * 4, 256, 0, h->s>>>(h->va, h->vaf, h->nnz);
    CK(h, cudaGetLastError());
  }
  if (p <= h->p_cap32) return BLCOC_OK;
  h->graph.reset();
  free_ws32(h);
  const size_t blk = (size_t)h->n * p * sizeof(float2);
  for (float2*& b : h->w32) CK(h, cudaMalloc(&b, blk));
  h->p_cap32 = p;
  h->gen++;
  return BLCOC_OK;
}

blcoc_status ensure_ws(blcoc_ctx* h, int p) {
  if (p <= h->p_cap) return BLCOC_OK;
  h->graph.reset();
  free_ws(h);
  const size_t blk = (size_t)h->n * p * sizeof(double2);
  CK(h, cudaMalloc(&h->W, blk));
  CK(h, cudaMalloc(&h->S, blk));
  CK(h, cudaMalloc(&h->U, blk));
  CK(h, cudaMalloc(&h->V, blk));
  CK(h, cudaMalloc(&h->Q, blk));
  CK(h, cudaMalloc(&h->mats, (size_t)M_NSLOTS * PMAX * PMAX * sizeof(double2)));
  CK(h, cudaMemset(h->mats, 0, (size_t)M_NSLOTS * PMAX * PMAX * sizeof(double2)));
  const int ne = max_ne(PMAX);
  h->partials_cap = (size_t)h->num_sms * 4 * ne;
  CK(h, cudaMalloc(&h->partials, h->partials_cap * sizeof(double2)));
  h->stage1_cap = (size_t)RED_SPLIT * 2 * ne;
  CK(h, cudaMalloc(&h->stage1, h->stage1_cap * sizeof(double)));
  h->p_cap = p;
  h->gen++;
  return BLCOC_OK;
}

}  // namespace

// ------------------------------------------------------------------------------ solve loop
namespace {

struct Solver {
  blcoc_ctx* h;
  const KernelSet* K;
  int PP, p, method;
  const double2* B;
  double2* X;
  // block buffers: the FP64 workspace, or (mixed precision) the complex64 one
  double2 *bW = nullptr, *bS = nullptr, *bU = nullptr, *bV = nullptr, *bQ = nullptr;
  void use_fp64_blocks() {
    bW = h->W;
    bS = h->S;
    bU = h->U;
    bV = h->V;
    bQ = h->Q;
  }
  void use_c64_blocks() {
    bW = reinterpret_cast<double2*>(h->w32[0]);
    bS = reinterpret_cast<double2*>(h->w32[1]);
    bU = reinterpret_cast<double2*>(h->w32[2]);
    bV = reinterpret_cast<double2*>(h->w32[3]);
    bQ = reinterpret_cast<double2*>(h->w32[4]);
  }
  PassArgs base() const {
    PassArgs a{};
    a.A = CsrDev{h->n, h->nnz, h->rp, h->ci, h->va, h->vaf};
    a.p = p;
    a.W = bW ? bW : h->W;
    a.S = bS ? bS : h->S;
    a.U = bU ? bU : h->U;
    a.V = bV ? bV : h->V;
    a.Q = bQ ? bQ : h->Q;
    a.X = X;
    a.B = B;
    a.mats = h->mats;
    a.partials = h->partials;
    a.ctrl = h->ctrl;
    a.oz = oz;
    return a;
  }
  int launches = 0;
  std::vector<Timer>* timers = nullptr;   // when set, each pass kernel is bracketed by events
  int batch_iter = 0;
  bool capturing = false;                 // events inside a graph must be external record nodes
  void record(cudaEvent_t e) {
    if (capturing) cudaEventRecordWithFlags(e, h->s, cudaEventRecordExternal);
    else cudaEventRecord(e, h->s);
  }
  cudaEvent_t next_event() {
    if (h->evnext == h->evpool.size()) {
      cudaEvent_t e = nullptr;
      cudaEventCreate(&e);
      h->evpool.push_back(e);
    }
    return h->evpool[h->evnext++];
  }
  void pass(LaunchFn f, int kind, int ne, int flag, double2* in = nullptr, int tkind = -1) {
    PassArgs a = base();
    if (in) a.W = in;   // spmm_gram gathers a.W
    a.ne = ne;
    a.flag = flag;
    a.grid = K->grid(h->n, kind, sms());
    Timer t{tkind >= 0 ? tkind : kind, batch_iter, nullptr, nullptr};
    const bool timed = timers && (time_only < 0 || kind == time_only);
    if (timed) {
      t.e0 = next_event();
      t.e1 = next_event();
      record(t.e0);
    }
    f(a, h->s);
    if (timed) {
      record(t.e1);
      timers->push_back(t);
    }
    ++launches;
    last_grid = a.grid;
  }
  int last_grid = 0;
  void timed_begin(Timer& t, int kind) {
    t = Timer{kind, batch_iter, nullptr, nullptr};
    if (timers) {
      t.e0 = next_event();
      t.e1 = next_event();
      record(t.e0);
    }
  }
  void timed_end(Timer& t) {
    if (timers) {
      record(t.e1);
      timers->push_back(t);
    }
  }
  bool time_small = true;   // with timers: also bracket the reductions and p x p stages
  int time_only = -1;       // with timers: >= 0 brackets only the row passes of this kind
  void set_timing_mode(int mode) {
    time_small = mode == 1;
    time_only = mode == 3 ? (method == BLCOC_COCR_RQ ? (int)K_COCR_C : (int)K_COCG_1) : -1;
  }
  void reduce(int ne, const Ctrl* ctrl, bool fb_only = false) {
    Timer t;
    if (time_small) timed_begin(t, kKindReduce);
    launch_reduce(h->partials, last_grid, ne, h->stage1, ctrl, h->s, fb_only);
    if (time_small) timed_end(t);
    ++launches;
  }
  int plain = 0;   // 1: plain block method (Algorithm 1 / derived block COCG)
  uint2* oz = nullptr;   // factor fragments when the applies run on the tensor cores
  int grid_sms = 0;   // SMs the row passes size their grid for (0 = all)
  int sms() const { return grid_sms > 0 ? grid_sms : h->num_sms; }
  void small(SmallKind k, int ne) {
    Timer t;
    if (time_small) timed_begin(t, kKindSmall0 + (int)k);
    launch_small(k, p, method + 16 * plain + 32 * qr2, h->stage1, ne, h->mats, h->ctrl, h->hist, h->s, oz,
                 k == SK_CHOL ? cond : 0ull);
    if (time_small) timed_end(t);
    ++launches;
  }
  // kinds must match PassKind in blcoc_rowpass.cuh
  enum { K_RESID = 0, K_SPMM_GRAM, K_SPMM_PLAIN, K_COCR_A, K_COCR_C, K_COCG_1, K_COCG_2, K_AXPY, K_QR2 };
  int qr2 = 0;   // CholQR2: after each Cholesky QR, W <- W T1 and a second factor
  int spmm_split = 1;   // SpMM row bundle: lane groups splitting each row's nonzeros (1, 2, 4)
  LaunchFn spmm_fn() const {
    if (spmm_split == 4 && K->spmm_gram_s4) return K->spmm_gram_s4;
    if (spmm_split == 2 && K->spmm_gram_s2) return K->spmm_gram_s2;
    return K->spmm_gram;
  }
  // CholQR2's second pass and factor (setup: the factor of R_0)
  // (cocg: the pass also forms Q1^T Q1, from which the stage forms Q^T Q of the final basis)
  void second_qr(bool setup) {
    if (!qr2 || plain) return;
    const int E = tri_count(p), ne = method == BLCOC_COCG_RQ ? 2 * E : E;
    pass(K->qr2, K_QR2, ne, method == BLCOC_COCG_RQ ? F_SYM2 : 0, nullptr, kKindQR2);
    reduce(ne, h->ctrl);
    small(setup ? SK_CHOL2_SETUP : SK_CHOL2, ne);
  }
  // Shifted-CholQR3 fallback (rq methods with single-pass Cholesky QR): when the p x p
  // stage before had to shift the Gram, two Cholesky QR passes complete the factorisation;
  // otherwise these kernels return at once.
  int qr_fb = 0;
  void fallback_launches(bool setup) {
    const int E = tri_count(p), ne = method == BLCOC_COCG_RQ ? 2 * E : E;
    for (int k = 0; k < 2; ++k) {
      pass(K->qr2, K_QR2, ne, F_FB | (method == BLCOC_COCG_RQ ? F_SYM2 : 0), nullptr, kKindQR2);
      reduce(ne, h->ctrl, true);
      small(setup ? SK_CHOL_FB_SETUP : SK_CHOL_FB, ne);
    }
  }
  // Shifted-CholQR3 fallback after a Cholesky QR.  Launched directly, its kernels return at
  // once unless the preceding stage started it.  In a captured iteration they form the body
  // of a conditional IF node whose handle that stage (SK_CHOL) sets, so a replay that needs
  // no fallback runs none of them.
  void fallback_qr(bool setup) {
    if (!qr_fb) return;
    if (!setup && cond != 0) {
      const bool ok = fallback_conditional();
      cond = 0;
      if (ok) return;
      cond_failed = true;   // the caller discards this capture and captures plain launches
    }
    fallback_launches(setup);
  }
  // conditional graph node of the current iteration's fallback (captured graphs)
  unsigned long long cond = 0;
  bool cond_failed = false;
  void cond_begin() {
    cond = 0;
    if (!capturing || !qr_fb || !h->cond_ok || cond_failed) return;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t cg = nullptr;
    cudaGraphConditionalHandle hd = 0;
    if (cudaStreamGetCaptureInfo(h->s, &st, nullptr, &cg) != cudaSuccess || st != cudaStreamCaptureStatusActive ||
        cudaGraphConditionalHandleCreate(&hd, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess) {
      cudaGetLastError();
      cond_failed = true;
      return;
    }
    cond = (unsigned long long)hd;
  }
  bool fallback_conditional() {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(h->s, &st, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive)
      return cudaGetLastError(), false;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = (cudaGraphConditionalHandle)cond;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np) != cudaSuccess ||
        cudaStreamUpdateCaptureDependencies(h->s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
      return cudaGetLastError(), false;
    if (!h->sbody && cudaStreamCreateWithFlags(&h->sbody, cudaStreamNonBlocking) != cudaSuccess)
      return cudaGetLastError(), false;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(h->sbody, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess)
      return cudaGetLastError(), false;
    // the body's launches: on the body stream, untimed (event nodes are not allowed in a
    // conditional body) and not counted (they run only when needed)
    cudaStream_t main_s = h->s;
    std::vector<Timer>* keep_timers = timers;
    const bool keep_small = time_small;
    const int keep_launches = launches;
    h->s = h->sbody;
    timers = nullptr;
    time_small = false;
    fallback_launches(false);
    h->s = main_s;
    timers = keep_timers;
    time_small = keep_small;
    launches = keep_launches;
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(h->sbody, &out) != cudaSuccess) return cudaGetLastError(), false;
    return true;
  }
  void chol_stage(int ne) {
    cond_begin();
    small(SK_CHOL, ne);
  }

  // inner = 1: the right-hand side of this solve is the residual itself (refinement
  // step), so the stopping test is relative to ||R||_F instead of ||B||_F.
  void setup_residual(int inner = 0) {
    const int E = tri_count(p);
    pass(K->resid, K_RESID, 2 * E + 1, method == BLCOC_COCG_RQ ? 2 : 0);
    reduce(2 * E + 1, h->ctrl);
    small(inner ? SK_SETUP_INNER : SK_SETUP, 2 * E + 1);
    second_qr(true);
    fallback_qr(true);
  }
  void setup_rest() {
    const int E = tri_count(p);
    if (method == BLCOC_COCR_RQ) {
      pass(spmm_fn(), K_SPMM_GRAM, E, 1);   // V_0 = A Q_0, gram W^T A W
      reduce(E, h->ctrl);
      small(SK_COCR_H0, E);
      pass(K->cocr_passC, K_COCR_C, E, 1);     // S_0 = Q_0, U_0 = V_0, gram U^T U
      reduce(E, h->ctrl);
    } else {
      pass(K->cocg_pass2, K_COCG_2, 0, 1);     // S_0 = Q_0
      pass(spmm_fn(), K_SPMM_GRAM, E, 0, base().S);   // A S_0, gram S^T A S
      reduce(E, h->ctrl);
    }
  }
  bool uexpl = false;
  void iteration() {
    const int E = tri_count(p);
    if (method == BLCOC_COCR_RQ && uexpl) {
      small(SK_ALPHA, E);
      pass(K->cocr_passA, K_COCR_A, E, 0);
      reduce(E, h->ctrl);
      chol_stage(E);
      second_qr(false);
      fallback_qr(false);
      pass(spmm_fn(), K_SPMM_GRAM, E, 0);            // Y = A W, gram W^T Y (for H+ of the beta' step)
      reduce(E, h->ctrl);
      small(SK_COCR_BETA, E);
      pass(K->cocr_passC, K_COCR_C, 0, 4);               // Q, X, S (no U recurrence)
      {
        PassArgs a = base();
        a.W = a.S;                                       // gather S_{m+1}
        a.V = a.U;                                       // U_{m+1} = A S_{m+1}
        a.ne = E;
        a.flag = 4;                                      // gram U^T U
        a.grid = K->grid(h->n, K_SPMM_GRAM, sms());
        Timer t;
        const bool timed = time_only < 0;
        if (timed) timed_begin(t, K_SPMM_GRAM);
        spmm_fn()(a, h->s);
        if (timed) timed_end(t);
        ++launches;
        last_grid = a.grid;
      }
      reduce(E, h->ctrl);
    } else if (method == BLCOC_COCR_RQ) {
      small(SK_ALPHA, E);
      pass(K->cocr_passA, K_COCR_A, E, 0);
      reduce(E, h->ctrl);
      chol_stage(E);
      second_qr(false);
      fallback_qr(false);
      pass(spmm_fn(), K_SPMM_GRAM, E, 1);
      reduce(E, h->ctrl);
      small(SK_COCR_BETA, E);
      pass(K->cocr_passC, K_COCR_C, E, 0);
      reduce(E, h->ctrl);
    } else {
      small(SK_ALPHA, E);
      pass(K->cocg_pass1, K_COCG_1, 2 * E, 0);
      reduce(2 * E, h->ctrl);
      chol_stage(2 * E);
      second_qr(false);
      fallback_qr(false);
      pass(K->cocg_pass2, K_COCG_2, 0, 0);
      pass(spmm_fn(), K_SPMM_GRAM, E, 0, base().S);   // A S_{m+1}, gram S^T A S
      reduce(E, h->ctrl);
    }
  }
  void true_residual() {
    const int E = tri_count(p);
    PassArgs a = base();
    a.ne = 2 * E + 1;
    a.flag = 1 | 16;   // norm only, run after the solve finished
    a.grid = K->grid(h->n, K_RESID, h->num_sms);
    K->resid(a, h->s);
    ++launches;
    launch_reduce(h->partials, a.grid, 2 * E + 1, h->stage1, nullptr, h->s);
    ++launches;
    launch_small(SK_TRR, p, method, h->stage1, 2 * E + 1, h->mats, h->ctrl, h->hist, h->s);
    ++launches;
  }
};

// Control-block fields of the shifted-CholQR3 fallback: on, and the shift coefficient
// 11 (n p + p (p + 1)) u of Fukaya et al. (applied to trace(W^H W) >= ||W||_2^2).
void set_qr_fallback(Ctrl& c, int on, int64_t n, int p) {
  c.qr_fb_on = on;
  c.qr_fb = 0;
  c.qr_shift = on ? 11.0 * ((double)n * p + (double)p * (p + 1)) * 0x1p-53 : 0.0;
}

bool is_host_ptr(const void* ptr) {
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace

extern "C" {

const char* blcoc_status_string(blcoc_status s) {
  switch (s) {
    case BLCOC_OK: return "BLCOC_OK";
    case BLCOC_ERR_INVALID_ARG: return "BLCOC_ERR_INVALID_ARG";
    case BLCOC_ERR_NOT_SYMMETRIC: return "BLCOC_ERR_NOT_SYMMETRIC";
    case BLCOC_ERR_CUDA: return "BLCOC_ERR_CUDA";
    case BLCOC_ERR_OOM: return "BLCOC_ERR_OOM";
    case BLCOC_NOT_CONVERGED: return "BLCOC_NOT_CONVERGED";
    case BLCOC_BREAKDOWN: return "BLCOC_BREAKDOWN";
    case BLCOC_ERR_TIMEOUT: return "BLCOC_ERR_TIMEOUT";
  }
  return "BLCOC_UNKNOWN";
}

const char* blcoc_last_error(blcoc_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

blcoc_status blcoc_destroy(blcoc_handle h) {
  if (!h) return BLCOC_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->dev);
  if (h->s) cudaStreamSynchronize(h->s);
  h->graph.reset();
  free_ws(h);
  free_ws32(h);
  if (h->vaf) cudaFree(h->vaf);
  if (h->ozbuf) cudaFree(h->ozbuf);
  if (h->Bst) cudaFree(h->Bst);
  if (h->Xst) cudaFree(h->Xst);
  if (h->rp) cudaFree(h->rp);
  if (h->ci) cudaFree(h->ci);
  if (h->va) cudaFree(h->va);
  if (h->hist) cudaFree(h->hist);
  if (h->ctrl) cudaFree(h->ctrl);
  if (h->flags) cudaFree(h->flags);
  if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  if (h->ev) cudaEventDestroy(h->ev);
  if (h->s) cudaStreamDestroy(h->s);
  if (h->sbody) cudaStreamDestroy(h->sbody);
  delete h;
  cudaSetDevice(cur);
  return BLCOC_OK;
}

blcoc_status blcoc_create(blcoc_handle* out, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                          const void* vals, int host_ptrs, void* cuda_stream) {
  if (!out) return invalid(nullptr, "out is NULL");
  *out = nullptr;
  if (n < 1 || nnz < 1 || nnz >= (int64_t)1 << 31 || n >= (int64_t)1 << 31)
    return invalid(nullptr, "n and nnz must satisfy 1 <= n, nnz < 2^31");
  if (!row_ptr || !col_idx || !vals) return invalid(nullptr, "CSR pointer is NULL");
  blcoc_ctx* h = new blcoc_ctx();
  blcoc_status st = BLCOC_OK;
  auto fail = [&](blcoc_status s) {
    if (s != BLCOC_OK) {
      g_create_error = h->err;
      blcoc_destroy(h);
    }
    return s;
  };
#define CKC(call)                                                   \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return fail(cuda_fail(h, e_, #call));    \
  } while (0)
  CKC(cudaGetDevice(&h->dev));
  CKC(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev));
  h->user_stream = (cudaStream_t)cuda_stream;
  h->n = n;
  h->nnz = nnz;
  CKC(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
  CKC(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming));
  CKC(cudaMalloc(&h->rp, (n + 1) * sizeof(int)));
  CKC(cudaMalloc(&h->ci, nnz * sizeof(int)));
  CKC(cudaMalloc(&h->va, nnz * sizeof(double2)));
  CKC(cudaMalloc(&h->ctrl, sizeof(Ctrl)));
  CKC(cudaMalloc(&h->flags, 4 * sizeof(int)));
  CKC(cudaMallocHost(&h->h_ctrl, sizeof(Ctrl)));
  const cudaMemcpyKind kind = host_ptrs ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CKC(cudaEventRecord(h->ev, h->user_stream));
  CKC(cudaStreamWaitEvent(h->s, h->ev, 0));
  CKC(cudaMemcpyAsync(h->rp, row_ptr, (n + 1) * sizeof(int), kind, h->s));
  CKC(cudaMemcpyAsync(h->ci, col_idx, nnz * sizeof(int), kind, h->s));
  CKC(cudaMemcpyAsync(h->va, vals, nnz * sizeof(double2), kind, h->s));
  CKC(cudaMemsetAsync(h->flags, 0, 4 * sizeof(int), h->s));
  launch_validate(n, nnz, h->rp, h->ci, h->va, h->flags, 0, h->s);
  CKC(cudaGetLastError());
  int hf[4] = {0, 0, 0, 0};
  CKC(cudaMemcpyAsync(hf, h->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CKC(cudaStreamSynchronize(h->s));
  if (hf[0] != 0) {
    h->err = "CSR structure invalid: row_ptr must start at 0, be non-decreasing and end at nnz; col_idx must be in "
             "[0,n) and strictly increasing within each row";
    return fail(BLCOC_ERR_INVALID_ARG);
  }
  launch_validate(n, nnz, h->rp, h->ci, h->va, h->flags, 1, h->s);
  CKC(cudaGetLastError());
  CKC(cudaMemcpyAsync(hf, h->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CKC(cudaStreamSynchronize(h->s));
  if (hf[1] != 0) {
    h->err = "A is not symmetric: some a_ij has no a_ji or |a_ij - a_ji| > 1e-12 max(|a_ij|, |a_ji|)";
    return fail(BLCOC_ERR_NOT_SYMMETRIC);
  }
  prepare_small_kernels();
  (void)st;
#undef CKC
  *out = h;
  return BLCOC_OK;
}

blcoc_status blcoc_set_values(blcoc_handle h, const void* vals, int host_ptrs) {
  if (!h || !vals) return invalid(h, "NULL argument");
  CK(h, cudaSetDevice(h->dev));
  CK(h, cudaEventRecord(h->ev, h->user_stream));
  CK(h, cudaStreamWaitEvent(h->s, h->ev, 0));
  CK(h, cudaMemcpyAsync(h->va, vals, h->nnz * sizeof(double2),
                        host_ptrs ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->s));
  CK(h, cudaMemsetAsync(h->flags, 0, 4 * sizeof(int), h->s));
  launch_validate(h->n, h->nnz, h->rp, h->ci, h->va, h->flags, 1, h->s);
  CK(h, cudaGetLastError());
  int hf[4] = {0, 0, 0, 0};
  CK(h, cudaMemcpyAsync(hf, h->flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(h, cudaStreamSynchronize(h->s));
  if (hf[1] != 0) {
    h->err = "A is not symmetric: some |a_ij - a_ji| > 1e-12 max(|a_ij|, |a_ji|)";
    return BLCOC_ERR_NOT_SYMMETRIC;
  }
  if (h->vaf) {   // keep the complex64 copy in step
    k_vals_to_c64<<<h->num_sms * 4, 256, 0, h->s>>>(h->va, h->vaf, h->nnz);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->s));
  }
  return BLCOC_OK;
}

blcoc_status blcoc_sampled_grad(blcoc_handle h, const void* Lambda, const void* X, int p, void* grad_vals) {
  if (!h || !Lambda || !X || !grad_vals) return invalid(h, "NULL argument");
  if (p < 1 || p > BLCOC_MAX_P) return invalid(h, "p must be in [1, 32]");
  CK(h, cudaSetDevice(h->dev));
  CK(h, cudaEventRecord(h->ev, h->user_stream));
  CK(h, cudaStreamWaitEvent(h->s, h->ev, 0));
  launch_sampled_grad(h->n, h->rp, h->ci, (const double2*)Lambda, (const double2*)X, p, (double2*)grad_vals,
                      h->num_sms, h->s);
  CK(h, cudaGetLastError());
  CK(h, cudaEventRecord(h->ev, h->s));
  CK(h, cudaStreamWaitEvent(h->user_stream, h->ev, 0));
  CK(h, cudaStreamSynchronize(h->s));
  return BLCOC_OK;
}

blcoc_status blcoc_set_option(blcoc_handle h, const char* key, int64_t value) {
  if (!h || !key) return invalid(h, "NULL handle or key");
  if (!strcmp(key, "graph")) {
    if (value != 0 && value != 1) return invalid(h, "graph must be 0 or 1");
    h->use_graph = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "graph_conditional")) {
    if (value != 0 && value != 1) return invalid(h, "graph_conditional must be 0 or 1");
    if (h->cond_ok != (int)value) h->graph.reset();
    h->cond_ok = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "timing")) {
    if (value < 0 || value > 3) return invalid(h, "timing must be 0, 1, 2 or 3");
    if (h->timing != (int)value) h->graph.reset();
    h->timing = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "inner_tol_exp")) {
    if (value < -15 || value > -1) return invalid(h, "inner_tol_exp must be in [-15, -1]");
    h->inner_tol_exp = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "inner_maxit")) {
    if (value < 0 || value > (1 << 30)) return invalid(h, "inner_maxit must be >= 0");
    h->inner_maxit = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "outer_maxit")) {
    if (value < 1 || value > 10000) return invalid(h, "outer_maxit must be in [1, 10000]");
    h->outer_maxit = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "poll")) {
    if (value < 1 || value > 4096) return invalid(h, "poll must be in [1, 4096]");
    if (h->poll != (int)value) h->graph.reset();
    h->poll = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "fp64_tc")) {
    if (value != 0 && value != 1) return invalid(h, "fp64_tc must be 0 or 1");
    h->graph.reset();
    h->fp64_tc = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "u_explicit") || !strcmp(key, "u_explicit_mixed")) {
    if (value != 0 && value != 1) return invalid(h, "u_explicit must be 0 or 1");
    h->graph.reset();
    (key[10] == 0 ? h->u_explicit : h->u_explicit_mixed) = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "spmm_split")) {
    if (value != 0 && value != 1 && value != 2 && value != 4) return invalid(h, "spmm_split must be 0, 1, 2 or 4");
    h->graph.reset();
    h->spmm_split = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "qr_fallback")) {
    if (value != 0 && value != 1) return invalid(h, "qr_fallback must be 0 or 1");
    h->graph.reset();
    h->qr_fallback = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "qr_passes")) {
    if (value != 1 && value != 2) return invalid(h, "qr_passes must be 1 or 2");
    h->graph.reset();
    h->qr_passes = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "persistent_timeout_ms")) {
    if (value < 1 || value > 600000) return invalid(h, "persistent_timeout_ms must be in [1, 600000]");
    h->persistent_timeout_ms = (int)value;
    return BLCOC_OK;
  }
  if (!strcmp(key, "persistent_stall")) {
    if (value != 0 && value != 1) return invalid(h, "persistent_stall must be 0 or 1");
    h->persistent_stall = (int)value;
    return BLCOC_OK;
  }
  return invalid(h, "unknown option");
}

blcoc_status blcoc_get_stat(blcoc_handle h, const char* key, int64_t* value) {
  if (!h || !key || !value) return invalid(h, "NULL argument");
  if (!strcmp(key, "launches")) { *value = h->stat_launches; return BLCOC_OK; }
  if (!strcmp(key, "graph_replays")) { *value = h->stat_replays; return BLCOC_OK; }
  if (!strcmp(key, "outer_iters")) { *value = h->outer_iters; return BLCOC_OK; }
  if (!strcmp(key, "persistent_graph")) { *value = h->stat_persistent_graph; return BLCOC_OK; }
  if (!strcmp(key, "spmm_split")) { *value = h->stat_spmm_split; return BLCOC_OK; }
  if (!strcmp(key, "qr_fallbacks")) { *value = h->h_ctrl ? h->h_ctrl->fb_count : 0; return BLCOC_OK; }
  for (int k = 0; k < kNumKinds; ++k) {
    const std::string nm(kKindNames[k]);
    if (("kt_ns." + nm) == key) { *value = (int64_t)(h->kt_ms[k] * 1e6); return BLCOC_OK; }
    if (("kt_n." + nm) == key) { *value = h->kt_n[k]; return BLCOC_OK; }
  }
  return invalid(h, "unknown stat");
}

blcoc_status blcoc_spmm(blcoc_handle h, const void* X, void* Y, int p) {
  if (!h) return invalid(h, "NULL handle");
  if (p < 1 || p > BLCOC_MAX_P) return invalid(h, "p must be in [1, 32]");
  if (!X || !Y || X == Y) return invalid(h, "X, Y must be distinct non-NULL device pointers");
  CK(h, cudaSetDevice(h->dev));
  int PP = 0;
  const KernelSet* K = kernels_for(p, &PP);
  K->prepare();
  PassArgs a{};
  a.A = CsrDev{h->n, h->nnz, h->rp, h->ci, h->va};
  a.p = p;
  a.W = (double2*)X;
  a.V = (double2*)Y;
  a.ctrl = h->ctrl;
  a.flag = 16;
  a.grid = K->grid(h->n, 2, h->num_sms);
  CK(h, cudaEventRecord(h->ev, h->user_stream));
  CK(h, cudaStreamWaitEvent(h->s, h->ev, 0));
  K->spmm_plain(a, h->s);
  CK(h, cudaGetLastError());
  CK(h, cudaStreamSynchronize(h->s));
  return BLCOC_OK;
}

blcoc_status blcoc_residual_norm(blcoc_handle h, const void* B, const void* X, int p, double* out) {
  if (!h) return invalid(h, "NULL handle");
  if (p < 1 || p > BLCOC_MAX_P) return invalid(h, "p must be in [1, 32]");
  if (!B || !X || !out) return invalid(h, "NULL pointer");
  CK(h, cudaSetDevice(h->dev));
  blcoc_status st = ensure_ws(h, p);
  if (st != BLCOC_OK) return st;
  int PP = 0;
  Solver sv{h, kernels_for(p, &PP), PP, p, BLCOC_COCR_RQ, (const double2*)B, (double2*)X};
  sv.K->prepare();
  CK(h, cudaEventRecord(h->ev, h->user_stream));
  CK(h, cudaStreamWaitEvent(h->s, h->ev, 0));
  sv.true_residual();
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->s));
  CK(h, cudaStreamSynchronize(h->s));
  *out = h->h_ctrl->trr;
  return BLCOC_OK;
}

}  // extern "C"

namespace {

// Replays batches of `poll` iterations (captured once as a CUDA graph, or launched
// directly) until the control block reports the end of the solve.  `gkey` identifies
// the kernel sequence of the graph (method and working precision).
blcoc_status run_iterations(blcoc_ctx* h, Solver& sv, const GraphKey& gkey, int maxit) {
  const int batch = h->poll;
  const bool use_graph = h->use_graph != 0;
  std::vector<Timer> direct_timers;
  if (use_graph) {
    Graph& g = h->graph;
    if (!(g.exec && g.p == sv.p && g.key == gkey && g.batch == batch && g.X == sv.X && g.gen == h->gen &&
          g.timing == h->timing)) {
      g.reset();
      h->evnext = 0;
      cudaGraph_t graph = nullptr;
      for (;;) {   // a second capture with plain launches if a conditional node was refused
        CK(h, cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
        const int before = sv.launches;
        g.timers.clear();
        h->evnext = 0;
        sv.timers = h->timing ? &g.timers : nullptr;
        sv.set_timing_mode(h->timing);
        sv.capturing = true;
        for (int i = 0; i < batch; ++i) {
          sv.batch_iter = i;
          sv.iteration();
        }
        sv.capturing = false;
        sv.timers = nullptr;
        g.timing = h->timing;
        g.launches = sv.launches - before;
        sv.launches = before;
        cudaError_t e = cudaStreamEndCapture(h->s, &graph);
        if (sv.cond_failed) {
          if (graph) cudaGraphDestroy(graph);
          graph = nullptr;
          cudaGetLastError();
          h->cond_ok = 0;
          sv.cond_failed = false;
          continue;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        break;
      }
      cudaError_t e = cudaSuccess;
      e = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        g.exec = nullptr;
        return cuda_fail(h, e, "cudaGraphInstantiate");
      }
      g.p = sv.p;
      g.key = gkey;
      g.batch = batch;
      g.X = sv.X;
      g.gen = h->gen;
    }
  }
  int iter_before = 0;
  for (int done_iters = 0;; done_iters += batch) {
    const std::vector<Timer>* timers = nullptr;
    if (use_graph) {
      CK(h, cudaGraphLaunch(h->graph.exec, h->s));
      sv.launches += h->graph.launches;
      h->stat_replays++;
      timers = &h->graph.timers;
    } else {
      direct_timers.clear();
      if (h->timing) {
        h->evnext = 0;
        sv.timers = &direct_timers;
        sv.set_timing_mode(h->timing);
      }
      for (int i = 0; i < batch; ++i) {
        sv.batch_iter = i;
        sv.iteration();
      }
      sv.timers = nullptr;
      CK(h, cudaGetLastError());
      timers = &direct_timers;
    }
    CK(h, cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    if (h->timing && timers) {
      // kernels of iterations past the end returned at once: not counted
      const int ran = h->h_ctrl->iter - iter_before;
      for (const Timer& t : *timers) {
        if (t.iter >= ran) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess) {
          h->kt_ms[t.kind] += ms;
          h->kt_n[t.kind] += 1;
        } else {
          cudaGetLastError();   // timing is best effort; never fail the solve for it
        }
      }
    }
    iter_before = h->h_ctrl->iter;
    if (h->h_ctrl->done) break;
    if (done_iters > maxit + 2 * batch) {
      h->err = "iteration control did not stop";
      return BLCOC_ERR_CUDA;
    }
  }
  return BLCOC_OK;
}

blcoc_status finish_solve(blcoc_ctx* h, Solver& sv, void* X, bool hostX, size_t bytes) {
  if (hostX) CK(h, cudaMemcpyAsync(X, h->Xst, bytes, cudaMemcpyDeviceToHost, h->s));
  CK(h, cudaEventRecord(h->ev, h->s));
  CK(h, cudaStreamWaitEvent(h->user_stream, h->ev, 0));
  CK(h, cudaStreamSynchronize(h->s));
  h->stat_launches = sv.launches;
  return BLCOC_OK;
}

// Mixed precision: iterative refinement whose residual R = B - A X, the
// p x p solves and the Cholesky QR are FP64, and whose inner correction solve A D = R
// (bl_cocr_rq or bl_cocg_rq) runs its SpMM, Grams and block updates in complex64.
blcoc_status solve_mixed(blcoc_ctx* h, const double2* dB, double2* dX, void* X, bool hostX, int p, int inner_method,
                         double tol, int maxit) {
  NvtxRange range("blcoc mixed-precision refinement");
  blcoc_status st = ensure_ws32(h, p);
  if (st != BLCOC_OK) return st;
  const size_t bytes = (size_t)h->n * p * sizeof(double2);
  int PP = 0;
  Solver sv{h, kernels_for(p, &PP, true), PP, p, inner_method, dB, dX};
  sv.K->prepare();
  sv.use_c64_blocks();
  sv.uexpl = h->u_explicit_mixed != 0;
  sv.qr2 = h->qr_passes == 2 ? 1 : 0;
  double2* D = reinterpret_cast<double2*>(h->w32[5]);
  GraphKey gkey;
  gkey.method = inner_method;
  gkey.mixed = 1;
  gkey.uexpl = sv.uexpl ? 1 : 0;
  gkey.qr2 = sv.qr2;
  gkey.split = sv.spmm_split;
  std::vector<double> outer_hist;
  int total_inner = 0, outer = 0, done = 2, last_bd = 0;
  double bnorm = 0.0, relres = 0.0;
  for (;; ++outer) {
    // FP64 residual of the current X, stored in complex64 as the inner right-hand side
    Ctrl c0{};
    const int left = maxit - total_inner;
    c0.maxit = h->inner_maxit > 0 && h->inner_maxit < left ? h->inner_maxit : left;
    c0.tol = std::pow(10.0, (double)h->inner_tol_exp);
    CK(h, cudaMemcpyAsync(h->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, h->s));
    sv.X = dX;
    sv.setup_residual(1);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    const Ctrl c = *h->h_ctrl;
    if (outer == 0) bnorm = std::sqrt(c.pad[0]);
    if (bnorm == 0.0) {   // B = 0: X = 0 solves it exactly
      CK(h, cudaMemsetAsync(dX, 0, bytes, h->s));
      outer_hist.push_back(0.0);
      done = 1;
      relres = 0.0;
      break;
    }
    relres = c.trr / bnorm;
    outer_hist.push_back(relres);
    if (!std::isfinite(relres)) { done = 3; last_bd = 5; break; }
    if (relres <= tol) { done = 1; break; }
    if (total_inner >= maxit || outer >= h->outer_maxit) { done = 2; break; }
    if (c.done == 3) { done = 3; last_bd = c.bd_code; break; }   // residual block without full rank
    CK(h, cudaMemsetAsync(D, 0, (size_t)h->n * p * sizeof(float2), h->s));
    sv.X = D;
    sv.setup_rest();
    CK(h, cudaGetLastError());
    st = run_iterations(h, sv, gkey, c0.maxit);
    if (st != BLCOC_OK) return st;
    const Ctrl ci = *h->h_ctrl;
    total_inner += ci.iter;
    if (ci.done == 3 && ci.iter == 0) { done = 3; last_bd = ci.bd_code; break; }
    // X += D in FP64
    PassArgs a = sv.base();
    a.X = dX;
    a.V = D;
    a.grid = sv.K->grid(h->n, 7, h->num_sms);
    sv.K->axpy(a, h->s);
    ++sv.launches;
    CK(h, cudaGetLastError());
  }
  h->outer_iters = outer;
  h->iters = total_inner;
  h->trr = relres;
  h->relres = relres;
  h->hist_h = outer_hist;
  h->xi_h.assign(2 * p * p, 0.0);
  st = finish_solve(h, sv, X, hostX, bytes);
  if (st != BLCOC_OK) return st;
  switch (done) {
    case 1: return BLCOC_OK;
    case 2: return BLCOC_NOT_CONVERGED;
    default: {
      char buf[128];
      snprintf(buf, sizeof buf, "breakdown in refinement step %d (site %d)", outer, last_bd);
      h->err = buf;
      return BLCOC_BREAKDOWN;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------------ batched solves
namespace {

// SpMM row-bundle autotuner: time the SpMM (it writes the handle's V and partial slots,
// which every solve overwrites) with 1, 2 and 4 lane groups per row and keep the fastest;
// cached per (n, nnz per row, p, FP64 or tensor-core kernel set).
std::mutex g_spmm_mutex;
std::map<std::string, int> g_spmm_cache;

int tune_spmm_split(blcoc_ctx* h, Solver& sv, bool tc) {
  const std::string key = std::to_string(h->n) + "/" + std::to_string((h->nnz * 10 + h->n / 2) / h->n) + "/" +
                          std::to_string(sv.p) + "/" + (tc ? "tc" : "fp64");
  {
    std::lock_guard<std::mutex> lock(g_spmm_mutex);
    auto it = g_spmm_cache.find(key);
    if (it != g_spmm_cache.end()) return it->second;
  }
  PassArgs a = sv.base();
  a.ne = tri_count(sv.p);
  a.flag = 16;   // run whatever the control block says; no T apply
  a.grid = sv.K->grid(h->n, Solver::K_SPMM_GRAM, h->num_sms);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = 1;
  float best_ms = 1e30f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    const int cand[3] = {1, 2, 4};
    for (int c : cand) {
      sv.spmm_split = c;
      LaunchFn f = sv.spmm_fn();
      if (c != 1 && f == sv.K->spmm_gram) continue;   // bundle wider than a warp
      f(a, h->s);                                     // warm-up
      cudaEventRecord(e0, h->s);
      for (int r = 0; r < 3; ++r) f(a, h->s);
      cudaEventRecord(e1, h->s);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  sv.spmm_split = best;
  std::lock_guard<std::mutex> lock(g_spmm_mutex);
  g_spmm_cache[key] = best;
  return best;
}

// Launch shapes chosen by the batch autotuner, per batch signature (form, method, and
// every system's n, nnz and p).
std::mutex g_tune_mutex;
std::map<std::string, int> g_tune_cache;

std::string tune_key(int form, int method, int nsys, const blcoc_handle* hs, const int* p) {
  std::string k = std::to_string(form) + "/" + std::to_string(method);
  for (int i = 0; i < nsys; ++i)
    k += "/" + std::to_string(hs[i]->n) + "," + std::to_string(hs[i]->nnz) + "," + std::to_string(p[i]);
  return k;
}
int tune_lookup(const std::string& k) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune_cache.find(k);
  return it == g_tune_cache.end() ? -1 : it->second;
}
void tune_store(const std::string& k, int v) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[k] = v;
}

// Iterations of a batch in the persistent kernel: one launch (with the copies that arm its
// ring, scheduler state and per-system counters, captured as one CUDA graph) runs every
// system until it stops.  Autotuning: successive calls with the same batch signature try
// the candidate grid sizes (resident CTAs per SM) in turn, then keep the fastest per
// system-iteration.
struct PersTune {
  std::vector<double> ms;   // per candidate; < 0: not tried yet
};
std::map<std::string, PersTune> g_pers_tune;

blcoc_status iterate_persistent(int nsys, const blcoc_handle* hs, std::vector<Solver>& sv, std::vector<char>& live,
                                const int* p, int method, int maxit, int autotune, const std::string& tkey,
                                int64_t* launches, double* total_ms, int64_t* total_iters, std::string* shape_msg) {
  (void)maxit;
  blcoc_ctx* h0 = hs[0];
  int pmax = 1, nlive = 0;
  for (int i = 0; i < nsys; ++i) {
    pmax = p[i] > pmax ? p[i] : pmax;
    nlive += live[i] ? 1 : 0;
  }
  if (nlive == 0) return BLCOC_OK;
  const size_t smem = persistent_smem(pmax, method);
  int occ = 0;
  CK(h0, persistent_ctas_per_sm(smem, &occ));
  if (occ < 1) return invalid(h0, "batched (persistent): the kernel does not fit on an SM");
  const int maxk = occ < 3 ? occ : 3;
  std::vector<int> cand;   // resident CTAs per SM: as many as fit first
  for (int k = maxk; k >= 1; --k) cand.push_back(k);
  int pick = 0, trying = -1;
  if (autotune) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    PersTune& t = g_pers_tune[tkey];
    if (t.ms.size() != cand.size()) t.ms.assign(cand.size(), -1.0);
    for (size_t c = 0; c < cand.size() && trying < 0; ++c)
      if (t.ms[c] < 0) trying = (int)c;
    if (trying >= 0) {
      pick = trying;
    } else {
      for (size_t c = 1; c < cand.size(); ++c)
        if (t.ms[c] < t.ms[pick]) pick = (int)c;
    }
  }
  const int G = cand[pick] * h0->num_sms;

  std::vector<PersSys> hsys(nsys);
  int64_t M = 0;
  for (int i = 0; i < nsys; ++i) {
    hsys[i].a = sv[i].base();
    hsys[i].stage1 = hs[i]->stage1;
    hsys[i].hist = hs[i]->hist;
    hsys[i].pp = sv[i].PP;
    const bool cocr = method == BLCOC_COCR_RQ;
    hsys[i].vg[0] = sv[i].K->grid(hs[i]->n, cocr ? Solver::K_COCR_A : Solver::K_COCG_1, hs[i]->num_sms);
    hsys[i].vg[1] = sv[i].K->grid(hs[i]->n, Solver::K_SPMM_GRAM, hs[i]->num_sms);
    hsys[i].vg[2] = sv[i].K->grid(hs[i]->n, cocr ? Solver::K_COCR_C : Solver::K_COCG_2, hs[i]->num_sms);
    int mx = RED_SPLIT;
    for (int v : hsys[i].vg) mx = v > mx ? v : mx;
    M += mx;
  }
  const unsigned cap = (unsigned)(2 * M + 2 * nsys + 64);
  // pinned image of [scheduler state][per-system counters][ring]
  const size_t off_run = sizeof(SchedState), off_ring = off_run + (size_t)nsys * sizeof(SysRun);
  const size_t bytes = off_ring + (size_t)cap * sizeof(QItem);

  cudaStream_t ms = nullptr;
  PersSys* d_sys = nullptr;
  unsigned char* d_buf = nullptr;
  unsigned char* h_buf = nullptr;
  SchedState* h_done = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  blcoc_status st = BLCOC_OK;
  do {
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&ms, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess ||
        (e = cudaMalloc(&d_sys, nsys * sizeof(PersSys))) != cudaSuccess ||
        (e = cudaMalloc(&d_buf, bytes)) != cudaSuccess ||
        (e = cudaMallocHost(&h_buf, bytes + sizeof(SchedState))) != cudaSuccess) {
      st = cuda_fail(h0, e, "batched (persistent): workspace");
      break;
    }
    h_done = reinterpret_cast<SchedState*>(h_buf + bytes);
    SchedState* hs0 = reinterpret_cast<SchedState*>(h_buf);
    SysRun* hrun = reinterpret_cast<SysRun*>(h_buf + off_run);
    QItem* hring = reinterpret_cast<QItem*>(h_buf + off_ring);
    *hs0 = SchedState{};
    for (unsigned k = 0; k < cap; ++k) hring[k] = QItem{~0ull, (unsigned long long)k, 0, 0, 0, 0};
    unsigned long long tail = 0;
    const int items0 = method == BLCOC_COCR_RQ ? 2 : 1;   // cocr: the alpha' step and the elimination of H_m
    for (int i = 0; i < nsys; ++i) {
      hrun[i] = SysRun{0, live[i] ? items0 : 0};
      if (live[i] && !h0->persistent_stall) {   // the test hook publishes nothing: every wait runs out
        for (int it = 0; it < items0; ++it) {
          hring[tail] = QItem{tail, tail, i, 0, it, 0};
          ++tail;
        }
      }
    }
    hs0->tail = tail;
    hs0->active = nlive;
    for (int i = 0; i < nsys; ++i) {   // the batch stream starts after every setup
      if ((e = cudaEventRecord(hs[i]->ev, hs[i]->s)) != cudaSuccess || (e = cudaStreamWaitEvent(ms, hs[i]->ev, 0)) != cudaSuccess)
        break;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_sys, hsys.data(), nsys * sizeof(PersSys), cudaMemcpyHostToDevice, ms);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ms);
    if (e != cudaSuccess) {
      st = cuda_fail(h0, e, "batched (persistent): system table");
      break;
    }
    SchedState* d_sch = reinterpret_cast<SchedState*>(d_buf);
    SysRun* d_run = reinterpret_cast<SysRun*>(d_buf + off_run);
    QItem* d_ring = reinterpret_cast<QItem*>(d_buf + off_ring);
    const long long tmo = (long long)h0->persistent_timeout_ms * 1000000LL;
    auto enqueue = [&]() -> cudaError_t {
      cudaError_t r = cudaMemcpyAsync(d_buf, h_buf, bytes, cudaMemcpyHostToDevice, ms);
      if (r == cudaSuccess) r = launch_persistent(d_sys, method, d_sch, d_ring, cap, d_run, tmo, G, smem, ms);
      if (r == cudaSuccess) r = cudaMemcpyAsync(h_done, d_sch, sizeof(SchedState), cudaMemcpyDeviceToHost, ms);
      return r;
    };
    bool use_graph = true;
    {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal);
      cudaError_t e2 = e == cudaSuccess ? enqueue() : e;
      cudaError_t e3 = e == cudaSuccess ? cudaStreamEndCapture(ms, &g) : e;
      if (e2 == cudaSuccess && e3 == cudaSuccess) e3 = cudaGraphInstantiate(&exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e2 != cudaSuccess || e3 != cudaSuccess) {
        use_graph = false;
        exec = nullptr;
        cudaGetLastError();
      }
    }
    if ((e = cudaEventRecord(t0, ms)) != cudaSuccess) {
      st = cuda_fail(h0, e, "batched (persistent): event");
      break;
    }
    e = use_graph ? cudaGraphLaunch(exec, ms) : enqueue();
    if (e == cudaSuccess) e = cudaEventRecord(t1, ms);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ms);
    if (e != cudaSuccess) {
      st = cuda_fail(h0, e, "batched (persistent): launch");
      break;
    }
    *launches += 1;
    h0->stat_persistent_graph = use_graph ? 1 : 0;
    if (h_done->err) {
      h0->err = "batched (persistent): a wait for work exceeded persistent_timeout_ms";
      st = BLCOC_ERR_TIMEOUT;
      break;
    }
    float msr = 0.f;
    cudaEventElapsedTime(&msr, t0, t1);
    int64_t its = 0;
    for (int i = 0; i < nsys; ++i) {
      if (!live[i]) continue;
      if ((e = cudaMemcpy(hs[i]->h_ctrl, hs[i]->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost)) != cudaSuccess) break;
      its += hs[i]->h_ctrl->iter;
      live[i] = 0;
    }
    if (e != cudaSuccess) {
      st = cuda_fail(h0, e, "batched (persistent): control blocks");
      break;
    }
    *total_ms += msr;
    *total_iters += its;
    if (autotune && its > 0) {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      PersTune& t = g_pers_tune[tkey];
      if (trying >= 0) t.ms[trying] = msr / (double)its;
    }
    char buf[200];
    snprintf(buf, sizeof buf, "persistent kernel: %d CTAs (%d per SM), dataflow work queue, %s%s", G, cand[pick],
             use_graph ? "CUDA graph" : "direct launch",
             autotune ? (trying >= 0 ? ", autotune: timing this candidate" : ", autotuned") : "");
    *shape_msg = buf;
  } while (false);
  if (exec) cudaGraphExecDestroy(exec);
  if (ms) cudaStreamSynchronize(ms);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (d_sys) cudaFree(d_sys);
  if (d_buf) cudaFree(d_buf);
  if (h_buf) cudaFreeHost(h_buf);
  if (ms) cudaStreamDestroy(ms);
  return st;
}

}  // namespace

extern "C" {

blcoc_status blcoc_solve(blcoc_handle h, const void* B, void* X, int p, blcoc_method method, double tol, int maxit) {
  NvtxRange range("blcoc_solve");
  if (!h) return invalid(h, "NULL handle");
  h->err.clear();
  if (p < 1 || p > BLCOC_MAX_P) return invalid(h, "p must be in [1, 32]");
  if (method != BLCOC_COCG_RQ && method != BLCOC_COCR_RQ && method != BLCOC_COCG_RQ_MIXED &&
      method != BLCOC_COCR_RQ_MIXED && method != BLCOC_COCG && method != BLCOC_COCR)
    return invalid(h, "unknown method");
  if (!(tol >= 0.0) || std::isinf(tol)) return invalid(h, "tol must be finite and >= 0");
  if (maxit < 0) return invalid(h, "maxit must be >= 0");
  if (!B || !X || B == X) return invalid(h, "B and X must be distinct non-NULL pointers");
  CK(h, cudaSetDevice(h->dev));
  blcoc_status st = ensure_ws(h, p);
  if (st != BLCOC_OK) return st;
  if (h->hist_cap < maxit + 1) {
    h->graph.reset();   // a captured graph writes the history through the old pointer
    if (h->hist) cudaFree(h->hist);
    h->hist = nullptr;
    h->hist_cap = 0;
    CK(h, cudaMalloc(&h->hist, (size_t)(maxit + 1) * sizeof(double)));
    h->hist_cap = maxit + 1;
  }
  const size_t bytes = (size_t)h->n * p * sizeof(double2);
  const bool hostB = is_host_ptr(B), hostX = is_host_ptr(X);
  if ((hostB || hostX) && h->st_cap < p) {
    if (h->Bst) cudaFree(h->Bst);
    if (h->Xst) cudaFree(h->Xst);
    h->Bst = h->Xst = nullptr;
    h->st_cap = 0;
    CK(h, cudaMalloc(&h->Bst, (size_t)h->n * p * sizeof(double2)));
    CK(h, cudaMalloc(&h->Xst, (size_t)h->n * p * sizeof(double2)));
    h->st_cap = p;
  }
  CK(h, cudaEventRecord(h->ev, h->user_stream));
  CK(h, cudaStreamWaitEvent(h->s, h->ev, 0));
  const double2* dB = (const double2*)B;
  double2* dX = (double2*)X;
  if (hostB) {
    CK(h, cudaMemcpyAsync(h->Bst, B, bytes, cudaMemcpyHostToDevice, h->s));
    dB = h->Bst;
  }
  if (hostX) {
    CK(h, cudaMemcpyAsync(h->Xst, X, bytes, cudaMemcpyHostToDevice, h->s));
    dX = h->Xst;
  }
  h->stat_replays = 0;
  h->outer_iters = 0;
  for (int k = 0; k < kNumKinds; ++k) {
    h->kt_ms[k] = 0.0;
    h->kt_n[k] = 0;
  }
  if (method == BLCOC_COCG_RQ_MIXED || method == BLCOC_COCR_RQ_MIXED)
    return solve_mixed(h, dB, dX, X, hostX, p, method == BLCOC_COCR_RQ_MIXED ? BLCOC_COCR_RQ : BLCOC_COCG_RQ, tol,
                       maxit);

  const bool plain = method == BLCOC_COCG || method == BLCOC_COCR;
  const int base_method = plain ? (method == BLCOC_COCR ? BLCOC_COCR_RQ : BLCOC_COCG_RQ) : (int)method;
  int PP = 0;
  Solver sv{h, kernels_for(p, &PP), PP, p, base_method, dB, dX};
  const bool tc = h->fp64_tc && !plain && PP >= 8;
  if (tc) {
    if (!h->ozbuf) CK(h, cudaMalloc(&h->ozbuf, (size_t)OZ_NSLOTS * OZ_SLOT_U2 * sizeof(uint2)));
    sv.K = tc_kernels(PP);
    sv.oz = h->ozbuf;
  }
  sv.K->prepare();
  sv.use_fp64_blocks();
  sv.plain = plain ? 1 : 0;
  sv.uexpl = !plain && h->u_explicit != 0;
  sv.qr2 = h->qr_passes == 2 ? 1 : 0;
  sv.qr_fb = (!plain && !sv.qr2 && h->qr_fallback) ? 1 : 0;
  sv.spmm_split = h->spmm_split == 0 ? tune_spmm_split(h, sv, tc) : h->spmm_split;
  h->stat_spmm_split = sv.spmm_fn() == sv.K->spmm_gram ? 1 : sv.spmm_split;
  Ctrl c0{};
  c0.maxit = maxit;
  c0.tol = tol;
  set_qr_fallback(c0, sv.qr_fb, h->n, p);
  CK(h, cudaMemcpyAsync(h->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, h->s));
  {
    NvtxRange r("blcoc setup");
    sv.setup_residual();
  }
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->s));
  CK(h, cudaStreamSynchronize(h->s));
  bool zero_rhs = false;
  if (h->h_ctrl->done == 1 && h->h_ctrl->sumsq_b == 0.0) {
    zero_rhs = true;
    CK(h, cudaMemsetAsync(dX, 0, bytes, h->s));
  } else if (!h->h_ctrl->done) {
    sv.setup_rest();
    CK(h, cudaGetLastError());
    NvtxRange r("blcoc iterations");
    GraphKey gkey;
    gkey.method = (int)method;
    gkey.uexpl = sv.uexpl ? 1 : 0;
    gkey.plain = sv.plain;
    gkey.tc = tc ? 1 : 0;
    gkey.qr2 = sv.qr2;
    gkey.qr_fb = sv.qr_fb;
    gkey.split = h->stat_spmm_split;
    st = run_iterations(h, sv, gkey, maxit);
    if (st != BLCOC_OK) return st;
  }
  // true residual of the returned iterate
  NvtxRange rr("blcoc true residual");
  sv.B = dB;
  sv.X = dX;
  sv.true_residual();
  CK(h, cudaGetLastError());
  CK(h, cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->s));
  CK(h, cudaStreamSynchronize(h->s));
  const Ctrl c = *h->h_ctrl;
  h->iters = zero_rhs ? 0 : c.iter;
  const double nb = std::sqrt(c.sumsq_b);
  h->trr = zero_rhs ? 0.0 : (nb > 0 ? c.trr / nb : NAN);
  h->hist_h.assign(zero_rhs ? 1 : c.nhist, 0.0);
  if (!zero_rhs && c.nhist > 0)
    CK(h, cudaMemcpy(h->hist_h.data(), h->hist, (size_t)c.nhist * sizeof(double), cudaMemcpyDeviceToHost));
  if (zero_rhs) h->relres = 0.0;
  else if (c.done == 3) h->relres = c.nhist > 0 ? h->hist_h[c.nhist - 1] : h->trr;
  else h->relres = c.relres;
  h->xi_h.assign(2 * p * p, 0.0);
  CK(h, cudaMemcpy(h->xi_h.data(), h->mats + M_XI * PMAX * PMAX, (size_t)p * p * sizeof(double2),
                   cudaMemcpyDeviceToHost));
  st = finish_solve(h, sv, X, hostX, bytes);
  if (st != BLCOC_OK) return st;
  if (zero_rhs) return BLCOC_OK;
  switch (c.done) {
    case 1: return BLCOC_OK;
    case 2: return BLCOC_NOT_CONVERGED;
    case 3: {
      char buf[128];
      snprintf(buf, sizeof buf, "breakdown at iteration %d (site %d)", c.iter, c.bd_code);
      h->err = buf;
      return BLCOC_BREAKDOWN;
    }
    default: h->err = "solve ended in an unknown state"; return BLCOC_ERR_CUDA;
  }
}

static blcoc_status solve_batched_impl(int form, int nsys, const blcoc_handle* hs, const void* const* B,
                                       void* const* X, const int* p, blcoc_method method, double tol, int maxit,
                                       int autotune, double* ms_per_iter_out) {
  NvtxRange range(form == 1 ? "blcoc_solve_batched_persistent" : "blcoc_solve_batched");
  if (nsys < 1 || !hs || !B || !X || !p) return invalid(nullptr, "blcoc_solve_batched: NULL argument or nsys < 1");
  if (method != BLCOC_COCG_RQ && method != BLCOC_COCR_RQ) return invalid(nullptr, "batched: rq methods only");
  if (!(tol >= 0.0) || std::isinf(tol) || maxit < 0) return invalid(nullptr, "batched: bad tol or maxit");
  const int dev = hs[0]->dev;
  for (int i = 0; i < nsys; ++i) {
    if (!hs[i] || hs[i]->dev != dev) return invalid(nullptr, "batched: handles must be non-NULL and on one device");
    if (p[i] < 1 || p[i] > BLCOC_MAX_P) return invalid(nullptr, "batched: p must be in [1, 32]");
    if (form == 1 && p[i] > PERSISTENT_PMAX) return invalid(nullptr, "batched (persistent): p must be in [1, 16]");
    if (form == 1 && hs[i] && (hs[i]->qr_passes != 1 || hs[i]->fp64_tc || hs[i]->u_explicit))
      return invalid(nullptr,
                     "batched (persistent): qr_passes = 2, fp64_tc and u_explicit are not supported; use "
                     "blcoc_solve_batched");
    if (!B[i] || !X[i] || B[i] == X[i]) return invalid(nullptr, "batched: B[i], X[i] must be distinct device pointers");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return invalid(nullptr, "batched: each system needs its own handle");
  }
  blcoc_ctx* h0 = hs[0];
  CK(h0, cudaSetDevice(dev));
  std::vector<Solver> sv;
  sv.reserve(nsys);
  std::vector<char> live(nsys, 0);
  for (int i = 0; i < nsys; ++i) {
    blcoc_ctx* h = hs[i];
    h->err.clear();
    blcoc_status st = ensure_ws(h, p[i]);
    if (st != BLCOC_OK) return st;
    if (h->hist_cap < maxit + 1) {
      h->graph.reset();   // a captured graph writes the history through the old pointer
      if (h->hist) cudaFree(h->hist);
      h->hist = nullptr;
      h->hist_cap = 0;
      CK(h, cudaMalloc(&h->hist, (size_t)(maxit + 1) * sizeof(double)));
      h->hist_cap = maxit + 1;
    }
    CK(h, cudaEventRecord(h->ev, h->user_stream));
    CK(h, cudaStreamWaitEvent(h->s, h->ev, 0));
    int PP = 0;
    sv.push_back(Solver{h, kernels_for(p[i], &PP), PP, p[i], (int)method, (const double2*)B[i], (double2*)X[i]});
    // per-system options, as in blcoc_solve: tensor-core block updates, explicit U, CholQR2
    if (form == 0 && h->fp64_tc && PP >= 8) {
      if (!h->ozbuf) CK(h, cudaMalloc(&h->ozbuf, (size_t)OZ_NSLOTS * OZ_SLOT_U2 * sizeof(uint2)));
      sv.back().K = tc_kernels(PP);
      sv.back().oz = h->ozbuf;
    }
    sv.back().K->prepare();
    sv.back().use_fp64_blocks();
    sv.back().qr2 = h->qr_passes == 2 ? 1 : 0;
    sv.back().uexpl = method == BLCOC_COCR_RQ && h->u_explicit != 0;
    // the graph form runs the shifted-CholQR3 fallback as blcoc_solve does; the persistent
    // kernel has no stages for it
    sv.back().qr_fb = (form == 0 && !sv.back().qr2 && h->qr_fallback) ? 1 : 0;
    if (form == 0) {   // SpMM row bundle: the handle's, or timed per (n, nnz/row, p) when autotuning
      const bool tc_i = sv.back().oz != nullptr;
      sv.back().spmm_split = (autotune || h->spmm_split == 0) ? tune_spmm_split(h, sv.back(), tc_i) : h->spmm_split;
      h->stat_spmm_split = sv.back().spmm_fn() == sv.back().K->spmm_gram ? 1 : sv.back().spmm_split;
    }
    Ctrl c0{};
    c0.maxit = maxit;
    c0.tol = tol;
    set_qr_fallback(c0, sv.back().qr_fb, h->n, p[i]);
    CK(h, cudaMemcpyAsync(h->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, h->s));
    sv.back().setup_residual();
    CK(h, cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->s));
  }
  for (int i = 0; i < nsys; ++i) {
    blcoc_ctx* h = hs[i];
    CK(h, cudaStreamSynchronize(h->s));
    if (h->h_ctrl->done == 1 && h->h_ctrl->sumsq_b == 0.0) {
      CK(h, cudaMemsetAsync(X[i], 0, (size_t)h->n * p[i] * sizeof(double2), h->s));
    } else if (!h->h_ctrl->done) {
      sv[i].setup_rest();
      live[i] = 1;
    }
    CK(h, cudaGetLastError());
  }
  int64_t launches = 0;
  double total_ms = 0.0;
  int64_t total_iters = 0;
  blcoc_status st = BLCOC_OK;
  std::string shape_msg;
  const std::string tkey = tune_key(form, (int)method, nsys, hs, p);
  if (form == 0) {
    cudaStream_t main_s = nullptr;
    cudaEvent_t fork_ev = nullptr;
    std::vector<cudaEvent_t> join(nsys, nullptr);
    CK(h0, cudaStreamCreateWithFlags(&main_s, cudaStreamNonBlocking));
    CK(h0, cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    for (auto& e : join) CK(h0, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEvent_t t0, t1;
    CK(h0, cudaEventCreate(&t0));
    CK(h0, cudaEventCreate(&t1));
    for (int i = 0; i < nsys; ++i) {   // the batch stream starts after every setup
      CK(h0, cudaEventRecord(join[i], hs[i]->s));
      CK(h0, cudaStreamWaitEvent(main_s, join[i], 0));
    }
    // one graph: every live system's `poll` iterations as a parallel branch
    auto capture = [&](int poll, int grid_sms, cudaGraphExec_t* exec, int* nlaunch) -> blcoc_status {
      cudaGraph_t graph = nullptr;
      int launches = 0;
      for (;;) {   // a second capture with plain launches if a conditional node was refused
        CK(h0, cudaStreamBeginCapture(main_s, cudaStreamCaptureModeThreadLocal));
        CK(h0, cudaEventRecord(fork_ev, main_s));
        launches = 0;
        bool refused = false;
        for (int i = 0; i < nsys; ++i) {
          if (!live[i]) continue;
          CK(h0, cudaStreamWaitEvent(hs[i]->s, fork_ev, 0));
          sv[i].grid_sms = grid_sms;
          sv[i].capturing = true;
          const int before = sv[i].launches;
          for (int k = 0; k < poll; ++k) sv[i].iteration();
          sv[i].capturing = false;
          launches += sv[i].launches - before;
          sv[i].launches = before;
          refused = refused || sv[i].cond_failed;
          CK(h0, cudaEventRecord(join[i], hs[i]->s));
          CK(h0, cudaStreamWaitEvent(main_s, join[i], 0));
        }
        cudaError_t e = cudaStreamEndCapture(main_s, &graph);
        if (refused) {
          if (graph) cudaGraphDestroy(graph);
          graph = nullptr;
          cudaGetLastError();
          for (int i = 0; i < nsys; ++i) {
            hs[i]->cond_ok = 0;
            sv[i].cond_failed = false;
          }
          continue;
        }
        if (e != cudaSuccess) return cuda_fail(h0, e, "batched: cudaStreamEndCapture");
        break;
      }
      cudaError_t e = cudaSuccess;
      e = cudaGraphInstantiate(exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(h0, e, "batched: cudaGraphInstantiate");
      *nlaunch = launches;
      return BLCOC_OK;
    };
    // candidate launch shapes: grid sized for all / half / a quarter of the SMs (several
    // systems then share the GPU), graph batches of 8, 16 or 32 iterations
    struct Shape { int poll, grid_sms; };
    std::vector<Shape> cand = {{16, h0->num_sms}};
    if (autotune) cand = {{16, h0->num_sms}, {16, h0->num_sms / 2}, {16, h0->num_sms / 4}, {8, h0->num_sms / 2},
                          {32, h0->num_sms / 2}};
    const int cached = autotune ? tune_lookup(tkey) : -1;
    if (cached >= 0 && cached < (int)cand.size()) cand = {cand[cached]};
    size_t ci = 0;
    int best = -1, cur = -1;
    double best_ms = 1e300;
    cudaGraphExec_t exec = nullptr;
    int exec_launches = 0, exec_poll = 0;
    for (int round = 0;; ++round) {
      bool any = false;
      for (int i = 0; i < nsys; ++i) any = any || live[i];
      if (!any) break;
      const int idx = (ci < cand.size()) ? (int)ci : best;
      const Shape sh = cand[idx];
      if (!exec || idx != cur) {   // (re)capture only when the launch shape changes
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        st = capture(sh.poll, sh.grid_sms, &exec, &exec_launches);
        if (st != BLCOC_OK) break;
        exec_poll = sh.poll;
        cur = idx;
      }
      std::vector<int> it_before(nsys);
      for (int i = 0; i < nsys; ++i) it_before[i] = hs[i]->h_ctrl->iter;
      CK(h0, cudaEventRecord(t0, main_s));
      CK(h0, cudaGraphLaunch(exec, main_s));
      CK(h0, cudaEventRecord(t1, main_s));
      launches += exec_launches;
      for (int i = 0; i < nsys; ++i)
        if (live[i]) CK(h0, cudaMemcpyAsync(hs[i]->h_ctrl, hs[i]->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, main_s));
      CK(h0, cudaStreamSynchronize(main_s));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      int64_t its = 0;
      for (int i = 0; i < nsys; ++i)
        if (live[i]) {
          its += hs[i]->h_ctrl->iter - it_before[i];
          if (hs[i]->h_ctrl->done) live[i] = 0;
          if (round > (maxit + exec_poll) / (exec_poll > 0 ? exec_poll : 1) + 8) {
            h0->err = "batched: iteration control did not stop";
            st = BLCOC_ERR_CUDA;
          }
        }
      total_ms += ms;
      total_iters += its;
      if (ci < cand.size()) {   // autotuning round: time per system-iteration
        const double per = its > 0 ? ms / (double)its : 1e300;
        if (per < best_ms) {
          best_ms = per;
          best = (int)ci;
        }
        ++ci;
      }
      if (st != BLCOC_OK) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (autotune && cached < 0 && best >= 0 && st == BLCOC_OK) tune_store(tkey, best);
    if (best >= 0) {
      char buf[160];
      snprintf(buf, sizeof buf, "autotuned launch shape: graph batch %d iterations, grid for %d SMs",
               cand[best].poll, cand[best].grid_sms);
      shape_msg = buf;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    for (auto& e : join) cudaEventDestroy(e);
    cudaEventDestroy(fork_ev);
    cudaStreamDestroy(main_s);
    if (ms_per_iter_out) *ms_per_iter_out = total_iters > 0 ? total_ms / (double)total_iters : 0.0;
  } else {
    st = iterate_persistent(nsys, hs, sv, live, p, (int)method, maxit, autotune, tkey, &launches, &total_ms,
                            &total_iters, &shape_msg);
    if (ms_per_iter_out) *ms_per_iter_out = total_iters > 0 ? total_ms / (double)total_iters : 0.0;
  }
  // finish every system like a single solve: true residual, history, status
  blcoc_status worst = st;
  for (int i = 0; i < nsys && st == BLCOC_OK; ++i) {
    blcoc_ctx* h = hs[i];
    Solver& s1 = sv[i];
    s1.grid_sms = 0;
    s1.true_residual();
    CK(h, cudaMemcpyAsync(h->h_ctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->s));
    CK(h, cudaStreamSynchronize(h->s));
    const Ctrl c = *h->h_ctrl;
    h->iters = c.iter;
    const double nb = std::sqrt(c.sumsq_b);
    h->trr = nb > 0 ? c.trr / nb : 0.0;
    h->hist_h.assign(c.nhist, 0.0);
    if (c.nhist > 0)
      CK(h, cudaMemcpy(h->hist_h.data(), h->hist, (size_t)c.nhist * sizeof(double), cudaMemcpyDeviceToHost));
    h->relres = c.done == 3 ? (c.nhist > 0 ? h->hist_h[c.nhist - 1] : h->trr) : c.relres;
    h->xi_h.assign(2 * p[i] * p[i], 0.0);
    CK(h, cudaEventRecord(h->ev, h->s));
    CK(h, cudaStreamWaitEvent(h->user_stream, h->ev, 0));
    h->stat_launches = launches;
    blcoc_status si = c.done == 1 || nb == 0 ? BLCOC_OK : (c.done == 2 ? BLCOC_NOT_CONVERGED : BLCOC_BREAKDOWN);
    if (si != BLCOC_OK && worst == BLCOC_OK) worst = si;
  }
  if (!shape_msg.empty() && worst == BLCOC_OK && h0) h0->err = shape_msg;
  return worst;
}

blcoc_status blcoc_solve_batched(int nsys, const blcoc_handle* hs, const void* const* B, void* const* X,
                                 const int* p, blcoc_method method, double tol, int maxit, int autotune,
                                 double* ms_per_iter_out) {
  return solve_batched_impl(0, nsys, hs, B, X, p, method, tol, maxit, autotune, ms_per_iter_out);
}

blcoc_status blcoc_solve_batched_persistent(int nsys, const blcoc_handle* hs, const void* const* B, void* const* X,
                                            const int* p, blcoc_method method, double tol, int maxit, int autotune,
                                            double* ms_per_iter_out) {
  return solve_batched_impl(1, nsys, hs, B, X, p, method, tol, maxit, autotune, ms_per_iter_out);
}

blcoc_status blcoc_get_info(blcoc_handle h, int* iters, double* relres_recursive, double* relres_true, double* hist,
                            int hist_len) {
  if (!h) return invalid(h, "NULL handle");
  if (iters) *iters = h->iters;
  if (relres_recursive) *relres_recursive = h->relres;
  if (relres_true) *relres_true = h->trr;
  if (hist && hist_len > 0) {
    const int k = (int)h->hist_h.size() < hist_len ? (int)h->hist_h.size() : hist_len;
    for (int i = 0; i < k; ++i) hist[i] = h->hist_h[i];
  }
  return BLCOC_OK;
}

blcoc_status blcoc_get_xi(blcoc_handle h, double* xi_out) {
  if (!h || !xi_out) return invalid(h, "NULL argument");
  for (size_t i = 0; i < h->xi_h.size(); ++i) xi_out[i] = h->xi_h[i];
  return BLCOC_OK;
}

}  // extern "C"

/*
 * blcoc.h - C ABI of libblcoc.so: block COCG / block COCR with residual
 * orthonormalization for complex symmetric sparse systems, on one GB300 GPU.
 *
 * Problem (Sec. 1, Eq. 1.1): A X = B with A in C^{n x n} complex symmetric
 * (A = A^T, A != A^H), sparse; X, B in C^{n x p}, p << n.
 *
 * Methods: bl_cocg_rq (Algorithm 2, Sec. 2.2) and bl_cocr_rq (Algorithm 3, Sec. 2.2).
 * Every coefficient uses the unconjugated bilinear form Y^T Z (Table 1); only the
 * thin QR of the residual block is orthonormal in the Hermitian sense, Q^H Q = I_p.
 * The QR is computed as a Cholesky QR: tau^H tau = W^H W with tau upper triangular
 * and a real positive diagonal, Q = W tau^{-1} (same factor as a Householder QR whose
 * diagonal is normalised to be real and positive).
 *
 * Data layout
 *   - complex numbers are interleaved (re, im) doubles (C99 double _Complex,
 *     numpy complex128, torch.complex128);
 *   - an n x p block is row-major with row stride p: element (i, j) at offset i*p + j;
 *   - A is CSR with both triangles stored: int32 row_ptr[n+1] (row_ptr[0] = 0,
 *     non-decreasing, row_ptr[n] = nnz < 2^31), int32 col_idx[nnz] strictly
 *     increasing within each row, values vals[nnz].
 *
 * Threading: a handle is not thread safe; use one handle per host thread.
 * Errors: every entry point returns a blcoc_status; nothing throws across the ABI.
 * blcoc_last_error() gives a one-line description of the last failure on a handle.
 */
#ifndef BLCOC_H
#define BLCOC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct blcoc_ctx* blcoc_handle;

typedef enum {
  BLCOC_OK = 0,
  BLCOC_ERR_INVALID_ARG = 1,   /* a size, pointer, method or tolerance is out of range  */
  BLCOC_ERR_NOT_SYMMETRIC = 2, /* create: pattern or values of A are not symmetric       */
  BLCOC_ERR_CUDA = 3,          /* a CUDA runtime call failed (see blcoc_last_error)      */
  BLCOC_ERR_OOM = 4,           /* device allocation failed                               */
  BLCOC_NOT_CONVERGED = 5,     /* maxit iterations ran without reaching tol              */
  BLCOC_BREAKDOWN = 6,         /* the residual block lost rank, a p x p system was
                                  singular, or a coefficient became non-finite          */
  BLCOC_ERR_TIMEOUT = 7        /* reserved: a device wait gave up                        */
} blcoc_status;

/* Methods.  The _MIXED forms are iterative refinement around the rq methods: the residual
 * R = B - A X, the p x p solves and the Cholesky QR are FP64; each correction solve
 * A D = R runs bl_cocg_rq / bl_cocr_rq with complex64 SpMM, Grams and block updates to a
 * relative tolerance 10^inner_tol_exp (blcoc_set_option), then X += D in FP64.  tol is
 * then on the true residual ||B - A X||_F / ||B||_F and maxit bounds the total inner
 * iterations; blcoc_get_info returns the inner iteration count and, as hist, the true
 * relative residual after each refinement step. */
/* BLCOC_COCR is the plain block COCR of Algorithm 1 (Sec. 2.1) and BLCOC_COCG the plain
 * block COCG (Sec. 2.1, Eqs. 2.1-2.2 with Table 1's COCG conditions:
 * alpha = (P^T A P)^{-1} R^T R, beta = (R_m^T R_m)^{-1} R_{m+1}^T R_{m+1}); both stop when
 * ||R_m||_F / ||B||_F <= tol (Algorithm 1 normalises by ||R_0||_F, equal for X0 = 0). */
typedef enum {
  BLCOC_COCG_RQ = 0,
  BLCOC_COCR_RQ = 1,
  BLCOC_COCG_RQ_MIXED = 2,
  BLCOC_COCR_RQ_MIXED = 3,
  BLCOC_COCG = 4,
  BLCOC_COCR = 5
} blcoc_method;

/* Largest number of right-hand sides one solve accepts. */
#define BLCOC_MAX_P 32

/*
 * blcoc_create - upload A and check it.
 *   out       : receives the handle (set to NULL on failure).
 *   n, nnz    : order and number of stored entries, 1 <= n, 1 <= nnz < 2^31.
 *   row_ptr, col_idx, vals : CSR arrays as described above; vals holds 2*nnz doubles.
 *   host_ptrs : 1 if the three arrays are host memory, 0 if device memory.
 *   cuda_stream : a cudaStream_t (NULL = legacy default stream). Every solve first
 *               waits for the work already queued on it; the library runs its own
 *               kernels on an internal stream of the same device.
 * The arrays are deep-copied to the device; the caller keeps ownership of them.
 * Checks (on the GPU): row_ptr monotone, 0 <= col_idx < n, strictly increasing within
 * rows, and for every stored a_ij a stored a_ji with |a_ij - a_ji| <= 1e-12 max(|a_ij|,
 * |a_ji|) (Sec. 1: A = A^T).  Failure: BLCOC_ERR_INVALID_ARG or BLCOC_ERR_NOT_SYMMETRIC.
 * The device is the current CUDA device of the calling thread.
 */
blcoc_status blcoc_create(blcoc_handle* out, int64_t n, int64_t nnz, const int32_t* row_ptr,
                          const int32_t* col_idx, const void* vals, int host_ptrs, void* cuda_stream);

/*
 * blcoc_solve - run Algorithm 2 (BLCOC_COCG_RQ) or Algorithm 3 (BLCOC_COCR_RQ).
 *   B     : n x p right-hand sides (read only).
 *   X     : n x p, on entry the initial guess X_0, on exit the last iterate.
 *   p     : 1 <= p <= BLCOC_MAX_P.
 *   tol   : stop at the top of iteration m when ||xi_m||_F / ||B||_F <= tol
 *           (the test at the top of each iteration of Algorithms 2-3); tol >= 0 (tol = 0
 *           runs exactly maxit iterations).
 *   maxit : maximum number of iterations, maxit >= 0.
 * B and X may be device pointers or host pointers (pageable or pinned); host data is
 * copied through handle-owned device buffers.  B must not alias X.
 * Workspace (about 6 n x p blocks) is owned by the handle and grows to the largest p
 * used.  The call blocks until the solve ends.
 * On return the caller's stream (given at create) is ordered after the solve's work.
 * Returns BLCOC_OK (converged), BLCOC_NOT_CONVERGED, BLCOC_BREAKDOWN (X then holds
 * the last complete iterate), or an error code.  ||B||_F = 0 returns X = 0, OK.
 */
blcoc_status blcoc_solve(blcoc_handle h, const void* B, void* X, int p, blcoc_method method, double tol,
                         int maxit);

/*
 * blcoc_solve_batched - solve nsys independent systems A_i X_i = B_i (one handle each,
 * p[i] right-hand sides) with the same rq method, tol and maxit.  Every system keeps its
 * own workspace, control block and p x p factors; one CUDA graph holds all live systems'
 * next iterations as parallel branches, so one graph launch advances every unconverged
 * system (converged ones return at once) and small systems share the GPU.
 * With autotune != 0 the first rounds run under different launch shapes (row-pass grids
 * sized for all / 1/2 / 1/4 of the SMs, graph batches of 8 / 16 / 32 iterations) and the
 * fastest per system-iteration is kept; blcoc_last_error(hs[0]) then names it.
 * B[i], X[i]: device pointers.  ms_per_iter_out (may be NULL): device time per
 * system-iteration over the whole batch.  Per-system results: blcoc_get_info(hs[i]).
 * Returns BLCOC_OK if every system converged, else the first non-OK status.
 * Each system runs with its own handle's options (fp64_tc, u_explicit, qr_passes,
 * qr_fallback), as blcoc_solve would.
 * The paper solves one system at a time; batching many is this library's addition.
 */
blcoc_status blcoc_solve_batched(int nsys, const blcoc_handle* hs, const void* const* B, void* const* X,
                                 const int* p, blcoc_method method, double tol, int maxit, int autotune,
                                 double* ms_per_iter_out);

/*
 * blcoc_solve_batched_persistent - the same batch (arguments, results and statuses as
 * blcoc_solve_batched; p[i] <= 16, rq methods, handles without the options qr_passes = 2,
 * fp64_tc and u_explicit; the shifted-CholQR3 fallback of option qr_fallback is not run,
 * so a failed Cholesky QR is a breakdown) with every iteration of every system in
 * ONE persistent kernel launch.  An iteration of Algorithm 2 or 3 (Sec. 2.2) is a chain
 * of stages per system (row passes, their reductions, the p x p stages); the items of a
 * stage (a row pass's 32-row chunk groups, the reduction slices, one p x p solve) wait in
 * a ring of work items, the resident CTAs take them as they become ready, and the CTA
 * that finishes a stage publishes the system's next one.  So systems advance
 * independently (per-system work queues), one system's p x p stages overlap the others'
 * row passes, and a system whose stopping test (top of an iteration) has fired publishes
 * nothing more (convergence mask).  The launch and the copies that arm it are one CUDA
 * graph (a direct launch if capture is refused; blcoc_get_stat(hs[0], "persistent_graph")
 * says which).  Each system's iterates, history and residuals are bitwise those of a
 * separate blcoc_solve (with qr_fallback = 0 where that fallback would have run).
 * With autotune != 0, successive calls with the same batch signature (every system's n,
 * nnz and p) time the candidate grid sizes (resident CTAs per SM) in turn and then keep
 * the fastest per system-iteration; blcoc_last_error(hs[0]) names the shape used.
 * Every wait of the kernel (for work, for a free ring slot) gives up after the option
 * "persistent_timeout_ms" of hs[0] (default 10000 ms); the call then returns
 * BLCOC_ERR_TIMEOUT (the handles stay usable; X holds an unfinished iterate).
 * Scratch (a system table, the ring, counters) is allocated per call.  The paper has no
 * batched form.
 */
blcoc_status blcoc_solve_batched_persistent(int nsys, const blcoc_handle* hs, const void* const* B, void* const* X,
                                            const int* p, blcoc_method method, double tol, int maxit, int autotune,
                                            double* ms_per_iter_out);

/*
 * blcoc_get_info - results of the last solve.
 *   iters            : number of iterations taken (the iterate X holds is X_iters).
 *   relres_recursive : ||xi_iters||_F / ||B||_F.
 *   relres_true      : ||B - A X||_F / ||B||_F recomputed from the returned X (Sec. 3,
 *                      "TRR" before the log10).
 *   hist, hist_len   : if hist != NULL, receives min(hist_len, iters + 1) values
 *                      hist[m] = ||xi_m||_F / ||B||_F.
 * Any output pointer may be NULL.
 */
blcoc_status blcoc_get_info(blcoc_handle h, int* iters, double* relres_recursive, double* relres_true,
                            double* hist, int hist_len);

/*
 * blcoc_get_xi - the p x p factor xi_iters of the last solve (R = Q xi, Sec. 2.2),
 * row-major, 2*p*p doubles, written to host memory.
 */
blcoc_status blcoc_get_xi(blcoc_handle h, double* xi_out);

/*
 * blcoc_spmm - Y = A X for an n x p block (the A V product of Algorithms 2-3).
 * X, Y are device pointers, 1 <= p <= BLCOC_MAX_P, Y must not alias X.  Runs on the
 * handle's stream order (waits for the creation stream, returns after completion).
 */
blcoc_status blcoc_spmm(blcoc_handle h, const void* X, void* Y, int p);

/*
 * blcoc_residual_norm - ||B - A X||_F for n x p device blocks B, X (Sec. 3's true
 * residual).  The result is written to *out (host).  Uses handle-owned workspace.
 */
blcoc_status blcoc_residual_norm(blcoc_handle h, const void* B, const void* X, int p, double* out);

/*
 * blcoc_set_values - replace the values of A, keeping its pattern (for example between
 * optimisation steps of the differentiable solve).  vals: nnz complex values in the
 * order of the handle's col_idx; host_ptrs as in blcoc_create.  The symmetry check of
 * blcoc_create is repeated; on BLCOC_ERR_NOT_SYMMETRIC the handle holds the new values
 * and must not be used for solves until valid values are set.
 */
blcoc_status blcoc_set_values(blcoc_handle h, const void* vals, int host_ptrs);

/*
 * blcoc_sampled_grad - the gradient of a real loss through X = A^{-1} B with respect to
 * the stored values of A: grad_vals[e] = - sum_k Lambda[i][k] conj(X[j][k]) for entry e
 * at (i, j), where Lambda = A^{-H} G is the adjoint solution for the upstream gradient G
 * (conjugate-Wirtinger convention; with A = A^T, Lambda = conj(A^{-1} conj(G)), one more
 * solve with the same A).  Lambda, X: n x p device blocks; grad_vals: nnz device values.
 * The paper defines the solve (Sec. 1, Eq. 1.1); its derivative is standard calculus.
 */
blcoc_status blcoc_sampled_grad(blcoc_handle h, const void* Lambda, const void* X, int p, void* grad_vals);

/*
 * blcoc_set_option - tuning switches (key, value):
 *   "graph"      : 1 (default) replays the iteration as a CUDA graph, 0 launches kernels.
 *   "poll"       : iterations between two host checks of the convergence flag (default 16).
 *   "inner_tol_exp": mixed methods: inner relative tolerance 10^value, value in [-15, -1]
 *                  (default -5).
 *   "inner_maxit": mixed methods: iteration limit of one correction solve (0 = the
 *                  remaining budget, default).
 *   "outer_maxit": mixed methods: refinement steps (default 40).
 *   "u_explicit" : BLCOC_COCR_RQ: 1 forms U_{m+1} = A S_{m+1} with a second sparse
 *                  product per iteration instead of Algorithm 3's recurrence
 *                  U_{m+1} = V_{m+1} + U_m beta'_m (equal in exact arithmetic; the
 *                  recurrence is the default, 0).
 *   "fp64_tc"    : BLCOC_COCR_RQ and BLCOC_COCG_RQ with 5 <= p <= 32: 1 runs the p x p
 *                  block updates (right-multiplications by alpha', alpha'xi, beta',
 *                  tau^{-1}) on the bf16 tensor cores by exact integer slicing of both
 *                  operands (eight 7-bit digits, 43 slice products, exact fp32 partial
 *                  sums), to about FP64 accuracy; for BLCOC_COCR_RQ with p <= 16 the Grams
 *                  W^H W and W^T A W as well.  The other Grams, the sparse product and the
 *                  p x p stages stay FP64.  0 (default) computes everything with FP64 FMAs
 *                  (so do p <= 4, the plain methods and the complex64 inner solves).
 *   "u_explicit_mixed": the same for the complex64 inner solves of BLCOC_COCR_RQ_MIXED
 *                  (default 1: the recurrence drifts quickly in single precision).
 *   "qr_passes"  : rq methods: 1 (default) forms the thin QR of W (Sec. 2.2, Q^H Q = I)
 *                  as a Cholesky QR: tau from the Gram W^H W of the pass that forms W,
 *                  Q = W tau^{-1} applied lazily; its orthogonality error grows like
 *                  cond(W)^2 eps.  2: CholQR2 - after every Cholesky QR (setup included)
 *                  one more pass replaces W by Q1 = W tau1^{-1} and forms Q1^H Q1, a second
 *                  Cholesky factor tau2 follows and tau = tau2 tau1 (error about cond(W)
 *                  eps, like a Householder QR).  One extra read/write pass of W per
 *                  iteration.  Not available in blcoc_solve_batched_persistent.
 *   "qr_fallback": rq methods with qr_passes = 1: 1 (default) - when the Cholesky QR of
 *                  a residual block fails (a pivot not above 64 eps of its column's
 *                  squared norm: the block is too ill-conditioned for cond^2 eps), it is
 *                  redone as shifted CholQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto,
 *                  Yanagisawa): Cholesky of W^H W + s I with s = 11 (n p + p(p+1)) u
 *                  trace(W^H W), then two Cholesky QR passes; a breakdown is reported
 *                  only if the resulting factor has a diagonal entry below 1e-14 of its
 *                  largest (the rank test of a Householder QR).  The fallback's six
 *                  kernels run in every iteration and return at once unless it is
 *                  needed (see "graph_conditional").  0: a failed Cholesky QR is a
 *                  breakdown.
 *   "graph_conditional": 1 - in the CUDA graph of the iterations the QR fallback's six
 *                  kernels form the body of a conditional node that the Cholesky stage
 *                  enables only when a fallback has started, so an iteration that needs
 *                  none launches none of them (same results bit for bit).  0 (default):
 *                  plain launches; Nsight Compute does not profile the kernel nodes of a
 *                  graph that can hold conditional nodes.  If the runtime refuses the
 *                  conditional node the option turns itself off.  Also read per handle by
 *                  blcoc_solve_batched.
 *   "spmm_split" : the SpMM's row bundle.  1 (default): p lanes per row (one per column),
 *                  each summing the row's nonzeros in order.  2 or 4: that many lane groups
 *                  split each row's nonzeros (interleaved) and their partial sums are
 *                  combined in a fixed order (where p * split <= 32; otherwise 1).  0: a
 *                  timed sweep of 1 / 2 / 4 on the first solve, cached for the process per
 *                  (n, nonzeros per row, p); blcoc_solve_batched with autotune != 0 also
 *                  tunes it per system.  Results are bitwise reproducible for a given
 *                  bundle.  blcoc_get_stat(h, "spmm_split") reports the bundle used.
 *                  (The persistent batch always uses 1.)
 *   "persistent_timeout_ms": blcoc_solve_batched_persistent (read from hs[0]): limit of
 *                  one wait of the kernel, in [1, 600000] ms (default 10000).
 *   "persistent_stall": blcoc_solve_batched_persistent (read from hs[0]), a test of the
 *                  time limit: 1 publishes no first work item, so every wait for work
 *                  runs out and the call returns BLCOC_ERR_TIMEOUT (0 = off, default).
 *   "timing"     : 1 brackets every kernel of the iterations with CUDA events on
 *                  the internal stream (also inside the graph) and accumulates per-kernel
 *                  device time; 2 brackets only the row-pass kernels (less overhead:
 *                  two event records per pass); 3 only the dominant row pass (pass C of
 *                  bl_cocr_rq, pass 1 of bl_cocg_rq); 0 (default) records nothing.
 * Returns BLCOC_ERR_INVALID_ARG for an unknown key or value.
 */
blcoc_status blcoc_set_option(blcoc_handle h, const char* key, int64_t value);

/* blcoc_get_stat - counters of the last solve: "launches" (kernels launched by the
 * solve, including those inside graph replays), "graph_replays", "outer_iters",
 * "persistent_graph" (last persistent batch: 1 graph replays, 0 direct launches, -1 none),
 * "spmm_split" (SpMM row bundle of the last solve), "qr_fallbacks" (shifted-CholQR3
 * fallbacks started in the last solve)
 * (refinement steps of a mixed solve), and with the
 * "timing" option "kt_ns.<kernel>" (total device nanoseconds) and "kt_n.<kernel>"
 * (launches that did work) for <kernel> in resid, spmm_gram, spmm_plain, cocr_passA,
 * cocr_passC, cocg_pass1, cocg_pass2, reduce, small_setup, small_H0, small_alpha,
 * small_chol, small_beta, small_trr. */
blcoc_status blcoc_get_stat(blcoc_handle h, const char* key, int64_t* value);

/*
 * blcoc_residual_norm_noalloc - ||B - A X||_F, allocating no device memory.
 *
 * For callers that cannot call cudaMalloc (for example code running while a memory
 * pool or caching allocator is held by its owner, or inside another library's
 * allocation-free section): it takes no handle, because creating one allocates.  The
 * paper has no counterpart; the value is the same true residual as
 * blcoc_residual_norm (up to summation order).
 *   n, row_ptr, col_idx, vals : CSR of A in device memory (same layout as blcoc_create;
 *                               not checked here: pass a matrix that blcoc_create accepts).
 *   B, X       : n x p device blocks, 1 <= p <= BLCOC_MAX_P, n < 2^31.
 *   norm_out   : device pointer; receives ||B - A X||_F in norm_out[0].
 *   cuda_stream: stream the two kernels are queued on (NULL = legacy default); the call
 *                returns without waiting for them.
 * Scratch: a static device array of BLCOC_NOALLOC_MAX_CTAS doubles (8 KB) that every
 * GPU loading the library holds until exit; the row pass uses at most that many CTAs, so
 * any n fits.  Each call overwrites the slots it reads; calls that overlap on the GPU
 * (other streams, other threads) race on the shared array.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.
 * Errors: BLCOC_ERR_INVALID_ARG for n or p out of range or a NULL pointer (message in
 * blcoc_last_error(NULL)), BLCOC_ERR_CUDA if the set-up or a launch fails.
 */
#define BLCOC_NOALLOC_MAX_CTAS 1024
blcoc_status blcoc_residual_norm_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                         const void* vals, const void* B, const void* X, int p,
                                         double* norm_out, void* cuda_stream);

/*
 * blcoc_probe_peak - measured FMA throughput of the current device, in flop/s (an FMA
 * counts as 2), for the ALU roofline the row passes are reported against.
 *   kind        : 0 = FP64 (DFMA), 1 = FP32 (FFMA).
 *   flops_per_s : receives the best of three timed launches (after one warm-up) of a
 *                 kernel in which every resident thread runs eight independent FMA chains.
 * Takes about 0.2 s; allocates 8 bytes of device memory and a stream for the call.
 * The paper has no counterpart (a measuring utility).  Errors: BLCOC_ERR_INVALID_ARG,
 * BLCOC_ERR_CUDA / BLCOC_ERR_OOM (message in blcoc_last_error(NULL)).
 */
blcoc_status blcoc_probe_peak(int kind, double* flops_per_s);

/* blcoc_destroy - free the handle and everything it owns.  NULL is accepted. */
blcoc_status blcoc_destroy(blcoc_handle h);

/* blcoc_status_string - static name of a status code. */
const char* blcoc_status_string(blcoc_status s);

/* blcoc_last_error - one-line description of the last failure on h ("" if none);
 * valid until the next call on h.  h = NULL gives the last create failure. */
const char* blcoc_last_error(blcoc_handle h);

#ifdef __cplusplus
}
#endif

#endif /* BLCOC_H */

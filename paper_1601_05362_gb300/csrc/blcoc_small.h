// Host launchers of the p x p kernels, the Gram reduction and the CSR checks.
#pragma once
#include "blcoc_common.cuh"

namespace blcoc {

enum SmallKind { SK_SETUP = 0, SK_COCR_H0, SK_ALPHA, SK_CHOL, SK_COCR_BETA, SK_TRR, SK_SETUP_INNER, SK_CHOL2, SK_CHOL2_SETUP,
                 SK_CHOL_FB, SK_CHOL_FB_SETUP };

void prepare_small_kernels();
// ctrl == nullptr: run even after the solve has finished (final residual pass).
// fb_only: run only while a shifted-CholQR3 fallback is in progress (ctrl->qr_fb > 0).
void launch_reduce(const double2* partials, int nparts, int ne, double* stage1, const Ctrl* ctrl, cudaStream_t s,
                   bool fb_only = false);
// method: 0 cocg / 1 cocr, + 16 for the plain forms, + 32 for CholQR2.
// oz != nullptr: also write the exact-slice fragments of the factors formed (tensor-core
// applies of the FP64 path).  cond (SK_CHOL only, inside a captured graph): the conditional
// node handle the stage sets to 1 when a shifted-CholQR3 fallback has started, 0 otherwise.
void launch_small(SmallKind kind, int p, int method, const double* stage1, int ne, double2* mats, Ctrl* ctrl,
                  double* hist, cudaStream_t s, uint2* oz = nullptr, unsigned long long cond = 0);
void launch_sampled_grad(int64_t n, const int* rp, const int* ci, const double2* Lam, const double2* X, int p,
                         double2* out, int num_sms, cudaStream_t s);
void launch_validate(int64_t n, int64_t nnz, const int* rp, const int* ci, const double2* va, int* flags, int which,
                     cudaStream_t s);

}  // namespace blcoc

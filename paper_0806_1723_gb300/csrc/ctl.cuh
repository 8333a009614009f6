// Device control block of one solve: norms, CG scalars, iteration count, status and
// the relative-residual history.  Written only by single-block kernels.
#pragma once

#include <cuda_runtime.h>

namespace lasto {

constexpr int CTL_HIST = 256;

struct Ctl {
    double bnorm;      // ||b_eff||_2
    double rz;         // <r, z>_vol of the current iteration
    double alpha, beta;
    double rel;        // last relative residual seen by the loop
    double true_rel;   // recomputed ||b - A u|| / ||b_eff|| after the loop
    double tol;        // requested relative tolerance
    double tol_iter;   // tolerance the loop checks (CG: half of tol, so the true residual meets tol)
    int iter, max_iter, status, done;
    // inner FP32 CG of the mixed form (defect correction): scalars of the current inner solve
    double rz_in, alpha_in, beta_in, rr0_in, tol_in, tol_in_eff;
    int iter_in, max_in, outer, go_in;
    double hist[CTL_HIST];
};

enum FinOp {
    FIN_BNORM = 0, FIN_ALPHA = 1, FIN_BETA = 2, FIN_START = 3, FIN_CHECK = 4, FIN_TRUE = 5,
    FIN_IN_START = 6, FIN_IN_ALPHA = 7, FIN_IN_BETA = 8, FIN_IN_CHECK = 9, FIN_OUTER = 10
};

cudaError_t launch_ctl_init(Ctl* ctl, double tol, double tol_iter, int max_iter, cudaStream_t s);

}  // namespace lasto

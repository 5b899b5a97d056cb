// Krylov drivers with the network as preconditioner (solvers.cu) and the
// context helpers they share with the ABI layer (api.cu).
#pragma once

#include <vector>

#include "common.cuh"

namespace mgcnn {

// api.cu: synchronise the context's stream (a fused kernel's timeout flag turns
// into ERR_TIMEOUT); ||v||^2 into the device scalar `slot`; read a device scalar;
// one application e = B r (u_skip: e = u + B r) in the context's precision.
Status sync(mgcnn_ctx* c);
Status sumsq(mgcnn_ctx* c, const double* v, size_t N, int slot);
Status read_scalar(mgcnn_ctx* c, int slot, double* out);
Status vcycle_any(mgcnn_ctx* c, const double* r, double* e, const double* u_skip);

// solvers.cu.  df, du: device arrays (f, and u in: initial guess, out: iterate);
// *iters inner iterations; hist as documented at the ABI entries.
Status krylov_solve(mgcnn_ctx* c, const double* df, double* du, double tol, int maxit, int restart, int* iters,
                    std::vector<double>& hist);
Status pcg_solve(mgcnn_ctx* c, const double* df, double* du, double tol, int maxit, int* iters,
                 std::vector<double>& hist);
Status minres_solve(mgcnn_ctx* c, const double* df, double* du, double tol, int maxit, int* iters,
                    std::vector<double>& hist);

}  // namespace mgcnn

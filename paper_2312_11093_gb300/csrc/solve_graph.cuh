// Device-side solve loop (solve_graph.cu).
#pragma once

#include "common.cuh"

namespace mgcnn {

// fn2_known > 0: ||f||^2, already in the context's scalar slot 1 (not recomputed).
Status solve_on_device(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int* iters,
                       double* relres, bool* used, double fn2_known = -1.0);
void graph_release(mgcnn_ctx* c);

}  // namespace mgcnn

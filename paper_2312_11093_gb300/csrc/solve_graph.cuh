// Device-side solve loop (solve_graph.cu).
#pragma once

#include "common.cuh"

namespace mgcnn {

Status solve_on_device(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int* iters,
                       double* relres, bool* used);
void graph_release(mgcnn_ctx* c);

}  // namespace mgcnn

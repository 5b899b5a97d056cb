// Batched setup / solve of many problems of uneven grid sizes (batch.cu).
#pragma once

#include "common.cuh"
#include "mixed.cuh"

namespace mgcnn {

// Problems of one grid size, stored back to back in every buffer.
struct BatchClass {
  int n = 0, B = 0, L = 0;
  std::vector<int> members;                    // caller's problem indices
  int nl[kMaxLevels] = {};
  DevBuf coef;                                 // [2][B][(n+2)^2] nodal k, level ping-pong
  DevBuf op[kMaxLevels];                       // [B][5][N_l] FP64 operators
  DevBuf s16[kMaxLevels], xa[kMaxLevels], xb[kMaxLevels];  // [B][N_l][8] BF16
  DevBuf xl[kMaxLevels];                                     // low part of the up sweep's output (l >= 1)
  DevBuf dinv32, r32;                          // [B][N] FP32
  DevBuf f, u;                                 // [B][N] FP64
  DevBuf partial;                              // [B][blocks]
  DevBuf rn2, fn2;                             // [B]
  DevBuf alpha;                                // [B][2] input scale of the fused V-cycle
  DevBuf state;                                // int [3][B]: active, iters, status
  DevBuf hist;                                 // [B][maxit + 1]
  DevBuf feat, ca, cb, za, zb, s32;            // FP32 setup scratch
  DevBuf scratch;                              // [B][N] FP64 (autotuning output)
  DevBuf kV, kZ;                               // FGMRES: [restart + 1][B][N] and [restart][B][N] FP64
  DevBuf kpart, kdbl, kint;                    // FGMRES: dot partials, per-problem scalars and matrices, flags
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  FusedLevels fl;
};

void batch_release(mgcnn_ctx* c);
// omega non-null: analytic setup tensors of the 8-channel GMG V(1, 0) network
// (Jacobi weights per level) instead of the setup network
Status setup_batched(mgcnn_ctx* c, int nprob, const double* const* coeff, const int* ns,
                     const LevelWeights* omega = nullptr);
Status solve_batched(mgcnn_ctx* c, int nprob, const double* const* rhs, double* const* u, double tol, int maxit,
                     int* iters, double* relres, int* status);
// batch_krylov.cu: flexible GMRES(restart) of every problem, the batch's network as preconditioner
Status solve_batched_krylov(mgcnn_ctx* c, int nprob, const double* const* rhs, double* const* u, double tol,
                            int maxit, int restart, int* iters, double* relres, int* status);

}  // namespace mgcnn

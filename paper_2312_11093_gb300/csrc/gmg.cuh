// Classical GMG comparator (gmg.cu).
#pragma once

#include "common.cuh"

namespace mgcnn {

struct GmgLevels {
  int L = 0;
  int n[kMaxLevels] = {};
  const double* op[kMaxLevels] = {};   // rediscretised operator per level
  double* r[kMaxLevels] = {};          // right-hand side per level (level 0: the residual)
  double* e[kMaxLevels] = {};          // correction per level (result)
  double* t[kMaxLevels] = {};          // Jacobi ping-pong
};

// level l smooths with weight omega.at(l, g.L)
Status gmg_vcycle(const GmgLevels& g, int l, int nu1, int nu2, const LevelWeights& omega, cudaStream_t st);

}  // namespace mgcnn

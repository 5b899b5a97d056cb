// Training-path buffers and entry points (train.cu).
#pragma once

#include "common.cuh"

namespace mgcnn {

// Per-size batch of training problems: every tensor is [B][N_l][...].
struct TrainGroup {
  int n = 0, B = 0, K = 0, L = 0;
  std::vector<Level> lv;
  DevBuf op[kMaxLevels];                       // FP64 operators [B][5][N_l]
  DevBuf c[kMaxLevels], s[kMaxLevels];         // setup: coef_l, setup_out_l
  DevBuf z[kMaxLevels][kSetupLayers];          // inputs of the setup layers (z[l][0] unused: c[l])
  DevBuf t[kMaxLevels][kSetupLayers];          // tanh outputs of the setup layers
  DevBuf sbar[kMaxLevels], cbar[kMaxLevels], zb[kMaxLevels], tmp[kMaxLevels];
  DevBuf x0[kMaxLevels], xdown[kMaxLevels], xfin[kMaxLevels];
  DevBuf xd[kMaxLevels][kMaxSweeps];           // inputs of the ResNetDown layers
  DevBuf xu[kMaxLevels][kMaxSweeps];           // inputs of the ResNetUp layers (xu[l][0] = pre-up state)
  DevBuf xbf[kMaxLevels], xbd[kMaxLevels], xbt[kMaxLevels];  // adjoints (up, down, scratch)
  DevBuf coef, feat;
  DevBuf rs;                                   // r_0 .. r_K, [K+1][B][N]
  DevBuf gv, ev, eb, rb;                       // g_k, B r_k, e_bar, B^T e_bar
  DevBuf fn2, rn2, npart, wpart;
  DevBuf dinvT, rin;                           // 1/a_C (finest) in T; network input D^{-1} r_k
};

void train_release(mgcnn_ctx* c);
template <typename T>
Status loss_grad_impl(mgcnn_ctx* c, int nprob, const double* const* coeff, const double* const* rhs, const int* ns,
                      int K, double* loss, bool want_grad);
Status adam_step(mgcnn_ctx* c, const double* grad, double lr, double b1, double b2, double eps);

}  // namespace mgcnn

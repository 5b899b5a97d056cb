// Mixed-precision solve phase (BF16 tensors, FP32 accumulation) -- host side.
#pragma once

#include "common.cuh"

namespace mgcnn {

bool mixed_channels_supported(int C);
// Packs the solve-phase weights for the tensor-core kernels (after w64 is set).
Status mixed_set_weights(mgcnn_ctx* c);
// Setup phase in FP32, setup tensors stored BF16 (channel-padded).
Status setup_mixed(mgcnn_ctx* c);
// e = B r (or e = u + B r with u_skip) with r, e in FP64 at the boundary.
Status vcycle_mixed(mgcnn_ctx* c, const double* r, double* e, const double* u_skip);
// Same, from an FP32 residual whose squared norm is already on the device.
Status vcycle_mixed_r32(mgcnn_ctx* c, const float* r32, const double* norm2_dev, double* e, const double* u_skip);
Status mixed_set_setup_level(mgcnn_ctx* c, int l, const double* src);
Status mixed_get_setup_level(mgcnn_ctx* c, int l, double* dst);
// GMG-equivalent setup tensors of level l into the BF16 store.
Status mixed_gmg_setup_level(mgcnn_ctx* c, int l, double omega);
void mixed_release(mgcnn_ctx* c);
// mixed_fused.cu: fused level kernels (8 channels, one layer per ResNet)
constexpr int kFusedVariants = 5;        // tile shapes 16x32, 8x32, 16x16, 32x32, 24x32
class TmaMaps;
struct FusedLevels {
  int L = 0, batch = 1;
  TmaMaps* maps = nullptr;               // tensor-map cache of the owner (context or batch class)
  int* err = nullptr;                    // device flag: a block's tile copies timed out
  float* alpha = nullptr;                // device [batch][2]: input scale alpha and 1 / alpha per problem
  int n[kMaxLevels] = {};
  int var_down[kMaxLevels] = {};         // tile variant per level (autotuned)
  int var_up[kMaxLevels] = {};
  const __nv_bfloat16* s[kMaxLevels] = {};
  __nv_bfloat16* xa[kMaxLevels] = {};
  __nv_bfloat16* xb[kMaxLevels] = {};
};
struct FusedWeights {
  const uint32_t *f_down, *f_up, *f_R;   // mma B fragments (device)
  const uint32_t *f_out_hi, *f_out_lo;   // W_out as an 8 -> 8 layer (output channel 0), BF16 hi + lo parts
  const uint32_t* f_tcnn;                // TCNN by pixel-parity class (taps 0,2 | 6,8 | 1,7 | 3,5 | 4)
  SmallWeights small;                    // by value, see SmallWeights
};
Status fused_vcycle_levels(const FusedLevels& fl, const float* r32, const double* norm2, double* e,
                           const double* u_skip, const FusedWeights& w, const int* active, cudaStream_t st,
                           mgcnn_ctx* prof_ctx);
Status fused_autotune(FusedLevels& fl, const float* r32, const double* norm2, double* scratch,
                      const FusedWeights& w, cudaStream_t st, int reps);
// Pointers into ctx->wmix for the fused kernels (valid after mixed_set_weights).
FusedWeights fused_weights(const mgcnn_ctx* c);
bool fused_supported(const mgcnn_ctx* c);
// setup_fused.cu: Algorithm 2 for 8 channels, one fused kernel per level
struct SetupWeights {
  const uint32_t* frags;      // mma B fragments (device)
  SetupSmallWeights small;    // by value
};
SetupWeights setup_weights(const mgcnn_ctx* c);
Status setup_fused_levels(int L, const int* n, int batch, const double* const* op, __nv_bfloat16* const* s,
                          __nv_bfloat16* const* coef, const SetupWeights& w, int mode, cudaStream_t st);
// [N][C] FP32 -> [N][cp] BF16, zero padded
Status pad_setup_bf16(const float* src, __nv_bfloat16* dst, size_t N, int C, int cp, cudaStream_t st);
Status vcycle_fused_cp8(mgcnn_ctx* c, const float* r32, const double* norm2, double* e, const double* u_skip,
                        const FusedWeights& w);
// Defined in api.cu: Algorithm 2 in FP32 into out[l] ([n_l^2][C] floats).
Status run_setup_net_fp32(mgcnn_ctx* c, float* const* out);

}  // namespace mgcnn

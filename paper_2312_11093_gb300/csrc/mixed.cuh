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
constexpr int kUpVariants = 8;           // the up kernel also: 24x30, 32x30, 22x30 (finest level: rows of 32 layer
                                         // outputs; 22x30 keeps four blocks per SM with both coarse tiles)
constexpr int kTcnnQuadRegs = 16;        // TCNN B fragments per lane: 4 fine pixels x 2 k steps x 2
constexpr int kOutTapRegs = 8;           // W_out B fragments per lane: 2 tap tiles x (hi, lo) x 2 k halves
class TmaMaps;
// Inputs of the finest down kernel when it computes the residual itself.
struct ResidIn {
  const double* u = nullptr;             // n^2
  const double* f = nullptr;             // n^2
  const double* op = nullptr;            // 5 n^2 (a_C, a_W, a_E, a_S, a_N)
  const float* dinv32 = nullptr;         // optional n^2: the network input is D^{-1} r
  double* partial = nullptr;             // per block: sum of r^2 over its owned pixels
};
// Outputs of the finest up kernel when it also forms the next cycle's residual
// from u + e (inputs f, op, dinv32 as in ResidIn).
struct ResidOut {
  const double* f = nullptr;             // n^2
  const double* op = nullptr;            // 5 n^2
  const float* dinv32 = nullptr;         // optional n^2
  float* r32 = nullptr;                  // FP32 D^{-1} r, rows of r32_pitch(n)
  double* partial = nullptr;             // per block: sum of r^2 over its owned pixels
};
struct FusedLevels {
  int L = 0, batch = 1;
  TmaMaps* maps = nullptr;               // tensor-map cache of the owner (context or batch class)
  int* err = nullptr;                    // device flag: a block's tile copies timed out
  float* alpha = nullptr;                // device [batch][2]: input scale alpha and 1 / alpha per problem
  bool pdl = false;                      // launch the level kernels with programmatic dependent launch
  int tail_n = 0;                        // levels of at most this grid side run as one cooperative kernel (0: off)
  unsigned* tail_bar = nullptr;          // that kernel's grid barrier: two zeroed words of the owner's
  int tail_share = 1;                    // tail kernels that may run at once (batch classes): each takes at
                                         // most 1 / tail_share of the resident blocks, so all fit together
  int n[kMaxLevels] = {};
  int var_down[kMaxLevels] = {};         // tile variant per level (autotuned)
  int var_up[kMaxLevels] = {};
  const __nv_bfloat16* s[kMaxLevels] = {};
  __nv_bfloat16* xa[kMaxLevels] = {};
  __nv_bfloat16* xb[kMaxLevels] = {};
  __nv_bfloat16* xbl[kMaxLevels] = {};   // low BF16 part of the up sweep's x_fin (levels >= 1)
};
struct FusedWeights {
  const uint32_t *f_down, *f_up, *f_R;   // mma B fragments (device)
  const uint32_t* f_out_taps;            // W_out by tap (kOutTapWords, see pack_out_taps), BF16 hi + lo parts
  const uint32_t* f_tcnn;                // TCNN of 2 x 2 fine-pixel quads (kTcnnQuadRegs x 32 words)
  SmallWeights small;                    // by value, see SmallWeights
  int out_lo = 1;                        // 0: W_out is exact in BF16 (its lo part is zero), one pass suffices
};
struct FusedCycleOpt {
  bool after_fused_down0 = false;        // the finest down kernel ran already, with the residual fused in
  const ResidOut* resid_out = nullptr;   // the finest up kernel forms the next residual
};
Status fused_vcycle_levels(const FusedLevels& fl, const float* r32, const double* norm2, double* e,
                           const double* u_skip, const FusedWeights& w, const int* active, cudaStream_t st,
                           mgcnn_ctx* prof_ctx, FusedCycleOpt opt = {});
// The finest down kernel with the residual fused in: r = f - A u (FP64) on the
// kernel's tiles, r^2 partial sums (one per block, fused_down0_blocks of them)
// into ra.partial, then the level as usual with the input scale already in
// fl.alpha (fused_set_alpha).  One problem only.
Status fused_down0_resid(const FusedLevels& fl, const ResidIn& ra, const FusedWeights& w, const int* active,
                         cudaStream_t st, mgcnn_ctx* prof_ctx);
Status fused_set_alpha(const FusedLevels& fl, const double* norm2, cudaStream_t st);
int fused_down0_blocks(int n, int variant);  // blocks of a finest-level launch of tile variant `variant`
size_t fused_partials_max(int n);          // the largest fused_down0_blocks over the tile variants
Status fused_autotune(FusedLevels& fl, const float* r32, const double* norm2, double* scratch,
                      const FusedWeights& w, cudaStream_t st, int reps, const ResidIn* ra = nullptr,
                      const ResidOut* ro = nullptr);
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
// The stationary iteration's cycle with the residual fused into the finest down
// kernel (mgcnn_solve, mixed path with the fused kernels):
//   fused_cycle_setup    once per solve: partial-sum space, autotuning, the
//                        input scale from ||f||^2 (device scalar fn2_dev)
//   per cycle k:
//   fused_cycle_residual r_k = f - A u_k and the finest down level; ||r_k||^2
//                        into rn2_dev
//   (convergence test on rn2_dev)
//   fused_cycle_rest     levels 1.. down, all levels up, u += B r_k; the next
//                        input scale from rn2_dev
// `active` (nullable) is the device flag that makes the kernels return at once.
bool fused_residual_applies(const mgcnn_ctx* c);
// MGCNN_OPT_FUSED_RESIDUAL as it applies to this context: 0 separate residual
// pass, 1 residual in the finest down kernel (the functions above), 2 residual in
// the finest up kernel:
//   upres_cycle_setup  once per solve: autotuning, r_0 (stand-alone kernel) and
//                      ||r_0||^2 into rn2_dev
//   per cycle k (after the convergence test on rn2_dev):
//   upres_cycle        the whole V-cycle, u_out = u_in + B r_k, and r_{k+1}
//                      (FP32 copy and ||r_{k+1}||^2 into rn2_dev) formed by the
//                      finest up kernel; u_in and u_out must differ (a tile reads
//                      u_in around its pixels while the neighbours write u_out)
int fused_residual_mode(const mgcnn_ctx* c);
Status upres_cycle_setup(mgcnn_ctx* c, const double* f, const double* u, double* rn2_dev, cudaStream_t st);
Status upres_cycle(mgcnn_ctx* c, const double* f, const double* u_in, double* u_out, double* rn2_dev,
                   const int* active, cudaStream_t st, bool profile);
Status fused_cycle_setup(mgcnn_ctx* c, const double* f, const double* u, const double* fn2_dev);
Status fused_cycle_residual(mgcnn_ctx* c, const double* f, const double* u, double* rn2_dev, const int* active,
                            cudaStream_t st, bool profile);
Status fused_cycle_rest(mgcnn_ctx* c, double* u, const double* rn2_dev, const int* active, cudaStream_t st,
                        bool profile);
// Defined in api.cu: Algorithm 2 in FP32 into out[l] ([n_l^2][C] floats).
Status run_setup_net_fp32(mgcnn_ctx* c, float* const* out);

}  // namespace mgcnn

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
bool fused_supported(const mgcnn_ctx* c);
Status vcycle_fused_cp8(mgcnn_ctx* c, const float* r32, const double* norm2, double* e, const double* u_skip,
                        const uint32_t* f_down, const uint32_t* f_up, const uint32_t* f_R, const float* w_in,
                        const float* w_out, const float* w_P);
// Defined in api.cu: Algorithm 2 in FP32 into out[l] ([n_l^2][C] floats).
Status run_setup_net_fp32(mgcnn_ctx* c, float* const* out);

}  // namespace mgcnn

// Launchers shared between translation units (host-side prototypes).
#pragma once

#include "common.cuh"

namespace mgcnn {

// ---- operator.cu: discretisation, residual, reductions ---------------------
constexpr int kResidualBlock = 256;
constexpr int kReduceBlock = 1024;

// Blocks used by launch_residual / launch_sumsq for N values; the caller
// sizes the partial-sum buffer with it.
inline int reduction_blocks(size_t N) { return grid_for(N, kResidualBlock); }
// The residual kernel's blocks (and partial sums): kResidualPix pixels per thread.
constexpr int kResidualPix = 8;
inline int residual_blocks(size_t N) { return grid_for(N, (size_t)kResidualBlock * kResidualPix); }

// Row pitch (floats) of the FP32 network input r32: rows start on 16-byte
// boundaries so that tiles of it can be copied by TMA.  r32 of a problem is
// n rows of r32_pitch(n) floats (the pad columns are never read).
__host__ __device__ inline int r32_pitch(int n) { return (n + 3) & ~3; }
__host__ __device__ inline size_t r32_floats(int n) { return (size_t)n * r32_pitch(n); }

// batch > 1: problems of the same size stored back to back (blockIdx.y selects one).
// arith: arithmetic instead of geometric full weighting of k (MGCNN_OPT_COARSE_K)
Status launch_restrict_k(const double* k, double* kc, int m, cudaStream_t st, int batch = 1, bool arith = false);
Status launch_inject_mu(const double* mu, double* mc, int n, cudaStream_t st);
Status launch_stencil_div(const double* k, double* op, int n, double bx, double by, cudaStream_t st, int batch = 1);
Status launch_stencil_nondiv(const double* mu, double* op, int n, double vx, double vy, cudaStream_t st);
Status launch_count_bad(const double* v, size_t N, int* count, cudaStream_t st);
template <typename FT>
Status launch_features(const double* op, FT* feat, int n, cudaStream_t st, int batch = 1);
// r = f - A u (FP64), optional FP32 copy r32 (times dinv32 when given; row
// pitch r32_pitch(n)), per-block partial sums of r^2.
// With batch > 1 every array is per problem, back to back; partial is [batch][blocks].
Status launch_residual(const double* f, const double* u, const double* op, double* r, float* r32,
                       double* partial, int n, cudaStream_t st, const float* dinv32 = nullptr, int batch = 1);
// dinv = 1/a_C (FP64, may be null, and FP32) from the first plane of op.
Status launch_diag_inverse(const double* op, double* dinv, float* dinv32, size_t N, cudaStream_t st, int batch = 1);
// per-block partial sums of v^2: residual_blocks(N) of them
Status launch_sumsq(const double* v, size_t N, double* partial, cudaStream_t st);
// out[0] = sum of partial[0..count) in a fixed order (deterministic).
Status launch_reduce(const double* partial, int count, double* out, cudaStream_t st);
// Setup tensors of the networks whose solve phase is classical GMG (weighted
// Jacobi, full weighting, bilinear): the 13-channel V(nu1, nu2) network or the
// 8-channel V(1, 0) network; out [N][channels] FP64.
constexpr int kGmgChannels = 13;
constexpr int kGmgV10Channels = 8;
Status launch_gmg_setup(const double* op, double* out, int n, double omega, cudaStream_t st,
                        bool input_diag_level = false, int channels = kGmgChannels);
// The 8-channel V(1, 0) setup tensors straight into the BF16 [batch][N][8] layout.
Status launch_gmg_v10_setup_bf16(const double* op, __nv_bfloat16* out, int n, double omega, cudaStream_t st,
                                 bool input_diag_level, int batch = 1);
Status launch_axpy_to(const double* u, const double* e, double* out, size_t N, cudaStream_t st);
// Setup tensors of the BPX network (symmetric variant) on level `level`:
// out[p][0] = sqrt(omega 4^level / a_C(p)) / eps with eps = MGCNN_BPX_EPS, the
// other channels 0; out [N][channels] FP64.
Status launch_bpx_setup(const double* op, double* out, int n, int level, double omega, int channels,
                        cudaStream_t st);
// krylov.cu: vector kernels of the Krylov drivers (FP64, fixed-order sums)
size_t krylov_partial_count(size_t N, int nvec);   // doubles of the dots scratch
Status launch_apply_A(const double* op, const double* x, double* y, int n, cudaStream_t st);
// out[i] = <V_i, w>, i < nvec (V: nvec vectors of N back to back)
Status launch_block_dots(const double* V, int nvec, const double* w, size_t N, double* partial, double* out,
                         cudaStream_t st);
// y += sign * sum_i coef[i] V_i (coef on the device)
Status launch_combine(double* y, const double* V, int nvec, const double* coef, double sign, size_t N,
                      cudaStream_t st);
Status launch_scale(const double* x, double* y, double a, size_t N, cudaStream_t st);
// y <- a x + b y (b == 0: y is not read); out <- a x + b y + c z (out may alias y or z)
Status launch_axpby(double* y, const double* x, double a, double b, size_t N, cudaStream_t st);
Status launch_lincomb3(double* out, const double* x, double a, const double* y, double b, const double* z, double c,
                       size_t N, cudaStream_t st);

// ---- net_generic.cu: FP64 / FP32 direct convolution kernels ----------------
template <typename T>
struct ConvArgs {
  const T* x = nullptr;     // input  [N][CI]
  const T* s = nullptr;     // optional per-pixel input scale [N][CI] (Eq. heteroresnet)
  const T* W = nullptr;     // weights [CO][CI][3][3]
  const T* bias = nullptr;  // optional [CO]
  const T* s_out = nullptr;  // optional per-pixel output scale [N][CO], applied before the skip
                            // (the adjoint layer x + s * (K^T x) of the symmetric network)
  const T* skip = nullptr;  // optional residual input [N][CO], added after the activation
  const double* diag = nullptr;  // optional: divide the result by diag[p] (FP64 a_C)
  double out_scale = 1.0;        // multiply the result (after skip) by this constant
  T* y = nullptr;           // output [N][CO]
  int n = 0;                // grid side
  int tanh_act = 0;         // 1: y = tanh(conv + bias) (+ skip)
  // batch of problems of the same size: blockIdx.y selects the problem and
  // each pointer advances by its stride (elements; 0 = shared by the batch)
  int batch = 1;
  size_t x_bs = 0, s_bs = 0, skip_bs = 0, diag_bs = 0, y_bs = 0;   // s_bs also strides s_out
};

template <typename T>
Status conv_same(int CI, int CO, const ConvArgs<T>& a, cudaStream_t st);
// batch > 1: consecutive problems of the same size, tensors back to back.
template <typename T>
Status rcnn(int C, const T* x, const T* W, T* y, int n_fine, cudaStream_t st, int batch = 1);
template <typename T>
Status tcnn_add(int C, const T* xc, const T* W, T* y, int n_fine, cudaStream_t st, int batch = 1);
template <typename T>
Status convert(const double* src, T* dst, size_t count, cudaStream_t st);
bool channels_supported(int C);

}  // namespace mgcnn

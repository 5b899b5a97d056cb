// Direct 3x3 convolutions of the setup and solve networks in FP64 or FP32.
//
// These are the plain per-pixel kernels of the FP64 path (one thread computes
// every output channel of one pixel, all 9 taps x C_in inputs) and of the
// FP32 setup/training path.  Semantics follow PyTorch (Sec. 2.4 of
// arXiv 2312.11093, Eqs. conv and transconv):
//   same:  y[p][co] = sum_{ci,a,b} W[co][ci][a][b] x[p + (a-1, b-1)][ci], zero padding
//   RCNN:  y[J][I][co] = sum W[co][ci][a][b] x[2J+a][2I+b][ci]   (stride 2, no padding)
//   TCNN:  y[2J+a][2I+b][co] += sum_ci W[ci][co][a][b] x[J][I][ci]
// Tensors are pixel-major, channel-minor ([j][i][c]).
#include "ops.cuh"

namespace mgcnn {

template <typename T> __device__ __forceinline__ T dev_tanh(T v);
template <> __device__ __forceinline__ double dev_tanh<double>(double v) { return tanh(v); }
template <> __device__ __forceinline__ float dev_tanh<float>(float v) { return tanhf(v); }

// Same-size 3x3 convolution with the optional pieces of the network's layers:
//   heterogeneous ResNet (Eq. heteroresnet): y = K (s * x) + x        (s, skip)
//   its adjoint (symmetric network):          y = s * (K x) + x        (s_out, skip)
//   NonLinearResNet (Eq. resnet_nonlinear):  y = tanh(K x + b) + x    (bias, tanh, skip)
//   setup output scaling:                    y /= diag                (diag)
template <typename T, int CI, int CO>
__global__ void __launch_bounds__(128) conv_same_kernel(ConvArgs<T> a) {
  const int n = a.n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  const size_t bi = blockIdx.y;
  a.x += bi * a.x_bs;
  if (a.s) a.s += bi * a.s_bs;
  if (a.s_out) a.s_out += bi * a.s_bs;   // same layout as s
  if (a.skip) a.skip += bi * a.skip_bs;
  if (a.diag) a.diag += bi * a.diag_bs;
  a.y += bi * a.y_bs;
  const int j = p / n, i = p - j * n;
  T acc[CO];
#pragma unroll
  for (int co = 0; co < CO; ++co) acc[co] = a.bias ? a.bias[co] : T(0);
  for (int ta = 0; ta < 3; ++ta) {
    const int jj = j + ta - 1;
    if (jj < 0 || jj >= n) continue;
    for (int tb = 0; tb < 3; ++tb) {
      const int ii = i + tb - 1;
      if (ii < 0 || ii >= n) continue;
      const size_t q = (size_t)jj * n + ii;
      const int tap = ta * 3 + tb;
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) {
        T v = a.x[q * CI + ci];
        if (a.s) v *= a.s[q * CI + ci];
#pragma unroll
        for (int co = 0; co < CO; ++co) acc[co] += a.W[(co * CI + ci) * 9 + tap] * v;
      }
    }
  }
#pragma unroll
  for (int co = 0; co < CO; ++co) {
    T v = acc[co];
    if (a.tanh_act) v = dev_tanh<T>(v);
    if (a.s_out) v *= a.s_out[(size_t)p * CO + co];
    if (a.skip) v += a.skip[(size_t)p * CO + co];
    if (a.diag) v = (T)((double)v / a.diag[p]);
    if (a.out_scale != 1.0) v = (T)((double)v * a.out_scale);
    a.y[(size_t)p * CO + co] = v;
  }
}

template <typename T, int C>
__global__ void __launch_bounds__(128) rcnn_kernel(const T* __restrict__ x, const T* __restrict__ W,
                                                   T* __restrict__ y, int n) {
  const int nc = (n - 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc * nc) return;
  x += (size_t)blockIdx.y * n * n * C;
  y += (size_t)blockIdx.y * nc * nc * C;
  const int J = p / nc, I = p - J * nc;
  T acc[C];
#pragma unroll
  for (int co = 0; co < C; ++co) acc[co] = T(0);
  for (int ta = 0; ta < 3; ++ta) {
    for (int tb = 0; tb < 3; ++tb) {
      const size_t q = (size_t)(2 * J + ta) * n + (2 * I + tb);
      const int tap = ta * 3 + tb;
#pragma unroll
      for (int ci = 0; ci < C; ++ci) {
        const T v = x[q * C + ci];
#pragma unroll
        for (int co = 0; co < C; ++co) acc[co] += W[(co * C + ci) * 9 + tap] * v;
      }
    }
  }
#pragma unroll
  for (int co = 0; co < C; ++co) y[(size_t)p * C + co] = acc[co];
}

// Gather form of the transposed convolution: fine pixel (j, i) receives tap
// (a, b) of coarse pixel (J, I) when 2J + a = j and 2I + b = i.
template <typename T, int C>
__global__ void __launch_bounds__(128) tcnn_add_kernel(const T* __restrict__ xc, const T* __restrict__ W,
                                                       T* __restrict__ y, int n) {
  const int nc = (n - 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  xc += (size_t)blockIdx.y * nc * nc * C;
  y += (size_t)blockIdx.y * n * n * C;
  const int j = p / n, i = p - j * n;
  T acc[C];
#pragma unroll
  for (int co = 0; co < C; ++co) acc[co] = T(0);
  for (int ta = 0; ta < 3; ++ta) {
    const int dj = j - ta;
    if (dj < 0 || (dj & 1)) continue;
    const int J = dj >> 1;
    if (J >= nc) continue;
    for (int tb = 0; tb < 3; ++tb) {
      const int di = i - tb;
      if (di < 0 || (di & 1)) continue;
      const int I = di >> 1;
      if (I >= nc) continue;
      const size_t q = (size_t)J * nc + I;
      const int tap = ta * 3 + tb;
#pragma unroll
      for (int ci = 0; ci < C; ++ci) {
        const T v = xc[q * C + ci];
#pragma unroll
        for (int co = 0; co < C; ++co) acc[co] += W[(ci * C + co) * 9 + tap] * v;
      }
    }
  }
#pragma unroll
  for (int co = 0; co < C; ++co) y[(size_t)p * C + co] += acc[co];
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ src, T* __restrict__ dst, size_t count) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) dst[p] = (T)src[p];
}

// 2 channels serve the BPX form of the symmetric network (FP64 only: the mixed
// path has its own list)
bool channels_supported(int C) { return C == 2 || C == 4 || C == 8 || C == 12 || C == 13 || C == 16; }

namespace {

template <typename T, int CI, int CO>
Status conv_same_launch(const ConvArgs<T>& a, cudaStream_t st) {
  conv_same_kernel<T, CI, CO><<<dim3(grid_for((size_t)a.n * a.n, 128), a.batch), 128, 0, st>>>(a);
  MG_LAUNCH("conv_same_kernel");
  return {};
}

// Dispatch a kernel template over the supported hidden-channel counts.
#define MG_DISPATCH_C(C, ...)                                 \
  switch (C) {                                                \
    case 2: { constexpr int CC = 2; __VA_ARGS__; } break;     \
    case 4: { constexpr int CC = 4; __VA_ARGS__; } break;     \
    case 8: { constexpr int CC = 8; __VA_ARGS__; } break;     \
    case 12: { constexpr int CC = 12; __VA_ARGS__; } break;   \
    case 13: { constexpr int CC = 13; __VA_ARGS__; } break;   \
    case 16: { constexpr int CC = 16; __VA_ARGS__; } break;   \
    default: return make_status(MGCNN_ERR_SIZE, "unsupported channel count %d", C); \
  }

}  // namespace

template <typename T>
Status conv_same(int CI, int CO, const ConvArgs<T>& a, cudaStream_t st) {
  if (CI == CO) {
    MG_DISPATCH_C(CI, return (conv_same_launch<T, CC, CC>(a, st)));
  } else if (CI == 1) {
    MG_DISPATCH_C(CO, return (conv_same_launch<T, 1, CC>(a, st)));
  } else if (CO == 1) {
    MG_DISPATCH_C(CI, return (conv_same_launch<T, CC, 1>(a, st)));
  } else if (CI == kFeatures) {
    MG_DISPATCH_C(CO, return (conv_same_launch<T, kFeatures, CC>(a, st)));
  }
  return make_status(MGCNN_ERR_SIZE, "conv_same: unsupported channels %d -> %d", CI, CO);
}

template <typename T>
Status rcnn(int C, const T* x, const T* W, T* y, int n_fine, cudaStream_t st, int batch) {
  const int nc = (n_fine - 1) / 2;
  MG_DISPATCH_C(C, {
    rcnn_kernel<T, CC><<<dim3(grid_for((size_t)nc * nc, 128), batch), 128, 0, st>>>(x, W, y, n_fine);
    MG_LAUNCH("rcnn_kernel");
  });
  return {};
}

template <typename T>
Status tcnn_add(int C, const T* xc, const T* W, T* y, int n_fine, cudaStream_t st, int batch) {
  MG_DISPATCH_C(C, {
    tcnn_add_kernel<T, CC><<<dim3(grid_for((size_t)n_fine * n_fine, 128), batch), 128, 0, st>>>(xc, W, y, n_fine);
    MG_LAUNCH("tcnn_add_kernel");
  });
  return {};
}

template <typename T>
Status convert(const double* src, T* dst, size_t count, cudaStream_t st) {
  convert_kernel<T><<<grid_for(count, 256), 256, 0, st>>>(src, dst, count);
  MG_LAUNCH("convert_kernel");
  return {};
}

template Status conv_same<double>(int, int, const ConvArgs<double>&, cudaStream_t);
template Status conv_same<float>(int, int, const ConvArgs<float>&, cudaStream_t);
template Status rcnn<double>(int, const double*, const double*, double*, int, cudaStream_t, int);
template Status rcnn<float>(int, const float*, const float*, float*, int, cudaStream_t, int);
template Status tcnn_add<double>(int, const double*, const double*, double*, int, cudaStream_t, int);
template Status tcnn_add<float>(int, const float*, const float*, float*, int, cudaStream_t, int);
template Status convert<float>(const double*, float*, size_t, cudaStream_t);
template Status convert<__nv_bfloat16>(const double*, __nv_bfloat16*, size_t, cudaStream_t);

}  // namespace mgcnn

// Vector kernels of the Krylov drivers (MGCNN as a Krylov preconditioner:
// flexible GMRES, and CG / MINRES for the symmetric network): y = A x on the
// finest grid, the dot products of one vector with a block of vectors, linear
// combinations with device coefficients, and axpby / three-term combinations
// with host scalars.
// FP64 throughout; every reduction sums in a fixed order (one partial per block,
// then one block per coefficient), so results repeat bit for bit.
#include "ops.cuh"

namespace mgcnn {

namespace {

constexpr int KB = 256;            // threads per block
constexpr int KPIX = 8;            // pixels per thread
constexpr int KCHUNK = KB * KPIX;  // pixels per block

__device__ __forceinline__ double block_sum_d(double v, double* smem) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();   // smem may still be read by the previous call
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? smem[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y = A x, the 5-point operator (planes a_C, a_W, a_E, a_S, a_N of n^2 each).
__global__ void __launch_bounds__(KB) apply_kernel(const double* __restrict__ op, const double* __restrict__ x,
                                                   double* __restrict__ y, int n) {
  const size_t N = (size_t)n * n;
  const int base = blockIdx.x * KCHUNK + threadIdx.x;
#pragma unroll
  for (int k = 0; k < KPIX; ++k) {
    const int p = base + k * KB;
    if (p >= (int)N) continue;
    const int j = p / n, i = p - j * n;
    double v = op[p] * x[p];
    if (i > 0) v = fma(op[N + p], x[p - 1], v);
    if (i < n - 1) v = fma(op[2 * N + p], x[p + 1], v);
    if (j > 0) v = fma(op[3 * N + p], x[p - n], v);
    if (j < n - 1) v = fma(op[4 * N + p], x[p + n], v);
    y[p] = v;
  }
}

// partial[i * gridDim.x + b] = sum over block b's pixels of V_i[p] w[p], i < nvec
// (nvec <= kMaxDots).  Each thread keeps its KPIX values of w in registers and
// streams the basis vectors past them; a vector's sum is reduced within each
// warp by shuffles (no block-wide barrier per vector, so the loads of the next
// vectors stay in flight), the eight warp sums meet in shared memory once at the
// end and are added in warp order.
constexpr int kMaxDots = 72;
__global__ void __launch_bounds__(KB) dots_partial_kernel(const double* __restrict__ V, int nvec,
                                                          const double* __restrict__ w, size_t N,
                                                          double* __restrict__ partial) {
  __shared__ double wsum[kMaxDots][KB / 32];
  const size_t base = (size_t)blockIdx.x * KCHUNK + threadIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double wv[KPIX];
#pragma unroll
  for (int k = 0; k < KPIX; ++k) {
    const size_t p = base + (size_t)k * KB;
    wv[k] = p < N ? w[p] : 0.0;
  }
#pragma unroll 2
  for (int i = 0; i < nvec; ++i) {
    const double* v = V + (size_t)i * N;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < KPIX; ++k) {
      const size_t p = base + (size_t)k * KB;
      if (p < N) acc = fma(v[p], wv[k], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) wsum[i][warp] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvec; i += KB) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < KB / 32; ++q) t += wsum[i][q];
    partial[(size_t)i * gridDim.x + blockIdx.x] = t;
  }
}

// out[i] = sum_b partial[i * nblk + b], one block per i, fixed order.
__global__ void __launch_bounds__(KB) dots_final_kernel(const double* __restrict__ partial, int nblk,
                                                        double* __restrict__ out) {
  __shared__ double smem[32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += KB) acc += partial[(size_t)blockIdx.x * nblk + b];
  acc = block_sum_d(acc, smem);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// y[p] <- y[p] + sign * sum_i coef[i] V_i[p], the terms added in the order i = 0, 1, ...
// The KPIX pixels of a thread advance together through the vectors, so every
// step of the loop issues KPIX independent loads.
__global__ void __launch_bounds__(KB) combine_kernel(double* __restrict__ y, const double* __restrict__ V, int nvec,
                                                     const double* __restrict__ coef, double sign, size_t N) {
  const size_t base = (size_t)blockIdx.x * KCHUNK + threadIdx.x;
  double acc[KPIX];
#pragma unroll
  for (int k = 0; k < KPIX; ++k) {
    const size_t p = base + (size_t)k * KB;
    acc[k] = p < N ? y[p] : 0.0;
  }
#pragma unroll 2
  for (int i = 0; i < nvec; ++i) {
    const double c = sign * coef[i];
    const double* v = V + (size_t)i * N;
#pragma unroll
    for (int k = 0; k < KPIX; ++k) {
      const size_t p = base + (size_t)k * KB;
      if (p < N) acc[k] = fma(c, v[p], acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < KPIX; ++k) {
    const size_t p = base + (size_t)k * KB;
    if (p < N) y[p] = acc[k];
  }
}

__global__ void __launch_bounds__(KB) scale_kernel(const double* __restrict__ x, double* __restrict__ y, double a,
                                                   size_t N) {
  const size_t p = (size_t)blockIdx.x * KB + threadIdx.x;
  if (p < N) y[p] = a * x[p];
}

// y <- a x + b y; b == 0 does not read y (it may hold anything, NaN included)
__global__ void __launch_bounds__(KB) axpby_kernel(double* __restrict__ y, const double* __restrict__ x, double a,
                                                   double b, size_t N) {
  const size_t p = (size_t)blockIdx.x * KB + threadIdx.x;
  if (p >= N) return;
  y[p] = (b == 0.0) ? a * x[p] : fma(a, x[p], b * y[p]);
}

// out <- a x + b y + c z, the terms added in that order; out may alias y or z
__global__ void __launch_bounds__(KB) lincomb3_kernel(double* out, const double* x, double a, const double* y,
                                                      double b, const double* z, double c, size_t N) {
  const size_t p = (size_t)blockIdx.x * KB + threadIdx.x;
  if (p >= N) return;
  const double v = a * x[p] + b * y[p];
  out[p] = v + c * z[p];
}

int chunks(size_t N) { return (int)((N + KCHUNK - 1) / KCHUNK); }

}  // namespace

size_t krylov_partial_count(size_t N, int nvec) { return (size_t)chunks(N) * nvec; }

Status launch_apply_A(const double* op, const double* x, double* y, int n, cudaStream_t st) {
  apply_kernel<<<chunks((size_t)n * n), KB, 0, st>>>(op, x, y, n);
  MG_LAUNCH("apply_kernel");
  return {};
}

Status launch_block_dots(const double* V, int nvec, const double* w, size_t N, double* partial, double* out,
                         cudaStream_t st) {
  if (nvec < 1 || nvec > kMaxDots) return make_status(MGCNN_ERR_ARG, "%d dot products, at most %d", nvec, kMaxDots);
  const int nb = chunks(N);
  dots_partial_kernel<<<nb, KB, 0, st>>>(V, nvec, w, N, partial);
  MG_LAUNCH("dots_partial_kernel");
  dots_final_kernel<<<nvec, KB, 0, st>>>(partial, nb, out);
  MG_LAUNCH("dots_final_kernel");
  return {};
}

Status launch_combine(double* y, const double* V, int nvec, const double* coef, double sign, size_t N,
                      cudaStream_t st) {
  combine_kernel<<<chunks(N), KB, 0, st>>>(y, V, nvec, coef, sign, N);
  MG_LAUNCH("combine_kernel");
  return {};
}

Status launch_scale(const double* x, double* y, double a, size_t N, cudaStream_t st) {
  scale_kernel<<<grid_for(N, KB), KB, 0, st>>>(x, y, a, N);
  MG_LAUNCH("scale_kernel");
  return {};
}

Status launch_axpby(double* y, const double* x, double a, double b, size_t N, cudaStream_t st) {
  axpby_kernel<<<grid_for(N, KB), KB, 0, st>>>(y, x, a, b, N);
  MG_LAUNCH("axpby_kernel");
  return {};
}

Status launch_lincomb3(double* out, const double* x, double a, const double* y, double b, const double* z, double c,
                       size_t N, cudaStream_t st) {
  lincomb3_kernel<<<grid_for(N, KB), KB, 0, st>>>(out, x, a, y, b, z, c, N);
  MG_LAUNCH("lincomb3_kernel");
  return {};
}

}  // namespace mgcnn

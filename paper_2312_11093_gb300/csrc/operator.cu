// Discretisation (A on every level), FP64 residual and deterministic reductions.
//
// Operator: Remark 2.1 (divergence form) and Sec. 2.5 (non-divergence form)
// of arXiv 2312.11093, 5-point stencil with first-order upwind convection,
// zero Dirichlet boundary (zero padding).  Coarse operators are
// rediscretisations (Sec. 2.3) with the coefficient carried down by full
// weighting of log k (divergence form) or by sampling mu (non-divergence form).
#include <cmath>

#include "fpconv.cuh"
#include "ops.cuh"

namespace mgcnn {

// ---------------------------------------------------------------------------
// Coarse coefficient: log k_c(J, I) = weighted mean of log k over the fine
// nodes (2J + a - 1, 2I + b - 1), weights (1,2,1)x(1,2,1), renormalised over
// the nodes that exist (or, with `arith`, the weighted mean of k itself).
// m = fine nodes per side incl. the ring.
//
// FP64 log and exp cost dozens of FP64-pipe instructions each, and FP64 runs
// at 1/58 of the FP32 rate here, so interior coarse nodes (all nine fine nodes
// present, weights summing to 16) use the equivalent weighted geometric mean
//   k_c = (prod k^w)^(1/16),
// formed from the binary mantissas m in [1, 2) and exponents e of the nine k
// (k = m 2^e): P = prod m^w lies in [1, 2^16), E = sum w e, and
//   k_c = P^(1/16) * 2^(r/16) * 2^q  with E = 16 q + r, 0 <= r < 16,
// P^(1/16) by Newton-Raphson from an FP32 start (root16_newton), 2^(r/16) from
// a table made on the host.
// Ring nodes (renormalised weights) and subnormal k take the log / exp form.
struct Pow2Sixteenths {
  double t[16];   // t[r] = 2^(r/16)
};

__device__ __forceinline__ double split_pow2(double x, int& e) {
  const long long b = __double_as_longlong(x);
  e = (int)((b >> 52) & 0x7ff) - 1023;
  return __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
}

__global__ void restrict_k_kernel(const double* __restrict__ k, double* __restrict__ kc, int m,
                                  const Pow2Sixteenths p2, int arith) {
  const int mc = (m + 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= mc * mc) return;
  k += (size_t)blockIdx.y * m * m;      // problem blockIdx.y of a batch stored back to back
  kc += (size_t)blockIdx.y * mc * mc;
  const int J = p / mc, I = p - J * mc;
  if (arith) {
    // arithmetic full weighting: sum w k / sum w over the fine nodes that exist
    const double w[3] = {1.0, 2.0, 1.0};
    double num = 0.0, den = 0.0;
    for (int a = 0; a < 3; ++a) {
      const int jj = 2 * J + a - 1;
      for (int b = 0; b < 3; ++b) {
        const int ii = 2 * I + b - 1;
        if (jj < 0 || jj >= m || ii < 0 || ii >= m) continue;
        num += w[a] * w[b] * k[(size_t)jj * m + ii];
        den += w[a] * w[b];
      }
    }
    kc[p] = num / den;
    return;
  }
  if (J >= 1 && I >= 1 && 2 * J + 1 < m && 2 * I + 1 < m) {
    const double* k0 = k + (size_t)(2 * J - 1) * m + (2 * I - 1);
    int e[9];
    double v[9];
    bool normal = true;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      v[t] = split_pow2(k0[(size_t)(t / 3) * m + t % 3], e[t]);
      normal = normal && e[t] > -1023;
    }
    if (normal) {
      const double corners = (v[0] * v[2]) * (v[6] * v[8]);
      const double edges = (v[1] * v[3]) * (v[5] * v[7]);
      const double c2 = v[4] * v[4];
      const double P = corners * (edges * edges) * (c2 * c2);
      const int E = (e[0] + e[2] + e[6] + e[8]) + 2 * (e[1] + e[3] + e[5] + e[7]) + 4 * e[4];
      const double root = root16_newton(P);
      const int q = E >> 4, r = E & 15;
      kc[p] = (root * p2.t[r]) * __longlong_as_double((long long)(q + 1023) << 52);
      return;
    }
  }
  const double w[3] = {1.0, 2.0, 1.0};
  double num = 0.0, den = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int jj = 2 * J + a - 1;
    for (int b = 0; b < 3; ++b) {
      const int ii = 2 * I + b - 1;
      if (jj < 0 || jj >= m || ii < 0 || ii >= m) continue;
      num += w[a] * w[b] * log(k[(size_t)jj * m + ii]);
      den += w[a] * w[b];
    }
  }
  kc[p] = exp(num / den);
}

Status launch_restrict_k(const double* k, double* kc, int m, cudaStream_t st, int batch, bool arith) {
  static const Pow2Sixteenths p2 = [] {
    Pow2Sixteenths t{};
    for (int r = 0; r < 16; ++r) t.t[r] = std::exp2(r / 16.0);
    return t;
  }();
  const int mc = (m + 1) / 2;
  restrict_k_kernel<<<dim3(grid_for((size_t)mc * mc, 256), batch), 256, 0, st>>>(k, kc, m, p2, arith ? 1 : 0);
  MG_LAUNCH("restrict_k_kernel");
  return {};
}

__global__ void inject_mu_kernel(const double* __restrict__ mu, double* __restrict__ mc, int n) {
  const int nc = (n - 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc * nc) return;
  const int J = p / nc, I = p - J * nc;
  mc[p] = mu[(size_t)(2 * J + 1) * n + 2 * I + 1];
}

Status launch_inject_mu(const double* mu, double* mc, int n, cudaStream_t st) {
  const int nc = (n - 1) / 2;
  inject_mu_kernel<<<grid_for((size_t)nc * nc, 256), 256, 0, st>>>(mu, mc, n);
  MG_LAUNCH("inject_mu_kernel");
  return {};
}

// ---------------------------------------------------------------------------
// Divergence form: faces carry the harmonic mean of the two nodal k.
//   a_W = -k_w/h^2 - max(bx,0)/h   a_E = -k_e/h^2 + min(bx,0)/h
//   a_S = -k_s/h^2 - max(by,0)/h   a_N = -k_n/h^2 + min(by,0)/h
//   a_C = (k_w + k_e + k_s + k_n)/h^2 + (|bx| + |by|)/h
// Output layout: op[0..N) = a_C, then a_W, a_E, a_S, a_N.
// The constant terms come from the host (StencilConsts); the four harmonic
// means 2 k_c k_o / (k_c + k_o) share one reciprocal of the product of the
// four sums, by Newton-Raphson from an FP32 start (recip_newton: an FP64
// divide is a long FP64-pipe sequence), with the plain divisions as the
// fallback when that product's exponent leaves [-1000, 1000].
struct StencilConsts {
  double ih2;          // 1 / h^2
  double cW, cE, cS, cN, cC;   // max(bx,0)/h, min(bx,0)/h, max(by,0)/h, min(by,0)/h, (|bx|+|by|)/h
};

__global__ void stencil_div_kernel(const double* __restrict__ k, double* __restrict__ op, int n,
                                   const StencilConsts sc) {
  const size_t N = (size_t)n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int)N) return;
  const int j = p / n, i = p - j * n;
  const int m = n + 2;
  k += (size_t)blockIdx.y * m * m;
  op += (size_t)blockIdx.y * 5 * N;
  const double kc = k[(size_t)(j + 1) * m + (i + 1)];
  const double kwn = k[(size_t)(j + 1) * m + i];
  const double ken = k[(size_t)(j + 1) * m + (i + 2)];
  const double ksn = k[(size_t)j * m + (i + 1)];
  const double knn = k[(size_t)(j + 2) * m + (i + 1)];
  const double sW = kc + kwn, sE = kc + ken, sS = kc + ksn, sN = kc + knn;
  const double pWE = sW * sE, pSN = sS * sN;
  const double D = pWE * pSN;
  const double T = kc * (2.0 * sc.ih2);   // 2 k_c / h^2
  double iW, iE, iS, iN;                  // 1 / s_o
  const int ed = (int)((__double_as_longlong(D) >> 52) & 0x7ff) - 1023;
  if (ed >= -1000 && ed <= 1000) {
    const double R = recip_newton(D);
    const double rWE = R * pSN, rSN = R * pWE;   // 1 / (sW sE), 1 / (sS sN)
    iW = sE * rWE;
    iE = sW * rWE;
    iS = sN * rSN;
    iN = sS * rSN;
  } else {
    iW = 1.0 / sW;
    iE = 1.0 / sE;
    iS = 1.0 / sS;
    iN = 1.0 / sN;
  }
  // k_o / h^2 = (2 k_c / h^2) k_o / s_o
  const double kw = T * kwn * iW, ke = T * ken * iE, ks = T * ksn * iS, kn = T * knn * iN;
  op[1 * N + p] = -kw - sc.cW;
  op[2 * N + p] = -ke + sc.cE;
  op[3 * N + p] = -ks - sc.cS;
  op[4 * N + p] = -kn + sc.cN;
  op[p] = (kw + ke) + (ks + kn) + sc.cC;
}

Status launch_stencil_div(const double* k, double* op, int n, double bx, double by, cudaStream_t st, int batch) {
  const double h = 1.0 / (n + 1);
  const StencilConsts sc{1.0 / (h * h), std::fmax(bx, 0.0) / h, std::fmin(bx, 0.0) / h, std::fmax(by, 0.0) / h,
                         std::fmin(by, 0.0) / h, (std::fabs(bx) + std::fabs(by)) / h};
  stencil_div_kernel<<<dim3(grid_for((size_t)n * n, 256), batch), 256, 0, st>>>(k, op, n, sc);
  MG_LAUNCH("stencil_div_kernel");
  return {};
}

// Non-divergence form: (1/h){(mu/h) Lap5 + v_x^+ dx^- + v_x^- dx^+ + v_y^+ dy^- + v_y^- dy^+}.
__global__ void stencil_nondiv_kernel(const double* __restrict__ mu, double* __restrict__ op, int n,
                                      double vx, double vy) {
  const size_t N = (size_t)n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int)N) return;
  const double h = 1.0 / (n + 1);
  const double lap = mu[p] / (h * h);
  op[1 * N + p] = -lap - fmax(vx, 0.0) / h;
  op[2 * N + p] = -lap + fmin(vx, 0.0) / h;
  op[3 * N + p] = -lap - fmax(vy, 0.0) / h;
  op[4 * N + p] = -lap + fmin(vy, 0.0) / h;
  op[p] = 4.0 * lap + (fmax(vx, 0.0) - fmin(vx, 0.0) + fmax(vy, 0.0) - fmin(vy, 0.0)) / h;
}

Status launch_stencil_nondiv(const double* mu, double* op, int n, double vx, double vy, cudaStream_t st) {
  stencil_nondiv_kernel<<<grid_for((size_t)n * n, 256), 256, 0, st>>>(mu, op, n, vx, vy);
  MG_LAUNCH("stencil_nondiv_kernel");
  return {};
}

// Counts entries that are not finite or not > 0 (coefficients must be positive).
__global__ void count_bad_kernel(const double* __restrict__ v, size_t N, int* __restrict__ count) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  int bad = 0;
  if (p < N) {
    const double x = v[p];
    bad = !(isfinite(x) && x > 0.0);
  }
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) atomicAdd(count, 1);
}

Status launch_count_bad(const double* v, size_t N, int* count, cudaStream_t st) {
  MG_CUDA(cudaMemsetAsync(count, 0, sizeof(int), st));
  count_bad_kernel<<<grid_for(N, 256), 256, 0, st>>>(v, N, count);
  MG_LAUNCH("count_bad_kernel");
  return {};
}

// Setup-network input (reading of the Remark "Matrix coefficients as input"):
// [a_W/a_C, a_E/a_C, a_S/a_C, a_N/a_C, log10(h^2 a_C)], layout [N][5].
template <typename FT>
__global__ void features_kernel(const double* __restrict__ op, FT* __restrict__ feat, int n) {
  const size_t N = (size_t)n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int)N) return;
  op += (size_t)blockIdx.y * 5 * N;
  feat += (size_t)blockIdx.y * N * kFeatures;
  if constexpr (sizeof(FT) == sizeof(float)) {
    // FP32 features feed the BF16 network: FP32 arithmetic (FP64 divides and
    // log10 would cost dozens of slow FP64-pipe instructions per node)
    const float np1 = (float)(n + 1);
    const float aC = (float)op[p];
    const float inv = 1.0f / aC;
    feat[(size_t)p * kFeatures + 0] = (float)op[1 * N + p] * inv;
    feat[(size_t)p * kFeatures + 1] = (float)op[2 * N + p] * inv;
    feat[(size_t)p * kFeatures + 2] = (float)op[3 * N + p] * inv;
    feat[(size_t)p * kFeatures + 3] = (float)op[4 * N + p] * inv;
    feat[(size_t)p * kFeatures + 4] = log10f(aC / (np1 * np1));
  } else {
    const double h = 1.0 / (n + 1);
    const double aC = op[p];
    feat[(size_t)p * kFeatures + 0] = (FT)(op[1 * N + p] / aC);
    feat[(size_t)p * kFeatures + 1] = (FT)(op[2 * N + p] / aC);
    feat[(size_t)p * kFeatures + 2] = (FT)(op[3 * N + p] / aC);
    feat[(size_t)p * kFeatures + 3] = (FT)(op[4 * N + p] / aC);
    feat[(size_t)p * kFeatures + 4] = (FT)log10(h * h * aC);
  }
}

template <typename FT>
Status launch_features(const double* op, FT* feat, int n, cudaStream_t st, int batch) {
  features_kernel<FT><<<dim3(grid_for((size_t)n * n, 256), batch), 256, 0, st>>>(op, feat, n);
  MG_LAUNCH("features_kernel");
  return {};
}
template Status launch_features<double>(const double*, double*, int, cudaStream_t, int);
template Status launch_features<float>(const double*, float*, int, cudaStream_t, int);

// ---------------------------------------------------------------------------
// Block-level sum of one double per thread; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* smem) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? smem[threadIdx.x] : 0.0;
  if (warp == 0) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// r = f - A u, FP64 (Eq. 1); per-block partial of sum r^2.
// FP64 runs at 1/58 of the FP32 rate here, so the kernel keeps FP64 work to the
// minimum: five FMAs for f - A u, one for r^2, the FP32 copy converted with
// integer operations (fpconv.cuh), and the block reduction once per
// kResidualPix pixels per thread (thread t of block b takes pixels
// b * kResidualPix * blockDim + k * blockDim + t, k = 0.., summed in that order).
__global__ void __launch_bounds__(kResidualBlock)
residual_kernel(const double* __restrict__ f, const double* __restrict__ u, const double* __restrict__ op,
                double* __restrict__ r, float* __restrict__ r32, double* __restrict__ partial, int n,
                const float* __restrict__ dinv32) {
  __shared__ double smem[32];
  const size_t N = (size_t)n * n;
  {
    const size_t b = blockIdx.y;   // problem of a batch stored back to back
    f += b * N;
    u += b * N;
    op += b * 5 * N;
    if (r) r += b * N;
    if (r32) r32 += b * (size_t)n * ((n + 3) & ~3);
    if (dinv32) dinv32 += b * N;
    partial += b * gridDim.x;
  }
  double rr = 0.0;
  const int base = blockIdx.x * (kResidualPix * kResidualBlock) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < kResidualPix; ++k) {
    const int p = base + k * kResidualBlock;
    if (p < (int)N) {
      const int j = p / n, i = p - j * n;
      const double uW = (i > 0) ? u[p - 1] : 0.0;
      const double uE = (i < n - 1) ? u[p + 1] : 0.0;
      const double uS = (j > 0) ? u[p - n] : 0.0;
      const double uN = (j < n - 1) ? u[p + n] : 0.0;
      double rv = fma(-op[p], u[p], f[p]);
      rv = fma(-op[N + p], uW, rv);
      rv = fma(-op[2 * N + p], uE, rv);
      rv = fma(-op[3 * N + p], uS, rv);
      rv = fma(-op[4 * N + p], uN, rv);
      if (r) r[p] = rv;
      if (r32) {
        const float rf = f64_to_f32_rn(rv);
        r32[(size_t)j * ((n + 3) & ~3) + i] = dinv32 ? rf * dinv32[p] : rf;
      }
      rr = fma(rv, rv, rr);
    }
  }
  rr = block_sum(rr, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = rr;
}

Status launch_residual(const double* f, const double* u, const double* op, double* r, float* r32,
                       double* partial, int n, cudaStream_t st, const float* dinv32, int batch) {
  const size_t N = (size_t)n * n;
  residual_kernel<<<dim3(residual_blocks(N), batch), kResidualBlock, 0, st>>>(f, u, op, r, r32, partial, n, dinv32);
  MG_LAUNCH("residual_kernel");
  return {};
}

// 1/a_C: the FP32 copy (the mixed path's network input scale) in FP32 from the
// integer-converted diagonal, the same value whether or not the FP64 copy
// (FP64 division) is wanted too.
__global__ void diag_inverse_kernel(const double* __restrict__ op, double* __restrict__ dinv,
                                    float* __restrict__ dinv32, size_t N) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  op += (size_t)blockIdx.y * 5 * N;
  dinv32 += (size_t)blockIdx.y * N;
  dinv32[p] = 1.0f / f64_to_f32_rn(op[p]);
  if (dinv) dinv[(size_t)blockIdx.y * N + p] = 1.0 / op[p];
}

Status launch_diag_inverse(const double* op, double* dinv, float* dinv32, size_t N, cudaStream_t st, int batch) {
  diag_inverse_kernel<<<dim3(grid_for(N, 256), batch), 256, 0, st>>>(op, dinv, dinv32, N);
  MG_LAUNCH("diag_inverse_kernel");
  return {};
}

// per-block partial sums of v^2, kResidualPix values per thread (the residual
// kernel's blocks: residual_blocks(N) partial sums)
__global__ void __launch_bounds__(kResidualBlock)
sumsq_kernel(const double* __restrict__ v, size_t N, double* __restrict__ partial) {
  __shared__ double smem[32];
  const size_t base = (size_t)blockIdx.x * (kResidualPix * kResidualBlock) + threadIdx.x;
  double x = 0.0;
#pragma unroll
  for (int k = 0; k < kResidualPix; ++k) {
    const size_t p = base + (size_t)k * kResidualBlock;
    if (p < N) x = fma(v[p], v[p], x);
  }
  x = block_sum(x, smem);
  if (threadIdx.x == 0) partial[blockIdx.x] = x;
}

Status launch_sumsq(const double* v, size_t N, double* partial, cudaStream_t st) {
  sumsq_kernel<<<residual_blocks(N), kResidualBlock, 0, st>>>(v, N, partial);
  MG_LAUNCH("sumsq_kernel");
  return {};
}

// One block sums the partials: thread t adds partial[t], partial[t + 1024], ...
// in order, then a fixed tree -- the same result on every run.
__global__ void __launch_bounds__(kReduceBlock)
reduce_kernel(const double* __restrict__ partial, int count, double* __restrict__ out) {
  __shared__ double smem[32];
  double v = 0.0;
  for (int t = threadIdx.x; t < count; t += blockDim.x) v += partial[t];
  v = block_sum(v, smem);
  if (threadIdx.x == 0) out[0] = v;
}

Status launch_reduce(const double* partial, int count, double* out, cudaStream_t st) {
  reduce_kernel<<<1, kReduceBlock, 0, st>>>(partial, count, out);
  MG_LAUNCH("reduce_kernel");
  return {};
}

// Setup tensors that turn Algorithm 3 into classical GMG (13 channels: E_C..E_N,
// G_C..G_N, F_J, F_G, D).  A stencil acting on e is rewritten in source-side
// form, sum_o a_o(p) e(p+o) = sum_o a_o(q-o) e(q) with q = p + o, so the setup
// tensor multiplying a layer's input carries the coefficient of tap o:
//   s[E_o](q) = -omega a_o(q-o) / a_C(q-o),  s[G_o](q) = -a_o(q-o)   (0 if q-o is outside)
//   s[F_J] = omega / a_C,  s[F_G] = 1,  s[D] = 0.
__global__ void gmg_setup_kernel(const double* __restrict__ op, double* __restrict__ out, int n, double omega,
                                 int input_diag_level) {
  const size_t N = (size_t)n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int)N) return;
  const int j = p / n, i = p - j * n;
  const int dy[5] = {0, 0, 0, -1, 1}, dx[5] = {0, -1, 1, 0, 0};  // C, W, E, S, N
  double* o = out + (size_t)p * kGmgChannels;
  for (int k = 0; k < 5; ++k) {
    const int pj = j - dy[k], pi = i - dx[k];
    double sE = 0.0, sG = 0.0;
    if (pj >= 0 && pj < n && pi >= 0 && pi < n) {
      const size_t q = (size_t)pj * n + pi;
      const double a = op[k * N + q];
      sE = -omega * a / op[q];
      sG = -a;
    }
    o[k] = sE;
    o[5 + k] = sG;
  }
  // rhs copies: r at coarse levels; D^{-1} r at the finest level when the input is normalised
  o[10] = input_diag_level ? omega : omega / op[p];
  o[11] = input_diag_level ? op[p] : 1.0;
  o[12] = 0.0;
}

// Setup tensors of the 8-channel network (one down, one up layer) that is GMG
// V(1, 0): the down layer does the Jacobi sweep from e = 0 and the defect of its
// result in one pass, d(p) = (1 - omega) r(p) - sum_{o != C} omega a_o(p) r(p+o) / a_C(p+o),
// so the off-centre setup tensors divide by the SOURCE node's diagonal:
//   s[T_o](q) = -omega a_o(q-o) / a_C(q) (o = W, E, S, N; 0 if q-o is outside),
//   s[F_G] = 1 - omega,  s[F_J] = omega / a_C,  s[D] = s[E] = 0.
// With the normalised input at the finest level (rhs copies hold D^{-1} r):
//   s[T_o](q) = -omega a_o(q-o),  s[F_G] = (1 - omega) a_C,  s[F_J] = omega.
// The eight values of node p (problem blockIdx.y of a batch stored back to back).
__device__ __forceinline__ void gmg_v10_values(const double* __restrict__ op, int n, double omega,
                                               int input_diag_level, int p, double* o) {
  const size_t N = (size_t)n * n;
  const int j = p / n, i = p - j * n;
  const int dy[4] = {0, 0, -1, 1}, dx[4] = {-1, 1, 0, 0};  // W, E, S, N
  const double aCq = op[p];
  const double inv = input_diag_level ? 1.0 : 1.0 / aCq;   // one FP64 divide per node
  for (int k = 0; k < 4; ++k) {
    const int pj = j - dy[k], pi = i - dx[k];
    double v = 0.0;
    if (pj >= 0 && pj < n && pi >= 0 && pi < n) v = -omega * op[(k + 1) * N + (size_t)pj * n + pi] * inv;
    o[k] = v;
  }
  o[4] = input_diag_level ? (1.0 - omega) * aCq : 1.0 - omega;
  o[5] = omega * inv;
  o[6] = 0.0;
  o[7] = 0.0;
}

__global__ void gmg_v10_setup_kernel(const double* __restrict__ op, double* __restrict__ out, int n, double omega,
                                     int input_diag_level) {
  const size_t N = (size_t)n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int)N) return;
  gmg_v10_values(op, n, omega, input_diag_level, p, out + (size_t)p * kGmgV10Channels);
}

// BF16 variant for the mixed-precision path: one 16-byte pixel per node, for a
// batch of problems stored back to back.  BF16 keeps 8 bits, so the values are
// formed in FP32 (24 bits) from the FP64 stencil converted with integer
// operations (fpconv.cuh) -- the FP64 pipe, about 1/58 of the FP32 rate here,
// stays idle -- and rounded once to BF16 (within 2^-9 of the FP64 values, plus
// FP32 rounding far below that).
__global__ void gmg_v10_setup_bf16_kernel(const double* __restrict__ op, __nv_bfloat16* __restrict__ out, int n,
                                          float omega, int input_diag_level) {
  const size_t N = (size_t)n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int)N) return;
  op += (size_t)blockIdx.y * 5 * N;
  out += (size_t)blockIdx.y * N * kGmgV10Channels;
  const int j = p / n, i = p - j * n;
  const int dy[4] = {0, 0, -1, 1}, dx[4] = {-1, 1, 0, 0};  // W, E, S, N
  const float aCq = f64_to_f32_rn(op[p]);
  const float inv = input_diag_level ? 1.0f : 1.0f / aCq;
  float o[8];
  for (int k = 0; k < 4; ++k) {
    const int pj = j - dy[k], pi = i - dx[k];
    o[k] = (pj >= 0 && pj < n && pi >= 0 && pi < n)
               ? -omega * f64_to_f32_rn(op[(k + 1) * N + (size_t)pj * n + pi]) * inv
               : 0.0f;
  }
  o[4] = input_diag_level ? (1.0f - omega) * aCq : 1.0f - omega;
  o[5] = omega * inv;
  o[6] = 0.0f;
  o[7] = 0.0f;
  __nv_bfloat162 h[4];
  for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(o[2 * k], o[2 * k + 1]);
  reinterpret_cast<uint4*>(out)[p] = *reinterpret_cast<const uint4*>(h);
}

Status launch_gmg_v10_setup_bf16(const double* op, __nv_bfloat16* out, int n, double omega, cudaStream_t st,
                                 bool input_diag_level, int batch) {
  gmg_v10_setup_bf16_kernel<<<dim3(grid_for((size_t)n * n, 256), batch), 256, 0, st>>>(op, out, n, (float)omega,
                                                                                        input_diag_level ? 1 : 0);
  MG_LAUNCH("gmg_v10_setup_bf16_kernel");
  return {};
}

Status launch_gmg_setup(const double* op, double* out, int n, double omega, cudaStream_t st,
                        bool input_diag_level, int channels) {
  if (channels == kGmgV10Channels) {
    gmg_v10_setup_kernel<<<grid_for((size_t)n * n, 256), 256, 0, st>>>(op, out, n, omega, input_diag_level ? 1 : 0);
    MG_LAUNCH("gmg_v10_setup_kernel");
    return {};
  }
  gmg_setup_kernel<<<grid_for((size_t)n * n, 256), 256, 0, st>>>(op, out, n, omega, input_diag_level ? 1 : 0);
  MG_LAUNCH("gmg_setup_kernel");
  return {};
}

__global__ void axpy_to_kernel(const double* __restrict__ u, const double* __restrict__ e,
                               double* __restrict__ out, size_t N) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) out[p] = u[p] + e[p];
}

Status launch_axpy_to(const double* u, const double* e, double* out, size_t N, cudaStream_t st) {
  axpy_to_kernel<<<grid_for(N, 256), 256, 0, st>>>(u, e, out, N);
  MG_LAUNCH("axpy_to_kernel");
  return {};
}

}  // namespace mgcnn

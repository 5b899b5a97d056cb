// Classical geometric multigrid on the GPU (Sec. 2.3 of arXiv 2312.11093),
// the comparator of the learned solver: V(nu1, nu2) cycles of weighted Jacobi
// (weight omega), full-weighting restriction of the defect, bilinear
// prolongation, rediscretised coarse operators (the context's operator on
// every level), inside the stationary iteration of Eq. 1.  FP64 throughout.
// The coarsest grid is smoothed (nu1 + nu2 sweeps), not solved directly.
#include <cmath>

#include "gmg.cuh"
#include "ops.cuh"

namespace mgcnn {

namespace {

// e_out = e_in + omega (r - A e_in) / a_C; with e_in == nullptr, e_in = 0.
__global__ void jacobi_kernel(const double* __restrict__ op, const double* __restrict__ r,
                              const double* __restrict__ ein, double* __restrict__ eout, int n, double omega) {
  const size_t N = (size_t)n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int)N) return;
  const double aC = op[p];
  if (!ein) {
    eout[p] = omega * r[p] / aC;
    return;
  }
  const int j = p / n, i = p - j * n;
  const double eC = ein[p];
  double Ae = aC * eC;
  if (i > 0) Ae += op[N + p] * ein[p - 1];
  if (i < n - 1) Ae += op[2 * N + p] * ein[p + 1];
  if (j > 0) Ae += op[3 * N + p] * ein[p - n];
  if (j < n - 1) Ae += op[4 * N + p] * ein[p + n];
  eout[p] = eC + omega * (r[p] - Ae) / aC;
}

// r_c[J][I] = sum_ab FW[a][b] d[2J + a][2I + b], d = r - A e (computed on the fly).
__global__ void defect_restrict_kernel(const double* __restrict__ op, const double* __restrict__ r,
                                       const double* __restrict__ e, double* __restrict__ rc, int n) {
  const int nc = (n - 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc * nc) return;
  const size_t N = (size_t)n * n;
  const int J = p / nc, I = p - J * nc;
  const double w1[3] = {1.0, 2.0, 1.0};
  double acc = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int j = 2 * J + a;
    for (int b = 0; b < 3; ++b) {
      const int i = 2 * I + b;
      const size_t q = (size_t)j * n + i;
      double Ae = op[q] * e[q];
      if (i > 0) Ae += op[N + q] * e[q - 1];
      if (i < n - 1) Ae += op[2 * N + q] * e[q + 1];
      if (j > 0) Ae += op[3 * N + q] * e[q - n];
      if (j < n - 1) Ae += op[4 * N + q] * e[q + n];
      acc += w1[a] * w1[b] * (r[q] - Ae);
    }
  }
  rc[p] = acc / 16.0;
}

// e[2J + a][2I + b] += BIL[a][b] e_c[J][I], gather form.
__global__ void prolong_add_kernel(const double* __restrict__ ec, double* __restrict__ e, int n) {
  const int nc = (n - 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  const int j = p / n, i = p - j * n;
  const double w1[3] = {1.0, 2.0, 1.0};
  double acc = 0.0;
  for (int a = 0; a < 3; ++a) {
    const int dj = j - a;
    if (dj < 0 || (dj & 1) || (dj >> 1) >= nc) continue;
    for (int b = 0; b < 3; ++b) {
      const int di = i - b;
      if (di < 0 || (di & 1) || (di >> 1) >= nc) continue;
      acc += w1[a] * w1[b] * ec[(size_t)(dj >> 1) * nc + (di >> 1)];
    }
  }
  e[p] += acc / 4.0;
}

// Setup tensors of the BPX network (symmetric variant of the learned solver,
// the additive multilevel counterpart of the V-cycle above): the carrier
// channel's scale that makes the smoother copy sqrt(omega 4^l / a_C) R_l r; the
// division by eps (a power of two) is exact.
__global__ void bpx_setup_kernel(const double* __restrict__ op, double* __restrict__ out, int n, double w4l,
                                 int channels) {
  const size_t N = (size_t)n * n;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  double* o = out + p * channels;
  o[0] = sqrt(w4l / op[p]) / MGCNN_BPX_EPS;
  for (int c = 1; c < channels; ++c) o[c] = 0.0;
}

}  // namespace

Status launch_bpx_setup(const double* op, double* out, int n, int level, double omega, int channels,
                        cudaStream_t st) {
  bpx_setup_kernel<<<grid_for((size_t)n * n, 256), 256, 0, st>>>(op, out, n, omega * std::ldexp(1.0, 2 * level),
                                                                 channels);
  MG_LAUNCH("bpx_setup_kernel");
  return {};
}

// One V(nu1, nu2) cycle on level l for A_l e = r_l from e = 0; the result is in e[l].
// Level l smooths with the weight omega.at(l, g.L).
Status gmg_vcycle(const GmgLevels& g, int l, int nu1, int nu2, const LevelWeights& omegas, cudaStream_t st) {
  const double omega = omegas.at(l, g.L);
  const int n = g.n[l];
  const size_t N = (size_t)n * n;
  const int grid = grid_for(N, 256);
  double* e = g.e[l];
  double* t = g.t[l];
  const bool coarsest = l + 1 == g.L;
  const int pre = coarsest ? nu1 + nu2 : nu1;
  // pre-smoothing (the first sweep starts from e = 0)
  for (int s = 0; s < pre; ++s) {
    jacobi_kernel<<<grid, 256, 0, st>>>(g.op[l], g.r[l], s == 0 ? nullptr : e, t, n, omega);
    MG_LAUNCH("jacobi_kernel");
    std::swap(e, t);
  }
  if (pre == 0) MG_CUDA(cudaMemsetAsync(e, 0, N * sizeof(double), st));
  if (!coarsest) {
    const int nc = g.n[l + 1];
    defect_restrict_kernel<<<grid_for((size_t)nc * nc, 256), 256, 0, st>>>(g.op[l], g.r[l], e, g.r[l + 1], n);
    MG_LAUNCH("defect_restrict_kernel");
    MG_TRY(gmg_vcycle(g, l + 1, nu1, nu2, omegas, st));
    prolong_add_kernel<<<grid, 256, 0, st>>>(g.e[l + 1], e, n);
    MG_LAUNCH("prolong_add_kernel");
    for (int s = 0; s < nu2; ++s) {
      jacobi_kernel<<<grid, 256, 0, st>>>(g.op[l], g.r[l], e, t, n, omega);
      MG_LAUNCH("jacobi_kernel");
      std::swap(e, t);
    }
  }
  // leave the result in g.e[l]
  if (e != g.e[l]) MG_CUDA(cudaMemcpyAsync(g.e[l], e, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return {};
}

}  // namespace mgcnn

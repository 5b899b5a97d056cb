// Flexible GMRES for a batch of uneven problems, with the batch's mixed
// network as right preconditioner (Sec. 2.2: the network approximates A^{-1}
// and may precondition a Krylov method).  Every problem of a size class runs
// its own Arnoldi process; the processes advance in lockstep, one inner
// iteration of every still-active problem per pass, on the class's buffers:
//   z_j = B v_j            the fused V-cycle of the class (FP32 D^{-1} v_j in)
//   w   = A z_j            FP64 5-point product
//   h   = V^T w, w -= V h  classical Gram-Schmidt, twice, fixed-order sums
//   v_{j+1} = w / ||w||
// with the Hessenberg matrix, its Givens rotations and the residual estimate
// per problem on the device (one thread per problem).  At the end of a cycle
// (restart iterations, or the estimate below tol, or maxit) u += Z y and the
// next cycle starts from the true FP64 residual.  The classes run concurrently
// on their own streams; the host reads one counter per inner pass to stop
// early once no problem is left in its cycle.
#include <algorithm>
#include <cmath>

#include "batch.cuh"
#include "ops.cuh"

namespace mgcnn {

namespace {

constexpr int kBkThreads = 256;
constexpr int kBkPix = 8;                    // pixels per thread of the dot-product blocks
constexpr int kBkSpan = kBkThreads * kBkPix;

int bk_blocks(size_t N) { return (int)((N + kBkSpan - 1) / kBkSpan); }

// per-problem ints: [field][B]
enum { kAlive = 0, kInner, kIter, kStat, kCyc, kMm, kIntFields };

// per-problem doubles (offsets in units of B): fn, beta, inv, hn2, one, r2,
// then the small matrices
struct BkLayout {
  int B = 0, m = 0;
  size_t fn = 0, beta = 0, inv = 0, hn2 = 0, one = 0, r2 = 0;
  size_t H = 0, cs = 0, sn = 0, g = 0, y = 0, hc = 0, total = 0;
  explicit BkLayout(int B_, int m_) : B(B_), m(m_) {
    size_t o = 0;
    fn = o; o += B;
    beta = o; o += B;
    inv = o; o += B;
    hn2 = o; o += B;
    one = o; o += B;
    r2 = o; o += B;
    H = o; o += (size_t)B * (m + 1) * m;        // H[b][i * m + j]
    cs = o; o += (size_t)B * m;
    sn = o; o += (size_t)B * m;
    g = o; o += (size_t)B * (m + 1);
    y = o; o += (size_t)B * m;
    hc = o; o += (size_t)2 * B * (m + 1);       // Gram-Schmidt coefficients of the two passes [pass][b][i]
    total = o;
  }
};

__device__ __forceinline__ double bk_block_sum(double v, double* smem) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? smem[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[(b * pstride + i) * nblk + blk] = sum over the block's pixels of
// V_i[b] * w[b], i < nvec <= kBkMaxVec; V_i[b] = V + (i * B + b) * N, w[b] = w +
// b * wstride.  Problems with flag[b] == 0 are skipped (flag may be null).  A
// vector's sum is reduced within each warp by shuffles, with no block-wide
// barrier per vector (the next vectors' loads stay in flight); the warp sums are
// added in warp order at the end.
constexpr int kBkMaxVec = MGCNN_KRYLOV_MAX_RESTART + 1;
__global__ void __launch_bounds__(kBkThreads) bk_dots_kernel(const double* __restrict__ V, int nvec,
                                                             const double* __restrict__ w, size_t wstride, size_t N,
                                                             int B, const int* __restrict__ flag,
                                                             double* __restrict__ partial, int pstride) {
  __shared__ double wsum[kBkMaxVec][kBkThreads / 32];
  const int b = blockIdx.y;
  if (flag && !flag[b]) return;
  const int nblk = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t base = (size_t)blockIdx.x * kBkSpan + threadIdx.x;
  double wv[kBkPix];
#pragma unroll
  for (int t = 0; t < kBkPix; ++t) {
    const size_t p = base + (size_t)t * kBkThreads;
    wv[t] = p < N ? w[(size_t)b * wstride + p] : 0.0;
  }
#pragma unroll 2
  for (int i = 0; i < nvec; ++i) {
    const double* v = V + ((size_t)i * B + b) * N;
    double s = 0.0;
#pragma unroll
    for (int t = 0; t < kBkPix; ++t) {
      const size_t p = base + (size_t)t * kBkThreads;
      if (p < N) s += v[p] * wv[t];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[i][warp] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvec; i += kBkThreads) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kBkThreads / 32; ++q) t += wsum[i][q];
    partial[((size_t)b * pstride + i) * nblk + blockIdx.x] = t;
  }
}

// out[b * ostride + i] = sum_t partial[(b * pstride + i) * count + t], one
// 1024-thread block per (i, b), a fixed order.
__global__ void __launch_bounds__(1024) bk_reduce_kernel(const double* __restrict__ partial, int count, int pstride,
                                                         const int* __restrict__ flag, double* __restrict__ out,
                                                         int ostride) {
  __shared__ double smem[32];
  const int i = blockIdx.x, b = blockIdx.y;
  if (flag && !flag[b]) return;
  const double* p = partial + ((size_t)b * pstride + i) * count;
  double v = 0.0;
  for (int t = threadIdx.x; t < count; t += blockDim.x) v += p[t];
  v = bk_block_sum(v, smem);
  if (threadIdx.x == 0) out[(size_t)b * ostride + i] = v;
}

// y[b] += sign * sum_{i < cnt} coef[b * cstride + i] * V_i[b], cnt = nvec, or
// count[b] when count is given; problems with flag[b] == 0 are skipped.  A
// thread's kCombPix pixels advance together through the vectors, so every step
// issues kCombPix independent loads.
constexpr int kCombPix = 4;
__global__ void bk_combine_kernel(double* __restrict__ y, const double* __restrict__ V, int nvec,
                                  const int* __restrict__ count, const double* __restrict__ coef, int cstride,
                                  double sign, size_t N, int B, const int* __restrict__ flag) {
  const int b = blockIdx.y;
  if (flag && !flag[b]) return;
  const size_t base = (size_t)blockIdx.x * blockDim.x * kCombPix + threadIdx.x;
  const int cnt = count ? count[b] : nvec;
  double s[kCombPix];
#pragma unroll
  for (int t = 0; t < kCombPix; ++t) s[t] = 0.0;
#pragma unroll 2
  for (int i = 0; i < cnt; ++i) {
    const double c = coef[(size_t)b * cstride + i];
    const double* v = V + ((size_t)i * B + b) * N;
#pragma unroll
    for (int t = 0; t < kCombPix; ++t) {
      const size_t p = base + (size_t)t * blockDim.x;
      if (p < N) s[t] += c * v[p];
    }
  }
#pragma unroll
  for (int t = 0; t < kCombPix; ++t) {
    const size_t p = base + (size_t)t * blockDim.x;
    if (p < N) y[(size_t)b * N + p] += sign * s[t];
  }
}

// x[b] *= s[b] for problems with flag[b]
__global__ void bk_scale_kernel(double* __restrict__ x, const double* __restrict__ s, size_t N,
                                const int* __restrict__ flag) {
  const int b = blockIdx.y;
  if (!flag[b]) return;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) x[(size_t)b * N + p] *= s[b];
}

// r32[b] (row pitch r32_pitch(n)) = FP32 v[b] (times dinv32[b] when given)
__global__ void bk_to_f32_kernel(const double* __restrict__ v, float* __restrict__ r32,
                                 const float* __restrict__ dinv32, int n, const int* __restrict__ flag) {
  const int b = blockIdx.y;
  if (!flag[b]) return;
  const size_t N = (size_t)n * n;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int j = (int)(p / n), i = (int)(p - (size_t)j * n);
  const float x = (float)v[(size_t)b * N + p];
  r32[(size_t)b * r32_floats(n) + (size_t)j * r32_pitch(n) + i] = dinv32 ? x * dinv32[(size_t)b * N + p] : x;
}

// w[b] = A_b z[b], the FP64 5-point operator of problem b (planes aC, aW, aE, aS, aN)
__global__ void bk_apply_kernel(const double* __restrict__ op, const double* __restrict__ z, double* __restrict__ w,
                                int n, const int* __restrict__ flag) {
  const int b = blockIdx.y;
  if (!flag[b]) return;
  const size_t N = (size_t)n * n;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int j = (int)(p / n), i = (int)(p - (size_t)j * n);
  const double* a = op + (size_t)b * 5 * N;
  const double* x = z + (size_t)b * N;
  double s = a[p] * x[p];
  if (i > 0) s += a[N + p] * x[p - 1];
  if (i + 1 < n) s += a[2 * N + p] * x[p + 1];
  if (j > 0) s += a[3 * N + p] * x[p - n];
  if (j + 1 < n) s += a[4 * N + p] * x[p + n];
  w[(size_t)b * N + p] = s;
}

struct BkParams {
  double tol, divtol;
  int maxit, m, B;
};

// Start: fn from fn2, the f = 0 and non-finite cases, iteration counters.
__global__ void bk_init_kernel(double* __restrict__ D, int* __restrict__ I, double* __restrict__ u,
                               double* __restrict__ hist, size_t N, BkParams P, size_t fn_off, size_t one_off) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P.B) return;
  const double fn2 = D[fn_off + b];
  D[one_off + b] = 1.0;
  I[kIter * P.B + b] = 0;
  I[kInner * P.B + b] = 0;
  I[kCyc * P.B + b] = 0;
  int alive = 1, stat = MGCNN_OK;
  if (!isfinite(fn2)) {
    alive = 0;
    stat = MGCNN_ERR_NONFINITE;
    hist[(size_t)b * (P.maxit + 1)] = fn2;
  } else if (fn2 == 0.0) {
    alive = 0;
    hist[(size_t)b * (P.maxit + 1)] = 0.0;
    for (size_t p = 0; p < N; ++p) u[(size_t)b * N + p] = 0.0;
  }
  D[fn_off + b] = sqrt(fn2);
  I[kAlive * P.B + b] = alive;
  I[kStat * P.B + b] = stat;
}

// Before a cycle: ||r||/||f|| from the true residual, the stopping tests, and
// for a problem that goes on the cycle's start (beta, g, H = 0, v_0 scale).
__global__ void bk_restart_kernel(double* __restrict__ D, int* __restrict__ I, double* __restrict__ hist,
                                  BkParams P, BkLayout Ly, int* __restrict__ counter) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P.B || !I[kAlive * P.B + b]) return;
  const int it = I[kIter * P.B + b];
  const double r2 = D[Ly.r2 + b];
  const double rel = sqrt(r2) / D[Ly.fn + b];
  hist[(size_t)b * (P.maxit + 1) + it] = rel;
  int stat = -100;
  if (!isfinite(rel)) stat = MGCNN_ERR_NONFINITE;
  else if (rel <= P.tol) stat = MGCNN_OK;
  else if (P.divtol > 0.0 && rel > P.divtol) stat = MGCNN_ERR_DIVERGED;
  else if (it >= P.maxit) stat = MGCNN_NOT_CONVERGED;
  if (stat != -100) {
    I[kAlive * P.B + b] = 0;
    I[kStat * P.B + b] = stat;
    return;
  }
  const int m = P.m;
  const double beta = sqrt(r2);
  D[Ly.beta + b] = beta;
  D[Ly.inv + b] = 1.0 / beta;
  double* H = D + Ly.H + (size_t)b * (m + 1) * m;
  for (int q = 0; q < (m + 1) * m; ++q) H[q] = 0.0;
  double* g = D + Ly.g + (size_t)b * (m + 1);
  for (int q = 0; q <= m; ++q) g[q] = 0.0;
  g[0] = beta;
  I[kMm * P.B + b] = min(m, P.maxit - it);
  I[kCyc * P.B + b] = 0;
  I[kInner * P.B + b] = 1;
  atomicAdd(counter, 1);
}

// After inner step j of every problem still in its cycle: column j of H from the
// two Gram-Schmidt passes and ||w||, the earlier rotations applied to it, a new
// rotation, the residual estimate, and whether the cycle goes on.
__global__ void bk_givens_kernel(double* __restrict__ D, int* __restrict__ I, double* __restrict__ hist, int j,
                                 BkParams P, BkLayout Ly, int* __restrict__ counter) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P.B || !I[kInner * P.B + b]) return;
  const int m = P.m;
  double* H = D + Ly.H + (size_t)b * (m + 1) * m;
  double* cs = D + Ly.cs + (size_t)b * m;
  double* sn = D + Ly.sn + (size_t)b * m;
  double* g = D + Ly.g + (size_t)b * (m + 1);
  const double* h0 = D + Ly.hc + (size_t)b * (m + 1);
  const double* h1 = D + Ly.hc + ((size_t)P.B + b) * (m + 1);
  const double hn = sqrt(D[Ly.hn2 + b]);
  for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = (0.0 + h0[i]) + h1[i];
  H[(size_t)(j + 1) * m + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
    H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
    H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
  }
  const double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
  const double d = hypot(a, c);
  cs[j] = a / d;
  sn[j] = c / d;
  H[(size_t)j * m + j] = d;
  H[(size_t)(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  I[kCyc * P.B + b] = j + 1;
  const int it = I[kIter * P.B + b] + 1;
  I[kIter * P.B + b] = it;
  const double est = fabs(g[j + 1]) / D[Ly.fn + b];
  if (est <= P.tol || it >= P.maxit || !isfinite(est) || j == I[kMm * P.B + b] - 1) {
    I[kInner * P.B + b] = 0;   // the cycle ends here: update, then the true residual
    return;
  }
  hist[(size_t)b * (P.maxit + 1) + it] = est;
  D[Ly.inv + b] = 1.0 / hn;
  atomicAdd(counter, 1);
}

// y = R^{-1} g on the rotated H (back substitution, k = the cycle's length)
__global__ void bk_solve_y_kernel(double* __restrict__ D, const int* __restrict__ I, BkParams P, BkLayout Ly) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P.B) return;
  const int k = I[kCyc * P.B + b], m = P.m;
  const double* H = D + Ly.H + (size_t)b * (m + 1) * m;
  const double* g = D + Ly.g + (size_t)b * (m + 1);
  double* y = D + Ly.y + (size_t)b * m;
  for (int i = k - 1; i >= 0; --i) {
    double t = g[i];
    for (int q = i + 1; q < k; ++q) t -= H[(size_t)i * m + q] * y[q];
    y[i] = t / H[(size_t)i * m + i];
  }
}

__global__ void bk_end_cycle_kernel(int* __restrict__ I, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) I[kCyc * B + b] = 0;
}

}  // namespace

Status solve_batched_krylov(mgcnn_ctx* c, int nprob, const double* const* rhs, double* const* u, double tol,
                            int maxit, int restart, int* iters, double* relres, int* status) {
  if (!c->bready) return make_status(MGCNN_ERR_STATE, "mgcnn_setup_batched has not been called");
  if (nprob != c->bn) return make_status(MGCNN_ERR_ARG, "batch has %d problems, setup had %d", nprob, c->bn);
  if (restart < 1 || restart > MGCNN_KRYLOV_MAX_RESTART)
    return make_status(MGCNN_ERR_ARG, "restart must be in 1..%d", MGCNN_KRYLOV_MAX_RESTART);
  for (int i = 0; i < nprob; ++i)
    if (!rhs[i] || !u[i]) return make_status(MGCNN_ERR_ARG, "null array for problem %d", i);
  const int m = restart;
  cudaStream_t st = c->bstream;
  c->bmaxit = -1;   // the history buffers may move: the stationary path captures its graph again
  const FusedWeights w = fused_weights(c);
  int* counter = c->bcount.as<int>();
  // workspace and inputs
  for (BatchClass& k : c->bcls) {
    const size_t N = (size_t)k.n * k.n;
    const BkLayout Ly(k.B, m);
    MG_TRY(ensure(k.kV, (size_t)(m + 1) * k.B * N * sizeof(double)));
    MG_TRY(ensure(k.kZ, (size_t)m * k.B * N * sizeof(double)));
    MG_TRY(ensure(k.kpart, (size_t)k.B * (m + 1) * std::max(bk_blocks(N), residual_blocks(N)) * sizeof(double)));
    MG_TRY(ensure(k.kdbl, Ly.total * sizeof(double)));
    MG_TRY(ensure(k.kint, (size_t)kIntFields * k.B * sizeof(int)));
    MG_TRY(ensure(k.hist, (size_t)k.B * (maxit + 1) * sizeof(double)));
    for (int b = 0; b < k.B; ++b) {
      const int i = k.members[b];
      MG_CUDA(cudaMemcpyAsync(k.f.as<double>() + b * N, rhs[i], N * sizeof(double), cudaMemcpyDefault, st));
      MG_CUDA(cudaMemcpyAsync(k.u.as<double>() + b * N, u[i], N * sizeof(double), cudaMemcpyDefault, st));
    }
    double* D = k.kdbl.as<double>();
    const int nb = bk_blocks(N);
    bk_dots_kernel<<<dim3(nb, k.B), kBkThreads, 0, st>>>(k.f.as<double>(), 1, k.f.as<double>(), N, N, k.B, nullptr,
                                                         k.kpart.as<double>(), 1);
    MG_LAUNCH("bk_dots_kernel");
    bk_reduce_kernel<<<dim3(1, k.B), 1024, 0, st>>>(k.kpart.as<double>(), nb, 1, nullptr, D + Ly.fn, 1);
    MG_LAUNCH("bk_reduce_kernel");
    const BkParams P{tol, c->divtol, maxit, m, k.B};
    bk_init_kernel<<<grid_for(k.B, 128), 128, 0, st>>>(D, k.kint.as<int>(), k.u.as<double>(), k.hist.as<double>(), N,
                                                       P, Ly.fn, Ly.one);
    MG_LAUNCH("bk_init_kernel");
  }
  // the classes run concurrently on their own streams between a fork and a join on `st`
  auto fork = [&]() -> Status {
    MG_CUDA(cudaEventRecord(c->bfork, st));
    for (BatchClass& k : c->bcls) MG_CUDA(cudaStreamWaitEvent(k.stream, c->bfork, 0));
    return {};
  };
  auto join = [&]() -> Status {
    for (BatchClass& k : c->bcls) {
      MG_CUDA(cudaEventRecord(k.done, k.stream));
      MG_CUDA(cudaStreamWaitEvent(st, k.done, 0));
    }
    return {};
  };
  int h_count = 0;
  auto read_counter = [&]() -> Status {
    MG_CUDA(cudaMemcpyAsync(&h_count, counter, sizeof(int), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    return {};
  };
  for (;;) {
    // true residual into v_0, ||r||^2, stopping tests, cycle start
    MG_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    MG_TRY(fork());
    for (BatchClass& k : c->bcls) {
      const size_t N = (size_t)k.n * k.n;
      const BkLayout Ly(k.B, m);
      double* D = k.kdbl.as<double>();
      const BkParams P{tol, c->divtol, maxit, m, k.B};
      cudaStream_t st = k.stream;
      MG_TRY(launch_residual(k.f.as<double>(), k.u.as<double>(), k.op[0].as<double>(), k.kV.as<double>(), nullptr,
                             k.kpart.as<double>(), k.n, st, nullptr, k.B));
      const int nr = residual_blocks(N);
      bk_reduce_kernel<<<dim3(1, k.B), 1024, 0, st>>>(k.kpart.as<double>(), nr, 1, k.kint.as<int>() + kAlive * k.B,
                                                      D + Ly.r2, 1);
      MG_LAUNCH("bk_reduce_kernel");
      bk_restart_kernel<<<grid_for(k.B, 128), 128, 0, st>>>(D, k.kint.as<int>(), k.hist.as<double>(), P, Ly, counter);
      MG_LAUNCH("bk_restart_kernel");
      bk_scale_kernel<<<dim3(grid_for(N, 256), k.B), 256, 0, st>>>(k.kV.as<double>(), D + Ly.inv, N,
                                                                   k.kint.as<int>() + kInner * k.B);
      MG_LAUNCH("bk_scale_kernel");
    }
    MG_TRY(join());
    MG_TRY(read_counter());
    if (h_count == 0) break;
    for (int j = 0; j < m; ++j) {
      MG_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
      MG_TRY(fork());
      for (BatchClass& k : c->bcls) {
        const size_t N = (size_t)k.n * k.n;
        const BkLayout Ly(k.B, m);
        double* D = k.kdbl.as<double>();
        int* inner = k.kint.as<int>() + kInner * k.B;
        const BkParams P{tol, c->divtol, maxit, m, k.B};
        cudaStream_t st = k.stream;
        double* V = k.kV.as<double>();
        double* Vj = V + (size_t)j * k.B * N;
        double* Wv = V + (size_t)(j + 1) * k.B * N;      // w is formed in the slot of v_{j+1}
        double* Zj = k.kZ.as<double>() + (size_t)j * k.B * N;
        const dim3 pg(grid_for(N, 256), k.B);
        bk_to_f32_kernel<<<pg, 256, 0, st>>>(Vj, k.r32.as<float>(), c->cfg.input_diag ? k.dinv32.as<float>() : nullptr,
                                             k.n, inner);
        MG_LAUNCH("bk_to_f32_kernel");
        MG_TRY(fused_vcycle_levels(k.fl, k.r32.as<float>(), D + Ly.one, Zj, nullptr, w, inner, st, nullptr));
        bk_apply_kernel<<<pg, 256, 0, st>>>(k.op[0].as<double>(), Zj, Wv, k.n, inner);
        MG_LAUNCH("bk_apply_kernel");
        const int nb = bk_blocks(N);
        for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
          double* hc = D + Ly.hc + (size_t)pass * k.B * (m + 1);
          bk_dots_kernel<<<dim3(nb, k.B), kBkThreads, 0, st>>>(V, j + 1, Wv, N, N, k.B, inner, k.kpart.as<double>(),
                                                               m + 1);
          MG_LAUNCH("bk_dots_kernel");
          bk_reduce_kernel<<<dim3(j + 1, k.B), 1024, 0, st>>>(k.kpart.as<double>(), nb, m + 1, inner, hc, m + 1);
          MG_LAUNCH("bk_reduce_kernel");
          bk_combine_kernel<<<dim3(grid_for(N, 256 * kCombPix), k.B), 256, 0, st>>>(Wv, V, j + 1, nullptr, hc, m + 1,
                                                                                    -1.0, N, k.B, inner);
          MG_LAUNCH("bk_combine_kernel");
        }
        bk_dots_kernel<<<dim3(nb, k.B), kBkThreads, 0, st>>>(Wv, 1, Wv, N, N, k.B, inner, k.kpart.as<double>(), 1);
        MG_LAUNCH("bk_dots_kernel");
        bk_reduce_kernel<<<dim3(1, k.B), 1024, 0, st>>>(k.kpart.as<double>(), nb, 1, inner, D + Ly.hn2, 1);
        MG_LAUNCH("bk_reduce_kernel");
        bk_givens_kernel<<<grid_for(k.B, 128), 128, 0, st>>>(D, k.kint.as<int>(), k.hist.as<double>(), j, P, Ly,
                                                             counter);
        MG_LAUNCH("bk_givens_kernel");
        bk_scale_kernel<<<pg, 256, 0, st>>>(Wv, D + Ly.inv, N, inner);
        MG_LAUNCH("bk_scale_kernel");
      }
      MG_TRY(join());
      MG_TRY(read_counter());
      if (h_count == 0) break;
    }
    // u += Z y for every problem that ran a cycle
    MG_TRY(fork());
    for (BatchClass& k : c->bcls) {
      const size_t N = (size_t)k.n * k.n;
      const BkLayout Ly(k.B, m);
      double* D = k.kdbl.as<double>();
      const BkParams P{tol, c->divtol, maxit, m, k.B};
      cudaStream_t st = k.stream;
      bk_solve_y_kernel<<<grid_for(k.B, 128), 128, 0, st>>>(D, k.kint.as<int>(), P, Ly);
      MG_LAUNCH("bk_solve_y_kernel");
      bk_combine_kernel<<<dim3(grid_for(N, 256 * kCombPix), k.B), 256, 0, st>>>(k.u.as<double>(), k.kZ.as<double>(), m,
                                                                     k.kint.as<int>() + kCyc * k.B, D + Ly.y, m, 1.0,
                                                                     N, k.B, nullptr);
      MG_LAUNCH("bk_combine_kernel");
      bk_end_cycle_kernel<<<grid_for(k.B, 128), 128, 0, st>>>(k.kint.as<int>(), k.B);
      MG_LAUNCH("bk_end_cycle_kernel");
    }
    MG_TRY(join());
  }
  // results back
  Status overall;
  for (BatchClass& k : c->bcls) {
    const size_t N = (size_t)k.n * k.n;
    std::vector<int> I((size_t)kIntFields * k.B);
    std::vector<double> h((size_t)k.B * (maxit + 1));
    MG_CUDA(cudaMemcpyAsync(I.data(), k.kint.p, I.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaMemcpyAsync(h.data(), k.hist.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    for (int b = 0; b < k.B; ++b)
      MG_CUDA(cudaMemcpyAsync(u[k.members[b]], k.u.as<double>() + b * N, N * sizeof(double), cudaMemcpyDefault, st));
    MG_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < k.B; ++b) {
      const int i = k.members[b];
      const int it = I[(size_t)kIter * k.B + b], stat = I[(size_t)kStat * k.B + b];
      if (iters) iters[i] = it;
      if (relres) relres[i] = h[(size_t)b * (maxit + 1) + std::min(it, maxit)];
      if (status) status[i] = stat;
      if (stat < 0 && overall.code >= 0) overall = make_status(stat, "problem %d: %s", i, mgcnn_status_string(stat));
      else if (stat == MGCNN_NOT_CONVERGED && overall.code == MGCNN_OK)
        overall = make_status(MGCNN_NOT_CONVERGED, "problem %d did not converge in %d iterations", i, maxit);
    }
  }
  return overall;
}

}  // namespace mgcnn

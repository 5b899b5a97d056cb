// Training: the K-cycle residual loss and its hand-written adjoint (Sec. 3.4,
// Eq. loss of arXiv 2312.11093, unrolled over K stationary cycles), in FP32
// or FP64, batched over problems of equal grid size, plus Adam.
//
//   r_0 = f,  r_{k+1} = r_k - A B(r_k),   L = (1/N) sum_i ||r_K,i||^2 / ||f_i||^2
//
// Reverse sweep, g_k = dL/dr_k:  g_K = 2 r_K / (N ||f||^2),
//   g_k = g_{k+1} + B^T(-A^T g_{k+1}),
// and cycle k contributes the weight gradient of <B(r_k), -A^T g_{k+1}>.
// Only r_k is kept per cycle; the intermediates of B are recomputed in the
// reverse sweep (per-cycle checkpointing).  Setup-tensor gradients from every
// cycle accumulate, then flow back through Algorithm 2 (tanh ResNet and the
// setup RCNN) once.
//
// Adjoints of the layers (PyTorch semantics, same weight arrays):
//   same conv  y = K x      ->  x_bar = K^T y_bar: the same conv with the
//                               weights transposed in (co, ci) and flipped in space
//   RCNN  (stride 2)        ->  TCNN with the same array, and vice versa
//   y = x + K (s * x)       ->  t = K^T y_bar; x_bar = y_bar + s * t; s_bar += x * t
//   y = tanh(K z + b) + z   ->  d = y_bar (1 - tanh^2); z_bar = y_bar + K^T d
// Weight gradients are correlations of an output adjoint with the layer input
// over all pixels of all problems; one gather-correlate kernel serves the
// same, strided and transposed layers, reduced deterministically.
#include <algorithm>
#include <cmath>

#include "ops.cuh"
#include "train.cuh"

namespace mgcnn {

namespace {

// ---------------------------------------------------------------------------
// elementwise and small kernels

template <typename T>
__global__ void transpose_flip_kernel(const T* __restrict__ W, T* __restrict__ WT, int CO, int CI) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= CO * CI * 9) return;
  const int tap = p % 9, ci = (p / 9) % CI, co = p / (9 * CI);
  WT[((size_t)ci * CO + co) * 9 + (8 - tap)] = W[p];
}

// x_bar = y_bar + s * t ;  s_bar += x_in * t
template <typename T>
__global__ void resnet_bwd_kernel(const T* __restrict__ ybar, const T* __restrict__ s, const T* __restrict__ xin,
                                  const T* __restrict__ t, T* __restrict__ xbar, T* __restrict__ sbar, size_t count) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const T tv = t[p];
  sbar[p] += xin[p] * tv;
  xbar[p] = ybar[p] + s[p] * tv;
}

// d = z_bar * (1 - t^2)
template <typename T>
__global__ void tanh_bwd_kernel(const T* __restrict__ zbar, const T* __restrict__ t, T* __restrict__ d, size_t count) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const T tv = t[p];
  d[p] = zbar[p] * (T(1) - tv * tv);
}

// out[b][p][c] = in[b][p][c] / aC[b][p]; aC is the first plane of op [b][5][N]
template <typename T>
__global__ void div_diag_kernel(const T* __restrict__ in, const double* __restrict__ op, T* __restrict__ out,
                                size_t N, int C, int B) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * N * C) return;
  const size_t pix = q / C;
  const size_t b = pix / N, p = pix - b * N;
  out[q] = (T)((double)in[q] / op[b * 5 * N + p]);
}

// d[b][p] = 1 / a_C[b][p] (first plane of op [b][5][N])
template <typename T>
__global__ void dinv_kernel(const double* __restrict__ op, T* __restrict__ d, size_t N, int B) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (size_t)B * N) return;
  const size_t b = q / N, p = q - b * N;
  d[q] = (T)(1.0 / op[b * 5 * N + p]);
}

template <typename T>
__global__ void copy_cast_kernel(const double* __restrict__ src, T* __restrict__ dst, size_t count) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) dst[p] = (T)src[p];
}

// out = base - A v  (transpose = 0)  or  out = -A^T v  (transpose = 1, base ignored),
// op [b][5][N] FP64 (a_C, a_W, a_E, a_S, a_N), v/out [b][N].
template <typename T>
__global__ void stencil_kernel(const double* __restrict__ op, const T* __restrict__ v, const T* __restrict__ base,
                               T* __restrict__ out, int n, int transpose) {
  const size_t N = (size_t)n * n;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int)N) return;
  const size_t b = blockIdx.y;
  op += b * 5 * N;
  v += b * N;
  out += b * N;
  const int j = p / n, i = p - j * n;
  const T vC = v[p];
  T acc = (T)op[p] * vC;
  if (!transpose) {
    if (i > 0) acc += (T)op[N + p] * v[p - 1];
    if (i < n - 1) acc += (T)op[2 * N + p] * v[p + 1];
    if (j > 0) acc += (T)op[3 * N + p] * v[p - n];
    if (j < n - 1) acc += (T)op[4 * N + p] * v[p + n];
    out[p] = base[b * N + p] - acc;
  } else {
    // (A^T v)_q = sum_p A[p][q] v_p: q is the W neighbour of q+1, the E neighbour of q-1, ...
    if (i < n - 1) acc += (T)op[N + p + 1] * v[p + 1];
    if (i > 0) acc += (T)op[2 * N + p - 1] * v[p - 1];
    if (j < n - 1) acc += (T)op[3 * N + p + n] * v[p + n];
    if (j > 0) acc += (T)op[4 * N + p - n] * v[p - n];
    out[p] = -acc;
  }
}

// Per-problem sum of squares: partial[b][blk], one double per block.
template <typename T>
__global__ void sumsq_batched_kernel(const T* __restrict__ v, size_t N, double* __restrict__ partial) {
  __shared__ double sm[32];
  const size_t b = blockIdx.y;
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double x = (p < N) ? (double)v[b * N + p] : 0.0;
  x *= x;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    x = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (threadIdx.x == 0) partial[b * gridDim.x + blockIdx.x] = x;
  }
}

// out[b] = sum_k partial[b][k], fixed order
__global__ void rows_sum_kernel(const double* __restrict__ partial, int cols, double* __restrict__ out, int rows) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= rows) return;
  double s = 0.0;
  for (int k = 0; k < cols; ++k) s += partial[(size_t)b * cols + k];
  out[b] = s;
}

// g = 2 r / (Ntot ||f||^2) per problem
template <typename T>
__global__ void loss_seed_kernel(const T* __restrict__ r, const double* __restrict__ fn2, double Ntot,
                                 T* __restrict__ g, size_t N) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t b = blockIdx.y;
  if (p < N) g[b * N + p] = (T)(2.0 * (double)r[b * N + p] / (Ntot * fn2[b]));
}

// ---------------------------------------------------------------------------
// Weight gradient: out[ia][ib][tap] += sum over positions p of A[p][ia] * G(p, tap)[ib]
//   MODE 0 (same conv):  p = fine pixel, A = y_bar, G = input at p + (a-1, b-1), zero outside
//   MODE 1 (RCNN):       p = coarse pixel, A = y_bar (coarse), G = fine input at (2J+a, 2I+b)
//   MODE 2 (TCNN):       p = coarse pixel, A = coarse input, G = fine y_bar at (2J+a, 2I+b)
// Positions run over all problems of the batch.  Each block walks tiles of
// kPos positions, staging A and the gathered G in shared memory; each thread
// owns a fixed set of outputs and keeps their sums in registers; the block
// writes its partial sums, reduced afterwards in a fixed order.
constexpr int kPos = 32;
constexpr int kWgThreads = 256;

template <typename T, int MODE, int NA, int NB>
__global__ void __launch_bounds__(kWgThreads) wgrad_kernel(const T* __restrict__ A, const T* __restrict__ G,
                                                           int n_pos_side, int n_g_side, int B,
                                                           double* __restrict__ partial) {
  constexpr int NOUT = NA * NB * 9;
  constexpr int PER = (NOUT + kWgThreads - 1) / kWgThreads;
  __shared__ T sA[kPos][NA];
  __shared__ T sG[kPos][9][NB];
  const size_t Np = (size_t)n_pos_side * n_pos_side;
  const size_t Ng = (size_t)n_g_side * n_g_side;
  const size_t total = Np * B;
  double acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.0;
  for (size_t base = (size_t)blockIdx.x * kPos; base < total; base += (size_t)gridDim.x * kPos) {
    __syncthreads();
    for (int e = threadIdx.x; e < kPos * NA; e += blockDim.x) {
      const int pp = e / NA, ia = e - pp * NA;
      const size_t gp = base + pp;
      sA[pp][ia] = (gp < total) ? A[gp * NA + ia] : T(0);
    }
    for (int e = threadIdx.x; e < kPos * 9 * NB; e += blockDim.x) {
      const int pp = e / (9 * NB), rem = e - pp * 9 * NB, tap = rem / NB, ib = rem - tap * NB;
      const size_t gp = base + pp;
      T v = T(0);
      if (gp < total) {
        const size_t b = gp / Np, q = gp - b * Np;
        const int j = (int)(q / n_pos_side), i = (int)(q - (size_t)j * n_pos_side);
        int jj, ii;
        if (MODE == 0) {
          jj = j + tap / 3 - 1;
          ii = i + tap % 3 - 1;
        } else {
          jj = 2 * j + tap / 3;
          ii = 2 * i + tap % 3;
        }
        if (jj >= 0 && jj < n_g_side && ii >= 0 && ii < n_g_side) v = G[(b * Ng + (size_t)jj * n_g_side + ii) * NB + ib];
      }
      sG[pp][tap][ib] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int o = threadIdx.x + k * kWgThreads;
      if (o < NOUT) {
        const int ia = o / (NB * 9), rem = o - ia * NB * 9, ib = rem / 9, tap = rem - ib * 9;
        double s = 0.0;
        for (int pp = 0; pp < kPos; ++pp) s += (double)sA[pp][ia] * (double)sG[pp][tap][ib];
        acc[k] += s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int o = threadIdx.x + k * kWgThreads;
    if (o < NOUT) partial[(size_t)blockIdx.x * NOUT + o] = acc[k];
  }
}

// grad[o] += sum_blk partial[blk][o]
__global__ void wgrad_reduce_kernel(const double* __restrict__ partial, int blocks, int nout, double* __restrict__ grad) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  double s = 0.0;
  for (int k = 0; k < blocks; ++k) s += partial[(size_t)k * nout + o];
  grad[o] += s;
}

// bias gradient: grad[c] += sum over all pixels of d[.][c]
template <typename T>
__global__ void bias_grad_kernel(const T* __restrict__ d, size_t pixels, int C, double* __restrict__ partial) {
  extern __shared__ double sb[];
  for (int c = threadIdx.x; c < C; c += blockDim.x) sb[c] = 0.0;
  __syncthreads();
  double loc[16];
  for (int c = 0; c < C; ++c) loc[c] = 0.0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < pixels; p += (size_t)gridDim.x * blockDim.x)
    for (int c = 0; c < C; ++c) loc[c] += (double)d[p * C + c];
  for (int c = 0; c < C; ++c) {
    double v = loc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sb[c], v);  // shared-memory only, per block
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) partial[(size_t)blockIdx.x * C + c] = sb[c];
}

__global__ void adam_kernel(double* __restrict__ w, double* __restrict__ m, double* __restrict__ v,
                            const double* __restrict__ g, size_t count, double lr, double b1, double b2, double eps,
                            double c1, double c2) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const double gv = g[p];
  const double mv = b1 * m[p] + (1.0 - b1) * gv;
  const double vv = b2 * v[p] + (1.0 - b2) * gv * gv;
  m[p] = mv;
  v[p] = vv;
  w[p] -= lr * (mv / c1) / (sqrt(vv / c2) + eps);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

template <typename T>
struct Trainer {
  mgcnn_ctx* c;
  TrainGroup& g;
  const T* W;     // weights in T
  const T* WT;    // transposed-flipped copies (same offsets as W for the same-conv layers)
  double* grad;   // FP64 gradient accumulator (weight-blob layout)
  cudaStream_t st;
  int C;
  const WeightLayout& wl;

  Trainer(mgcnn_ctx* c_, TrainGroup& g_, const T* W_, const T* WT_, double* grad_)
      : c(c_), g(g_), W(W_), WT(WT_), grad(grad_), st(c_->stream), C(c_->cfg.channels), wl(c_->wl) {}

  T* buf(DevBuf& b) { return b.as<T>(); }
  size_t N(int l) const { return g.lv[l].N(); }
  int nl(int l) const { return g.lv[l].n; }

  // ---- forward pieces -------------------------------------------------------
  Status conv(int CI, int CO, const T* x, const T* s, const T* Wp, const T* bias, const T* skip,
              const double* diag, T* y, int l, int tanh_act = 0) {
    ConvArgs<T> a;
    a.x = x; a.s = s; a.W = Wp; a.bias = bias; a.skip = skip; a.diag = diag; a.y = y; a.n = nl(l);
    a.tanh_act = tanh_act; a.batch = g.B;
    a.x_bs = N(l) * CI; a.s_bs = N(l) * CI; a.skip_bs = N(l) * CO; a.y_bs = N(l) * CO; a.diag_bs = 5 * N(l);
    return conv_same<T>(CI, CO, a, st);
  }

  // Algorithm 2 for the batch; keeps c_l, z_i, t_i (tanh outputs) and s_l.
  Status setup_forward() {
    const size_t CC9 = (size_t)C * C * 9;
    MG_TRY(conv(kFeatures, C, buf(g.feat), nullptr, W + wl.sw_in, W + wl.sb_in, nullptr, nullptr, buf(g.c[0]), 0));
    for (int l = 0; l < g.L; ++l) {
      const T* z = buf(g.c[l]);
      for (int i = 0; i < kSetupLayers; ++i) {
        // t_i = tanh(K_i z_i + b_i) (stored), z_{i+1} = t_i + z_i
        MG_TRY(conv(C, C, z, nullptr, W + wl.sw + i * CC9, W + wl.sb + (size_t)i * C, nullptr, nullptr,
                    buf(g.t[l][i]), l, 1));
        T* znext = (i == kSetupLayers - 1) ? buf(g.tmp[l]) : buf(g.z[l][i + 1]);
        add(buf(g.t[l][i]), z, znext, g.B * N(l) * C);
        if (i + 1 < kSetupLayers) z = znext;
      }
      // s_l = z_4 / a_C, z_4 (h_l/h_1)^2, or z_4
      if (c->cfg.scale_by_diag == 1) {
        div_diag_kernel<T><<<grid_for(g.B * N(l) * C, 256), 256, 0, st>>>(buf(g.tmp[l]), g.op[l].as<double>(),
                                                                           buf(g.s[l]), N(l), C, g.B);
        MG_LAUNCH("div_diag_kernel");
      } else {
        scale_copy(buf(g.tmp[l]), buf(g.s[l]), g.B * N(l) * C, level_factor(l));
      }
      if (l + 1 < g.L) MG_TRY(rcnn<T>(C, buf(g.c[l]), W + wl.sw_R, buf(g.c[l + 1]), nl(l), st, g.B));
    }
    return {};
  }

  void add(const T* a, const T* b, T* out, size_t count);

  // The up loop needs x_pre_up[l] = x_down[l] before the coarser level adds into it.
  Status solve_forward_full(const T* r, T* e) {
    // copy of x_down into the pre-up slot happens as soon as x_down exists
    const size_t CC9 = (size_t)C * C * 9;
    MG_TRY(conv(1, C, r, nullptr, W + wl.w_in, nullptr, nullptr, nullptr, buf(g.x0[0]), 0));
    for (int l = 0; l < g.L; ++l) {
      MG_CUDA(cudaMemcpyAsync(g.xd[l][0].p, g.x0[l].p, g.B * N(l) * C * sizeof(T), cudaMemcpyDeviceToDevice, st));
      for (int i = 0; i < wl.nu_d; ++i) {
        T* y = (i == wl.nu_d - 1) ? buf(g.xdown[l]) : buf(g.xd[l][i + 1]);
        MG_TRY(conv(C, C, buf(g.xd[l][i]), buf(g.s[l]), W + wl.w_down + i * CC9, nullptr, buf(g.xd[l][i]), nullptr, y, l));
      }
      MG_CUDA(cudaMemcpyAsync(g.xu[l][0].p, g.xdown[l].p, g.B * N(l) * C * sizeof(T), cudaMemcpyDeviceToDevice, st));
      if (l + 1 < g.L) MG_TRY(rcnn<T>(C, buf(g.xdown[l]), W + wl.w_R, buf(g.x0[l + 1]), nl(l), st, g.B));
    }
    for (int l = g.L - 1; l >= 0; --l) {
      for (int i = 0; i < wl.nu_u; ++i) {
        T* y = (i == wl.nu_u - 1) ? buf(g.xfin[l]) : buf(g.xu[l][i + 1]);
        MG_TRY(conv(C, C, buf(g.xu[l][i]), buf(g.s[l]), W + wl.w_up + i * CC9, nullptr, buf(g.xu[l][i]), nullptr, y, l));
      }
      if (l > 0) MG_TRY(tcnn_add<T>(C, buf(g.xfin[l]), W + wl.w_P, buf(g.xu[l - 1][0]), nl(l - 1), st, g.B));
    }
    MG_TRY(conv(C, 1, buf(g.xfin[0]), nullptr, W + wl.w_out, nullptr, nullptr, nullptr, e, 0));
    return {};
  }

  // ---- weight gradients -------------------------------------------------------
  template <int MODE, int NA, int NB>
  Status wgrad_launch(const T* A, const T* G, int pos_side, int g_side, double* gout) {
    constexpr int NOUT = NA * NB * 9;
    const size_t total = (size_t)pos_side * pos_side * g.B;
    int blocks = (int)std::min<size_t>((total + kPos - 1) / kPos, 2 * 152);
    MG_TRY(ensure(g.wpart, (size_t)blocks * NOUT * sizeof(double)));
    wgrad_kernel<T, MODE, NA, NB><<<blocks, kWgThreads, 0, st>>>(A, G, pos_side, g_side, g.B, g.wpart.as<double>());
    MG_LAUNCH("wgrad_kernel");
    wgrad_reduce_kernel<<<grid_for(NOUT, 128), 128, 0, st>>>(g.wpart.as<double>(), blocks, NOUT, gout);
    MG_LAUNCH("wgrad_reduce_kernel");
    return {};
  }

  // dispatch over (NA, NB) for C and the 1-channel / 5-feature layers
  template <int MODE>
  Status wgrad(int NA, int NB, const T* A, const T* G, int pos_side, int g_side, double* gout) {
    switch (C) {
#define MG_WG_CASE(CC)                                                                     \
  case CC:                                                                                 \
    if (NA == CC && NB == CC) return wgrad_launch<MODE, CC, CC>(A, G, pos_side, g_side, gout); \
    if (NA == CC && NB == 1) return wgrad_launch<MODE, CC, 1>(A, G, pos_side, g_side, gout);   \
    if (NA == 1 && NB == CC) return wgrad_launch<MODE, 1, CC>(A, G, pos_side, g_side, gout);   \
    if (NA == CC && NB == kFeatures) return wgrad_launch<MODE, CC, kFeatures>(A, G, pos_side, g_side, gout); \
    break;
      MG_WG_CASE(4)
      MG_WG_CASE(8)
      MG_WG_CASE(12)
      MG_WG_CASE(13)
      MG_WG_CASE(16)
#undef MG_WG_CASE
      default: break;
    }
    return make_status(MGCNN_ERR_SIZE, "wgrad: unsupported channels %d x %d", NA, NB);
  }

  Status bias_grad(const T* d, size_t pixels, double* gout) {
    const int blocks = (int)std::min<size_t>(grid_for(pixels, 256), 2 * 152);
    MG_TRY(ensure(g.wpart, (size_t)blocks * C * sizeof(double)));
    bias_grad_kernel<T><<<blocks, 256, C * sizeof(double), st>>>(d, pixels, C, g.wpart.as<double>());
    MG_LAUNCH("bias_grad_kernel");
    wgrad_reduce_kernel<<<1, 128, 0, st>>>(g.wpart.as<double>(), blocks, C, gout);
    MG_LAUNCH("wgrad_reduce_kernel");
    return {};
  }

  // ---- backward pieces ----------------------------------------------------------
  // y = x + K(s * x) at level l with y_bar in `yb`; writes x_bar into `xb_out`.
  Status resnet_backward(int l, const T* yb, const T* xin, const T* Wl, const T* WTl, double* gW, T* xb_out) {
    const size_t cnt = g.B * N(l) * C;
    // z = s * x (for the weight gradient)
    mul(buf(g.s[l]), xin, buf(g.tmp[l]), cnt);
    MG_TRY(wgrad<0>(C, C, yb, buf(g.tmp[l]), nl(l), nl(l), gW));
    // t = K^T y_bar
    MG_TRY(conv(C, C, yb, nullptr, WTl, nullptr, nullptr, nullptr, buf(g.tmp[l]), l));
    resnet_bwd_kernel<T><<<grid_for(cnt, 256), 256, 0, st>>>(yb, buf(g.s[l]), xin, buf(g.tmp[l]), xb_out,
                                                              buf(g.sbar[l]), cnt);
    MG_LAUNCH("resnet_bwd_kernel");
    (void)Wl;
    return {};
  }

  void mul(const T* a, const T* b, T* out, size_t count);
  void scale_copy(const T* a, T* out, size_t count, double factor);
  // (h_l / h_1)^2 for the grid setup scaling, else 1
  double level_factor(int l) const { return c->cfg.scale_by_diag == 2 ? (double)(1u << (2 * l)) : 1.0; }

  // B^T e_bar at input r (intermediates from solve_forward_full); accumulates weight
  // grads and s_bar; writes r_bar.
  Status solve_backward(const T* r, const T* ebar, T* rbar, const T* WTin, const T* WTout,
                        const T* WTdown, const T* WTup) {
    const size_t CC9 = (size_t)C * C * 9;
    // e = W_out * x_fin[0]
    MG_TRY(wgrad<0>(1, C, ebar, buf(g.xfin[0]), nl(0), nl(0), grad + wl.w_out));
    MG_TRY(conv(1, C, ebar, nullptr, WTout, nullptr, nullptr, nullptr, buf(g.xbf[0]), 0));
    for (int l = 0; l < g.L; ++l) {
      // x_bar of x_fin[l] is in xbf[l]; go back through the up layers
      for (int i = wl.nu_u - 1; i >= 0; --i) {
        T* out = buf(g.xbt[l]);
        MG_TRY(resnet_backward(l, buf(g.xbf[l]), buf(g.xu[l][i]), W + wl.w_up + i * CC9, WTup + i * CC9,
                               grad + wl.w_up + i * CC9, out));
        std::swap(g.xbf[l], g.xbt[l]);
      }
      // pre-up = x_down (+ TCNN(x_fin[l+1])): x_bar_down[l] = x_bar_preup; x_bar_fin[l+1] = RCNN_P(x_bar_preup)
      MG_CUDA(cudaMemcpyAsync(g.xbd[l].p, g.xbf[l].p, g.B * N(l) * C * sizeof(T), cudaMemcpyDeviceToDevice, st));
      if (l + 1 < g.L) {
        MG_TRY(rcnn<T>(C, buf(g.xbf[l]), W + wl.w_P, buf(g.xbf[l + 1]), nl(l), st, g.B));
        MG_TRY(wgrad<2>(C, C, buf(g.xfin[l + 1]), buf(g.xbf[l]), nl(l + 1), nl(l), grad + wl.w_P));
      }
    }
    for (int l = g.L - 1; l >= 0; --l) {
      for (int i = wl.nu_d - 1; i >= 0; --i) {
        T* out = buf(g.xbt[l]);
        MG_TRY(resnet_backward(l, buf(g.xbd[l]), buf(g.xd[l][i]), W + wl.w_down + i * CC9, WTdown + i * CC9,
                               grad + wl.w_down + i * CC9, out));
        std::swap(g.xbd[l], g.xbt[l]);
      }
      if (l > 0) {
        // x0[l] = RCNN_R(x_down[l-1]): x_bar_down[l-1] += TCNN_R(x_bar_x0[l]); dR
        MG_TRY(tcnn_add<T>(C, buf(g.xbd[l]), W + wl.w_R, buf(g.xbd[l - 1]), nl(l - 1), st, g.B));
        MG_TRY(wgrad<1>(C, C, buf(g.xbd[l]), buf(g.xdown[l - 1]), nl(l), nl(l - 1), grad + wl.w_R));
      } else {
        MG_TRY(wgrad<0>(C, 1, buf(g.xbd[0]), r, nl(0), nl(0), grad + wl.w_in));
        MG_TRY(conv(C, 1, buf(g.xbd[0]), nullptr, WTin, nullptr, nullptr, nullptr, rbar, 0));
      }
    }
    return {};
  }

  // Algorithm 2 backward from s_bar.
  Status setup_backward(const T* WTs) {
    const size_t CC9 = (size_t)C * C * 9;
    for (int l = g.L - 1; l >= 0; --l) {
      const size_t cnt = g.B * N(l) * C;
      T* zb = buf(g.zb[l]);
      if (c->cfg.scale_by_diag == 1) {
        div_diag_kernel<T><<<grid_for(cnt, 256), 256, 0, st>>>(buf(g.sbar[l]), g.op[l].as<double>(), zb, N(l), C, g.B);
        MG_LAUNCH("div_diag_kernel");
      } else {
        scale_copy(buf(g.sbar[l]), zb, cnt, level_factor(l));
      }
      for (int i = kSetupLayers - 1; i >= 0; --i) {
        T* d = buf(g.tmp[l]);
        tanh_bwd_kernel<T><<<grid_for(cnt, 256), 256, 0, st>>>(zb, buf(g.t[l][i]), d, cnt);
        MG_LAUNCH("tanh_bwd_kernel");
        const T* zin = (i == 0) ? buf(g.c[l]) : buf(g.z[l][i]);
        MG_TRY(wgrad<0>(C, C, d, zin, nl(l), nl(l), grad + wl.sw + i * CC9));
        MG_TRY(bias_grad(d, g.B * N(l), grad + wl.sb + (size_t)i * C));
        // z_bar_i = z_bar_{i+1} + K_i^T d
        MG_TRY(conv(C, C, d, nullptr, WTs + i * CC9, nullptr, zb, nullptr, buf(g.xbt[l]), l));
        MG_CUDA(cudaMemcpyAsync(zb, g.xbt[l].p, cnt * sizeof(T), cudaMemcpyDeviceToDevice, st));
      }
      // c_bar[l] = z_bar_0 + (from level l+1, already added below)
      add(zb, buf(g.cbar[l]), buf(g.cbar[l]), cnt);
      if (l > 0) {
        // c_l = RCNN_s(c_{l-1})
        MG_TRY(tcnn_add<T>(C, buf(g.cbar[l]), W + wl.sw_R, buf(g.cbar[l - 1]), nl(l - 1), st, g.B));
        MG_TRY(wgrad<1>(C, C, buf(g.cbar[l]), buf(g.c[l - 1]), nl(l), nl(l - 1), grad + wl.sw_R));
      }
    }
    MG_TRY(wgrad<0>(C, kFeatures, buf(g.cbar[0]), buf(g.feat), nl(0), nl(0), grad + wl.sw_in));
    MG_TRY(bias_grad(buf(g.cbar[0]), g.B * N(0), grad + wl.sb_in));
    return {};
  }
};

// add / mul are also used in place (out == a), so their pointers are not __restrict__
template <typename T>
__global__ void add_kernel(const T* a, const T* b, T* out, size_t count) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) out[p] = a[p] + b[p];
}
template <typename T>
__global__ void mul_kernel(const T* a, const T* b, T* out, size_t count) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) out[p] = a[p] * b[p];
}

template <typename T>
__global__ void scale_copy_kernel(const T* __restrict__ a, T* __restrict__ out, size_t count, T factor) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) out[p] = a[p] * factor;
}

template <typename T>
void Trainer<T>::scale_copy(const T* a, T* out, size_t count, double factor) {
  scale_copy_kernel<T><<<grid_for(count, 256), 256, 0, st>>>(a, out, count, (T)factor);
  count_launch();
}

template <typename T>
void Trainer<T>::add(const T* a, const T* b, T* out, size_t count) {
  add_kernel<T><<<grid_for(count, 256), 256, 0, st>>>(a, b, out, count);
  count_launch();
}
template <typename T>
void Trainer<T>::mul(const T* a, const T* b, T* out, size_t count) {
  mul_kernel<T><<<grid_for(count, 256), 256, 0, st>>>(a, b, out, count);
  count_launch();
}

// ---------------------------------------------------------------------------
// group buffers

namespace {

Status alloc_group(mgcnn_ctx* c, TrainGroup& g, int n, int B, int K, size_t tsize) {
  int Lmax = 0;
  while ((1 << (Lmax + 1)) - 1 <= n) ++Lmax;
  Lmax -= 1;
  const int C = c->cfg.channels;
  g.n = n;
  g.B = B;
  g.K = K;
  g.L = c->cfg.levels > 0 ? std::min(c->cfg.levels, Lmax) : Lmax;
  g.lv.assign(g.L, Level{});
  int nl = n;
  for (int l = 0; l < g.L; ++l) {
    g.lv[l].n = nl;
    g.lv[l].h = 1.0 / (nl + 1);
    nl = (nl - 1) / 2;
  }
  const size_t N0 = g.lv[0].N();
  auto T_ = [&](DevBuf& b, size_t count) { return ensure(b, count * tsize); };
  for (int l = 0; l < g.L; ++l) {
    const size_t NC = (size_t)B * g.lv[l].N() * C;
    MG_TRY(ensure(g.op[l], (size_t)B * 5 * g.lv[l].N() * sizeof(double)));
    for (DevBuf* b : {&g.c[l], &g.s[l], &g.sbar[l], &g.tmp[l], &g.x0[l], &g.xdown[l], &g.xfin[l], &g.xbf[l],
                      &g.xbd[l], &g.xbt[l], &g.zb[l], &g.cbar[l]})
      MG_TRY(T_(*b, NC));
    for (int i = 0; i < kSetupLayers; ++i) {
      MG_TRY(T_(g.z[l][i], NC));
      MG_TRY(T_(g.t[l][i], NC));
    }
    for (int i = 0; i < c->wl.nu_d; ++i) MG_TRY(T_(g.xd[l][i], NC));
    for (int i = 0; i < c->wl.nu_u; ++i) MG_TRY(T_(g.xu[l][i], NC));
  }
  MG_TRY(ensure(g.coef, (size_t)(n + 2) * (n + 2) * sizeof(double) * 2));
  MG_TRY(T_(g.feat, (size_t)B * N0 * kFeatures));
  MG_TRY(T_(g.rs, (size_t)(K + 1) * B * N0));
  MG_TRY(T_(g.gv, (size_t)B * N0));
  MG_TRY(T_(g.ev, (size_t)B * N0));
  MG_TRY(T_(g.eb, (size_t)B * N0));
  MG_TRY(T_(g.rb, (size_t)B * N0));
  MG_TRY(T_(g.dinvT, (size_t)B * N0));
  MG_TRY(T_(g.rin, (size_t)B * N0));
  MG_TRY(ensure(g.fn2, (size_t)B * sizeof(double)));
  MG_TRY(ensure(g.rn2, (size_t)B * sizeof(double)));
  MG_TRY(ensure(g.npart, (size_t)B * grid_for(N0, 256) * sizeof(double)));
  return {};
}

}  // namespace

void train_release(mgcnn_ctx* c) {
  for (TrainGroup& g : c->groups) {
    for (int l = 0; l < kMaxLevels; ++l) {
      for (DevBuf* b : {&g.op[l], &g.c[l], &g.s[l], &g.sbar[l], &g.tmp[l], &g.x0[l], &g.xdown[l], &g.xfin[l],
                        &g.xbf[l], &g.xbd[l], &g.xbt[l], &g.zb[l], &g.cbar[l]})
        release(*b);
      for (int i = 0; i < kSetupLayers; ++i) {
        release(g.z[l][i]);
        release(g.t[l][i]);
      }
      for (int i = 0; i < kMaxSweeps; ++i) {
        release(g.xd[l][i]);
        release(g.xu[l][i]);
      }
    }
    for (DevBuf* b : {&g.coef, &g.feat, &g.rs, &g.gv, &g.ev, &g.eb, &g.rb, &g.fn2, &g.rn2, &g.npart, &g.wpart,
                      &g.dinvT, &g.rin})
      release(*b);
  }
  c->groups.clear();
  release(c->grad);
  release(c->wT);
  release(c->adam_m);
  release(c->adam_v);
}

// Loss (and gradient) over problems grouped by size.  Arrays: coeff[i] nodal k
// ((n_i+2)^2; the non-divergence form: mu on the n_i^2 interior nodes) and
// rhs[i] (n_i^2), device or host.
template <typename T>
Status loss_grad_impl(mgcnn_ctx* c, int nprob, const double* const* coeff, const double* const* rhs, const int* ns,
                      int K, double* loss, bool want_grad) {
  const int C = c->cfg.channels;
  const WeightLayout& wl = c->wl;
  const size_t CC9 = (size_t)C * C * 9;
  cudaStream_t st = c->stream;
  const T* W = (sizeof(T) == 8) ? reinterpret_cast<const T*>(c->w64.p) : reinterpret_cast<const T*>(c->w32.p);
  // transposed-flipped weights for the data adjoints (same offsets as the blob)
  MG_TRY(ensure(c->wT, wl.total * sizeof(T)));
  T* WT = c->wT.as<T>();
  auto tflip = [&](size_t off, int CO, int CI) -> Status {
    transpose_flip_kernel<T><<<grid_for((size_t)CO * CI * 9, 256), 256, 0, st>>>(W + off, WT + off, CO, CI);
    MG_LAUNCH("transpose_flip_kernel");
    return {};
  };
  MG_TRY(tflip(wl.w_in, C, 1));
  MG_TRY(tflip(wl.w_out, 1, C));
  for (int i = 0; i < wl.nu_d; ++i) MG_TRY(tflip(wl.w_down + i * CC9, C, C));
  for (int i = 0; i < wl.nu_u; ++i) MG_TRY(tflip(wl.w_up + i * CC9, C, C));
  for (int i = 0; i < kSetupLayers; ++i) MG_TRY(tflip(wl.sw + i * CC9, C, C));
  MG_TRY(ensure(c->grad, wl.total * sizeof(double)));
  MG_CUDA(cudaMemsetAsync(c->grad.p, 0, wl.total * sizeof(double), st));
  // group problems by size, in order of first appearance
  std::vector<int> sizes;
  for (int i = 0; i < nprob; ++i)
    if (std::find(sizes.begin(), sizes.end(), ns[i]) == sizes.end()) sizes.push_back(ns[i]);
  if (c->groups.size() < sizes.size()) c->groups.resize(sizes.size());
  double total = 0.0;
  for (size_t gi = 0; gi < sizes.size(); ++gi) {
    const int n = sizes[gi];
    std::vector<int> members;
    for (int i = 0; i < nprob; ++i)
      if (ns[i] == n) members.push_back(i);
    TrainGroup& g = c->groups[gi];
    const int B = (int)members.size();
    MG_TRY(alloc_group(c, g, n, B, K, sizeof(T)));
    const size_t N0 = g.lv[0].N();
    // operators and features per problem; f into r_0
    const bool div = c->cfg.pde == MGCNN_PDE_DIV_HARMONIC;
    for (int b = 0; b < B; ++b) {
      const int i = members[b];
      const int m = n + 2;
      double* k0 = g.coef.as<double>();
      double* k1 = k0 + (size_t)m * m;
      const size_t cn = div ? (size_t)m * m : N0;
      MG_CUDA(cudaMemcpyAsync(k0, coeff[i], cn * sizeof(double), cudaMemcpyDefault, st));
      for (int l = 0; l < g.L; ++l) {
        const int nlv = g.lv[l].n;
        double* opl = g.op[l].as<double>() + (size_t)b * 5 * g.lv[l].N();
        double* kin = (l % 2 == 0) ? k0 : k1;
        double* kout = (l % 2 == 0) ? k1 : k0;
        if (div) {
          MG_TRY(launch_stencil_div(kin, opl, nlv, c->cfg.bx, c->cfg.by, st));
          if (l + 1 < g.L) MG_TRY(launch_restrict_k(kin, kout, nlv + 2, st, 1, c->coarse_k_arith != 0));
        } else {
          MG_TRY(launch_stencil_nondiv(kin, opl, nlv, c->cfg.bx, c->cfg.by, st));
          if (l + 1 < g.L) MG_TRY(launch_inject_mu(kin, kout, nlv, st));
        }
      }
      MG_TRY(launch_features<T>(g.op[0].as<double>() + (size_t)b * 5 * N0, g.feat.as<T>() + (size_t)b * N0 * kFeatures,
                                n, st));
      // f -> r_0, staged through the FP64 coefficient scratch (stream order keeps it free)
      MG_CUDA(cudaMemcpyAsync(k0, rhs[i], N0 * sizeof(double), cudaMemcpyDefault, st));
      copy_cast_kernel<T><<<grid_for(N0, 256), 256, 0, st>>>(k0, g.rs.as<T>() + (size_t)b * N0, N0);
      MG_LAUNCH("copy_cast_kernel");
    }
    Trainer<T> tr(c, g, W, WT, c->grad.as<double>());
    const bool idiag = c->cfg.input_diag != 0;
    if (idiag) {
      dinv_kernel<T><<<grid_for((size_t)B * N0, 256), 256, 0, st>>>(g.op[0].as<double>(), g.dinvT.as<T>(), N0, B);
      MG_LAUNCH("dinv_kernel");
    }
    // network input for cycle k: r_k, or D^{-1} r_k
    auto net_input = [&](const T* rk) -> const T* {
      if (!idiag) return rk;
      tr.mul(rk, g.dinvT.as<T>(), g.rin.as<T>(), (size_t)B * N0);
      return g.rin.as<T>();
    };
    MG_TRY(tr.setup_forward());
    // K cycles, storing r_k
    for (int k = 0; k < K; ++k) {
      T* rk = g.rs.as<T>() + (size_t)k * B * N0;
      T* rk1 = rk + (size_t)B * N0;
      MG_TRY(tr.solve_forward_full(net_input(rk), g.ev.as<T>()));
      stencil_kernel<T><<<dim3(grid_for(N0, 256), B), 256, 0, st>>>(g.op[0].as<double>(), g.ev.as<T>(), rk, rk1, n, 0);
      MG_LAUNCH("stencil_kernel");
    }
    // per-problem norms of f and r_K
    const int nb = grid_for(N0, 256);
    sumsq_batched_kernel<T><<<dim3(nb, B), 256, 0, st>>>(g.rs.as<T>(), N0, g.npart.as<double>());
    MG_LAUNCH("sumsq_batched_kernel");
    rows_sum_kernel<<<grid_for(B, 64), 64, 0, st>>>(g.npart.as<double>(), nb, g.fn2.as<double>(), B);
    MG_LAUNCH("rows_sum_kernel");
    const T* rK = g.rs.as<T>() + (size_t)K * B * N0;
    sumsq_batched_kernel<T><<<dim3(nb, B), 256, 0, st>>>(rK, N0, g.npart.as<double>());
    MG_LAUNCH("sumsq_batched_kernel");
    rows_sum_kernel<<<grid_for(B, 64), 64, 0, st>>>(g.npart.as<double>(), nb, g.rn2.as<double>(), B);
    MG_LAUNCH("rows_sum_kernel");
    std::vector<double> fn2(B), rn2(B);
    MG_CUDA(cudaMemcpyAsync(fn2.data(), g.fn2.p, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaMemcpyAsync(rn2.data(), g.rn2.p, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < B; ++b) {
      if (!(fn2[b] > 0.0) || !std::isfinite(rn2[b]))
        return make_status(MGCNN_ERR_NONFINITE, "zero right-hand side or non-finite residual in the batch");
      total += rn2[b] / fn2[b];
    }
    if (!want_grad) continue;
    // reverse sweep
    for (int l = 0; l < g.L; ++l) {
      MG_CUDA(cudaMemsetAsync(g.sbar[l].p, 0, (size_t)B * g.lv[l].N() * C * sizeof(T), st));
      MG_CUDA(cudaMemsetAsync(g.cbar[l].p, 0, (size_t)B * g.lv[l].N() * C * sizeof(T), st));
    }
    loss_seed_kernel<T><<<dim3(nb, B), 256, 0, st>>>(rK, g.fn2.as<double>(), (double)nprob, g.gv.as<T>(), N0);
    MG_LAUNCH("loss_seed_kernel");
    for (int k = K - 1; k >= 0; --k) {
      const T* rk = g.rs.as<T>() + (size_t)k * B * N0;
      // e_bar = -A^T g
      stencil_kernel<T><<<dim3(grid_for(N0, 256), B), 256, 0, st>>>(g.op[0].as<double>(), g.gv.as<T>(), nullptr,
                                                                     g.eb.as<T>(), n, 1);
      MG_LAUNCH("stencil_kernel");
      const T* rin = net_input(rk);
      MG_TRY(tr.solve_forward_full(rin, g.ev.as<T>()));
      MG_TRY(tr.solve_backward(rin, g.eb.as<T>(), g.rb.as<T>(), WT + wl.w_in, WT + wl.w_out, WT + wl.w_down,
                               WT + wl.w_up));
      // d(D^{-1} r)/dr = D^{-1}
      if (idiag) tr.mul(g.rb.as<T>(), g.dinvT.as<T>(), g.rb.as<T>(), (size_t)B * N0);
      tr.add(g.gv.as<T>(), g.rb.as<T>(), g.gv.as<T>(), (size_t)B * N0);
    }
    MG_TRY(tr.setup_backward(WT + wl.sw));
  }
  *loss = total / nprob;
  return {};
}

template Status loss_grad_impl<float>(mgcnn_ctx*, int, const double* const*, const double* const*, const int*, int,
                                      double*, bool);
template Status loss_grad_impl<double>(mgcnn_ctx*, int, const double* const*, const double* const*, const int*, int,
                                       double*, bool);

Status adam_step(mgcnn_ctx* c, const double* grad, double lr, double b1, double b2, double eps) {
  const size_t n = c->wl.total;
  if (c->adam_m.bytes < n * sizeof(double)) {
    MG_TRY(ensure(c->adam_m, n * sizeof(double)));
    MG_TRY(ensure(c->adam_v, n * sizeof(double)));
    MG_CUDA(cudaMemsetAsync(c->adam_m.p, 0, n * sizeof(double), c->stream));
    MG_CUDA(cudaMemsetAsync(c->adam_v.p, 0, n * sizeof(double), c->stream));
    c->adam_t = 0;
  }
  c->adam_t += 1;
  const double c1 = 1.0 - std::pow(b1, (double)c->adam_t), c2 = 1.0 - std::pow(b2, (double)c->adam_t);
  adam_kernel<<<grid_for(n, 256), 256, 0, c->stream>>>(c->w64.as<double>(), c->adam_m.as<double>(),
                                                        c->adam_v.as<double>(), grad, n, lr, b1, b2, eps, c1, c2);
  MG_LAUNCH("adam_kernel");
  return {};
}

}  // namespace mgcnn

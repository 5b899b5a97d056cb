// C ABI of libmgcnn.so (declared in include/mgcnn.h).
//
// Drives the setup phase (Algorithm 2 of arXiv 2312.11093), the solve phase
// (Algorithm 3) and the stationary iteration (Eq. 1) on one GPU.  Every
// arithmetic step runs in this library's kernels; this file only sequences
// launches, owns device buffers and moves data across the ABI.
#include <atomic>
#include <algorithm>
#include <cmath>

#include "ops.cuh"
#include "tma.cuh"
#include "mixed.cuh"
#include "train.cuh"
#include "batch.cuh"
#include "gmg.cuh"
#include "solve_graph.cuh"
#include "solvers.cuh"

using namespace mgcnn;

// ---------------------------------------------------------------------------
// Internal helpers
namespace mgcnn {

Status make_status(int code, const char* fmt, ...) {
  Status s;
  s.code = code;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  s.msg = buf;
  return s;
}

Status cuda_status(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? MGCNN_ERR_NOMEM : MGCNN_ERR_CUDA;
  if (e == cudaErrorMemoryAllocation) cudaGetLastError();  // not sticky: clear it
  return make_status(code, "%s: %s", what, cudaGetErrorString(e));
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

Status ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return {};
  release(b);
  if (bytes == 0) return {};
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
  b.p = p;
  b.bytes = bytes;
  return {};
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int prof_begin(mgcnn_ctx* c, int kind) {
  if (!c->prof) return -1;
  if (c->ev_used == c->ev_start.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return -1;
    }
    c->ev_start.push_back(a);
    c->ev_stop.push_back(b);
    c->ev_kind.push_back(kind);
  }
  const size_t i = c->ev_used++;
  c->ev_kind[i] = kind;
  cudaEventRecord(c->ev_start[i], c->stream);
  return (int)i;
}

void prof_end(mgcnn_ctx* c, int slot) {
  if (slot >= 0) cudaEventRecord(c->ev_stop[slot], c->stream);
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace mgcnn

namespace {

int finish(mgcnn_ctx* c, const Status& s) {
  if (c) c->last_error = s.ok() ? std::string() : s.msg;
  return s.code;
}

int levels_of(int n) {
  int m = 0;
  while ((1 << m) - 1 < n) ++m;
  if (n < 3 || (1 << m) - 1 != n) return -1;
  return m - 1;
}

// Device view of a caller array of `count` doubles: the array itself if it is
// device memory, else a copy in `stage`.
Status stage_in(mgcnn_ctx* c, const double* src, size_t count, DevBuf& stage, const double** out) {
  if (is_device_pointer(src)) {
    *out = src;
    return {};
  }
  MG_TRY(ensure(stage, count * sizeof(double)));
  MG_CUDA(cudaMemcpyAsync(stage.p, src, count * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  *out = stage.as<double>();
  return {};
}

// Where to write an output of `count` doubles: the caller's device array, or
// `stage` (copied back by stage_out_finish).
Status stage_out(const double* dst, size_t count, DevBuf& stage, double** out, bool* host) {
  if (is_device_pointer(dst)) {
    *out = const_cast<double*>(dst);
    *host = false;
    return {};
  }
  MG_TRY(ensure(stage, count * sizeof(double)));
  *out = stage.as<double>();
  *host = true;
  return {};
}

// mgcnn_solve's inputs from host memory go on the context's copy stream, so
// that they can overlap the setup kernels that mgcnn_setup / mgcnn_setup_gmg
// leave running on the context's stream (those touch neither c->f nor c->u,
// and every other call synchronises before it returns); join_copies orders the
// stream after them.
Status copy_stream(mgcnn_ctx* c) {
  if (!c->cstream) MG_CUDA(cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
  if (!c->cevent) MG_CUDA(cudaEventCreateWithFlags(&c->cevent, cudaEventDisableTiming));
  return {};
}

Status stage_in_overlapped(mgcnn_ctx* c, const double* src, size_t count, DevBuf& stage, const double** out,
                           bool* copied) {
  if (is_device_pointer(src)) {
    *out = src;
    return {};
  }
  MG_TRY(ensure(stage, count * sizeof(double)));
  MG_TRY(copy_stream(c));
  MG_CUDA(cudaMemcpyAsync(stage.p, src, count * sizeof(double), cudaMemcpyHostToDevice, c->cstream));
  *out = stage.as<double>();
  *copied = true;
  return {};
}

Status join_copies(mgcnn_ctx* c, bool copied) {
  if (!copied) return {};
  MG_CUDA(cudaEventRecord(c->cevent, c->cstream));
  MG_CUDA(cudaStreamWaitEvent(c->stream, c->cevent, 0));
  return {};
}

Status stage_out_finish(mgcnn_ctx* c, double* dst, const double* dev, size_t count, bool host) {
  if (host) MG_CUDA(cudaMemcpyAsync(dst, dev, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return {};
}

}  // namespace

namespace mgcnn {

Status sync(mgcnn_ctx* c) {
  MG_CUDA(cudaStreamSynchronize(c->stream));
  if (c->kerr.p) {
    int flag = 0;
    MG_CUDA(cudaMemcpyAsync(&flag, c->kerr.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    if (flag) {
      // the flag and the grid barriers a kernel may have left mid-way
      MG_CUDA(cudaMemsetAsync(c->kerr.p, 0, kErrWords * sizeof(int), c->stream));
      MG_CUDA(cudaStreamSynchronize(c->stream));
      return make_status(MGCNN_ERR_TIMEOUT,
                         "a fused kernel gave up waiting for its tile copies (TMA) or for a grid barrier");
    }
  }
  return {};
}

// ||v||_2^2 of N doubles into scalars[slot] on the device.
Status sumsq(mgcnn_ctx* c, const double* v, size_t N, int slot) {
  MG_TRY(launch_sumsq(v, N, c->partial.as<double>(), c->stream));
  MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N), c->scalars.as<double>() + slot, c->stream));
  return {};
}

Status read_scalar(mgcnn_ctx* c, int slot, double* out) {
  MG_CUDA(cudaMemcpyAsync(c->h_scalars + slot, c->scalars.as<double>() + slot, sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream));
  MG_TRY(sync(c));
  *out = c->h_scalars[slot];
  return {};
}

}  // namespace mgcnn

namespace {

size_t setup_tensor_count(const mgcnn_ctx* c) {
  size_t t = 0;
  for (int l = 0; l < c->L; ++l) t += c->lv[l].N() * c->cfg.channels;
  return t;
}

// ---- setup network (Algorithm 2) in FP64 or FP32 --------------------------
// out[l] receives setup_out_l, [n_l^2][C].
template <typename T>
Status run_setup_net(mgcnn_ctx* c, const T* W, T* const* out) {
  const int C = c->cfg.channels;
  const WeightLayout& wl = c->wl;
  const size_t CC9 = (size_t)C * C * 9;
  const size_t N0 = c->lv[0].N();
  MG_TRY(ensure(c->feat, N0 * kFeatures * sizeof(T)));
  MG_TRY(ensure(c->setup_a, N0 * C * sizeof(T)));
  MG_TRY(ensure(c->setup_b, N0 * C * sizeof(T)));
  MG_TRY(ensure(c->setup_c, N0 * C * sizeof(T)));
  MG_TRY(ensure(c->setup_d, N0 * C * sizeof(T)));
  T* feat = c->feat.as<T>();
  T* cA = c->setup_a.as<T>();
  T* cB = c->setup_b.as<T>();
  T* zA = c->setup_c.as<T>();
  T* zB = c->setup_d.as<T>();
  MG_TRY(launch_features<T>(c->op[0].as<double>(), feat, c->lv[0].n, c->stream));
  {
    ConvArgs<T> a;
    a.x = feat; a.W = W + wl.sw_in; a.bias = W + wl.sb_in; a.y = cA; a.n = c->lv[0].n;
    MG_TRY(conv_same<T>(kFeatures, C, a, c->stream));
  }
  for (int l = 0; l < c->L; ++l) {
    const int nl = c->lv[l].n;
    const T* zin = cA;
    for (int i = 0; i < kSetupLayers; ++i) {
      T* zout = (i == kSetupLayers - 1) ? out[l] : ((i % 2 == 0) ? zA : zB);
      ConvArgs<T> a;
      a.x = zin; a.W = W + wl.sw + i * CC9; a.bias = W + wl.sb + (size_t)i * C;
      a.skip = zin; a.tanh_act = 1; a.y = zout; a.n = nl;
      if (i == kSetupLayers - 1 && c->cfg.scale_by_diag == 1) a.diag = c->op[l].as<double>();
      if (i == kSetupLayers - 1 && c->cfg.scale_by_diag == 2) a.out_scale = (double)(1u << (2 * l));  // (h_l/h_1)^2
      MG_TRY(conv_same<T>(C, C, a, c->stream));
      zin = zout;
    }
    if (l < c->L - 1) {
      MG_TRY(rcnn<T>(C, cA, W + wl.sw_R, cB, nl, c->stream));
      std::swap(cA, cB);
    }
  }
  return {};
}

// ---- solve phase (Algorithm 3) in FP64 ------------------------------------
// e = B r, or e = u + B r when `u_skip` is given (the update of Eq. 1, fused
// into the last layer).
Status vcycle_fp64(mgcnn_ctx* c, const double* r, double* e, const double* u_skip) {
  const int C = c->cfg.channels;
  const WeightLayout& wl = c->wl;
  const size_t CC9 = (size_t)C * C * 9;
  const double* W = c->w64.as<double>();
  double* x[kMaxLevels];
  double* t[kMaxLevels];
  for (int l = 0; l < c->L; ++l) {
    x[l] = c->xa[l].as<double>();
    t[l] = c->xb[l].as<double>();
  }
  {
    ConvArgs<double> a;
    a.x = r; a.W = W + wl.w_in; a.y = x[0]; a.n = c->lv[0].n;
    if (c->cfg.input_diag) a.s = c->dinv.as<double>();   // Net(D^{-1} r)
    MG_TRY(conv_same<double>(1, C, a, c->stream));
  }
  for (int l = 0; l < c->L; ++l) {
    for (int i = 0; i < wl.nu_d; ++i) {
      ConvArgs<double> a;
      a.x = x[l]; a.s = c->s64[l].as<double>(); a.W = W + wl.w_down + i * CC9;
      a.skip = x[l]; a.y = t[l]; a.n = c->lv[l].n;
      MG_TRY(conv_same<double>(C, C, a, c->stream));
      std::swap(x[l], t[l]);
    }
    if (l < c->L - 1) MG_TRY(rcnn<double>(C, x[l], W + wl.w_R, x[l + 1], c->lv[l].n, c->stream));
  }
  for (int l = c->L - 1; l >= 0; --l) {
    for (int i = 0; i < wl.nu_u; ++i) {
      ConvArgs<double> a;
      a.x = x[l]; a.W = W + wl.w_up + i * CC9;
      // symmetric variant: the adjoint layer x + s * (K^T x) (w_up holds K^T)
      if (c->symmetric)
        a.s_out = c->s64[l].as<double>();
      else
        a.s = c->s64[l].as<double>();
      a.skip = x[l]; a.y = t[l]; a.n = c->lv[l].n;
      MG_TRY(conv_same<double>(C, C, a, c->stream));
      std::swap(x[l], t[l]);
    }
    if (l > 0) MG_TRY(tcnn_add<double>(C, x[l], W + wl.w_P, x[l - 1], c->lv[l - 1].n, c->stream));
  }
  {
    ConvArgs<double> a;
    a.x = x[0]; a.W = W + wl.w_out; a.skip = u_skip; a.y = e; a.n = c->lv[0].n;
    MG_TRY(conv_same<double>(C, 1, a, c->stream));
  }
  return {};
}

}  // namespace

namespace mgcnn {

Status vcycle_any(mgcnn_ctx* c, const double* r, double* e, const double* u_skip) {
  if (c->cfg.precision == MGCNN_PREC_FP64) return vcycle_fp64(c, r, e, u_skip);
  return vcycle_mixed(c, r, e, u_skip);
}

}  // namespace mgcnn

namespace {

// ---- symmetric variant (Remark "Symmetric problem", Sec. 3.3) ---------------
// Tied weights: w_up[i] = the adjoint kernel of w_down[nu-1-i] (channels
// swapped, taps flipped: tap t = 3a + b -> 8 - t), w_P = w_R (the transposed
// conv with the RCNN weights is RCNN^T), w_out = the adjoint of w_in.
void tie_weights(const WeightLayout& wl, double* w) {
  const int C = wl.C, nu = wl.nu_d;
  const size_t CC9 = (size_t)C * C * 9;
  for (int i = 0; i < nu; ++i) {
    const double* kd = w + wl.w_down + (size_t)(nu - 1 - i) * CC9;
    double* ku = w + wl.w_up + (size_t)i * CC9;
    for (int co = 0; co < C; ++co)
      for (int ci = 0; ci < C; ++ci)
        for (int t = 0; t < 9; ++t) ku[((size_t)co * C + ci) * 9 + t] = kd[((size_t)ci * C + co) * 9 + (8 - t)];
  }
  std::copy(w + wl.w_R, w + wl.w_R + CC9, w + wl.w_P);
  for (int ch = 0; ch < C; ++ch)
    for (int t = 0; t < 9; ++t) w[wl.w_out + (size_t)ch * 9 + t] = w[wl.w_in + (size_t)ch * 9 + (8 - t)];
}

// Copy a weight blob (host or device memory) into the context, tied first in
// the symmetric mode.
Status load_weights(mgcnn_ctx* c, const double* w) {
  const size_t count = c->wl.total;
  MG_TRY(ensure(c->w64, count * sizeof(double)));
  MG_TRY(ensure(c->w32, count * sizeof(float)));
  std::vector<double> tied;
  if (c->symmetric) {
    tied.resize(count);
    MG_CUDA(cudaMemcpyAsync(tied.data(), w, count * sizeof(double), cudaMemcpyDefault, c->stream));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    tie_weights(c->wl, tied.data());
    w = tied.data();
  }
  MG_CUDA(cudaMemcpyAsync(c->w64.p, w, count * sizeof(double), cudaMemcpyDefault, c->stream));
  MG_TRY(convert<float>(c->w64.as<double>(), c->w32.as<float>(), count, c->stream));
  MG_TRY(mixed_set_weights(c));
  return sync(c);   // before `tied` goes away
}

Status require_symmetric_problem(const mgcnn_ctx* c) {
  if (!c->symmetric) return make_status(MGCNN_ERR_STATE, "CG and MINRES need the symmetric network (MGCNN_OPT_SYMMETRIC)");
  if (c->cfg.pde != MGCNN_PDE_DIV_HARMONIC || c->cfg.bx != 0.0 || c->cfg.by != 0.0)
    return make_status(MGCNN_ERR_ARG, "CG and MINRES need a symmetric A: the divergence form with b = 0");
  return {};
}

Status require_setup(const mgcnn_ctx* c) {
  if (!c->have_setup) return make_status(MGCNN_ERR_STATE, "mgcnn_setup has not been called");
  return {};
}

// Levels, buffers, coefficient check and the operator on every level (A1).
Status setup_operators(mgcnn_ctx* c, const double* coeff, int n) {
  const int Lmax = levels_of(n);
  if (Lmax < 1) return make_status(MGCNN_ERR_SIZE, "n=%d is not 2^m-1 with m>=2", n);
  if (Lmax > kMaxLevels) return make_status(MGCNN_ERR_SIZE, "n=%d too large", n);
  const int L = c->cfg.levels > 0 ? c->cfg.levels : Lmax;
  if (L > Lmax) return make_status(MGCNN_ERR_SIZE, "%d levels requested, n=%d allows %d", L, n, Lmax);
  c->have_setup = false;
  c->sgraph_valid = false;           // buffers may move: recapture the device loop
  if (c->n != n) c->tuned = c->tile_fixed >= 0;   // tile shapes are tuned per grid size
  c->n = n;
  c->L = L;
  c->lv.assign(L, Level{});
  int nl = n;
  for (int l = 0; l < L; ++l) {
    c->lv[l].n = nl;
    c->lv[l].h = 1.0 / (nl + 1);
    nl = (nl - 1) / 2;
  }
  const int C = c->cfg.channels;
  const bool div = c->cfg.pde == MGCNN_PDE_DIV_HARMONIC;
  for (int l = 0; l < L; ++l) {
    const size_t N = c->lv[l].N();
    const size_t cn = div ? (size_t)(c->lv[l].n + 2) * (c->lv[l].n + 2) : N;
    MG_TRY(ensure(c->coef[l], cn * sizeof(double)));
    MG_TRY(ensure(c->op[l], 5 * N * sizeof(double)));
    if (c->cfg.precision == MGCNN_PREC_FP64) {
      MG_TRY(ensure(c->xa[l], N * C * sizeof(double)));
      MG_TRY(ensure(c->xb[l], N * C * sizeof(double)));
      MG_TRY(ensure(c->s64[l], N * C * sizeof(double)));
    }
  }
  const size_t N0 = c->lv[0].N();
  MG_TRY(ensure(c->partial, std::max((size_t)reduction_blocks(N0), fused_partials_max(c->lv[0].n)) * sizeof(double)));
  MG_TRY(ensure(c->r, N0 * sizeof(double)));
  MG_TRY(ensure(c->e, N0 * sizeof(double)));
  // coefficient in, checked positive and finite
  const size_t cn0 = div ? (size_t)(n + 2) * (n + 2) : N0;
  MG_CUDA(cudaMemcpyAsync(c->coef[0].p, coeff, cn0 * sizeof(double), cudaMemcpyDefault, c->stream));
  int* bad = reinterpret_cast<int*>(c->scalars.as<double>() + 7);
  MG_TRY(launch_count_bad(c->coef[0].as<double>(), cn0, bad, c->stream));
  int hbad = 0;
  MG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MG_TRY(sync(c));
  if (hbad) return make_status(MGCNN_ERR_NONFINITE, "coefficient field has non-finite or non-positive entries");
  MG_TRY(ensure(c->dinv, N0 * sizeof(double)));
  MG_TRY(ensure(c->dinv32, N0 * sizeof(float)));
  // operators on every level (Sec. 2.3: rediscretisation)
  for (int l = 0; l < L; ++l) {
    const int nlv = c->lv[l].n;
    if (div) {
      MG_TRY(launch_stencil_div(c->coef[l].as<double>(), c->op[l].as<double>(), nlv, c->cfg.bx, c->cfg.by, c->stream));
      if (l < L - 1)
        MG_TRY(launch_restrict_k(c->coef[l].as<double>(), c->coef[l + 1].as<double>(), nlv + 2, c->stream, 1,
                                 c->coarse_k_arith != 0));
    } else {
      MG_TRY(launch_stencil_nondiv(c->coef[l].as<double>(), c->op[l].as<double>(), nlv, c->cfg.bx, c->cfg.by, c->stream));
      if (l < L - 1) MG_TRY(launch_inject_mu(c->coef[l].as<double>(), c->coef[l + 1].as<double>(), nlv, c->stream));
    }
  }
  // the FP64 copy of 1/a_C feeds the FP64 network only (an FP64 division per unknown)
  MG_TRY(launch_diag_inverse(c->op[0].as<double>(),
                             c->cfg.precision == MGCNN_PREC_FP64 ? c->dinv.as<double>() : nullptr,
                             c->dinv32.as<float>(), N0, c->stream));
  return {};
}

Status do_setup(mgcnn_ctx* c, const double* coeff, int n) {
  if (!c->have_weights) return make_status(MGCNN_ERR_STATE, "weights not set");
  MG_TRY(setup_operators(c, coeff, n));
  const int L = c->L;
  // setup network (Algorithm 2)
  if (c->cfg.precision == MGCNN_PREC_FP64) {
    double* outs[kMaxLevels];
    for (int l = 0; l < L; ++l) outs[l] = c->s64[l].as<double>();
    MG_TRY(run_setup_net<double>(c, c->w64.as<double>(), outs));
  } else {
    MG_TRY(setup_mixed(c));
  }
  // no synchronisation: the setup kernels run on after the call returns (the
  // solve's input copies overlap them); a kernel error surfaces at the next
  // synchronising call
  MG_CUDA(cudaGetLastError());
  c->have_setup = true;
  return {};
}

}  // namespace

// Used by the mixed-precision translation unit.
namespace mgcnn {
Status run_setup_net_fp32(mgcnn_ctx* c, float* const* out) {
  return run_setup_net<float>(c, c->w32.as<float>(), out);
}
}  // namespace mgcnn

// ---------------------------------------------------------------------------
// ABI
extern "C" {

size_t mgcnn_weight_count(const mgcnn_config* cfg) {
  if (!cfg || !channels_supported(cfg->channels) || cfg->down_layers < 1 || cfg->up_layers < 1) return 0;
  WeightLayout wl;
  wl.build(cfg->channels, cfg->down_layers, cfg->up_layers);
  return wl.total;
}

int mgcnn_create(const mgcnn_config* cfg, mgcnn_ctx** out) {
  if (!cfg || !out) return MGCNN_ERR_ARG;
  *out = nullptr;
  if (!channels_supported(cfg->channels) || cfg->down_layers < 1 || cfg->up_layers < 1 ||
      cfg->down_layers > 16 || cfg->up_layers > 16 || cfg->levels < 0 || cfg->levels > kMaxLevels)
    return MGCNN_ERR_SIZE;
  if ((cfg->precision != MGCNN_PREC_FP64 && cfg->precision != MGCNN_PREC_MIXED_BF16) ||
      (cfg->pde != MGCNN_PDE_DIV_HARMONIC && cfg->pde != MGCNN_PDE_NONDIV) ||
      !std::isfinite(cfg->bx) || !std::isfinite(cfg->by))
    return MGCNN_ERR_ARG;
  if (cfg->precision == MGCNN_PREC_MIXED_BF16 && !mixed_channels_supported(cfg->channels)) return MGCNN_ERR_SIZE;
  if (cfg->scale_by_diag < 0 || cfg->scale_by_diag > 2) return MGCNN_ERR_ARG;
  mgcnn_ctx* c = new (std::nothrow) mgcnn_ctx();
  if (!c) return MGCNN_ERR_NOMEM;
  c->cfg = *cfg;
  c->wl.build(cfg->channels, cfg->down_layers, cfg->up_layers);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MGCNN_ERR_CUDA;
  }
  Status s = ensure(c->scalars, 8 * sizeof(double));
  if (s.ok()) s = ensure(c->kerr, kErrWords * sizeof(int));
  if (s.ok() && cudaMemset(c->kerr.p, 0, kErrWords * sizeof(int)) != cudaSuccess)
    s = make_status(MGCNN_ERR_CUDA, "cudaMemset");
  if (s.ok()) {
    c->tma = new (std::nothrow) TmaMaps();
    if (!c->tma) s = make_status(MGCNN_ERR_NOMEM, "tensor map cache");
  }
  if (s.ok() && cudaMallocHost(&c->h_scalars, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    s = make_status(MGCNN_ERR_NOMEM, "cudaMallocHost");
  }
  if (!s.ok()) {
    mgcnn_destroy(c);
    return s.code;
  }
  *out = c;
  return MGCNN_OK;
}

void mgcnn_destroy(mgcnn_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->cstream) cudaStreamSynchronize(c->cstream);
  release(c->w64); release(c->w32);
  for (int l = 0; l < kMaxLevels; ++l) {
    release(c->coef[l]); release(c->op[l]); release(c->s64[l]); release(c->s16[l]);
    release(c->xa[l]); release(c->xb[l]);
  }
  release(c->setup_a); release(c->setup_b); release(c->setup_c); release(c->setup_d);
  release(c->feat); release(c->f); release(c->u); release(c->u2); release(c->r); release(c->e);
  release(c->r32); release(c->partial); release(c->scalars);
  mixed_release(c);
  train_release(c);
  batch_release(c);
  graph_release(c);
  for (int l = 0; l < kMaxLevels; ++l) {
    release(c->gmg_r[l]);
    release(c->gmg_e[l]);
    release(c->gmg_t[l]);
  }
  for (size_t i = 0; i < c->ev_start.size(); ++i) {
    cudaEventDestroy(c->ev_start[i]);
    cudaEventDestroy(c->ev_stop[i]);
  }
  if (c->cevent) cudaEventDestroy(c->cevent);
  if (c->cstream) cudaStreamDestroy(c->cstream);
  if (c->h_scalars) cudaFreeHost(c->h_scalars);
  release(c->kerr);
  for (DevBuf* b : {&c->kV, &c->kZ, &c->kw, &c->kr, &c->kcoef, &c->kpart}) release(*b);
  release(c->alpha32);
  delete c->tma;
  delete c;
}

int mgcnn_set_stream(mgcnn_ctx* c, void* stream) {
  if (!c) return MGCNN_ERR_ARG;
  Status st = sync(c);   // work a setup left on the old stream
  c->stream = static_cast<cudaStream_t>(stream);
  return finish(c, st);
}

int mgcnn_set_weights(mgcnn_ctx* c, const double* w, size_t count) {
  if (!c || !w) return MGCNN_ERR_ARG;
  if (count != c->wl.total)
    return finish(c, make_status(MGCNN_ERR_ARG, "weight count %zu, expected %zu", count, c->wl.total));
  Status s = [&]() -> Status {
    MG_TRY(load_weights(c, w));
    c->have_weights = true;
    return {};
  }();
  return finish(c, s);
}

int mgcnn_setup(mgcnn_ctx* c, const double* coeff, int n) {
  if (!c || !coeff) return MGCNN_ERR_ARG;
  return finish(c, do_setup(c, coeff, n));
}

namespace {

Status setup_gmg_levels(mgcnn_ctx* c, const double* coeff, int n, const LevelWeights& omega) {
  const bool v10 = c->cfg.channels == kGmgV10Channels && c->cfg.down_layers == 1 && c->cfg.up_layers == 1;
  if (c->cfg.channels != kGmgChannels && !v10)
    return make_status(MGCNN_ERR_SIZE, "GMG-equivalent setup needs %d channels, or %d channels with one down "
                       "and one up layer", kGmgChannels, kGmgV10Channels);
  if (!omega.valid()) return make_status(MGCNN_ERR_ARG, "every Jacobi weight must be in (0, 2)");
  MG_TRY(setup_operators(c, coeff, n));
  for (int l = 0; l < c->L; ++l) {
    const double w = omega.at(l, c->L);
    if (c->cfg.precision == MGCNN_PREC_FP64)
      MG_TRY(launch_gmg_setup(c->op[l].as<double>(), c->s64[l].as<double>(), c->lv[l].n, w, c->stream,
                              l == 0 && c->cfg.input_diag, c->cfg.channels));
    else
      MG_TRY(mixed_gmg_setup_level(c, l, w));
  }
  // no synchronisation, as in do_setup
  MG_CUDA(cudaGetLastError());
  c->have_setup = true;
  return {};
}

}  // namespace

int mgcnn_setup_gmg(mgcnn_ctx* c, const double* coeff, int n, double omega) {
  if (!c || !coeff) return MGCNN_ERR_ARG;
  return finish(c, setup_gmg_levels(c, coeff, n, LevelWeights::uniform(omega)));
}

int mgcnn_setup_gmg_levels(mgcnn_ctx* c, const double* coeff, int n, const double* omega) {
  if (!c || !coeff || !omega) return MGCNN_ERR_ARG;
  return finish(c, setup_gmg_levels(c, coeff, n, LevelWeights{omega[0], omega[1], omega[2]}));
}

int mgcnn_setup_bpx(mgcnn_ctx* c, const double* coeff, int n, double omega) {
  if (!c || !coeff) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    if (!c->symmetric) return make_status(MGCNN_ERR_STATE, "the BPX setup needs the symmetric network");
    if (!(omega > 0.0 && omega <= 2.0)) return make_status(MGCNN_ERR_ARG, "omega must be in (0, 2]");
    MG_TRY(setup_operators(c, coeff, n));
    for (int l = 0; l < c->L; ++l)
      MG_TRY(launch_bpx_setup(c->op[l].as<double>(), c->s64[l].as<double>(), c->lv[l].n, l, omega, c->cfg.channels,
                              c->stream));
    MG_TRY(sync(c));
    c->have_setup = true;
    return {};
  }();
  return finish(c, st);
}

size_t mgcnn_setup_tensor_count(const mgcnn_ctx* c) {
  if (!c || !c->have_setup) return 0;
  return setup_tensor_count(c);
}

int mgcnn_set_setup_tensors(mgcnn_ctx* c, const double* s, size_t count) {
  if (!c || !s) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    if (count != setup_tensor_count(c))
      return make_status(MGCNN_ERR_ARG, "setup tensor count %zu, expected %zu", count, setup_tensor_count(c));
    const double* ds = nullptr;
    MG_TRY(stage_in(c, s, count, c->setup_a, &ds));
    size_t off = 0;
    for (int l = 0; l < c->L; ++l) {
      const size_t m = c->lv[l].N() * c->cfg.channels;
      if (c->cfg.precision == MGCNN_PREC_FP64)
        MG_CUDA(cudaMemcpyAsync(c->s64[l].p, ds + off, m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      else
        MG_TRY(mixed_set_setup_level(c, l, ds + off));
      off += m;
    }
    return sync(c);
  }();
  return finish(c, st);
}

int mgcnn_get_setup_tensors(mgcnn_ctx* c, double* s, size_t count) {
  if (!c || !s) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    if (count != setup_tensor_count(c))
      return make_status(MGCNN_ERR_ARG, "setup tensor count %zu, expected %zu", count, setup_tensor_count(c));
    double* ds = nullptr;
    bool host = false;
    MG_TRY(stage_out(s, count, c->setup_b, &ds, &host));
    size_t off = 0;
    for (int l = 0; l < c->L; ++l) {
      const size_t m = c->lv[l].N() * c->cfg.channels;
      if (c->cfg.precision == MGCNN_PREC_FP64)
        MG_CUDA(cudaMemcpyAsync(ds + off, c->s64[l].p, m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      else
        MG_TRY(mixed_get_setup_level(c, l, ds + off));
      off += m;
    }
    MG_TRY(stage_out_finish(c, s, ds, count, host));
    return sync(c);
  }();
  return finish(c, st);
}

int mgcnn_get_operator(mgcnn_ctx* c, int level, double* out, size_t count) {
  if (!c || !out) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    if (level < 0 || level >= c->L) return make_status(MGCNN_ERR_ARG, "level %d out of range", level);
    const size_t m = 5 * c->lv[level].N();
    if (count != m) return make_status(MGCNN_ERR_ARG, "operator count %zu, expected %zu", count, m);
    MG_CUDA(cudaMemcpyAsync(out, c->op[level].p, m * sizeof(double), cudaMemcpyDefault, c->stream));
    return sync(c);
  }();
  return finish(c, st);
}

int mgcnn_residual(mgcnn_ctx* c, const double* f, const double* u, double* r, double* norm2) {
  if (!c || !f || !u || !r) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    const size_t N = c->lv[0].N();
    const double *df = nullptr, *du = nullptr;
    MG_TRY(stage_in(c, f, N, c->f, &df));
    MG_TRY(stage_in(c, u, N, c->u, &du));
    double* dr = nullptr;
    bool host = false;
    MG_TRY(stage_out(r, N, c->r, &dr, &host));
    MG_TRY(launch_residual(df, du, c->op[0].as<double>(), dr, nullptr, c->partial.as<double>(), c->n, c->stream));
    MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N), c->scalars.as<double>(), c->stream));
    MG_TRY(stage_out_finish(c, r, dr, N, host));
    double v = 0.0;
    MG_TRY(read_scalar(c, 0, &v));
    if (norm2) *norm2 = v;
    return {};
  }();
  return finish(c, st);
}

int mgcnn_vcycle(mgcnn_ctx* c, const double* r, double* e) {
  if (!c || !r || !e) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    const size_t N = c->lv[0].N();
    const double* dr = nullptr;
    MG_TRY(stage_in(c, r, N, c->f, &dr));
    double* de = nullptr;
    bool host = false;
    MG_TRY(stage_out(e, N, c->e, &de, &host));
    MG_TRY(vcycle_any(c, dr, de, nullptr));
    MG_TRY(stage_out_finish(c, e, de, N, host));
    return sync(c);
  }();
  return finish(c, st);
}

int mgcnn_solve_krylov(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int restart, int* iters,
                       double* relres) {
  if (!c || !f || !u || !iters || maxit < 0 || !(tol >= 0.0) || restart < 1 || restart > MGCNN_KRYLOV_MAX_RESTART)
    return MGCNN_ERR_ARG;
  *iters = 0;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    const size_t N = c->lv[0].N();
    const double* df = nullptr;
    MG_TRY(stage_in(c, f, N, c->f, &df));
    double* du = nullptr;
    bool host = false;
    MG_TRY(stage_out(u, N, c->u, &du, &host));
    if (host) MG_CUDA(cudaMemcpyAsync(du, u, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    std::vector<double> hist;
    const Status s = krylov_solve(c, df, du, tol, maxit, restart, iters, hist);
    if (relres) std::copy(hist.begin(), hist.end(), relres);
    MG_TRY(stage_out_finish(c, u, du, N, host));
    MG_TRY(sync(c));
    if (!s.ok()) return s;
    if (hist.back() > tol)
      return make_status(MGCNN_NOT_CONVERGED, "no convergence in %d iterations (relres %.3e)", maxit, hist.back());
    return {};
  }();
  return finish(c, st);
}

// PCG (method 0) or MINRES (method 1) with the symmetric network.
static int symmetric_entry(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int* iters,
                           double* relres, int method) {
  if (!c || !f || !u || !iters || maxit < 0 || !(tol >= 0.0)) return MGCNN_ERR_ARG;
  *iters = 0;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    MG_TRY(require_symmetric_problem(c));
    const size_t N = c->lv[0].N();
    const double* df = nullptr;
    MG_TRY(stage_in(c, f, N, c->f, &df));
    double* du = nullptr;
    bool host = false;
    MG_TRY(stage_out(u, N, c->u, &du, &host));
    if (host) MG_CUDA(cudaMemcpyAsync(du, u, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    std::vector<double> hist;
    const Status s = method == 0 ? pcg_solve(c, df, du, tol, maxit, iters, hist)
                                 : minres_solve(c, df, du, tol, maxit, iters, hist);
    if (relres) std::copy(hist.begin(), hist.end(), relres);
    MG_TRY(stage_out_finish(c, u, du, N, host));
    MG_TRY(sync(c));
    if (!s.ok()) return s;
    if (hist.back() > tol)
      return make_status(MGCNN_NOT_CONVERGED, "no convergence in %d iterations (relres %.3e)", maxit, hist.back());
    return {};
  }();
  return finish(c, st);
}

int mgcnn_solve_pcg(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int* iters, double* relres) {
  return symmetric_entry(c, f, u, tol, maxit, iters, relres, 0);
}

int mgcnn_solve_minres(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int* iters, double* relres) {
  return symmetric_entry(c, f, u, tol, maxit, iters, relres, 1);
}

int mgcnn_solve(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int* iters, double* relres) {
  if (!c || !f || !u || !iters || maxit < 0 || !(tol >= 0.0)) return MGCNN_ERR_ARG;
  *iters = 0;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    const size_t N = c->lv[0].N();
    const double* df = nullptr;
    bool copied = false;
    MG_TRY(stage_in_overlapped(c, f, N, c->f, &df, &copied));
    double* du = nullptr;
    bool host = false;
    MG_TRY(stage_out(u, N, c->u, &du, &host));
    if (host) {
      MG_TRY(copy_stream(c));
      MG_CUDA(cudaMemcpyAsync(du, u, N * sizeof(double), cudaMemcpyHostToDevice, c->cstream));
      copied = true;
    }
    MG_TRY(join_copies(c, copied));
    MG_TRY(sumsq(c, df, N, 1));
    double fn2 = 0.0;
    MG_TRY(read_scalar(c, 1, &fn2));
    if (!std::isfinite(fn2)) return make_status(MGCNN_ERR_NONFINITE, "right-hand side is not finite");
    if (fn2 == 0.0) {
      MG_CUDA(cudaMemsetAsync(du, 0, N * sizeof(double), c->stream));
      if (relres) relres[0] = 0.0;
      MG_TRY(stage_out_finish(c, u, du, N, host));
      return sync(c);
    }
    if (c->device_loop && !c->prof) {   // profiling brackets need plain stream launches
      bool used = false;
      Status d = solve_on_device(c, df, du, tol, maxit, iters, relres, &used, fn2);
      if (used || !d.ok()) {
        MG_TRY(stage_out_finish(c, u, du, N, host));
        MG_TRY(sync(c));
        return d;
      }
    }
    Status result;
    const bool mixed = c->cfg.precision == MGCNN_PREC_MIXED_BF16;
    // mixed path with the fused kernels: the finest down kernel computes r_k itself
    const bool fres = fused_residual_applies(c);
    const bool upres = fused_residual_mode(c) == 2;   // the finest up kernel forms the next residual
    if (fres) MG_TRY(fused_cycle_setup(c, df, du, c->scalars.as<double>() + 1));
    if (upres) {
      MG_TRY(ensure(c->u2, N * sizeof(double)));
      MG_TRY(upres_cycle_setup(c, df, du, c->scalars.as<double>(), c->stream));
    }
    double* ucur = du;   // upres: the iterate alternates between du and c->u2
    for (int k = 0;; ++k) {
      if (fres) {
        MG_TRY(fused_cycle_residual(c, df, du, c->scalars.as<double>(), nullptr, c->stream, true));
      } else if (upres) {
        // ||r_k||^2 is in scalars[0] already
      } else {
        // mixed: the V-cycle consumes an FP32 copy of r (scaled in-kernel), FP64 r is not stored
        const int ps = prof_begin(c, kProfResidual);
        MG_TRY(launch_residual(df, du, c->op[0].as<double>(), mixed ? nullptr : c->r.as<double>(),
                               mixed ? c->r32.as<float>() : nullptr, c->partial.as<double>(), c->n, c->stream,
                               c->cfg.input_diag ? c->dinv32.as<float>() : nullptr));
        prof_end(c, ps);
        MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N), c->scalars.as<double>(), c->stream));
      }
      double rn2 = 0.0;
      MG_TRY(read_scalar(c, 0, &rn2));
      const double rel = std::sqrt(rn2 / fn2);
      *iters = k;
      if (!std::isfinite(rel)) {
        result = make_status(MGCNN_ERR_NONFINITE, "residual norm is not finite at cycle %d", k);
        break;
      }
      if (relres) relres[k] = rel;
      if (c->divtol > 0.0 && rel > c->divtol) {
        result = make_status(MGCNN_ERR_DIVERGED, "relres %.3e above the divergence limit at cycle %d", rel, k);
        break;
      }
      if (rel <= tol) break;
      if (k == maxit) {
        result = make_status(MGCNN_NOT_CONVERGED, "no convergence in %d cycles (relres %.3e)", maxit, rel);
        break;
      }
      if (fres)
        MG_TRY(fused_cycle_rest(c, du, c->scalars.as<double>(), nullptr, c->stream, true));
      else if (upres) {
        double* unext = (ucur == du) ? c->u2.as<double>() : du;
        MG_TRY(upres_cycle(c, df, ucur, unext, c->scalars.as<double>(), nullptr, c->stream, true));
        ucur = unext;
      }
      else if (mixed)
        MG_TRY(vcycle_mixed_r32(c, c->r32.as<float>(), c->scalars.as<double>(), du, du));
      else
        MG_TRY(vcycle_fp64(c, c->r.as<double>(), du, du));
    }
    if (ucur != du) MG_CUDA(cudaMemcpyAsync(du, ucur, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    MG_TRY(stage_out_finish(c, u, du, N, host));
    MG_TRY(sync(c));
    return result;
  }();
  return finish(c, st);
}

static Status refresh_weights(mgcnn_ctx* c) {
  MG_TRY(convert<float>(c->w64.as<double>(), c->w32.as<float>(), c->wl.total, c->stream));
  MG_TRY(mixed_set_weights(c));
  return {};
}

static Status loss_grad_any(mgcnn_ctx* c, int nprob, const double* const* coeff, const double* const* rhs,
                            const int* n, int K, double* loss, bool want_grad) {
  if (!c->have_weights) return make_status(MGCNN_ERR_STATE, "weights not set");
  if (c->symmetric) return make_status(MGCNN_ERR_STATE, "training is not available for the symmetric network");
  if (nprob < 1 || K < 1 || K > 64) return make_status(MGCNN_ERR_ARG, "need nprob >= 1 and 1 <= K <= 64");
  for (int i = 0; i < nprob; ++i) {
    if (!coeff[i] || !rhs[i]) return make_status(MGCNN_ERR_ARG, "null problem array %d", i);
    if (levels_of(n[i]) < 1 || levels_of(n[i]) > kMaxLevels) return make_status(MGCNN_ERR_SIZE, "bad n=%d", n[i]);
  }
  if (c->cfg.precision == MGCNN_PREC_FP64) return loss_grad_impl<double>(c, nprob, coeff, rhs, n, K, loss, want_grad);
  return loss_grad_impl<float>(c, nprob, coeff, rhs, n, K, loss, want_grad);
}

int mgcnn_loss_grad(mgcnn_ctx* c, int nprob, const double* const* coeff, const double* const* rhs, const int* n,
                    int K, double* loss, double* grad) {
  if (!c || !coeff || !rhs || !n || !loss) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(loss_grad_any(c, nprob, coeff, rhs, n, K, loss, grad != nullptr));
    if (grad) MG_CUDA(cudaMemcpyAsync(grad, c->grad.p, c->wl.total * sizeof(double), cudaMemcpyDefault, c->stream));
    return sync(c);
  }();
  return finish(c, st);
}

int mgcnn_adam_step(mgcnn_ctx* c, const double* grad, double lr, double beta1, double beta2, double eps) {
  if (!c || !grad) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    if (!c->have_weights) return make_status(MGCNN_ERR_STATE, "weights not set");
    const double* dg = nullptr;
    MG_TRY(stage_in(c, grad, c->wl.total, c->e, &dg));
    MG_TRY(adam_step(c, dg, lr, beta1, beta2, eps));
    MG_TRY(refresh_weights(c));
    c->have_setup = false;  // setup tensors belong to the old weights
    return sync(c);
  }();
  return finish(c, st);
}

int mgcnn_train_step(mgcnn_ctx* c, int nprob, const double* const* coeff, const double* const* rhs, const int* n,
                     int K, double lr, double* loss, double* grad) {
  if (!c || !coeff || !rhs || !n || !loss) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(loss_grad_any(c, nprob, coeff, rhs, n, K, loss, true));
    if (grad) MG_CUDA(cudaMemcpyAsync(grad, c->grad.p, c->wl.total * sizeof(double), cudaMemcpyDefault, c->stream));
    MG_TRY(adam_step(c, c->grad.as<double>(), lr, 0.9, 0.999, 1e-8));
    MG_TRY(refresh_weights(c));
    c->have_setup = false;
    return sync(c);
  }();
  return finish(c, st);
}

int mgcnn_get_weights(mgcnn_ctx* c, double* w, size_t count) {
  if (!c || !w) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    if (!c->have_weights) return make_status(MGCNN_ERR_STATE, "weights not set");
    if (count != c->wl.total) return make_status(MGCNN_ERR_ARG, "weight count %zu, expected %zu", count, c->wl.total);
    MG_CUDA(cudaMemcpyAsync(w, c->w64.p, count * sizeof(double), cudaMemcpyDefault, c->stream));
    return sync(c);
  }();
  return finish(c, st);
}

int mgcnn_setup_batched(mgcnn_ctx* c, int nprob, const double* const* coeff, const int* n) {
  if (!c || !coeff || !n) return MGCNN_ERR_ARG;
  return finish(c, setup_batched(c, nprob, coeff, n));
}

int mgcnn_check_wait_timeout(mgcnn_ctx* c) {
  if (!c) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(launch_wait_check(c->kerr.as<int>(), 8, c->stream));
    return sync(c);   // turns the device flag into ERR_TIMEOUT and clears it
  }();
  return finish(c, st);
}

int mgcnn_setup_batched_gmg(mgcnn_ctx* c, int nprob, const double* const* coeff, const int* n, double omega) {
  if (!c || !coeff || !n) return MGCNN_ERR_ARG;
  const LevelWeights w = LevelWeights::uniform(omega);
  if (!w.valid()) return finish(c, make_status(MGCNN_ERR_ARG, "omega must be in (0, 2)"));
  return finish(c, setup_batched(c, nprob, coeff, n, &w));
}

int mgcnn_setup_batched_gmg_levels(mgcnn_ctx* c, int nprob, const double* const* coeff, const int* n,
                                   const double* omega) {
  if (!c || !coeff || !n || !omega) return MGCNN_ERR_ARG;
  const LevelWeights w{omega[0], omega[1], omega[2]};
  if (!w.valid()) return finish(c, make_status(MGCNN_ERR_ARG, "every Jacobi weight must be in (0, 2)"));
  return finish(c, setup_batched(c, nprob, coeff, n, &w));
}

int mgcnn_solve_batched(mgcnn_ctx* c, int nprob, const double* const* rhs, double* const* u, double tol, int maxit,
                        int* iters, double* relres, int* status) {
  if (!c || !rhs || !u || maxit < 0 || !(tol >= 0.0)) return MGCNN_ERR_ARG;
  return finish(c, solve_batched(c, nprob, rhs, u, tol, maxit, iters, relres, status));
}

int mgcnn_solve_batched_krylov(mgcnn_ctx* c, int nprob, const double* const* rhs, double* const* u, double tol,
                               int maxit, int restart, int* iters, double* relres, int* status) {
  if (!c || !rhs || !u || maxit < 0 || !(tol >= 0.0)) return MGCNN_ERR_ARG;
  return finish(c, solve_batched_krylov(c, nprob, rhs, u, tol, maxit, restart, iters, relres, status));
}

namespace {

int gmg_solve_levels(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int nu1, int nu2,
                     const LevelWeights& omega, int* iters, double* relres) {
  if (!c || !f || !u || !iters || maxit < 0 || !(tol >= 0.0) || nu1 < 0 || nu2 < 0 || nu1 + nu2 < 1 ||
      !omega.valid())
    return MGCNN_ERR_ARG;
  *iters = 0;
  Status st = [&]() -> Status {
    MG_TRY(require_setup(c));
    const size_t N = c->lv[0].N();
    GmgLevels g;
    g.L = c->L;
    for (int l = 0; l < c->L; ++l) {
      const size_t Nl = c->lv[l].N();
      MG_TRY(ensure(c->gmg_r[l], Nl * sizeof(double)));
      MG_TRY(ensure(c->gmg_e[l], Nl * sizeof(double)));
      MG_TRY(ensure(c->gmg_t[l], Nl * sizeof(double)));
      g.n[l] = c->lv[l].n;
      g.op[l] = c->op[l].as<double>();
      g.r[l] = c->gmg_r[l].as<double>();
      g.e[l] = c->gmg_e[l].as<double>();
      g.t[l] = c->gmg_t[l].as<double>();
    }
    const double* df = nullptr;
    MG_TRY(stage_in(c, f, N, c->f, &df));
    double* du = nullptr;
    bool host = false;
    MG_TRY(stage_out(u, N, c->u, &du, &host));
    if (host) MG_CUDA(cudaMemcpyAsync(du, u, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    MG_TRY(sumsq(c, df, N, 1));
    double fn2 = 0.0;
    MG_TRY(read_scalar(c, 1, &fn2));
    if (!std::isfinite(fn2)) return make_status(MGCNN_ERR_NONFINITE, "right-hand side is not finite");
    Status result;
    if (fn2 == 0.0) {
      MG_CUDA(cudaMemsetAsync(du, 0, N * sizeof(double), c->stream));
      if (relres) relres[0] = 0.0;
    } else {
      for (int k = 0;; ++k) {
        MG_TRY(launch_residual(df, du, c->op[0].as<double>(), g.r[0], nullptr, c->partial.as<double>(), c->n,
                               c->stream));
        MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N), c->scalars.as<double>(), c->stream));
        double rn2 = 0.0;
        MG_TRY(read_scalar(c, 0, &rn2));
        const double rel = std::sqrt(rn2 / fn2);
        *iters = k;
        if (!std::isfinite(rel)) {
          result = make_status(MGCNN_ERR_NONFINITE, "residual norm is not finite at cycle %d", k);
          break;
        }
        if (relres) relres[k] = rel;
        if (rel <= tol) break;
        if (k == maxit) {
          result = make_status(MGCNN_NOT_CONVERGED, "no convergence in %d cycles (relres %.3e)", maxit, rel);
          break;
        }
        MG_TRY(gmg_vcycle(g, 0, nu1, nu2, omega, c->stream));
        MG_TRY(launch_axpy_to(du, g.e[0], du, N, c->stream));
      }
    }
    MG_TRY(stage_out_finish(c, u, du, N, host));
    MG_TRY(sync(c));
    return result;
  }();
  return finish(c, st);
}

}  // namespace

int mgcnn_gmg_solve(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int nu1, int nu2, double omega,
                    int* iters, double* relres) {
  return gmg_solve_levels(c, f, u, tol, maxit, nu1, nu2, LevelWeights::uniform(omega), iters, relres);
}

int mgcnn_gmg_solve_levels(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int nu1, int nu2,
                           const double* omega, int* iters, double* relres) {
  if (!omega) return MGCNN_ERR_ARG;
  return gmg_solve_levels(c, f, u, tol, maxit, nu1, nu2, LevelWeights{omega[0], omega[1], omega[2]}, iters, relres);
}

int mgcnn_set_option(mgcnn_ctx* c, int option, int value) {
  if (!c) return MGCNN_ERR_ARG;
  switch (option) {
    case MGCNN_OPT_FUSED:
      c->fused = value ? 1 : 0;
      c->sgraph_valid = false;
      return finish(c, {});
    case MGCNN_OPT_DEVICE_LOOP:
      c->device_loop = value ? 1 : 0;
      return finish(c, {});
    case MGCNN_OPT_COARSE_K:
      if (value < 0 || value > 1) return finish(c, make_status(MGCNN_ERR_ARG, "coarse k rule is 0 or 1"));
      c->coarse_k_arith = value;
      return finish(c, {});
    case MGCNN_OPT_DIVTOL:
      if (value < 0 || value > 300) return finish(c, make_status(MGCNN_ERR_ARG, "divergence exponent is 0..300"));
      c->divtol = value == 0 ? 0.0 : std::pow(10.0, value);
      return finish(c, {});
    case MGCNN_OPT_COARSE_TAIL:
      if (value < 0) return finish(c, make_status(MGCNN_ERR_ARG, "coarse tail grid side must be >= 0"));
      c->tail_n = value;
      c->sgraph_valid = false;
      c->bmaxit = -1;   // batch graphs are captured again
      return finish(c, {});
    case MGCNN_OPT_FUSED_RESIDUAL:
      if (value < 0 || value > 2) return finish(c, make_status(MGCNN_ERR_ARG, "fused residual mode is 0, 1 or 2"));
      c->fuse_residual = value;
      c->sgraph_valid = false;
      c->tuned = c->tile_fixed >= 0;   // the finest down kernel is tuned in the mode it runs in
      return finish(c, {});
    case MGCNN_OPT_SYMMETRIC: {
      if (value != 0 && value != 1) return finish(c, make_status(MGCNN_ERR_ARG, "symmetric option is 0 or 1"));
      if (value) {
        if (c->cfg.precision != MGCNN_PREC_FP64)
          return finish(c, make_status(MGCNN_ERR_ARG, "the symmetric network runs in FP64 precision"));
        if (c->cfg.input_diag)
          return finish(c, make_status(MGCNN_ERR_ARG, "the symmetric network needs input_diag = 0"));
        if (c->wl.nu_d != c->wl.nu_u)
          return finish(c, make_status(MGCNN_ERR_ARG, "the symmetric network needs down_layers == up_layers"));
      }
      const bool retie = value && !c->symmetric && c->have_weights;
      c->symmetric = value;
      if (!retie) return finish(c, {});
      std::vector<double> w(c->wl.total);
      Status st = [&]() -> Status {
        MG_CUDA(cudaMemcpyAsync(w.data(), c->w64.p, w.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        MG_CUDA(cudaStreamSynchronize(c->stream));
        return load_weights(c, w.data());
      }();
      return finish(c, st);
    }
    case MGCNN_OPT_TILE:
      if (value < -1 || value >= kUpVariants)
        return finish(c, make_status(MGCNN_ERR_ARG, "tile shape %d not in -1..%d", value, kUpVariants - 1));
      c->tile_fixed = value;
      c->sgraph_valid = false;   // the captured loop holds the old shapes
      if (value >= 0) {
        // the up-kernel-only shapes pair with the down kernel's 24 x 32
        for (int l = 0; l < kMaxLevels; ++l) {
          c->tile_var[0][l] = value < kFusedVariants ? value : 4;
          c->tile_var[1][l] = value;
        }
        c->tuned = true;
      } else {
        c->tuned = false;
      }
      return finish(c, {});
    default:
      return finish(c, make_status(MGCNN_ERR_ARG, "unknown option %d", option));
  }
}

long long mgcnn_kernel_launches(void) { return g_launches.load(); }

int mgcnn_profile(mgcnn_ctx* c, int enable) {
  if (!c) return MGCNN_ERR_ARG;
  c->prof = enable ? 1 : 0;
  c->ev_used = 0;
  return finish(c, {});
}

int mgcnn_profile_read(mgcnn_ctx* c, double* ms, long long* counts, int nkinds) {
  if (!c || !ms || !counts || nkinds < 1) return MGCNN_ERR_ARG;
  Status st = [&]() -> Status {
    MG_TRY(sync(c));
    for (int k = 0; k < nkinds; ++k) {
      ms[k] = 0.0;
      counts[k] = 0;
    }
    for (size_t i = 0; i < c->ev_used; ++i) {
      const int k = c->ev_kind[i];
      if (k >= nkinds) continue;
      float t = 0.f;
      MG_CUDA(cudaEventElapsedTime(&t, c->ev_start[i], c->ev_stop[i]));
      ms[k] += t;
      counts[k] += 1;
    }
    c->ev_used = 0;
    return {};
  }();
  return finish(c, st);
}

const char* mgcnn_status_string(int s) {
  switch (s) {
    case MGCNN_OK: return "MGCNN_OK";
    case MGCNN_NOT_CONVERGED: return "MGCNN_NOT_CONVERGED";
    case MGCNN_ERR_ARG: return "MGCNN_ERR_ARG";
    case MGCNN_ERR_SIZE: return "MGCNN_ERR_SIZE";
    case MGCNN_ERR_STATE: return "MGCNN_ERR_STATE";
    case MGCNN_ERR_NOMEM: return "MGCNN_ERR_NOMEM";
    case MGCNN_ERR_CUDA: return "MGCNN_ERR_CUDA";
    case MGCNN_ERR_NONFINITE: return "MGCNN_ERR_NONFINITE";
    case MGCNN_ERR_TIMEOUT: return "MGCNN_ERR_TIMEOUT";
    case MGCNN_ERR_DIVERGED: return "MGCNN_ERR_DIVERGED";
    default: return "MGCNN_UNKNOWN_STATUS";
  }
}

const char* mgcnn_last_error(const mgcnn_ctx* c) { return c ? c->last_error.c_str() : ""; }

}  // extern "C"

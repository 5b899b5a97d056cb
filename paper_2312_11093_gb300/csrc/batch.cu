// Batched solves of many coefficient fields and right-hand sides of uneven
// grid sizes (the stationary iteration of Eq. 1 with the mixed-precision solve
// phase of Algorithm 3, one problem per field), as one CUDA graph launch per
// batch: a conditional WHILE node whose body is one cycle of the whole batch.
//
// Problems are grouped into size classes; every buffer of a class holds its
// problems back to back, so each kernel of the cycle covers a whole class
// (grid.z or grid.y = problem).  One cycle of the whole batch is
//   per class, on its own stream (fork/join inside the graph):
//     FP64 residual + per-problem norm      (residual_kernel, batched reduce)
//     convergence check on the device        (active mask, cycle counts, history)
//     fused V-cycle, tile shape per level chosen by the autotuner; blocks of
//     converged problems return at once
//   joined: the loop test (another cycle while any problem is active, at most
//     maxit + 2 cycles) sets the WHILE node's condition on the device
// The host launches the graph once and reads the per-problem states after it.
// (Where conditional graph nodes are unavailable the same body is captured
// as a plain graph and launched once per cycle, with a 4-byte readback each.)
// Setup (operators on every level, Algorithm 2 in FP32, BF16 setup tensors) is
// batched per class the same way.
#include <algorithm>
#include <cmath>

#include "batch.cuh"
#include "ops.cuh"

namespace mgcnn {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ double block_sum_1024(double v, double* smem) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? smem[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// out[b] = sum_k partial[b][k]; one 1024-thread block per problem, the same
// strided order and tree as the single-problem reduction (bit-identical norms).
__global__ void __launch_bounds__(kReduceBlock) rows_reduce_kernel(const double* __restrict__ partial, int count,
                                                                   double* __restrict__ out) {
  __shared__ double smem[32];
  partial += (size_t)blockIdx.x * count;
  double v = 0.0;
  for (int t = threadIdx.x; t < count; t += blockDim.x) v += partial[t];
  v = block_sum_1024(v, smem);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// per-problem partial sums of f^2 (same blocks as the residual kernel)
__global__ void __launch_bounds__(kResidualBlock) sumsq_rows_kernel(const double* __restrict__ v, size_t N,
                                                                    double* __restrict__ partial) {
  __shared__ double smem[32];
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double x = (p < N) ? v[(size_t)blockIdx.y * N + p] : 0.0;
  x = block_sum_1024(x * x, smem);
  if (threadIdx.x == 0) partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = x;
}

// state = [active | iters | status] (3 x B ints)
// First node of a cycle: clear the active-problem count.
__global__ void batch_cycle_begin_kernel(int* __restrict__ counter) {
  if (threadIdx.x == 0 && blockIdx.x == 0) counter[0] = 0;
}

// Last node of a cycle: count it and run another while any problem is active
// (bounded by `limit` cycles).  counter[1] holds the cycles run by this launch.
__global__ void batch_loop_kernel(int* __restrict__ counter, int limit, cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int cycles = counter[1] + 1;
  counter[1] = cycles;
  cudaGraphSetConditional(loop, (counter[0] > 0 && cycles < limit) ? 1u : 0u);
}

__global__ void batch_init_kernel(const double* __restrict__ fn2, int* __restrict__ state, double* __restrict__ u,
                                  size_t N, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double v = fn2[b];
  int act = 1, stat = MGCNN_OK;
  if (!isfinite(v)) {
    act = 0;
    stat = MGCNN_ERR_NONFINITE;
  } else if (v == 0.0) {
    act = 0;   // f = 0: u = 0 is the solution
    for (size_t p = 0; p < N; ++p) u[(size_t)b * N + p] = 0.0;
  }
  state[b] = act;
  state[B + b] = 0;
  state[2 * B + b] = stat;
}

// Before cycle k of an active problem: record ||r_k|| / ||f||, stop on tol,
// maxit or a non-finite norm, otherwise count the cycle about to be applied.
__global__ void batch_check_kernel(const double* __restrict__ rn2, const double* __restrict__ fn2,
                                   int* __restrict__ state, double* __restrict__ hist, int hist_stride,
                                   const double* __restrict__ params, int B, int* __restrict__ counter) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !state[b]) return;
  const double tol = params[0];
  const int maxit = (int)params[1];
  const double divtol = params[2];
  const int it = state[B + b];
  const double rel = sqrt(rn2[b] / fn2[b]);
  if (!isfinite(rel)) {
    state[b] = 0;
    state[2 * B + b] = MGCNN_ERR_NONFINITE;
    return;
  }
  hist[(size_t)b * hist_stride + it] = rel;
  if (divtol > 0.0 && rel > divtol) {
    state[b] = 0;
    state[2 * B + b] = MGCNN_ERR_DIVERGED;
    return;
  }
  if (rel <= tol) {
    state[b] = 0;
    return;
  }
  if (it >= maxit) {
    state[b] = 0;
    state[2 * B + b] = MGCNN_NOT_CONVERGED;
    return;
  }
  state[B + b] = it + 1;
  atomicAdd(counter, 1);
}

__global__ void fill_kernel(double* __restrict__ p, size_t count, double v) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}

int levels_of_n(int n) {
  int m = 0;
  while ((1 << m) - 1 < n) ++m;
  if (n < 3 || (1 << m) - 1 != n) return -1;
  return m - 1;
}

// Algorithm 2 in FP32 for a class, setup tensors into s16[l] (BF16, 8 channels).
Status batched_setup_net(mgcnn_ctx* c, BatchClass& k) {
  const int C = c->cfg.channels;
  const WeightLayout& wl = c->wl;
  const size_t CC9 = (size_t)C * C * 9;
  const float* W = c->w32.as<float>();
  const size_t N0 = (size_t)k.n * k.n;
  cudaStream_t st = k.stream;
  float* feat = k.feat.as<float>();
  float* cA = k.ca.as<float>();
  float* cB = k.cb.as<float>();
  float* zA = k.za.as<float>();
  float* zB = k.zb.as<float>();
  float* s32 = k.s32.as<float>();
  MG_TRY(launch_features<float>(k.op[0].as<double>(), feat, k.n, st, k.B));
  {
    ConvArgs<float> a;
    a.x = feat; a.W = W + wl.sw_in; a.bias = W + wl.sb_in; a.y = cA; a.n = k.n;
    a.batch = k.B; a.x_bs = N0 * kFeatures; a.y_bs = N0 * C;
    MG_TRY(conv_same<float>(kFeatures, C, a, st));
  }
  for (int l = 0; l < k.L; ++l) {
    const int nl = k.nl[l];
    const size_t N = (size_t)nl * nl;
    const float* zin = cA;
    for (int i = 0; i < kSetupLayers; ++i) {
      float* zout = (i == kSetupLayers - 1) ? s32 : ((i % 2 == 0) ? zA : zB);
      ConvArgs<float> a;
      a.x = zin; a.W = W + wl.sw + i * CC9; a.bias = W + wl.sb + (size_t)i * C; a.skip = zin; a.tanh_act = 1;
      a.y = zout; a.n = nl; a.batch = k.B; a.x_bs = a.skip_bs = a.y_bs = N * C; a.diag_bs = 5 * N;
      if (i == kSetupLayers - 1 && c->cfg.scale_by_diag == 1) a.diag = k.op[l].as<double>();
      if (i == kSetupLayers - 1 && c->cfg.scale_by_diag == 2) a.out_scale = (double)(1u << (2 * l));
      MG_TRY(conv_same<float>(C, C, a, st));
      zin = zout;
    }
    MG_TRY(pad_setup_bf16(s32, k.s16[l].as<bf16>(), (size_t)k.B * N, C, 8, st));
    if (l + 1 < k.L) {
      MG_TRY(rcnn<float>(C, cA, W + wl.sw_R, cB, nl, st, k.B));
      std::swap(cA, cB);
    }
  }
  return {};
}

// omega non-null: the analytic setup tensors of the 8-channel GMG V(1, 0)
// network (level l's Jacobi weight omega->at(l, L)) instead of the setup network.
Status setup_class(mgcnn_ctx* c, BatchClass& k, const double* const* coeff, const LevelWeights* omega) {
  const int C = c->cfg.channels;
  const int m0 = k.n + 2;
  const size_t N0 = (size_t)k.n * k.n;
  k.L = levels_of_n(k.n);
  if (c->cfg.levels > 0) k.L = std::min(k.L, c->cfg.levels);
  int nl = k.n;
  for (int l = 0; l < k.L; ++l) {
    k.nl[l] = nl;
    nl = (nl - 1) / 2;
  }
  if (!k.stream) MG_CUDA(cudaStreamCreateWithFlags(&k.stream, cudaStreamNonBlocking));
  if (!k.done) MG_CUDA(cudaEventCreateWithFlags(&k.done, cudaEventDisableTiming));
  const size_t B = k.B;
  MG_TRY(ensure(k.coef, 2 * B * m0 * m0 * sizeof(double)));
  for (int l = 0; l < k.L; ++l) {
    const size_t N = (size_t)k.nl[l] * k.nl[l];
    MG_TRY(ensure(k.op[l], B * 5 * N * sizeof(double)));
    MG_TRY(ensure(k.s16[l], B * N * 8 * sizeof(bf16)));
    MG_TRY(ensure(k.xa[l], B * N * 8 * sizeof(bf16)));
    MG_TRY(ensure(k.xb[l], B * N * 8 * sizeof(bf16)));
    if (l > 0) MG_TRY(ensure(k.xl[l], B * N * 8 * sizeof(bf16)));
  }
  MG_TRY(ensure(k.dinv32, B * N0 * sizeof(float)));
  MG_TRY(ensure(k.r32, B * r32_floats(k.n) * sizeof(float)));
  MG_TRY(ensure(k.f, B * N0 * sizeof(double)));
  MG_TRY(ensure(k.u, B * N0 * sizeof(double)));
  MG_TRY(ensure(k.scratch, B * N0 * sizeof(double)));
  MG_TRY(ensure(k.partial, B * reduction_blocks(N0) * sizeof(double)));
  MG_TRY(ensure(k.rn2, B * sizeof(double)));
  MG_TRY(ensure(k.alpha, 2 * B * sizeof(float)));
  MG_TRY(ensure(k.fn2, B * sizeof(double)));
  MG_TRY(ensure(k.state, 3 * B * sizeof(int)));
  if (!c->fused) {   // FP32 scratch of the unfused setup network only
    MG_TRY(ensure(k.feat, B * N0 * kFeatures * sizeof(float)));
    for (DevBuf* b : {&k.ca, &k.cb, &k.za, &k.zb, &k.s32}) MG_TRY(ensure(*b, B * N0 * C * sizeof(float)));
  }
  cudaStream_t st = k.stream;
  // coefficients in, checked positive and finite
  double* k0 = k.coef.as<double>();
  for (size_t b = 0; b < B; ++b)
    MG_CUDA(cudaMemcpyAsync(k0 + b * m0 * m0, coeff[k.members[b]], (size_t)m0 * m0 * sizeof(double), cudaMemcpyDefault, st));
  int* bad = k.state.as<int>();
  MG_TRY(launch_count_bad(k0, B * m0 * m0, bad, st));
  int hbad = 0;
  MG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
  if (hbad) return make_status(MGCNN_ERR_NONFINITE, "a coefficient field of size %d has non-positive entries", k.n);
  // operators on every level; k ping-pongs between the two halves of coef
  double* kh[2] = {k0, k0 + B * m0 * m0};
  for (int l = 0; l < k.L; ++l) {
    MG_TRY(launch_stencil_div(kh[l & 1], k.op[l].as<double>(), k.nl[l], c->cfg.bx, c->cfg.by, st, k.B));
    if (l + 1 < k.L)
      MG_TRY(launch_restrict_k(kh[l & 1], kh[(l + 1) & 1], k.nl[l] + 2, st, k.B, c->coarse_k_arith != 0));
  }
  MG_TRY(launch_diag_inverse(k.op[0].as<double>(), nullptr, k.dinv32.as<float>(), N0, st, k.B));
  if (omega) {
    for (int l = 0; l < k.L; ++l)
      MG_TRY(launch_gmg_v10_setup_bf16(k.op[l].as<double>(), k.s16[l].as<bf16>(), k.nl[l], omega->at(l, k.L), st,
                                       l == 0 && c->cfg.input_diag, k.B));
  } else if (c->fused) {
    const double* ops[kMaxLevels];
    bf16* ss[kMaxLevels];
    bf16* cs[kMaxLevels];
    for (int l = 0; l < k.L; ++l) {
      ops[l] = k.op[l].as<double>();
      ss[l] = k.s16[l].as<bf16>();
      cs[l] = k.xb[l].as<bf16>();
    }
    const SetupWeights sw = setup_weights(c);
    MG_TRY(setup_fused_levels(k.L, k.nl, k.B, ops, ss, cs, sw, c->cfg.scale_by_diag, st));
  } else {
    MG_TRY(batched_setup_net(c, k));
  }
  // level geometry for the fused kernels, then autotune the tile shapes
  k.fl = FusedLevels{};
  k.fl.L = k.L;
  k.fl.batch = k.B;
  k.fl.maps = c->tma;
  k.fl.err = c->kerr.as<int>();
  k.fl.alpha = k.alpha.as<float>();
  for (int l = 0; l < k.L; ++l) {
    k.fl.n[l] = k.nl[l];
    k.fl.s[l] = k.s16[l].as<bf16>();
    k.fl.xa[l] = k.xa[l].as<bf16>();
    k.fl.xb[l] = k.xb[l].as<bf16>();
    k.fl.xbl[l] = k.xl[l].as<bf16>();
  }
  // tile shapes: reuse the choice made for an earlier class of the same size and
  // batch (the timing depends only on the shapes), else time the variants
  for (const auto& tc : c->tuned_classes)
    if (tc.n == k.n && tc.batch == k.B) {
      for (int l = 0; l < k.L; ++l) {
        k.fl.var_down[l] = tc.var[0][l];
        k.fl.var_up[l] = tc.var[1][l];
      }
      MG_CUDA(cudaStreamSynchronize(st));
      return {};
    }
  fill_kernel<<<grid_for(B, 128), 128, 0, st>>>(k.rn2.as<double>(), B, 1.0);
  MG_LAUNCH("fill_kernel");
  MG_CUDA(cudaMemsetAsync(k.r32.p, 0, B * r32_floats(k.n) * sizeof(float), st));
  MG_TRY(fused_autotune(k.fl, k.r32.as<float>(), k.rn2.as<double>(), k.scratch.as<double>(), fused_weights(c), st, 5));
  mgcnn_ctx::TunedClass tc{k.n, k.B, {}};
  for (int l = 0; l < k.L; ++l) {
    tc.var[0][l] = k.fl.var_down[l];
    tc.var[1][l] = k.fl.var_up[l];
  }
  c->tuned_classes.push_back(tc);
  MG_CUDA(cudaStreamSynchronize(st));
  return {};
}

// One cycle of the whole batch (all classes forked on their streams), captured
// from `main`.
Status record_cycle(mgcnn_ctx* c, cudaStream_t main, const FusedWeights& w) {
  batch_cycle_begin_kernel<<<1, 32, 0, main>>>(c->bcount.as<int>());
  MG_LAUNCH("batch_cycle_begin_kernel");
  MG_CUDA(cudaEventRecord(c->bfork, main));
  // coarse tail: one grid-barrier word pair per class; the classes run
  // concurrently, so their tail kernels split the resident blocks
  int pair = 1;
  const int share = std::min((int)c->bcls.size(), kTailBarriers - 1);
  for (BatchClass& k : c->bcls) {
    const size_t N0 = (size_t)k.n * k.n;
    const int nblk = residual_blocks(N0);
    int* state = k.state.as<int>();
    FusedLevels fl = k.fl;
    fl.tail_n = pair < kTailBarriers ? c->tail_n : 0;
    fl.tail_bar = c->kerr.as<unsigned>() + kTailBarrierWord + 2 * pair;
    fl.tail_share = share;
    ++pair;
    MG_CUDA(cudaStreamWaitEvent(k.stream, c->bfork, 0));
    MG_TRY(launch_residual(k.f.as<double>(), k.u.as<double>(), k.op[0].as<double>(), nullptr, k.r32.as<float>(),
                           k.partial.as<double>(), k.n, k.stream,
                           c->cfg.input_diag ? k.dinv32.as<float>() : nullptr, k.B));
    rows_reduce_kernel<<<k.B, kReduceBlock, 0, k.stream>>>(k.partial.as<double>(), nblk, k.rn2.as<double>());
    MG_LAUNCH("rows_reduce_kernel");
    batch_check_kernel<<<grid_for(k.B, 128), 128, 0, k.stream>>>(k.rn2.as<double>(), k.fn2.as<double>(), state,
                                                                  k.hist.as<double>(), c->bmaxit + 1,
                                                                  c->bparams.as<double>(), k.B, c->bcount.as<int>());
    MG_LAUNCH("batch_check_kernel");
    MG_TRY(fused_vcycle_levels(fl, k.r32.as<float>(), k.rn2.as<double>(), k.u.as<double>(), k.u.as<double>(), w,
                               state, k.stream, nullptr));
    MG_CUDA(cudaEventRecord(k.done, k.stream));
    MG_CUDA(cudaStreamWaitEvent(main, k.done, 0));
  }
  return {};
}

Status capture_cycle_once(mgcnn_ctx* c);

// The batch's graph: a conditional WHILE node around one cycle (bwhile), or,
// where that cannot be built, the plain cycle graph launched once per cycle;
// without the coarse tail kernel where neither holds it.
Status capture_cycle(mgcnn_ctx* c) {
  Status s = capture_cycle_once(c);
  if (!s.ok() && c->tail_n > 0) {
    cudaGetLastError();
    c->tail_n = 0;
    s = capture_cycle_once(c);
  }
  return s;
}

Status capture_cycle_once(mgcnn_ctx* c) {
  if (c->bgraph) {
    cudaGraphExecDestroy(c->bgraph);
    c->bgraph = nullptr;
  }
  cudaStream_t main = c->bstream;
  const FusedWeights w = fused_weights(c);
  const long long launches0 = mgcnn_kernel_launches();
  c->bwhile = false;
  {
    cudaGraph_t g = nullptr;
    MG_CUDA(cudaGraphCreate(&g, 0));
    Status s = [&]() -> Status {
      cudaGraphConditionalHandle loop;
      MG_CUDA(cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = loop;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      MG_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
      cudaGraph_t body = np.conditional.phGraph_out[0];
      MG_CUDA(cudaStreamBeginCaptureToGraph(main, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      Status cap = [&]() -> Status {
        MG_TRY(record_cycle(c, main, w));
        batch_loop_kernel<<<1, 32, 0, main>>>(c->bcount.as<int>(), c->bmaxit + 2, loop);
        MG_LAUNCH("batch_loop_kernel");
        return {};
      }();
      cudaGraph_t captured = body;
      const cudaError_t e = cudaStreamEndCapture(main, &captured);
      MG_TRY(cap);
      if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
      MG_CUDA(cudaGraphInstantiate(&c->bgraph, g, 0));
      return {};
    }();
    cudaGraphDestroy(g);
    c->bgraph_kernels = mgcnn_kernel_launches() - launches0;   // kernels per cycle, counted per launch later
    add_launches(-c->bgraph_kernels);
    if (s.ok()) {
      c->bwhile = true;
      return {};
    }
    cudaGetLastError();
    if (c->bgraph) cudaGraphExecDestroy(c->bgraph);
    c->bgraph = nullptr;
  }
  // plain graph of one cycle
  const long long launches1 = mgcnn_kernel_launches();
  cudaGraph_t g = nullptr;
  MG_CUDA(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
  Status s = record_cycle(c, main, w);
  cudaError_t e = cudaStreamEndCapture(main, &g);
  if (!s.ok()) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
  c->bgraph_kernels = mgcnn_kernel_launches() - launches1;   // kernels captured, not launched
  add_launches(-c->bgraph_kernels);
  e = cudaGraphInstantiate(&c->bgraph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate");
  return {};
}

}  // namespace

void batch_release(mgcnn_ctx* c) {
  if (c->bgraph) cudaGraphExecDestroy(c->bgraph);
  c->bgraph = nullptr;
  for (BatchClass& k : c->bcls) {
    release(k.coef);
    for (int l = 0; l < kMaxLevels; ++l) {
      release(k.op[l]); release(k.s16[l]); release(k.xa[l]); release(k.xb[l]); release(k.xl[l]);
    }
    for (DevBuf* b : {&k.dinv32, &k.r32, &k.f, &k.u, &k.partial, &k.rn2, &k.alpha, &k.fn2, &k.state, &k.hist, &k.feat,
                      &k.ca, &k.cb, &k.za, &k.zb, &k.s32, &k.scratch, &k.kV, &k.kZ, &k.kpart, &k.kdbl, &k.kint})
      release(*b);
    if (k.stream) cudaStreamDestroy(k.stream);
    if (k.done) cudaEventDestroy(k.done);
  }
  c->bcls.clear();
  release(c->bparams);
  release(c->bcount);
  if (c->h_bcount) cudaFreeHost(c->h_bcount);
  c->h_bcount = nullptr;
  if (c->bfork) cudaEventDestroy(c->bfork);
  c->bfork = nullptr;
  if (c->bstream) cudaStreamDestroy(c->bstream);
  c->bstream = nullptr;
  c->bready = false;
}

Status setup_batched(mgcnn_ctx* c, int nprob, const double* const* coeff, const int* ns, const LevelWeights* omega) {
  if (!c->have_weights) return make_status(MGCNN_ERR_STATE, "weights not set");
  if (c->cfg.precision != MGCNN_PREC_MIXED_BF16 || !fused_supported(c) || c->cfg.pde != MGCNN_PDE_DIV_HARMONIC)
    return make_status(MGCNN_ERR_SIZE, "batched solves need MIXED_BF16, 8 channels, one layer per ResNet, "
                                       "divergence form");
  if (nprob < 1) return make_status(MGCNN_ERR_ARG, "empty batch");
  for (int i = 0; i < nprob; ++i) {
    if (!coeff[i]) return make_status(MGCNN_ERR_ARG, "null coefficient array %d", i);
    const int L = levels_of_n(ns[i]);
    if (L < 1 || L > kMaxLevels) return make_status(MGCNN_ERR_SIZE, "problem %d: n=%d is not 2^m-1", i, ns[i]);
  }
  batch_release(c);
  MG_CUDA(cudaStreamCreateWithFlags(&c->bstream, cudaStreamNonBlocking));
  MG_CUDA(cudaEventCreateWithFlags(&c->bfork, cudaEventDisableTiming));
  MG_TRY(ensure(c->bparams, 3 * sizeof(double)));
  MG_TRY(ensure(c->bcount, 2 * sizeof(int)));
  MG_CUDA(cudaMallocHost(&c->h_bcount, 2 * sizeof(int)));
  // size classes in order of first appearance
  c->bn = nprob;
  c->bcls_of.assign(nprob, 0);
  c->bidx_of.assign(nprob, 0);
  for (int i = 0; i < nprob; ++i) {
    int ci = -1;
    for (size_t q = 0; q < c->bcls.size(); ++q)
      if (c->bcls[q].n == ns[i]) ci = (int)q;
    if (ci < 0) {
      c->bcls.emplace_back();
      c->bcls.back().n = ns[i];
      ci = (int)c->bcls.size() - 1;
    }
    c->bcls_of[i] = ci;
    c->bidx_of[i] = (int)c->bcls[ci].members.size();
    c->bcls[ci].members.push_back(i);
  }
  for (BatchClass& k : c->bcls) {
    k.B = (int)k.members.size();
    MG_TRY(setup_class(c, k, coeff, omega));
  }
  c->bmaxit = -1;
  c->bready = true;
  return {};
}

Status solve_batched(mgcnn_ctx* c, int nprob, const double* const* rhs, double* const* u, double tol, int maxit,
                     int* iters, double* relres, int* status) {
  if (!c->bready) return make_status(MGCNN_ERR_STATE, "mgcnn_setup_batched has not been called");
  if (nprob != c->bn) return make_status(MGCNN_ERR_ARG, "batch has %d problems, setup had %d", nprob, c->bn);
  for (int i = 0; i < nprob; ++i)
    if (!rhs[i] || !u[i]) return make_status(MGCNN_ERR_ARG, "null array for problem %d", i);
  cudaStream_t main = c->bstream;
  // inputs into the class buffers; f norms; initial state
  for (BatchClass& k : c->bcls) {
    const size_t N0 = (size_t)k.n * k.n;
    for (int b = 0; b < k.B; ++b) {
      const int i = k.members[b];
      MG_CUDA(cudaMemcpyAsync(k.f.as<double>() + b * N0, rhs[i], N0 * sizeof(double), cudaMemcpyDefault, main));
      MG_CUDA(cudaMemcpyAsync(k.u.as<double>() + b * N0, u[i], N0 * sizeof(double), cudaMemcpyDefault, main));
    }
    const int nblk = reduction_blocks(N0);
    sumsq_rows_kernel<<<dim3(nblk, k.B), kResidualBlock, 0, main>>>(k.f.as<double>(), N0, k.partial.as<double>());
    MG_LAUNCH("sumsq_rows_kernel");
    rows_reduce_kernel<<<k.B, kReduceBlock, 0, main>>>(k.partial.as<double>(), nblk, k.fn2.as<double>());
    MG_LAUNCH("rows_reduce_kernel");
    batch_init_kernel<<<grid_for(k.B, 128), 128, 0, main>>>(k.fn2.as<double>(), k.state.as<int>(), k.u.as<double>(),
                                                            N0, k.B);
    MG_LAUNCH("batch_init_kernel");
  }
  const double params[3] = {tol, (double)maxit, c->divtol};
  MG_CUDA(cudaMemcpyAsync(c->bparams.p, params, sizeof(params), cudaMemcpyHostToDevice, main));
  if (maxit != c->bmaxit) {
    for (BatchClass& k : c->bcls) MG_TRY(ensure(k.hist, (size_t)k.B * (maxit + 1) * sizeof(double)));
    c->bmaxit = maxit;
    MG_TRY(capture_cycle(c));
  }
  if (c->bwhile) {
    // every cycle of every problem in one graph launch
    MG_CUDA(cudaMemsetAsync(c->bcount.p, 0, 2 * sizeof(int), main));
    MG_CUDA(cudaGraphLaunch(c->bgraph, main));
    MG_CUDA(cudaMemcpyAsync(c->h_bcount, c->bcount.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, main));
    MG_CUDA(cudaStreamSynchronize(main));
    add_launches(c->bgraph_kernels * (long long)c->h_bcount[1]);
  } else {
    // each graph launch checks every active problem and applies one cycle
    for (int cyc = 0; cyc <= maxit + 1; ++cyc) {
      MG_CUDA(cudaGraphLaunch(c->bgraph, main));
      add_launches(c->bgraph_kernels);
      MG_CUDA(cudaMemcpyAsync(c->h_bcount, c->bcount.p, sizeof(int), cudaMemcpyDeviceToHost, main));
      MG_CUDA(cudaStreamSynchronize(main));
      if (*c->h_bcount == 0) break;
    }
  }
  // results back
  Status overall;
  for (BatchClass& k : c->bcls) {
    const size_t N0 = (size_t)k.n * k.n;
    std::vector<int> st(3 * k.B);
    std::vector<double> h((size_t)k.B * (maxit + 1));
    MG_CUDA(cudaMemcpyAsync(st.data(), k.state.p, st.size() * sizeof(int), cudaMemcpyDeviceToHost, main));
    MG_CUDA(cudaMemcpyAsync(h.data(), k.hist.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, main));
    for (int b = 0; b < k.B; ++b) {
      const int i = k.members[b];
      MG_CUDA(cudaMemcpyAsync(u[i], k.u.as<double>() + b * N0, N0 * sizeof(double), cudaMemcpyDefault, main));
    }
    MG_CUDA(cudaStreamSynchronize(main));
    for (int b = 0; b < k.B; ++b) {
      const int i = k.members[b];
      const int it = st[k.B + b], stat = st[2 * k.B + b];
      if (iters) iters[i] = it;
      if (relres) relres[i] = h[(size_t)b * (maxit + 1) + std::min(it, maxit)];
      if (status) status[i] = stat;
      if (stat < 0 && overall.code >= 0) overall = make_status(stat, "problem %d: %s", i, mgcnn_status_string(stat));
      else if (stat == MGCNN_NOT_CONVERGED && overall.code == MGCNN_OK)
        overall = make_status(MGCNN_NOT_CONVERGED, "problem %d did not converge in %d cycles", i, maxit);
    }
  }
  return overall;
}

}  // namespace mgcnn

// The stationary iteration (Eq. 1 of arXiv 2312.11093) run on the device: the
// whole solve is one launch of a CUDA graph whose only node is a conditional
// WHILE loop.  The loop body -- FP64 residual and norm, convergence test,
// mixed-precision V-cycle (fused level kernels; by default the residual is
// computed inside the finest down kernel) -- is captured once per setup;
// the test kernel records ||r_k|| / ||f||, stops the loop on the tolerance,
// on maxit or on a non-finite norm (cudaGraphSetConditional), and otherwise
// counts the cycle about to be applied.  The V-cycle kernels of the final
// pass see the cleared active flag and return at once.  No host round trip
// happens between cycles.
#include <cmath>

#include "mixed.cuh"
#include "ops.cuh"
#include "solve_graph.cuh"

namespace mgcnn {

namespace {

// state: [0] active, [1] cycles applied, [2] status
__global__ void solve_check_kernel(const double* __restrict__ rn2, const double* __restrict__ fn2,
                                   int* __restrict__ state, double* __restrict__ hist,
                                   const double* __restrict__ params, cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!state[0]) {
    cudaGraphSetConditional(loop, 0);
    return;
  }
  const double tol = params[0];
  const int maxit = (int)params[1];
  const double divtol = params[2];
  const int it = state[1];
  const double rel = sqrt(rn2[0] / fn2[0]);
  if (!isfinite(rel)) {
    state[0] = 0;
    state[2] = MGCNN_ERR_NONFINITE;
    cudaGraphSetConditional(loop, 0);
    return;
  }
  hist[it] = rel;
  if (divtol > 0.0 && rel > divtol) {
    state[0] = 0;
    state[2] = MGCNN_ERR_DIVERGED;
    cudaGraphSetConditional(loop, 0);
    return;
  }
  if (rel <= tol || it >= maxit) {
    state[0] = 0;
    state[2] = (rel <= tol) ? MGCNN_OK : MGCNN_NOT_CONVERGED;
    cudaGraphSetConditional(loop, 0);
    return;
  }
  state[1] = it + 1;
}

Status build_graph(mgcnn_ctx* c) {
  if (c->sgraph) {
    cudaGraphExecDestroy(c->sgraph);
    c->sgraph = nullptr;
  }
  const size_t N0 = c->lv[0].N();
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
    cudaStream_t st = c->gstream;
    MG_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const long long launches0 = mgcnn_kernel_launches();
    Status cap = [&]() -> Status {
      double* sc = c->scalars.as<double>();
      if (fused_residual_mode(c) == 2) {
        // two cycles per pass, u -> u2 -> u: the test on ||r_k||, then the whole
        // cycle, whose finest up kernel forms r_{k+1} and its norm for the next
        // test (r_0 comes before the loop); a stop after the first half leaves
        // the iterate in u2 (odd cycle count)
        double* ua = c->u.as<double>();
        double* ub = c->u2.as<double>();
        for (int half = 0; half < 2; ++half) {
          solve_check_kernel<<<1, 32, 0, st>>>(sc, sc + 1, c->gstate.as<int>(), c->ghist.as<double>(),
                                               c->gparams.as<double>(), loop);
          MG_LAUNCH("solve_check_kernel");
          MG_TRY(upres_cycle(c, c->f.as<double>(), half ? ub : ua, half ? ua : ub, sc, c->gstate.as<int>(), st,
                             false));
        }
        return {};
      }
      if (fused_residual_applies(c)) {
        // r_k and the finest down level in one kernel, ||r_k||^2, the test, the
        // rest of the cycle (u += B r_k) and the next input scale
        MG_TRY(fused_cycle_residual(c, c->f.as<double>(), c->u.as<double>(), sc, nullptr, st, false));
        solve_check_kernel<<<1, 32, 0, st>>>(sc, sc + 1, c->gstate.as<int>(), c->ghist.as<double>(),
                                             c->gparams.as<double>(), loop);
        MG_LAUNCH("solve_check_kernel");
        return fused_cycle_rest(c, c->u.as<double>(), sc, c->gstate.as<int>(), st, false);
      }
      MG_TRY(launch_residual(c->f.as<double>(), c->u.as<double>(), c->op[0].as<double>(), nullptr,
                             c->r32.as<float>(), c->partial.as<double>(), c->n, st,
                             c->cfg.input_diag ? c->dinv32.as<float>() : nullptr));
      MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N0), sc, st));
      solve_check_kernel<<<1, 32, 0, st>>>(sc, sc + 1, c->gstate.as<int>(), c->ghist.as<double>(),
                                           c->gparams.as<double>(), loop);
      MG_LAUNCH("solve_check_kernel");
      FusedLevels fl;
      fl.L = c->L;
      fl.batch = 1;
      fl.maps = c->tma;
      fl.err = c->kerr.as<int>();
      fl.alpha = c->alpha32.as<float>();
      fl.pdl = c->pdl;
      fl.tail_n = c->tail_n;
      fl.tail_bar = c->kerr.as<unsigned>() + kTailBarrierWord;
      for (int l = 0; l < c->L; ++l) {
        fl.n[l] = c->lv[l].n;
        fl.s[l] = c->s16[l].as<__nv_bfloat16>();
        fl.xa[l] = c->x16a[l].as<__nv_bfloat16>();
        fl.xb[l] = c->x16b[l].as<__nv_bfloat16>();
        fl.xbl[l] = c->x16l[l].as<__nv_bfloat16>();
        fl.var_down[l] = c->tile_var[0][l];
        fl.var_up[l] = c->tile_var[1][l];
      }
      MG_TRY(fused_vcycle_levels(fl, c->r32.as<float>(), sc, c->u.as<double>(), c->u.as<double>(), fused_weights(c),
                                 c->gstate.as<int>(), st, nullptr));
      return {};
    }();
    cudaGraph_t captured = body;
    const cudaError_t e = cudaStreamEndCapture(st, &captured);
    c->sgraph_kernels = mgcnn_kernel_launches() - launches0;   // kernels per cycle, counted per launch later
    add_launches(-c->sgraph_kernels);
    MG_TRY(cap);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
    MG_CUDA(cudaGraphInstantiate(&c->sgraph, g, 0));
    return {};
  }();
  cudaGraphDestroy(g);
  return s;
}

}  // namespace

void graph_release(mgcnn_ctx* c) {
  if (c->sgraph) cudaGraphExecDestroy(c->sgraph);
  c->sgraph = nullptr;
  if (c->gstream) cudaStreamDestroy(c->gstream);
  c->gstream = nullptr;
  release(c->gstate);
  release(c->ghist);
  release(c->gparams);
}

// Device-side solve for the mixed path with the fused kernels.  f, u: device
// arrays of n^2 doubles (u in place).  *used = false when the graph could not be
// built (the caller then runs the host loop); the context remembers that.
Status solve_on_device(mgcnn_ctx* c, const double* f, double* u, double tol, int maxit, int* iters,
                       double* relres, bool* used, double fn2_known) {
  *used = false;
  if (c->graph_failed || !(c->cfg.precision == MGCNN_PREC_MIXED_BF16 && c->fused && fused_supported(c))) return {};
  const size_t N0 = c->lv[0].N();
  cudaStream_t st = c->stream;
  MG_TRY(ensure(c->gstate, 4 * sizeof(int)));
  MG_TRY(ensure(c->alpha32, 2 * sizeof(float)));
  MG_TRY(ensure(c->gparams, 3 * sizeof(double)));
  if (c->ghist.bytes < (size_t)(maxit + 1) * sizeof(double)) {
    MG_TRY(ensure(c->ghist, (size_t)(maxit + 1) * sizeof(double)));
    c->sgraph_valid = false;
  }
  MG_TRY(ensure(c->f, N0 * sizeof(double)));
  MG_TRY(ensure(c->u, N0 * sizeof(double)));
  if (f != c->f.as<double>()) MG_CUDA(cudaMemcpyAsync(c->f.p, f, N0 * sizeof(double), cudaMemcpyDefault, st));
  if (u != c->u.as<double>()) MG_CUDA(cudaMemcpyAsync(c->u.p, u, N0 * sizeof(double), cudaMemcpyDefault, st));
  // ||f||^2 into scalars[1] (unless the caller has it there already)
  double fn2 = fn2_known;
  if (!(fn2_known > 0.0)) {
    MG_TRY(launch_sumsq(c->f.as<double>(), N0, c->partial.as<double>(), st));
    MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N0), c->scalars.as<double>() + 1, st));
    MG_CUDA(cudaMemcpyAsync(c->h_scalars + 1, c->scalars.as<double>() + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    fn2 = c->h_scalars[1];
  }
  if (!std::isfinite(fn2)) return make_status(MGCNN_ERR_NONFINITE, "right-hand side is not finite");
  *used = true;
  *iters = 0;
  if (fn2 == 0.0) {
    MG_CUDA(cudaMemsetAsync(u, 0, N0 * sizeof(double), st));
    if (relres) relres[0] = 0.0;
    MG_CUDA(cudaStreamSynchronize(st));
    return {};
  }
  if (fused_residual_mode(c) == 2) {
    // tile shapes (tuned once per setup before the graph fixes them), then r_0
    // and ||r_0||^2 before the loop
    if (c->u2.bytes < N0 * sizeof(double)) {
      MG_TRY(ensure(c->u2, N0 * sizeof(double)));
      c->sgraph_valid = false;
    }
    const bool was_tuned = c->tuned;
    MG_TRY(upres_cycle_setup(c, c->f.as<double>(), c->u.as<double>(), c->scalars.as<double>(), st));
    if (!was_tuned) c->sgraph_valid = false;
  } else if (fused_residual_applies(c)) {
    // tile shapes (tuned once per setup before the graph fixes them) and the
    // first cycle's input scale from ||f||
    const bool was_tuned = c->tuned;
    MG_TRY(fused_cycle_setup(c, c->f.as<double>(), c->u.as<double>(), c->scalars.as<double>() + 1));
    if (!was_tuned) c->sgraph_valid = false;
  } else if (!c->tuned) {
    // tile shapes: tuned once per setup before the graph fixes them
    FusedLevels fl;
    fl.L = c->L;
    fl.batch = 1;
    fl.maps = c->tma;
    fl.err = c->kerr.as<int>();
    fl.alpha = c->alpha32.as<float>();
    for (int l = 0; l < c->L; ++l) {
      fl.n[l] = c->lv[l].n;
      fl.s[l] = c->s16[l].as<__nv_bfloat16>();
      fl.xa[l] = c->x16a[l].as<__nv_bfloat16>();
      fl.xb[l] = c->x16b[l].as<__nv_bfloat16>();
      fl.xbl[l] = c->x16l[l].as<__nv_bfloat16>();
    }
    MG_TRY(fused_autotune(fl, c->r32.as<float>(), c->scalars.as<double>() + 1, c->e.as<double>(), fused_weights(c),
                          st, 5));
    for (int l = 0; l < c->L; ++l) {
      c->tile_var[0][l] = fl.var_down[l];
      c->tile_var[1][l] = fl.var_up[l];
    }
    c->tuned = true;
    c->sgraph_valid = false;
  }
  if (!c->gstream) MG_CUDA(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
  if (!c->sgraph_valid) {
    Status b = build_graph(c);
    if (!b.ok() && c->tail_n > 0) {
      // no cooperative kernel in this graph: a launch per coarse level
      cudaGetLastError();
      c->tail_n = 0;
      b = build_graph(c);
    }
    if (!b.ok() && c->pdl) {
      // programmatic edges not available in this graph: plain launches
      cudaGetLastError();
      c->pdl = false;
      b = build_graph(c);
    }
    if (!b.ok()) {
      cudaGetLastError();
      c->graph_failed = true;   // conditional graphs unavailable: host loop from now on
      *used = false;
      return {};
    }
    c->sgraph_valid = true;
  }
  const double params[3] = {tol, (double)maxit, c->divtol};
  const int state0[4] = {1, 0, MGCNN_OK, 0};
  MG_CUDA(cudaMemcpyAsync(c->gparams.p, params, sizeof(params), cudaMemcpyHostToDevice, st));
  MG_CUDA(cudaMemcpyAsync(c->gstate.p, state0, sizeof(state0), cudaMemcpyHostToDevice, st));
  MG_CUDA(cudaGraphLaunch(c->sgraph, st));
  int state[4];
  MG_CUDA(cudaMemcpyAsync(state, c->gstate.p, sizeof(state), cudaMemcpyDeviceToHost, st));
  MG_CUDA(cudaStreamSynchronize(st));
  // with the residual formed in the up kernel an odd number of cycles leaves the
  // iterate in u2
  const double* ures = (fused_residual_mode(c) == 2 && (state[1] & 1)) ? c->u2.as<double>() : c->u.as<double>();
  if (u != ures) MG_CUDA(cudaMemcpyAsync(u, ures, N0 * sizeof(double), cudaMemcpyDefault, st));
  MG_CUDA(cudaStreamSynchronize(st));
  *iters = state[1];
  // graph passes run: one per cycle plus the final test (two cycles per pass with
  // the residual formed in the up kernel)
  const long long passes = (fused_residual_mode(c) == 2) ? state[1] / 2 + 1 : state[1] + 1;
  add_launches(c->sgraph_kernels * passes);
  if (relres) {
    const int nh = state[2] == MGCNN_ERR_NONFINITE ? state[1] : state[1] + 1;
    if (nh > 0) MG_CUDA(cudaMemcpy(relres, c->ghist.p, nh * sizeof(double), cudaMemcpyDeviceToHost));
  }
  if (state[2] == MGCNN_ERR_NONFINITE)
    return make_status(MGCNN_ERR_NONFINITE, "residual norm is not finite at cycle %d", state[1]);
  if (state[2] == MGCNN_NOT_CONVERGED)
    return make_status(MGCNN_NOT_CONVERGED, "no convergence in %d cycles", maxit);
  if (state[2] == MGCNN_ERR_DIVERGED)
    return make_status(MGCNN_ERR_DIVERGED, "relres %.3e above the divergence limit at cycle %d",
                       relres ? relres[state[1]] : 0.0, state[1]);
  return {};
}

}  // namespace mgcnn

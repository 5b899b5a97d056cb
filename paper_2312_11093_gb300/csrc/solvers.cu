// Krylov methods with the MGCNN network as preconditioner (Sec. 2.2: the
// network approximates A^{-1} and can precondition a Krylov method; Remark
// "Symmetric problem": CG / MINRES with the symmetric network).  Host-driven
// loops over the library's FP64 vector kernels (krylov.cu), the residual
// kernel and one V-cycle per inner iteration; scalars come back to the host
// once per inner product.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ops.cuh"
#include "solvers.cuh"

namespace mgcnn {

namespace {

// <x, y> in FP64 with the fixed-order block reduction, read back to the host.
Status dot_host(mgcnn_ctx* c, const double* x, const double* y, size_t N, double* out) {
  double* d = c->kcoef.as<double>();
  MG_TRY(launch_block_dots(x, 1, y, N, c->kpart.as<double>(), d, c->stream));
  MG_CUDA(cudaMemcpyAsync(c->h_scalars + 7, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MG_TRY(sync(c));
  *out = c->h_scalars[7];
  return {};
}

// Shared start of the two drivers: ||f||, the f = 0 case, workspace of `nvec`
// vectors, r = f - A u in vector 0.  Returns fn = 0 when the solve is done.
Status sym_start(mgcnn_ctx* c, const double* df, double* du, int nvec, double* fn, double* rn) {
  const size_t N = c->lv[0].N();
  MG_TRY(sumsq(c, df, N, 1));
  double fn2 = 0.0;
  MG_TRY(read_scalar(c, 1, &fn2));
  if (!std::isfinite(fn2)) return make_status(MGCNN_ERR_NONFINITE, "right-hand side is not finite");
  *fn = std::sqrt(fn2);
  if (fn2 == 0.0) {
    MG_CUDA(cudaMemsetAsync(du, 0, N * sizeof(double), c->stream));
    return {};
  }
  MG_TRY(ensure(c->kV, (size_t)nvec * N * sizeof(double)));
  MG_TRY(ensure(c->kcoef, 8 * sizeof(double)));
  MG_TRY(ensure(c->kpart, krylov_partial_count(N, 1) * sizeof(double)));
  double* r = c->kV.as<double>();
  MG_TRY(launch_residual(df, du, c->op[0].as<double>(), r, nullptr, c->partial.as<double>(), c->n, c->stream));
  MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N), c->scalars.as<double>() + 3, c->stream));
  double r2 = 0.0;
  MG_TRY(read_scalar(c, 3, &r2));
  *rn = std::sqrt(r2);
  return {};
}

}  // namespace

// Flexible GMRES(restart) with the network as right preconditioner: z_j = B v_j
// (one V-cycle of the context's precision), Arnoldi with classical Gram-Schmidt
// applied twice, Givens rotations on the host, u += Z y at the end of a cycle and
// a restart from the true FP64 residual.  df, du: device arrays.  hist gets
// ||r|| / ||f|| before the first and after every inner iteration (the recursive
// estimate inside a cycle, the true residual at its end).
Status krylov_solve(mgcnn_ctx* c, const double* df, double* du, double tol, int maxit, int restart, int* iters,
                    std::vector<double>& hist) {
  const size_t N = c->lv[0].N();
  const int n = c->n, m = restart;
  cudaStream_t st = c->stream;
  *iters = 0;
  hist.clear();
  MG_TRY(sumsq(c, df, N, 1));
  double fn2 = 0.0;
  MG_TRY(read_scalar(c, 1, &fn2));
  if (!std::isfinite(fn2)) return make_status(MGCNN_ERR_NONFINITE, "right-hand side is not finite");
  if (fn2 == 0.0) {
    MG_CUDA(cudaMemsetAsync(du, 0, N * sizeof(double), st));
    hist.push_back(0.0);
    return {};
  }
  const double fn = std::sqrt(fn2);
  MG_TRY(ensure(c->kV, (size_t)(m + 1) * N * sizeof(double)));
  MG_TRY(ensure(c->kZ, (size_t)m * N * sizeof(double)));
  MG_TRY(ensure(c->kw, N * sizeof(double)));
  MG_TRY(ensure(c->kr, N * sizeof(double)));
  MG_TRY(ensure(c->kcoef, (size_t)3 * (m + 1) * sizeof(double)));
  MG_TRY(ensure(c->kpart, krylov_partial_count(N, m + 1) * sizeof(double)));
  double* V = c->kV.as<double>();
  double* Z = c->kZ.as<double>();
  double* w = c->kw.as<double>();
  double* r = c->kr.as<double>();
  double* coef = c->kcoef.as<double>();
  auto true_residual = [&](double* beta) -> Status {
    MG_TRY(launch_residual(df, du, c->op[0].as<double>(), r, nullptr, c->partial.as<double>(), n, st));
    MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N), c->scalars.as<double>() + 3, st));
    double b2 = 0.0;
    MG_TRY(read_scalar(c, 3, &b2));
    *beta = std::sqrt(b2);
    return {};
  };
  double beta = 0.0;
  MG_TRY(true_residual(&beta));
  hist.push_back(beta / fn);
  int it = 0;
  std::vector<double> H, cs, sn, g, y, hc(2 * (size_t)(m + 1));
  while (hist.back() > tol && it < maxit && std::isfinite(hist.back())) {
    const int mm = std::min(m, maxit - it);
    H.assign((size_t)(mm + 1) * mm, 0.0);   // H[i * mm + j]
    cs.assign(mm, 0.0);
    sn.assign(mm, 0.0);
    g.assign(mm + 1, 0.0);
    g[0] = beta;
    MG_TRY(launch_scale(r, V, 1.0 / beta, N, st));
    int k = 0;
    for (int j = 0; j < mm; ++j) {
      MG_TRY(vcycle_any(c, V + (size_t)j * N, Z + (size_t)j * N, nullptr));
      MG_TRY(launch_apply_A(c->op[0].as<double>(), Z + (size_t)j * N, w, n, st));
      for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
        double* cp = coef + (size_t)pass * (m + 1);
        MG_TRY(launch_block_dots(V, j + 1, w, N, c->kpart.as<double>(), cp, st));
        MG_TRY(launch_combine(w, V, j + 1, cp, -1.0, N, st));
      }
      MG_TRY(sumsq(c, w, N, 4));
      MG_CUDA(cudaMemcpyAsync(hc.data(), coef, hc.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      double hn2 = 0.0;
      MG_TRY(read_scalar(c, 4, &hn2));
      const double hn = std::sqrt(hn2);
      for (int i = 0; i <= j; ++i) H[(size_t)i * mm + j] = (0.0 + hc[i]) + hc[(size_t)(m + 1) + i];
      H[(size_t)(j + 1) * mm + j] = hn;
      for (int i = 0; i < j; ++i) {   // earlier rotations on column j, then a new one
        const double a = H[(size_t)i * mm + j], b = H[(size_t)(i + 1) * mm + j];
        H[(size_t)i * mm + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * mm + j] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[(size_t)j * mm + j], b = H[(size_t)(j + 1) * mm + j];
      const double d = std::hypot(a, b);
      cs[j] = a / d;
      sn[j] = b / d;
      H[(size_t)j * mm + j] = d;
      H[(size_t)(j + 1) * mm + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      ++it;
      const double est = std::fabs(g[j + 1]) / fn;
      if (est <= tol || it >= maxit || !std::isfinite(est) || j == mm - 1) break;   // then the true residual
      hist.push_back(est);
      MG_TRY(launch_scale(w, V + (size_t)(j + 1) * N, 1.0 / hn, N, st));
    }
    y.assign(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {   // back substitution on the rotated H
      double t = g[i];
      for (int q = i + 1; q < k; ++q) t -= H[(size_t)i * mm + q] * y[q];
      y[i] = t / H[(size_t)i * mm + i];
    }
    double* cy = coef + 2 * (size_t)(m + 1);
    MG_CUDA(cudaMemcpyAsync(cy, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, st));
    MG_TRY(launch_combine(du, Z, k, cy, 1.0, N, st));
    MG_TRY(true_residual(&beta));
    hist.push_back(beta / fn);
  }
  *iters = it;
  if (!std::isfinite(hist.back())) return make_status(MGCNN_ERR_NONFINITE, "residual norm is not finite");
  return {};
}

// Preconditioned CG: z = B r, p = z + beta p, alpha = (r, z) / (p, A p),
// beta = (r_new, z_new) / (r, z), r updated recursively.  hist[k] = ||r_k|| / ||f||.
Status pcg_solve(mgcnn_ctx* c, const double* df, double* du, double tol, int maxit, int* iters,
                 std::vector<double>& hist) {
  const size_t N = c->lv[0].N();
  cudaStream_t st = c->stream;
  *iters = 0;
  hist.clear();
  double fn = 0.0, rn = 0.0;
  MG_TRY(sym_start(c, df, du, 4, &fn, &rn));
  if (fn == 0.0) {
    hist.push_back(0.0);
    return {};
  }
  double* r = c->kV.as<double>();
  double* z = r + N;
  double* p = z + N;
  double* q = p + N;
  hist.push_back(rn / fn);
  double rz = 0.0;
  int it = 0;
  while (hist.back() > tol && it < maxit && std::isfinite(hist.back())) {
    MG_TRY(vcycle_any(c, r, z, nullptr));
    double rz_new = 0.0;
    MG_TRY(dot_host(c, r, z, N, &rz_new));
    MG_TRY(launch_axpby(p, z, 1.0, it == 0 ? 0.0 : rz_new / rz, N, st));   // p = z + beta p
    rz = rz_new;
    MG_TRY(launch_apply_A(c->op[0].as<double>(), p, q, c->n, st));
    double pq = 0.0;
    MG_TRY(dot_host(c, p, q, N, &pq));
    const double alpha = rz / pq;
    MG_TRY(launch_axpby(du, p, alpha, 1.0, N, st));
    MG_TRY(launch_axpby(r, q, -alpha, 1.0, N, st));
    ++it;
    MG_TRY(sumsq(c, r, N, 4));
    double r2 = 0.0;
    MG_TRY(read_scalar(c, 4, &r2));
    hist.push_back(std::sqrt(r2) / fn);
  }
  *iters = it;
  if (!std::isfinite(hist.back())) return make_status(MGCNN_ERR_NONFINITE, "residual norm is not finite");
  return {};
}

// Preconditioned MINRES (Lanczos on B A in the B^{-1} inner product; Givens
// rotations on the tridiagonal least-squares problem as its columns arrive;
// search directions w_k = (v_k - eps_k w_{k-2} - delta_k w_{k-1}) / gamma_k).
// hist[k] = ||r_k||_B / ||r_0||_B from the recursion.
Status minres_solve(mgcnn_ctx* c, const double* df, double* du, double tol, int maxit, int* iters,
                    std::vector<double>& hist) {
  const size_t N = c->lv[0].N();
  cudaStream_t st = c->stream;
  *iters = 0;
  hist.clear();
  double fn = 0.0, rn = 0.0;
  MG_TRY(sym_start(c, df, du, 7, &fn, &rn));
  if (fn == 0.0) {
    hist.push_back(0.0);
    return {};
  }
  double* buf = c->kV.as<double>();
  double* r_cur = buf;            // r_k (unpreconditioned Lanczos vector, scaled by beta_k)
  double* r_prev = buf + N;       // r_{k-1}
  double* y = buf + 2 * N;        // B r_k
  double* v = buf + 3 * N;
  double* t = buf + 4 * N;
  double* w_prev2 = buf + 5 * N;  // w_{k-2}
  double* w_prev = buf + 6 * N;   // w_{k-1}
  MG_CUDA(cudaMemsetAsync(w_prev2, 0, 2 * N * sizeof(double), st));
  MG_TRY(vcycle_any(c, r_cur, y, nullptr));
  double ry = 0.0;
  MG_TRY(dot_host(c, r_cur, y, N, &ry));
  if (!(ry >= 0.0)) return make_status(MGCNN_ERR_NONFINITE, "preconditioner is not positive definite");
  const double beta1 = std::sqrt(ry);
  hist.push_back(beta1 == 0.0 ? 0.0 : 1.0);
  double beta_prev = 0.0, beta = beta1, cs = -1.0, sn = 0.0, dbar = 0.0, eps = 0.0, phibar = beta1;
  int it = 0;
  while (beta1 != 0.0 && it < maxit) {
    MG_TRY(launch_scale(y, v, 1.0 / beta, N, st));
    MG_TRY(launch_apply_A(c->op[0].as<double>(), v, t, c->n, st));
    if (it > 0) MG_TRY(launch_axpby(t, r_prev, -beta / beta_prev, 1.0, N, st));
    double alpha = 0.0;
    MG_TRY(dot_host(c, v, t, N, &alpha));
    MG_TRY(launch_axpby(t, r_cur, -alpha / beta, 1.0, N, st));
    // r_{k-1} <- r_k, r_k <- t (the old r_{k-1} buffer becomes the next t)
    double* old_prev = r_prev;
    r_prev = r_cur;
    r_cur = t;
    t = old_prev;
    MG_TRY(vcycle_any(c, r_cur, y, nullptr));
    MG_TRY(dot_host(c, r_cur, y, N, &ry));
    if (!(ry >= 0.0)) return make_status(MGCNN_ERR_NONFINITE, "preconditioner is not positive definite");
    beta_prev = beta;
    beta = std::sqrt(ry);
    const double eps_old = eps;
    const double delta = cs * dbar + sn * alpha;
    const double gbar = sn * dbar - cs * alpha;
    eps = sn * beta;
    dbar = -cs * beta;
    const double gamma = std::hypot(gbar, beta);
    cs = gbar / gamma;
    sn = beta / gamma;
    const double phi = cs * phibar;
    phibar = sn * phibar;
    // w_k into the w_{k-2} buffer, then rotate the two
    MG_TRY(launch_lincomb3(w_prev2, v, 1.0 / gamma, w_prev2, -eps_old / gamma, w_prev, -delta / gamma, N, st));
    std::swap(w_prev2, w_prev);
    MG_TRY(launch_axpby(du, w_prev, phi, 1.0, N, st));
    ++it;
    hist.push_back(std::fabs(phibar) / beta1);
    if (hist.back() <= tol || !std::isfinite(hist.back()) || beta == 0.0) break;
  }
  *iters = it;
  if (!std::isfinite(hist.back())) return make_status(MGCNN_ERR_NONFINITE, "residual norm is not finite");
  return {};
}

}  // namespace mgcnn

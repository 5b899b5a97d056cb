/*
 * mgcnn.h -- C ABI of the GB300 MGCNN solver library (libmgcnn.so).
 *
 * MGCNN (Xie, Lv, Zhang, "MGCNN: a learnable multigrid solver for sparse
 * linear systems from PDEs on structured grids", arXiv 2312.11093) solves
 * A_coef sol = rhs (Sec. 2.1, "Solver as Decoder") for a 5-point
 * convection-diffusion operator on an n x n interior grid of the unit square
 * with zero Dirichlet boundary, by the stationary iteration
 *     sol^{k+1} = sol^k + B (rhs - A sol^k)                  (Sec. 2.2, Eq. 1)
 * where B is the solve phase of a multigrid-shaped CNN (Sec. 3.3, Algorithm 3)
 * whose per-level setup tensors come from a setup network run once per
 * coefficient field (Sec. 3.2, Algorithm 2).
 *
 * Conventions for every entry point
 *   - Grids: n = 2^m - 1, m >= 2 (n = 3, 7, 15, ..., 4095).  Level sizes
 *     n_1 = n, n_{l+1} = (n_l - 1)/2 down to 3; L = log2(n+1) - 1 levels unless
 *     the config asks for fewer.  h = 1/(n+1).
 *   - Scalar fields are row-major [j][i], x = i h, y = j h (y grows with j);
 *     interior fields have n*n entries, nodal coefficient fields that include
 *     the boundary ring (n+2)*(n+2).
 *   - Multi-channel tensors (setup tensors) are [j][i][c] per level, levels
 *     concatenated finest first.
 *   - Array arguments may be HOST or DEVICE pointers: the library asks the
 *     driver which (cudaPointerGetAttributes).  Device arrays are used in
 *     place (they must live on the context's device); host arrays are copied
 *     to the context's device buffers and results copied back, on the
 *     context's stream, before the call returns.
 *   - The caller owns every array it passes; the context owns its device
 *     workspaces.  Nothing allocated by the library is freed by the caller
 *     except through mgcnn_destroy.
 *   - Calls on one context are not thread-safe.  No C++ exception and no
 *     exit() crosses the ABI; every failure is a negative status code and a
 *     message retrievable with mgcnn_last_error.
 *   - Every call that returns a status synchronises the context's stream
 *     before returning, unless its comment says otherwise.
 */
#ifndef MGCNN_H
#define MGCNN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes.  >0: the result is valid but a limit was hit. */
enum {
  MGCNN_OK = 0,
  MGCNN_NOT_CONVERGED = 1,   /* maxit cycles applied without reaching tol        */
  MGCNN_ERR_ARG = -1,        /* null pointer, bad count, bad enum value          */
  MGCNN_ERR_SIZE = -2,       /* n not 2^m-1, too many levels, unsupported C      */
  MGCNN_ERR_STATE = -3,      /* e.g. solve before setup, weights never set       */
  MGCNN_ERR_NOMEM = -4,      /* device allocation failed                         */
  MGCNN_ERR_CUDA = -5,       /* a CUDA runtime call or kernel launch failed      */
  MGCNN_ERR_NONFINITE = -6,  /* NaN/Inf in an input or in the iterate's residual */
  MGCNN_ERR_TIMEOUT = -7,    /* a bounded device-side wait gave up               */
  MGCNN_ERR_DIVERGED = -8    /* ||r||/||f|| rose above the limit MGCNN_OPT_DIVTOL */
};

/* Arithmetic of the solve phase.  The residual, the update and the
 * convergence norm are FP64 in every mode (defect correction). */
enum {
  MGCNN_PREC_FP64 = 0,       /* setup and solve networks in FP64                 */
  MGCNN_PREC_MIXED_BF16 = 1  /* setup in FP32; solve network with BF16 tensors,
                                BF16 x BF16 products, FP32 accumulation          */
};

/* Discretisation that turns the coefficient field into A. */
enum {
  /* -div(k grad u) + b.grad u = f (Remark 2.1, Eq. convection_diffusion_div):
   * nodal k on the (n+2)^2 nodes incl. the boundary ring, face k the harmonic
   * mean of its two nodes, first-order upwind convection.  Coarse levels
   * rediscretise with k restricted by full weighting of log k. */
  MGCNN_PDE_DIV_HARMONIC = 0,
  /* -mu Lap u + v.grad u = f (Sec. 2.5, Eqs. convection_diffusion(_kernel)):
   * nodal mu on the n^2 interior nodes, 5-point Laplacian scaled by mu plus
   * first-order upwind convection; coarse levels sample mu (injection). */
  MGCNN_PDE_NONDIV = 1
};

typedef struct mgcnn_ctx mgcnn_ctx;

typedef struct {
  int channels;      /* C, hidden channels of both networks (Sec. 4.2: 4, 8, 12);
                        supported: 4, 8, 12, 13, 16, and 2 in FP64 precision
                        (the BPX form of the symmetric network)                 */
  int down_layers;   /* layers ("sweeps") in ResNetDown, >= 1 (Sec. 3.3)      */
  int up_layers;     /* layers in ResNetUp, >= 1                               */
  int precision;     /* MGCNN_PREC_*                                           */
  int pde;           /* MGCNN_PDE_*                                            */
  int scale_by_diag; /* scaling of each level's setup tensor (Algorithm 2 output):
                        0: none; 1: divided by a_C of its level's operator
                        (Jacobi-like D^{-1}); 2: multiplied by (h_l/h_1)^2 =
                        4^(l-1), the coefficient-free level ratio of D^{-1}     */
  int input_diag;    /* 1: the solve network is applied to D^{-1} r, D = diag(A)
                        of the finest level (B r = Net(D^{-1} r)): the pointwise
                        analogue of the paper's normalisation of the stencil to
                        O(1) entries (Sec. 2.5); 0: Net(r)                       */
  int levels;        /* 0: L = log2(n+1)-1 (coarsest 3x3); else 1..that L     */
  double bx, by;     /* constant velocity b (or v) of the convection term      */
} mgcnn_config;

/* Number of doubles in a weight blob for this config.  Layout, in order, all
 * row-major and shared by every level (principle P3, Sec. 3.1):
 *   solve phase (Algorithm 3; no bias, no activation -- principle P2)
 *     w_in   [C][1][3][3]        reChannelCNN rhs -> C channels
 *     w_down [nu_d][C][C][3][3]  ResNetDown kernels K_down, [c_out][c_in]
 *     w_up   [nu_u][C][C][3][3]  ResNetUp kernels K_up
 *     w_R    [C][C][3][3]        RCNN, stride 2, [c_out][c_in]
 *     w_P    [C][C][3][3]        TCNN, stride 2, [c_in][c_out]
 *     w_out  [1][C][3][3]        reChannelCNN C -> solution
 *   setup phase (Algorithm 2; F = 5 input features)
 *     sw_in  [C][5][3][3], sb_in [C]         reChannelCNN of the features
 *     sw     [4][C][C][3][3], sb [4][C]      NonLinearResNet, tanh (Eq. resnet_nonlinear)
 *     sw_R   [C][C][3][3]                    setup RCNN (Eq. setup1)
 * Tap [a][b] of a same-size layer reads pixel (j+a-1, i+b-1); of RCNN, fine
 * pixel (2J+a, 2I+b) (0-based interior indices); TCNN adds W[.][.][a][b] x[J][I]
 * into fine pixel (2J+a, 2I+b).  Returns 0 for an invalid config. */
size_t mgcnn_weight_count(const mgcnn_config* cfg);

/* Create a context on the current CUDA device.  *out receives the handle.
 * Errors: ARG (null), SIZE (unsupported channels/layers), CUDA. */
int mgcnn_create(const mgcnn_config* cfg, mgcnn_ctx** out);

/* Free every device buffer and the handle.  Accepts NULL. */
void mgcnn_destroy(mgcnn_ctx* ctx);

/* Bind the context to a CUDA stream (cudaStream_t passed as void*; NULL is
 * the legacy default stream).  All later work is issued on it; work still
 * running on the previous stream (a setup's kernels) is waited for first. */
int mgcnn_set_stream(mgcnn_ctx* ctx, void* stream);

/* Load the weight blob (layout of mgcnn_weight_count; count must equal it).
 * The blob is copied; the caller may free it afterwards.  Errors: ARG. */
int mgcnn_set_weights(mgcnn_ctx* ctx, const double* w, size_t count);

/* Setup phase for one coefficient field (Sec. 3.2, Algorithm 2), once per
 * problem.  coeff: DIV_HARMONIC -> nodal k, (n+2)^2 doubles, all > 0;
 * NONDIV -> nodal mu, n^2 doubles, all > 0.  Builds the operator on every
 * level (Sec. 2.3: rediscretised coarse operators), runs the setup network
 * on all levels and keeps the setup tensors on the device.
 * Errors: ARG, SIZE, STATE (weights not set), NOMEM, NONFINITE (k <= 0 or
 * non-finite), CUDA.
 * Synchronisation: the call returns once coeff has been copied and checked; the
 * setup kernels run on the context's stream after it returns (every later call
 * on the context is ordered after them, and mgcnn_solve's copies of host inputs
 * overlap them); an error they meet is reported by the next call that
 * synchronises. */
int mgcnn_setup(mgcnn_ctx* ctx, const double* coeff, int n);

/* Setup for the 13-channel network whose solve phase is exactly classical
 * geometric multigrid V(nu1, nu2) (Sec. 2.3: weighted Jacobi with weight
 * omega, full-weighting restriction, bilinear prolongation, rediscretised
 * coarse operators), used as a learning-free reference network and as the GMG
 * comparator.  Builds the operators like mgcnn_setup, then sets the setup
 * tensors analytically instead of running the setup network:
 *   s[E_o](q) = -omega a_o(q-o)/a_C(q-o), s[G_o](q) = -a_o(q-o) for o in
 *   {C, W, E, S, N} (channels 0-4 and 5-9), s[F_J] = omega/a_C, s[F_G] = 1,
 *   s[D] = 0 (channels 10, 11, 12); with input_diag the finest level's
 *   right-hand-side copies hold D^{-1} r, so there s[F_J] = omega, s[F_G] = a_C.
 * The matching weights (ResNetDown = nu1 Jacobi layers + one defect layer,
 * ResNetUp = nu2 Jacobi layers) must be loaded with mgcnn_set_weights; the
 * Python binding's gmg_weights() builds that blob.
 * A context with channels == 8, down_layers == 1 and up_layers == 1 (the
 * learned network's shape) gets instead the setup tensors of the 8-channel
 * network that is GMG V(1, 0): one down layer does the Jacobi sweep from
 * e = 0 and the defect of its result, d = (1-omega) r - sum_{o != C} omega
 * a_o(p) r(p+o)/a_C(p+o); the up layer is the identity.  Channels T_W, T_E,
 * T_S, T_N, F_G, F_J, D, E (0-7):
 *   s[T_o](q) = -omega a_o(q-o)/a_C(q), s[F_G] = 1 - omega, s[F_J] = omega/a_C,
 *   s[D] = s[E] = 0; with input_diag at the finest level
 *   s[T_o](q) = -omega a_o(q-o), s[F_G] = (1 - omega) a_C, s[F_J] = omega.
 * Its weights come from the binding's gmg_v10_weights().
 * Errors: SIZE (any other channels / layer counts), ARG (omega not in (0,2)),
 * as mgcnn_setup.  Synchronisation as mgcnn_setup. */
int mgcnn_setup_gmg(mgcnn_ctx* ctx, const double* coeff, int n, double omega);

/* mgcnn_setup_gmg with a Jacobi weight per level (Sec. 2.3 leaves the weight
 * open): omega[0] on the finest level, omega[2] on the coarsest, omega[1] on
 * every level in between; a one-level grid takes omega[0].  omega: 3 host
 * doubles, each in (0, 2), read before the call returns.  Level l's setup
 * tensors are those of mgcnn_setup_gmg with that level's weight, so the solve
 * phase is GMG with weighted Jacobi at weight omega_l on level l.  On the
 * lognormal workloads over-relaxing the levels between the finest and the
 * coarsest, e.g. {0.8, 1.5, 1.0}, cuts the V(1, 0) network's cycle count by
 * about a quarter against a uniform 0.8.  Errors as mgcnn_setup_gmg, ARG
 * (null omega, a weight outside (0, 2)). */
int mgcnn_setup_gmg_levels(mgcnn_ctx* ctx, const double* coeff, int n, const double* omega);

/* Number of doubles of all setup tensors of the current setup:
 * sum_l n_l^2 * C.  0 before setup. */
size_t mgcnn_setup_tensor_count(const mgcnn_ctx* ctx);

/* Replace the setup tensors produced by mgcnn_setup with caller-supplied ones
 * (layout [level][j][i][c], finest level first; count as above).  Used to run
 * the solve phase with analytically built setup tensors, e.g. the weights and
 * tensors that make Algorithm 3 reproduce classical GMG.  Errors: STATE
 * (no setup), ARG. */
int mgcnn_set_setup_tensors(mgcnn_ctx* ctx, const double* s, size_t count);

/* Copy the setup tensors out as doubles (layout as above). */
int mgcnn_get_setup_tensors(mgcnn_ctx* ctx, double* s, size_t count);

/* Copy the level-l operator out: 5 arrays of n_l^2 doubles, in the order
 * a_C, a_W, a_E, a_S, a_N, with (A u)_p = sum_o a_o(p) u(p+o), zero outside. */
int mgcnn_get_operator(mgcnn_ctx* ctx, int level, double* out, size_t count);

/* r = f - A u on the finest grid (Eq. 1) in FP64, and ||r||_2^2 in FP64 into
 * *norm2 (host pointer; may be NULL).  f, u, r: n^2 doubles. */
int mgcnn_residual(mgcnn_ctx* ctx, const double* f, const double* u, double* r, double* norm2);

/* One application e = B r of the solve phase (Algorithm 3) in the context's
 * precision: FP64, or for MIXED_BF16 the scaled BF16 network with r and e in
 * FP64 at the boundary.  r, e: n^2 doubles. */
int mgcnn_vcycle(mgcnn_ctx* ctx, const double* r, double* e);

/* The stationary iteration (Eq. 1) with B the solve phase:
 *   for k = 0, 1, ...: r_k = f - A u_k; stop if ||r_k||_2 / ||f||_2 <= tol or
 *   k == maxit; u_{k+1} = u_k + B r_k.
 * u: n^2 doubles, in: initial guess, out: the last iterate.  f = 0 gives
 * u = 0, *iters = 0.  *iters receives the number of cycles applied; relres
 * (may be NULL) receives ||r_k||/||f|| for k = 0..*iters (room for maxit+1).
 * Returns OK, NOT_CONVERGED (maxit reached), NONFINITE (a residual norm was
 * NaN/Inf; u holds the last finite iterate's update), STATE, ARG, CUDA. */
int mgcnn_solve(mgcnn_ctx* ctx, const double* f, double* u, double tol, int maxit,
                int* iters, double* relres);

/* The solve network as the right preconditioner of flexible GMRES (Sec. 2.2:
 * the network approximates A^{-1}; besides the stationary iteration of Eq. 1
 * it can precondition a Krylov method).  Each inner iteration applies one
 * V-cycle z_j = B v_j in the context's precision (the mixed network differs
 * slightly from one input to the next, hence the flexible variant, which keeps
 * the z_j) and one FP64 product A z_j; Arnoldi orthogonalises by classical
 * Gram-Schmidt applied twice, the least-squares problem uses Givens rotations,
 * and every `restart` iterations (1..MGCNN_KRYLOV_MAX_RESTART) the iterate is
 * updated, u += Z y, and the cycle restarts from the true FP64 residual.
 * Stops when ||r|| / ||f|| <= tol (the recursive estimate inside a cycle, the
 * true residual at its end) or after maxit inner iterations.  f, u as in
 * mgcnn_solve; *iters = inner iterations; relres (may be NULL, room for
 * maxit + 1) receives ||r|| / ||f|| before the first and after every inner
 * iteration (the true residual at each cycle's end).  Workspace: 2 restart + 3
 * vectors of n^2 doubles.  Returns OK, NOT_CONVERGED, NONFINITE, STATE, ARG,
 * NOMEM, CUDA. */
#define MGCNN_KRYLOV_MAX_RESTART 64
int mgcnn_solve_krylov(mgcnn_ctx* ctx, const double* f, double* u, double tol, int maxit, int restart,
                       int* iters, double* relres);

/* Symmetric variant (Remark "Symmetric problem", Sec. 3.3: a symmetric solver
 * for a symmetric problem, with MINRES as the outer method).  Turned on by
 * mgcnn_set_option(ctx, MGCNN_OPT_SYMMETRIC, 1), which needs precision FP64,
 * input_diag 0 and down_layers == up_layers (else ERR_ARG).  The network then
 * shares weights between ResNetDown and ResNetUp and between RCNN and TCNN in
 * the adjoint sense: each up map is the transpose of its down map, so
 *   up layer i (of nu):  x <- x + s_l * (K_i^T x),  K_i^T the same-size conv
 *                        with w_down[nu-1-i]'s channels swapped and taps flipped
 *                        (the setup tensor applied after the conv),
 *   TCNN = the transposed conv with w_R (exactly RCNN^T),
 *   reChannel-out = the adjoint of reChannel-in,
 * and B = W_in^T M_1 W_in with M_l = D_l^T (I + R^T M_{l+1} R) D_l, D_l the
 * level's down layers: B is symmetric positive semidefinite for any weights and
 * setup tensors (definite when the down layers are nonsingular and W_in is
 * injective).  mgcnn_set_weights then overwrites the blob's w_up, w_P and w_out
 * with the tied values (mgcnn_get_weights returns them); turning the option on
 * with weights already loaded ties them at once.  Training (mgcnn_train_step,
 * mgcnn_loss_grad) is not available in this mode (ERR_STATE).
 *
 * mgcnn_setup_bpx: operators as mgcnn_setup, and setup tensors that make the
 * symmetric network the additive multilevel (BPX) preconditioner
 *   B = sum_l 4^l R_l^T (omega D_l^{-1}) R_l  +  eps^2 sum_l R_l^T R_l,
 * R_l = full weighting applied l times, D_l = diagonal of the level-l operator,
 * eps = MGCNN_BPX_EPS: s_l[0] = sqrt(omega 4^l / a_C,l) / eps, other channels 0.
 * It expects the BPX weights: w_in[0][0][1][1] = eps, w_down[0][1][0][1][1] = 1,
 * w_R[0][0] = (1/16)[1 2 1; 2 4 2; 1 2 1], everything else 0 (the tied entries
 * follow).  Needs the symmetric mode (ERR_STATE) and omega in (0, 2] (ERR_ARG).
 *
 * mgcnn_solve_pcg: preconditioned conjugate gradients, z = B r, with the
 * residual updated recursively; stops when ||r_k||_2 / ||f||_2 <= tol or after
 * maxit iterations (one V-cycle each).  relres (may be NULL, room for maxit+1)
 * receives ||r_k|| / ||f|| for k = 0..*iters (k = 0: the true residual of the
 * initial guess).
 * mgcnn_solve_minres: preconditioned MINRES (Lanczos on B A in the B^{-1} inner
 * product, Givens rotations on the tridiagonal least-squares problem); iterate
 * k minimises ||f - A u||_B over the Krylov space; stops when that norm
 * relative to its value at the initial guess is <= tol (relres receives these
 * ratios, 1 at k = 0) or after maxit iterations.
 * Both need the symmetric mode (ERR_STATE) and a symmetric A: pde
 * DIV_HARMONIC with b = 0 (ERR_ARG otherwise).  f, u, *iters as in
 * mgcnn_solve; f = 0 gives u = 0, *iters = 0.  Workspace: 4 (PCG) or 7
 * (MINRES) vectors of n^2 doubles.  A preconditioner that is not positive
 * definite ends MINRES with NONFINITE (the square root of a negative inner
 * product) and may end PCG with NONFINITE.  Returns OK, NOT_CONVERGED,
 * NONFINITE, STATE, ARG, NOMEM, CUDA. */
#define MGCNN_BPX_EPS 0x1p-26
int mgcnn_setup_bpx(mgcnn_ctx* ctx, const double* coeff, int n, double omega);
int mgcnn_solve_pcg(mgcnn_ctx* ctx, const double* f, double* u, double tol, int maxit, int* iters, double* relres);
int mgcnn_solve_minres(mgcnn_ctx* ctx, const double* f, double* u, double tol, int maxit, int* iters,
                       double* relres);

/* Classical geometric multigrid (Sec. 2.3), the comparator of the learned
 * solver, on the context's operators (mgcnn_setup or mgcnn_setup_gmg must have
 * run): the stationary iteration of Eq. 1 with B one V(nu1, nu2) cycle of
 * weighted Jacobi (weight omega in (0,2)), full-weighting restriction of the
 * defect, bilinear prolongation and the rediscretised coarse operators; the
 * coarsest grid gets nu1 + nu2 sweeps.  FP64.  f, u, iters, relres as
 * mgcnn_solve.  Errors: ARG (nu1 + nu2 < 1, omega), STATE, NONFINITE, CUDA. */
int mgcnn_gmg_solve(mgcnn_ctx* ctx, const double* f, double* u, double tol, int maxit, int nu1, int nu2,
                    double omega, int* iters, double* relres);

/* mgcnn_gmg_solve with a Jacobi weight per level: omega (3 host doubles, each
 * in (0, 2)) as in mgcnn_setup_gmg_levels, omega[0] on the finest level,
 * omega[2] on the coarsest, omega[1] in between.  Errors as mgcnn_gmg_solve,
 * ARG for a null omega or a weight outside (0, 2). */
int mgcnn_gmg_solve_levels(mgcnn_ctx* ctx, const double* f, double* u, double tol, int maxit, int nu1, int nu2,
                           const double* omega, int* iters, double* relres);

/* ---- Batched solves ------------------------------------------------------------
 * Many coefficient fields and right-hand sides of uneven grid sizes at once:
 * the setup phase (Sec. 3.2) for every field, then the stationary iteration
 * (Eq. 1) for every problem, each stopping on its own tolerance test.
 * Problems of equal n are grouped; one cycle of the whole batch (residual,
 * convergence test and V-cycle of every still-active problem) is one CUDA
 * graph, replayed until no problem is active, with one 4-byte readback per
 * cycle.  The level kernels' tile shapes are chosen per grid size by timing
 * (autotuned in mgcnn_setup_batched).  Requires MIXED_BF16, 8 channels, one
 * layer per ResNet and the divergence form; otherwise ERR_SIZE.
 * coeff[i]: nodal k of problem i, (n[i]+2)^2 doubles; host or device; copied. */
int mgcnn_setup_batched(mgcnn_ctx* ctx, int nprob, const double* const* coeff, const int* n);

/* As mgcnn_setup_batched, but every problem gets the analytic setup tensors of
 * the 8-channel GMG V(1, 0) network (the ones mgcnn_setup_gmg builds on such a
 * context, Jacobi weight omega) instead of running the setup network; load
 * that network's weights first.  Errors as mgcnn_setup_batched, ARG for omega
 * outside (0, 2). */
int mgcnn_setup_batched_gmg(mgcnn_ctx* ctx, int nprob, const double* const* coeff, const int* n, double omega);

/* mgcnn_setup_batched_gmg with the per-level Jacobi weights of
 * mgcnn_setup_gmg_levels (omega: 3 host doubles, finest / in between /
 * coarsest), applied to every problem on its own level hierarchy.  Errors as
 * mgcnn_setup_batched_gmg. */
int mgcnn_setup_batched_gmg_levels(mgcnn_ctx* ctx, int nprob, const double* const* coeff, const int* n,
                                   const double* omega);

/* rhs[i], u[i]: n[i]^2 doubles (host or device); u[i] is the initial guess on
 * entry and the last iterate on return.  iters[i] (may be NULL) receives the
 * cycles applied, relres[i] (may be NULL) the last ||r||/||f||, status[i]
 * (may be NULL) OK / NOT_CONVERGED / ERR_NONFINITE per problem.  Returns OK if
 * every problem converged, else the first error, else NOT_CONVERGED. */
int mgcnn_solve_batched(mgcnn_ctx* ctx, int nprob, const double* const* rhs, double* const* u, double tol,
                        int maxit, int* iters, double* relres, int* status);

/* Flexible GMRES(restart) for every problem of the batch (after
 * mgcnn_setup_batched or mgcnn_setup_batched_gmg(_levels)), the batch's mixed
 * network as right preconditioner, as mgcnn_solve_krylov does for one problem:
 * z_j = B v_j, Arnoldi by classical Gram-Schmidt applied twice, Givens
 * rotations, u += Z y at the end of a cycle and a restart from the true FP64
 * residual.  The problems of a size class advance in lockstep, one inner
 * iteration of each problem still in its cycle per pass; the Hessenberg
 * matrices, rotations and estimates stay on the device.  iters[i]: inner
 * iterations of problem i; relres[i]: the last ||r||/||f|| (the true residual
 * at the end of its last cycle); status[i]: OK, NOT_CONVERGED (maxit inner
 * iterations), ERR_NONFINITE, or ERR_DIVERGED (MGCNN_OPT_DIVTOL, tested before
 * each cycle).  restart: 1..MGCNN_KRYLOV_MAX_RESTART.  Workspace per problem:
 * 2 restart + 1 vectors of n_i^2 doubles.  Returns as mgcnn_solve_batched;
 * ARG for a restart outside its range. */
int mgcnn_solve_batched_krylov(mgcnn_ctx* ctx, int nprob, const double* const* rhs, double* const* u, double tol,
                               int maxit, int restart, int* iters, double* relres, int* status);

/* ---- Training (Sec. 3.4, Eq. loss) ------------------------------------------
 * Loss of a batch of problems after K stationary cycles from u = 0,
 *     r_0 = f,  r_{k+1} = r_k - A B(r_k),   L = (1/N) sum_i ||r_K,i||^2 / ||f_i||^2
 * (the paper's loss is the K = 1 case of this unrolled form), and its exact
 * gradient with respect to every weight of the setup and solve networks,
 * from a hand-written adjoint (reverse sweep over the cycles with per-cycle
 * checkpointing: only r_k is kept, B's intermediates are recomputed).
 * coeff[i]: nodal k of problem i, (n[i]+2)^2 doubles (the non-divergence
 * form: mu on the n[i]^2 interior nodes); rhs[i]: f, n[i]^2 doubles; host or
 * device.  Problems of equal n are batched together.
 * Arithmetic: FP64 for an FP64 context, FP32 otherwise (gradients are
 * accumulated in FP64).  grad (weight_count doubles, host or device) may be
 * NULL to evaluate the loss only.  Divergence form only.
 * Errors: STATE (no weights), ARG, SIZE, NONFINITE (zero f or non-finite loss). */
int mgcnn_loss_grad(mgcnn_ctx* ctx, int nprob, const double* const* coeff, const double* const* rhs,
                    const int* n, int K, double* loss, double* grad);

/* One Adam update (Kingma & Ba; the paper trains with Adam, Appendix A) of the
 * context's weights with gradient `grad` (weight_count doubles, host or
 * device): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  Moments live in
 * the context and start at zero.  Invalidates the current setup. */
int mgcnn_adam_step(mgcnn_ctx* ctx, const double* grad, double lr, double beta1, double beta2, double eps);

/* mgcnn_loss_grad followed by mgcnn_adam_step (beta 0.9, 0.999, eps 1e-8)
 * with the gradient kept on the device; grad may be NULL. */
int mgcnn_train_step(mgcnn_ctx* ctx, int nprob, const double* const* coeff, const double* const* rhs,
                     const int* n, int K, double lr, double* loss, double* grad);

/* Copy the context's current weights (layout of mgcnn_weight_count) out. */
int mgcnn_get_weights(mgcnn_ctx* ctx, double* w, size_t count);

/* Implementation options (no counterpart in the paper).
 * MGCNN_OPT_FUSED (default 1): in MIXED_BF16 mode with 8 channels and one
 * layer per ResNet, run each level of the V-cycle as two fused kernels (down:
 * [reChannel-in] + ResNetDown + RCNN; up: TCNN-add + ResNetUp [+ reChannel-out
 * and the FP64 update]); 0 runs one kernel per layer.  Both compute the same
 * function; roundings to BF16 happen at different points.
 * MGCNN_OPT_DEVICE_LOOP (default 1): where the fused kernels apply, mgcnn_solve
 * runs the whole stationary iteration as one launch of a CUDA graph with a
 * conditional WHILE node (residual, norm, convergence test and V-cycle on the
 * device, no host round trip per cycle; the graph is captured once per setup,
 * f and u are copied through the context's buffers); 0 runs the host loop
 * (one 8-byte readback per cycle).  Both give identical iterates.
 * MGCNN_OPT_TILE (default -1): tile shape of the fused kernels.  -1: the first
 * solve after a setup on a new grid size times every shape on every level and
 * keeps the fastest; 0..7: that shape on every level, no timing (0 = 16 x 32,
 * 1 = 8 x 32, 2 = 16 x 16, 3 = 32 x 32, 4 = 24 x 32 fine pixels per block,
 * rows x columns; 5 = 24 x 30, 6 = 32 x 30 and 7 = 22 x 30 for the up kernels
 * with 24 x 32 for the down kernels, whose restriction needs other widths);
 * other values:
 * ERR_ARG.  Every shape gives bit-identical results: a pixel's arithmetic does
 * not depend on the tile that holds it.  Applies to mgcnn_solve and
 * mgcnn_solve_krylov; the batched solves keep their own timing.
 * MGCNN_OPT_SYMMETRIC (default 0): the symmetric network variant, see
 * mgcnn_setup_bpx; 1 on, 0 off (weights stay as they are). */
/* MGCNN_OPT_FUSED_RESIDUAL (default 0): where mgcnn_solve forms each cycle's FP64
 * residual r = f - A u and its norm when the fused kernels apply.  0: a separate
 * residual pass before each cycle.  1: inside the finest-level down kernel, on
 * that kernel's tiles and their halo.  2: inside the finest-level up kernel, from
 * the u + e it has just formed (its tiles carry a halo of one more pixel), for
 * the next cycle; the first residual comes from the separate pass.  The same
 * FP64 arithmetic per unknown in all three (bit-identical iterates); the norm is
 * summed in a different order.  Modes 1 and 2 run slower than the separate pass
 * on this GPU (the fused kernels add latency-bound FP64 loads to a kernel that
 * is latency-bound already, mode 1 also FP64 work on the halo), so 0 is the
 * default. */
/* MGCNN_OPT_COARSE_TAIL (default 0): where the fused kernels apply, the levels
 * below the finest whose grid side is at most this value (and at most 255),
 * when there are at least two of them, run down and back up in one cooperative
 * kernel with grid-wide barriers between the levels (16 x 32 tiles) instead of
 * two launches per level: the same arithmetic per pixel, results bit-identical.
 * Slower than a launch per level on a GB300 (each level step inside one kernel,
 * tile copies and the barrier included, takes longer than a level kernel
 * launched programmatically after the previous one), so off by default.
 * 0: one launch per level, as also where the device offers no cooperative launch
 * or a CUDA graph of the solve cannot hold one (the context then keeps 0).
 * The classes of a batch share the device's resident blocks between their tail
 * kernels; contexts whose solves overlap on one device do not, and should set 0
 * (the barrier waits are bounded: past about a second the call fails
 * with MGCNN_ERR_TIMEOUT instead of hanging). */
/* MGCNN_OPT_DIVTOL (default 0, off): a value d in 1..300 stops mgcnn_solve and
 * each problem of mgcnn_solve_batched once ||r_k||/||f|| > 10^d, before cycle k,
 * with status MGCNN_ERR_DIVERGED (iters = k, relres[k] recorded, u the iterate
 * u_k); the usual divergence test of iterative solvers, which ends a failing
 * problem long before maxit.  mgcnn_solve_batched_krylov applies it to the true
 * residual before each restart cycle; mgcnn_solve_krylov does not use it.
 * Errors: ARG for a value outside 0..300. */
/* MGCNN_OPT_COARSE_K (default 0): how the divergence form's k reaches the
 * coarse grids before rediscretisation (Sec. 2.3 leaves it open).  0: full
 * weighting of log k (a geometric mean), 1: full weighting of k itself (an
 * arithmetic mean, never below the geometric one, so stiffer coarse
 * operators).  On smooth lognormal k the geometric mean converges in fewer
 * cycles.  On piecewise-constant high-contrast k the geometric mean makes the
 * coarse-grid correction over-correct and the V-cycle diverge.  The arithmetic
 * mean keeps the V-cycle stable there, a preconditioner that flexible GMRES
 * (mgcnn_solve_krylov) turns into a solver.  Takes effect at the next setup;
 * the non-divergence form injects mu either way.  Errors: ARG for other values. */
enum { MGCNN_OPT_FUSED = 1, MGCNN_OPT_DEVICE_LOOP = 2, MGCNN_OPT_TILE = 3, MGCNN_OPT_SYMMETRIC = 4,
       MGCNN_OPT_FUSED_RESIDUAL = 5, MGCNN_OPT_COARSE_TAIL = 6, MGCNN_OPT_DIVTOL = 7, MGCNN_OPT_COARSE_K = 8 };
int mgcnn_set_option(mgcnn_ctx* ctx, int option, int value);

/* Instrumentation (no counterpart in the paper; used by the benchmark).
 * mgcnn_kernel_launches: kernels launched by this library in this process.
 * mgcnn_profile(ctx, 1): from now on bracket the finest-level launch of each
 * kernel class, and the fused kernels of every level, with CUDA events on the
 * context's stream; mgcnn_profile_read returns, per class, the summed
 * milliseconds and the number of launches since the last read (classes: 0
 * residual, 1 ResNet layer, 2 restriction, 3 prolongation-add into the finest
 * level, 4 reChannel-in, 5 reChannel-out with update, 6 fused down kernel, 7
 * fused up kernel of the finest level; 8 + l fused down kernel and 21 + l
 * fused up kernel of level l = 1..12, 34 classes in all) and clears them.
 * Timing adds one event pair per bracketed launch.  While profiling is on, mgcnn_solve runs its host-driven loop (not
 * the device-side loop of MGCNN_OPT_DEVICE_LOOP), so that every bracketed
 * kernel is a plain launch on the context's stream. */
long long mgcnn_kernel_launches(void);
/* Check of the failure path of the fused kernels' tile waits (no counterpart in
 * the paper): one block waits on a tile copy that is never issued, gives up
 * after eight suspended waits of at most 1 ms, and sets the context's device
 * error flag; the call then returns MGCNN_ERR_TIMEOUT, as a solve whose copies
 * never arrived would, and the context stays usable (the flag is cleared).
 * Nothing faults or hangs. */
int mgcnn_check_wait_timeout(mgcnn_ctx* ctx);
int mgcnn_profile(mgcnn_ctx* ctx, int enable);
int mgcnn_profile_read(mgcnn_ctx* ctx, double* ms, long long* counts, int nkinds);

/* r = f - A u and ||r||_2^2 without allocating anything (no counterpart in the
 * paper: an interface for callers that cannot call cudaMalloc -- hosts that
 * give the library a fixed device-memory budget owned by their own allocator,
 * where a hidden allocation would break that budget, or tools that may only
 * touch the buffers they were handed).
 * op: the operator of one grid as 5 planes of n*n doubles (a_C, a_W, a_E, a_S,
 * a_N, layout of mgcnn_get_operator); f, u, r: n*n doubles.  All four must be
 * DEVICE pointers owned by the caller (host pointers: ERR_ARG, since staging
 * them would need an allocation).  norm2: host pointer or NULL.  stream:
 * cudaStream_t as void* (NULL: legacy default stream); the call synchronises it.
 * Same kernels and the same deterministic reduction as mgcnn_residual.
 * Scratch: the per-block partial sums live in a fixed array inside the library
 * (8,193 doubles, 64 KiB, held by every GPU that loads the library until the
 * process exits), so n*n may not exceed 16,777,216 (n <= 4096): larger grids
 * return ERR_SIZE before anything is launched.  The first call on a device
 * looks the array's device address up (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call
 * overwrites the array and all calls share it: calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * Allocates no device or pinned memory. */
int mgcnn_residual_noalloc(const double* op, const double* f, const double* u, double* r, int n,
                           double* norm2, void* stream);

/* Human-readable name of a status code (static storage). */
const char* mgcnn_status_string(int status);

/* Message describing the last failure on this context ("" if none). */
const char* mgcnn_last_error(const mgcnn_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MGCNN_H */

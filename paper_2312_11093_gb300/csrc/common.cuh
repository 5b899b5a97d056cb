// Internal definitions shared by the translation units of libmgcnn.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mgcnn.h"

namespace mgcnn {

constexpr int kFeatures = 5;      // setup-network input features per node
constexpr int kSetupLayers = 4;   // NonLinearResNet depth (Sec. 3.2: "four layers")
constexpr int kMaxLevels = 13;    // n <= 16383
constexpr int kMaxSweeps = 16;    // layers per ResNetDown / ResNetUp
struct TrainGroup;
struct BatchClass;

// Status carried through the library; converted to the ABI code at the boundary.
struct Status {
  int code = MGCNN_OK;
  std::string msg;
  bool ok() const { return code == MGCNN_OK; }
};

// A device allocation that grows on demand and is freed by the context.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

// Offsets (in elements) of each weight tensor in the flat weight blob.
struct WeightLayout {
  int C = 0, nu_d = 0, nu_u = 0;
  size_t w_in, w_down, w_up, w_R, w_P, w_out, sw_in, sb_in, sw, sb, sw_R, total;
  void build(int C_, int nd, int nu) {
    C = C_; nu_d = nd; nu_u = nu;
    size_t CC9 = (size_t)C * C * 9, o = 0;
    w_in = o;   o += (size_t)C * 9;
    w_down = o; o += (size_t)nu_d * CC9;
    w_up = o;   o += (size_t)nu_u * CC9;
    w_R = o;    o += CC9;
    w_P = o;    o += CC9;
    w_out = o;  o += (size_t)C * 9;
    sw_in = o;  o += (size_t)C * kFeatures * 9;
    sb_in = o;  o += (size_t)C;
    sw = o;     o += (size_t)kSetupLayers * CC9;
    sb = o;     o += (size_t)kSetupLayers * C;
    sw_R = o;   o += CC9;
    total = o;
  }
};

struct Level {
  int n = 0;          // interior nodes per side
  double h = 0;       // mesh width 1/(n+1)
  size_t N() const { return (size_t)n * n; }
};

// Jacobi weights of the analytic (GMG-equivalent) setup tensors: `fine` on the
// finest level, `coarsest` on the coarsest, `mid` on every level in between; a
// one-level hierarchy takes `fine` (weighted Jacobi of Sec. 2.3 with the weight
// chosen per level).
struct LevelWeights {
  double fine = 0.0, mid = 0.0, coarsest = 0.0;
  static LevelWeights uniform(double w) { return {w, w, w}; }
  bool valid() const {
    for (double w : {fine, mid, coarsest})
      if (!(w > 0.0 && w < 2.0)) return false;
    return true;
  }
  double at(int l, int L) const { return l == 0 ? fine : (l == L - 1 ? coarsest : mid); }
};

class TmaMaps;   // tma.cuh

// FP32 weights of the fused down kernel's input layer W_in (8 channels), passed
// by value: they sit in the kernel-parameter constant bank and the unrolled
// loop reads them as constant operands, with no shared-memory loads.
// Layout w_in[t][co] (t = 3 a + b).
struct SmallWeights {
  float w_in[72];
};

// FP32 weights of the fused setup kernel's small layers, by value like
// SmallWeights: v[0..32) = b_i [4][8], v[32..392) = W_cin [8][5][9],
// v[392..400) = b_cin [8].
struct SetupSmallWeights {
  float v[400];
};

}  // namespace mgcnn

// The opaque context of the ABI.
struct mgcnn_ctx {
  mgcnn_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string last_error;

  mgcnn::WeightLayout wl;
  bool have_weights = false;
  mgcnn::DevBuf w64, w32;                 // weight blob in FP64 and FP32

  bool have_setup = false;
  int n = 0, L = 0;
  std::vector<mgcnn::Level> lv;
  mgcnn::DevBuf coef[mgcnn::kMaxLevels];  // nodal k (or mu) per level
  mgcnn::DevBuf op[mgcnn::kMaxLevels];    // 5 x n_l^2 FP64 stencil per level
  mgcnn::DevBuf s64[mgcnn::kMaxLevels];   // setup tensors FP64 [n_l^2][C]
  mgcnn::DevBuf s16[mgcnn::kMaxLevels];   // setup tensors BF16 [n_l^2][C]
  mgcnn::DevBuf xa[mgcnn::kMaxLevels];    // state ping-pong buffers, per level
  mgcnn::DevBuf xb[mgcnn::kMaxLevels];
  mgcnn::DevBuf setup_a, setup_b, setup_c, setup_d;  // setup-phase scratch
  mgcnn::DevBuf feat;                     // setup features [n^2][5]
  mgcnn::DevBuf f, u, r, e;               // finest-grid FP64 vectors (staging / work)
  mgcnn::DevBuf u2;                       // second iterate buffer: with the residual formed in the up
                                          // kernel, cycles alternate u -> u2 -> u (halo reads of u_k
                                          // must not see a neighbour's u_{k+1})
  mgcnn::DevBuf r32;                      // FP32 network input (r or D^{-1} r) for the mixed path
  mgcnn::DevBuf dinv, dinv32;             // 1/a_C of the finest level, FP64 and FP32
  mgcnn::DevBuf partial;                  // per-block partial sums of reductions
  // mixed-precision path (mixed.cu)
  int cp = 0;                             // channels padded for the tensor cores (8 or 16)
  int fused = 1;                          // use the fused level kernels when they apply
  int fuse_residual = 0;                  // mgcnn_solve: where the residual is formed (MGCNN_OPT_FUSED_RESIDUAL)
  int tail_n = 0;                         // MGCNN_OPT_COARSE_TAIL: the levels of at most this grid side in one
                                          // cooperative kernel (0: a launch per level; reset to 0 if refused)
  bool pdl = true;                        // level kernels with programmatic dependent launch (off if a graph
                                          // with programmatic edges cannot be built)
  int tile_var[2][mgcnn::kMaxLevels] = {};  // autotuned tile variants (down, up) per level
  bool tuned = false;                       // set by the first solve after a setup
  int tile_fixed = -1;                      // MGCNN_OPT_TILE: a fixed tile variant, or -1 (autotune)
  int symmetric = 0;                        // MGCNN_OPT_SYMMETRIC: tied adjoint up sweep (FP64)
  struct TunedClass {                       // tile variants chosen for batched classes, per (n, batch)
    int n, batch;
    int var[2][mgcnn::kMaxLevels];
  };
  std::vector<TunedClass> tuned_classes;
  mgcnn::DevBuf x16a[mgcnn::kMaxLevels];  // BF16 state ping-pong, [n_l^2][cp]
  mgcnn::DevBuf x16b[mgcnn::kMaxLevels];
  mgcnn::DevBuf x16l[mgcnn::kMaxLevels];  // low BF16 part of the up sweep's output, levels >= 1
  mgcnn::DevBuf wmix;                     // packed weights: mma fragments + FP32 small layers
  mgcnn::TmaMaps* tma = nullptr;          // tensor maps of the fused kernels' TMA tile loads
  mgcnn::DevBuf kerr;                     // device flag: a kernel gave up waiting for its tile copies
  mgcnn::DevBuf alpha32;                  // input scale of the fused V-cycle (alpha, 1 / alpha)
  mgcnn::SmallWeights small_w{};          // host copy of the fused down kernel's W_in
  int out_lo = 1;                         // W_out has a nonzero BF16 lo part (the fused up kernel's second pass)
  mgcnn::SetupSmallWeights setup_small_w{};  // host copy of the fused setup kernel's small layers
  mgcnn::DevBuf s32tmp;                   // FP32 setup output before the BF16 cast
  mgcnn::DevBuf scalars;                  // device scalars (norms)
  // training (train.cu)
  std::vector<mgcnn::TrainGroup> groups;
  mgcnn::DevBuf grad, wT, adam_m, adam_v;
  long long adam_t = 0;
  // device-side solve loop (solve_graph.cu)
  int device_loop = 1;                    // option: run mgcnn_solve as one conditional CUDA graph
  double divtol = 0.0;                    // MGCNN_OPT_DIVTOL: stop when ||r||/||f|| > divtol (0: never)
  int coarse_k_arith = 0;                 // MGCNN_OPT_COARSE_K: arithmetic full weighting of k
  bool graph_failed = false, sgraph_valid = false;
  cudaGraphExec_t sgraph = nullptr;
  long long sgraph_kernels = 0;
  cudaStream_t gstream = nullptr;
  cudaStream_t cstream = nullptr;         // host-to-device copies of mgcnn_solve's inputs, overlapping the
  cudaEvent_t cevent = nullptr;           // setup kernels still running on `stream`; joined by this event
  mgcnn::DevBuf gstate, ghist, gparams;
  // classical GMG comparator (gmg.cu): per-level rhs, correction, ping-pong
  mgcnn::DevBuf gmg_r[mgcnn::kMaxLevels], gmg_e[mgcnn::kMaxLevels], gmg_t[mgcnn::kMaxLevels];
  // flexible GMRES (mgcnn_solve_krylov): basis V, preconditioned directions Z, work vectors,
  // Gram-Schmidt coefficients and the dots' per-block partial sums
  mgcnn::DevBuf kV, kZ, kw, kr, kcoef, kpart;
  // batched solves (batch.cu)
  std::vector<mgcnn::BatchClass> bcls;
  int bn = 0, bmaxit = -1;
  bool bready = false;
  std::vector<int> bcls_of, bidx_of;
  cudaStream_t bstream = nullptr;
  cudaEvent_t bfork = nullptr;
  cudaGraphExec_t bgraph = nullptr;
  bool bwhile = false;                    // bgraph is the whole batch (WHILE node), not one cycle
  long long bgraph_kernels = 0;
  mgcnn::DevBuf bparams, bcount;         // bcount: [0] problems active after this cycle's checks, [1] cycles
  int* h_bcount = nullptr;
  // optional per-kernel timing (mgcnn_profile)
  int prof = 0;
  std::vector<cudaEvent_t> ev_start, ev_stop;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  double* h_scalars = nullptr;            // pinned host mirror of `scalars`
};

namespace mgcnn {

Status make_status(int code, const char* fmt, ...);
Status cuda_status(cudaError_t e, const char* what);
Status ensure(DevBuf& b, size_t bytes);
void release(DevBuf& b);
bool is_device_pointer(const void* p);

#define MG_CUDA(call)                                              \
  do {                                                             \
    cudaError_t _e = (call);                                       \
    if (_e != cudaSuccess) return ::mgcnn::cuda_status(_e, #call); \
  } while (0)

// Every kernel launch site is followed by MG_LAUNCH, which also counts it.
void count_launch();
void add_launches(long long k);   // kernels launched through a CUDA graph
#define MG_LAUNCH(what)                                            \
  do {                                                             \
    ::mgcnn::count_launch();                                       \
    cudaError_t _e = cudaGetLastError();                           \
    if (_e != cudaSuccess) return ::mgcnn::cuda_status(_e, what);  \
  } while (0)

// Profiling kinds: finest-level launches bracketed by events when enabled.
enum ProfKind { kProfResidual = 0, kProfResnet = 1, kProfRestrict = 2, kProfProlong = 3, kProfIn = 4,
                kProfOut = 5, kProfDown0 = 6, kProfUp0 = 7,
                // fused down / up kernel of level l >= 1: kProfDownLevel + l, kProfUpLevel + l;
                // the coarse tail kernel takes the unused slot of level 0
                kProfDownLevel = 8, kProfTail = kProfDownLevel, kProfUpLevel = 8 + kMaxLevels,
                kProfKinds = 8 + 2 * kMaxLevels };
// The context's device error flag (kerr) is the first of kErrWords words; from
// word kTailBarrierWord on, pairs of words hold the coarse tail kernels' grid
// barriers (arrival count, generation; zero when no kernel is inside one): pair
// 0 for the context's single problem, pair 1 + i for class i of a batch.
constexpr int kErrWords = 64, kTailBarrierWord = 2, kTailBarriers = (kErrWords - kTailBarrierWord) / 2;
int prof_begin(mgcnn_ctx* c, int kind);   // -1 when profiling is off
void prof_end(mgcnn_ctx* c, int slot);

#define MG_TRY(expr)                       \
  do {                                     \
    ::mgcnn::Status _s = (expr);           \
    if (!_s.ok()) return _s;               \
  } while (0)

inline int grid_for(size_t work, int block) {
  return (int)((work + block - 1) / block);
}

}  // namespace mgcnn

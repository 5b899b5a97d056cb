// Fused level kernels of the mixed-precision solve phase for 8 channels
// (one 16-byte BF16 vector per pixel) and one layer per ResNetDown/Up, the
// configuration of the paper's experiments (Sec. 4.1: sweeps = 1, C = 8).
//
// Down kernel, level l (Algorithm 3, down loop):
//   [finest level: x_1 = alpha W_in * r, FP32 FMAs, weights as constants]
//   x_l <- x_l + K_down (s_l * x_l)            tensor cores (implicit GEMM, skip folded in)
//   x_{l+1} = RCNN(x_l)                        tensor cores, stride 2
// One block owns an FH x FW fine tile (16 x 32, 8 x 32, 16 x 16, 32 x 32 or 24 x 32, autotuned)
// and the coarse tile under it.  The restriction needs one extra fine row and
// column, which the block recomputes instead of reading a neighbour's.
//
// Up kernel, level l (Algorithm 3, up loop):
//   x_l <- x_l + TCNN(x_{l+1})                 tensor cores, per pixel-parity class
//   x_l <- x_l + K_up (s_l * x_l)              tensor cores (skip folded in)
//   [finest level: e = W_out * x_1 / alpha     tensor cores, BF16 hi + lo weights
//    u <- u + e                                FP64, full warps]
// One block owns an FH x FW fine tile, with a 1-pixel halo of the layer input
// (2 at the finest level, where W_out needs the layer output's halo).
//
// Tiles arrive by TMA (tma.cuh; zero fill outside the grid).  Tensor-core
// tiling: a warp computes 16 output pixels x 8 channels with mma.m16n8k16 (+
// m16n8k8), A rows fetched by ldmatrix from per-lane shared-memory addresses,
// so a strip can be any 16 pixels of an odd-sized region.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>

#include "fpconv.cuh"
#include "mixed.cuh"
#include "ops.cuh"
#include "tma.cuh"

namespace mgcnn {

using bf16 = __nv_bfloat16;
using bf162 = __nv_bfloat162;

namespace {

// Fine tile owned by a block: FH x FW, a template parameter chosen per level
// size by the autotuner (variants below).
constexpr int NT = 256;              // threads per block (8 warps)
constexpr int NW = NT / 32;

// ldmatrix on 32-bit shared-window addresses: tile bases are converted once
// and offsets added in bytes, instead of converting a generic pointer per load
__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void ldsm_x4(uint32_t* r, uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t* r, uint32_t a) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
// The MMAs only read and write registers, so they are not volatile: the
// compiler may schedule them around the (volatile) shared-memory loads.
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma1688(float* d, uint32_t a0, uint32_t a1, uint32_t b0) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ uint32_t f2bf(float a, float b) {
  bf162 r = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&r);
}
// s * x of 8 channels with packed BF16 multiplies: the product of two BF16
// values is exact in FP32, so rounding it once to BF16 here gives the bits that
// widening, multiplying in FP32 and rounding back would.
__device__ __forceinline__ uint32_t bmul2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("mul.rn.bf16x2 %0, %1, %2;\n" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ float2 bf2_to_f2(uint32_t v) {
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}
__device__ __forceinline__ uint4 mul8(uint4 a, uint4 b) {
  return make_uint4(bmul2(a.x, b.x), bmul2(a.y, b.y), bmul2(a.z, b.z), bmul2(a.w, b.w));
}

// Sum of one double per thread over the block (fixed order: warp shuffles, then
// the warps' sums by warp 0); the result is valid in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = (lane < NW) ? red[lane] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The tiles of a block live in dynamic shared memory (the 32 x 32 variant needs
// more than the 48 KB of static shared memory); every array starts on a 128-byte
// boundary (TMA destinations).
constexpr int pad8(int pixels) { return (pixels + 7) / 8 * 8; }   // uint4 count -> multiple of 128 bytes
// The down kernel's layer output tile split by column parity: row pitch XP
// pixels, column c at c / 2 (even c) or XE + c / 2 (odd c).  The restriction's
// A rows (16 coarse pixels of a row, stride two in fine columns) then sit on
// consecutive pixels, free of shared-memory bank conflicts; XE = 4 (mod 8)
// keeps the layer's stores of eight consecutive columns conflict-free too.
constexpr int split_xe(int xw) { return ((xw + 1) / 2 + 3) / 8 * 8 + 4; }
constexpr int split_xp(int xw) { return split_xe(xw) + xw / 2; }
template <int XW>
struct SplitCols {
  static constexpr int XE = split_xe(XW);
  static constexpr int XP = split_xp(XW);
  static __device__ __forceinline__ int col(int c) { return (c & 1) ? XE + (c >> 1) : (c >> 1); }
  // the restriction's taps (a, b): row a, column b of the coarse pixel's 3 x 3 window
  uint32_t off[4];
  __device__ __forceinline__ SplitCols() {
    const int kh = (threadIdx.x & 31) >> 4;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int t = 2 * s + kh, b = t % 3;
      off[s] = 16u * ((t / 3) * XP + (b == 1 ? XE : b / 2));
    }
  }
  static constexpr uint32_t off8 = 16u * (2 * XP + 1);
};

// Bytes of the down kernel's layer-output slot (the split-column tile where a
// restriction follows): on the finest level it first
// holds u (FP64) on the residual region plus one pixel when the residual is
// computed in the kernel.
template <int FH, int FW, bool FIRST, bool HAS_R>
constexpr size_t down_xd_bytes() {
  constexpr int XH = FH + (HAS_R ? 1 : 0), XW = FW + (HAS_R ? 1 : 0);
  constexpr size_t xd = HAS_R ? 16u * pad8(XH * split_xp(XW)) : 0u;
  constexpr size_t us = FIRST ? (8u * (XH + 6) * (XW + 6) + 127) / 128 * 128 : 0u;
  return (FIRST && us > xd) ? us : xd;
}
// The finest level's residual tile: RH rows of r (halo 2 around the layer
// output region) staged by TMA from column i0 - 4 (a 16-byte aligned start) in
// rows of down_rwt floats (a multiple of 4), so region column c sits at tile
// column c + 2.
template <int FW, bool HAS_R>
constexpr int down_rwt() {
  constexpr int RW = FW + (HAS_R ? 1 : 0) + 4;
  return (RW + 2 + 3) / 4 * 4;
}
template <int FH, int FW, bool FIRST, bool HAS_R>
constexpr size_t down_smem_bytes() {
  constexpr int XH = FH + (HAS_R ? 1 : 0), XW = FW + (HAS_R ? 1 : 0), ZH = XH + 2, ZW = XW + 2;
  constexpr int RH = ZH + 2;
  return 16u * (2 * pad8(ZH * ZW)) + down_xd_bytes<FH, FW, FIRST, HAS_R>() +
         (FIRST ? 4u * RH * down_rwt<FW, HAS_R>() : 0u);
}
// Up-kernel regions for an FH x FW owned tile at (j0, i0), fine coordinates:
//   O (layer output):   owned + halo H (H = 1 at the finest level, where W_out
//                       needs the layer output around the owned pixels)
//   P (layer input):    O + halo 1
//   Q (staged x_down, s): P, extended by one row / column on each side where
//                       needed so that it is made of whole quads -- 2 x 2 blocks
//                       (2J+1.., 2I+1..) of fine pixels -- when a coarser level
//                       feeds the TCNN (Q starts on an odd row and column)
//   coarse pixels (J, I) of the quads plus one row and column (the quads'
//   sources J..J+1, I..I+1)
//   E (finest level):   where e = W_out * x_fin and u + e are formed: the owned
//                       pixels, plus a halo of one when the kernel also forms
//                       the next residual (RES), which needs u + e around
//                       every owned pixel; O = E + halo 1
template <int FH, int FW, bool LAST, bool HAS_P, bool RES = false>
struct UpGeom {
  static_assert(LAST || !RES, "the residual is formed on the finest level only");
  static constexpr int HE = RES ? 1 : 0;
  static constexpr int EH = FH + 2 * HE, EW = FW + 2 * HE;
  static constexpr int H = LAST ? HE + 1 : 0;
  static constexpr int OH = FH + 2 * H, OW = FW + 2 * H;
  static constexpr int PH = OH + 2, PW = OW + 2;
  static constexpr int QOFF = (HAS_P && (H & 1)) ? 1 : 0;  // P's offset inside Q (Q starts on an odd row)
  static constexpr int QH = PH + 2 * QOFF, QW = PW + 2 * QOFF;
  static constexpr int NQH = QH / 2, NQW = QW / 2;         // quads
  static constexpr int CQH = NQH + 1, CQW = NQW + 1;       // coarse pixels staged
  static_assert(!HAS_P || (QH % 2 == 0 && QW % 2 == 0), "whole quads");
  // finest level, after the layer: e (FP32) on E, then u + e (FP64) on E, in the z tile
  static_assert(!LAST || EH * EW * (4 + 8) + 8 <= 16 * QH * QW, "E staging in the z tile");
};
// Tiles: ps, zs on Q; pl on O; the coarse tiles cs (hi) and cl (lo).
template <int FH, int FW, bool LAST, bool HAS_P, bool RES = false>
constexpr size_t up_smem_bytes() {
  using G = UpGeom<FH, FW, LAST, HAS_P, RES>;
  return 16u * (2 * pad8(G::QH * G::QW) + pad8(G::OH * G::OW) + (HAS_P ? 2 * pad8(G::CQH * G::CQW) : 0));
}
extern __shared__ __align__(128) unsigned char fused_dsm[];

// Per-lane tap offsets of a shared-memory tile with row pitch PITCH (in
// pixels): this lane's four taps 2s + kh (kh = lane / 16) of the x4 loads and
// the ninth tap, relative to the tap-(0,0) pixel of the lane's A row.
template <int PITCH>
struct TapOffsets {
  uint32_t off[4];   // bytes (16 per pixel)
  __device__ __forceinline__ TapOffsets() {
    const int kh = (threadIdx.x & 31) >> 4;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int t = 2 * s + kh;
      off[s] = 16u * ((t / 3) * PITCH + t % 3);
    }
  }
  static constexpr uint32_t off8 = 16u * (2 * PITCH + 2);
};

// strip_conv with precomputed addressing: base_m is the tap-(0,0) pixel of
// A row m = (lane & 7) + 8 ((lane >> 3) & 1) (the x4 loads), base_l the one of
// row lane & 15 (the ninth tap's x2 load).
template <class Taps>
__device__ __forceinline__ void strip_conv_taps(const uint4* tile, const uint32_t* wf, int base_m, int base_l,
                                                const Taps& to, float* acc) {
  const uint32_t am = sa(tile) + 16u * base_m, al = sa(tile) + 16u * base_l;
  uint32_t a[4][4], a8[2];
#pragma unroll
  for (int s = 0; s < 4; ++s) ldsm_x4(a[s], am + to.off[s]);
  ldsm_x2(a8, al + Taps::off8);
#pragma unroll
  for (int s = 0; s < 4; ++s) mma16816(acc, a[s], wf[2 * s], wf[2 * s + 1]);
  mma1688(acc, a8[0], a8[1], wf[8]);
}

template <int PITCH>
__device__ __forceinline__ void strip_conv_at(const uint4* tile, const uint32_t* wf, int base_m, int base_l,
                                              const TapOffsets<PITCH>& to, float* acc) {
  strip_conv_taps(tile, wf, base_m, base_l, to, acc);
}

// One ResNet layer strip y = x + K z (Eq. heteroresnet) with the skip folded
// into the last MMA step: K = 80, the ninth tap's 8 channels of z followed by
// the 8 channels of x at the centre pixel, whose B block is the identity.  zt
// (tile of z) and xt (tile of x) share the pitch; base_m as in strip_conv_at,
// fI the identity half of the last step's B fragment.
template <int PITCH>
__device__ __forceinline__ void layer_strip(const uint4* zt, const uint4* xt, const uint32_t* wf, uint32_t fI,
                                            int base_m, const TapOffsets<PITCH>& to, float* acc) {
  const int lane = threadIdx.x & 31;
  const uint32_t am = sa(zt) + 16u * base_m;
  uint32_t a[5][4];
#pragma unroll
  for (int s = 0; s < 4; ++s) ldsm_x4(a[s], am + to.off[s]);
  // lanes 0-15 address rows 0-15 of tap 8 of z (k 0-7), lanes 16-31 the same
  // rows of x at the centre pixel (k 8-15)
  ldsm_x4(a[4], (lane < 16) ? am + TapOffsets<PITCH>::off8 : sa(xt) + 16u * (base_m + PITCH + 1));
#pragma unroll
  for (int s = 0; s < 4; ++s) mma16816(acc, a[s], wf[2 * s], wf[2 * s + 1]);
  mma16816(acc, a[4], wf[8], fI);
}

// The identity block of the last step's B fragment: k = 8 + ci, n = co, one
// where ci == co (this lane holds ci = 2q, 2q + 1 for co = g).
// Programmatic dependent launch: a level kernel launched with the programmatic
// stream-serialisation attribute may start while its predecessor finishes; it
// runs its prologue (barrier set-up, weight fragments), then waits here until
// the predecessor grid has completed and its memory is visible.  Without the
// attribute both instructions have no effect.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t identity_frag() {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const uint32_t one = 0x3F80u;   // BF16 1.0
  return (2 * q == g ? one : 0u) | ((2 * q + 1 == g ? one : 0u) << 16);
}

// The input scale of the network, alpha ~ sqrt(N / ||r||^2), keeps the BF16
// state near unit size whatever the scale of f.  It is a power of two, so
// scaling by it and back is exact: the cycle's result does not depend on the
// norm it was taken from (nor on that norm's summation order).
__device__ __forceinline__ double alpha_of(const double* norm2, size_t N) {
  const double v = *norm2;
  if (!(v > 0.0) || !isfinite(v)) return 1.0;
  const int e = ilogb(sqrt((double)N / v));
  return ldexp(1.0, max(-120, min(120, e)));
}

// alpha2[2b] = alpha, alpha2[2b + 1] = 1 / alpha, once per cycle and problem:
// an FP64 square root is dozens of FP64-pipe instructions, too many to repeat
// in every block of the level kernels.
__global__ void alpha_kernel(const double* __restrict__ norm2, float* __restrict__ alpha2, size_t N, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const double a = alpha_of(norm2 + b, N);
  alpha2[2 * b] = (float)a;
  alpha2[2 * b + 1] = (float)(1.0 / a);
}

Status launch_alpha(const FusedLevels& fl, const double* norm2, cudaStream_t st) {
  if (!fl.alpha) return make_status(MGCNN_ERR_STATE, "fused levels without an alpha buffer");
  alpha_kernel<<<(fl.batch + 127) / 128, 128, 0, st>>>(norm2, fl.alpha, (size_t)fl.n[0] * fl.n[0], fl.batch);
  MG_LAUNCH("alpha_kernel");
  return {};
}

// ---------------------------------------------------------------------------
// Down kernel.  Regions, in fine coordinates relative to (j0, i0) = (2 J0, 2 I0):
//   X (layer output kept):   rows 0..XH-1, cols 0..XW-1 (XH = 16 + R, XW = 32 + R)
//   Z (layer input, halo 1): rows -1..XH,  cols -1..XW
//   Rg (residual, halo 2):   rows -2..XH+1, cols -2..XW+1   (finest level only)
// The down kernel's work on the tile (tbx, tby) of problem tbz (one block).
template <int FH, int FW, bool FIRST, bool HAS_R, bool RESID>
__device__ __forceinline__ void down_body(const float* __restrict__ r, const float* __restrict__ alpha2,
                                          const ResidIn& ra, const SmallWeights& sw, const CUtensorMap& map_x,
                                          const CUtensorMap& map_s, const CUtensorMap& map_r,
                                          const uint32_t* __restrict__ fK, const uint32_t* __restrict__ fR,
                                          bf16* __restrict__ xdown, bf16* __restrict__ xc, int n,
                                          const int* __restrict__ active, int* __restrict__ err, int tbx, int tby,
                                          int tbz) {
  static_assert(FH % 2 == 0 && FW % 2 == 0 && (FH / 2) * (FW / 2) % 16 == 0, "tile shape");
  static_assert(FIRST || !RESID, "the residual is fused into the finest level only");
  constexpr int XH = FH + (HAS_R ? 1 : 0), XW = FW + (HAS_R ? 1 : 0);
  constexpr int ZH = XH + 2, ZW = XW + 2;
  constexpr int RH = ZH + 2, RW = ZW + 2, RWT = down_rwt<FW, HAS_R>();
  // zs: s, then z = s * x_in in place (BF16); xs: x_in, for the skip.  Both are
  // TMA destinations: the box of rows j0-1.. and columns i0-1.. of the tensor,
  // zero outside the grid.  rs (finest level): r on rows j0-2.., columns
  // i0-4.., zero outside the grid (TMA, or the fused residual pass).
  uint4* zs = reinterpret_cast<uint4*>(fused_dsm);
  uint4* xs = zs + pad8(ZH * ZW);
  uint4* xd = xs + pad8(ZH * ZW);                                   // layer output
  float* rs = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(xd) +
                                      down_xd_bytes<FH, FW, FIRST, HAS_R>());   // finest level only
  __shared__ __align__(8) uint64_t bar;
  const int j0 = tby * FH, i0 = tbx * FW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t N = (size_t)n * n;
  // problem tbz of a batch of equal-size problems stored back to back
  const int bz = tbz;
  {
    const size_t Nc = (size_t)((n - 1) / 2) * ((n - 1) / 2);
    if (FIRST) r += bz * N;
    xdown += bz * N * 8;
    if (HAS_R) xc += bz * Nc * 8;
  }
  // prologue (may overlap the previous kernel's end): weight fragments, barrier
  uint32_t wk[9], wr[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    wk[k] = fK[k * 32 + lane];
    if (HAS_R) wr[k] = fR[k * 32 + lane];
  }
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  pdl_wait();
  if (active && !active[bz]) return;
  constexpr bool R_TMA = FIRST && !RESID;
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, (FIRST ? 1u : 2u) * ZH * ZW * 16u + (R_TMA ? 4u * RH * RWT : 0u));
    tma_load_pix(zs, &map_s, i0 - 1, j0 - 1, bz, &bar);
    if (!FIRST) tma_load_pix(xs, &map_x, i0 - 1, j0 - 1, bz, &bar);
    if (R_TMA) tma_load_f32(rs, &map_r, i0 - 4, j0 - 2, bz, &bar);
  }
  __syncthreads();   // barrier initialised

  if constexpr (FIRST && RESID) {
    // r = f - A u (FP64, Eq. 1) on the residual region: the same five FMAs, in
    // the same order, as the stand-alone residual kernel; u with a halo of one
    // more pixel is staged in the layer-output tile, which is free until the
    // layer.  The block's owned pixels add r^2 to its partial sum.
    constexpr int UH = RH + 2, UW = RW + 2;
    static_assert(UH * UW * sizeof(double) <= down_xd_bytes<FH, FW, FIRST, HAS_R>(), "u staging");
    double* us = reinterpret_cast<double*>(xd);
    for (int e = threadIdx.x; e < UH * UW; e += NT) {
      const int ur = e / UW, uc = e - ur * UW;
      const int gj = j0 + ur - 3, gi = i0 + uc - 3;
      us[e] = (gj >= 0 && gj < n && gi >= 0 && gi < n) ? ra.u[(size_t)gj * n + gi] : 0.0;
    }
    __syncthreads();
    double rr2 = 0.0;
#pragma unroll 2
    for (int e = threadIdx.x; e < RH * RW; e += NT) {
      const int rr = e / RW, cc = e - rr * RW;
      const int gj = j0 + rr - 2, gi = i0 + cc - 2;
      float v = 0.f;
      if (gj >= 0 && gj < n && gi >= 0 && gi < n) {
        const size_t p = (size_t)gj * n + gi;
        const double* uc = us + (rr + 1) * UW + cc + 1;
        double rv = fma(-ra.op[p], uc[0], ra.f[p]);
        rv = fma(-ra.op[N + p], uc[-1], rv);
        rv = fma(-ra.op[2 * N + p], uc[1], rv);
        rv = fma(-ra.op[3 * N + p], uc[-UW], rv);
        rv = fma(-ra.op[4 * N + p], uc[UW], rv);
        if (rr >= 2 && rr < 2 + FH && cc >= 2 && cc < 2 + FW) rr2 = fma(rv, rv, rr2);
        const float rf = f64_to_f32_rn(rv);
        v = ra.dinv32 ? rf * ra.dinv32[p] : rf;
      }
      rs[rr * RWT + cc + 2] = v;
    }
    __shared__ double red[NW];
    rr2 = block_sum_fixed(rr2, red);
    if (threadIdx.x == 0) ra.partial[blockIdx.y * gridDim.x + blockIdx.x] = rr2;
  }
  // the copies of the block's tiles (a uniform decision: every thread agrees
  // before any of them returns)
  const bool landed = mbar_wait_bounded(&bar, 0);
  if (!__syncthreads_and(landed)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  if constexpr (FIRST) {
    // x_in = alpha (W_in * r) on Z, rounded to BF16 (zero outside the grid); z =
    // s * x_in.  alpha is a power of two, so scaling the sums is exact.
    const float alpha = alpha2[2 * bz];   // the finest level's input scale
    for (int e = threadIdx.x; e < ZH * ZW; e += NT) {
      const int zr = e / ZW, zc = e - zr * ZW;
      const int gj = j0 + zr - 1, gi = i0 + zc - 1;
      uint4 xv = make_uint4(0, 0, 0, 0);
      if (gj >= 0 && gj < n && gi >= 0 && gi < n) {
        float rv[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) rv[t] = rs[(zr + t / 3) * RWT + zc + t % 3 + 2];
        // channel pairs on packed FP32 FMAs: per lane the same fused multiply-adds in
        // the same tap order as one channel at a time
        float2 o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float2 a = make_float2(0.f, 0.f);
#pragma unroll
          for (int t = 0; t < 9; ++t)
            a = __ffma2_rn(make_float2(sw.w_in[t * 8 + 2 * k], sw.w_in[t * 8 + 2 * k + 1]), make_float2(rv[t], rv[t]), a);
          o[k] = make_float2(alpha * a.x, alpha * a.y);
        }
        xv = make_uint4(f2bf(o[0].x, o[0].y), f2bf(o[1].x, o[1].y), f2bf(o[2].x, o[2].y), f2bf(o[3].x, o[3].y));
      }
      xs[e] = xv;
      zs[e] = mul8(xv, zs[e]);
    }
  } else {
    for (int e = threadIdx.x; e < ZH * ZW; e += NT) zs[e] = mul8(xs[e], zs[e]);
  }
  __syncthreads();

  // layer: X = x_in + K (s * x_in); every lane's A-row address is its pixel's
  // tile position plus fixed tap offsets.
  const int g = lane >> 2, q = lane & 3;
  const int mrow = (lane & 7) + ((lane >> 3) & 1) * 8, lrow = lane & 15;
  {
    // strips of 16 consecutive pixels of the Z tile's rows 0..XH-1 (pitch ZW,
    // so a strip's A rows are consecutive tile pixels even where it wraps to
    // the next row: no shared-memory bank conflicts); pixel p of a row is the
    // tap-(0,0) pixel of X pixel p, the last ZW - XW of each row are dropped.
    // The division by the compile-time pitch is a multiply.
    constexpr int NX = XH * ZW, NSTRIP = (NX + 15) / 16;
    static_assert(pad8(ZH * ZW) >= ZH * ZW + ZW - XW, "the dropped pixels' taps stay inside the z tile");
    const TapOffsets<ZW> to;
    const uint32_t fI = identity_frag();
    for (int st = warp; st < NSTRIP; st += NW) {
      const int pm = min(st * 16 + mrow, NX - 1);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      layer_strip<ZW>(zs, xs, wk, fI, pm, to, acc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = st * 16 + g + 8 * h;
        const int xr = p / ZW, xcol = p - xr * ZW;
        if (p >= NX || xcol >= XW) continue;
        const uint32_t o = f2bf(acc[2 * h], acc[2 * h + 1]);
        if constexpr (HAS_R) reinterpret_cast<uint32_t*>(&xd[xr * SplitCols<XW>::XP + SplitCols<XW>::col(xcol)])[q] = o;
        const int gj = j0 + xr, gi = i0 + xcol;
        if (xr < FH && xcol < FW && gj < n && gi < n)
          reinterpret_cast<uint32_t*>(xdown + ((size_t)gj * n + gi) * 8)[q] = o;
      }
    }
  }
  if constexpr (HAS_R) {
    __syncthreads();
    // restriction: coarse (J0 + cr, I0 + cc) over the CH x CW coarse tile, taps
    // (2 cr + a, 2 cc + b) of X; strips of 16 coarse pixels in row-major order
    constexpr int CH = FH / 2, CW = FW / 2;
    const int nc = (n - 1) / 2;
    const int J0 = tby * CH, I0 = tbx * CW;
    using SC = SplitCols<XW>;
    const SC tr;
    for (int st = warp; st < CH * CW / 16; st += NW) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const int pm = st * 16 + mrow, pl = st * 16 + lrow;
      // tap (0, 0) of coarse (cr, cc) is X pixel (2 cr, 2 cc): split column cc
      strip_conv_taps(xd, wr, 2 * (pm / CW) * SC::XP + pm % CW, 2 * (pl / CW) * SC::XP + pl % CW, tr, acc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = st * 16 + g + 8 * h, cr = p / CW, cc = p - cr * CW;
        const int J = J0 + cr, I = I0 + cc;
        if (J < nc && I < nc)
          reinterpret_cast<uint32_t*>(xc + ((size_t)J * nc + I) * 8)[q] = f2bf(acc[2 * h], acc[2 * h + 1]);
      }
    }
  }
  pdl_trigger();   // the next kernel may start its prologue
}

template <int FH, int FW, bool FIRST, bool HAS_R, bool RESID>
__global__ void __launch_bounds__(NT, 4) down_kernel(const float* __restrict__ r, const float* __restrict__ alpha2,
                                                  const __grid_constant__ ResidIn ra,
                                                  const __grid_constant__ SmallWeights sw,
                                                  const __grid_constant__ CUtensorMap map_x,
                                                  const __grid_constant__ CUtensorMap map_s,
                                                  const __grid_constant__ CUtensorMap map_r,
                                                  const uint32_t* __restrict__ fK, const uint32_t* __restrict__ fR,
                                                  bf16* __restrict__ xdown, bf16* __restrict__ xc, int n,
                                                  const int* __restrict__ active, int* __restrict__ err) {
  down_body<FH, FW, FIRST, HAS_R, RESID>(r, alpha2, ra, sw, map_x, map_s, map_r, fK, fR, xdown, xc, n, active, err,
                                         blockIdx.x, blockIdx.y, blockIdx.z);
}

// TCNN-add on the tensor cores over the quads of Q: each 16 quads are a GEMM
// [16 x 96] x [96 x 8] per fine pixel (r, c) of the quad, whose A row holds the
// quad's four coarse sources (J+dJ, I+dI) as their high BF16 parts (k 0-31) and
// low BF16 parts (k 32-63), gathered by ldmatrix from per-lane addresses, and
// the fine pixel's own x_down (k 64-95, through an identity block: the U-net
// skip of Algorithm 3 added in FP32).  Every quad has the same structure, so
// one set of B fragments serves all of them and both parts (fq, see
// pack_tcnn_frags).  Epilogue: x_pre = hi + lo BF16 (hi into ps, lo into pl on
// the layer-output region O, the layer adds it to its skip) and z = s * x_pre
// from the FP32 sum into zs.  Coarse pixels outside the coarse grid are staged
// as zeros, which makes the sum zero on every fine pixel outside the fine grid.
// Work items: (strip of 16 quads, quad row r), so that the warps' shares differ
// by at most half a strip.
template <class G>
__device__ __forceinline__ void tcnn_quads(uint4* ps, uint4* zs, uint4* pl, const uint4* cs, const uint4* cl,
                                           const uint32_t* fq) {
  constexpr int NQ = G::NQH * G::NQW, NS = (NQ + 15) / 16;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3, kh = lane >> 4;
  const int mrow = (lane & 7) + ((lane >> 3) & 1) * 8;
  const uint32_t fI = identity_frag();
  const uint32_t cs0 = sa(cs), cl0 = sa(cl), ps0 = sa(ps);
  for (int it = warp; it < 2 * NS; it += NW) {
    const int st = it >> 1, r = it & 1;
    // A rows: quad (qr, qc) of this lane's ldmatrix row
    const int qm = min(st * 16 + mrow, NQ - 1), qr = qm / G::NQW, qc = qm - qr * G::NQW;
    uint32_t a0[4], a1[4], b0[4], b1[4], ax[4];
    const uint32_t co = 16u * (qr * G::CQW + qc + kh);
    ldsm_x4(a0, cs0 + co);                             // sources (J, I) | (J, I+1), high parts
    ldsm_x4(a1, cs0 + co + 16u * G::CQW);              // sources (J+1, I) | (J+1, I+1)
    ldsm_x4(b0, cl0 + co);                             // the same, low parts
    ldsm_x4(b1, cl0 + co + 16u * G::CQW);
    ldsm_x4(ax, ps0 + 16u * ((2 * qr + r) * G::QW + 2 * qc + kh));   // x_down of fine (r, 0) | (r, 1)
    // this lane's two output quads (rows g and g + 8 of the strip)
    int pe[2], po[2];
    bool ok[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int qe = st * 16 + g + 8 * h, er = qe / G::NQW, ec = qe - er * G::NQW;
      ok[h] = qe < NQ;
      pe[h] = 2 * er * G::QW + 2 * ec;
      // the quad's first fine pixel in O coordinates (Q pixel (qr, qc) is O pixel
      // (qr - QOFF - 1, qc - QOFF - 1)), packed as row * 65536 + column + offset
      po[h] = (2 * er - G::QOFF - 1 + 2) * 65536 + (2 * ec - G::QOFF - 1 + 2);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      // B fragments of fine pixel t = 2 r + c (selected, so that fq stays in registers)
      uint32_t bw[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) bw[k] = r ? fq[8 + 4 * c + k] : fq[4 * c + k];
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      mma16816(acc, a0, bw[0], bw[1]);
      mma16816(acc, a1, bw[2], bw[3]);
      mma16816(acc, b0, bw[0], bw[1]);
      mma16816(acc, b1, bw[2], bw[3]);
      mma16816(acc, ax, c ? 0u : fI, c ? fI : 0u);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!ok[h]) continue;
        const int e = pe[h] + r * G::QW + c;
        const uint32_t xo = f2bf(acc[2 * h], acc[2 * h + 1]);
        reinterpret_cast<uint32_t*>(&ps[e])[q] = xo;
        uint32_t* zp = reinterpret_cast<uint32_t*>(&zs[e]) + q;
        const float2 hi = bf2_to_f2(xo), sv = bf2_to_f2(*zp);
        *zp = f2bf(sv.x * acc[2 * h], sv.y * acc[2 * h + 1]);
        const int orow = (po[h] >> 16) - 2 + r, ocol = (po[h] & 0xffff) - 2 + c;
        if (orow >= 0 && orow < G::OH && ocol >= 0 && ocol < G::OW)
          reinterpret_cast<uint32_t*>(&pl[orow * G::OW + ocol])[q] = f2bf(acc[2 * h] - hi.x, acc[2 * h + 1] - hi.y);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Up kernel (geometry in UpGeom).  Level l: x_pre = x_down + TCNN(x_{l+1}) on P
// (or x_down on the coarsest level), layer x_fin = x_pre + K_up (s * x_pre) on O;
// finest level: e = W_out * x_fin / alpha, u_out = u_in + e.  The up path
// carries x_pre and x_fin as BF16 hi + lo pairs (about 16 significant bits):
// rounding the coarse-grid correction to BF16 on its way up costs cycles of
// the stationary iteration (37 instead of 30 at 4095^2, measured by emulating
// the roundings); a level's x_fin goes to the next finer level as xfin (hi)
// and xfin_lo (lo), which that level's TCNN reads through map_c and map_cl.
// The up kernel's work on the tile (tbx, tby) of problem tbz (one block).
template <int FH, int FW, bool LAST, bool HAS_P, bool RES>
__device__ __forceinline__ void up_body(const CUtensorMap& map_xd, const CUtensorMap& map_s, const CUtensorMap& map_c,
                                        const CUtensorMap& map_cl, const uint32_t* __restrict__ fK,
                                        const uint32_t* __restrict__ fTc, const uint32_t* __restrict__ fOutTaps,
                                        const float* __restrict__ alpha2, const double* __restrict__ u_in,
                                        bf16* __restrict__ xfin, bf16* __restrict__ xfin_lo,
                                        double* __restrict__ u_out, int n, const int* __restrict__ active,
                                        int* __restrict__ err, const ResidOut& ro, int out_lo, int tbx, int tby,
                                        int tbz) {
  using G = UpGeom<FH, FW, LAST, HAS_P, RES>;
  constexpr int H = G::H, OH = G::OH, OW = G::OW, QW = G::QW, QOFF = G::QOFF;
  constexpr int HE = G::HE, EH = G::EH, EW = G::EW;
  // TMA destinations (zero outside the grid): ps = x_down on Q, then x_pre's
  // high BF16 part; zs = s on Q, then s * x_pre; cs, cl = the quads' coarse
  // pixels (high, low parts).  pl = the low part of x_pre on O; on the finest
  // level the layer output's parts then replace x_pre's in ps and pl, and W_out's
  // per-tap planes use zs, cs and cl (contiguous)
  uint4* ps = reinterpret_cast<uint4*>(fused_dsm);
  uint4* pl = ps + pad8(G::QH * QW);
  uint4* zs = pl + pad8(OH * OW);
  uint4* cs = zs + pad8(G::QH * QW);                                   // coarser level only
  uint4* cl = cs + pad8(G::CQH * G::CQW);
  __shared__ __align__(8) uint64_t bar;
  const int j0 = tby * FH, i0 = tbx * FW;
  const int qj0 = j0 - H - 1 - QOFF, qi0 = i0 - H - 1 - QOFF;         // Q's corner (odd when HAS_P)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bz = tbz;
  {
    const size_t N = (size_t)n * n;
    if (LAST) {
      if (u_in) u_in += bz * N;
      u_out += bz * N;
    } else {
      xfin += bz * N * 8;
      xfin_lo += bz * N * 8;
    }
  }
  // weight fragments of the TCNN and of the layer, loaded before the tiles land
  uint32_t fq[kTcnnQuadRegs], wk[9];
#pragma unroll
  for (int k = 0; k < kTcnnQuadRegs; ++k) fq[k] = HAS_P ? fTc[k * 32 + lane] : 0u;
#pragma unroll
  for (int k = 0; k < 9; ++k) wk[k] = fK[k * 32 + lane];
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  pdl_wait();
  if (active && !active[bz]) return;
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, (2u * G::QH * QW + (HAS_P ? 2u * G::CQH * G::CQW : 0u)) * 16u);
    tma_load_pix(ps, &map_xd, qi0, qj0, bz, &bar);
    tma_load_pix(zs, &map_s, qi0, qj0, bz, &bar);
    // the first quad's coarse source: J = (qj0 - 1) / 2 (exact, qj0 odd)
    if (HAS_P) {
      tma_load_pix(cs, &map_c, (qi0 - 1) / 2, (qj0 - 1) / 2, bz, &bar);
      tma_load_pix(cl, &map_cl, (qi0 - 1) / 2, (qj0 - 1) / 2, bz, &bar);
    }
  }
  __syncthreads();   // barrier initialised
  const bool landed = mbar_wait_bounded(&bar, 0);
  if (!__syncthreads_and(landed)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }

  if constexpr (HAS_P) {
    tcnn_quads<G>(ps, zs, pl, cs, cl, fq);
  } else {
    for (int e = threadIdx.x; e < G::QH * QW; e += NT) zs[e] = mul8(ps[e], zs[e]);
    for (int e = threadIdx.x; e < OH * OW; e += NT) pl[e] = make_uint4(0u, 0u, 0u, 0u);   // x_pre = x_down
  }
  __syncthreads();

  // layer on O: strips of 16 pixels of O in row-major order (a strip may wrap
  // to the next row); O pixel (orow, ocol) reads the taps around Q pixel
  // (orow + QOFF + 1, ocol + QOFF + 1).  (Strips at the Q tile's pitch, free of
  // the wrap's bank conflicts, cost more in the extra pixels than they save.)
  const int g = lane >> 2, q = lane & 3;
  {
    constexpr int NO = OH * OW, NSTRIP = (NO + 15) / 16;
    const int mrow = (lane & 7) + ((lane >> 3) & 1) * 8;
    const TapOffsets<QW> to;
    const uint32_t fI = identity_frag();
    for (int st = warp; st < NSTRIP; st += NW) {
      const int pm = min(st * 16 + mrow, NO - 1), rm = pm / OW;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      layer_strip<QW>(zs, ps, wk, fI, (rm + QOFF) * QW + (pm - rm * OW) + QOFF, to, acc);
      {
        // the skip's low part: x_lo at the pixel itself through an identity block
        uint32_t a[2];
        ldsm_x2(a, sa(pl) + 16u * min(st * 16 + (lane & 15), NO - 1));
        mma1688(acc, a[0], a[1], fI);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = st * 16 + g + 8 * h;
        if (p >= NO) continue;
        const int orow = p / OW, ocol = p - orow * OW;
        const uint32_t o = f2bf(acc[2 * h], acc[2 * h + 1]);
        const int gj = j0 - H + orow, gi = i0 - H + ocol;
        if constexpr (LAST) {
          // the output as hi + lo BF16, zero outside the grid (W_out's zero
          // padding), in place: only this strip reads these pixels of ps and pl
          const bool in = gj >= 0 && gj < n && gi >= 0 && gi < n;
          const float2 hi = bf2_to_f2(o);
          reinterpret_cast<uint32_t*>(&ps[(orow + QOFF + 1) * QW + ocol + QOFF + 1])[q] = in ? o : 0u;
          reinterpret_cast<uint32_t*>(&pl[p])[q] = in ? f2bf(acc[2 * h] - hi.x, acc[2 * h + 1] - hi.y) : 0u;
        } else if (gj < n && gi < n) {
          // x_fin to the next finer level as hi + lo BF16
          const float2 hi = bf2_to_f2(o);
          const size_t gp = ((size_t)gj * n + gi) * 8;
          reinterpret_cast<uint32_t*>(xfin + gp)[q] = o;
          reinterpret_cast<uint32_t*>(xfin_lo + gp)[q] = f2bf(acc[2 * h] - hi.x, acc[2 * h + 1] - hi.y);
        }
      }
    }
  }
  if constexpr (LAST) {
    // W_out (Eq. reCh-out: 8 channels -> 1) tap by tap.  Every O pixel's layer
    // output y (hi + lo BF16 in ps and pl) meets the tap weights once, in one
    // K = 16 MMA per 16 pixels: D_t(o) = sum_ch (hi + lo)(y(o))[ch] w_t[ch]
    // (w split as hi + lo BF16 too: the products hi(w) hi(y) + hi(w) lo(y) +
    // lo(w) hi(y), about 16 bits on each side, summed in FP32), written to
    // per-tap planes in shared memory; then e(E pixel) = sum over taps t = 0..8
    // of D_t at the pixel's tap t, in that order, in FP32.  E pixel (er, ec)
    // is O pixel (er + 1, ec + 1); tap (a, b) reads O pixel (er + a, ec + b).
    // The planes take PASS taps at a time (PASS = 6 where zs and cs hold six
    // planes, else 3), in consecutive passes.
    uint32_t bt[kOutTapRegs];
#pragma unroll
    for (int k = 0; k < kOutTapRegs; ++k) bt[k] = fOutTaps[k * 32 + lane];
    // E pixels of this thread: with rows of 17..32 pixels, E row er = warp + NW k
    // to one warp (lane = column), so that a warp's reads of a tap plane are one
    // row, consecutive words, free of bank conflicts; else consecutive pixels
    constexpr int NE = EH * EW;
    constexpr bool ROWS = EW > 16 && EW <= 32;
    constexpr int NU = ROWS ? (EH + NW - 1) / NW : (NE + NT - 1) / NT;
    auto epix = [&](int k, int& er, int& ec) -> bool {
      if constexpr (ROWS) {
        er = warp + NW * k;
        ec = lane;
        return er < EH && ec < EW;
      } else {
        const int e = threadIdx.x + k * NT;
        er = e / EW;
        ec = e - er * EW;
        return e < NE;
      }
    };
    // this thread's u values of the update below, loaded now so that their
    // latency passes during W_out (zero outside the grid)
    double uv[NU];
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      int er, ec;
      const bool valid = epix(k, er, ec);
      const int gj = j0 - HE + er, gi = i0 - HE + ec;
      uv[k] = (u_in && valid && gj >= 0 && gj < n && gi >= 0 && gi < n) ? u_in[(size_t)gj * n + gi] : 0.0;
    }
    constexpr int NO = OH * OW, NSO = (NO + 15) / 16;
    constexpr int PL = (NO + 27) / 32 * 32 + 4;    // plane pitch (floats), 4 (mod 32): conflict-free stores
    constexpr int FREE = 16 * (pad8(G::QH * QW) + (HAS_P ? 2 * pad8(G::CQH * G::CQW) : 0));
    constexpr int PASS = 6 * PL * 4 <= FREE ? 6 : 3;
    static_assert(PASS * PL * 4 <= FREE, "W_out planes in the z and coarse tiles");
    float* dpl = reinterpret_cast<float*>(zs);
    float esum[NU];
#pragma unroll
    for (int k = 0; k < NU; ++k) esum[k] = 0.f;
    __syncthreads();   // the layer's y is complete; z and the coarse tile are free
#pragma unroll
    for (int t0 = 0; t0 < 9; t0 += PASS) {
      // B tile of this pass: taps 6 b .. 6 b + 5 in columns n = tap - 6 b
      const int b = t0 / 6, base = 6 * b;
      for (int st = warp; st < NSO; st += NW) {
        // A rows: 16 O pixels; lanes 0-15 address hi(y) in ps, 16-31 lo(y) in pl
        const int pr = min(st * 16 + (lane & 15), NO - 1), orr = pr / OW, oc = pr - orr * OW;
        uint32_t a[4];
        ldsm_x4(a, lane < 16 ? sa(ps) + 16u * ((orr + QOFF + 1) * QW + oc + QOFF + 1) : sa(pl) + 16u * pr);
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(d, a, bt[4 * b + 0], bt[4 * b + 1]);
        if (out_lo) mma16816(d, a, bt[4 * b + 2], bt[4 * b + 3]);   // a zero lo part adds exactly nothing
        // lane (g, q): taps base + 2q, base + 2q + 1 of pixels g and g + 8 of the strip
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int p = st * 16 + g + 8 * h;
          if (p >= NO) continue;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int tp = base + 2 * q + j - t0;   // plane of this tap in the pass
            if (tp >= 0 && tp < PASS && t0 + tp < 9) dpl[tp * PL + p] = d[2 * h + j];
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < NU; ++k) {
        int er, ec;
        if (!epix(k, er, ec)) continue;
#pragma unroll
        for (int tp = 0; tp < PASS && t0 + tp < 9; ++tp) {
          const int t = t0 + tp;
          esum[k] += dpl[tp * PL + (er + t / 3) * OW + ec + t % 3];
        }
      }
      __syncthreads();   // the next pass (or the u + e staging) overwrites the planes
    }
    const float inv_alpha = alpha2[2 * bz + 1];
    double* un = reinterpret_cast<double*>(zs);    // u + e on E (residual in this kernel)
#pragma unroll
    for (int k = 0; k < NU; ++k) {
      int er, ec;
      if (!epix(k, er, ec)) continue;
      const int gj = j0 - HE + er, gi = i0 - HE + ec;
      const bool in = gj >= 0 && gj < n && gi >= 0 && gi < n;
      const double un_e = in ? uv[k] + f32_to_f64_exact(esum[k] * inv_alpha) : 0.0;
      if (RES) un[er * EW + ec] = un_e;
      if (in && er >= HE && er < HE + FH && ec >= HE && ec < HE + FW) u_out[(size_t)gj * n + gi] = un_e;
    }
    if constexpr (RES) {
      // the next cycle's residual on the owned pixels: r = f - A u (FP64, Eq. 1)
      // with the same five FMAs, in the same order, as the stand-alone residual
      // kernel, from u + e of this block (its halo pixels hold the same bits as
      // the neighbouring blocks' owned pixels: every pixel's e is the same
      // instruction sequence on the same data); the FP32 copy of D^{-1} r for
      // the next cycle and the block's partial sum of r^2
      __syncthreads();
      const size_t N = (size_t)n * n;
      double rr2 = 0.0;
      const int pitch = r32_pitch(n);
      for (int e = threadIdx.x; e < FH * FW; e += NT) {
        const int rr = e / FW, cc = e - rr * FW;
        const int gj = j0 + rr, gi = i0 + cc;
        if (gj >= n || gi >= n) continue;
        const size_t p = (size_t)gj * n + gi;
        const double* uc = un + (rr + 1) * EW + cc + 1;
        double rv = fma(-ro.op[p], uc[0], ro.f[p]);
        rv = fma(-ro.op[N + p], uc[-1], rv);
        rv = fma(-ro.op[2 * N + p], uc[1], rv);
        rv = fma(-ro.op[3 * N + p], uc[-EW], rv);
        rv = fma(-ro.op[4 * N + p], uc[EW], rv);
        rr2 = fma(rv, rv, rr2);
        const float rf = f64_to_f32_rn(rv);
        ro.r32[(size_t)gj * pitch + gi] = ro.dinv32 ? rf * ro.dinv32[p] : rf;
      }
      __shared__ double red[NW];
      rr2 = block_sum_fixed(rr2, red);
      if (threadIdx.x == 0) ro.partial[blockIdx.y * gridDim.x + blockIdx.x] = rr2;
    }
  }
  pdl_trigger();
}

template <int FH, int FW, bool LAST, bool HAS_P, bool RES>
__global__ void __launch_bounds__(NT, 4) up_kernel(const __grid_constant__ CUtensorMap map_xd,
                                                const __grid_constant__ CUtensorMap map_s,
                                                const __grid_constant__ CUtensorMap map_c,
                                                const __grid_constant__ CUtensorMap map_cl,
                                                const uint32_t* __restrict__ fK, const uint32_t* __restrict__ fTc,
                                                const uint32_t* __restrict__ fOutTaps,
                                                const float* __restrict__ alpha2, const double* __restrict__ u_in,
                                                bf16* __restrict__ xfin, bf16* __restrict__ xfin_lo,
                                                double* __restrict__ u_out, int n, const int* __restrict__ active,
                                                int* __restrict__ err, const __grid_constant__ ResidOut ro,
                                                int out_lo) {
  up_body<FH, FW, LAST, HAS_P, RES>(map_xd, map_s, map_c, map_cl, fK, fTc, fOutTaps, alpha2, u_in, xfin, xfin_lo,
                                    u_out, n, active, err, ro, out_lo, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// The coarse tail of the cycle in one launch.  From level `lt` down (grids of
// at most kTailMaxN points per side) every level's kernel is a few blocks whose
// cost is launch and ramp time, so one cooperative kernel runs them all: the
// blocks take the tiles of level lt's down step, then of level lt+1, ... the
// coarsest, then the up steps back to lt, a grid-wide barrier between the
// levels.  Same tile bodies (16 x 32 tiles), same arithmetic per pixel.
constexpr int kTailFH = 16, kTailFW = 32, kTailMaxN = 255, kTailMaxLevels = 8;
struct TailLevel {
  CUtensorMap dx, ds;              // down: the level's input x (box of Z), s (box of Z)
  CUtensorMap ux, us, uc, ucl;     // up: x_down, s (boxes of Q), the coarser level's x hi, lo (coarse box)
  bf16 *xa, *xb, *xbl, *xc;        // x_down, x (input, then output of the up step: hi), its lo, coarser level's x
  int n, tx, ty;                   // grid side, tiles per row / column
};
struct TailArgs {
  TailLevel lv[kTailMaxLevels];
  int nl, batch;
  const uint32_t *f_down, *f_R, *f_up, *f_tcnn;
  const int* active;
  int* err;
  unsigned* bar;                   // [0] arrivals, [1] generation (zero when idle)
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of the tail (all blocks resident: cooperative launch).  The
// block's global writes are made visible to the other blocks, TMA loads
// included; the wait is bounded (false and the error flag past the limit).
__device__ __forceinline__ bool tail_sync(unsigned* bar, int* err) {
  // the block's writes are ordered before thread 0's release by the CTA barrier
  // and the cumulative fence that follows it
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned gen = ld_acquire(bar + 1);
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);   // the last arrival resets the count, then opens the next generation
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      ok = 0;
      for (int i = 0; i < (1 << 21) && !ok; ++i)   // about a second of L2 round trips
        if (ld_acquire(bar + 1) != gen) ok = 1;
      if (!ok) atomicExch(err, 1);
    }
    __threadfence();
    asm volatile("fence.proxy.async.global;" ::: "memory");   // the TMA loads this thread issues next
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__global__ void __launch_bounds__(NT, 4) tail_kernel(const __grid_constant__ TailArgs ta) {
  const ResidIn no_ra{};
  const ResidOut no_ro{};
  const SmallWeights no_sw{};
  for (int k = 0; k < ta.nl; ++k) {
    const TailLevel& L = ta.lv[k];
    const int per = L.tx * L.ty, tiles = per * ta.batch;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int bz = t / per, tl = t - bz * per, ty = tl / L.tx, tx = tl - ty * L.tx;
      if (k + 1 < ta.nl)
        down_body<kTailFH, kTailFW, false, true, false>(nullptr, nullptr, no_ra, no_sw, L.dx, L.ds, L.ds, ta.f_down,
                                                        ta.f_R, L.xa, L.xc, L.n, ta.active, ta.err, tx, ty, bz);
      else
        down_body<kTailFH, kTailFW, false, false, false>(nullptr, nullptr, no_ra, no_sw, L.dx, L.ds, L.ds, ta.f_down,
                                                         ta.f_R, L.xa, nullptr, L.n, ta.active, ta.err, tx, ty, bz);
      // the next tile's copies overwrite the shared tiles this one read and wrote
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
    }
    if (!tail_sync(ta.bar, ta.err)) return;
  }
  for (int k = ta.nl - 1; k >= 0; --k) {
    const TailLevel& L = ta.lv[k];
    const int per = L.tx * L.ty, tiles = per * ta.batch;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int bz = t / per, tl = t - bz * per, ty = tl / L.tx, tx = tl - ty * L.tx;
      if (k + 1 < ta.nl)
        up_body<kTailFH, kTailFW, false, true, false>(L.ux, L.us, L.uc, L.ucl, ta.f_up, ta.f_tcnn, nullptr, nullptr,
                                                      nullptr, L.xb, L.xbl, nullptr, L.n, ta.active, ta.err, no_ro, 0,
                                                      tx, ty, bz);
      else
        up_body<kTailFH, kTailFW, false, false, false>(L.ux, L.us, L.us, L.us, ta.f_up, ta.f_tcnn, nullptr,
                                                       nullptr, nullptr, L.xb, L.xbl, nullptr, L.n, ta.active, ta.err,
                                                       no_ro, 0, tx, ty, bz);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
    }
    if (k > 0 && !tail_sync(ta.bar, ta.err)) return;
  }
}

// Dynamic shared memory of a kernel instantiation: above 48 KB the kernel must be
// allowed it once per device (cudaFuncSetAttribute); the (device, kernel) pairs
// already allowed are remembered, under a lock (contexts may live in different
// threads).  Returns the byte count for the launch; a refused attribute shows
// up as the launch's error.
size_t dyn_smem_allow(const void* kernel, size_t bytes) {
  static std::mutex lock;
  static std::vector<std::pair<int, const void*>> allowed;
  if (bytes <= 48 * 1024) return bytes;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bytes;
  std::lock_guard<std::mutex> g(lock);
  const std::pair<int, const void*> key{dev, kernel};
  if (std::find(allowed.begin(), allowed.end(), key) == allowed.end() &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
    allowed.push_back(key);
  return bytes;
}

template <typename K>
size_t dyn_smem(K* kernel, size_t bytes) {
  return dyn_smem_allow(reinterpret_cast<const void*>(kernel), bytes);
}

// Launch of a level kernel; with `pdl` the launch may begin while the previous
// kernel in the stream finishes (programmatic stream serialisation: the kernel
// waits for it in pdl_wait before touching its output).
template <typename... KArgs, typename... Args>
cudaError_t launch_level(void (*kernel)(KArgs...), dim3 grid, size_t smem, cudaStream_t st, bool pdl,
                         Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Tensor map of a level tensor for a box of bw x bh pixels (copied out of the
// cache at once: a later lookup may move the cache's storage).
Status pix8_map(const FusedLevels& fl, const void* base, int n, int bw, int bh, CUtensorMap* out) {
  const CUtensorMap* m = fl.maps ? fl.maps->pix8(base, n, fl.batch, bw, bh) : nullptr;
  if (!m) return make_status(MGCNN_ERR_CUDA, "cannot encode a TMA tensor map (n %d, box %d x %d)", n, bw, bh);
  *out = *m;
  return {};
}

// Tile variants (FH x FW): 0 = 16 x 32, 1 = 8 x 32, 2 = 16 x 16, 3 = 32 x 32,
// 4 = 24 x 32.  FH must be even and (FH / 2) x (FW / 2) a multiple of 16 (the
// restriction's strips of 16 coarse pixels).
template <int FH, int FW>
Status launch_down(int l, const FusedLevels& fl, const float* r32, const double* norm2, const FusedWeights& w,
                   const int* active, cudaStream_t st, const ResidIn* ra) {
  const int nl = fl.n[l];
  const bool first = l == 0, has_r = l + 1 < fl.L;
  if (ra && (!first || fl.batch != 1)) return make_status(MGCNN_ERR_STATE, "fused residual: finest level, one problem");
  const dim3 grid((nl + FW - 1) / FW, (nl + FH - 1) / FH, fl.batch);
  __nv_bfloat16* xc = has_r ? fl.xb[l + 1] : nullptr;
  const int R = has_r ? 1 : 0, ZH = FH + R + 2, ZW = FW + R + 2;
  CUtensorMap ms, mx;
  MG_TRY(pix8_map(fl, fl.s[l], nl, ZW, ZH, &ms));
  if (first)
    mx = ms;   // not read on the finest level
  else
    MG_TRY(pix8_map(fl, fl.xb[l], nl, ZW, ZH, &mx));
  const ResidIn rin = ra ? *ra : ResidIn{};
  CUtensorMap mr = ms;   // not read unless the finest level stages r32 by TMA
  if (first && !ra) {
    const int RH = FH + R + 4, RWT = has_r ? down_rwt<FW, true>() : down_rwt<FW, false>();
    const CUtensorMap* m = fl.maps ? fl.maps->f32(r32, nl, r32_pitch(nl), fl.batch, RWT, RH) : nullptr;
    if (!m) return make_status(MGCNN_ERR_CUDA, "cannot encode the residual's TMA tensor map (n %d)", nl);
    mr = *m;
  }
  cudaError_t le = cudaSuccess;
  auto run = [&](auto* kernel, size_t smem) {
    le = launch_level(kernel, grid, dyn_smem(kernel, smem), st, fl.pdl, r32, (const float*)fl.alpha, rin, w.small, mx,
                      ms, mr, w.f_down, w.f_R, fl.xa[l], xc, nl, active, fl.err);
  };
  if (ra && has_r)
    run(down_kernel<FH, FW, true, true, true>, down_smem_bytes<FH, FW, true, true>());
  else if (ra)
    run(down_kernel<FH, FW, true, false, true>, down_smem_bytes<FH, FW, true, false>());
  else if (first && has_r)
    run(down_kernel<FH, FW, true, true, false>, down_smem_bytes<FH, FW, true, true>());
  else if (first)
    run(down_kernel<FH, FW, true, false, false>, down_smem_bytes<FH, FW, true, false>());
  else if (has_r)
    run(down_kernel<FH, FW, false, true, false>, down_smem_bytes<FH, FW, false, true>());
  else
    run(down_kernel<FH, FW, false, false, false>, down_smem_bytes<FH, FW, false, false>());
  if (le != cudaSuccess) return cuda_status(le, "down_kernel launch");
  MG_LAUNCH("down_kernel");
  return {};
}

template <int FH, int FW>
Status launch_up(int l, const FusedLevels& fl, const double* norm2, double* e, const double* u_skip,
                 const FusedWeights& w, const int* active, cudaStream_t st, const ResidOut* ro) {
  const int nl = fl.n[l];
  const bool last = l == 0, has_p = l + 1 < fl.L;
  if (ro && (!last || fl.batch != 1)) return make_status(MGCNN_ERR_STATE, "fused residual: finest level, one problem");
  const dim3 grid((nl + FW - 1) / FW, (nl + FH - 1) / FH, fl.batch);
  const ResidOut rout = ro ? *ro : ResidOut{};
  if (!last && !fl.xbl[l]) return make_status(MGCNN_ERR_STATE, "level %d: no buffer for the low part of x_fin", l);
  if (has_p && !fl.xbl[l + 1]) return make_status(MGCNN_ERR_STATE, "level %d: no low part of x_fin", l + 1);
  auto run = [&](auto* kernel, size_t smem, bf16* xfin, auto geom) -> Status {
    using G = decltype(geom);
    CUtensorMap mxd, ms, mc, mcl;
    MG_TRY(pix8_map(fl, fl.xa[l], nl, G::QW, G::QH, &mxd));
    MG_TRY(pix8_map(fl, fl.s[l], nl, G::QW, G::QH, &ms));
    if (has_p) {
      MG_TRY(pix8_map(fl, fl.xb[l + 1], fl.n[l + 1], G::CQW, G::CQH, &mc));
      MG_TRY(pix8_map(fl, fl.xbl[l + 1], fl.n[l + 1], G::CQW, G::CQH, &mcl));
    } else {
      mc = mcl = ms;   // not read on the coarsest level
    }
    bf16* xfin_lo = last ? nullptr : fl.xbl[l];
    const cudaError_t le = launch_level(kernel, grid, dyn_smem(kernel, smem), st, fl.pdl, mxd, ms, mc, mcl, w.f_up,
                                        w.f_tcnn, w.f_out_taps, (const float*)fl.alpha, u_skip, xfin, xfin_lo, e,
                                        nl, active, fl.err, rout, w.out_lo);
    if (le != cudaSuccess) return cuda_status(le, "up_kernel launch");
    return {};
  };
  if (ro && has_p)
    MG_TRY(run(up_kernel<FH, FW, true, true, true>, up_smem_bytes<FH, FW, true, true, true>(), nullptr,
               UpGeom<FH, FW, true, true, true>{}));
  else if (ro)
    MG_TRY(run(up_kernel<FH, FW, true, false, true>, up_smem_bytes<FH, FW, true, false, true>(), nullptr,
               UpGeom<FH, FW, true, false, true>{}));
  else if (last && has_p)
    MG_TRY(run(up_kernel<FH, FW, true, true, false>, up_smem_bytes<FH, FW, true, true>(), nullptr,
               UpGeom<FH, FW, true, true>{}));
  else if (last)
    MG_TRY(run(up_kernel<FH, FW, true, false, false>, up_smem_bytes<FH, FW, true, false>(), nullptr,
               UpGeom<FH, FW, true, false>{}));
  else if (has_p)
    MG_TRY(run(up_kernel<FH, FW, false, true, false>, up_smem_bytes<FH, FW, false, true>(), fl.xb[l],
               UpGeom<FH, FW, false, true>{}));
  else
    MG_TRY(run(up_kernel<FH, FW, false, false, false>, up_smem_bytes<FH, FW, false, false>(), fl.xb[l],
               UpGeom<FH, FW, false, false>{}));
  MG_LAUNCH("up_kernel");
  return {};
}

int tail_capacity();

// The coarse tail (tail_kernel): the levels from `lt` to the coarsest in one
// cooperative launch, when at least two levels qualify (grid side at most
// fl.tail_n and kTailMaxN, level 1 or coarser, at most kTailMaxLevels levels).
int tail_start(const FusedLevels& fl) {
  if (fl.tail_n <= 0 || !fl.tail_bar || tail_capacity() <= 0) return fl.L;
  int lt = fl.L;
  for (int l = fl.L - 1; l >= 1 && fl.n[l] <= std::min(fl.tail_n, kTailMaxN) && fl.L - l <= kTailMaxLevels; --l)
    lt = l;
  return fl.L - lt >= 2 ? lt : fl.L;
}

constexpr size_t tail_smem_bytes() {
  return std::max(std::max(down_smem_bytes<kTailFH, kTailFW, false, true>(),
                           down_smem_bytes<kTailFH, kTailFW, false, false>()),
                  std::max(up_smem_bytes<kTailFH, kTailFW, false, true>(),
                           up_smem_bytes<kTailFH, kTailFW, false, false>()));
}

// Blocks of the tail kernel that fit on the device at once (0: no cooperative
// launch), once per device.
int tail_capacity() {
  static std::mutex lock;
  static std::vector<std::pair<int, int>> known;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> g(lock);
  for (const auto& k : known)
    if (k.first == dev) return k.second;
  int coop = 0, sms = 0, per_sm = 0;
  const size_t smem = dyn_smem(tail_kernel, tail_smem_bytes());
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tail_kernel, NT, smem) != cudaSuccess) {
    cudaGetLastError();
    coop = 0;
  }
  const int cap = coop ? per_sm * sms : 0;
  known.emplace_back(dev, cap);
  return cap;
}

template <bool HAS_R, bool HAS_P>
Status tail_level_maps(const FusedLevels& fl, int l, TailLevel* t) {
  using G = UpGeom<kTailFH, kTailFW, false, HAS_P>;
  const int n = fl.n[l], R = HAS_R ? 1 : 0, ZH = kTailFH + R + 2, ZW = kTailFW + R + 2;
  MG_TRY(pix8_map(fl, fl.xb[l], n, ZW, ZH, &t->dx));
  MG_TRY(pix8_map(fl, fl.s[l], n, ZW, ZH, &t->ds));
  MG_TRY(pix8_map(fl, fl.xa[l], n, G::QW, G::QH, &t->ux));
  MG_TRY(pix8_map(fl, fl.s[l], n, G::QW, G::QH, &t->us));
  if (HAS_P) {
    MG_TRY(pix8_map(fl, fl.xb[l + 1], fl.n[l + 1], G::CQW, G::CQH, &t->uc));
    MG_TRY(pix8_map(fl, fl.xbl[l + 1], fl.n[l + 1], G::CQW, G::CQH, &t->ucl));
  } else {
    t->uc = t->ucl = t->us;   // not read on the coarsest level
  }
  return {};
}

// Levels lt .. L-1 down and back up in one cooperative launch.  Returns
// MGCNN_ERR_CUDA (launch refused) without side effects on the level state.
Status launch_tail(const FusedLevels& fl, int lt, const FusedWeights& w, const int* active, cudaStream_t st) {
  const int cap = tail_capacity();
  if (cap <= 0) return make_status(MGCNN_ERR_CUDA, "no cooperative launch on this device");
  TailArgs ta{};
  ta.nl = fl.L - lt;
  ta.batch = fl.batch;
  ta.f_down = w.f_down;
  ta.f_R = w.f_R;
  ta.f_up = w.f_up;
  ta.f_tcnn = w.f_tcnn;
  ta.active = active;
  ta.err = fl.err;
  ta.bar = fl.tail_bar;
  int tiles = 0;
  for (int k = 0; k < ta.nl; ++k) {
    const int l = lt + k;
    TailLevel& t = ta.lv[k];
    if (l + 1 < fl.L)
      MG_TRY((tail_level_maps<true, true>(fl, l, &t)));
    else
      MG_TRY((tail_level_maps<false, false>(fl, l, &t)));
    t.xa = fl.xa[l];
    t.xb = fl.xb[l];
    t.xbl = fl.xbl[l];
    t.xc = l + 1 < fl.L ? fl.xb[l + 1] : nullptr;
    t.n = fl.n[l];
    t.tx = (t.n + kTailFW - 1) / kTailFW;
    t.ty = (t.n + kTailFH - 1) / kTailFH;
    tiles = std::max(tiles, t.tx * t.ty * fl.batch);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::max(1, std::min(tiles, cap / std::max(1, fl.tail_share))));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = dyn_smem(tail_kernel, tail_smem_bytes());
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t le = cudaLaunchKernelEx(&cfg, tail_kernel, ta);
  if (le != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(le, "tail_kernel launch");
  }
  return {};
}

constexpr int kTileH[kUpVariants] = {16, 8, 16, 32, 24, 24, 32, 22};
constexpr int kTileW[kUpVariants] = {32, 32, 16, 32, 32, 30, 30, 30};

Status launch_down_variant(int v, int l, const FusedLevels& fl, const float* r32, const double* norm2,
                           const FusedWeights& w, const int* active, cudaStream_t st, const ResidIn* ra = nullptr) {
  switch (v) {
    case 1: return launch_down<8, 32>(l, fl, r32, norm2, w, active, st, ra);
    case 2: return launch_down<16, 16>(l, fl, r32, norm2, w, active, st, ra);
    case 3: return launch_down<32, 32>(l, fl, r32, norm2, w, active, st, ra);
    case 4: return launch_down<24, 32>(l, fl, r32, norm2, w, active, st, ra);
    default: return launch_down<16, 32>(l, fl, r32, norm2, w, active, st, ra);
  }
}

Status launch_up_variant(int v, int l, const FusedLevels& fl, const double* norm2, double* e, const double* u_skip,
                         const FusedWeights& w, const int* active, cudaStream_t st, const ResidOut* ro = nullptr) {
  switch (v) {
    case 1: return launch_up<8, 32>(l, fl, norm2, e, u_skip, w, active, st, ro);
    case 2: return launch_up<16, 16>(l, fl, norm2, e, u_skip, w, active, st, ro);
    case 3: return launch_up<32, 32>(l, fl, norm2, e, u_skip, w, active, st, ro);
    case 4: return launch_up<24, 32>(l, fl, norm2, e, u_skip, w, active, st, ro);
    // up kernel only (the restriction needs (FH / 2) (FW / 2) a multiple of 16):
    // on the finest level the layer output is 32 pixels wide, whole strips of 16
    case 5: return launch_up<24, 30>(l, fl, norm2, e, u_skip, w, active, st, ro);
    case 6: return launch_up<32, 30>(l, fl, norm2, e, u_skip, w, active, st, ro);
    case 7: return launch_up<22, 30>(l, fl, norm2, e, u_skip, w, active, st, ro);
    default: return launch_up<16, 32>(l, fl, norm2, e, u_skip, w, active, st, ro);
  }
}

}  // namespace

// One V-cycle with the fused level kernels (CP = 8) for a batch of `batch`
// equal-size problems stored back to back: level l state in xa[l] (down state)
// and xb[l] (restricted input, then final up state), setup tensors s[l];
// r32/norm2/u/e per problem.  `active` (nullable, [batch]) skips converged
// problems.  fl.var_down / fl.var_up pick each level's tile variant.  With
// opt.after_fused_down0 the finest down kernel has already run (it computed the
// residual itself) and the input scale was set before it: the cycle continues
// from level 1 and leaves the scale alone.
Status fused_vcycle_levels(const FusedLevels& fl, const float* r32, const double* norm2, double* e,
                           const double* u_skip, const FusedWeights& w, const int* active, cudaStream_t st,
                           mgcnn_ctx* prof_ctx, FusedCycleOpt opt) {
  const int L = fl.L, lt = tail_start(fl);
  if (!opt.after_fused_down0) MG_TRY(launch_alpha(fl, norm2, st));
  for (int l = opt.after_fused_down0 ? 1 : 0; l < lt; ++l) {
    const int ps = prof_ctx ? prof_begin(prof_ctx, l == 0 ? kProfDown0 : kProfDownLevel + l) : -1;
    MG_TRY(launch_down_variant(fl.var_down[l], l, fl, r32, norm2, w, active, st));
    if (prof_ctx) prof_end(prof_ctx, ps);
  }
  if (lt < L) {
    const int ps = prof_ctx ? prof_begin(prof_ctx, kProfTail) : -1;
    MG_TRY(launch_tail(fl, lt, w, active, st));
    MG_LAUNCH("tail_kernel");
    if (prof_ctx) prof_end(prof_ctx, ps);
  }
  for (int l = lt - 1; l >= 0; --l) {
    const int ps = prof_ctx ? prof_begin(prof_ctx, l == 0 ? kProfUp0 : kProfUpLevel + l) : -1;
    MG_TRY(launch_up_variant(fl.var_up[l], l, fl, norm2, e, u_skip, w, active, st, l == 0 ? opt.resid_out : nullptr));
    if (prof_ctx) prof_end(prof_ctx, ps);
  }
  return {};
}

Status fused_down0_resid(const FusedLevels& fl, const ResidIn& ra, const FusedWeights& w, const int* active,
                         cudaStream_t st, mgcnn_ctx* prof_ctx) {
  const int ps = prof_ctx ? prof_begin(prof_ctx, kProfDown0) : -1;
  MG_TRY(launch_down_variant(fl.var_down[0], 0, fl, nullptr, nullptr, w, active, st, &ra));
  if (prof_ctx) prof_end(prof_ctx, ps);
  return {};
}

Status fused_set_alpha(const FusedLevels& fl, const double* norm2, cudaStream_t st) { return launch_alpha(fl, norm2, st); }

int fused_down0_blocks(int n, int variant) {
  return ((n + kTileW[variant] - 1) / kTileW[variant]) * ((n + kTileH[variant] - 1) / kTileH[variant]);
}

size_t fused_partials_max(int n) {
  size_t m = 0;
  for (int v = 0; v < kUpVariants; ++v) m = std::max(m, (size_t)fused_down0_blocks(n, v));
  return m;
}

// Autotuner: for every level, time each tile variant of the down and up kernels
// (CUDA events, `reps` launches after one warm-up launch) on the real buffers
// and keep the fastest.  The up kernel of the finest level writes its FP64
// output to `scratch` (n_0^2 x batch doubles) so that no caller data changes.
// With `ra` the finest down kernel is timed as it runs in the cycle, computing
// the residual (its partial sums go to ra->partial).
Status fused_autotune(FusedLevels& fl, const float* r32, const double* norm2, double* scratch,
                      const FusedWeights& w, cudaStream_t st, int reps, const ResidIn* ra, const ResidOut* ro) {
  cudaEvent_t e0, e1;
  MG_CUDA(cudaEventCreate(&e0));
  MG_CUDA(cudaEventCreate(&e1));
  Status result = launch_alpha(fl, norm2, st);
  for (int l = 0; l < fl.L && result.ok(); ++l) {
    const ResidIn* rl = (l == 0) ? ra : nullptr;
    const ResidOut* rol = (l == 0) ? ro : nullptr;
    float best_d = 1e30f, best_u = 1e30f;
    // two timed rounds per variant, keeping the faster one: a single short
    // round is easily disturbed (clock ramp, other work on the GPU)
    for (int round = 0; round < 2 && result.ok(); ++round)
      for (int v = 0; v < kUpVariants && result.ok(); ++v) {
        float t = 0.f;
        if (v < kFusedVariants) {
          result = launch_down_variant(v, l, fl, r32, norm2, w, nullptr, st, rl);
          if (!result.ok()) break;
          cudaEventRecord(e0, st);
          for (int k = 0; k < reps && result.ok(); ++k)
            result = launch_down_variant(v, l, fl, r32, norm2, w, nullptr, st, rl);
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&t, e0, e1);
          if (t < best_d) { best_d = t; fl.var_down[l] = v; }
        }
        result = launch_up_variant(v, l, fl, norm2, scratch, nullptr, w, nullptr, st, rol);
        if (!result.ok()) break;
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps && result.ok(); ++k)
          result = launch_up_variant(v, l, fl, norm2, scratch, nullptr, w, nullptr, st, rol);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best_u) { best_u = t; fl.var_up[l] = v; }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return result;
}

bool fused_supported(const mgcnn_ctx* c) {
  return c->cp == 8 && c->wl.nu_d == 1 && c->wl.nu_u == 1;
}

// The context's single-problem level set (tile variants as tuned).
FusedLevels ctx_levels(mgcnn_ctx* c) {
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
    fl.s[l] = c->s16[l].as<bf16>();
    fl.xa[l] = c->x16a[l].as<bf16>();
    fl.xb[l] = c->x16b[l].as<bf16>();
    fl.xbl[l] = c->x16l[l].as<bf16>();
    fl.var_down[l] = c->tile_var[0][l];
    fl.var_up[l] = c->tile_var[1][l];
  }
  return fl;
}

// First V-cycle after a setup: time the tile variants per level (outputs to the
// context's scratch vector and partial sums, so no caller data changes) and keep
// the fastest.  With `ra` the finest down kernel is tuned with the residual fused in.
Status ctx_autotune(mgcnn_ctx* c, const float* r32, const double* norm2, const ResidIn* ra,
                    const ResidOut* ro = nullptr) {
  MG_TRY(ensure(c->alpha32, 2 * sizeof(float)));
  if (c->tuned) return {};
  FusedLevels fl = ctx_levels(c);
  MG_TRY(fused_autotune(fl, r32, norm2, c->e.as<double>(), fused_weights(c), c->stream, 5, ra, ro));
  for (int l = 0; l < c->L; ++l) {
    c->tile_var[0][l] = fl.var_down[l];
    c->tile_var[1][l] = fl.var_up[l];
  }
  c->tuned = true;
  c->sgraph_valid = false;
  return {};
}

// e = B r (u_skip == nullptr) or e = u_skip + B r for the context's single problem.
Status vcycle_fused_cp8(mgcnn_ctx* c, const float* r32, const double* norm2, double* e, const double* u_skip,
                        const FusedWeights& w) {
  MG_TRY(ctx_autotune(c, r32, norm2, nullptr));
  return fused_vcycle_levels(ctx_levels(c), r32, norm2, e, u_skip, w, nullptr, c->stream, c);
}

int fused_residual_mode(const mgcnn_ctx* c) {
  return (c->cfg.precision == MGCNN_PREC_MIXED_BF16 && c->fused && fused_supported(c)) ? c->fuse_residual : 0;
}

bool fused_residual_applies(const mgcnn_ctx* c) { return fused_residual_mode(c) == 1; }

ResidOut ctx_resid_out(mgcnn_ctx* c, const double* f) {
  ResidOut ro;
  ro.f = f;
  ro.op = c->op[0].as<double>();
  ro.dinv32 = c->cfg.input_diag ? c->dinv32.as<float>() : nullptr;
  ro.r32 = c->r32.as<float>();
  ro.partial = c->partial.as<double>();
  return ro;
}

Status upres_cycle_setup(mgcnn_ctx* c, const double* f, const double* u, double* rn2_dev, cudaStream_t st) {
  MG_TRY(ensure(c->partial, std::max((size_t)reduction_blocks(c->lv[0].N()), fused_partials_max(c->n)) *
                                sizeof(double)));
  const ResidOut ro = ctx_resid_out(c, f);
  MG_TRY(ctx_autotune(c, c->r32.as<float>(), rn2_dev, nullptr, &ro));
  // r_0 and ||r_0||^2 by the stand-alone kernel; later residuals come from the up kernel
  MG_TRY(launch_residual(f, u, c->op[0].as<double>(), nullptr, c->r32.as<float>(), c->partial.as<double>(), c->n, st,
                         c->cfg.input_diag ? c->dinv32.as<float>() : nullptr));
  return launch_reduce(c->partial.as<double>(), residual_blocks(c->lv[0].N()), rn2_dev, st);
}

Status upres_cycle(mgcnn_ctx* c, const double* f, const double* u_in, double* u_out, double* rn2_dev,
                   const int* active, cudaStream_t st, bool profile) {
  if (u_in == u_out) return make_status(MGCNN_ERR_STATE, "the residual-forming cycle needs two iterate buffers");
  const FusedLevels fl = ctx_levels(c);
  const ResidOut ro = ctx_resid_out(c, f);
  FusedCycleOpt opt;
  opt.resid_out = &ro;
  MG_TRY(fused_vcycle_levels(fl, c->r32.as<float>(), rn2_dev, u_out, u_in, fused_weights(c), active, st,
                             profile ? c : nullptr, opt));
  return launch_reduce(c->partial.as<double>(), fused_down0_blocks(c->n, fl.var_up[0]), rn2_dev, st);
}

ResidIn ctx_resid_in(mgcnn_ctx* c, const double* f, const double* u) {
  ResidIn ra;
  ra.u = u;
  ra.f = f;
  ra.op = c->op[0].as<double>();
  ra.dinv32 = c->cfg.input_diag ? c->dinv32.as<float>() : nullptr;
  ra.partial = c->partial.as<double>();
  return ra;
}

Status fused_cycle_setup(mgcnn_ctx* c, const double* f, const double* u, const double* fn2_dev) {
  MG_TRY(ensure(c->partial, std::max((size_t)reduction_blocks(c->lv[0].N()), fused_partials_max(c->n)) *
                                sizeof(double)));
  const ResidIn ra = ctx_resid_in(c, f, u);
  MG_TRY(ctx_autotune(c, nullptr, fn2_dev, &ra));
  return fused_set_alpha(ctx_levels(c), fn2_dev, c->stream);
}

Status fused_cycle_residual(mgcnn_ctx* c, const double* f, const double* u, double* rn2_dev, const int* active,
                            cudaStream_t st, bool profile) {
  const FusedLevels fl = ctx_levels(c);
  MG_TRY(fused_down0_resid(fl, ctx_resid_in(c, f, u), fused_weights(c), active, st, profile ? c : nullptr));
  return launch_reduce(c->partial.as<double>(), fused_down0_blocks(c->n, fl.var_down[0]), rn2_dev, st);
}

Status fused_cycle_rest(mgcnn_ctx* c, double* u, const double* rn2_dev, const int* active, cudaStream_t st,
                        bool profile) {
  const FusedLevels fl = ctx_levels(c);
  FusedCycleOpt opt;
  opt.after_fused_down0 = true;
  MG_TRY(fused_vcycle_levels(fl, nullptr, rn2_dev, u, u, fused_weights(c), active, st, profile ? c : nullptr, opt));
  return fused_set_alpha(fl, rn2_dev, st);
}

}  // namespace mgcnn

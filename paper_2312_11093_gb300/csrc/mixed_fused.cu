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
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma1688(float* d, uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ float2 bf2f(uint32_t v) { return __bfloat1622float2(*reinterpret_cast<bf162*>(&v)); }
__device__ __forceinline__ uint32_t f2bf(float a, float b) {
  bf162 r = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&r);
}
__device__ __forceinline__ uint4 mul8(uint4 a, uint4 b) {
  float2 x, y;
  uint4 o;
  x = bf2f(a.x); y = bf2f(b.x); o.x = f2bf(x.x * y.x, x.y * y.y);
  x = bf2f(a.y); y = bf2f(b.y); o.y = f2bf(x.x * y.x, x.y * y.y);
  x = bf2f(a.z); y = bf2f(b.z); o.z = f2bf(x.x * y.x, x.y * y.y);
  x = bf2f(a.w); y = bf2f(b.w); o.w = f2bf(x.x * y.x, x.y * y.y);
  return o;
}

// The tiles of a block live in dynamic shared memory (the 32 x 32 variant needs
// more than the 48 KB of static shared memory); every array starts on a 128-byte
// boundary (TMA destinations).
constexpr int pad8(int pixels) { return (pixels + 7) / 8 * 8; }   // uint4 count -> multiple of 128 bytes
template <int FH, int FW, bool FIRST, bool HAS_R>
constexpr size_t down_smem_bytes() {
  constexpr int XH = FH + (HAS_R ? 1 : 0), XW = FW + (HAS_R ? 1 : 0), ZH = XH + 2, ZW = XW + 2;
  constexpr int RH = ZH + 2, RW = ZW + 2;
  return 16u * (2 * pad8(ZH * ZW) + pad8(XH * XW)) + (FIRST ? 4u * RH * RW : 0u);
}
template <int FH, int FW, bool LAST, bool HAS_P>
constexpr size_t up_smem_bytes() {
  constexpr int H = LAST ? 1 : 0, OH = FH + 2 * H, OW = FW + 2 * H, PH = OH + 2, PW = OW + 2;
  constexpr int CH = PH / 2 + 2, CW = PW / 2 + 2;
  return 16u * (2 * pad8(PH * PW) + (HAS_P ? pad8(CH * CW) : 0) + (LAST ? OH * OW : 0));
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
template <int PITCH>
__device__ __forceinline__ void strip_conv_at(const uint4* tile, const uint32_t* wf, int base_m, int base_l,
                                              const TapOffsets<PITCH>& to, float* acc) {
  const uint32_t am = sa(tile) + 16u * base_m, al = sa(tile) + 16u * base_l;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    uint32_t a[4];
    ldsm_x4(a, am + to.off[s]);
    mma16816(acc, a, wf[2 * s], wf[2 * s + 1]);
  }
  uint32_t a[2];
  ldsm_x2(a, al + TapOffsets<PITCH>::off8);
  mma1688(acc, a[0], a[1], wf[8]);
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
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    uint32_t a[4];
    ldsm_x4(a, am + to.off[s]);
    mma16816(acc, a, wf[2 * s], wf[2 * s + 1]);
  }
  // lanes 0-15 address rows 0-15 of tap 8 of z (k 0-7), lanes 16-31 the same
  // rows of x at the centre pixel (k 8-15)
  uint32_t a[4];
  ldsm_x4(a, (lane < 16) ? am + TapOffsets<PITCH>::off8 : sa(xt) + 16u * (base_m + PITCH + 1));
  mma16816(acc, a, wf[8], fI);
}

// The identity block of the last step's B fragment: k = 8 + ci, n = co, one
// where ci == co (this lane holds ci = 2q, 2q + 1 for co = g).
__device__ __forceinline__ uint32_t identity_frag() {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const uint32_t one = 0x3F80u;   // BF16 1.0
  return (2 * q == g ? one : 0u) | ((2 * q + 1 == g ? one : 0u) << 16);
}

__device__ __forceinline__ double alpha_of(const double* norm2, size_t N) {
  const double v = *norm2;
  return (v > 0.0) ? sqrt((double)N / v) : 1.0;
}

// alpha2[2b] = alpha = sqrt(N / ||r_b||^2), alpha2[2b + 1] = 1 / alpha, once per
// cycle and problem: an FP64 divide and square root are dozens of FP64-pipe
// instructions, too many to repeat in every block of the level kernels.
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
template <int FH, int FW, bool FIRST, bool HAS_R>
__global__ void __launch_bounds__(NT, 4) down_kernel(const float* __restrict__ r, const float* __restrict__ alpha2,
                                                  const __grid_constant__ SmallWeights sw,
                                                  const __grid_constant__ CUtensorMap map_x,
                                                  const __grid_constant__ CUtensorMap map_s,
                                                  const uint32_t* __restrict__ fK, const uint32_t* __restrict__ fR,
                                                  bf16* __restrict__ xdown, bf16* __restrict__ xc, int n,
                                                  const int* __restrict__ active, int* __restrict__ err) {
  static_assert(FH % 2 == 0 && FW % 2 == 0 && (FH / 2) * (FW / 2) % 16 == 0, "tile shape");
  constexpr int XH = FH + (HAS_R ? 1 : 0), XW = FW + (HAS_R ? 1 : 0);
  constexpr int ZH = XH + 2, ZW = XW + 2;
  constexpr int RH = ZH + 2, RW = ZW + 2;
  // zs: s, then z = s * x_in in place (BF16); xs: x_in, for the skip.  Both are
  // TMA destinations: the box of rows j0-1.. and columns i0-1.. of the tensor,
  // zero outside the grid.
  uint4* zs = reinterpret_cast<uint4*>(fused_dsm);
  uint4* xs = zs + pad8(ZH * ZW);
  uint4* xd = xs + pad8(ZH * ZW);                                   // layer output
  float* rs = reinterpret_cast<float*>(xd + pad8(XH * XW));         // finest level only
  __shared__ __align__(8) uint64_t bar;
  const int j0 = blockIdx.y * FH, i0 = blockIdx.x * FW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t N = (size_t)n * n;
  // problem blockIdx.z of a batch of equal-size problems stored back to back
  const int bz = blockIdx.z;
  if (active && !active[bz]) return;
  {
    const size_t Nc = (size_t)((n - 1) / 2) * ((n - 1) / 2);
    if (FIRST) r += bz * N;
    xdown += bz * N * 8;
    if (HAS_R) xc += bz * Nc * 8;
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, (FIRST ? 1u : 2u) * ZH * ZW * 16u);
    tma_load_pix(zs, &map_s, i0 - 1, j0 - 1, bz, &bar);
    if (!FIRST) tma_load_pix(xs, &map_x, i0 - 1, j0 - 1, bz, &bar);
  }

  uint32_t wk[9], wr[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    wk[k] = fK[k * 32 + lane];
    if (HAS_R) wr[k] = fR[k * 32 + lane];
  }
  __syncthreads();   // barrier initialised

  if constexpr (FIRST) {
    const float alpha = alpha2[2 * bz];   // the finest level's input scale
    #pragma unroll 4
    for (int e = threadIdx.x; e < RH * RW; e += NT) {
      const int rr = e / RW, cc = e - rr * RW;
      const int gj = j0 + rr - 2, gi = i0 + cc - 2;
      rs[e] = (gj >= 0 && gj < n && gi >= 0 && gi < n) ? alpha * r[(size_t)gj * n + gi] : 0.f;
    }
  }
  // the copies of the block's tiles (a uniform decision: every thread agrees
  // before any of them returns)
  const bool landed = mbar_wait_bounded(&bar, 0);
  if (!__syncthreads_and(landed)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  if constexpr (FIRST) {
    // x_in = W_in * (alpha r) on Z, rounded to BF16 (zero outside the grid); z = s * x_in
    for (int e = threadIdx.x; e < ZH * ZW; e += NT) {
      const int zr = e / ZW, zc = e - zr * ZW;
      const int gj = j0 + zr - 1, gi = i0 + zc - 1;
      uint4 xv = make_uint4(0, 0, 0, 0);
      if (gj >= 0 && gj < n && gi >= 0 && gi < n) {
        float rv[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) rv[t] = rs[(zr + t / 3) * RW + zc + t % 3];
        float o[8];
#pragma unroll
        for (int co = 0; co < 8; ++co) {
          float a = 0.f;
#pragma unroll
          for (int t = 0; t < 9; ++t) a += sw.w_in[t * 8 + co] * rv[t];
          o[co] = a;
        }
        xv = make_uint4(f2bf(o[0], o[1]), f2bf(o[2], o[3]), f2bf(o[4], o[5]), f2bf(o[6], o[7]));
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
    // strips of 16 consecutive pixels of X in row-major order (a strip may wrap
    // to the next row); the division by the compile-time width is a multiply
    constexpr int NX = XH * XW, NSTRIP = (NX + 15) / 16;
    const TapOffsets<ZW> to;
    const uint32_t fI = identity_frag();
    for (int st = warp; st < NSTRIP; st += NW) {
      const int pm = min(st * 16 + mrow, NX - 1), rm = pm / XW;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      layer_strip<ZW>(zs, xs, wk, fI, rm * ZW + (pm - rm * XW), to, acc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = st * 16 + g + 8 * h;
        if (p >= NX) continue;
        const int xr = p / XW, xcol = p - xr * XW;
        const uint32_t o = f2bf(acc[2 * h], acc[2 * h + 1]);
        reinterpret_cast<uint32_t*>(&xd[xr * XW + xcol])[q] = o;
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
    const int J0 = blockIdx.y * CH, I0 = blockIdx.x * CW;
    const TapOffsets<XW> tr;
    for (int st = warp; st < CH * CW / 16; st += NW) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const int pm = st * 16 + mrow, pl = st * 16 + lrow;
      strip_conv_at<XW>(xd, wr, 2 * (pm / CW) * XW + 2 * (pm % CW), 2 * (pl / CW) * XW + 2 * (pl % CW), tr, acc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = st * 16 + g + 8 * h, cr = p / CW, cc = p - cr * CW;
        const int J = J0 + cr, I = I0 + cc;
        if (J < nc && I < nc)
          reinterpret_cast<uint32_t*>(xc + ((size_t)J * nc + I) * 8)[q] = f2bf(acc[2 * h], acc[2 * h + 1]);
      }
    }
  }
}

// Shared-memory view of an up-kernel block for the TCNN pass.
struct TcnnTile {
  uint4* ps;          // P region: x_down in, x_pre out
  uint4* zs;          // P region: s in, s * x_pre out
  const uint4* cs;    // staged coarse pixels (zero outside the coarse grid)
  int pj0, pi0;       // global coordinates of P's corner
  int cj0, ci0;       // global coordinates of cs's corner
  int n;
};

// TCNN-add on the tensor cores, one parity class (gj & 1 == A, gi & 1 == B) of
// the fine pixels of P at a time.  A fine row 2J + a gets coarse row J through
// tap row a: a in {0, 2} for even rows, a = 1 for odd rows (likewise columns),
// so a class has a fixed tap list -- 4, 2, 2 or 1 taps, i.e. K = 32, 16, 16 or
// 8 -- and each 16 class pixels are a GEMM [16 x K] x [K x 8]
// whose A rows are coarse pixels gathered by ldmatrix (per-lane addresses; the
// zero-filled staging covers coarse pixels outside the grid).  fT holds the B
// fragments in the step order (taps 0, 2 | 6, 8 | 1, 7 | 3, 5 | 4).
// Epilogue: x_pre = x_down + TCNN rounded once to BF16, z = s * x_pre.
template <int A, int B, int PH, int PW, int CW>
__device__ __forceinline__ void tcnn_class_mma(const TcnnTile& t, const uint32_t* fT, int st, int lane) {
  // the class's pixels in row-major order over an NRM x NCM grid (class rows
  // and columns, at most); strips of 16 of them, wrapping across class rows
  constexpr int NRM = (PH + 1) / 2, NCM = (PW + 1) / 2, NP = NRM * NCM;
  const int r0 = (A ^ t.pj0) & 1, c0 = (B ^ t.pi0) & 1;   // first P row / column of the class
  const int nr_cls = (PH - r0 + 1) >> 1, nc_cls = (PW - c0 + 1) >> 1;
  const int mrow = (lane & 7) + ((lane >> 3) & 1) * 8, kh = lane >> 4;
  // fine pixel of A row m (clamped into the class so that every address is valid)
  auto fine = [&](int m, int& gj, int& gi) {
    const int p = min(st * 16 + m, NP - 1);
    const int rr = p / NCM, cc = p - rr * NCM;
    gj = t.pj0 + r0 + 2 * min(rr, nr_cls - 1);
    gi = t.pi0 + c0 + 2 * min(cc, nc_cls - 1);
  };
  // shared-memory pixel of coarse (J, I) for fine (gj, gi) through tap (ta, tb)
  const uint32_t cs0 = sa(t.cs);
  auto at = [&](int gj, int gi, int ta, int tb) {
    return cs0 + 16u * ((((gj - ta) >> 1) - t.cj0) * CW + (((gi - tb) >> 1) - t.ci0));
  };
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  uint32_t a[4];
  int gj, gi;
  if constexpr (A == 1 && B == 1) {
    fine(lane & 15, gj, gi);
    ldsm_x2(a, at(gj, gi, 1, 1));              // tap (1,1)
    mma1688(acc, a[0], a[1], fT[8]);
  } else {
    fine(mrow, gj, gi);
    if constexpr (A == 0 && B == 0) {
      // step 0: taps (0,0) | (0,2); step 1: taps (2,0) | (2,2)
      ldsm_x4(a, at(gj, gi, 0, kh ? 2 : 0));
      mma16816(acc, a, fT[0], fT[1]);
      ldsm_x4(a, at(gj, gi, 2, kh ? 2 : 0));
      mma16816(acc, a, fT[2], fT[3]);
    } else if constexpr (A == 0 && B == 1) {
      ldsm_x4(a, at(gj, gi, kh ? 2 : 0, 1));   // taps (0,1) | (2,1)
      mma16816(acc, a, fT[4], fT[5]);
    } else {
      ldsm_x4(a, at(gj, gi, 1, kh ? 2 : 0));   // taps (1,0) | (1,2)
      mma16816(acc, a, fT[6], fT[7]);
    }
  }
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int p = st * 16 + g + 8 * h;
    const int rr = p / NCM, cc = p - rr * NCM;
    const int pr = r0 + 2 * rr, pc = c0 + 2 * cc;
    const int ogj = t.pj0 + pr, ogi = t.pi0 + pc;
    if (p >= NP || rr >= nr_cls || cc >= nc_cls || ogj < 0 || ogj >= t.n || ogi < 0 || ogi >= t.n) continue;
    const int pe = pr * PW + pc;
    const float2 xin = bf2f(reinterpret_cast<const uint32_t*>(&t.ps[pe])[q]);
    const uint32_t xo = f2bf(xin.x + acc[2 * h], xin.y + acc[2 * h + 1]);
    reinterpret_cast<uint32_t*>(&t.ps[pe])[q] = xo;
    const float2 xf = bf2f(xo), sf = bf2f(reinterpret_cast<const uint32_t*>(&t.zs[pe])[q]);
    reinterpret_cast<uint32_t*>(&t.zs[pe])[q] = f2bf(xf.x * sf.x, xf.y * sf.y);
  }
}

// All four classes, strips spread over the warps.
template <int PH, int PW, int CW>
__device__ __forceinline__ void tcnn_mma(const TcnnTile& t, const uint32_t* fT) {
  constexpr int NRM = (PH + 1) / 2, NCM = (PW + 1) / 2, PER = (NRM * NCM + 15) / 16;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int st = warp; st < 4 * PER; st += NW) {
    const int cls = st / PER, sl = st - cls * PER;
    if (cls == 0)
      tcnn_class_mma<0, 0, PH, PW, CW>(t, fT, sl, lane);
    else if (cls == 1)
      tcnn_class_mma<0, 1, PH, PW, CW>(t, fT, sl, lane);
    else if (cls == 2)
      tcnn_class_mma<1, 0, PH, PW, CW>(t, fT, sl, lane);
    else
      tcnn_class_mma<1, 1, PH, PW, CW>(t, fT, sl, lane);
  }
}

// ---------------------------------------------------------------------------
// Up kernel.  Output tile 16 x 32 at (j0, i0).  H = halo of the layer output
// that is needed (1 at the finest level for W_out, else 0).
//   O (layer output):  rows -H..15+H, cols -H..31+H        (OH x OW)
//   P (layer input x_pre = x_down + TCNN(x_c)): O plus halo 1  (PH x PW)
//   coarse rows/cols J: floor((j0 - H - 1) / 2) - 1 .. , enough for P
template <int FH, int FW, bool LAST, bool HAS_P>
__global__ void __launch_bounds__(NT, 4) up_kernel(const __grid_constant__ CUtensorMap map_xd,
                                                const __grid_constant__ CUtensorMap map_s,
                                                const __grid_constant__ CUtensorMap map_c,
                                                const uint32_t* __restrict__ fK, const uint32_t* __restrict__ fTc,
                                                const uint32_t* __restrict__ fOutHi,
                                                const uint32_t* __restrict__ fOutLo,
                                                const float* __restrict__ alpha2, const double* __restrict__ u_in,
                                                bf16* __restrict__ xfin, double* __restrict__ u_out, int n,
                                                const int* __restrict__ active, int* __restrict__ err) {
  constexpr int H = LAST ? 1 : 0;
  constexpr int OH = FH + 2 * H, OW = FW + 2 * H;
  constexpr int PH = OH + 2, PW = OW + 2;
  constexpr int CH = PH / 2 + 2, CW = PW / 2 + 2;   // coarse rows / cols staged
  // TMA destinations (zero outside the grid): ps = x_down on P, then x_pre;
  // zs = s on P, then s * x_pre; cs = the coarse pixels under P
  uint4* ps = reinterpret_cast<uint4*>(fused_dsm);
  uint4* zs = ps + pad8(PH * PW);
  uint4* cs = zs + pad8(PH * PW);                                    // coarser level only
  uint4* os = cs + (HAS_P ? pad8(CH * CW) : 0);                      // finest level only
  __shared__ __align__(8) uint64_t bar;
  const int j0 = blockIdx.y * FH, i0 = blockIdx.x * FW;
  const int pj0 = j0 - H - 1, pi0 = i0 - H - 1;      // global coords of P's corner
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bz = blockIdx.z;
  if (active && !active[bz]) return;
  {
    const size_t N = (size_t)n * n;
    if (LAST) {
      if (u_in) u_in += bz * N;
      u_out += bz * N;
    } else {
      xfin += bz * N * 8;
    }
  }
  // coarse corner: the smallest J with 2J + 2 >= pj0
  const int cj0 = (pj0 - 2 >= 0) ? (pj0 - 2) / 2 : -((2 - pj0 + 1) / 2);
  const int ci0 = (pi0 - 2 >= 0) ? (pi0 - 2) / 2 : -((2 - pi0 + 1) / 2);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, (2u * PH * PW + (HAS_P ? CH * CW : 0u)) * 16u);
    tma_load_pix(ps, &map_xd, pi0, pj0, bz, &bar);
    tma_load_pix(zs, &map_s, pi0, pj0, bz, &bar);
    if (HAS_P) tma_load_pix(cs, &map_c, ci0, cj0, bz, &bar);
  }

  uint32_t wk[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) wk[k] = fK[k * 32 + lane];
  __syncthreads();   // barrier initialised
  const bool landed = mbar_wait_bounded(&bar, 0);
  if (!__syncthreads_and(landed)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }

  // x_pre on P: per parity class (gj & 1, gi & 1) of the fine pixel, the TCNN
  // taps that reach it -- 4, 2, 2 or 1, known at compile time, so the weights are
  // constant operands -- x_pre = x_down + TCNN(x_c) rounded once, z = s * x_pre.
  if constexpr (HAS_P) {
    uint32_t fT[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) fT[k] = fTc[k * 32 + lane];
    const TcnnTile t{ps, zs, cs, pj0, pi0, cj0, ci0, n};
    tcnn_mma<PH, PW, CW>(t, fT);
  } else {
    for (int e = threadIdx.x; e < PH * PW; e += NT) zs[e] = mul8(ps[e], zs[e]);
  }
  __syncthreads();

  // layer on O, row-aligned strips as in the down kernel
  const int g = lane >> 2, q = lane & 3;
  {
    constexpr int NO = OH * OW, NSTRIP = (NO + 15) / 16;   // row-major strips, as in the down kernel
    const int mrow = (lane & 7) + ((lane >> 3) & 1) * 8;
    const TapOffsets<PW> to;
    const uint32_t fI = identity_frag();
    for (int st = warp; st < NSTRIP; st += NW) {
      const int pm = min(st * 16 + mrow, NO - 1), rm = pm / OW;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      layer_strip<PW>(zs, ps, wk, fI, rm * PW + (pm - rm * OW), to, acc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = st * 16 + g + 8 * h;
        if (p >= NO) continue;
        const int orow = p / OW, ocol = p - orow * OW;
        const uint32_t o = f2bf(acc[2 * h], acc[2 * h + 1]);
        const int gj = j0 - H + orow, gi = i0 - H + ocol;
        if constexpr (LAST) {
          // zero outside the grid: W_out's zero padding
          reinterpret_cast<uint32_t*>(&os[orow * OW + ocol])[q] = (gj >= 0 && gj < n && gi >= 0 && gi < n) ? o : 0u;
        } else {
          if (gj < n && gi < n) reinterpret_cast<uint32_t*>(xfin + ((size_t)gj * n + gi) * 8)[q] = o;
        }
      }
    }
  }
  if constexpr (LAST) {
    // W_out on the tensor cores: an 8 -> 8 channel layer whose only nonzero
    // output channel is 0, with the FP32 weights split as hi + lo BF16 (the two
    // products are accumulated in FP32, so the weights keep ~16 bits); strips of
    // 16 owned pixels of one row, as in the layer above
    uint32_t wh[9], wl[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      wh[k] = fOutHi[k * 32 + lane];
      wl[k] = fOutLo[k * 32 + lane];
    }
    __syncthreads();
    const float inv_alpha = alpha2[2 * bz + 1];
    float* ev = reinterpret_cast<float*>(ps);   // FH x FW corrections
    static_assert(FH * FW * sizeof(float) <= PH * PW * sizeof(uint4), "correction staging");
    constexpr int SPRO = (FW + 15) / 16;
    const int mrow = (lane & 7) + ((lane >> 3) & 1) * 8, lrow = lane & 15;
    const TapOffsets<OW> to;
    for (int st = warp; st < FH * SPRO; st += NW) {
      const int rr = st / SPRO, c0 = (st - rr * SPRO) * 16;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const int bm = rr * OW + min(c0 + mrow, FW - 1), bl = rr * OW + min(c0 + lrow, FW - 1);
      strip_conv_at<OW>(os, wh, bm, bl, to, acc);
      strip_conv_at<OW>(os, wl, bm, bl, to, acc);
      // output channel 0 sits in the q == 0 lanes: stage it in shared memory
      // (the P tiles are free now) so that the FP64 update below runs on
      // full warps -- an FP64 instruction costs the same with 8 lanes or 32
      if (q == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cc = c0 + g + 8 * h;
          if (cc < FW) ev[rr * FW + cc] = acc[2 * h] * inv_alpha;
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < FH * FW; e += NT) {
      const int rr = e / FW, cc = e - rr * FW;
      const int gj = j0 + rr, gi = i0 + cc;
      if (gj >= n || gi >= n) continue;
      const size_t qg = (size_t)gj * n + gi;
      u_out[qg] = (u_in ? u_in[qg] : 0.0) + f32_to_f64_exact(ev[e]);
    }
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
                   const int* active, cudaStream_t st) {
  const int nl = fl.n[l];
  const bool first = l == 0, has_r = l + 1 < fl.L;
  const dim3 grid((nl + FW - 1) / FW, (nl + FH - 1) / FH, fl.batch);
  __nv_bfloat16* xc = has_r ? fl.xb[l + 1] : nullptr;
  const int R = has_r ? 1 : 0, ZH = FH + R + 2, ZW = FW + R + 2;
  CUtensorMap ms, mx;
  MG_TRY(pix8_map(fl, fl.s[l], nl, ZW, ZH, &ms));
  if (first)
    mx = ms;   // not read on the finest level
  else
    MG_TRY(pix8_map(fl, fl.xb[l], nl, ZW, ZH, &mx));
  auto run = [&](auto* kernel, size_t smem) {
    kernel<<<grid, NT, dyn_smem(kernel, smem), st>>>(r32, fl.alpha, w.small, mx, ms, w.f_down, w.f_R, fl.xa[l], xc,
                                                      nl, active, fl.err);
  };
  if (first && has_r)
    run(down_kernel<FH, FW, true, true>, down_smem_bytes<FH, FW, true, true>());
  else if (first)
    run(down_kernel<FH, FW, true, false>, down_smem_bytes<FH, FW, true, false>());
  else if (has_r)
    run(down_kernel<FH, FW, false, true>, down_smem_bytes<FH, FW, false, true>());
  else
    run(down_kernel<FH, FW, false, false>, down_smem_bytes<FH, FW, false, false>());
  MG_LAUNCH("down_kernel");
  return {};
}

template <int FH, int FW>
Status launch_up(int l, const FusedLevels& fl, const double* norm2, double* e, const double* u_skip,
                 const FusedWeights& w, const int* active, cudaStream_t st) {
  const int nl = fl.n[l];
  const bool last = l == 0, has_p = l + 1 < fl.L;
  const dim3 grid((nl + FW - 1) / FW, (nl + FH - 1) / FH, fl.batch);
  const int H = last ? 1 : 0, PH = FH + 2 * H + 2, PW = FW + 2 * H + 2;
  CUtensorMap mxd, ms, mc;
  MG_TRY(pix8_map(fl, fl.xa[l], nl, PW, PH, &mxd));
  MG_TRY(pix8_map(fl, fl.s[l], nl, PW, PH, &ms));
  if (has_p)
    MG_TRY(pix8_map(fl, fl.xb[l + 1], fl.n[l + 1], PW / 2 + 2, PH / 2 + 2, &mc));
  else
    mc = ms;   // not read on the coarsest level
  auto run = [&](auto* kernel, size_t smem, bf16* xfin) {
    kernel<<<grid, NT, dyn_smem(kernel, smem), st>>>(mxd, ms, mc, w.f_up, w.f_tcnn, w.f_out_hi, w.f_out_lo, fl.alpha,
                                                      u_skip, xfin, e, nl, active, fl.err);
  };
  if (last && has_p)
    run(up_kernel<FH, FW, true, true>, up_smem_bytes<FH, FW, true, true>(), nullptr);
  else if (last)
    run(up_kernel<FH, FW, true, false>, up_smem_bytes<FH, FW, true, false>(), nullptr);
  else if (has_p)
    run(up_kernel<FH, FW, false, true>, up_smem_bytes<FH, FW, false, true>(), fl.xb[l]);
  else
    run(up_kernel<FH, FW, false, false>, up_smem_bytes<FH, FW, false, false>(), fl.xb[l]);
  MG_LAUNCH("up_kernel");
  return {};
}

Status launch_down_variant(int v, int l, const FusedLevels& fl, const float* r32, const double* norm2,
                           const FusedWeights& w, const int* active, cudaStream_t st) {
  switch (v) {
    case 1: return launch_down<8, 32>(l, fl, r32, norm2, w, active, st);
    case 2: return launch_down<16, 16>(l, fl, r32, norm2, w, active, st);
    case 3: return launch_down<32, 32>(l, fl, r32, norm2, w, active, st);
    case 4: return launch_down<24, 32>(l, fl, r32, norm2, w, active, st);
    default: return launch_down<16, 32>(l, fl, r32, norm2, w, active, st);
  }
}

Status launch_up_variant(int v, int l, const FusedLevels& fl, const double* norm2, double* e, const double* u_skip,
                         const FusedWeights& w, const int* active, cudaStream_t st) {
  switch (v) {
    case 1: return launch_up<8, 32>(l, fl, norm2, e, u_skip, w, active, st);
    case 2: return launch_up<16, 16>(l, fl, norm2, e, u_skip, w, active, st);
    case 3: return launch_up<32, 32>(l, fl, norm2, e, u_skip, w, active, st);
    case 4: return launch_up<24, 32>(l, fl, norm2, e, u_skip, w, active, st);
    default: return launch_up<16, 32>(l, fl, norm2, e, u_skip, w, active, st);
  }
}

}  // namespace

// One V-cycle with the fused level kernels (CP = 8) for a batch of `batch`
// equal-size problems stored back to back: level l state in xa[l] (down state)
// and xb[l] (restricted input, then final up state), setup tensors s[l];
// r32/norm2/u/e per problem.  `active` (nullable, [batch]) skips converged
// problems.  fl.var_down / fl.var_up pick each level's tile variant.
Status fused_vcycle_levels(const FusedLevels& fl, const float* r32, const double* norm2, double* e,
                           const double* u_skip, const FusedWeights& w, const int* active, cudaStream_t st,
                           mgcnn_ctx* prof_ctx) {
  const int L = fl.L;
  MG_TRY(launch_alpha(fl, norm2, st));
  for (int l = 0; l < L; ++l) {
    const int ps = (l == 0 && prof_ctx) ? prof_begin(prof_ctx, kProfDown0) : -1;
    MG_TRY(launch_down_variant(fl.var_down[l], l, fl, r32, norm2, w, active, st));
    if (prof_ctx) prof_end(prof_ctx, ps);
  }
  for (int l = L - 1; l >= 0; --l) {
    const int ps = (l == 0 && prof_ctx) ? prof_begin(prof_ctx, kProfUp0) : -1;
    MG_TRY(launch_up_variant(fl.var_up[l], l, fl, norm2, e, u_skip, w, active, st));
    if (prof_ctx) prof_end(prof_ctx, ps);
  }
  return {};
}

// Autotuner: for every level, time each tile variant of the down and up kernels
// (CUDA events, `reps` launches after one warm-up launch) on the real buffers
// and keep the fastest.  The up kernel of the finest level writes its FP64
// output to `scratch` (n_0^2 x batch doubles) so that no caller data changes.
Status fused_autotune(FusedLevels& fl, const float* r32, const double* norm2, double* scratch,
                      const FusedWeights& w, cudaStream_t st, int reps) {
  cudaEvent_t e0, e1;
  MG_CUDA(cudaEventCreate(&e0));
  MG_CUDA(cudaEventCreate(&e1));
  Status result = launch_alpha(fl, norm2, st);
  for (int l = 0; l < fl.L && result.ok(); ++l) {
    float best_d = 1e30f, best_u = 1e30f;
    // two timed rounds per variant, keeping the faster one: a single short
    // round is easily disturbed (clock ramp, other work on the GPU)
    for (int round = 0; round < 2 && result.ok(); ++round)
      for (int v = 0; v < kFusedVariants && result.ok(); ++v) {
        float t = 0.f;
        result = launch_down_variant(v, l, fl, r32, norm2, w, nullptr, st);
        if (!result.ok()) break;
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps && result.ok(); ++k) result = launch_down_variant(v, l, fl, r32, norm2, w, nullptr, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best_d) { best_d = t; fl.var_down[l] = v; }
        result = launch_up_variant(v, l, fl, norm2, scratch, nullptr, w, nullptr, st);
        if (!result.ok()) break;
        cudaEventRecord(e0, st);
        for (int k = 0; k < reps && result.ok(); ++k) result = launch_up_variant(v, l, fl, norm2, scratch, nullptr, w, nullptr, st);
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

// e = B r (u_skip == nullptr) or e = u_skip + B r for the context's single problem.
Status vcycle_fused_cp8(mgcnn_ctx* c, const float* r32, const double* norm2, double* e, const double* u_skip,
                        const FusedWeights& w) {
  FusedLevels fl;
  fl.L = c->L;
  fl.batch = 1;
  fl.maps = c->tma;
  fl.err = c->kerr.as<int>();
  MG_TRY(ensure(c->alpha32, 2 * sizeof(float)));
  fl.alpha = c->alpha32.as<float>();
  for (int l = 0; l < c->L; ++l) {
    fl.n[l] = c->lv[l].n;
    fl.s[l] = c->s16[l].as<bf16>();
    fl.xa[l] = c->x16a[l].as<bf16>();
    fl.xb[l] = c->x16b[l].as<bf16>();
  }
  if (!c->tuned) {
    // first V-cycle after a setup: time the tile variants per level (output to
    // the context's scratch vector, so no caller data changes), keep the fastest
    MG_TRY(fused_autotune(fl, r32, norm2, c->e.as<double>(), w, c->stream, 5));
    for (int l = 0; l < c->L; ++l) {
      c->tile_var[0][l] = fl.var_down[l];
      c->tile_var[1][l] = fl.var_up[l];
    }
    c->tuned = true;
  }
  for (int l = 0; l < c->L; ++l) {
    fl.var_down[l] = c->tile_var[0][l];
    fl.var_up[l] = c->tile_var[1][l];
  }
  return fused_vcycle_levels(fl, r32, norm2, e, u_skip, w, nullptr, c->stream, c);
}

}  // namespace mgcnn

// Mixed-precision solve phase: BF16 tensors, BF16 x BF16 products, FP32
// accumulation, inside an FP64 defect-correction loop.
//
// Algorithm 3 of arXiv 2312.11093 (solve phase) with every tensor of the
// network stored in BF16, pixel-major with the channel count padded to CP = 8
// or 16 so that one pixel is one or two 16-byte vectors.  The C x C 3x3
// layers (ResNetDown/Up, Eq. heteroresnet, and the stride-2 RCNN) are
// implicit GEMMs on the tensor cores: M = 16 output pixels per warp tile,
// N = CP output channels, K = 9 taps x CP input channels, A fragments loaded
// with ldmatrix straight from the shared-memory input tile (each pixel row is
// one 16-byte ldmatrix row, a tap is an address offset), B fragments (the
// weights) held in registers for the whole kernel.  The thin layers
// (reChannelCNN 1->C and C->1, and the transposed convolution, which touches
// only 2.25 taps per fine pixel) run on FP32 CUDA cores.
//
// Defect correction: the residual r (FP64, computed elsewhere) enters scaled
// by alpha = sqrt(N)/||r||_2 -- exact by linearity (P2, Sec. 3.1) -- and the
// correction leaves as e/alpha, added to u in FP64.
#include <algorithm>
#include <cmath>

#include "mixed.cuh"
#include "ops.cuh"

namespace mgcnn {

using bf16 = __nv_bfloat16;
using bf162 = __nv_bfloat162;

bool mixed_channels_supported(int C) { return C == 4 || C == 8 || C == 12 || C == 13 || C == 16; }

namespace {

int padded_channels(int C) { return C <= 8 ? 8 : 16; }

// Packed-weight layout inside ctx->wmix.
struct MixLayout {
  int cp = 0, nreg = 0;
  size_t frag_words = 0;                 // uint32 words per packed C x C conv
  size_t down = 0, up = 0, R = 0;        // byte offsets of the fragment blocks
  size_t w_in = 0, w_out = 0, w_P = 0;   // byte offsets of FP32 arrays
  size_t s_frag = 0, s_fp = 0;           // setup network: 5 fragment blocks, FP32 biases + W_cin (CP = 8)
  size_t out_taps = 0;                   // W_out fragments by tap for the fused up kernel (CP = 8)
  size_t tcnn = 0;                       // TCNN fragments of the 2 x 2 fine-pixel quads (CP = 8)
  size_t bytes = 0;
};

MixLayout mix_layout(const mgcnn_ctx* c) {
  MixLayout m;
  m.cp = padded_channels(c->cfg.channels);
  m.nreg = (m.cp == 8) ? 9 : 36;
  m.frag_words = (size_t)m.nreg * 32;
  size_t o = 0;
  m.down = o; o += (size_t)c->wl.nu_d * m.frag_words * 4;
  m.up = o;   o += (size_t)c->wl.nu_u * m.frag_words * 4;
  m.R = o;    o += m.frag_words * 4;
  m.w_in = o;  o += (size_t)m.cp * 9 * 4;
  m.w_out = o; o += (size_t)m.cp * 9 * 4;
  m.w_P = o;   o += (size_t)m.cp * m.cp * 9 * 4;
  m.s_frag = o; o += 5 * m.frag_words * 4;
  m.s_fp = o;   o += (4 * 8 + 8 * kFeatures * 9 + 8) * 4;
  m.out_taps = o; o += (size_t)kOutTapRegs * 32 * 4;
  m.tcnn = o;   o += (size_t)kTcnnQuadRegs * 32 * 4;
  m.bytes = o;
  return m;
}

uint16_t f2bf_host(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
  u += 0x7fffu + ((u >> 16) & 1u);                       // round to nearest even
  return (uint16_t)(u >> 16);
}

// mma.m16n8k16 / m16n8k8 B fragments of a C x C 3x3 conv W[co][ci][a][b].
// B[k][n] with k = tap * CP + ci (zero for ci >= C), n = co (zero for co >= C).
// Per lane (g = lane/4, q = lane%4) a 32-bit register holds B[k0][n], B[k0+1][n]
// (low half = lower k) with k0 = 16 s + 2 q (first) or + 8 (second register).
// B fragments of the TCNN W[ci][co][a][b] for the fused up kernel's quad GEMM.
// A quad is the 2 x 2 block of fine pixels (2J+1+r, 2I+1+c), r, c in {0, 1};
// it receives the transposed convolution from the coarse pixels (J+dJ, I+dI),
// dJ, dI in {0, 1}, through tap (1 + r - 2 dJ, 1 + c - 2 dI) (zero weight where
// that tap lies outside 0..2).  A rows are quads, k = (dJ, dI, ci): k step dJ
// holds (dI = 0, ci) at k 0-7 and (dI = 1, ci) at k 8-15; n-tile t = 2 r + c is
// fine pixel (r, c), n = co.  Register index (2 t + dJ) * 2 + half.
void pack_tcnn_frags(const double* W, int C, uint32_t* out) {
  auto B = [&](int a, int b, int ci, int co) -> float {
    if (a < 0 || a > 2 || b < 0 || b > 2 || ci >= C || co >= C) return 0.0f;
    return (float)W[((size_t)ci * C + co) * 9 + a * 3 + b];
  };
  for (int lane = 0; lane < 32; ++lane) {
    const int g = lane >> 2, q = lane & 3;
    for (int t = 0; t < 4; ++t) {
      const int r = t >> 1, c = t & 1;
      for (int dJ = 0; dJ < 2; ++dJ)
        for (int dI = 0; dI < 2; ++dI) {
          const int a = 1 + r - 2 * dJ, b = 1 + c - 2 * dI;
          out[((2 * t + dJ) * 2 + dI) * 32 + lane] = (uint32_t)f2bf_host(B(a, b, 2 * q, g)) |
                                                     ((uint32_t)f2bf_host(B(a, b, 2 * q + 1, g)) << 16);
        }
    }
  }
}

// W_out (one output channel) by tap, for the fused up kernel's product
// D[pixel][tap] = sum_ch (hi(y) + lo(y))[ch] w_tap[ch] as one K = 16 MMA over
// A = [hi(y) | lo(y)]: B tile b holds taps 6 b .. (n = tap - 6 b; n past tap 8
// zero), as [w_hi ; w_hi] (hl = 0) and [w_lo ; 0] (hl = 1, the weights' low
// parts times hi(y)).  Word ((b * 2 + hl) * 2 + reg) * 32 + lane; reg 0 holds k
// = 2q, 2q + 1 (channels of hi(y)), reg 1 k = 8 + 2q, 9 + 2q (those of lo(y)).
// whi[ch * 9 + tap] and wlo[ch * 9 + tap] are the BF16-exact hi and lo parts of w_out.
void pack_out_taps(const std::vector<double>& whi, const std::vector<double>& wlo, uint32_t* out) {
  for (int b = 0; b < 2; ++b)
    for (int hl = 0; hl < 2; ++hl)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, q = lane & 3, tap = 6 * b + g;
        const bool valid = b == 0 ? g < 6 : g < 3;
        const std::vector<double>& w = hl ? wlo : whi;
        auto wv = [&](int ch) -> uint32_t { return valid ? f2bf_host((float)w[ch * 9 + tap]) : 0u; };
        const uint32_t pr = wv(2 * q) | (wv(2 * q + 1) << 16);
        out[((b * 2 + hl) * 2 + 0) * 32 + lane] = pr;
        out[((b * 2 + hl) * 2 + 1) * 32 + lane] = hl ? 0u : pr;
      }
}

void pack_frags(const double* W, int C, int cp, uint32_t* out) {
  auto B = [&](int k, int nn) -> float {
    const int tap = k / cp, ci = k % cp;
    if (tap >= 9 || ci >= C || nn >= C) return 0.0f;
    return (float)W[((size_t)nn * C + ci) * 9 + tap];
  };
  auto pair = [&](int k, int nn) -> uint32_t {
    return (uint32_t)f2bf_host(B(k, nn)) | ((uint32_t)f2bf_host(B(k + 1, nn)) << 16);
  };
  if (cp == 8) {
    // 4 k16 steps (taps 2s, 2s+1) then one k8 step (tap 8); regs i = 2s + r, i = 8
    for (int lane = 0; lane < 32; ++lane) {
      const int g = lane >> 2, q = lane & 3;
      for (int s = 0; s < 4; ++s) {
        out[(2 * s + 0) * 32 + lane] = pair(16 * s + 2 * q, g);
        out[(2 * s + 1) * 32 + lane] = pair(16 * s + 2 * q + 8, g);
      }
      out[8 * 32 + lane] = pair(64 + 2 * q, g);
    }
  } else {
    // 9 k16 steps (one tap each) x 2 n8 tiles; regs i = (tap * 2 + t) * 2 + r
    for (int lane = 0; lane < 32; ++lane) {
      const int g = lane >> 2, q = lane & 3;
      for (int tap = 0; tap < 9; ++tap)
        for (int t = 0; t < 2; ++t) {
          out[((tap * 2 + t) * 2 + 0) * 32 + lane] = pair(16 * tap + 2 * q, 8 * t + g);
          out[((tap * 2 + t) * 2 + 1) * 32 + lane] = pair(16 * tap + 2 * q + 8, 8 * t + g);
        }
    }
  }
}

// ---------------------------------------------------------------------------
// device helpers
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t* r, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
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

__device__ __forceinline__ uint32_t mul_bf16x2(uint32_t a, uint32_t b) {
  const float2 fa = __bfloat1622float2(*reinterpret_cast<const bf162*>(&a));
  const float2 fb = __bfloat1622float2(*reinterpret_cast<const bf162*>(&b));
  bf162 r = __floats2bfloat162_rn(fa.x * fb.x, fa.y * fb.y);
  return *reinterpret_cast<uint32_t*>(&r);
}
__device__ __forceinline__ uint4 mul_bf16x8(uint4 a, uint4 b) {
  return make_uint4(mul_bf16x2(a.x, b.x), mul_bf16x2(a.y, b.y), mul_bf16x2(a.z, b.z), mul_bf16x2(a.w, b.w));
}

__device__ __forceinline__ double alpha_from(const double* norm2, size_t N) {
  const double v = *norm2;
  return (v > 0.0) ? sqrt((double)N / v) : 1.0;
}

// Implicit-GEMM accumulation of one warp tile: 16 output pixels x CP channels.
// addr(m, tap) returns the shared-memory pixel index of the A row m for tap.
template <int CP, typename Addr>
__device__ __forceinline__ void warp_conv(const bf16* tile, const uint32_t* wf, Addr addr, float (*acc)[4]) {
  const int lane = threadIdx.x & 31;
  const int m = (lane & 7) + ((lane >> 3) & 1) * 8;
  const int kh = lane >> 4;
  if constexpr (CP == 8) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      uint32_t a[4];
      ldsm_x4(a, tile + (size_t)addr(m, 2 * s + kh) * CP);
      mma16816(acc[0], a, wf[2 * s], wf[2 * s + 1]);
    }
    uint32_t a[2];
    ldsm_x2(a, tile + (size_t)addr(lane & 15, 8) * CP);
    mma1688(acc[0], a[0], a[1], wf[8]);
  } else {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      uint32_t a[4];
      ldsm_x4(a, tile + (size_t)addr(m, tap) * CP + kh * 8);
      mma16816(acc[0], a, wf[(tap * 2 + 0) * 2], wf[(tap * 2 + 0) * 2 + 1]);
      mma16816(acc[1], a, wf[(tap * 2 + 1) * 2], wf[(tap * 2 + 1) * 2 + 1]);
    }
  }
}

constexpr int TH = 8, TW = 32;            // output tile of the C x C kernels
constexpr int kWarps = 4;                 // 16 strips of 16 pixels, 4 per warp

// y = x + K (s * x)   (Eq. heteroresnet), one layer of ResNetDown / ResNetUp.
template <int CP>
__global__ void __launch_bounds__(kWarps * 32) resnet_mma_kernel(const bf16* __restrict__ x, const bf16* __restrict__ s,
                                                                 const uint32_t* __restrict__ frag,
                                                                 bf16* __restrict__ y, int n) {
  constexpr int PH = TH + 2, PW = TW + 2, NV = CP / 8;
  constexpr int NREG = (CP == 8) ? 9 : 36;
  __shared__ __align__(16) bf16 zs[PH * PW * CP];
  __shared__ __align__(16) bf16 xs[PH * PW * CP];
  const int j0 = blockIdx.y * TH, i0 = blockIdx.x * TW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t wf[NREG];
#pragma unroll
  for (int k = 0; k < NREG; ++k) wf[k] = frag[k * 32 + lane];
  for (int idx = threadIdx.x; idx < PH * PW; idx += blockDim.x) {
    const int pr = idx / PW, pc = idx - pr * PW;
    const int gj = j0 + pr - 1, gi = i0 + pc - 1;
    uint4* zd = reinterpret_cast<uint4*>(zs + (size_t)idx * CP);
    uint4* xd = reinterpret_cast<uint4*>(xs + (size_t)idx * CP);
    if (gj >= 0 && gj < n && gi >= 0 && gi < n) {
      const size_t q = ((size_t)gj * n + gi) * CP;
      const uint4* xp = reinterpret_cast<const uint4*>(x + q);
      const uint4* sp = reinterpret_cast<const uint4*>(s + q);
#pragma unroll
      for (int h = 0; h < NV; ++h) {
        const uint4 xv = xp[h];
        xd[h] = xv;
        zd[h] = mul_bf16x8(xv, sp[h]);
      }
    } else {
#pragma unroll
      for (int h = 0; h < NV; ++h) xd[h] = zd[h] = make_uint4(0, 0, 0, 0);
    }
  }
  __syncthreads();
  const int g = lane >> 2, q = lane & 3;
  for (int st = warp; st < 2 * TH; st += kWarps) {
    const int r = st >> 1, col0 = (st & 1) * 16;
    float acc[2][4] = {};
    warp_conv<CP>(zs, wf, [&](int m, int tap) { return (r + tap / 3) * PW + (col0 + m + tap % 3); }, acc);
    const int gj = j0 + r;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int px = col0 + g + 8 * half;
      const int gi = i0 + px;
      if (gj >= n || gi >= n) continue;
#pragma unroll
      for (int t = 0; t < CP / 8; ++t) {
        const int ch = 8 * t + 2 * q;
        const float2 xv = __bfloat1622float2(*reinterpret_cast<const bf162*>(xs + ((size_t)(r + 1) * PW + px + 1) * CP + ch));
        const bf162 o = __floats2bfloat162_rn(xv.x + acc[t][2 * half], xv.y + acc[t][2 * half + 1]);
        *reinterpret_cast<bf162*>(y + ((size_t)gj * n + gi) * CP + ch) = o;
      }
    }
  }
}

// RCNN: y[J][I] = sum_tap W x[2J+a][2I+b] (stride 2, no padding).
template <int CP>
__global__ void __launch_bounds__(kWarps * 32) rcnn_mma_kernel(const bf16* __restrict__ x, const uint32_t* __restrict__ frag,
                                                               bf16* __restrict__ y, int n) {
  constexpr int FH = 2 * TH + 1, FW = 2 * TW + 1, NV = CP / 8;
  constexpr int NREG = (CP == 8) ? 9 : 36;
  __shared__ __align__(16) bf16 xs[FH * FW * CP];
  const int nc = (n - 1) / 2;
  const int J0 = blockIdx.y * TH, I0 = blockIdx.x * TW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t wf[NREG];
#pragma unroll
  for (int k = 0; k < NREG; ++k) wf[k] = frag[k * 32 + lane];
  for (int idx = threadIdx.x; idx < FH * FW; idx += blockDim.x) {
    const int pr = idx / FW, pc = idx - pr * FW;
    const int gj = 2 * J0 + pr, gi = 2 * I0 + pc;
    uint4* xd = reinterpret_cast<uint4*>(xs + (size_t)idx * CP);
    if (gj < n && gi < n) {
      const uint4* xp = reinterpret_cast<const uint4*>(x + ((size_t)gj * n + gi) * CP);
#pragma unroll
      for (int h = 0; h < NV; ++h) xd[h] = xp[h];
    } else {
#pragma unroll
      for (int h = 0; h < NV; ++h) xd[h] = make_uint4(0, 0, 0, 0);
    }
  }
  __syncthreads();
  const int g = lane >> 2, q = lane & 3;
  for (int st = warp; st < 2 * TH; st += kWarps) {
    const int r = st >> 1, col0 = (st & 1) * 16;
    float acc[2][4] = {};
    warp_conv<CP>(xs, wf, [&](int m, int tap) { return (2 * r + tap / 3) * FW + 2 * (col0 + m) + tap % 3; }, acc);
    const int J = J0 + r;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int I = I0 + col0 + g + 8 * half;
      if (J >= nc || I >= nc) continue;
#pragma unroll
      for (int t = 0; t < CP / 8; ++t) {
        const int ch = 8 * t + 2 * q;
        *reinterpret_cast<bf162*>(y + ((size_t)J * nc + I) * CP + ch) =
            __floats2bfloat162_rn(acc[t][2 * half], acc[t][2 * half + 1]);
      }
    }
  }
}

// y_fine += TCNN(x_coarse), gather form, FP32 accumulate.  W: [ci][co][9] FP32, padded.
template <int CP>
__global__ void __launch_bounds__(128) tcnn_add_kernel16(const bf16* __restrict__ xc, const float* __restrict__ W,
                                                         bf16* __restrict__ y, int n) {
  const int nc = (n - 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  const int j = p / n, i = p - j * n;
  float acc[CP];
#pragma unroll
  for (int co = 0; co < CP; ++co) acc[co] = 0.f;
  for (int ta = 0; ta < 3; ++ta) {
    const int dj = j - ta;
    if (dj < 0 || (dj & 1) || (dj >> 1) >= nc) continue;
    for (int tb = 0; tb < 3; ++tb) {
      const int di = i - tb;
      if (di < 0 || (di & 1) || (di >> 1) >= nc) continue;
      const bf16* xq = xc + ((size_t)(dj >> 1) * nc + (di >> 1)) * CP;
      const int tap = ta * 3 + tb;
#pragma unroll
      for (int ci = 0; ci < CP; ci += 2) {
        const float2 v = __bfloat1622float2(*reinterpret_cast<const bf162*>(xq + ci));
#pragma unroll
        for (int co = 0; co < CP; ++co)
          acc[co] += W[(ci * CP + co) * 9 + tap] * v.x + W[((ci + 1) * CP + co) * 9 + tap] * v.y;
      }
    }
  }
  bf16* yp = y + (size_t)p * CP;
#pragma unroll
  for (int co = 0; co < CP; co += 2) {
    const float2 v = __bfloat1622float2(*reinterpret_cast<const bf162*>(yp + co));
    *reinterpret_cast<bf162*>(yp + co) = __floats2bfloat162_rn(v.x + acc[co], v.y + acc[co + 1]);
  }
}

// x_1 = alpha * W_in * r  (reChannelCNN 1 -> C), FP32 math, BF16 out.
template <int CP>
__global__ void __launch_bounds__(128) in_kernel16(const float* __restrict__ r, const double* __restrict__ norm2,
                                                   const float* __restrict__ W, bf16* __restrict__ x, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  const int j = p / n, i = p - j * n;
  const float alpha = (float)alpha_from(norm2, (size_t)n * n);
  float rv[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int jj = j + t / 3 - 1, ii = i + t % 3 - 1;
    rv[t] = (jj >= 0 && jj < n && ii >= 0 && ii < n) ? r[(size_t)jj * r32_pitch(n) + ii] : 0.f;
  }
  bf16* xp = x + (size_t)p * CP;
#pragma unroll
  for (int co = 0; co < CP; co += 2) {
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      a0 += W[co * 9 + t] * rv[t];
      a1 += W[(co + 1) * 9 + t] * rv[t];
    }
    *reinterpret_cast<bf162*>(xp + co) = __floats2bfloat162_rn(alpha * a0, alpha * a1);
  }
}

// e = (W_out * x_1) / alpha  (reChannelCNN C -> 1) in FP32; out = u + e in FP64.
template <int CP>
__global__ void __launch_bounds__(128) out_kernel16(const bf16* __restrict__ x, const float* __restrict__ W,
                                                    const double* __restrict__ norm2, const double* __restrict__ u,
                                                    double* __restrict__ out, int n) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n * n) return;
  const int j = p / n, i = p - j * n;
  float acc = 0.f;
  for (int t = 0; t < 9; ++t) {
    const int jj = j + t / 3 - 1, ii = i + t % 3 - 1;
    if (jj < 0 || jj >= n || ii < 0 || ii >= n) continue;
    const bf16* xq = x + ((size_t)jj * n + ii) * CP;
#pragma unroll
    for (int ci = 0; ci < CP; ci += 2) {
      const float2 v = __bfloat1622float2(*reinterpret_cast<const bf162*>(xq + ci));
      acc += W[ci * 9 + t] * v.x + W[(ci + 1) * 9 + t] * v.y;
    }
  }
  const double e = (double)acc / alpha_from(norm2, (size_t)n * n);
  out[p] = u ? u[p] + e : e;
}

// [N][C] float/double -> [N][CP] BF16 (zero padded), and back.
template <typename S>
__global__ void pad_to_bf16_kernel(const S* __restrict__ src, bf16* __restrict__ dst, size_t N, int C, int cp) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N * cp) return;
  const size_t pix = p / cp;
  const int ch = (int)(p - pix * cp);
  dst[p] = __float2bfloat16_rn(ch < C ? (float)src[pix * C + ch] : 0.f);
}

__global__ void unpad_bf16_kernel(const bf16* __restrict__ src, double* __restrict__ dst, size_t N, int C, int cp) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N * C) return;
  const size_t pix = p / C;
  const int ch = (int)(p - pix * C);
  dst[p] = (double)__bfloat162float(src[pix * cp + ch]);
}

// dst (row pitch r32_pitch(n)) = FP32 src (times scale)
__global__ void to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, int n,
                              const float* __restrict__ scale) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (size_t)n * n) return;
  const int j = (int)(p / n), i = (int)(p - (size_t)j * n);
  dst[(size_t)j * r32_pitch(n) + i] = scale ? (float)src[p] * scale[p] : (float)src[p];
}

template <int CP>
Status vcycle_cp(mgcnn_ctx* c, const float* r32, const double* norm2, double* e, const double* u_skip) {
  const MixLayout ml = mix_layout(c);
  const char* wb = c->wmix.as<char>();
  const uint32_t* f_down = reinterpret_cast<const uint32_t*>(wb + ml.down);
  const uint32_t* f_up = reinterpret_cast<const uint32_t*>(wb + ml.up);
  const uint32_t* f_R = reinterpret_cast<const uint32_t*>(wb + ml.R);
  const float* w_in = reinterpret_cast<const float*>(wb + ml.w_in);
  const float* w_out = reinterpret_cast<const float*>(wb + ml.w_out);
  const float* w_P = reinterpret_cast<const float*>(wb + ml.w_P);
  if (CP == 8 && c->fused && fused_supported(c))
    return vcycle_fused_cp8(c, r32, norm2, e, u_skip, fused_weights(c));
  bf16* x[kMaxLevels];
  bf16* t[kMaxLevels];
  for (int l = 0; l < c->L; ++l) {
    x[l] = c->x16a[l].as<bf16>();
    t[l] = c->x16b[l].as<bf16>();
  }
  cudaStream_t st = c->stream;
  const int n0 = c->lv[0].n;
  int ps = prof_begin(c, kProfIn);
  in_kernel16<CP><<<grid_for((size_t)n0 * n0, 128), 128, 0, st>>>(r32, norm2, w_in, x[0], n0);
  MG_LAUNCH("in_kernel16");
  prof_end(c, ps);
  for (int l = 0; l < c->L; ++l) {
    const int nl = c->lv[l].n;
    const dim3 grid((nl + TW - 1) / TW, (nl + TH - 1) / TH);
    for (int i = 0; i < c->wl.nu_d; ++i) {
      ps = (l == 0) ? prof_begin(c, kProfResnet) : -1;
      resnet_mma_kernel<CP><<<grid, kWarps * 32, 0, st>>>(x[l], c->s16[l].as<bf16>(), f_down + i * ml.frag_words, t[l], nl);
      MG_LAUNCH("resnet_mma_kernel(down)");
      prof_end(c, ps);
      std::swap(x[l], t[l]);
    }
    if (l < c->L - 1) {
      const int nc = c->lv[l + 1].n;
      const dim3 g2((nc + TW - 1) / TW, (nc + TH - 1) / TH);
      ps = (l == 0) ? prof_begin(c, kProfRestrict) : -1;
      rcnn_mma_kernel<CP><<<g2, kWarps * 32, 0, st>>>(x[l], f_R, x[l + 1], nl);
      MG_LAUNCH("rcnn_mma_kernel");
      prof_end(c, ps);
    }
  }
  for (int l = c->L - 1; l >= 0; --l) {
    const int nl = c->lv[l].n;
    const dim3 grid((nl + TW - 1) / TW, (nl + TH - 1) / TH);
    for (int i = 0; i < c->wl.nu_u; ++i) {
      ps = (l == 0) ? prof_begin(c, kProfResnet) : -1;
      resnet_mma_kernel<CP><<<grid, kWarps * 32, 0, st>>>(x[l], c->s16[l].as<bf16>(), f_up + i * ml.frag_words, t[l], nl);
      MG_LAUNCH("resnet_mma_kernel(up)");
      prof_end(c, ps);
      std::swap(x[l], t[l]);
    }
    if (l > 0) {
      const int nf = c->lv[l - 1].n;
      ps = (l == 1) ? prof_begin(c, kProfProlong) : -1;
      tcnn_add_kernel16<CP><<<grid_for((size_t)nf * nf, 128), 128, 0, st>>>(x[l], w_P, x[l - 1], nf);
      MG_LAUNCH("tcnn_add_kernel16");
      prof_end(c, ps);
    }
  }
  ps = prof_begin(c, kProfOut);
  out_kernel16<CP><<<grid_for((size_t)n0 * n0, 128), 128, 0, st>>>(x[0], w_out, norm2, u_skip, e, n0);
  MG_LAUNCH("out_kernel16");
  prof_end(c, ps);
  return {};
}

}  // namespace

FusedWeights fused_weights(const mgcnn_ctx* c) {
  const MixLayout ml = mix_layout(c);
  const char* wb = c->wmix.as<char>();
  return FusedWeights{reinterpret_cast<const uint32_t*>(wb + ml.down), reinterpret_cast<const uint32_t*>(wb + ml.up),
                      reinterpret_cast<const uint32_t*>(wb + ml.R), reinterpret_cast<const uint32_t*>(wb + ml.out_taps),
                      reinterpret_cast<const uint32_t*>(wb + ml.tcnn),
                      c->small_w, c->out_lo};
}

Status mixed_set_weights(mgcnn_ctx* c) {
  if (c->cfg.precision != MGCNN_PREC_MIXED_BF16) return {};
  const int C = c->cfg.channels;
  c->cp = padded_channels(C);
  const MixLayout ml = mix_layout(c);
  std::vector<double> w(c->wl.total);
  MG_CUDA(cudaMemcpyAsync(w.data(), c->w64.p, w.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MG_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<char> blob(ml.bytes, 0);
  const size_t CC9 = (size_t)C * C * 9;
  for (int i = 0; i < c->wl.nu_d; ++i)
    pack_frags(w.data() + c->wl.w_down + i * CC9, C, ml.cp, reinterpret_cast<uint32_t*>(blob.data() + ml.down) + i * ml.frag_words);
  for (int i = 0; i < c->wl.nu_u; ++i)
    pack_frags(w.data() + c->wl.w_up + i * CC9, C, ml.cp, reinterpret_cast<uint32_t*>(blob.data() + ml.up) + i * ml.frag_words);
  pack_frags(w.data() + c->wl.w_R, C, ml.cp, reinterpret_cast<uint32_t*>(blob.data() + ml.R));
  float* win = reinterpret_cast<float*>(blob.data() + ml.w_in);
  float* wout = reinterpret_cast<float*>(blob.data() + ml.w_out);
  float* wP = reinterpret_cast<float*>(blob.data() + ml.w_P);
  for (int co = 0; co < C; ++co)
    for (int t = 0; t < 9; ++t) {
      win[co * 9 + t] = (float)w[c->wl.w_in + co * 9 + t];
      wout[co * 9 + t] = (float)w[c->wl.w_out + co * 9 + t];
    }
  for (int ci = 0; ci < C; ++ci)
    for (int co = 0; co < C; ++co)
      for (int t = 0; t < 9; ++t) wP[(ci * ml.cp + co) * 9 + t] = (float)w[c->wl.w_P + ((size_t)ci * C + co) * 9 + t];
  if (ml.cp == 8) {
    // W_out as an 8 -> 8 layer with output channel 0 only, split into BF16 hi + lo
    std::vector<double> whi(8 * 8 * 9, 0.0), wlo(8 * 8 * 9, 0.0);
    for (int ci = 0; ci < C; ++ci)
      for (int t = 0; t < 9; ++t) {
        const float v = (float)w[c->wl.w_out + ci * 9 + t];
        const uint32_t hb = (uint32_t)f2bf_host(v) << 16;
        float hi;
        std::memcpy(&hi, &hb, 4);
        whi[ci * 9 + t] = hi;
        wlo[ci * 9 + t] = (double)(v - hi);
      }
    c->out_lo = 0;
    for (double v : wlo) c->out_lo |= (v != 0.0);
    pack_out_taps(whi, wlo, reinterpret_cast<uint32_t*>(blob.data() + ml.out_taps));
    pack_tcnn_frags(w.data() + c->wl.w_P, C, reinterpret_cast<uint32_t*>(blob.data() + ml.tcnn));
    // W_in of the fused down kernel, zero beyond C channels
    SmallWeights& sw = c->small_w;
    sw = SmallWeights{};
    for (int t = 0; t < 9; ++t)
      for (int ch = 0; ch < C; ++ch) sw.w_in[t * 8 + ch] = (float)w[c->wl.w_in + ch * 9 + t];
  }
  if (C == 8) {
    // fused setup network: 4 tanh layers and the setup RCNN as fragments; b_i, W_cin, b_cin in FP32
    uint32_t* sf = reinterpret_cast<uint32_t*>(blob.data() + ml.s_frag);
    for (int i = 0; i < kSetupLayers; ++i) pack_frags(w.data() + c->wl.sw + i * CC9, C, ml.cp, sf + i * ml.frag_words);
    pack_frags(w.data() + c->wl.sw_R, C, ml.cp, sf + 4 * ml.frag_words);
    float* sp = reinterpret_cast<float*>(blob.data() + ml.s_fp);
    for (int i = 0; i < 4 * 8; ++i) sp[i] = (float)w[c->wl.sb + i];
    for (int i = 0; i < 8 * kFeatures * 9; ++i) sp[32 + i] = (float)w[c->wl.sw_in + i];
    for (int i = 0; i < 8; ++i) sp[32 + 8 * kFeatures * 9 + i] = (float)w[c->wl.sb_in + i];
    static_assert(32 + 8 * kFeatures * 9 + 8 == sizeof(SetupSmallWeights) / sizeof(float), "setup small weights");
    std::copy(sp, sp + 400, c->setup_small_w.v);
  }
  MG_TRY(ensure(c->wmix, ml.bytes));
  MG_CUDA(cudaMemcpyAsync(c->wmix.p, blob.data(), ml.bytes, cudaMemcpyHostToDevice, c->stream));
  MG_CUDA(cudaStreamSynchronize(c->stream));
  return {};
}

SetupWeights setup_weights(const mgcnn_ctx* c) {
  const MixLayout ml = mix_layout(c);
  const char* wb = c->wmix.as<char>();
  return SetupWeights{reinterpret_cast<const uint32_t*>(wb + ml.s_frag), c->setup_small_w};
}

Status setup_mixed(mgcnn_ctx* c) {
  const int C = c->cfg.channels;
  const int cp = c->cp;
  if (C == 8 && c->fused) {
    // one fused kernel per level; coef_l (l >= 1) is kept in the level's second state buffer
    const double* ops[kMaxLevels];
    bf16* ss[kMaxLevels];
    bf16* cs[kMaxLevels];
    int ns[kMaxLevels];
    for (int l = 0; l < c->L; ++l) {
      const size_t N = c->lv[l].N();
      MG_TRY(ensure(c->s16[l], N * cp * sizeof(bf16)));
      MG_TRY(ensure(c->x16a[l], N * cp * sizeof(bf16)));
      MG_TRY(ensure(c->x16b[l], N * cp * sizeof(bf16)));
      if (l > 0) MG_TRY(ensure(c->x16l[l], N * cp * sizeof(bf16)));
      ops[l] = c->op[l].as<double>();
      ss[l] = c->s16[l].as<bf16>();
      cs[l] = c->x16b[l].as<bf16>();
      ns[l] = c->lv[l].n;
    }
    MG_TRY(ensure(c->r32, r32_floats(c->lv[0].n) * sizeof(float)));
    const SetupWeights sw = setup_weights(c);
    return setup_fused_levels(c->L, ns, 1, ops, ss, cs, sw, c->cfg.scale_by_diag, c->stream);
  }
  size_t total = 0;
  for (int l = 0; l < c->L; ++l) total += c->lv[l].N() * C;
  MG_TRY(ensure(c->s32tmp, total * sizeof(float)));
  float* outs[kMaxLevels];
  size_t off = 0;
  for (int l = 0; l < c->L; ++l) {
    outs[l] = c->s32tmp.as<float>() + off;
    off += c->lv[l].N() * C;
    MG_TRY(ensure(c->s16[l], c->lv[l].N() * cp * sizeof(bf16)));
    MG_TRY(ensure(c->x16a[l], c->lv[l].N() * cp * sizeof(bf16)));
    MG_TRY(ensure(c->x16b[l], c->lv[l].N() * cp * sizeof(bf16)));
    if (l > 0) MG_TRY(ensure(c->x16l[l], c->lv[l].N() * cp * sizeof(bf16)));
  }
  MG_TRY(ensure(c->r32, r32_floats(c->lv[0].n) * sizeof(float)));
  MG_TRY(run_setup_net_fp32(c, outs));
  for (int l = 0; l < c->L; ++l) {
    const size_t N = c->lv[l].N();
    pad_to_bf16_kernel<float><<<grid_for(N * cp, 256), 256, 0, c->stream>>>(outs[l], c->s16[l].as<bf16>(), N, C, cp);
    MG_LAUNCH("pad_to_bf16_kernel");
  }
  return {};
}

Status pad_setup_bf16(const float* src, bf16* dst, size_t N, int C, int cp, cudaStream_t st) {
  pad_to_bf16_kernel<float><<<grid_for(N * cp, 256), 256, 0, st>>>(src, dst, N, C, cp);
  MG_LAUNCH("pad_to_bf16_kernel");
  return {};
}

Status mixed_gmg_setup_level(mgcnn_ctx* c, int l, double omega) {
  const size_t N = c->lv[l].N();
  const int cp = c->cp;
  MG_TRY(ensure(c->s16[l], N * cp * sizeof(bf16)));
  MG_TRY(ensure(c->x16a[l], N * cp * sizeof(bf16)));
  MG_TRY(ensure(c->x16b[l], N * cp * sizeof(bf16)));
  if (l > 0) MG_TRY(ensure(c->x16l[l], N * cp * sizeof(bf16)));
  MG_TRY(ensure(c->r32, r32_floats(c->lv[0].n) * sizeof(float)));
  const int C = c->cfg.channels;
  if (C == kGmgV10Channels)   // straight into the BF16 layout
    return launch_gmg_v10_setup_bf16(c->op[l].as<double>(), c->s16[l].as<bf16>(), c->lv[l].n, omega, c->stream,
                                     l == 0 && c->cfg.input_diag);
  MG_TRY(ensure(c->setup_a, N * C * sizeof(double)));
  MG_TRY(launch_gmg_setup(c->op[l].as<double>(), c->setup_a.as<double>(), c->lv[l].n, omega, c->stream,
                          l == 0 && c->cfg.input_diag, C));
  pad_to_bf16_kernel<double><<<grid_for(N * cp, 256), 256, 0, c->stream>>>(c->setup_a.as<double>(),
                                                                            c->s16[l].as<bf16>(), N, C, cp);
  MG_LAUNCH("pad_to_bf16_kernel");
  return {};
}

Status mixed_set_setup_level(mgcnn_ctx* c, int l, const double* src) {
  const size_t N = c->lv[l].N();
  pad_to_bf16_kernel<double><<<grid_for(N * c->cp, 256), 256, 0, c->stream>>>(src, c->s16[l].as<bf16>(), N,
                                                                                c->cfg.channels, c->cp);
  MG_LAUNCH("pad_to_bf16_kernel");
  return {};
}

Status mixed_get_setup_level(mgcnn_ctx* c, int l, double* dst) {
  const size_t N = c->lv[l].N();
  const int C = c->cfg.channels;
  unpad_bf16_kernel<<<grid_for(N * C, 256), 256, 0, c->stream>>>(c->s16[l].as<bf16>(), dst, N, C, c->cp);
  MG_LAUNCH("unpad_bf16_kernel");
  return {};
}

Status vcycle_mixed_r32(mgcnn_ctx* c, const float* r32, const double* norm2_dev, double* e, const double* u_skip) {
  if (c->cp == 8) return vcycle_cp<8>(c, r32, norm2_dev, e, u_skip);
  return vcycle_cp<16>(c, r32, norm2_dev, e, u_skip);
}

Status vcycle_mixed(mgcnn_ctx* c, const double* r, double* e, const double* u_skip) {
  const size_t N = c->lv[0].N();
  to_f32_kernel<<<grid_for(N, 256), 256, 0, c->stream>>>(r, c->r32.as<float>(), c->lv[0].n,
                                                         c->cfg.input_diag ? c->dinv32.as<float>() : nullptr);
  MG_LAUNCH("to_f32_kernel");
  double* norm2 = c->scalars.as<double>() + 2;
  MG_TRY(launch_sumsq(r, N, c->partial.as<double>(), c->stream));
  MG_TRY(launch_reduce(c->partial.as<double>(), residual_blocks(N), norm2, c->stream));
  return vcycle_mixed_r32(c, c->r32.as<float>(), norm2, e, u_skip);
}

void mixed_release(mgcnn_ctx* c) {
  for (int l = 0; l < kMaxLevels; ++l) {
    release(c->x16a[l]);
    release(c->x16b[l]);
    release(c->x16l[l]);
  }
  release(c->wmix);
  release(c->s32tmp);
}

}  // namespace mgcnn

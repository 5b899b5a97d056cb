// Fused setup phase (Algorithm 2) for 8 channels: one kernel per level.
//
// Level l:  z_0 = coef_l;  z_{i+1} = tanh(K_i z_i + b_i) + z_i  (i = 0..3, Eq.
// resnet_nonlinear);  setup_out_l = z_4 * scale_l;  coef_{l+1} = RCNN_s(coef_l)
// (Eq. setup1).  At the finest level coef_1 = W_cin * features + b_cin is
// formed from the operator in the same kernel (features: [a_W, a_E, a_S, a_N]/a_C
// and log10(h^2 a_C)).
//
// A block owns a 16 x 32 fine tile.  The four layers shrink a 4-pixel halo of
// coef_l one pixel per layer (24 x 40 -> 22 x 38 -> 20 x 36 -> 18 x 34 -> 16 x 32);
// z stays in FP32 in shared memory for the skip sum and tanh, a BF16 copy feeds
// the tensor cores (mma.m16n8k16 + m16n8k8, FP32 accumulation).  The restriction
// reads the 17 x 33 corner of the staged coef_l.  coef_l is stored in BF16
// between levels.  Output: BF16 setup tensor [N][8] and BF16 coef_{l+1}.
#include <cmath>

#include "mixed.cuh"
#include "ops.cuh"

namespace mgcnn {

using bf16 = __nv_bfloat16;
using bf162 = __nv_bfloat162;

namespace {

constexpr int SH = 16, SW = 32;        // owned fine tile
constexpr int HALO = kSetupLayers;     // one pixel per layer
constexpr int NT = 256, NW = NT / 32;
constexpr int CH0 = SH + 2 * HALO, CW0 = SW + 2 * HALO;   // staged coef tile 24 x 40

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
__device__ __forceinline__ uint32_t f2bf(float a, float b) {
  bf162 r = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&r);
}

template <typename Pix>
__device__ __forceinline__ void strip_conv(const uint4* tile, const uint32_t* wf, Pix pix, float* acc) {
  const int lane = threadIdx.x & 31;
  const int m = (lane & 7) + ((lane >> 3) & 1) * 8;
  const int kh = lane >> 4;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    uint32_t a[4];
    ldsm_x4(a, tile + pix(m, 2 * s + kh));
    mma16816(acc, a, wf[2 * s], wf[2 * s + 1]);
  }
  uint32_t a[2];
  ldsm_x2(a, tile + pix(lane & 15, 8));
  mma1688(acc, a[0], a[1], wf[8]);
}

struct SetupSmem {
  float zf[2][CH0 * CW0][8];   // FP32 z, ping-pong between layers
  uint4 zb[2][CH0 * CW0];      // BF16 copy of z (tensor-core operand)
};

// frags: 5 packed B-fragment blocks (4 setup layers, setup RCNN), 9 x 32 words each.
// sw: FP32 small weights by value (b_i [4][8], W_cin [8][5][9], b_cin [8]).
template <bool FIRST, bool HAS_R>
__global__ void __launch_bounds__(NT) setup_level_kernel(const double* __restrict__ op, const bf16* __restrict__ cin,
                                                         const uint32_t* __restrict__ frags,
                                                         const __grid_constant__ SetupSmallWeights sw, int mode,
                                                         float lscale, bf16* __restrict__ sout,
                                                         bf16* __restrict__ cout, int n) {
  const float* fp = sw.v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SetupSmem& sm = *reinterpret_cast<SetupSmem*>(smem_raw);
  const int j0 = blockIdx.y * SH, i0 = blockIdx.x * SW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t N = (size_t)n * n;
  const size_t bz = blockIdx.z;   // problem of a batch stored back to back
  op += bz * 5 * N;
  if (!FIRST) cin += bz * N * 8;
  sout += bz * N * 8;
  if (HAS_R) cout += bz * (size_t)((n - 1) / 2) * ((n - 1) / 2) * 8;

  // finest level: the five features once per pixel of the 26 x 42 region under
  // the staged tile, in FP32 (they feed a BF16 network), into the second z
  // buffer, which the first layer overwrites only later; zero outside the grid,
  // where W_cin's zero padding leaves them out of the sum
  constexpr int FH = CH0 + 2, FW = CW0 + 2;
  static_assert(FH * FW * kFeatures <= CH0 * CW0 * 8, "feature staging");
  float* fts = &sm.zf[1][0][0];
  if constexpr (FIRST) {
    const float np1 = (float)(n + 1);
    const float h2 = 1.0f / (np1 * np1);
    for (int e = threadIdx.x; e < FH * FW; e += NT) {
      const int r = e / FW, c = e - r * FW;
      const int gj = j0 + r - HALO - 1, gi = i0 + c - HALO - 1;
      float ft[kFeatures] = {0.f, 0.f, 0.f, 0.f, 0.f};
      if (gj >= 0 && gj < n && gi >= 0 && gi < n) {
        const size_t q = (size_t)gj * n + gi;
        const float aC = (float)op[q];
        const float inv = 1.0f / aC;
        ft[0] = (float)op[N + q] * inv;
        ft[1] = (float)op[2 * N + q] * inv;
        ft[2] = (float)op[3 * N + q] * inv;
        ft[3] = (float)op[4 * N + q] * inv;
        ft[4] = log10f(h2 * aC);
      }
#pragma unroll
      for (int fi = 0; fi < kFeatures; ++fi) fts[e * kFeatures + fi] = ft[fi];
    }
    __syncthreads();
  }
  // stage coef_l on the 24 x 40 tile (zero outside the grid: zero padding)
  for (int e = threadIdx.x; e < CH0 * CW0; e += NT) {
    const int r = e / CW0, c = e - r * CW0;
    const int gj = j0 + r - HALO, gi = i0 + c - HALO;
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (gj >= 0 && gj < n && gi >= 0 && gi < n) {
      if constexpr (FIRST) {
        // coef_1 = W_cin * features + b_cin (taps outside the grid are zero)
        const float* wcin = fp + 32;
        const float* bcin = fp + 32 + 8 * 5 * 9;
#pragma unroll
        for (int co = 0; co < 8; ++co) v[co] = bcin[co];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          const float* ft = fts + ((r + t / 3) * FW + c + t % 3) * kFeatures;
#pragma unroll
          for (int co = 0; co < 8; ++co)
#pragma unroll
            for (int fi = 0; fi < 5; ++fi) v[co] += wcin[(co * 5 + fi) * 9 + t] * ft[fi];
        }
      } else {
        const uint4 cv = reinterpret_cast<const uint4*>(cin)[(size_t)gj * n + gi];
        const bf162* p2 = reinterpret_cast<const bf162*>(&cv);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 f = __bfloat1622float2(p2[k]);
          v[2 * k] = f.x;
          v[2 * k + 1] = f.y;
        }
      }
    }
#pragma unroll
    for (int co = 0; co < 8; ++co) sm.zf[0][e][co] = v[co];
    sm.zb[0][e] = make_uint4(f2bf(v[0], v[1]), f2bf(v[2], v[3]), f2bf(v[4], v[5]), f2bf(v[6], v[7]));
  }
  __syncthreads();
  const int g = lane >> 2, q = lane & 3;

  if constexpr (HAS_R) {
    // coef_{l+1} = RCNN_s(coef_l) from the staged BF16 coef (before the layers
    // reuse its buffer): coarse (J0 + cr, I0 + cc), taps (2 cr + a, 2 cc + b)
    uint32_t wr[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) wr[k] = frags[(4 * 9 + k) * 32 + lane];
    const int nc = (n - 1) / 2;
    const int J0 = blockIdx.y * (SH / 2), I0 = blockIdx.x * (SW / 2);
    for (int st = warp; st < (SH / 2) * (SW / 2) / 16; st += NW) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      strip_conv(sm.zb[0], wr, [&](int m, int tap) {
        const int p = st * 16 + m, cr = p / (SW / 2), cc = p % (SW / 2);
        return (2 * cr + tap / 3 + HALO) * CW0 + 2 * cc + tap % 3 + HALO;
      }, acc);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int p = st * 16 + g + 8 * hh, cr = p / (SW / 2), cc = p % (SW / 2);
        const int J = J0 + cr, I = I0 + cc;
        if (J < nc && I < nc)
          reinterpret_cast<uint32_t*>(cout + ((size_t)J * nc + I) * 8)[q] = f2bf(acc[2 * hh], acc[2 * hh + 1]);
      }
    }
    __syncthreads();
  }

  // four layers on a region that shrinks by one pixel per side per layer; the
  // region of layer i's output is (CH0 - 2(i+1)) x (CW0 - 2(i+1)), stored in the
  // same 24 x 40 indexing (offset i+1)
  for (int i = 0; i < kSetupLayers; ++i) {
    uint32_t wf[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) wf[k] = frags[(i * 9 + k) * 32 + lane];
    const float* bias = fp + i * 8;
    const int src = i & 1, dst = src ^ 1;
    const int off = i + 1, OH = CH0 - 2 * off, OW = CW0 - 2 * off;
    const int nstrip = (OH * OW + 15) / 16;
    for (int st = warp; st < nstrip; st += NW) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      strip_conv(sm.zb[src], wf, [&](int m, int tap) {
        int p = st * 16 + m;
        p = p < OH * OW ? p : OH * OW - 1;
        const int orow = p / OW + off, ocol = p % OW + off;
        return (orow + tap / 3 - 1) * CW0 + ocol + tap % 3 - 1;
      }, acc);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int p = st * 16 + g + 8 * hh;
        if (p >= OH * OW) continue;
        const int orow = p / OW + off, ocol = p % OW + off;
        const int e = orow * CW0 + ocol;
        const int gj = j0 + orow - HALO, gi = i0 + ocol - HALO;
        const bool in = gj >= 0 && gj < n && gi >= 0 && gi < n;
        const int ch = 2 * q;
        // zero outside the grid: the next layer's zero padding
        const float z0 = in ? tanhf(acc[2 * hh] + bias[ch]) + sm.zf[src][e][ch] : 0.f;
        const float z1 = in ? tanhf(acc[2 * hh + 1] + bias[ch + 1]) + sm.zf[src][e][ch + 1] : 0.f;
        sm.zf[dst][e][ch] = z0;
        sm.zf[dst][e][ch + 1] = z1;
        reinterpret_cast<uint32_t*>(&sm.zb[dst][e])[q] = f2bf(z0, z1);
      }
    }
    __syncthreads();
  }
  // setup_out = z_4 * scale on the owned tile (buffer 0 after four layers)
  for (int e = threadIdx.x; e < SH * SW; e += NT) {
    const int r = e / SW, c = e - r * SW;
    const int gj = j0 + r, gi = i0 + c;
    if (gj >= n || gi >= n) continue;
    const int t = (r + HALO) * CW0 + c + HALO;
    float sc = lscale;
    if (mode == 1) sc = 1.0f / (float)op[(size_t)gj * n + gi];
    const float* z = sm.zf[0][t];
    reinterpret_cast<uint4*>(sout)[(size_t)gj * n + gi] =
        make_uint4(f2bf(z[0] * sc, z[1] * sc), f2bf(z[2] * sc, z[3] * sc), f2bf(z[4] * sc, z[5] * sc),
                   f2bf(z[6] * sc, z[7] * sc));
  }
}

}  // namespace

size_t setup_fused_smem() { return sizeof(SetupSmem); }

// Algorithm 2 for `batch` problems of the same size: op[l] operators ([B][5][N_l]),
// s[l] setup tensors out ([B][N_l][8] BF16), coef[l] (l >= 1) BF16 coefficient
// storage ([B][N_l][8]).  mode / level scale as mgcnn_config.scale_by_diag.
Status setup_fused_levels(int L, const int* n, int batch, const double* const* op, __nv_bfloat16* const* s,
                          __nv_bfloat16* const* coef, const SetupWeights& w, int mode, cudaStream_t st) {
  const uint32_t* frags = w.frags;
  static bool attr_set = false;
  const size_t smem = sizeof(SetupSmem);
  if (!attr_set) {
    MG_CUDA(cudaFuncSetAttribute(setup_level_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MG_CUDA(cudaFuncSetAttribute(setup_level_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MG_CUDA(cudaFuncSetAttribute(setup_level_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MG_CUDA(cudaFuncSetAttribute(setup_level_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  for (int l = 0; l < L; ++l) {
    const bool first = l == 0, has_r = l + 1 < L;
    const dim3 grid((n[l] + SW - 1) / SW, (n[l] + SH - 1) / SH, batch);
    const float lscale = (mode == 2) ? (float)(1u << (2 * l)) : 1.0f;
    const bf16* cin = first ? nullptr : coef[l];
    bf16* cout = has_r ? coef[l + 1] : nullptr;
    if (first && has_r)
      setup_level_kernel<true, true><<<grid, NT, smem, st>>>(op[l], cin, frags, w.small, mode, lscale, s[l], cout, n[l]);
    else if (first)
      setup_level_kernel<true, false><<<grid, NT, smem, st>>>(op[l], cin, frags, w.small, mode, lscale, s[l], cout, n[l]);
    else if (has_r)
      setup_level_kernel<false, true><<<grid, NT, smem, st>>>(op[l], cin, frags, w.small, mode, lscale, s[l], cout, n[l]);
    else
      setup_level_kernel<false, false><<<grid, NT, smem, st>>>(op[l], cin, frags, w.small, mode, lscale, s[l], cout, n[l]);
    MG_LAUNCH("setup_level_kernel");
  }
  return {};
}

}  // namespace mgcnn

// Host side of the TMA tile loads: tensor-map encoding through the driver entry
// point (no link-time dependency on libcuda) and a per-context cache.
#include "tma.cuh"

namespace mgcnn {

namespace {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeFn>(p);
  }();
  return fn;
}

}  // namespace

const CUtensorMap* TmaMaps::pix8(const void* base, int n, int batch, int bw, int bh) {
  for (const Entry& e : entries_)
    if (e.kind == 0 && e.base == base && e.n == n && e.batch == batch && e.bw == bw && e.bh == bh) return &e.map;
  EncodeFn enc = encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || bw < 1 || bw > 256 || bh < 1 || bh > 256) return nullptr;
  Entry e{base, n, batch, bw, bh, 0, {}};
  const cuuint64_t dims[4] = {8, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)batch};
  const cuuint64_t strides[3] = {16, 16ull * n, 16ull * n * n};
  const cuuint32_t box[4] = {8, (cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  if (enc(&e.map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, elem,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return nullptr;
  if (entries_.size() >= 256) entries_.clear();   // bounded: maps are re-made on demand
  entries_.push_back(e);
  return &entries_.back().map;
}

const CUtensorMap* TmaMaps::f32(const void* base, int n, int pitch, int batch, int bw, int bh) {
  for (const Entry& e : entries_)
    if (e.kind == 1 && e.base == base && e.n == n && e.batch == batch && e.bw == bw && e.bh == bh) return &e.map;
  EncodeFn enc = encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || (pitch & 3) || pitch < n || (bw & 3) || bw < 4 ||
      bw > 256 || bh < 1 || bh > 256)
    return nullptr;
  Entry e{base, n, batch, bw, bh, 1, {}};
  const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {4ull * pitch, 4ull * pitch * n};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t elem[3] = {1, 1, 1};
  if (enc(&e.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, elem,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return nullptr;
  if (entries_.size() >= 256) entries_.clear();
  entries_.push_back(e);
  return &entries_.back().map;
}

}  // namespace mgcnn

namespace mgcnn {

namespace {

// Check of the bounded-wait path of the TMA tile loads: thread 0 arms an
// mbarrier for 16 bytes that no copy will ever deliver, every thread waits
// with at most `rounds` suspended tries (kMbarSuspendNs each), and a block that
// gives up records the error flag, exactly as the level kernels do.
__global__ void wait_check_kernel(int* err, int rounds) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16u);
  }
  __syncthreads();
  bool landed = false;
  for (int i = 0; i < rounds && !landed; ++i) landed = mbar_try_wait(&bar, 0);
  if (!__syncthreads_and(landed) && threadIdx.x == 0) atomicExch(err, 1);
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(&bar)) : "memory");
}

}  // namespace

Status launch_wait_check(int* err, int rounds, cudaStream_t st) {
  wait_check_kernel<<<1, 64, 0, st>>>(err, rounds);
  MG_LAUNCH("wait_check_kernel");
  return {};
}

}  // namespace mgcnn

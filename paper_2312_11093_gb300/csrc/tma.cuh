// Tensor-memory-accelerator (TMA) tile loads for the fused level kernels.
//
// The BF16 network tensors are stored pixel-major, 8 channels per pixel
// (16 bytes), problems of a batch back to back: as a TMA tensor that is
// {8 channels, n columns, n rows, batch} with byte strides {16, 16 n, 16 n^2}
// -- every stride a multiple of 16 bytes for any n, and the innermost box
// extent (8 BF16) exactly 16 bytes, so any pixel-aligned box can be copied.
// A box may start at a negative row or column (the halo of a tile at the grid
// edge): TMA fills the elements outside the tensor with zeros, which is the
// zero padding of Eq. conv.  The channel coordinate is always 0.
//
// A block waits for its copies on an mbarrier with an iteration limit; past
// it the kernel records an error in a device flag (read by the host after the
// call) and returns instead of waiting forever.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "common.cuh"

namespace mgcnn {

// Launches one block whose tile wait can never complete (no copy is issued):
// its bounded wait gives up after `rounds` suspended tries and sets *err.
Status launch_wait_check(int* err, int rounds, cudaStream_t st);

// Host: encoder and a small cache of tensor maps (base pointer, grid, batch, box).
class TmaMaps {
 public:
  // Map of a [batch][n][n][8] BF16 tensor with box bw x bh pixels; nullptr on failure.
  const CUtensorMap* pix8(const void* base, int n, int batch, int bw, int bh);
  // Map of a [batch][n][pitch] FP32 array (n x n values per problem, rows of
  // `pitch` floats, pitch a multiple of 4) with box bw x bh values; bw * 4 must
  // be a multiple of 16.
  const CUtensorMap* f32(const void* base, int n, int pitch, int batch, int bw, int bh);
  void clear() { entries_.clear(); }

 private:
  struct Entry {
    const void* base;
    int n, batch, bw, bh, kind;   // kind 0: pix8, 1: f32
    CUtensorMap map;
  };
  std::vector<Entry> entries_;
};

#ifdef __CUDACC__
// A waiting thread is suspended until the phase completes or kMbarSuspendNs
// pass (it issues nothing meanwhile); a block gives up after kMbarWaitLimit
// such rounds, about two seconds.
constexpr int kMbarWaitLimit = 2048;
constexpr uint32_t kMbarSuspendNs = 1000000;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(kMbarSuspendNs)
      : "memory");
  return ok != 0;
}

// true when the barrier's phase `parity` completed within the limit
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kMbarWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Box of the 3-D FP32 array at (column x, row y, problem z); x must be a
// multiple of 4 (16-byte aligned start).
__device__ __forceinline__ void tma_load_f32(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Box of the 4-D pixel tensor at (channel 0, column x, row y, problem z) into
// shared memory, completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_pix(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
#endif

}  // namespace mgcnn

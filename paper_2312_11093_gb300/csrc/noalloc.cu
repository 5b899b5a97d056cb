// Residual and norm for callers that cannot allocate device memory.
//
// mgcnn_residual_noalloc runs the same FP64 residual kernel and the same
// deterministic two-pass norm as the context-based mgcnn_residual, but its
// per-block partial sums live in a fixed array defined in this file instead of
// a buffer obtained from cudaMalloc.  Every GPU that loads the library keeps
// that array (kNoAllocMaxBlocks + 1 doubles, 64 KiB) until the process exits.
#include <mutex>

#include "ops.cuh"

namespace mgcnn {
namespace {

// Largest grid served: n^2 <= 16,777,216 unknowns (n <= 4096).  Each block of
// the residual kernel covers kResidualBlock * kResidualPix = 2048 unknowns and
// leaves one partial sum, so 8,192 partial sums suffice; the last slot receives
// the reduced sum.
constexpr size_t kNoAllocMaxUnknowns = 16777216;
constexpr int kNoAllocMaxBlocks = (int)(kNoAllocMaxUnknowns / ((size_t)kResidualBlock * kResidualPix));
static_assert(kNoAllocMaxUnknowns % ((size_t)kResidualBlock * kResidualPix) == 0, "whole residual blocks");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 1];

// Device address of g_noalloc_scratch per device.  In host code the array's name
// is only a host-side stand-in, so the address is looked up once per device
// (with that device current) and reused.
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

Status scratch_for_current_device(double** out) {
  int dev = 0;
  MG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return make_status(MGCNN_ERR_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    MG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return {};
}

}  // namespace
}  // namespace mgcnn

using namespace mgcnn;

extern "C" int mgcnn_residual_noalloc(const double* op, const double* f, const double* u, double* r, int n,
                                      double* norm2, void* stream) {
  if (!op || !f || !u || !r || n < 1) return MGCNN_ERR_ARG;
  // the bound is checked on the unknown count in size_t before any block count
  // is formed (those are int and would wrap for huge n)
  const size_t N = (size_t)n * (size_t)n;
  if (N > kNoAllocMaxUnknowns) return MGCNN_ERR_SIZE;
  if (residual_blocks(N) > kNoAllocMaxBlocks) return MGCNN_ERR_SIZE;
  for (const void* p : {(const void*)op, (const void*)f, (const void*)u, (const void*)r})
    if (!is_device_pointer(p)) return MGCNN_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Status s = [&]() -> Status {
    double* scratch = nullptr;
    MG_TRY(scratch_for_current_device(&scratch));
    // every block overwrites its partial sum and the reduction overwrites the
    // last slot, so nothing left by an earlier call needs clearing
    MG_TRY(launch_residual(f, u, op, r, nullptr, scratch, n, st));
    MG_TRY(launch_reduce(scratch, residual_blocks(N), scratch + kNoAllocMaxBlocks, st));
    if (norm2) MG_CUDA(cudaMemcpyAsync(norm2, scratch + kNoAllocMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, st));
    MG_CUDA(cudaStreamSynchronize(st));
    return {};
  }();
  return s.code;
}

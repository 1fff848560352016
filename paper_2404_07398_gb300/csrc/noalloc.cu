// ifilt_spectrum_noalloc: the spectrum computation of ifilt_spectrum with its
// device scratch in a fixed array of this library instead of memory taken
// from an allocator, for callers that must not allocate device memory during
// a call (see include/ifilt.h).
#include <atomic>
#include <mutex>

#include "internal.h"

namespace ifilt {
namespace {

constexpr int kMaxCols = 512;   // n_fields * n_k (and n_k) at most
constexpr int kBlocks = 128;    // partial sums per (field, k)
// layout: k [kMaxCols] | energy [kMaxCols] | spec [kMaxCols] | kmid [kMaxCols] | partial [kMaxCols * kBlocks]
constexpr size_t kScratchDoubles = 4 * (size_t)kMaxCols + (size_t)kMaxCols * kBlocks;

// 532 KB, resident on every device that loads the library until the process exits.
static __device__ __align__(256) double g_spectrum_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};  // device -> address of g_spectrum_scratch on that device

// The array's name in host code is only a host-side handle; its device
// address is looked up with that device current: on the first call on the
// device, and again on every call made outside a stream capture, so that an
// address cached before a device reset (which reloads the module) is never
// used.  Inside a capture the address cached by an earlier call is used.
double* scratch_address(int dev, cudaStream_t st) {
  if (dev < 0 || dev >= kMaxDevices) fail(IFILT_EINVAL, "device ordinal %d out of range", dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  IFILT_CUDA(cudaStreamIsCapturing(st, &cap));
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap != cudaStreamCaptureStatusNone) {
    if (!g_addr[dev])
      fail(IFILT_EINVAL, "the first ifilt_spectrum_noalloc call on device %d must come before any stream capture", dev);
    return g_addr[dev];
  }
  void* p = nullptr;
  IFILT_CUDA(cudaGetSymbolAddress(&p, g_spectrum_scratch));
  g_addr[dev] = static_cast<double*>(p);
  return g_addr[dev];
}

}  // namespace

size_t spectrum_noalloc_max_columns() { return kMaxCols; }

ifilt_status spectrum_noalloc(ifilt_mesh_s* m, int32_t F, int32_t K, const double* k, const double* filtered,
                              double* energy, double* spec, double* kmid, cudaStream_t st) {
  if ((int64_t)F * K > kMaxCols)
    fail(IFILT_EINVAL, "n_fields * n_k = %lld exceeds the fixed scratch of %d columns",
         (long long)F * K, kMaxCols);
  int dev = 0;
  IFILT_CUDA(cudaGetDevice(&dev));
  double* base = scratch_address(dev, st);
  double* k_dev = base;
  double* e_dev = base + kMaxCols;
  double* s_dev = base + 2 * kMaxCols;
  double* km_dev = base + 3 * kMaxCols;
  double* part = base + 4 * kMaxCols;
  // every scratch element the kernels read is written first in this call, so
  // nothing has to be cleared
  IFILT_CUDA(cudaMemcpyAsync(k_dev, k, (size_t)K * sizeof(double), cudaMemcpyHostToDevice, st));
  spectrum_device(m, F, K, k_dev, filtered, e_dev, s_dev, km_dev, part, kBlocks, st);
  IFILT_CUDA(cudaMemcpyAsync(energy, e_dev, (size_t)F * K * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (spec && K > 1)
    IFILT_CUDA(cudaMemcpyAsync(spec, s_dev, (size_t)F * (K - 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (kmid && K > 1)
    IFILT_CUDA(cudaMemcpyAsync(kmid, km_dev, (size_t)(K - 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  IFILT_CUDA(cudaStreamSynchronize(st));
  return IFILT_OK;
}

}  // namespace ifilt

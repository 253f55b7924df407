// Allocation-free entry point: first column of (T_M + sigma I)^{-1} with the
// divide-and-conquer scratch in a fixed, file-scope device array.
//
// For callers that must not allocate device memory once they are running:
// applications that reserve all GPU memory up front under a fixed budget,
// services that forbid allocation after initialisation, or code that shares a
// device whose memory is owned by another allocator.  The regular path
// (mgwr_create / mgwr_inverse_column) allocates its scratch with cudaMalloc.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/mgwr.h"
#include "mgwr_internal.h"

namespace {

// Largest M served (the smem FFT path's limit as well).
constexpr int kNoallocMaxM = 4096;
// Slot 0 holds sigma; the complex work area (3 M values) starts 32 bytes in.
constexpr int kSigmaSlots = 4;
constexpr size_t kScratchDoubles = kSigmaSlots + 6 * (size_t)kNoallocMaxM;  // 196,640 bytes

// Every device that loads this library holds this array until the process exits.
static __device__ __align__(256) double g_inverse_column_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, resolved once per
// device (the host-side symbol is only a stand-in and must not reach a kernel).
cudaError_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_inverse_column_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Writes sigma, passed by value, into its slot of the scratch array: no host
// buffer is involved, so the call stays stream-ordered and never waits for a
// pageable copy.
__global__ void k_store_sigma(double* slot, double sigma) { *slot = sigma; }

}  // namespace

extern "C" int mgwr_inverse_column_noalloc(const double* r_dev, int M, double sigma, double* k_dev,
                                           void* stream) {
  if (r_dev == nullptr || k_dev == nullptr) return MGWR_E_INVAL;
  if (M < 4 || (M & (M - 1)) != 0) return MGWR_E_INVAL;
  if (M > kNoallocMaxM) return MGWR_E_TOOBIG;
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) return MGWR_E_INVAL;
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return MGWR_E_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // sigma goes into its slot by a one-thread kernel on the caller's stream; the
  // work area needs no clearing (every entry is written before it is read
  // inside the kernel)
  k_store_sigma<<<1, 1, 0, s>>>(scratch, sigma);
  cudaError_t e = mgwr::counted(cudaGetLastError());
  if (e == cudaSuccess)
    e = mgwr::launch_inverse_columns(k_dev, r_dev, scratch, 1, M, 1,
                                     reinterpret_cast<mgwr::Cx<double>*>(scratch + kSigmaSlots), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MGWR_E_CUDA;
  }
  return MGWR_OK;
}

// Arithmetic peak probe: the FP64 and FP32 FMA throughput of the device, the
// denominators of the FP64- and FP32-issue rooflines (the HBM and bf16 ones
// come from measured copy and GEMM runs).  Every thread runs independent FMA
// chains; the probe tries 8 and 16 chains per thread at 4 and 8 blocks of 256
// threads per SM and reports the best, the shape that keeps the pipe busiest.
#include <cuda_runtime.h>

#include "../../include/mgwr.h"
#include "mgwr_internal.h"

namespace {

constexpr int kThreads = 256;

template <class T, int CHAINS>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, T b, T c, int iters) {
  T a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

// TFLOP/s of `flops_target` worth of FMA rounds at `per_sm` blocks per SM,
// timed with events on stream s after one untimed launch.
template <class T, int CHAINS>
int probe_shape(T* out, cudaStream_t s, int sms, int per_sm, double flops_target, double* tflops) {
  const int blocks = per_sm * sms;
  const double per_round = 2.0 * CHAINS * (double)blocks * kThreads;
  const int iters = (int)(flops_target / per_round) + 1;
  // b slightly below 1 and a small c keep every chain bounded
  const T b = (T)0.999999, c = (T)1e-6;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = MGWR_E_CUDA;
  float ms = 0.f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    k_fma_chains<T, CHAINS><<<blocks, kThreads, 0, s>>>(out, b, c, iters / 8 + 1);
    mgwr::counted(cudaGetLastError());
    cudaEventRecord(e0, s);
    k_fma_chains<T, CHAINS><<<blocks, kThreads, 0, s>>>(out, b, c, iters);
    mgwr::counted(cudaGetLastError());
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) == cudaSuccess &&
        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
      *tflops = per_round * iters / (ms * 1e-3) / 1e12;
      st = MGWR_OK;
    }
  }
  if (e0 != nullptr) cudaEventDestroy(e0);
  if (e1 != nullptr) cudaEventDestroy(e1);
  return st;
}

// best of the four shapes, each about flops_target of work
template <class T>
int probe(int sms, double flops_target, double* best) {
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)8 * sms * kThreads) != cudaSuccess) return MGWR_E_NOMEM;
  cudaStream_t s = nullptr;
  int st = MGWR_E_CUDA;
  *best = 0.0;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess) {
    for (int per_sm : {4, 8}) {
      double t8 = 0.0, t16 = 0.0;
      st = probe_shape<T, 8>(out, s, sms, per_sm, flops_target, &t8);
      if (st != MGWR_OK) break;
      st = probe_shape<T, 16>(out, s, sms, per_sm, flops_target, &t16);
      if (st != MGWR_OK) break;
      *best = t8 > *best ? t8 : *best;
      *best = t16 > *best ? t16 : *best;
    }
    cudaStreamDestroy(s);
  }
  cudaFree(out);
  return st;
}

}  // namespace

extern "C" int mgwr_peak_probe(double* fp64_tflops, double* fp32_tflops) {
  if (fp64_tflops == nullptr || fp32_tflops == nullptr) return MGWR_E_INVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return MGWR_E_CUDA;
  // about 0.2 s a shape on a GB300 (FP64 at 1/64 of the FP32 rate)
  const int st = probe<double>(sms, 2.5e11, fp64_tflops);
  if (st != MGWR_OK) return st;
  return probe<float>(sms, 1.6e13, fp32_tflops);
}

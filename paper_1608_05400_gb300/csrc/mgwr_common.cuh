// Device helpers and launch utilities shared by the kernel translation units
// of the MGWR library (point enumeration, neighbour lines, per-type arithmetic
// of the defect, reductions, launch geometry).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "mgwr_dd.cuh"
#include "mgwr_fft.cuh"
#include "mgwr_internal.h"

namespace mgwr {

// Minimum resident blocks per SM asked of the compiler (it sets the register
// cap), counted in butterfly slots (threads x E, E butterflies per thread):
// 1024 slots for the FP32 engine kernels (64 registers per slot), 768 for the
// FP64 / double-float ones (85 registers per slot at 256 threads per block).
template <class R>
constexpr int min_blocks(int block, int E = 1) {
  return sizeof(R) == 4 ? (1024 / (block * E) > 1 ? 1024 / (block * E) : 1)
                        : (768 / (block * E) > 1 ? 768 / (block * E) : 1);
}

// Threads per line pair: L/8.  Blocks hold 256 threads (several pairs) up to
// L = 2048 and one pair of L/8 threads beyond.
inline int block_threads(int L) { return L / 8 > 256 ? L / 8 : 256; }

inline int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

template <class K>
inline cudaError_t prepare_smem(K kernel, size_t smem) {
  if (smem > 48 * 1024) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  return cudaSuccess;
}

// Number of SMs of the current device (queried once per process).
inline int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      v = 152;
    }
    return v > 0 ? v : 152;
  }();
  return n;
}

// Threads per block for line pairs of TL (< 256) threads each: 256, halved
// (down to one warp, and not below TL) while the grid would give some SMs no
// block at all.  Short lines on small grids (coarse levels, small 1-D
// problems) then spread over the SMs instead of queueing up to 256 / TL pairs
// on one; the arithmetic of each pair is the same in every block size.
inline int spread_block(int TL, int npairs, int batch) {
  int block = 256;
  const long long sms = sm_count();
  while (block > 32 && block > TL &&
         (long long)((npairs + block / TL - 1) / (block / TL)) * batch < sms)
    block /= 2;
  return block;
}

inline unsigned elementwise_grid(size_t total) {
  size_t blocks = (total + 255) / 256;
  const size_t cap = 152 * 16;
  return (unsigned)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}


// FFT lengths with a compile-time specialisation (L = 2^7 .. 2^13, M = 64 ..
// 4096), used for FP32, where index arithmetic competes with the butterflies;
// the FP64 and double-float kernels are bound by their arithmetic and keep the
// run-time shape, which needs fewer registers.
#define MGWR_FIXED_LOGL(X) X(7) X(8) X(9) X(10) X(11) X(12) X(13)

// ---------------------------------------------------------------------------------
// point enumeration
// ---------------------------------------------------------------------------------

// Number of points of parity `par`: (i & 1) == par in 1-D, ((i + j) & 1) == par in 2-D.
__host__ __device__ __forceinline__ int colour_count(int d, int n, int par) {
  if (d == 1) return (n - par + 1) / 2;
  return ((n - 1) / 2) * n + (n - par + 1) / 2;
}

// k-th point of parity `par` in row-major order (p = i + n*j).
__device__ __forceinline__ int colour_point(int k, int d, int n, int par, int& i, int& j) {
  if (d == 1) {
    i = par + 2 * k;
    j = 0;
    return i;
  }
  const int a = k / n;
  const int rem = k - a * n;
  const int c0 = (n - par + 1) / 2;  // points in row 2a (first i = par)
  if (rem < c0) {
    j = 2 * a;
    i = par + 2 * rem;
  } else {
    j = 2 * a + 1;
    i = (par ^ 1) + 2 * (rem - c0);
  }
  return i + n * j;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* bits, double v) {
  // non-negative doubles order like their bit patterns; NaN (all exponent bits
  // set, non-zero mantissa) compares above +inf and so propagates
  atomicMax(bits, (unsigned long long)__double_as_longlong(v));
}

template <class R>
__device__ __forceinline__ R absmax_nan(R a, R b) {
  // max that lets NaN win
  return (a != a || a > b) ? a : b;
}

// Per arithmetic type: the magnitude type of norms, |x|, and the difference
// and sum used by the defect's stencil and final subtraction (exact
// renormalisation for double-float, where these operands nearly cancel).
template <class R>
struct Arith;
template <>
struct Arith<double> {
  using Mag = double;
  static __device__ __forceinline__ double mag(double x) { return fabs(x); }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
};
template <>
struct Arith<float> {
  using Mag = float;
  static __device__ __forceinline__ float mag(float x) { return fabsf(x); }
  static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
};
template <>
struct Arith<dd> {
  using Mag = float;
  static __device__ __forceinline__ float mag(dd x) { return dd_abs_hi(x); }
  static __device__ __forceinline__ dd sub(dd a, dd b) { return dd_add_accurate(a, -b); }
  static __device__ __forceinline__ dd add(dd a, dd b) { return dd_add_accurate(a, b); }
};


// The 2d neighbour lines of point (i, j) in `base` (its line starts at pM), with
// the shared zero line standing in for neighbours outside the grid (zero
// Dirichlet data), so that the loops over time need no branches.
template <class R>
__device__ __forceinline__ void neighbour_lines(const R* base, const R* zero, int d, int n, int i,
                                                int j, size_t pM, int M, const R* (&q)[4]) {
  q[0] = i > 0 ? base + pM - M : zero;
  q[1] = i < n - 1 ? base + pM + M : zero;
  if (d == 2) {
    const size_t nM = (size_t)n * M;
    q[2] = j > 0 ? base + pM - nM : zero;
    q[3] = j < n - 1 ? base + pM + nM : zero;
  } else {
    q[2] = q[3] = zero;
  }
}


// Sum of the neighbour lines of point (i, j) at time m, zero outside the grid,
// with the bounds tested per access (fewer live registers than holding the
// neighbour pointers; used by the FP64 and double-float kernels, whose
// arithmetic, not their index work, bounds them).
template <class R>
__device__ __forceinline__ R neighbour_sum(const R* __restrict__ u, int d, int n, int i, int j,
                                           size_t pM, int M, int m) {
  R s = R(0);
  if (i > 0) s = s + u[pM - M + m];
  if (i < n - 1) s = s + u[pM + M + m];
  if (d == 2) {
    const size_t nM = (size_t)n * M;
    if (j > 0) s = s + u[pM - nM + m];
    if (j < n - 1) s = s + u[pM + nM + m];
  }
  return s;
}

// sum over the 2d directions of (u_p - u_q), u_q = 0 outside the grid, with every
// difference formed before the sum (same bounds handling as neighbour_sum)
template <class R>
__device__ __forceinline__ R stencil_differences(const R* __restrict__ u, R up, int d, int n, int i,
                                                 int j, size_t pM, int M, int m) {
  using A = Arith<R>;
  R s = A::add(i > 0 ? A::sub(up, u[pM - M + m]) : up, i < n - 1 ? A::sub(up, u[pM + M + m]) : up);
  if (d == 2) {
    const size_t nM = (size_t)n * M;
    s = A::add(s, A::add(j > 0 ? A::sub(up, u[pM - nM + m]) : up,
                         j < n - 1 ? A::sub(up, u[pM + nM + m]) : up));
  }
  return s;
}

}  // namespace mgwr

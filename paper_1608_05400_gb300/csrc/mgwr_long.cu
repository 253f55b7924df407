// Long time lines (M > kShortMaxM): the causal convolutions of the smoother
// and of the defect (Sec. 5) split into P = M / B blocks of B = kLongB time
// steps and are evaluated as a uniformly partitioned convolution, so every
// transform keeps the engine length Lb = 2B of the short lines.  Output block i
// of y = k * x is
//     y_i = sum_{j <= i} T_{i-j} x_j,
// where the Toeplitz block of lag d holds the kernel values k[dB + s] for
// -B < s < B.  Laid out cyclically on Lb points (s < 0 at Lb + s, position B
// unused) they form the segment c_d, and because x_j fills only the first B of
// its Lb points no lag wraps:
//     y_i = first B values of IFFT( sum_{j <= i} FFT(c_{i-j}) . FFT(x_j) ).
// Pass 1 transforms every input block of every line pair into scratch; pass 2
// accumulates the spectrum products of output block i in registers, inverts,
// and finishes the block (smoother update or defect with its norm).
//
// Spectra here (scratch and kernel segments) are stored position-major within
// a block: slot q of radix-8 butterfly b sits at q * Lb/8 + b, so the
// accumulation loop of pass 2 reads whole warps of consecutive values (for
// every engine split E: thread t owns the butterflies t + e Lb/(8E)).
#include <type_traits>

#include "mgwr_common.cuh"

namespace mgwr {

namespace {

constexpr int kLb = 2 * kLongB;  // transform length
constexpr int kLogLb = 13;       // log2(kLb)
constexpr int kL8 = kLb / 8;     // radix-8 butterflies per stage
// threads per line pair (one pair per block) for engine split E
template <int E>
constexpr int long_threads() { return kL8 / E; }
static_assert((1 << kLogLb) == kLb, "the long path is written for kLongB = 4096");

// Shape type per arithmetic: the FP32 kernels unroll the fixed length, the
// wider types keep the run-time shape (fewer registers at 1024 threads).
template <class R>
using LongShape = typename std::conditional<sizeof(R) == 4, FixedShape<kLogLb>, FftShape>::type;

// The k-th point of parity `par` (or the k-th point of the grid when every
// point is taken), with its grid coordinates.
__device__ __forceinline__ int pair_point(int k, int d, int n, int par, bool every, int& i,
                                          int& j) {
  if (!every) return colour_point(k, d, n, par, i, j);
  i = d == 1 ? k : k % n;
  j = d == 1 ? 0 : k / n;
  return k;
}

}  // namespace

// ---- pass 1: spectra of the input blocks ---------------------------------------

// MODE 0 (smoother): x = f + hinv2 * (sum of neighbour lines) on the points of
// parity `par`, or x = f on every point (all_points, one-point solve);
// MODE 1 (defect): x = u on every point.
// Block (pair * P + j, instance): input block j of one line pair.
template <class R, int MODE, int E>
__global__ void __launch_bounds__(long_threads<E>(), 1)
    k_long_forward(const R* __restrict__ f, const R* __restrict__ u, Cx<R>* __restrict__ scratch,
                   const Cx<R>* __restrict__ tw, int d, int n, int M, int P, int par,
                   int all_points, R hinv2, int npts, int npairs, size_t fstride) {
  extern __shared__ unsigned char smem_raw[];
  const int pair = blockIdx.x / P, j = blockIdx.x - pair * P, inst = blockIdx.y;
  f += inst * fstride;
  u += inst * fstride;
  Cx<R>* buf = reinterpret_cast<Cx<R>*>(smem_raw);
  const LongShape<R> sh(kLogLb);
  const int t = threadIdx.x;
  const bool every = MODE == 1 || all_points;
  const int kA = 2 * pair, kB = 2 * pair + 1;
  const bool hasB = kB < npts;
  int iA, jA, iB = 0, jB = 0;
  const int pA = pair_point(kA, d, n, par, every, iA, jA);
  const int pB = hasB ? pair_point(kB, d, n, par, every, iB, jB) : 0;
  const size_t pAM = (size_t)pA * M, pBM = (size_t)pB * M;
  const int m0 = j * kLongB;
  auto load = [&](int a) -> Cx<R> {
    const int m = m0 + a;
    Cx<R> x{R(0), R(0)};
    if constexpr (MODE == 0) {
      x.x = f[pAM + m];
      if (!all_points) x.x = x.x + hinv2 * neighbour_sum(u, d, n, iA, jA, pAM, M, m);
      if (hasB) {
        x.y = f[pBM + m];
        if (!all_points) x.y = x.y + hinv2 * neighbour_sum(u, d, n, iB, jB, pBM, M, m);
      }
    } else {
      x.x = u[pAM + m];
      if (hasB) x.y = u[pBM + m];
    }
    return x;
  };
  Cx<R> v[E][8];
  const GroupSync sync(long_threads<E>(), long_threads<E>(), 0);
  fft_forward<E>(buf, t, sh, tw, load, v, sync);
  Cx<R>* out = scratch + (((size_t)inst * npairs + pair) * P + j) * kLb + t;
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q * kL8 + e * long_threads<E>()] = v[e][q];
}

// ---- pass 2: accumulate, invert, finish ------------------------------------------

// Block (pair * P + i, instance): output block i of one line pair.
// MODE 0: u = y (delta = y - u_old when delta != null); MODE 1: r = f - y -
// hinv2 * sum of (u_p - u_q), with |r|_inf folded into norm_bits[instance].
template <class R, class RO, int MODE, int E>
__global__ void __launch_bounds__(long_threads<E>(), 1)
    k_long_inverse(const R* __restrict__ f, R* __restrict__ u, R* __restrict__ delta,
                   RO* __restrict__ r, const Cx<R>* __restrict__ scratch,
                   const Cx<R>* __restrict__ seg, size_t seg_stride,
                   const Cx<R>* __restrict__ tw, int d, int n, int M, int P, int par,
                   int all_points, R hinv2, int npts, int npairs, size_t fstride,
                   unsigned long long* __restrict__ norm_bits) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[long_threads<E>() / 32];
  const int pair = blockIdx.x / P, i = blockIdx.x - pair * P, inst = blockIdx.y;
  f += inst * fstride;
  u += inst * fstride;
  if (delta != nullptr) delta += inst * fstride;
  if (r != nullptr) r += inst * fstride;
  seg += inst * seg_stride;
  Cx<R>* buf = reinterpret_cast<Cx<R>*>(smem_raw);
  const LongShape<R> sh(kLogLb);
  const int t = threadIdx.x;
  const bool every = MODE == 1 || all_points;
  const int kA = 2 * pair, kB = 2 * pair + 1;
  const bool hasB = kB < npts;
  int iA, jA, iB = 0, jB = 0;
  const int pA = pair_point(kA, d, n, par, every, iA, jA);
  const int pB = hasB ? pair_point(kB, d, n, par, every, iB, jB) : 0;
  const size_t pAM = (size_t)pA * M, pBM = (size_t)pB * M;

  // spectrum of output block i: sum over input blocks j <= i of K(i - j) . X(j)
  const Cx<R>* xs = scratch + ((size_t)inst * npairs + pair) * P * kLb + t;
  const Cx<R>* ks = seg + t;
  constexpr int TL = long_threads<E>();
  Cx<R> v[E][8];
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int q = 0; q < 8; ++q) v[e][q] = Cx<R>{R(0), R(0)};
#pragma unroll 1
  for (int jb = 0; jb <= i; ++jb) {
    const Cx<R>* xj = xs + (size_t)jb * kLb;
    const Cx<R>* kd = ks + (size_t)(i - jb) * kLb;
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int q = 0; q < 8; ++q)
        v[e][q] = cadd(v[e][q], cmul(xj[q * kL8 + e * TL], kd[q * kL8 + e * TL]));
  }

  const int m0 = i * kLongB;
  using A = Arith<R>;
  typename A::Mag amax = 0;
  auto store = [&](int a, Cx<R> y) {
    const int m = m0 + a;
    if constexpr (MODE == 0) {
      if (delta != nullptr) delta[pAM + m] = y.x - u[pAM + m];
      u[pAM + m] = y.x;
      if (hasB) {
        if (delta != nullptr) delta[pBM + m] = y.y - u[pBM + m];
        u[pBM + m] = y.y;
      }
    } else {
      const R ra = A::sub(A::sub(f[pAM + m], y.x),
                          hinv2 * stencil_differences(u, u[pAM + m], d, n, iA, jA, pAM, M, m));
      r[pAM + m] = RO(ra);
      amax = absmax_nan(A::mag(ra), amax);
      if (hasB) {
        const R rb = A::sub(A::sub(f[pBM + m], y.y),
                            hinv2 * stencil_differences(u, u[pBM + m], d, n, iB, jB, pBM, M, m));
        r[pBM + m] = RO(rb);
        amax = absmax_nan(A::mag(rb), amax);
      }
    }
  };
  const GroupSync sync(TL, TL, 0);
  fft_inverse<E>(buf, t, sh, tw, v, store, sync);

  if constexpr (MODE == 1) {
    if (norm_bits != nullptr) {
      double a = (double)amax;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a = absmax_nan(__shfl_xor_sync(0xffffffffu, a, o), a);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
      __syncthreads();
      if (threadIdx.x < 32) {
        a = threadIdx.x < TL / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a = absmax_nan(__shfl_xor_sync(0xffffffffu, a, o), a);
        if (threadIdx.x == 0) atomic_max_nonneg(norm_bits + inst, a);
      }
    }
  }
}

// ---- kernel segment spectra (FP64 setup) -----------------------------------------

// Block (line, segment dseg): spectrum of the cyclic segment c_dseg of the
// length-M kernel `lines[line]`: c[s] = k[dseg B + s] for 0 <= s < B,
// c[Lb + s] = k[dseg B + s] for -B < s < 0 (zero where the lag leaves
// [0, M)), c[B] = 0; scaled by 1/Lb, position-major.
__global__ void __launch_bounds__(kL8, 1)
    k_long_spectra(Cx<double>* __restrict__ spec, const double* __restrict__ lines, int M, int P,
                   const Cx<double>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  const int line = blockIdx.x, dseg = blockIdx.y;
  Cx<double>* buf = reinterpret_cast<Cx<double>*>(smem_raw);
  const FftShape sh(kLogLb);
  const double* k = lines + (size_t)line * M;
  auto load = [&](int s) -> Cx<double> {
    const int lag = s < kLongB ? dseg * kLongB + s : (s > kLongB ? dseg * kLongB + s - kLb : -1);
    return Cx<double>{lag >= 0 && lag < M ? k[lag] : 0.0, 0.0};
  };
  Cx<double> v[1][8];
  const GroupSync sync(kL8, kL8, 0);
  fft_forward<1, double, FftShape, decltype(load), true>(buf, threadIdx.x, sh, tw, load, v, sync);
  const double inv = 1.0 / (double)kLb;
  Cx<double>* out = spec + ((size_t)line * P + dseg) * kLb + threadIdx.x;
#pragma unroll
  for (int q = 0; q < 8; ++q) out[q * kL8] = Cx<double>{v[0][q].x * inv, v[0][q].y * inv};
}

// ---- launchers -------------------------------------------------------------------

template <class R, int E>
cudaError_t sweep_long_launch(dim3 grid, size_t smem, cudaStream_t s, const R* f, R* u, R* delta,
                              const Cx<R>* spec, size_t spec_stride, const Cx<R>* tw,
                              Cx<R>* scratch, int d, int n, int M, int P, int par, int all_points,
                              R hinv2, int npts, int npairs, size_t fstride) {
  cudaError_t e = prepare_smem(k_long_forward<R, 0, E>, smem);
  if (e != cudaSuccess) return e;
  k_long_forward<R, 0, E><<<grid, long_threads<E>(), smem, s>>>(
      f, u, scratch, tw, d, n, M, P, par, all_points, hinv2, npts, npairs, fstride);
  e = counted(cudaGetLastError());
  if (e != cudaSuccess) return e;
  e = prepare_smem(k_long_inverse<R, R, 0, E>, smem);
  if (e != cudaSuccess) return e;
  k_long_inverse<R, R, 0, E><<<grid, long_threads<E>(), smem, s>>>(
      f, u, delta, (R*)nullptr, scratch, spec, spec_stride, tw, d, n, M, P, par, all_points,
      hinv2, npts, npairs, fstride, nullptr);
  return counted(cudaGetLastError());
}

template <class R>
cudaError_t launch_sweep_long(const R* f, R* u, R* delta, const Cx<R>* spec, size_t spec_stride,
                              const Cx<R>* tw, Cx<R>* scratch, const LevelShape& ls, int par,
                              bool all_points, R hinv2, int E, cudaStream_t s) {
  const int d = ls.d, n = ls.n, M = ls.M, P = M / kLongB;
  const int npts = all_points ? (d == 1 ? n : n * n) : colour_count(d, n, par);
  const int npairs = (npts + 1) / 2;
  if (npairs == 0 || ls.batch == 0) return cudaSuccess;
  if (scratch == nullptr || M % kLongB != 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)Pad<R>::len(kLb) * sizeof(Cx<R>);
  const dim3 grid((unsigned)((size_t)npairs * P), (unsigned)ls.batch);
  const size_t fstride = ls.field_stride();
  if (effective_split(M, 8, E) == 2)
    return sweep_long_launch<R, 2>(grid, smem, s, f, u, delta, spec, spec_stride, tw, scratch, d,
                                   n, M, P, par, all_points ? 1 : 0, hinv2, npts, npairs, fstride);
  return sweep_long_launch<R, 1>(grid, smem, s, f, u, delta, spec, spec_stride, tw, scratch, d, n,
                                 M, P, par, all_points ? 1 : 0, hinv2, npts, npairs, fstride);
}

template <class R, class RO, int E>
cudaError_t defect_long_launch(dim3 grid, size_t smem, cudaStream_t s, const R* u, const R* f,
                               RO* r, const Cx<R>* tspec, size_t spec_stride, const Cx<R>* tw,
                               Cx<R>* scratch, int d, int n, int M, int P, R hinv2, int npts,
                               int npairs, size_t fstride, unsigned long long* norm_bits) {
  cudaError_t e = prepare_smem(k_long_forward<R, 1, E>, smem);
  if (e != cudaSuccess) return e;
  k_long_forward<R, 1, E><<<grid, long_threads<E>(), smem, s>>>(
      f, u, scratch, tw, d, n, M, P, 0, 1, hinv2, npts, npairs, fstride);
  e = counted(cudaGetLastError());
  if (e != cudaSuccess) return e;
  e = prepare_smem(k_long_inverse<R, RO, 1, E>, smem);
  if (e != cudaSuccess) return e;
  k_long_inverse<R, RO, 1, E><<<grid, long_threads<E>(), smem, s>>>(
      f, const_cast<R*>(u), (R*)nullptr, r, scratch, tspec, spec_stride, tw, d, n, M, P, 0, 1,
      hinv2, npts, npairs, fstride, norm_bits);
  return counted(cudaGetLastError());
}

template <class R, class RO>
cudaError_t launch_defect_long(const R* u, const R* f, RO* r, const Cx<R>* tspec,
                               size_t spec_stride, const Cx<R>* tw, Cx<R>* scratch,
                               const LevelShape& ls, R hinv2, unsigned long long* norm_bits,
                               int E, cudaStream_t s) {
  const int d = ls.d, n = ls.n, M = ls.M, P = M / kLongB;
  const int npts = d == 1 ? n : n * n;
  const int npairs = (npts + 1) / 2;
  if (ls.batch == 0) return cudaSuccess;
  if (scratch == nullptr || M % kLongB != 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)Pad<R>::len(kLb) * sizeof(Cx<R>);
  const dim3 grid((unsigned)((size_t)npairs * P), (unsigned)ls.batch);
  const size_t fstride = ls.field_stride();
  if (effective_split(M, 8, E) == 2)
    return defect_long_launch<R, RO, 2>(grid, smem, s, u, f, r, tspec, spec_stride, tw, scratch,
                                        d, n, M, P, hinv2, npts, npairs, fstride, norm_bits);
  return defect_long_launch<R, RO, 1>(grid, smem, s, u, f, r, tspec, spec_stride, tw, scratch, d,
                                      n, M, P, hinv2, npts, npairs, fstride, norm_bits);
}

cudaError_t launch_spectra_long(Cx<double>* spec, const double* lines, int count, int M,
                                const Cx<double>* tw, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  if (M % kLongB != 0) return cudaErrorInvalidValue;
  const int P = M / kLongB;
  const size_t smem = (size_t)Pad<double>::len(kLb) * sizeof(Cx<double>);
  cudaError_t e = prepare_smem(k_long_spectra, smem);
  if (e != cudaSuccess) return e;
  k_long_spectra<<<dim3((unsigned)count, (unsigned)P), kL8, smem, s>>>(spec, lines, M, P, tw);
  return counted(cudaGetLastError());
}

template cudaError_t launch_sweep_long<double>(const double*, double*, double*, const Cx<double>*,
                                               size_t, const Cx<double>*, Cx<double>*,
                                               const LevelShape&, int, bool, double, int,
                                               cudaStream_t);
template cudaError_t launch_sweep_long<dd>(const dd*, dd*, dd*, const Cx<dd>*, size_t,
                                           const Cx<dd>*, Cx<dd>*, const LevelShape&, int, bool,
                                           dd, int, cudaStream_t);
template cudaError_t launch_sweep_long<float>(const float*, float*, float*, const Cx<float>*,
                                              size_t, const Cx<float>*, Cx<float>*,
                                              const LevelShape&, int, bool, float, int,
                                              cudaStream_t);
#define MGWR_INST_LONG_DEFECT(R, RO)                                                          \
  template cudaError_t launch_defect_long<R, RO>(const R*, const R*, RO*, const Cx<R>*,        \
                                                 size_t, const Cx<R>*, Cx<R>*,                 \
                                                 const LevelShape&, R, unsigned long long*,    \
                                                 int, cudaStream_t);
MGWR_INST_LONG_DEFECT(double, double)
MGWR_INST_LONG_DEFECT(double, float)
MGWR_INST_LONG_DEFECT(double, dd)
MGWR_INST_LONG_DEFECT(float, float)
MGWR_INST_LONG_DEFECT(dd, float)
MGWR_INST_LONG_DEFECT(dd, dd)
#undef MGWR_INST_LONG_DEFECT

}  // namespace mgwr

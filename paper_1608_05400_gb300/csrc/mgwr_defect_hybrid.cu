// Outer defect of the mixed-precision refinement in its cheap form, for the
// outer steps whose defect is still large: the time convolution T_M u in FP32
// (one FP32 FFT convolution of the rounded iterate, error about 1e-6 of
// |T_M u|), the source and the stencil f - A_h u in the iterate's own
// arithmetic (double or double-float), where the rounding of u to FP32 would
// otherwise be amplified by |A_h| ~ 4d/h^2.
#include "mgwr_common.cuh"
#include "mgwr_fft_rp.cuh"

namespace mgwr {

namespace {

__device__ __forceinline__ float to_float(double x) { return (float)x; }
__device__ __forceinline__ float to_float(dd x) { return float(x); }
__device__ __forceinline__ double widen(float x, double) { return (double)x; }
__device__ __forceinline__ dd widen(float x, dd) { return dd(x, 0.f); }

}  // namespace

template <class Tin, int BLOCK, class SH>
__global__ void __launch_bounds__(BLOCK, min_blocks<float>(BLOCK))
    k_defect_hybrid(const Tin* __restrict__ u, const Tin* __restrict__ f, float* __restrict__ r,
                    const Cx<float>* __restrict__ tspec, const Cx<float>* __restrict__ tw,
                    const Tin* __restrict__ zero, int d, int n, int M, int logL, Tin hinv2,
                    int npts, int npairs, unsigned long long* __restrict__ norm_bits,
                    size_t fstride, size_t sstride) {
  extern __shared__ unsigned char smem_raw[];
  u += blockIdx.y * fstride;
  f += blockIdx.y * fstride;
  r += blockIdx.y * fstride;
  tspec += blockIdx.y * sstride;
  if (norm_bits != nullptr) norm_bits += blockIdx.y;
  __shared__ double red[BLOCK / 32];
  Cx<float>* smem = reinterpret_cast<Cx<float>*>(smem_raw);
  const SH sh(logL);
  const int TL = sh.L8;
  const int g = threadIdx.x / TL;
  const int t = threadIdx.x - g * TL;
  const int groups = BLOCK / TL;
  const int pair = blockIdx.x * groups + g;
  Cx<float>* buf = smem + g * Pad<float>::len(sh.L);
  const GroupSync sync(TL, BLOCK, g);

  const bool valid = pair < npairs;
  const int pA = 2 * pair, pB = 2 * pair + 1;
  const bool hasB = valid && pB < npts;
  const size_t pAM = (size_t)pA * M, pBM = (size_t)pB * M;
  const int iA = d == 1 ? pA : pA % n, jA = d == 1 ? 0 : pA / n;
  const int iB = d == 1 ? pB : pB % n, jB = d == 1 ? 0 : pB / n;
  const Tin* uA = valid ? u + pAM : zero;
  const Tin* uB = hasB ? u + pBM : zero;
  auto load = [&](int m) -> Cx<float> { return Cx<float>{to_float(uA[m]), to_float(uB[m])}; };
  Cx<float> v[1][8];
  fft_forward<1>(buf, t, sh, tw, load, v, sync);
#pragma unroll
  for (int q = 0; q < 8; ++q) v[0][q] = cmul(v[0][q], tspec[8 * t + q]);
  using A = Arith<Tin>;
  typename A::Mag amax = 0;
  auto store = [&](int m, Cx<float> y) {
    if (valid) {
      const Tin ra = A::sub(A::sub(f[pAM + m], hinv2 * stencil_differences(u, uA[m], d, n, iA, jA,
                                                                             pAM, M, m)),
                            widen(y.x, Tin()));
      r[pAM + m] = float(ra);
      amax = absmax_nan(A::mag(ra), amax);
      if (hasB) {
        const Tin rb = A::sub(A::sub(f[pBM + m], hinv2 * stencil_differences(u, uB[m], d, n, iB,
                                                                               jB, pBM, M, m)),
                              widen(y.y, Tin()));
        r[pBM + m] = float(rb);
        amax = absmax_nan(A::mag(rb), amax);
      }
    }
  };
  fft_inverse<1>(buf, t, sh, tw, v, store, sync);

  if (norm_bits != nullptr) {
    double a = (double)amax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = absmax_nan(__shfl_xor_sync(0xffffffffu, a, o), a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
      a = threadIdx.x < BLOCK / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a = absmax_nan(__shfl_xor_sync(0xffffffffu, a, o), a);
      if (threadIdx.x == 0) atomic_max_nonneg(norm_bits, a);
    }
  }
}

template <class Tin, int BLOCK, class SH>
cudaError_t hybrid_launch(dim3 grid, size_t smem, cudaStream_t s, const Tin* u, const Tin* f,
                          float* r, const Cx<float>* tspec, const Cx<float>* tw, const Tin* zero,
                          int d, int n, int M, int logL, Tin hinv2, int npts, int npairs,
                          unsigned long long* norm_bits, size_t fstride, size_t sstride) {
  cudaError_t e = prepare_smem(k_defect_hybrid<Tin, BLOCK, SH>, smem);
  if (e != cudaSuccess) return e;
  k_defect_hybrid<Tin, BLOCK, SH><<<grid, BLOCK, smem, s>>>(u, f, r, tspec, tw, zero, d, n, M,
                                                            logL, hinv2, npts, npairs, norm_bits,
                                                            fstride, sstride);
  return cudaSuccess;
}

template <class Tin>
cudaError_t launch_defect_hybrid(const Tin* u, const Tin* f, float* r, const Cx<float>* tspec,
                                 size_t spec_stride, const Cx<float>* tw, const Tin* zero,
                                 const LevelShape& ls, Tin hinv2, unsigned long long* norm_bits,
                                 cudaStream_t s) {
  const int d = ls.d, n = ls.n, M = ls.M;
  if (M > kShortMaxM) return cudaErrorInvalidValue;
  const int L = 2 * M, logL = ilog2(L);
  const int npts = d == 1 ? n : n * n;
  const int npairs = (npts + 1) / 2;
  if (ls.batch == 0) return cudaSuccess;
  const size_t fstride = ls.field_stride();
  const int block = block_threads(L);
  const int groups = block / (L / 8);
  const size_t smem = (size_t)groups * Pad<float>::len(L) * sizeof(Cx<float>);
  const dim3 grid((unsigned)((npairs + groups - 1) / groups), (unsigned)ls.batch);
  cudaError_t e;
  switch (logL) {
#define MGWR_CASE(LG)                                                                           \
  case LG:                                                                                      \
    e = hybrid_launch<Tin, ((1 << LG) / 8 > 256 ? (1 << LG) / 8 : 256), FixedShape<LG>>(        \
        grid, smem, s, u, f, r, tspec, tw, zero, d, n, M, logL, hinv2, npts, npairs, norm_bits, \
        fstride, spec_stride);                                                                  \
    break;
    MGWR_FIXED_LOGL(MGWR_CASE)
#undef MGWR_CASE
    default:
      e = hybrid_launch<Tin, 256, FftShape>(grid, smem, s, u, f, r, tspec, tw, zero, d, n, M, logL,
                                            hinv2, npts, npairs, norm_bits, fstride, spec_stride);
      break;
  }
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

// The same defect with T_M u on the register-pass engine (mgwr_fft_rp.cuh):
// tspec in that engine's spectral order.
template <class Tin, int LOGL, int R0, int R1, int R2, int T>
__global__ void __launch_bounds__(kRpBlock, 2)
    k_defect_hybrid_rp(const Tin* __restrict__ u, const Tin* __restrict__ f, float* __restrict__ r,
                       const Cx<float>* __restrict__ tspec, const Cx<float>* __restrict__ tw,
                       const Tin* __restrict__ zero, int d, int n, int M, Tin hinv2, int npts,
                       int npairs, unsigned long long* __restrict__ norm_bits, size_t fstride,
                       size_t sstride) {
  using P = rp::Plan<LOGL, R0, R1, R2, T>;
  constexpr int PAIRS = kRpBlock / T;
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[kRpBlock / 32];
  u += blockIdx.y * fstride;
  f += blockIdx.y * fstride;
  r += blockIdx.y * fstride;
  tspec += blockIdx.y * sstride;
  if (norm_bits != nullptr) norm_bits += blockIdx.y;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int pair = blockIdx.x * PAIRS + g;
  Cx<float>* buf = reinterpret_cast<Cx<float>*>(smem_raw) + g * P::SMEM;
  const bool valid = pair < npairs;
  const int pA = 2 * pair, pB = 2 * pair + 1;
  const bool hasB = valid && pB < npts;
  const size_t pAM = (size_t)pA * M, pBM = (size_t)pB * M;
  const int iA = d == 1 ? pA : pA % n, jA = d == 1 ? 0 : pA / n;
  const int iB = d == 1 ? pB : pB % n, jB = d == 1 ? 0 : pB / n;
  const Tin* uA = valid ? u + pAM : zero;
  const Tin* uB = hasB ? u + pBM : zero;
  auto load = [&](int m) -> Cx<float> { return Cx<float>{to_float(uA[m]), to_float(uB[m])}; };
  using A = Arith<Tin>;
  typename A::Mag amax = 0;
  auto store = [&](int m, Cx<float> y) {
    if (valid) {
      const Tin ra = A::sub(A::sub(f[pAM + m], hinv2 * stencil_differences(u, uA[m], d, n, iA, jA,
                                                                             pAM, M, m)),
                            widen(y.x, Tin()));
      r[pAM + m] = float(ra);
      amax = absmax_nan(A::mag(ra), amax);
      if (hasB) {
        const Tin rb = A::sub(A::sub(f[pBM + m], hinv2 * stencil_differences(u, uB[m], d, n, iB,
                                                                               jB, pBM, M, m)),
                              widen(y.y, Tin()));
        r[pBM + m] = float(rb);
        amax = absmax_nan(A::mag(rb), amax);
      }
    }
  };
  rp::convolve<LOGL, R0, R1, R2, T, PAIRS>(buf, t, g, tspec, tw, load, store);
  if (norm_bits != nullptr) {
    double a = (double)amax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = absmax_nan(__shfl_xor_sync(0xffffffffu, a, o), a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
      a = threadIdx.x < kRpBlock / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a = absmax_nan(__shfl_xor_sync(0xffffffffu, a, o), a);
      if (threadIdx.x == 0) atomic_max_nonneg(norm_bits, a);
    }
  }
}

template <class Tin>
cudaError_t launch_defect_hybrid_rp(const Tin* u, const Tin* f, float* r, const Cx<float>* tspec,
                                    size_t spec_stride, const Cx<float>* tw, const Tin* zero,
                                    const LevelShape& ls, Tin hinv2, unsigned long long* norm_bits,
                                    cudaStream_t s) {
  const int d = ls.d, n = ls.n, M = ls.M;
  if (!radix_length(M)) return cudaErrorInvalidValue;
  const int npts = d == 1 ? n : n * n;
  const int npairs = (npts + 1) / 2;
  if (ls.batch == 0) return cudaSuccess;
  const size_t fstride = ls.field_stride();
  cudaError_t e = cudaErrorInvalidValue;
  switch (ilog2(2 * M)) {
#define MGWR_RP_HYBRID(LG, A, B, C, T)                                                             case LG: {                                                                                         using P = rp::Plan<LG, A, B, C, T>;                                                              const size_t smem = (size_t)(kRpBlock / T) * P::SMEM * sizeof(Cx<float>);                        e = prepare_smem(k_defect_hybrid_rp<Tin, LG, A, B, C, T>, smem);                                 if (e != cudaSuccess) return e;                                                                  const dim3 grid((unsigned)((npairs + kRpBlock / T - 1) / (kRpBlock / T)), (unsigned)ls.batch);     k_defect_hybrid_rp<Tin, LG, A, B, C, T><<<grid, kRpBlock, smem, s>>>(                                u, f, r, tspec, tw, zero, d, n, M, hinv2, npts, npairs, norm_bits, fstride, spec_stride);     break;                                                                                         }
    MGWR_RP_PLANS(MGWR_RP_HYBRID)
#undef MGWR_RP_HYBRID
    default:
      break;
  }
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

template cudaError_t launch_defect_hybrid_rp<double>(const double*, const double*, float*,
                                                     const Cx<float>*, size_t, const Cx<float>*,
                                                     const double*, const LevelShape&, double,
                                                     unsigned long long*, cudaStream_t);
template cudaError_t launch_defect_hybrid_rp<dd>(const dd*, const dd*, float*, const Cx<float>*,
                                                 size_t, const Cx<float>*, const dd*,
                                                 const LevelShape&, dd, unsigned long long*,
                                                 cudaStream_t);
template cudaError_t launch_defect_hybrid<double>(const double*, const double*, float*,
                                                  const Cx<float>*, size_t, const Cx<float>*,
                                                  const double*, const LevelShape&, double,
                                                  unsigned long long*, cudaStream_t);
template cudaError_t launch_defect_hybrid<dd>(const dd*, const dd*, float*, const Cx<float>*,
                                              size_t, const Cx<float>*, const dd*,
                                              const LevelShape&, dd, unsigned long long*,
                                              cudaStream_t);

}  // namespace mgwr

// Defect kernel r = f - (T_M (x) I + A_h) u and its launcher for all FFT
// lengths; the arithmetic types are instantiated in mgwr_defect_*.cu (one
// translation unit each, compiled in parallel).
#pragma once

#include "mgwr_common.cuh"

namespace mgwr {

// ---------------------------------------------------------------------------------
// defect r = f - (T_M (x) I + A_h) u  (Algorithm 1; Sec. 5 circulant-embedding matvec)
// ---------------------------------------------------------------------------------

template <class R, class RO, int BLOCK, class SH>
__global__ void __launch_bounds__(BLOCK, min_blocks<R>(BLOCK))
    k_defect(const R* __restrict__ u, const R* __restrict__ f, RO* __restrict__ r,
             const Cx<R>* __restrict__ tspec, const Cx<R>* __restrict__ tw,
             const R* __restrict__ zero, int d, int n, int M, int logL, R hinv2, int npts,
             int npairs, unsigned long long* __restrict__ norm_bits, size_t fstride,
             size_t sstride) {
  extern __shared__ unsigned char smem_raw[];
  u += blockIdx.y * fstride;
  f += blockIdx.y * fstride;
  r += blockIdx.y * fstride;
  tspec += blockIdx.y * sstride;
  if (norm_bits != nullptr) norm_bits += blockIdx.y;
  __shared__ double red[BLOCK / 32];
  Cx<R>* smem = reinterpret_cast<Cx<R>*>(smem_raw);
  const SH sh(logL);
  const int TL = sh.L8;
  const int g = threadIdx.x / TL;
  const int t = threadIdx.x - g * TL;
  const int groups = BLOCK / TL;
  const int pair = blockIdx.x * groups + g;
  Cx<R>* buf = smem + g * Pad<R>::len(sh.L);

  const bool valid = pair < npairs;
  const int pA = 2 * pair, pB = 2 * pair + 1;
  const bool hasB = valid && pB < npts;
  const size_t pAM = (size_t)pA * M, pBM = (size_t)pB * M;
  const int iA = d == 1 ? pA : pA % n, jA = d == 1 ? 0 : pA / n;
  const int iB = d == 1 ? pB : pB % n, jB = d == 1 ? 0 : pB / n;
  const R* uA = valid ? u + pAM : zero;
  const R* uB = hasB ? u + pBM : zero;
  const R *qA[4], *qB[4];
  if constexpr (sizeof(R) == 4) {
    neighbour_lines(u, zero, d, n, iA, jA, pAM, M, qA);
    neighbour_lines(u, zero, d, n, iB, jB, pBM, M, qB);
  }
  auto load = [&](int m) -> Cx<R> { return Cx<R>{uA[m], uB[m]}; };
  Cx<R> v[8];
  fft_forward(buf, t, sh, tw, load, v);
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = cmul(v[q], tspec[8 * t + q]);
  using A = Arith<R>;
  typename A::Mag amax = 0;
  // r = f - (T_M u) - h^-2 sum_q (u_p - u_q): every difference is formed before
  // the sum, so smooth u loses no digits to the stencil's cancellation
  auto stencil = [&](R up, const R* const (&q)[4], int i, int j, size_t pM, int m) -> R {
    if constexpr (sizeof(R) == 4) {
      R s = A::add(A::sub(up, q[0][m]), A::sub(up, q[1][m]));
      if (d == 2) s = A::add(s, A::add(A::sub(up, q[2][m]), A::sub(up, q[3][m])));
      return s;
    } else {
      return stencil_differences(u, up, d, n, i, j, pM, M, m);
    }
  };
  auto store = [&](int m, Cx<R> y) {
    if (valid) {
      const R ua = uA[m];
      const R ra = A::sub(A::sub(f[pAM + m], y.x), hinv2 * stencil(ua, qA, iA, jA, pAM, m));
      r[pAM + m] = RO(ra);
      amax = absmax_nan(A::mag(ra), amax);
      if (hasB) {
        const R ub = uB[m];
        const R rb = A::sub(A::sub(f[pBM + m], y.y), hinv2 * stencil(ub, qB, iB, jB, pBM, m));
        r[pBM + m] = RO(rb);
        amax = absmax_nan(A::mag(rb), amax);
      }
    }
  };
  fft_inverse(buf, t, sh, tw, v, store);

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

template <class R, class RO, int BLOCK, class SH>
cudaError_t defect_launch(dim3 grid, size_t smem, cudaStream_t s, const R* u, const R* f, RO* r,
                          const Cx<R>* tspec, const Cx<R>* tw, const R* zero, int d, int n, int M,
                          int logL, R hinv2, int npts, int npairs, unsigned long long* norm_bits,
                          size_t fstride, size_t sstride) {
  cudaError_t e = prepare_smem(k_defect<R, RO, BLOCK, SH>, smem);
  if (e != cudaSuccess) return e;
  k_defect<R, RO, BLOCK, SH><<<grid, BLOCK, smem, s>>>(u, f, r, tspec, tw, zero, d, n, M, logL,
                                                       hinv2, npts, npairs, norm_bits, fstride,
                                                       sstride);
  return cudaSuccess;
}

template <class R, class RO>
cudaError_t launch_defect(const R* u, const R* f, RO* r, const Cx<R>* tspec, size_t spec_stride,
                          const Cx<R>* tw, const R* zero, Cx<R>* scratch, const LevelShape& ls,
                          R hinv2, unsigned long long* norm_bits, cudaStream_t s) {
  if (ls.M > kShortMaxM)
    return launch_defect_long<R, RO>(u, f, r, tspec, spec_stride, tw, scratch, ls, hinv2,
                                     norm_bits, s);
  const int d = ls.d, n = ls.n, M = ls.M;
  const int L = 2 * M, logL = ilog2(L);
  const int npts = d == 1 ? n : n * n;
  const int npairs = (npts + 1) / 2;
  if (ls.batch == 0) return cudaSuccess;
  const size_t fstride = ls.field_stride();
  const int block = block_threads(L);
  const int groups = block / (L / 8);
  const size_t smem = (size_t)groups * Pad<R>::len(L) * sizeof(Cx<R>);
  const dim3 grid((unsigned)((npairs + groups - 1) / groups), (unsigned)ls.batch);
  cudaError_t e;
  if constexpr (sizeof(R) == 4) {
    switch (logL) {
#define MGWR_CASE(LG)                                                                          \
  case LG:                                                                                     \
    e = defect_launch<R, RO, ((1 << LG) / 8 > 256 ? (1 << LG) / 8 : 256), FixedShape<LG>>(     \
        grid, smem, s, u, f, r, tspec, tw, zero, d, n, M, logL, hinv2, npts, npairs, norm_bits, \
        fstride, spec_stride);                                                                 \
    break;
      MGWR_FIXED_LOGL(MGWR_CASE)
#undef MGWR_CASE
      default:
        e = defect_launch<R, RO, 256, FftShape>(grid, smem, s, u, f, r, tspec, tw, zero, d, n, M,
                                                logL, hinv2, npts, npairs, norm_bits, fstride,
                                                spec_stride);
        break;
    }
  } else {
    switch (block) {
      case 256:
        e = defect_launch<R, RO, 256, FftShape>(grid, smem, s, u, f, r, tspec, tw, zero, d, n, M,
                                                logL, hinv2, npts, npairs, norm_bits, fstride,
                                                spec_stride);
        break;
      case 512:
        e = defect_launch<R, RO, 512, FftShape>(grid, smem, s, u, f, r, tspec, tw, zero, d, n, M,
                                                logL, hinv2, npts, npairs, norm_bits, fstride,
                                                spec_stride);
        break;
      default:
        e = defect_launch<R, RO, 1024, FftShape>(grid, smem, s, u, f, r, tspec, tw, zero, d, n,
                                                 M, logL, hinv2, npts, npairs, norm_bits, fstride,
                                                 spec_stride);
        break;
    }
  }
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

}  // namespace mgwr

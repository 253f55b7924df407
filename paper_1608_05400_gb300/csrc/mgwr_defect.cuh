// Defect kernel r = f - (T_M (x) I + A_h) u and its launcher for all FFT
// lengths; the arithmetic types are instantiated in mgwr_defect_*.cu (one
// translation unit each, compiled in parallel).
#pragma once

#include <type_traits>

#include "mgwr_common.cuh"

namespace mgwr {

// ---------------------------------------------------------------------------------
// defect r = f - (T_M (x) I + A_h) u  (Algorithm 1; Sec. 5 circulant-embedding matvec)
// ---------------------------------------------------------------------------------

// The defect's value in the output type: a conversion, or for an FP64 defect
// kept in double-float the split without FP64 arithmetic (dd_split_int).
template <class RO, class R>
__device__ __forceinline__ RO out_value(R x) {
  if constexpr (std::is_same<RO, dd>::value && std::is_same<R, double>::value)
    return dd_split_int(x);
  else
    return RO(x);
}

template <class R, class RO, int BLOCK, class SH, int E>
__global__ void __launch_bounds__(BLOCK, min_blocks<R>(BLOCK, E))
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
  const int TL = sh.L8 / E;  // threads per line pair
  const int g = threadIdx.x / TL;
  const int t = threadIdx.x - g * TL;
  const int groups = BLOCK / TL;
  const int pair = blockIdx.x * groups + g;
  Cx<R>* buf = smem + g * Pad<R>::len(sh.L);
  const GroupSync sync(TL, BLOCK, g);

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
  Cx<R> v[E][8];
  fft_forward<E>(buf, t, sh, tw, load, v, sync);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int b = t + e * TL;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[e][q] = cmul(v[e][q], tspec[8 * b + q]);
  }
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
      r[pAM + m] = out_value<RO>(ra);
      amax = absmax_nan(A::mag(ra), amax);
      if (hasB) {
        const R ub = uB[m];
        const R rb = A::sub(A::sub(f[pBM + m], y.y), hinv2 * stencil(ub, qB, iB, jB, pBM, m));
        r[pBM + m] = out_value<RO>(rb);
        amax = absmax_nan(A::mag(rb), amax);
      }
    }
  };
  fft_inverse<E>(buf, t, sh, tw, v, store, sync);

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

template <class R, class RO, int BLOCK, class SH, int E>
cudaError_t defect_launch(dim3 grid, size_t smem, cudaStream_t s, const R* u, const R* f, RO* r,
                          const Cx<R>* tspec, const Cx<R>* tw, const R* zero, int d, int n, int M,
                          int logL, R hinv2, int npts, int npairs, unsigned long long* norm_bits,
                          size_t fstride, size_t sstride) {
  cudaError_t e = prepare_smem(k_defect<R, RO, BLOCK, SH, E>, smem);
  if (e != cudaSuccess) return e;
  k_defect<R, RO, BLOCK, SH, E><<<grid, BLOCK, smem, s>>>(u, f, r, tspec, tw, zero, d, n, M,
                                                          logL, hinv2, npts, npairs, norm_bits,
                                                          fstride, sstride);
  return cudaSuccess;
}

template <class R, class RO>
cudaError_t launch_defect(const R* u, const R* f, RO* r, const Cx<R>* tspec, size_t spec_stride,
                          const Cx<R>* tw, const R* zero, Cx<R>* scratch, const LevelShape& ls,
                          R hinv2, unsigned long long* norm_bits, int E, cudaStream_t s) {
  if (ls.M > kShortMaxM)
    return launch_defect_long<R, RO>(u, f, r, tspec, spec_stride, tw, scratch, ls, hinv2,
                                     norm_bits, E, s);
  const int d = ls.d, n = ls.n, M = ls.M;
  const int L = 2 * M, logL = ilog2(L);
  E = effective_split(M, (int)sizeof(R) == 4 ? 4 : 8, E) & ~kStaged;
  const int npts = d == 1 ? n : n * n;
  const int npairs = (npts + 1) / 2;
  if (ls.batch == 0) return cudaSuccess;
  const size_t fstride = ls.field_stride();
  const int TL = L / (8 * E);
  int block = TL > 256 ? TL : 256;
  if constexpr (sizeof(R) == 8) {
    if (E == 1 && TL < 256) block = spread_block(TL, npairs, ls.batch);
  }
  const int groups = block / TL;
  const size_t smem = (size_t)groups * Pad<R>::len(L) * sizeof(Cx<R>);
  const dim3 grid((unsigned)((npairs + groups - 1) / groups), (unsigned)ls.batch);
  cudaError_t e = cudaErrorInvalidValue;
#define MGWR_DEFECT_ARGS \
  grid, smem, s, u, f, r, tspec, tw, zero, d, n, M, logL, hinv2, npts, npairs, norm_bits, fstride, spec_stride
  if constexpr (sizeof(R) == 4) {
    switch (logL * 8 + E) {
#define MGWR_CASE_E(LG, EE)                                                                       \
  case LG * 8 + EE:                                                                               \
    e = defect_launch<R, RO, ((1 << LG) / (8 * EE) > 256 ? (1 << LG) / (8 * EE) : 256),          \
                      FixedShape<LG>, EE>(MGWR_DEFECT_ARGS);                                      \
    break;
#define MGWR_CASE(LG) MGWR_CASE_E(LG, 1) MGWR_CASE_E(LG, 2) MGWR_CASE_E(LG, 4)
      MGWR_FIXED_LOGL(MGWR_CASE)
#undef MGWR_CASE
#undef MGWR_CASE_E
      default:
        e = defect_launch<R, RO, 256, FftShape, 1>(MGWR_DEFECT_ARGS);
        break;
    }
  } else {
    switch (block * 8 + E) {
      case 32 * 8 + 1: e = defect_launch<R, RO, 32, FftShape, 1>(MGWR_DEFECT_ARGS); break;
      case 64 * 8 + 1: e = defect_launch<R, RO, 64, FftShape, 1>(MGWR_DEFECT_ARGS); break;
      case 128 * 8 + 1: e = defect_launch<R, RO, 128, FftShape, 1>(MGWR_DEFECT_ARGS); break;
      case 256 * 8 + 1: e = defect_launch<R, RO, 256, FftShape, 1>(MGWR_DEFECT_ARGS); break;
      case 512 * 8 + 1: e = defect_launch<R, RO, 512, FftShape, 1>(MGWR_DEFECT_ARGS); break;
      case 1024 * 8 + 1: e = defect_launch<R, RO, 1024, FftShape, 1>(MGWR_DEFECT_ARGS); break;
      case 256 * 8 + 2: e = defect_launch<R, RO, 256, FftShape, 2>(MGWR_DEFECT_ARGS); break;
      case 512 * 8 + 2: e = defect_launch<R, RO, 512, FftShape, 2>(MGWR_DEFECT_ARGS); break;
      case 256 * 8 + 4: e = defect_launch<R, RO, 256, FftShape, 4>(MGWR_DEFECT_ARGS); break;
      default: break;
    }
  }
#undef MGWR_DEFECT_ARGS
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

}  // namespace mgwr

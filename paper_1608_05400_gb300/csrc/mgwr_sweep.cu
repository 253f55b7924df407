// Smoother kernel (one colour half-sweep) and its launcher, all FFT lengths.
#include "mgwr_common.cuh"

namespace mgwr {

// ---------------------------------------------------------------------------------
// smoother: one colour half-sweep (Sec. 3 Eq. red-black, Sec. 6 Eq. red-black_2d)
// ---------------------------------------------------------------------------------

template <class R, int BLOCK, class SH, int E>
__global__ void __launch_bounds__(BLOCK, min_blocks<R>(BLOCK, E))
    k_sweep(const R* __restrict__ f, R* __restrict__ u, R* __restrict__ delta,
            const Cx<R>* __restrict__ spec, const Cx<R>* __restrict__ tw,
            const R* __restrict__ zero, int d, int n, int M, int logL, int par, int all_points,
            R hinv2, int npts, int npairs, size_t fstride, size_t sstride) {
  extern __shared__ unsigned char smem_raw[];
  // instance of a batch: blockIdx.y
  f += blockIdx.y * fstride;
  u += blockIdx.y * fstride;
  if (delta != nullptr) delta += blockIdx.y * fstride;
  spec += blockIdx.y * sstride;
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
  const int kA = 2 * pair, kB = 2 * pair + 1;
  const bool hasB = valid && kB < npts;
  int iA = 0, jA = 0, iB = 0, jB = 0, pA = 0, pB = 0;
  if (valid) {
    if (all_points) {
      pA = kA;
      pB = kB;
    } else {
      pA = colour_point(kA, d, n, par, iA, jA);
      if (hasB) pB = colour_point(kB, d, n, par, iB, jB);
    }
  }
  const size_t pAM = (size_t)pA * M, pBM = (size_t)pB * M;
  // lines read by the gather; absent lines (no partner B, out-of-range group,
  // one-point solve without neighbours) read the zero line
  const R* fA = valid ? f + pAM : zero;
  const R* fB = hasB ? f + pBM : zero;
  const R *qA[4], *qB[4];
  if constexpr (sizeof(R) == 4) {
    neighbour_lines(u, zero, d, n, iA, jA, pAM, M, qA);
    neighbour_lines(u, zero, d, n, iB, jB, pBM, M, qB);
    if (!valid || all_points) qA[0] = qA[1] = qA[2] = qA[3] = zero;
    if (!hasB || all_points) qB[0] = qB[1] = qB[2] = qB[3] = zero;
  }

  auto load = [&](int m) -> Cx<R> {
    if constexpr (sizeof(R) == 4) {  // branch-free through the neighbour pointers
      if (d == 2)
        return Cx<R>{fA[m] + hinv2 * ((qA[0][m] + qA[1][m]) + (qA[2][m] + qA[3][m])),
                     fB[m] + hinv2 * ((qB[0][m] + qB[1][m]) + (qB[2][m] + qB[3][m]))};
      return Cx<R>{fA[m] + hinv2 * (qA[0][m] + qA[1][m]), fB[m] + hinv2 * (qB[0][m] + qB[1][m])};
    } else {  // bounds tested per access: fewer live registers
      Cx<R> b{fA[m], fB[m]};
      if (valid && !all_points) b.x = b.x + hinv2 * neighbour_sum(u, d, n, iA, jA, pAM, M, m);
      if (hasB && !all_points) b.y = b.y + hinv2 * neighbour_sum(u, d, n, iB, jB, pBM, M, m);
      return b;
    }
  };
  Cx<R> v[E][8];
  fft_forward<E>(buf, t, sh, tw, load, v, sync);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int b = t + e * TL;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[e][q] = cmul(v[e][q], spec[8 * b + q]);
  }
  R* uA = u + pAM;
  R* uB = u + pBM;
  auto store = [&](int m, Cx<R> y) {
    if (valid) {
      if (delta != nullptr) delta[pAM + m] = y.x - uA[m];
      uA[m] = y.x;
      if (hasB) {
        if (delta != nullptr) delta[pBM + m] = y.y - uB[m];
        uB[m] = y.y;
      }
    }
  };
  fft_inverse<E>(buf, t, sh, tw, v, store, sync);
}

template <class R, int BLOCK, class SH, int E>
cudaError_t sweep_launch(dim3 grid, size_t smem, cudaStream_t s, const R* f, R* u, R* delta,
                         const Cx<R>* spec, const Cx<R>* tw, const R* zero, int d, int n, int M,
                         int logL, int par, bool all_points, R hinv2, int npts, int npairs,
                         size_t fstride, size_t sstride) {
  cudaError_t e = prepare_smem(k_sweep<R, BLOCK, SH, E>, smem);
  if (e != cudaSuccess) return e;
  k_sweep<R, BLOCK, SH, E><<<grid, BLOCK, smem, s>>>(f, u, delta, spec, tw, zero, d, n, M, logL,
                                                     par, all_points, hinv2, npts, npairs, fstride,
                                                     sstride);
  return cudaSuccess;
}

template <class R>
cudaError_t launch_sweep(const R* f, R* u, R* delta, const Cx<R>* spec, size_t spec_stride,
                         const Cx<R>* tw, const R* zero, Cx<R>* scratch, const LevelShape& ls,
                         int par, bool all_points, R hinv2, int E, cudaStream_t s) {
  if (ls.M > kShortMaxM)
    return launch_sweep_long(f, u, delta, spec, spec_stride, tw, scratch, ls, par, all_points,
                             hinv2, E, s);
  const int d = ls.d, n = ls.n, M = ls.M;
  const int L = 2 * M, logL = ilog2(L);
  E = effective_split(M, (int)sizeof(R) == 4 ? 4 : 8, E);
  if constexpr (sizeof(R) == 4) {
    if ((E & kStaged) && !all_points)
      return launch_sweep_staged(f, u, delta, spec, spec_stride, tw, zero, ls, par, hinv2, E, s);
  }
  E &= ~(kStaged | kTensor | kRadix);
  const int npts = all_points ? (d == 1 ? n : n * n) : colour_count(d, n, par);
  const int npairs = (npts + 1) / 2;
  if (npairs == 0 || ls.batch == 0) return cudaSuccess;
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
#define MGWR_SWEEP_ARGS                                                                     \
  grid, smem, s, f, u, delta, spec, tw, zero, d, n, M, logL, par, all_points, hinv2, npts, \
      npairs, fstride, spec_stride
  if constexpr (sizeof(R) == 4) {
    switch (logL * 8 + E) {
#define MGWR_CASE_E(LG, EE)                                                                   \
  case LG * 8 + EE:                                                                           \
    e = sweep_launch<R, ((1 << LG) / (8 * EE) > 256 ? (1 << LG) / (8 * EE) : 256), FixedShape<LG>, \
                     EE>(MGWR_SWEEP_ARGS);                                                    \
    break;
#define MGWR_CASE(LG) MGWR_CASE_E(LG, 1) MGWR_CASE_E(LG, 2) MGWR_CASE_E(LG, 4)
      MGWR_FIXED_LOGL(MGWR_CASE)
#undef MGWR_CASE
#undef MGWR_CASE_E
      default:
        e = sweep_launch<R, 256, FftShape, 1>(MGWR_SWEEP_ARGS);
        break;
    }
  } else {
    switch (block * 8 + E) {
      case 32 * 8 + 1: e = sweep_launch<R, 32, FftShape, 1>(MGWR_SWEEP_ARGS); break;
      case 64 * 8 + 1: e = sweep_launch<R, 64, FftShape, 1>(MGWR_SWEEP_ARGS); break;
      case 128 * 8 + 1: e = sweep_launch<R, 128, FftShape, 1>(MGWR_SWEEP_ARGS); break;
      case 256 * 8 + 1: e = sweep_launch<R, 256, FftShape, 1>(MGWR_SWEEP_ARGS); break;
      case 512 * 8 + 1: e = sweep_launch<R, 512, FftShape, 1>(MGWR_SWEEP_ARGS); break;
      case 1024 * 8 + 1: e = sweep_launch<R, 1024, FftShape, 1>(MGWR_SWEEP_ARGS); break;
      case 256 * 8 + 2: e = sweep_launch<R, 256, FftShape, 2>(MGWR_SWEEP_ARGS); break;
      case 512 * 8 + 2: e = sweep_launch<R, 512, FftShape, 2>(MGWR_SWEEP_ARGS); break;
      case 256 * 8 + 4: e = sweep_launch<R, 256, FftShape, 4>(MGWR_SWEEP_ARGS); break;
      default: break;
    }
  }
#undef MGWR_SWEEP_ARGS
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

template cudaError_t launch_sweep<double>(const double*, double*, double*, const Cx<double>*,
                                          size_t, const Cx<double>*, const double*, Cx<double>*,
                                          const LevelShape&, int, bool, double, int, cudaStream_t);
template cudaError_t launch_sweep<float>(const float*, float*, float*, const Cx<float>*, size_t,
                                         const Cx<float>*, const float*, Cx<float>*,
                                         const LevelShape&, int, bool, float, int, cudaStream_t);

template cudaError_t launch_sweep<dd>(const dd*, dd*, dd*, const Cx<dd>*, size_t, const Cx<dd>*,
                                      const dd*, Cx<dd>*, const LevelShape&, int, bool, dd, int,
                                      cudaStream_t);

}  // namespace mgwr

// FP32 smoother half-sweep on the register-pass FFT engine (mgwr_fft_rp.cuh),
// and the permutation of the inverse-column spectra into its spectral order.
#include "mgwr_common.cuh"
#include "mgwr_fft_rp.cuh"

namespace mgwr {

namespace {

// Radix plans per transform length (L = 2^7 .. 2^13): two or three passes,
// the last of radix 32; T threads per line pair, 256 threads per block.
#define MGWR_RP_PLANS(X)      \
  X(13, 16, 16, 32, 256)      \
  X(12, 8, 16, 32, 128)       \
  X(11, 8, 8, 32, 64)         \
  X(10, 32, 32, 0, 32)        \
  X(9, 16, 32, 0, 16)         \
  X(8, 8, 32, 0, 8)           \
  X(7, 4, 32, 0, 4)

constexpr int kRpBlock = 256;

__host__ __device__ inline int rp_plan(int logL, int* r) {
  switch (logL) {
#define MGWR_RP_PLAN_CASE(LG, A, B, C, T) \
  case LG:                                \
    r[0] = A;                             \
    r[1] = B;                             \
    r[2] = C;                             \
    return C != 0 ? 3 : 2;
    MGWR_RP_PLANS(MGWR_RP_PLAN_CASE)
#undef MGWR_RP_PLAN_CASE
    default:
      return 0;
  }
}

// Radices of the shared-memory engine of mgwr_fft.cuh for length 2^logL:
// radix-8 stages, then radix 2^(logL mod 3) when that is not 0.
__host__ __device__ inline int engine_plan(int logL, int* r) {
  int np = 0;
  for (int k = 0; k < logL / 3; ++k) r[np++] = 8;
  if (logL % 3 != 0) r[np++] = 1 << (logL % 3);
  return np;
}

// Barrier of the T threads of one line pair (PAIRS pairs per block).
template <int T, int PAIRS>
__device__ __forceinline__ void group_sync(int g) {
  if constexpr (PAIRS == 1) {
    __syncthreads();
  } else if constexpr (T <= 32) {
    __syncwarp();  // every group of a warp runs the same barrier sequence
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(T) : "memory");
  }
}

template <int LOGL, int R0, int R1, int R2, int T>
__global__ void __launch_bounds__(kRpBlock, 2)
    k_sweep_rp(const float* __restrict__ f, float* __restrict__ u, float* __restrict__ delta,
               const Cx<float>* __restrict__ spec, const Cx<float>* __restrict__ tw,
               const float* __restrict__ zero, int d, int n, int M, int par, float hinv2,
               int npts, int npairs, size_t fstride, size_t sstride) {
  using P = rp::Plan<LOGL, R0, R1, R2, T>;
  using C = Cx<float>;
  constexpr int PAIRS = kRpBlock / T;
  extern __shared__ unsigned char smem_raw[];
  f += blockIdx.y * fstride;
  u += blockIdx.y * fstride;
  if (delta != nullptr) delta += blockIdx.y * fstride;
  spec += blockIdx.y * sstride;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int pair = blockIdx.x * PAIRS + g;
  C* buf = reinterpret_cast<C*>(smem_raw) + g * P::SMEM;

  const bool valid = pair < npairs;
  const int kA = 2 * pair, kB = 2 * pair + 1;
  const bool hasB = valid && kB < npts;
  int iA = 0, jA = 0, iB = 0, jB = 0, pA = 0, pB = 0;
  if (valid) {
    pA = colour_point(kA, d, n, par, iA, jA);
    if (hasB) pB = colour_point(kB, d, n, par, iB, jB);
  }
  const size_t pAM = (size_t)pA * M, pBM = (size_t)pB * M;
  const float* fA = valid ? f + pAM : zero;
  const float* fB = hasB ? f + pBM : zero;
  const float *qA[4], *qB[4];
  neighbour_lines(u, zero, d, n, iA, jA, pAM, M, qA);
  neighbour_lines(u, zero, d, n, iB, jB, pBM, M, qB);
  if (!valid) qA[0] = qA[1] = qA[2] = qA[3] = zero;
  if (!hasB) qB[0] = qB[1] = qB[2] = qB[3] = zero;

  // ---- pass 0: gather the right-hand sides (every load of the thread issued
  // before the first DFT), half-input DFT, twiddles
  constexpr int NB0 = P::S0 / T;
  C in[NB0][R0 / 2];
#pragma unroll
  for (int i = 0; i < NB0; ++i) {
#pragma unroll
    for (int q = 0; q < R0 / 2; ++q) {
      const int m = t + T * i + q * P::S0;
      if (d == 2)
        in[i][q] = C{fA[m] + hinv2 * ((qA[0][m] + qA[1][m]) + (qA[2][m] + qA[3][m])),
                     fB[m] + hinv2 * ((qB[0][m] + qB[1][m]) + (qB[2][m] + qB[3][m]))};
      else
        in[i][q] = C{fA[m] + hinv2 * (qA[0][m] + qA[1][m]), fB[m] + hinv2 * (qB[0][m] + qB[1][m])};
    }
  }
#pragma unroll
  for (int i = 0; i < NB0; ++i) {
    const int j = t + T * i;
    const rp::TwBase<R0> tb(tw, j);
    C v[R0];
#pragma unroll
    for (int q = 0; q < R0 / 2; ++q) v[q] = in[i][q];
    rp::dft_half<R0>(v);
    rp::twiddle_apply<R0, false>(v, tb);
#pragma unroll
    for (int k = 0; k < R0; ++k) buf[P::idx(j + k * P::S0)] = v[k];
  }
  group_sync<T, PAIRS>(g);

  // ---- pass 1 when there are three: radix R1 on groups of G1, twiddles w_G1^{jk}
  if constexpr (P::NP == 3) {
    constexpr int NB1 = (P::L / R1) / T;
#pragma unroll 1
    for (int i = 0; i < NB1; ++i) {
      const int beta = t + T * i;
      const int grp = beta / P::S1, j = beta - grp * P::S1;
      const int base = grp * P::G1 + j;
      const rp::TwBase<R1> tb(tw, j * R0);
      C v[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) v[q] = buf[P::idx(base + q * P::S1)];
      rp::Dft<R1, false>::run(v);
      rp::twiddle_apply<R1, false>(v, tb);
#pragma unroll
      for (int q = 0; q < R1; ++q) buf[P::idx(base + q * P::S1)] = v[q];
    }
    group_sync<T, PAIRS>(g);
  }

  // ---- last pass (contiguous RL values), spectrum product, its inverse
  constexpr int RL = P::RL;
  constexpr int NBL = (P::L / RL) / T;
#pragma unroll 1
  for (int i = 0; i < NBL; ++i) {
    const int base = (t + T * i) * RL;
    C v[RL];
#pragma unroll
    for (int q = 0; q < RL; ++q) v[q] = buf[P::idx(base + q)];
    rp::Dft<RL, false>::run(v);
    const float4* sp = reinterpret_cast<const float4*>(spec + base);
#pragma unroll
    for (int q = 0; q < RL / 2; ++q) {
      const float4 s2 = __ldg(sp + q);
      v[2 * q] = cmul(v[2 * q], C{s2.x, s2.y});
      v[2 * q + 1] = cmul(v[2 * q + 1], C{s2.z, s2.w});
    }
    rp::Dft<RL, true>::run(v);
#pragma unroll
    for (int q = 0; q < RL; ++q) buf[P::idx(base + q)] = v[q];
  }
  group_sync<T, PAIRS>(g);

  // ---- inverse of pass 1
  if constexpr (P::NP == 3) {
    constexpr int NB1 = (P::L / R1) / T;
#pragma unroll 1
    for (int i = 0; i < NB1; ++i) {
      const int beta = t + T * i;
      const int grp = beta / P::S1, j = beta - grp * P::S1;
      const int base = grp * P::G1 + j;
      const rp::TwBase<R1> tb(tw, j * R0);
      C v[R1];
#pragma unroll
      for (int q = 0; q < R1; ++q) v[q] = buf[P::idx(base + q * P::S1)];
      rp::twiddle_apply<R1, true>(v, tb);
      rp::Dft<R1, true>::run(v);
#pragma unroll
      for (int q = 0; q < R1; ++q) buf[P::idx(base + q * P::S1)] = v[q];
    }
    group_sync<T, PAIRS>(g);
  }

  // ---- inverse of pass 0: the first M outputs, the update and the change record
  float* uA = u + pAM;
  float* uB = u + pBM;
#pragma unroll
  for (int i = 0; i < NB0; ++i) {
    const int j = t + T * i;
    const rp::TwBase<R0> tb(tw, j);
    C v[R0];
#pragma unroll
    for (int k = 0; k < R0; ++k) v[k] = buf[P::idx(j + k * P::S0)];
    rp::twiddle_apply<R0, true>(v, tb);
    rp::Dft<R0, true>::run(v);
    if (valid) {
#pragma unroll
      for (int q = 0; q < R0 / 2; ++q) {
        const int m = j + q * P::S0;
        if (delta != nullptr) delta[pAM + m] = v[q].x - uA[m];
        uA[m] = v[q].x;
        if (hasB) {
          if (delta != nullptr) delta[pBM + m] = v[q].y - uB[m];
          uB[m] = v[q].y;
        }
      }
    }
  }
}

// spec_rp[c L + rp position of k] = (float) spec64[c L + engine position of k]
__global__ void k_spectra_rp(Cx<float>* __restrict__ dst, const Cx<double>* __restrict__ src,
                             size_t lines, int logL) {
  const int L = 1 << logL;
  int re[16], rr[3];
  const int ne = engine_plan(logL, re);
  const int nr = rp_plan(logL, rr);
  const size_t total = lines * (size_t)L;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
       x += (size_t)gridDim.x * blockDim.x) {
    const size_t c = x / L;
    const int k = (int)(x - c * L);
    const Cx<double> s = src[c * L + rp_position(k, re, ne)];
    dst[c * L + rp_position(k, rr, nr)] = Cx<float>{(float)s.x, (float)s.y};
  }
}

template <int LOGL, int R0, int R1, int R2, int T>
cudaError_t sweep_rp_launch(dim3 grid, cudaStream_t s, const float* f, float* u, float* delta,
                            const Cx<float>* spec, const Cx<float>* tw, const float* zero, int d,
                            int n, int M, int par, float hinv2, int npts, int npairs,
                            size_t fstride, size_t sstride) {
  using P = rp::Plan<LOGL, R0, R1, R2, T>;
  const size_t smem = (size_t)(kRpBlock / T) * P::SMEM * sizeof(Cx<float>);
  cudaError_t e = prepare_smem(k_sweep_rp<LOGL, R0, R1, R2, T>, smem);
  if (e != cudaSuccess) return e;
  k_sweep_rp<LOGL, R0, R1, R2, T><<<grid, kRpBlock, smem, s>>>(
      f, u, delta, spec, tw, zero, d, n, M, par, hinv2, npts, npairs, fstride, sstride);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_sweep_rp(const float* f, float* u, float* delta, const Cx<float>* spec,
                            size_t spec_stride, const Cx<float>* tw, const float* zero,
                            const LevelShape& ls, int par, float hinv2, cudaStream_t s) {
  const int d = ls.d, n = ls.n, M = ls.M;
  if (!radix_length(M)) return cudaErrorInvalidValue;
  const int logL = ilog2(2 * M);
  const int npts = colour_count(d, n, par);
  const int npairs = (npts + 1) / 2;
  if (npairs == 0 || ls.batch == 0) return cudaSuccess;
  const size_t fstride = ls.field_stride();
  cudaError_t e = cudaErrorInvalidValue;
  switch (logL) {
#define MGWR_RP_LAUNCH(LG, A, B, C, T)                                                       \
  case LG: {                                                                                 \
    const dim3 grid((unsigned)((npairs + kRpBlock / T - 1) / (kRpBlock / T)), (unsigned)ls.batch); \
    e = sweep_rp_launch<LG, A, B, C, T>(grid, s, f, u, delta, spec, tw, zero, d, n, M, par,   \
                                        hinv2, npts, npairs, fstride, spec_stride);          \
    break;                                                                                   \
  }
    MGWR_RP_PLANS(MGWR_RP_LAUNCH)
#undef MGWR_RP_LAUNCH
    default:
      break;
  }
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

cudaError_t launch_spectra_rp(Cx<float>* dst, const Cx<double>* src, size_t lines, int M,
                              cudaStream_t s) {
  if (!radix_length(M)) return cudaErrorInvalidValue;
  const size_t total = lines * 2 * (size_t)M;
  k_spectra_rp<<<elementwise_grid(total), 256, 0, s>>>(dst, src, lines, ilog2(2 * M));
  return counted(cudaGetLastError());
}

}  // namespace mgwr

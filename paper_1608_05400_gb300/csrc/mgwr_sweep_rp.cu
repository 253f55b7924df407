// FP32 smoother half-sweep on the register-pass FFT engine (mgwr_fft_rp.cuh),
// and the permutation of the inverse-column spectra into its spectral order.
#include "mgwr_common.cuh"
#include "mgwr_fft_rp.cuh"

namespace mgwr {

namespace {

// PAIRED: the first pass takes adjacent butterflies two at a time, with 8-byte
// gathers and stores (rp::convolve2), else one at a time (rp::convolve); the
// tuner picks per level (faster for 256-step lines, slower for 1024 and 4096).
template <int LOGL, int R0, int R1, int R2, int R3, int T, bool PAIRED>
__global__ void __launch_bounds__(kRpBlock, (rp::Plan<LOGL, R0, R1, R2, R3, T>::MIN_BLOCKS))
    k_sweep_rp(const float* __restrict__ f, float* __restrict__ u, float* __restrict__ delta,
               const Cx<float>* __restrict__ spec, const Cx<float>* __restrict__ tw,
               const float* __restrict__ zero, int d, int n, int M, int par, float hinv2,
               int npts, int npairs, size_t fstride, size_t sstride) {
  using P = rp::Plan<LOGL, R0, R1, R2, R3, T>;
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

  if constexpr (!PAIRED) {
    auto load = [&](int m) -> C {
      if (d == 2)
        return C{fA[m] + hinv2 * ((qA[0][m] + qA[1][m]) + (qA[2][m] + qA[3][m])),
                 fB[m] + hinv2 * ((qB[0][m] + qB[1][m]) + (qB[2][m] + qB[3][m]))};
      return C{fA[m] + hinv2 * (qA[0][m] + qA[1][m]), fB[m] + hinv2 * (qB[0][m] + qB[1][m])};
    };
    float* uA = u + pAM;
    float* uB = u + pBM;
    auto store = [&](int m, C y) {
      if (valid) {
        if (delta != nullptr) delta[pAM + m] = y.x - uA[m];
        uA[m] = y.x;
        if (hasB) {
          if (delta != nullptr) delta[pBM + m] = y.y - uB[m];
          uB[m] = y.y;
        }
      }
    };
    rp::convolve<LOGL, R0, R1, R2, R3, T, PAIRS>(buf, t, g, rp::GlobalTables{tw, spec}, load,
                                                 store);
    return;
  }
  // times m and m + 1 (m even) of a line as one 8-byte load
  auto ld2 = [](const float* p, int m) { return *reinterpret_cast<const float2*>(p + m); };
  auto load2 = [&](int m) -> rp::Pair2 {
    const float2 a = ld2(fA, m), b = ld2(fB, m);
    const float2 a0 = ld2(qA[0], m), a1 = ld2(qA[1], m), b0 = ld2(qB[0], m), b1 = ld2(qB[1], m);
    float2 sa{a0.x + a1.x, a0.y + a1.y}, sb{b0.x + b1.x, b0.y + b1.y};
    if (d == 2) {
      const float2 a2 = ld2(qA[2], m), a3 = ld2(qA[3], m), b2 = ld2(qB[2], m), b3 = ld2(qB[3], m);
      sa = float2{sa.x + (a2.x + a3.x), sa.y + (a2.y + a3.y)};
      sb = float2{sb.x + (b2.x + b3.x), sb.y + (b2.y + b3.y)};
    }
    return rp::Pair2{C{a.x + hinv2 * sa.x, b.x + hinv2 * sb.x},
                     C{a.y + hinv2 * sa.y, b.y + hinv2 * sb.y}};
  };
  float* uA = u + pAM;
  float* uB = u + pBM;
  auto store2 = [&](int m, C y0, C y1) {
    if (valid) {
      float2* ua = reinterpret_cast<float2*>(uA + m);
      if (delta != nullptr) {
        const float2 o = *ua;
        *reinterpret_cast<float2*>(delta + pAM + m) = float2{y0.x - o.x, y1.x - o.y};
      }
      *ua = float2{y0.x, y1.x};
      if (hasB) {
        float2* ub = reinterpret_cast<float2*>(uB + m);
        if (delta != nullptr) {
          const float2 o = *ub;
          *reinterpret_cast<float2*>(delta + pBM + m) = float2{y0.y - o.x, y1.y - o.y};
        }
        *ub = float2{y0.y, y1.y};
      }
    }
  };
  auto store_all = [&](int j, const C (&y)[2][R0 / 2]) {
#pragma unroll
    for (int q = 0; q < R0 / 2; ++q) store2(j + q * P::S0, y[0][q], y[1][q]);
  };
  rp::convolve2<LOGL, R0, R1, R2, R3, T, PAIRS>(buf, t, g, rp::GlobalTables{tw, spec}, load2,
                                                store_all);
}

// The paired half-sweep with resident blocks: kRpResBlock threads (that many /
// T line pairs at a time) per block and one block per SM, each block looping
// over line pairs with the spectrum and the twiddle bases copied once into
// shared memory (rp::SharedTables), where k_sweep_rp reads them through the
// caches for every butterfly; the line between the two points of a pair is
// loaded once; the black half-sweep loads the old values of a butterfly's
// outputs before its first store.  The same arithmetic as the
// paired k_sweep_rp: bitwise the same results.
template <int LOGL, int R0, int R1, int R2, int R3, int T>
__global__ void __launch_bounds__(kRpResBlock, 1)
    k_sweep_rp_res(const float* __restrict__ f, float* __restrict__ u, float* __restrict__ delta,
                   const Cx<float>* __restrict__ spec, const Cx<float>* __restrict__ tw,
                   const float* __restrict__ zero, int d, int n, int M, int par, float hinv2,
                   int npts, int npairs, size_t fstride, size_t sstride) {
  using P = rp::Plan<LOGL, R0, R1, R2, R3, T>;
  using TB = rp::SharedTables<LOGL, R0, R1, R2, R3>;
  using C = Cx<float>;
  constexpr int PAIRS = kRpResBlock / T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  f += blockIdx.y * fstride;
  u += blockIdx.y * fstride;
  if (delta != nullptr) delta += blockIdx.y * fstride;
  spec += blockIdx.y * sstride;
  unsigned char* tmem = smem_raw + (size_t)PAIRS * P::SMEM * sizeof(C);
  TB::fill(tmem, tw, spec, threadIdx.x, kRpResBlock);
  __syncthreads();
  const TB tab(tmem);
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  C* buf = reinterpret_cast<C*>(smem_raw) + g * P::SMEM;
  auto ld2 = [](const float* p, int m) { return *reinterpret_cast<const float2*>(p + m); };

  // every group runs the block's iterations (its barriers are the group's);
  // a pair beyond the last reads the zero line and stores nothing
  for (int first = blockIdx.x * PAIRS; first < npairs; first += gridDim.x * PAIRS) {
    const int pair = first + g;
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
    // the two points of a pair on one row share the line between them
    const bool shared = qB[0] == qA[1] && hasB;
    auto load2 = [&](int m) -> rp::Pair2 {
      const float2 a = ld2(fA, m), b = ld2(fB, m);
      const float2 a0 = ld2(qA[0], m), a1 = ld2(qA[1], m), b1 = ld2(qB[1], m);
      const float2 b0 = shared ? a1 : ld2(qB[0], m);
      float2 sa{a0.x + a1.x, a0.y + a1.y}, sb{b0.x + b1.x, b0.y + b1.y};
      if (d == 2) {
        const float2 a2 = ld2(qA[2], m), a3 = ld2(qA[3], m), b2 = ld2(qB[2], m),
                     b3 = ld2(qB[3], m);
        sa = float2{sa.x + (a2.x + a3.x), sa.y + (a2.y + a3.y)};
        sb = float2{sb.x + (b2.x + b3.x), sb.y + (b2.y + b3.y)};
      }
      return rp::Pair2{C{a.x + hinv2 * sa.x, b.x + hinv2 * sb.x},
                       C{a.y + hinv2 * sa.y, b.y + hinv2 * sb.y}};
    };
    float* uA = u + pAM;
    float* uB = u + pBM;
    // outputs of butterflies j, j + 1: times j + q S0 and j + 1 + q S0
    auto store_all = [&](int j, const C (&y)[2][R0 / 2]) {
      if (!valid) return;
      if (delta != nullptr) {
        float2 oa[R0 / 2], ob[R0 / 2];
#pragma unroll
        for (int q = 0; q < R0 / 2; ++q) {
          oa[q] = ld2(uA, j + q * P::S0);
          ob[q] = hasB ? ld2(uB, j + q * P::S0) : float2{0.f, 0.f};
        }
#pragma unroll
        for (int q = 0; q < R0 / 2; ++q) {
          const int m = j + q * P::S0;
          *reinterpret_cast<float2*>(delta + pAM + m) =
              float2{y[0][q].x - oa[q].x, y[1][q].x - oa[q].y};
          *reinterpret_cast<float2*>(uA + m) = float2{y[0][q].x, y[1][q].x};
          if (hasB) {
            *reinterpret_cast<float2*>(delta + pBM + m) =
                float2{y[0][q].y - ob[q].x, y[1][q].y - ob[q].y};
            *reinterpret_cast<float2*>(uB + m) = float2{y[0][q].y, y[1][q].y};
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < R0 / 2; ++q) {
          const int m = j + q * P::S0;
          *reinterpret_cast<float2*>(uA + m) = float2{y[0][q].x, y[1][q].x};
          if (hasB) *reinterpret_cast<float2*>(uB + m) = float2{y[0][q].y, y[1][q].y};
        }
      }
    };
    rp::convolve2<LOGL, R0, R1, R2, R3, T, PAIRS>(buf, t, g, tab, load2, store_all);
    rp::group_sync<T, PAIRS>(g);  // the next pair's first pass rewrites buf
  }
}

// spec_rp[c L + rp position of k] = (float) spec64[c L + engine position of k]
// (rp positions of the sweeps' plans, or of the carried defect's when `defect`)
__global__ void k_spectra_rp(Cx<float>* __restrict__ dst, const Cx<double>* __restrict__ src,
                             size_t lines, int logL, bool defect) {
  const int L = 1 << logL;
  int re[16], rr[4];
  const int ne = engine_plan(logL, re);
  const int nr = rp_plan(logL, rr, defect);
  const size_t total = lines * (size_t)L;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total;
       x += (size_t)gridDim.x * blockDim.x) {
    const size_t c = x / L;
    const int k = (int)(x - c * L);
    const Cx<double> s = src[c * L + rp_position(k, re, ne)];
    dst[c * L + rp_position(k, rr, nr)] = Cx<float>{(float)s.x, (float)s.y};
  }
}

template <int LOGL, int R0, int R1, int R2, int R3, int T, bool PAIRED>
cudaError_t sweep_rp_launch(dim3 grid, cudaStream_t s, const float* f, float* u, float* delta,
                            const Cx<float>* spec, const Cx<float>* tw, const float* zero, int d,
                            int n, int M, int par, float hinv2, int npts, int npairs,
                            size_t fstride, size_t sstride) {
  using P = rp::Plan<LOGL, R0, R1, R2, R3, T>;
  const size_t smem = (size_t)(kRpBlock / T) * P::SMEM * sizeof(Cx<float>);
  cudaError_t e = prepare_smem(k_sweep_rp<LOGL, R0, R1, R2, R3, T, PAIRED>, smem);
  if (e != cudaSuccess) return e;
  k_sweep_rp<LOGL, R0, R1, R2, R3, T, PAIRED><<<grid, kRpBlock, smem, s>>>(
      f, u, delta, spec, tw, zero, d, n, M, par, hinv2, npts, npairs, fstride, sstride);
  return cudaSuccess;
}

// Resident form: one block of kRpResBlock threads per SM (across the batch's
// instances, at least one block per instance), never more blocks than pairs
// need.
template <int LOGL, int R0, int R1, int R2, int R3, int T>
cudaError_t sweep_rp_res_launch(int batch, cudaStream_t s, const float* f, float* u, float* delta,
                                const Cx<float>* spec, const Cx<float>* tw, const float* zero,
                                int d, int n, int M, int par, float hinv2, int npts, int npairs,
                                size_t fstride, size_t sstride) {
  using P = rp::Plan<LOGL, R0, R1, R2, R3, T>;
  using TB = rp::SharedTables<LOGL, R0, R1, R2, R3>;
  constexpr int PAIRS = kRpResBlock / T;
  constexpr size_t smem = (size_t)PAIRS * P::SMEM * sizeof(Cx<float>) + TB::BYTES;
  static_assert(smem <= 227 * 1024, "resident sweep exceeds the shared memory of a block");
  cudaError_t e = prepare_smem(k_sweep_rp_res<LOGL, R0, R1, R2, R3, T>, smem);
  if (e != cudaSuccess) return e;
  const int need = (npairs + PAIRS - 1) / PAIRS;
  int per = sm_count() / batch;
  if (per < 1) per = 1;
  const dim3 grid((unsigned)(need < per ? need : per), (unsigned)batch);
  k_sweep_rp_res<LOGL, R0, R1, R2, R3, T><<<grid, kRpResBlock, smem, s>>>(
      f, u, delta, spec, tw, zero, d, n, M, par, hinv2, npts, npairs, fstride, sstride);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_sweep_rp(const float* f, float* u, float* delta, const Cx<float>* spec,
                            size_t spec_stride, const Cx<float>* tw, const float* zero,
                            const LevelShape& ls, int par, float hinv2, int form,
                            cudaStream_t s) {
  const int d = ls.d, n = ls.n, M = ls.M;
  if (!radix_length(M)) return cudaErrorInvalidValue;
  const int logL = ilog2(2 * M);
  const int npts = colour_count(d, n, par);
  const int npairs = (npts + 1) / 2;
  if (npairs == 0 || ls.batch == 0) return cudaSuccess;
  const size_t fstride = ls.field_stride();
  cudaError_t e = cudaErrorInvalidValue;
  switch (logL) {
#define MGWR_RP_LAUNCH(LG, A, B, C, D, T)                                                    \
  case LG: {                                                                                 \
    const dim3 grid((unsigned)((npairs + kRpBlock / T - 1) / (kRpBlock / T)), (unsigned)ls.batch); \
    if (form == kRpResident)                                                                 \
      e = sweep_rp_res_launch<LG, A, B, C, D, T>(ls.batch, s, f, u, delta, spec, tw, zero, d, \
                                                 n, M, par, hinv2, npts, npairs, fstride,    \
                                                 spec_stride);                               \
    else if (form == kRpPaired)                                                              \
      e = sweep_rp_launch<LG, A, B, C, D, T, true>(grid, s, f, u, delta, spec, tw, zero, d, n,  \
                                                   M, par, hinv2, npts, npairs, fstride,     \
                                                   spec_stride);                             \
    else                                                                                     \
      e = sweep_rp_launch<LG, A, B, C, D, T, false>(grid, s, f, u, delta, spec, tw, zero, d, n, \
                                                    M, par, hinv2, npts, npairs, fstride,    \
                                                    spec_stride);                            \
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
                              bool defect, cudaStream_t s) {
  if (!radix_length(M)) return cudaErrorInvalidValue;
  const size_t total = lines * 2 * (size_t)M;
  k_spectra_rp<<<elementwise_grid(total), 256, 0, s>>>(dst, src, lines, ilog2(2 * M), defect);
  return counted(cudaGetLastError());
}

}  // namespace mgwr

// Outer defect of the mixed-precision refinement in its cheap form: the
// defect is carried from one outer step to the next by the correction e that
// the step's FP32 cycles computed (u_new = u_old + e, so
// r_new = r_old - (T_M (x) I + A_h) e), with the time convolution T_M e as one
// FP32 FFT convolution of e, and the stencil A_h e and the subtraction in
// double-float, where the stencil's cancellation on the smooth e would
// otherwise lose |A_h| ~ 4d/h^2 of its digits (FP32 arithmetic only: GB300
// runs FP64 at 1/64 of the FP32 rate).  The FP32 convolution errs by about
// 1e-6 of |T_M e|, and |T_M e| is about the size of r_old, so the carried
// defect errs by about 1e-6 of the defect at the last full computation,
// however far the steps since have reduced it (residual replacement: the
// solve computes the full defect again once that error could matter).  Both
// mixed modes hold the carried defect in double-float, whose 2^-48 rounding
// is far below that error.
#include "mgwr_common.cuh"
#include "mgwr_fft_rp.cuh"

namespace mgwr {

namespace {

// sum over the 2d neighbour lines q of (e_p - e_q) at time m as a double-float
// pair: every difference of two FP32 values is exact as a TwoSum pair, the
// leading words are summed by TwoSum and the trailing ones plainly (error
// about 2^-48 of the differences' magnitudes).  Neighbours outside the grid
// are the zero line, so the difference is e_p there.
__device__ __forceinline__ dd exact_differences(const float* const (&q)[4], float ep, int d,
                                                int m) {
  dd acc = dd_two_sum(ep, -q[0][m]);
  const int nq = 2 * d;
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    if (k < nq) {
      const dd t = dd_two_sum(ep, -q[k][m]);
      const dd s = dd_two_sum(acc.hi, t.hi);
      acc = dd(s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, t.lo)));
    }
  }
  return dd_fast_two_sum(acc.hi, acc.lo);
}

// the per-instance maximum of |r_new| into norm_bits (one atomic per block)
template <int BLOCK>
__device__ __forceinline__ void block_norm(double a, double* red,
                                           unsigned long long* __restrict__ norm_bits) {
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

// One line pair's update, shared by both engines: the store of the inverse
// transform's outputs y = T_M e (A and B lines in y.x and y.y).  hinv2 = 1/h^2
// = (n + 1)^2 is a power of 4 (n + 1 is a power of two), so scaling a
// double-float pair by it is exact word by word.
template <class W>
struct UpdateStore {
  const float* e;
  const W* r_in;
  W* r_out;
  float* r32;
  float hinv2;
  int d;
  bool valid, hasB;
  size_t pAM, pBM;
  const float *qA[4], *qB[4];
  float* amax;
  __device__ __forceinline__ void one(size_t pM, int m, const float* const (&q)[4],
                                      float ty) const {
    const dd s = exact_differences(q, e[pM + m], d, m);
    const dd as = dd_add_float(dd(hinv2 * s.hi, hinv2 * s.lo), ty);  // (A e) at this value
    const dd r = dd_add_accurate(r_in[pM + m], -as);
    r_out[pM + m] = r;
    r32[pM + m] = float(r);
    *amax = absmax_nan(fabsf(r.hi), *amax);
  }
  __device__ __forceinline__ void operator()(int m, Cx<float> y) const {
    if (!valid) return;
    one(pAM, m, qA, y.x);
    if (hasB) one(pBM, m, qB, y.y);
  }
};

}  // namespace

// r_in and r_out may be the same field (each value is read, then written, by
// the same thread); e is only read.
template <class W, int BLOCK, class SH>
__global__ void __launch_bounds__(BLOCK, min_blocks<float>(BLOCK))
    k_defect_update(const float* __restrict__ e, const W* r_in, W* r_out, float* __restrict__ r32,
                    const Cx<float>* __restrict__ tspec, const Cx<float>* __restrict__ tw,
                    const float* __restrict__ zero, int d, int n, int M, int logL, float hinv2,
                    int npts, int npairs, unsigned long long* __restrict__ norm_bits,
                    size_t fstride, size_t sstride) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[BLOCK / 32];
  const size_t off = blockIdx.y * fstride;
  tspec += blockIdx.y * sstride;
  const SH sh(logL);
  const int TL = sh.L8;
  const int g = threadIdx.x / TL;
  const int t = threadIdx.x - g * TL;
  const int pair = blockIdx.x * (BLOCK / TL) + g;
  Cx<float>* buf = reinterpret_cast<Cx<float>*>(smem_raw) + g * Pad<float>::len(sh.L);
  const GroupSync sync(TL, BLOCK, g);

  const bool valid = pair < npairs;
  const int pA = 2 * pair, pB = 2 * pair + 1;
  const bool hasB = valid && pB < npts;
  float amax = 0.f;
  UpdateStore<W> store;
  store.e = e + off;
  store.r_in = r_in + off;
  store.r_out = r_out + off;
  store.r32 = r32 + off;
  store.hinv2 = hinv2;
  store.d = d;
  store.valid = valid;
  store.hasB = hasB;
  store.pAM = (size_t)pA * M;
  store.pBM = (size_t)pB * M;
  store.amax = &amax;
  neighbour_lines(store.e, zero, d, n, d == 1 ? pA : pA % n, d == 1 ? 0 : pA / n, store.pAM, M,
                  store.qA);
  neighbour_lines(store.e, zero, d, n, d == 1 ? pB : pB % n, d == 1 ? 0 : pB / n, store.pBM, M,
                  store.qB);
  const float* eA = valid ? store.e + store.pAM : zero;
  const float* eB = hasB ? store.e + store.pBM : zero;
  auto load = [&](int m) -> Cx<float> { return Cx<float>{eA[m], eB[m]}; };
  Cx<float> v[1][8];
  fft_forward<1>(buf, t, sh, tw, load, v, sync);
#pragma unroll
  for (int q = 0; q < 8; ++q) v[0][q] = cmul(v[0][q], tspec[8 * t + q]);
  fft_inverse<1>(buf, t, sh, tw, v, store, sync);
  if (norm_bits != nullptr) block_norm<BLOCK>((double)amax, red, norm_bits + blockIdx.y);
}

// The same on the register-pass engine (mgwr_fft_rp.cuh, the carried defect's
// plan table): tspec in that plan's spectral order.
template <class W, int LOGL, int R0, int R1, int R2, int R3, int T>
__global__ void __launch_bounds__(kRpBlock, (rp::Plan<LOGL, R0, R1, R2, R3, T>::MIN_BLOCKS))
    k_defect_update_rp(const float* __restrict__ e, const W* r_in, W* r_out,
                       float* __restrict__ r32, const Cx<float>* __restrict__ tspec,
                       const Cx<float>* __restrict__ tw, const float* __restrict__ zero, int d,
                       int n, int M, float hinv2, int npts, int npairs,
                       unsigned long long* __restrict__ norm_bits, size_t fstride,
                       size_t sstride) {
  using P = rp::Plan<LOGL, R0, R1, R2, R3, T>;
  constexpr int PAIRS = kRpBlock / T;
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[kRpBlock / 32];
  const size_t off = blockIdx.y * fstride;
  tspec += blockIdx.y * sstride;
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int pair = blockIdx.x * PAIRS + g;
  Cx<float>* buf = reinterpret_cast<Cx<float>*>(smem_raw) + g * P::SMEM;
  const bool valid = pair < npairs;
  const int pA = 2 * pair, pB = 2 * pair + 1;
  const bool hasB = valid && pB < npts;
  float amax = 0.f;
  UpdateStore<W> store;
  store.e = e + off;
  store.r_in = r_in + off;
  store.r_out = r_out + off;
  store.r32 = r32 + off;
  store.hinv2 = hinv2;
  store.d = d;
  store.valid = valid;
  store.hasB = hasB;
  store.pAM = (size_t)pA * M;
  store.pBM = (size_t)pB * M;
  store.amax = &amax;
  neighbour_lines(store.e, zero, d, n, d == 1 ? pA : pA % n, d == 1 ? 0 : pA / n, store.pAM, M,
                  store.qA);
  neighbour_lines(store.e, zero, d, n, d == 1 ? pB : pB % n, d == 1 ? 0 : pB / n, store.pBM, M,
                  store.qB);
  const float* eA = valid ? store.e + store.pAM : zero;
  const float* eB = hasB ? store.e + store.pBM : zero;
  auto load = [&](int m) -> Cx<float> { return Cx<float>{eA[m], eB[m]}; };
  rp::convolve<LOGL, R0, R1, R2, R3, T, PAIRS>(buf, t, g, rp::GlobalTables{tw, tspec}, load,
                                               store);
  if (norm_bits != nullptr) block_norm<kRpBlock>((double)amax, red, norm_bits + blockIdx.y);
}

namespace {

template <class W, int BLOCK, class SH>
cudaError_t update_launch(dim3 grid, size_t smem, cudaStream_t s, const float* e, const W* r_in,
                          W* r_out, float* r32, const Cx<float>* tspec, const Cx<float>* tw,
                          const float* zero, int d, int n, int M, int logL, float hinv2, int npts,
                          int npairs, unsigned long long* norm_bits, size_t fstride,
                          size_t sstride) {
  cudaError_t err = prepare_smem(k_defect_update<W, BLOCK, SH>, smem);
  if (err != cudaSuccess) return err;
  k_defect_update<W, BLOCK, SH><<<grid, BLOCK, smem, s>>>(e, r_in, r_out, r32, tspec, tw, zero, d,
                                                          n, M, logL, hinv2, npts, npairs,
                                                          norm_bits, fstride, sstride);
  return cudaSuccess;
}

}  // namespace

template <class W>
cudaError_t launch_defect_update(const float* e, const W* r_in, W* r_out, float* r32,
                                 const Cx<float>* tspec, size_t spec_stride, const Cx<float>* tw,
                                 const float* zero, const LevelShape& ls, float hinv2,
                                 unsigned long long* norm_bits, cudaStream_t s) {
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
  // the run-time shape only: the solver takes the register-pass form for every
  // length it serves (64 <= M <= kShortMaxM), this one for the shorter lines
  cudaError_t err = cudaErrorInvalidValue;
  switch (block) {
    case 256:
      err = update_launch<W, 256, FftShape>(grid, smem, s, e, r_in, r_out, r32, tspec, tw, zero, d,
                                            n, M, logL, hinv2, npts, npairs, norm_bits, fstride,
                                            spec_stride);
      break;
    case 512:
      err = update_launch<W, 512, FftShape>(grid, smem, s, e, r_in, r_out, r32, tspec, tw, zero, d,
                                            n, M, logL, hinv2, npts, npairs, norm_bits, fstride,
                                            spec_stride);
      break;
    case 1024:
      err = update_launch<W, 1024, FftShape>(grid, smem, s, e, r_in, r_out, r32, tspec, tw, zero,
                                             d, n, M, logL, hinv2, npts, npairs, norm_bits,
                                             fstride, spec_stride);
      break;
    default:
      break;
  }
  if (err != cudaSuccess) return err;
  return counted(cudaGetLastError());
}

template <class W>
cudaError_t launch_defect_update_rp(const float* e, const W* r_in, W* r_out, float* r32,
                                    const Cx<float>* tspec, size_t spec_stride,
                                    const Cx<float>* tw, const float* zero, const LevelShape& ls,
                                    float hinv2, unsigned long long* norm_bits, cudaStream_t s) {
  const int d = ls.d, n = ls.n, M = ls.M;
  if (!radix_length(M)) return cudaErrorInvalidValue;
  const int npts = d == 1 ? n : n * n;
  const int npairs = (npts + 1) / 2;
  if (ls.batch == 0) return cudaSuccess;
  const size_t fstride = ls.field_stride();
  cudaError_t err = cudaErrorInvalidValue;
  switch (ilog2(2 * M)) {
#define MGWR_RP_UPDATE(LG, A, B, C, D, T)                                                        \
  case LG: {                                                                                    \
    using P = rp::Plan<LG, A, B, C, D, T>;                                                         \
    const size_t smem = (size_t)(kRpBlock / T) * P::SMEM * sizeof(Cx<float>);                   \
    err = prepare_smem(k_defect_update_rp<W, LG, A, B, C, D, T>, smem);                            \
    if (err != cudaSuccess) return err;                                                         \
    const dim3 grid((unsigned)((npairs + kRpBlock / T - 1) / (kRpBlock / T)),                   \
                    (unsigned)ls.batch);                                                        \
    k_defect_update_rp<W, LG, A, B, C, D, T><<<grid, kRpBlock, smem, s>>>(                         \
        e, r_in, r_out, r32, tspec, tw, zero, d, n, M, hinv2, npts, npairs, norm_bits, fstride, \
        spec_stride);                                                                           \
    break;                                                                                      \
  }
    MGWR_RP_DEFECT_PLANS(MGWR_RP_UPDATE)
#undef MGWR_RP_UPDATE
    default:
      break;
  }
  if (err != cudaSuccess) return err;
  return counted(cudaGetLastError());
}

template cudaError_t launch_defect_update<dd>(const float*, const dd*, dd*, float*,
                                             const Cx<float>*, size_t, const Cx<float>*,
                                             const float*, const LevelShape&, float,
                                             unsigned long long*, cudaStream_t);
template cudaError_t launch_defect_update_rp<dd>(const float*, const dd*, dd*, float*,
                                                const Cx<float>*, size_t, const Cx<float>*,
                                                const float*, const LevelShape&, float,
                                                unsigned long long*, cudaStream_t);

}  // namespace mgwr

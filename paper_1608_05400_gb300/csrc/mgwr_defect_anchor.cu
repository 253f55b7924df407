// Full outer defect of MGWR_MIXED in a cheaper arithmetic, for solves to
// tolerances of at least 1e-10: the anchors of the carried defects
// (launch_defect_update) and the defects that decide the stop.
// r = (f - A_h u) - T_M u of the FP64 iterate u, with the stencil, the source
// and the subtractions in FP64 (exact differences first, as in the FP64
// defect) and T_M u by a double-float FFT convolution of u split into
// double-float pairs (dd_split_int).  The split drops u's last five bits
// (2^-48 |u|, far below the convolution's own error) and only reaches T_M u,
// not the stencil, so the defect errs by about 2^-44 of |T_M u|: a few 1e-14 of
// the right-hand side's scale, on any grid.  GB300 runs double-float
// butterflies (FP32 pipes) several times faster than FP64 ones (1/64 of the
// FP32 rate); the FP64 work left is eight operations per value (the stencil's
// seven sums and one fused multiply-add; the splits use integer and FP32
// operations).  The norm is that of the FP32 leading words, within 2^-24 of
// the defect's own.
#include "mgwr_common.cuh"

namespace mgwr {

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, min_blocks<dd>(BLOCK))
    k_defect_anchor(const double* __restrict__ u, const double* __restrict__ f,
                    dd* __restrict__ r, float* __restrict__ r32, const Cx<dd>* __restrict__ tspec,
                    const Cx<dd>* __restrict__ tw, const double* __restrict__ zero, int d, int n,
                    int M, int logL, double hinv2, int npts, int npairs,
                    unsigned long long* __restrict__ norm_bits, size_t fstride, size_t sstride) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[BLOCK / 32];
  const size_t off = blockIdx.y * fstride;
  u += off;
  f += off;
  r += off;
  r32 += off;
  tspec += blockIdx.y * sstride;
  const FftShape sh(logL);
  const int TL = sh.L8;
  const int g = threadIdx.x / TL;
  const int t = threadIdx.x - g * TL;
  const int pair = blockIdx.x * (BLOCK / TL) + g;
  Cx<dd>* buf = reinterpret_cast<Cx<dd>*>(smem_raw) + g * Pad<dd>::len(sh.L);
  const GroupSync sync(TL, BLOCK, g);

  const bool valid = pair < npairs;
  const int pA = 2 * pair, pB = 2 * pair + 1;
  const bool hasB = valid && pB < npts;
  const size_t pAM = (size_t)pA * M, pBM = (size_t)pB * M;
  const int iA = d == 1 ? pA : pA % n, jA = d == 1 ? 0 : pA / n;
  const int iB = d == 1 ? pB : pB % n, jB = d == 1 ? 0 : pB / n;
  const double* uA = valid ? u + pAM : zero;
  const double* uB = hasB ? u + pBM : zero;
  auto load = [&](int m) -> Cx<dd> { return Cx<dd>{dd_split_int(uA[m]), dd_split_int(uB[m])}; };
  Cx<dd> v[1][8];
  fft_forward<1>(buf, t, sh, tw, load, v, sync);
#pragma unroll
  for (int q = 0; q < 8; ++q) v[0][q] = cmul(v[0][q], tspec[8 * t + q]);
  float amax = 0.f;
  // one value (line start pM, time m, T_M u there in y): f - h^-2 sum (u_p - u_q)
  // in FP64 (one fused step after the differences), split, and T_M u
  // subtracted in double-float
  auto one = [&](size_t pM, int m, int i, int j, dd y, double up) {
    const double a = fma(-hinv2, stencil_differences(u, up, d, n, i, j, pM, M, m), f[pM + m]);
    const dd rd = dd_add_accurate(dd_split_int(a), -y);
    r[pM + m] = rd;
    r32[pM + m] = float(rd);
    amax = absmax_nan(fabsf(rd.hi), amax);
  };
  auto store = [&](int m, Cx<dd> y) {
    if (valid) {
      one(pAM, m, iA, jA, y.x, uA[m]);
      if (hasB) one(pBM, m, iB, jB, y.y, uB[m]);
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
      if (threadIdx.x == 0) atomic_max_nonneg(norm_bits + blockIdx.y, a);
    }
  }
}

namespace {

template <int BLOCK>
cudaError_t anchor_launch(dim3 grid, size_t smem, cudaStream_t s, const double* u,
                          const double* f, dd* r, float* r32, const Cx<dd>* tspec,
                          const Cx<dd>* tw, const double* zero, int d, int n, int M, int logL,
                          double hinv2, int npts, int npairs, unsigned long long* norm_bits,
                          size_t fstride, size_t sstride) {
  cudaError_t e = prepare_smem(k_defect_anchor<BLOCK>, smem);
  if (e != cudaSuccess) return e;
  k_defect_anchor<BLOCK><<<grid, BLOCK, smem, s>>>(u, f, r, r32, tspec, tw, zero, d, n, M, logL,
                                                   hinv2, npts, npairs, norm_bits, fstride,
                                                   sstride);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_defect_anchor(const double* u, const double* f, dd* r, float* r32,
                                 const Cx<dd>* tspec, size_t spec_stride, const Cx<dd>* tw,
                                 const double* zero, const LevelShape& ls, double hinv2,
                                 unsigned long long* norm_bits, cudaStream_t s) {
  const int d = ls.d, n = ls.n, M = ls.M;
  if (M > kShortMaxM || M < 4) return cudaErrorInvalidValue;
  const int L = 2 * M, logL = ilog2(L);
  const int npts = d == 1 ? n : n * n;
  const int npairs = (npts + 1) / 2;
  if (ls.batch == 0) return cudaSuccess;
  const size_t fstride = ls.field_stride();
  const int block = block_threads(L);
  const int groups = block / (L / 8);
  const size_t smem = (size_t)groups * Pad<dd>::len(L) * sizeof(Cx<dd>);
  const dim3 grid((unsigned)((npairs + groups - 1) / groups), (unsigned)ls.batch);
  cudaError_t e = cudaErrorInvalidValue;
#define MGWR_ANCHOR_ARGS \
  grid, smem, s, u, f, r, r32, tspec, tw, zero, d, n, M, logL, hinv2, npts, npairs, norm_bits, \
      fstride, spec_stride
  switch (block) {
    case 256: e = anchor_launch<256>(MGWR_ANCHOR_ARGS); break;
    case 512: e = anchor_launch<512>(MGWR_ANCHOR_ARGS); break;
    case 1024: e = anchor_launch<1024>(MGWR_ANCHOR_ARGS); break;
    default: break;
  }
#undef MGWR_ANCHOR_ARGS
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

}  // namespace mgwr

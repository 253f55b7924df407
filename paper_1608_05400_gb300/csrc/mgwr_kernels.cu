// CUDA kernels of the MGWR solver (sm_103a): defect after a smoothing step,
// grid transfers, precision conversions and the FP64 setup (coefficients,
// inverse columns, twiddles, spectra).  The smoother and the full defect live
// in mgwr_sweep.cu and mgwr_defect.cu.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>

#include "mgwr_common.cuh"

namespace mgwr {

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

cudaError_t counted(cudaError_t e) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

long long launch_counter() { return g_launches.load(); }

void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Line-wise kernels: a group of TPL threads owns one time line (TPL =
// min(64, M/W), 256 for lines of more than 1024 vectors; 256 / TPL lines per
// 256-thread block); each thread moves W =
// 16 / sizeof(R) consecutive time values per step with 16-byte accesses (every
// line starts on a 16-byte boundary: M is a power of two >= 4 and the fields
// are allocated 256-byte aligned).  Index arithmetic is done once per line.
constexpr int kLineBlock = 256;

template <class R>
struct Vec {
  static constexpr int W = 16 / sizeof(R);
  R v[W];
};

template <class R>
__device__ __forceinline__ Vec<R> vload(const R* p) {
  Vec<R> x;
  *reinterpret_cast<uint4*>(x.v) = __ldg(reinterpret_cast<const uint4*>(p));
  return x;
}

// the same for a line the kernel also writes (no read-only cache path)
template <class R>
__device__ __forceinline__ Vec<R> vload_rw(const R* p) {
  Vec<R> x;
  *reinterpret_cast<uint4*>(x.v) = *reinterpret_cast<const uint4*>(p);
  return x;
}

template <class R>
__device__ __forceinline__ void vstore(R* p, const Vec<R>& x) {
  *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(x.v);
}

template <class R>
struct LineMap {
  int line, m0, step;
  __device__ __forceinline__ explicit LineMap(int log_tpl) {
    const int tpl = 1 << log_tpl;
    line = blockIdx.x * (kLineBlock >> log_tpl) + (threadIdx.x >> log_tpl);
    m0 = Vec<R>::W * (threadIdx.x & (tpl - 1));
    step = Vec<R>::W * tpl;
  }
};

// Block-wide maximum of `amax` folded into *norm_bits (any block of whole warps,
// at most 1024 threads).
__device__ __forceinline__ void block_absmax(double amax, unsigned long long* norm_bits) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = absmax_nan(__shfl_xor_sync(0xffffffffu, amax, o), amax);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x < 32) {
    amax = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = absmax_nan(__shfl_xor_sync(0xffffffffu, amax, o), amax);
    if (threadIdx.x == 0) atomic_max_nonneg(norm_bits, amax);
  }
}

// Defect right after a complete red-black smoothing step, without a
// convolution.  The second (black) half-sweep left every black point solving
// its own equation exactly, so the defect is 0 there; at a red point the
// equation was solved with the old black neighbours, so its defect is
// h^-2 * sum over its black neighbours of (new - old) = h^-2 sum delta.
template <class R>
__global__ void __launch_bounds__(kLineBlock)
    k_defect_from_delta(const R* __restrict__ delta, R* __restrict__ r, const R* __restrict__ zero,
                        int d, int n, int M, int log_tpl, int npts, int red_par, R hinv2,
                        unsigned long long* __restrict__ norm_bits, size_t fstride) {
  constexpr int W = Vec<R>::W;
  const LineMap<R> lm(log_tpl);
  delta += blockIdx.y * fstride;
  r += blockIdx.y * fstride;
  if (norm_bits != nullptr) norm_bits += blockIdx.y;
  double amax = 0.0;
  if (lm.line < npts) {
    const int p = lm.line;
    const int i = d == 1 ? p : p % n, j = d == 1 ? 0 : p / n;
    const int par = d == 1 ? (i & 1) : ((i + j) & 1);
    R* rp = r + (size_t)p * M;
    if (par != red_par) {
      Vec<R> z;
#pragma unroll
      for (int k = 0; k < W; ++k) z.v[k] = R(0);
      for (int m = lm.m0; m < M; m += lm.step) vstore(rp + m, z);
    } else {
      // neighbour lines, the zero line outside the grid; four reads, three
      // additions and one product per value
      const size_t pM = (size_t)p * M, nM = (size_t)n * M;
      const R* w = i > 0 ? delta + pM - M : zero;
      const R* e = i < n - 1 ? delta + pM + M : zero;
      const R* so = d == 2 && j > 0 ? delta + pM - nM : zero;
      const R* no = d == 2 && j < n - 1 ? delta + pM + nM : zero;
      const bool four = d == 2;
      for (int m = lm.m0; m < M; m += lm.step) {
        const Vec<R> a = vload(w + m), b = vload(e + m);
        Vec<R> c, g, out;
        if (four) {
          c = vload(so + m);
          g = vload(no + m);
        }
#pragma unroll
        for (int k = 0; k < W; ++k) {
          R sum = a.v[k] + b.v[k];
          if (four) sum = sum + (c.v[k] + g.v[k]);
          out.v[k] = hinv2 * sum;
          amax = absmax_nan((double)Arith<R>::mag(out.v[k]), amax);
        }
        vstore(rp + m, out);
      }
    }
  }
  if (norm_bits != nullptr) block_absmax(amax, norm_bits);
}

// ---------------------------------------------------------------------------------
// grid transfers on whole time lines (Algorithm 1; Sec. 3 and Sec. 6)
// ---------------------------------------------------------------------------------

// Full weighting, (1/4)[1 2 1] per dimension; also clears the coarse correction.
template <class R>
__global__ void __launch_bounds__(kLineBlock)
    k_restrict(const R* __restrict__ r, R* __restrict__ fc, R* __restrict__ uc, int d, int n, int M,
               int log_tpl, int ncpts, size_t fstride, size_t cstride) {
  constexpr int W = Vec<R>::W;
  const LineMap<R> lm(log_tpl);
  r += blockIdx.y * fstride;
  fc += blockIdx.y * cstride;
  uc += blockIdx.y * cstride;
  if (lm.line >= ncpts) return;
  const int nc = (n - 1) / 2;
  const int P = lm.line;
  R* fo = fc + (size_t)P * M;
  R* uo = uc + (size_t)P * M;
  Vec<R> z;
#pragma unroll
  for (int k = 0; k < W; ++k) z.v[k] = R(0);
  if (d == 1) {
    const R* c = r + (size_t)(2 * P + 1) * M;
    for (int m = lm.m0; m < M; m += lm.step) {
      const Vec<R> a = vload(c + m - M), b = vload(c + m), e = vload(c + m + M);
      Vec<R> out;
#pragma unroll
      for (int k = 0; k < W; ++k) out.v[k] = R(0.25) * (a.v[k] + R(2) * b.v[k] + e.v[k]);
      vstore(fo + m, out);
      vstore(uo + m, z);
    }
  } else {
    const int I = P % nc, J = P / nc;
    const size_t nM = (size_t)n * M;
    // centre line of the 3 x 3 fine stencil and the rows below / above it
    const R* c = r + ((size_t)(2 * I + 1) + (size_t)(2 * J + 1) * n) * M;
    const R* cs = c - nM;
    const R* cn = c + nM;
    for (int m = lm.m0; m < M; m += lm.step) {
      Vec<R> out;
      {
        const Vec<R> a = vload(cs + m - M), b = vload(cs + m), e = vload(cs + m + M);
#pragma unroll
        for (int k = 0; k < W; ++k) out.v[k] = a.v[k] + R(2) * b.v[k] + e.v[k];
      }
      {
        const Vec<R> a = vload(c + m - M), b = vload(c + m), e = vload(c + m + M);
#pragma unroll
        for (int k = 0; k < W; ++k) out.v[k] = out.v[k] + R(2) * (a.v[k] + R(2) * b.v[k] + e.v[k]);
      }
      {
        const Vec<R> a = vload(cn + m - M), b = vload(cn + m), e = vload(cn + m + M);
#pragma unroll
        for (int k = 0; k < W; ++k) out.v[k] = R(0.0625) * (out.v[k] + (a.v[k] + R(2) * b.v[k] + e.v[k]));
      }
      vstore(fo + m, out);
      vstore(uo + m, z);
    }
  }
}

// a * b rounded on its own (never fused into a following addition), as when
// the product is stored and read back.
__device__ __forceinline__ float mul_rounded(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rounded(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ dd mul_rounded(dd a, dd b) { return a * b; }

// Full weighting of the defect that a complete red-black step leaves (the
// defect from the black half-sweep's changes, see k_defect_from_delta) without
// storing that defect: every fine value of the stencil is formed where it is
// needed, 0 at a black point and hinv2 * (sum of the black neighbours'
// changes) at a red one, and the stencil sums them in k_restrict's order, so
// fc is bitwise what k_defect_from_delta followed by k_restrict gives.  Reads
// the black changes (half a fine field, neighbours shared through L2) instead
// of writing and reading back a whole fine defect; also clears uc.
template <class R>
__global__ void __launch_bounds__(kLineBlock)
    k_restrict_delta(const R* __restrict__ delta, R* __restrict__ fc, R* __restrict__ uc,
                     const R* __restrict__ zero, int d, int n, int M, int log_tpl, int ncpts,
                     int red_par, R hinv2, size_t fstride, size_t cstride) {
  constexpr int W = Vec<R>::W;
  const LineMap<R> lm(log_tpl);
  delta += blockIdx.y * fstride;
  fc += blockIdx.y * cstride;
  uc += blockIdx.y * cstride;
  if (lm.line >= ncpts) return;
  const int nc = (n - 1) / 2;
  const int P = lm.line;
  R* fo = fc + (size_t)P * M;
  R* uo = uc + (size_t)P * M;
  Vec<R> z;
#pragma unroll
  for (int k = 0; k < W; ++k) z.v[k] = R(0);
  const size_t nM = (size_t)n * M;
  // the defect at fine point (i, j), time values m .. m+W-1
  auto r_at = [&](int i, int j, int m) -> Vec<R> {
    const bool red = d == 1 ? (i & 1) == red_par : ((i + j) & 1) == red_par;
    if (!red) return z;
    const size_t pM = ((size_t)i + (size_t)j * n) * M;
    const R* w = i > 0 ? delta + pM - M : zero;
    const R* e = i < n - 1 ? delta + pM + M : zero;
    const Vec<R> a = vload(w + m), b = vload(e + m);
    Vec<R> out;
    if (d == 2) {
      const R* so = j > 0 ? delta + pM - nM : zero;
      const R* no = j < n - 1 ? delta + pM + nM : zero;
      const Vec<R> c = vload(so + m), g = vload(no + m);
#pragma unroll
      for (int k = 0; k < W; ++k) out.v[k] = mul_rounded(hinv2, (a.v[k] + b.v[k]) + (c.v[k] + g.v[k]));
    } else {
#pragma unroll
      for (int k = 0; k < W; ++k) out.v[k] = mul_rounded(hinv2, a.v[k] + b.v[k]);
    }
    return out;
  };
  if (d == 1) {
    const int c = 2 * P + 1;
    for (int m = lm.m0; m < M; m += lm.step) {
      const Vec<R> a = r_at(c - 1, 0, m), b = r_at(c, 0, m), e = r_at(c + 1, 0, m);
      Vec<R> out;
#pragma unroll
      for (int k = 0; k < W; ++k) out.v[k] = R(0.25) * (a.v[k] + R(2) * b.v[k] + e.v[k]);
      vstore(fo + m, out);
      vstore(uo + m, z);
    }
  } else {
    const int ci = 2 * (P % nc) + 1, cj = 2 * (P / nc) + 1;
    for (int m = lm.m0; m < M; m += lm.step) {
      Vec<R> out;
      {
        const Vec<R> a = r_at(ci - 1, cj - 1, m), b = r_at(ci, cj - 1, m), e = r_at(ci + 1, cj - 1, m);
#pragma unroll
        for (int k = 0; k < W; ++k) out.v[k] = a.v[k] + R(2) * b.v[k] + e.v[k];
      }
      {
        const Vec<R> a = r_at(ci - 1, cj, m), b = r_at(ci, cj, m), e = r_at(ci + 1, cj, m);
#pragma unroll
        for (int k = 0; k < W; ++k) out.v[k] = out.v[k] + R(2) * (a.v[k] + R(2) * b.v[k] + e.v[k]);
      }
      {
        const Vec<R> a = r_at(ci - 1, cj + 1, m), b = r_at(ci, cj + 1, m), e = r_at(ci + 1, cj + 1, m);
#pragma unroll
        for (int k = 0; k < W; ++k) out.v[k] = R(0.0625) * (out.v[k] + (a.v[k] + R(2) * b.v[k] + e.v[k]));
      }
      vstore(fo + m, out);
      vstore(uo + m, z);
    }
  }
}

// The 2-D k_restrict_delta with each thread walking kRowRun coarse points of one
// coarse row for one vector of time values: the stencils of neighbouring
// coarse points share a fine column (the right column of one is the left of the
// next), so each fine defect value is formed once per walk instead of once per
// stencil that holds it (12 vector loads of changes per coarse value instead of
// 20).  Every value is formed and summed exactly as in k_restrict_delta: the
// same bits.
constexpr int kRowRun = 8;

template <class R>
__global__ void __launch_bounds__(kLineBlock)
    k_restrict_delta_rows(const R* __restrict__ delta, R* __restrict__ fc, R* __restrict__ uc,
                          const R* __restrict__ zero, int n, int M, int red_par, R hinv2,
                          size_t fstride, size_t cstride) {
  constexpr int W = Vec<R>::W;
  delta += blockIdx.y * fstride;
  fc += blockIdx.y * cstride;
  uc += blockIdx.y * cstride;
  const int nc = (n - 1) / 2;
  const int MV = M / W;                        // time vectors per line
  const int runs = (nc + kRowRun - 1) / kRowRun;  // walks per coarse row
  const size_t items = (size_t)nc * runs * MV;
  const size_t nM = (size_t)n * M;
  Vec<R> z;
#pragma unroll
  for (int k = 0; k < W; ++k) z.v[k] = R(0);
  // the defect at fine point (i, j), time values m .. m+W-1 (as in k_restrict_delta)
  auto r_at = [&](int i, int j, int m) -> Vec<R> {
    if (((i + j) & 1) != red_par) return z;
    const size_t pM = ((size_t)i + (size_t)j * n) * M;
    const R* w = i > 0 ? delta + pM - M : zero;
    const R* e = i < n - 1 ? delta + pM + M : zero;
    const R* so = j > 0 ? delta + pM - nM : zero;
    const R* no = j < n - 1 ? delta + pM + nM : zero;
    const Vec<R> a = vload(w + m), b = vload(e + m), c = vload(so + m), g = vload(no + m);
    Vec<R> out;
#pragma unroll
    for (int k = 0; k < W; ++k) out.v[k] = mul_rounded(hinv2, (a.v[k] + b.v[k]) + (c.v[k] + g.v[k]));
    return out;
  };
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < items;
       x += (size_t)gridDim.x * blockDim.x) {
    const int mv = (int)(x % MV);
    const size_t rest = x / MV;
    const int run = (int)(rest % runs);
    const int row = (int)(rest / runs);
    const int m = mv * W;
    const int cj = 2 * row + 1;
    const int p0 = run * kRowRun;
    const int p1 = p0 + kRowRun < nc ? p0 + kRowRun : nc;
    // the left column (rows cj-1, cj, cj+1) of the first stencil
    Vec<R> l0 = r_at(2 * p0, cj - 1, m), l1 = r_at(2 * p0, cj, m), l2 = r_at(2 * p0, cj + 1, m);
    for (int p = p0; p < p1; ++p) {
      const int ci = 2 * p + 1;
      const Vec<R> c0 = r_at(ci, cj - 1, m), c1 = r_at(ci, cj, m), c2 = r_at(ci, cj + 1, m);
      const Vec<R> q0 = r_at(ci + 1, cj - 1, m), q1 = r_at(ci + 1, cj, m),
                   q2 = r_at(ci + 1, cj + 1, m);
      Vec<R> out;
#pragma unroll
      for (int k = 0; k < W; ++k) out.v[k] = l0.v[k] + R(2) * c0.v[k] + q0.v[k];
#pragma unroll
      for (int k = 0; k < W; ++k) out.v[k] = out.v[k] + R(2) * (l1.v[k] + R(2) * c1.v[k] + q1.v[k]);
#pragma unroll
      for (int k = 0; k < W; ++k)
        out.v[k] = R(0.0625) * (out.v[k] + (l2.v[k] + R(2) * c2.v[k] + q2.v[k]));
      const size_t P = (size_t)row * nc + p;
      vstore(fc + P * M + m, out);
      vstore(uc + P * M + m, z);
      l0 = q0;
      l1 = q1;
      l2 = q2;
    }
  }
}

// 1-D interpolation taps of fine index i from the coarse grid (nc points):
// fine 2J+1 takes coarse J (one tap, weight 1); fine 2J takes the mean of
// coarse J-1 and J (two taps, weight 1/2), or half of the one inside the grid
// at the ends.  All taps of a point share one weight, so the interpolated
// value is that weight times a plain sum of one, two or four coarse lines.
struct Taps {
  int i0, i1, count;
  bool half;
  __device__ __forceinline__ Taps(int i, int nc) {
    if (i & 1) {
      i0 = i1 = (i - 1) >> 1;
      count = 1;
      half = false;
    } else {
      const int J = i >> 1;
      half = true;
      if (J - 1 >= 0 && J < nc) {
        i0 = J - 1;
        i1 = J;
        count = 2;
      } else {
        i0 = i1 = J - 1 >= 0 ? J - 1 : J;
        count = 1;
      }
    }
  }
};

template <class R>
__global__ void __launch_bounds__(kLineBlock)
    k_prolong(R* __restrict__ u, const R* __restrict__ uc, int d, int n, int M, int log_tpl,
              int npts, size_t fstride, size_t cstride) {
  constexpr int W = Vec<R>::W;
  const LineMap<R> lm(log_tpl);
  u += blockIdx.y * fstride;
  uc += blockIdx.y * cstride;
  if (lm.line >= npts) return;
  const int nc = (n - 1) / 2;
  const int p = lm.line;
  R* up = u + (size_t)p * M;
  const Taps tx(d == 1 ? p : p % n, nc);
  const Taps ty(d == 1 ? 1 : p / n, nc);  // 1-D: a single tap of weight 1 in y
  const size_t row0 = d == 1 ? 0 : (size_t)ty.i0 * nc, row1 = d == 1 ? 0 : (size_t)ty.i1 * nc;
  const R* a = uc + ((size_t)tx.i0 + row0) * M;
  const R* b = uc + ((size_t)tx.i1 + row0) * M;
  const R* c = uc + ((size_t)tx.i0 + row1) * M;
  const R* e = uc + ((size_t)tx.i1 + row1) * M;
  const bool unit = !tx.half && !ty.half;
  const R w = R((tx.half ? 0.5 : 1.0) * (ty.half ? 0.5 : 1.0));
  const int taps = tx.count * ty.count;  // 1, 2 (in x or in y) or 4
  // the second tap of a two-tap point: the other coarse line in x, or in y
  const R* second = ty.count == 2 ? c : b;
  for (int m = lm.m0; m < M; m += lm.step) {
    Vec<R> sum = vload(a + m);
    if (taps == 4) {
      const Vec<R> vb = vload(b + m), vc = vload(c + m), ve = vload(e + m);
#pragma unroll
      for (int k = 0; k < W; ++k) sum.v[k] = (sum.v[k] + vb.v[k]) + (vc.v[k] + ve.v[k]);
    } else if (taps == 2) {
      const Vec<R> vs = vload(second + m);
#pragma unroll
      for (int k = 0; k < W; ++k) sum.v[k] = sum.v[k] + vs.v[k];
    }
    Vec<R> cur = vload_rw(up + m);
#pragma unroll
    for (int k = 0; k < W; ++k) cur.v[k] = unit ? cur.v[k] + sum.v[k] : cur.v[k] + w * sum.v[k];
    vstore(up + m, cur);
  }
}

// The 2-D k_prolong with each thread walking kProlongRun fine points of one fine
// row for one vector of time values: a coarse column serves the three fine
// columns around it, so each coarse value (one or two coarse rows) is loaded
// once per walk and kept while the walk needs it, instead of once per fine
// point that interpolates from it.  Every fine value takes the same taps in the
// same order as in k_prolong: the same bits.
constexpr int kProlongRun = 16;

template <class R>
__global__ void __launch_bounds__(kLineBlock)
    k_prolong_rows(R* __restrict__ u, const R* __restrict__ uc, int n, int M, size_t fstride,
                   size_t cstride) {
  constexpr int W = Vec<R>::W;
  u += blockIdx.y * fstride;
  uc += blockIdx.y * cstride;
  const int nc = (n - 1) / 2;
  const int MV = M / W;
  const int runs = (n + kProlongRun - 1) / kProlongRun;
  const size_t items = (size_t)n * runs * MV;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < items;
       x += (size_t)gridDim.x * blockDim.x) {
    const int mv = (int)(x % MV);
    const size_t rest = x / MV;
    const int run = (int)(rest % runs);
    const int j = (int)(rest / runs);
    const int m = mv * W;
    const Taps ty(j, nc);
    const R* row0 = uc + (size_t)ty.i0 * nc * M + m;
    const R* row1 = uc + (size_t)ty.i1 * nc * M + m;
    // the last two coarse columns loaded (index, value in coarse rows i0 and i1)
    int ca = -1, cb = -1;
    Vec<R> a0, a1, b0, b1;
    auto column = [&](int c, Vec<R>& v0, Vec<R>& v1) {
      if (c == cb) {
        v0 = b0;
        v1 = b1;
        return;
      }
      if (c == ca) {
        v0 = a0;
        v1 = a1;
        return;
      }
      ca = cb;
      a0 = b0;
      a1 = b1;
      cb = c;
      b0 = vload(row0 + (size_t)c * M);
      if (ty.count == 2) b1 = vload(row1 + (size_t)c * M);
      v0 = b0;
      v1 = b1;
    };
    const int i_end = (run + 1) * kProlongRun < n ? (run + 1) * kProlongRun : n;
    for (int i = run * kProlongRun; i < i_end; ++i) {
      const Taps tx(i, nc);
      Vec<R> l0, l1, r0, r1;
      column(tx.i0, l0, l1);  // a, c
      column(tx.i1, r0, r1);  // b, e
      const int taps = tx.count * ty.count;
      Vec<R> sum = l0;
      if (taps == 4) {
#pragma unroll
        for (int k = 0; k < W; ++k) sum.v[k] = (sum.v[k] + r0.v[k]) + (l1.v[k] + r1.v[k]);
      } else if (taps == 2) {
        const Vec<R>& second = ty.count == 2 ? l1 : r0;
#pragma unroll
        for (int k = 0; k < W; ++k) sum.v[k] = sum.v[k] + second.v[k];
      }
      const bool unit = !tx.half && !ty.half;
      const R w = R((tx.half ? 0.5 : 1.0) * (ty.half ? 0.5 : 1.0));
      R* up = u + ((size_t)i + (size_t)j * n) * M + m;
      Vec<R> cur = vload_rw(up);
#pragma unroll
      for (int k = 0; k < W; ++k) cur.v[k] = unit ? cur.v[k] + sum.v[k] : cur.v[k] + w * sum.v[k];
      vstore(up, cur);
    }
  }
}

// double <-> double-float conversions and the double-float update
// dst = src as double-float pairs (RN32(x), RN32(x - RN32(x))), without FP64
// arithmetic for the values a solve holds (dd_split_rn).
__global__ void k_split(dd* __restrict__ dst, const double* __restrict__ src, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = dd_split_rn(src[i]);
}

__global__ void k_join(double* __restrict__ dst, const dd* __restrict__ src, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i].hi + (double)src[i].lo;
}

__global__ void k_round_dd(float* __restrict__ dst, const dd* __restrict__ src, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = float(src[i]);
}

__global__ void k_split_cx(Cx<dd>* __restrict__ dst, const Cx<double>* __restrict__ src,
                           size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const double x = src[i].x, y = src[i].y;
    const float xh = (float)x, yh = (float)y;
    dst[i] = Cx<dd>{dd(xh, (float)(x - (double)xh)), dd(yh, (float)(y - (double)yh))};
  }
}

__global__ void k_refine_dd(dd* __restrict__ u, const float* __restrict__ e, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    u[i] = dd_add_float(u[i], e[i]);
}

__global__ void k_refine_dd2(dd* __restrict__ u, const dd* __restrict__ e, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    u[i] = dd_add_accurate(u[i], e[i]);
}

__global__ void k_refine(double* __restrict__ u, const float* __restrict__ e, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    u[i] += (double)e[i];
}

__global__ void k_round(float* __restrict__ dst, const double* __restrict__ src, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// Per instance (blockIdx.y), in one pass over x: |x|_inf folded into
// norm_bits[instance], and where given out = (float) x and out_dd = x as
// double-float pairs (k_split's).  The defect of u = 0 is f itself, so this
// is the initial defect of a solve from zero, rounded for the first inner
// cycles and split for the outer defect the first steps carry.  No FP64
// arithmetic: the conversions by dd_split_rn, the norm as the largest
// magnitude bit pattern (non-negative doubles order like their bits, a NaN
// above infinity).
__global__ void __launch_bounds__(128)
    k_absmax_round(const double* __restrict__ x, float* __restrict__ out, dd* __restrict__ out_dd,
                   size_t per, unsigned long long* __restrict__ norm_bits) {
  x += blockIdx.y * per;
  if (out != nullptr) out += blockIdx.y * per;
  if (out_dd != nullptr) out_dd += blockIdx.y * per;
  unsigned long long amax = 0;
  for (size_t i = blockIdx.x * (size_t)128 + threadIdx.x; i < per; i += (size_t)gridDim.x * 128) {
    const double v = x[i];
    if (out != nullptr || out_dd != nullptr) {
      const dd p = dd_split_rn(v);
      if (out != nullptr) out[i] = p.hi;
      if (out_dd != nullptr) out_dd[i] = p;
    }
    const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    amax = a > amax ? a : amax;
  }
  block_absmax(__longlong_as_double((long long)amax), norm_bits + blockIdx.y);
}

// Initial value g of every instance (blockIdx.y): u = g along time (initial
// iterate u^0(t) = g) and f += c d_m g (the u_0 term of the L1 scheme).
__global__ void k_initial(double* __restrict__ u, double* __restrict__ f,
                          const double* __restrict__ g, const double* __restrict__ dk,
                          const double* __restrict__ c, int N, int M) {
  const size_t stride = (size_t)N * M;
  u += blockIdx.y * stride;
  f += blockIdx.y * stride;
  g += (size_t)blockIdx.y * N;
  dk += (size_t)blockIdx.y * (M + 1);
  const double cb = c[blockIdx.y];
  for (int p = blockIdx.x; p < N; p += gridDim.x) {
    const double gp = g[p];
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
      u[(size_t)p * M + m] = gp;
      f[(size_t)p * M + m] += cb * dk[m + 1] * gp;
    }
  }
}

// ---------------------------------------------------------------------------------
// setup, FP64: L1 coefficients, inverse columns, twiddles, spectra
// ---------------------------------------------------------------------------------

// r_1 = c; r_2 = c (2^beta - 2); for i >= 3 the second difference
//   i^b - 2(i-1)^b + (i-2)^b = (i-1)^b [(1+y)^b + (1-y)^b - 2],  y = 1/(i-1),
// is summed as its binomial series 2 sum_{k>=1} C(b, 2k) y^{2k}, whose terms all
// have the sign of C(b, 2) < 0, so no cancellation occurs.  d_m (for the
// initial-value term) is accumulated by the telescoping sum d_m = sum r_i / c.
__global__ void k_coefficients(double* __restrict__ r, int M, const double* __restrict__ alphas,
                               const double* __restrict__ cs) {
  r += (size_t)blockIdx.y * M;
  const double b = 1.0 - alphas[blockIdx.y];
  const double c = cs[blockIdx.y];
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < M; i0 += gridDim.x * blockDim.x) {
    const int i = i0 + 1;
    double val;
    if (i == 1) {
      val = 1.0;
    } else if (i == 2) {
      val = exp2(b) - 2.0;
    } else {
      const double y = 1.0 / (double)(i - 1);
      const double y2 = y * y;
      double term = 0.5 * b * (b - 1.0) * y2;  // C(b,2) y^2
      double sum = term;
      for (int k = 1; k < 200; ++k) {
        // C(b,2k+2)/C(b,2k) = (b-2k)(b-2k-1) / ((2k+1)(2k+2))
        term *= (b - 2.0 * k) * (b - 2.0 * k - 1.0) / ((2.0 * k + 1.0) * (2.0 * k + 2.0)) * y2;
        sum += term;
        if (fabs(term) <= 1e-18 * fabs(sum)) break;
      }
      val = 2.0 * sum * pow((double)(i - 1), b);
    }
    r[i0] = c * val;
  }
}

// d_0 = 0, d_m = d_{m-1} + r_m / c (sequential; setup only).
__global__ void k_weights_from_column(double* __restrict__ dk, const double* __restrict__ r, int M,
                                      const double* __restrict__ cs, int batch) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst < batch) {
    dk += (size_t)inst * (M + 1);
    r += (size_t)inst * M;
    const double c = cs[inst];
    double acc = 0.0;
    dk[0] = 0.0;
    for (int m = 1; m <= M; ++m) {
      acc += r[m - 1] / c;
      dk[m] = acc;
    }
  }
}

// In-place radix-2 FFT of length N = 2^logN in global memory by one block
// (bit reversal, then decimation-in-time passes); twiddles from sincospi.
__device__ void block_fft_radix2(Cx<double>* x, int N, int logN, bool inv) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int rr = (int)(__brev((unsigned)i) >> (32 - logN));
    if (rr > i) {
      const Cx<double> tmp = x[i];
      x[i] = x[rr];
      x[rr] = tmp;
    }
  }
  __syncthreads();
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1;
    for (int bidx = threadIdx.x; bidx < N / 2; bidx += blockDim.x) {
      const int grp = bidx / half, jj = bidx - grp * half;
      const int i0 = grp * len + jj, i1 = i0 + half;
      double s, co;
      sincospi((inv ? 2.0 : -2.0) * (double)jj / (double)len, &s, &co);
      const Cx<double> w{co, s};
      const Cx<double> a = x[i0], bb = cmul(x[i1], w);
      x[i0] = cadd(a, bb);
      x[i1] = csub(a, bb);
    }
    __syncthreads();
  }
}

// One block per level.  First column k of (T_M + sigma I)^{-1} by divide and
// conquer (Sec. 5, smoothing procedure): with a = (r_1 + sigma, r_2, ...),
// T_{2n}^{-1} = [T_n^{-1} 0; -T_n^{-1} P_n T_n^{-1}  T_n^{-1}], so the new half
// of the column is k[n..2n) = -(k_n * c)[0..n) with c = (a * k_n)[n..2n), both
// causal products done as cyclic convolutions of length 2n.  The first
// 2^p0 = 16 entries come from forward substitution.
__global__ void k_inverse_columns(double* __restrict__ kcol, const double* __restrict__ r,
                                  const double* __restrict__ sigma, int M,
                                  Cx<double>* __restrict__ work) {
  // block (l, b): level l of instance b; columns and work are instance-major
  const int l = blockIdx.x;
  const size_t slot = (size_t)blockIdx.y * gridDim.x + l;
  r += (size_t)blockIdx.y * M;
  double* k = kcol + slot * M;
  Cx<double>* X = work + slot * 3 * M;
  Cx<double>* Y = X + M;
  Cx<double>* Z = Y + M;
  const double a0 = r[0] + sigma[l];
  const int n0 = M < 16 ? M : 16;
  if (threadIdx.x == 0) {
    k[0] = 1.0 / a0;
    for (int m = 1; m < n0; ++m) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += r[m - j] * k[j];
      k[m] = -s / a0;
    }
  }
  __syncthreads();
  for (int nn = n0; nn < M; nn *= 2) {
    const int N2 = 2 * nn;
    int logN = 0;
    while ((1 << logN) < N2) ++logN;
    const double inv = 1.0 / (double)N2;
    for (int i = threadIdx.x; i < N2; i += blockDim.x) {
      X[i] = Cx<double>{i == 0 ? a0 : r[i], 0.0};
      Y[i] = Cx<double>{i < nn ? k[i] : 0.0, 0.0};
    }
    __syncthreads();
    block_fft_radix2(X, N2, logN, false);
    block_fft_radix2(Y, N2, logN, false);
    for (int i = threadIdx.x; i < N2; i += blockDim.x) Z[i] = cmul(X[i], Y[i]);
    __syncthreads();
    block_fft_radix2(Z, N2, logN, true);
    // c = (a * k_n)[n..2n): entries n.. of the cyclic product (no wrap for those)
    for (int i = threadIdx.x; i < N2; i += blockDim.x)
      X[i] = Cx<double>{i < nn ? Z[nn + i].x * inv : 0.0, 0.0};
    __syncthreads();
    block_fft_radix2(X, N2, logN, false);
    for (int i = threadIdx.x; i < N2; i += blockDim.x) Z[i] = cmul(X[i], Y[i]);
    __syncthreads();
    block_fft_radix2(Z, N2, logN, true);
    for (int i = threadIdx.x; i < nn; i += blockDim.x) k[nn + i] = -Z[i].x * inv;
    __syncthreads();
  }
}

__global__ void k_twiddles(Cx<double>* __restrict__ tw, int L) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)m / (double)L, &s, &c);
    tw[m] = Cx<double>{c, s};
  }
}

// Spectrum of one real line per thread group, in the engine's spectral order,
// scaled by 1/L.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_spectra(Cx<double>* __restrict__ spec, const double* __restrict__ lines, int count, int M,
              int logL, const Cx<double>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  Cx<double>* smem = reinterpret_cast<Cx<double>*>(smem_raw);
  const FftShape sh(logL);
  const int TL = sh.L8;
  const int g = threadIdx.x / TL;
  const int t = threadIdx.x - g * TL;
  const int groups = BLOCK / TL;
  const int line = blockIdx.x * groups + g;
  const bool valid = line < count;
  Cx<double>* buf = smem + g * Pad<double>::len(sh.L);
  const double* x = lines + (size_t)(valid ? line : 0) * M;
  auto load = [&](int m) -> Cx<double> { return Cx<double>{valid ? x[m] : 0.0, 0.0}; };
  Cx<double> v[1][8];
  const GroupSync sync(TL, BLOCK, g);
  fft_forward<1>(buf, t, sh, tw, load, v, sync);
  const double inv = 1.0 / (double)sh.L;
  if (valid) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      spec[(size_t)line * sh.L + 8 * t + q] = Cx<double>{v[0][q].x * inv, v[0][q].y * inv};
  }
}

__global__ void k_round_cx(Cx<float>* __restrict__ dst, const Cx<double>* __restrict__ src,
                           size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = Cx<float>{(float)src[i].x, (float)src[i].y};
}

// ---------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------



// Launch geometry of the line-wise kernels: log2 of the threads per line and
// the number of 256-thread blocks for `lines` lines of M values of R.
template <class R>
inline void line_grid(int M, int lines, int* log_tpl, unsigned* blocks) {
  const int per = M / Vec<R>::W;
  // 64 threads per line up to 1024 vectors (measured best at M = 256 .. 4096);
  // the partitioned long lines take 256 (1-D 4095 x 65536 double-float solve:
  // 564 -> 527 ms; at M = 1024 the wider groups lost 2-3 %)
  const int tpl = per <= 1024 ? (per < 64 ? per : 64) : 256;
  *log_tpl = ilog2(tpl);
  const int lpb = kLineBlock / tpl;
  *blocks = (unsigned)((lines + lpb - 1) / lpb);
}

template <class R>
cudaError_t launch_defect_from_delta(const R* delta, R* r, const R* zero, const LevelShape& ls,
                                     int red_par, R hinv2, unsigned long long* norm_bits,
                                     cudaStream_t s) {
  const int npts = ls.d == 1 ? ls.n : ls.n * ls.n;
  if (ls.batch == 0) return cudaSuccess;
  int log_tpl;
  unsigned blocks;
  line_grid<R>(ls.M, npts, &log_tpl, &blocks);
  k_defect_from_delta<R><<<dim3(blocks, ls.batch), kLineBlock, 0, s>>>(
      delta, r, zero, ls.d, ls.n, ls.M, log_tpl, npts, red_par, hinv2, norm_bits,
      ls.field_stride());
  return counted(cudaGetLastError());
}

template <class R>
cudaError_t launch_restrict(const R* r, R* fc, R* uc, const LevelShape& ls, cudaStream_t s) {
  const int nc = (ls.n - 1) / 2;
  const int ncpts = ls.d == 1 ? nc : nc * nc;
  if (ncpts == 0 || ls.batch == 0) return cudaSuccess;
  int log_tpl;
  unsigned blocks;
  line_grid<R>(ls.M, ncpts, &log_tpl, &blocks);
  k_restrict<R><<<dim3(blocks, ls.batch), kLineBlock, 0, s>>>(r, fc, uc, ls.d, ls.n, ls.M, log_tpl, ncpts,
                                                       ls.field_stride(), (size_t)ncpts * ls.M);
  return counted(cudaGetLastError());
}

template <class R>
cudaError_t launch_restrict_delta(const R* delta, R* fc, R* uc, const R* zero, const LevelShape& ls,
                                  int red_par, R hinv2, cudaStream_t s) {
  const int nc = (ls.n - 1) / 2;
  const int ncpts = ls.d == 1 ? nc : nc * nc;
  if (ncpts == 0 || ls.batch == 0) return cudaSuccess;
  if (ls.d == 2) {
    const size_t items = (size_t)nc * ((nc + kRowRun - 1) / kRowRun) * (ls.M / Vec<R>::W);
    const unsigned blocks = elementwise_grid(items);
    k_restrict_delta_rows<R><<<dim3(blocks, ls.batch), kLineBlock, 0, s>>>(
        delta, fc, uc, zero, ls.n, ls.M, red_par, hinv2, ls.field_stride(), (size_t)ncpts * ls.M);
    return counted(cudaGetLastError());
  }
  int log_tpl;
  unsigned blocks;
  line_grid<R>(ls.M, ncpts, &log_tpl, &blocks);
  k_restrict_delta<R><<<dim3(blocks, ls.batch), kLineBlock, 0, s>>>(
      delta, fc, uc, zero, ls.d, ls.n, ls.M, log_tpl, ncpts, red_par, hinv2, ls.field_stride(),
      (size_t)ncpts * ls.M);
  return counted(cudaGetLastError());
}

template <class R>
cudaError_t launch_prolong(R* u, const R* uc, const LevelShape& ls, cudaStream_t s) {
  const int npts = ls.d == 1 ? ls.n : ls.n * ls.n;
  const int nc = (ls.n - 1) / 2;
  const size_t cstride = (size_t)(ls.d == 1 ? nc : nc * nc) * ls.M;
  if (ls.batch == 0) return cudaSuccess;
  // short lines (at most 1 KB: one time vector per thread of the per-line kernel,
  // whose index work per point then dominates) walk rows; longer ones keep the
  // per-line kernel, near the HBM roof there (2-D 511 x 511, M = 4096: 21.9 ms per
  // solve against 29.0 for the row walk; 4096 x 63 x 63, M = 256: 127 against 108)
  if (ls.d == 2 && nc > 0 && (size_t)ls.M * sizeof(R) <= 1024) {
    const size_t items =
        (size_t)ls.n * ((ls.n + kProlongRun - 1) / kProlongRun) * (ls.M / Vec<R>::W);
    k_prolong_rows<R><<<dim3(elementwise_grid(items), ls.batch), kLineBlock, 0, s>>>(
        u, uc, ls.n, ls.M, ls.field_stride(), cstride);
    return counted(cudaGetLastError());
  }
  int log_tpl;
  unsigned blocks;
  line_grid<R>(ls.M, npts, &log_tpl, &blocks);
  k_prolong<R><<<dim3(blocks, ls.batch), kLineBlock, 0, s>>>(u, uc, ls.d, ls.n, ls.M, log_tpl, npts,
                                                      ls.field_stride(), cstride);
  return counted(cudaGetLastError());
}

cudaError_t launch_refine_dd2(dd* u, const dd* e, size_t count, cudaStream_t s) {
  k_refine_dd2<<<elementwise_grid(count), 256, 0, s>>>(u, e, count);
  return counted(cudaGetLastError());
}

cudaError_t launch_refine(double* u, const float* e, size_t count, cudaStream_t s) {
  k_refine<<<elementwise_grid(count), 256, 0, s>>>(u, e, count);
  return counted(cudaGetLastError());
}

cudaError_t launch_split(dd* dst, const double* src, size_t count, cudaStream_t s) {
  k_split<<<elementwise_grid(count), 256, 0, s>>>(dst, src, count);
  return counted(cudaGetLastError());
}

cudaError_t launch_join(double* dst, const dd* src, size_t count, cudaStream_t s) {
  k_join<<<elementwise_grid(count), 256, 0, s>>>(dst, src, count);
  return counted(cudaGetLastError());
}

cudaError_t launch_round_dd(const dd* x, float* out, size_t count, cudaStream_t s) {
  k_round_dd<<<elementwise_grid(count), 256, 0, s>>>(out, x, count);
  return counted(cudaGetLastError());
}

cudaError_t launch_split_cx(Cx<dd>* dst, const Cx<double>* src, size_t count, cudaStream_t s) {
  k_split_cx<<<elementwise_grid(count), 256, 0, s>>>(dst, src, count);
  return counted(cudaGetLastError());
}

cudaError_t launch_refine_dd(dd* u, const float* e, size_t count, cudaStream_t s) {
  k_refine_dd<<<elementwise_grid(count), 256, 0, s>>>(u, e, count);
  return counted(cudaGetLastError());
}

cudaError_t launch_round(float* dst, const double* src, size_t count, cudaStream_t s) {
  k_round<<<elementwise_grid(count), 256, 0, s>>>(dst, src, count);
  return counted(cudaGetLastError());
}

namespace {

__global__ void k_loop_init(LoopState* st, double tol, int max_iter) {
  st->tol = tol;
  st->rel = 0.0;
  st->max_iter = max_iter;
  st->iters = 0;
}

// One warp: the largest relative defect over the instances (NaN wins), then
// the loop's condition.
__global__ void k_loop_decide(const unsigned long long* __restrict__ norm_bits,
                              const double* __restrict__ r0, int batch, LoopState* st,
                              cudaGraphConditionalHandle loop) {
  double worst = 0.0;
  for (int b = threadIdx.x; b < batch; b += 32) {
    const double nv = __longlong_as_double((long long)norm_bits[b]);
    const double rel = r0[b] > 0.0 ? nv / r0[b] : (nv == 0.0 ? 0.0 : nv);
    worst = absmax_nan(isinf(rel) ? (double)NAN : rel, worst);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) worst = absmax_nan(__shfl_xor_sync(0xffffffffu, worst, o), worst);
  if (threadIdx.x == 0) {
    st->iters += 1;
    st->rel = worst;
    const bool more = worst == worst && worst > st->tol && st->iters < st->max_iter;
    cudaGraphSetConditional(loop, more ? 1u : 0u);
  }
}

}  // namespace

cudaError_t launch_loop_init(LoopState* st, double tol, int max_iter, cudaStream_t s) {
  k_loop_init<<<1, 1, 0, s>>>(st, tol, max_iter);
  return counted(cudaGetLastError());
}

cudaError_t launch_loop_decide(const unsigned long long* norm_bits, const double* r0, int batch,
                               LoopState* st, cudaGraphConditionalHandle loop, cudaStream_t s) {
  k_loop_decide<<<1, 32, 0, s>>>(norm_bits, r0, batch, st, loop);
  return counted(cudaGetLastError());
}

cudaError_t launch_absmax_round(const double* x, float* out, dd* out_dd, size_t per, int batch,
                                unsigned long long* norm_bits, cudaStream_t s) {
  if (per == 0 || batch == 0) return cudaSuccess;
  size_t bx = (per + 128 * 16 - 1) / (128 * 16);
  if (bx > 2432) bx = 2432;
  k_absmax_round<<<dim3((unsigned)bx, (unsigned)batch), 128, 0, s>>>(x, out, out_dd, per,
                                                                     norm_bits);
  return counted(cudaGetLastError());
}

cudaError_t launch_initial(double* u, double* f, const double* g, const double* dk, const double* c,
                           int N, int M, int batch, cudaStream_t s) {
  const unsigned bx = (unsigned)(N < 1024 ? N : 1024);
  k_initial<<<dim3(bx, batch), 256, 0, s>>>(u, f, g, dk, c, N, M);
  return counted(cudaGetLastError());
}

cudaError_t launch_coefficients(double* r, double* dk, int M, const double* alphas,
                                const double* cs, int batch, cudaStream_t s) {
  k_coefficients<<<dim3((M + 255) / 256, batch), 256, 0, s>>>(r, M, alphas, cs);
  cudaError_t e = counted(cudaGetLastError());
  if (e != cudaSuccess) return e;
  k_weights_from_column<<<(batch + 63) / 64, 64, 0, s>>>(dk, r, M, cs, batch);
  return counted(cudaGetLastError());
}

cudaError_t launch_inverse_columns(double* kcol, const double* r, const double* sigma, int nlev,
                                   int M, int batch, Cx<double>* work, cudaStream_t s) {
  k_inverse_columns<<<dim3(nlev, batch), 512, 0, s>>>(kcol, r, sigma, M, work);
  return counted(cudaGetLastError());
}

cudaError_t launch_twiddles(Cx<double>* tw, int L, cudaStream_t s) {
  k_twiddles<<<(L + 255) / 256, 256, 0, s>>>(tw, L);
  return counted(cudaGetLastError());
}

cudaError_t launch_spectra(Cx<double>* spec, const double* lines, int count, int M,
                           const Cx<double>* tw, cudaStream_t s) {
  if (M > kShortMaxM) return launch_spectra_long(spec, lines, count, M, tw, s);
  const int L = 2 * M, logL = ilog2(L);
  const int block = block_threads(L);
  const int groups = block / (L / 8);
  const size_t smem = (size_t)groups * Pad<double>::len(L) * sizeof(Cx<double>);
  const unsigned grid = (unsigned)((count + groups - 1) / groups);
  cudaError_t e;
  switch (block) {
    case 256:
      e = prepare_smem(k_spectra<256>, smem);
      if (e != cudaSuccess) return e;
      k_spectra<256><<<grid, 256, smem, s>>>(spec, lines, count, M, logL, tw);
      break;
    case 512:
      e = prepare_smem(k_spectra<512>, smem);
      if (e != cudaSuccess) return e;
      k_spectra<512><<<grid, 512, smem, s>>>(spec, lines, count, M, logL, tw);
      break;
    default:
      e = prepare_smem(k_spectra<1024>, smem);
      if (e != cudaSuccess) return e;
      k_spectra<1024><<<grid, 1024, smem, s>>>(spec, lines, count, M, logL, tw);
      break;
  }
  return counted(cudaGetLastError());
}

cudaError_t launch_round_cx(Cx<float>* dst, const Cx<double>* src, size_t count, cudaStream_t s) {
  k_round_cx<<<elementwise_grid(count), 256, 0, s>>>(dst, src, count);
  return counted(cudaGetLastError());
}

// explicit instantiations
#define MGWR_INST_R(R)                                                                         \
  template cudaError_t launch_defect_from_delta<R>(const R*, R*, const R*, const LevelShape&,  \
                                                   int, R, unsigned long long*, cudaStream_t); \
  template cudaError_t launch_restrict<R>(const R*, R*, R*, const LevelShape&, cudaStream_t);  \
  template cudaError_t launch_prolong<R>(R*, const R*, const LevelShape&, cudaStream_t);     \
  template cudaError_t launch_restrict_delta<R>(const R*, R*, R*, const R*, const LevelShape&, \
                                                int, R, cudaStream_t);
MGWR_INST_R(double)
MGWR_INST_R(float)
MGWR_INST_R(dd)
#undef MGWR_INST_R


}  // namespace mgwr

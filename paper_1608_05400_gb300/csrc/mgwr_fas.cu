// Waveform relaxation FAS for the 1-D nonlinear problem of Sec. 7
// (Eq. anomalous_diffusion): D_t^alpha u = d/dx(D(u) du/dx) + c du/dx + f on
// (0,1) x (0,T], zero boundary and initial values, discretised with the L1
// scheme (Eq. L1_scheme2), the conservative flux difference of
// Eq. spatial_discretization (a_{n+-1/2} the mean of D at the two nodes) and
// upwind convection (forward difference for c >= 0, backward for c < 0).
//
// Kernels (FP64):
//   k_fas_line   the nonlinear red-black waveform smoother: one warp per time line
//                of one colour; the line is marched in time, each step a scalar
//                Newton solve (the step's equation is strictly increasing in the
//                unknown), the history sum of the L1 matrix shared by the warp's
//                lanes from a shared-memory copy of the line;
//   k_fas_apply  out = base + sign * N_h(u), N_h the discrete operator (time term
//                T_M u by direct sums from shared memory, flux and upwind
//                differences), with its max-norm: the defect f - N_h(u) and the
//                FAS coarse right-hand side N_2h(R u) + R r;
//   k_fas_restrict2, k_fas_correct   full weighting of the iterate and the
//                defect, and u += P (u_c - R u).
// The history sums are direct (O(M^2) per line, as the scheme is written):
// the paper's nonlinear tables use M <= 256, and M is limited to 1024 here, so
// both kernels stay within the default 48 KB of dynamic shared memory.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mgwr.h"
#include "mgwr_common.cuh"

namespace mgwr {
namespace {

constexpr int kFasMaxM = 1024;
constexpr int kLineWarps = 4;     // time lines per block of k_fas_line
constexpr int kApplyThreads = 256;
constexpr int kNewtonMax = 100;   // Newton iterations per time step before giving up

__device__ __forceinline__ double coef_D(int kind, double v) {
  return kind == MGWR_FAS_D_POROUS ? 1.0 + v * v : 1.0;
}


// Lines of one colour: points i = 2k + parity (k < count), or every point when
// all_points (the one-point grid).  Dynamic shared memory: (1 + kLineWarps) * M
// doubles.  status bit 0 is set when Newton's method did not settle in a step.
__global__ void __launch_bounds__(32 * kLineWarps)
    k_fas_line(double* __restrict__ u, const double* __restrict__ f,
               const double* __restrict__ r, int n, int M, double h, double c, int coef,
               int parity, int all_points, int* __restrict__ status) {
  extern __shared__ double sm[];
  double* rs = sm;  // r_1..r_M of T_M
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* line = sm + M + (size_t)warp * M;
  for (int j = threadIdx.x; j < M; j += blockDim.x) rs[j] = r[j];
  const int count = all_points ? n : (parity ? n / 2 : (n + 1) / 2);
  const int k = blockIdx.x * kLineWarps + warp;
  const bool active = k < count;
  const int i = all_points ? k : 2 * k + parity;
  if (active)
    for (int j = lane; j < M; j += 32) line[j] = u[(size_t)i * M + j];
  __syncthreads();
  if (!active) return;
  const double* up = (i + 1 < n) ? u + (size_t)(i + 1) * M : nullptr;
  const double* um = (i > 0) ? u + (size_t)(i - 1) * M : nullptr;
  const double* fi = f + (size_t)i * M;
  const double r1 = rs[0], h2 = h * h, half_h2 = 0.5 / h2, c_h = c / h, ac_h = fabs(c_h);
  const double kappa = coef == MGWR_FAS_D_POROUS ? 1.0 : 0.0;  // D(v) = 1 + kappa v^2
  // per-line constants (no FP64 division inside the time loop)
  const double a3 = kappa / h2, a3x3 = 3.0 * a3;
  bool ok = true;
  for (int m = 0; m < M; ++m) {
    // sum_{j<m} (T_M)_{mj} u_j, (T_M)_{mj} = r_{m-j+1}
    double part = 0.0;
    for (int j = lane; j < m; j += 32) part = fma(rs[m - j], line[j], part);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const double hist = __shfl_sync(0xffffffffu, part, 0);
    const double P = up ? up[m] : 0.0, Q = um ? um[m] : 0.0;
    const double Dp = 1.0 + kappa * P * P, Dm = 1.0 + kappa * Q * Q, fm = fi[m];
    // The step's equation g(v) = r_1 v + hist - diffusion(v) - convection(v) - f = 0
    // as the cubic a0 + a1 v + a2 v^2 + a3 v^3: with D(v) = 1 + kappa v^2,
    //   2 h^2 diffusion = (Dp+1) P + (Dm+1) Q - (Dp+Dm+2) v + kappa (P+Q) v^2 - 2 kappa v^3.
    const double flux0 = ((Dp + 1.0) * P + (Dm + 1.0) * Q) * half_h2;
    const double conv0 = c >= 0.0 ? c_h * P : -c_h * Q;
    const double a2 = -kappa * (P + Q) * half_h2, a2x2 = 2.0 * a2;
    const double a1 = r1 + (Dp + Dm + 2.0) * half_h2 + ac_h;
    const double a0 = hist - fm - flux0 - conv0;
    // the size of the equation's terms, in units of v (a tolerance scale only, so the
    // FP32 reciprocal of a1 is accurate enough)
    const double s0 =
        (fabs(hist) + fabs(fm) + fabs(flux0) + fabs(conv0)) * (double)(1.0f / (float)a1);
    // Newton's method in FP32 to about 1e-6, then two FP64 Newton steps with the
    // FP32 reciprocal of g' (each contracts the error by about 1e-7)
    const float b0 = (float)a0, b1 = (float)a1, b2 = (float)a2, b3 = (float)a3;
    const float s0f = (float)s0;
    float vf = (float)line[m];
    for (int it = 0; it < 30; ++it) {
      const float gf = fmaf(fmaf(fmaf(b3, vf, b2), vf, b1), vf, b0);
      const float dgf = fmaf(fmaf(3.0f * b3, vf, 2.0f * b2), vf, b1);
      const float sf = gf / dgf;
      vf -= sf;
      if (fabsf(sf) <= 1e-6f * (fabsf(vf) + s0f)) break;
    }
    double v = isfinite(vf) ? (double)vf : line[m];
    double step = 0.0;
    for (int k = 0; k < 2; ++k) {
      const double g = fma(fma(fma(a3, v, a2), v, a1), v, a0);
      const double dg = fma(fma(a3x3, v, a2x2), v, a1);
      const float dgs = fabsf((float)dg);
      if (!(dgs >= FLT_MIN && dgs <= FLT_MAX)) {
        // g' outside FP32's normal range: its FP32 reciprocal would be 0 or inf,
        // so leave the step to the plain FP64 Newton solve below
        step = NAN;
        break;
      }
      step = g * (double)(1.0f / (float)dg);
      v -= step;
    }
    if (!(fabs(step) <= 1e-12 * (fabs(v) + s0) + 1e-300)) {
      // not settled (extreme or non-finite data): plain FP64 Newton from the start
      v = line[m];
      bool done = false, settled = false;
      for (int it = 0; it < kNewtonMax; ++it) {
        const double g = fma(fma(fma(a3, v, a2), v, a1), v, a0);
        const double dg = fma(fma(a3x3, v, a2x2), v, a1);
        step = g / dg;
        v -= step;
        if (done) {
          settled = true;
          break;
        }
        done = fabs(step) <= 1e-13 * (fabs(v) + s0) + 1e-300;
      }
      if (!settled) ok = false;
    }
    __syncwarp();
    if (lane == 0) line[m] = v;
    __syncwarp();
  }
  for (int j = lane; j < M; j += 32) u[(size_t)i * M + j] = line[j];
  if (!ok && lane == 0) atomicOr(status, 1);
}

// The same half-sweep as k_fas_line by a whole-line fixed point instead of a
// march in time: with the splitting N(v) = (T_M + sigma I) v - (sigma v - phi(v)),
// phi the point's spatial term (flux difference and upwind convection with its
// neighbours' lines fixed), sigma = 2/h^2 + |c|/h the spatial term's slope at
// D = 1, every iteration is
//     v <- (T_M + sigma I)^{-1} (f + sigma v - phi(v)),
// one causal convolution per line with the inverse column of T_M + sigma I
// (spectrum kspec) on the FFT engine, two lines per thread group.  For D = 1
// it is the linear smoother (one iteration); otherwise it contracts by about
// max |1 - phi'(v) / sigma| and runs until the largest change of the pair is at
// the convolution's rounding level (4e-15 of its largest value), or stops
// falling below 1e-12 of it, at most max_it times (status bit 1 set when
// neither is reached).  One line pair per block of L/8 threads (E = 1).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_fas_fixed(double* __restrict__ u, const double* __restrict__ f,
                const Cx<double>* __restrict__ kspec, const Cx<double>* __restrict__ tw, int n,
                int M, int logL, double hinv, double hinv2, double c, double sigma, int coef,
                int parity, int all_points, int max_it, int* __restrict__ status,
                unsigned long long* __restrict__ iterations) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
  __shared__ int done_flag;
  Cx<double>* buf = reinterpret_cast<Cx<double>*>(smem_raw);
  const FftShape sh(logL);
  const int t = threadIdx.x;
  const GroupSync sync(BLOCK, BLOCK, 0);
  const int count = all_points ? n : (parity ? n / 2 : (n + 1) / 2);
  const int kA = 2 * blockIdx.x, kB = kA + 1;
  const bool hasB = kB < count;
  const int iA = all_points ? kA : 2 * kA + parity;
  const int iB = all_points ? kB : 2 * kB + parity;
  double* uA = u + (size_t)iA * M;
  double* uB = u + (size_t)(hasB ? iB : iA) * M;
  const double* fA = f + (size_t)iA * M;
  const double* fB = f + (size_t)(hasB ? iB : iA) * M;
  // neighbour lines (the other colour, fixed in this half-sweep); none on the one-point grid
  const double* pA = (!all_points && iA + 1 < n) ? u + (size_t)(iA + 1) * M : nullptr;
  const double* qA = (!all_points && iA > 0) ? u + (size_t)(iA - 1) * M : nullptr;
  const double* pB = (!all_points && iB + 1 < n) ? u + (size_t)(iB + 1) * M : nullptr;
  const double* qB = (!all_points && iB > 0) ? u + (size_t)(iB - 1) * M : nullptr;
  // f + sigma v - phi(v) at one point: phi(v) = -(diffusion + convection)
  auto rhs = [&](double fm, double v, double P, double Q) {
    const double D0 = coef_D(coef, v);
    const double a_plus = 0.5 * (coef_D(coef, P) + D0);
    const double a_minus = 0.5 * (coef_D(coef, Q) + D0);
    const double diffusion = (a_plus * (P - v) - a_minus * (v - Q)) * hinv2;
    const double convection = c >= 0.0 ? c * (P - v) * hinv : c * (v - Q) * hinv;
    return fm + sigma * v + (diffusion + convection);
  };
  auto load = [&](int m) -> Cx<double> {
    const double bA = rhs(fA[m], uA[m], pA ? pA[m] : 0.0, qA ? qA[m] : 0.0);
    const double bB = hasB ? rhs(fB[m], uB[m], pB ? pB[m] : 0.0, qB ? qB[m] : 0.0) : 0.0;
    return Cx<double>{bA, bB};
  };
  bool settled = false;
  int it = 0;
  double d_prev = 0.0;  // the last iteration's largest change (thread 0)
  for (; it < max_it; ++it) {
    double dmax = 0.0, vmax = 0.0;
    auto store = [&](int m, Cx<double> y) {
      dmax = fmax(dmax, fabs(y.x - uA[m]));
      vmax = fmax(vmax, fabs(y.x));
      uA[m] = y.x;
      if (hasB) {
        dmax = fmax(dmax, fabs(y.y - uB[m]));
        vmax = fmax(vmax, fabs(y.y));
        uB[m] = y.y;
      }
    };
    Cx<double> v[1][8];
    fft_forward<1>(buf, t, sh, tw, load, v, sync);
#pragma unroll
    for (int q = 0; q < 8; ++q) v[0][q] = cmul(v[0][q], kspec[8 * t + q]);
    fft_inverse<1>(buf, t, sh, tw, v, store, sync);
    // the pair's largest change and value (non-finite values count as not settled)
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if (BLOCK >= 32 && (t & 31) == 0) {
      red[0][t >> 5] = dmax;
      red[1][t >> 5] = vmax;
    }
    __syncthreads();
    if (t == 0) {
      double d = 0.0, w = 0.0;
      for (int k = 0; k < (BLOCK >= 32 ? BLOCK / 32 : 1); ++k) {
        d = fmax(d, BLOCK >= 32 ? red[0][k] : dmax);
        w = fmax(w, BLOCK >= 32 ? red[1][k] : vmax);
      }
      // settled: the change is at the level of the convolution's rounding (the
      // right-hand side holds sigma v, so v carries about log2(L) eps of itself),
      // or it has stopped falling within 1e-12 of the line
      done_flag = (w <= DBL_MAX && (d <= 4e-15 * w || (d <= 1e-12 * w && d >= 0.5 * d_prev))) ? 1 : 0;
      d_prev = d;
    }
    __syncthreads();  // also orders this iteration's stores before the next loads
    if (done_flag) {
      settled = true;
      ++it;
      break;
    }
  }
  if (t == 0) {
    if (!settled) atomicOr(status, 2);
    atomicAdd(iterations, (unsigned long long)it * (hasB ? 2 : 1));  // line iterations
  }
}

// out = base + sign * N_h(u) on every point (one block per line), and the
// max-norm of out into *norm_bits (the bits of a non-negative double; a
// non-finite value counts as +inf).  Dynamic shared memory: 2 * M doubles.
__global__ void __launch_bounds__(kApplyThreads)
    k_fas_apply(const double* __restrict__ u, const double* __restrict__ r,
                const double* __restrict__ base, double* __restrict__ out, int n, int M,
                double h, double c, int coef, double sign,
                unsigned long long* __restrict__ norm_bits) {
  extern __shared__ double sm[];
  __shared__ double wmax[kApplyThreads / 32];
  double* rs = sm;
  double* line = sm + M;
  const int i = blockIdx.x;
  const size_t row = (size_t)i * M;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    rs[j] = r[j];
    line[j] = u[row + j];
  }
  __syncthreads();
  const double h2 = h * h;
  double local = 0.0;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    double t = 0.0;
    for (int j = 0; j <= m; ++j) t = fma(rs[m - j], line[j], t);
    const double w0 = line[m];
    const double wp = i + 1 < n ? u[row + M + m] : 0.0;
    const double wm = i > 0 ? u[row - M + m] : 0.0;
    const double D0 = coef_D(coef, w0);
    const double a_plus = 0.5 * (coef_D(coef, wp) + D0);
    const double a_minus = 0.5 * (coef_D(coef, wm) + D0);
    const double diffusion = (a_plus * (wp - w0) - a_minus * (w0 - wm)) / h2;
    const double convection = c >= 0.0 ? c * (wp - w0) / h : c * (w0 - wm) / h;
    const double val = base[row + m] + sign * (t - (diffusion + convection));
    out[row + m] = val;
    const double a = fabs(val);
    local = fmax(local, a <= DBL_MAX ? a : (double)INFINITY);
  }
  for (int o = 16; o > 0; o >>= 1) local = fmax(local, __shfl_xor_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0 && norm_bits != nullptr) {
    double mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, wmax[w]);
    atomicMax(norm_bits, (unsigned long long)__double_as_longlong(mx));
  }
}

// Full weighting (1/4)[1 2 1] of two fine fields (n = 2 nc + 1 lines) at once.
__global__ void k_fas_restrict2(const double* __restrict__ a, double* __restrict__ ac,
                                const double* __restrict__ b, double* __restrict__ bc, int nc,
                                int M) {
  const size_t total = (size_t)nc * M;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t J = idx / M, m = idx % M;
    const size_t f0 = 2 * J * M + m;  // fine line 2J, then 2J+1 and 2J+2
    ac[idx] = 0.25 * ((a[f0] + 2.0 * a[f0 + M]) + a[f0 + 2 * M]);
    bc[idx] = 0.25 * ((b[f0] + 2.0 * b[f0 + M]) + b[f0 + 2 * M]);
  }
}

// u (n = 2 nc + 1 lines) += P (uc - ubar): fine line 2J+1 takes coarse J, fine
// line 2J the mean of coarse J-1 and J (zero beyond the boundary).
__global__ void k_fas_correct(double* __restrict__ u, const double* __restrict__ uc,
                              const double* __restrict__ ubar, int nc, int M) {
  const int n = 2 * nc + 1;
  const size_t total = (size_t)n * M;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(idx / M);
    const size_t m = idx % M;
    double p;
    if (I & 1) {
      const size_t cj = (size_t)((I - 1) / 2) * M + m;
      p = uc[cj] - ubar[cj];
    } else {
      const int J = I / 2;
      p = 0.0;
      if (J >= 1) p += 0.5 * (uc[(size_t)(J - 1) * M + m] - ubar[(size_t)(J - 1) * M + m]);
      if (J < nc) p += 0.5 * (uc[(size_t)J * M + m] - ubar[(size_t)J * M + m]);
    }
    u[idx] += p;
  }
}

}  // namespace
}  // namespace mgwr

// ---- handle -------------------------------------------------------------------------

using mgwr::Cx;

struct mgwr_fas {
  int n = 0, M = 0, nlev = 0, coef = 0, order = MGWR_ORDER_TEXT;
  double T = 0.0, alpha = 0.0, c = 0.0;
  cudaStream_t stream = nullptr;  // the stream every launch and copy goes to
  cudaStream_t own = nullptr;     // the stream the handle created
  double* r = nullptr;       // r_1..r_M of T_M
  double* dk = nullptr;      // d_0..d_M (written by the coefficient kernel)
  double* params = nullptr;  // alpha, tau^-alpha / Gamma(2 - alpha)
  std::vector<double*> u, f, rr, ubar;  // per level, coarsest first
  unsigned long long* flags = nullptr;  // [0] max-norm bits, [1] line-solve status,
                                        // [2] fixed-point line iterations so far
  // whole-line fixed-point smoother (k_fas_fixed): twiddles, per-level inverse
  // columns of T_M + sigma_l I and their spectra; null when M is not a power of
  // two in 128 .. 1024, where the time march serves
  int smoother = MGWR_FAS_SMOOTHER_AUTO;
  Cx<double>* tw = nullptr;
  double* kcol = nullptr;
  Cx<double>* kspec = nullptr;
  std::vector<double> sigma;
  size_t line_smem = 0, apply_smem = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

namespace {

int fas_fail(mgwr_fas_t h, int code, const std::string& msg) {
  if (h != nullptr) h->err = msg;
  return code;
}

int fas_cuda(mgwr_fas_t h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MGWR_OK;
  cudaGetLastError();
  return fas_fail(h, MGWR_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

inline int level_n(int l) { return (1 << (l + 1)) - 1; }
inline double level_h(int l) { return 1.0 / (double)(level_n(l) + 1); }
inline size_t field_bytes(const mgwr_fas* h, int l) {
  return sizeof(double) * (size_t)level_n(l) * h->M;
}

// red = the colour visited first: 1-D text order odd i, table order even i
inline int colour_parity(const mgwr_fas* h, int colour) {
  const int red = h->order == MGWR_ORDER_TEXT ? 1 : 0;
  return colour == MGWR_RED ? red : 1 - red;
}

bool fixed_point(const mgwr_fas* h) {
  return h->kspec != nullptr && h->smoother != MGWR_FAS_SMOOTHER_MARCH;
}

constexpr int kFixedMaxIt = 200;  // fixed-point iterations per half-sweep before giving up

cudaError_t launch_line(mgwr_fas* h, int l, int parity, int all_points) {
  const int n = level_n(l);
  const int count = all_points ? n : (parity ? n / 2 : (n + 1) / 2);
  if (count == 0) return cudaSuccess;
  if (fixed_point(h)) {
    const int L = 2 * h->M, logL = mgwr::ilog2(L);
    const double hl = level_h(l);
    const unsigned grid = (unsigned)((count + 1) / 2);
    const size_t smem = mgwr::Pad<double>::len(L) * sizeof(Cx<double>);
    const Cx<double>* ks = h->kspec + (size_t)l * L;
    int* st = reinterpret_cast<int*>(h->flags + 1);
#define MGWR_FIXED_LAUNCH(B)                                                                    \
  mgwr::k_fas_fixed<B><<<grid, B, smem, h->stream>>>(h->u[l], h->f[l], ks, h->tw, n, h->M, logL, \
                                                     1.0 / hl, 1.0 / (hl * hl), h->c,           \
                                                     h->sigma[l], h->coef, parity, all_points,   \
                                                     kFixedMaxIt, st, h->flags + 2)
    switch (L / 8) {
      case 32: MGWR_FIXED_LAUNCH(32); break;
      case 64: MGWR_FIXED_LAUNCH(64); break;
      case 128: MGWR_FIXED_LAUNCH(128); break;
      default: MGWR_FIXED_LAUNCH(256); break;
    }
#undef MGWR_FIXED_LAUNCH
    return mgwr::counted(cudaGetLastError());
  }
  const int blocks = (count + mgwr::kLineWarps - 1) / mgwr::kLineWarps;
  mgwr::k_fas_line<<<blocks, 32 * mgwr::kLineWarps, h->line_smem, h->stream>>>(
      h->u[l], h->f[l], h->r, n, h->M, level_h(l), h->c, h->coef, parity, all_points,
      reinterpret_cast<int*>(h->flags + 1));
  return mgwr::counted(cudaGetLastError());
}

cudaError_t launch_apply(mgwr_fas* h, int l, const double* u, const double* base, double* out,
                         double sign, bool norm) {
  mgwr::k_fas_apply<<<level_n(l), mgwr::kApplyThreads, h->apply_smem, h->stream>>>(
      u, h->r, base, out, level_n(l), h->M, level_h(l), h->c, h->coef, sign,
      norm ? h->flags : nullptr);
  return mgwr::counted(cudaGetLastError());
}

inline int grid_for(size_t total) {
  const size_t b = (total + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

cudaError_t smooth_steps(mgwr_fas* h, int l, int steps) {
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < steps && e == cudaSuccess; ++s) {
    e = launch_line(h, l, colour_parity(h, MGWR_RED), 0);
    if (e == cudaSuccess) e = launch_line(h, l, colour_parity(h, MGWR_BLACK), 0);
  }
  return e;
}

// One FAS cycle at level l on the handle's stream (no synchronisation).
cudaError_t fas_cycle(mgwr_fas* h, int l, int nu1, int nu2, int gamma) {
  if (l == 0) return launch_line(h, 0, 0, 1);
  cudaError_t e = smooth_steps(h, l, nu1);
  if (e != cudaSuccess) return e;
  // r = f - N_h(u)
  if ((e = launch_apply(h, l, h->u[l], h->f[l], h->rr[l], -1.0, false)) != cudaSuccess) return e;
  const int nc = level_n(l - 1);
  // ubar = R u, R r (into the coarse defect field, free until the coarse cycle)
  mgwr::k_fas_restrict2<<<grid_for((size_t)nc * h->M), 256, 0, h->stream>>>(
      h->u[l], h->ubar[l - 1], h->rr[l], h->rr[l - 1], nc, h->M);
  if ((e = mgwr::counted(cudaGetLastError())) != cudaSuccess) return e;
  // f_c = N_2h(ubar) + R r; the coarse iterate starts from ubar
  if ((e = launch_apply(h, l - 1, h->ubar[l - 1], h->rr[l - 1], h->f[l - 1], 1.0, false)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(h->u[l - 1], h->ubar[l - 1], field_bytes(h, l - 1),
                           cudaMemcpyDeviceToDevice, h->stream)) != cudaSuccess)
    return e;
  for (int g = 0; g < gamma; ++g)
    if ((e = fas_cycle(h, l - 1, nu1, nu2, gamma)) != cudaSuccess) return e;
  // u += P (u_c - ubar)
  mgwr::k_fas_correct<<<grid_for((size_t)level_n(l) * h->M), 256, 0, h->stream>>>(
      h->u[l], h->u[l - 1], h->ubar[l - 1], nc, h->M);
  if ((e = mgwr::counted(cudaGetLastError())) != cudaSuccess) return e;
  return smooth_steps(h, l, nu2);
}

// Reads the max-norm and Newton status written since the last clear (synchronises).
int read_flags(mgwr_fas* h, double* norm, bool* newton_failed) {
  unsigned long long host[2] = {0, 0};
  int s = fas_cuda(h, cudaMemcpyAsync(host, h->flags, sizeof(host), cudaMemcpyDeviceToHost,
                                      h->stream), "read flags");
  if (s == MGWR_OK) s = fas_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
  if (s != MGWR_OK) return s;
  if (norm) {
    double v;
    std::memcpy(&v, &host[0], sizeof(v));
    *norm = v;
  }
  if (newton_failed) *newton_failed = (host[1] & 3ull) != 0;
  return MGWR_OK;
}

cudaError_t clear_norm(mgwr_fas* h) {
  return cudaMemsetAsync(h->flags, 0, sizeof(unsigned long long), h->stream);
}

int defect_norm(mgwr_fas* h, int l, double* norm) {
  int s = fas_cuda(h, clear_norm(h), "clear norm");
  if (s == MGWR_OK)
    s = fas_cuda(h, launch_apply(h, l, h->u[l], h->f[l], h->rr[l], -1.0, true), "defect");
  bool failed = false;
  if (s == MGWR_OK) s = read_flags(h, norm, &failed);
  if (s == MGWR_OK && failed)
    s = fas_fail(h, MGWR_E_NUMERIC, "a line solve did not settle (Newton's method or the whole-line fixed point)");
  return s;
}

double* field_of(mgwr_fas* h, int l, int which) {
  switch (which) {
    case MGWR_U: return h->u[l];
    case MGWR_F: return h->f[l];
    case MGWR_R: return h->rr[l];
    default: return nullptr;
  }
}

void release(mgwr_fas* h) {
  auto fr = [](double* p) { if (p) cudaFree(p); };
  for (auto* v : {&h->u, &h->f, &h->rr, &h->ubar})
    for (double* p : *v) fr(p);
  fr(h->r);
  fr(h->dk);
  fr(h->params);
  fr(h->kcol);
  if (h->kspec) cudaFree(h->kspec);
  if (h->tw) cudaFree(h->tw);
  if (h->flags) cudaFree(h->flags);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->own) cudaStreamDestroy(h->own);
}

}  // namespace

extern "C" {

int mgwr_fas_create(int n, int M, double T, double alpha, double c, int coefficient,
                    mgwr_fas_t* out) {
  if (out == nullptr) return MGWR_E_INVAL;
  *out = nullptr;
  if (n < 1 || n > 4095 || ((n + 1) & n) != 0) return MGWR_E_INVAL;
  if (M < 1 || M > mgwr::kFasMaxM) return MGWR_E_INVAL;
  if (!(T > 0.0) || !std::isfinite(T) || !(alpha > 0.0) || !(alpha <= 1.0)) return MGWR_E_INVAL;
  if (!std::isfinite(c)) return MGWR_E_INVAL;
  if (coefficient != MGWR_FAS_D_POROUS && coefficient != MGWR_FAS_D_CONSTANT) return MGWR_E_INVAL;
  // the smoother starts each Newton solve in FP32: its coefficients, the L1 scale
  // tau^-alpha / Gamma(2 - alpha) and |c| / h, must stay far inside FP32's range
  const double l1_scale = std::pow(T / M, -alpha) / std::tgamma(2.0 - alpha);
  if (!(l1_scale <= 1e30) || !(std::fabs(c) <= 1e30)) return MGWR_E_INVAL;
  mgwr_fas* h = new (std::nothrow) mgwr_fas;
  if (h == nullptr) return MGWR_E_NOMEM;
  h->n = n;
  h->M = M;
  h->T = T;
  h->alpha = alpha;
  h->c = c;
  h->coef = coefficient;
  while (level_n(h->nlev) < n) ++h->nlev;
  ++h->nlev;  // levels 0..nlev-1 with level_n(nlev-1) = n
  h->line_smem = sizeof(double) * (size_t)(1 + mgwr::kLineWarps) * M;
  h->apply_smem = sizeof(double) * 2 * (size_t)M;
  auto bail = [&](int code) {
    release(h);
    delete h;
    return code;
  };
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    cudaGetLastError();
    return bail(MGWR_E_CUDA);
  }
  h->stream = h->own;
  auto alloc = [&](double** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return false;
    }
    return true;
  };
  bool ok = alloc(&h->r, sizeof(double) * M) && alloc(&h->dk, sizeof(double) * (M + 1)) &&
            alloc(&h->params, sizeof(double) * 2);
  if (ok && cudaMalloc(&h->flags, 3 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    h->flags = nullptr;
    ok = false;
  }
  for (int l = 0; ok && l < h->nlev; ++l) {
    double *u = nullptr, *f = nullptr, *r = nullptr, *ub = nullptr;
    ok = alloc(&u, field_bytes(h, l)) && alloc(&f, field_bytes(h, l)) &&
         alloc(&r, field_bytes(h, l)) && alloc(&ub, field_bytes(h, l));
    h->u.push_back(u);
    h->f.push_back(f);
    h->rr.push_back(r);
    h->ubar.push_back(ub);
  }
  if (!ok) return bail(MGWR_E_NOMEM);
  // (1 + kLineWarps) * 1024 and 2 * 1024 doubles: within the default 48 KB
  static_assert((1 + mgwr::kLineWarps) * mgwr::kFasMaxM * sizeof(double) <= 48 * 1024,
                "k_fas_line shared memory");
  cudaError_t e = cudaSuccess;
  const double params[2] = {alpha, l1_scale};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->params, params, sizeof(params), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = mgwr::launch_coefficients(h->r, h->dk, M, h->params, h->params + 1, 1, h->stream);
  for (int l = 0; e == cudaSuccess && l < h->nlev; ++l) {
    e = cudaMemsetAsync(h->u[l], 0, field_bytes(h, l), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->f[l], 0, field_bytes(h, l), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->rr[l], 0, field_bytes(h, l), h->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->flags, 0, 3 * sizeof(unsigned long long), h->stream);
  // the fixed-point smoother's setup (Sec. 5): per level sigma_l = 2/h_l^2 + |c|/h_l,
  // the first column of (T_M + sigma_l I)^{-1} by divide and conquer, its spectrum
  if (e == cudaSuccess && M >= 128 && (M & (M - 1)) == 0) {
    const int L = 2 * M;
    for (int l = 0; l < h->nlev; ++l) {
      const double hl = level_h(l);
      h->sigma.push_back(2.0 / (hl * hl) + std::fabs(c) / hl);
    }
    double* sig_dev = nullptr;
    Cx<double>* work = nullptr;
    ok = alloc(&h->kcol, sizeof(double) * (size_t)h->nlev * M) &&
         alloc(&sig_dev, sizeof(double) * (size_t)h->nlev) &&
         cudaMalloc(&h->kspec, sizeof(Cx<double>) * (size_t)h->nlev * L) == cudaSuccess &&
         cudaMalloc(&h->tw, sizeof(Cx<double>) * (size_t)L) == cudaSuccess &&
         cudaMalloc(&work, sizeof(Cx<double>) * (size_t)h->nlev * 3 * M) == cudaSuccess;
    if (ok) {
      e = cudaMemcpyAsync(sig_dev, h->sigma.data(), sizeof(double) * h->nlev,
                          cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess)
        e = mgwr::launch_inverse_columns(h->kcol, h->r, sig_dev, h->nlev, M, 1, work, h->stream);
      if (e == cudaSuccess) e = mgwr::launch_twiddles(h->tw, L, h->stream);
      if (e == cudaSuccess)
        e = mgwr::launch_spectra(h->kspec, h->kcol, h->nlev, M, h->tw, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    } else {
      cudaGetLastError();
    }
    if (sig_dev) cudaFree(sig_dev);
    if (work) cudaFree(work);
    if (!ok) return bail(MGWR_E_NOMEM);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(MGWR_E_CUDA);
  }
  *out = h;
  return MGWR_OK;
}

int mgwr_fas_destroy(mgwr_fas_t h) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (h->stream) cudaStreamSynchronize(h->stream);
  release(h);
  delete h;
  return MGWR_OK;
}

const char* mgwr_fas_last_error(mgwr_fas_t h) { return h ? h->err.c_str() : "null handle"; }

int mgwr_fas_set_order(mgwr_fas_t h, int order) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (order != MGWR_ORDER_TEXT && order != MGWR_ORDER_TABLE)
    return fas_fail(h, MGWR_E_INVAL, "order must be MGWR_ORDER_TEXT or MGWR_ORDER_TABLE");
  h->order = order;
  return MGWR_OK;
}

int mgwr_fas_set_stream(mgwr_fas_t h, void* stream) {
  if (h == nullptr) return MGWR_E_INVAL;
  int s = fas_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
  if (s == MGWR_OK) h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own;
  return s;
}

int mgwr_fas_reset(mgwr_fas_t h) {
  if (h == nullptr) return MGWR_E_INVAL;
  const int L = h->nlev - 1;
  int s = fas_cuda(h, cudaMemsetAsync(h->u[L], 0, field_bytes(h, L), h->stream), "clear u");
  if (s == MGWR_OK)
    s = fas_cuda(h, cudaMemsetAsync(h->flags, 0, 2 * sizeof(unsigned long long), h->stream),
                 "clear flags");
  return s;
}

int mgwr_fas_levels(mgwr_fas_t h, int* levels) {
  if (h == nullptr || levels == nullptr) return MGWR_E_INVAL;
  *levels = h->nlev;
  return MGWR_OK;
}

int mgwr_fas_field_set(mgwr_fas_t h, int level, int which, const double* host) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (level < 0 || level >= h->nlev || host == nullptr || field_of(h, level, which) == nullptr)
    return fas_fail(h, MGWR_E_INVAL, "bad level, field or pointer");
  int s = fas_cuda(h, cudaMemcpyAsync(field_of(h, level, which), host, field_bytes(h, level),
                                      cudaMemcpyHostToDevice, h->stream), "field_set");
  if (s == MGWR_OK) s = fas_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
  return s;
}

int mgwr_fas_field_get(mgwr_fas_t h, int level, int which, double* host) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (level < 0 || level >= h->nlev || host == nullptr || field_of(h, level, which) == nullptr)
    return fas_fail(h, MGWR_E_INVAL, "bad level, field or pointer");
  int s = fas_cuda(h, cudaMemcpyAsync(host, field_of(h, level, which), field_bytes(h, level),
                                      cudaMemcpyDeviceToHost, h->stream), "field_get");
  if (s == MGWR_OK) s = fas_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
  return s;
}

int mgwr_fas_set_rhs(mgwr_fas_t h, const double* f) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (f == nullptr) return fas_fail(h, MGWR_E_INVAL, "null right-hand side");
  const int L = h->nlev - 1;
  int s = fas_cuda(h, cudaMemsetAsync(h->u[L], 0, field_bytes(h, L), h->stream), "clear u");
  if (s == MGWR_OK)
    s = fas_cuda(h, cudaMemsetAsync(h->flags, 0, 2 * sizeof(unsigned long long), h->stream),
                 "clear flags");
  if (s == MGWR_OK) s = mgwr_fas_field_set(h, L, MGWR_F, f);
  return s;
}

int mgwr_fas_set_initial(mgwr_fas_t h, const double* u0) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (u0 == nullptr) return fas_fail(h, MGWR_E_INVAL, "null initial iterate");
  const int s = fas_cuda(
      h, cudaMemsetAsync(h->flags, 0, 2 * sizeof(unsigned long long), h->stream), "clear flags");
  return s == MGWR_OK ? mgwr_fas_field_set(h, h->nlev - 1, MGWR_U, u0) : s;
}

int mgwr_fas_get_solution(mgwr_fas_t h, double* u_host) {
  if (h == nullptr) return MGWR_E_INVAL;
  return mgwr_fas_field_get(h, h->nlev - 1, MGWR_U, u_host);
}

int mgwr_fas_defect(mgwr_fas_t h, int level, double* norm_inf) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (level < 0 || level >= h->nlev) return fas_fail(h, MGWR_E_INVAL, "bad level");
  double nrm = 0.0;
  const int s = defect_norm(h, level, &nrm);
  if (s == MGWR_OK && norm_inf) *norm_inf = nrm;
  return s;
}

int mgwr_fas_residual(mgwr_fas_t h, double* norm_inf, double* r_host) {
  if (h == nullptr) return MGWR_E_INVAL;
  const int L = h->nlev - 1;
  int s = mgwr_fas_defect(h, L, norm_inf);
  if (s == MGWR_OK && r_host) s = mgwr_fas_field_get(h, L, MGWR_R, r_host);
  return s;
}

int mgwr_fas_set_smoother(mgwr_fas_t h, int smoother) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (smoother != MGWR_FAS_SMOOTHER_AUTO && smoother != MGWR_FAS_SMOOTHER_MARCH &&
      smoother != MGWR_FAS_SMOOTHER_FIXED)
    return fas_fail(h, MGWR_E_INVAL, "unknown smoother");
  if (smoother == MGWR_FAS_SMOOTHER_FIXED && h->kspec == nullptr)
    return fas_fail(h, MGWR_E_INVAL, "the fixed-point smoother needs M a power of two in 128..1024");
  h->smoother = smoother;
  return MGWR_OK;
}

int mgwr_fas_line_iterations(mgwr_fas_t h, long long* count) {
  if (h == nullptr || count == nullptr) return MGWR_E_INVAL;
  unsigned long long v = 0;
  int s = fas_cuda(h, cudaMemcpyAsync(&v, h->flags + 2, sizeof(v), cudaMemcpyDeviceToHost,
                                      h->stream), "read count");
  if (s == MGWR_OK) s = fas_cuda(h, cudaStreamSynchronize(h->stream), "synchronize");
  if (s == MGWR_OK) *count = (long long)v;
  return s;
}

int mgwr_fas_smooth(mgwr_fas_t h, int level, int colour) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (level < 0 || level >= h->nlev || (colour != MGWR_RED && colour != MGWR_BLACK))
    return fas_fail(h, MGWR_E_INVAL, "bad level or colour");
  int s = fas_cuda(h, launch_line(h, level, colour_parity(h, colour), 0), "smooth");
  bool failed = false;
  if (s == MGWR_OK) s = read_flags(h, nullptr, &failed);
  if (s == MGWR_OK && failed)
    s = fas_fail(h, MGWR_E_NUMERIC, "a line solve did not settle (Newton's method or the whole-line fixed point)");
  return s;
}

int mgwr_fas_cycle(mgwr_fas_t h, int cycle, int nu1, int nu2) {
  if (h == nullptr) return MGWR_E_INVAL;
  if ((cycle != 1 && cycle != 2) || nu1 < 0 || nu2 < 0 || nu1 + nu2 < 1 || nu1 > 16 || nu2 > 16)
    return fas_fail(h, MGWR_E_INVAL, "bad cycle parameters");
  int s = fas_cuda(h, fas_cycle(h, h->nlev - 1, nu1, nu2, cycle), "cycle");
  bool failed = false;
  if (s == MGWR_OK) s = read_flags(h, nullptr, &failed);
  if (s == MGWR_OK && failed)
    s = fas_fail(h, MGWR_E_NUMERIC, "a line solve did not settle (Newton's method or the whole-line fixed point)");
  return s;
}

int mgwr_fas_solve(mgwr_fas_t h, int cycle, int nu1, int nu2, double tol, int max_cycles,
                   mgwr_stats* stats) {
  if (h == nullptr) return MGWR_E_INVAL;
  if ((cycle != 1 && cycle != 2) || nu1 < 0 || nu2 < 0 || nu1 + nu2 < 1 || nu1 > 16 ||
      nu2 > 16 || !(tol >= 0.0) || max_cycles < 0)
    return fas_fail(h, MGWR_E_INVAL, "bad solve parameters");
  const int L = h->nlev - 1;
  mgwr_stats st{};
  double r0 = 0.0;
  int s = defect_norm(h, L, &r0);
  if (s != MGWR_OK) return s;
  if (!std::isfinite(r0)) return fas_fail(h, MGWR_E_NUMERIC, "non-finite initial defect");
  if (r0 == 0.0) {
    if (stats) *stats = st;
    return MGWR_OK;
  }
  st.relres = 1.0;
  s = fas_cuda(h, cudaEventRecord(h->ev0, h->stream), "event");
  while (s == MGWR_OK && st.cycles < max_cycles && st.relres > tol) {
    s = fas_cuda(h, fas_cycle(h, L, nu1, nu2, cycle), "cycle");
    double nrm = 0.0;
    if (s == MGWR_OK) s = defect_norm(h, L, &nrm);
    if (s != MGWR_OK) break;
    ++st.cycles;
    st.relres = nrm / r0;
    if (!std::isfinite(st.relres)) s = fas_fail(h, MGWR_E_NUMERIC, "non-finite defect");
  }
  if (cudaEventRecord(h->ev1, h->stream) == cudaSuccess &&
      cudaEventSynchronize(h->ev1) == cudaSuccess) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) st.seconds = 1e-3 * ms;
  }
  cudaGetLastError();
  st.factor = st.cycles > 0 ? std::pow(st.relres, 1.0 / st.cycles) : 0.0;
  if (stats) *stats = st;
  if (s != MGWR_OK) return s;
  return st.relres <= tol ? MGWR_OK
                          : fas_fail(h, MGWR_E_NOCONV, "max_cycles reached before tol");
}

}  // extern "C"

// Internal declarations shared by the kernel and host translation units of the
// MGWR library.  Not part of the public ABI (see include/mgwr.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "mgwr_dd.cuh"

namespace mgwr {

template <class R>
struct alignas(2 * sizeof(R)) Cx {
  R x, y;
};

// Spectral layout of every length-L FFT in this library: the forward
// transform is a decimation-in-frequency radix-8 cascade (last stage radix 8,
// 4 or 2) that leaves its output in digit-reversed order; spectra are stored
// in that order, pre-scaled by 1/L, and the inverse cascade consumes it.  Only
// products of two such spectra are ever formed, so the order never matters.

// Shape of one level of a batch of same-shape instances: n^d lines of M
// values per instance, instances stored one after another.
struct LevelShape {
  int d, n, M, batch;
  size_t field_stride() const { return (size_t)(d == 1 ? n : n * n) * M; }
};

// Time lines up to kShortMaxM values are convolved with one transform of
// length 2M.  Longer lines (partitioned convolution) are cut into blocks of
// kLongB values, each transformed at length 2 kLongB; their spectra and the
// kernel segments keep the total length 2M per line (P = M / kLongB segments
// of 2 kLongB values).  engine_length(M) is the transform length, and so the
// length of the twiddle table.
constexpr int kShortMaxM = 4096;
constexpr int kLongB = 4096;
constexpr int kMaxM = 1 << 20;
inline int engine_length(int M) { return M <= kShortMaxM ? 2 * M : 2 * kLongB; }
// Butterflies per thread of the FFT engine for a transform of length L:
// E in {1, 2, 4} and at most L/8; any other request selects 1.
// A split value may carry kStaged: the FP32 sweep of lines of 64 .. 4096 steps
// then runs persistently with its input lines staged in shared memory by bulk
// copies (mgwr_sweep_staged.cu); every other launch ignores the bit.
constexpr int kStaged = 16;
// A split value may instead carry kTensor: the FP32 sweep of lines of 64, 128
// or 256 steps then runs on the tensor cores (mgwr_sweep_tc.cu).
constexpr int kTensor = 32;
inline bool tensor_length(int M) { return M == 64 || M == 128 || M == 256; }
// Or kRadix: the FP32 sweep of lines of 64 .. 4096 steps then runs on the
// register-pass engine (mgwr_sweep_rp.cu, radix-32 passes in registers).
constexpr int kRadix = 64;
inline bool radix_length(int M) { return M >= 64 && M <= kShortMaxM; }
inline int engine_split(int L, int E) {
  E &= ~(kStaged | kTensor | kRadix);
  if (E != 2 && E != 4) E = 1;
  while (E > 1 && L / 8 < E) E >>= 1;
  return E;
}
// The split a launch on lines of M values in an arithmetic of `word` bytes
// really uses when E is requested: the partitioned convolution has E = 1 or
// 2, the FP32 kernels split only their compile-time lengths 2^7 .. 2^13.
inline int effective_split(int M, int word, int E) {
  const int staged = E & kStaged;
  const int tensor = E & kTensor;
  const int radix = E & kRadix;
  E &= ~(kStaged | kTensor | kRadix);
  if (M > kShortMaxM) return E == 2 ? 2 : 1;
  const int L = 2 * M;
  E = engine_split(L, E);
  if (word == 4 && (L < 128 || L > 8192)) return 1;
  if (word == 4 && radix && radix_length(M)) return E | kRadix;
  if (word == 4 && tensor && tensor_length(M)) return 1 | kTensor;
  return word == 4 ? (E | staged) : E;
}
// Complex values of the partitioned-convolution scratch for one launch on a
// level of shape ls: per instance, per line pair, the spectra of all blocks.
inline size_t long_scratch_count(const LevelShape& ls) {
  if (ls.M <= kShortMaxM) return 0;
  const size_t pts = (size_t)(ls.d == 1 ? ls.n : ls.n * ls.n);
  return (size_t)ls.batch * ((pts + 1) / 2) * 2 * (size_t)ls.M;
}

// ---- launchers (kernels in mgwr_kernels.cu); all return the launch status ----
// Every launcher covers all `batch` instances (blockIdx.y = instance).

// One colour half-sweep (Sec. 3 Eq. red-black, Sec. 6 Eq. red-black_2d): for
// each point p of parity `par`, u_p = k * (f_p + hinv2 * sum of neighbour
// lines), k the inverse column whose spectrum is `spec` (instance b's at
// spec + b * spec_stride).  all_points: every point, no neighbour term
// (one-point coarsest solve).  delta != null: also delta_p = u_p(new) -
// u_p(old) on the swept lines.
// `zero` is a line of M zeros standing in for neighbours outside the grid.
// For M > kShortMaxM, `scratch` holds long_scratch_count(ls) values (unused
// otherwise, may be null).
// E: butterflies per thread of the FFT engine (engine_split; the launch shape
// only, results are identical for every E).
template <class R>
cudaError_t launch_sweep(const R* f, R* u, R* delta, const Cx<R>* spec, size_t spec_stride,
                         const Cx<R>* tw, const R* zero, Cx<R>* scratch, const LevelShape& ls,
                         int par, bool all_points, R hinv2, int E, cudaStream_t s);

// launch_sweep<float> for 64 <= M <= kShortMaxM without all_points, E carrying
// kStaged: a persistent grid (as many CTAs as fit on the GPU) walks the line
// pairs; while a group transforms one pair, the f and neighbour lines of its
// next pair are copied into shared memory by cp.async.bulk, completing on an
// mbarrier.  Same arithmetic in the same order as the direct-load kernel, so
// the results are bitwise identical.  A wait that gives up (half a second) sets
// a device flag read by take_stage_timeout.
cudaError_t launch_sweep_staged(const float* f, float* u, float* delta, const Cx<float>* spec,
                                size_t spec_stride, const Cx<float>* tw, const float* zero,
                                const LevelShape& ls, int par, float hinv2, int E,
                                cudaStream_t s);
// Reads and clears the flag of the staged sweep's bounded waits (synchronous).
cudaError_t take_stage_timeout(bool* hit);

// One colour half-sweep of FP32 lines of M = 64, 128 or 256 steps on the
// tensor cores (tcgen05.mma, bf16 x 3 pieces, FP32 accumulation): as
// launch_sweep without all_points, with the inverse column of instance b given
// as its Toeplitz band (band + b * bstride, tc_band_bytes(M) bytes, written by
// launch_band_bf16x3).  Results agree with the FFT engine's to FP32 rounding
// (not bitwise).  A wait that gives up (half a second) sets a flag read by
// take_tc_timeout.
cudaError_t launch_sweep_tc(const float* f, float* u, float* delta, const unsigned char* band,
                            size_t bstride, const LevelShape& ls, int par, float hinv2,
                            cudaStream_t s);
// Bytes of one Toeplitz band: three bf16 pieces of M rows x 32 columns.
size_t tc_band_bytes(int M);
// band + line * tc_band_bytes(M): the band of the inverse column kcol[line]
// (rows t, columns k < 32: k_{t-k}, 0 for t < k) split into three bf16 pieces
// (x = x0 + x1 + x2), in the tensor-core kernel's shared-memory layout.
cudaError_t launch_band_bf16x3(const double* kcol, unsigned char* band, int M, size_t lines,
                               cudaStream_t s);
cudaError_t take_tc_timeout(bool* hit);

// One colour half-sweep of FP32 lines of 64 .. 4096 steps on the register-pass
// FFT engine (mgwr_fft_rp.cuh): as launch_sweep without all_points, with the
// inverse-column spectra in that engine's spectral order (launch_spectra_rp).
// Results agree with the shared-memory engine's to FP32 rounding, not bitwise.
// paired: the first pass's adjacent butterflies two at a time with 8-byte
// global accesses (the split's E: 1 | kRadix single, 2 | kRadix paired).
// Forms of the register-pass sweep: first-pass butterflies one at a time,
// two adjacent at a time (8-byte gathers and stores), or paired with resident
// blocks holding the spectrum and twiddle bases in shared memory.
constexpr int kRpSingle = 1, kRpPaired = 2, kRpResident = 4;
cudaError_t launch_sweep_rp(const float* f, float* u, float* delta, const Cx<float>* spec,
                            size_t spec_stride, const Cx<float>* tw, const float* zero,
                            const LevelShape& ls, int par, float hinv2, int form,
                            cudaStream_t s);
// dst[c L ..] = the FP64 spectra src[c L ..] (length L = 2M, the shared-memory
// engine's order) rounded to FP32 and permuted into the register-pass engine's
// order (the sweeps' plans, or the carried defect's when `defect`), for
// `lines` lines.
cudaError_t launch_spectra_rp(Cx<float>* dst, const Cx<double>* src, size_t lines, int M,
                              bool defect, cudaStream_t s);

// Defect after a red-black step from the black half-sweep's delta: r = 0 on the
// black points, r = hinv2 * sum of neighbour deltas on the red points
// (parity red_par); |r|_inf of instance b folded into norm_bits[b].
template <class R>
cudaError_t launch_defect_from_delta(const R* delta, R* r, const R* zero, const LevelShape& ls,
                                     int red_par, R hinv2, unsigned long long* norm_bits,
                                     cudaStream_t s);

// r = f - T_M u - A_h u for all points; |r|_inf of instance b folded into
// norm_bits[b] (bit pattern of a non-negative double, atomicMax) when non-null.
// `scratch` as for launch_sweep.
template <class R, class RO>
cudaError_t launch_defect(const R* u, const R* f, RO* r, const Cx<R>* tspec, size_t spec_stride,
                          const Cx<R>* tw, const R* zero, Cx<R>* scratch, const LevelShape& ls,
                          R hinv2, unsigned long long* norm_bits, int E, cudaStream_t s);

// The same two operations for M > kShortMaxM by partitioned convolution
// (mgwr_long.cu); `spec` / `tspec` hold the kernel segment spectra written by
// launch_spectra for that M.
template <class R>
cudaError_t launch_sweep_long(const R* f, R* u, R* delta, const Cx<R>* spec, size_t spec_stride,
                              const Cx<R>* tw, Cx<R>* scratch, const LevelShape& ls, int par,
                              bool all_points, R hinv2, int E, cudaStream_t s);
template <class R, class RO>
cudaError_t launch_defect_long(const R* u, const R* f, RO* r, const Cx<R>* tspec,
                               size_t spec_stride, const Cx<R>* tw, Cx<R>* scratch,
                               const LevelShape& ls, R hinv2, unsigned long long* norm_bits,
                               int E, cudaStream_t s);

// fc = full weighting of r (fine n -> coarse (n-1)/2), uc = 0.
template <class R>
cudaError_t launch_restrict(const R* r, R* fc, R* uc, const LevelShape& fine, cudaStream_t s);

// fc = full weighting of the defect after a red-black step, formed from the
// black half-sweep's changes delta (as launch_defect_from_delta would write
// it, red points of parity red_par) without storing it; uc = 0.  Bitwise the
// same fc as launch_defect_from_delta followed by launch_restrict.
template <class R>
cudaError_t launch_restrict_delta(const R* delta, R* fc, R* uc, const R* zero, const LevelShape& fine,
                                  int red_par, R hinv2, cudaStream_t s);

// u (fine, n) += linear / bilinear interpolation of uc (coarse (n-1)/2).
template <class R>
cudaError_t launch_prolong(R* u, const R* uc, const LevelShape& fine, cudaStream_t s);

// u += (double) e, elementwise.
cudaError_t launch_refine(double* u, const float* e, size_t count, cudaStream_t s);
// double-float: dst = split(src); dst = hi + lo; u += e; complex split.
cudaError_t launch_split(dd* dst, const double* src, size_t count, cudaStream_t s);
cudaError_t launch_join(double* dst, const dd* src, size_t count, cudaStream_t s);
cudaError_t launch_refine_dd(dd* u, const float* e, size_t count, cudaStream_t s);
// u += e in double-float (both double-float; the sum renormalised twice).
cudaError_t launch_refine_dd2(dd* u, const dd* e, size_t count, cudaStream_t s);
cudaError_t launch_split_cx(Cx<dd>* dst, const Cx<double>* src, size_t count, cudaStream_t s);
// dst = (float) src.
cudaError_t launch_round(float* dst, const double* src, size_t count, cudaStream_t s);
// Per instance b (x holds batch * per values): |x_b|_inf folded into
// norm_bits[b]; out_b = (float) x_b when out != null.
// State of a solve loop run on the device (a CUDA graph WHILE node whose body
// is one iteration and k_loop_decide): the stopping tolerance and iteration
// bound it was given, the iterations done and the last relative defect.
struct LoopState {
  double tol;
  double rel;
  int max_iter;
  int iters;
};
cudaError_t launch_loop_init(LoopState* st, double tol, int max_iter, cudaStream_t s);
// After an iteration: rel = max_b norm_b / r0_b (norm_bits as in the defect
// kernels; r0_b = 0 takes the norm itself), iters += 1, and the loop's
// condition set to continue while rel > tol, rel is finite and iters <
// max_iter.
cudaError_t launch_loop_decide(const unsigned long long* norm_bits, const double* r0, int batch,
                               LoopState* st, cudaGraphConditionalHandle loop, cudaStream_t s);
// Per instance (batch instances of `per` values): |x|_inf into norm_bits, and
// in the same pass, where not null, out = (float) x and out_dd = x split as
// launch_split does.
cudaError_t launch_absmax_round(const double* x, float* out, dd* out_dd, size_t per, int batch,
                                unsigned long long* norm_bits, cudaStream_t s);

// Outer defect of the mixed modes carried by the correction of an outer step
// (residual replacement): r_out = r_in - (T_M (x) I + A_h) e, where e is the
// step's FP32 correction (u_new = u_old + e), T_M e an FP32 FFT convolution
// (FP32 spectra `tspec`, twiddles `tw`) and the stencil on e, widened, and the
// subtraction in double-float (W = dd, the one instantiation); r_out also
// rounded into r32, |r_out|_inf of instance b into norm_bits[b].  r_in and
// r_out may be the same field.  hinv2 = 1/h^2 must be a power of 4 (exact in
// FP32 and in every scaling by it), as every level of the solver's grids has.
// Its error is that of one FP32 convolution of e, about 1e-6 of |T_M e|.  Lines of M <= kShortMaxM only (else
// cudaErrorInvalidValue).  zero: M FP32 zeros.
template <class W>
cudaError_t launch_defect_update(const float* e, const W* r_in, W* r_out, float* r32,
                                 const Cx<float>* tspec, size_t spec_stride, const Cx<float>* tw,
                                 const float* zero, const LevelShape& ls, float hinv2,
                                 unsigned long long* norm_bits, cudaStream_t s);
// The same on the register-pass engine (64 <= M <= kShortMaxM), tspec in its
// spectral order (launch_spectra_rp).
template <class W>
cudaError_t launch_defect_update_rp(const float* e, const W* r_in, W* r_out, float* r32,
                                    const Cx<float>* tspec, size_t spec_stride,
                                    const Cx<float>* tw, const float* zero, const LevelShape& ls,
                                    float hinv2, unsigned long long* norm_bits, cudaStream_t s);
// Full outer defect of an FP64 iterate with T_M u by a double-float FFT
// convolution of u split into double-float pairs (double-float spectra `tspec`,
// twiddles `tw`) and the stencil, source and subtractions in FP64: r = f -
// (T_M (x) I + A_h) u within about 2^-44 of |T_M u|, written in double-float to
// r and rounded to FP32 into r32; |r|_inf of instance b into norm_bits[b].  Lines
// of 4 <= M <= kShortMaxM (else cudaErrorInvalidValue).  zero: M FP64 zeros.
cudaError_t launch_defect_anchor(const double* u, const double* f, dd* r, float* r32,
                                 const Cx<dd>* tspec, size_t spec_stride, const Cx<dd>* tw,
                                 const double* zero, const LevelShape& ls, double hinv2,
                                 unsigned long long* norm_bits, cudaStream_t s);
// out = (float) x for a double-float field of `count` values.
cudaError_t launch_round_dd(const dd* x, float* out, size_t count, cudaStream_t s);
// Per instance b: u = broadcast of g_b along time (initial iterate u^0(t) = g);
// f += c_b d_{b,m} g_b.  g: batch * N, dk: batch * (M+1), c: batch (device).
cudaError_t launch_initial(double* u, double* f, const double* g, const double* dk, const double* c,
                           int N, int M, int batch, cudaStream_t s);

// ---- setup (FP64) ----
// Per instance b: r[b*M + i] = r_{i+1}, dk[b*(M+1) + m] = d_m (d_0 = 0), from
// alphas[b] and cs[b] = tau_b^-alpha_b / Gamma(2 - alpha_b) (device arrays).
cudaError_t launch_coefficients(double* r, double* dk, int M, const double* alphas,
                                const double* cs, int batch, cudaStream_t s);
// kcol[(b*nlev + l)*M ..] = first column of (T_{M,b} + sigma[l] I)^{-1} by
// divide and conquer with FFT convolutions; work: 3*M complex per (b, l).
cudaError_t launch_inverse_columns(double* kcol, const double* r, const double* sigma, int nlev,
                                   int M, int batch, Cx<double>* work, cudaStream_t s);
// tw[m] = exp(-2 pi i m / L), m < L.
cudaError_t launch_twiddles(Cx<double>* tw, int L, cudaStream_t s);
// spec[k*2M ..] = FFT_2M(pad(lines[k*M ..])) / 2M in the library's spectral
// order (M <= kShortMaxM); for longer M the kernel segment spectra of the
// partitioned convolution (launch_spectra_long), also 2M values per line.
// tw: engine_length(M) twiddles.
cudaError_t launch_spectra(Cx<double>* spec, const double* lines, int count, int M,
                           const Cx<double>* tw, cudaStream_t s);
cudaError_t launch_spectra_long(Cx<double>* spec, const double* lines, int count, int M,
                                const Cx<double>* tw, cudaStream_t s);
cudaError_t launch_round_cx(Cx<float>* dst, const Cx<double>* src, size_t count, cudaStream_t s);

// Kernel launches issued through the launchers above (process-wide counter),
// including those replayed from captured graphs (add_launches).
long long launch_counter();
void add_launches(long long n);
// Counts a kernel launch in that counter and passes the launch status through.
cudaError_t counted(cudaError_t e);

}  // namespace mgwr

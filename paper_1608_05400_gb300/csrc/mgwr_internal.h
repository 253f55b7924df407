// Internal declarations shared by the kernel and host translation units of the
// MGWR library.  Not part of the public ABI (see include/mgwr.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

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

// ---- launchers (kernels in mgwr_kernels.cu); all return the launch status ----

// One colour half-sweep (Sec. 3 Eq. red-black, Sec. 6 Eq. red-black_2d): for
// each point p of parity `par`, u_p = k * (f_p + hinv2 * sum of neighbour
// lines), k the inverse column whose spectrum is `spec`.  all_points: every
// point, no neighbour term (one-point coarsest solve).  delta != null: also
// delta_p = u_p(new) - u_p(old) on the swept lines.
template <class R>
cudaError_t launch_sweep(const R* f, R* u, R* delta, const Cx<R>* spec, const Cx<R>* tw, int d,
                         int n, int M, int par, bool all_points, R hinv2, cudaStream_t s);

// Defect after a red-black step from the black half-sweep's delta: r = 0 on the
// black points, r = hinv2 * sum of neighbour deltas on the red points
// (parity red_par); |r|_inf folded into *norm_bits when non-null.
template <class R>
cudaError_t launch_defect_from_delta(const R* delta, R* r, int d, int n, int M, int red_par,
                                     R hinv2, unsigned long long* norm_bits, cudaStream_t s);

// r = f - T_M u - A_h u for all points; |r|_inf folded into *norm_bits
// (bit pattern of a non-negative double, atomicMax) when norm_bits != null.
template <class R, class RO>
cudaError_t launch_defect(const R* u, const R* f, RO* r, const Cx<R>* tspec, const Cx<R>* tw,
                          int d, int n, int M, R hinv2, unsigned long long* norm_bits,
                          cudaStream_t s);

// fc = full weighting of r (fine n -> coarse (n-1)/2), uc = 0.
template <class R>
cudaError_t launch_restrict(const R* r, R* fc, R* uc, int d, int n, int M, cudaStream_t s);

// u (fine, n) += linear / bilinear interpolation of uc (coarse (n-1)/2).
template <class R>
cudaError_t launch_prolong(R* u, const R* uc, int d, int n, int M, cudaStream_t s);

// u += (double) e, elementwise.
cudaError_t launch_refine(double* u, const float* e, size_t count, cudaStream_t s);
// dst = (float) src.
cudaError_t launch_round(float* dst, const double* src, size_t count, cudaStream_t s);
// u = broadcast of g along time (initial iterate u^0(t) = g); f += c d_m g.
cudaError_t launch_initial(double* u, double* f, const double* g, const double* dk, double c,
                           int N, int M, cudaStream_t s);

// ---- setup (FP64) ----
// r[i] = r_{i+1}, i < M; dk[m] = d_m, m <= M (L1 weights, d_0 = 0).
cudaError_t launch_coefficients(double* r, double* dk, int M, double alpha, double c,
                                cudaStream_t s);
// For each level l < nlev: kcol[l*M ..] = first column of (T_M + sigma[l] I)^{-1}
// by divide and conquer with FFT convolutions; work: 3*M complex per level.
cudaError_t launch_inverse_columns(double* kcol, const double* r, const double* sigma,
                                   int nlev, int M, Cx<double>* work, cudaStream_t s);
// tw[m] = exp(-2 pi i m / L), m < L.
cudaError_t launch_twiddles(Cx<double>* tw, int L, cudaStream_t s);
// spec[k*L ..] = FFT_L(pad(lines[k*M ..])) / L in the library's spectral order.
cudaError_t launch_spectra(Cx<double>* spec, const double* lines, int count, int M,
                           const Cx<double>* tw, cudaStream_t s);
cudaError_t launch_round_cx(Cx<float>* dst, const Cx<double>* src, size_t count, cudaStream_t s);

// Kernel launches issued through the launchers above (process-wide counter).
long long launch_counter();

}  // namespace mgwr

// Shared-memory FFT engine for causal time-line convolutions (Sec. 5).
//
// Every time-line operator of the method is a lower-triangular Toeplitz matrix
// (T_M for the defect, the inverse (T_M + sigma I)^{-1} for the smoother).  Its
// product with a line x is the first M entries of the cyclic convolution of the
// zero-padded length-L = 2M sequences (Sec. 5, circulant embedding C_2M).  Two
// real lines are packed as the real and imaginary parts of one complex line, so
// one complex transform serves two spatial points.
//
// One thread group of L/(8E) threads owns one line pair; each thread does E
// radix-8 butterflies per stage (E = 1, 2 or 4: the launch shape, chosen per
// length and arithmetic by the tuner; groups of at most 32 threads synchronise
// with warp barriers only).  Forward transform: decimation in frequency,
// radix-8 stages (the first one reads the input from global memory and skips
// the zero upper half), a last stage of radix 8, 4 or 2 whose butterflies each
// thread does on 8 contiguous values.  The spectrum
// product is applied in registers right there, followed by the matching
// inverse stage, so the result never needs reordering: the inverse cascade
// runs the forward one backwards with conjugate twiddles and writes only the
// first M outputs.
#pragma once

#include <type_traits>

#include "mgwr_internal.h"

namespace mgwr {

template <class R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R>
__device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <class R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <class R>
__device__ __forceinline__ Cx<R> cmulc(Cx<R> a, Cx<R> b) {
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// Double-float complex arithmetic: butterfly sums without the closing
// renormalisation, products as fused two-term dot products (mgwr_dd.cuh).
template <>
__device__ __forceinline__ Cx<dd> cadd<dd>(Cx<dd> a, Cx<dd> b) {
  return {dd_add_lazy(a.x, b.x), dd_add_lazy(a.y, b.y)};
}
template <>
__device__ __forceinline__ Cx<dd> csub<dd>(Cx<dd> a, Cx<dd> b) {
  return {dd_sub_lazy(a.x, b.x), dd_sub_lazy(a.y, b.y)};
}
template <>
__device__ __forceinline__ Cx<dd> cmul<dd>(Cx<dd> a, Cx<dd> b) {
  return {dd_dot2(a.x, b.x, -a.y, b.y), dd_dot2(a.x, b.y, a.y, b.x)};
}
template <>
__device__ __forceinline__ Cx<dd> cmulc<dd>(Cx<dd> a, Cx<dd> b) {
  return {dd_dot2(a.x, b.x, a.y, b.y), dd_dot2(a.y, b.x, -a.x, b.y)};
}

// Multiplication by powers of w8 = exp(-+2 pi i / 8) (INV: the + sign).
template <bool INV, class R>
__device__ __forceinline__ Cx<R> mul_w1(Cx<R> a) {
  const R s = R(0.70710678118654752440);
  return INV ? Cx<R>{(a.x - a.y) * s, (a.x + a.y) * s} : Cx<R>{(a.x + a.y) * s, (a.y - a.x) * s};
}
template <bool INV, class R>
__device__ __forceinline__ Cx<R> mul_w2(Cx<R> a) {
  return INV ? Cx<R>{-a.y, a.x} : Cx<R>{a.y, -a.x};
}
template <bool INV, class R>
__device__ __forceinline__ Cx<R> mul_w3(Cx<R> a) {
  const R s = R(0.70710678118654752440);
  return INV ? Cx<R>{-(a.x + a.y) * s, (a.x - a.y) * s} : Cx<R>{(a.y - a.x) * s, -(a.x + a.y) * s};
}

// Length-4 DFT, natural order in and out.
template <bool INV, class R>
__device__ __forceinline__ void dft4(Cx<R>& a0, Cx<R>& a1, Cx<R>& a2, Cx<R>& a3) {
  const Cx<R> c0 = cadd(a0, a2), d0 = csub(a0, a2);
  const Cx<R> c1 = cadd(a1, a3), d1 = mul_w2<INV>(csub(a1, a3));
  a0 = cadd(c0, c1);
  a2 = csub(c0, c1);
  a1 = cadd(d0, d1);
  a3 = csub(d0, d1);
}

template <class R>
__device__ __forceinline__ void dft2(Cx<R>& a0, Cx<R>& a1) {
  const Cx<R> s = cadd(a0, a1);
  a1 = csub(a0, a1);
  a0 = s;
}

// c + s q for a real s, one fused multiply-add per component.
__device__ __forceinline__ Cx<float> cfma(float s, Cx<float> q, Cx<float> c) {
  return {fmaf(s, q.x, c.x), fmaf(s, q.y, c.y)};
}
__device__ __forceinline__ Cx<double> cfma(double s, Cx<double> q, Cx<double> c) {
  return {fma(s, q.x, c.x), fma(s, q.y, c.y)};
}

// Odd half of a length-8 DFT from b0 = x0 - x4, t1 = x1 - x5, b2 = w2 (x2 - x6),
// t3 = x3 - x7: the length-4 DFT of (b0, w1 t1, b2, w3 t3), written to v[1],
// v[3], v[5], v[7].  With IEEE types, w1 t1 and w3 t3 are s p1 and s p3
// (s = 1/sqrt 2, p1 and p3 sums of t's components), and s is applied by the
// fused multiply-adds of the outputs: 16 operations instead of 20.
template <bool INV, class R>
__device__ __forceinline__ void dft8_odd(Cx<R> (&v)[8], Cx<R> b0, Cx<R> t1, Cx<R> b2, Cx<R> t3) {
  if constexpr (std::is_same<R, dd>::value) {
    Cx<R> b1 = mul_w1<INV>(t1), b3 = mul_w3<INV>(t3);
    dft4<INV>(b0, b1, b2, b3);
    v[1] = b0; v[3] = b1; v[5] = b2; v[7] = b3;
  } else {
    const R s = R(0.70710678118654752440);
    const Cx<R> p1 = INV ? Cx<R>{t1.x - t1.y, t1.x + t1.y} : Cx<R>{t1.x + t1.y, t1.y - t1.x};
    const Cx<R> p3 = INV ? Cx<R>{-(t3.x + t3.y), t3.x - t3.y} : Cx<R>{t3.y - t3.x, -(t3.x + t3.y)};
    const Cx<R> c0 = cadd(b0, b2), d0 = csub(b0, b2);
    const Cx<R> q = cadd(p1, p3), r = mul_w2<INV>(csub(p1, p3));
    v[1] = cfma(s, q, c0);
    v[5] = cfma(-s, q, c0);
    v[3] = cfma(s, r, d0);
    v[7] = cfma(-s, r, d0);
  }
}

// Length-8 DFT (one radix-2 layer, then two length-4 DFTs), natural order.
template <bool INV, class R>
__device__ __forceinline__ void dft8(Cx<R> (&v)[8]) {
  Cx<R> a0 = cadd(v[0], v[4]), a1 = cadd(v[1], v[5]), a2 = cadd(v[2], v[6]), a3 = cadd(v[3], v[7]);
  const Cx<R> b0 = csub(v[0], v[4]), t1 = csub(v[1], v[5]);
  const Cx<R> b2 = mul_w2<INV>(csub(v[2], v[6])), t3 = csub(v[3], v[7]);
  dft4<INV>(a0, a1, a2, a3);
  dft8_odd<INV>(v, b0, t1, b2, t3);
  v[0] = a0; v[2] = a1; v[4] = a2; v[6] = a3;
}

// Forward length-8 DFT of (v0, v1, v2, v3, 0, 0, 0, 0).
template <class R>
__device__ __forceinline__ void dft8_half_input(Cx<R> (&v)[8]) {
  Cx<R> a0 = v[0], a1 = v[1], a2 = v[2], a3 = v[3];
  const Cx<R> b0 = v[0], t1 = v[1], b2 = mul_w2<false>(v[2]), t3 = v[3];
  dft4<false>(a0, a1, a2, a3);
  dft8_odd<false>(v, b0, t1, b2, t3);
  v[0] = a0; v[2] = a1; v[4] = a2; v[6] = a3;
}

// Shared-memory index of transform position x.  16-byte elements: one pad
// slot per 8 values.  8-byte elements: no padding; bits 4..9 of x are folded
// into its bits 0..3 by an XOR (a bijection on every aligned block of 16), so
// the three access patterns of the stages below (consecutive positions, the
// span-s butterflies of the middle stages, 8 consecutive values per thread)
// each put the 16 lanes of a half-warp on 16 different bank pairs.
template <class R>
struct Pad {
  static constexpr bool wide = sizeof(Cx<R>) >= 16;
  static __device__ __forceinline__ int idx(int x) {
    if constexpr (wide) return x + (x >> 3);
    return x ^ (((x >> 3) & 14) ^ ((x >> 6) & 15));
  }
  static __host__ __device__ __forceinline__ int len(int L) { return wide ? L + (L >> 3) : L; }
};

// Last-stage butterflies on the 8 contiguous values a thread owns.
template <bool INV, class R>
__device__ __forceinline__ void last_stage(Cx<R> (&v)[8], int rlast) {
  if (rlast == 8) {
    dft8<INV>(v);
  } else if (rlast == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
    dft4<INV>(v[4], v[5], v[6], v[7]);
  } else {
    dft2(v[0], v[1]);
    dft2(v[2], v[3]);
    dft2(v[4], v[5]);
    dft2(v[6], v[7]);
  }
}

// Stage plan of a length-L = 2^logL transform: radix-8 stages 0 .. s8-1 and,
// when logL is not a multiple of 3, a last stage of radix 2^(logL mod 3).
// Stage 0 reads global memory; "middle" stages 1 .. kmid_end-1 run through
// shared memory; the last stage (span 1) is done on 8 contiguous values.
struct FftShape {  // run-time length
  static constexpr bool kFixed = false;
  int L, logL, L8, rlast, kmid_end;
  __device__ __forceinline__ explicit FftShape(int logL_) : L(1 << logL_), logL(logL_) {
    L8 = L >> 3;
    const int rem = logL % 3;
    rlast = rem == 0 ? 8 : (1 << rem);
    const int s8 = logL / 3;
    kmid_end = rem == 0 ? s8 - 1 : s8;
  }
};

template <int LOGL>
struct FixedShape {  // compile-time length: every index below folds to a constant offset
  static constexpr bool kFixed = true;
  static constexpr int logL = LOGL, L = 1 << LOGL, L8 = L >> 3;
  static constexpr int rlast = LOGL % 3 == 0 ? 8 : (1 << (LOGL % 3));
  static constexpr int kmid_end = LOGL % 3 == 0 ? LOGL / 3 - 1 : LOGL / 3;
  __device__ __forceinline__ explicit FixedShape(int) {}
};

// v[q] *= w^(j q) (CONJ: by the conjugate), q = 1..7, w = exp(-2 pi i / L),
// jstride = j L / S for a sub-transform of length S.  FP32 forms the seven
// powers from w, w^2, w^4 (three table loads, four products; error a few
// ulps); the wider types load each twiddle right before its product, which
// keeps fewer values live.
template <bool CONJ, class R>
__device__ __forceinline__ void twiddle_mul(Cx<R> (&v)[8], const Cx<R>* __restrict__ tw,
                                            int jstride) {
  if constexpr (sizeof(R) == 4) {
    Cx<R> w[8];
    w[1] = tw[jstride];
    w[2] = tw[2 * jstride];
    w[4] = tw[4 * jstride];
    w[3] = cmul(w[1], w[2]);
    w[5] = cmul(w[1], w[4]);
    w[6] = cmul(w[2], w[4]);
    w[7] = cmul(w[3], w[4]);
#pragma unroll
    for (int q = 1; q < 8; ++q) v[q] = CONJ ? cmulc(v[q], w[q]) : cmul(v[q], w[q]);
  } else {
#pragma unroll
    for (int q = 1; q < 8; ++q)
      v[q] = CONJ ? cmulc(v[q], tw[jstride * q]) : cmul(v[q], tw[jstride * q]);
  }
}

// Barrier of the thread group that owns one line pair: the warp barrier when
// the group fits in a warp, a named barrier (id 1 + group index) when several
// groups of whole warps share the CTA, the CTA barrier when the group is the
// CTA.  All three order the group's shared-memory accesses.
struct GroupSync {
  int kind;  // 0: CTA, 1: warp, 2: named
  int id, nthreads;
  __device__ __forceinline__ GroupSync(int group_threads, int block_threads, int group) {
    if (group_threads >= block_threads) {
      kind = 0;
    } else if (group_threads <= 32) {
      kind = 1;
    } else {
      kind = 2;
    }
    id = 1 + group;
    nthreads = group_threads;
  }
  __device__ __forceinline__ void operator()() const {
    if (kind == 0) {
      __syncthreads();
    } else if (kind == 1) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
  }
};

// Radix-8 middle stage k (span L >> 3(k+1)) of butterfly b, forward or inverse,
// in shared memory.
template <bool INV, class R, class SH>
__device__ __forceinline__ void middle_stage(Cx<R>* buf, int b, const SH& sh, int k,
                                             const Cx<R>* __restrict__ tw) {
  using P = Pad<R>;
  const int shift = 3 * (k + 1);
  const int s = sh.L >> shift;
  const int j = b & (s - 1);
  const int base = ((b - j) << 3) + j;
  Cx<R> v[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = buf[P::idx(base + q * s)];
  if (!INV) {
    dft8<false>(v);
    twiddle_mul<false>(v, tw, j << (3 * k));
  } else {
    twiddle_mul<true>(v, tw, j << (3 * k));
    dft8<true>(v);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) buf[P::idx(base + q * s)] = v[q];
}

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// Forward transform of one line pair by a group of T = L/(8E) threads: thread
// t does the radix-8 butterflies b = t + eT, e < E, of every stage.  `load(m)`
// returns the pair's input at time index m (called for m = b + q L/8, q < 4:
// the upper half of the line is zero padding; with FULL, q < 8: every position
// carries data).  On return the thread holds, in v[e], the transform values at
// spectral positions 8b .. 8b+7 of its butterfly b = t + eT.  Every thread of
// the group must call this (it synchronises the group through `sync`).
// `after_input()` runs in every thread right after the group barrier that
// follows the last `load` call of the group.
template <int E, class R, class SH, class Load, bool FULL = false, class Hook = NoHook>
__device__ __forceinline__ void fft_forward(Cx<R>* buf, int t, const SH& sh,
                                            const Cx<R>* __restrict__ tw, Load load,
                                            Cx<R> (&v)[E][8], const GroupSync& sync,
                                            Hook after_input = Hook()) {
  using P = Pad<R>;
  const int T = sh.L8 / E;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int b = t + e * T;
    if constexpr (FULL) {
#pragma unroll
      for (int q = 0; q < 8; ++q) v[e][q] = load(b + q * sh.L8);
      dft8<false>(v[e]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) v[e][q] = load(b + q * sh.L8);
      dft8_half_input(v[e]);
    }
    if (sh.logL == 3) return;  // single stage: thread 0 holds positions 0..7 (E = 1)
    twiddle_mul<false>(v[e], tw, b);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[P::idx(b + q * sh.L8)] = v[e][q];
  }
  sync();
  after_input();
  if constexpr (SH::kFixed) {
#pragma unroll
    for (int k = 1; k < sh.kmid_end; ++k) {
#pragma unroll
      for (int e = 0; e < E; ++e) middle_stage<false>(buf, t + e * T, sh, k, tw);
      sync();
    }
  } else {
#pragma unroll 1
    for (int k = 1; k < sh.kmid_end; ++k) {
#pragma unroll
      for (int e = 0; e < E; ++e) middle_stage<false>(buf, t + e * T, sh, k, tw);
      sync();
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int b = t + e * T;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[e][q] = buf[P::idx(8 * b + q)];
    last_stage<false>(v[e], sh.rlast);
  }
}

// Inverse transform starting from the spectral values in v (v[e] at positions
// 8b..8b+7, b = t + eT, already multiplied).  `store(m, value)` receives the
// outputs for m < L/2.
template <int E, class R, class SH, class Store>
__device__ __forceinline__ void fft_inverse(Cx<R>* buf, int t, const SH& sh,
                                            const Cx<R>* __restrict__ tw, Cx<R> (&v)[E][8],
                                            Store store, const GroupSync& sync) {
  using P = Pad<R>;
  const int T = sh.L8 / E;
  if (sh.logL == 3) {
    dft8<true>(v[0]);
#pragma unroll
    for (int q = 0; q < 4; ++q) store(q, v[0][q]);
    return;
  }
  // each thread rewrites only the 8E positions it read in fft_forward
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int b = t + e * T;
    last_stage<true>(v[e], sh.rlast);
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[P::idx(8 * b + q)] = v[e][q];
  }
  sync();
  if constexpr (SH::kFixed) {
#pragma unroll
    for (int k = sh.kmid_end - 1; k >= 1; --k) {
#pragma unroll
      for (int e = 0; e < E; ++e) middle_stage<true>(buf, t + e * T, sh, k, tw);
      sync();
    }
  } else {
#pragma unroll 1
    for (int k = sh.kmid_end - 1; k >= 1; --k) {
#pragma unroll
      for (int e = 0; e < E; ++e) middle_stage<true>(buf, t + e * T, sh, k, tw);
      sync();
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int b = t + e * T;
    Cx<R> w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) w[q] = buf[P::idx(b + q * sh.L8)];
    twiddle_mul<true>(w, tw, b);
    dft8<true>(w);
#pragma unroll
    for (int q = 0; q < 4; ++q) store(b + q * sh.L8, w[q]);
  }
}

}  // namespace mgwr

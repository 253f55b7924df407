// Register-pass FFT engine for FP32 causal time-line convolutions (Sec. 5).
//
// The same circulant embedding as mgwr_fft.cuh (two real lines packed as one
// complex line of length L = 2M, zero upper half, spectrum product, first M
// outputs of the inverse), organised for fewer instructions per value: each
// pass of the decimation-in-frequency transform is one radix-R DFT of R <= 32
// values held in registers (two to four passes instead of four or five
// radix-8 stages), so every value crosses shared memory once per pass and the
// inter-pass twiddles are applied only at pass boundaries.  The last pass
// holds R contiguous positions per butterfly: the spectrum product and the
// first inverse pass follow in registers.  Shared memory is padded by one slot
// per R_last values, which makes every access of every pass conflict-free for
// 8-byte elements (and its address a base plus an immediate offset).
//
// Plan (R0, R1[, R2[, R3]]): pass p has radix R_p, stride S_p = G_p / R_p on groups of
// G_p = L / (R_0 .. R_{p-1}) positions; butterfly j < S_p of a group reads
// positions j + q S_p, applies the DFT and, except in the last pass, the
// twiddles w_{G_p}^{j k}, and writes output k to j + k S_p.  Position
// p = sum_i d_i L / (R_0 .. R_i) then holds frequency k = sum_i d_i R_0 .. R_{i-1}
// (spectra are stored in that order: rp_position).
#pragma once

#include "mgwr_fft.cuh"

namespace mgwr {
namespace rp {

using C = Cx<float>;

// cos(2 pi e / N) and sin(2 pi e / N) at compile time: the angle is reduced to
// [-pi, pi] and the power series summed in double (|x| <= pi: 30 terms leave
// a truncation far below double rounding).
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double series_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
constexpr double series_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double reduced_angle(int e, int N) {
  const int r = ((e % N) + N) % N;
  return kTwoPi * (double)(2 * r > N ? r - N : r) / (double)N;
}
constexpr double root_cos(int e, int N) { return series_cos(reduced_angle(e, N)); }
constexpr double root_sin(int e, int N) { return series_sin(reduced_angle(e, N)); }

// a * w_N^E with w_N = exp(-2 pi i / N) (INV: exp(+2 pi i / N)); E, N compile-time.
// Multiples of N/8 use the exact forms of mgwr_fft.cuh.
template <int N, int E, bool INV>
__device__ __forceinline__ C rot(C a) {
  constexpr int e = ((E % N) + N) % N;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (2 * e == N) {
    return C{-a.x, -a.y};
  } else if constexpr (4 * e == N) {
    return mul_w2<INV>(a);
  } else if constexpr (4 * e == 3 * N) {
    return mul_w2<!INV>(a);
  } else if constexpr (8 * e == N) {
    return mul_w1<INV>(a);
  } else if constexpr (8 * e == 3 * N) {
    return mul_w3<INV>(a);
  } else if constexpr (8 * e == 5 * N) {
    const C b = mul_w1<INV>(a);
    return C{-b.x, -b.y};
  } else if constexpr (8 * e == 7 * N) {
    const C b = mul_w3<INV>(a);
    return C{-b.x, -b.y};
  } else {
    constexpr float c = (float)root_cos(e, N);
    constexpr float s = (float)root_sin(e, N);
    // forward root c - i s, inverse c + i s
    return INV ? C{fmaf(a.x, c, -a.y * s), fmaf(a.y, c, a.x * s)}
               : C{fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s)};
  }
}

// In-place length-R DFT, natural order in and out (INV: conjugate roots, no
// scaling).  R = A * B with n = n1 B + n2, k = k1 + A k2:
//   X[k1 + A k2] = sum_n2 w_B^{n2 k2} w_R^{n2 k1} sum_n1 x[n1 B + n2] w_A^{n1 k1}.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  static __device__ __forceinline__ void run(C (&v)[2]) { dft2(v[0], v[1]); }
};
template <bool INV>
struct Dft<4, INV> {
  static __device__ __forceinline__ void run(C (&v)[4]) { dft4<INV>(v[0], v[1], v[2], v[3]); }
};
template <bool INV>
struct Dft<8, INV> {
  static __device__ __forceinline__ void run(C (&v)[8]) { dft8<INV>(v); }
};

template <int A, int B, bool INV>
__device__ __forceinline__ void dft_ab(C (&v)[A * B]) {
  constexpr int R = A * B;
  C y[B][A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
    C a[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) a[n1] = v[n1 * B + n2];
    Dft<A, INV>::run(a);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) y[n2][k1] = a[k1];
  }
  // twiddles w_R^{n2 k1} (compile-time exponents)
#define MGWR_RP_TW(N2, K1) \
  if constexpr ((N2) < B && (K1) < A) y[N2][K1] = rot<R, (N2) * (K1), INV>(y[N2][K1]);
#define MGWR_RP_TW_ROW(N2) \
  MGWR_RP_TW(N2, 1) MGWR_RP_TW(N2, 2) MGWR_RP_TW(N2, 3) MGWR_RP_TW(N2, 4) MGWR_RP_TW(N2, 5) \
  MGWR_RP_TW(N2, 6) MGWR_RP_TW(N2, 7)
  MGWR_RP_TW_ROW(1) MGWR_RP_TW_ROW(2) MGWR_RP_TW_ROW(3) MGWR_RP_TW_ROW(4)
  MGWR_RP_TW_ROW(5) MGWR_RP_TW_ROW(6) MGWR_RP_TW_ROW(7)
#undef MGWR_RP_TW_ROW
#undef MGWR_RP_TW
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    C b[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) b[n2] = y[n2][k1];
    Dft<B, INV>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = b[k2];
  }
}

template <bool INV>
struct Dft<16, INV> {
  static __device__ __forceinline__ void run(C (&v)[16]) { dft_ab<4, 4, INV>(v); }
};
template <bool INV>
struct Dft<32, INV> {
  static __device__ __forceinline__ void run(C (&v)[32]) { dft_ab<4, 8, INV>(v); }
};

// Forward DFT of (v[0], .., v[R/2 - 1], 0, .., 0): the first pass, whose upper
// half is the zero padding.  Even outputs are the length-R/2 DFT of the input,
// odd outputs that of the input times w_R^n.
template <int R>
__device__ __forceinline__ void dft_half(C (&v)[R]) {
  if constexpr (R == 8) {
    dft8_half_input(v);
  } else if constexpr (R == 2) {
    v[1] = v[0];
  } else {
    constexpr int H = R / 2;
    C e[H], o[H];
#pragma unroll
    for (int q = 0; q < H; ++q) e[q] = v[q];
    o[0] = v[0];
#define MGWR_RP_HT(Q) \
  if constexpr ((Q) < H) o[Q] = rot<R, (Q), false>(v[Q]);
    MGWR_RP_HT(1) MGWR_RP_HT(2) MGWR_RP_HT(3) MGWR_RP_HT(4) MGWR_RP_HT(5) MGWR_RP_HT(6)
    MGWR_RP_HT(7) MGWR_RP_HT(8) MGWR_RP_HT(9) MGWR_RP_HT(10) MGWR_RP_HT(11) MGWR_RP_HT(12)
    MGWR_RP_HT(13) MGWR_RP_HT(14) MGWR_RP_HT(15)
#undef MGWR_RP_HT
    Dft<H, false>::run(e);
    Dft<H, false>::run(o);
#pragma unroll
    for (int q = 0; q < H; ++q) {
      v[2 * q] = e[q];
      v[2 * q + 1] = o[q];
    }
  }
}

// The table values w^{b e1} (b = 1, 2, 4 and RA, 2 RA) from which twiddle_apply
// forms the twiddles of a radix-R butterfly: loaded ahead of the butterfly's
// data so that their latency overlaps the data loads and the DFT.
template <int R>
struct TwBase {
  static constexpr int RA = R > 8 ? 8 : R;
  static constexpr int RB = R / RA;
  // rows of a table of the bases (b = 1, 2, 4, RA, 2 RA, those present)
  static constexpr int I_H1 = 1 + (RA >= 4) + (RA >= 8);
  static constexpr int NB = I_H1 + (RB >= 2) + (RB >= 4);
  static constexpr int exponent(int i) {
    return i < I_H1 ? (1 << i) : (i == I_H1 ? RA : 2 * RA);
  }
  C a1, a2, a4, h1, h2;
  __device__ __forceinline__ TwBase(const C* __restrict__ tw, int e1) {
    a1 = tw[e1];
    if constexpr (RA >= 4) a2 = tw[2 * e1];
    if constexpr (RA >= 8) a4 = tw[4 * e1];
    if constexpr (RB >= 2) h1 = tw[RA * e1];
    if constexpr (RB >= 4) h2 = tw[2 * RA * e1];
  }
  // The same values from a table whose row i holds base i for butterflies j < S.
  struct FromRows {};
  __device__ __forceinline__ TwBase(FromRows, const C* tab, int j, int S) {
    a1 = tab[j];
    if constexpr (RA >= 4) a2 = tab[S + j];
    if constexpr (RA >= 8) a4 = tab[2 * S + j];
    if constexpr (RB >= 2) h1 = tab[I_H1 * S + j];
    if constexpr (RB >= 4) h2 = tab[(I_H1 + 1) * S + j];
  }
};

// v[k] *= w_L^{k e1} (INV: conjugate), k = 1 .. R-1, from the bases of TwBase.
// With k = RA k_hi + k_lo (RA = min(R, 8)) the other powers of each factor are
// products of the bases, and w^{k e1} is the product of its two factors,
// formed right before it is used (few live registers); every twiddle is a
// product of at most four table values.
template <int R, bool INV>
__device__ __forceinline__ void twiddle_apply(C (&v)[R], const TwBase<R>& tb) {
  constexpr int RA = TwBase<R>::RA, RB = TwBase<R>::RB;
  C a[RA];
  a[1] = tb.a1;
  if constexpr (RA >= 4) {
    a[2] = tb.a2;
    a[3] = cmul(a[1], a[2]);
  }
  if constexpr (RA == 8) {
    a[4] = tb.a4;
    a[5] = cmul(a[1], a[4]);
    a[6] = cmul(a[2], a[4]);
    a[7] = cmul(a[3], a[4]);
  }
  C hb[RB > 1 ? RB : 2];
  if constexpr (RB >= 2) hb[1] = tb.h1;
  if constexpr (RB == 4) {
    hb[2] = tb.h2;
    hb[3] = cmul(hb[1], hb[2]);
  }
#pragma unroll
  for (int kh = 0; kh < RB; ++kh) {
#pragma unroll
    for (int kl = 0; kl < RA; ++kl) {
      const int k = kh * RA + kl;
      if (k == 0) continue;
      const C w = kh == 0 ? a[kl] : (kl == 0 ? hb[kh] : cmul(a[kl], hb[kh]));
      v[k] = INV ? cmulc(v[k], w) : cmul(v[k], w);
    }
  }
}

// Compile-time plan of a length-2^LOGL transform with radices R0, R1 and, when
// not 0, R2 and R3; T threads per line pair.  Four-pass plans keep every radix
// at most 16, so that a thread needs fewer registers and three blocks fit an
// SM (MIN_BLOCKS), for one more pass through shared memory.
template <int LOGL, int R0, int R1, int R2, int R3, int T>
struct Plan {
  static constexpr int L = 1 << LOGL;
  static constexpr int NP = R3 != 0 ? 4 : R2 != 0 ? 3 : 2;
  static constexpr int RL = NP == 4 ? R3 : NP == 3 ? R2 : R1;  // radix of the last pass
  static constexpr int LOG_RL = RL == 32 ? 5 : RL == 16 ? 4 : RL == 8 ? 3 : RL == 4 ? 2 : 1;
  static constexpr int S0 = L / R0;             // pass 0: one group of L
  static constexpr int G1 = S0, S1 = G1 / R1;   // pass 1
  static constexpr int G2 = S1, S2 = G2 / (R2 != 0 ? R2 : 1);  // pass 2
  static constexpr int SMEM = L + L / RL;       // padded complex slots per line pair
  static constexpr int MIN_BLOCKS = NP == 4 ? 3 : 2;
  static_assert(R0 * R1 * (R2 != 0 ? R2 : 1) * (R3 != 0 ? R3 : 1) == L,
                "radices must multiply to L");
  static_assert((L / R0) % T == 0 && (L / R1) % T == 0 && (L / RL) % T == 0 &&
                    (L / (R2 != 0 ? R2 : 1)) % T == 0,
                "every pass must give each thread the same number of butterflies");
  static __device__ __forceinline__ int idx(int p) { return p + (p >> LOG_RL); }
};

// Where a convolution takes its twiddle bases and spectrum from.  Global
// tables (tw[e] = w_L^e; spectrum in the plan's spectral order) are read
// through the caches by every butterfly.
struct GlobalTables {
  const C* __restrict__ tw;
  const C* __restrict__ spec;
  // bases of butterfly j of twiddled pass PASS (exponent stride TWS)
  template <int PASS, int R, int TWS>
  __device__ __forceinline__ TwBase<R> base(int j) const {
    return TwBase<R>(tw, j * TWS);
  }
  // spectrum values 2q, 2q + 1 of last-pass butterfly beta (RL values each)
  template <int RL>
  __device__ __forceinline__ float4 spec2(int beta, int q) const {
    return __ldg(reinterpret_cast<const float4*>(spec + (size_t)beta * RL) + q);
  }
};

// The same values copied into shared memory once per block, for kernels whose
// blocks stay resident and convolve many line pairs.  Twiddled pass p (all but
// the last) has a table of TwBase<R_p>::NB rows of S_p values, row i holding
// w_L^{b_i TWS_p j} for its butterflies j < S_p (b_i the exponents of the
// bases); the spectrum is kept per last-pass butterfly, RL values followed by
// one unused 16-byte slot, so that the 16-byte reads of a warp's 32
// butterflies fall on distinct banks in every wavefront.
template <int LOGL, int R0, int R1, int R2, int R3>
struct SharedTables {
  static constexpr int L = 1 << LOGL;
  static constexpr int NP = R3 != 0 ? 4 : R2 != 0 ? 3 : 2;
  static constexpr int RL = NP == 4 ? R3 : NP == 3 ? R2 : R1;
  // butterflies per group and exponent strides of the twiddled passes
  static constexpr int S0 = L / R0, TWS0 = 1;
  static constexpr int S1 = NP >= 3 ? L / (R0 * R1) : 0, TWS1 = R0;
  static constexpr int S2 = NP == 4 ? L / (R0 * R1 * R2) : 0, TWS2 = R0 * R1;
  static constexpr int N0 = TwBase<R0>::NB * S0;
  static constexpr int N1 = NP >= 3 ? TwBase<R1>::NB * S1 : 0;
  static constexpr int N2 = NP == 4 ? TwBase<R2 != 0 ? R2 : 2>::NB * S2 : 0;
  static constexpr int SPEC_ROW = RL / 2 + 1;             // float4 slots per butterfly
  static constexpr int SPEC_F4 = (L / RL) * SPEC_ROW;
  // bytes: spectrum (16-byte slots) first, then the twiddle rows
  static constexpr size_t BYTES = (size_t)SPEC_F4 * 16 + (size_t)(N0 + N1 + N2) * sizeof(C);

  const float4* sp;
  const C* t0;
  const C* t1;
  const C* t2;

  __device__ __forceinline__ explicit SharedTables(unsigned char* mem) {
    sp = reinterpret_cast<const float4*>(mem);
    t0 = reinterpret_cast<const C*>(mem + (size_t)SPEC_F4 * 16);
    t1 = t0 + N0;
    t2 = t1 + N1;
  }

  template <int R, int S, int TWS>
  static __device__ __forceinline__ void fill_rows(C* dst, const C* __restrict__ tw, int tid,
                                                   int nthr) {
    for (int x = tid; x < TwBase<R>::NB * S; x += nthr) {
      const int i = x / S, j = x - i * S;
      dst[x] = tw[TwBase<R>::exponent(i) * TWS * j];
    }
  }
  // Copies the tables from global memory (all threads of the block; the
  // caller synchronises the block before the first use).
  static __device__ __forceinline__ void fill(unsigned char* mem, const C* __restrict__ tw,
                                              const C* __restrict__ spec, int tid, int nthr) {
    float4* sd = reinterpret_cast<float4*>(mem);
    const float4* ss = reinterpret_cast<const float4*>(spec);
    for (int x = tid; x < (L / RL) * (RL / 2); x += nthr) {
      const int beta = x / (RL / 2), q = x - beta * (RL / 2);
      sd[beta * SPEC_ROW + q] = __ldg(ss + x);
    }
    C* d0 = reinterpret_cast<C*>(mem + (size_t)SPEC_F4 * 16);
    fill_rows<R0, S0, TWS0>(d0, tw, tid, nthr);
    if constexpr (NP >= 3) fill_rows<R1, S1, TWS1>(d0 + N0, tw, tid, nthr);
    if constexpr (NP == 4) fill_rows<R2, S2, TWS2>(d0 + N0 + N1, tw, tid, nthr);
  }

  template <int PASS, int R, int TWS>
  __device__ __forceinline__ TwBase<R> base(int j) const {
    using FR = typename TwBase<R>::FromRows;
    if constexpr (PASS == 0) return TwBase<R>(FR{}, t0, j, S0);
    else if constexpr (PASS == 1) return TwBase<R>(FR{}, t1, j, S1);
    else return TwBase<R>(FR{}, t2, j, S2);
  }
  template <int RL_>
  __device__ __forceinline__ float4 spec2(int beta, int q) const {
    return sp[beta * SPEC_ROW + q];
  }
};

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

// A middle pass (neither the first nor the last): radix R butterflies on
// groups of G positions with stride S, twiddles w_G^{jk} = w_L^{j k TWS}
// (TWS = L / G) after the forward DFT, before the inverse one; then the
// group's barrier.
template <class P, int PASS, int R, int G, int S, int TWS, bool INV, int T, int PAIRS, class Tab>
__device__ __forceinline__ void mid_pass(C* buf, int t, int g, const Tab& tab) {
  constexpr int NB = (P::L / R) / T;
#pragma unroll 1
  for (int i = 0; i < NB; ++i) {
    const int beta = t + T * i;
    const int grp = beta / S, j = beta - grp * S;
    const int base = grp * G + j;
    const TwBase<R> tb = tab.template base<PASS, R, TWS>(j);
    C v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = buf[P::idx(base + q * S)];
    if constexpr (INV) {
      twiddle_apply<R, true>(v, tb);
      Dft<R, true>::run(v);
    } else {
      Dft<R, false>::run(v);
      twiddle_apply<R, false>(v, tb);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) buf[P::idx(base + q * S)] = v[q];
  }
  group_sync<T, PAIRS>(g);
}

// The forward middle passes of plan P (pass 1 of three- and four-pass plans,
// pass 2 of four-pass ones), and their inverses in reverse order.
template <class P, int R0, int R1, int R2, int T, int PAIRS, class Tab>
__device__ __forceinline__ void mid_passes_forward(C* buf, int t, int g, const Tab& tab) {
  if constexpr (P::NP >= 3) mid_pass<P, 1, R1, P::G1, P::S1, R0, false, T, PAIRS>(buf, t, g, tab);
  if constexpr (P::NP == 4)
    mid_pass<P, 2, R2, P::G2, P::S2, R0 * R1, false, T, PAIRS>(buf, t, g, tab);
}
template <class P, int R0, int R1, int R2, int T, int PAIRS, class Tab>
__device__ __forceinline__ void mid_passes_inverse(C* buf, int t, int g, const Tab& tab) {
  if constexpr (P::NP == 4)
    mid_pass<P, 2, R2, P::G2, P::S2, R0 * R1, true, T, PAIRS>(buf, t, g, tab);
  if constexpr (P::NP >= 3) mid_pass<P, 1, R1, P::G1, P::S1, R0, true, T, PAIRS>(buf, t, g, tab);
}

// One line pair's causal convolution by the T threads t of group g: the first
// M = L/2 values of IFFT(FFT(x) * spec), x zero-padded to L.  load(m) gives
// the pair's input at time m < M (both lines as one complex value; every call
// of the thread is made before its first DFT, so the loads overlap);
// store(m, y) receives output m < M.  tab: the twiddle bases and the kernel's
// spectrum (in this plan's spectral order, pre-scaled by 1/L; GlobalTables or
// SharedTables).  buf: P::SMEM complex values of shared memory for the group.
template <int LOGL, int R0, int R1, int R2, int R3, int T, int PAIRS, class Tab, class Load,
          class Store>
__device__ __forceinline__ void convolve(C* buf, int t, int g, const Tab& tab, Load load,
                                         Store store) {
  using P = Plan<LOGL, R0, R1, R2, R3, T>;
  // ---- pass 0: every input of the thread, then half-input DFTs and twiddles
  constexpr int NB0 = P::S0 / T;
  C in[NB0][R0 / 2];
#pragma unroll
  for (int i = 0; i < NB0; ++i) {
#pragma unroll
    for (int q = 0; q < R0 / 2; ++q) in[i][q] = load(t + T * i + q * P::S0);
  }
#pragma unroll
  for (int i = 0; i < NB0; ++i) {
    const int j = t + T * i;
    const TwBase<R0> tb = tab.template base<0, R0, 1>(j);
    C v[R0];
#pragma unroll
    for (int q = 0; q < R0 / 2; ++q) v[q] = in[i][q];
    dft_half<R0>(v);
    twiddle_apply<R0, false>(v, tb);
#pragma unroll
    for (int k = 0; k < R0; ++k) buf[P::idx(j + k * P::S0)] = v[k];
  }
  group_sync<T, PAIRS>(g);

  // ---- the middle passes: radix R1 (and R2) on groups of G1 (G2), twiddles w_G^{jk}
  mid_passes_forward<P, R0, R1, R2, T, PAIRS>(buf, t, g, tab);

  // ---- last pass (contiguous RL values), spectrum product, its inverse
  constexpr int RL = P::RL;
  constexpr int NBL = (P::L / RL) / T;
#pragma unroll 1
  for (int i = 0; i < NBL; ++i) {
    const int base = (t + T * i) * RL;
    C v[RL];
#pragma unroll
    for (int q = 0; q < RL; ++q) v[q] = buf[P::idx(base + q)];
    Dft<RL, false>::run(v);
#pragma unroll
    for (int q = 0; q < RL / 2; ++q) {
      const float4 s2 = tab.template spec2<RL>(t + T * i, q);
      v[2 * q] = cmul(v[2 * q], C{s2.x, s2.y});
      v[2 * q + 1] = cmul(v[2 * q + 1], C{s2.z, s2.w});
    }
    Dft<RL, true>::run(v);
#pragma unroll
    for (int q = 0; q < RL; ++q) buf[P::idx(base + q)] = v[q];
  }
  group_sync<T, PAIRS>(g);

  // ---- inverses of the middle passes
  mid_passes_inverse<P, R0, R1, R2, T, PAIRS>(buf, t, g, tab);

  // ---- inverse of pass 0: the first M outputs
#pragma unroll 1
  for (int i = 0; i < NB0; ++i) {
    const int j = t + T * i;
    const TwBase<R0> tb = tab.template base<0, R0, 1>(j);
    C v[R0];
#pragma unroll
    for (int k = 0; k < R0; ++k) v[k] = buf[P::idx(j + k * P::S0)];
    twiddle_apply<R0, true>(v, tb);
    Dft<R0, true>::run(v);
#pragma unroll
    for (int q = 0; q < R0 / 2; ++q) store(j + q * P::S0, v[q]);
  }
}

// Two consecutive complex inputs of the first pass (times m and m + 1).
struct Pair2 {
  C a, b;
};

// The same convolution with the first pass's butterflies taken two adjacent at
// a time (j = 2 (t + T i) and j + 1), so that the inputs and outputs of a
// thread come as pairs of consecutive times: load2(m) gives the inputs at m and
// m + 1 (Pair2), store_all(j, y) receives the outputs of the butterflies j and
// j + 1, y[h][q] at time j + h + q L / R0 (q < R0 / 2); the global accesses are
// then 8-byte vectors (half the load and store instructions), for 2-way bank
// conflicts on the first pass's shared-memory accesses.  tab: the twiddle
// bases and the kernel's spectrum (in this plan's spectral order, pre-scaled
// by 1/L).  buf: P::SMEM complex values of shared memory for the group.
template <int LOGL, int R0, int R1, int R2, int R3, int T, int PAIRS, class Tab, class Load2,
          class StoreAll>
__device__ __forceinline__ void convolve2(C* buf, int t, int g, const Tab& tab, Load2 load2,
                                          StoreAll store_all) {
  using P = Plan<LOGL, R0, R1, R2, R3, T>;
  // ---- pass 0: every input of the thread, then half-input DFTs and twiddles
  constexpr int NB0 = P::S0 / T;
  static_assert(NB0 % 2 == 0, "the first pass takes butterflies in adjacent pairs");
  Pair2 in[NB0 / 2][R0 / 2];
#pragma unroll
  for (int i = 0; i < NB0 / 2; ++i) {
#pragma unroll
    for (int q = 0; q < R0 / 2; ++q) in[i][q] = load2(2 * (t + T * i) + q * P::S0);
  }
#pragma unroll
  for (int i = 0; i < NB0; ++i) {
    const int j = 2 * (t + T * (i >> 1)) + (i & 1);
    const TwBase<R0> tb = tab.template base<0, R0, 1>(j);
    C v[R0];
#pragma unroll
    for (int q = 0; q < R0 / 2; ++q) v[q] = (i & 1) ? in[i >> 1][q].b : in[i >> 1][q].a;
    dft_half<R0>(v);
    twiddle_apply<R0, false>(v, tb);
#pragma unroll
    for (int k = 0; k < R0; ++k) buf[P::idx(j + k * P::S0)] = v[k];
  }
  group_sync<T, PAIRS>(g);

  // ---- the middle passes: radix R1 (and R2) on groups of G1 (G2), twiddles w_G^{jk}
  mid_passes_forward<P, R0, R1, R2, T, PAIRS>(buf, t, g, tab);

  // ---- last pass (contiguous RL values), spectrum product, its inverse
  constexpr int RL = P::RL;
  constexpr int NBL = (P::L / RL) / T;
#pragma unroll 1
  for (int i = 0; i < NBL; ++i) {
    const int base = (t + T * i) * RL;
    C v[RL];
#pragma unroll
    for (int q = 0; q < RL; ++q) v[q] = buf[P::idx(base + q)];
    Dft<RL, false>::run(v);
#pragma unroll
    for (int q = 0; q < RL / 2; ++q) {
      const float4 s2 = tab.template spec2<RL>(t + T * i, q);
      v[2 * q] = cmul(v[2 * q], C{s2.x, s2.y});
      v[2 * q + 1] = cmul(v[2 * q + 1], C{s2.z, s2.w});
    }
    Dft<RL, true>::run(v);
#pragma unroll
    for (int q = 0; q < RL; ++q) buf[P::idx(base + q)] = v[q];
  }
  group_sync<T, PAIRS>(g);

  // ---- inverses of the middle passes
  mid_passes_inverse<P, R0, R1, R2, T, PAIRS>(buf, t, g, tab);

  // ---- inverse of pass 0: the first M outputs, two adjacent butterflies at a time
#pragma unroll 1
  for (int i = 0; i < NB0 / 2; ++i) {
    const int j = 2 * (t + T * i);
    C y[2][R0 / 2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const TwBase<R0> tb = tab.template base<0, R0, 1>(j + h);
      C v[R0];
#pragma unroll
      for (int k = 0; k < R0; ++k) v[k] = buf[P::idx(j + h + k * P::S0)];
      twiddle_apply<R0, true>(v, tb);
      Dft<R0, true>::run(v);
#pragma unroll
      for (int q = 0; q < R0 / 2; ++q) y[h][q] = v[q];
    }
    store_all(j, y);
  }
}

}  // namespace rp

// Radix plans per transform length (L = 2^7 .. 2^13): two to four passes,
// (LOGL, R0, R1, R2, R3, T), T threads per line pair, 256 threads per block.
// The sweeps take two or three passes, the last of radix 32.  The carried
// outer defect (launch_defect_update_rp), whose store phase is heavier, takes
// four passes of radix <= 16 at L = 8192 (80 registers: three blocks per SM
// instead of two; 12.8 against 17.2 ms on 2-D 511 x 511, M = 4096, where the
// sweep measured 4.1 against 3.2 ms per half-sweep).
#define MGWR_RP_PLANS(X)        \
  X(13, 16, 16, 32, 0, 256)     \
  X(12, 8, 16, 32, 0, 128)      \
  X(11, 8, 8, 32, 0, 64)        \
  X(10, 8, 4, 32, 0, 32)        \
  X(9, 16, 32, 0, 0, 16)        \
  X(8, 8, 32, 0, 0, 8)          \
  X(7, 4, 32, 0, 0, 4)
#define MGWR_RP_DEFECT_PLANS(X) \
  X(13, 8, 8, 8, 16, 256)       \
  X(12, 8, 16, 32, 0, 128)      \
  X(11, 8, 8, 32, 0, 64)        \
  X(10, 8, 4, 32, 0, 32)        \
  X(9, 16, 32, 0, 0, 16)        \
  X(8, 8, 32, 0, 0, 8)          \
  X(7, 4, 32, 0, 0, 4)

constexpr int kRpBlock = 256;     // threads per block of the register-pass kernels
constexpr int kRpResBlock = 512;  // and of the resident sweep (one block per SM)

// Radices of the plan for length 2^logL into r[0..4) (the carried defect's
// table when `defect`); returns their count, 0 for a length without a plan.
__host__ __device__ inline int rp_plan(int logL, int* r, bool defect = false) {
#define MGWR_RP_PLAN_CASE(LG, A, B, C, D, T) \
  case LG:                                   \
    r[0] = A;                                \
    r[1] = B;                                \
    r[2] = C;                                \
    r[3] = D;                                \
    return D != 0 ? 4 : C != 0 ? 3 : 2;
  if (defect) {
    switch (logL) {
      MGWR_RP_DEFECT_PLANS(MGWR_RP_PLAN_CASE)
      default:
        return 0;
    }
  }
  switch (logL) {
    MGWR_RP_PLANS(MGWR_RP_PLAN_CASE)
    default:
      return 0;
  }
#undef MGWR_RP_PLAN_CASE
}

// Radices of the shared-memory engine of mgwr_fft.cuh for length 2^logL:
// radix-8 stages, then radix 2^(logL mod 3) when that is not 0.
__host__ __device__ inline int engine_plan(int logL, int* r) {
  int np = 0;
  for (int k = 0; k < logL / 3; ++k) r[np++] = 8;
  if (logL % 3 != 0) r[np++] = 1 << (logL % 3);
  return np;
}

// Position of frequency k in the spectral order of a DIF transform with the
// radices r[0..np) (host and device; used to permute spectra between engines).
__host__ __device__ inline int rp_position(int k, const int* r, int np) {
  int L = 1;
  for (int i = 0; i < np; ++i) L *= r[i];
  int p = 0, w = L, base = 1;
  for (int i = 0; i < np; ++i) {
    const int dgt = (k / base) % r[i];
    w /= r[i];
    p += dgt * w;
    base *= r[i];
  }
  return p;
}

}  // namespace mgwr

// Smoother half-sweep on the tensor cores (FP32 fields, lines of 64 .. 256
// steps; Sec. 3 Eq. red-black, Sec. 6 Eq. red-black_2d).
//
// For short lines the triangular Toeplitz product u_p = k * b_p (k the inverse
// column of (T_M + sigma I), b_p = f_p + h^-2 * sum of neighbour lines) is
// computed as a dense product: for a tile of 128 lines of one colour,
// U[128 x M] = B[128 x M] * Kt[M x M] with Kt[k][t] = k[t - k] (0 for t < k),
// on tcgen05.mma (kind::f16, bf16 operands, FP32 accumulator in tensor memory).
// Both operands are split into three bf16 pieces (x = x0 + x1 + x2, 24
// significant bits) and the six products of pieces whose orders add up to at
// most 2 are accumulated, so the result carries FP32 accuracy.  Per line this
// is 6 M^2 multiply-adds against the FFT engine's ~10 M log2(2M) operations on
// the SIMT pipes, which the tensor cores more than repay up to M = 256.
//
// Per CTA (17 warps): the band of Kt for the first 32 time steps (row t,
// column k: k_{t-k}), built once per instance and level at setup in the
// K-major no-swizzle layout (8 x 16-byte core matrices), arrives in shared
// memory by one bulk copy (cp.async.bulk on an mbarrier); because Kt is
// Toeplitz, the band of steps 32c .. 32c+31 is the same band shifted down by
// 32c rows, so chunk c multiplies into accumulator columns 32c .. M-1 only
// (N = M - 32c: the triangle above the diagonal is never computed).  Two
// producer groups of 8 warps gather the 128 lines' b values of alternate
// chunks, split them and write them into their own buffer in the same layout,
// then arrive on the buffer's "full" mbarrier; one warp waits for each chunk,
// issues its twelve MMAs and commits them to the buffer's "empty" mbarrier,
// which the group waits for before refilling.  No CTA-wide barrier separates
// the chunks, so one group's memory latency overlaps the other's work.  Every
// wait is bounded.  The epilogue reads the accumulator with tcgen05.ld and
// writes u (and the change record).
#include <cuda_bf16.h>

#include "mgwr_common.cuh"
#include "mgwr_tma.cuh"

namespace mgwr {

// Set when a CTA gave up waiting for its MMAs (read by take_tc_timeout).
__device__ unsigned g_tc_timeout;

namespace {

constexpr int kTileRows = 128;  // lines per CTA: the MMA's M
constexpr int kChunk = 32;      // time steps per shared-memory chunk (two K = 16 steps)
// 16 producer warps in two groups of 8 (alternate chunks), one MMA-issuing warp
constexpr int kGroupThreads = 256;
constexpr int kIssuerWarp = 2 * kGroupThreads / 32;
constexpr int kIssuer = kIssuerWarp * 32;
constexpr int kThreads = kIssuer + 32;

// Byte offset of element (r, k) in a K-major tile of kChunk columns: core
// matrices of 8 rows x 16 bytes; the kChunk / 8 core matrices of a row group
// are adjacent (128 bytes apart: the descriptor's leading byte offset), row
// groups follow each other (kChunk / 8 * 128 bytes: the stride byte offset).
__device__ __forceinline__ int core_off(int r, int kcore) {
  return (r >> 3) * (kChunk / 8) * 128 + kcore * 128 + (r & 7) * 16;
}

__device__ __forceinline__ uint64_t smem_desc(unsigned addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;                 // leading byte offset: next K core
  d |= (uint64_t)((kChunk / 8 * 128) >> 4) << 32;  // stride byte offset: next 8 rows
  d |= (uint64_t)1 << 46;                          // descriptor version (tcgen05)
  return d;                                        // base offset 0, no swizzle
}

// Instruction descriptor: FP32 accumulator, bf16 A and B, both K-major,
// N = n columns, M = 128 rows.
__host__ __device__ constexpr uint32_t mma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kTileRows >> 4) << 24);
}

// x = x0 + x1 + x2 in bf16 (each piece the rounding of what the others leave).
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b,
                                       __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Which pieces (of B and of Kt) the six products use.
__constant__ int kPieceA[6] = {0, 0, 1, 0, 1, 2};
__constant__ int kPieceB[6] = {0, 1, 0, 2, 1, 0};

}  // namespace

template <int M>
__global__ void __launch_bounds__(kThreads, 2)
    k_sweep_tc(const float* __restrict__ f, float* __restrict__ u, float* __restrict__ delta,
               const unsigned char* __restrict__ band, int d, int n, int par, float hinv2,
               int npts, int tiles_per_inst, size_t fstride, size_t bstride) {
  constexpr int kA = kTileRows * kChunk * 2;  // bytes per piece of a b-values chunk
  constexpr int kB = M * kChunk * 2;          // bytes per piece of the Kt band
  constexpr int kNumChunks = M / kChunk;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // full[b]: producer group b has written a chunk into buffer b (one arrival per
  // thread of the group); empty[b]: the MMAs reading buffer b have completed
  // (commit); done: every MMA has completed (commit); band: the band has arrived
  __shared__ __align__(8) uint64_t bars[6];
  uint64_t* const full = bars;
  uint64_t* const empty = bars + 2;
  uint64_t* const done = bars + 4;
  uint64_t* const band_bar = bars + 5;
  __shared__ unsigned tmem_slot;
  __shared__ int rowp[kTileRows];
  __shared__ unsigned rowm[kTileRows];
  unsigned char* sA = smem_raw;               // 2 buffers x 3 pieces
  unsigned char* sB = smem_raw + 6 * kA;      // 3 pieces

  const int inst = blockIdx.x / tiles_per_inst;
  const int rt = blockIdx.x - inst * tiles_per_inst;
  f += (size_t)inst * fstride;
  u += (size_t)inst * fstride;
  if (delta != nullptr) delta += (size_t)inst * fstride;
  band += (size_t)inst * bstride;
  const int warp = threadIdx.x >> 5;

  // rows of the tile: the colour's points rt*128 .. rt*128+127 and their neighbours
  if (threadIdx.x < kTileRows) {
    const int k = rt * kTileRows + threadIdx.x;
    unsigned m = 0;
    int p = 0;
    if (k < npts) {
      int i = 0, j = 0;
      p = colour_point(k, d, n, par, i, j);
      m = 16u | (i > 0 ? 1u : 0u) | (i < n - 1 ? 2u : 0u);
      if (d == 2) m |= (j > 0 ? 4u : 0u) | (j < n - 1 ? 8u : 0u);
    }
    rowp[threadIdx.x] = p;
    rowm[threadIdx.x] = m;
  }
  if (threadIdx.x == kIssuer) {
    mbar_init(&full[0], kGroupThreads);
    mbar_init(&full[1], kGroupThreads);
    mbar_init(&empty[0], 1);
    mbar_init(&empty[1], 1);
    mbar_init(done, 1);
    mbar_init(band_bar, 1);
    mbar_fence_init();
    // the three pieces of the band: 3 * kB contiguous bytes (16-byte multiples)
    mbar_arrive_expect_tx(band_bar, 3u * kB);
    bulk_copy_g2s(sB, band, 3u * kB, band_bar);
  }
  if (warp == kIssuerWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(M)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;
  const size_t nM = (size_t)n * M;
  bool ok = true;

  if (warp == kIssuerWarp) {
    // one thread issues every chunk's MMAs as soon as its buffer is full
    if (threadIdx.x == kIssuer) {
      int issued = -1;
      ok = mbar_wait_bounded(band_bar, 0u);
      const bool band_ok = ok;
      for (int ch = 0; ok && ch < kNumChunks; ++ch) {
        const int b = ch & 1;
        if (!mbar_wait_bounded(&full[b], (unsigned)((ch >> 1) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        // chunk ch reaches output steps 32 ch .. M-1: N = M - 32 ch columns from 32 ch
        const uint32_t idesc = mma_idesc(M - ch * kChunk);
        const unsigned dcol = tmem + (unsigned)(ch * kChunk);
        unsigned char* sAb = sA + b * 3 * kA;
#pragma unroll
        for (int s = 0; s < kChunk / 16; ++s) {
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            const uint64_t da = smem_desc(smem_u32(sAb + kPieceA[c] * kA) + s * 256);
            const uint64_t db = smem_desc(smem_u32(sB + kPieceB[c] * kB) + s * 256);
            mma_bf16(dcol, da, db, idesc, (ch > 0 || s > 0 || c > 0) ? 1u : 0u);
          }
        }
        mma_commit(&empty[b]);
        issued = ch;
      }
      if (ok) {
        mma_commit(done);
      } else {
        atomicOr(&g_tc_timeout, 1u);
        // the band's bulk copy may still be writing shared memory: give it one more
        // bounded wait before the CTA can end
        if (!band_ok) (void)mbar_wait_bounded(band_bar, 0u);
        // what was issued finishes before the accumulator is released
        if (issued >= 0) (void)mbar_wait_bounded(&empty[issued & 1], (unsigned)((issued >> 1) & 1));
      }
    }
    __syncwarp();
  } else {
    // producer group g (warps 8g .. 8g+7) fills buffer g with chunks g, g + 2, ...
    const int g = warp >> 3;
    const int gt = threadIdx.x - g * kGroupThreads;
    unsigned char* sAb = sA + g * 3 * kA;
    for (int ch = g, k = 0; ch < kNumChunks; ch += 2, ++k) {
      // the MMAs of this buffer's previous chunk have read it
      if (k >= 1 && !mbar_wait_bounded(&empty[g], (unsigned)((k - 1) & 1))) {
        ok = false;
        break;
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int item = gt + s * kGroupThreads;
        const int r = item >> 2, kc = item & 3;
        const int m0 = ch * kChunk + kc * 8;
        const unsigned msk = rowm[r];
        float b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = 0.f;
        if (msk & 16u) {
          const size_t pM = (size_t)rowp[r] * M + m0;
          // 8 steps of a line, 0 for a neighbour outside the grid
          auto line8 = [&](const float* src, bool present, float (&o)[8]) {
            if (present) {
              const float4 x = __ldg(reinterpret_cast<const float4*>(src));  // read-only in this kernel
              const float4 y = __ldg(reinterpret_cast<const float4*>(src + 4));
              o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
              o[4] = y.x; o[5] = y.y; o[6] = y.z; o[7] = y.w;
            } else {
#pragma unroll
              for (int q = 0; q < 8; ++q) o[q] = 0.f;
            }
          };
          // the neighbour sum in the FFT sweep's order: (west + east) + (south + north)
          float fv[8], a[8], c[8], s2[8];
          line8(u + pM - M, (msk & 1u) != 0, a);
          line8(u + pM + M, (msk & 2u) != 0, c);
#pragma unroll
          for (int q = 0; q < 8; ++q) s2[q] = a[q] + c[q];
          if (d == 2) {
            line8(u + pM - nM, (msk & 4u) != 0, a);
            line8(u + pM + nM, (msk & 8u) != 0, c);
#pragma unroll
            for (int q = 0; q < 8; ++q) s2[q] = s2[q] + (a[q] + c[q]);
          }
          line8(f + pM, true, fv);
#pragma unroll
          for (int q = 0; q < 8; ++q) b[q] = fv[q] + hinv2 * s2[q];
        }
        __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split3(b[q], p0[q], p1[q], p2[q]);
        const int off = core_off(r, kc);
        *reinterpret_cast<uint4*>(sAb + off) =
            make_uint4(pack2(p0[0], p0[1]), pack2(p0[2], p0[3]), pack2(p0[4], p0[5]), pack2(p0[6], p0[7]));
        *reinterpret_cast<uint4*>(sAb + kA + off) =
            make_uint4(pack2(p1[0], p1[1]), pack2(p1[2], p1[3]), pack2(p1[4], p1[5]), pack2(p1[6], p1[7]));
        *reinterpret_cast<uint4*>(sAb + 2 * kA + off) =
            make_uint4(pack2(p2[0], p2[1]), pack2(p2[2], p2[3]), pack2(p2[4], p2[5]), pack2(p2[6], p2[7]));
      }
      fence_proxy_async_smem();  // these stores before the MMAs' reads
      mbar_arrive(&full[g]);
    }
    // the accumulator is complete once every MMA has
    if (ok && !mbar_wait_bounded(done, 0u)) ok = false;
    if (!ok && gt == 0) atomicOr(&g_tc_timeout, 1u);
  }
  // every thread agrees on the outcome before the accumulator is read
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  tc_fence_after();

  // epilogue: warp w < 16 reads lanes 32 (w % 4) .. +31 (its rows), columns of quarter w / 4
  if (ok && warp < 2 * kGroupThreads / 32) {
    const int w = warp, lane = threadIdx.x & 31;
    const int r = 32 * (w & 3) + lane;
    const unsigned msk = rowm[r];
    float* ur = u + (size_t)rowp[r] * M;
    float* dr = delta != nullptr ? delta + (size_t)rowp[r] * M : nullptr;
#pragma unroll 1
    for (int c = (w >> 2) * (M / 4); c < (w >> 2) * (M / 4) + M / 4; c += 8) {
      unsigned v[8];
      const unsigned addr = tmem + ((unsigned)(32 * (w & 3)) << 16) + (unsigned)c;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (msk & 16u) {
        const float4 y0 = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]),
                                      __uint_as_float(v[2]), __uint_as_float(v[3]));
        const float4 y1 = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]),
                                      __uint_as_float(v[6]), __uint_as_float(v[7]));
        if (dr != nullptr) {
          const float4 o0 = *reinterpret_cast<const float4*>(ur + c);
          const float4 o1 = *reinterpret_cast<const float4*>(ur + c + 4);
          *reinterpret_cast<float4*>(dr + c) =
              make_float4(y0.x - o0.x, y0.y - o0.y, y0.z - o0.z, y0.w - o0.w);
          *reinterpret_cast<float4*>(dr + c + 4) =
              make_float4(y1.x - o1.x, y1.y - o1.y, y1.z - o1.z, y1.w - o1.w);
        }
        *reinterpret_cast<float4*>(ur + c) = y0;
        *reinterpret_cast<float4*>(ur + c + 4) = y1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kIssuerWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(M)
                 : "memory");
}

namespace {

template <int M>
cudaError_t tc_launch(const float* f, float* u, float* delta, const unsigned char* band,
                      size_t bstride, const LevelShape& ls, int par, float hinv2, cudaStream_t s) {
  const int npts = colour_count(ls.d, ls.n, par);
  if (npts == 0 || ls.batch == 0) return cudaSuccess;
  const int tiles = (npts + kTileRows - 1) / kTileRows;
  const long long grid = (long long)tiles * ls.batch;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  constexpr int kA = kTileRows * kChunk * 2, kB = M * kChunk * 2;
  // shared memory also caps the CTAs per SM so that their tensor-memory columns
  // (M each) fit the SM's 512 at once
  size_t smem = 6 * (size_t)kA + 3 * (size_t)kB;
  const size_t per_sm_cap = 512 / M;  // CTAs whose accumulators fit together
  const size_t min_smem = (228 * 1024) / (per_sm_cap + 1) + 1;
  if (smem < min_smem) smem = min_smem;
  auto kern = k_sweep_tc<M>;
  cudaError_t e = prepare_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, kThreads, smem, s>>>(f, u, delta, band, ls.d, ls.n, par, hinv2, npts,
                                              tiles, ls.field_stride(), bstride);
  return cudaSuccess;
}

// The Kt band of every (instance, level) line of inverse columns: line l,
// piece q, row t, column k (k < 32) holds piece q of k_{t-k} (0 for t < k), at
// byte l * 3 * 64 M + q * 64 M + core_off(t, k / 8) + 2 (k % 8).
__global__ void k_band_bf16x3(const double* __restrict__ kcol, unsigned char* __restrict__ band,
                              int M, size_t lines) {
  const size_t per_line = (size_t)M * kChunk;
  const size_t total = lines * per_line;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t line = i / per_line;
    const int rest = (int)(i - line * per_line);
    const int t = rest / kChunk, k = rest - t * kChunk;
    const double x = t >= k ? kcol[line * M + (t - k)] : 0.0;
    const __nv_bfloat16 a = __double2bfloat16(x);
    const double r1 = x - (double)__bfloat162float(a);
    const __nv_bfloat16 b = __double2bfloat16(r1);
    const __nv_bfloat16 c = __double2bfloat16(r1 - (double)__bfloat162float(b));
    unsigned char* o = band + line * 3 * (size_t)(2 * per_line) + core_off(t, k >> 3) + 2 * (k & 7);
    *reinterpret_cast<__nv_bfloat16*>(o) = a;
    *reinterpret_cast<__nv_bfloat16*>(o + 2 * per_line) = b;
    *reinterpret_cast<__nv_bfloat16*>(o + 4 * per_line) = c;
  }
}

}  // namespace

cudaError_t launch_sweep_tc(const float* f, float* u, float* delta, const unsigned char* band,
                            size_t bstride, const LevelShape& ls, int par, float hinv2,
                            cudaStream_t s) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (ls.M) {
    case 64: e = tc_launch<64>(f, u, delta, band, bstride, ls, par, hinv2, s); break;
    case 128: e = tc_launch<128>(f, u, delta, band, bstride, ls, par, hinv2, s); break;
    case 256: e = tc_launch<256>(f, u, delta, band, bstride, ls, par, hinv2, s); break;
    default: break;
  }
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

size_t tc_band_bytes(int M) { return 3 * (size_t)M * kChunk * 2; }

cudaError_t launch_band_bf16x3(const double* kcol, unsigned char* band, int M, size_t lines,
                               cudaStream_t s) {
  k_band_bf16x3<<<elementwise_grid(lines * (size_t)M * kChunk), 256, 0, s>>>(kcol, band, M, lines);
  return counted(cudaGetLastError());
}

cudaError_t take_tc_timeout(bool* hit) {
  unsigned v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(v));
  if (e != cudaSuccess) return e;
  *hit = v != 0;
  if (v != 0) {
    const unsigned z = 0;
    e = cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof(z));
  }
  return e;
}

}  // namespace mgwr

// Smoother half-sweep with its input lines staged by bulk copies (FP32, lines
// of 64 .. 4096 steps; Sec. 3 Eq. red-black, Sec. 6 Eq. red-black_2d).
//
// A persistent grid of as many CTAs as fit on the GPU walks the line pairs of
// every instance.  Each thread group owning one pair has its own staging area
// in shared memory and its own mbarrier: while the group transforms one pair,
// the f lines and the neighbour lines of its next pair arrive there through
// cp.async.bulk (the TMA unit's untiled copies), so the gather that starts each
// transform reads shared memory instead of waiting on HBM.  The arithmetic is
// the direct-load kernel's, term for term, so results are bitwise identical.
#include "mgwr_common.cuh"
#include "mgwr_tma.cuh"

namespace mgwr {

// Bit 0: a group gave up waiting for its copies; bit 1: a pair needed more
// staging slots than it has (read by take_stage_timeout).
__device__ unsigned g_stage_timeout;

namespace {

// Staged lines per group: fA, fB and at most seven distinct neighbour lines.
// Two points of a pair in one row share a neighbour (B's left is A's right);
// a pair that wraps to the next row has A in the last or B in the first column
// of the other colour, so one of A's right and B's left lies outside the grid.
// Lines outside the grid (zero Dirichlet data) take no slot.
constexpr int kSlots = 9;

// The lines a group gathers for one item (one line pair of one instance):
// line k (fA, fB, A's four neighbours, B's four) is staged at off[k] floats
// into the group's area when bit k of `present` is set, else it is zero.
struct PairLines {
  int inst;
  bool valid, hasB;
  int pA, pB;
  unsigned present;  // lines that carry data
  unsigned copies;   // lines whose slot this item fills (B's left reuses A's right)
  int off[10];
};

__device__ __forceinline__ void pair_lines(PairLines& P, int item, int g, int groups, int nblk,
                                           int npairs, int npts, int d, int n, int par, int M) {
  P.inst = item / nblk;
  const int pair = (item - P.inst * nblk) * groups + g;
  P.valid = pair < npairs;
  const int kA = 2 * pair, kB = kA + 1;
  P.hasB = P.valid && kB < npts;
  int iA = 0, jA = 0, iB = 0, jB = 0;
  P.pA = P.valid ? colour_point(kA, d, n, par, iA, jA) : 0;
  P.pB = P.hasB ? colour_point(kB, d, n, par, iB, jB) : 0;
  unsigned present = (P.valid ? 1u : 0u) | (P.hasB ? 2u : 0u);
  if (P.valid) {
    present |= (iA > 0 ? 4u : 0u) | (iA < n - 1 ? 8u : 0u);
    if (d == 2) present |= (jA > 0 ? 16u : 0u) | (jA < n - 1 ? 32u : 0u);
  }
  if (P.hasB) {
    present |= (iB > 0 ? 64u : 0u) | (iB < n - 1 ? 128u : 0u);
    if (d == 2) present |= (jB > 0 ? 256u : 0u) | (jB < n - 1 ? 512u : 0u);
  }
  // B's left neighbour (pB - 1) is A's right one (pA + 1)
  const bool shared_lr = (present & 64u) && (present & 8u) && P.pB - 1 == P.pA + 1;
  P.present = present;
  P.copies = shared_lr ? (present & ~64u) : present;
  if (__popc(P.copies) > kSlots) {  // cannot happen (see kSlots); flagged, never overruns
    P.present = P.copies = 0;
    atomicOr(&g_stage_timeout, 2u);
  }
  int next = 0;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    P.off[k] = 0;
    if ((P.copies >> k) & 1u) P.off[k] = (next++) * M;
  }
  if (shared_lr) P.off[6] = P.off[3];
}

// Global start of line k of an item (instance offset `base`, M values per line).
__device__ __forceinline__ const float* line_src(const PairLines& P, int k, const float* f,
                                                 const float* u, int n, int M) {
  const long long p = k < 2 ? (k == 0 ? P.pA : P.pB) : (k < 6 ? P.pA : P.pB);
  const int dir = k < 2 ? -1 : (k - 2) & 3;
  const long long step = dir == 0 ? -1 : dir == 1 ? 1 : dir == 2 ? -(long long)n : (long long)n;
  return k < 2 ? f + p * M : u + (p + step) * M;
}

// One arrival announcing the item's bytes, then one bulk copy per staged line
// (lines are whole time lines: M * 4 bytes, a multiple of 16, at 16-byte
// aligned addresses on both sides).
__device__ __forceinline__ void issue_copies(const PairLines& P, const float* f, const float* u,
                                             float* stage, uint64_t* bar, int n, int M) {
  const unsigned bytes = (unsigned)M * (unsigned)sizeof(float);
  mbar_arrive_expect_tx(bar, bytes * (unsigned)__popc(P.copies));
#pragma unroll
  for (int k = 0; k < 10; ++k)
    if ((P.copies >> k) & 1u) bulk_copy_g2s(stage + P.off[k], line_src(P, k, f, u, n, M), bytes, bar);
}

// The copies of item `item` into `stage` (one thread of the group; kept out of
// line so that its index work does not add to the transform's registers).
__device__ __noinline__ void stage_item(int item, int g, int groups, int nblk, int npairs, int npts,
                                        int d, int n, int par, int M, const float* f,
                                        const float* u, size_t fstride, float* stage,
                                        uint64_t* bar) {
  PairLines Q;
  pair_lines(Q, item, g, groups, nblk, npairs, npts, d, n, par, M);
  const size_t off = (size_t)Q.inst * fstride;
  fence_proxy_async_smem();
  issue_copies(Q, f + off, u + off, stage, bar, n, M);
}

}  // namespace

template <int BLOCK, class SH, int E>
__global__ void __launch_bounds__(BLOCK, min_blocks<float>(BLOCK, E))
    k_sweep_staged(const float* __restrict__ f, float* __restrict__ u, float* __restrict__ delta,
                   const Cx<float>* __restrict__ spec, const Cx<float>* __restrict__ tw, int d,
                   int n, int par, float hinv2, int npts, int npairs, int nblk, int nitems,
                   size_t fstride, size_t sstride) {
  constexpr int TL = SH::L8 / E;  // threads per line pair
  constexpr int groups = BLOCK / TL;
  constexpr int M = SH::L / 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t bars[groups];
  const SH sh(SH::logL);
  const int g = threadIdx.x / TL;
  const int t = threadIdx.x - g * TL;
  Cx<float>* const bufs = reinterpret_cast<Cx<float>*>(smem_raw);
  Cx<float>* buf = bufs + g * Pad<float>::len(SH::L);
  float* stage = reinterpret_cast<float*>(bufs + groups * Pad<float>::len(SH::L)) +
                 (size_t)g * kSlots * M;
  const GroupSync sync(TL, BLOCK, g);
  if (threadIdx.x < groups) mbar_init(&bars[threadIdx.x], 1);
  mbar_fence_init();
  __syncthreads();
  uint64_t* bar = &bars[g];

  int item = blockIdx.x;
  if (t == 0 && item < nitems)
    stage_item(item, g, groups, nblk, npairs, npts, d, n, par, M, f, u, fstride, stage, bar);
  for (unsigned j = 0; item < nitems; ++j, item += gridDim.x) {
    // one thread per group waits; the CTA barrier also ends every read of buf by
    // the previous item, and a group that gave up ends the whole CTA (every group
    // runs the same items, so all threads leave at the same point)
    int failed = 0;
    if (t == 0) failed = mbar_wait_bounded(bar, j & 1u) ? 0 : 1;
    if (__syncthreads_or(failed)) {
      if (failed) {
        atomicOr(&g_stage_timeout, 1u);
        (void)mbar_wait_bounded(bar, j & 1u);  // the copies in flight land before the CTA ends
      }
      return;
    }
    (void)mbar_try_wait(bar, j & 1u);  // completed phase: acquire the staged lines here too
    PairLines P;
    pair_lines(P, item, g, groups, nblk, npairs, npts, d, n, par, M);
    // line k at time m: the staged value, or the zero Dirichlet value outside the grid
    auto rd = [&](int k, int m) -> float {
      return ((P.present >> k) & 1u) ? stage[P.off[k] + m] : 0.f;
    };
    auto load = [&](int m) -> Cx<float> {
      if (d == 2)
        return Cx<float>{rd(0, m) + hinv2 * ((rd(2, m) + rd(3, m)) + (rd(4, m) + rd(5, m))),
                         rd(1, m) + hinv2 * ((rd(6, m) + rd(7, m)) + (rd(8, m) + rd(9, m)))};
      return Cx<float>{rd(0, m) + hinv2 * (rd(2, m) + rd(3, m)),
                       rd(1, m) + hinv2 * (rd(6, m) + rd(7, m))};
    };
    // once the group has read its staged lines, the next item's copies start
    const int next = item + (int)gridDim.x;
    auto refill = [&]() {
      if (t == 0 && next < nitems)
        stage_item(next, g, groups, nblk, npairs, npts, d, n, par, M, f, u, fstride, stage, bar);
    };
    Cx<float> v[E][8];
    fft_forward<E>(buf, t, sh, tw, load, v, sync, refill);
    const Cx<float>* sp = spec + (size_t)P.inst * sstride;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int b = t + e * TL;
#pragma unroll
      for (int q = 0; q < 8; ++q) v[e][q] = cmul(v[e][q], sp[8 * b + q]);
    }
    const size_t ioff = (size_t)P.inst * fstride;
    float* uA = u + ioff + (size_t)P.pA * M;
    float* uB = u + ioff + (size_t)P.pB * M;
    float* dA = delta != nullptr ? delta + ioff + (size_t)P.pA * M : nullptr;
    float* dB = delta != nullptr ? delta + ioff + (size_t)P.pB * M : nullptr;
    const bool valid = P.valid, hasB = P.hasB;
    auto store = [&](int m, Cx<float> y) {
      if (valid) {
        if (dA != nullptr) dA[m] = y.x - uA[m];
        uA[m] = y.x;
        if (hasB) {
          if (dB != nullptr) dB[m] = y.y - uB[m];
          uB[m] = y.y;
        }
      }
    };
    fft_inverse<E>(buf, t, sh, tw, v, store, sync);
  }
}

namespace {

template <int BLOCK, class SH, int E>
cudaError_t staged_launch(const float* f, float* u, float* delta, const Cx<float>* spec,
                          size_t sstride, const Cx<float>* tw, const LevelShape& ls, int par, float hinv2, int npts, int npairs,
                          cudaStream_t s) {
  constexpr int TL = SH::L8 / E;
  constexpr int groups = BLOCK / TL;
  constexpr int M = SH::L / 2;
  auto kern = k_sweep_staged<BLOCK, SH, E>;
  const size_t smem = (size_t)groups * (Pad<float>::len(SH::L) * sizeof(Cx<float>) +
                                        (size_t)kSlots * M * sizeof(float));
  cudaError_t e = prepare_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem)) !=
      cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int nblk = (npairs + groups - 1) / groups;
  const long long nitems = (long long)nblk * ls.batch;
  if (nitems > 0x7fffffffLL) return cudaErrorInvalidValue;
  const long long cap = (long long)per_sm * sms;
  const unsigned grid = (unsigned)(nitems < cap ? nitems : cap);
  kern<<<grid, BLOCK, smem, s>>>(f, u, delta, spec, tw, ls.d, ls.n, par, hinv2, npts, npairs,
                                 nblk, (int)nitems, ls.field_stride(), sstride);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_sweep_staged(const float* f, float* u, float* delta, const Cx<float>* spec,
                                size_t spec_stride, const Cx<float>* tw, const float* zero,
                                const LevelShape& ls, int par, float hinv2, int E,
                                cudaStream_t s) {
  (void)zero;  // lines outside the grid are not read: the kernel adds zeros
  const int M = ls.M;
  if (M < 64 || M > kShortMaxM) return cudaErrorInvalidValue;
  const int npts = colour_count(ls.d, ls.n, par);
  const int npairs = (npts + 1) / 2;
  if (npairs == 0 || ls.batch == 0) return cudaSuccess;
  E = engine_split(2 * M, E);
  const int logL = ilog2(2 * M);
  cudaError_t e = cudaErrorInvalidValue;
#define MGWR_STAGED_ARGS f, u, delta, spec, spec_stride, tw, ls, par, hinv2, npts, npairs, s
  switch (logL * 8 + E) {
#define MGWR_CASE_E(LG, EE)                                                                    \
  case LG * 8 + EE:                                                                            \
    e = staged_launch<((1 << LG) / (8 * EE) > 256 ? (1 << LG) / (8 * EE) : 256), FixedShape<LG>, \
                      EE>(MGWR_STAGED_ARGS);                                                   \
    break;
#define MGWR_CASE(LG) MGWR_CASE_E(LG, 1) MGWR_CASE_E(LG, 2) MGWR_CASE_E(LG, 4)
    MGWR_FIXED_LOGL(MGWR_CASE)
#undef MGWR_CASE
#undef MGWR_CASE_E
    default:
      break;
  }
#undef MGWR_STAGED_ARGS
  if (e != cudaSuccess) return e;
  return counted(cudaGetLastError());
}

cudaError_t take_stage_timeout(bool* hit) {
  unsigned v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_stage_timeout, sizeof(v));
  if (e != cudaSuccess) return e;
  *hit = v != 0;
  if (v != 0) {
    const unsigned z = 0;
    e = cudaMemcpyToSymbol(g_stage_timeout, &z, sizeof(z));
  }
  return e;
}

}  // namespace mgwr

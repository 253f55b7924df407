// Host side of the MGWR library: handle (a batch of same-shape instances),
// level hierarchy, Algorithm 1 driver, FP64 / mixed-precision solve loops and
// the C ABI of include/mgwr.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/mgwr.h"
#include "mgwr_internal.h"

using mgwr::Cx;
using mgwr::LevelShape;

namespace {

// What the defect work field r_l of a level currently stands for (all
// instances of a batch are always in the same state).
enum RState {
  R_STALE = 0,    // nothing known: the defect needs the full (convolution) form
  R_ZERO_U = 1,   // u_l = 0 (just restricted into): the defect is f_l itself
  R_DELTA = 2,    // last op was a complete red-black step: defect from its delta
  R_CURRENT = 3,  // r_l holds the defect of the current (u_l, f_l)
};

// Default switch of the mixed modes' outer defect (mgwr_set_outer_switch): an
// outer step carries the defect by its correction (launch_defect_update, error
// about 1e-6 of the defect at the last full computation, the anchor) while
// the relative defect is at least this fraction of the anchor's, so that the
// carried error stays near 1e-4 of the defect it updates.
constexpr double kLooseOuter = 1e-2;

// Forms of a mixed-mode outer defect: in full in the outer arithmetic; carried
// by the step's correction (launch_defect_update); in full with T_M u by a
// double-float convolution (launch_defect_anchor, MGWR_MIXED to a tolerance of
// at least kAnchorTol).
enum OuterForm { kOuterFull = 0, kOuterCarry = 1, kOuterAnchor = 2 };

// Tolerances at or above which MGWR_MIXED computes its full outer defects (the
// anchors of the carried ones, and those that decide the stop) with T_M u in
// double-float (launch_defect_anchor): the form's error, about 2^-44 |T_M u|
// (a few 1e-14 of the right-hand side's scale, against about 1e-15 for an FP64
// convolution), stays below 1e-3 of them.  Below, every full defect is FP64.
constexpr double kAnchorTol = 1e-10;

template <class R>
struct Hier {
  std::vector<R*> u, f, r;        // per level: batch * N_l * M values each
  std::vector<R*> dl;             // per level: black-point changes of the last step
  std::vector<int> rs;            // per level: RState of r
  Cx<R>* spec = nullptr;          // batch * nlev * L: spectra of the inverse columns
  Cx<R>* spec_rp = nullptr;       // the same in the register-pass engine's order (FP32)
  Cx<R>* tspec_rp = nullptr;      // the Toeplitz spectra in that order (FP32)
  Cx<R>* tspec = nullptr;         // batch * L: spectra of the Toeplitz columns
  Cx<R>* tw = nullptr;            // L twiddles
  R* zero = nullptr;              // M zeros: the neighbour line outside the grid
  bool ready = false;             // spectra present
  bool full = false;              // every level's u, f, r, dl allocated
};

// The per-level defect states of a handle's three hierarchies.  Enqueuing an
// iteration updates them as if it ran; a captured iteration graph keeps what
// its capture left and a replay sets them to it, so that the next iteration's
// key (and the launches it selects) follows the device's state.
struct RsState {
  std::vector<int> r64, r32, rdd;
};

}  // namespace

struct mgwr_handle {
  int d = 1, n = 1, M = 4, L = 8, nlev = 1, B = 1;
  int Lt = 8;  // transform length of the convolution engine (twiddle table length)
  std::vector<double> alpha, T, c;  // per instance; c = tau^-alpha / Gamma(2 - alpha)
  int precision = MGWR_FP64, order = MGWR_ORDER_TEXT;
  int inner = 0;  // inner cycles per outer defect; 0 = the precision's default (inner_cycles)
  int inner_now = 0;  // inner cycles of the outer step being enqueued (0: inner_cycles)
  double loose_above = kLooseOuter;  // mgwr_set_outer_switch
  std::vector<int> nl;          // interior points per dimension, level 0 = 1
  std::vector<double> hinv2;    // 1/h_l^2
  std::vector<double> sigma;    // 2d/h_l^2
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  double* r = nullptr;          // batch * M: r_1..r_M
  double* dk = nullptr;         // batch * (M+1): d_0..d_M
  double* kcol = nullptr;       // batch * nlev * M inverse columns
  unsigned char* tc_band = nullptr;  // their Toeplitz bands in bf16 pieces (tensor-core sweeps)
  double* c_dev = nullptr;      // batch
  Hier<double> h64;
  Hier<float> h32;
  Hier<mgwr::dd> hdd;  // MGWR_DD: every level in double-float
  // double-float copies of the finest iterate / right-hand side and of the
  // Toeplitz spectra, for the outer defect of MGWR_MIXED_DD
  mgwr::dd* u_dd = nullptr;
  mgwr::dd* f_dd = nullptr;
  mgwr::dd* zero_dd = nullptr;
  Cx<mgwr::dd>* tspec_dd = nullptr;
  Cx<mgwr::dd>* tw_dd = nullptr;
  // partitioned-convolution scratch for M > kShortMaxM: the block spectra of
  // the largest launch (finest level, all points), in 16-byte complex values;
  // shared by every precision (one launch at a time on the handle's stream)
  Cx<double>* scratch = nullptr;
  size_t scratch_count = 0;
  unsigned long long* norm_bits = nullptr;  // device, one per instance
  unsigned long long* norm_host = nullptr;  // pinned, one per instance
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<double> r0, relres;  // per instance
  bool r0_valid = false;
  std::vector<void*> allocs;
  std::string err;
  // FFT-engine split (butterflies per thread) per kernel class and level; 0 = default
  std::vector<int> split[MGWR_NUM_KERNEL_CLASSES];
  // solve-loop iterations captured as CUDA graphs (one per form of the
  // iteration: settings and outer-defect form), replayed every iteration
  bool use_graphs = true;
  struct IterGraph {
    long long key;        // (precision, cycle, nu1, nu2, inner, order, outer form, finest state)
    cudaGraphExec_t exec;
    bool exact;           // its norms come from the full defect in the working precision
    long long kernels;    // kernel launches recorded in the graph
    RsState after;        // the defect states the iteration leaves
  };
  std::vector<IterGraph> graphs;
  // the rest of an MGWR_FP64 solve as one graph launch: a WHILE node whose body
  // is one iteration (its launches without the copy of the norms to the host)
  // and k_loop_decide, which ends it on the device (run_device_loop)
  struct LoopGraph {
    long long key = -1;   // iteration_key of the body (-1: none)
    cudaGraphExec_t exec = nullptr;
    bool exact = true;    // the body's norms come from the full defect
    long long kernels = 0;  // kernel launches of one body iteration
    bool unusable = false;  // the body's iteration is not uniform for this key
  } loop;
  bool use_device_loop = true;              // mgwr_set_device_loop
  mgwr::LoopState* loop_dev = nullptr;      // device state of the loop
  mgwr::LoopState* loop_pin = nullptr;      // pinned copy read after it
  double* r0_dev = nullptr;                 // per-instance reference norms (device)
  double* r0_pin = nullptr;                 // pinned staging of r0
  // pipelined transfers (mgwr_stage_rhs / mgwr_take_rhs / mgwr_stage_solution):
  // device staging of the next right-hand side and of the last solution, each
  // copied to or from the host on a stream of its own
  double* stage_in = nullptr;
  double* stage_out = nullptr;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev_in = nullptr;      // the staged right-hand side has landed
  cudaEvent_t ev_taken = nullptr;   // stage_in copied into f: it may be refilled
  cudaEvent_t ev_staged = nullptr;  // stage_out holds the solution to send
  cudaEvent_t ev_sent = nullptr;    // stage_out sent to the host: it may be refilled
  bool rhs_pending = false;
  // the finest iterate is zero (right-hand side just set without initial values)
  bool u_zero = false;
  // mixed modes: the form of the outer defect of the iteration being enqueued
  int outer_form = kOuterFull;
  // where the outer defect in double-float is held for the carried form: -1
  // nowhere (full form only), 0 the right-hand side f_dd (u = 0), 1 outer_field
  int outer_src = -1;
  // the finest outer defect of MGWR_MIXED, M <= kShortMaxM, in double-float (outer_field)
  double* r_outer = nullptr;
  // per-kernel-class timing (mgwr_profile): event pairs around each launch
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Mark { int cls; int ev; double lines; };
  std::vector<Mark> marks;
  long long prof_launches[MGWR_NUM_KERNEL_CLASSES] = {};
  double prof_ms[MGWR_NUM_KERNEL_CLASSES] = {};
  double prof_lines[MGWR_NUM_KERNEL_CLASSES] = {};
};

namespace {

const char* kNullHandleMsg = "null handle";

int fail(mgwr_t h, int code, const std::string& msg) {
  if (h != nullptr) h->err = msg;
  return code;
}

#define MGWR_CK(h, call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail((h), MGWR_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MGWR_TRY(call)            \
  do {                            \
    int s_ = (call);              \
    if (s_ != MGWR_OK) return s_; \
  } while (0)

// Stream-ordered allocation on the handle's stream: creating or destroying a
// handle does not synchronise the device, so handles on other streams (other
// server slots) keep running.
template <class P>
int dev_alloc(mgwr_t h, P** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMallocAsync(&q, bytes < 16 ? 16 : bytes, h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MGWR_E_NOMEM, std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " +
                                     cudaGetErrorString(e));
  }
  h->allocs.push_back(q);
  *p = static_cast<P*>(q);
  return MGWR_OK;
}

// Allocates a zero-filled field once.
template <class R>
int ensure_field(mgwr_t h, R** p, size_t count) {
  if (*p != nullptr) return MGWR_OK;
  MGWR_TRY(dev_alloc(h, p, count * sizeof(R)));
  MGWR_CK(h, cudaMemsetAsync(*p, 0, count * sizeof(R), h->stream));
  return MGWR_OK;
}

bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }

// Engine kernel classes of a hierarchy's arithmetic.
template <class R>
constexpr int sweep_class() {
  return std::is_same<R, float>::value ? MGWR_K_SWEEP32
         : std::is_same<R, mgwr::dd>::value ? MGWR_K_SWEEP_DD : MGWR_K_SWEEP64;
}
template <class R>
constexpr int defect_class() {
  return std::is_same<R, float>::value ? MGWR_K_DEFECT32
         : std::is_same<R, mgwr::dd>::value ? MGWR_K_DEFECT_DD : MGWR_K_DEFECT64;
}

// A staged sweep that gave up waiting for its copies (never expected: a copy of
// a valid line always lands) turns into an error of the call that ran it.
int check_staging(mgwr_t h) {
  bool hit = false;
  MGWR_CK(h, mgwr::take_stage_timeout(&hit));
  if (hit) return fail(h, MGWR_E_CUDA, "staged sweep: wait for bulk copies gave up");
  MGWR_CK(h, mgwr::take_tc_timeout(&hit));
  if (hit) return fail(h, MGWR_E_CUDA, "tensor-core sweep: wait for its MMAs gave up");
  return MGWR_OK;
}

int split_of(const mgwr_handle* h, int cls, int l) {
  return h->split[cls].empty() ? 0 : h->split[cls][l];
}

RsState save_rs(const mgwr_handle* h) { return RsState{h->h64.rs, h->h32.rs, h->hdd.rs}; }

void load_rs(mgwr_t h, const RsState& s) {
  h->h64.rs = s.r64;
  h->h32.rs = s.r32;
  h->hdd.rs = s.rdd;
}

void drop_graph(mgwr_t h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  if (h->loop.exec != nullptr) cudaGraphExecDestroy(h->loop.exec);
  h->loop = mgwr_handle::LoopGraph{};
}

// The handle's partitioned-convolution scratch viewed as complex values of R
// (null for M <= kShortMaxM, where no launch uses it).
template <class R>
Cx<R>* scratch_for(mgwr_t h) {
  static_assert(sizeof(Cx<R>) <= sizeof(Cx<double>), "scratch holds 16-byte values");
  return reinterpret_cast<Cx<R>*>(h->scratch);
}

size_t points(const mgwr_handle* h, int l) {
  return h->d == 1 ? (size_t)h->nl[l] : (size_t)h->nl[l] * h->nl[l];
}

// values of one level field over the whole batch
size_t level_count(const mgwr_handle* h, int l) { return points(h, l) * h->M * h->B; }

LevelShape shape(const mgwr_handle* h, int l) { return LevelShape{h->d, h->nl[l], h->M, h->B}; }

int parity(const mgwr_handle* h, int colour) {
  int red_par;
  if (h->d == 1)
    red_par = h->order == MGWR_ORDER_TEXT ? 1 : 0;
  else
    red_par = 0;
  return colour == MGWR_RED ? red_par : red_par ^ 1;
}

// Every field of every level (u, f, r, dl) of a hierarchy.  The black-change
// field dl is zero-filled once, so lines that are never swept black stay finite
// and the zero-weight boundary reads of the defect-from-changes kernel are safe.
template <class R>
int ensure_full(mgwr_t h, Hier<R>& H) {
  if (H.full) return MGWR_OK;
  for (int l = 0; l < h->nlev; ++l) {
    const size_t cnt = level_count(h, l);
    MGWR_TRY(ensure_field(h, &H.u[l], cnt));
    MGWR_TRY(ensure_field(h, &H.f[l], cnt));
    MGWR_TRY(ensure_field(h, &H.r[l], cnt));
    if (l > 0) MGWR_TRY(ensure_field(h, &H.dl[l], cnt));
  }
  H.full = true;
  return MGWR_OK;
}

template <class R>
void init_hier(mgwr_t h, Hier<R>& H) {
  H.u.assign(h->nlev, nullptr);
  H.f.assign(h->nlev, nullptr);
  H.r.assign(h->nlev, nullptr);
  H.dl.assign(h->nlev, nullptr);
  H.rs.assign(h->nlev, R_STALE);
}

int ensure_h32(mgwr_t h) {
  if (h->h32.ready) return MGWR_OK;
  Hier<float>& H = h->h32;
  MGWR_TRY(ensure_full(h, H));
  MGWR_TRY(ensure_field(h, &H.zero, (size_t)h->M));
  const size_t nspec = (size_t)h->B * h->nlev * h->L;
  MGWR_TRY(dev_alloc(h, &H.spec, sizeof(Cx<float>) * nspec));
  MGWR_TRY(dev_alloc(h, &H.tspec, sizeof(Cx<float>) * (size_t)h->B * h->L));
  MGWR_TRY(dev_alloc(h, &H.tw, sizeof(Cx<float>) * (size_t)h->Lt));
  MGWR_CK(h, mgwr::launch_round_cx(H.spec, h->h64.spec, nspec, h->stream));
  MGWR_CK(h, mgwr::launch_round_cx(H.tspec, h->h64.tspec, (size_t)h->B * h->L, h->stream));
  MGWR_CK(h, mgwr::launch_round_cx(H.tw, h->h64.tw, (size_t)h->Lt, h->stream));
  if (mgwr::radix_length(h->M)) {
    MGWR_TRY(dev_alloc(h, &H.spec_rp, sizeof(Cx<float>) * nspec));
    MGWR_CK(h, mgwr::launch_spectra_rp(H.spec_rp, h->h64.spec, (size_t)h->B * h->nlev, h->M,
                                       false, h->stream));
    MGWR_TRY(dev_alloc(h, &H.tspec_rp, sizeof(Cx<float>) * (size_t)h->B * h->L));
    MGWR_CK(h, mgwr::launch_spectra_rp(H.tspec_rp, h->h64.tspec, (size_t)h->B, h->M, true,
                                       h->stream));
  }
  if (mgwr::tensor_length(h->M)) {
    const size_t lines = (size_t)h->B * h->nlev;
    MGWR_TRY(dev_alloc(h, &h->tc_band, mgwr::tc_band_bytes(h->M) * lines));
    MGWR_CK(h, mgwr::launch_band_bf16x3(h->kcol, h->tc_band, h->M, lines, h->stream));
  }
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  H.ready = true;
  return MGWR_OK;
}

// The double-float Toeplitz spectra and twiddles, split from FP64.
int ensure_dd_spectra(mgwr_t h) {
  if (h->tspec_dd != nullptr) return MGWR_OK;
  MGWR_TRY(dev_alloc(h, &h->tspec_dd, sizeof(Cx<mgwr::dd>) * (size_t)h->B * h->L));
  MGWR_TRY(dev_alloc(h, &h->tw_dd, sizeof(Cx<mgwr::dd>) * (size_t)h->Lt));
  MGWR_CK(h, mgwr::launch_split_cx(h->tspec_dd, h->h64.tspec, (size_t)h->B * h->L, h->stream));
  MGWR_CK(h, mgwr::launch_split_cx(h->tw_dd, h->h64.tw, (size_t)h->Lt, h->stream));
  return MGWR_OK;
}

int ensure_dd(mgwr_t h) {
  if (h->u_dd != nullptr) return MGWR_OK;
  const size_t cnt = level_count(h, h->nlev - 1);
  MGWR_TRY(ensure_field(h, &h->u_dd, cnt));
  MGWR_TRY(ensure_field(h, &h->f_dd, cnt));
  MGWR_TRY(ensure_field(h, &h->zero_dd, (size_t)h->M));
  return ensure_dd_spectra(h);
}

// The double-float hierarchy of MGWR_DD: every level's fields in double-float,
// the inverse-column and Toeplitz spectra and the twiddles split from FP64.
int ensure_hdd(mgwr_t h) {
  if (h->hdd.ready) return MGWR_OK;
  MGWR_TRY(ensure_dd(h));
  Hier<mgwr::dd>& H = h->hdd;
  MGWR_TRY(ensure_full(h, H));
  const size_t nspec = (size_t)h->B * h->nlev * h->L;
  MGWR_TRY(dev_alloc(h, &H.spec, sizeof(Cx<mgwr::dd>) * nspec));
  MGWR_CK(h, mgwr::launch_split_cx(H.spec, h->h64.spec, nspec, h->stream));
  H.tspec = h->tspec_dd;
  H.tw = h->tw_dd;
  H.zero = h->zero_dd;
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  H.ready = true;
  return MGWR_OK;
}

// ---- per-class timing ----------------------------------------------------------

// Records an event before a launch of class `cls` covering `lines` time lines;
// returns the index to close with prof_end (or -1 when profiling is off).
int prof_begin(mgwr_t h, int cls, double lines) {
  if (!h->profiling) return -1;
  const int idx = (int)h->marks.size();
  const int ev = 2 * idx;
  while ((int)h->ev_pool.size() < ev + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->ev_pool.push_back(e);
  }
  cudaEventRecord(h->ev_pool[ev], h->stream);
  h->marks.push_back({cls, ev, lines});
  return idx;
}

void prof_end(mgwr_t h, int idx) {
  if (idx < 0) return;
  cudaEventRecord(h->ev_pool[h->marks[idx].ev + 1], h->stream);
}

// Folds all recorded launch times into the per-class totals (synchronises).
void prof_collect(mgwr_t h) {
  if (h->marks.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (const auto& mk : h->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[mk.ev], h->ev_pool[mk.ev + 1]) == cudaSuccess) {
      h->prof_launches[mk.cls] += 1;
      h->prof_ms[mk.cls] += ms;
      h->prof_lines[mk.cls] += mk.lines;
    }
  }
  h->marks.clear();
}

// ---- Algorithm 1 components ------------------------------------------------------

template <class R>
int coarsest(mgwr_t h, Hier<R>& H) {
  const int pm = prof_begin(h, MGWR_K_COARSEST, (double)h->B);
  MGWR_CK(h, mgwr::launch_sweep<R>(H.f[0], H.u[0], (R*)nullptr, H.spec, (size_t)h->nlev * h->L,
                                    H.tw, H.zero, scratch_for<R>(h), shape(h, 0), 0, true, R(0),
                                    split_of(h, sweep_class<R>(), 0) &
                                        ~(mgwr::kTensor | mgwr::kRadix),
                                    h->stream));
  prof_end(h, pm);
  H.rs[0] = R_STALE;
  return MGWR_OK;
}

// One colour half-sweep of level l >= 1 (parity par) of the fields f -> u with
// launch shape E: the tensor-core form for FP32 lines of 64 .. 256 steps when E
// carries kTensor, else the FFT engine.
template <class R>
cudaError_t level_sweep(mgwr_t h, Hier<R>& H, int l, const R* f, R* u, R* delta,
                        const LevelShape& ls, int par, int E) {
  if constexpr (std::is_same<R, float>::value) {
    const int eff = mgwr::effective_split(h->M, 4, E);
    if ((eff & mgwr::kTensor) && h->tc_band != nullptr) {
      const size_t bb = mgwr::tc_band_bytes(h->M);
      return mgwr::launch_sweep_tc(f, u, delta, h->tc_band + (size_t)l * bb, (size_t)h->nlev * bb,
                                   ls, par, (float)h->hinv2[l], h->stream);
    }
    if ((eff & mgwr::kRadix) && H.spec_rp != nullptr)
      return mgwr::launch_sweep_rp(f, u, delta, H.spec_rp + (size_t)l * h->L,
                                   (size_t)h->nlev * h->L, H.tw, H.zero, ls, par,
                                   (float)h->hinv2[l], eff & ~mgwr::kRadix, h->stream);
  }
  return mgwr::launch_sweep<R>(f, u, delta, H.spec + (size_t)l * h->L, (size_t)h->nlev * h->L,
                               H.tw, H.zero, scratch_for<R>(h), ls, par, false, R(h->hinv2[l]),
                               E & ~(mgwr::kTensor | mgwr::kRadix), h->stream);
}

// One colour half-sweep at level l >= 1; delta != null also records the change of
// every swept line (used by the black half-sweep ending a smoothing step).
template <class R>
int sweep_colour(mgwr_t h, Hier<R>& H, int l, int colour, R* delta) {
  const int par = parity(h, colour);
  const size_t N = points(h, l);
  const double lines = (double)h->B * (double)(par == 0 ? (N + 1) / 2 : N / 2);
  const int pm = prof_begin(h, sweep_class<R>(), lines);
  MGWR_CK(h, level_sweep(h, H, l, H.f[l], H.u[l], delta, shape(h, l), par,
                         split_of(h, sweep_class<R>(), l)));
  prof_end(h, pm);
  return MGWR_OK;
}

template <class R>
int smooth_colour(mgwr_t h, Hier<R>& H, int l, int colour) {
  if (l == 0) return coarsest(h, H);  // one point: its half-sweep is the exact solve
  MGWR_TRY(sweep_colour(h, H, l, colour, (R*)nullptr));
  H.rs[l] = R_STALE;
  return MGWR_OK;
}

// `steps` red-black smoothing steps; with `record`, the last black half-sweep
// records its changes so that a defect that follows needs no convolution
// (without, the level's defect state is stale).
template <class R>
int smooth(mgwr_t h, Hier<R>& H, int l, int steps, bool record = true) {
  for (int s = 0; s < steps; ++s) {
    MGWR_TRY(sweep_colour(h, H, l, MGWR_RED, (R*)nullptr));
    MGWR_TRY(sweep_colour(h, H, l, MGWR_BLACK,
                          record && s == steps - 1 ? H.dl[l] : (R*)nullptr));
  }
  if (steps > 0) H.rs[l] = record ? R_DELTA : R_STALE;
  return MGWR_OK;
}

// Full defect r = f - (T_M (x) I + A_h) u with one FFT convolution per line.
template <class R>
int defect(mgwr_t h, Hier<R>& H, int l, unsigned long long* norm_bits) {
  const int pm = prof_begin(h, defect_class<R>(),
                            (double)(points(h, l) * h->B));
  MGWR_CK(h, (mgwr::launch_defect<R, R>(H.u[l], H.f[l], H.r[l], H.tspec, (size_t)h->L, H.tw,
                                         H.zero, scratch_for<R>(h), shape(h, l), R(h->hinv2[l]), norm_bits,
                                         split_of(h, defect_class<R>(), l),
                                         h->stream)));
  prof_end(h, pm);
  H.rs[l] = R_CURRENT;
  return MGWR_OK;
}

// Defect of level l from the last smoothing step's changes (no convolution).
template <class R>
int defect_from_delta(mgwr_t h, Hier<R>& H, int l, unsigned long long* norm_bits) {
  const int pm = prof_begin(h, MGWR_K_DEFECT_DELTA, (double)(points(h, l) * h->B));
  MGWR_CK(h, mgwr::launch_defect_from_delta<R>(H.dl[l], H.r[l], H.zero, shape(h, l),
                                                parity(h, MGWR_RED), R(h->hinv2[l]), norm_bits,
                                                h->stream));
  prof_end(h, pm);
  H.rs[l] = R_CURRENT;
  return MGWR_OK;
}

// Pointer to the defect of level l for the restriction, produced the cheapest
// way the level's state allows (Algorithm 1, "compute the defect").
template <class R>
int current_defect(mgwr_t h, Hier<R>& H, int l, const R** out) {
  switch (H.rs[l]) {
    case R_ZERO_U:
      *out = H.f[l];
      return MGWR_OK;
    case R_DELTA:
      MGWR_TRY(defect_from_delta(h, H, l, nullptr));
      break;
    case R_CURRENT:
      break;
    default:
      MGWR_TRY(defect(h, H, l, nullptr));
      break;
  }
  *out = H.r[l];
  return MGWR_OK;
}

template <class R>
int restrict_into(mgwr_t h, Hier<R>& H, int l, const R* r) {
  const int pm = prof_begin(h, MGWR_K_RESTRICT, (double)(points(h, l - 1) * h->B));
  MGWR_CK(h, mgwr::launch_restrict<R>(r, H.f[l - 1], H.u[l - 1], shape(h, l), h->stream));
  prof_end(h, pm);
  H.rs[l - 1] = R_ZERO_U;
  return MGWR_OK;
}

template <class R>
int prolong_into(mgwr_t h, Hier<R>& H, int l) {
  const int pm = prof_begin(h, MGWR_K_PROLONG, (double)(points(h, l) * h->B));
  MGWR_CK(h, mgwr::launch_prolong<R>(H.u[l], H.u[l - 1], shape(h, l), h->stream));
  prof_end(h, pm);
  H.rs[l] = R_STALE;
  return MGWR_OK;
}

// Restriction of the defect a smoothing step left (state R_DELTA) straight from
// the black half-sweep's changes: the fine defect is never stored.
template <class R>
int restrict_delta_into(mgwr_t h, Hier<R>& H, int l) {
  const int pm = prof_begin(h, MGWR_K_RESTRICT, (double)(points(h, l - 1) * h->B));
  MGWR_CK(h, mgwr::launch_restrict_delta<R>(H.dl[l], H.f[l - 1], H.u[l - 1], H.zero, shape(h, l),
                                             parity(h, MGWR_RED), R(h->hinv2[l]), h->stream));
  prof_end(h, pm);
  H.rs[l - 1] = R_ZERO_U;
  return MGWR_OK;
}

// Algorithm 1's "compute the defect and restrict it" for level l.  The fused
// form pays for FP32 fields (2-D 511 x 511, M = 4096: 41 -> 25 ms per solve for
// both steps); for the 8-byte types it measured slower than the two line
// kernels (2-D 255 x 255, M = 1024, FP64: 13.8 -> 20 ms: twice the iterations
// per byte, and 2 blocks per SM at its register count).
template <class R>
int defect_restrict(mgwr_t h, Hier<R>& H, int l) {
  if (sizeof(R) == 4 && H.rs[l] == R_DELTA) return restrict_delta_into(h, H, l);
  const R* r = nullptr;
  MGWR_TRY(current_defect(h, H, l, &r));
  return restrict_into(h, H, l, r);
}

// One cycle from level l.  `keep`: the post-smoothing records its changes for
// a defect of level l that follows before any other smoothing of it.  Below
// the top that happens only in cycles without pre-smoothing that visit a
// level more than once (the next visit restricts the defect the last one
// left); every other visit starts from a restricted right-hand side.
template <class R>
int cycle(mgwr_t h, Hier<R>& H, int l, int gamma, int nu1, int nu2, bool keep = true) {
  if (l == 0) return coarsest(h, H);
  MGWR_TRY(smooth(h, H, l, nu1));
  MGWR_TRY(defect_restrict(h, H, l));
  for (int g = 0; g < gamma; ++g)
    MGWR_TRY(cycle(h, H, l - 1, gamma, nu1, nu2, gamma > 1 && nu1 == 0));
  MGWR_TRY(prolong_into(h, H, l));
  MGWR_TRY(smooth(h, H, l, nu2, keep));
  return MGWR_OK;
}

int clear_norms(mgwr_t h) {
  MGWR_CK(h, cudaMemsetAsync(h->norm_bits, 0, sizeof(unsigned long long) * h->B, h->stream));
  return MGWR_OK;
}

// Reads the per-instance norm accumulators (cleared before the producing kernel).
int read_norms(mgwr_t h, std::vector<double>& out) {
  MGWR_CK(h, cudaMemcpyAsync(h->norm_host, h->norm_bits, sizeof(unsigned long long) * h->B,
                             cudaMemcpyDeviceToHost, h->stream));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  out.resize(h->B);
  for (int b = 0; b < h->B; ++b) std::memcpy(&out[b], &h->norm_host[b], sizeof(double));
  return MGWR_OK;
}

// The field that holds a solve's finest outer defect in double-float for the
// carried form (launch_defect_update; 8 bytes a value): its own field r_outer
// in MGWR_MIXED; in MGWR_MIXED_DD the FP64 iterate's field, which a solve
// leaves unused while it holds the iterate in double-float (u_dd, joined back
// at its end), so only solves may write it.  Null where no line length or
// precision has the carried form.
mgwr::dd* outer_field(const mgwr_handle* h) {
  static_assert(sizeof(mgwr::dd) == sizeof(double), "a double-float value fills a double's slot");
  if (h->M > mgwr::kShortMaxM) return nullptr;
  if (h->precision == MGWR_MIXED) return reinterpret_cast<mgwr::dd*>(h->r_outer);
  if (h->precision == MGWR_MIXED_DD) return reinterpret_cast<mgwr::dd*>(h->h64.u[h->nlev - 1]);
  return nullptr;
}

// Whether the solves of this handle carry outer defects (a field for them,
// and a finite switch: at +inf every outer defect is full and none is kept).
bool carries(const mgwr_handle* h) {
  return outer_field(h) != nullptr && std::isfinite(h->loose_above);
}

// The full outer defect of the mixed modes (FP64 for MGWR_MIXED, double-float
// for MGWR_MIXED_DD) rounded into the FP32 right-hand side, norms into
// norm_bits (cleared by the caller); when the handle carries its outer defect,
// first into outer_field in double-float, then rounded from there.  Called by
// solves only (outer_field may be the FP64 iterate's field).
int enqueue_outer_full(mgwr_t h) {
  const int L = h->nlev - 1;
  const size_t cnt = level_count(h, L);
  const bool ddef = h->precision == MGWR_MIXED_DD;
  mgwr::dd* keep = carries(h) ? outer_field(h) : nullptr;
  const int pd = prof_begin(h, ddef ? MGWR_K_DEFECT_DD : MGWR_K_DEFECT64, (double)(points(h, L) * h->B));
  if (ddef && keep != nullptr)
    MGWR_CK(h, (mgwr::launch_defect<mgwr::dd, mgwr::dd>(
                   h->u_dd, h->f_dd, keep, h->tspec_dd, (size_t)h->L, h->tw_dd, h->zero_dd,
                   scratch_for<mgwr::dd>(h), shape(h, L), mgwr::dd(h->hinv2[L]), h->norm_bits,
                   split_of(h, MGWR_K_DEFECT_DD, L), h->stream)));
  else if (ddef)
    MGWR_CK(h, (mgwr::launch_defect<mgwr::dd, float>(
                   h->u_dd, h->f_dd, h->h32.f[L], h->tspec_dd, (size_t)h->L, h->tw_dd, h->zero_dd,
                   scratch_for<mgwr::dd>(h), shape(h, L), mgwr::dd(h->hinv2[L]), h->norm_bits,
                   split_of(h, MGWR_K_DEFECT_DD, L), h->stream)));
  else if (keep != nullptr)
    MGWR_CK(h, (mgwr::launch_defect<double, mgwr::dd>(
                   h->h64.u[L], h->h64.f[L], keep, h->h64.tspec, (size_t)h->L, h->h64.tw,
                   h->h64.zero, scratch_for<double>(h), shape(h, L), h->hinv2[L], h->norm_bits,
                   split_of(h, MGWR_K_DEFECT64, L), h->stream)));
  else
    MGWR_CK(h, (mgwr::launch_defect<double, float>(
                   h->h64.u[L], h->h64.f[L], h->h32.f[L], h->h64.tspec, (size_t)h->L, h->h64.tw,
                   h->h64.zero, scratch_for<double>(h), shape(h, L), h->hinv2[L], h->norm_bits,
                   split_of(h, MGWR_K_DEFECT64, L), h->stream)));
  prof_end(h, pd);
  if (keep != nullptr) MGWR_CK(h, mgwr::launch_round_dd(keep, h->h32.f[L], cnt, h->stream));
  h->h32.rs[L] = R_STALE;
  return MGWR_OK;
}

// MGWR_MIXED: whether its full outer defects may take the double-float
// convolution form (launch_defect_anchor): the handle carries its defects (so
// the next steps start from the one it leaves in outer_field), has the
// double-float Toeplitz spectra, and solves to a tolerance (at least
// kAnchorTol) that the form's error cannot reach.  Such defects also decide the
// stop; a switch at +inf keeps every outer defect in FP64.
bool anchor_ok(const mgwr_handle* h, double tol) {
  return h->precision == MGWR_MIXED && carries(h) && h->tspec_dd != nullptr && tol >= kAnchorTol;
}

// The outer defect of MGWR_MIXED in the double-float-convolution form into
// outer_field and, rounded, the FP32 right-hand side, norms into norm_bits.
int enqueue_anchor(mgwr_t h) {
  const int L = h->nlev - 1;
  const int pa = prof_begin(h, MGWR_K_DEFECT_DD, (double)(points(h, L) * h->B));
  MGWR_CK(h, mgwr::launch_defect_anchor(h->h64.u[L], h->h64.f[L], outer_field(h), h->h32.f[L],
                                        h->tspec_dd, (size_t)h->L, h->tw_dd, h->h64.zero,
                                        shape(h, L), h->hinv2[L], h->norm_bits, h->stream));
  prof_end(h, pa);
  h->h32.rs[L] = R_STALE;
  return MGWR_OK;
}

// FP64 defect of the finest iterate with its per-instance infinity norms.  In
// mixed mode the defect is written, rounded, as the FP32 right-hand side.
int finest_defect_norms(mgwr_t h, std::vector<double>& norms, bool to_h32) {
  const int L = h->nlev - 1;
  MGWR_TRY(clear_norms(h));
  if (to_h32) {
    MGWR_TRY(enqueue_outer_full(h));
  } else {
    const int pm = prof_begin(h, MGWR_K_DEFECT64, (double)(points(h, L) * h->B));
    MGWR_TRY(ensure_field(h, &h->h64.r[L], level_count(h, L)));
    MGWR_CK(h, (mgwr::launch_defect<double, double>(h->h64.u[L], h->h64.f[L], h->h64.r[L],
                                                     h->h64.tspec, (size_t)h->L, h->h64.tw,
                                                     h->h64.zero, scratch_for<double>(h), shape(h, L), h->hinv2[L], h->norm_bits,
                                                    split_of(h, MGWR_K_DEFECT64, L),
                                                     h->stream)));
    h->h64.rs[L] = R_CURRENT;
    prof_end(h, pm);
  }
  return read_norms(h, norms);
}

// Double-float defect of the finest iterate, rounded into the FP32 right-hand
// side, with per-instance norms (MGWR_MIXED_DD).
int finest_defect_norms_dd(mgwr_t h, std::vector<double>& norms) {
  MGWR_TRY(clear_norms(h));
  MGWR_TRY(enqueue_outer_full(h));
  return read_norms(h, norms);
}

// Relative defects from norms; returns the largest, NaN if any is not finite.
double relative(mgwr_t h, const std::vector<double>& norms, std::vector<double>& rel) {
  rel.resize(h->B);
  double worst = 0.0;
  for (int b = 0; b < h->B; ++b) {
    rel[b] = h->r0[b] > 0.0 ? norms[b] / h->r0[b] : (norms[b] == 0.0 ? 0.0 : norms[b]);
    if (!std::isfinite(rel[b])) worst = NAN;
    if (worst == worst) worst = std::max(worst, rel[b]);
  }
  return worst;
}

// Double-float defect of the double-float iterate (u_dd, f_dd) into the
// double-float hierarchy's finest right-hand side, norms into norm_bits
// (MGWR_DD's outer defect; the iterate itself never passes through a
// convolution, so its rounding stays at the double-float level).
int outer_defect_ddd(mgwr_t h) {
  const int L = h->nlev - 1;
  const int pd = prof_begin(h, MGWR_K_DEFECT_DD, (double)(points(h, L) * h->B));
  MGWR_CK(h, (mgwr::launch_defect<mgwr::dd, mgwr::dd>(
                 h->u_dd, h->f_dd, h->hdd.f[L], h->tspec_dd, (size_t)h->L, h->tw_dd, h->zero_dd,
                 scratch_for<mgwr::dd>(h), shape(h, L), mgwr::dd(h->hinv2[L]), h->norm_bits,
                 split_of(h, MGWR_K_DEFECT_DD, L), h->stream)));
  prof_end(h, pd);
  h->hdd.rs[L] = R_STALE;
  return MGWR_OK;
}

// Inner cycles per outer defect of the refinements.  Default 2: the outer
// steps that carry their defect by the correction (launch_defect_update) cost
// about one FP32 cycle, so the full FP64 defects (about eight FP32 cycles on
// GB300, FP64 running at 1/64 of the FP32 rate) are needed only as anchors and
// for the stopping test, whatever the number of steps (2-D 511 x 511, M = 4096
// to 1e-8: 5 outer steps of 2 cycles 797 ms, of 3 cycles 906 ms in
// MGWR_MIXED; 513 against 623 ms in MGWR_MIXED_DD).
int inner_cycles(const mgwr_handle* h) {
  if (h->inner > 0) return h->inner;
  return 2;
}

// Inner cycles of the outer step being enqueued: inner_cycles, or one more on
// the step that the solve loop predicts will finish with it.
int step_cycles(const mgwr_handle* h) { return h->inner_now > 0 ? h->inner_now : inner_cycles(h); }

// One cycle on hierarchy H and the finest defect norms (from the smoothing
// changes when the cycle ended with a smoothing step: *exact = false).
template <class R>
int enqueue_plain(mgwr_t h, Hier<R>& H, int cyc, int nu1, int nu2, bool* exact) {
  const int L = h->nlev - 1;
  MGWR_TRY(cycle(h, H, L, cyc, nu1, nu2));
  MGWR_TRY(clear_norms(h));
  if (H.rs[L] == R_DELTA) {
    MGWR_TRY(defect_from_delta(h, H, L, h->norm_bits));
    *exact = false;
  } else {
    MGWR_TRY(defect(h, H, L, h->norm_bits));
    *exact = true;
  }
  return MGWR_OK;
}

// Enqueues one iteration of the solve loop and the copy of its per-instance
// norms to pinned host memory, with no host synchronisation (so that it can be
// captured into a graph).  FP64: one cycle, then the finest defect norms (from
// the smoothing changes when the cycle ended with a smoothing step, *exact =
// false).  Mixed: `inner` FP32 cycles on the defect equation from e = 0, the
// update, and the outer defect (double or double-float) with its norms.
// MGWR_DD: the same with double-float inner cycles and outer defect.
int enqueue_iteration(mgwr_t h, int cyc, int nu1, int nu2, bool* exact, bool copy_norms = true) {
  const int L = h->nlev - 1;
  const size_t cnt = level_count(h, L);
  if (h->precision == MGWR_FP64) {
    MGWR_TRY(enqueue_plain(h, h->h64, cyc, nu1, nu2, exact));
  } else if (h->precision == MGWR_DD) {
    // double-float cycles on the defect equation from e = 0, the update of the
    // double-float iterate, its double-float defect as the next right-hand side
    MGWR_CK(h, cudaMemsetAsync(h->hdd.u[L], 0, cnt * sizeof(mgwr::dd), h->stream));
    h->hdd.rs[L] = R_ZERO_U;
    // the next inner cycle restricts the post-smoothing's defect only without
    // pre-smoothing; after the last one the outer defect is computed in full
    for (int k = 0; k < step_cycles(h); ++k)
      MGWR_TRY(cycle(h, h->hdd, L, cyc, nu1, nu2, nu1 == 0 && k + 1 < step_cycles(h)));
    const int pm = prof_begin(h, MGWR_K_REFINE, (double)(points(h, L) * h->B));
    MGWR_CK(h, mgwr::launch_refine_dd2(h->u_dd, h->hdd.u[L], cnt, h->stream));
    prof_end(h, pm);
    MGWR_TRY(clear_norms(h));
    MGWR_TRY(outer_defect_ddd(h));
    *exact = true;
  } else {
    const bool ddef = h->precision == MGWR_MIXED_DD;
    MGWR_CK(h, cudaMemsetAsync(h->h32.u[L], 0, cnt * sizeof(float), h->stream));
    h->h32.rs[L] = R_ZERO_U;  // f32 holds the outer defect, e32 = 0
    for (int k = 0; k < step_cycles(h); ++k)
      MGWR_TRY(cycle(h, h->h32, L, cyc, nu1, nu2, nu1 == 0 && k + 1 < step_cycles(h)));
    const int pm = prof_begin(h, MGWR_K_REFINE, (double)(points(h, L) * h->B));
    if (ddef)
      MGWR_CK(h, mgwr::launch_refine_dd(h->u_dd, h->h32.u[L], cnt, h->stream));
    else
      MGWR_CK(h, mgwr::launch_refine(h->h64.u[L], h->h32.u[L], cnt, h->stream));
    prof_end(h, pm);
    MGWR_TRY(clear_norms(h));
    if (h->outer_form == kOuterCarry) {
      // the defect carried by the correction e = h32.u: outer_field = r - A e, with
      // r the double-float right-hand side f_dd after MGWR_MIXED_DD's start from
      // u = 0, else outer_field
      const int pl = prof_begin(h, MGWR_K_DEFECT32, (double)(points(h, L) * h->B));
      const bool rp = h->h32.tspec_rp != nullptr;  // the register-pass engine serves M
      const Cx<float>* ts = rp ? h->h32.tspec_rp : h->h32.tspec;
      mgwr::dd* ro = outer_field(h);
      const mgwr::dd* ri = h->outer_src == 0 ? h->f_dd : ro;
      const float hi2 = (float)h->hinv2[L];  // (n + 1)^2, a power of 4
      MGWR_CK(h, rp ? mgwr::launch_defect_update_rp<mgwr::dd>(
                          h->h32.u[L], ri, ro, h->h32.f[L], ts, (size_t)h->L, h->h32.tw,
                          h->h32.zero, shape(h, L), hi2, h->norm_bits, h->stream)
                    : mgwr::launch_defect_update<mgwr::dd>(
                          h->h32.u[L], ri, ro, h->h32.f[L], ts, (size_t)h->L, h->h32.tw,
                          h->h32.zero, shape(h, L), hi2, h->norm_bits, h->stream));
      prof_end(h, pl);
      h->h32.rs[L] = R_STALE;
      *exact = false;
    } else if (h->outer_form == kOuterAnchor) {
      MGWR_TRY(enqueue_anchor(h));
      *exact = true;
    } else {
      MGWR_TRY(enqueue_outer_full(h));
      *exact = true;
    }
  }
  if (copy_norms)
    MGWR_CK(h, cudaMemcpyAsync(h->norm_host, h->norm_bits, sizeof(unsigned long long) * h->B,
                               cudaMemcpyDeviceToHost, h->stream));
  return MGWR_OK;
}

// Runs one iteration: replays the captured graph when it matches the current
// settings (capturing it first if needed), else enqueues the launches
// directly; then waits and decodes the norms.
// Identifies the launch sequence of the next iteration: the settings, the
// outer-defect form and the state of the finest FP64 defect field it starts
// from (the first FP64 iteration from u = 0 restricts f itself).
long long iteration_key(const mgwr_handle* h, int cyc, int nu1, int nu2) {
  const int rs_in = h->precision == MGWR_FP64 ? h->h64.rs[h->nlev - 1] : 0;
  return ((((((long long)h->precision * 4 + cyc) * 32 + nu1) * 32 + nu2) * 32 * 4 +
           (long long)step_cycles(h) * 4 + h->order) * 4 + (h->outer_form == kOuterCarry    ? 1 + h->outer_src
                                                        : h->outer_form == kOuterAnchor ? 3
                                                                                        : 0)) *
             4 + rs_in;
}

int run_iteration(mgwr_t h, int cyc, int nu1, int nu2, std::vector<double>& norms, bool* exact) {
  const long long key = iteration_key(h, cyc, nu1, nu2);
  if (h->use_graphs && !h->profiling) {
    const mgwr_handle::IterGraph* slot = nullptr;
    for (const auto& g : h->graphs)
      if (g.key == key) slot = &g;
    if (slot == nullptr) {
      if (h->graphs.size() >= 4) drop_graph(h);  // settings changed: start over
      cudaGraph_t g = nullptr;
      MGWR_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      bool ex = true;
      const long long before = mgwr::launch_counter();
      const int st = enqueue_iteration(h, cyc, nu1, nu2, &ex);
      const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
      // captured launches do not run; count them when the graph is replayed
      const long long captured = mgwr::launch_counter() - before;
      mgwr::add_launches(-captured);
      if (st != MGWR_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      MGWR_CK(h, e);
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      MGWR_CK(h, ei);
      h->graphs.push_back({key, exec, ex, captured, save_rs(h)});
      slot = &h->graphs.back();
    }
    load_rs(h, slot->after);
    MGWR_CK(h, cudaGraphLaunch(slot->exec, h->stream));
    mgwr::add_launches(slot->kernels);
    *exact = slot->exact;
  } else {
    MGWR_TRY(enqueue_iteration(h, cyc, nu1, nu2, exact));
  }
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  norms.resize(h->B);
  for (int b = 0; b < h->B; ++b) std::memcpy(&norms[b], &h->norm_host[b], sizeof(double));
  return MGWR_OK;
}

int check_level(mgwr_t h, int hierarchy, int level) {
  if (hierarchy != MGWR_H64 && hierarchy != MGWR_H32 && hierarchy != MGWR_HDD)
    return fail(h, MGWR_E_INVAL, "hierarchy must be MGWR_H64, MGWR_H32 or MGWR_HDD");
  if (level < 0 || level >= h->nlev) return fail(h, MGWR_E_INVAL, "level out of range");
  if (hierarchy == MGWR_H32 && !h->h32.ready)
    return fail(h, MGWR_E_STATE, "the FP32 hierarchy exists only after mgwr_set_precision(MGWR_MIXED)");
  if (hierarchy == MGWR_HDD && !h->hdd.ready)
    return fail(h, MGWR_E_STATE, "the double-float hierarchy exists only after mgwr_set_precision(MGWR_DD)");
  if (hierarchy == MGWR_H64) MGWR_TRY(ensure_full(h, h->h64));
  return MGWR_OK;
}

// Calls f with the hierarchy a component call addresses (checked before).
template <class F>
int with_hier(mgwr_t h, int hierarchy, F f) {
  if (hierarchy == MGWR_H64) return f(h->h64);
  if (hierarchy == MGWR_H32) return f(h->h32);
  return f(h->hdd);
}

int check_cycle_args(mgwr_t h, int cyc, int nu1, int nu2) {
  if (cyc != 1 && cyc != 2) return fail(h, MGWR_E_INVAL, "cycle must be 1 (V) or 2 (W)");
  if (nu1 < 0 || nu2 < 0 || nu1 > 16 || nu2 > 16 || nu1 + nu2 == 0)
    return fail(h, MGWR_E_INVAL, "need 0 <= nu1, nu2 <= 16 and nu1 + nu2 >= 1");
  return MGWR_OK;
}

// ---- FFT-engine launch-shape tuner ---------------------------------------------

// Splits chosen by mgwr_autotune, per (kernel class, d, n, M, batch): handles of a
// shape that was tuned before start with its choices.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, std::vector<int>> g_tune;

void load_tuned(mgwr_t h) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (int c = 0; c < MGWR_NUM_KERNEL_CLASSES; ++c) {
    auto it = g_tune.find(std::make_tuple(c, h->d, h->n, h->M, h->B));
    if (it != g_tune.end()) h->split[c] = it->second;
  }
}

void set_split(mgwr_t h, int cls, int l, int E) {
  if (h->split[cls].empty()) h->split[cls].assign(h->nlev, 0);
  h->split[cls][l] = E;
}

// The sample the tuner times on level l: as many instances (at most the batch,
// at least one) as keep it within 2^27 values, all pairs of those instances.
LevelShape tune_sample(const mgwr_handle* h, int l) {
  const size_t cap = size_t(1) << 27;
  const size_t per = points(h, l) * (size_t)h->M;
  size_t b = per >= cap ? 1 : cap / per;
  if (b > (size_t)h->B) b = h->B;
  return LevelShape{h->d, h->nl[l], h->M, (int)b};
}

// Mean device time of `reps` launches after one warm-up launch.
template <class F>
int time_launches(mgwr_t h, F launch, float* ms) {
  MGWR_CK(h, launch());
  const int reps = 5;
  MGWR_CK(h, cudaEventRecord(h->ev0, h->stream));
  for (int i = 0; i < reps; ++i) MGWR_CK(h, launch());
  MGWR_CK(h, cudaEventRecord(h->ev1, h->stream));
  MGWR_CK(h, cudaEventSynchronize(h->ev1));
  float t = 0.f;
  MGWR_CK(h, cudaEventElapsedTime(&t, h->ev0, h->ev1));
  *ms = t / reps;
  return MGWR_OK;
}

// Times every split E in {1, 2, 4} of one kernel class with `launch(E)` and
// keeps the fastest; a larger E must beat the best smaller one by 3 %.  FP32
// sweeps also try each E with staged input lines (E | kStaged), which must
// beat the best direct-load launch by 3 % as well.
template <class F>
int tune_class(mgwr_t h, int cls, int l, int word, F launch) {
  int best = 1;
  float best_ms = 0.f;
  const int cands[10] = {1, 2, 4, 1 | mgwr::kStaged, 2 | mgwr::kStaged, 4 | mgwr::kStaged,
                         1 | mgwr::kTensor, 1 | mgwr::kRadix, 2 | mgwr::kRadix, 4 | mgwr::kRadix};
  const int ncand = cls == MGWR_K_SWEEP32 ? 10 : 3;
  for (int c = 0; c < ncand; ++c) {
    const int E = cands[c];
    if (mgwr::effective_split(h->M, word, E) != E) continue;  // same launch as a smaller E
    float ms = 0.f;
    MGWR_TRY(time_launches(h, [&] { return launch(E); }, &ms));
    if (E == 1 || ms < 0.97f * best_ms) {
      best = E;
      best_ms = ms;
    }
  }
  set_split(h, cls, l, best);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[std::make_tuple(cls, h->d, h->n, h->M, h->B)] = h->split[cls];
  return MGWR_OK;
}

// Sweeps (red points, every level >= 1 and the one-point solve) and defects
// (every level) of the samples, written to a scratch field, in the arithmetic
// `R` of hierarchy H; no state of the handle changes.
template <class R>
int tune_hierarchy(mgwr_t h, Hier<R>& H, int cls_sweep, int cls_defect) {
  size_t count = 0;
  for (int l = 0; l < h->nlev; ++l) {
    const LevelShape ls = tune_sample(h, l);
    count = std::max(count, ls.field_stride() * ls.batch);
  }
  R *out = nullptr, *dlt = nullptr;
  MGWR_TRY(dev_alloc(h, &out, count * sizeof(R)));
  MGWR_TRY(dev_alloc(h, &dlt, count * sizeof(R)));
  MGWR_CK(h, cudaMemsetAsync(out, 0, count * sizeof(R), h->stream));
  int st = MGWR_OK;
  for (int l = h->nlev - 1; l >= 0 && st == MGWR_OK; --l) {
    const LevelShape ls = tune_sample(h, l);
    st = ensure_field(h, &H.u[l], level_count(h, l));
    if (st == MGWR_OK) st = ensure_field(h, &H.f[l], level_count(h, l));
    if (st == MGWR_OK)
      st = tune_class(h, cls_sweep, l, sizeof(R) == 4 ? 4 : 8, [&](int E) {
        // one smoothing step as the cycle runs it: red, then black recording its changes
        const Cx<R>* spec = H.spec + (size_t)l * h->L;
        const size_t sstride = (size_t)h->nlev * h->L;
        if (l == 0)
          return mgwr::launch_sweep<R>(H.f[0], out, (R*)nullptr, spec, sstride, H.tw, H.zero,
                                       scratch_for<R>(h), ls, 0, true, R(0),
                                       E & ~(mgwr::kTensor | mgwr::kRadix), h->stream);
        const cudaError_t e =
            level_sweep(h, H, l, H.f[l], out, (R*)nullptr, ls, parity(h, MGWR_RED), E);
        if (e != cudaSuccess) return e;
        return level_sweep(h, H, l, H.f[l], out, dlt, ls, parity(h, MGWR_BLACK), E);
      });
    if (st == MGWR_OK)
      st = tune_class(h, cls_defect, l, sizeof(R) == 4 ? 4 : 8, [&](int E) {
        return mgwr::launch_defect<R, R>(H.u[l], H.f[l], out, H.tspec, (size_t)h->L, H.tw,
                                         H.zero, scratch_for<R>(h), ls, R(h->hinv2[l]), nullptr,
                                         E, h->stream);
      });
  }
  for (void* p : {(void*)out, (void*)dlt}) {
    cudaFreeAsync(p, h->stream);
    h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), p));
  }
  return st;
}

// Outer defect of the mixed modes (FP64 or double-float iterate, FP32 output)
// on the finest-level sample.
int tune_outer(mgwr_t h) {
  const int Lf = h->nlev - 1;
  const LevelShape ls = tune_sample(h, Lf);
  const size_t count = ls.field_stride() * ls.batch;
  float* out = nullptr;
  MGWR_TRY(dev_alloc(h, &out, count * sizeof(float)));
  int st;
  if (h->precision == MGWR_MIXED_DD)
    st = tune_class(h, MGWR_K_DEFECT_DD, Lf, 8, [&](int E) {
      return mgwr::launch_defect<mgwr::dd, float>(h->u_dd, h->f_dd, out, h->tspec_dd, (size_t)h->L,
                                                  h->tw_dd, h->zero_dd, scratch_for<mgwr::dd>(h),
                                                  ls, mgwr::dd(h->hinv2[Lf]), nullptr, E,
                                                  h->stream);
    });
  else
    st = tune_class(h, MGWR_K_DEFECT64, Lf, 8, [&](int E) {
      return mgwr::launch_defect<double, float>(h->h64.u[Lf], h->h64.f[Lf], out, h->h64.tspec,
                                                (size_t)h->L, h->h64.tw, h->h64.zero,
                                                scratch_for<double>(h), ls, h->hinv2[Lf],
                                                nullptr, E, h->stream);
    });
  cudaFreeAsync(out, h->stream);
  h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), (void*)out));
  return st;
}

// Handles allocate their fields stream-ordered from the device's default memory
// pool.  With the pool's default release threshold (0) every synchronisation
// hands freed memory back to the driver, and the next handle maps it again
// (for a 2-D 511 x 511, M = 4096 handle: 57 ms to create, 76 ms to destroy);
// keeping freed memory in this process's pool makes a new handle of a size
// seen before cheap.  The pool and its threshold belong to this process only.
void keep_pool_memory() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t threshold = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  }
  cudaGetLastError();
  done.push_back(dev);
}

// The per-instance setup of Sec. 5 from h->alpha, h->c: the L1 Toeplitz
// columns, the inverse columns of every level by divide and conquer, and the
// FP64 spectra of both (twiddles already in place).  Temporaries come
// stream-ordered from the pool and are returned; synchronises the stream.
int setup_columns(mgwr_t h) {
  const size_t B = h->B;
  const int M = h->M;
  double *sig_dev = nullptr, *alpha_dev = nullptr;
  Cx<double>* work = nullptr;
  int s = dev_alloc(h, &alpha_dev, sizeof(double) * B);
  if (s == MGWR_OK) s = dev_alloc(h, &sig_dev, sizeof(double) * h->nlev);
  if (s == MGWR_OK) s = dev_alloc(h, &work, sizeof(Cx<double>) * B * h->nlev * 3 * M);
  cudaError_t e = cudaSuccess;
  if (s == MGWR_OK) {
    e = cudaMemcpyAsync(sig_dev, h->sigma.data(), sizeof(double) * h->nlev,
                        cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->c_dev, h->c.data(), sizeof(double) * B, cudaMemcpyHostToDevice,
                          h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(alpha_dev, h->alpha.data(), sizeof(double) * B, cudaMemcpyHostToDevice,
                          h->stream);
    if (e == cudaSuccess)
      e = mgwr::launch_coefficients(h->r, h->dk, M, alpha_dev, h->c_dev, h->B, h->stream);
    if (e == cudaSuccess)
      e = mgwr::launch_inverse_columns(h->kcol, h->r, sig_dev, h->nlev, M, h->B, work, h->stream);
    if (e == cudaSuccess)
      e = mgwr::launch_spectra(h->h64.spec, h->kcol, h->B * h->nlev, M, h->h64.tw, h->stream);
    if (e == cudaSuccess)
      e = mgwr::launch_spectra(h->h64.tspec, h->r, h->B, M, h->h64.tw, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  // the temporaries are no longer needed
  for (void* p : {(void*)work, (void*)sig_dev, (void*)alpha_dev}) {
    if (p == nullptr) continue;
    cudaFreeAsync(p, h->stream);
    h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), p));
  }
  if (s != MGWR_OK) return s;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MGWR_E_CUDA, std::string("setup: ") + cudaGetErrorString(e));
  }
  h->h64.ready = true;
  return MGWR_OK;
}

// The copies of the FP64 setup that the other arithmetics keep (rounded FP32
// spectra, their register-pass order, the tensor-core bands, double-float
// splits), recomputed after setup_columns changed the FP64 ones.
int refresh_derived(mgwr_t h) {
  const size_t nspec = (size_t)h->B * h->nlev * h->L;
  if (h->h32.ready) {
    MGWR_CK(h, mgwr::launch_round_cx(h->h32.spec, h->h64.spec, nspec, h->stream));
    MGWR_CK(h, mgwr::launch_round_cx(h->h32.tspec, h->h64.tspec, (size_t)h->B * h->L, h->stream));
    if (h->h32.spec_rp != nullptr)
      MGWR_CK(h, mgwr::launch_spectra_rp(h->h32.spec_rp, h->h64.spec, (size_t)h->B * h->nlev,
                                         h->M, false, h->stream));
    if (h->h32.tspec_rp != nullptr)
      MGWR_CK(h, mgwr::launch_spectra_rp(h->h32.tspec_rp, h->h64.tspec, (size_t)h->B, h->M,
                                         true, h->stream));
    if (h->tc_band != nullptr)
      MGWR_CK(h, mgwr::launch_band_bf16x3(h->kcol, h->tc_band, h->M, (size_t)h->B * h->nlev,
                                          h->stream));
  }
  if (h->tspec_dd != nullptr)
    MGWR_CK(h, mgwr::launch_split_cx(h->tspec_dd, h->h64.tspec, (size_t)h->B * h->L, h->stream));
  if (h->hdd.ready)
    MGWR_CK(h, mgwr::launch_split_cx(h->hdd.spec, h->h64.spec, nspec, h->stream));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return MGWR_OK;
}

int create_impl(int d, int n, int M, const double* T, const double* alpha, int batch,
                mgwr_t* out) {
  if (out == nullptr) return MGWR_E_INVAL;
  *out = nullptr;
  if (d != 1 && d != 2) return MGWR_E_INVAL;
  if (n < 1 || !is_pow2((long long)n + 1)) return MGWR_E_INVAL;
  if ((d == 1 && n > 32767) || (d == 2 && n > 4095)) return MGWR_E_INVAL;
  if (!is_pow2(M) || M < 4 || M > mgwr::kMaxM) return MGWR_E_INVAL;
  if (batch < 1 || batch > 65535 || T == nullptr || alpha == nullptr) return MGWR_E_INVAL;
  for (int b = 0; b < batch; ++b) {
    if (!(T[b] > 0.0) || !std::isfinite(T[b])) return MGWR_E_INVAL;
    if (!(alpha[b] > 0.0) || !(alpha[b] <= 1.0)) return MGWR_E_INVAL;
  }

  keep_pool_memory();
  mgwr_t h = new (std::nothrow) mgwr_handle;
  if (h == nullptr) return MGWR_E_NOMEM;
  h->d = d;
  h->n = n;
  h->M = M;
  h->L = 2 * M;
  h->Lt = mgwr::engine_length(M);
  h->B = batch;
  h->alpha.assign(alpha, alpha + batch);
  h->T.assign(T, T + batch);
  for (int b = 0; b < batch; ++b) {
    const double tau = T[b] / M;
    h->c.push_back(std::pow(tau, -alpha[b]) / std::tgamma(2.0 - alpha[b]));
  }
  h->r0.assign(batch, 0.0);
  h->relres.assign(batch, 0.0);
  std::vector<int> sizes{n};
  while (sizes.back() > 1) sizes.push_back((sizes.back() - 1) / 2);
  h->nl.assign(sizes.rbegin(), sizes.rend());
  h->nlev = (int)h->nl.size();
  for (int l = 0; l < h->nlev; ++l) {
    const double hl = 1.0 / (h->nl[l] + 1);
    h->hinv2.push_back(1.0 / (hl * hl));
    h->sigma.push_back(2.0 * d / (hl * hl));
  }
  init_hier(h, h->h64);
  init_hier(h, h->h32);
  init_hier(h, h->hdd);

  auto bail = [&](int code) {
    mgwr_destroy(h);
    return code;
  };
  if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return bail(MGWR_E_CUDA);
  }
  h->stream = h->own_stream;
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
      cudaMallocHost(&h->norm_host, sizeof(unsigned long long) * batch) != cudaSuccess) {
    cudaGetLastError();
    return bail(MGWR_E_CUDA);
  }
  const size_t B = batch;
  int s;
  if ((s = dev_alloc(h, &h->norm_bits, sizeof(unsigned long long) * B)) != MGWR_OK) return bail(s);
  if ((s = dev_alloc(h, &h->r, sizeof(double) * B * M)) != MGWR_OK) return bail(s);
  if ((s = dev_alloc(h, &h->dk, sizeof(double) * B * (M + 1))) != MGWR_OK) return bail(s);
  if ((s = dev_alloc(h, &h->kcol, sizeof(double) * B * h->nlev * M)) != MGWR_OK) return bail(s);
  if ((s = dev_alloc(h, &h->c_dev, sizeof(double) * B)) != MGWR_OK) return bail(s);
  if ((s = dev_alloc(h, &h->h64.spec, sizeof(Cx<double>) * B * h->nlev * h->L)) != MGWR_OK)
    return bail(s);
  if ((s = dev_alloc(h, &h->h64.tspec, sizeof(Cx<double>) * B * h->L)) != MGWR_OK) return bail(s);
  if ((s = dev_alloc(h, &h->h64.tw, sizeof(Cx<double>) * (size_t)h->Lt)) != MGWR_OK) return bail(s);
  if (h->M > mgwr::kShortMaxM) {
    h->scratch_count = mgwr::long_scratch_count(shape(h, h->nlev - 1));
    if ((s = dev_alloc(h, &h->scratch, sizeof(Cx<double>) * h->scratch_count)) != MGWR_OK)
      return bail(s);
  }
  if (mgwr::launch_twiddles(h->h64.tw, h->Lt, h->stream) != cudaSuccess) {
    cudaGetLastError();
    return bail(MGWR_E_CUDA);
  }
  if ((s = setup_columns(h)) != MGWR_OK) return bail(s);
  h->h64.ready = true;
  // the finest iterate and right-hand side always exist; the rest on demand
  const int Lf = h->nlev - 1;
  if ((s = ensure_field(h, &h->h64.zero, (size_t)M)) != MGWR_OK) return bail(s);
  if ((s = ensure_field(h, &h->h64.u[Lf], level_count(h, Lf))) != MGWR_OK) return bail(s);
  if ((s = ensure_field(h, &h->h64.f[Lf], level_count(h, Lf))) != MGWR_OK) return bail(s);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return bail(MGWR_E_CUDA);
  }
  load_tuned(h);
  *out = h;
  return MGWR_OK;
}

}  // namespace

// =================================================================================
// C ABI
// =================================================================================

extern "C" {

const char* mgwr_status_string(int s) {
  switch (s) {
    case MGWR_OK: return "ok";
    case MGWR_E_INVAL: return "invalid argument";
    case MGWR_E_NOMEM: return "out of memory";
    case MGWR_E_TOOBIG: return "request exceeds budget";
    case MGWR_E_NOCONV: return "not converged";
    case MGWR_E_NUMERIC: return "non-finite residual";
    case MGWR_E_AGAIN: return "try again";
    case MGWR_E_TIMEOUT: return "timed out";
    case MGWR_E_CUDA: return "CUDA error";
    case MGWR_E_STATE: return "invalid state";
    default: return "unknown status";
  }
}

const char* mgwr_last_error(mgwr_t h) { return h == nullptr ? kNullHandleMsg : h->err.c_str(); }

int mgwr_destroy(mgwr_t h) {
  if (h == nullptr) return MGWR_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->norm_host) cudaFreeHost(h->norm_host);
  if (h->loop_pin) cudaFreeHost(h->loop_pin);
  if (h->r0_pin) cudaFreeHost(h->r0_pin);
  if (h->loop.exec) cudaGraphExecDestroy(h->loop.exec);
  if (h->copy_in) cudaStreamSynchronize(h->copy_in);
  if (h->copy_out) cudaStreamSynchronize(h->copy_out);
  for (cudaEvent_t e : {h->ev_in, h->ev_taken, h->ev_staged, h->ev_sent})
    if (e) cudaEventDestroy(e);
  if (h->copy_in) cudaStreamDestroy(h->copy_in);
  if (h->copy_out) cudaStreamDestroy(h->copy_out);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return MGWR_OK;
}

int mgwr_create(int d, int n, int M, double T, double alpha, mgwr_t* out) {
  return create_impl(d, n, M, &T, &alpha, 1, out);
}

int mgwr_create_batch(int d, int n, int M, const double* T, const double* alpha, int batch,
                      mgwr_t* out) {
  return create_impl(d, n, M, T, alpha, batch, out);
}

int mgwr_set_problem(mgwr_t h, const double* T, const double* alpha) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (T == nullptr || alpha == nullptr) return fail(h, MGWR_E_INVAL, "null T or alpha");
  for (int b = 0; b < h->B; ++b) {
    if (!(T[b] > 0.0) || !std::isfinite(T[b]) || !(alpha[b] > 0.0) || !(alpha[b] <= 1.0))
      return fail(h, MGWR_E_INVAL, "need T > 0 finite and 0 < alpha <= 1");
  }
  bool same = true;
  for (int b = 0; b < h->B; ++b) same = same && T[b] == h->T[b] && alpha[b] == h->alpha[b];
  h->r0_valid = false;
  if (same) return MGWR_OK;  // the setup of this (T, alpha) is already resident
  for (int b = 0; b < h->B; ++b) {
    h->T[b] = T[b];
    h->alpha[b] = alpha[b];
    h->c[b] = std::pow(T[b] / h->M, -alpha[b]) / std::tgamma(2.0 - alpha[b]);
  }
  MGWR_TRY(setup_columns(h));
  return refresh_derived(h);
}

int mgwr_batch_size(mgwr_t h, int* batch) {
  if (h == nullptr || batch == nullptr) return MGWR_E_INVAL;
  *batch = h->B;
  return MGWR_OK;
}

int mgwr_instance_relres(mgwr_t h, double* relres) {
  if (h == nullptr || relres == nullptr) return MGWR_E_INVAL;
  std::copy(h->relres.begin(), h->relres.end(), relres);
  return MGWR_OK;
}

namespace {
bool known_precision(int p) {
  return p == MGWR_FP64 || p == MGWR_MIXED || p == MGWR_MIXED_DD || p == MGWR_DD || p == MGWR_AUTO;
}
// FP32 rounding of a correction e limits what one outer step of the FP32
// refinement can remove to about 4 eps32 / (pi h)^2 of the defect (the ratio of
// the discrete Laplacian's largest to smallest eigenvalue times eps32); from
// 0.2 on (h <= 1/4096) the outer steps cost more than double-float inner cycles,
// whose reduction per step is that of FP64 cycles.
constexpr double kAutoLimit = 0.2;
int resolve_precision(int n, int precision) {
  if (precision != MGWR_AUTO) return precision;
  const double h = 1.0 / ((double)n + 1.0);
  const double pi = 3.14159265358979323846;
  const double limit = 4.0 * 0x1p-24 / (pi * pi * h * h);
  return limit >= kAutoLimit ? MGWR_DD : MGWR_MIXED_DD;
}
}  // namespace

int mgwr_auto_precision(int d, int n, int M, int precision, int* resolved) {
  if (resolved == nullptr || (d != 1 && d != 2) || n < 1 || !is_pow2((long long)n + 1) ||
      !is_pow2(M) || M < 4 || M > mgwr::kMaxM || !known_precision(precision))
    return MGWR_E_INVAL;
  *resolved = resolve_precision(n, precision);
  return MGWR_OK;
}

int mgwr_get_precision(mgwr_t h, int* precision) {
  if (h == nullptr || precision == nullptr) return MGWR_E_INVAL;
  *precision = h->precision;
  return MGWR_OK;
}

int mgwr_set_precision(mgwr_t h, int precision) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (known_precision(precision)) precision = resolve_precision(h->n, precision);
  if (precision != MGWR_FP64 && precision != MGWR_MIXED && precision != MGWR_MIXED_DD &&
      precision != MGWR_DD)
    return fail(h, MGWR_E_INVAL,
                "precision must be MGWR_FP64, MGWR_MIXED, MGWR_MIXED_DD, MGWR_DD or MGWR_AUTO");
  if (precision == MGWR_DD) MGWR_TRY(ensure_hdd(h));
  if (precision == MGWR_MIXED || precision == MGWR_MIXED_DD) {
    MGWR_TRY(ensure_h32(h));
    // the double-float outer defect of MGWR_MIXED, for the carried form
    // (MGWR_MIXED_DD keeps its own in the FP64 iterate's field during a solve)
    // and the double-float spectra of its anchors (launch_defect_anchor)
    if (precision == MGWR_MIXED && h->M <= mgwr::kShortMaxM) {
      MGWR_TRY(ensure_field(h, &h->r_outer, level_count(h, h->nlev - 1)));
      MGWR_TRY(ensure_dd_spectra(h));
      MGWR_CK(h, cudaStreamSynchronize(h->stream));
    }
  }
  if (precision == MGWR_MIXED_DD) {
    MGWR_TRY(ensure_dd(h));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
  }
  h->precision = precision;
  return MGWR_OK;
}

int mgwr_set_order(mgwr_t h, int order) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (order != MGWR_ORDER_TEXT && order != MGWR_ORDER_TABLE)
    return fail(h, MGWR_E_INVAL, "order must be MGWR_ORDER_TEXT or MGWR_ORDER_TABLE");
  h->order = order;
  return MGWR_OK;
}

int mgwr_set_stream(mgwr_t h, void* stream) {
  if (h == nullptr) return MGWR_E_INVAL;
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  h->stream = stream != nullptr ? static_cast<cudaStream_t>(stream) : h->own_stream;
  return MGWR_OK;
}

int mgwr_set_graphs(mgwr_t h, int enable) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->use_graphs = enable != 0;
  return MGWR_OK;
}

int mgwr_set_device_loop(mgwr_t h, int enable) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->use_device_loop = enable != 0;
  return MGWR_OK;
}

int mgwr_set_engine_split(mgwr_t h, int kernel_class, int level, int split) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (kernel_class != MGWR_K_SWEEP64 && kernel_class != MGWR_K_SWEEP32 &&
      kernel_class != MGWR_K_DEFECT64 && kernel_class != MGWR_K_DEFECT32 &&
      kernel_class != MGWR_K_DEFECT_DD && kernel_class != MGWR_K_SWEEP_DD)
    return fail(h, MGWR_E_INVAL, "kernel class has no FFT engine");
  const int variants = mgwr::kStaged | mgwr::kTensor | mgwr::kRadix;
  const int E = split & ~variants;
  if (E != 1 && E != 2 && E != 4) return fail(h, MGWR_E_INVAL, "split must be 1, 2 or 4");
  if ((split & variants) && kernel_class != MGWR_K_SWEEP32)
    return fail(h, MGWR_E_INVAL, "staged, tensor-core and register-pass sweeps exist for FP32 only");
  const int v = split & variants;
  if (v != 0 && (v & (v - 1)) != 0)
    return fail(h, MGWR_E_INVAL, "staged, tensor-core and register-pass sweeps are exclusive");
  if (level < -1 || level >= h->nlev) return fail(h, MGWR_E_INVAL, "level out of range");
  if (level == -1)
    h->split[kernel_class].assign(h->nlev, split);
  else
    set_split(h, kernel_class, level, split);
  drop_graph(h);
  return MGWR_OK;
}

int mgwr_get_engine_split(mgwr_t h, int kernel_class, int level, int* split) {
  if (h == nullptr || split == nullptr || kernel_class < 0 ||
      kernel_class >= MGWR_NUM_KERNEL_CLASSES || level < -1 || level >= h->nlev)
    return MGWR_E_INVAL;
  const int word = kernel_class == MGWR_K_SWEEP32 || kernel_class == MGWR_K_DEFECT32 ? 4 : 8;
  *split = mgwr::effective_split(h->M, word,
                                 split_of(h, kernel_class, level == -1 ? h->nlev - 1 : level));
  return MGWR_OK;
}

int mgwr_autotune(mgwr_t h) {
  if (h == nullptr) return MGWR_E_INVAL;
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  if (h->precision == MGWR_FP64) {
    MGWR_TRY(tune_hierarchy(h, h->h64, MGWR_K_SWEEP64, MGWR_K_DEFECT64));
  } else if (h->precision == MGWR_DD) {
    MGWR_TRY(tune_hierarchy(h, h->hdd, MGWR_K_SWEEP_DD, MGWR_K_DEFECT_DD));
  } else {
    MGWR_TRY(tune_hierarchy(h, h->h32, MGWR_K_SWEEP32, MGWR_K_DEFECT32));
    MGWR_TRY(tune_outer(h));
  }
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  drop_graph(h);
  return check_staging(h);
}

int mgwr_set_outer_switch(mgwr_t h, double rel) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (!(rel >= 0.0)) return fail(h, MGWR_E_INVAL, "the switch must be a number >= 0");
  h->loose_above = rel;
  return MGWR_OK;
}

int mgwr_set_inner_cycles(mgwr_t h, int cycles) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (cycles < 1 || cycles > 16) return fail(h, MGWR_E_INVAL, "inner cycles must be in 1..16");
  h->inner = cycles;
  return MGWR_OK;
}

static int set_rhs_impl(mgwr_t h, const double* f, const double* g, cudaMemcpyKind kind) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (f == nullptr) return fail(h, MGWR_E_INVAL, "f must not be null");
  const int L = h->nlev - 1;
  const size_t N = points(h, L);
  const size_t bytes = level_count(h, L) * sizeof(double);
  MGWR_CK(h, cudaMemcpyAsync(h->h64.f[L], f, bytes, kind, h->stream));
  if (g != nullptr) {
    double* g_dev = nullptr;
    MGWR_TRY(dev_alloc(h, &g_dev, N * h->B * sizeof(double)));
    MGWR_CK(h, cudaMemcpyAsync(g_dev, g, N * h->B * sizeof(double), kind, h->stream));
    MGWR_CK(h, mgwr::launch_initial(h->h64.u[L], h->h64.f[L], g_dev, h->dk, h->c_dev, (int)N, h->M,
                                     h->B, h->stream));
    MGWR_CK(h, cudaFreeAsync(g_dev, h->stream));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
    h->allocs.pop_back();
  } else {
    MGWR_CK(h, cudaMemsetAsync(h->h64.u[L], 0, bytes, h->stream));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
  }
  h->u_zero = g == nullptr;
  h->r0_valid = false;
  h->h64.rs[L] = R_STALE;
  return MGWR_OK;
}

int mgwr_set_rhs(mgwr_t h, const double* f, const double* g) {
  return set_rhs_impl(h, f, g, cudaMemcpyHostToDevice);
}

int mgwr_set_rhs_dev(mgwr_t h, const double* f_dev, const double* g_dev) {
  return set_rhs_impl(h, f_dev, g_dev, cudaMemcpyDeviceToDevice);
}

int mgwr_set_initial(mgwr_t h, const double* u0) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  if (u0 == nullptr) return fail(h, MGWR_E_INVAL, "u0 must not be null");
  const int L = h->nlev - 1;
  MGWR_CK(h, cudaMemcpyAsync(h->h64.u[L], u0, level_count(h, L) * sizeof(double),
                             cudaMemcpyHostToDevice, h->stream));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  h->r0_valid = false;
  h->h64.rs[L] = R_STALE;
  return MGWR_OK;
}

}  // extern "C"

namespace {

// State of one solve between its iterations: the loop of mgwr_solve, split so
// that a group of handles can run each iteration of all its members as one
// graph launch (mgwr_group_*) with exactly the launches a solo solve makes.
struct SolveState {
  int cyc = 1, nu1 = 1, nu2 = 1, max_cycles = 1;
  double tol = 0.0;
  bool mixed = false, ddef = false, ddc = false;
  double rel = 0.0;
  int status = MGWR_OK;
  int cycles = 0, outer = 0;
  bool rel_exact = true;  // rel comes from the full defect (not from smoothing changes)
  // refinements: defect reduction of the last outer step and its inner cycles
  double last_q = 0.0;
  int last_k = 0;
  // mixed modes: per-instance relative defect at the last full outer defect
  // (the anchor of the carried defects since)
  std::vector<double> anchor;
  // the iteration being run
  double rel_before = 0.0;
  int k_now = 1;
  std::vector<double> norms;
};

// The full defect of the finest level in the outer precision, with norms (in
// the refinements written as the inner right-hand side).
int solve_full_defect(mgwr_t h, SolveState& S) {
  if (S.mixed && anchor_ok(h, S.tol)) {
    MGWR_TRY(clear_norms(h));
    MGWR_TRY(enqueue_anchor(h));
    return read_norms(h, S.norms);
  }
  if (S.ddc) {
    MGWR_TRY(clear_norms(h));
    MGWR_TRY(outer_defect_ddd(h));
    return read_norms(h, S.norms);
  }
  if (S.ddef) return finest_defect_norms_dd(h, S.norms);
  return finest_defect_norms(h, S.norms, S.mixed);
}

// Checks the arguments, starts the timing and computes the initial defect and
// its norms (synchronises the handle's stream).
int solve_begin(mgwr_t h, SolveState& S, int cyc, int nu1, int nu2, double tol, int max_cycles) {
  MGWR_TRY(check_cycle_args(h, cyc, nu1, nu2));
  if (!(tol >= 0.0) || max_cycles < 1) return fail(h, MGWR_E_INVAL, "need tol >= 0, max_cycles >= 1");
  S = SolveState{};
  S.cyc = cyc;
  S.nu1 = nu1;
  S.nu2 = nu2;
  S.tol = tol;
  S.max_cycles = max_cycles;
  // refinement: inner cycles on the defect equation (FP32 or double-float),
  // the outer defect in FP64 or double-float
  S.mixed = h->precision != MGWR_FP64;
  S.ddef = h->precision == MGWR_MIXED_DD || h->precision == MGWR_DD;
  S.ddc = h->precision == MGWR_DD;  // double-float inner cycles
  if (h->precision == MGWR_FP64) MGWR_TRY(ensure_full(h, h->h64));
  const int L = h->nlev - 1;
  const size_t cntL = level_count(h, L);
  MGWR_CK(h, cudaEventRecord(h->ev0, h->stream));
  if (S.ddef) {
    MGWR_CK(h, mgwr::launch_split(h->u_dd, h->h64.u[L], cntL, h->stream));
    if (!h->u_zero) MGWR_CK(h, mgwr::launch_split(h->f_dd, h->h64.f[L], cntL, h->stream));
  }
  if (h->u_zero) {
    // the defect of u = 0 is f itself (Algorithm 1 from the zero iterate): its
    // norm, its FP32 rounding for the first inner cycles and its double-float
    // split (f_dd, or the outer defect MGWR_MIXED carries from) in one pass
    MGWR_TRY(clear_norms(h));
    mgwr::dd* fdd = S.ddef ? h->f_dd
                    : (S.mixed && !S.ddc && carries(h)) ? outer_field(h)
                                                        : nullptr;
    MGWR_CK(h, mgwr::launch_absmax_round(h->h64.f[L], S.mixed && !S.ddc ? h->h32.f[L] : nullptr,
                                         fdd, cntL / h->B, h->B, h->norm_bits, h->stream));
    if (S.ddc) {
      MGWR_CK(h, mgwr::launch_split(h->hdd.f[L], h->h64.f[L], cntL, h->stream));
      h->hdd.rs[L] = R_STALE;
    } else if (S.mixed) {
      h->h32.rs[L] = R_STALE;
    } else {
      h->h64.rs[L] = R_ZERO_U;
    }
    MGWR_TRY(read_norms(h, S.norms));
  } else {
    MGWR_TRY(solve_full_defect(h, S));
  }
  if (!h->r0_valid) {
    h->r0 = S.norms;
    h->r0_valid = true;
  }
  S.rel = relative(h, S.norms, h->relres);
  // the outer defect to carry from: from u = 0 f itself (f_dd in MGWR_MIXED_DD;
  // split into outer_field in MGWR_MIXED), else the full defect just computed
  // (kept in outer_field by enqueue_outer_full)
  h->outer_src = -1;
  if (S.mixed && !S.ddc && carries(h))
    h->outer_src = h->u_zero && S.ddef ? 0 : 1;  // from u = 0: split above
  S.anchor = h->relres;
  return MGWR_OK;
}

// Mixed modes: whether the next outer defect may be carried by the step's
// correction.  Its error is about 1e-6 of the anchor (the defect at the last
// full computation); every instance must still be at least the switch times
// its anchor, or have an anchor so small against the tolerance that the
// carried error cannot decide its stopping test (which the full defect
// confirms anyway).
bool carry_next(const mgwr_handle* h, const SolveState& S) {
  if (!S.mixed || S.ddc || h->outer_src < 0) return false;
  const double x = h->loose_above;
  for (int b = 0; b < h->B; ++b) {
    const double a = x * S.anchor[b];
    if (!(h->relres[b] >= a || a <= S.tol)) return false;
  }
  return true;
}

// Decides whether another iteration runs (false: the loop ends, S.status set)
// and prepares its form on the handle (outer-defect form, inner cycles).
bool solve_plan(mgwr_t h, SolveState& S) {
  if (S.rel <= S.tol) return false;
  if (!std::isfinite(S.rel)) {
    S.status = MGWR_E_NUMERIC;
    return false;
  }
  if ((S.mixed ? S.outer : S.cycles) >= S.max_cycles) {
    S.status = MGWR_E_NOCONV;
    return false;
  }
  // outer defects of the mixed modes carried by the correction while the
  // defect is large against the anchor (mgwr_set_outer_switch)
  h->outer_form = carry_next(h, S)    ? kOuterCarry
                   : anchor_ok(h, S.tol) ? kOuterAnchor
                                       : kOuterFull;
  // Refinements: when the last step's reduction predicts that this step ends
  // just above the tolerance, but below half of it with one cycle more, this
  // step takes that cycle instead of leaving a whole outer step (and its outer
  // defect) for it.  One more cycle gains the last step's mean reduction per
  // cycle only down to the floor of the inner precision: the rounding of the
  // correction e (eps |e|) has a defect of about 4d/h^2 eps |e| against the
  // smooth defect d pi^2 |e| left after a cycle, so no outer step reduces the
  // defect below about 4 eps / (pi h)^2 (FP32: 6e-3 at h = 1/512).
  h->inner_now = 0;
  if (S.mixed && S.last_k > 0 && S.last_q > 0.0 && S.last_q < 1.0) {
    const int k = inner_cycles(h);
    const double per_cycle = std::pow(S.last_q, 1.0 / S.last_k);
    const double hf = 1.0 / (h->n + 1);
    const double eps = S.ddc ? std::ldexp(1.0, -44) : std::ldexp(1.0, -24);
    const double pi = 3.14159265358979323846;
    const double floor_q = 4.0 * eps / (pi * pi * hf * hf);
    const double q_more = std::max(S.last_q * per_cycle, floor_q);
    if (S.rel * S.last_q > S.tol && S.rel * q_more <= 0.5 * S.tol) h->inner_now = k + 1;
  }
  S.rel_before = S.rel;
  S.k_now = S.mixed ? step_cycles(h) : 1;
  return true;
}

// Takes in the norms an iteration left in the handle's pinned buffer (the
// stream is synchronised); the stopping decision is always taken on the full
// defect, computed here when the iteration's norms came from smoothing changes.
int solve_after(mgwr_t h, SolveState& S, bool exact) {
  h->inner_now = 0;
  S.norms.resize(h->B);
  for (int b = 0; b < h->B; ++b) std::memcpy(&S.norms[b], &h->norm_host[b], sizeof(double));
  S.cycles += S.k_now;
  S.rel = relative(h, S.norms, h->relres);
  if (S.mixed && S.rel_before > 0.0) {
    S.last_q = S.rel / S.rel_before;
    S.last_k = S.k_now;
  }
  const bool mixed_outer = S.mixed && !S.ddc;
  if (mixed_outer) {
    // outer_field now holds the step's outer defect (carried or full)
    h->outer_src = carries(h) ? 1 : -1;
    if (exact) S.anchor = h->relres;
  }
  h->outer_form = kOuterFull;
  if (!exact && S.rel <= S.tol) {
    MGWR_TRY(solve_full_defect(h, S));
    S.rel = relative(h, S.norms, h->relres);
    exact = true;
    if (mixed_outer) S.anchor = h->relres;
  }
  S.rel_exact = exact;
  ++S.outer;
  return MGWR_OK;
}

// Builds the device loop of the current iteration form: a WHILE node whose body
// is one iteration without the copy of its norms and k_loop_decide.  The body's
// iteration must leave the finest state as it found it (the same
// iteration_key), so that every pass of the loop runs the launches of the host
// loop's replayed iterations; otherwise the key is marked unusable.
int build_device_loop(mgwr_t h, int cyc, int nu1, int nu2, long long key) {
  if (h->loop.exec != nullptr) cudaGraphExecDestroy(h->loop.exec);
  h->loop = mgwr_handle::LoopGraph{};
  h->loop.key = key;
  cudaGraph_t g = nullptr;
  MGWR_CK(h, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    MGWR_CK(h, e);
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    MGWR_CK(h, e);
  }
  // the capture updates the hierarchies' defect states as if the iteration ran
  const RsState pre = save_rs(h);
  bool ex = true;
  const long long before = mgwr::launch_counter();
  int st = enqueue_iteration(h, cyc, nu1, nu2, &ex, false);
  if (st == MGWR_OK)
    st = mgwr::launch_loop_decide(h->norm_bits, h->r0_dev, h->B, h->loop_dev, cond, h->stream) ==
                 cudaSuccess
             ? MGWR_OK
             : MGWR_E_CUDA;
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(h->stream, &captured);
  const long long kernels = mgwr::launch_counter() - before;
  mgwr::add_launches(-kernels);  // captured launches run when the graph does
  if (st != MGWR_OK || e != cudaSuccess) {
    cudaGraphDestroy(g);
    if (st != MGWR_OK) return st;
    MGWR_CK(h, e);
  }
  const bool uniform = iteration_key(h, cyc, nu1, nu2) == key && h->h64.rs == pre.r64 &&
                       h->h32.rs == pre.r32 && h->hdd.rs == pre.rdd;
  if (!uniform) {  // keep the host loop, and the states the capture changed
    cudaGraphDestroy(g);
    load_rs(h, pre);
    h->loop.unusable = true;
    return MGWR_OK;
  }
  e = cudaGraphInstantiate(&h->loop.exec, g, 0);
  cudaGraphDestroy(g);
  MGWR_CK(h, e);
  h->loop.exact = ex;
  h->loop.kernels = kernels;
  return MGWR_OK;
}

// MGWR_FP64 with graphs: runs the remaining iterations of the solve as one
// graph launch (the device decides when to stop, within max_cycles), then takes
// in the last norms and the iteration count as solve_after would.  *ran =
// false when the form has no device loop (the caller runs the host loop).
int run_device_loop(mgwr_t h, SolveState& S, bool* ran) {
  *ran = false;
  const int left = S.max_cycles - S.cycles;
  if (h->precision != MGWR_FP64 || !h->use_graphs || !h->use_device_loop || h->profiling ||
      left < 2)
    return MGWR_OK;
  const long long key = iteration_key(h, S.cyc, S.nu1, S.nu2);
  if (h->loop.key == key && h->loop.unusable) return MGWR_OK;
  if (h->loop_dev == nullptr) {
    MGWR_TRY(dev_alloc(h, &h->loop_dev, sizeof(mgwr::LoopState)));
    MGWR_TRY(dev_alloc(h, &h->r0_dev, sizeof(double) * h->B));
    if (cudaMallocHost(&h->loop_pin, sizeof(mgwr::LoopState)) != cudaSuccess ||
        cudaMallocHost(&h->r0_pin, sizeof(double) * h->B) != cudaSuccess)
      return fail(h, MGWR_E_NOMEM, "pinned loop state");
  }
  if (h->loop.key != key || h->loop.exec == nullptr) {
    MGWR_TRY(build_device_loop(h, S.cyc, S.nu1, S.nu2, key));
    if (h->loop.unusable) return MGWR_OK;
  }
  for (int b = 0; b < h->B; ++b) h->r0_pin[b] = h->r0[b];
  MGWR_CK(h, cudaMemcpyAsync(h->r0_dev, h->r0_pin, sizeof(double) * h->B, cudaMemcpyHostToDevice,
                             h->stream));
  MGWR_CK(h, mgwr::launch_loop_init(h->loop_dev, S.tol, left, h->stream));
  MGWR_CK(h, cudaGraphLaunch(h->loop.exec, h->stream));
  MGWR_CK(h, cudaMemcpyAsync(h->loop_pin, h->loop_dev, sizeof(mgwr::LoopState),
                             cudaMemcpyDeviceToHost, h->stream));
  std::vector<double> norms;
  MGWR_TRY(read_norms(h, norms));  // synchronises the stream
  const int iters = h->loop_pin->iters;
  mgwr::add_launches(h->loop.kernels * iters);
  *ran = true;
  S.norms = norms;
  S.cycles += iters;
  S.outer += iters;
  S.rel = relative(h, S.norms, h->relres);
  bool exact = h->loop.exact;
  if (!exact && S.rel <= S.tol) {  // the stop is decided on the full defect
    MGWR_TRY(solve_full_defect(h, S));
    S.rel = relative(h, S.norms, h->relres);
    exact = true;
  }
  S.rel_exact = exact;
  return MGWR_OK;
}

// Ends a solve: the iterate back in FP64, the full defect when the last norms
// were not, the timing and the statistics.
int solve_end(mgwr_t h, SolveState& S, mgwr_stats* st) {
  const int L = h->nlev - 1;
  const size_t cntL = level_count(h, L);
  h->u_zero = false;
  h->outer_form = kOuterFull;
  h->outer_src = -1;
  if (S.ddef) MGWR_CK(h, mgwr::launch_join(h->h64.u[L], h->u_dd, cntL, h->stream));
  if (!S.rel_exact) {  // report the full defect also when stopping on max_cycles
    MGWR_TRY(finest_defect_norms(h, S.norms, false));
    S.rel = relative(h, S.norms, h->relres);
  }
  int status = S.status;
  if (!std::isfinite(S.rel)) status = MGWR_E_NUMERIC;
  MGWR_CK(h, cudaEventRecord(h->ev1, h->stream));
  MGWR_CK(h, cudaEventSynchronize(h->ev1));
  MGWR_TRY(check_staging(h));
  prof_collect(h);
  float ms = 0.f;
  MGWR_CK(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  mgwr_stats local{};
  local.cycles = S.cycles;
  local.outer = S.outer;
  local.relres = S.rel;
  local.factor = S.cycles > 0 && S.rel > 0.0 ? std::pow(S.rel, 1.0 / S.cycles) : 0.0;
  local.seconds = ms * 1e-3;
  if (st != nullptr) *st = local;
  if (status == MGWR_E_NOCONV) h->err = "max_cycles reached before the tolerance";
  if (status == MGWR_E_NUMERIC) h->err = "non-finite residual norm";
  return status;
}

}  // namespace

extern "C" {

int mgwr_solve(mgwr_t h, int cyc, int nu1, int nu2, double tol, int max_cycles, mgwr_stats* st) {
  if (h == nullptr) return MGWR_E_INVAL;
  SolveState S;
  MGWR_TRY(solve_begin(h, S, cyc, nu1, nu2, tol, max_cycles));
  while (solve_plan(h, S)) {
    if (S.cycles >= 1) {  // past the first iteration, whose start differs from u = 0
      bool ran = false;
      MGWR_TRY(run_device_loop(h, S, &ran));
      if (ran) continue;
    }
    bool exact = true;
    std::vector<double> unused;
    MGWR_TRY(run_iteration(h, cyc, nu1, nu2, unused, &exact));
    MGWR_TRY(solve_after(h, S, exact));
  }
  return solve_end(h, S, st);
}

}  // extern "C"

// A group of handles solved together: each member runs exactly the launches of
// its own solve (mgwr_solve), and every iteration of all running members is
// one CUDA graph launch whose branches, one per member, run concurrently on
// the device.  Members may differ in every setting (d, n, M, batch, precision,
// cycle); they join and leave between iterations.
struct mgwr_group {
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;
  struct Member {
    mgwr_t h = nullptr;
    SolveState S;
    cudaEvent_t join = nullptr;
  };
  std::vector<Member> running;
  struct Done {
    mgwr_t h;
    int status;
    mgwr_stats st;
  };
  std::deque<Done> finished;
  // instantiated iteration graphs by the (member, iteration key) list they serve
  struct Entry {
    std::vector<std::pair<mgwr_t, long long>> key;
    cudaGraphExec_t exec = nullptr;
    std::vector<char> exact;
    std::vector<RsState> after;  // per member: the defect states its iteration leaves
    long long kernels = 0;
    unsigned long long used = 0;
  };
  std::vector<Entry> graphs;
  unsigned long long clock = 0;
  long long launches = 0, member_iterations = 0;
  int max_members = 0;
  std::string err;
};

namespace {

constexpr size_t kGroupGraphs = 8;

void group_drop_graphs_of(mgwr_group* g, mgwr_t h) {
  for (size_t i = 0; i < g->graphs.size();) {
    bool uses = false;
    for (const auto& k : g->graphs[i].key) uses = uses || k.first == h;
    if (uses) {
      cudaGraphExecDestroy(g->graphs[i].exec);
      g->graphs.erase(g->graphs.begin() + i);
    } else {
      ++i;
    }
  }
}

void group_finish(mgwr_group* g, size_t i, int status) {
  mgwr_group::Member& m = g->running[i];
  mgwr_stats st{};
  int code = status;
  if (code == MGWR_OK) code = solve_end(m.h, m.S, &st);
  group_drop_graphs_of(g, m.h);
  cudaEventDestroy(m.join);
  g->finished.push_back({m.h, code, st});
  g->running.erase(g->running.begin() + i);
}

// Captures one iteration of every running member (their launches on their own
// streams, forked from and joined to the group's stream) as one graph.
int group_capture(mgwr_group* g, mgwr_group::Entry& e) {
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    g->err = cudaGetErrorString(ce);
    return MGWR_E_CUDA;
  }
  const long long before = mgwr::launch_counter();
  int st = MGWR_OK;
  if (cudaEventRecord(g->fork, g->stream) != cudaSuccess) st = MGWR_E_CUDA;
  e.exact.assign(g->running.size(), 1);
  for (size_t i = 0; i < g->running.size() && st == MGWR_OK; ++i) {
    mgwr_group::Member& m = g->running[i];
    const mgwr_group::Member& mm = m;
    if (cudaStreamWaitEvent(m.h->stream, g->fork, 0) != cudaSuccess) {
      st = MGWR_E_CUDA;
      break;
    }
    bool ex = true;
    st = enqueue_iteration(m.h, mm.S.cyc, mm.S.nu1, mm.S.nu2, &ex);
    e.exact[i] = ex ? 1 : 0;
    e.after.push_back(save_rs(m.h));
    if (st == MGWR_OK && (cudaEventRecord(m.join, m.h->stream) != cudaSuccess ||
                          cudaStreamWaitEvent(g->stream, m.join, 0) != cudaSuccess))
      st = MGWR_E_CUDA;
  }
  ce = cudaStreamEndCapture(g->stream, &graph);
  const long long captured = mgwr::launch_counter() - before;
  mgwr::add_launches(-captured);  // counted when the graph runs
  if (st == MGWR_OK && ce != cudaSuccess) st = MGWR_E_CUDA;
  if (st == MGWR_OK && cudaGraphInstantiate(&e.exec, graph, 0) != cudaSuccess) st = MGWR_E_CUDA;
  if (graph != nullptr) cudaGraphDestroy(graph);
  if (st != MGWR_OK) {
    cudaGetLastError();
    g->err = "capture of the group iteration failed";
    return st;
  }
  e.kernels = captured;
  return MGWR_OK;
}

}  // namespace

extern "C" {

int mgwr_group_create(mgwr_group_t* out) {
  if (out == nullptr) return MGWR_E_INVAL;
  *out = nullptr;
  mgwr_group_t g = new (std::nothrow) mgwr_group;
  if (g == nullptr) return MGWR_E_NOMEM;
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    mgwr_group_destroy(g);
    return MGWR_E_CUDA;
  }
  *out = g;
  return MGWR_OK;
}

int mgwr_group_destroy(mgwr_group_t g) {
  if (g == nullptr) return MGWR_OK;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (auto& e : g->graphs) cudaGraphExecDestroy(e.exec);
  for (auto& m : g->running) cudaEventDestroy(m.join);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->stream) cudaStreamDestroy(g->stream);
  cudaGetLastError();
  delete g;
  return MGWR_OK;
}

const char* mgwr_group_last_error(mgwr_group_t g) {
  return g == nullptr ? "null group" : g->err.c_str();
}

int mgwr_group_add(mgwr_group_t g, mgwr_t h, int cyc, int nu1, int nu2, double tol,
                   int max_cycles) {
  if (g == nullptr || h == nullptr) return MGWR_E_INVAL;
  if (h->profiling) return fail(h, MGWR_E_STATE, "a profiled handle cannot join a group");
  for (const auto& m : g->running)
    if (m.h == h || m.h->stream == h->stream)
      return fail(h, MGWR_E_STATE, "the handle, or its stream, is already in the group");
  mgwr_group::Member m;
  m.h = h;
  MGWR_TRY(solve_begin(h, m.S, cyc, nu1, nu2, tol, max_cycles));
  if (cudaEventCreateWithFlags(&m.join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MGWR_E_CUDA, "event creation failed");
  }
  g->running.push_back(m);
  return MGWR_OK;
}

int mgwr_group_step(mgwr_group_t g, int* running) {
  if (g == nullptr) return MGWR_E_INVAL;
  // members whose solve has ended leave; the others prepare their next iteration
  for (size_t i = 0; i < g->running.size();) {
    if (!solve_plan(g->running[i].h, g->running[i].S))
      group_finish(g, i, MGWR_OK);
    else
      ++i;
  }
  if (g->running.empty()) {
    if (running != nullptr) *running = 0;
    return MGWR_OK;
  }
  std::vector<std::pair<mgwr_t, long long>> key;
  for (const auto& m : g->running)
    key.emplace_back(m.h, iteration_key(m.h, m.S.cyc, m.S.nu1, m.S.nu2));
  mgwr_group::Entry* e = nullptr;
  for (auto& c : g->graphs)
    if (c.key == key) e = &c;
  if (e == nullptr) {
    if (g->graphs.size() >= kGroupGraphs) {  // the least recently used one goes
      size_t old = 0;
      for (size_t i = 1; i < g->graphs.size(); ++i)
        if (g->graphs[i].used < g->graphs[old].used) old = i;
      cudaGraphExecDestroy(g->graphs[old].exec);
      g->graphs.erase(g->graphs.begin() + old);
    }
    mgwr_group::Entry fresh;
    fresh.key = key;
    MGWR_TRY(group_capture(g, fresh));
    g->graphs.push_back(std::move(fresh));
    e = &g->graphs.back();
  }
  e->used = ++g->clock;
  for (size_t i = 0; i < g->running.size(); ++i) load_rs(g->running[i].h, e->after[i]);
  cudaError_t ce = cudaGraphLaunch(e->exec, g->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(g->stream);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    g->err = cudaGetErrorString(ce);
    return MGWR_E_CUDA;
  }
  mgwr::add_launches(e->kernels);
  g->launches++;
  g->member_iterations += (long long)g->running.size();
  g->max_members = std::max(g->max_members, (int)g->running.size());
  const std::vector<char> exact = e->exact;
  for (size_t i = 0, k = 0; i < g->running.size(); ++k) {
    const int st = solve_after(g->running[i].h, g->running[i].S, exact[k] != 0);
    if (st != MGWR_OK)
      group_finish(g, i, st);
    else
      ++i;
  }
  if (running != nullptr) *running = (int)g->running.size();
  return MGWR_OK;
}

int mgwr_group_collect(mgwr_group_t g, mgwr_t* h, int* status, mgwr_stats* st) {
  if (g == nullptr || h == nullptr) return MGWR_E_INVAL;
  if (g->finished.empty()) return MGWR_E_AGAIN;
  const mgwr_group::Done d = g->finished.front();
  g->finished.pop_front();
  *h = d.h;
  if (status != nullptr) *status = d.status;
  if (st != nullptr) *st = d.st;
  return MGWR_OK;
}

int mgwr_group_info(mgwr_group_t g, long long* launches, long long* member_iterations,
                    int* max_members) {
  if (g == nullptr) return MGWR_E_INVAL;
  if (launches != nullptr) *launches = g->launches;
  if (member_iterations != nullptr) *member_iterations = g->member_iterations;
  if (max_members != nullptr) *max_members = g->max_members;
  return MGWR_OK;
}

int mgwr_group_solve(mgwr_t* handles, int count, int cyc, int nu1, int nu2, double tol,
                     int max_cycles, int* status, mgwr_stats* stats) {
  if (handles == nullptr || count < 1 || status == nullptr) return MGWR_E_INVAL;
  for (int i = 0; i < count; ++i)
    if (handles[i] == nullptr) return MGWR_E_INVAL;
  mgwr_group_t g = nullptr;
  MGWR_TRY(mgwr_group_create(&g));
  int st = MGWR_OK;
  for (int i = 0; i < count; ++i) {
    status[i] = mgwr_group_add(g, handles[i], cyc, nu1, nu2, tol, max_cycles);
    if (status[i] != MGWR_OK && st == MGWR_OK) st = status[i];
  }
  int left = 1;
  while (st == MGWR_OK && left > 0) st = mgwr_group_step(g, &left);
  mgwr_t h = nullptr;
  int code = 0;
  mgwr_stats one{};
  while (mgwr_group_collect(g, &h, &code, &one) == MGWR_OK) {
    for (int i = 0; i < count; ++i) {
      if (handles[i] != h) continue;
      status[i] = code;
      if (stats != nullptr) stats[i] = one;
    }
  }
  mgwr_group_destroy(g);
  return st;
}

int mgwr_residual(mgwr_t h, double* relres, double* r_host) {
  if (h == nullptr) return MGWR_E_INVAL;
  std::vector<double> norms;
  MGWR_TRY(finest_defect_norms(h, norms, false));
  if (!h->r0_valid) {
    h->r0 = norms;
    h->r0_valid = true;
  }
  const double rel = relative(h, norms, h->relres);
  if (relres != nullptr) *relres = rel;
  if (r_host != nullptr) {
    const int L = h->nlev - 1;
    MGWR_CK(h, cudaMemcpyAsync(r_host, h->h64.r[L], level_count(h, L) * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
  }
  return MGWR_OK;
}

// ---- pipelined transfers ---------------------------------------------------------

static int ensure_staging(mgwr_t h) {
  if (h->stage_in != nullptr) return MGWR_OK;
  const size_t cnt = level_count(h, h->nlev - 1);
  MGWR_TRY(dev_alloc(h, &h->stage_out, cnt * sizeof(double)));
  MGWR_TRY(dev_alloc(h, &h->stage_in, cnt * sizeof(double)));
  MGWR_CK(h, cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking));
  MGWR_CK(h, cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&h->ev_in, &h->ev_taken, &h->ev_staged, &h->ev_sent})
    MGWR_CK(h, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  // the staging buffers come from the handle's stream-ordered pool: the copy
  // streams may use them once that allocation has completed
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return MGWR_OK;
}

int mgwr_stage_rhs(mgwr_t h, const double* f_host) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (f_host == nullptr) return fail(h, MGWR_E_INVAL, "f must not be null");
  if (h->rhs_pending) return fail(h, MGWR_E_STATE, "a staged right-hand side is not taken yet");
  MGWR_TRY(ensure_staging(h));
  const size_t bytes = level_count(h, h->nlev - 1) * sizeof(double);
  MGWR_CK(h, cudaStreamWaitEvent(h->copy_in, h->ev_taken, 0));
  MGWR_CK(h, cudaMemcpyAsync(h->stage_in, f_host, bytes, cudaMemcpyHostToDevice, h->copy_in));
  MGWR_CK(h, cudaEventRecord(h->ev_in, h->copy_in));
  h->rhs_pending = true;
  return MGWR_OK;
}

int mgwr_take_rhs(mgwr_t h) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (!h->rhs_pending) return fail(h, MGWR_E_STATE, "no staged right-hand side");
  const int L = h->nlev - 1;
  const size_t bytes = level_count(h, L) * sizeof(double);
  MGWR_CK(h, cudaStreamWaitEvent(h->stream, h->ev_in, 0));
  MGWR_CK(h, cudaMemcpyAsync(h->h64.f[L], h->stage_in, bytes, cudaMemcpyDeviceToDevice, h->stream));
  MGWR_CK(h, cudaEventRecord(h->ev_taken, h->stream));
  MGWR_CK(h, cudaMemsetAsync(h->h64.u[L], 0, bytes, h->stream));
  h->rhs_pending = false;
  h->u_zero = true;
  h->r0_valid = false;
  h->h64.rs[L] = R_STALE;
  return MGWR_OK;
}

int mgwr_stage_solution(mgwr_t h, double* u_host) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (u_host == nullptr) return fail(h, MGWR_E_INVAL, "u must not be null");
  MGWR_TRY(ensure_staging(h));
  const int L = h->nlev - 1;
  const size_t bytes = level_count(h, L) * sizeof(double);
  MGWR_CK(h, cudaStreamWaitEvent(h->stream, h->ev_sent, 0));
  MGWR_CK(h, cudaMemcpyAsync(h->stage_out, h->h64.u[L], bytes, cudaMemcpyDeviceToDevice, h->stream));
  MGWR_CK(h, cudaEventRecord(h->ev_staged, h->stream));
  MGWR_CK(h, cudaStreamWaitEvent(h->copy_out, h->ev_staged, 0));
  MGWR_CK(h, cudaMemcpyAsync(u_host, h->stage_out, bytes, cudaMemcpyDeviceToHost, h->copy_out));
  MGWR_CK(h, cudaEventRecord(h->ev_sent, h->copy_out));
  return MGWR_OK;
}

int mgwr_wait_staged(mgwr_t h) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (h->copy_in != nullptr) MGWR_CK(h, cudaStreamSynchronize(h->copy_in));
  if (h->copy_out != nullptr) MGWR_CK(h, cudaStreamSynchronize(h->copy_out));
  return MGWR_OK;
}

int mgwr_get_solution(mgwr_t h, double* u_host) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (u_host == nullptr) return fail(h, MGWR_E_INVAL, "u must not be null");
  const int L = h->nlev - 1;
  MGWR_CK(h, cudaMemcpyAsync(u_host, h->h64.u[L], level_count(h, L) * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return MGWR_OK;
}

int mgwr_get_solution_dev(mgwr_t h, double* u_dev) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (u_dev == nullptr) return fail(h, MGWR_E_INVAL, "u must not be null");
  const int L = h->nlev - 1;
  MGWR_CK(h, cudaMemcpyAsync(u_dev, h->h64.u[L], level_count(h, L) * sizeof(double),
                             cudaMemcpyDeviceToDevice, h->stream));
  return MGWR_OK;
}

int mgwr_num_levels(mgwr_t h, int* levels) {
  if (h == nullptr || levels == nullptr) return MGWR_E_INVAL;
  *levels = h->nlev;
  return MGWR_OK;
}

int mgwr_level_n(mgwr_t h, int level, int* n_level) {
  if (h == nullptr || n_level == nullptr) return MGWR_E_INVAL;
  if (level < 0 || level >= h->nlev) return fail(h, MGWR_E_INVAL, "level out of range");
  *n_level = h->nl[level];
  return MGWR_OK;
}

static void* field_ptr(mgwr_t h, int hierarchy, int level, int which) {
  void* p = nullptr;
  with_hier(h, hierarchy, [&](auto& H) {
    p = which == MGWR_U ? (void*)H.u[level] : which == MGWR_F ? (void*)H.f[level] : (void*)H.r[level];
    return MGWR_OK;
  });
  return p;
}

int mgwr_field_set(mgwr_t h, int hierarchy, int level, int which, const double* host) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  MGWR_TRY(check_level(h, hierarchy, level));
  if (which < MGWR_U || which > MGWR_R || host == nullptr)
    return fail(h, MGWR_E_INVAL, "bad field or null pointer");
  const size_t cnt = level_count(h, level);
  void* dst = field_ptr(h, hierarchy, level, which);
  if (hierarchy == MGWR_H64) {
    MGWR_CK(h, cudaMemcpyAsync(dst, host, cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  } else if (hierarchy == MGWR_H32) {
    std::vector<float> tmp(cnt);
    for (size_t i = 0; i < cnt; ++i) tmp[i] = (float)host[i];
    MGWR_CK(h, cudaMemcpyAsync(dst, tmp.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
  } else {
    std::vector<mgwr::dd> tmp(cnt);
    for (size_t i = 0; i < cnt; ++i) {
      const float hi = (float)host[i];
      tmp[i] = mgwr::dd(hi, (float)(host[i] - (double)hi));
    }
    MGWR_CK(h, cudaMemcpyAsync(dst, tmp.data(), cnt * sizeof(mgwr::dd), cudaMemcpyHostToDevice,
                               h->stream));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
  }
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  if (hierarchy == MGWR_H64 && level == h->nlev - 1) h->r0_valid = false;
  with_hier(h, hierarchy, [&](auto& H) {
    H.rs[level] = R_STALE;
    return MGWR_OK;
  });
  return MGWR_OK;
}

int mgwr_field_get(mgwr_t h, int hierarchy, int level, int which, double* host) {
  if (h == nullptr) return MGWR_E_INVAL;
  MGWR_TRY(check_level(h, hierarchy, level));
  if (which < MGWR_U || which > MGWR_R || host == nullptr)
    return fail(h, MGWR_E_INVAL, "bad field or null pointer");
  const size_t cnt = level_count(h, level);
  const void* src = field_ptr(h, hierarchy, level, which);
  if (hierarchy == MGWR_H64) {
    MGWR_CK(h, cudaMemcpyAsync(host, src, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
  } else if (hierarchy == MGWR_H32) {
    std::vector<float> tmp(cnt);
    MGWR_CK(h, cudaMemcpyAsync(tmp.data(), src, cnt * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < cnt; ++i) host[i] = (double)tmp[i];
  } else {
    std::vector<mgwr::dd> tmp(cnt);
    MGWR_CK(h, cudaMemcpyAsync(tmp.data(), src, cnt * sizeof(mgwr::dd), cudaMemcpyDeviceToHost,
                               h->stream));
    MGWR_CK(h, cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < cnt; ++i) host[i] = (double)tmp[i].hi + (double)tmp[i].lo;
  }
  return MGWR_OK;
}

int mgwr_smooth(mgwr_t h, int hierarchy, int level, int colour) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  MGWR_TRY(check_level(h, hierarchy, level));
  if (colour != MGWR_RED && colour != MGWR_BLACK) return fail(h, MGWR_E_INVAL, "bad colour");
  MGWR_TRY(with_hier(h, hierarchy, [&](auto& H) { return smooth_colour(h, H, level, colour); }));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return check_staging(h);
}

// largest per-instance norm of the last reduction
static double max_norm(mgwr_t h, const std::vector<double>& norms) {
  double m = 0.0;
  for (double v : norms) m = (v != v || v > m) ? v : m;
  (void)h;
  return m;
}

int mgwr_smooth_defect(mgwr_t h, int hierarchy, int level, double* norm_inf) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  MGWR_TRY(check_level(h, hierarchy, level));
  if (level == 0) return fail(h, MGWR_E_INVAL, "level 0 has a direct solve, not a smoother");
  MGWR_TRY(clear_norms(h));
  MGWR_TRY(with_hier(h, hierarchy, [&](auto& H) {
    MGWR_TRY(smooth(h, H, level, 1));
    return defect_from_delta(h, H, level, h->norm_bits);
  }));
  std::vector<double> norms;
  MGWR_TRY(read_norms(h, norms));
  if (norm_inf != nullptr) *norm_inf = max_norm(h, norms);
  return MGWR_OK;
}

int mgwr_smooth_restrict(mgwr_t h, int hierarchy, int level) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  MGWR_TRY(check_level(h, hierarchy, level));
  if (level == 0) return fail(h, MGWR_E_INVAL, "level 0 has no coarser level");
  MGWR_TRY(with_hier(h, hierarchy, [&](auto& H) {
    MGWR_TRY(smooth(h, H, level, 1));
    return defect_restrict(h, H, level);
  }));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return check_staging(h);
}

int mgwr_defect(mgwr_t h, int hierarchy, int level, double* norm_inf) {
  if (h == nullptr) return MGWR_E_INVAL;
  MGWR_TRY(check_level(h, hierarchy, level));
  MGWR_TRY(clear_norms(h));
  MGWR_TRY(with_hier(h, hierarchy, [&](auto& H) { return defect(h, H, level, h->norm_bits); }));
  std::vector<double> norms;
  MGWR_TRY(read_norms(h, norms));
  if (norm_inf != nullptr) *norm_inf = max_norm(h, norms);
  return MGWR_OK;
}

int mgwr_restrict(mgwr_t h, int hierarchy, int level) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  MGWR_TRY(check_level(h, hierarchy, level));
  if (level == 0) return fail(h, MGWR_E_INVAL, "level 0 has no coarser level");
  MGWR_TRY(with_hier(h, hierarchy, [&](auto& H) { return restrict_into(h, H, level, H.r[level]); }));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return MGWR_OK;
}

int mgwr_prolong(mgwr_t h, int hierarchy, int level) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  MGWR_TRY(check_level(h, hierarchy, level));
  if (level == 0) return fail(h, MGWR_E_INVAL, "level 0 has no coarser level");
  MGWR_TRY(with_hier(h, hierarchy, [&](auto& H) { return prolong_into(h, H, level); }));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return MGWR_OK;
}

int mgwr_coarsest(mgwr_t h, int hierarchy) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  MGWR_TRY(check_level(h, hierarchy, 0));
  MGWR_TRY(with_hier(h, hierarchy, [&](auto& H) { return coarsest(h, H); }));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return MGWR_OK;
}

int mgwr_cycle(mgwr_t h, int hierarchy, int cyc, int nu1, int nu2) {
  if (h == nullptr) return MGWR_E_INVAL;
  h->u_zero = false;
  MGWR_TRY(check_level(h, hierarchy, h->nlev - 1));
  MGWR_TRY(check_cycle_args(h, cyc, nu1, nu2));
  MGWR_TRY(with_hier(h, hierarchy,
                     [&](auto& H) { return cycle(h, H, h->nlev - 1, cyc, nu1, nu2); }));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return check_staging(h);
}

int mgwr_toeplitz_column(mgwr_t h, double* r_host) {
  if (h == nullptr || r_host == nullptr) return MGWR_E_INVAL;
  MGWR_CK(h, cudaMemcpyAsync(r_host, h->r, sizeof(double) * h->M * h->B, cudaMemcpyDeviceToHost,
                             h->stream));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return MGWR_OK;
}

int mgwr_inverse_column(mgwr_t h, int level, double* k_host) {
  if (h == nullptr || k_host == nullptr) return MGWR_E_INVAL;
  if (level < 0 || level >= h->nlev) return fail(h, MGWR_E_INVAL, "level out of range");
  for (int b = 0; b < h->B; ++b)
    MGWR_CK(h, cudaMemcpyAsync(k_host + (size_t)b * h->M,
                               h->kcol + ((size_t)b * h->nlev + level) * h->M,
                               sizeof(double) * h->M, cudaMemcpyDeviceToHost, h->stream));
  MGWR_CK(h, cudaStreamSynchronize(h->stream));
  return MGWR_OK;
}

int mgwr_profile(mgwr_t h, int enable) {
  if (h == nullptr) return MGWR_E_INVAL;
  prof_collect(h);
  h->profiling = enable != 0;
  for (int k = 0; k < MGWR_NUM_KERNEL_CLASSES; ++k) {
    h->prof_launches[k] = 0;
    h->prof_ms[k] = 0.0;
    h->prof_lines[k] = 0.0;
  }
  return MGWR_OK;
}

int mgwr_profile_read(mgwr_t h, int kernel_class, long long* launches, double* ms, double* lines) {
  if (h == nullptr) return MGWR_E_INVAL;
  if (kernel_class < 0 || kernel_class >= MGWR_NUM_KERNEL_CLASSES)
    return fail(h, MGWR_E_INVAL, "bad kernel class");
  prof_collect(h);
  if (launches) *launches = h->prof_launches[kernel_class];
  if (ms) *ms = h->prof_ms[kernel_class];
  if (lines) *lines = h->prof_lines[kernel_class];
  return MGWR_OK;
}

int mgwr_footprint(int d, int n, int M, int batch, int precision, size_t* bytes) {
  if (bytes == nullptr) return MGWR_E_INVAL;
  if ((d != 1 && d != 2) || n < 1 || !is_pow2((long long)n + 1) || !is_pow2(M) || M < 4 ||
      M > mgwr::kMaxM || batch < 1 || !known_precision(precision))
    return MGWR_E_INVAL;
  precision = resolve_precision(n, precision);
  // mirrors the allocations of create_impl, ensure_full, ensure_h32 and ensure_hdd, each
  // rounded up to 512 bytes, plus 2 MiB of allocator slack per handle
  auto r512 = [](size_t b) { return (b + 511) / 512 * 512; };
  const size_t B = batch, L = 2 * (size_t)M, Lt = (size_t)mgwr::engine_length(M);
  std::vector<size_t> pts;
  for (int m = n;; m = (m - 1) / 2) {
    pts.push_back(d == 1 ? (size_t)m : (size_t)m * m);
    if (m == 1) break;
  }
  const size_t nlev = pts.size();
  size_t total = 2u << 20;
  total += r512(8 * B) + r512(8 * B * M) + r512(8 * B * (M + 1)) + r512(8 * B * nlev * M);
  total += 2 * r512(8 * B) + r512(8 * nlev);
  total += r512(16 * B * nlev * 3 * M);  // divide-and-conquer work (freed after setup)
  total += r512(16 * B * nlev * L) + r512(16 * B * L) + r512(16 * Lt);
  if (M > mgwr::kShortMaxM)  // partitioned-convolution scratch: all block spectra of the finest level
    total += r512(16 * B * ((pts[0] + 1) / 2) * L);
  if (precision == MGWR_FP64) {
    for (size_t l = 0; l < nlev; ++l) total += (l + 1 < nlev ? 4 : 3) * r512(8 * B * pts[l] * M);
  } else if (precision == MGWR_DD) {
    total += 2 * r512(8 * B * pts[0] * M);  // FP64 finest iterate and right-hand side
    total += 2 * r512(8 * B * pts[0] * M);  // double-float copies of the finest pair (ensure_dd)
    for (size_t l = 0; l < nlev; ++l) total += (l + 1 < nlev ? 4 : 3) * r512(8 * B * pts[l] * M);
    total += r512(16 * B * nlev * L) + r512(16 * B * L) + r512(16 * Lt) + r512(8 * (size_t)M);
  } else {
    total += 2 * r512(8 * B * pts[0] * M);  // FP64 finest iterate and right-hand side
    for (size_t l = 0; l < nlev; ++l) total += (l + 1 < nlev ? 4 : 3) * r512(4 * B * pts[l] * M);
    total += r512(8 * B * nlev * L) + r512(8 * B * L) + r512(8 * Lt);
    if (mgwr::tensor_length(M)) total += r512(192 * B * nlev * (size_t)M);  // Toeplitz bands
    if (mgwr::radix_length(M))  // register-pass spectra
      total += r512(8 * B * nlev * L) + r512(8 * B * L);
    if (precision == MGWR_MIXED_DD)
      total += 2 * r512(8 * B * pts[0] * M) + r512(16 * B * L) + r512(16 * Lt);
    if (precision == MGWR_MIXED && M <= (size_t)mgwr::kShortMaxM)  // carried defect, anchor spectra
      total += r512(8 * B * pts[0] * M) + r512(16 * B * L) + r512(16 * Lt);
  }
  *bytes = total;
  return MGWR_OK;
}

int mgwr_launch_count(mgwr_t h, long long* count) {
  (void)h;
  if (count == nullptr) return MGWR_E_INVAL;
  *count = mgwr::launch_counter();
  return MGWR_OK;
}

}  // extern "C"

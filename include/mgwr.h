/*
 * mgwr.h -- C ABI of the GB300 multigrid waveform relaxation (MGWR) solver for
 * the time-fractional heat equation
 *
 *     D_t^alpha u - Laplace u = f   on (0,1)^d x (0,T],  d in {1,2},  0 < alpha <= 1,
 *     u = 0 on the boundary,        u(x,0) = g(x),
 *
 * discretised as in the paper: the L1 scheme in time (Sec. 2, Eq. L1_scheme2;
 * Sec. 6, Eq. L1_scheme_2d) and the 3-point / 5-point Laplacian in space
 * (Sec. 2, Eq. discrete_model_IVP_1; Sec. 6, Eq. discrete_model_IVP_2d_1), on
 * n^d interior points (n = 2^k - 1, h = 1/(n+1)) and M uniform time steps
 * (tau = T/M).  The solver is Algorithm 1 (WRMG): red-black waveform
 * relaxation smoother (Sec. 3 Eq. red-black; Sec. 6 Eq. red-black_2d), defect
 * (Algorithm 1), full-weighting restriction and linear / bilinear
 * interpolation of whole time lines, coarsening in space down to one point.
 * All time-line operators are applied as FFT convolutions (Sec. 5).
 *
 * Data layout (every field, host or device): N = n^d time lines of M values,
 * index p*M + m, p = i (1-D) or p = i + n*j (2-D, i along x), m = 0..M-1 at
 * time t_{m+1} = (m+1) tau.  Values are IEEE double.  A handle holds a batch of
 * `batch` instances of the same (d, n, M) with their own T and alpha
 * (mgwr_create_batch; mgwr_create makes a batch of one); every field then
 * holds the instances one after another: instance b at offset b*N*M.
 *
 * Ownership: the caller owns every pointer it passes; the library copies in
 * and out.  The library owns all device memory it allocates (cudaMalloc) and
 * frees it in mgwr_destroy.  Device pointers ("_dev" calls) must be
 * cudaMalloc'd memory on the handle's device, 16-byte aligned.
 *
 * Errors: every call returns MGWR_OK (0) or a negative MGWR_E_* code;
 * mgwr_last_error(h) gives a message for the last failing call on h (static
 * text for a NULL handle).  No call aborts the process or faults the device on
 * invalid arguments: they are checked on the host first.
 *
 * Threads: a handle is not thread-safe; use one handle per host thread.  All
 * device work of a handle runs on its stream (mgwr_set_stream, default: a
 * stream the handle creates).
 */
#ifndef MGWR_H
#define MGWR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MGWR_OK 0
#define MGWR_E_INVAL (-1)   /* invalid argument                              */
#define MGWR_E_NOMEM (-2)   /* device or host allocation failed              */
#define MGWR_E_TOOBIG (-3)  /* request larger than a configured budget        */
#define MGWR_E_NOCONV (-4)  /* max_cycles reached before the tolerance        */
#define MGWR_E_NUMERIC (-5) /* non-finite residual norm                       */
#define MGWR_E_AGAIN (-6)   /* not ready / queue full; retry                  */
#define MGWR_E_TIMEOUT (-7) /* bounded wait ended                             */
#define MGWR_E_CUDA (-8)    /* CUDA runtime error (message in last_error)     */
#define MGWR_E_STATE (-9)   /* call not valid in the handle's current state   */

/* arithmetic of a solve (mgwr_set_precision) */
#define MGWR_FP64 0  /* every kernel in IEEE double                          */
#define MGWR_MIXED 1 /* FP32 V-cycles on the defect, FP64 defect + update     */
#define MGWR_MIXED_DD 2 /* FP32 V-cycles; defect + update in double-float    */
#define MGWR_DD 3       /* refinement with double-float inner cycles         */
#define MGWR_AUTO 4     /* MGWR_MIXED_DD or MGWR_DD by the grid (below)      */
/* MGWR_MIXED keeps the finest iterate, the update and the stencil part of
 * every outer defect in IEEE double.  Its full outer defects take the time
 * convolution T_M u in double-float (FP32 instructions, error about 2^-44
 * |T_M u|, against about 1e-15 |T_M u| in FP64) when the tolerance is at least
 * 1e-10 and the outer switch is finite (mgwr_set_outer_switch), else in FP64;
 * its stopping test uses that defect.
 * MGWR_MIXED_DD keeps the finest iterate and right-hand side as double-float
 * pairs (hi + lo of two floats, about 48 significant bits) and computes the
 * outer defect and the update with FP32 instructions only (GB300 runs FP32 64x
 * faster than FP64).  Its stopping test uses that defect; mgwr_residual gives
 * the IEEE-double defect of the result.
 * MGWR_DD is the same refinement with its inner cycles on a third hierarchy
 * in double-float (8 bytes per value): each outer step reduces the defect as
 * `inner` FP64 cycles do, also where FP32 rounding limits the mixed refinement
 * (4 eps32 / (pi h)^2 close to 1), with FP32 instructions only.  The iterate
 * itself never passes through a convolution (only corrections do), so the
 * rounding of the transforms, about 2^-44 of a field's scale, is not amplified
 * by the discrete Laplacian's 4/h^2.  Its norms and stopping test use the
 * double-float defect.
 * MGWR_AUTO resolves, when it is set, to MGWR_DD where the FP32 limit of an
 * outer step, 4 eps32 / (pi h)^2 with h the finest spacing, is 0.2 or more
 * (h <= 1/4096), else to MGWR_MIXED_DD (mgwr_auto_precision). */

/* which hierarchy a component call addresses */
#define MGWR_H64 64  /* the double-precision hierarchy                         */
#define MGWR_H32 32  /* the single-precision hierarchy (MGWR_MIXED only)       */
#define MGWR_HDD 48  /* the double-float hierarchy (MGWR_DD only)              */

/* fields of a level */
#define MGWR_U 0 /* iterate (finest) or coarse correction e (coarser levels)  */
#define MGWR_F 1 /* right-hand side (finest) or restricted defect              */
#define MGWR_R 2 /* defect work field                                           */

/* smoother colours and colour orders */
#define MGWR_RED 0   /* the colour visited first                              */
#define MGWR_BLACK 1 /* the colour visited second                             */
#define MGWR_ORDER_TEXT 0  /* 1-D: even mesh index n first (0-based odd i)   */
#define MGWR_ORDER_TABLE 1 /* 1-D: odd mesh index n first (0-based even i)   */
/* In 2-D both orders visit even n+l (0-based even i+j) first.  The text of
 * Sec. 3 (below Eq. red-black) says even n first; the 1-D iteration counts of
 * Table table_it_1d are reproduced with the odd-n-first order. */

typedef struct mgwr_handle* mgwr_t;

typedef struct {
  int cycles;       /* WRMG cycles done (MGWR_MIXED: inner FP32 cycles)        */
  int outer;        /* FP64 defect evaluations after the initial one           */
  double relres;    /* ||f - A u||_inf / ||f - A u0||_inf at return            */
  double factor;    /* mean convergence factor relres^(1/cycles)               */
  double seconds;   /* device time of the solve (CUDA events)                  */
} mgwr_stats;

/* ---- lifecycle --------------------------------------------------------- */

/* Create a solver for (d, n, M, T, alpha).  d in {1,2}; n = 2^k - 1 with
 * 1 <= k <= 15 (1-D) or 1 <= k <= 12 (2-D); M = 2^j with 4 <= M <= 2^20;
 * T > 0 finite; 0 < alpha <= 1.  Allocates the double-precision hierarchy
 * and computes on the GPU, in FP64: the L1 Toeplitz column r_1..r_M
 * (Sec. 5 Eq. Toeplitz_matrix), the first column of (T_M + 2d/h_l^2 I)^{-1}
 * for every level l by divide and conquer (Sec. 5, smoothing procedure), and
 * their length-2M spectra (Sec. 5, circulant embedding).  For M > 4096 every
 * time-line convolution is partitioned into blocks of 4096 steps (transforms
 * of length 8192; the spectra are those of the 2M/8192 kernel segments), and
 * the handle also holds a scratch area of 16 bytes x ceil(n^d/2) x 2M per
 * instance for the block spectra (mgwr_footprint counts it).  Device memory
 * comes stream-ordered from the device's default memory pool, whose release
 * threshold the first handle on a device raises to its maximum: memory that
 * handles free stays reserved by this process for the next handles (a setting
 * of this process's pool, not of the GPU).  Returns MGWR_E_INVAL for bad
 * arguments, MGWR_E_NOMEM if device memory runs out. */
int mgwr_create(int d, int n, int M, double T, double alpha, mgwr_t* out);
/* A batch of `batch` (1..65535) independent problems of the same (d, n, M),
 * instance b with final time T[b] and order alpha[b] (host arrays).  Every
 * kernel launch serves all instances (one launch per step of the cycle, the
 * instance index in the grid's second dimension); setup is done for each
 * instance as in mgwr_create.  Sizes and layout: see the data-layout note. */
int mgwr_create_batch(int d, int n, int M, const double* T, const double* alpha, int batch,
                      mgwr_t* out);
int mgwr_batch_size(mgwr_t h, int* batch);
/* Gives the handle's instances new final times T[b] and orders alpha[b]
 * (batch values each, host; as for mgwr_create_batch) without allocating:
 * the L1 columns, the inverse columns of every level and their spectra
 * (Sec. 5) are recomputed in place, with every copy the handle's precisions
 * keep.  Nothing is recomputed when the values are the ones the handle has.
 * The right-hand side and iterate stay; the next solve measures its relative
 * defect from its own start.  A handle set up this way solves bitwise as one
 * created with these values.  MGWR_E_INVAL for bad values. */
int mgwr_set_problem(mgwr_t h, const double* T, const double* alpha);
/* Per-instance relative defect ||f_b - A u_b||_inf / ||f_b - A u0_b||_inf after
 * the last mgwr_solve / mgwr_residual (batch doubles). */
int mgwr_instance_relres(mgwr_t h, double* relres);
int mgwr_destroy(mgwr_t h);
const char* mgwr_last_error(mgwr_t h);
const char* mgwr_status_string(int status);

/* MGWR_FP64 (default), MGWR_MIXED or MGWR_MIXED_DD (both allocate the FP32
 * hierarchy), MGWR_DD (allocates the double-float hierarchy), or MGWR_AUTO
 * (one of MGWR_MIXED_DD and MGWR_DD, resolved now; mgwr_get_precision reads
 * which). */
int mgwr_set_precision(mgwr_t h, int precision);
int mgwr_get_precision(mgwr_t h, int* precision);
/* The precision MGWR_AUTO resolves to for a finest grid of n points per
 * dimension (host arithmetic, no CUDA call; d and M are checked as in
 * mgwr_create).  Other precisions are returned unchanged. */
int mgwr_auto_precision(int d, int n, int M, int precision, int* resolved);
/* MGWR_ORDER_TEXT (default) or MGWR_ORDER_TABLE. */
int mgwr_set_order(mgwr_t h, int order);
/* cudaStream_t to run on (NULL: the handle's own stream). */
int mgwr_set_stream(mgwr_t h, void* stream);
/* Inner cycles per outer defect in the refinements (1..16).  Default 2 in
 * every refinement: most outer steps carry their defect by the correction at
 * the cost of about one FP32 cycle (mgwr_set_outer_switch), and the full
 * defects they leave (anchors and the stopping test) do not grow with the
 * number of steps. */
int mgwr_set_inner_cycles(mgwr_t h, int cycles);
/* Mixed modes (MGWR_MIXED, MGWR_MIXED_DD), lines of M <= 4096: the outer
 * defect of a step's result u + e is carried from the step's starting defect r
 * by its correction, r - (T_M (x) I + A_h) e, with A_h e and the subtraction in
 * the outer precision and T_M e by one FP32 convolution of e (residual
 * replacement), instead of computed in full (a convolution in the outer
 * precision, the solve's dearest kernel in MGWR_MIXED).  A carried defect errs
 * by about 1e-6 of the defect at the last full computation (the anchor), so a
 * step carries it while its starting relative defect is at least `rel` times
 * the anchor's (default 1e-2; 0: every step; +inf: none), in every instance of
 * a batch whose anchor is not already below the tolerance / rel; the other
 * steps compute it in full and so set a new anchor.  Every stopping decision is
 * taken on a full defect.  At +inf no defect is carried and MGWR_MIXED's full
 * defects all take their convolution in FP64.  The paper has no counterpart
 * (its solver is one precision).  MGWR_E_INVAL for rel < 0 or NaN. */
int mgwr_set_outer_switch(mgwr_t h, double rel);

/* Launch shape of the FFT-engine kernels (no counterpart in the paper; the
 * results are bitwise the same for every shape).  For kernel class
 * MGWR_K_SWEEP64, MGWR_K_SWEEP32, MGWR_K_SWEEP_DD (also the one-point solves
 * of that arithmetic), MGWR_K_DEFECT64, MGWR_K_DEFECT32 or MGWR_K_DEFECT_DD, `split`
 * = E in {1, 2, 4} radix-8 butterflies per thread and stage: a group of
 * L/(8E) threads transforms one line pair of length L = 2M (8192 for
 * M > 4096, where E is 1 or 2), synchronising with warp barriers when the
 * group fits in one warp.  A request a length cannot take falls back to the
 * nearest smaller E; mgwr_get_engine_split reports the E launches use.
 * For MGWR_K_SWEEP32 (not the one-point solve) with 64 <= M <= 4096, `split`
 * may also be E | MGWR_SPLIT_STAGED: a persistent kernel whose thread groups
 * receive the f and neighbour lines of their next line pair in shared memory
 * through bulk asynchronous copies (cp.async.bulk, completing on an mbarrier)
 * while they transform the current pair; bitwise the same results.  Its waits
 * give up after half a second, and the call that ran it then returns
 * MGWR_E_CUDA.  MGWR_E_INVAL for another class or split. */
#define MGWR_SPLIT_STAGED 16
/* For MGWR_K_SWEEP32 (not the one-point solve) with M = 64, 128 or 256,
 * `split` may instead be 1 | MGWR_SPLIT_TENSOR: the half-sweep as a dense
 * product with the lower-triangular Toeplitz matrix of the inverse column on
 * the tensor cores (tcgen05.mma with bf16 operands split into three pieces
 * each, FP32 accumulation in tensor memory), 128 lines per CTA.  Results agree
 * with the FFT engine's to FP32 rounding, not bitwise.  Other lengths fall
 * back to the FFT engine.  Its waits give up after half a second, and the call
 * that ran it then returns MGWR_E_CUDA. */
#define MGWR_SPLIT_TENSOR 32
/* For MGWR_K_SWEEP32 (not the one-point solve) with 64 <= M <= 4096, `split`
 * may instead be 1 | MGWR_SPLIT_RADIX: the half-sweep on the register-pass FFT
 * engine, whose transform of length 2M runs as two or three passes of radix
 * 4 .. 32 DFTs held in registers (last pass radix 32, spectrum product and
 * first inverse pass in registers), so every value crosses shared memory once
 * per pass.  Results agree with the other engine's to FP32 rounding, not
 * bitwise.  2 | MGWR_SPLIT_RADIX takes the first pass's adjacent butterflies
 * two at a time, with 8-byte global loads and stores (the same arithmetic;
 * results agree to FP32 rounding).  4 | MGWR_SPLIT_RADIX runs that paired form
 * with resident blocks (one 512-thread block per SM, looping over the line
 * pairs) that keep the spectrum and the twiddle bases in shared memory; its
 * results are bitwise those of 2 | MGWR_SPLIT_RADIX.  Other lengths fall back
 * to the FFT engine. */
#define MGWR_SPLIT_RADIX 64
int mgwr_set_engine_split(mgwr_t h, int kernel_class, int level, int split);
int mgwr_get_engine_split(mgwr_t h, int kernel_class, int level, int* split);
/* Tuner: times every E of each engine class the current precision runs (the
 * sweep and the full defect of its cycle hierarchy on every level, and in
 * the mixed modes the outer defect) on the handle's own data (per level, as
 * many instances as fit 2^27 values, at least one), writing to a temporary
 * field, and keeps the fastest per level (a larger E, staged input lines or
 * the tensor-core sweep must win by 3 %).  The
 * handle's state is unchanged.  The choices are also recorded process-wide
 * for (class, d, n, M, batch): handles created later with that shape start
 * with them.  mgwr_set_engine_split / mgwr_get_engine_split address
 * one level (0 .. num_levels-1) or, with level -1, every level (set) and the
 * finest (get).  Synchronises the
 * handle's stream. */
int mgwr_autotune(mgwr_t h);
/* enable != 0 (default): mgwr_solve captures one iteration of its loop (the
 * cycle's launches, the defect norms and their copy to the host) as a CUDA
 * graph on first use and replays it, one graph launch per iteration; 0:
 * launches are issued one by one.  Results are identical either way.  The
 * capture uses thread-local capture mode on the handle's stream. */
int mgwr_set_graphs(mgwr_t h, int enable);
/* enable != 0 (default): an MGWR_FP64 solve with graphs runs its iterations
 * after the first as one graph launch, a conditional (WHILE) node whose body is
 * one iteration followed by a one-warp kernel that computes the relative
 * defect from the iteration's norms and ends the loop on the device once it is
 * at most tol, is not finite, or max_cycles is reached; the host then reads the
 * iteration count and the norms once, and confirms a stop with the full defect
 * as the host loop does.  Used when the iteration leaves the hierarchy's state
 * as it found it (every V or W cycle from the second on).  Results are those of
 * the host loop, bitwise.  0: one graph launch and one host wait per iteration. */
int mgwr_set_device_loop(mgwr_t h, int enable);

/* ---- problem data -------------------------------------------------------- */

/* Right-hand side f (N*M doubles, host) and initial values g (N doubles, host,
 * NULL = 0).  g enters as + c d_m g in the right-hand side (Sec. 2
 * Eq. L1_scheme2, c = tau^-alpha / Gamma(2-alpha)) and as the initial
 * iterate u^0(t) = g (Sec. 3, below Eq. GS_ODEs).  Resets the iterate. */
int mgwr_set_rhs(mgwr_t h, const double* f, const double* g);
/* Same with device pointers; the copies run on the handle's stream. */
int mgwr_set_rhs_dev(mgwr_t h, const double* f_dev, const double* g_dev);
/* Overwrite the iterate (N*M doubles, host). */
int mgwr_set_initial(mgwr_t h, const double* u0);

/* ---- solve --------------------------------------------------------------- */

/* Run WRMG cycles (cycle = 1: V, 2: W; nu1 pre- and nu2 post-smoothing steps,
 * each one red and one black half-sweep) from the current iterate until
 * ||f - A u||_inf <= tol * ||f - A u0||_inf for every instance of the batch, or
 * max_cycles cycles (MGWR_MIXED: max_cycles FP64 defect evaluations).  A is the
 * whole space-time operator T_M (x) I + A_h (Sec. 5).  Returns MGWR_OK,
 * MGWR_E_NOCONV (stats still filled) or MGWR_E_NUMERIC (non-finite norm).
 * stats may be NULL. */
int mgwr_solve(mgwr_t h, int cycle, int nu1, int nu2, double tol, int max_cycles,
               mgwr_stats* stats);
/* ---- groups: several solves advancing together --------------------------- */
/* A group runs the solves of several handles together (no counterpart in the
 * paper).  Members may differ in every respect (d, n, M, batch, T, alpha,
 * precision, cycle, tolerance); each runs exactly the launches mgwr_solve
 * would, so its result is bitwise the one it gets alone, and each iteration of
 * all running members is one CUDA graph launch on the group's stream whose
 * branches, one per member on the member's own stream, run concurrently on
 * the device (graphs of the recent member combinations are kept, at most 8).
 * Handles join (mgwr_group_add, which computes the initial defect) and leave
 * (their solve ended: collected with mgwr_group_collect) between iterations,
 * so a serving loop admits new work while other solves are in flight.  While
 * in a group a handle must not be used otherwise, and no two members may share
 * a stream.  Group calls are not thread-safe per group. */
typedef struct mgwr_group* mgwr_group_t;
int mgwr_group_create(mgwr_group_t* out);
int mgwr_group_destroy(mgwr_group_t g);
const char* mgwr_group_last_error(mgwr_group_t g);
/* Starts h's solve as mgwr_solve does (arguments as there): the initial defect
 * is computed now, synchronously on h's stream.  MGWR_E_STATE for a handle
 * with profiling on, or one already in the group or sharing a member's
 * stream. */
int mgwr_group_add(mgwr_group_t g, mgwr_t h, int cycle, int nu1, int nu2, double tol,
                   int max_cycles);
/* One iteration of every running member (one graph launch, synchronous).
 * Members whose solve has ended move to the finished list; *running (may be
 * NULL) gets the number still running. */
int mgwr_group_step(mgwr_group_t g, int* running);
/* Takes the oldest finished member: its handle, mgwr_solve's status for it and
 * its statistics.  MGWR_E_AGAIN when none has finished. */
int mgwr_group_collect(mgwr_group_t g, mgwr_t* h, int* status, mgwr_stats* stats);
/* Graph launches so far, member iterations they ran, most members in one. */
int mgwr_group_info(mgwr_group_t g, long long* launches, long long* member_iterations,
                    int* max_members);
/* All `count` handles solved as one group until every solve has ended;
 * status[i] and stats[i] (stats may be NULL) as mgwr_solve's for handles[i].
 * Returns MGWR_OK, or the first error of the group itself. */
int mgwr_group_solve(mgwr_t* handles, int count, int cycle, int nu1, int nu2, double tol,
                     int max_cycles, int* status, mgwr_stats* stats);

/* Defect of the current iterate in FP64: *relres = ||f - A u||_inf /
 * ||f - A u0||_inf (u0 the iterate at set_rhs / set_initial), optional copy of
 * the defect to r_host (N*M doubles). */
int mgwr_residual(mgwr_t h, double* relres, double* r_host);
int mgwr_get_solution(mgwr_t h, double* u_host);
int mgwr_get_solution_dev(mgwr_t h, double* u_dev);

/* Pipelined transfers, for a stream of problems through one handle: the next
 * right-hand side travels to the device and the last solution to the host
 * while a solve runs, so that only two device-to-device copies of one field
 * (about 2.5 ms each at 2-D 511 x 511, M = 4096) stay between the solves.
 * Each call returns at once; the copies run on two streams of the handle's
 * own (created, with two device staging fields of N*M doubles, on first use).
 * - mgwr_stage_rhs: starts copying f_host (N*M doubles, pinned for the copy
 *   to overlap) into the input staging field.  f_host must stay unchanged
 *   until the copy has landed: until mgwr_wait_staged, or the mgwr_solve
 *   after the matching mgwr_take_rhs, returns.  MGWR_E_STATE while a staged
 *   right-hand side is not taken yet.
 * - mgwr_take_rhs: makes the staged right-hand side the handle's (as
 *   mgwr_set_rhs(h, f, NULL) does, without a host wait): the handle's stream
 *   waits for the copy, then copies it into place and zeroes the iterate.
 *   MGWR_E_STATE when nothing is staged.
 * - mgwr_stage_solution: copies the current solution into the output staging
 *   field on the handle's stream (after the previous one has left it), then to
 *   u_host (N*M doubles, pinned) on the output stream.  u_host holds it once
 *   mgwr_wait_staged returns.
 * - mgwr_wait_staged: waits for both transfer streams.
 * A pipelined step: mgwr_take_rhs; mgwr_stage_rhs(next f); mgwr_solve;
 * mgwr_stage_solution(u); and mgwr_wait_staged after the last. */
int mgwr_stage_rhs(mgwr_t h, const double* f_host);
int mgwr_take_rhs(mgwr_t h);
int mgwr_stage_solution(mgwr_t h, double* u_host);
int mgwr_wait_staged(mgwr_t h);

/* ---- components (one step of Algorithm 1 on one level) ------------------ */
/* hier is MGWR_H64 or MGWR_H32; level 0 is the one-point grid, level
 * num_levels-1 the finest.  Fields are exchanged as doubles in both
 * hierarchies (rounded to float on the way into MGWR_H32). */
int mgwr_num_levels(mgwr_t h, int* levels);
int mgwr_level_n(mgwr_t h, int level, int* n_level);
int mgwr_field_set(mgwr_t h, int hier, int level, int which, const double* host);
int mgwr_field_get(mgwr_t h, int hier, int level, int which, double* host);
/* One colour half-sweep of the waveform smoother at `level`: every point p of
 * the colour solves (T_M + 2d/h^2 I) u_p = f_p + h^-2 sum_{q~p} u_q
 * (Sec. 3 Eq. red-black; Sec. 6 Eq. red-black_2d) by convolving with the
 * precomputed inverse column (Sec. 5). */
int mgwr_smooth(mgwr_t h, int hier, int level, int colour);
/* r = f - (T_M (x) I + A_h) u at `level` (Algorithm 1, defect; Sec. 5
 * circulant-embedding matvec); *norm_inf = max |r| (may be NULL). */
int mgwr_defect(mgwr_t h, int hier, int level, double* norm_inf);
/* One smoothing step (red then black half-sweep) at level >= 1, then the
 * defect of the result into field R without a convolution: the black
 * half-sweep leaves each black point's equation satisfied, so the defect is 0
 * there and h^-2 * (sum over the black neighbours of their change) at red
 * points.  Equal to mgwr_defect after mgwr_smooth(RED), mgwr_smooth(BLACK) up
 * to rounding; the solver uses it for every defect that follows smoothing. */
int mgwr_smooth_defect(mgwr_t h, int hier, int level, double* norm_inf);
/* f_{level-1} = full weighting of r_level; u_{level-1} = 0 (Algorithm 1). */
int mgwr_restrict(mgwr_t h, int hier, int level);
/* Algorithm 1's pre-smoothing step, defect and restriction as the cycle runs
 * them at `level` >= 1: one smoothing step (red then black half-sweep), then
 * f_{level-1} = full weighting of the defect f - A u and u_{level-1} = 0.  For
 * MGWR_H32 the defect is formed inside the restriction from the black
 * half-sweep's changes (0 at black points, h^-2 times the sum of the black
 * neighbours' changes at red points) and never stored; for the other
 * hierarchies it is written to field R first (mgwr_smooth_defect) and then
 * restricted.  Field R of `level` is left unspecified. */
int mgwr_smooth_restrict(mgwr_t h, int hier, int level);
/* u_level += linear / bilinear interpolation of u_{level-1} (Algorithm 1). */
int mgwr_prolong(mgwr_t h, int hier, int level);
/* Exact solve on the one-point grid: u_0 = (T_M + 2d/h_0^2 I)^{-1} f_0. */
int mgwr_coarsest(mgwr_t h, int hier);
/* One WRMG cycle at the finest level of `hier` (no convergence test). */
int mgwr_cycle(mgwr_t h, int hier, int cycle, int nu1, int nu2);

/* ---- setup results (FP64, computed on the GPU at mgwr_create) ----------- */
int mgwr_toeplitz_column(mgwr_t h, double* r_host);            /* batch x (r_1..r_M) */
int mgwr_inverse_column(mgwr_t h, int level, double* k_host);  /* batch x (k_1..k_M) */

/* Allocation-free variant of the inverse-column setup (the paper has no
 * counterpart; it serves callers that cannot allocate device memory while
 * they run, e.g. services that reserve their whole GPU budget at start-up or
 * forbid allocation after initialisation).  Computes k_1..k_M, the first
 * column of (T + sigma I)^{-1} for the lower-triangular Toeplitz T with first
 * column r_1..r_M, by the same divide-and-conquer kernel as mgwr_create, on
 * `stream` (a cudaStream_t, NULL = legacy default stream).  r_dev and k_dev
 * are device pointers (M doubles each, caller-owned).  The kernel's scratch
 * (sigma plus 3*M complex values) is a fixed 196,640-byte array compiled into
 * the library, which every GPU that loads the library keeps until the process
 * exits; so M is limited to 4096: larger M returns MGWR_E_TOOBIG, and a bad
 * pointer, M not a power of two >= 4 or sigma < 0 returns MGWR_E_INVAL.
 * Nothing is allocated.  sigma reaches the array by value, through a
 * one-thread kernel on `stream` ahead of the inverse-column kernel, so the
 * call is ordered on `stream` like any kernel launch and does not wait for the
 * GPU.  The first call on each device looks up the array's device address
 * (make it before any stream capture).  All calls share the one array: calls
 * whose work overlaps on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. */
int mgwr_inverse_column_noalloc(const double* r_dev, int M, double sigma, double* k_dev,
                                void* stream);

/* Device bytes a handle of this shape needs at its peak (setup included), for
 * admission control; host-only arithmetic, no CUDA call. */
int mgwr_footprint(int d, int n, int M, int batch, int precision, size_t* bytes);

/* ---- serving: submit / poll ----------------------------------------------- */
/* A server admits queued requests while the sum of their footprints
 * (mgwr_footprint) and of its idle handles stays within `hbm_budget` bytes,
 * at most `max_slots` at a time.  A worker thread per slot prepares each
 * admitted request's handle (an idle handle of the same d, n, M and resolved
 * precision, set up in place for the request's T and alpha by
 * mgwr_set_problem, else a new one; at most 32 idle handles are kept, the least
 * recently used evicted first, also when their memory keeps a request out) and
 * copies its data in; then the request joins the server's group
 * (mgwr_group_*): per size class (space-time unknowns n^d M below 2^22, below
 * 2^26, larger) one batcher thread advances every running request of the
 * class together, each iteration of all of them one CUDA graph launch whose
 * branches run concurrently on the device (the classes' launches overlap too,
 * and small solves do not wait for the iterations of large ones).  A request that arrives while others run starts
 * at the next iteration boundary; its result is bitwise what it gets alone.
 * Admission order (mgwr_server_set_policy; the paper has no counterpart):
 * MGWR_POLICY_FIFO (default), the oldest request that fits runs first;
 * MGWR_POLICY_SMALLEST, the request with the fewest space-time unknowns n^d*M
 * that fits (ties: the oldest), which keeps small requests from waiting behind
 * large ones.  Under both, a request passed over 64 times blocks the others
 * until it fits.  Thread-safe: submit and poll from any thread. */
#define MGWR_POLICY_FIFO 0
#define MGWR_POLICY_SMALLEST 1
typedef struct mgwr_server* mgwr_server_t;
typedef struct {
  int d, n, M;            /* shape, as for mgwr_create                         */
  double T, alpha;
  const double* f;        /* N*M right-hand side, host; copied by mgwr_submit  */
  const double* g;        /* N initial values or NULL; copied                 */
  int precision;          /* MGWR_FP64, MGWR_MIXED, MGWR_MIXED_DD, MGWR_DD, AUTO */
  int order;              /* MGWR_ORDER_TEXT or MGWR_ORDER_TABLE              */
  int cycle, nu1, nu2;    /* as for mgwr_solve                                */
  double tol;
  int max_cycles;
} mgwr_request;
typedef struct {
  int status;             /* mgwr_solve's status (or the failing call's)       */
  mgwr_stats stats;
  double queue_s;         /* submit -> admission, seconds                      */
  double latency_s;       /* submit -> result ready, seconds                   */
} mgwr_result;
typedef struct {
  long long queued, admitted, completed;
  size_t in_use_bytes, peak_bytes, budget_bytes;  /* in use: running + idle handles */
  int slots;
  int max_group_members;      /* most solves advanced by one graph launch        */
  long long group_launches;   /* graph launches of the group so far              */
  long long member_iterations;/* solve iterations those launches ran             */
  long long reused_handles;   /* requests served by an idle handle of their shape */
  double submit_copy_s;       /* host seconds mgwr_submit spent copying f         */
  double prepare_s;           /* slot seconds preparing handles, uploading data   */
  double finish_s;            /* slot seconds downloading results                 */
  double pin_s;               /* host seconds page-locking new pool buffers       */
  long long pinned_buffers;   /* pool buffers page-locked so far                  */
} mgwr_server_info;
/* MGWR_E_INVAL (bad arguments), MGWR_E_CUDA (no device). */
int mgwr_server_create(size_t hbm_budget, int max_slots, mgwr_server_t* out);
/* Stops the workers after their current requests; queued requests are dropped. */
int mgwr_server_destroy(mgwr_server_t s);
/* MGWR_POLICY_FIFO or MGWR_POLICY_SMALLEST; applies to requests admitted from
 * now on.  MGWR_E_INVAL for another value. */
int mgwr_server_set_policy(mgwr_server_t s, int policy);
/* Copies the request's data and queues it: MGWR_OK with *ticket set,
 * MGWR_E_INVAL (bad request), MGWR_E_TOOBIG (footprint above the budget),
 * MGWR_E_AGAIN (queue full), MGWR_E_NOMEM (no host memory for the copy).
 * The copy of f, and later the result, are held in page-locked host memory
 * from a pool the server keeps (up to 32 GiB of released buffers are reused;
 * pageable memory when no page-locked memory can be had). */
int mgwr_submit(mgwr_server_t s, const mgwr_request* rq, uint64_t* ticket);
/* Zero-copy submission (no counterpart in the paper): a page-locked host
 * buffer of at least `count` doubles from the server's pool, into which the
 * caller writes a request's f (N*M doubles, time-contiguous as for
 * mgwr_submit) and which mgwr_submit_buffer then queues without copying it.
 * The buffer belongs to the caller until it is submitted or released;
 * mgwr_server_destroy frees buffers still lent.  MGWR_E_INVAL (bad
 * arguments), MGWR_E_NOMEM (no page-locked memory). */
int mgwr_server_buffer(mgwr_server_t s, size_t count, double** buf);
/* mgwr_submit with f in `buf` from mgwr_server_buffer (rq->f is ignored):
 * on MGWR_OK the server owns the buffer (back to its pool once the data is on
 * the device); on any error the caller still holds it.  Also MGWR_E_INVAL
 * for a buffer the server did not lend or one smaller than N*M doubles. */
int mgwr_submit_buffer(mgwr_server_t s, const mgwr_request* rq, double* buf, uint64_t* ticket);
/* Gives a lent buffer back unsubmitted (MGWR_E_INVAL if it is not lent). */
int mgwr_server_release(mgwr_server_t s, double* buf);
/* Waits up to timeout_us (0: no wait) for the ticket.  MGWR_E_AGAIN (not
 * ready, timeout 0) or MGWR_E_TIMEOUT (not ready after the wait); MGWR_OK:
 * u_out (N*M doubles, may be NULL) and *res filled and the ticket released;
 * MGWR_E_INVAL for an unknown ticket. */
int mgwr_poll(mgwr_server_t s, uint64_t ticket, int timeout_us, double* u_out, mgwr_result* res);
int mgwr_server_stats(mgwr_server_t s, mgwr_server_info* info);

/* Number of CUDA kernel launches issued through the library so far
 * (process-wide; h may be NULL). */
int mgwr_launch_count(mgwr_t h, long long* count);

/* Arithmetic peaks of the current device, the denominators of the FP64- and
 * FP32-issue rooflines: TFLOP/s of dependent-FMA chains, the best of 8 or 16
 * independent chains per thread at 4 or 8 blocks of 256 threads per SM, FP64
 * then FP32, each shape timed with CUDA events after an untimed launch (about
 * 0.2 s a shape on a GB300).  Runs on a private stream and synchronises it;
 * MGWR_E_INVAL for null outputs, MGWR_E_CUDA / MGWR_E_NOMEM on a CUDA failure. */
int mgwr_peak_probe(double* fp64_tflops, double* fp32_tflops);

/* ---- per-kernel-class timing ------------------------------------------- */
/* Kernel classes for mgwr_profile_read. */
#define MGWR_K_SWEEP64 0    /* FP64 colour half-sweeps (levels >= 1)          */
#define MGWR_K_SWEEP32 1    /* FP32 colour half-sweeps                         */
#define MGWR_K_DEFECT64 2   /* FP64 defects (incl. the convergence test)       */
#define MGWR_K_DEFECT32 3   /* FP32 defects                                    */
#define MGWR_K_RESTRICT 4   /* full weighting                                   */
#define MGWR_K_PROLONG 5    /* interpolation + correction                       */
#define MGWR_K_COARSEST 6   /* one-point solves                                 */
#define MGWR_K_REFINE 7     /* mixed-precision update u64 += e32                */
#define MGWR_K_DEFECT_DELTA 8 /* defect after a smoothing step, no convolution  */
#define MGWR_K_DEFECT_DD 9  /* double-float defects (MGWR_MIXED_DD outer, MGWR_DD) */
#define MGWR_K_SWEEP_DD 10  /* double-float colour half-sweeps (MGWR_DD)        */
#define MGWR_NUM_KERNEL_CLASSES 11
/* enable != 0: from now on every launch of the solver is bracketed by CUDA
 * events on the handle's stream (clears the totals).  Adds event records
 * between launches; meant for a measurement run, not for timed runs. */
int mgwr_profile(mgwr_t h, int enable);
/* Totals since mgwr_profile: launches, summed device milliseconds, and the
 * number of time lines the launches processed (points swept / defect points /
 * coarse points restricted / fine points corrected). */
int mgwr_profile_read(mgwr_t h, int kernel_class, long long* launches, double* ms, double* lines);

/* ---- nonlinear problem: waveform relaxation FAS (Sec. 7) ---------------- */
/* The 1-D problem of Eq. anomalous_diffusion,
 *     D_t^alpha u = d/dx( D(u) du/dx ) + c du/dx + f   on (0,1) x (0,T],
 * zero boundary and initial values, discretised with the L1 scheme in time
 * (Eq. L1_scheme2), the conservative flux difference of Eq.
 * spatial_discretization (a_{n+-1/2} = (D(u_{n+-1}) + D(u_n)) / 2, D(0) at the
 * boundary) and upwind convection (forward difference c (u_{n+1} - u_n)/h for
 * c >= 0, backward for c < 0), on n = 2^k - 1 interior points (h = 1/(n+1)) and
 * M time steps (tau = T/M).  It is solved by the full approximation scheme
 * (FAS): a nonlinear red-black waveform smoother in which every point of one
 * colour solves its own time line with its neighbours' lines fixed (marching in
 * time, a Newton solve per step), the residual N_h-defect, full weighting of the
 * iterate and the defect, coarse right-hand side N_2h(R u) + R r on
 * rediscretised coarse levels, linear interpolation of the coarse change, and
 * an exact line solve on the one-point grid.  All arithmetic is IEEE double.
 * Fields (host) are n time lines of M values, index i*M + m, m at t_{m+1}.
 * Ownership, errors and threads as for mgwr_t; a handle runs on a stream it
 * creates.  The history sums are direct (O(M^2) per line). */
typedef struct mgwr_fas* mgwr_fas_t;
#define MGWR_FAS_D_POROUS 0   /* D(u) = 1 + u^2 (Table table_nonlinear)          */
#define MGWR_FAS_D_CONSTANT 1 /* D(u) = 1: the linear model (Sec. 2) when c = 0  */
/* n = 2^k - 1 with 1 <= k <= 12; 1 <= M <= 1024; T > 0 finite; 0 < alpha <= 1;
 * |c| <= 1e30; the L1 scale (T/M)^-alpha / Gamma(2 - alpha) <= 1e30 (the smoother
 * starts each Newton solve in FP32); coefficient one of MGWR_FAS_D_*.  The iterate starts at zero and
 * the right-hand side at zero.  MGWR_E_INVAL / MGWR_E_NOMEM / MGWR_E_CUDA. */
int mgwr_fas_create(int n, int M, double T, double alpha, double c, int coefficient,
                    mgwr_fas_t* out);
int mgwr_fas_destroy(mgwr_fas_t h);
const char* mgwr_fas_last_error(mgwr_fas_t h);
/* MGWR_ORDER_TEXT (default) or MGWR_ORDER_TABLE, as for the linear solver; the
 * cycle counts of Table table_nonlinear are reproduced with MGWR_ORDER_TABLE. */
int mgwr_fas_set_order(mgwr_fas_t h, int order);
/* The nonlinear smoother's line solve (the paper names a nonlinear red-black
 * Gauss-Seidel waveform relaxation and leaves the line solve open):
 * MGWR_FAS_SMOOTHER_MARCH marches each line in time, a scalar Newton solve per
 * step (one warp per line); MGWR_FAS_SMOOTHER_FIXED iterates on whole lines,
 * v <- (T_M + sigma I)^{-1} (f + sigma v - phi(v)) with phi the point's spatial
 * term (its neighbours' lines fixed) and sigma = 2/h^2 + |c|/h, each iteration
 * one FFT convolution per line with the precomputed inverse column of
 * T_M + sigma I (Sec. 5), until the largest change is at the convolution's
 * rounding level (4e-15 of the line pair's largest value) or stops falling
 * within 1e-12 of it (at most 200 iterations; else the call reports
 * MGWR_E_NUMERIC); both give the line's solution to rounding.
 * MGWR_FAS_SMOOTHER_AUTO (default): the fixed point when M is a power of two in
 * 128 .. 1024, else the march.  MGWR_E_INVAL for the fixed point on other M. */
#define MGWR_FAS_SMOOTHER_AUTO 0
#define MGWR_FAS_SMOOTHER_MARCH 1
#define MGWR_FAS_SMOOTHER_FIXED 2
int mgwr_fas_set_smoother(mgwr_fas_t h, int smoother);
/* Whole-line fixed-point iterations run so far, summed over lines (zero when
 * only the march ran); for measuring the smoother's work. */
int mgwr_fas_line_iterations(mgwr_fas_t h, long long* count);
/* f: n*M doubles (host).  Resets the iterate to zero and clears a recorded
 * Newton failure. */
int mgwr_fas_set_rhs(mgwr_fas_t h, const double* f);
/* u0: n*M doubles (host): the iterate the next cycle or solve starts from
 * (also clears a recorded Newton failure). */
int mgwr_fas_set_initial(mgwr_fas_t h, const double* u0);
/* Zero the iterate and clear a recorded Newton failure (device work only, no
 * copy): the next solve starts again from u = 0 with the same right-hand side. */
int mgwr_fas_reset(mgwr_fas_t h);
/* Run the handle's work on `stream` (a cudaStream_t of the current device; NULL:
 * the handle's own stream).  Synchronises the previous stream first; the caller
 * keeps the stream alive while the handle uses it. */
int mgwr_fas_set_stream(mgwr_fas_t h, void* stream);
/* FAS cycles (cycle = 1: V, 2: W; nu1 / nu2 pre- / post-smoothing steps, each a
 * red and a black half-sweep) from the current iterate until the max-norm of
 * f - N_h(u) is at most tol times its value at the start of the call, or
 * max_cycles cycles.  Returns MGWR_OK, MGWR_E_NOCONV (stats filled), or
 * MGWR_E_NUMERIC (a non-finite defect, or a Newton solve in the smoother that
 * did not settle in 100 steps).  stats may be NULL (outer is 0). */
int mgwr_fas_solve(mgwr_fas_t h, int cycle, int nu1, int nu2, double tol, int max_cycles,
                   mgwr_stats* stats);
/* One FAS cycle from the current iterate. */
int mgwr_fas_cycle(mgwr_fas_t h, int cycle, int nu1, int nu2);
/* max-norm of f - N_h(u) of the current iterate; optional copy to r_host (n*M). */
int mgwr_fas_residual(mgwr_fas_t h, double* norm_inf, double* r_host);
int mgwr_fas_get_solution(mgwr_fas_t h, double* u_host);
/* Component calls on level `level` (0 = the one-point grid, mgwr_fas_levels()-1
 * = the finest): one colour half-sweep of the nonlinear smoother, and copies of
 * a level's iterate / right-hand side / defect (which = MGWR_U / MGWR_F /
 * MGWR_R; n_level*M doubles, n_level = 2^(level+1) - 1). */
int mgwr_fas_levels(mgwr_fas_t h, int* levels);
int mgwr_fas_smooth(mgwr_fas_t h, int level, int colour);
int mgwr_fas_defect(mgwr_fas_t h, int level, double* norm_inf);
int mgwr_fas_field_set(mgwr_fas_t h, int level, int which, const double* host);
int mgwr_fas_field_get(mgwr_fas_t h, int level, int which, double* host);

#ifdef __cplusplus
}
#endif
#endif /* MGWR_H */

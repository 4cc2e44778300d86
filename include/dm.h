/*
 * dm.h -- C ABI of the GB300 (sm_103a) decomposition-method solver for
 * block-tridiagonal linear systems.
 *
 * Method: P. A. Belov, E. R. Nugumanov, S. L. Yakovlev, "Decomposition
 * method for block-tridiagonal matrix systems", arXiv:1505.06864.
 *
 * The system (the paper's Eq. 1, with this library's letters) is
 *
 *     A_i X_{i-1} + B_i X_i + C_i X_{i+1} = b_i,   i = 1..N,   A_1 = C_N = 0,
 *
 * B_i the m x m diagonal block (the paper's C_i), C_i the super-diagonal
 * block (the paper's B_i), m the block size (the paper's n), nrhs the number
 * of right-hand-side columns (the paper's l), P the number of subsystems
 * (the paper's M).
 *
 * Memory layout of every array argument: float64, row-major blocks stored one
 * after another.  A, B, C: [N][m][m] (element (i, r, c) at i*m*m + r*m + c);
 * b, x: [N][m][nrhs] (element (i, r, c) at i*m*nrhs + r*nrhs + c).  The
 * entries of A_1 (index 0) and C_N (index N-1) are ignored.  Each pointer may
 * be host memory (pageable or pinned) or device memory of the current CUDA
 * device; the library detects which.  The caller keeps ownership of every
 * array; the library copies what it needs before the call returns (dm_submit
 * excepted, see there).
 *
 * Return values: DM_OK (0) on success, a negative DM_E* code on failure.
 * Nothing is thrown across the ABI.  dm_last_error() gives a text for the
 * calling thread's last failure.  A plan handle may be used by one thread at
 * a time; different plans may be used concurrently from different threads.
 */
#ifndef DM_GB300_H
#define DM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DM_OK 0
#define DM_PENDING 1      /* dm_poll: the request has not finished */
#define DM_EINVAL (-1)    /* invalid argument (sizes, P, levels, precision, NULL pointer) */
#define DM_ENOMEM (-2)    /* device memory could not be allocated / admission refused */
#define DM_ESINGULAR (-3) /* a pivot of some block inverse was zero, not finite, or (float64
                             blocked inverse) of magnitude below 2^-1022 or at least 2^1022 */
#define DM_ENOTCONV (-4)  /* iterative refinement did not reach its tolerance */
#define DM_EAGAIN (-5)    /* no serving slot free right now; try again */
#define DM_ECUDA (-6)     /* a CUDA runtime call failed */
#define DM_ESTATE (-7)    /* call out of order (e.g. dm_solve before dm_factor) */
#define DM_ETIMEOUT (-8)  /* a bounded device-side wait gave up */

/* precision of the block factorisation at the top level.  The supplementary
 * (interface) system is always factored and solved in float64, and the
 * residual of iterative refinement is always evaluated in float64. */
#define DM_FP64 0    /* plain float64 throughout; no refinement */
#define DM_FP32 1    /* float32 factors on CUDA cores + float64 refinement */
#define DM_TF32 2    /* tcgen05 kind::tf32 block products, float32 accumulate + refinement */
#define DM_BF16X3 3  /* tcgen05 kind::f16 split-bf16 (hi*hi + hi*lo + lo*hi) + refinement */

/* How the residual r = b - T x is computed (dm_set_residual). */
#define DM_RESIDUAL_FP64 0   /* float64 fused multiply-adds on the CUDA cores */
#define DM_RESIDUAL_SLICED 1 /* exact bf16 slice products on the tensor cores, float64-accurate */
#define DM_RESIDUAL_AUTO 2   /* SLICED for the systems where it is faster (m^2 nrhs >= 2^17), else FP64 */

typedef struct dm_plan_s* dm_plan_t;

/* Facts about a plan, filled by dm_plan_query. */
typedef struct dm_plan_info {
  int N, m, nrhs;        /* sizes (first system of a batch plan) */
  int P;                 /* subsystems at the top level (the paper's M) */
  int levels;            /* 1: supplementary system by block Thomas; L > 1: by DM with L-1 levels */
  int P2;                /* subsystems of the supplementary system when levels > 1, else 1 */
  int precision;         /* DM_FP64 / DM_FP32 / DM_TF32 / DM_BF16X3 */
  int count;             /* systems in the plan (1 unless made by dm_plan_batch) */
  int last_iters;        /* refinement iterations taken by the last dm_solve */
  int max_rows;          /* longest subsystem (block rows swept sequentially) */
  size_t device_bytes;   /* device memory held by the plan */
  double last_relres;    /* max_k ||b - T x||_2 / ||b||_2 over columns of the last solve */
  double last_correction;/* last refinement step ||dx||_2 / ||x||_2 (0 for DM_FP64) */
  double factor_flops;   /* algorithmic flops of one dm_factor (2 per multiply-add) */
  double solve_flops;    /* algorithmic flops of one solve sweep (without refinement) */
  int residual_mode;     /* DM_RESIDUAL_FP64 or DM_RESIDUAL_SLICED */
  int residual_tc_systems; /* systems whose residual runs on the tensor cores */
  int J;                 /* sub-subsystems per subsystem (dm_plan_inside), else 1 */
} dm_plan_info;

/* Plan the solution of one system of N block rows, blocks m x m, nrhs
 * right-hand-side columns, split into P subsystems (Section 2 of the paper;
 * 1 <= P <= (N+1)/2, every subsystem keeps >= 1 row; P = 1 is the block Thomas
 * algorithm of Section 3).  levels >= 1: the supplementary system of Eq. (e232)
 * is solved by block Thomas (levels = 1) or by DM recursively (levels > 1,
 * Section 4.2.1, its subsystem count from Eq. (SuppMatrM)).  P = 0 and
 * levels = 0 take the measured choice of dm_autotune for this shape and
 * precision if there is one, else (and for P = 0 or levels = 0 alone) the
 * paper's optimum: Eq. (MAXSpeedP) for P, depth 2 when P >= 21 (depth 3 when
 * the supplementary system then has >= 8 subsystems: on the GPU each level's
 * last block Thomas chain is latency-bound).  Limits: 1 <= m <= 512, 1 <= nrhs <= 64.  Allocates the
 * device workspace (factors, sweep vectors, supplementary systems) after an
 * admission check against the free device memory; returns DM_EINVAL or
 * DM_ENOMEM on failure.  The plan's copy of A, B, C (3 N m^2 doubles) is
 * allocated by the first dm_factor that copies (none if the plan borrows its
 * inputs, see dm_set_borrow_inputs).  *out is set only on success. */
int dm_plan(dm_plan_t* out, int N, int m, int nrhs, int P, int levels, int precision);

/* dm_plan with flags.  DM_PLAN_EQUAL_TIME sizes the subsystems for equal
 * operation counts (Section 5.1, second case; sizes from Table 2): the first
 * and last subsystems longer than the middle ones (about 7/4 and 7/6 of them
 * for nrhs << m).  On the GPU every step of all subsystems is one launch, so
 * the longest subsystem sets the step count: equal sizes (flags = 0) are
 * normally faster there. */
#define DM_PLAN_EQUAL_TIME 1
/* Float64 block products (DM_FP64 plans and every supplementary level) are by
 * default computed on the tensor cores by exact digit slicing where the level
 * has one block size m with m % 8 == 0 and m <= 256: every float64 operand is
 * cut into nine 6-bit digit slices (bf16) with a power-of-two scale per row
 * (left operand) or column (right operand), the 53 digit products with
 * s + t <= 11 are accumulated exactly (integers below 2^24 in float32), and
 * the sums are combined in float64 -- an error bound of the size of the
 * float64 dot product's.  DM_PLAN_FP64_FMA keeps them on the float64 pipe. */
#define DM_PLAN_FP64_FMA 2
/* The float64 block inverse of those levels is by default blocked
 * Gauss-Jordan (panels of 32 columns in float64, their rank-32 trailing
 * updates as digit-sliced tensor-core products); DM_PLAN_FP64_INV_COLUMN
 * takes the column-by-column Gauss-Jordan kernel instead (same pivoting). */
#define DM_PLAN_FP64_INV_COLUMN 4
int dm_plan_ex(dm_plan_t* out, int N, int m, int nrhs, int P, int levels, int precision, int flags);

/* DM inside the subsystems (Section 4.2.2; counts Eqs. DMrec121, DMrec1212,
 * DMrec122; serial counts Eq. DMrec3 and, with outer_levels = 2, Eq. DMrec4).
 * The system is split into M subsystems (equal sizes as in dm_plan), and the
 * subsystem equations of Eq. (e231) are themselves solved by DM: every
 * subsystem is split into J sub-subsystems (the same rule; each needs >= 1
 * row, i.e. every subsystem >= 2J - 1 rows), their J - 1 inner separators
 * form the subsystem's inner supplementary system, and the M - 1 outer
 * separators the supplementary system of Eq. (e232), solved by block Thomas
 * (outer_levels = 1) or by DM (outer_levels = 2, its subsystem count from
 * Eq. SuppMatrM).  The sub-subsystems' sweeps (M J of them, each about
 * (N - M + 1) / (M J) rows long) run in parallel, so the sequential chain is
 * J times shorter than with M subsystems.  Executed as DM with the M J
 * sub-subsystems whose supplementary system is split into M parts at the
 * outer separators: each part is one subsystem's inner supplementary system,
 * and the subsystem spikes Z^k of Eq. (e231) are applied in this factored
 * form (sub-subsystem spikes, inner supplementary solution) rather than
 * formed over all rows; x is the same.  Arguments and errors as for dm_plan;
 * DM_EINVAL also for M < 1, J < 2, outer_levels not 1 or 2, or subsystems
 * too short for J. */
int dm_plan_inside(dm_plan_t* out, int N, int m, int nrhs, int M, int J, int outer_levels, int precision);

/* Complex systems (the paper's application, Section 7, has complex
 * boundary conditions).  Arrays are complex128 as interleaved (real,
 * imaginary) double pairs with the real layouts: A, B, C [N][m][m], b, x
 * [N][m][nrhs]; host or device pointers as for the real calls.  The plan
 * solves the real embedding of the system: every complex block X + iY becomes
 * the real 2m x 2m block [[X, -Y], [Y, X]] and every right-hand-side block
 * u + iv the 2m x nrhs block [u; v], a real block-tridiagonal system with the
 * same N, P and recursion, on which every precision and kernel of the real
 * path runs unchanged (twice the multiply-adds of complex arithmetic).
 * Limits: m <= 256 (m <= 128 for DM_TF32 / DM_BF16X3).  The plan holds the
 * embedded blocks (3 N (2m)^2 doubles) and a staging buffer for host arrays.
 * dm_solve_complex returns DM_ENOTCONV as dm_solve does; relres_out is the
 * relative residual of the embedded system, equal to that of the complex one.
 * dm_factor / dm_solve on such a plan take the embedded real arrays. */
int dm_plan_complex(dm_plan_t* out, int N, int m, int nrhs, int P, int levels, int precision);
int dm_factor_complex(dm_plan_t plan, const double* A, const double* B, const double* C);
int dm_solve_complex(dm_plan_t plan, const double* b, double* x, double* relres_out);

/* Subsystem sizes (rows, in order) a plan with these arguments uses; host
 * only.  `lengths` receives P values (P = the effective P: 0 = the tuner's). */
int dm_partition_sizes(int N, int m, int nrhs, int P, int flags, int* lengths);

/* Plan `count` independent systems (sizes N[s], m[s], nrhs[s]) that are
 * factored and solved together, every stage of all systems in the same
 * launches.  Partition counts and recursion depth are chosen per system by
 * the tuner.  Arrays of a batch are the systems' arrays concatenated in order
 * (system s starts at sum_{s'<s} N[s'] m[s']^2 for A, B, C and at
 * sum_{s'<s} N[s'] m[s'] nrhs[s'] for b, x).  relres_out of dm_solve then points to
 * `count` doubles. */
int dm_plan_batch(dm_plan_t* out, int count, const int* N, const int* m, const int* nrhs, int precision);

/* Factor: forward and backward sweeps of every subsystem for its spikes
 * (Eq. e231, the W_R right-hand sides), assembly of the supplementary matrix
 * (Eq. e2311) and its float64 factorisation (Eq. e232).  The factors stay on
 * the device until dm_destroy; dm_factor may be called again with new blocks.
 * Returns DM_ESINGULAR if a pivot vanished or its reciprocal is not a normal
 * float64 number (dm_last_error names the block row),
 * DM_ENOMEM if the first call cannot allocate the plan's input copies. */
int dm_factor(dm_plan_t plan, const double* A, const double* B, const double* C);

/* Solve T x = b with the resident factors: subsystem sweeps for z^k
 * (Eq. e231), supplementary right-hand side (Eq. e2311), supplementary solve
 * for h (Eq. e232), back-substitution (Eq. endSolution), float64 residual.
 * For precision != DM_FP64 the solve is repeated on float64 residuals
 * (iterative refinement) until ||dx||/||x|| <= tol (dm_set_refinement) or the
 * iteration cap; DM_ENOTCONV then, with the best x written.  x may alias b.
 * relres_out (may be NULL) receives max over columns of ||b - T x||/||b||. */
int dm_solve(dm_plan_t plan, const double* b, double* x, double* relres_out);

/* Measured tuning: time candidate decompositions -- P from the paper's
 * optimum (Eq. MAXSpeedP), its half and double, and multiples of half the SM
 * count; recursion depth 1, 2, 3 -- on a synthetic diagonally dominant system
 * of this shape (drawn on the device, freed afterwards), for dm_factor +
 * dm_solve at `precision`, and return the fastest (*ms_out: its time per
 * factor + solve).  The choice is remembered per (N, m, nrhs, precision) for
 * the process and, if the environment variable DM_TUNE_CACHE names a file,
 * in that file; dm_plan with P = 0 and levels = 0 then uses it.  Needs room
 * for the synthetic system and one plan at a time; a call for a remembered
 * shape returns at once. */
int dm_autotune(int N, int m, int nrhs, int precision, int* P, int* levels, double* ms_out);

/* dm_autotune that also times the kernel variants at the chosen (P, levels):
 * for float64 plans whose levels can use the digit-sliced products, the
 * products on the float64 pipe (DM_PLAN_FP64_FMA) and the column-by-column
 * inverse (DM_PLAN_FP64_INV_COLUMN); *flags receives the fastest variant's
 * plan flags (0: the defaults), which dm_plan with P = 0 and levels = 0 then
 * applies.  flags may be NULL. */
int dm_autotune_ex(int N, int m, int nrhs, int precision, int* P, int* levels, int* flags, double* ms_out);

/* The measured choice stored for this shape and precision (by dm_autotune /
 * dm_autotune_ex in this process, or read from the DM_TUNE_CACHE file at the
 * first lookup), which dm_plan with P = 0 and levels = 0 applies.  Host only:
 * no GPU work.  DM_EINVAL if there is none.  flags may be NULL. */
int dm_tuned(int N, int m, int nrhs, int precision, int* P, int* levels, int* flags);

/* Continuous batching.  dm_submit queues a solve of b on the plan's resident
 * factors; dm_submit_system queues a factor (of A, B, C) followed by a solve.
 * Both return at once with a ticket.  A process-wide server runs the queued
 * requests on `slots` worker streams (default 8, set by dm_serve_slots before
 * the first submit): a worker takes the oldest request whose plan has nothing
 * in flight, so requests on different plans run concurrently on the device
 * and new requests are admitted as slots free up; requests on one plan run in
 * submission order.  b, x (and A, B, C) must stay valid and unchanged until
 * dm_poll reports completion, and the plan must not be used directly
 * meanwhile.  DM_EAGAIN if the queue is full.  dm_destroy waits for a plan's
 * queued requests.  (Device memory is admitted at dm_plan, which refuses a
 * plan that does not fit in the free device memory with DM_ENOMEM.) */
int dm_submit(dm_plan_t plan, const double* b, double* x, uint64_t* ticket);
int dm_submit_system(dm_plan_t plan, const double* A, const double* B, const double* C,
                     const double* b, double* x, uint64_t* ticket);

/* Poll a ticket: *status = DM_PENDING while queued or running, else the
 * request's final status (DM_OK or an error code); relres_out (may be NULL)
 * receives its relative residual.  A finished ticket is forgotten after the
 * poll that reports it.  DM_EINVAL for an unknown ticket. */
int dm_poll(uint64_t ticket, int* status, double* relres_out);

/* dm_poll that also reports, for a finished request, when it was submitted,
 * started on a worker and finished (times[0..2], seconds on a monotonic clock
 * with an arbitrary origin); times untouched while DM_PENDING. */
int dm_poll_times(uint64_t ticket, int* status, double* relres_out, double* times);

/* Number of serving worker streams (1..64); only before the first submit. */
int dm_serve_slots(int slots);

/* A narrow request: b and x hold ncols right-hand-side columns
 * ([N][m][ncols], 1 <= ncols <= the plan's nrhs), solved on the plan's
 * resident factors.  Narrow requests queued on one plan are merged: a worker
 * packs the columns of consecutive queued narrow requests (in submission
 * order, while they fit in nrhs) into one solve of the plan's nrhs columns,
 * unused columns zero, and unpacks each request's columns into its x; each
 * request's relres is the worst of its own columns.  The columns pass through
 * the plan's residual buffer and a gather kernel, so b and x may be host or
 * device memory as for dm_solve.  Real single-system plans only (DM_EINVAL
 * otherwise); other errors as dm_submit. */
int dm_submit_cols(dm_plan_t plan, const double* b, double* x, int ncols, uint64_t* ticket);

/* Latency budget for admission (seconds; 0, the default, admits everything
 * the queue holds).  The server keeps per plan a moving average of the
 * measured service time of factor + solve and of solve requests (a narrow
 * request is charged its columns' share of a solve).  A submit whose
 * predicted latency -- the queued and remaining running work divided by the
 * slots, but at least the work queued or running on its own plan, plus its
 * own service time -- exceeds the budget is refused with DM_EAGAIN and
 * nothing is queued.  Plans not yet measured predict zero.  May be changed at
 * any time.  DM_EINVAL for a negative, NaN or absurd (> 1e6 s) budget. */
int dm_serve_budget(double seconds);

/* Serving counters since the process started: out[0] requests admitted,
 * out[1] refused (budget or full queue), out[2] worker runs (a run serves one
 * request or one merged group), out[3] requests served in merged groups of
 * two or more. */
int dm_serve_stats(long long* out);

/* The application case of the paper's Section 7: the right-hand side is zero
 * except its last block row b_N ([m][nrhs]) and only x_N ([m][nrhs]) is
 * wanted.  Every subsystem's z vanishes except the last one's, whose forward
 * sweep is a single step; only the last separator's supplementary right-hand
 * side is non-zero; x_N = z_N - Z_L h (Eqs. e2311, endSolution).  Float64
 * single-system plans only (DM_EINVAL otherwise); no residual is computed. */
int dm_solve_last(dm_plan_t plan, const double* b_last, double* x_last);

/* The decomposition dm_plan would choose for P = 0 / levels = 0 (the tuner's
 * seed: P from Eq. (MAXSpeedP), recursion from the P >= 21 condition after
 * Eq. (SuppMatrM) -- one level more when P2 >= 8 --, P2 from Eq. (SuppMatrM)).  Host only: allocates nothing and
 * needs no GPU.  Inputs P, levels as for dm_plan (0 = choose); outputs the
 * effective P, levels and P2.  DM_EINVAL for invalid sizes. */
int dm_plan_tune(int N, int m, int nrhs, int* P, int* levels, int* P2);

/* Per-kernel timing for benchmarks.  Every kernel the library launches for a
 * plan belongs to a class (inv, fwd_factor, back_factor, assemble_h,
 * fwd_solve, back_solve, assemble_f, backsub, sep_copy, residual,
 * axpy_norms).  With profiling enabled each launch is bracketed by a pair of
 * CUDA events recorded on the plan's stream.  dm_profile first writes (when
 * out != NULL) one entry per class and recursion depth seen since the
 * previous call (name "fwd_factor" for the top level, "fwd_factor@1" for its
 * supplementary system, "@2" one level further, "@3" for all deeper) -- launches,
 * summed event time in ms, and the launches' algorithmic flops (2 per
 * multiply-add) and bytes (operands read once, results written once) --
 * then clears the sums and switches profiling on (enable = 1) or off. */
typedef struct dm_profile_entry {
  char name[24];
  long long launches;
  double ms, flops, bytes;
} dm_profile_entry;
int dm_profile(dm_plan_t plan, int enable, dm_profile_entry* out, int max_entries, int* n_entries);

/* Number of kernels this plan has launched so far (always counted). */
long long dm_launch_count(dm_plan_t plan);

/* Factor and solve one system without allocating anything, for callers that
 * cannot call cudaMalloc (code running while another component owns the
 * device memory pool, plug-ins whose host forbids allocation on the solve
 * path, real-time loops that must not enter the allocator).  The paper has no
 * counterpart: this is a deployment variant of dm_plan(N, m, nrhs, P, 1,
 * DM_FP64) + dm_factor + dm_solve and gives the same x.
 *
 * A, B, C ([N][m][m]), b and x ([N][m][nrhs]) must be device pointers on the
 * current device; x must not alias b.  The workspace is one static 32 MiB
 * __device__ array compiled into the library (held by every GPU that loads
 * it until the process exits): the system must fit it, roughly
 * 4 N m^2 + 5 (P-1) m^2 doubles below 4 Mi, and P <= 256, else DM_EINVAL
 * (nothing is launched).  The supplementary system is solved by block Thomas.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents: calls
 * whose work overlaps on the GPU (other threads, other streams) race and give
 * wrong results, so serialise them.  Work is queued on `stream` (NULL: the
 * default stream) and the call returns after it finished.  DM_ESINGULAR as
 * for dm_factor. */
int dm_solve_noalloc(int N, int m, int nrhs, int P, const double* A, const double* B, const double* C,
                     const double* b, double* x, void* stream);

/* Borrow the inputs instead of copying them: the plan keeps no copy of A, B,
 * C (3 N m^2 doubles per system; freed if already made) and from then on dm_factor
 * takes device pointers only and uses them in place; they must stay valid and
 * unchanged until the next dm_factor or dm_destroy (the residual of every
 * dm_solve reads them).  For systems that fill a large part of device memory.
 * Cannot be switched off. */
int dm_set_borrow_inputs(dm_plan_t plan, int enable);

/* Factor sweeps: run the left-spike tiles (off the inversion chain) on a
 * second stream that overlaps the next block inversion (enable = 1) or in
 * the same launches as the rest (0, the default; on GB300 both run at the
 * same speed for float64, whose FP64 pipes both stages share). */
int dm_set_side_stream(dm_plan_t plan, int enable);

/* Optional settings and queries. */
int dm_set_stream(dm_plan_t plan, void* cuda_stream);            /* cudaStream_t for the plan's launches */
int dm_set_refinement(dm_plan_t plan, double tol, int max_iters); /* default 1e-12, 30 */

/* Residual method (the paper has none: it stops at the direct solve; the
 * refinement of the mixed precisions needs r = b - T x in float64 accuracy).
 * DM_RESIDUAL_SLICED cuts every float64 entry of a block row [A_i B_i C_i]
 * and of [x_{i-1}; x_i; x_{i+1}] into nine 6-bit digits scaled by the row's
 * (column's) largest power of two, multiplies digit matrices exactly on the
 * bf16 tensor cores (integer partial sums below 2^24 in float32), and sums
 * the digit products in float64: error per entry below
 * 3m 2^-50 max|row of [A B C]| max|column of x|, the float64 dot product's own
 * bound.  It serves systems with m <= 128 and nrhs <= 16; the others of the
 * plan use DM_RESIDUAL_FP64.  DM_RESIDUAL_AUTO picks SLICED per system where
 * it measured faster on GB300 (m^2 nrhs >= 2^17: m = 128 with nrhs >= 8,
 * m = 96 with nrhs >= 15): the float64 kernel's cost grows with nrhs, the
 * sliced kernel's mostly with m^2.  Default: AUTO for DM_FP32 / DM_TF32 /
 * DM_BF16X3 plans, FP64 for DM_FP64 plans.  DM_EINVAL for other modes. */
int dm_set_residual(dm_plan_t plan, int mode);

/* r = b - T x with the plan's blocks (after dm_factor) in the plan's residual
 * mode; x, b, r are [N][m][nrhs] float64 (host or device; r may alias b),
 * relres_out (may be NULL) receives max over columns of ||r|| / ||b||.  For
 * checking a solution computed elsewhere, or a residual method against
 * another.  DM_ESTATE before dm_factor. */
int dm_residual(dm_plan_t plan, const double* x, const double* b, double* r, double* relres_out);
int dm_plan_query(dm_plan_t plan, dm_plan_info* info);

/* Measured arithmetic peak of the current device, for roofline denominators
 * (the paper has no counterpart).  kind: DM_PROBE_FP64 / DM_PROBE_FP32 -- the
 * inner loop of a register-tiled matrix product (4 x 4 accumulators per
 * thread, each fused multiply-add reading two shared operands) at full
 * occupancy;
 * DM_PROBE_TF32 / DM_PROBE_BF16 -- one CTA per SM issuing back-to-back
 * tcgen05.mma (M = 128, N = 256, float32 accumulate) from shared memory.
 * One warm-up launch, then `repeat` launches of about 0.1 s timed with CUDA
 * events; *tflops_out receives the best (flops = 2 per multiply-add),
 * *ms_out (may be NULL) that launch's time.  Allocates 64 bytes.  Changes no
 * clock or power setting. */
#define DM_PROBE_FP64 0
#define DM_PROBE_FP32 1
#define DM_PROBE_TF32 2
#define DM_PROBE_BF16 3
int dm_peak_probe(int kind, int repeat, double* tflops_out, double* ms_out);

void dm_destroy(dm_plan_t plan);
const char* dm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DM_GB300_H */

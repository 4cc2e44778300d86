// Host-side plan structures of the decomposition-method solver.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <memory>
#include <string>
#include <vector>

#include "dm_internal.cuh"

namespace dm {

// Kernel classes of the profiler (one per launcher).
enum KClass {
  K_INV, K_FWD_FACTOR, K_BACK_FACTOR, K_ASSEMBLE_H, K_FWD_SOLVE, K_BACK_SOLVE, K_ASSEMBLE_F,
  K_BACKSUB, K_SEP_COPY, K_RESIDUAL, K_AXPY, K_SWEEP_SOLVE, K_TC_CONVERT, K_INV_PANEL, K_INV_UPDATE, K_BANDED,
  K_NCLASS
};
extern const char* const kClassNames[K_NCLASS];

// Launch counter and optional CUDA-event timing of every launch.
struct Prof {
  bool on = false;
  long long launches = 0;
  struct Rec {
    int cls;
    cudaEvent_t e0, e1;
    double flops, bytes;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  // sums per class and recursion depth (0 = the top level; deeper levels
  // share the last slot)
  static constexpr int kDepths = 4;
  int depth = 0;  // depth of the level whose kernels are being launched
  long long n[K_NCLASS * kDepths] = {};
  double ms[K_NCLASS * kDepths] = {}, flops[K_NCLASS * kDepths] = {}, bytes[K_NCLASS * kDepths] = {};
  cudaEvent_t take();
  void begin(cudaStream_t st, cudaEvent_t* e0);
  void end(cudaStream_t st, cudaEvent_t e0, int cls, double fl, double by, int kernels);
  int collect();  // fold finished records into the per-class sums
  void reset();
  ~Prof();
};

// Algorithmic flops (2 per multiply-add) and bytes (operands read once, results
// written once) of one launch.
struct Cost {
  double flops = 0, bytes = 0;
};

// Side stream for work off the inversion chain, with the two events that
// order it against the main stream.
struct Aux {
  cudaStream_t st = nullptr;
  cudaEvent_t ev_main = nullptr, ev_aux = nullptr;
};

// Sizes and decomposition of one system.
struct SysSpec {
  int N = 0, m = 0, r = 0;
  int P = 1;       // subsystems (the paper's M)
  int levels = 1;  // 1: supplementary system by block Thomas; L > 1: by DM, L-1 levels
  int P2 = 1;      // subsystems of the supplementary system when levels > 1
  int flags = 0;   // DM_PLAN_* (subsystem sizing)
  int J = 1;       // >= 2: DM inside each of P / J subsystems (nested lengths, P2 = P / J)
};

// Operand copies of the tensor-core step kernels (dm_tc2.cu) for a float32
// level with one block size m (m % 8 == 0, m <= 256): TF32 (mode 0, float32
// values) or split bf16 (mode 1, hi blocks then lo blocks, `cap` blocks
// apart).  Full copies hold every block of the level; rolling ones one block
// per subsystem (two for the spikes of the backward sweep).
struct Tc2Level {
  bool on = false;
  int mode = 0;
  void* A = nullptr;     // A_i row-major (mode 0: the float32 copy A32)
  void* CT = nullptr;    // C_i transposed
  void* Acal = nullptr;  // Acal_t row-major (mode 1 only; mode 0 reads the float32 factor)
  void* G = nullptr;     // G_t row-major, rolling (mode 1 only)
  void *AcalT = nullptr, *YT = nullptr, *ZLT = nullptr, *ZRT = nullptr;  // transposed, rolling
  long long capA = 0, capCT = 0, capAcal = 0, capG = 0, capAcalT = 0, capYT = 0, capZLT = 0, capZRT = 0;
  // tensor maps: left G, A, Acal; right CT, YT, AcalT, ZLT, ZRT
  alignas(64) unsigned char maps[8][128];
};

// Digit slices of a float64 level with one block size m (m % 8 == 0,
// m <= 256) for the products on the tensor cores (dm_oz.cu): nine bf16
// slices per block ([block][slice][row][column]) and one exponent per row
// ([block][m] ints).  Full copies: A (rows), C^T (columns of C), Acal (rows);
// rolling, per subsystem: G_t (rows), Acal_t^T, Y_t^T, and two slots each of
// ZL^T, ZR^T (columns); Y: Y_{t+1} per subsystem in float64.
struct OzLevel {
  bool on = false;
  void *A = nullptr, *CT = nullptr, *Acal = nullptr, *G = nullptr;
  void *AcalT = nullptr, *YT = nullptr, *ZLT = nullptr, *ZRT = nullptr;
  int *eA = nullptr, *eCT = nullptr, *eAcal = nullptr, *eG = nullptr;
  int *eAcalT = nullptr, *eYT = nullptr, *eZLT = nullptr, *eZRT = nullptr;
  double* Y = nullptr;
  // tensor maps: left G, A, Acal; right CT, YT, AcalT, ZLT, ZRT
  alignas(64) unsigned char maps[8][128];
  // blocked Gauss-Jordan inversion: panel slices U, V ([subsystem][9][m][32]),
  // their exponents, the pivot rows, and the two panel maps
  bool gj = false;
  void *U = nullptr, *V = nullptr;
  int *eU = nullptr, *eV = nullptr, *piv = nullptr;
  alignas(64) unsigned char gj_maps[2][128];
  // the supplementary blocks on the tensor cores (levels with a supplementary level)
  bool asm_on = false;
  OzAsm as;
  // banded A and C: the largest |row - column| of a nonzero entry, found by
  // the input slicing on the device (null: detection off, DM_BANDED=0), and
  // its copy in page-locked host memory after each factorisation (for the
  // profiling costs of the next one; the device decides the path)
  int* band = nullptr;
  int* band_host = nullptr;
};

// One level of the recursion: a set of independent systems, each split into
// subsystems, with the float64 supplementary systems one level down.
struct Level {
  bool f32 = false;  // factors stored and multiplied in float32 (else float64)
  int tc_mode = -1;   // float32 factors: -1 CUDA cores, 0 tcgen05 TF32, 1 tcgen05 split bf16
  int* d_err = nullptr;  // set by a tensor-core kernel whose bounded wait expired
  float *A32 = nullptr, *B32 = nullptr, *C32 = nullptr;  // float32 copies streamed by the tensor-core sweeps
  alignas(64) unsigned char tmaps[3 * 128];  // TMA tensor maps of G, A32, Acal (TF32 level, one block size)
  bool has_tma = false;
  Tc2Level tc2;
  OzLevel oz;
  bool fp64_fma = false;  // float64 products on the FP64 pipe even where digit slicing applies
  bool inv_column = false;  // the column-by-column float64 inverse even where the blocked one applies
  int nsys = 0;
  std::vector<SysSpec> spec;
  std::vector<long long> blk0, vec0;  // per-system offsets of row 0
  long long nblk = 0, nvec = 0;       // elements of the [rows][m][m] and [rows][m][r] arrays
  int max_m = 1, max_r = 1, Nmax = 0, Lmax = 0, nparts = 0, nseps = 0;
  int nrows = 0;  // block rows of all systems
  std::vector<PartDesc> parts;
  std::vector<SepDesc> seps;
  std::vector<SysDesc> sysd;
  std::vector<int> active_fwd, active_back;  // subsystems still active at each step (prefix counts)
  // per-step launch costs
  std::vector<Cost> c_inv, c_fwd, c_back, c_fwds, c_backs;
  std::vector<Cost> c_fwdA, c_fwdB;  // the two launches of a forward step of the tensor-core step kernels
  std::vector<Cost> c_fwdA0;         // launch A's first product (G_t C_t) alone
  Cost c_cvt;                         // one operand conversion of the level's blocks
  std::vector<double> fwd_chain_frac;  // share of c_fwd[t] in the type-0 (chain) tiles
  std::vector<int> last_part;           // per system: index in parts of its last subsystem
  Cost c_asm_h, c_asm_f, c_backsub, c_resid, c_axpy, c_sepcopy;
  Cost c_resid_tc;     // the part of c_resid computed by the tensor-core residual
  int nres_tc = 0;     // systems whose residual runs on the tensor cores
  PartDesc* d_parts = nullptr;
  SepDesc* d_seps = nullptr;
  SysDesc* d_sys = nullptr;
  int* status = nullptr;
  double *A = nullptr, *B = nullptr, *C = nullptr;  // float64 blocks of the level's systems
  void *G = nullptr, *Acal = nullptr, *ZL = nullptr, *ZR = nullptr, *z = nullptr;
  double *F = nullptr, *X = nullptr;  // right-hand sides and solutions (supplementary: fh and h)
  std::unique_ptr<Level> supp;
  bool sweep = false;  // both z sweeps in one persistent cluster launch
  int sweep_cs = 0;    // its cluster size
  int depth = 0;  // 0 = the top level, 1 = its supplementary system, ...
  std::vector<void*> owned;

  int build(const std::vector<SysSpec>& specs, bool fp32_factors, int tensor_mode = -1);
  void release(void* p);  // free one owned buffer now
  bool lazy_inputs = false;  // A, B, C copies allocated at the first copying factor
  int ensure_inputs();
  void compute_costs();
  size_t bytes_needed() const;
  int allocate();
  ~Level();
};

// A captured launch sequence: the first use runs eagerly, the second captures
// it into a CUDA graph, later uses replay the graph.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  int uses = 0;
  long long launches = 0;  // kernels in one replay
  bool broken = false;     // capture failed: stay eager
};

struct Plan {
  int precision = 0;
  int device = 0;  // the CUDA device current at dm_plan: every launch of the plan goes there
  Level top;
  cudaStream_t stream = nullptr, own_stream = nullptr;
  double* R = nullptr;    // float64 residual
  double* Dx = nullptr;   // refinement correction
  double* nrm = nullptr;  // [nsys][4][kMaxR] column norms
  std::vector<double> h_nrm, relres;
  bool factored = false;
  double tol = 1e-12;
  int max_iters = 30;
  int last_iters = 0;
  double last_corr = 0.0;
  double factor_flops = 0, solve_flops = 0;
  size_t device_bytes = 0;
  Prof prof;
  Aux aux;
  bool use_graphs = true;
  GraphCache g_factor, g_solve, g_iter_first, g_iter_next;
  bool borrow = false;  // use the caller's device A, B, C in place (no copy)
  bool overlap = false;  // left-spike tiles on the side stream
  const double *bA = nullptr, *bB = nullptr, *bC = nullptr;
  int resid_mode = 0;  // DM_RESIDUAL_FP64 or DM_RESIDUAL_SLICED
  // complex systems (dm_plan_complex): the real embedding of block size 2m
  bool cplx = false;
  int cm = 0;                             // the complex block size m
  double *embA = nullptr, *embB = nullptr, *embC = nullptr;  // [N][2m][2m] real blocks
  double *cstage = nullptr;               // complex staging for host inputs / outputs
  double *bR = nullptr, *xR = nullptr;    // [N][2m][nrhs] real right-hand side / solution
  size_t cstage_bytes = 0;
  std::vector<void*> cbuf;                // the buffers above (freed with the plan)
  unsigned* rowhi = nullptr;  // per point row of the top level: largest high word of [A_i B_i C_i]'s row
  unsigned* colhi = nullptr;  // per block row x 16: largest high word of each column of x_i
  void row_scales();          // rowhi from the resident blocks (after each factorisation)
  void reset_graphs();
  int set_residual_mode(int mode);
  // r = b - T x (float64-accurate) with the column norms into nrm; all device pointers
  void residual(const double* x_dev, const double* b_dev, double* r_dev);
  int check_residual_error();
  template <typename F>
  int run(GraphCache& g, F&& body);

  int init(const std::vector<SysSpec>& specs, int precision);
  int solve_last(const double* b_last, double* x_last);
  int factor(const double* A, const double* B, const double* C);
  int solve(const double* b, double* x, double* relres_out);
  int solve_device(const double* b_dev, double* x_dev);
  // max ||b - T x|| / ||b|| over columns [c0, c0 + nc) of system 0's last solve
  double column_relres(int c0, int nc) const;
  ~Plan();
};

int set_error(int code, const char* fmt, ...);
extern thread_local std::string g_last_error;  // text of the calling thread's last failure

// Return DM_ECUDA with the failing call's text from an int-returning function.
#define DM_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return ::dm::set_error(DM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                              \
  } while (0)
void partition_plan(int N, int P, std::vector<int>& starts, std::vector<int>& lens, std::vector<int>& seps);
void partition_lengths(int N, int P, int m, int r, int flags, std::vector<int>& lens);
void nested_lengths(int N, int M, int J, std::vector<int>& lens);
int tuner_seed_p(int N, int m, int r);
int supp_partitions(int Ms, int P, int r, int m);
int make_spec(int N, int m, int r, int P, int levels, SysSpec* out);
void factor_level(Level& L, cudaStream_t st, Prof& pf, Aux* aux = nullptr);
void solve_level(Level& L, const double* F, double* X, cudaStream_t st, Prof& pf);
void level_flops(const Level& L, double* ffac, double* fsol);
int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t st);
int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st);
bool is_device_ptr(const void* p);

void serve_drain(struct dm_plan_s* plan);
bool tuned_lookup(int N, int m, int r, int prec, int* P, int* levels, int* flags = nullptr);
int autotune(int N, int m, int r, int prec, int* P_out, int* lv_out, double* ms_out, int* flags_out, bool variants);

}  // namespace dm

// The opaque handle of the C ABI.
struct dm_plan_s {
  dm::Plan plan;
};

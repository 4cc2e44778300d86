// Internal declarations shared by the solver's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dm {

// Flags of a subsystem (partition) descriptor.
enum : int {
  HAS_LEFT = 1,   // subsystem k > 0: spike for h^{k-1} (top block A of its first row)
  HAS_RIGHT = 2,  // subsystem k < P-1: spike for h^k (bottom block C of its last row)
};

// One subsystem S^k of one system (Section 2).  Its rows are contiguous in
// the system's row space; block offsets are element offsets into the level's
// [rows][m][m] arrays, vector offsets into its [rows][m][nrhs] arrays.
struct PartDesc {
  long long blk;    // offset of the subsystem's first row block
  long long vec;    // offset of the subsystem's first right-hand-side block
  long long hprev;  // offset of h^{k-1} in the supplementary level's vectors (HAS_LEFT)
  long long hnext;  // offset of h^k in the supplementary level's vectors (HAS_RIGHT)
  int m, r, L;      // block size, right-hand-side columns, rows of the subsystem
  int flags;
  int sys;          // system index within the level
  int row0;         // row index (within its system) of the subsystem's first row
};

// Separator row j of one system (between subsystems j and j+1).
enum : int { HAS_HA = 1, HAS_HC = 2 };
struct SepDesc {
  long long blk_q, vec_q;        // the separator row q
  long long blk_prev, vec_prev;  // row q-1 (last row of subsystem j)
  long long blk_next, vec_next;  // row q+1 (first row of subsystem j+1)
  long long hblk, hvec;          // row j of the supplementary system (its level's offsets)
  int m, r, flags, sys;
};

// One system of a level (for row-parallel kernels such as the residual).
struct SysDesc {
  long long blk, vec;  // offsets of row 0
  int N, m, r;
  int row0;            // first row of the system when the rows of all systems are numbered consecutively
  int sliced;          // residual on the tensor cores (k_residual_sliced) instead of float64 CUDA cores
  int eoff;            // offset of the system's rows in the per-row scale arrays (sum of N m before it)
};

// ---- launchers (dm_kernels.cu); T = double or float (factor storage type)
template <typename T>
void launch_inv(const PartDesc* parts, int nparts, int t, const double* B, T* G, int* status,
                int max_m, cudaStream_t st);
// type_lo..type_hi-1 select the tile types: 0 = Acal_t and the next Schur
// block (the inversion chain), 1 = left spike (off the chain).
template <typename T>
void launch_fwd_factor(const PartDesc* parts, int nparts, int t, int max_m, const double* A,
                       const double* B, const double* C, T* G, T* Acal, T* ZL, T* ZR, cudaStream_t st,
                       int type_lo = 0, int type_hi = 2);
template <typename T>
void launch_back_factor(const PartDesc* parts, int nparts, int s, int max_m, const T* Acal, T* ZL,
                        T* ZR, cudaStream_t st);
template <typename T>
void launch_fwd_solve(const PartDesc* parts, int nparts, int t, int max_m, int max_r,
                      const double* A, const T* G, const double* F, T* z, cudaStream_t st);
// Both right-hand-side sweeps of a level in one persistent launch (one
// cluster per subsystem); false when the level's shape needs the per-step
// kernels (more than 16 right-hand sides or panels beyond shared memory).
// Cluster size for the persistent solve sweep of `nparts` subsystems (0: use
// the per-step kernels).
int sweep_cluster_choice(int elem_bytes, int max_m, int max_r, int nparts);
template <typename T>
void launch_sweep_solve(const PartDesc* parts, int nparts, int cs, int max_m, int max_r, const double* A,
                        const T* G, const T* Acal, const double* F, T* z, cudaStream_t st);
template <typename T>
void launch_back_solve(const PartDesc* parts, int nparts, int s, int max_m, int max_r,
                       const T* Acal, T* z, cudaStream_t st);
template <typename T>
void launch_assemble_h(const SepDesc* seps, int nseps, int max_m, const double* A, const double* B,
                       const double* C, const T* ZL, const T* ZR, double* HA, double* HB,
                       double* HC, cudaStream_t st);
template <typename T>
void launch_assemble_f(const SepDesc* seps, int nseps, int max_m, int max_r, const double* A,
                       const double* C, const double* F, const T* z, double* fh, cudaStream_t st);
template <typename T>
void launch_backsub(const PartDesc* parts, int nparts, int Lmax, int max_m, int max_r, const T* ZL,
                    const T* ZR, const T* z, const double* h, double* x, cudaStream_t st);
void launch_sep_copy(const SepDesc* seps, int nseps, int max_m, int max_r, const double* h,
                     double* x, cudaStream_t st);
// r = b - T x (float64), per-system column norms: nrm[s*4*64 + 0*64 + c] = ||r_c||^2,
// [1] = ||b_c||^2 (both accumulated by atomics; zeroed by the caller).
// With `band` (a level's band flag, see OzOut::band) at most kBandMax, the A
// and C products run over the band only.
void launch_residual(const SysDesc* sys, int nsys, int nrows, int max_m, int max_r, const double* A,
                     const double* B, const double* C, const double* x, const double* b, double* r,
                     double* nrm, cudaStream_t st, const int* band = nullptr);
// x += d, nrm[2] += ||d_c||^2, nrm[3] += ||x_c||^2 (after the update)
// Residual b - T x of the systems with SysDesc::sliced set, float64-accurate
// from exact bf16 slice products on the tensor cores (m <= 128, r <= 16).
bool residual_sliced_fits(int m, int r);
// Per point row of the sliced systems: the largest high word (sign cleared)
// of the row of [A_i B_i C_i] -- computed once per factorisation.
void launch_row_scales(const SysDesc* sys, int nsys, int nrows, const double* A, const double* B,
                       const double* C, unsigned* rowhi, cudaStream_t st);
// Per block row of the sliced systems: the largest high word of each column
// of x_i ([global block row][16]), before each sliced residual.
void launch_col_scales(const SysDesc* sys, int nsys, int nrows, const double* x, unsigned* colhi, cudaStream_t st);
void launch_residual_sliced(const SysDesc* sys, int nsys, int nrows, const double* A, const double* B,
                            const double* C, const double* x, const double* b, double* r, double* nrm,
                            const unsigned* rowhi, const unsigned* colhi, int* errflag, cudaStream_t st);
void launch_axpy_norms(const SysDesc* sys, int nsys, int nrows, int max_m, int max_r, const double* d,
                       double* x, double* nrm, cudaStream_t st);

// tcgen05 block products of the float32 factor sweeps (dm_tc.cu); mode 0 =
// TF32, 1 = split bf16 (three products).  m <= 256.
// tmaps: host copy of the level's tensor maps (make_tma_maps) or nullptr.
void launch_fwd_factor_tc(int mode, const PartDesc* parts, int nparts, int t, int max_m, const float* A,
                          const float* B, const float* C, float* G, float* Acal, float* ZL, float* ZR,
                          int* errflag, cudaStream_t st, int type_lo, int type_hi, const void* tmaps);
void launch_to_f32(const double* src, float* dst, long long n, cudaStream_t st);
void launch_back_factor_tc(int mode, const PartDesc* parts, int nparts, int s, int max_m, const float* Acal,
                           float* ZL, float* ZR, int* errflag, cudaStream_t st, const void* tmaps);
bool make_tma_maps(const float* G, const float* A32, const float* Acal, long long rows, int m, void* out);
int tma_maps_bytes();
constexpr int kMaxMTensor = 256;
// Peak probe: one CTA per SM issuing back-to-back tcgen05 MMAs (mode 0 TF32,
// 1 bf16); returns the launch's flops.
double launch_mma_probe(int mode, int iters, int* errflag, cudaStream_t st);

// Tensor-core step kernels with TMA-fed operand copies (dm_tc2.cu); see
// Tc2Level.  kind 0: G_t [C_t | Y_t]; 1: A_{t+1} [Acal_t | Bcal_t];
// 2: Acal_t [ZL_{t+1} | ZR_{t+1}] (backward step).
// Destinations of the step kernels' epilogues (element offsets of the operand
// copies are block index x m^2; `cap_*` are the copies' block capacities,
// i.e. where their lo parts start).
struct Tc2Out {
  const float* B32;
  float *G, *Acal, *ZL, *ZR;
  void *acal_l, *acalT, *yT, *zlT, *zrT;
  long long cap_acal_l, cap_acalT, cap_yT, cap_zlT, cap_zrT;
};
bool tc2_eligible(int m);

// Float64 products on the tensor cores by exact digit slicing (dm_oz.cu):
// the step kernels' products with float64 operands and results, the operands
// as nine bf16 digit slices with per-row (left) / per-column (right) scales.
struct OzOut {
  const double* B;
  double *G, *Acal, *ZL, *ZR, *Y;  // Y: Y_{t+1} per subsystem (rolling, float64)
  // the supplementary blocks (Eq. e2311), one separator per CTA row
  const SepDesc* seps;
  double *HA, *HB, *HC;
  // the level's largest |row - column| of a nonzero entry of A and C (null:
  // not detected); at most kBandMax: the products with a banded operand run
  // in the banded kernels and the tensor-core tiles for them are skipped
  const int* band;
};
constexpr int kBandMax = 6;
bool oz_eligible(int m);
int oz_slice_blocks_bytes(int m);
bool oz_make_map(const void* base, long long blocks, int m, int box_rows, void* out, int kdim = 0);
int oz_box_rows_left();
int oz_box_rows_right();
int oz_box_rows_gj();  // rows of the right operand's box in the inverse's trailing updates
// The supplementary blocks of a sliced level (Eq. e2311) as digit-sliced
// products: C_q row slices and the four boundary spike blocks' column slices
// per separator, then HB = B_q - A_q ZR - C_q ZL, HA = -A_q ZL, HC = -C_q ZR.
struct OzAsm {
  void *Cq, *S;   // [separator][9][m][m] C_q rows; [4 separator + b][9][m][m] spike columns
  int *eCq, *eS;  // their scales
  alignas(64) unsigned char maps[2][128];  // left Cq, right S
};
void launch_oz_assemble(const SepDesc* seps, int nseps, int m, const double* B, const double* C, const double* ZL,
                        const double* ZR, double* HA, double* HB, double* HC, const OzAsm& a, const int* eA,
                        const void* mapA, int* errflag, const int* band, cudaStream_t st);
void launch_oz_slice_all(bool cols, const double* src, int nblocks, int m, void* dst, int* exps, const int* band,
                         cudaStream_t st);
// The level's band into *band (atomicMax; the caller zeroes it first): the
// largest |row - column| of a nonzero entry of the n entries of A and of C.
void launch_band_detect(const double* A, const double* C, long long n, int m, int* band, cudaStream_t st);
// Products with a banded operand (half-bandwidth w = *band <= kBandMax, else
// nothing is done): G_t C_t of launch A, both products of launch B, and the
// supplementary blocks; float64 multiply-adds over the band only.
void launch_band_gc(const PartDesc* parts, int nparts, int t, int m, const double* G, const double* C, double* Acal,
                    double* ZR, const int* band, cudaStream_t st);
void launch_band_b(const PartDesc* parts, int nparts, int t, int m, const double* A, const double* B,
                   const double* Acal, const double* ZL, double* G, double* Y, const int* band, cudaStream_t st);
void launch_band_h(const SepDesc* seps, int nseps, int m, const double* A, const double* B, const double* C,
                   const double* ZL, const double* ZR, double* HA, double* HB, double* HC, const int* band,
                   cudaStream_t st);
struct OzSliceJob {
  const double* src;
  void* dst;
  int* exps;
  int kind;  // see k_oz_slice_jobs
};
struct OzSliceJobs {
  OzSliceJob job[4];
  const int* band = nullptr;  // kinds 2 and 3 (launch B's operands) are skipped when banded
};
void launch_oz_slice_jobs(const PartDesc* parts, int nparts, int step, int m, const OzSliceJobs& jobs, int njobs,
                          cudaStream_t st);
void launch_oz_step(int kind, const PartDesc* parts, int nparts, int step, int m, const OzOut& out, const int* lexp,
                    const int* rexp0, const int* rexp1, const void* maps3, int* errflag, cudaStream_t st,
                    int aux = 0);
// Blocked Gauss-Jordan inversion with the rank-32 updates as digit-sliced
// tensor-core products; maps2 = the panel-slice maps (U with 128-row boxes,
// V with 48-row boxes), piv [nparts][m] (the column permutation), Us / Vs
// [nparts][9][m][32] bf16, Uexp / Vexp [nparts][m]; Gs / eG receive the row
// slices of the inverses ([nparts][9][m][m] bf16, [nparts][m]).
void launch_gj_inverse(const PartDesc* parts, int nparts, int t, int m, const double* B, double* G, int* piv,
                       void* Us, int* Uexp, void* Vs, int* Vexp, const void* maps2, int* status, int* errflag,
                       void* Gs, int* eG, cudaStream_t st);
// its phases (launch_gj_inverse runs them in order)
void launch_gj_begin(const PartDesc* parts, int nparts, int t, int m, const double* B, double* G, cudaStream_t st);
void launch_gj_panel(const PartDesc* parts, int nparts, int t, int m, int pnl, double* G, int* piv, void* Us,
                     int* Uexp, void* Vs, int* Vexp, int* status, cudaStream_t st);
void launch_gj_update(const PartDesc* parts, int nparts, int t, int m, int pnl, double* G, const int* Uexp,
                      const int* Vexp, const void* maps2, int* errflag, cudaStream_t st);
void launch_gj_finish(const PartDesc* parts, int nparts, int t, int m, double* G, const int* piv, void* Gs, int* eG,
                      cudaStream_t st);
int tc2_ntile(int m);
bool tc2_make_map(int mode, const void* base, long long blocks, int m, int box_rows, void* out);
int tc2_map_bytes();
void launch_tc2_convert(int mode, const double* src64, const float* src32, const PartDesc* parts, int nq, int t, int m,
                        bool trans, void* dst, long long cap_blocks, cudaStream_t st);
void launch_tc2_step(int mode, int kind, const PartDesc* parts, int nparts, int step, int m, const int lo[3],
                     const Tc2Out& out, const void* maps3, int* errflag, cudaStream_t st);

constexpr int kMaxM = 512;
constexpr int kMaxR = 64;

}  // namespace dm

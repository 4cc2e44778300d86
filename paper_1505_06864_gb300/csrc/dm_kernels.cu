// Level-synchronous block kernels of the decomposition method (SIMT path).
//
// Every kernel works on a table of subsystems (PartDesc) or separators
// (SepDesc) so that one launch advances the same step of every subsystem of
// every system in a level: step t of the forward sweep processes row t of all
// subsystems at once (Section 3's recurrences run down each subsystem, the
// subsystems are independent, Section 2).  Block products are computed in
// "panels": all m rows of an m x W slab of the result, W = 32 (m <= 256) or
// 16 (m <= 512) columns, so a CTA can chain two products on the same slab
// (e.g. Acal_t = G_t C_t followed by D_{t+1} = B_{t+1} - A_{t+1} Acal_t).
//
// T is the factor storage/arithmetic type: double for DM_FP64 and for every
// supplementary level, float for the mixed-precision top level (its block
// products on CUDA cores; the tcgen05 kernels replace them where enabled).
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>
#include <unordered_map>

#include <cooperative_groups.h>

#include "dm_internal.cuh"

namespace dm {

namespace {

constexpr int kThreads = 256;  // 16 x 16 thread grid of the panel products

// ---------------------------------------------------------------------------
// Panel product core.  Computes rows r0..r0+63 of L (m x m, row-major, leading
// dimension m, element type TL) times Rs (m x W in shared memory, row stride
// W), accumulating into acc.  Thread (ty, tx) owns rows r0 + ty + 16a (a < 4)
// and columns tx + 16b (b < W/16).  Lc holds two 64 x 17 staging tiles for L.
template <typename T, typename TL, int W>
__device__ __forceinline__ void mm_rowblock(T (&acc)[4][W / 16], const TL* __restrict__ L, int m,
                                            int r0, const T* __restrict__ Rs, T* __restrict__ Lc) {
  // Lc holds two 64 x 17 staging tiles: the chunk being multiplied and the
  // next one, whose global loads are issued before the current chunk's FMAs.
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  constexpr int PER = 64 * 16 / kThreads;  // elements per thread per chunk
  T nxt[PER];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * kThreads;
      const int rr = e >> 4, kk = e & 15, row = r0 + rr, col = k0 + kk;
      nxt[u] = (row < m && col < m) ? (T)L[(long long)row * m + col] : (T)0;
    }
  };
  auto stash = [&](T* buf) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * kThreads;
      buf[(e >> 4) * 17 + (e & 15)] = nxt[u];
    }
  };
  fetch(0);
  stash(Lc);
  __syncthreads();
  int cur = 0;
  for (int k0 = 0; k0 < m; k0 += 16) {
    const bool more = k0 + 16 < m;
    if (more) fetch(k0 + 16);
    const T* Lt = Lc + cur * (64 * 17);
    const int kmax = min(16, m - k0);
    for (int kk = 0; kk < kmax; ++kk) {
      T lv[4], rv[W / 16];
#pragma unroll
      for (int a = 0; a < 4; ++a) lv[a] = Lt[(ty + 16 * a) * 17 + kk];
#pragma unroll
      for (int b = 0; b < W / 16; ++b) rv[b] = Rs[(k0 + kk) * W + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < W / 16; ++b) acc[a][b] = fma(lv[a], rv[b], acc[a][b]);
    }
    if (more) stash(Lc + (cur ^ 1) * (64 * 17));
    __syncthreads();
    cur ^= 1;
  }
}

// out = L1 * R1 (+ L2 * R2 when L2 != nullptr), delivered element by element
// to epi(row, col, value) for row < m and every col < W.
template <typename T, typename TL1, typename TL2, int W, typename Epi>
__device__ __forceinline__ void panel_mm(int m, const TL1* L1, const T* R1, const TL2* L2,
                                         const T* R2, T* Lc, Epi epi) {
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int r0 = 0; r0 < m; r0 += 64) {
    T acc[4][W / 16];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < W / 16; ++b) acc[a][b] = (T)0;
    mm_rowblock<T, TL1, W>(acc, L1, m, r0, R1, Lc);
    if (L2 != nullptr) mm_rowblock<T, TL2, W>(acc, L2, m, r0, R2, Lc);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int row = r0 + ty + 16 * a;
      if (row < m) {
#pragma unroll
        for (int b = 0; b < W / 16; ++b) epi(row, tx + 16 * b, acc[a][b]);
      }
    }
  }
}

// Rs[k][c] = scale * src[k * ld + c0 + c] for k < rows, c < W; zero past `cols`.
template <typename T, typename TS, int W>
__device__ __forceinline__ void load_panel(T* Rs, const TS* __restrict__ src, int rows, int ld,
                                           int c0, int cols, T scale) {
  for (int e = threadIdx.x; e < rows * W; e += kThreads) {
    const int k = e / W, c = e - k * W;
    Rs[e] = (c0 + c < cols) ? scale * (T)src[(long long)k * ld + c0 + c] : (T)0;
  }
}

template <typename T>
__host__ __device__ constexpr size_t panel_smem(int m, int W, int npanels) {
  return sizeof(T) * ((size_t)npanels * m * W + 2 * 64 * 17);
}

template <int W>
__host__ __device__ constexpr int ntiles(int cols) { return (cols + W - 1) / W; }

// ---------------------------------------------------------------------------
// Block inverse G_t = D_t^{-1} by Gauss-Jordan elimination with partial
// (row) pivoting, in place (m^3 multiply-adds, the paper's cost for an
// inversion in Section 4).  One CTA per subsystem.  D_t was written into G's
// row-t slot by the previous forward step; at t = 0 it is B of the
// subsystem's first row.  The working matrix lives in shared memory when it
// fits, else in the G slot itself (global memory, L2-resident).
template <typename T>
__global__ void __launch_bounds__(512) k_inv(const PartDesc* __restrict__ parts, int t,
                                             const double* __restrict__ B, T* __restrict__ G,
                                             int* __restrict__ status, int smem_max_m) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.x];
  if (t >= p.L) return;
  const int m = p.m;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const long long o = p.blk + (long long)t * m * m;
  T* g = G + o;
  int* perm = reinterpret_cast<int*>(smem_raw);
  int* idx = perm + kMaxM;
  T* colk = reinterpret_cast<T*>(idx + kMaxM);
  T* rowk = colk + kMaxM;
  __shared__ int s_p, s_bad;
  __shared__ T s_inv, s_akk, s_apk;
  const bool in_smem = m <= smem_max_m;
  T* a;
  int lda;
  if (in_smem) {
    a = rowk + kMaxM;
    lda = m + 1;
  } else {
    a = g;
    lda = m;
  }
  if (tid == 0) s_bad = 0;
  const int i0 = tid >> 5, istep = nthr >> 5, j0 = tid & 31;
  if (t == 0) {
    const double* bsrc = B + o;
    for (int i = i0; i < m; i += istep)
      for (int j = j0; j < m; j += 32) a[i * lda + j] = (T)bsrc[(long long)i * m + j];
  } else if (in_smem) {
    for (int i = i0; i < m; i += istep)
      for (int j = j0; j < m; j += 32) a[i * lda + j] = g[(long long)i * m + j];
  }
  __syncthreads();

  for (int k = 0; k < m; ++k) {
    if (tid < 32) {
      // pivot search over rows k..m-1 of column k; ties go to the lowest row
      T best = (T)-1;
      int bi = k;
      for (int i = k + tid; i < m; i += 32) {
        const T v = fabs(a[i * lda + k]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        const T akk = a[k * lda + k], apk = a[bi * lda + k];
        T inv = (T)1 / apk;
        if (!(fabs(apk) > (T)0) || !isfinite(inv)) {
          s_bad = 1;
          inv = (T)0;
        }
        perm[k] = bi;
        s_p = bi;
        s_inv = inv;
        s_akk = akk;
        s_apk = apk;
      }
    }
    __syncthreads();
    const int pr = s_p;
    const T inv = s_inv;
    for (int j = tid; j < m; j += nthr) {
      const T vk = a[k * lda + j], vp = a[pr * lda + j];
      if (pr != k) {
        a[k * lda + j] = vp;
        a[pr * lda + j] = vk;
      }
      rowk[j] = vp * inv;
    }
    for (int i = tid; i < m; i += nthr)
      colk[i] = (i == k) ? s_apk : (i == pr ? s_akk : a[i * lda + k]);
    __syncthreads();
    for (int i = i0; i < m; i += istep) {
      const T ci = colk[i];
      if (i == k) {
        for (int j = j0; j < m; j += 32) a[i * lda + j] = (j == k) ? inv : rowk[j];
      } else {
        for (int j = j0; j < m; j += 32)
          a[i * lda + j] = (j == k) ? -ci * inv : fma(-ci, rowk[j], a[i * lda + j]);
      }
    }
    __syncthreads();
  }
  // D^{-1} = inv(Pi D) Pi: undo the row exchanges on the columns, last first.
  if (in_smem) {
    if (tid == 0) {
      for (int c = 0; c < m; ++c) idx[c] = c;
      for (int k = m - 1; k >= 0; --k) {
        const int q = perm[k];
        const int tmp = idx[k];
        idx[k] = idx[q];
        idx[q] = tmp;
      }
    }
    __syncthreads();
    for (int i = i0; i < m; i += istep)
      for (int j = j0; j < m; j += 32) g[(long long)i * m + j] = a[i * lda + idx[j]];
  } else {
    for (int k = m - 1; k >= 0; --k) {
      const int q = perm[k];
      if (q != k) {
        for (int i = tid; i < m; i += nthr) {
          const T v = a[i * lda + k];
          a[i * lda + k] = a[i * lda + q];
          a[i * lda + q] = v;
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0 && s_bad) atomicMin(status + p.sys, p.row0 + t + 1);
}

// ---------------------------------------------------------------------------
// The same block inverse with the columns split over a thread-block cluster
// of `cs` CTAs: CTA r keeps columns [r w, (r+1) w) of the working matrix in
// its shared memory (w = ceil(m / cs)).  Step k: the CTA owning column k
// searches the pivot in that column, exchanges rows k and p in it and
// publishes the column (and p) in its shared memory; one cluster barrier;
// every CTA reads the published column through distributed shared memory,
// exchanges rows k and p in its own columns and applies the rank-1 update to
// them.  The published column is double-buffered: a CTA can only overwrite
// buffer k&1 at step k+2, after every CTA has passed step k+1's barrier and
// therefore finished reading it.  No CTA of a cluster returns early except
// all together, and a final barrier keeps every CTA's shared memory alive
// until the last remote read.
template <typename T>
__global__ void __launch_bounds__(256) k_inv_cluster(const PartDesc* __restrict__ parts, int t,
                                                     const double* __restrict__ B, T* __restrict__ G,
                                                     int* __restrict__ status, int cs) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const PartDesc p = parts[blockIdx.x / cs];
  if (t >= p.L) return;  // the same for every CTA of the cluster
  const int m = p.m;
  const int w = (m + cs - 1) / cs, c0 = rank * w, wc = max(0, min(w, m - c0));
  const int lda = w + 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  T* pub = reinterpret_cast<T*>(smem_raw);  // [2][kMaxM]
  T* colk = pub + 2 * kMaxM;                // [kMaxM]
  T* rowk = colk + kMaxM;                   // [128]
  T* a = rowk + 128;                        // [m][w+1]
  int* perm = reinterpret_cast<int*>(a + (size_t)m * lda);  // [kMaxM]
  int* idx = perm + kMaxM;                                  // [kMaxM]
  int* inv_idx = idx + kMaxM;                               // [kMaxM]
  __shared__ int pubp[2];
  __shared__ int s_bad;
  const long long o = p.blk + (long long)t * m * m;
  T* g = G + o;
  if (tid == 0) s_bad = 0;
  for (int e = tid; e < m * wc; e += nthr) {
    const int i = e / wc, jl = e - i * wc;
    a[i * lda + jl] = (t == 0) ? (T)B[o + (long long)i * m + c0 + jl] : g[(long long)i * m + c0 + jl];
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  // Pivot search over rows k..m-1 of local column kl (ties to the lowest row)
  // by one warp, then publication of the column as it reads after exchanging
  // rows k and p, into pub[k & 1] / pubp[k & 1].
  auto search_publish = [&](int k, int kl) {
    T best = (T)-1;
    int bi = k;
    for (int i = k + lane; i < m; i += 32) {
      const T v = fabs(a[i * lda + kl]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T ob = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    bi = __shfl_sync(0xffffffffu, bi, 0);
    const T akk = a[k * lda + kl], apk = a[bi * lda + kl];
    T* pb = pub + (k & 1) * kMaxM;
    for (int i = lane; i < m; i += 32) pb[i] = (i == k) ? apk : (i == bi ? akk : a[i * lda + kl]);
    if (lane == 0) pubp[k & 1] = bi;
  };
  if (rank == 0 && warp == 0) search_publish(0, 0);  // step 0's column is owned by CTA 0
  for (int k = 0; k < m; ++k) {
    const int owner = k / w, kl = k - owner * w;
    const int buf = k & 1;
    const bool own = (rank == owner);
    cl.sync();  // step k's pivot column is published
    const T* rb = cl.map_shared_rank(pub + buf * kMaxM, owner);
    const int pr = *cl.map_shared_rank(&pubp[buf], owner);
    const T piv = rb[k];
    T inv = (T)1 / piv;
    if (!(fabs(piv) > (T)0) || !isfinite(inv)) {
      inv = (T)0;
      if (tid == 0 && own) s_bad = 1;
    }
    for (int i = tid; i < m; i += nthr) colk[i] = rb[i];
    for (int jl = tid; jl < wc; jl += nthr) {
      const T vk = a[k * lda + jl], vp = a[pr * lda + jl];
      if (pr != k) {
        a[k * lda + jl] = vp;
        a[pr * lda + jl] = vk;
      }
      rowk[jl] = vp * inv;
    }
    if (tid == 0) perm[k] = pr;
    __syncthreads();
    // lookahead: the owner of column k+1 updates that column first, and its
    // warp 0 searches and publishes step k+1's pivot column while the other
    // warps apply the rest of step k's update
    const int k1 = k + 1, owner1 = k1 < m ? k1 / w : -1, kl1 = k1 - owner1 * w;
    const bool next_here = (rank == owner1);
    if (next_here) {
      const T rj = rowk[kl1];
      for (int i = tid; i < m; i += nthr)
        a[i * lda + kl1] = (i == k) ? rj : fma(-colk[i], rj, a[i * lda + kl1]);
      __syncthreads();
    }
    const bool searcher = next_here && warp == 0;
    if (searcher) search_publish(k1, kl1);
    // rank-1 update of the local columns (column k+1 done above); rowk in registers
    const int w0 = next_here ? 1 : 0, nw = nwarp - w0;
    if (!searcher) {
      for (int jl = lane; jl < wc; jl += 32) {
        if (next_here && jl == kl1) continue;
        const T rj = rowk[jl];
        int i = warp - w0;
        for (; i + 3 * nw < m; i += 4 * nw) {
          const int i1 = i + nw, i2 = i + 2 * nw, i3 = i + 3 * nw;
          const T c0v = colk[i], c1v = colk[i1], c2v = colk[i2], c3v = colk[i3];
          const T a0 = a[i * lda + jl], a1 = a[i1 * lda + jl], a2 = a[i2 * lda + jl], a3 = a[i3 * lda + jl];
          a[i * lda + jl] = (i == k) ? rj : fma(-c0v, rj, a0);
          a[i1 * lda + jl] = (i1 == k) ? rj : fma(-c1v, rj, a1);
          a[i2 * lda + jl] = (i2 == k) ? rj : fma(-c2v, rj, a2);
          a[i3 * lda + jl] = (i3 == k) ? rj : fma(-c3v, rj, a3);
        }
        for (; i < m; i += nw) a[i * lda + jl] = (i == k) ? rj : fma(-colk[i], rj, a[i * lda + jl]);
      }
    }
    __syncthreads();
    // column k itself becomes the k-th column of the running inverse
    if (own)
      for (int i = tid; i < m; i += nthr) a[i * lda + kl] = (i == k) ? inv : -colk[i] * inv;
  }
  cl.sync();  // every remote read of this CTA's buffers is done
  if (tid == 0) {
    for (int c = 0; c < m; ++c) idx[c] = c;
    for (int k = m - 1; k >= 0; --k) {
      const int q = perm[k];
      const int tmp = idx[k];
      idx[k] = idx[q];
      idx[q] = tmp;
    }
    for (int c = 0; c < m; ++c) inv_idx[idx[c]] = c;
  }
  __syncthreads();
  // column c0 + jl of inv(Pi D) is column inv_idx[c0 + jl] of D^{-1}
  for (int e = tid; e < m * wc; e += nthr) {
    const int i = e / wc, jl = e - i * wc;
    g[(long long)i * m + inv_idx[c0 + jl]] = a[i * lda + jl];
  }
  if (tid == 0 && s_bad) atomicMin(status + p.sys, p.row0 + t + 1);
}

// ---------------------------------------------------------------------------
// Blocked form of the same Gauss-Jordan inverse (partial pivoting inside the
// block, column unscramble at the end): the columns are processed in panels
// of NB.  The CTA that owns a panel's columns eliminates the panel alone (one
// warp, warp-synchronous: pivot search by shuffles, row exchange, scaling and
// elimination restricted to the panel), which leaves the panel holding the
// NB non-trivial columns of the panel's composed elimination matrix
// M = I + X.  After one cluster barrier every CTA copies the panel and its
// pivots (distributed shared memory), applies the exchanges to its own
// columns, keeps the NB pivot rows Y, and applies the rank-NB update
//   a[i][j] <- (i a pivot row of the panel ? 0 : a[i][j]) + sum_l M[i][l] Y[l][j]
// to its other columns.  Lookahead: the owner of the next panel updates that
// panel's columns first, and its warp 0 eliminates the next panel while the
// other warps finish the update, so a panel costs one cluster barrier and the
// elimination of the next panel is hidden behind the update.  All loop bounds
// are uniform over the cluster; a final barrier keeps every CTA's shared
// memory alive until the last remote read.
struct InvPanel {
  int owner, kl0, nbk, k0;
};

__host__ __device__ __forceinline__ size_t up16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T, int NB>
__host__ __device__ size_t inv_blocked_layout(int m, int w, size_t* off_pan, size_t* off_y, size_t* off_perm) {
  const size_t a = up16(sizeof(T) * (size_t)m * (w + 1));
  const size_t pan = up16(sizeof(T) * (size_t)m * NB);
  const size_t y = up16(sizeof(T) * (size_t)NB * w);
  if (off_pan) *off_pan = a;
  if (off_y) *off_y = a + pan;
  if (off_perm) *off_perm = a + pan + y;
  return a + pan + y + 3 * sizeof(int) * (size_t)m;
}

template <typename T, int NB>
__global__ void __launch_bounds__(256) k_inv_blocked(const PartDesc* __restrict__ parts, int t,
                                                     const double* __restrict__ B, T* __restrict__ G,
                                                     int* __restrict__ status, int cs) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const PartDesc p = parts[blockIdx.x / cs];
  if (t >= p.L) return;  // the same for every CTA of the cluster
  const int m = p.m;
  const int w = (m + cs - 1) / cs, c0 = rank * w, wc = max(0, min(w, m - c0));
  const int lda = w + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  size_t op, oy, oq;
  inv_blocked_layout<T, NB>(m, w, &op, &oy, &oq);
  T* a = reinterpret_cast<T*>(smem_raw);           // [m][lda]: this CTA's columns
  T* pan = reinterpret_cast<T*>(smem_raw + op);    // [m][NB]: the current panel
  T* Y = reinterpret_cast<T*>(smem_raw + oy);      // [NB][w]: pivot rows of the own columns
  int* perm = reinterpret_cast<int*>(smem_raw + oq);
  int* idx = perm + m;
  int* inv_idx = idx + m;
  __shared__ int s_bad;
  const long long o = p.blk + (long long)t * m * m;
  T* g = G + o;
  if (tid == 0) s_bad = 0;
  for (int e = tid; e < m * wc; e += blockDim.x) {
    const int i = e / wc, jl = e - i * wc;
    a[i * lda + jl] = (t == 0) ? (T)B[o + (long long)i * m + c0 + jl] : g[(long long)i * m + c0 + jl];
  }
  __syncthreads();

  // panels in column order: owner r, local columns [kl0, kl0 + nbk)
  auto owner_cols = [&](int r) { return max(0, min(w, m - r * w)); };
  auto first_panel = [&]() { return InvPanel{0, 0, min(NB, owner_cols(0)), 0}; };
  auto next_panel = [&](InvPanel q) {
    q.kl0 += NB;
    if (q.kl0 >= owner_cols(q.owner)) {
      q.owner += 1;
      q.kl0 = 0;
    }
    q.nbk = q.owner < cs ? min(NB, owner_cols(q.owner) - q.kl0) : 0;
    q.k0 = q.owner * w + q.kl0;
    return q;
  };

  // Elimination of a panel by one warp (columns kl0.. of this CTA, rows 0..m-1).
  auto eliminate = [&](const InvPanel& q) {
    for (int j = 0; j < q.nbk; ++j) {
      const int k = q.k0 + j, kl = q.kl0 + j;
      T best = (T)-1;
      int bi = k;
      for (int i = k + lane; i < m; i += 32) {
        const T v = fabs(a[i * lda + kl]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      bi = __shfl_sync(0xffffffffu, bi, 0);
      if (bi != k && lane < q.nbk) {
        T* rk = a + k * lda + q.kl0 + lane;
        T* rp = a + bi * lda + q.kl0 + lane;
        const T tmp = *rk;
        *rk = *rp;
        *rp = tmp;
      }
      if (lane == 0) perm[k] = bi;
      __syncwarp();
      const T piv = a[k * lda + kl];
      T inv = (T)1 / piv;
      if (!(fabs(piv) > (T)0) || !isfinite(inv)) {
        inv = (T)0;
        if (lane == 0) s_bad = 1;
      }
      T rk[NB];
#pragma unroll
      for (int l = 0; l < NB; ++l) rk[l] = l < q.nbk ? a[k * lda + q.kl0 + l] * inv : (T)0;
      __syncwarp();
      for (int i = lane; i < m; i += 32) {
        T* ai = a + i * lda + q.kl0;
        if (i == k) {
#pragma unroll
          for (int l = 0; l < NB; ++l)
            if (l < q.nbk) ai[l] = (l == j) ? inv : rk[l];
        } else {
          const T cik = ai[j];
#pragma unroll
          for (int l = 0; l < NB; ++l)
            if (l < q.nbk) ai[l] = (l == j) ? -cik * inv : fma(-cik, rk[l], ai[l]);
        }
      }
      __syncwarp();
    }
  };

  // Rank-NB update of local columns jl in [lo, hi) except [x0, x1) and
  // [y0, y1), by warps wf .. wf + nw - 1 (lanes over columns, warps over rows).
  auto update = [&](const InvPanel& q, int lo, int hi, int x0, int x1, int y0, int y1, int wf, int nw) {
    const int wi = warp - wf;
    if (wi < 0 || wi >= nw) return;
    for (int jl = lo + lane; jl < hi; jl += 32) {
      if ((jl >= x0 && jl < x1) || (jl >= y0 && jl < y1)) continue;
      T yc[NB];
#pragma unroll
      for (int l = 0; l < NB; ++l) yc[l] = Y[l * w + jl];
      for (int i = wi; i < m; i += nw) {
        const T* pi = pan + i * NB;
        T acc = (i >= q.k0 && i < q.k0 + q.nbk) ? (T)0 : a[i * lda + jl];
#pragma unroll
        for (int l = 0; l < NB; ++l) acc = fma(pi[l], yc[l], acc);
        a[i * lda + jl] = acc;
      }
    }
  };

  InvPanel q = first_panel();
  if (rank == q.owner && warp == 0) eliminate(q);
  while (q.owner < cs && q.nbk > 0) {
    cl.sync();  // panel q eliminated by its owner
    const bool own = rank == q.owner;
    const T* ra = cl.map_shared_rank(a, q.owner);
    const int* rperm = cl.map_shared_rank(perm, q.owner);
    for (int e = tid; e < m * NB; e += blockDim.x) {
      const int i = e / NB, l = e - i * NB;
      pan[e] = l < q.nbk ? ra[i * lda + q.kl0 + l] : (T)0;
    }
    if (tid < q.nbk) perm[q.k0 + tid] = rperm[q.k0 + tid];
    __syncthreads();
    // exchanges and pivot rows of the own columns (the owner's panel excluded)
    const int x0 = own ? q.kl0 : 0, x1 = own ? q.kl0 + q.nbk : 0;
    for (int jl = tid; jl < wc; jl += blockDim.x) {
      if (jl >= x0 && jl < x1) continue;
      for (int l = 0; l < q.nbk; ++l) {
        const int k = q.k0 + l, pr = perm[k];
        if (pr != k) {
          const T tmp = a[k * lda + jl];
          a[k * lda + jl] = a[pr * lda + jl];
          a[pr * lda + jl] = tmp;
        }
      }
#pragma unroll
      for (int l = 0; l < NB; ++l) Y[l * w + jl] = l < q.nbk ? a[(q.k0 + l) * lda + jl] : (T)0;
    }
    __syncthreads();
    const InvPanel q1 = next_panel(q);
    const bool next_here = q1.owner < cs && q1.nbk > 0 && rank == q1.owner;
    if (next_here) {
      update(q, q1.kl0, q1.kl0 + q1.nbk, x0, x1, 0, 0, 0, 8);
      __syncthreads();
      if (warp == 0)
        eliminate(q1);
      else
        update(q, 0, wc, x0, x1, q1.kl0, q1.kl0 + q1.nbk, 1, 7);
    } else {
      update(q, 0, wc, x0, x1, 0, 0, 0, 8);
    }
    q = q1;
  }
  cl.sync();  // every remote read of this CTA's columns is done
  if (tid == 0) {
    for (int c = 0; c < m; ++c) idx[c] = c;
    for (int k = m - 1; k >= 0; --k) {
      const int r = perm[k];
      const int tmp = idx[k];
      idx[k] = idx[r];
      idx[r] = tmp;
    }
    for (int c = 0; c < m; ++c) inv_idx[idx[c]] = c;
  }
  __syncthreads();
  for (int e = tid; e < m * wc; e += blockDim.x) {
    const int i = e / wc, jl = e - i * wc;
    g[(long long)i * m + inv_idx[c0 + jl]] = a[i * lda + jl];
  }
  if (tid == 0 && s_bad) atomicMin(status + p.sys, p.row0 + t + 1);
}

// ---------------------------------------------------------------------------
// Register-resident Gauss-Jordan inverse (Section 3's explicit block inverse;
// partial pivoting inside the block), columns split over a cluster of cs CTAs
// (cs = 1: one CTA).  Each CTA holds the m x w slab of its columns in
// registers: a 32 x 32 thread grid, thread (ty = lane, tx = warp) owning rows
// ty + 32a (a < RT) and local columns tx + 32b (b < CT), so a warp holds whole
// columns.  Pivoting is implicit: rows are never exchanged; step k takes the
// unused row p_k with the largest |a[i][k]| as its pivot row, and the working
// matrix ends as W[p_r][c] = inv(D)[r][p_c], written out in that order.
// Step k (one barrier):
//   * the warp owning column k (in the owner CTA) has published the column,
//     p_k and 1 / pivot (its pivot search ran at the end of step k-1:
//     warp-wide max of |a| then min of the row index among the maxima);
//   * every thread reads the column for its rows (distributed shared memory
//     in a cluster), takes row p_k of its columns from lane p_k mod 32 of its
//     own warp by a shuffle, and applies the rank-1 update in registers,
//     fixing up row p_k and column k;
//   * the warp owning column k+1 searches and publishes its pivot.
// The slab is staged through shared memory on entry and exit (coalesced
// global traffic).  Loop bounds are uniform over the cluster; a final barrier
// keeps every CTA's shared memory alive until the last remote read.
constexpr int kInvRegThreads = 1024;

template <typename T>
__host__ __device__ size_t inv_reg_smem(int m, int w) {
  // slab [m][w+1] + published columns [2][m] + published reciprocals [2] (T),
  // then pivot row per step [m] and published pivot rows [2] (int)
  return sizeof(T) * ((size_t)m * (w + 1) + 2 * (size_t)m + 2) + sizeof(int) * ((size_t)m + 2);
}

// f(integral_constant<I>) for the I in [0, N) equal to v (uniform v: one
// branch taken, the others skipped), so register arrays stay statically
// indexed.
template <int N, int I = 0, typename F>
__device__ __forceinline__ void dispatch_index(int v, F&& f) {
  if constexpr (I < N) {
    if (v == I)
      f(std::integral_constant<int, I>());
    else
      dispatch_index<N, I + 1>(v, f);
  }
}

// Warp-wide argmax of v >= 0 (lowest index among equal maxima; lanes
// without a candidate pass idx = m).
__device__ __forceinline__ int warp_argmax(float v, int idx) {
  const unsigned bits = idx < INT_MAX ? __float_as_uint(v) : 0u;
  const unsigned vmax = __reduce_max_sync(0xffffffffu, bits);
  return (int)__reduce_min_sync(0xffffffffu, bits == vmax ? (unsigned)idx : 0xffffffffu);
}
__device__ __forceinline__ int warp_argmax(double v, int idx) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  return idx;
}
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

template <typename T, int RT, int CT>
__global__ void __launch_bounds__(kInvRegThreads) k_inv_reg(const PartDesc* __restrict__ parts, int t,
                                                            const double* __restrict__ B, T* __restrict__ G,
                                                            int* __restrict__ status, int cs) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const PartDesc p = parts[blockIdx.x / cs];
  if (t >= p.L) return;  // the same for every CTA of the cluster
  const int m = p.m;
  const int w = (m + cs - 1) / cs, c0 = rank * w, wc = max(0, min(w, m - c0));
  const int lds = w + 1;
  const int tid = threadIdx.x;
  const int ty = tid & 31, tx = tid >> 5;
  T* slab = reinterpret_cast<T*>(smem_raw);  // [m][lds]
  T* pubc = slab + (size_t)m * lds;          // [2][m]: published column k
  T* pubinv = pubc + 2 * (size_t)m;          // [2]: published 1 / pivot
  int* pivrow = reinterpret_cast<int*>(pubinv + 2);  // [m]: pivot row of step k
  int* pubp = pivrow + m;                            // [2]: published pivot row
  __shared__ int s_bad;
  const long long o = p.blk + (long long)t * m * m;
  T* g = G + o;
  if (tid == 0) s_bad = 0;
  for (int e = tid; e < m * wc; e += blockDim.x) {
    const int i = e / wc, jl = e - i * wc;
    slab[i * lds + jl] = (t == 0) ? (T)B[o + (long long)i * m + c0 + jl] : g[(long long)i * m + c0 + jl];
  }
  __syncthreads();
  T A[RT][CT];
#pragma unroll
  for (int a = 0; a < RT; ++a)
#pragma unroll
    for (int b = 0; b < CT; ++b) {
      const int i = ty + 32 * a, jl = tx + 32 * b;
      A[a][b] = (i < m && jl < wc) ? slab[i * lds + jl] : (T)0;
    }
  unsigned used = 0;  // bit a: row ty + 32a has been a pivot row

  // Pivot search of column k by the warp owning it (NaN counted as 0) and
  // publication of the column, the pivot row and the pivot's reciprocal (0
  // for a zero or non-finite pivot, which also flags the block).
  auto search = [&](int k) {
    T* pc = pubc + (k & 1) * m;
    dispatch_index<CT>((k - c0) >> 5, [&](auto bc) {
      constexpr int BK = decltype(bc)::value;
      T best = (T)0;
      int bi = INT_MAX;
#pragma unroll
      for (int a = 0; a < RT; ++a) {
        const int i = ty + 32 * a;
        const T x = A[a][BK];
        if (i < m) {
          pc[i] = x;
          T v = fabs(x);
          if (!(v >= (T)0)) v = (T)0;
          if (!((used >> a) & 1u) && (bi == INT_MAX || v > best)) { best = v; bi = i; }
        }
      }
      const int pk = warp_argmax(best, bi);
      __syncwarp();
      if (ty == 0) {
        const int q = min(max(pk, 0), m - 1);
        const T piv = pc[q];
        T inv = recip(piv);
        if (!(fabs(piv) > (T)0) || !isfinite(inv)) {
          inv = (T)0;
          s_bad = 1;
        }
        pubp[k & 1] = q;
        pubinv[k & 1] = inv;
      }
    });
  };

  auto owner_of = [&](int k) { return k / w; };
  if (rank == 0 && tx == 0) search(0);
  for (int k = 0; k < m; ++k) {
    const int ok = owner_of(k), jk = k - ok * w;
    if (cs > 1) cl.sync(); else __syncthreads();  // column k, p_k, 1 / pivot published
    const T* pc = pubc + (k & 1) * m;
    int pk;
    T inv;
    T c[RT];
    if (cs > 1) {
      const T* rc = cl.map_shared_rank(pc, ok);
      pk = *cl.map_shared_rank(pubp + (k & 1), ok);
      inv = *cl.map_shared_rank(pubinv + (k & 1), ok);
#pragma unroll
      for (int a = 0; a < RT; ++a) {
        const int i = ty + 32 * a;
        c[a] = i < m ? rc[i] : (T)0;
      }
    } else {
      pk = pubp[k & 1];
      inv = pubinv[k & 1];
#pragma unroll
      for (int a = 0; a < RT; ++a) {
        const int i = ty + 32 * a;
        c[a] = i < m ? pc[i] : (T)0;
      }
    }
    const int ap = pk >> 5, lp = pk & 31;
    // row p_k of this warp's columns, from the lane that holds it
    T rs[CT];
    dispatch_index<RT>(ap, [&](auto ac) {
      constexpr int AP = decltype(ac)::value;
#pragma unroll
      for (int b = 0; b < CT; ++b) rs[b] = __shfl_sync(0xffffffffu, A[AP][b], lp) * inv;
    });
    if (ty == lp) used |= 1u << ap;
    if (tid == 0) pivrow[k] = pk;
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int b = 0; b < CT; ++b) A[a][b] = fma(-c[a], rs[b], A[a][b]);
    if (ty == lp)
      dispatch_index<RT>(ap, [&](auto ac) {
        constexpr int AP = decltype(ac)::value;
#pragma unroll
        for (int b = 0; b < CT; ++b) A[AP][b] = rs[b];
      });
    if (rank == ok && tx == (jk & 31))
      dispatch_index<CT>(jk >> 5, [&](auto bc) {
        constexpr int BK = decltype(bc)::value;
#pragma unroll
        for (int a = 0; a < RT; ++a) A[a][BK] = (ty + 32 * a == pk) ? inv : -c[a] * inv;
      });
    // lookahead: the warp owning column k+1 searches its pivot now
    const int k1 = k + 1;
    if (k1 < m && rank == owner_of(k1) && tx == ((k1 - owner_of(k1) * w) & 31)) search(k1);
  }
  if (cs > 1) cl.sync(); else __syncthreads();  // every remote read of this CTA is done
#pragma unroll
  for (int a = 0; a < RT; ++a)
#pragma unroll
    for (int b = 0; b < CT; ++b) {
      const int i = ty + 32 * a, jl = tx + 32 * b;
      if (i < m && jl < wc) slab[i * lds + jl] = A[a][b];
    }
  __syncthreads();
  // inv(D)[r][p_c] = W[p_r][c] for the columns c = c0 .. c0+wc-1 of W held here
  for (int e = tid; e < m * wc; e += blockDim.x) {
    const int r = e / wc, jl = e - r * wc;
    g[(long long)r * m + pivrow[c0 + jl]] = slab[pivrow[r] * lds + jl];
  }
  if (tid == 0 && s_bad) atomicMin(status + p.sys, p.row0 + t + 1);
}

// ---------------------------------------------------------------------------
// Forward step t of the factor sweep (Section 3, applied to subsystem S^k
// with right-hand sides W_R^k, Eq. e231).  Tile types:
//   0: Acal_t[:, J] = G_t C_t[:, J], then D_{t+1}[:, J] = B_{t+1}[:, J] - A_{t+1} Acal_t[:, J]
//      (written into G's row t+1 slot for the next inversion).  At the last
//      row of a subsystem with a right spike the product G_t C_t is the
//      spike's only non-zero forward block and goes to ZR.
//   1: left spike (k > 0): Bcal_t = G_t A_first at t = 0, else G_t (-A_t Bcal_{t-1}).
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_fwd_factor(const PartDesc* __restrict__ parts, int t,
                                                         int tiles, int type_lo, const double* __restrict__ A,
                                                         const double* __restrict__ B,
                                                         const double* __restrict__ C,
                                                         T* __restrict__ G, T* __restrict__ Acal,
                                                         T* __restrict__ ZL, T* __restrict__ ZR) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.y];
  if (t >= p.L) return;
  const int m = p.m;
  const int tb = blockIdx.x / tiles, type = type_lo + tb, c0 = (blockIdx.x - tb * tiles) * W;
  if (c0 >= m) return;
  T* Rs = reinterpret_cast<T*>(smem_raw);
  T* Xs = Rs + m * W;
  T* Lc = Xs + m * W;
  const long long mm = (long long)m * m;
  const long long o = p.blk + (long long)t * mm;
  const T* Gt = G + o;
  if (type == 0) {
    const bool last = (t == p.L - 1);
    if (last && !(p.flags & HAS_RIGHT)) return;
    load_panel<T, double, W>(Rs, C + o, m, m, c0, m, (T)1);
    __syncthreads();
    T* dst = last ? ZR + o : Acal + o;
    panel_mm<T, T, T, W>(m, Gt, Rs, (const T*)nullptr, (const T*)nullptr, Lc,
                         [&](int row, int col, T v) {
                           Xs[row * W + col] = v;
                           if (c0 + col < m) dst[(long long)row * m + c0 + col] = v;
                         });
    if (last) return;
    __syncthreads();
    const double* Bn = B + o + mm;
    T* Dn = G + o + mm;
    panel_mm<T, double, double, W>(m, A + o + mm, Xs, (const double*)nullptr, (const T*)nullptr, Lc,
                                   [&](int row, int col, T v) {
                                     if (c0 + col < m) {
                                       const long long e = (long long)row * m + c0 + col;
                                       Dn[e] = (T)Bn[e] - v;
                                     }
                                   });
  } else {
    if (!(p.flags & HAS_LEFT)) return;
    if (t == 0) {
      load_panel<T, double, W>(Rs, A + o, m, m, c0, m, (T)1);
    } else {
      load_panel<T, T, W>(Xs, ZL + o - mm, m, m, c0, m, (T)1);
      __syncthreads();
      panel_mm<T, double, double, W>(m, A + o, Xs, (const double*)nullptr, (const T*)nullptr, Lc,
                                     [&](int row, int col, T v) { Rs[row * W + col] = -v; });
    }
    __syncthreads();
    T* dst = ZL + o;
    panel_mm<T, T, T, W>(m, Gt, Rs, (const T*)nullptr, (const T*)nullptr, Lc,
                         [&](int row, int col, T v) {
                           if (c0 + col < m) dst[(long long)row * m + c0 + col] = v;
                         });
  }
}

// Backward step s of the spike sweeps, row t = L-2-s of each subsystem:
//   0: ZL_t = Bcal_t - Acal_t ZL_{t+1}   (in place over the forward blocks)
//   1: ZR_t = -Acal_t ZR_{t+1}           (the right spike's forward blocks above its last row are zero)
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_back_factor(const PartDesc* __restrict__ parts, int s,
                                                          int tiles, const T* __restrict__ Acal,
                                                          T* __restrict__ ZL, T* __restrict__ ZR) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.y];
  const int t = p.L - 2 - s;
  if (t < 0) return;
  const int m = p.m;
  const int type = blockIdx.x / tiles, c0 = (blockIdx.x - type * tiles) * W;
  if (c0 >= m) return;
  if (type == 0 && !(p.flags & HAS_LEFT)) return;
  if (type == 1 && !(p.flags & HAS_RIGHT)) return;
  T* Rs = reinterpret_cast<T*>(smem_raw);
  T* Lc = Rs + m * W;
  const long long mm = (long long)m * m;
  const long long o = p.blk + (long long)t * mm;
  T* Y = (type == 0 ? ZL : ZR) + o;
  load_panel<T, T, W>(Rs, Y + mm, m, m, c0, m, (T)1);
  __syncthreads();
  const bool keep = (type == 0);
  panel_mm<T, T, T, W>(m, Acal + o, Rs, (const T*)nullptr, (const T*)nullptr, Lc,
                       [&](int row, int col, T v) {
                         if (c0 + col < m) {
                           const long long e = (long long)row * m + c0 + col;
                           Y[e] = (keep ? Y[e] : (T)0) - v;
                         }
                       });
}

// Forward step t for a right-hand side: z_t = G_t (F_t - A_t z_{t-1}).
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_fwd_solve(const PartDesc* __restrict__ parts, int t,
                                                        int tiles, const double* __restrict__ A,
                                                        const T* __restrict__ G,
                                                        const double* __restrict__ F,
                                                        T* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.y];
  if (t >= p.L) return;
  const int m = p.m, r = p.r;
  const int c0 = blockIdx.x * W;
  if (c0 >= r) return;
  T* Rs = reinterpret_cast<T*>(smem_raw);
  T* Xs = Rs + m * W;
  T* Lc = Xs + m * W;
  const long long mm = (long long)m * m, mr = (long long)m * r;
  const long long o = p.blk + (long long)t * mm, v = p.vec + (long long)t * mr;
  const double* Ft = F + v;
  if (t == 0) {
    load_panel<T, double, W>(Rs, Ft, m, r, c0, r, (T)1);
  } else {
    load_panel<T, T, W>(Xs, z + v - mr, m, r, c0, r, (T)1);
    __syncthreads();
    panel_mm<T, double, double, W>(m, A + o, Xs, (const double*)nullptr, (const T*)nullptr, Lc,
                                   [&](int row, int col, T val) {
                                     Rs[row * W + col] =
                                         (c0 + col < r) ? (T)Ft[(long long)row * r + c0 + col] - val : (T)0;
                                   });
  }
  __syncthreads();
  T* dst = z + v;
  panel_mm<T, T, T, W>(m, G + o, Rs, (const T*)nullptr, (const T*)nullptr, Lc,
                       [&](int row, int col, T val) {
                         if (c0 + col < r) dst[(long long)row * r + c0 + col] = val;
                       });
}

// Backward step s for a right-hand side: z_t -= Acal_t z_{t+1}, t = L-2-s.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_back_solve(const PartDesc* __restrict__ parts, int s,
                                                         int tiles, const T* __restrict__ Acal,
                                                         T* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.y];
  const int t = p.L - 2 - s;
  if (t < 0) return;
  const int m = p.m, r = p.r;
  const int c0 = blockIdx.x * W;
  if (c0 >= r) return;
  T* Rs = reinterpret_cast<T*>(smem_raw);
  T* Lc = Rs + m * W;
  const long long mm = (long long)m * m, mr = (long long)m * r;
  const long long o = p.blk + (long long)t * mm, v = p.vec + (long long)t * mr;
  T* Y = z + v;
  load_panel<T, T, W>(Rs, Y + mr, m, r, c0, r, (T)1);
  __syncthreads();
  panel_mm<T, T, T, W>(m, Acal + o, Rs, (const T*)nullptr, (const T*)nullptr, Lc,
                       [&](int row, int col, T val) {
                         if (c0 + col < r) {
                           const long long e = (long long)row * r + c0 + col;
                           Y[e] = Y[e] - val;
                         }
                       });
}

// Supplementary matrix (Eq. e2311), separator j at row q, in float64:
//   0: HB_j = B_q - A_q ZR^j[q-1] - C_q ZL^{j+1}[q+1]
//   1: HA_j = -A_q ZL^j[q-1]        (j > 0)
//   2: HC_j = -C_q ZR^{j+1}[q+1]    (j < P-2)
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_assemble_h(const SepDesc* __restrict__ seps, int tiles,
                                                         const double* __restrict__ A,
                                                         const double* __restrict__ B,
                                                         const double* __restrict__ C,
                                                         const T* __restrict__ ZL,
                                                         const T* __restrict__ ZR,
                                                         double* __restrict__ HA,
                                                         double* __restrict__ HB,
                                                         double* __restrict__ HC) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SepDesc sp = seps[blockIdx.y];
  const int m = sp.m;
  const int type = blockIdx.x / tiles, c0 = (blockIdx.x - type * tiles) * W;
  if (c0 >= m) return;
  if (type == 1 && !(sp.flags & HAS_HA)) return;
  if (type == 2 && !(sp.flags & HAS_HC)) return;
  // the level's arithmetic: float32 products (and sums) on float32 levels,
  // whose spikes carry float32 accuracy anyway; H itself is float64
  T* R1 = reinterpret_cast<T*>(smem_raw);
  T* R2 = R1 + m * W;
  T* Lc = R2 + m * W;
  const double* Aq = A + sp.blk_q;
  const double* Cq = C + sp.blk_q;
  if (type == 0) {
    load_panel<T, T, W>(R1, ZR + sp.blk_prev, m, m, c0, m, (T)1);
    load_panel<T, T, W>(R2, ZL + sp.blk_next, m, m, c0, m, (T)1);
    __syncthreads();
    const double* Bq = B + sp.blk_q;
    double* dst = HB + sp.hblk;
    panel_mm<T, double, double, W>(m, Aq, R1, Cq, R2, Lc, [&](int row, int col, T v) {
      if (c0 + col < m) {
        const long long e = (long long)row * m + c0 + col;
        dst[e] = Bq[e] - (double)v;
      }
    });
  } else {
    const T* Z = (type == 1) ? ZL + sp.blk_prev : ZR + sp.blk_next;
    const double* Lop = (type == 1) ? Aq : Cq;
    double* dst = ((type == 1) ? HA : HC) + sp.hblk;
    load_panel<T, T, W>(R1, Z, m, m, c0, m, (T)1);
    __syncthreads();
    panel_mm<T, double, double, W>(m, Lop, R1, (const double*)nullptr, (const T*)nullptr, Lc,
                                   [&](int row, int col, T v) {
                                     if (c0 + col < m) dst[(long long)row * m + c0 + col] = -(double)v;
                                   });
  }
}

// Supplementary right-hand side (Eq. e2311): fh_j = F_q - A_q z^j[q-1] - C_q z^{j+1}[q+1].
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_assemble_f(const SepDesc* __restrict__ seps, int tiles,
                                                         const double* __restrict__ A,
                                                         const double* __restrict__ C,
                                                         const double* __restrict__ F,
                                                         const T* __restrict__ z,
                                                         double* __restrict__ fh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SepDesc sp = seps[blockIdx.y];
  const int m = sp.m, r = sp.r;
  const int c0 = blockIdx.x * W;
  if (c0 >= r) return;
  double* R1 = reinterpret_cast<double*>(smem_raw);
  double* R2 = R1 + m * W;
  double* Lc = R2 + m * W;
  load_panel<double, T, W>(R1, z + sp.vec_prev, m, r, c0, r, 1.0);
  load_panel<double, T, W>(R2, z + sp.vec_next, m, r, c0, r, 1.0);
  __syncthreads();
  const double* Fq = F + sp.vec_q;
  double* dst = fh + sp.hvec;
  panel_mm<double, double, double, W>(m, A + sp.blk_q, R1, C + sp.blk_q, R2, Lc,
                                      [&](int row, int col, double v) {
                                        if (c0 + col < r) {
                                          const long long e = (long long)row * r + c0 + col;
                                          dst[e] = Fq[e] - v;
                                        }
                                      });
}

// Back-substitution (Eq. endSolution) for row t of each subsystem, in float64:
//   x_t = z_t - ZL_t h^{k-1} - ZR_t h^k.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_backsub(const PartDesc* __restrict__ parts, int tiles,
                                                      const T* __restrict__ ZL,
                                                      const T* __restrict__ ZR,
                                                      const T* __restrict__ z,
                                                      const double* __restrict__ h,
                                                      double* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.y];
  const int t = blockIdx.x / tiles;
  if (t >= p.L) return;
  const int m = p.m, r = p.r;
  const int c0 = (blockIdx.x - t * tiles) * W;
  if (c0 >= r) return;
  double* R1 = reinterpret_cast<double*>(smem_raw);
  double* R2 = R1 + m * W;
  double* Lc = R2 + m * W;
  const long long mm = (long long)m * m, mr = (long long)m * r;
  const long long o = p.blk + (long long)t * mm, v = p.vec + (long long)t * mr;
  const bool hl = p.flags & HAS_LEFT, hr = p.flags & HAS_RIGHT;
  if (hl) load_panel<double, double, W>(R1, h + p.hprev, m, r, c0, r, 1.0);
  if (hr) load_panel<double, double, W>(R2, h + p.hnext, m, r, c0, r, 1.0);
  __syncthreads();
  const T* zt = z + v;
  double* xt = x + v;
  auto epi = [&](int row, int col, double val) {
    if (c0 + col < r) {
      const long long e = (long long)row * r + c0 + col;
      xt[e] = (double)zt[e] - val;
    }
  };
  if (hl && hr) {
    panel_mm<double, T, T, W>(m, ZL + o, R1, ZR + o, R2, Lc, epi);
  } else if (hl) {
    panel_mm<double, T, T, W>(m, ZL + o, R1, (const T*)nullptr, (const double*)nullptr, Lc, epi);
  } else if (hr) {
    panel_mm<double, T, T, W>(m, ZR + o, R2, (const T*)nullptr, (const double*)nullptr, Lc, epi);
  } else {
    for (int e = threadIdx.x; e < m * W; e += kThreads) {
      const int row = e / W, col = e - row * W;
      if (c0 + col < r) xt[(long long)row * r + c0 + col] = (double)zt[(long long)row * r + c0 + col];
    }
  }
}

// ---------------------------------------------------------------------------
// Narrow products for right-hand sides (r <= 16 columns): one output row per
// thread.  Each thread streams its row of the m x m block from global memory
// (every load brings a whole line into L1, so a warp keeps 32 lines in flight
// and the following k hit L1) against the panel R ([m][RB] in shared memory,
// read as broadcasts); no cross-lane reduction.  RB is the CTA's own column
// bucket (1, 2, 4, 8 or 16 >= its r), so a batch with mixed right-hand-side
// counts spends no multiply-add on another system's padding.
__host__ __device__ constexpr int rbucket(int r) { return r <= 1 ? 1 : r <= 2 ? 2 : r <= 4 ? 4 : r <= 8 ? 8 : 16; }

// f(integral_constant<RB>) with RB = rbucket(r), instantiated only for RB <= RM
template <int RM, typename F>
__device__ __forceinline__ void with_rb(int r, F&& f) {
  const int rb = rbucket(r);
  if (rb == 1) { f(std::integral_constant<int, 1>()); return; }
  if constexpr (RM >= 2) if (rb == 2) { f(std::integral_constant<int, 2>()); return; }
  if constexpr (RM >= 4) if (rb == 4) { f(std::integral_constant<int, 4>()); return; }
  if constexpr (RM >= 8) if (rb == 8) { f(std::integral_constant<int, 8>()); return; }
  if constexpr (RM >= 16) f(std::integral_constant<int, 16>());
}

template <typename T, typename TL1, typename TL2, int RB, typename Epi>
__device__ __forceinline__ void rows_mm(int m, const TL1* __restrict__ L1, const T* __restrict__ R1,
                                        const TL2* __restrict__ L2, const T* __restrict__ R2, Epi epi) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    T acc[RB];
#pragma unroll
    for (int c = 0; c < RB; ++c) acc[c] = (T)0;
    const TL1* l1 = L1 + (long long)i * m;
#pragma unroll 4
    for (int k = 0; k < m; ++k) {
      const T lv = (T)l1[k];
#pragma unroll
      for (int c = 0; c < RB; ++c) acc[c] = fma(lv, R1[k * RB + c], acc[c]);
    }
    if (L2 != nullptr) {
      const TL2* l2 = L2 + (long long)i * m;
#pragma unroll 4
      for (int k = 0; k < m; ++k) {
        const T lv = (T)l2[k];
#pragma unroll
        for (int c = 0; c < RB; ++c) acc[c] = fma(lv, R2[k * RB + c], acc[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < RB; ++c) epi(i, c, acc[c]);
  }
}

// Rs[k][c] = src[k * r + c] for c < r, zero up to RB.
template <typename T, typename TS, int RB>
__device__ __forceinline__ void load_narrow(T* Rs, const TS* __restrict__ src, int m, int r) {
  for (int e = threadIdx.x; e < m * RB; e += blockDim.x) {
    const int k = e / RB, c = e - k * RB;
    Rs[e] = c < r ? (T)src[(long long)k * r + c] : (T)0;
  }
}

// ---------------------------------------------------------------------------
// Both right-hand-side sweeps of a level in one launch (Section 3 applied to
// the subsystems: z_t = G_t (F_t - A_t z_{t-1}) for t = 0..L-1, then
// z_t -= Acal_t z_{t+1} for t = L-2..0), one thread-block cluster of CS CTAs
// per subsystem.  CTA `rank` owns rows [rank*rpc, (rank+1)*rpc) of every
// block; each of its rows is a dot product over LPR lanes (coalesced loads of
// the block row, many in flight per lane, xor-shuffle reduction), against the
// full m x RB panel that every CTA holds in shared memory, column-major
// ([c][k], conflict-free).  A CTA pushes the rows it computes into the panel
// of every CTA of its cluster (distributed shared memory) and the cluster
// barrier publishes them, so a step costs two cluster barriers forward and
// one backward instead of a kernel launch.  All loop bounds are uniform over
// a cluster (the subsystem's L and m), so every CTA passes every barrier.
constexpr int kSweepThreads = 256;

// Lanes per row: the largest power of two <= 32 with lpr * rows <= threads
// (at least 4; a CTA with more rows than groups loops over them).
__host__ __device__ constexpr int sweep_lpr(int rows) {
  return rows <= 8 ? 32 : rows <= 16 ? 16 : rows <= 32 ? 8 : rows <= 64 ? 4 : rows <= 128 ? 2 : 1;
}

// acc[c] = sum_k Lrow[k] X[c * ld + k] over the LPR lanes of a group
// (result in every lane of the group).  `valid` false contributes zeros but
// still takes part in the shuffles (the whole warp executes them).
template <typename T, typename TL, int RB, int LPR>
__device__ __forceinline__ void group_dot(bool valid, const TL* __restrict__ Lrow, const T* X, int ld, int m,
                                          int lane, T (&acc)[RB]) {
#pragma unroll
  for (int c = 0; c < RB; ++c) acc[c] = (T)0;
  if (valid) {
    constexpr int U = (sizeof(T) == 8 && RB >= 16) ? 4 : 8;  // loads in flight per lane
    int k = lane;
    for (; k + LPR * (U - 1) < m; k += LPR * U) {
      TL v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = Lrow[k + u * LPR];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < RB; ++c) acc[c] = fma((T)v[u], X[c * ld + k + u * LPR], acc[c]);
    }
    for (; k < m; k += LPR) {
      const T v = (T)Lrow[k];
#pragma unroll
      for (int c = 0; c < RB; ++c) acc[c] = fma(v, X[c * ld + k], acc[c]);
    }
  }
  if constexpr (LPR > 1) {
#pragma unroll
    for (int off = LPR / 2; off > 0; off >>= 1)
#pragma unroll
      for (int c = 0; c < RB; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off, LPR);
  }
}

namespace cg = cooperative_groups;

template <typename T, int RB, int LPR>
__device__ void sweep_body(const PartDesc& p, int rank, int cs, const double* __restrict__ A,
                           const T* __restrict__ G, const T* __restrict__ Acal, const double* __restrict__ F,
                           T* __restrict__ z, T* Zp0, T* Zp1, T* Rs) {
  cg::cluster_group cl = cg::this_cluster();
  const int m = p.m, r = p.r, L = p.L;
  const int rpc = (m + cs - 1) / cs;
  const int r0 = min(m, rank * rpc), r1 = min(m, r0 + rpc);
  constexpr int GROUPS = kSweepThreads / LPR;
  const int g = threadIdx.x / LPR, lane = threadIdx.x % LPR;
  const long long mm = (long long)m * m, mr = (long long)m * r;
  // the rows this CTA computes go into the panel `dst` of every CTA
  auto push = [&](T* dst, int row, int c, T v) {
    for (int q = 0; q < cs; ++q) *cl.map_shared_rank(dst + c * m + row, q) = v;
  };
  // forward sweep
  for (int t = 0; t < L; ++t) {
    const long long o = p.blk + t * mm, v = p.vec + t * mr;
    const double* Ft = F + v;
    if (t == 0) {
      for (int e = threadIdx.x; e < m * RB; e += blockDim.x) {
        const int c = e / m, k = e - c * m;
        Rs[e] = c < r ? (T)Ft[(long long)k * r + c] : (T)0;
      }
      __syncthreads();
    } else {
      for (int i0 = r0; i0 < r1; i0 += GROUPS) {
        const int row = i0 + g;
        const bool ok = row < r1;
        T acc[RB];
        group_dot<T, double, RB, LPR>(ok, A + o + (long long)row * m, Zp0, m, m, lane, acc);
#pragma unroll
        for (int c = 0; c < RB; ++c)
          if (ok && c % LPR == lane) push(Rs, row, c, c < r ? (T)Ft[(long long)row * r + c] - acc[c] : (T)0);
      }
      cl.sync();
    }
    T* zt = z + v;
    for (int i0 = r0; i0 < r1; i0 += GROUPS) {
      const int row = i0 + g;
      const bool ok = row < r1;
      T acc[RB];
      group_dot<T, T, RB, LPR>(ok, G + o + (long long)row * m, Rs, m, m, lane, acc);
#pragma unroll
      for (int c = 0; c < RB; ++c)
        if (ok && c % LPR == lane) {
          if (c < r) zt[(long long)row * r + c] = acc[c];
          push(Zp0, row, c, c < r ? acc[c] : (T)0);
        }
    }
    cl.sync();
  }
  // backward sweep: Zp0 holds z_{L-1}; panels alternate between Zp0 and Zp1
  T* cur = Zp0;
  T* nxt = Zp1;
  for (int t = L - 2; t >= 0; --t) {
    const long long o = p.blk + t * mm, v = p.vec + t * mr;
    T* zt = z + v;
    for (int i0 = r0; i0 < r1; i0 += GROUPS) {
      const int row = i0 + g;
      const bool ok = row < r1;
      T acc[RB];
      group_dot<T, T, RB, LPR>(ok, Acal + o + (long long)row * m, cur, m, m, lane, acc);
#pragma unroll
      for (int c = 0; c < RB; ++c)
        if (ok && c % LPR == lane) {
          T val = (T)0;
          if (c < r) {
            const long long e = (long long)row * r + c;
            val = zt[e] - acc[c];
            zt[e] = val;
          }
          push(nxt, row, c, val);
        }
    }
    cl.sync();
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
}

template <typename T, int RM>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_solve_n(const PartDesc* __restrict__ parts, int cs,
                                                                 const double* __restrict__ A,
                                                                 const T* __restrict__ G,
                                                                 const T* __restrict__ Acal,
                                                                 const double* __restrict__ F, T* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const PartDesc p = parts[blockIdx.x / cs];
  const int m = p.m;
  // panels laid out for this subsystem's m (at most the launch's max_m)
  T* Zp0 = reinterpret_cast<T*>(smem_raw);
  T* Zp1 = Zp0 + m * RM;
  T* Rs = Zp1 + m * RM;
  const int rpc = (m + cs - 1) / cs;
  const int lpr = sweep_lpr(rpc);
  with_rb<RM>(p.r, [&](auto rbc) {
    constexpr int RB = decltype(rbc)::value;
    switch (lpr) {
      case 32: sweep_body<T, RB, 32>(p, rank, cs, A, G, Acal, F, z, Zp0, Zp1, Rs); break;
      case 16: sweep_body<T, RB, 16>(p, rank, cs, A, G, Acal, F, z, Zp0, Zp1, Rs); break;
      case 8: sweep_body<T, RB, 8>(p, rank, cs, A, G, Acal, F, z, Zp0, Zp1, Rs); break;
      default: sweep_body<T, RB, 4>(p, rank, cs, A, G, Acal, F, z, Zp0, Zp1, Rs); break;  // rows looped
    }
  });
}

template <typename T, int RM>
__global__ void __launch_bounds__(256) k_fwd_solve_n(const PartDesc* __restrict__ parts, int t,
                                                     const double* __restrict__ A, const T* __restrict__ G,
                                                     const double* __restrict__ F, T* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.x];
  if (t >= p.L) return;
  const int m = p.m, r = p.r;
  with_rb<RM>(r, [&](auto rbc) {
    constexpr int RB = decltype(rbc)::value;
    T* Rs = reinterpret_cast<T*>(smem_raw);
    T* Xs = Rs + m * RB;
    const long long mm = (long long)m * m, mr = (long long)m * r;
    const long long o = p.blk + (long long)t * mm, v = p.vec + (long long)t * mr;
    const double* Ft = F + v;
    if (t == 0) {
      load_narrow<T, double, RB>(Rs, Ft, m, r);
    } else {
      load_narrow<T, T, RB>(Xs, z + v - mr, m, r);
      __syncthreads();
      rows_mm<T, double, double, RB>(m, A + o, Xs, (const double*)nullptr, (const T*)nullptr,
                                     [&](int row, int col, T val) {
                                       Rs[row * RB + col] = col < r ? (T)Ft[(long long)row * r + col] - val : (T)0;
                                     });
    }
    __syncthreads();
    T* dst = z + v;
    rows_mm<T, T, T, RB>(m, G + o, Rs, (const T*)nullptr, (const T*)nullptr, [&](int row, int col, T val) {
      if (col < r) dst[(long long)row * r + col] = val;
    });
  });
}

template <typename T, int RM>
__global__ void __launch_bounds__(256) k_back_solve_n(const PartDesc* __restrict__ parts, int s,
                                                      const T* __restrict__ Acal, T* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.x];
  const int t = p.L - 2 - s;
  if (t < 0) return;
  const int m = p.m, r = p.r;
  with_rb<RM>(r, [&](auto rbc) {
    constexpr int RB = decltype(rbc)::value;
    T* Rs = reinterpret_cast<T*>(smem_raw);
    const long long mm = (long long)m * m, mr = (long long)m * r;
    const long long o = p.blk + (long long)t * mm, v = p.vec + (long long)t * mr;
    T* Y = z + v;
    load_narrow<T, T, RB>(Rs, Y + mr, m, r);
    __syncthreads();
    rows_mm<T, T, T, RB>(m, Acal + o, Rs, (const T*)nullptr, (const T*)nullptr, [&](int row, int col, T val) {
      if (col < r) {
        const long long e = (long long)row * r + col;
        Y[e] = Y[e] - val;
      }
    });
  });
}

template <typename T, int RM>
__global__ void __launch_bounds__(256) k_assemble_f_n(const SepDesc* __restrict__ seps,
                                                      const double* __restrict__ A,
                                                      const double* __restrict__ C,
                                                      const double* __restrict__ F,
                                                      const T* __restrict__ z, double* __restrict__ fh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SepDesc sp = seps[blockIdx.x];
  const int m = sp.m, r = sp.r;
  with_rb<RM>(r, [&](auto rbc) {
    constexpr int RB = decltype(rbc)::value;
    double* R1 = reinterpret_cast<double*>(smem_raw);
    double* R2 = R1 + m * RB;
    load_narrow<double, T, RB>(R1, z + sp.vec_prev, m, r);
    load_narrow<double, T, RB>(R2, z + sp.vec_next, m, r);
    __syncthreads();
    const double* Fq = F + sp.vec_q;
    double* dst = fh + sp.hvec;
    rows_mm<double, double, double, RB>(m, A + sp.blk_q, R1, C + sp.blk_q, R2, [&](int row, int col, double v) {
      if (col < r) {
        const long long e = (long long)row * r + col;
        dst[e] = Fq[e] - v;
      }
    });
  });
}

// Back-substitution for row t = blockIdx.x of subsystem blockIdx.y, in the
// level's arithmetic (float32 levels: the spikes are float32, the products
// too; x is written in float64).
template <typename T, int RM>
__global__ void __launch_bounds__(256) k_backsub_n(const PartDesc* __restrict__ parts,
                                                   const T* __restrict__ ZL, const T* __restrict__ ZR,
                                                   const T* __restrict__ z, const double* __restrict__ h,
                                                   double* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const PartDesc p = parts[blockIdx.y];
  const int t = blockIdx.x;
  if (t >= p.L) return;
  const int m = p.m, r = p.r;
  with_rb<RM>(r, [&](auto rbc) {
    constexpr int RB = decltype(rbc)::value;
    T* R1 = reinterpret_cast<T*>(smem_raw);
    T* R2 = R1 + m * RB;
    const long long mm = (long long)m * m, mr = (long long)m * r;
    const long long o = p.blk + (long long)t * mm, v = p.vec + (long long)t * mr;
    const bool hl = p.flags & HAS_LEFT, hr = p.flags & HAS_RIGHT;
    if (hl) load_narrow<T, double, RB>(R1, h + p.hprev, m, r);
    if (hr) load_narrow<T, double, RB>(R2, h + p.hnext, m, r);
    __syncthreads();
    const T* zt = z + v;
    double* xt = x + v;
    auto epi = [&](int row, int col, T val) {
      if (col < r) {
        const long long e = (long long)row * r + col;
        xt[e] = (double)zt[e] - (double)val;
      }
    };
    if (hl && hr) {
      rows_mm<T, T, T, RB>(m, ZL + o, R1, ZR + o, R2, epi);
    } else if (hl) {
      rows_mm<T, T, T, RB>(m, ZL + o, R1, (const T*)nullptr, (const T*)nullptr, epi);
    } else if (hr) {
      rows_mm<T, T, T, RB>(m, ZR + o, R2, (const T*)nullptr, (const T*)nullptr, epi);
    } else {
      for (long long e = threadIdx.x; e < mr; e += blockDim.x) xt[e] = (double)zt[e];
    }
  });
}

__global__ void k_sep_copy(const SepDesc* __restrict__ seps, const double* __restrict__ h,
                           double* __restrict__ x) {
  const SepDesc sp = seps[blockIdx.x];
  const int n = sp.m * sp.r;
  for (int e = threadIdx.x; e < n; e += blockDim.x) x[sp.vec_q + e] = h[sp.hvec + e];
}

// ---------------------------------------------------------------------------
// Residual r_i = b_i - A_i x_{i-1} - B_i x_i - C_i x_{i+1} in float64, one CTA
// per block row of any system (rows of all systems numbered consecutively;
// the CTA finds its system by binary search over their first rows).  One
// output row per thread streaming the three block rows; x_{i-1}, x_i, x_{i+1}
// staged in shared memory RB columns at a time (RB = the system's bucket).
// Column sums of r^2 and b^2 go to nrm by atomics.
__device__ __forceinline__ int find_sys(const SysDesc* __restrict__ sys, int nsys, int row) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sys[mid].row0 <= row) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int RM>
__global__ void __launch_bounds__(256) k_residual(const SysDesc* __restrict__ sys, int nsys,
                                                  const double* __restrict__ A,
                                                  const double* __restrict__ B,
                                                  const double* __restrict__ C,
                                                  const double* __restrict__ x,
                                                  const double* __restrict__ b,
                                                  double* __restrict__ rout,
                                                  double* __restrict__ nrm,
                                                  const int* __restrict__ band) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2 * kMaxR];
  // A and C banded (half-bandwidth w <= kBandMax, found by the factorisation
  // of these blocks): their products run over the band only
  const int wb = band ? *band : kBandMax + 1;
  const int si = find_sys(sys, nsys, blockIdx.x);
  const SysDesc sd = sys[si];
  if (sd.sliced) return;  // residual on the tensor cores (k_residual_sliced)
  const int i = blockIdx.x - sd.row0;
  const int m = sd.m, r = sd.r;
  const long long mm = (long long)m * m, mr = (long long)m * r;
  const long long o = sd.blk + i * mm, v = sd.vec + i * mr;
  const int tid = threadIdx.x;
  for (int e = tid; e < 2 * r; e += blockDim.x) red[e] = 0.0;
  const bool hasA = i > 0, hasC = i < sd.N - 1;
  with_rb<RM>(r, [&](auto rbc) {
    constexpr int RB = decltype(rbc)::value;
    double* xs = reinterpret_cast<double*>(smem_raw);  // [3][m][RB]
    for (int c0 = 0; c0 < r; c0 += RB) {
      const int nc = min(RB, r - c0);
      __syncthreads();
      for (int e = tid; e < 3 * m * RB; e += blockDim.x) {
        const int which = e / (m * RB), rem = e - which * m * RB, k = rem / RB, c = rem - k * RB;
        const int row = i - 1 + which;
        xs[e] = (row >= 0 && row < sd.N && c < nc) ? x[sd.vec + row * mr + (long long)k * r + c0 + c] : 0.0;
      }
      __syncthreads();
      for (int row = tid; row < m; row += blockDim.x) {
        double acc[RB];
#pragma unroll
        for (int c = 0; c < RB; ++c) acc[c] = 0.0;
        const double* ar = A + o + (long long)row * m;
        const double* br = B + o + (long long)row * m;
        const double* cr = C + o + (long long)row * m;
        if (wb <= kBandMax) {
#pragma unroll 2
          for (int k = 0; k < m; ++k) {
            const double bv = br[k];
            const double* x0 = xs + (m + k) * RB;
#pragma unroll
            for (int c = 0; c < RB; ++c) acc[c] = fma(bv, x0[c], acc[c]);
          }
          for (int k = max(0, row - wb); k <= min(m - 1, row + wb); ++k) {
            const double av = hasA ? ar[k] : 0.0, cv = hasC ? cr[k] : 0.0;
            const double* xm = xs + k * RB;
            const double* xp = xm + 2 * m * RB;
#pragma unroll
            for (int c = 0; c < RB; ++c) acc[c] = fma(av, xm[c], fma(cv, xp[c], acc[c]));
          }
        } else {
#pragma unroll 2
          for (int k = 0; k < m; ++k) {
            const double av = hasA ? ar[k] : 0.0, bv = br[k], cv = hasC ? cr[k] : 0.0;
            const double* xm = xs + k * RB;
            const double* x0 = xm + m * RB;
            const double* xp = x0 + m * RB;
#pragma unroll
            for (int c = 0; c < RB; ++c) acc[c] = fma(av, xm[c], fma(bv, x0[c], fma(cv, xp[c], acc[c])));
          }
        }
#pragma unroll
        for (int c = 0; c < RB; ++c) {
          if (c < nc) {
            const long long e = v + (long long)row * r + c0 + c;
            const double bb = b[e];
            const double rv = bb - acc[c];
            rout[e] = rv;
            atomicAdd(&red[c0 + c], rv * rv);
            atomicAdd(&red[r + c0 + c], bb * bb);
          }
        }
      }
    }
  });
  __syncthreads();
  for (int c = tid; c < r; c += blockDim.x) {
    atomicAdd(&nrm[(long long)si * 4 * kMaxR + c], red[c]);
    atomicAdd(&nrm[(long long)si * 4 * kMaxR + kMaxR + c], red[r + c]);
  }
}

// x += d per block row (rows of all systems numbered consecutively), with
// column sums of d^2 and (updated) x^2.
__global__ void __launch_bounds__(256) k_axpy_norms(const SysDesc* __restrict__ sys, int nsys,
                                                    const double* __restrict__ d,
                                                    double* __restrict__ x,
                                                    double* __restrict__ nrm) {
  __shared__ double red[2 * kMaxR];
  const int si = find_sys(sys, nsys, blockIdx.x);
  const SysDesc sd = sys[si];
  const int i = blockIdx.x - sd.row0;
  const int r = sd.r;
  const long long mr = (long long)sd.m * r, v = sd.vec + i * mr;
  for (int e = threadIdx.x; e < 2 * r; e += blockDim.x) red[e] = 0.0;
  __syncthreads();
  for (long long e = threadIdx.x; e < mr; e += blockDim.x) {
    const double dv = d[v + e];
    const double xv = x[v + e] + dv;
    x[v + e] = xv;
    const int c = (int)(e % r);
    atomicAdd(&red[c], dv * dv);
    atomicAdd(&red[r + c], xv * xv);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    atomicAdd(&nrm[(long long)si * 4 * kMaxR + 2 * kMaxR + c], red[c]);
    atomicAdd(&nrm[(long long)si * 4 * kMaxR + 3 * kMaxR + c], red[r + c]);
  }
}

// Raise a kernel's dynamic shared memory limit once per kernel (to the
// largest size asked for so far), so that launches inside a stream capture
// make no attribute calls.
std::mutex g_smem_mu;
std::unordered_map<const void*, size_t> g_smem_granted;

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  // the default limit (48 KB) covers static + dynamic shared memory together
  if (bytes + 4096 <= 48 * 1024) return;
  const void* key = reinterpret_cast<const void*>(kernel);
  std::lock_guard<std::mutex> lk(g_smem_mu);
  size_t& g = g_smem_granted[key];
  if (bytes > g) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    g = bytes;
  }
}

template <typename T>
int inv_smem_max_m() {
  // working matrix (m x (m+1)) + perm/idx/colk/rowk, within 227 KB
  const size_t budget = 227 * 1024 - 2 * kMaxM * sizeof(int) - 2 * kMaxM * sizeof(T) - 256;
  int m = 1;
  while ((size_t)(m + 1) * (m + 2) * sizeof(T) <= budget) ++m;
  return m;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// r <= 16: call f with the smallest bucket RM >= r as a compile-time constant
template <typename F>
bool narrow_dispatch(int max_r, F&& f) {
  if (max_r <= 1) return f(std::integral_constant<int, 1>()), true;
  if (max_r <= 2) return f(std::integral_constant<int, 2>()), true;
  if (max_r <= 4) return f(std::integral_constant<int, 4>()), true;
  if (max_r <= 8) return f(std::integral_constant<int, 8>()), true;
  if (max_r <= 16) return f(std::integral_constant<int, 16>()), true;
  return false;
}

template <typename T>
size_t inv_cluster_smem(int max_m, int cs) {
  const int w = (max_m + cs - 1) / cs;
  return sizeof(T) * (3 * (size_t)kMaxM + 128 + (size_t)max_m * (w + 1)) + 3 * kMaxM * sizeof(int);
}

template <typename T>
int inv_cluster_size(int max_m) {
  // float64: ~32 columns per CTA so the FP64 pipes of cs SMs share a block
  // (up to 64 columns when that keeps the cluster at the portable 8 CTAs);
  // float32: one CTA up to m = 128, else 64 columns per CTA (the update is
  // cheap, barriers dominate).
  if (sizeof(T) == 4 && max_m <= 128) return 1;
  const int per = sizeof(T) == 8 ? 32 : 64;
  int cs = 1;
  while (cs * per < max_m) cs *= 2;
  if (cs > 8 && inv_cluster_smem<T>(max_m, 8) <= 227 * 1024 && (max_m + 7) / 8 <= 128) cs = 8;
  return cs;
}

// Whether a cluster of cs CTAs of `kernel` with `bytes` of shared memory each
// can run (cached per kernel, size and bytes).
template <typename K>
bool cluster_ok(K kernel, int cs, size_t bytes, int threads = 256) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, bool> known;
  const auto key = std::make_tuple(reinterpret_cast<const void*>(kernel), cs, bytes);
  std::lock_guard<std::mutex> lk(mu);
  auto it = known.find(key);
  if (it != known.end()) return it->second;
  if (cs > 8) cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  allow_smem(kernel, bytes);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) == cudaSuccess && nclusters > 0;
  cudaGetLastError();
  known[key] = ok;
  return ok;
}

template <typename K, typename... Args>
void launch_cluster(K kernel, int nclusters, int cs, int threads, size_t bytes, cudaStream_t st, Args... args) {
  allow_smem(kernel, bytes);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nclusters * cs);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// DM_INV_KERNEL=column / reg / panel forces one float32 inverse (for
// comparisons; reg falls back to column above m = 128).  0 = column,
// 1 = automatic, 2 = panel, 3 = reg.
int inv_variant() {
  static const int v = [] {
    const char* e = std::getenv("DM_INV_KERNEL");
    if (!e) return 1;
    const std::string s(e);
    return s == "column" ? 0 : s == "panel" ? 2 : s == "reg" ? 3 : 1;
  }();
  return v;
}

int device_sms() {
  static std::mutex mu;
  static std::unordered_map<int, int> known;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = known.find(dev);
  if (it != known.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 1;
  }
  known[dev] = sms;
  return sms;
}

// Thread tile (RT rows x CT columns per thread, 16 x 16 threads per CTA) and
// cluster size of the register-resident inverse for blocks up to max_m:
// float64 about 32 columns per CTA (the FP64 work of a block spread over
// several SMs), float32 up to 128 columns per CTA; at most 64 elements per
// thread.
template <typename T>
void inv_reg_shape(int max_m, int* rt, int* ct, int* cs) {
  auto p2 = [](int v) { int q = 1; while (q < v) q *= 2; return q; };
  const int r = p2((max_m + 31) / 32);
  const int per = sizeof(T) == 8 ? 32 : (max_m <= 128 ? 128 : 64);
  int c = 1;
  while (c * per < max_m) c *= 2;
  int w = (max_m + c - 1) / c;
  int cc = p2((w + 31) / 32);
  while (r * cc > 16 && c < 16) {
    c *= 2;
    w = (max_m + c - 1) / c;
    cc = p2((w + 31) / 32);
  }
  if (r > 16 || r * cc > 16) { *rt = *ct = *cs = 0; return; }
  *rt = r;
  *ct = cc;
  *cs = c;
}

template <typename T, typename F>
void inv_reg_dispatch(int rt, int ct, F&& f) {
#define DM_INV_REG_CASE(R, C) \
  if (rt == R && ct == C) return f(k_inv_reg<T, R, C>);
  DM_INV_REG_CASE(1, 1) DM_INV_REG_CASE(2, 1) DM_INV_REG_CASE(2, 2) DM_INV_REG_CASE(4, 1) DM_INV_REG_CASE(4, 2)
  DM_INV_REG_CASE(4, 4) DM_INV_REG_CASE(8, 1) DM_INV_REG_CASE(8, 2) DM_INV_REG_CASE(16, 1)
#undef DM_INV_REG_CASE
}

template <typename T>
void launch_inv(const PartDesc* parts, int nparts, int t, const double* B, T* G, int* status,
                int max_m, cudaStream_t st) {
  if (nparts <= 0) return;
  const int cs = inv_cluster_size<T>(max_m);
  // float32: the register-resident inverse while the blocks of a launch
  // leave SMs idle (latency-bound, up to m = 128), the panel-blocked inverse
  // when there are enough blocks to fill the GPU several times over
  // (throughput-bound); float64: column by column, whose per-pivot update
  // spreads the FP64 work over every warp of the cluster.
  if (sizeof(T) == 4 && inv_variant() != 0) {
    const bool many = inv_variant() == 3 ? false : nparts >= 2 * device_sms();
    if (!many && max_m <= 128 && inv_variant() != 2) {
      int rc = 0, cc = 0, ics = 0;
      inv_reg_shape<T>(max_m, &rc, &cc, &ics);
      const size_t bytes = inv_reg_smem<T>(max_m, (max_m + ics - 1) / ics);
      if (ics > 0 && bytes <= 227 * 1024) {
        bool launched = false;
        inv_reg_dispatch<T>(rc, cc, [&](auto kern) {
          if (ics <= 8 || cluster_ok(kern, ics, bytes, kInvRegThreads)) {
            launch_cluster(kern, nparts, ics, kInvRegThreads, bytes, st, parts, t, B, G, status, ics);
            launched = true;
          }
        });
        if (launched) return;
      }
    }
    if (cs <= 16 && (many || inv_variant() == 2)) {
      constexpr int NB = 8;
      const size_t bytes = inv_blocked_layout<T, NB>(max_m, (max_m + cs - 1) / cs, nullptr, nullptr, nullptr);
      if (bytes <= 227 * 1024 && (cs <= 8 || cluster_ok(k_inv_blocked<T, NB>, cs, bytes))) {
        launch_cluster(k_inv_blocked<T, NB>, nparts, cs, 256, bytes, st, parts, t, B, G, status, cs);
        return;
      }
    }
  }
  const size_t bytes = inv_cluster_smem<T>(max_m, cs);
  if (cs <= 16 && bytes <= 227 * 1024 && (cs <= 8 || cluster_ok(k_inv_cluster<T>, cs, bytes))) {
    launch_cluster(k_inv_cluster<T>, nparts, cs, 256, bytes, st, parts, t, B, G, status, cs);
    return;
  }
  // no cluster fits: one CTA per block, working matrix in global memory
  const int smax = inv_smem_max_m<T>();
  const size_t base = 2 * kMaxM * sizeof(int) + 2 * kMaxM * sizeof(T);
  const size_t gbytes = base + (max_m <= smax ? (size_t)max_m * (max_m + 1) * sizeof(T) : 0);
  allow_smem(k_inv<T>, gbytes);
  const int thr = max_m >= 128 ? 512 : (max_m >= 48 ? 256 : 128);
  // capacity actually allocated: every block up to max_m fits, or none does
  const int cap = max_m <= smax ? max_m : 0;
  k_inv<T><<<nparts, thr, gbytes, st>>>(parts, t, B, G, status, cap);
}

template <typename T>
void launch_fwd_factor(const PartDesc* parts, int nparts, int t, int max_m, const double* A,
                       const double* B, const double* C, T* G, T* Acal, T* ZL, T* ZR, cudaStream_t st,
                       int type_lo, int type_hi) {
  if (nparts <= 0 || type_hi <= type_lo) return;
  const int nt = type_hi - type_lo;
  if (max_m <= 256) {
    constexpr int W = 32;
    const int tiles = ntiles<W>(max_m);
    const size_t bytes = panel_smem<T>(max_m, W, 2);
    allow_smem(k_fwd_factor<T, W>, bytes);
    k_fwd_factor<T, W><<<dim3(nt * tiles, nparts), kThreads, bytes, st>>>(parts, t, tiles, type_lo, A, B, C, G, Acal,
                                                                          ZL, ZR);
  } else {
    constexpr int W = 16;
    const int tiles = ntiles<W>(max_m);
    const size_t bytes = panel_smem<T>(max_m, W, 2);
    allow_smem(k_fwd_factor<T, W>, bytes);
    k_fwd_factor<T, W><<<dim3(nt * tiles, nparts), kThreads, bytes, st>>>(parts, t, tiles, type_lo, A, B, C, G, Acal,
                                                                          ZL, ZR);
  }
}

template <typename T>
void launch_back_factor(const PartDesc* parts, int nparts, int s, int max_m, const T* Acal, T* ZL,
                        T* ZR, cudaStream_t st) {
  if (nparts <= 0) return;
  if (max_m <= 256) {
    constexpr int W = 32;
    const int tiles = ntiles<W>(max_m);
    const size_t bytes = panel_smem<T>(max_m, W, 1);
    allow_smem(k_back_factor<T, W>, bytes);
    k_back_factor<T, W><<<dim3(2 * tiles, nparts), kThreads, bytes, st>>>(parts, s, tiles, Acal, ZL, ZR);
  } else {
    constexpr int W = 16;
    const int tiles = ntiles<W>(max_m);
    const size_t bytes = panel_smem<T>(max_m, W, 1);
    allow_smem(k_back_factor<T, W>, bytes);
    k_back_factor<T, W><<<dim3(2 * tiles, nparts), kThreads, bytes, st>>>(parts, s, tiles, Acal, ZL, ZR);
  }
}

template <typename T>
void launch_fwd_solve(const PartDesc* parts, int nparts, int t, int max_m, int max_r,
                      const double* A, const T* G, const double* F, T* z, cudaStream_t st) {
  if (nparts <= 0) return;
  if (narrow_dispatch(max_r, [&](auto rm) {
        constexpr int RM = decltype(rm)::value;
        const size_t bytes = sizeof(T) * 2 * (size_t)max_m * RM;
        allow_smem(k_fwd_solve_n<T, RM>, bytes);
        k_fwd_solve_n<T, RM><<<nparts, 256, bytes, st>>>(parts, t, A, G, F, z);
      }))
    return;
  if (max_r <= 16) {
    constexpr int W = 16;
    const size_t bytes = panel_smem<T>(max_m, W, 2);
    allow_smem(k_fwd_solve<T, W>, bytes);
    k_fwd_solve<T, W><<<dim3(ntiles<W>(max_r), nparts), kThreads, bytes, st>>>(parts, t, 1, A, G, F, z);
  } else {
    constexpr int W = 32;
    const size_t bytes = panel_smem<T>(max_m, W, 2);
    allow_smem(k_fwd_solve<T, W>, bytes);
    k_fwd_solve<T, W><<<dim3(ntiles<W>(max_r), nparts), kThreads, bytes, st>>>(parts, t, 1, A, G, F, z);
  }
}

template <typename T>
void launch_back_solve(const PartDesc* parts, int nparts, int s, int max_m, int max_r,
                       const T* Acal, T* z, cudaStream_t st) {
  if (nparts <= 0) return;
  if (narrow_dispatch(max_r, [&](auto rm) {
        constexpr int RM = decltype(rm)::value;
        const size_t bytes = sizeof(T) * (size_t)max_m * RM;
        allow_smem(k_back_solve_n<T, RM>, bytes);
        k_back_solve_n<T, RM><<<nparts, 256, bytes, st>>>(parts, s, Acal, z);
      }))
    return;
  if (max_r <= 16) {
    constexpr int W = 16;
    const size_t bytes = panel_smem<T>(max_m, W, 1);
    allow_smem(k_back_solve<T, W>, bytes);
    k_back_solve<T, W><<<dim3(ntiles<W>(max_r), nparts), kThreads, bytes, st>>>(parts, s, 1, Acal, z);
  } else {
    constexpr int W = 32;
    const size_t bytes = panel_smem<T>(max_m, W, 1);
    allow_smem(k_back_solve<T, W>, bytes);
    k_back_solve<T, W><<<dim3(ntiles<W>(max_r), nparts), kThreads, bytes, st>>>(parts, s, 1, Acal, z);
  }
}

template <typename T, int RM>
cudaLaunchConfig_t sweep_config(int nparts, int cs, int max_m, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nparts * cs);
  cfg.blockDim = dim3(kSweepThreads);
  cfg.dynamicSmemBytes = sizeof(T) * 3 * (size_t)max_m * RM;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Largest cluster size (about 16 rows per CTA, at most the portable 8) at
// which all nparts clusters are resident together; 0 if none.
template <typename T>
int sweep_choice_t(int max_m, int max_r, int nparts) {
  if (max_r > 16 || sizeof(T) * 3 * (size_t)max_m * (size_t)rbucket(max_r) > 227 * 1024) return 0;
  if (nparts <= 0) return 0;
  int cs = 1;
  while (cs < 8 && cs * 16 < max_m) cs *= 2;
  int chosen = 0;
  narrow_dispatch(max_r, [&](auto rm) {
    constexpr int RM = decltype(rm)::value;
    allow_smem(k_sweep_solve_n<T, RM>, sizeof(T) * 3 * (size_t)max_m * RM);
    for (int c = cs; c >= 1 && !chosen; c /= 2) {
      cudaLaunchAttribute attr[1];
      cudaLaunchConfig_t cfg = sweep_config<T, RM>(nparts, c, max_m, nullptr, attr);
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_sweep_solve_n<T, RM>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
      if (nclusters >= nparts) chosen = c;
    }
  });
  return chosen;
}

int sweep_cluster_choice(int elem_bytes, int max_m, int max_r, int nparts) {
  return elem_bytes == 4 ? sweep_choice_t<float>(max_m, max_r, nparts) : sweep_choice_t<double>(max_m, max_r, nparts);
}

template <typename T>
void launch_sweep_solve(const PartDesc* parts, int nparts, int cs, int max_m, int max_r, const double* A,
                        const T* G, const T* Acal, const double* F, T* z, cudaStream_t st) {
  if (nparts <= 0 || cs <= 0) return;
  narrow_dispatch(max_r, [&](auto rm) {
    constexpr int RM = decltype(rm)::value;
    allow_smem(k_sweep_solve_n<T, RM>, sizeof(T) * 3 * (size_t)max_m * RM);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = sweep_config<T, RM>(nparts, cs, max_m, st, attr);
    cudaLaunchKernelEx(&cfg, k_sweep_solve_n<T, RM>, parts, cs, A, G, Acal, F, z);
  });
}

template <typename T>
void launch_assemble_h(const SepDesc* seps, int nseps, int max_m, const double* A, const double* B,
                       const double* C, const T* ZL, const T* ZR, double* HA, double* HB,
                       double* HC, cudaStream_t st) {
  if (nseps <= 0) return;
  if (max_m <= 256) {
    constexpr int W = 32;
    const int tiles = ntiles<W>(max_m);
    const size_t bytes = panel_smem<T>(max_m, W, 2);
    allow_smem(k_assemble_h<T, W>, bytes);
    k_assemble_h<T, W><<<dim3(3 * tiles, nseps), kThreads, bytes, st>>>(seps, tiles, A, B, C, ZL, ZR, HA, HB, HC);
  } else {
    constexpr int W = 16;
    const int tiles = ntiles<W>(max_m);
    const size_t bytes = panel_smem<T>(max_m, W, 2);
    allow_smem(k_assemble_h<T, W>, bytes);
    k_assemble_h<T, W><<<dim3(3 * tiles, nseps), kThreads, bytes, st>>>(seps, tiles, A, B, C, ZL, ZR, HA, HB, HC);
  }
}

template <typename T>
void launch_assemble_f(const SepDesc* seps, int nseps, int max_m, int max_r, const double* A,
                       const double* C, const double* F, const T* z, double* fh, cudaStream_t st) {
  if (nseps <= 0) return;
  if (narrow_dispatch(max_r, [&](auto rm) {
        constexpr int RM = decltype(rm)::value;
        const size_t bytes = sizeof(double) * 2 * (size_t)max_m * RM;
        allow_smem(k_assemble_f_n<T, RM>, bytes);
        k_assemble_f_n<T, RM><<<nseps, 256, bytes, st>>>(seps, A, C, F, z, fh);
      }))
    return;
  if (max_r <= 16) {
    constexpr int W = 16;
    const size_t bytes = panel_smem<double>(max_m, W, 2);
    allow_smem(k_assemble_f<T, W>, bytes);
    k_assemble_f<T, W><<<dim3(ntiles<W>(max_r), nseps), kThreads, bytes, st>>>(seps, 1, A, C, F, z, fh);
  } else {
    constexpr int W = 32;
    const size_t bytes = panel_smem<double>(max_m, W, 2);
    allow_smem(k_assemble_f<T, W>, bytes);
    k_assemble_f<T, W><<<dim3(ntiles<W>(max_r), nseps), kThreads, bytes, st>>>(seps, 1, A, C, F, z, fh);
  }
}

template <typename T>
void launch_backsub(const PartDesc* parts, int nparts, int Lmax, int max_m, int max_r, const T* ZL,
                    const T* ZR, const T* z, const double* h, double* x, cudaStream_t st) {
  if (nparts <= 0 || Lmax <= 0) return;
  if (narrow_dispatch(max_r, [&](auto rm) {
        constexpr int RM = decltype(rm)::value;
        const size_t bytes = sizeof(T) * 2 * (size_t)max_m * RM;
        allow_smem(k_backsub_n<T, RM>, bytes);
        k_backsub_n<T, RM><<<dim3(Lmax, nparts), 256, bytes, st>>>(parts, ZL, ZR, z, h, x);
      }))
    return;
  if (max_r <= 16) {
    constexpr int W = 16;
    const int tiles = ntiles<W>(max_r);
    const size_t bytes = panel_smem<double>(max_m, W, 2);
    allow_smem(k_backsub<T, W>, bytes);
    k_backsub<T, W><<<dim3(Lmax * tiles, nparts), kThreads, bytes, st>>>(parts, tiles, ZL, ZR, z, h, x);
  } else {
    constexpr int W = 32;
    const int tiles = ntiles<W>(max_r);
    const size_t bytes = panel_smem<double>(max_m, W, 2);
    allow_smem(k_backsub<T, W>, bytes);
    k_backsub<T, W><<<dim3(Lmax * tiles, nparts), kThreads, bytes, st>>>(parts, tiles, ZL, ZR, z, h, x);
  }
}

void launch_sep_copy(const SepDesc* seps, int nseps, int max_m, int max_r, const double* h,
                     double* x, cudaStream_t st) {
  if (nseps <= 0) return;
  k_sep_copy<<<nseps, 256, 0, st>>>(seps, h, x);
}

void launch_residual(const SysDesc* sys, int nsys, int nrows, int max_m, int max_r, const double* A,
                     const double* B, const double* C, const double* x, const double* b, double* r,
                     double* nrm, cudaStream_t st, const int* band) {
  if (nsys <= 0 || nrows <= 0) return;
  auto go = [&](auto rm) {
    constexpr int RM = decltype(rm)::value;
    const size_t bytes = sizeof(double) * 3 * (size_t)max_m * RM;
    allow_smem(k_residual<RM>, bytes);
    k_residual<RM><<<nrows, 256, bytes, st>>>(sys, nsys, A, B, C, x, b, r, nrm, band);
  };
  if (!narrow_dispatch(max_r, go)) go(std::integral_constant<int, 16>());
}

void launch_axpy_norms(const SysDesc* sys, int nsys, int nrows, int max_m, int max_r, const double* d,
                       double* x, double* nrm, cudaStream_t st) {
  if (nsys <= 0 || nrows <= 0) return;
  k_axpy_norms<<<nrows, 256, 0, st>>>(sys, nsys, d, x, nrm);
}

#define DM_INST(T)                                                                                  \
  template void launch_inv<T>(const PartDesc*, int, int, const double*, T*, int*, int, cudaStream_t); \
  template void launch_fwd_factor<T>(const PartDesc*, int, int, int, const double*, const double*,  \
                                     const double*, T*, T*, T*, T*, cudaStream_t, int, int);        \
  template void launch_back_factor<T>(const PartDesc*, int, int, int, const T*, T*, T*, cudaStream_t); \
  template void launch_fwd_solve<T>(const PartDesc*, int, int, int, int, const double*, const T*,   \
                                    const double*, T*, cudaStream_t);                               \
  template void launch_back_solve<T>(const PartDesc*, int, int, int, int, const T*, T*, cudaStream_t); \
  template void launch_sweep_solve<T>(const PartDesc*, int, int, int, int, const double*, const T*,   \
                                      const T*, const double*, T*, cudaStream_t);                    \
  template void launch_assemble_h<T>(const SepDesc*, int, int, const double*, const double*,        \
                                     const double*, const T*, const T*, double*, double*, double*,  \
                                     cudaStream_t);                                                 \
  template void launch_assemble_f<T>(const SepDesc*, int, int, int, const double*, const double*,   \
                                     const double*, const T*, double*, cudaStream_t);               \
  template void launch_backsub<T>(const PartDesc*, int, int, int, int, const T*, const T*, const T*, \
                                  const double*, double*, cudaStream_t);

DM_INST(double)
DM_INST(float)

}  // namespace dm

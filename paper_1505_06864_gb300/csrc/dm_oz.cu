// Float64 block products of the factor sweeps on the bf16 tensor cores by
// exact digit slicing (Ozaki's error-free splitting of matrix products; the
// digit extraction, accumulator grouping and pipeline are this library's).
//
// The products are the ones of the tensor-core step kernels (dm_tc2.cu):
// launch A = G_t [C_t | Y_t], launch B = A_{t+1} [Acal_t | Bcal_t], backward
// Acal_t [ZL_{t+1} | ZR_{t+1}] (Section 3 applied to Eq. e231), here with
// float64 operands and results.  Every operand block is cut into nine digit
// slices (dm_slices.cuh): a left operand L with one power-of-two scale per
// row r (|L[r][k]| < 2^e_r), a right operand R with one per column n
// (|R[k][n]| < 2^f_n), stored transposed (row n of the copy is column n of
// R).  Then
//
//   (L R)[r][n] = 2^(e_r + f_n) sum_{d=2..11} 2^(-6d) acc_d[r][n],
//   acc_d = sum_{s+t=d} Lslice_s Rslice_t,
//
// keeping the 53 slice pairs with s + t <= 11.  Each acc_d sums at most nine
// slice products over K = m <= 256 terms of magnitude <= 63^2: integers below
// 9 * 256 * 3969 < 2^24, so the float32 accumulation in tensor memory is
// exact.  The dropped pairs and the digit truncation bound the error of an
// entry by about K 2^-50 max_k |L[r][k]| max_k |R[k][n]|, the size of the
// float64 dot product's own bound.
//
// A CTA computes a 128 x 48 tile of one product: ten accumulators of 48
// columns (480 tensor-memory columns), a two-stage ring of 32-wide K slabs
// (nine left slices 72 KB + nine right slices 27 KB + a zero slice), one CTA
// per SM.  Per 16-wide K step one thread issues 14 MMAs: left slice s
// against right slices t = 1 .. T_s at once (stored consecutively, N = 48 per
// slice, at most five per instruction), into accumulators d = s + t.  With
// s = 1 the right slices run to a tenth, all-zero slice, so that the first
// K step's two instructions for s = 1 initialise all ten accumulators.  The
// epilogue combines the accumulators in 64-bit integers and scales once in
// float64 (GB300's float64 pipe is narrow).  Operand slices of results are
// made by separate slicing launches, which see whole rows and columns.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "dm_internal.cuh"
#include "dm_slices.cuh"
#include "dm_tcgen05.cuh"

namespace dm {
namespace oz {
using namespace ptx;

constexpr int kEpiWarps = 8;                 // epilogue warps 2 .. 9
constexpr int kThreads = 64 + 32 * kEpiWarps;  // warp 0: TMA producer, warp 1: MMA issuer
constexpr int MT = 128;          // rows per tile
constexpr int NT = 48;           // columns per tile
constexpr int NT3 = 32;          // columns per tile of the inverse's trailing updates (KIND 3)
constexpr int KS = 32;           // K elements per stage (64-byte rows, 64-byte swizzle)
constexpr int kStages = 2;
constexpr int S = kRsSlices;     // 9 slices
constexpr int NACC = 10;         // accumulators d = 2 .. 11
constexpr int ROWB = KS * 2;     // 64 bytes
constexpr int LSL = MT * ROWB;   // one left slice in a stage: 8 KB
constexpr int RSL = NT * ROWB;   // one right slice: 3 KB (2 KB for KIND 3, packed the same way)
constexpr int LBYTES = S * LSL;  // 72 KB
constexpr int RBYTES = (S + 1) * RSL;  // 30 KB with the zero slice
constexpr int STAGE = LBYTES + RBYTES;
constexpr int STG = 32 * 9;                  // an epilogue warp's 32 x 9 float64 staging tile
constexpr int SMEM = 1024 + kStages * STAGE + kEpiWarps * STG * 8;
constexpr uint32_t kCols = 512;
constexpr uint32_t kSbo = 8 * ROWB;  // 512-byte swizzle atoms
constexpr uint64_t kLayout = 4;       // 64-byte swizzle

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// The integer value of an integer-valued float32 |v| < 2^22: v + 1.5 2^23
// lies in [2^23, 2^24), where the float's low mantissa bits are v's.
__device__ __forceinline__ int acc_int_small(float v) { return __float_as_int(v + 12582912.0f) - 0x4B400000; }

// The integer value of an integer-valued float32 |v| < 2^24 from its bits.
__device__ __forceinline__ int acc_int(uint32_t b) {
  const uint32_t u = b & 0x7fffffffu;
  const uint32_t sh = min(150u - min(u >> 23, 150u), 31u);  // 23 - exponent; 31 for zero
  const int mag = (int)(((u & 0x7fffffu) | 0x800000u) >> sh);
  const int sg = (int)b >> 31;
  return (mag ^ sg) - sg;
}

// x 2^s as a float64, built from the bits: exact for |x| < 2^53 when the
// result is a normal number (the caller checks the exponent range).
__device__ __forceinline__ double i2d_scaled(long long x, int s) {
  const unsigned long long sg = (unsigned long long)x & 0x8000000000000000ull;
  const unsigned long long a = (unsigned long long)(x < 0 ? -x : x);
  const int lz = __clzll(a);                              // >= 11 for a < 2^53
  const unsigned long long mant = a << ((lz - 11) & 63);  // leading bit at 52
  // the leading bit adds one to the exponent field
  const unsigned long long ex = (unsigned long long)(1022 + 63 - lz + s);
  return a == 0 ? 0.0 : __longlong_as_double((long long)(sg | ((ex << 52) + mant)));
}

}  // namespace oz

struct OzMaps {
  CUtensorMap L, R0, R1;
};

namespace oz {

// KIND 0: launch A, 1: launch B (forward step `step`), 2: backward step
// `step`, over the subsystems.  Exponent arrays: [block][m] ints, indexed
// like the slices.
// KIND 3: the trailing update of panel `step` (columns K = [32 step, 32 step
// + 32)) of the blocked Gauss-Jordan inversion of block row `aux`:
// M[:, J] = (M[:, J] with the rows K zeroed) + U V, U the eliminated panel,
// V = M[K, J] before the update (both as slices, K = 32), J the other columns.
// KIND 4, 5: the supplementary blocks of a separator (Eq. e2311), left A_q /
// C_q: KIND 4 j = 0: HB = B_q - A_q ZR^j[q-1], j = 1: HA = -A_q ZL^j[q-1];
// KIND 5 j = 0: HB -= C_q ZL^{j+1}[q+1], j = 1: HC = -C_q ZR^{j+1}[q+1]
// (parts unused, out.seps instead).
//
// A tile = (subsystem or separator, product j, 128-row M-tile, 48-column
// N-tile); tile = ((unit * 2 + j) * ntm + M-tile) * ntn + N-tile (KIND 3,
// one product: (unit * ntm + M-tile) * ntn + N-tile).
struct OzTile {
  PartDesc p;
  SepDesc sd;
  int unit, j, tm, tn, t, zl, zr;
  bool act;
};

template <int KIND>
constexpr int nt_of() {
  return KIND == 3 ? NT3 : NT;
}

template <int KIND>
__device__ __forceinline__ OzTile oz_tile(int tile, const PartDesc* __restrict__ parts, const OzOut& out, int step,
                                          int aux, int m, int ntm, int ntn) {
  OzTile w{};
  constexpr int nj = KIND == 3 ? 1 : 2;  // KIND 3 has one product
  const int per = nj * ntm * ntn;
  w.unit = tile / per;
  const int rest = tile - w.unit * per;
  w.tn = rest % ntn;
  // KIND 3: the 32-column tile equal to panel `step` produces nothing and is
  // not enumerated (ntn counts the others)
  if (KIND == 3 && w.tn >= step) ++w.tn;
  const int r2 = rest / ntn;
  w.j = nj == 1 ? 0 : (r2 & 1);
  w.tm = nj == 1 ? r2 : (r2 >> 1);
  if constexpr (KIND >= 4)
    w.sd = out.seps[w.unit];
  else
    w.p = parts[w.unit];
  const PartDesc& p = w.p;
  const int j = w.j, pidx = w.unit;
  bool act;
  if (KIND == 4) {
    act = j == 0 || (w.sd.flags & HAS_HA) != 0;
  } else if (KIND == 5) {
    act = j == 0 || (w.sd.flags & HAS_HC) != 0;
  } else if (KIND == 0) {
    w.t = step;
    act = w.t < p.L && (j == 0 ? (w.t < p.L - 1 || (p.flags & HAS_RIGHT) != 0) : (p.flags & HAS_LEFT) != 0);
  } else if (KIND == 1) {
    w.t = step;
    act = w.t < p.L - 1 && (j == 0 || (p.flags & HAS_LEFT) != 0);
  } else if (KIND == 2) {
    w.t = p.L - 2 - step;
    act = w.t >= 0 && (j == 0 ? (p.flags & HAS_LEFT) != 0 : (p.flags & HAS_RIGHT) != 0);
  } else {
    w.t = aux;
    act = w.t < p.L && j == 0;
  }
  // products with a banded operand run in the banded kernels instead
  const bool banded = out.band && *out.band <= kBandMax;
  if (banded && ((KIND == 0 && j == 0) || KIND == 1 || KIND >= 4)) act = false;
  w.act = act && w.tm * MT < m && w.tn * nt_of<KIND>() < m;
  const long long mm = (long long)m * m;
  const int b0 = (int)(p.blk / mm), t = w.t;
  if (KIND == 4) {
    w.zl = (int)(w.sd.blk_q / mm);  // A_q (all blocks)
    w.zr = 4 * pidx + j;            // ZR^j[q-1]^T / ZL^j[q-1]^T
  } else if (KIND == 5) {
    w.zl = pidx;                    // C_q (per separator)
    w.zr = 4 * pidx + 2 + j;        // ZL^{j+1}[q+1]^T / ZR^{j+1}[q+1]^T
  } else if (KIND == 3) {
    w.zl = pidx;  // U slices (rolling)
    w.zr = pidx;  // V^T slices (rolling)
  } else if (KIND == 0) {
    w.zl = pidx;                     // G_t slices (rolling)
    w.zr = j == 0 ? b0 + t : pidx;   // C_t^T (all blocks) / Y_t^T (rolling)
  } else if (KIND == 1) {
    w.zl = b0 + t + 1;                          // A_{t+1}
    w.zr = j == 0 ? pidx : 2 * pidx + (t & 1);  // Acal_t^T / Bcal_t^T
  } else {
    w.zl = b0 + t;                    // Acal_t
    w.zr = 2 * pidx + ((t + 1) & 1);  // ZL_{t+1}^T / ZR_{t+1}^T
  }
  return w;
}

// Persistent: a CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x,
// ...  Warp 0 (one lane) streams every tile's K slabs by TMA into a two-stage
// ring and runs ahead into the next tile; warp 1 (one lane) issues the MMAs
// of a tile once the epilogue has drained the accumulators of the previous
// one (the ten accumulators take 480 of the 512 tensor-memory columns, so
// there is one set); warps 2-9 run the epilogue, loading what it needs
// besides the accumulators while the MMAs run.  Every wait is bounded; a
// role that gives up sets `err`, which the others see at their next tile.
template <int KIND>
__global__ void __launch_bounds__(kThreads, 1)
    k_oz_step(const PartDesc* __restrict__ parts, int step, int aux, int m, int ntm, int ntn, int ntiles, OzOut out,
              const int* __restrict__ lexp, const int* __restrict__ rexp0, const int* __restrict__ rexp1,
              int* __restrict__ errflag, const __grid_constant__ OzMaps maps) {
  constexpr int NTK = nt_of<KIND>();   // columns per tile
  constexpr int RSLK = NTK * ROWB;      // one right slice in a stage
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t full[kStages], empty[kStages], tfull, tempty, mdone;
  __shared__ uint32_t tmem_slot;
  __shared__ int err, nissued, ncons;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  double* stage_out = reinterpret_cast<double*>(base + kStages * STAGE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* verr = &err;
  // the zero right slice of both stages (never written by the copies)
  for (int st = 0; st < kStages; ++st)
    for (int i = threadIdx.x; i < RSLK / 16; i += kThreads)
      reinterpret_cast<uint4*>(base + st * STAGE + LBYTES + S * RSLK)[i] = make_uint4(0u, 0u, 0u, 0u);
  fence_async_shared();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&tfull, 1);
    mbar_init(&tempty, kEpiWarps);
    mbar_init(&mdone, 1);
    err = 0;
    nissued = 0;
    ncons = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_slot, kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const long long mm = (long long)m * m;
  const int nslab = KIND == 3 ? 1 : (m + KS - 1) / KS;
  constexpr uint32_t tx = (uint32_t)(S * (MT + NTK) * ROWB);

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*verr; tile += gridDim.x) {
        const OzTile w = oz_tile<KIND>(tile, parts, out, step, aux, m, ntm, ntn);
        if (!w.act) continue;
        const CUtensorMap* mr = w.j == 0 ? &maps.R0 : &maps.R1;
        bool ok = true;
        for (int s = 0; s < nslab; ++s, ++it) {
          const int st = it & 1;
          if (it >= kStages && !mbar_wait(&empty[st], (uint32_t)(((it >> 1) - 1) & 1))) {
            ok = false;
            break;
          }
          const uint32_t sb = smem_u32(base + st * STAGE);
          mbar_expect_tx(&full[st], tx);
          tma_load_4d(sb, &maps.L, s * KS, w.tm * MT, 0, w.zl, &full[st]);
          tma_load_4d(sb + LBYTES, mr, s * KS, w.tn * NTK, 0, w.zr, &full[st]);
        }
        if (!ok) {
          *verr = 1;
          break;
        }
      }
      nissued = it;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, lt = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*verr; tile += gridDim.x) {
        const OzTile w = oz_tile<KIND>(tile, parts, out, step, aux, m, ntm, ntn);
        if (!w.act) continue;
        // the accumulators of the previous tile have been read
        if (lt > 0 && !mbar_wait(&tempty, (uint32_t)((lt - 1) & 1))) {
          *verr = 1;
          break;
        }
        tc_fence_after();
        bool ok = true;
        for (int s = 0; s < nslab; ++s, ++it) {
          const int st = it & 1;
          if (!mbar_wait(&full[st], (uint32_t)((it >> 1) & 1))) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t la = smem_u32(base + st * STAGE), ra = la + LBYTES;
#pragma unroll
          for (int k = 0; k < KS / 16; ++k) {
            const uint32_t off = (uint32_t)(k * 32);
#pragma unroll
            for (int sl = 1; sl <= S; ++sl) {
              const int T = sl == 1 ? S + 1 : min(S, 11 - sl);  // s = 1 runs into the zero slice
              const uint64_t ad = kmajor_desc(la + (sl - 1) * LSL + off, kSbo, kLayout);
#pragma unroll
              for (int ta = 1; ta <= T; ta += 5) {
                const int cnt = min(5, T - ta + 1);
                const uint64_t bd = kmajor_desc(ra + (ta - 1) * RSLK + off, kSbo, kLayout);
                const uint32_t dcol = (uint32_t)((sl + ta - 2) * NTK);
                const uint32_t acc = (s == 0 && k == 0 && sl == 1) ? 0u : 1u;
                mma<1>(tmem + dcol, ad, bd, make_idesc(1u, MT, NTK * cnt), acc);
              }
            }
          }
          mma_commit(&empty[st]);
        }
        if (!ok) {
          *verr = 1;
          break;
        }
        mma_commit(&tfull);
        ++lt;
      }
      ncons = it;
      // every MMA issued here is complete before the accumulators are freed
      mma_commit(&mdone);
      mbar_wait(&mdone, 0u);
    }
    __syncwarp();
  } else {
    const int ew = warp - 2, quarter = warp & 3, half = ew >> 2;  // a warp reaches lanes 32 (warp % 4) ..
    double* stg = stage_out + ew * STG;
    const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
    const int cl = lane & 7, r0 = lane >> 3;
    const int k0 = 32 * step;  // KIND 3: the panel's columns and pivot rows
    int lt = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*verr; tile += gridDim.x) {
      const OzTile w = oz_tile<KIND>(tile, parts, out, step, aux, m, ntm, ntn);
      if (!w.act) continue;
      const int j = w.j, t = w.t, pidx = w.unit;
      const PartDesc& p = w.p;
      const SepDesc& sd = w.sd;
      const int* rexp = j == 0 ? rexp0 : rexp1;
      // Before the accumulators are ready: the row's scale, the column scales
      // of the warp's 24 columns (one per lane, passed by shuffle) and the
      // values the stores update (they do not depend on the products)
      const int rbase = w.tm * MT + quarter * 32, row = rbase + lane;
      const int er = row < m ? lexp[(long long)w.zl * m + row] : 0;
      int fexp = 0;
      {
        const int n = w.tn * NTK + half * (NTK / 2) + lane;
        if (lane < NTK / 2 && n < m) fexp = rexp[(long long)w.zr * m + n];
      }
      const bool rmw = KIND == 2 && j == 0, dnext = KIND == 1 && j == 0, gj = KIND == 3, hb = KIND >= 4 && j == 0;
      const bool upd = rmw || dnext || gj || hb;
      const long long o = p.blk + (long long)t * mm;
      const double* src = rmw    ? out.ZL + o
                          : gj   ? out.G + o
                          : hb   ? (KIND == 4 ? out.B + sd.blk_q : out.HB + sd.hblk)
                                 : out.B + o + mm;
      // the values chunk ci's stores update, loaded one chunk ahead
      auto load_in = [&](int ci, double (&in)[8]) {
        const int n = w.tn * NTK + half * (NTK / 2) + 8 * ci + cl;
        const bool outside = KIND != 3 || n < k0 || n >= k0 + 32;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rr = rbase + r0 + 4 * i;
          in[i] = (upd && n < m && outside && rr < m && !(gj && rr >= k0 && rr < k0 + 32)) ? src[(long long)rr * m + n]
                                                                                          : 0.0;
        }
      };
      double incur[8], innext[8];
      load_in(0, incur);
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull, (uint32_t)(lt & 1)));
      if (!ok) {
        *verr = 1;
        break;
      }
      tc_fence_after();
      // Accumulators of this thread's row (tensor-memory lane) for 8 columns
      // at a time.  Each acc_d is an integer-valued float below 2^24: its
      // integer comes from the float's bits (float32 and integer operations),
      // pairs P_j = acc_{2j+2} 64 + acc_{2j+3} are exact in 32 bits, and
      //   hi = P_0 2^12 + P_1 (< 2^39),  lo = (P_2 2^12 + P_3) 2^12 + P_4 (< 2^53)
      // give the sum exactly as hi 2^36 + lo.  Both become float64 from their
      // bits with the scale 2^(e_r + f_n - 66) in the exponent, and one
      // float64 add rounds their sum once (one issue slot; rounding the
      // 128-bit sum in integer arithmetic measured slower).  Warps of the
      // same lane quarter share the tile's columns.  Results are staged
      // through the warp's 32 x 9 float64 tile so that row-major writes are
      // coalesced.
      // acc_d below 2^22 for every d (then the float32 magic-number
      // conversion is exact): K = 32, or K = m <= 112 (acc_d <= 9 K 63^2)
      const bool small = KIND == 3 || m <= 112;
#pragma unroll
      for (int ci = 0; ci < NTK / 16; ++ci) {
        const int ch = half * (NTK / 2) + 8 * ci;
        // chunks past the block's last column, and (KIND 3) inside the
        // panel's columns, produce nothing: only the release of the
        // accumulators after the last chunk remains
        const int c0n = w.tn * NTK + ch;
        const bool dead = c0n >= m || (KIND == 3 && c0n >= k0 && c0n < k0 + 32);
        if (dead) {
          if (ci == NTK / 16 - 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty);
          } else {
            load_in(ci + 1, innext);
#pragma unroll
            for (int i = 0; i < 8; ++i) incur[i] = innext[i];
          }
          continue;
        }
        uint32_t r[NACC][8];
#pragma unroll
        for (int dd = 0; dd < NACC; ++dd) tmem_ld8_nowait(tl + (uint32_t)(dd * NTK + ch), r[dd]);
        tmem_wait_ld();
#pragma unroll
        for (int dd = 0; dd < NACC; ++dd) tmem_regs_after_wait(r[dd]);
        if (ci == NTK / 16 - 1) {  // the last accumulator read of this tile: the MMAs may go on
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty);
        } else {
          load_in(ci + 1, innext);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int n = w.tn * NTK + ch + c;
          const int k = er + __shfl_sync(0xffffffffu, fexp, 8 * ci + c);
          int a[NACC];
#pragma unroll
          for (int dd = 0; dd < NACC; ++dd)
            a[dd] = (dd < 4 || small) ? acc_int_small(__uint_as_float(r[dd][c])) : acc_int(r[dd][c]);
          const long long hi = (long long)(a[0] * 64 + a[1]) * 4096 + (a[2] * 64 + a[3]);
          const long long lo =
              ((long long)(a[4] * 64 + a[5]) * 4096 + (a[6] * 64 + a[7])) * 4096 + (a[8] * 64 + a[9]);
          double val = 0.0;
          const bool kept = KIND != 3 || n < k0 || n >= k0 + 32;  // KIND 3: not the panel's columns
          if (row < m && n < m && kept) {
            const float a2 = __uint_as_float(r[0][c]);
            if (a2 != a2)  // NaN or infinite operand: every digit is NaN, acc_2 included
              val = __longlong_as_double(0x7ff8000000000000ll);
            else if ((hi | lo) == 0)  // also the zero rows and columns, whose scale is the smallest
              val = 0.0;
            else if (k - 66 >= -1022 && k + 9 <= 1023)
              val = i2d_scaled(hi, k - 30) + i2d_scaled(lo, k - 66);
            else
              val = ldexp(fma((double)lo, 0x1p-36, (double)hi), k - 30);
          }
          stg[lane * 9 + c] = val;
        }
        __syncwarp();
        // row-major float64 results: lane = (row quarter, column), 8 row quads
        const int n = w.tn * NTK + ch + cl;
        const bool outside = KIND != 3 || n < k0 || n >= k0 + 32;
        if (n < m && outside) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int rl = r0 + 4 * i, rr = rbase + rl;
            if (rr >= m) continue;
            const double v = stg[rl * 9 + cl];
            const long long e = (long long)rr * m + n;
            if (KIND >= 4) {
              if (j == 0)
                out.HB[sd.hblk + e] = incur[i] - v;               // HB = B_q - A_q ZR, then HB -= C_q ZL
              else
                (KIND == 4 ? out.HA : out.HC)[sd.hblk + e] = -v;  // HA = -A_q ZL, HC = -C_q ZR
            } else if (KIND == 0) {
              double* d = (j == 0) ? (t < p.L - 1 ? out.Acal : out.ZR) : out.ZL;
              d[o + e] = v;
            } else if (dnext) {
              out.G[o + mm + e] = incur[i] - v;                    // D_{t+1} = B_{t+1} - A_{t+1} Acal_t
            } else if (KIND == 1) {
              out.Y[(long long)pidx * mm + e] = -v;                // Y_{t+1} = -A_{t+1} Bcal_t
            } else if (rmw) {
              out.ZL[o + e] = incur[i] - v;                        // ZL_t -= Acal_t ZL_{t+1}
            } else if (gj) {
              out.G[o + e] = incur[i] + v;                         // Gauss-Jordan trailing update
            } else {
              out.ZR[o + e] = -v;                                  // ZR_t = -Acal_t ZR_{t+1}
            }
          }
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 8; ++i) incur[i] = innext[i];
      }
      ++lt;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0)  // copies still in flight after an error
    for (int s = ncons; s < nissued; ++s) mbar_wait(&full[s & 1], (uint32_t)((s >> 1) & 1));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kCols);
  if (threadIdx.x == 0 && err && errflag) atomicExch(errflag, 1);
}

// ---------------------------------------------------------------- slicing
// A CTA slices one group of 32 rows (left operands) or 32 columns (right
// operands) of one float64 m x m block; a block takes ceil(m / 32) CTAs.

// Row slices (left operands): exps[r] = e with |v| < 2^e for the row's
// largest |v|; slice s element (r, k) at (q * 9 + s) m^2 + r m + k.  One
// warp per row, eight consecutive columns per lane (m % 8 == 0).
__device__ __forceinline__ void slice_rows_group(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                                                 long long qdst, int* __restrict__ exps, int m, int g) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long long mm = (long long)m * m;
  const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(src);
  const int rend = min(m, 32 * g + 32);
  for (int r = 32 * g + warp; r < rend; r += nw) {
    uint32_t hmax = 0;
    for (int c = lane; c < m; c += 32) hmax = max(hmax, (uint32_t)(bits[(long long)r * m + c] >> 32) & 0x7fffffffu);
#pragma unroll
    for (int o = 16; o; o >>= 1) hmax = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    const int e = scale_exponent(hmax);
    if (lane == 0) exps[qdst * m + r] = e;
    for (int c0 = lane * 8; c0 < m; c0 += 256) {
      uint32_t q[8][S];
#pragma unroll
      for (int u = 0; u < 8; ++u) digits9(bits[(long long)r * m + c0 + u], e, q[u]);
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        uint4 w;
        w.x = (q[0][sl] >> 16) | (q[1][sl] & 0xffff0000u);
        w.y = (q[2][sl] >> 16) | (q[3][sl] & 0xffff0000u);
        w.z = (q[4][sl] >> 16) | (q[5][sl] & 0xffff0000u);
        w.w = (q[6][sl] >> 16) | (q[7][sl] & 0xffff0000u);
        *reinterpret_cast<uint4*>(dst + (qdst * S + sl) * mm + (long long)r * m + c0) = w;
      }
    }
  }
}

// Column slices, transposed (right operands): exps[n] for column n, slice s
// element (n, k) = digit s of src[k][n] at (q * 9 + s) m^2 + n m + k.  The
// group's 32 column maxima first (eight warps over the rows), then 32 x 32
// tiles through shared memory; a thread writes four consecutive k of one n
// per slice (8-byte stores).  256 threads.
__device__ __forceinline__ void slice_cols_group(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                                                 long long qdst, int* __restrict__ exps, int m, int g,
                                                 uint32_t (*red)[32], int* s_e, unsigned long long (*tile)[33]) {
  const long long mm = (long long)m * m;
  const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(src);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = 32 * g + lane;
  uint32_t hmax = 0;
  if (n < m)
    for (int k = warp; k < m; k += 8) hmax = max(hmax, (uint32_t)(bits[(long long)k * m + n] >> 32) & 0x7fffffffu);
  red[warp][lane] = hmax;
  __syncthreads();
  if (warp == 0) {
    uint32_t h = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) h = max(h, red[w][lane]);
    const int e = scale_exponent(h);
    s_e[lane] = e;
    if (n < m) exps[qdst * m + n] = e;
  }
  __syncthreads();
  const int nl = threadIdx.x >> 3, kq = (threadIdx.x & 7) * 4;
  for (int k0 = 0; k0 < m; k0 += 32) {
    for (int y = warp; y < 32; y += 8) {
      const int k = k0 + y;
      tile[y][lane] = (k < m && n < m) ? bits[(long long)k * m + n] : 0ull;
    }
    __syncthreads();
    const int nn = 32 * g + nl, k = k0 + kq;
    if (nn < m && k < m) {  // m % 8 == 0: four consecutive k are all inside
      uint32_t q[4][S];
#pragma unroll
      for (int u = 0; u < 4; ++u) digits9(tile[kq + u][nl], s_e[nl], q[u]);
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        uint2 w;
        w.x = (q[0][sl] >> 16) | (q[1][sl] & 0xffff0000u);
        w.y = (q[2][sl] >> 16) | (q[3][sl] & 0xffff0000u);
        *reinterpret_cast<uint2*>(dst + (qdst * S + sl) * mm + (long long)nn * m + k) = w;
      }
    }
    __syncthreads();
  }
}

// Slices of every block of a level's array (A as rows, C as transposed
// columns): blockIdx.x = block * groups + group, looping past the grid.
// With `band` set and the level's A and C banded (*band <= kBandMax), nothing
// is done: only the tensor-core tiles the banded kernels replace read these.
template <bool COLS>
__global__ void __launch_bounds__(256) k_oz_slice_all(const double* __restrict__ src, int nblocks, int m,
                                                      __nv_bfloat16* __restrict__ dst, int* __restrict__ exps,
                                                      const int* __restrict__ band) {
  __shared__ uint32_t red[8][32];
  __shared__ int s_e[32];
  __shared__ unsigned long long tile[32][33];
  if (band && *band <= kBandMax) return;
  const long long mm = (long long)m * m;
  const int groups = (m + 31) / 32;
  for (long long i = blockIdx.x; i < (long long)nblocks * groups; i += gridDim.x) {
    const int q = (int)(i / groups), g = (int)(i - (long long)q * groups);
    if (COLS)
      slice_cols_group(src + q * mm, dst, q, exps, m, g, red, s_e, tile);
    else
      slice_rows_group(src + q * mm, dst, q, exps, m, g);
    __syncthreads();
  }
}

// Per-subsystem slicing jobs (k_oz_slice_jobs, blockIdx.x = subsystem), kind:
//   0 G_t rows -> rolling (q);            1 Acal_t rows -> all blocks (b0 + t);
//   2 Acal_t columns -> rolling (q);      3 ZL_t columns -> rolling slot (2q + t%2);
//   4 ZR_{L-1} columns (last row, right spike) -> slot;  5 Y_{t+1} columns -> rolling (q);
//   6 ZL_t columns, backward step;        7 ZR_t columns, backward step;
//   8 Y_0 = A_first columns -> rolling (q), at the start of a factorisation.
// ---------------------------------------------------------------- blocked Gauss-Jordan inversion
// The float64 block inverse G_t = D_t^{-1} with partial pivoting (the
// paper's inversion, Section 4; Gauss-Jordan as in the library's other
// inverses), blocked by panels of 32 columns so that 15/16 of its float64
// multiply-adds (the rank-32 trailing updates) run on the tensor cores as
// digit-sliced products (KIND 3 above).  For panel K = [k0, k0 + 32):
//   1. k_gj_panel (float64, a cluster of CTAs per block, a thread per row
//      holding the panel's 32 values): for each k in K, the pivot row r =
//      argmax_{i >= k} |M[i][k]| (ties to the lowest row) is exchanged with
//      row k, then in-place Gauss-Jordan restricted to the panel's columns:
//      row k scaled by 1/M[k][k] with 1/M[k][k] in column k, every other row
//      i minus M[i][k] times row k with -M[i][k]/M[k][k] in column k.  The
//      panel then holds U = [W; -M_RK W] (W = M_KK^{-1}); the kernel applies
//      the row exchanges to the other columns and writes U's row slices and
//      the column slices of V = M[K, J] (the pivot rows outside K).
//   2. k_oz_step<3>: M[:, J] = (M[:, J], rows K zeroed) + U V.
// After the last panel, k_gj_finish undoes the row exchanges on the columns
// (column c of the working matrix is column piv[c] of D^{-1}) and writes the
// row slices of the inverse.
__global__ void __launch_bounds__(256) k_gj_copy_b0(const PartDesc* __restrict__ parts, int m,
                                                    const double* __restrict__ B, double* __restrict__ G) {
  const PartDesc p = parts[blockIdx.x];
  const long long mm = (long long)m * m;
  for (long long e = threadIdx.x; e < mm; e += blockDim.x) G[p.blk + e] = B[p.blk + e];
}

// One panel, one cluster of kGjCS CTAs per block: CTA `rank` holds rows
// [rank R, rank R + R) (R = ceil(m / kGjCS)); warp w of it rows R rank + 16 w
// + (0..15), two lanes per row (lane = 16 h + row): lane half h holds panel
// columns 16 h .. 16 h + 15 in registers, rotated by one column per pivot (at
// pivot kk the row's register c of half h is panel column (kk + 16 h + c) mod
// 32, so the pivot column is always register 0 of half 0 and the loop needs
// no unrolling; after 32 pivots the order is back).
//
// GB300's float64 unit takes a warp instruction per about 68 cycles per SM
// sub-partition and a dependent one 66 cycles later (a division about 460),
// so the per-pivot chain keeps float64 instructions to the arithmetic: the
// pivot search orders the float64 bits of |M[i][k]| as integers, the checks
// read the bits, the reciprocal is taken once per CTA, the rank-1 update (16
// multiply-adds per lane) is spread over four warps per CTA, and it overlaps
// the cluster barrier by one pivot of lookahead.  With pivot kk's scaled row
// known, every row first updates only its next pivot column; the warps and
// then the CTA choose their best row for pivot kk + 1 on it (a strict order:
// magnitude, then lowest row), and that row is published as it is BEFORE
// pivot kk's update, with its multiplier f and the reciprocal of its updated
// pivot (row k + 1 likewise).  The CTA arrives at the cluster barrier, makes
// the bulk update of its rows, then waits; each lane then reads the kGjCS
// candidates and element `lane` (+ 1, the rotation) of each candidate row
// and of row k + 1 through distributed shared memory (one round of
// independent loads), picks the winner and applies pivot kk's update to that
// one element (the multiply-add its owner made).  The exchanges of rows
// outside the panel are applied after the last pivot as one permutation
// (pivot rows are always taken from rows >= k, so every row outside K that
// moves receives a row of K).
constexpr int kGjCS = 4;
constexpr int kGjThreads = 128;
constexpr int kGjWarps = kGjThreads / 32;
static_assert(kGjWarps * 16 * kGjCS >= kMaxMTensor, "a lane pair per row");

struct __align__(16) GjKey {
  unsigned long long key;  // 0: not eligible; 1: NaN; else |value| bits + 2
  int idx;                 // row (unique per thread, so the order is strict)
  int pad;
};

struct __align__(16) GjCand {
  unsigned long long key;
  int idx, pad;
  double inv;  // 1 / the candidate's updated pivot (0 when unusable)
  double f;    // the candidate's multiplier of the previous pivot
};

__device__ __forceinline__ bool gj_before(unsigned long long ok, int oi, unsigned long long k, int i) {
  return ok > k || (ok == k && oi < i);
}

__device__ __forceinline__ unsigned long long gj_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  return b > 0x7ff0000000000000ull ? 1ull : b + 2ull;
}

// zero, below 2^-1022 (whose reciprocal overflows), at or above 2^1022
// (whose reciprocal is not a normal number) or not finite
__device__ __forceinline__ bool gj_unusable(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  return b < 0x0010000000000000ull || b >= 0x7fd0000000000000ull;
}

// 1/x for a usable pivot x (2^-1022 <= |x| < 2^1022): the PTX reciprocal
// approximation rcp.approx.ftz.f64 refined by two Newton-Raphson steps for
// f(y) = 1/y - x, y <- y + y (1 - x y), each of which squares the relative
// error (within about one unit in the last place of 1/x).  It has no
// branch, so the compiler can interleave it with the pivot search.
__device__ __forceinline__ double gj_recip(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// The CTA's best of every lane's (key, idx): the warp's largest key (its high
// word, then its low word among the lanes with that high word) and the lowest
// row holding it, by three warp reductions; then the best of the warps' bests
// after a CTA barrier (the same result in every thread).
__device__ __forceinline__ GjKey gj_cta_best(unsigned long long key, int idx, GjKey* wbest, int warp, int lane) {
  const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
  const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
  const unsigned mi = __reduce_min_sync(0xffffffffu, hi == mh && lo == ml ? (unsigned)idx : 0xffffffffu);
  key = ((unsigned long long)mh << 32) | ml;
  idx = (int)mi;
  if (lane == 0) wbest[warp] = GjKey{key, idx, 0};
  __syncthreads();
  GjKey best = wbest[0];
#pragma unroll
  for (int w = 1; w < kGjWarps; ++w) {
    const GjKey o = wbest[w];
    if (gj_before(o.key, o.idx, best.key, best.idx)) best = o;
  }
  return best;
}

__device__ __forceinline__ GjCand gj_read_cand(const GjCand* c) {
  const uint4* v = reinterpret_cast<const uint4*>(c);
  const uint4 a = v[0], b = v[1];
  GjCand r;
  r.key = ((unsigned long long)a.y << 32) | a.x;
  r.idx = (int)a.z;
  r.pad = 0;
  r.inv = __hiloint2double((int)b.y, (int)b.x);
  r.f = __hiloint2double((int)b.w, (int)b.z);
  return r;
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

__global__ void __launch_bounds__(kGjThreads) k_gj_panel(const PartDesc* __restrict__ parts, int t, int m, int panel,
                                                        double* __restrict__ G, int* __restrict__ piv,
                                                        __nv_bfloat16* __restrict__ Us, int* __restrict__ Uexp,
                                                        __nv_bfloat16* __restrict__ Vs, int* __restrict__ Vexp,
                                                        int* __restrict__ status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  // published per pivot (double-buffered: a buffer is rewritten two pivots
  // later, after a cluster barrier that every reader of it has passed)
  __shared__ __align__(16) double crow[2][32], krow[2][32];
  __shared__ GjCand cand[2];
  __shared__ double kf[2];
  // this CTA's own
  __shared__ GjKey wbest[kGjWarps];
  __shared__ __align__(16) double sprow[kGjWarps][32], xrow[kGjWarps][32];
  __shared__ int piv_s[32], perm[kMaxMTensor], cperm[kMaxMTensor];
  const int rank = (int)cl.block_rank();
  const int q = blockIdx.x / kGjCS;
  const PartDesc p = parts[q];
  if (t >= p.L) return;  // the same for every CTA of the cluster
  const long long mm = (long long)m * m;
  double* M = G + p.blk + (long long)t * mm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, h = lane >> 4, rl = warp * 16 + (lane & 15);
  const int R = (m + kGjCS - 1) / kGjCS, i = rank * R + rl;
  const bool valid = rl < R && i < m;
  const int k0 = 32 * panel, kw = min(32, m - k0);  // kw % 8 == 0
  const int noidx = m + rank * kGjThreads + tid;   // an index no row has
  double reg[16];
#pragma unroll
  for (int c = 0; c < 16; c += 2) {
    double2 v2 = make_double2(0.0, 0.0);
    if (valid && 16 * h + c < kw) v2 = *reinterpret_cast<const double2*>(M + (long long)i * m + k0 + 16 * h + c);
    reg[c] = v2.x;
    reg[c + 1] = v2.y;
  }
  bool bad = false;
  double* sp = sprow[warp];
  double* xr = xrow[warp];
  int r;  // the current pivot row
  {
    // pivot k0: candidates from the rows as they are
    const bool elig = h == 0 && valid && i >= k0;
    const GjKey best = gj_cta_best(elig ? gj_key(reg[0]) : 0ull, elig ? i : noidx, wbest, warp, lane);
    if (valid && i == best.idx) {
#pragma unroll
      for (int c = 0; c < 16; c += 2)
        *reinterpret_cast<double2*>(&crow[0][16 * h + c]) = make_double2(reg[c], reg[c + 1]);
      if (h == 0) {
        cand[0].inv = gj_unusable(reg[0]) ? 0.0 : gj_recip(reg[0]);
        cand[0].f = 0.0;
      }
    }
    if (valid && i == k0)
#pragma unroll
      for (int c = 0; c < 16; c += 2)
        *reinterpret_cast<double2*>(&krow[0][16 * h + c]) = make_double2(reg[c], reg[c + 1]);
    if (tid == 0) cand[0].key = best.key, cand[0].idx = best.idx;
    cl.sync();
    GjCand w = gj_read_cand(cl.map_shared_rank(&cand[0], 0));
    double prow = cl.map_shared_rank(&crow[0][0], 0)[lane];
#pragma unroll
    for (int s = 1; s < kGjCS; ++s) {
      const GjCand o = gj_read_cand(cl.map_shared_rank(&cand[0], s));
      const double v = cl.map_shared_rank(&crow[0][0], s)[lane];
      if (gj_before(o.key, o.idx, w.key, w.idx)) w = o, prow = v;
    }
    const double xk = cl.map_shared_rank(&krow[0][0], k0 / R)[lane];
    const double p0 = __shfl_sync(0xffffffffu, prow, 0);
    double inv = w.inv;
    if (gj_unusable(p0)) inv = 0.0, bad = true;
    r = w.idx;
    if (r < k0 || r >= m) r = k0, inv = 0.0, bad = true;  // never: the winner is an eligible row
    sp[lane] = lane == 0 ? inv : prow * inv;  // the scaled pivot row
    xr[lane] = xk;                            // the old row k
    if (tid == 0) piv_s[0] = r;
    __syncwarp();
  }
  // the cluster's published candidates and rows, mapped once (buffer b at + b)
  const GjCand* rcand[kGjCS];
  const double* rcrow[kGjCS];
#pragma unroll
  for (int s = 0; s < kGjCS; ++s) {
    rcand[s] = cl.map_shared_rank(&cand[0], s);
    rcrow[s] = cl.map_shared_rank(&crow[0][0], s);
  }
  // the CTA holding row k + 1 and that row's place in it, advanced per pivot
  int ko = (k0 + 1) / R, kro = (k0 + 1) - ko * R;
#pragma unroll 1
  for (int kk = 0; kk < 32; ++kk) {
    if (kk >= kw) {  // padding columns of a narrow last panel: rotate only
      const double nxt = __shfl_xor_sync(0xffffffffu, reg[0], 16);
#pragma unroll
      for (int c = 0; c < 15; ++c) reg[c] = reg[c + 1];
      reg[15] = nxt;
      continue;
    }
    const int k = k0 + kk;
    const bool la = kk + 1 < kw, swap = i == r && i != k;  // row r takes the old row k
    if (swap)
#pragma unroll
      for (int c = 0; c < 16; c += 2) {
        const double2 v2 = *reinterpret_cast<const double2*>(&xr[16 * h + c]);
        reg[c] = v2.x;
        reg[c + 1] = v2.y;
      }
    const double other = __shfl_xor_sync(0xffffffffu, reg[0], 16);  // the other half's first column
    const double f = h == 0 ? reg[0] : other;  // the row's multiplier (column kk)
    if (la) {
      // the next pivot column of every row first, its candidates, and the
      // CTA's best row published before the update
      const int buf = (kk + 1) & 1;
      const double new1 = i == k ? sp[1] : fma(-f, sp[1], reg[1]);
      const bool elig = h == 0 && valid && i > k;
      const double rinv = gj_recip(new1);  // every row's, overlapping the search
      const GjKey best = gj_cta_best(elig ? gj_key(new1) : 0ull, elig ? i : noidx, wbest, warp, lane);
      if (valid && i == best.idx) {
#pragma unroll
        for (int c = 0; c < 16; c += 2)
          *reinterpret_cast<double2*>(&crow[buf][16 * h + c]) = make_double2(reg[c], reg[c + 1]);
        if (h == 0) {
          cand[buf].inv = gj_unusable(new1) ? 0.0 : rinv;
          cand[buf].f = f;
        }
      }
      if (valid && i == k + 1) {
#pragma unroll
        for (int c = 0; c < 16; c += 2)
          *reinterpret_cast<double2*>(&krow[buf][16 * h + c]) = make_double2(reg[c], reg[c + 1]);
        if (h == 0) kf[buf] = f;
      }
      if (tid == 0) cand[buf].key = best.key, cand[buf].idx = best.idx;
      cluster_arrive();
    }
    // pivot kk's update of this thread's row, rotated by one column
    if (valid) {
      double s16[16];  // this half's 16 values of the scaled pivot row
#pragma unroll
      for (int c = 0; c < 16; c += 2) {
        const double2 v2 = *reinterpret_cast<const double2*>(&sp[16 * h + c]);
        s16[c] = v2.x;
        s16[c + 1] = v2.y;
      }
      const double snext = sp[h == 0 ? 16 : 0];  // the next half's first value
      if (i == k) {
#pragma unroll
        for (int c = 0; c < 15; ++c) reg[c] = s16[c + 1];
        reg[15] = snext;
      } else {
#pragma unroll
        for (int c = 0; c < 15; ++c) reg[c] = fma(-f, s16[c + 1], reg[c + 1]);
        reg[15] = h == 0 ? fma(-f, snext, other) : -f * snext;
      }
    }
    if (la) {
      cluster_wait();
      const int buf = (kk + 1) & 1, src = (lane + 1) & 31;
      GjCand w = gj_read_cand(rcand[0] + buf);
      double pre = rcrow[0][32 * buf + src];
#pragma unroll
      for (int s = 1; s < kGjCS; ++s) {
        const GjCand o = gj_read_cand(rcand[s] + buf);
        const double v = rcrow[s][32 * buf + src];
        if (gj_before(o.key, o.idx, w.key, w.idx)) w = o, pre = v;
      }
      const double kpre = cl.map_shared_rank(&krow[buf][0], ko)[src];
      const double kfk = *cl.map_shared_rank(&kf[buf], ko);
      if (++kro == R) kro = 0, ++ko;
      // pivot kk's update of element `lane` of the winner and of row k + 1
      const double spc = sp[src];
      const double u = src == 0 ? -w.f * spc : fma(-w.f, spc, pre);
      const double x = src == 0 ? -kfk * spc : fma(-kfk, spc, kpre);
      // u at lane 0 is the winner's updated pivot, the same multiply-add of the
      // same operands its owner made: the owner's inv is 0 exactly when it is unusable
      double inv = w.inv;
      if (inv == 0.0) bad = true;
      r = w.idx;
      if (r <= k || r >= m) r = k + 1, inv = 0.0, bad = true;  // never: the winner is an eligible row
      __syncwarp();
      sp[lane] = lane == 0 ? inv : u * inv;
      xr[lane] = x;
      if (tid == 0) piv_s[kk + 1] = r;
      __syncwarp();
    }
  }
  // the eliminated panel and the row slices of U (scale per row over its 32 values)
  uint32_t hmax = 0;
#pragma unroll
  for (int c = 0; c < 16; ++c) hmax = max(hmax, (uint32_t)(__double_as_longlong(reg[c]) >> 32) & 0x7fffffffu);
  hmax = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, 16));
  if (valid) {
#pragma unroll
    for (int c = 0; c < 16; c += 2)
      if (16 * h + c < kw)
        *reinterpret_cast<double2*>(M + (long long)i * m + k0 + 16 * h + c) = make_double2(reg[c], reg[c + 1]);
    const int e = scale_exponent(hmax);
    if (h == 0) Uexp[(long long)q * m + i] = e;
    __nv_bfloat16* u = Us + (long long)q * S * m * 32 + (long long)i * 32 + 16 * h;
#pragma unroll
    for (int c0 = 0; c0 < 16; c0 += 8) {
      uint32_t d[8][S];
#pragma unroll
      for (int uu = 0; uu < 8; ++uu) digits9((unsigned long long)__double_as_longlong(reg[c0 + uu]), e, d[uu]);
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        uint4 w;
        w.x = (d[0][sl] >> 16) | (d[1][sl] & 0xffff0000u);
        w.y = (d[2][sl] >> 16) | (d[3][sl] & 0xffff0000u);
        w.z = (d[4][sl] >> 16) | (d[5][sl] & 0xffff0000u);
        w.w = (d[6][sl] >> 16) | (d[7][sl] & 0xffff0000u);
        *reinterpret_cast<uint4*>(u + (long long)sl * m * 32 + c0) = w;
      }
    }
  }
  // net row permutation of the pivots: position x ends up holding row perm[x];
  // rank 0 also carries the inversion's column permutation (the exchanges of
  // every panel so far applied in pivot order, from the identity at panel 0):
  // column c of the final working matrix is column piv[c] of D^{-1}
  int* colp = piv + (long long)q * m;
  for (int c = tid; c < m; c += kGjThreads) {
    perm[c] = c;
    if (rank == 0) cperm[c] = panel == 0 ? c : colp[c];
  }
  __syncthreads();
  if (tid == 0)
    for (int kk = 0; kk < kw; ++kk) {
      const int a = k0 + kk, b = piv_s[kk];
      int tmp = perm[a];
      perm[a] = perm[b];
      perm[b] = tmp;
      if (rank == 0) {
        tmp = cperm[a];
        cperm[a] = cperm[b];
        cperm[b] = tmp;
      }
    }
  __syncthreads();
  if (rank == 0)
    for (int c = tid; c < m; c += kGjThreads) colp[c] = cperm[c];
  // a thread per column outside the panel (shared among the cluster's CTAs):
  // the column slices of V = the pivot rows (transposed: row j of the copy
  // holds V[0..31][j]; zero inside the panel), then the rows outside K that
  // took part in an exchange receive their rows of K (read before written:
  // the V loads come first, from this thread's own column)
  for (int jcol = tid * kGjCS + rank; jcol < m; jcol += kGjCS * kGjThreads) {
    const bool inK = jcol >= k0 && jcol < k0 + kw;
    double vv[32];
    uint32_t vmax = 0;
#pragma unroll
    for (int kk = 0; kk < 32; ++kk) {
      vv[kk] = (!inK && kk < kw) ? M[(long long)perm[k0 + kk] * m + jcol] : 0.0;
      vmax = max(vmax, (uint32_t)(__double_as_longlong(vv[kk]) >> 32) & 0x7fffffffu);
    }
    if (!inK)
      for (int kk = 0; kk < kw; ++kk) {
        const int x = piv_s[kk];
        if (x >= k0 + kw) M[(long long)x * m + jcol] = M[(long long)perm[x] * m + jcol];
      }
    const int e = scale_exponent(vmax);
    Vexp[(long long)q * m + jcol] = e;
    __nv_bfloat16* vdst = Vs + (long long)q * S * m * 32 + (long long)jcol * 32;
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 8) {
      uint32_t d[8][S];
#pragma unroll
      for (int uu = 0; uu < 8; ++uu) digits9((unsigned long long)__double_as_longlong(vv[c0 + uu]), e, d[uu]);
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        uint4 w;
        w.x = (d[0][sl] >> 16) | (d[1][sl] & 0xffff0000u);
        w.y = (d[2][sl] >> 16) | (d[3][sl] & 0xffff0000u);
        w.z = (d[4][sl] >> 16) | (d[5][sl] & 0xffff0000u);
        w.w = (d[6][sl] >> 16) | (d[7][sl] & 0xffff0000u);
        *reinterpret_cast<uint4*>(vdst + (long long)sl * m * 32 + c0) = w;
      }
    }
  }
  if (rank == 0 && tid == 0 && bad) atomicMin(status + p.sys, p.row0 + t + 1);
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// After the last panel: the column permutation undone and the row slices of
// the block inverse G_t written (the left operand of the next products), one
// pass: a CTA takes 32 rows of one block (blockIdx.x = block * groups +
// group), a warp a row at a time: the row is read once, scattered to its
// final column order in shared memory (its largest magnitude does not depend
// on the order), then written back as float64 and as nine digit slices.
__global__ void __launch_bounds__(256) k_gj_finish(const PartDesc* __restrict__ parts, int t, int m,
                                                   double* __restrict__ G, const int* __restrict__ piv,
                                                   __nv_bfloat16* __restrict__ Gs, int* __restrict__ eG) {
  __shared__ int ip[kMaxMTensor];
  __shared__ __align__(16) double rowb[8][kMaxMTensor];
  const int groups = (m + 31) / 32;
  const int q = blockIdx.x / groups, g = blockIdx.x - q * groups;
  const PartDesc p = parts[q];
  if (t >= p.L) return;
  const long long mm = (long long)m * m;
  double* M = G + p.blk + (long long)t * mm;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = threadIdx.x; c < m; c += blockDim.x) ip[c] = piv[(long long)q * m + c];
  __syncthreads();
  double* rb = rowb[warp];
  const int rend = min(m, 32 * g + 32);
  for (int r = 32 * g + warp; r < rend; r += 8) {
    uint32_t hmax = 0;
    for (int c = lane; c < m; c += 32) {
      const double v = M[(long long)r * m + c];
      rb[ip[c]] = v;
      hmax = max(hmax, (uint32_t)(__double_as_longlong(v) >> 32) & 0x7fffffffu);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) hmax = max(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    const int e = scale_exponent(hmax);
    if (lane == 0) eG[(long long)q * m + r] = e;
    __syncwarp();
    for (int c0 = lane * 8; c0 < m; c0 += 256) {  // m % 8 == 0
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; u += 2) {
        const double2 d2 = *reinterpret_cast<const double2*>(rb + c0 + u);
        v[u] = d2.x;
        v[u + 1] = d2.y;
        *reinterpret_cast<double2*>(M + (long long)r * m + c0 + u) = d2;
      }
      uint32_t d[8][S];
#pragma unroll
      for (int u = 0; u < 8; ++u) digits9((unsigned long long)__double_as_longlong(v[u]), e, d[u]);
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        uint4 w;
        w.x = (d[0][sl] >> 16) | (d[1][sl] & 0xffff0000u);
        w.y = (d[2][sl] >> 16) | (d[3][sl] & 0xffff0000u);
        w.z = (d[4][sl] >> 16) | (d[5][sl] & 0xffff0000u);
        w.w = (d[6][sl] >> 16) | (d[7][sl] & 0xffff0000u);
        *reinterpret_cast<uint4*>(Gs + ((long long)q * S + sl) * mm + (long long)r * m + c0) = w;
      }
    }
    __syncwarp();
  }
}

// Several per-subsystem slicing jobs in one launch (blockIdx.y = job).
__global__ void __launch_bounds__(256) k_oz_slice_jobs(const PartDesc* __restrict__ parts, int step, int m,
                                                       OzSliceJobs jobs) {
  __shared__ uint32_t red[8][32];
  __shared__ int s_e[32];
  __shared__ unsigned long long tile[32][33];
  const OzSliceJob& jb = jobs.job[blockIdx.y];
  const int groups = (m + 31) / 32;
  const int q = blockIdx.x / groups, g = blockIdx.x - q * groups;
  const PartDesc p = parts[q];
  const long long mm = (long long)m * m;
  const bool hl = (p.flags & HAS_LEFT) != 0, hr = (p.flags & HAS_RIGHT) != 0;
  int t = step;
  bool act;
  long long sblk, dq;
  switch (jb.kind) {
    case 0: act = t < p.L; sblk = p.blk / mm + t; dq = q; break;
    case 1: act = t < p.L - 1; sblk = p.blk / mm + t; dq = p.blk / mm + t; break;
    case 2: act = t < p.L - 1; sblk = p.blk / mm + t; dq = q; break;
    case 3: act = t < p.L && hl; sblk = p.blk / mm + t; dq = 2 * q + (t & 1); break;
    case 4: act = t == p.L - 1 && hr; sblk = p.blk / mm + t; dq = 2 * q + (t & 1); break;
    case 5: act = t < p.L - 1 && hl; sblk = q; dq = q; break;
    case 6: t = p.L - 2 - step; act = t >= 0 && hl; sblk = p.blk / mm + t; dq = 2 * q + (t & 1); break;
    case 7: t = p.L - 2 - step; act = t >= 0 && hr; sblk = p.blk / mm + t; dq = 2 * q + (t & 1); break;
    default: act = hl; sblk = p.blk / mm; dq = q; break;
  }
  // launch B's right operands (Acal_t^T, ZL_t^T before the last row) are
  // not needed when its products run in the banded kernel
  if (jobs.band && *jobs.band <= kBandMax && (jb.kind == 2 || (jb.kind == 3 && t < p.L - 1))) act = false;
  if (!act) return;
  __nv_bfloat16* dst = static_cast<__nv_bfloat16*>(jb.dst);
  if (jb.kind == 0 || jb.kind == 1)
    slice_rows_group(jb.src + sblk * mm, dst, dq, jb.exps, m, g);
  else
    slice_cols_group(jb.src + sblk * mm, dst, dq, jb.exps, m, g, red, s_e, tile);
}

// The assembly's operands per separator s (blockIdx.x = s * groups + group,
// blockIdx.y = job): job 0 C_q rows -> Cq slot s; jobs 1-4 the boundary
// spike blocks as columns -> S slot 4 s + job - 1: ZR^j[q-1], ZL^j[q-1] (only
// with HA), ZL^{j+1}[q+1], ZR^{j+1}[q+1] (only with HC).
__global__ void __launch_bounds__(256) k_oz_slice_seps(const SepDesc* __restrict__ seps, int m,
                                                       const double* __restrict__ C, const double* __restrict__ ZL,
                                                       const double* __restrict__ ZR, __nv_bfloat16* __restrict__ Cq,
                                                       int* __restrict__ eCq, __nv_bfloat16* __restrict__ Sp,
                                                       int* __restrict__ eS, const int* __restrict__ band) {
  __shared__ uint32_t red[8][32];
  __shared__ int s_e[32];
  __shared__ unsigned long long tile[32][33];
  if (band && *band <= kBandMax) return;  // the banded assembly needs no slices
  const int groups = (m + 31) / 32;
  const int s = blockIdx.x / groups, g = blockIdx.x - s * groups, job = blockIdx.y;
  const SepDesc sd = seps[s];
  if (job == 0) {
    slice_rows_group(C + sd.blk_q, Cq, s, eCq, m, g);
    return;
  }
  if ((job == 2 && !(sd.flags & HAS_HA)) || (job == 4 && !(sd.flags & HAS_HC))) return;
  const double* src = job == 1 ? ZR + sd.blk_prev : job == 2 ? ZL + sd.blk_prev : job == 3 ? ZL + sd.blk_next
                                                                                         : ZR + sd.blk_next;
  slice_cols_group(src, Sp, 4LL * s + job - 1, eS, m, g, red, s_e, tile);
}

// ---------------------------------------------------------------- banded operands
// When every A and C block of the level has its nonzeros within w <= kBandMax
// of the diagonal (detected by the input slicing), the products with A or C
// as an operand cost (2w + 1) multiply-adds per entry instead of m: these
// float64 kernels compute them over the band (the other terms are exact
// zeros), and the tensor-core tiles and slices for them are skipped.  A CTA
// takes 32 rows of one block (blockIdx.x = unit * groups + group); a warp a
// row at a time, a lane every 32nd column; the band of the banded operand in
// shared memory, the dense operand read along rows (coalesced).

// launch A's first product: X = G_t C_t (Acal_t, or the right spike ZR_{L-1})
__global__ void __launch_bounds__(256) k_band_gc(const PartDesc* __restrict__ parts, int t, int m,
                                                 const double* __restrict__ G, const double* __restrict__ C,
                                                 double* __restrict__ Acal, double* __restrict__ ZR,
                                                 const int* __restrict__ band) {
  __shared__ double bd[2 * kBandMax + 1][kMaxMTensor];  // bd[d + w][n] = C[n + d][n]
  const int w = *band;
  if (w > kBandMax) return;
  const int groups = (m + 31) / 32;
  const int q = blockIdx.x / groups, g = blockIdx.x - q * groups;
  const PartDesc p = parts[q];
  if (t >= p.L || (t == p.L - 1 && !(p.flags & HAS_RIGHT))) return;
  const long long mm = (long long)m * m, o = p.blk + (long long)t * mm;
  const double* Gt = G + o;
  const double* Ct = C + o;
  double* X = (t < p.L - 1 ? Acal : ZR) + o;
  for (int i = threadIdx.x; i < (2 * w + 1) * m; i += blockDim.x) {
    const int dd = i / m, n = i - dd * m, k = n + dd - w;
    bd[dd][n] = (k >= 0 && k < m) ? Ct[(long long)k * m + n] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 32 * g + warp; r < min(m, 32 * g + 32); r += 8)
    for (int n = lane; n < m; n += 32) {
      double acc = 0.0;
      for (int d = -w; d <= w; ++d) {
        const int k = n + d;
        if (k >= 0 && k < m) acc = fma(Gt[(long long)r * m + k], bd[d + w][n], acc);
      }
      X[(long long)r * m + n] = acc;
    }
}

// Row r of the banded left operand L times the dense X: sum_{k=r-w..r+w} L[r][k] X[k][n].
__device__ __forceinline__ double band_row(const double* lb, const double* __restrict__ X, int r, int n, int m,
                                           int w) {
  double acc = 0.0;
  for (int d = -w; d <= w; ++d) {
    const int k = r + d;
    if (k >= 0 && k < m) acc = fma(lb[d + w], X[(long long)k * m + n], acc);
  }
  return acc;
}

// The 32 rows' bands of L into lb[row][d + w] = L[r][r + d].
__device__ __forceinline__ void load_row_band(double (*lb)[2 * kBandMax + 1], const double* __restrict__ L, int g, int m,
                                              int w) {
  for (int i = threadIdx.x; i < 32 * (2 * w + 1); i += blockDim.x) {
    const int rl = i / (2 * w + 1), dd = i - rl * (2 * w + 1), r = 32 * g + rl, k = r + dd - w;
    lb[rl][dd] = (r < m && k >= 0 && k < m) ? L[(long long)r * m + k] : 0.0;
  }
}

// launch B: D_{t+1} = B_{t+1} - A_{t+1} Acal_t (blockIdx.y = 0) and
// Y_{t+1} = -A_{t+1} Bcal_t (= ZL_t, blockIdx.y = 1, with a left spike)
__global__ void __launch_bounds__(256) k_band_b(const PartDesc* __restrict__ parts, int t, int m,
                                                const double* __restrict__ A, const double* __restrict__ B,
                                                const double* __restrict__ Acal, const double* __restrict__ ZL,
                                                double* __restrict__ G, double* __restrict__ Y,
                                                const int* __restrict__ band) {
  __shared__ double lb[32][2 * kBandMax + 1];
  const int w = *band;
  if (w > kBandMax) return;
  const int groups = (m + 31) / 32;
  const int q = blockIdx.x / groups, g = blockIdx.x - q * groups, j = blockIdx.y;
  const PartDesc p = parts[q];
  if (t >= p.L - 1 || (j == 1 && !(p.flags & HAS_LEFT))) return;
  const long long mm = (long long)m * m, o = p.blk + (long long)t * mm;
  load_row_band(lb, A + o + mm, g, m, w);
  __syncthreads();
  const double* X = (j == 0 ? Acal : ZL) + o;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 32 * g + warp; r < min(m, 32 * g + 32); r += 8)
    for (int n = lane; n < m; n += 32) {
      const double v = band_row(lb[r - 32 * g], X, r, n, m, w);
      const long long e = (long long)r * m + n;
      if (j == 0)
        G[o + mm + e] = B[o + mm + e] - v;  // D_{t+1}
      else
        Y[(long long)q * mm + e] = -v;      // Y_{t+1}
    }
}

// the supplementary blocks (Eq. e2311): blockIdx.y = 0: HB = B_q - A_q ZR^j[q-1]
// - C_q ZL^{j+1}[q+1]; 1: HA = -A_q ZL^j[q-1]; 2: HC = -C_q ZR^{j+1}[q+1]
__global__ void __launch_bounds__(256) k_band_h(const SepDesc* __restrict__ seps, int m, const double* __restrict__ A,
                                                const double* __restrict__ B, const double* __restrict__ C,
                                                const double* __restrict__ ZL, const double* __restrict__ ZR,
                                                double* __restrict__ HA, double* __restrict__ HB,
                                                double* __restrict__ HC, const int* __restrict__ band) {
  __shared__ double ab[32][2 * kBandMax + 1], cb[32][2 * kBandMax + 1];
  const int w = *band;
  if (w > kBandMax) return;
  const int groups = (m + 31) / 32;
  const int s = blockIdx.x / groups, g = blockIdx.x - s * groups, j = blockIdx.y;
  const SepDesc sd = seps[s];
  if ((j == 1 && !(sd.flags & HAS_HA)) || (j == 2 && !(sd.flags & HAS_HC))) return;
  if (j != 2) load_row_band(ab, A + sd.blk_q, g, m, w);
  if (j != 1) load_row_band(cb, C + sd.blk_q, g, m, w);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 32 * g + warp; r < min(m, 32 * g + 32); r += 8)
    for (int n = lane; n < m; n += 32) {
      const int rl = r - 32 * g;
      const long long e = (long long)r * m + n;
      if (j == 0)
        HB[sd.hblk + e] = B[sd.blk_q + e] - (band_row(ab[rl], ZR + sd.blk_prev, r, n, m, w) +
                                             band_row(cb[rl], ZL + sd.blk_next, r, n, m, w));
      else if (j == 1)
        HA[sd.hblk + e] = -band_row(ab[rl], ZL + sd.blk_prev, r, n, m, w);
      else
        HC[sd.hblk + e] = -band_row(cb[rl], ZR + sd.blk_next, r, n, m, w);
    }
}

// The level's band: the largest |row - column| of a nonzero entry (any bit
// but the sign set) of the A and C blocks, folded into *band.  Read only.
__global__ void __launch_bounds__(256) k_band_detect(const double* __restrict__ A, const double* __restrict__ C,
                                                     long long n, int m, int* __restrict__ band) {
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(A);
  const unsigned long long* c = reinterpret_cast<const unsigned long long*>(C);
  int wmax = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    if (((a[e] | c[e]) << 1) != 0) {
      const int col = (int)(e % m), row = (int)((e / m) % m);
      wmax = max(wmax, abs(row - col));
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  if ((threadIdx.x & 31) == 0 && wmax > 0) atomicMax(band, wmax);
}

}  // namespace oz

// ---------------------------------------------------------------- host side
namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                              const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn oz_encoder() {
  static EncodeFn enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    enc = reinterpret_cast<EncodeFn>(fn);
  }
  return enc;
}
}  // namespace

bool oz_eligible(int m) { return m >= 8 && m <= kMaxMTensor && m % 8 == 0; }

int oz_slice_blocks_bytes(int m) { return oz::S * m * m * 2; }

// 4-D map [block][slice][row][column] of a slice array (rows x kdim per
// slice; kdim = m for the sweeps' blocks, 32 for the inversion's panels),
// box 32 x box_rows x 9 x 1.
bool oz_make_map(const void* base, long long blocks, int m, int box_rows, void* out, int kdim) {
  EncodeFn enc = oz_encoder();
  if (kdim <= 0) kdim = m;
  if (!enc || blocks <= 0 || !oz_eligible(m)) return false;
  cuuint64_t dims[4] = {(cuuint64_t)kdim, (cuuint64_t)m, (cuuint64_t)oz::S, (cuuint64_t)blocks};
  cuuint64_t strides[3] = {(cuuint64_t)kdim * 2, (cuuint64_t)m * kdim * 2, (cuuint64_t)oz::S * m * kdim * 2};
  cuuint32_t box[4] = {(cuuint32_t)oz::KS, (cuuint32_t)box_rows, (cuuint32_t)oz::S, 1u};
  cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  CUresult r = enc(static_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int oz_box_rows_left() { return oz::MT; }
int oz_box_rows_right() { return oz::NT; }
int oz_box_rows_gj() { return oz::NT3; }

void launch_band_detect(const double* A, const double* C, long long n, int m, int* band, cudaStream_t st) {
  if (n <= 0 || !band) return;
  oz::k_band_detect<<<152 * 8, 256, 0, st>>>(A, C, n, m, band);
}

void launch_oz_slice_all(bool cols, const double* src, int nblocks, int m, void* dst, int* exps, const int* band,
                         cudaStream_t st) {
  if (nblocks <= 0) return;
  const long long work = (long long)nblocks * ((m + 31) / 32);
  const int grid = (int)std::min<long long>(work, 152LL * 16);
  if (cols)
    oz::k_oz_slice_all<true><<<grid, 256, 0, st>>>(src, nblocks, m, static_cast<__nv_bfloat16*>(dst), exps, band);
  else
    oz::k_oz_slice_all<false><<<grid, 256, 0, st>>>(src, nblocks, m, static_cast<__nv_bfloat16*>(dst), exps, band);
}

void launch_oz_slice_jobs(const PartDesc* parts, int nparts, int step, int m, const OzSliceJobs& jobs, int njobs,
                          cudaStream_t st) {
  if (nparts <= 0 || njobs <= 0) return;
  oz::k_oz_slice_jobs<<<dim3(nparts * ((m + 31) / 32), njobs), 256, 0, st>>>(parts, step, m, jobs);
}

// The blocked Gauss-Jordan inversion of block row t of every active
// subsystem (in place in G; t = 0 starts from B_0), as four phases: the copy
// of B_0, per panel of 32 columns the panel and its trailing update, and the
// finishing pass (the column permutation undone, the row slices written).
void launch_gj_begin(const PartDesc* parts, int nparts, int t, int m, const double* B, double* G, cudaStream_t st) {
  if (nparts > 0 && t == 0) oz::k_gj_copy_b0<<<nparts, 256, 0, st>>>(parts, m, B, G);
}

void launch_gj_panel(const PartDesc* parts, int nparts, int t, int m, int pnl, double* G, int* piv, void* Us,
                     int* Uexp, void* Vs, int* Vexp, int* status, cudaStream_t st) {
  if (nparts <= 0) return;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nparts * oz::kGjCS);
  cfg.blockDim = dim3(oz::kGjThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = oz::kGjCS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, oz::k_gj_panel, parts, t, m, pnl, G, piv, static_cast<__nv_bfloat16*>(Us), Uexp,
                     static_cast<__nv_bfloat16*>(Vs), Vexp, status);
}

void launch_gj_update(const PartDesc* parts, int nparts, int t, int m, int pnl, double* G, const int* Uexp,
                      const int* Vexp, const void* maps2, int* errflag, cudaStream_t st) {
  if (nparts <= 0) return;
  OzOut out{nullptr, G, nullptr, nullptr, nullptr, nullptr};
  unsigned char maps3[3 * 128];
  std::memcpy(maps3, maps2, 2 * 128);
  std::memcpy(maps3 + 2 * 128, static_cast<const unsigned char*>(maps2) + 128, 128);
  launch_oz_step(3, parts, nparts, pnl, m, out, Uexp, Vexp, Vexp, maps3, errflag, st, t);
}

void launch_gj_finish(const PartDesc* parts, int nparts, int t, int m, double* G, const int* piv, void* Gs, int* eG,
                      cudaStream_t st) {
  if (nparts <= 0) return;
  oz::k_gj_finish<<<nparts * ((m + 31) / 32), 256, 0, st>>>(parts, t, m, G, piv, static_cast<__nv_bfloat16*>(Gs),
                                                             eG);
}

void launch_gj_inverse(const PartDesc* parts, int nparts, int t, int m, const double* B, double* G, int* piv,
                       void* Us, int* Uexp, void* Vs, int* Vexp, const void* maps2, int* status, int* errflag,
                       void* Gs, int* eG, cudaStream_t st) {
  if (nparts <= 0) return;
  launch_gj_begin(parts, nparts, t, m, B, G, st);
  for (int pnl = 0; pnl < (m + 31) / 32; ++pnl) {
    launch_gj_panel(parts, nparts, t, m, pnl, G, piv, Us, Uexp, Vs, Vexp, status, st);
    if (m > 32) launch_gj_update(parts, nparts, t, m, pnl, G, Uexp, Vexp, maps2, errflag, st);
  }
  launch_gj_finish(parts, nparts, t, m, G, piv, Gs, eG, st);
}

void launch_oz_step(int kind, const PartDesc* parts, int nparts, int step, int m, const OzOut& out, const int* lexp,
                    const int* rexp0, const int* rexp1, const void* maps3, int* errflag, cudaStream_t st, int aux) {
  if (nparts <= 0) return;
  OzMaps mp;
  std::memcpy(&mp, maps3, sizeof mp);
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 1;
  }
  // KIND 3: 32-column tiles without the one that is the panel itself
  const int ntm = (m + oz::MT - 1) / oz::MT,
            ntn = kind == 3 ? (m + oz::NT3 - 1) / oz::NT3 - 1 : (m + oz::NT - 1) / oz::NT;
  const int ntiles = nparts * (kind == 3 ? 1 : 2) * ntm * ntn;
  if (ntiles <= 0) return;
  const int grid = std::min(ntiles, nsm);
#define DM_OZ(KIND_)                                                                                              \
  do {                                                                                                           \
    static bool set = false;                                                                                     \
    if (!set) {                                                                                                  \
      cudaFuncSetAttribute(oz::k_oz_step<KIND_>, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::SMEM);        \
      set = true;                                                                                                \
    }                                                                                                            \
    oz::k_oz_step<KIND_><<<grid, oz::kThreads, oz::SMEM, st>>>(parts, step, aux, m, ntm, ntn, ntiles, out, lexp, \
                                                               rexp0, rexp1, errflag, mp);                       \
  } while (0)
  if (kind == 0) DM_OZ(0);
  else if (kind == 1) DM_OZ(1);
  else if (kind == 2) DM_OZ(2);
  else if (kind == 3) DM_OZ(3);
  else if (kind == 4) DM_OZ(4);
  else DM_OZ(5);
#undef DM_OZ
}

void launch_oz_assemble(const SepDesc* seps, int nseps, int m, const double* B, const double* C, const double* ZL,
                        const double* ZR, double* HA, double* HB, double* HC, const OzAsm& a, const int* eA,
                        const void* mapA, int* errflag, const int* band, cudaStream_t st) {
  if (nseps <= 0) return;
  oz::k_oz_slice_seps<<<dim3(nseps * ((m + 31) / 32), 5), 256, 0, st>>>(
      seps, m, C, ZL, ZR, static_cast<__nv_bfloat16*>(a.Cq), a.eCq, static_cast<__nv_bfloat16*>(a.S), a.eS, band);
  OzOut out{B, nullptr, nullptr, nullptr, nullptr, nullptr, seps, HA, HB, HC, band};
  unsigned char maps3[3 * 128];
  std::memcpy(maps3, mapA, 128);
  std::memcpy(maps3 + 128, a.maps[1], 128);
  std::memcpy(maps3 + 256, a.maps[1], 128);
  launch_oz_step(4, nullptr, nseps, 0, m, out, eA, a.eS, a.eS, maps3, errflag, st);
  std::memcpy(maps3, a.maps[0], 128);
  launch_oz_step(5, nullptr, nseps, 0, m, out, a.eCq, a.eS, a.eS, maps3, errflag, st);
}

void launch_band_gc(const PartDesc* parts, int nparts, int t, int m, const double* G, const double* C, double* Acal,
                    double* ZR, const int* band, cudaStream_t st) {
  if (nparts <= 0 || !band) return;
  oz::k_band_gc<<<nparts * ((m + 31) / 32), 256, 0, st>>>(parts, t, m, G, C, Acal, ZR, band);
}

void launch_band_b(const PartDesc* parts, int nparts, int t, int m, const double* A, const double* B,
                   const double* Acal, const double* ZL, double* G, double* Y, const int* band, cudaStream_t st) {
  if (nparts <= 0 || !band) return;
  oz::k_band_b<<<dim3(nparts * ((m + 31) / 32), 2), 256, 0, st>>>(parts, t, m, A, B, Acal, ZL, G, Y, band);
}

void launch_band_h(const SepDesc* seps, int nseps, int m, const double* A, const double* B, const double* C,
                   const double* ZL, const double* ZR, double* HA, double* HB, double* HC, const int* band,
                   cudaStream_t st) {
  if (nseps <= 0 || !band) return;
  oz::k_band_h<<<dim3(nseps * ((m + 31) / 32), 3), 256, 0, st>>>(seps, m, A, B, C, ZL, ZR, HA, HB, HC, band);
}

}  // namespace dm

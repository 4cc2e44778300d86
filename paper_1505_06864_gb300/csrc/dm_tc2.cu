// Factor sweeps of the mixed precisions on the tensor cores, one launch per
// product pair, both operands moved by TMA from copies in the tensor cores'
// layout.
//
// The products of step t of every subsystem (Section 3 applied to Eq. e231)
// come in pairs that share their left operand:
//
//   launch A (after the inversion G_t = D_t^{-1}):
//       Acal_t = G_t C_t            (at the last row with a right spike: ZR = G C)
//       Bcal_t = G_t Y_t            (left spike; Y_0 = A_first, Y_t = -A_t Bcal_{t-1})
//   launch B (t < L-1):
//       D_{t+1} = B_{t+1} - A_{t+1} Acal_t
//       Y_{t+1} = -A_{t+1} Bcal_t
//   backward step (row t = L-2-s):
//       ZL_t -= Acal_t ZL_{t+1},    ZR_t = -Acal_t ZR_{t+1}
//
// so each launch is, per subsystem, one m x m left operand times two m x m
// right operands.  A CTA computes one 128-row tile of one of the two products
// (N = m columns, m <= 256): a producer thread streams 32-wide K slabs of both
// operands by TMA (3-D tensor maps [block][row][column], zero fill past the
// block's edge) into a two-stage shared-memory ring, a second thread issues
// tcgen05.mma into a float32 accumulator in tensor memory, and all four warps
// then read the accumulator (tcgen05.ld) and write the results.
//
// Operand copies.  TF32 (mode 0): float32 values, the left operands read from
// the float32 factor arrays themselves.  Split bf16 (mode 1): every operand
// value v is stored as hi = bf16(v) and lo = bf16(v - hi) (the lo blocks
// `cap` blocks after the hi ones) and a product is hi*hi + hi*lo + lo*hi.
// Right operands are stored transposed (K-major: row n holds column n of the
// block), written by the epilogue that produces them (or, for C and Y_0, by a
// conversion at the start of the factorisation); per-subsystem values that
// are consumed by the next launch only live in small rolling buffers indexed
// by the subsystem's position (two slots, by row parity, for the spikes of
// the backward sweep).  Every wait is bounded; on expiry the kernel records
// an error flag, waits (bounded) for its own copies in flight, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "dm_internal.cuh"
#include "dm_tcgen05.cuh"

namespace dm {
namespace tc2 {
using namespace ptx;

constexpr int kThreads = 128;
constexpr int MT = 128;     // MMA M: rows per tile
constexpr int KS = 32;      // K elements per pipeline stage
constexpr int kStages = 2;
constexpr int kCols = 256;  // tensor-memory columns: N <= 256 float32 accumulators

template <int MODE>
struct Cfg {
  static constexpr int esz = MODE == 0 ? 4 : 2;
  static constexpr int parts = MODE == 0 ? 1 : 2;           // hi (+ lo)
  static constexpr int row = KS * esz;                      // bytes of one operand row in a stage
  static constexpr uint64_t layout = MODE == 0 ? 2 : 4;     // 128- / 64-byte swizzle
  static constexpr uint32_t sbo = 8 * row;                  // one 8-row swizzle atom
  static constexpr int kstep = MODE == 0 ? 8 : 16;          // K of one instruction
  static constexpr int nk = KS / kstep;
  static constexpr int lpart = MT * row;                    // left tile, one part
  static constexpr int rpart = 256 * row;                   // right tile, one part
  static constexpr int stage = parts * (lpart + rpart);     // 48 KB in both modes
  static constexpr int smem = 1024 + kStages * stage;
  static constexpr uint32_t fmt = MODE == 0 ? 2u : 1u;
};

// Store one value into an operand copy (element e of the hi part; the lo part
// `cap` elements further).
template <int MODE>
__device__ __forceinline__ void put(void* base, long long cap, long long e, float v) {
  if (MODE == 0) {
    static_cast<float*>(base)[e] = round_tf32(v);
  } else {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    static_cast<__nv_bfloat16*>(base)[e] = hi;
    static_cast<__nv_bfloat16*>(base)[e + cap] = lo;
  }
}

// Four consecutive values of one row into a row-major operand copy (the
// element offset is a multiple of 4).
template <int MODE>
__device__ __forceinline__ void put4(void* base, long long cap, long long e, const float (&v)[4]) {
  if (MODE == 0) {
    *reinterpret_cast<float4*>(static_cast<float*>(base) + e) =
        make_float4(round_tf32(v[0]), round_tf32(v[1]), round_tf32(v[2]), round_tf32(v[3]));
  } else {
    uint32_t hi[2], lo[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]), h1 = __float2bfloat16_rn(v[2 * q + 1]);
      const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
      const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
      hi[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      lo[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(base) + e) = make_uint2(hi[0], hi[1]);
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(base) + e + cap) = make_uint2(lo[0], lo[1]);
  }
}

// 16 bytes of consecutive elements (4 float32 or 8 bf16 hi + 8 bf16 lo) at
// element offset e, a multiple of 4 (float32) or 8 (bf16).
template <int MODE>
__device__ __forceinline__ void putT(void* base, long long cap, long long e, const float (&v)[MODE == 0 ? 4 : 8]) {
  if (MODE == 0) {
    *reinterpret_cast<float4*>(static_cast<float*>(base) + e) =
        make_float4(round_tf32(v[0]), round_tf32(v[1]), round_tf32(v[2]), round_tf32(v[3]));
  } else {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]), h1 = __float2bfloat16_rn(v[2 * q + 1]);
      const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
      const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
      hi[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      lo[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(base) + e) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(base) + e + cap) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

}  // namespace tc2

struct Tc2Maps {
  CUtensorMap L, R0, R1;
};

namespace tc2 {

// KIND 0: launch A, 1: launch B (both at forward step `step`), 2: backward
// step `step`.  blockIdx.y = subsystem, blockIdx.x = 2 * M-tile + product.
template <int MODE, int KIND>
__global__ void __launch_bounds__(kThreads) k_tc_step(const PartDesc* __restrict__ parts, int step, int m, int ntile,
                                                      int lo_l, int lo_r0, int lo_r1, Tc2Out out,
                                                      int* __restrict__ errflag, const __grid_constant__ Tc2Maps maps) {
  using Cf = Cfg<MODE>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t full[kStages], empty[kStages], accb;
  __shared__ uint32_t tmem_slot;
  __shared__ int err, nissued, ncons;
  const int pidx = blockIdx.y;
  const PartDesc p = parts[pidx];
  const int tm = blockIdx.x >> 1, j = blockIdx.x & 1;
  if (tm * MT >= m) return;
  int t;
  bool act;
  if (KIND == 0) {
    t = step;
    act = t < p.L && (j == 0 ? (t < p.L - 1 || (p.flags & HAS_RIGHT) != 0) : (p.flags & HAS_LEFT) != 0);
  } else if (KIND == 1) {
    t = step;
    act = t < p.L - 1 && (j == 0 || (p.flags & HAS_LEFT) != 0);
  } else {
    t = p.L - 2 - step;
    act = t >= 0 && (j == 0 ? (p.flags & HAS_LEFT) != 0 : (p.flags & HAS_RIGHT) != 0);
  }
  if (!act) return;
  const long long mm = (long long)m * m;
  const int b0 = (int)(p.blk / mm);
  int zl, zr;
  if (KIND == 0) {
    zl = MODE == 0 ? b0 + t : pidx;  // G_t: the float32 factor array / the converted rolling copy
    zr = j == 0 ? b0 + t : pidx;     // C_t^T (all blocks) / Y_t^T (rolling)
  } else if (KIND == 1) {
    zl = b0 + t + 1;                            // A_{t+1}
    zr = j == 0 ? pidx : 2 * pidx + (t & 1);    // Acal_t^T / Bcal_t^T
  } else {
    zl = b0 + t;                                // Acal_t
    zr = 2 * pidx + ((t + 1) & 1);              // ZL_{t+1}^T / ZR_{t+1}^T
  }
  const CUtensorMap* mr = j == 0 ? &maps.R0 : &maps.R1;
  const int lo_r = j == 0 ? lo_r0 : lo_r1;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accb, 1);
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
  const int nslab = (m + KS - 1) / KS;
  const uint32_t tx = (uint32_t)(Cf::parts * (MT + ntile) * Cf::row);

  // Lane 0 of warp 0 produces, lane 0 of warp 1 issues the MMAs; the other
  // lanes of those warps park at __syncwarp (no spinning beside them), warps
  // 2 and 3 wait for the accumulator.
  if (warp == 0 && lane == 0) {
    // producer: K slab s into stage s % 2 once the MMAs of slab s - 2 are done
    uint32_t ph[kStages] = {0u, 0u};
    int s = 0;
    for (; s < nslab; ++s) {
      const int st = s & 1;
      if (s >= kStages) {
        if (!mbar_wait(&empty[st], ph[st])) {
          err = 1;
          break;
        }
        ph[st] ^= 1u;
      }
      const uint32_t sb = smem_u32(base + st * Cf::stage);
      mbar_expect_tx(&full[st], tx);
      tma_load_3d(sb, &maps.L, s * KS, tm * MT, zl, &full[st]);
      if (MODE == 1) tma_load_3d(sb + Cf::lpart, &maps.L, s * KS, tm * MT, zl + lo_l, &full[st]);
      tma_load_3d(sb + Cf::parts * Cf::lpart, mr, s * KS, 0, zr, &full[st]);
      if (MODE == 1) tma_load_3d(sb + Cf::parts * Cf::lpart + Cf::rpart, mr, s * KS, 0, zr + lo_r, &full[st]);
    }
    nissued = s;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = make_idesc(Cf::fmt, MT, ntile);
    int s = 0;
    for (; s < nslab; ++s) {
      const int st = s & 1;
      if (!mbar_wait(&full[st], (uint32_t)((s >> 1) & 1))) {
        err = 1;
        break;
      }
      tc_fence_after();
      const uint32_t la = smem_u32(base + st * Cf::stage), ll = la + Cf::lpart;
      const uint32_t ra = la + Cf::parts * Cf::lpart, rl = ra + Cf::rpart;
#pragma unroll
      for (int k = 0; k < Cf::nk; ++k) {
        const uint32_t off = (uint32_t)(k * Cf::kstep * Cf::esz);
        const uint64_t ad = kmajor_desc(la + off, Cf::sbo, Cf::layout);
        const uint64_t bd = kmajor_desc(ra + off, Cf::sbo, Cf::layout);
        mma<Cf::fmt>(tmem, ad, bd, idesc, (s | k) ? 1u : 0u);
        if (MODE == 1) {
          mma<Cf::fmt>(tmem, ad, kmajor_desc(rl + off, Cf::sbo, Cf::layout), idesc, 1u);
          mma<Cf::fmt>(tmem, kmajor_desc(ll + off, Cf::sbo, Cf::layout), bd, idesc, 1u);
        }
      }
      mma_commit(&empty[st]);
    }
    ncons = s;
    mma_commit(&accb);
  }
  if (warp < 2) __syncwarp();
  bool ok = mbar_wait(&accb, 0u);
  tc_fence_after();
  ok = __syncthreads_and(ok) && !err;

  if (ok) {
    // Epilogue in chunks of 32 columns.  Each thread holds one row of the
    // chunk (tensor-memory lane = row); transposed copies are written straight
    // from there (consecutive lanes = consecutive addresses), row-major
    // results go through a per-warp 32 x 33 tile in the (now idle) pipeline
    // buffers so that a warp writes 128 contiguous bytes of one row at a time.
    float* stg = reinterpret_cast<float*>(base) + warp * (32 * 33);
    const int rbase = tm * MT + warp * 32, row = rbase + lane;
    const bool rok = row < m;
    const long long o = p.blk + (long long)t * mm;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    // which outputs this tile has
    const bool acal = KIND == 0 && j == 0 && t < p.L - 1;          // Acal_t (+ row-major copy + transposed)
    const bool spike0 = KIND == 0 && !acal;                        // ZR seed (j = 0) or Bcal_t (j = 1)
    void* tr = nullptr;                                            // transposed copy
    long long tcap = 0, tz = 0;
    float sgn = 1.f;
    if (acal) tr = out.acalT, tcap = out.cap_acalT, tz = pidx;
    else if (spike0) tr = j == 0 ? out.zrT : out.zlT, tcap = j == 0 ? out.cap_zrT : out.cap_zlT, tz = 2 * pidx + (t & 1);
    else if (KIND == 1 && j == 1) tr = out.yT, tcap = out.cap_yT, tz = pidx, sgn = -1.f;
    else if (KIND == 2) tr = j == 0 ? out.zlT : out.zrT, tcap = j == 0 ? out.cap_zlT : out.cap_zrT,
                        tz = 2 * pidx + (t & 1), sgn = -1.f;
    float* rm = nullptr;  // row-major float32 result (KIND 1, j = 0 writes D_{t+1} into G instead)
    if (acal) rm = out.Acal;
    else if (spike0) rm = j == 0 ? out.ZR : out.ZL;
    else if (KIND == 2) rm = j == 0 ? out.ZL : out.ZR;
    const bool rmw = KIND == 2 && j == 0;  // ZL_t -= ...: the transposed copy needs the updated value
    for (int c0 = 0; c0 < ntile; c0 += 32) {
      {
        float v[32];
        float h[16];
        tmem_ld16(tl + (uint32_t)c0, h);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = h[i];
        if (c0 + 16 < ntile) {
          tmem_ld16(tl + (uint32_t)(c0 + 16), h);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[16 + i] = h[i];
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[16 + i] = 0.f;
        }
        if (c0 >= m) continue;
#pragma unroll
        for (int i = 0; i < 32; ++i) stg[lane * 33 + i] = v[i];
      }
      __syncwarp();
      // row-major results: lane = (row r0 + 4 i, columns cq .. cq + 3), float4
      // accesses (m % 8 == 0: a group of four columns is all inside or all out)
      const bool dnext = KIND == 1 && j == 0;  // D_{t+1} = B_{t+1} - A_{t+1} Acal_t into G
      if (rm || dnext) {
        const int r0 = lane >> 3, cq = (lane & 7) * 4, cc = c0 + cq;
        float4 in[8];
        if (dnext || rmw) {
          const float* src = KIND == 1 ? out.B32 + mm : rm;  // B_{t+1} / the forward ZL_t
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int rr = rbase + r0 + 4 * i;
            in[i] = (rr < m && cc < m) ? *reinterpret_cast<const float4*>(src + o + (long long)rr * m + cc)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = r0 + 4 * i, rr = rbase + r;
          if (rr >= m || cc >= m) continue;
          float* sp = stg + r * 33 + cq;
          float4 a = make_float4(sp[0], sp[1], sp[2], sp[3]);
          const long long e = (long long)rr * m + cc;
          if (dnext) {
            *reinterpret_cast<float4*>(out.G + o + mm + e) = make_float4(in[i].x - a.x, in[i].y - a.y, in[i].z - a.z,
                                                                        in[i].w - a.w);
          } else if (rmw) {
            a = make_float4(in[i].x - a.x, in[i].y - a.y, in[i].z - a.z, in[i].w - a.w);
            *reinterpret_cast<float4*>(rm + o + e) = a;
            sp[0] = a.x, sp[1] = a.y, sp[2] = a.z, sp[3] = a.w;
          } else {
            if (KIND == 2) a = make_float4(-a.x, -a.y, -a.z, -a.w);
            *reinterpret_cast<float4*>(rm + o + e) = a;
            if (acal && MODE == 1) {
              const float f4[4] = {a.x, a.y, a.z, a.w};
              put4<MODE>(out.acal_l, out.cap_acal_l * mm, (long long)(b0 + t) * mm + e, f4);
            }
          }
        }
        __syncwarp();
      }
      // transposed copies: lane = (column, a group of rows), 16-byte stores of
      // consecutive rows of one column (8 bf16 / 4 float32)
      if (tr) {
        constexpr int RG = MODE == 0 ? 4 : 8;      // rows per lane
        constexpr int LPC = 32 / RG;               // lanes per column
        constexpr int CPI = 32 / LPC;              // columns per pass
        const long long cap = tcap * mm, zb = tz * mm;
        const int g = (lane % LPC) * RG, cl = lane / LPC;
        const float sg = rmw ? 1.f : sgn;
#pragma unroll
        for (int q = 0; q < 32 / CPI; ++q) {
          const int c = q * CPI + cl, rr = rbase + g;
          if (c0 + c >= m || rr >= m) continue;
          float f[RG];
#pragma unroll
          for (int k = 0; k < RG; ++k) f[k] = sg * stg[(g + k) * 33 + c];
          putT<MODE>(tr, cap, zb + (long long)(c0 + c) * m + rr, f);
        }
      }
      __syncwarp();  // the staging tile is free for the next chunk
    }
  }
  // copies still in flight after an expired wait land before the CTA leaves
  if (threadIdx.x == 0)
    for (int s = ncons; s < nissued; ++s) mbar_wait(&full[s & 1], (uint32_t)((s >> 1) & 1));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kCols);
  if (threadIdx.x == 0 && !ok && errflag) atomicExch(errflag, 1);
}

// Operand copies from float64 (or float32) blocks, 32 x 32 tiles through
// shared memory so that transposed writes stay coalesced.  Block q (blockIdx.z
// and every gridDim.z-th after it, q < nq) is written to destination block q;
// its source is block q of `src`, or (by subsystem) the block of row t of
// subsystem q -- for the transposed Y_0 copy only subsystems with a left spike.
template <int MODE, typename TS, bool TRANS, bool BY_PART>
__global__ void __launch_bounds__(256) k_to_operand(const TS* __restrict__ src, const PartDesc* __restrict__ parts,
                                                    int nq, int t, int m, void* __restrict__ dst, long long cap_blocks) {
  __shared__ float tile[32][33];
  const long long mm = (long long)m * m;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int q = blockIdx.z; q < nq; q += gridDim.z) {
    long long sblk = q;
    if (BY_PART) {
      const PartDesc p = parts[q];
      if (t >= p.L || (TRANS && !(p.flags & HAS_LEFT))) continue;
      sblk = p.blk / mm + t;
    }
    __syncthreads();  // the previous block's reads of `tile` are done
    for (int k = ty; k < 32; k += 8) {
      const int r = r0 + k, c = c0 + tx;
      tile[k][tx] = (r < m && c < m) ? (float)src[sblk * mm + (long long)r * m + c] : 0.f;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
      // destination row dr, column dc (transposed: dst[c][r] = src[r][c])
      const int dr = (TRANS ? c0 : r0) + k, dc = (TRANS ? r0 : c0) + tx;
      if (dr < m && dc < m)
        put<MODE>(dst, cap_blocks * mm, (long long)q * mm + (long long)dr * m + dc, TRANS ? tile[tx][k] : tile[k][tx]);
    }
  }
}

}  // namespace tc2

// ---------------------------------------------------------------- host side
namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                              const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encoder() {
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

template <typename K>
void raise_smem(K kernel, int bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}
}  // namespace

bool tc2_eligible(int m) { return m >= 8 && m <= 256 && m % 8 == 0; }

int tc2_ntile(int m) { return (m + 15) / 16 * 16; }

// A 3-D map [blocks][m][m] of an operand copy (element type by mode), box
// 32 (K) x box_rows, swizzle matching the kernel's stage rows.
bool tc2_make_map(int mode, const void* base, long long blocks, int m, int box_rows, void* out) {
  EncodeFn enc = encoder();
  if (!enc || blocks <= 0 || !tc2_eligible(m)) return false;
  const int esz = mode == 0 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)m, (cuuint64_t)m, (cuuint64_t)blocks};
  cuuint64_t strides[2] = {(cuuint64_t)m * esz, (cuuint64_t)m * m * esz};
  cuuint32_t box[3] = {(cuuint32_t)tc2::KS, (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(static_cast<CUtensorMap*>(out), mode == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   mode == 0 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int tc2_map_bytes() { return (int)sizeof(CUtensorMap); }

// Conversions: all blocks of a level (A or C^T), or the block of row t of
// every subsystem (G_t, or A_first^T into the Y rolling buffer).
void launch_tc2_convert(int mode, const double* src64, const float* src32, const PartDesc* parts, int nq, int t, int m,
                        bool trans, void* dst, long long cap_blocks, cudaStream_t st) {
  if (nq <= 0) return;
  const dim3 grid((m + 31) / 32, (m + 31) / 32, std::min(nq, 65535));
  const bool bp = parts != nullptr;
#define DM_CVT(MODE_, TS_, SRC_)                                                                                      \
  do {                                                                                                                \
    if (trans) {                                                                                                      \
      if (bp) tc2::k_to_operand<MODE_, TS_, true, true><<<grid, 256, 0, st>>>(SRC_, parts, nq, t, m, dst, cap_blocks); \
      else tc2::k_to_operand<MODE_, TS_, true, false><<<grid, 256, 0, st>>>(SRC_, parts, nq, t, m, dst, cap_blocks);  \
    } else {                                                                                                          \
      if (bp) tc2::k_to_operand<MODE_, TS_, false, true><<<grid, 256, 0, st>>>(SRC_, parts, nq, t, m, dst, cap_blocks); \
      else tc2::k_to_operand<MODE_, TS_, false, false><<<grid, 256, 0, st>>>(SRC_, parts, nq, t, m, dst, cap_blocks); \
    }                                                                                                                 \
  } while (0)
  if (src64) {
    if (mode == 0) DM_CVT(0, double, src64);
    else DM_CVT(1, double, src64);
  } else {
    if (mode == 0) DM_CVT(0, float, src32);
    else DM_CVT(1, float, src32);
  }
#undef DM_CVT
}

// One launch of the step kernel: kind 0 / 1 (forward step t), 2 (backward step s).
void launch_tc2_step(int mode, int kind, const PartDesc* parts, int nparts, int step, int m, const int lo[3],
                     const Tc2Out& out, const void* maps3, int* errflag, cudaStream_t st) {
  if (nparts <= 0) return;
  Tc2Maps mp;
  std::memcpy(&mp, maps3, sizeof mp);
  const dim3 grid(2 * ((m + tc2::MT - 1) / tc2::MT), nparts);
  const int nt = tc2_ntile(m);
#define DM_STEP(MODE_, KIND_)                                                                                     \
  do {                                                                                                            \
    static bool set = false;                                                                                      \
    if (!set) {                                                                                                   \
      raise_smem(tc2::k_tc_step<MODE_, KIND_>, tc2::Cfg<MODE_>::smem);                                           \
      set = true;                                                                                                 \
    }                                                                                                             \
    tc2::k_tc_step<MODE_, KIND_><<<grid, tc2::kThreads, tc2::Cfg<MODE_>::smem, st>>>(parts, step, m, nt, lo[0],   \
                                                                                    lo[1], lo[2], out, errflag, mp); \
  } while (0)
  if (mode == 0) {
    if (kind == 0) DM_STEP(0, 0);
    else if (kind == 1) DM_STEP(0, 1);
    else DM_STEP(0, 2);
  } else {
    if (kind == 0) DM_STEP(1, 0);
    else if (kind == 1) DM_STEP(1, 1);
    else DM_STEP(1, 2);
  }
#undef DM_STEP
}

}  // namespace dm

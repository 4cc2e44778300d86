// Block products of the mixed-precision factor sweeps on the 5th-generation
// tensor cores (tcgen05, sm_103a).
//
// The sweeps' m x m x m products (Acal_t = G_t C_t, the next Schur block
// D_{t+1} = B_{t+1} - A_{t+1} Acal_t, the left spike G_t (-A_t Bcal_{t-1}),
// and the spike back-sweeps; Section 3 applied to Eq. e231) are computed in
// m x 64 output panels, one CTA of 128 threads per panel:
//
//   * the left operand (an m x m block, float64 or float32 in global memory)
//     streams through shared memory in K-slabs of one 128-byte swizzle atom,
//     converted to TF32 (DM_TF32) or split into bf16 hi + lo parts
//     (DM_BF16X3), double-buffered so that the loads of slab s+1 overlap the
//     MMAs of slab s;
//   * the right operand (the m x 64 panel) is held transposed (K-major) in
//     shared memory for the whole K;
//   * one thread issues tcgen05.mma (M = 128 rows per tile, N = 64, K = 8 for
//     TF32 / 16 for bf16) into a float32 accumulator in tensor memory and
//     commits to an mbarrier; DM_BF16X3 issues hi*hi + hi*lo + lo*hi;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
//     lanes 32w..32w+31 = rows of the tile) and either writes the result to
//     global memory or stages it, transposed, as the next product's right
//     operand (the chain Acal_t -> D_{t+1} stays in one CTA).
//
// Shared-memory operand layout: canonical K-major, 128-byte swizzle: rows of
// 128 bytes, 8-row atoms of 1024 bytes (stride-byte-offset 1024), the 16-byte
// chunk index XOR-ed with the row index within the atom.  Every wait on an
// mbarrier is bounded; on expiry the kernel records an error flag, stops
// issuing, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>

#include "dm_internal.cuh"
#include "dm_slices.cuh"

namespace dm {
namespace tc {

constexpr int kThreads = 128;
constexpr int NP = 64;          // panel width = MMA N
constexpr int MT = 128;         // MMA M (rows per tile)
constexpr int kMaxTiles = 2;    // m <= 256
constexpr uint32_t kWaitLimit = 1u << 26;

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One full warp: allocate `ncols` TMEM columns, address written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// K-major, 128-byte swizzle shared-memory matrix descriptor.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8-row atoms of 1024 bytes
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // SWIZZLE_128B
  return d;
}

// Instruction descriptor: float32 accumulate, K-major A and B, M x N.
// fmt: 2 = TF32 (kind::tf32), 1 = BF16 (kind::f16).
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (MODE == 0) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive float32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}

// byte offset of (row, byte-in-row kb) inside a K-major SW128 tile
__device__ __forceinline__ uint32_t sw128_off(int row, int kb) {
  const int chunk = kb >> 4;
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + (((chunk ^ (row & 7)) & 7) << 4) + (kb & 15));
}

// ---------------------------------------------------------------- operand staging
// Element size in shared memory and K elements per 128-byte atom.
template <int MODE>
struct Fmt {
  static constexpr int esz = MODE == 0 ? 4 : 2;
  static constexpr int katom = 128 / esz;   // 32 (tf32) or 64 (bf16)
  static constexpr int kstep = MODE == 0 ? 8 : 16;
  static constexpr int parts = MODE == 0 ? 1 : 2;  // hi (+ lo)
};

// Store value v at (row, k) of an operand whose K-slabs are `slab_bytes`
// apart (k = slab * katom + kk); part 0 = TF32 / bf16 hi, part 1 = bf16 lo
// at `lo_off` bytes further.
template <int MODE>
__device__ __forceinline__ void put(uint8_t* base, int slab_bytes, int lo_off, int row, int k, float v) {
  constexpr int KA = Fmt<MODE>::katom;
  const int s = k / KA, kk = k - s * KA;
  uint8_t* p = base + (size_t)s * slab_bytes;
  if (MODE == 0) {
    *reinterpret_cast<float*>(p + sw128_off(row, kk * 4)) = to_tf32(v);
  } else {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    *reinterpret_cast<__nv_bfloat16*>(p + sw128_off(row, kk * 2)) = hi;
    *reinterpret_cast<__nv_bfloat16*>(p + lo_off + sw128_off(row, kk * 2)) = lo;
  }
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// TMA: the byte count the next phase of `bar` waits for, and one 2-D tile
// load (box 32 x 128 float32 = one M-tile of one K-slab, 128-byte swizzle)
// that completes on `bar`.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Left-operand K-slab `slab` of the m x m row-major float32 block L (rows
// padded to MT * tiles, columns past m zero) into buffer `dst` (M-tile t at
// t * tile_bytes).  TF32 with m % 4 == 0: 16-byte cp.async copies straight
// into their swizzled chunks (the tensor core reads the float32 bits as TF32),
// asynchronous -- the caller waits.  Otherwise: 4-wide vector loads, TF32
// rounding or the bf16 hi/lo split in registers, stores to shared memory.
template <int MODE>
__device__ __forceinline__ void stage_left(uint8_t* dst, const float* __restrict__ L, int m, int slab, int tiles,
                                           int tile_bytes, int lo_off) {
  constexpr int KA = Fmt<MODE>::katom;
  const int k0 = slab * KA;
  const int rows = tiles * MT;
  const bool vec = (m & 3) == 0 && (reinterpret_cast<uintptr_t>(L) & 15) == 0;
  if (MODE == 0 && vec) {
    for (int e = threadIdx.x; e < rows * (KA / 4); e += kThreads) {
      const int r = e / (KA / 4), c = e - r * (KA / 4), k = k0 + 4 * c;
      const bool ok = r < m && k < m;
      const float* src = ok ? L + (long long)r * m + k : L;
      cp_async16(smem_u32(dst + (r / MT) * tile_bytes + sw128_off(r % MT, c * 16)), src, ok ? 16u : 0u);
    }
    cp_commit();
    return;
  }
  if (MODE == 1 && vec) {
    // 8 consecutive k per item: two float4 loads, one 16-byte chunk of bf16 hi
    // and one of bf16 lo (whole-chunk shared stores, no bank conflicts within
    // a row); U items per thread in flight.
    constexpr int U = 4;
    const int n8 = rows * (KA / 8);
    for (int e0 = threadIdx.x; e0 < n8; e0 += U * kThreads) {
      float4 v0[U], v1[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * kThreads;
        const int r = e / (KA / 8), k = k0 + 8 * (e - r * (KA / 8));
        const bool ok = e < n8 && r < m && k < m;
        const float* src = L + (long long)r * m + k;
        v0[u] = ok ? *reinterpret_cast<const float4*>(src) : make_float4(0.f, 0.f, 0.f, 0.f);
        v1[u] = ok ? *reinterpret_cast<const float4*>(src + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * kThreads;
        if (e >= n8) break;
        const int r = e / (KA / 8), c = e - r * (KA / 8);
        const float f[8] = {v0[u].x, v0[u].y, v0[u].z, v0[u].w, v1[u].x, v1[u].y, v1[u].z, v1[u].w};
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const __nv_bfloat16 h0 = __float2bfloat16_rn(f[2 * q]), h1 = __float2bfloat16_rn(f[2 * q + 1]);
          const __nv_bfloat16 l0 = __float2bfloat16_rn(f[2 * q] - __bfloat162float(h0));
          const __nv_bfloat16 l1 = __float2bfloat16_rn(f[2 * q + 1] - __bfloat162float(h1));
          hi[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
          lo[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        uint8_t* t = dst + (r / MT) * tile_bytes + sw128_off(r % MT, c * 16);
        *reinterpret_cast<uint4*>(t) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(t + lo_off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
    return;
  }
  if (vec) {
    constexpr int U = 4;  // independent vector loads in flight per thread
    const int n4 = rows * (KA / 4);
    for (int e0 = threadIdx.x; e0 < n4; e0 += U * kThreads) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * kThreads;
        const int r = e / (KA / 4), k = k0 + 4 * (e - r * (KA / 4));
        v[u] = (e < n4 && r < m && k < m) ? *reinterpret_cast<const float4*>(L + (long long)r * m + k)
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * kThreads;
        if (e >= n4) break;
        const int r = e / (KA / 4), kk = 4 * (e - r * (KA / 4));
        uint8_t* t = dst + (r / MT) * tile_bytes;
        put<MODE>(t, 0, lo_off, r % MT, kk + 0, v[u].x);
        put<MODE>(t, 0, lo_off, r % MT, kk + 1, v[u].y);
        put<MODE>(t, 0, lo_off, r % MT, kk + 2, v[u].z);
        put<MODE>(t, 0, lo_off, r % MT, kk + 3, v[u].w);
      }
    }
    return;
  }
  for (int e = threadIdx.x; e < rows * KA; e += kThreads) {
    const int r = e / KA, kk = e - r * KA, k = k0 + kk;
    const float v = (r < m && k < m) ? L[(long long)r * m + k] : 0.f;
    put<MODE>(dst + (r / MT) * tile_bytes, 0, lo_off, r % MT, kk, v);
  }
}

// Right operand: the m x NP panel R[k][c0 + n] (row stride ld, columns past
// `cols` zero, scaled by `sc`) stored transposed: row n, K index k.  A thread
// builds whole 16-byte chunks (4 TF32 values, or 8 bf16 hi + 8 bf16 lo) from
// coalesced reads of consecutive columns n across the warp.
template <int MODE, typename TR>
__device__ __forceinline__ void stage_right(uint8_t* dst, int slab_bytes, int lo_off, const TR* __restrict__ R,
                                            int m, int ld, int c0, int cols, float sc) {
  constexpr int KA = Fmt<MODE>::katom;
  constexpr int G = MODE == 0 ? 4 : 8;  // K values per 16-byte chunk
  constexpr int U = 4;                  // chunks per thread with their loads in flight together
  const int kpad = ((m + KA - 1) / KA) * KA;
  const int items = (kpad / G) * NP;
  for (int e0 = threadIdx.x; e0 < items; e0 += U * kThreads) {
    float v[U][G];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kThreads;
      const int kg = e / NP, n = e - kg * NP, k0 = kg * G;
      const bool col_ok = e < items && c0 + n < cols;
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int k = k0 + i;
        v[u][i] = (col_ok && k < m) ? sc * (float)R[(long long)k * ld + c0 + n] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kThreads;
      if (e >= items) break;
      const int kg = e / NP, n = e - kg * NP, k0 = kg * G;
      const int slab = k0 / KA, kk = k0 - slab * KA;
      uint8_t* p = dst + (size_t)slab * slab_bytes + sw128_off(n, kk * Fmt<MODE>::esz);
      if (MODE == 0) {
        *reinterpret_cast<uint4*>(p) =
            make_uint4(__float_as_uint(to_tf32(v[u][0])), __float_as_uint(to_tf32(v[u][1])),
                       __float_as_uint(to_tf32(v[u][2])), __float_as_uint(to_tf32(v[u][3])));
      } else {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const __nv_bfloat16 h0 = __float2bfloat16_rn(v[u][2 * q]), h1 = __float2bfloat16_rn(v[u][2 * q + 1]);
          const __nv_bfloat16 l0 = __float2bfloat16_rn(v[u][2 * q] - __bfloat162float(h0));
          const __nv_bfloat16 l1 = __float2bfloat16_rn(v[u][2 * q + 1] - __bfloat162float(h1));
          hi[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
          lo[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        *reinterpret_cast<uint4*>(p) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(p + lo_off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
  }
}

// Shared-memory plan of a CTA (bytes), m <= 256.
template <int MODE>
struct Smem {
  static constexpr int KA = Fmt<MODE>::katom;
  static constexpr int P = Fmt<MODE>::parts;
  static constexpr int tile_bytes = MT * 128 * P;     // one M-tile of one left K-slab (hi [+ lo])
  static constexpr int left_lo = MT * 128;            // lo part offset inside a tile
  static constexpr int lbuf_bytes = kMaxTiles * tile_bytes;
  static constexpr int rslab_bytes = NP * 128 * P;    // one K-slab of the right panel (hi [+ lo])
  static constexpr int right_lo = NP * 128;
  static constexpr int nslabs_max = 256 / KA;
  static constexpr int right_bytes = nslabs_max * rslab_bytes;
  static constexpr int total = 1024 /*align*/ + 2 * lbuf_bytes + right_bytes + 64;
};

// acc(TMEM) = L (m x m, float32) * Rpanel (K-major in `right`).  L's K-slabs
// stream through the two left buffers: slab s+1 is staged while the MMAs of
// slab s run.  `ph` tracks the two mbarriers' phases.  Returns false if a
// wait expired.
template <int MODE>
__device__ bool product(const float* __restrict__ L, int m, int tiles, uint8_t* lbuf0, uint8_t* right,
                        uint64_t* bars, uint32_t (&ph)[2], uint32_t tmem, bool elect, const CUtensorMap* tm,
                        long long row0, uint64_t* lbars, uint32_t (&lph)[2], int lbuf_bytes) {
  using S = Smem<MODE>;
  constexpr int KA = Fmt<MODE>::katom;
  constexpr int KS = Fmt<MODE>::kstep;
  constexpr uint32_t idesc = make_idesc(MODE == 0 ? 2u : 1u, MT, NP);
  const int nslab = (m + KA - 1) / KA;
  const bool tma = (MODE == 0) && tm != nullptr;
  bool ok = true;
  // stage K-slab `slab` of L into left buffer `buf`: TMA tiles (rows of the
  // next block row past m only feed output rows that are never stored;
  // columns past m are zero-filled) or cp.async / register copies
  auto stage = [&](int slab, int buf) {
    uint8_t* dstb = lbuf0 + buf * lbuf_bytes;
    if (tma) {
      if (elect) {
        mbar_expect_tx(&lbars[buf], (uint32_t)(tiles * MT * 128));
        for (int t = 0; t < tiles; ++t)
          tma_load_2d(smem_u32(dstb + t * S::tile_bytes), tm, slab * KA, (int)(row0 + t * MT), &lbars[buf]);
      }
    } else {
      stage_left<MODE>(dstb, L, m, slab, tiles, S::tile_bytes, S::left_lo);
    }
  };
  stage(0, 0);
  for (int s = 0; s < nslab; ++s) {
    const int b = s & 1;
    uint8_t* lb = lbuf0 + b * lbuf_bytes;
    if (tma) {
      if (!mbar_wait(&lbars[b], lph[b])) ok = false;
      lph[b] ^= 1u;
    } else {
      cp_wait_all();  // slab s (if it was copied asynchronously) has landed
      fence_async_shared();
    }
    if (!__syncthreads_and(ok)) return false;
    tc_fence_after();
    if (elect) {
      for (int t = 0; t < tiles; ++t) {
        const uint32_t dt = tmem + (uint32_t)(t * NP);
        const uint32_t la = smem_u32(lb + t * S::tile_bytes);
        const uint32_t ra = smem_u32(right + s * S::rslab_bytes);
        for (int j = 0; j < KA / KS; ++j) {
          const uint32_t kb = (uint32_t)(j * KS * Fmt<MODE>::esz);
          const uint64_t ad = sw128_desc(la + kb), bd = sw128_desc(ra + kb);
          const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
          mma<MODE>(dt, ad, bd, idesc, acc);
          if (MODE == 1) {
            const uint64_t bl = sw128_desc(ra + S::right_lo + kb);
            const uint64_t al = sw128_desc(la + S::left_lo + kb);
            mma<MODE>(dt, ad, bl, idesc, 1u);
            mma<MODE>(dt, al, bd, idesc, 1u);
          }
        }
      }
      mma_commit(&bars[b]);
    }
    if (s + 1 < nslab) {
      const int nb = (s + 1) & 1;
      if (s + 1 >= 2) {  // the MMAs of slab s-1 read buffer nb
        if (!mbar_wait(&bars[nb], ph[nb])) ok = false;
        ph[nb] ^= 1u;
      }
      stage(s + 1, nb);
    }
  }
  // drain: wait for the last one or two commits
  for (int s = (nslab >= 2 ? nslab - 2 : 0); s < nslab; ++s) {
    const int b = s & 1;
    if (!mbar_wait(&bars[b], ph[b])) ok = false;
    ph[b] ^= 1u;
  }
  tc_fence_after();
  return __syncthreads_and(ok);
}

// Epilogue: f(row, col, value) for every (row < m, col < NP) of the tiles' accumulators.
template <typename F>
__device__ __forceinline__ void drain_acc(uint32_t tmem, int tiles, int m, F&& f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = 0; t < tiles; ++t) {
    const int row = t * MT + warp * 32 + lane;
#pragma unroll
    for (int c = 0; c < NP; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * NP + c), v);
      if (row < m) {
#pragma unroll
        for (int i = 0; i < 16; ++i) f(row, c + i, v[i]);
      }
    }
  }
}

struct TcState {
  uint64_t bars[2];   // MMA completion per left buffer
  uint64_t lbars[2];  // TMA completion per left buffer
  uint32_t tmem;
  int err;
};

// Tensor maps of a level's float32 arrays (one 2-D view [rows][m] each).
struct TmaMaps {
  CUtensorMap G, A, Acal;
};

// Two left buffers of `lbuf_bytes` (the launch's M-tiles), then the right panel.
__device__ __forceinline__ uint8_t* carve(uint8_t* raw, uint8_t** lbuf, uint8_t** right, int lbuf_bytes) {
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  *lbuf = base;
  *right = base + 2 * lbuf_bytes;
  return base;
}

__device__ __forceinline__ void tc_setup(TcState* st, int ncols) {
  if (threadIdx.x < 32) tmem_alloc(&st->tmem, (uint32_t)ncols);
  if (threadIdx.x == 0) {
    mbar_init(&st->bars[0], 1);
    mbar_init(&st->bars[1], 1);
    mbar_init(&st->lbars[0], 1);
    mbar_init(&st->lbars[1], 1);
    st->err = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void tc_teardown(TcState* st, int ncols, int* errflag) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(st->tmem, (uint32_t)ncols);
  if (threadIdx.x == 0 && st->err && errflag) atomicExch(errflag, 1);
}

__device__ __forceinline__ int tmem_cols(int tiles) {
  const int need = tiles * NP;
  return need <= 32 ? 32 : (need <= 64 ? 64 : (need <= 128 ? 128 : 256));
}

// ---------------------------------------------------------------- kernels
// Forward factor step t, tile types as in the SIMT kernel:
//   0: Acal_t[:, J] = G_t C_t[:, J]; D_{t+1}[:, J] = B_{t+1}[:, J] - A_{t+1} Acal_t[:, J]
//      (last row with a right spike: ZR_t[:, J] = G_t C_t[:, J])
//   1: left spike: Bcal_t[:, J] = G_t A_first[:, J] (t = 0) or G_t (-A_t Bcal_{t-1}[:, J])
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_fwd_factor_tc(const PartDesc* __restrict__ parts, int t, int tiles_n,
                                                            int type_lo, const float* __restrict__ A,
                                                            const float* __restrict__ B,
                                                            const float* __restrict__ C, float* __restrict__ G,
                                                            float* __restrict__ Acal, float* __restrict__ ZL,
                                                            float* __restrict__ ZR, int* __restrict__ errflag,
                                                            const __grid_constant__ TmaMaps tmaps, int use_tma,
                                                            int cap_tiles) {
  using S = Smem<MODE>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ TcState st;
  const PartDesc p = parts[blockIdx.y];
  if (t >= p.L) return;
  const int m = p.m;
  const int tb = blockIdx.x / tiles_n, type = type_lo + tb, c0 = (blockIdx.x - tb * tiles_n) * NP;
  if (c0 >= m) return;
  const bool last = (t == p.L - 1);
  if (type == 0 && last && !(p.flags & HAS_RIGHT)) return;
  if (type == 1 && !(p.flags & HAS_LEFT)) return;
  uint8_t *lbuf, *right;
  const int lbuf_bytes = cap_tiles * S::tile_bytes;
  carve(smem_raw, &lbuf, &right, lbuf_bytes);
  const int tiles = (m + MT - 1) / MT;
  const int ncols = tmem_cols(tiles);
  tc_setup(&st, ncols);
  uint32_t ph[2] = {0u, 0u}, lph[2] = {0u, 0u};
  const bool elect = threadIdx.x == 0;
  const long long mm = (long long)m * m;
  const long long o = p.blk + (long long)t * mm;
  const CUtensorMap* tG = use_tma ? &tmaps.G : nullptr;
  const CUtensorMap* tA = use_tma ? &tmaps.A : nullptr;
  bool ok = true;
  if (type == 0) {
    stage_right<MODE, float>(right, S::rslab_bytes, S::right_lo, C + o, m, m, c0, m, 1.f);
    fence_async_shared();
    __syncthreads();
    ok = product<MODE>(G + o, m, tiles, lbuf, right, st.bars, ph, st.tmem, elect, tG, o / m, st.lbars, lph, lbuf_bytes);
    if (ok) {
      float* dst = last ? ZR + o : Acal + o;
      // result to global, and (not last) transposed into `right` for the next product
      drain_acc(st.tmem, tiles, m, [&](int row, int col, float v) {
        if (c0 + col < m) dst[(long long)row * m + c0 + col] = v;
      });
      if (!last) {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        drain_acc(st.tmem, tiles, m, [&](int row, int col, float v) {
          put<MODE>(right, S::rslab_bytes, S::right_lo, col, row, c0 + col < m ? v : 0.f);
        });
        fence_async_shared();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        ok = product<MODE>(A + o + mm, m, tiles, lbuf, right, st.bars, ph, st.tmem, elect, tA, (o + mm) / m,
                           st.lbars, lph, lbuf_bytes);
        if (ok) {
          const float* Bn = B + o + mm;
          float* Dn = G + o + mm;
          drain_acc(st.tmem, tiles, m, [&](int row, int col, float v) {
            if (c0 + col < m) {
              const long long e = (long long)row * m + c0 + col;
              Dn[e] = Bn[e] - v;
            }
          });
        }
      }
    }
  } else {
    if (t == 0) {
      stage_right<MODE, float>(right, S::rslab_bytes, S::right_lo, A + o, m, m, c0, m, 1.f);
    } else {
      stage_right<MODE, float>(right, S::rslab_bytes, S::right_lo, ZL + o - mm, m, m, c0, m, 1.f);
      fence_async_shared();
      __syncthreads();
      ok = product<MODE>(A + o, m, tiles, lbuf, right, st.bars, ph, st.tmem, elect, tA, o / m, st.lbars, lph, lbuf_bytes);
      if (ok) {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        drain_acc(st.tmem, tiles, m, [&](int row, int col, float v) {
          put<MODE>(right, S::rslab_bytes, S::right_lo, col, row, c0 + col < m ? -v : 0.f);
        });
      }
    }
    fence_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (ok) ok = product<MODE>(G + o, m, tiles, lbuf, right, st.bars, ph, st.tmem, elect, tG, o / m, st.lbars, lph, lbuf_bytes);
    if (ok) {
      float* dst = ZL + o;
      drain_acc(st.tmem, tiles, m, [&](int row, int col, float v) {
        if (c0 + col < m) dst[(long long)row * m + c0 + col] = v;
      });
    }
  }
  if (!ok && threadIdx.x == 0) st.err = 1;
  tc_teardown(&st, ncols, errflag);
}

// Backward factor step s, row t = L-2-s:  0: ZL_t -= Acal_t ZL_{t+1};  1: ZR_t = -Acal_t ZR_{t+1}.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_back_factor_tc(const PartDesc* __restrict__ parts, int s, int tiles_n,
                                                             const float* __restrict__ Acal, float* __restrict__ ZL,
                                                             float* __restrict__ ZR, int* __restrict__ errflag,
                                                             const __grid_constant__ TmaMaps tmaps, int use_tma,
                                                             int cap_tiles) {
  using S = Smem<MODE>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ TcState st;
  const PartDesc p = parts[blockIdx.y];
  const int t = p.L - 2 - s;
  if (t < 0) return;
  const int m = p.m;
  const int type = blockIdx.x / tiles_n, c0 = (blockIdx.x - type * tiles_n) * NP;
  if (c0 >= m) return;
  if (type == 0 && !(p.flags & HAS_LEFT)) return;
  if (type == 1 && !(p.flags & HAS_RIGHT)) return;
  uint8_t *lbuf, *right;
  const int lbuf_bytes = cap_tiles * S::tile_bytes;
  carve(smem_raw, &lbuf, &right, lbuf_bytes);
  const int tiles = (m + MT - 1) / MT;
  const int ncols = tmem_cols(tiles);
  tc_setup(&st, ncols);
  uint32_t ph[2] = {0u, 0u}, lph[2] = {0u, 0u};
  const long long mm = (long long)m * m;
  const long long o = p.blk + (long long)t * mm;
  float* Y = (type == 0 ? ZL : ZR) + o;
  stage_right<MODE, float>(right, S::rslab_bytes, S::right_lo, Y + mm, m, m, c0, m, 1.f);
  fence_async_shared();
  __syncthreads();
  bool ok = product<MODE>(Acal + o, m, tiles, lbuf, right, st.bars, ph, st.tmem, threadIdx.x == 0,
                         use_tma ? &tmaps.Acal : nullptr, o / m, st.lbars, lph, lbuf_bytes);
  if (ok) {
    const bool keep = (type == 0);
    drain_acc(st.tmem, tiles, m, [&](int row, int col, float v) {
      if (c0 + col < m) {
        const long long e = (long long)row * m + c0 + col;
        Y[e] = (keep ? Y[e] : 0.f) - v;
      }
    });
  }
  if (!ok && threadIdx.x == 0) st.err = 1;
  tc_teardown(&st, ncols, errflag);
}

// ---------------------------------------------------------------- sliced residual
// r = b - T x with float64 accuracy on the bf16 tensor cores (an exact
// splitting in the manner of Ozaki's error-free matrix products).  Block
// row i of a system is L = [A_i B_i C_i] (m x 3m) times X = [x_{i-1}; x_i;
// x_{i+1}] (3m x r).  Every row of L is scaled by 2^-e (e: the exponent of
// the row's largest magnitude) and every column of X by 2^-f, and each
// scaled value y in (-1, 1) is cut into nine base-64 digits read straight
// from its float64 bits: y = sign * sum_s d_s 2^(-6s) + (truncation below
// 2^-54), d_s in [0, 63] -- integers, exact in bf16.  Then
//   L X = 2^(e+f) sum_d 2^(-6d) acc_d,   acc_d = sum_{s+t=d} Lslice_s Xslice_t,
// keeping the pairs with s + t <= 11.  Each acc_d sums at most 9 slice
// products over K <= 384 terms of magnitude <= 63^2, so every partial sum is
// an integer below 2^24 and the float32 accumulation in tensor memory is
// exact; the ten acc_d are combined in float64.  The error per entry is
// below K * 2^-50 * max|L_row| * max|X_col| (digit truncation and the
// dropped pairs), within the float64 dot product's own bound.
//
// One CTA per block row (m <= 128, r <= 16), 256 threads.  K runs in chunks
// of 64: the CTA slices the chunk of L (128 x 64, nine slices, K-major
// 128-byte-swizzled bf16) and of X (16 x 64, nine slices + one zero slice,
// stored consecutively so that slices t = 1..T form one N = 16 T operand),
// then one thread issues per 16-wide K step nine MMAs: L slice s against X
// slices 1..T_s (T_1 = 10 with the zero slice, which initialises all ten
// accumulators; T_s = min(9, 11 - s) after), into the accumulators
// d = s+1 .. s+T_s (TMEM columns (d - 2) * 16).
constexpr int kRsThreads = 256;

constexpr int kRsNB = 16;                    // right-hand-side columns per tile
constexpr int kRsAcc = 10;                   // accumulators d = 2 .. 11
constexpr int kRsMaxM = 128;
struct RsSmem {
  static constexpr int a_slice = MT * 128;              // 128 rows x 64 bf16
  static constexpr int b_slice = kRsNB * 128;           // 16 columns x 64 bf16
  static constexpr int a_bytes = kRsSlices * a_slice;
  static constexpr int b_bytes = (kRsSlices + 1) * b_slice;
  static constexpr int total = 1024 + a_bytes + b_bytes;
};

__device__ __forceinline__ int rs_find_sys(const SysDesc* __restrict__ sys, int nsys, int row) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sys[mid].row0 <= row) lo = mid; else hi = mid - 1;
  }
  return lo;
}


__device__ __forceinline__ uint32_t abs_hi(unsigned long long bits) { return (uint32_t)(bits >> 32) & 0x7fffffffu; }

// two bf16 patterns (high halves of a, b) in one word: a low, b high
__device__ __forceinline__ uint32_t pack_bf16x2(uint32_t a, uint32_t b) { return (a >> 16) | (b & 0xffff0000u); }

// Largest high word (sign cleared) of every point row of [A_i B_i C_i] of the
// sliced systems: a warp per point row, one CTA per block row.
__global__ void __launch_bounds__(kRsThreads) k_row_scales(const SysDesc* __restrict__ sys, int nsys,
                                                           const double* __restrict__ A,
                                                           const double* __restrict__ B,
                                                           const double* __restrict__ C, unsigned* __restrict__ rowhi) {
  const int si = rs_find_sys(sys, nsys, blockIdx.x);
  const SysDesc sd = sys[si];
  if (!sd.sliced) return;
  const int i = blockIdx.x - sd.row0, m = sd.m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long o = sd.blk + (long long)i * m * m;
  const bool hasA = i > 0, hasC = i < sd.N - 1;
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(A + o);
  const unsigned long long* bb = reinterpret_cast<const unsigned long long*>(B + o);
  const unsigned long long* c = reinterpret_cast<const unsigned long long*>(C + o);
  for (int rr = warp; rr < m; rr += kRsThreads / 32) {
    uint32_t mx = 0;
    for (int k = lane; k < m; k += 32) {
      const long long e = (long long)rr * m + k;
      mx = max(mx, abs_hi(__ldg(bb + e)));
      if (hasA) mx = max(mx, abs_hi(__ldg(a + e)));
      if (hasC) mx = max(mx, abs_hi(__ldg(c + e)));
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) rowhi[sd.eoff + (long long)i * m + rr] = mx;
  }
}

// Largest high word of every column of every block x_i of the sliced systems
// ([global block row][16]): a warp per block row, lane = column + 16 * parity
// of the point row.
__global__ void __launch_bounds__(kRsThreads) k_col_scales(const SysDesc* __restrict__ sys, int nsys, int nrows,
                                                           const double* __restrict__ x, unsigned* __restrict__ colhi) {
  const int row = blockIdx.x * (kRsThreads / 32) + (threadIdx.x >> 5);
  if (row >= nrows) return;
  const int lane = threadIdx.x & 31;
  const SysDesc sd = sys[rs_find_sys(sys, nsys, row)];
  if (!sd.sliced) return;
  const int i = row - sd.row0, m = sd.m, r = sd.r;
  const int c = lane & 15, par = lane >> 4;
  const unsigned long long* xi = reinterpret_cast<const unsigned long long*>(x + sd.vec + (long long)i * m * r);
  uint32_t mx = 0;
  if (c < r)
    for (int k = par; k < m; k += 2) mx = max(mx, abs_hi(__ldg(xi + (long long)k * r + c)));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
  if (lane < 16) colhi[(long long)row * kRsNB + c] = mx;
}

__global__ void __launch_bounds__(kRsThreads, 1) k_residual_sliced(const SysDesc* __restrict__ sys, int nsys,
                                                                   const double* __restrict__ A,
                                                                   const double* __restrict__ B,
                                                                   const double* __restrict__ C,
                                                                   const double* __restrict__ x,
                                                                   const double* __restrict__ b,
                                                                   double* __restrict__ rout,
                                                                   double* __restrict__ nrm,
                                                                   const unsigned* __restrict__ rowhi,
                                                                   const unsigned* __restrict__ colhi,
                                                                   int* __restrict__ errflag) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ TcState st;
  __shared__ int s_erow[kRsMaxM];
  __shared__ int s_fcol[kRsNB];
  __shared__ double red[2 * kRsNB];
  const int si = rs_find_sys(sys, nsys, blockIdx.x);
  const SysDesc sd = sys[si];
  if (!sd.sliced) return;  // the float64 kernel handles this system
  const int i = blockIdx.x - sd.row0, m = sd.m, r = sd.r;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* As = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* Bs = As + RsSmem::a_bytes;
  const long long mm = (long long)m * m, mr = (long long)m * r;
  const bool hasA = i > 0, hasC = i < sd.N - 1;
  const unsigned long long* xbits = reinterpret_cast<const unsigned long long*>(x);
  // the K chunks: (block j, first column k0) over the blocks present
  const int nck = (m + 63) / 64;
  const int j0 = hasA ? 0 : 1, j1 = hasC ? 3 : 2;
  const int nchunks = (j1 - j0) * nck;
  auto chunk_src = [&](int q, int* j, int* k0) {
    *j = j0 + q / nck;
    *k0 = (q % nck) * 64;
  };
  auto lrow = [&](int j) {
    const double* base = j == 0 ? A : (j == 1 ? B : C);
    return reinterpret_cast<const unsigned long long*>(base + sd.blk + i * mm);
  };
  constexpr int IT = MT * 8 / kRsThreads;  // 8-wide groups of L per thread per chunk
  unsigned long long raw[IT][8];
  auto load_chunk = [&](int q) {
    int j, k0;
    chunk_src(q, &j, &k0);
    const unsigned long long* L = lrow(j);
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int e = tid + it * kRsThreads;
      const int rr = e >> 3, k = k0 + 8 * (e & 7);
#pragma unroll
      for (int u = 0; u < 8; ++u) raw[it][u] = (rr < m && k + u < m) ? __ldg(L + (long long)rr * m + k + u) : 0ull;
    }
  };
  load_chunk(0);  // in flight during the set-up below
  tc_setup(&st, 256);
  for (int rr = tid; rr < m; rr += kRsThreads) s_erow[rr] = scale_exponent(rowhi[sd.eoff + (long long)i * m + rr]);
  if (tid < kRsNB) {
    const long long g = (long long)blockIdx.x * kRsNB + tid;
    uint32_t h = colhi[g];
    if (hasA) h = max(h, colhi[g - kRsNB]);
    if (hasC) h = max(h, colhi[g + kRsNB]);
    s_fcol[tid] = scale_exponent(h);
  }
  if (tid < 2 * kRsNB) red[tid] = 0.0;
  for (int e = tid; e < RsSmem::b_slice / 16; e += kRsThreads)  // the zero slice after the nine X slices
    *reinterpret_cast<uint4*>(Bs + kRsSlices * RsSmem::b_slice + 16 * e) = make_uint4(0u, 0u, 0u, 0u);
  // rows m .. 127 of the L slices: zero for every chunk
  for (int e = tid; e < (MT - m) * 8 * kRsSlices; e += kRsThreads) {
    const int sl = e / ((MT - m) * 8), rem = e - sl * (MT - m) * 8;
    *reinterpret_cast<uint4*>(As + sl * RsSmem::a_slice + sw128_off(m + (rem >> 3), 16 * (rem & 7))) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  __syncthreads();

  uint32_t ph = 0;
  bool ok = true;
  for (int q = 0; q < nchunks; ++q) {
    int j, k0;
    chunk_src(q, &j, &k0);
    if (q > 0) {  // the previous chunk's MMAs have read shared memory
      if (!mbar_wait(&st.bars[0], ph)) ok = false;
      ph ^= 1u;
    }
    // L chunk (already in registers): nine digit slices; rows past m stay
    // as zeroed on entry, groups wholly past m are stored as zeros
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int e = tid + it * kRsThreads;
      const int rr = e >> 3, g8 = e & 7;
      if (rr >= m) continue;
      if (k0 + 8 * g8 >= m) {
#pragma unroll
        for (int sl = 0; sl < kRsSlices; ++sl)
          *reinterpret_cast<uint4*>(As + sl * RsSmem::a_slice + sw128_off(rr, 16 * g8)) = make_uint4(0u, 0u, 0u, 0u);
        continue;
      }
      const int er = s_erow[rr];
      uint32_t qv[8][kRsSlices];
#pragma unroll
      for (int u = 0; u < 8; ++u) digits9(raw[it][u], er, qv[u]);
#pragma unroll
      for (int sl = 0; sl < kRsSlices; ++sl)
        *reinterpret_cast<uint4*>(As + sl * RsSmem::a_slice + sw128_off(rr, 16 * g8)) =
            make_uint4(pack_bf16x2(qv[0][sl], qv[1][sl]), pack_bf16x2(qv[2][sl], qv[3][sl]),
                       pack_bf16x2(qv[4][sl], qv[5][sl]), pack_bf16x2(qv[6][sl], qv[7][sl]));
    }
    // X chunk: 16 columns x 8 groups of 8 consecutive K
    if (tid < kRsNB * 8) {
      const int c = tid >> 3, g8 = tid & 7, k = k0 + 8 * g8;
      const int fc = s_fcol[c];
      const long long xo = sd.vec + (long long)(i - 1 + j) * mr;
      uint32_t qv[8][kRsSlices];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        digits9((c < r && k + u < m) ? __ldg(xbits + xo + (long long)(k + u) * r + c) : 0ull, fc, qv[u]);
#pragma unroll
      for (int sl = 0; sl < kRsSlices; ++sl)
        *reinterpret_cast<uint4*>(Bs + sl * RsSmem::b_slice + sw128_off(c, 16 * g8)) =
            make_uint4(pack_bf16x2(qv[0][sl], qv[1][sl]), pack_bf16x2(qv[2][sl], qv[3][sl]),
                       pack_bf16x2(qv[4][sl], qv[5][sl]), pack_bf16x2(qv[6][sl], qv[7][sl]));
    }
    fence_async_shared();
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    tc_fence_after();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t kb = (uint32_t)(ks * 32);
        const uint64_t bd = sw128_desc(smem_u32(Bs) + kb);
#pragma unroll
        for (int sl = 0; sl < kRsSlices; ++sl) {
          const int T = sl == 0 ? kRsSlices + 1 : min(kRsSlices, 10 - sl);
          const uint64_t ad = sw128_desc(smem_u32(As + sl * RsSmem::a_slice) + kb);
          const uint32_t acc = (q == 0 && ks == 0 && sl == 0) ? 0u : 1u;
          const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((16 * T) >> 3) << 17) |
                                 ((uint32_t)(MT >> 4) << 24);
          mma<1>(st.tmem + (uint32_t)(sl * kRsNB), ad, bd, idesc, acc);
        }
      }
      mma_commit(&st.bars[0]);
    }
    if (q + 1 < nchunks) load_chunk(q + 1);  // next chunk's loads overlap these MMAs
  }
  if (nchunks > 0 && ok) {
    if (!mbar_wait(&st.bars[0], ph)) ok = false;
    ph ^= 1u;
  }
  tc_fence_after();
  ok = __syncthreads_and(ok);
  // epilogue: warps 0-3 own TMEM lanes 0-127 = rows
  const double* bi = b + sd.vec + i * mr;
  double* ri = rout + sd.vec + i * mr;
  if (warp < 4 && ok) {
    const int row = warp * 32 + lane;
    // sum_d acc_d 2^(-6d) from the exact integer accumulators: d = 2..6 and
    // d = 7..11 combined in two 64-bit integers (each below 2^49), then one
    // float64 fused multiply-add
    long long ih[kRsNB], il[kRsNB];
    uint32_t nan_cols = 0;  // a NaN digit (NaN or infinite input) reached the column
#pragma unroll
    for (int c = 0; c < kRsNB; ++c) ih[c] = il[c] = 0;
#pragma unroll
    for (int dd = 0; dd < kRsAcc; ++dd) {
      float v[16];
      tmem_ld16(st.tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(dd * kRsNB), v);
#pragma unroll
      for (int c = 0; c < kRsNB; ++c) {
        if (v[c] != v[c]) nan_cols |= 1u << c;
        const long long a = (long long)__float2int_rn(v[c]);
        if (dd < 5)
          ih[c] += a * (1ll << (6 * (4 - dd)));
        else
          il[c] += a * (1ll << (6 * (9 - dd)));
      }
    }
    double sum[kRsNB];
#pragma unroll
    for (int c = 0; c < kRsNB; ++c)
      sum[c] = ((nan_cols >> c) & 1u) ? __longlong_as_double(0x7ff8000000000000ll)
                                      : fma((double)il[c], 0x1p-66, (double)ih[c] * 0x1p-36);
    if (row < m) {
      const int er = s_erow[row];
#pragma unroll
      for (int c = 0; c < kRsNB; ++c)
        if (c < r) {
          const long long e = (long long)row * r + c;
          const double bb = bi[e];
          const double rv = bb - ldexp(sum[c], er + s_fcol[c]);
          ri[e] = rv;
          atomicAdd(&red[c], rv * rv);
          atomicAdd(&red[kRsNB + c], bb * bb);
        }
    }
  }
  __syncthreads();
  if (tid < r && ok) {
    atomicAdd(&nrm[(long long)si * 4 * kMaxR + tid], red[tid]);
    atomicAdd(&nrm[(long long)si * 4 * kMaxR + kMaxR + tid], red[kRsNB + tid]);
  }
  if (!ok && tid == 0) st.err = 1;
  tc_teardown(&st, 256, errflag);
}

// ---------------------------------------------------------------- throughput probe
// Peak tcgen05 throughput of one SM: one thread issues `iters` x 4
// back-to-back MMAs (M = 128, N = 256, one 128-byte K atom each: K = 32
// TF32 / 64 bf16 per 4 instructions) from zeroed shared-memory operands into
// one float32 accumulator, then commits and waits (bounded).  Launched with
// one CTA per SM; flops = 2 * 128 * 256 * K per instruction.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_mma_probe(int iters, int* __restrict__ errflag) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ TcState st;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int a_bytes = MT * 128, b_bytes = 256 * 128;
  for (int i = threadIdx.x; i < (a_bytes + b_bytes) / 16; i += kThreads)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
  fence_async_shared();
  tc_setup(&st, 256);
  if (threadIdx.x == 0) {
    constexpr uint32_t idesc = make_idesc(MODE == 0 ? 2u : 1u, MT, 256);
    const uint32_t a = smem_u32(base), b = a + a_bytes;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        mma<MODE>(st.tmem, sw128_desc(a + 32 * j), sw128_desc(b + 32 * j), idesc, (i | j) ? 1u : 0u);
    }
    mma_commit(&st.bars[0]);
    if (!mbar_wait(&st.bars[0], 0)) st.err = 1;
  }
  tc_teardown(&st, 256, errflag);
}

}  // namespace tc

// ---------------------------------------------------------------- launchers
namespace {
template <typename K>
void raise_smem_once(K kernel, int bytes, bool* done) {
  if (!*done) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    // the largest shared-memory carve-out, so that launches sized below the
    // maximum fit several CTAs per SM
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    *done = true;
  }
}
bool g_set_fwd[2], g_set_back[2];

// Shared memory of one launch: the left buffers for its M-tiles and the right
// panel for its K-slabs (blocks up to max_m), so that blocks of m <= 128 fit
// two CTAs per SM.
template <int MODE>
int tc_launch_smem(int max_m, int* cap_tiles) {
  using S = tc::Smem<MODE>;
  *cap_tiles = (max_m + tc::MT - 1) / tc::MT;
  const int nsl = (max_m + S::KA - 1) / S::KA;
  return 1024 + 2 * *cap_tiles * S::tile_bytes + nsl * S::rslab_bytes + 64;
}
}  // namespace

void launch_fwd_factor_tc(int mode, const PartDesc* parts, int nparts, int t, int max_m, const float* A,
                          const float* B, const float* C, float* G, float* Acal, float* ZL, float* ZR,
                          int* errflag, cudaStream_t st, int type_lo, int type_hi, const void* tmaps) {
  if (nparts <= 0 || type_hi <= type_lo) return;
  tc::TmaMaps tm;
  std::memset(&tm, 0, sizeof tm);
  if (tmaps) std::memcpy(&tm, tmaps, sizeof tm);
  const int use_tma = (tmaps != nullptr && mode == 0) ? 1 : 0;
  const int tiles_n = (max_m + tc::NP - 1) / tc::NP;
  const dim3 grid((type_hi - type_lo) * tiles_n, nparts);
  int cap = 0;
  if (mode == 0) {
    const int bytes = tc_launch_smem<0>(max_m, &cap);
    raise_smem_once(tc::k_fwd_factor_tc<0>, tc::Smem<0>::total, &g_set_fwd[0]);
    tc::k_fwd_factor_tc<0><<<grid, tc::kThreads, bytes, st>>>(parts, t, tiles_n, type_lo, A, B, C, G, Acal, ZL, ZR,
                                                              errflag, tm, use_tma, cap);
  } else {
    const int bytes = tc_launch_smem<1>(max_m, &cap);
    raise_smem_once(tc::k_fwd_factor_tc<1>, tc::Smem<1>::total, &g_set_fwd[1]);
    tc::k_fwd_factor_tc<1><<<grid, tc::kThreads, bytes, st>>>(parts, t, tiles_n, type_lo, A, B, C, G, Acal, ZL, ZR,
                                                              errflag, tm, 0, cap);
  }
}

void launch_back_factor_tc(int mode, const PartDesc* parts, int nparts, int s, int max_m, const float* Acal,
                           float* ZL, float* ZR, int* errflag, cudaStream_t st, const void* tmaps) {
  if (nparts <= 0) return;
  tc::TmaMaps tm;
  std::memset(&tm, 0, sizeof tm);
  if (tmaps) std::memcpy(&tm, tmaps, sizeof tm);
  const int use_tma = (tmaps != nullptr && mode == 0) ? 1 : 0;
  const int tiles_n = (max_m + tc::NP - 1) / tc::NP;
  const dim3 grid(2 * tiles_n, nparts);
  int cap = 0;
  if (mode == 0) {
    const int bytes = tc_launch_smem<0>(max_m, &cap);
    raise_smem_once(tc::k_back_factor_tc<0>, tc::Smem<0>::total, &g_set_back[0]);
    tc::k_back_factor_tc<0><<<grid, tc::kThreads, bytes, st>>>(parts, s, tiles_n, Acal, ZL, ZR, errflag, tm, use_tma,
                                                               cap);
  } else {
    const int bytes = tc_launch_smem<1>(max_m, &cap);
    raise_smem_once(tc::k_back_factor_tc<1>, tc::Smem<1>::total, &g_set_back[1]);
    tc::k_back_factor_tc<1><<<grid, tc::kThreads, bytes, st>>>(parts, s, tiles_n, Acal, ZL, ZR, errflag, tm, 0, cap);
  }
}

namespace {
__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; 2 * i + 1 < n; i += stride) {
    const double2 v = reinterpret_cast<const double2*>(src)[i];
    reinterpret_cast<float2*>(dst)[i] = make_float2((float)v.x, (float)v.y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) dst[n - 1] = (float)src[n - 1];
}
}  // namespace

// float32 copy of a float64 array (the blocks the tensor-core sweeps stream).
void launch_to_f32(const double* src, float* dst, long long n, cudaStream_t st) {
  if (n <= 0) return;
  int sms = 152;
  k_to_f32<<<sms * 4, 256, 0, st>>>(src, dst, n);
}

// 2-D tensor maps ([rows][m] float32, box 32 x 128, 128-byte swizzle, zero
// fill past the extent) of the three arrays the TF32 sweeps stream as left
// operands.  Returns false when the driver entry point is unavailable or m is
// not a multiple of 4 (row pitch must be a multiple of 16 bytes).
bool make_tma_maps(const float* G, const float* A32, const float* Acal, long long rows, int m, void* out) {
  if (m % 4 != 0 || rows <= 0) return false;
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    enc = reinterpret_cast<Encode>(fn);
  }
  tc::TmaMaps tm;
  std::memset(&tm, 0, sizeof tm);
  const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)m * sizeof(float)};
  const cuuint32_t box[2] = {32, 128};
  const cuuint32_t estr[2] = {1, 1};
  const float* src[3] = {G, A32, Acal};
  CUtensorMap* dst[3] = {&tm.G, &tm.A, &tm.Acal};
  for (int i = 0; i < 3; ++i)
    if (enc(dst[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(src[i]), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  std::memcpy(out, &tm, sizeof tm);
  return true;
}

int tma_maps_bytes() { return (int)sizeof(tc::TmaMaps); }

bool residual_sliced_fits(int m, int r) { return m >= 1 && m <= tc::kRsMaxM && r >= 1 && r <= tc::kRsNB; }

void launch_row_scales(const SysDesc* sys, int nsys, int nrows, const double* A, const double* B,
                       const double* C, unsigned* rowhi, cudaStream_t st) {
  if (nsys <= 0 || nrows <= 0) return;
  tc::k_row_scales<<<nrows, tc::kRsThreads, 0, st>>>(sys, nsys, A, B, C, rowhi);
}

void launch_col_scales(const SysDesc* sys, int nsys, int nrows, const double* x, unsigned* colhi, cudaStream_t st) {
  if (nsys <= 0 || nrows <= 0) return;
  const int per = tc::kRsThreads / 32;
  tc::k_col_scales<<<(nrows + per - 1) / per, tc::kRsThreads, 0, st>>>(sys, nsys, nrows, x, colhi);
}

void launch_residual_sliced(const SysDesc* sys, int nsys, int nrows, const double* A, const double* B,
                            const double* C, const double* x, const double* b, double* r, double* nrm,
                            const unsigned* rowhi, const unsigned* colhi, int* errflag, cudaStream_t st) {
  if (nsys <= 0 || nrows <= 0) return;
  static bool set = false;
  raise_smem_once(tc::k_residual_sliced, tc::RsSmem::total, &set);
  tc::k_residual_sliced<<<nrows, tc::kRsThreads, tc::RsSmem::total, st>>>(sys, nsys, A, B, C, x, b, r, nrm, rowhi,
                                                                          colhi, errflag);
}

// One CTA per SM (the dynamic shared memory keeps a second one out), `iters`
// x 4 MMAs each; returns the flops of the launch.
double launch_mma_probe(int mode, int iters, int* errflag, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int smem = 116 * 1024;
  if (mode == 0) {
    cudaFuncSetAttribute(tc::k_mma_probe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    tc::k_mma_probe<0><<<sms, tc::kThreads, smem, st>>>(iters, errflag);
  } else {
    cudaFuncSetAttribute(tc::k_mma_probe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    tc::k_mma_probe<1><<<sms, tc::kThreads, smem, st>>>(iters, errflag);
  }
  const double k_per_instr = mode == 0 ? 8.0 : 16.0;
  return 2.0 * tc::MT * 256.0 * k_per_instr * 4.0 * iters * sms;
}

int tc_smem_bytes(int mode) { return mode == 0 ? tc::Smem<0>::total : tc::Smem<1>::total; }

}  // namespace dm

// dm_solve_noalloc: factor and solve one small system without allocating.
//
// Some callers cannot call cudaMalloc: code that runs while another component
// owns the device's memory pool, plug-ins loaded into a host application that
// forbids allocations on its solve path, or real-time loops that must not
// touch the allocator.  This entry point serves them.  Its workspace (block
// inverses, spikes, sweep vectors, the supplementary system and the launch
// descriptors) lives in one file-scope __device__ array of kScratchBytes,
// which every GPU that loads the library holds until the process exits.
//
// It runs the library's existing float64 kernels in the same order as
// dm_plan(P, levels = 1, DM_FP64) + dm_factor + dm_solve, with every
// pointer of the plan's workspace replaced by a slice of the array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/dm.h"
#include "dm_internal.cuh"
#include "dm_plan.h"

namespace dm {
namespace {

constexpr size_t kScratchBytes = 32ull << 20;  // 32 MiB per device
constexpr int kNoallocMaxP = 256;
constexpr int kMaxDevices = 64;

// The workspace.  Host code must not use this name as an address: it is a
// host-side stand-in.  The device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(DM_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(DM_EINVAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return set_error(DM_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return DM_OK;
}

// Bump allocator over the scratch slice (256-byte aligned pieces).
struct Carve {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    used = (used + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + used);
    used += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

}  // namespace
}  // namespace dm

using namespace dm;

extern "C" int dm_solve_noalloc(int N, int m, int nrhs, int P, const double* A, const double* B,
                                const double* C, const double* b, double* x, void* stream) {
  if (!A || !B || !C || !b || !x) return set_error(DM_EINVAL, "NULL argument to dm_solve_noalloc");
  if (N < 1 || m < 1 || nrhs < 1 || P < 1) return set_error(DM_EINVAL, "N, m, nrhs, P must be >= 1");
  if (m > kMaxM || nrhs > kMaxR) return set_error(DM_EINVAL, "m or nrhs above the library limits");
  if (P > kNoallocMaxP) return set_error(DM_EINVAL, "dm_solve_noalloc supports P <= %d", kNoallocMaxP);
  if (P > 1 && 2 * P - 1 > N) return set_error(DM_EINVAL, "P = %d too large for N = %d", P, N);
  // every block row needs at least 4 doubles of workspace (G, Acal, ZL, ZR of
  // a 1 x 1 block): reject N beyond that before any size arithmetic
  if ((size_t)N > kScratchBytes / (4 * sizeof(double)))
    return set_error(DM_EINVAL, "N = %d above dm_solve_noalloc's workspace limit", N);
  const long long mm = (long long)m * m, mr = (long long)m * nrhs, Ms = P - 1, NN = N;
  // bytes this call needs in the scratch array (same carving order as below);
  // N <= 2^20 and m^2 <= 2^18 keep every term far inside 64 bits
  const unsigned long long need =
      256ull * 20 + sizeof(double) * (unsigned long long)(4 * NN * mm + NN * mr + 5 * Ms * mm + 3 * Ms * mr) +
      sizeof(PartDesc) * (unsigned long long)(P + 1) + sizeof(SepDesc) * (unsigned long long)std::max(1, P - 1) +
      2 * sizeof(int);
  if (need > kScratchBytes)
    return set_error(DM_EINVAL,
                     "system needs %llu bytes of workspace, above dm_solve_noalloc's static %zu bytes "
                     "(4 N m^2 + 5 (P-1) m^2 doubles must stay below about 4 Mi)",
                     need, (size_t)kScratchBytes);
  // every array must be device (or managed) memory of the current device,
  // and x must not overlap b: the kernels read b while they write x
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(DM_ECUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    const void* ptrs[5] = {A, B, C, b, x};
    const char* names[5] = {"A", "B", "C", "b", "x"};
    for (int i = 0; i < 5; ++i) {
      cudaPointerAttributes at;
      e = cudaPointerGetAttributes(&at, ptrs[i]);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(DM_EINVAL, "dm_solve_noalloc: %s is not a CUDA pointer (%s)", names[i], cudaGetErrorString(e));
      }
      if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
        return set_error(DM_EINVAL, "dm_solve_noalloc: %s must be device memory of the current device %d", names[i],
                         dev);
    }
    const unsigned long long vb = (unsigned long long)(NN * mr) * sizeof(double);
    const unsigned long long pb = (unsigned long long)(uintptr_t)b, px = (unsigned long long)(uintptr_t)x;
    if (px < pb + vb && pb < px + vb) return set_error(DM_EINVAL, "dm_solve_noalloc: x must not overlap b");
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  Carve cv{static_cast<unsigned char*>(base)};
  double* G = cv.take<double>(N * mm);
  double* Acal = cv.take<double>(N * mm);
  double* ZL = cv.take<double>(N * mm);
  double* ZR = cv.take<double>(N * mm);
  double* z = cv.take<double>(N * mr);
  double* HA = cv.take<double>(Ms * mm);
  double* HB = cv.take<double>(Ms * mm);
  double* HC = cv.take<double>(Ms * mm);
  double* HG = cv.take<double>(Ms * mm);
  double* HAcal = cv.take<double>(Ms * mm);
  double* hz = cv.take<double>(Ms * mr);
  double* hF = cv.take<double>(Ms * mr);
  double* hX = cv.take<double>(Ms * mr);
  PartDesc* d_parts = cv.take<PartDesc>(P);
  PartDesc* d_sp = cv.take<PartDesc>(1);
  SepDesc* d_seps = cv.take<SepDesc>(std::max(1, P - 1));
  int* status = cv.take<int>(2);

  // descriptors (host stack; subsystem lengths are non-increasing in k, so
  // the subsystems active at a step form a prefix as the kernels expect)
  PartDesc hp[kNoallocMaxP];
  SepDesc hs[kNoallocMaxP];
  const int rows = N - (P - 1), base_len = rows / P, extra = rows % P;
  int r0 = 0;
  for (int k = 0; k < P; ++k) {
    PartDesc& d = hp[k];
    d.L = base_len + (k < extra ? 1 : 0);
    d.blk = r0 * mm;
    d.vec = r0 * mr;
    d.m = m;
    d.r = nrhs;
    d.flags = (k > 0 ? HAS_LEFT : 0) | (k < P - 1 ? HAS_RIGHT : 0);
    d.sys = 0;
    d.row0 = r0;
    d.hprev = k > 0 ? (k - 1) * mr : 0;
    d.hnext = k < P - 1 ? k * mr : 0;
    r0 += d.L;
    if (k < P - 1) {
      SepDesc& s = hs[k];
      s.blk_q = r0 * mm;
      s.vec_q = r0 * mr;
      s.blk_prev = s.blk_q - mm;
      s.vec_prev = s.vec_q - mr;
      s.blk_next = s.blk_q + mm;
      s.vec_next = s.vec_q + mr;
      s.hblk = k * mm;
      s.hvec = k * mr;
      s.m = m;
      s.r = nrhs;
      s.flags = (k > 0 ? HAS_HA : 0) | (k < P - 2 ? HAS_HC : 0);
      s.sys = 0;
      ++r0;
    }
  }
  PartDesc sp;  // the supplementary system: one subsystem (block Thomas)
  sp.L = (int)Ms;
  sp.blk = 0;
  sp.vec = 0;
  sp.m = m;
  sp.r = nrhs;
  sp.flags = 0;
  sp.sys = 0;
  sp.row0 = 0;
  sp.hprev = sp.hnext = 0;
  const int Lmax = hp[0].L;

#define DM_NA(call)                                                                               \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return set_error(DM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
  DM_NA(cudaMemcpyAsync(d_parts, hp, sizeof(PartDesc) * P, cudaMemcpyHostToDevice, st));
  DM_NA(cudaMemcpyAsync(d_sp, &sp, sizeof(PartDesc), cudaMemcpyHostToDevice, st));
  if (P > 1) DM_NA(cudaMemcpyAsync(d_seps, hs, sizeof(SepDesc) * (P - 1), cudaMemcpyHostToDevice, st));
  // the array keeps the previous call's contents: reset what must start known
  DM_NA(cudaMemsetAsync(status, 0x7f, 2 * sizeof(int), st));
  if (P > 1) {
    DM_NA(cudaMemsetAsync(HA, 0, sizeof(double) * Ms * mm, st));
    DM_NA(cudaMemsetAsync(HC, 0, sizeof(double) * Ms * mm, st));
  }

  auto active_fwd = [&](int t) {
    int c = 0;
    while (c < P && hp[c].L > t) ++c;
    return c;
  };
  auto active_back = [&](int s) {
    int c = 0;
    while (c < P && hp[c].L >= s + 2) ++c;
    return c;
  };
  // factor: subsystem sweeps, assembly, supplementary block Thomas
  for (int t = 0; t < Lmax; ++t) {
    launch_inv<double>(d_parts, active_fwd(t), t, B, G, status, m, st);
    launch_fwd_factor<double>(d_parts, active_fwd(t), t, m, A, B, C, G, Acal, ZL, ZR, st);
  }
  for (int s = 0; s + 1 < Lmax; ++s) launch_back_factor<double>(d_parts, active_back(s), s, m, Acal, ZL, ZR, st);
  if (P > 1) {
    launch_assemble_h<double>(d_seps, P - 1, m, A, B, C, ZL, ZR, HA, HB, HC, st);
    for (int t = 0; t < Ms; ++t) {
      launch_inv<double>(d_sp, 1, t, HB, HG, status + 1, m, st);
      launch_fwd_factor<double>(d_sp, 1, t, m, HA, HB, HC, HG, HAcal, HAcal, HAcal, st);
    }
  }
  // solve
  for (int t = 0; t < Lmax; ++t) launch_fwd_solve<double>(d_parts, active_fwd(t), t, m, nrhs, A, G, b, z, st);
  for (int s = 0; s + 1 < Lmax; ++s) launch_back_solve<double>(d_parts, active_back(s), s, m, nrhs, Acal, z, st);
  if (P > 1) {
    launch_assemble_f<double>(d_seps, P - 1, m, nrhs, A, C, b, z, hF, st);
    for (int t = 0; t < Ms; ++t) launch_fwd_solve<double>(d_sp, 1, t, m, nrhs, HA, HG, hF, hz, st);
    for (int s = 0; s + 1 < Ms; ++s) launch_back_solve<double>(d_sp, 1, s, m, nrhs, HAcal, hz, st);
    launch_backsub<double>(d_sp, 1, (int)Ms, m, nrhs, HAcal, HAcal, hz, nullptr, hX, st);
    launch_backsub<double>(d_parts, P, Lmax, m, nrhs, ZL, ZR, z, hX, x, st);
    launch_sep_copy(d_seps, P - 1, m, nrhs, hX, x, st);
  } else {
    launch_backsub<double>(d_parts, 1, Lmax, m, nrhs, ZL, ZR, z, nullptr, x, st);
  }
  DM_NA(cudaGetLastError());
  int hstat[2] = {0, 0};
  DM_NA(cudaMemcpyAsync(hstat, status, sizeof hstat, cudaMemcpyDeviceToHost, st));
  DM_NA(cudaStreamSynchronize(st));
#undef DM_NA
  if (hstat[0] != 0x7f7f7f7f)
    return set_error(DM_ESINGULAR, "singular pivot: block row %d (0-based)", hstat[0] - 1);
  if (hstat[1] != 0x7f7f7f7f)
    return set_error(DM_ESINGULAR, "singular pivot in the supplementary system, row %d", hstat[1] - 1);
  return DM_OK;
}

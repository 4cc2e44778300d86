// dm_peak_probe: measured arithmetic peaks of the GPU the library runs on,
// for the roofline denominators of the benchmark (the paper has no
// counterpart).  Each probe is a kernel that does nothing but the one kind of
// arithmetic at full occupancy, timed with CUDA events on its own stream.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/dm.h"
#include "dm_internal.cuh"
#include "dm_plan.h"

namespace dm {
namespace {

// The inner loop of a register-tiled matrix product: a 4 x 4 tile of
// accumulators per thread, acc[i][j] += x[i] * y[j] (16 independent chains,
// each instruction reading an accumulator and two shared operands), 64 fused
// multiply-adds per iteration.  x, y come from the arguments so nothing
// folds; the result is stored only if it hits an impossible value.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T b, T c, T* __restrict__ sink) {
  T x[4], y[4], acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    x[i] = b + (T)(threadIdx.x + i) * (T)1e-3;
    y[i] = c + (T)i * (T)1e-3;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
      }
    }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) s += acc[i][j];
  }
  if (s == (T)-12345.0) sink[0] = s;
}

}  // namespace
}  // namespace dm

using namespace dm;

extern "C" int dm_peak_probe(int kind, int repeat, double* tflops_out, double* ms_out) {
  if (kind < DM_PROBE_FP64 || kind > DM_PROBE_BF16 || repeat < 1 || !tflops_out)
    return set_error(DM_EINVAL, "dm_peak_probe: kind in 0..3, repeat >= 1, tflops_out non-NULL");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return set_error(DM_ECUDA, "dm_peak_probe: no CUDA device");
  }
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* scratch = nullptr;
  int rc = DM_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&scratch, 64) != cudaSuccess) {
    cudaGetLastError();
    rc = set_error(DM_ECUDA, "dm_peak_probe: stream/event/scratch setup failed");
  }
  cudaMemsetAsync(scratch, 0, 64, st);
  double best = 0.0, best_ms = 0.0;
  // about 0.1 s per timed launch at the nominal rates
  const int blocks = sms * 4, threads = 256;
  for (int it = 0; rc == DM_OK && it <= repeat; ++it) {  // launch 0 warms up
    double flops = 0.0;
    cudaEventRecord(e0, st);
    if (kind == DM_PROBE_FP64) {
      const int iters = 6000;
      k_fma_probe<double><<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, static_cast<double*>(scratch));
      flops = 2.0 * 64 * (double)iters * blocks * threads;
    } else if (kind == DM_PROBE_FP32) {
      const int iters = 400000;
      k_fma_probe<float><<<blocks, threads, 0, st>>>(iters, 0.999999f, 1e-7f, static_cast<float*>(scratch));
      flops = 2.0 * 64 * (double)iters * blocks * threads;
    } else {
      flops = launch_mma_probe(kind == DM_PROBE_TF32 ? 0 : 1, kind == DM_PROBE_TF32 ? 300000 : 200000,
                               static_cast<int*>(scratch) + 8, st);
    }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      rc = set_error(DM_ECUDA, "dm_peak_probe: kernel failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (it > 0 && ms > 0.f && flops / (ms * 1e9) > best) best = flops / (ms * 1e9), best_ms = ms;
  }
  if (rc == DM_OK) {
    int err = 0;
    cudaMemcpy(&err, static_cast<int*>(scratch) + 8, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) rc = set_error(DM_ETIMEOUT, "dm_peak_probe: a bounded tensor-core wait expired");
  }
  if (scratch) cudaFree(scratch);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (rc == DM_OK) {
    *tflops_out = best;
    if (ms_out) *ms_out = best_ms;
  }
  return rc;
}

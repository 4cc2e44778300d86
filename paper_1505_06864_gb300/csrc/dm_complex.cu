// Complex block-tridiagonal systems (the paper's application has complex
// boundary conditions, Section 7) solved through their real embedding.
//
// A complex m x m block M = X + iY acts on z = u + iv as the real 2m x 2m
// block [[X, -Y], [Y, X]] acting on [u; v]: (X u - Y v) + i (Y u + X v).
// Applied to every block, the complex system A_i z_{i-1} + B_i z_i +
// C_i z_{i+1} = b_i becomes a real block-tridiagonal system of the same N and
// nrhs with block size 2m, and the decomposition method runs on it unchanged
// (every precision, recursion and kernel of the real path).  The cost is
// twice the multiply-adds of complex arithmetic on m x m blocks.  Complex
// arrays are interleaved (real, imaginary) pairs with the real path's
// layouts: blocks [N][m][m], right-hand sides [N][m][nrhs].
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "../../include/dm.h"
#include "dm_internal.cuh"
#include "dm_plan.h"

namespace dm {
namespace {

// dst [N][2m][2m] from src [N][m][m] complex: X at (r, c) and (m + r, m + c),
// -Y at (r, m + c), Y at (m + r, c).
__global__ void k_embed_blocks(const double2* __restrict__ src, double* __restrict__ dst, long long N, int m) {
  const long long mm = (long long)m * m, total = N * mm;
  const long long m2 = 2LL * m;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const long long i = q / mm;
    const int rc = (int)(q - i * mm), r = rc / m, c = rc - r * m;
    const double2 z = src[q];
    double* d = dst + i * m2 * m2;
    d[(long long)r * m2 + c] = z.x;
    d[(long long)r * m2 + m + c] = -z.y;
    d[(long long)(m + r) * m2 + c] = z.y;
    d[(long long)(m + r) * m2 + m + c] = z.x;
  }
}

// dst [N][2m][nrhs] from src [N][m][nrhs] complex: real parts in rows
// 0..m-1, imaginary parts in rows m..2m-1 of every block row.
__global__ void k_embed_vec(const double2* __restrict__ src, double* __restrict__ dst, long long N, int m, int r) {
  const long long mr = (long long)m * r, total = N * mr;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const long long i = q / mr, e = q - i * mr;
    const double2 z = src[q];
    dst[i * 2 * mr + e] = z.x;
    dst[i * 2 * mr + mr + e] = z.y;
  }
}

// The inverse of k_embed_vec.
__global__ void k_extract_vec(const double* __restrict__ src, double2* __restrict__ dst, long long N, int m, int r) {
  const long long mr = (long long)m * r, total = N * mr;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x)
    {
      const long long i = q / mr, e = q - i * mr;
      dst[q] = make_double2(src[i * 2 * mr + e], src[i * 2 * mr + mr + e]);
    }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace
}  // namespace dm

using namespace dm;

extern "C" {

int dm_plan_complex(dm_plan_t* out, int N, int m, int nrhs, int P, int levels, int precision) {
  if (!out) return set_error(DM_EINVAL, "out is NULL");
  if (m < 1 || 2 * m > kMaxM) return set_error(DM_EINVAL, "complex block size m = %d: 1 <= m <= %d", m, kMaxM / 2);
  if ((precision == DM_TF32 || precision == DM_BF16X3) && 2 * m > kMaxMTensor)
    return set_error(DM_EINVAL, "complex systems on the tensor cores need m <= %d", kMaxMTensor / 2);
  dm_plan_t p = nullptr;
  int rc = dm_plan(&p, N, 2 * m, nrhs, P, levels, precision);
  if (rc) return rc;
  std::unique_ptr<dm_plan_s> hold(p);
  Plan& pl = p->plan;
  pl.cplx = true;
  pl.cm = m;
  pl.borrow = true;  // the plan factors the embedded blocks in place
  const long long m2 = 2LL * m;
  const size_t blk = (size_t)N * m2 * m2 * sizeof(double), vec = (size_t)N * m2 * nrhs * sizeof(double);
  pl.cstage_bytes = std::max((size_t)N * m * m, (size_t)N * m * nrhs) * 2 * sizeof(double);
  void* b[6] = {};
  const size_t sz[6] = {blk, blk, blk, pl.cstage_bytes, vec, vec};
  for (int i = 0; i < 6; ++i) {
    if (cudaMalloc(&b[i], std::max<size_t>(sz[i], 16)) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < i; ++j) cudaFree(b[j]);
      return set_error(DM_ENOMEM, "cudaMalloc of the complex plan's %zu-byte buffer failed", sz[i]);
    }
    pl.cbuf.push_back(b[i]);
  }
  pl.embA = static_cast<double*>(b[0]);
  pl.embB = static_cast<double*>(b[1]);
  pl.embC = static_cast<double*>(b[2]);
  pl.cstage = static_cast<double*>(b[3]);
  pl.bR = static_cast<double*>(b[4]);
  pl.xR = static_cast<double*>(b[5]);
  pl.device_bytes += 3 * blk + pl.cstage_bytes + 2 * vec;
  *out = hold.release();
  return DM_OK;
}

int dm_factor_complex(dm_plan_t plan, const double* A, const double* B, const double* C) {
  if (!plan || !A || !B || !C) return set_error(DM_EINVAL, "NULL argument to dm_factor_complex");
  Plan& pl = plan->plan;
  if (!pl.cplx) return set_error(DM_ESTATE, "dm_factor_complex needs a plan made by dm_plan_complex");
  const SysSpec& sp = pl.top.spec[0];
  const int m = pl.cm;
  const long long N = sp.N;
  const size_t bytes = (size_t)N * m * m * 2 * sizeof(double);
  const double* src[3] = {A, B, C};
  double* dst[3] = {pl.embA, pl.embB, pl.embC};
  for (int k = 0; k < 3; ++k) {
    const double* s = src[k];
    if (!is_device_ptr(s)) {
      int rc = copy_in(pl.cstage, s, bytes, pl.stream);
      if (rc) return rc;
      s = pl.cstage;
    }
    k_embed_blocks<<<grid_for(N * m * m), 256, 0, pl.stream>>>(reinterpret_cast<const double2*>(s), dst[k], N, m);
    DM_CUDA(cudaGetLastError());
  }
  return pl.factor(pl.embA, pl.embB, pl.embC);
}

int dm_solve_complex(dm_plan_t plan, const double* b, double* x, double* relres_out) {
  if (!plan || !b || !x) return set_error(DM_EINVAL, "NULL argument to dm_solve_complex");
  Plan& pl = plan->plan;
  if (!pl.cplx) return set_error(DM_ESTATE, "dm_solve_complex needs a plan made by dm_plan_complex");
  if (!pl.factored) return set_error(DM_ESTATE, "dm_solve_complex before a successful dm_factor_complex");
  const SysSpec& sp = pl.top.spec[0];
  const int m = pl.cm, r = sp.r;
  const long long N = sp.N;
  const size_t bytes = (size_t)N * m * r * 2 * sizeof(double);
  const double* s = b;
  if (!is_device_ptr(s)) {
    int rc = copy_in(pl.cstage, s, bytes, pl.stream);
    if (rc) return rc;
    s = pl.cstage;
  }
  k_embed_vec<<<grid_for(N * m * r), 256, 0, pl.stream>>>(reinterpret_cast<const double2*>(s), pl.bR, N, m, r);
  DM_CUDA(cudaGetLastError());
  int rc = pl.solve(pl.bR, pl.xR, relres_out);
  if (rc != DM_OK && rc != DM_ENOTCONV) return rc;
  const bool dev = is_device_ptr(x);
  double2* d = reinterpret_cast<double2*>(dev ? x : pl.cstage);
  k_extract_vec<<<grid_for(N * m * r), 256, 0, pl.stream>>>(pl.xR, d, N, m, r);
  DM_CUDA(cudaGetLastError());
  if (!dev) {
    int rc2 = copy_out(x, pl.cstage, bytes, pl.stream);
    if (rc2) return rc2;
  }
  DM_CUDA(cudaStreamSynchronize(pl.stream));
  return rc;
}

}  // extern "C"

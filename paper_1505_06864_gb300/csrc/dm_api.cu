// C ABI of the decomposition-method solver: plans, factor, solve, refinement.
//
// A plan is a stack of levels.  Level 0 holds the user's systems split into
// subsystems (Section 2 of the paper).  Level 1 holds every system's
// supplementary system (Eq. e232: P-1 block rows assembled from the spikes),
// split again into subsystems when the recursion depth asks for DM there
// (Section 4.2.1), and so on; the last level is solved by the block Thomas
// algorithm (one subsystem per system, Section 3).  Every level runs the same
// level-synchronous kernels (dm_kernels.cu); level 0 may hold float32 factors
// (mixed precision), every deeper level is float64.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dm.h"
#include "dm_internal.cuh"
#include "dm_plan.h"

namespace dm {

thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

// ---------------------------------------------------------------------------
// Level construction
int Level::build(const std::vector<SysSpec>& specs, bool fp32_factors, int tensor_mode) {
  f32 = fp32_factors;
  tc_mode = fp32_factors ? tensor_mode : -1;
  nsys = (int)specs.size();
  spec = specs;
  blk0.assign(nsys, 0);
  vec0.assign(nsys, 0);
  long long b = 0, v = 0;
  max_m = 1;
  max_r = 1;
  Nmax = 0;
  for (int s = 0; s < nsys; ++s) {
    blk0[s] = b;
    vec0[s] = v;
    b += (long long)specs[s].N * specs[s].m * specs[s].m;
    v += (long long)specs[s].N * specs[s].m * specs[s].r;
    max_m = std::max(max_m, specs[s].m);
    max_r = std::max(max_r, specs[s].r);
    Nmax = std::max(Nmax, specs[s].N);
  }
  nblk = b;
  nvec = v;
  // supplementary systems: one per system with P > 1
  std::vector<SysSpec> sub;
  std::vector<int> sub_of(nsys, -1);
  for (int s = 0; s < nsys; ++s) {
    if (specs[s].P > 1) {
      SysSpec t;
      t.N = specs[s].P - 1;
      t.m = specs[s].m;
      t.r = specs[s].r;
      t.levels = specs[s].levels - 1;
      t.P = (t.levels >= 1 && specs[s].P2 > 1) ? specs[s].P2 : 1;
      t.P2 = (t.levels >= 2) ? supp_partitions(t.P - 1, t.P, t.r, t.m) : 1;
      if (t.P <= 1) { t.levels = 1; t.P = 1; }
      sub_of[s] = (int)sub.size();
      sub.push_back(t);
    }
  }
  if (!sub.empty()) {
    supp.reset(new Level());
    supp->depth = depth + 1;
    supp->fp64_fma = fp64_fma;
    supp->inv_column = inv_column;
    int rc = supp->build(sub, false);
    if (rc) return rc;
  }
  // subsystem and separator tables
  nrows = 0;
  long long eoff = 0;
  parts.clear();
  seps.clear();
  sysd.clear();
  for (int s = 0; s < nsys; ++s) {
    const SysSpec& sp = specs[s];
    SysDesc sd;
    sd.blk = blk0[s];
    sd.vec = vec0[s];
    sd.N = sp.N;
    sd.m = sp.m;
    sd.r = sp.r;
    sd.sliced = 0;
    sd.eoff = (int)eoff;
    eoff += (long long)sp.N * sp.m;
    sd.row0 = nrows;
    nrows += sp.N;
    sysd.push_back(sd);
    std::vector<int> starts, lens, sepr;
    if (sp.J >= 2)
      nested_lengths(sp.N, sp.P / sp.J, sp.J, lens);
    else
      partition_lengths(sp.N, sp.P, sp.m, sp.r, sp.flags, lens);
    {
      int r0 = 0;
      for (int k = 0; k < sp.P; ++k) {
        starts.push_back(r0);
        r0 += lens[k];
        if (k < sp.P - 1) sepr.push_back(r0++);
      }
    }
    const long long mm = (long long)sp.m * sp.m, mr = (long long)sp.m * sp.r;
    for (int k = 0; k < sp.P; ++k) {
      PartDesc pd;
      pd.blk = blk0[s] + starts[k] * mm;
      pd.vec = vec0[s] + starts[k] * mr;
      pd.m = sp.m;
      pd.r = sp.r;
      pd.L = lens[k];
      pd.flags = (k > 0 ? HAS_LEFT : 0) | (k < sp.P - 1 ? HAS_RIGHT : 0);
      pd.sys = s;
      pd.row0 = starts[k];
      pd.hprev = pd.hnext = 0;
      if (sp.P > 1) {
        const int ss = sub_of[s];
        if (k > 0) pd.hprev = supp->vec0[ss] + (long long)(k - 1) * mr;
        if (k < sp.P - 1) pd.hnext = supp->vec0[ss] + (long long)k * mr;
      }
      parts.push_back(pd);
    }
    for (int j = 0; j + 1 < sp.P; ++j) {
      const int q = sepr[j];
      SepDesc d;
      d.blk_q = blk0[s] + q * mm;
      d.vec_q = vec0[s] + q * mr;
      d.blk_prev = d.blk_q - mm;
      d.vec_prev = d.vec_q - mr;
      d.blk_next = d.blk_q + mm;
      d.vec_next = d.vec_q + mr;
      const int ss = sub_of[s];
      d.hblk = supp->blk0[ss] + (long long)j * mm;
      d.hvec = supp->vec0[ss] + (long long)j * mr;
      d.m = sp.m;
      d.r = sp.r;
      d.flags = (j > 0 ? HAS_HA : 0) | (j < sp.P - 2 ? HAS_HC : 0);
      d.sys = s;
      seps.push_back(d);
    }
  }
  // longest subsystems first: the subsystems still active at a step form a prefix
  std::stable_sort(parts.begin(), parts.end(),
                   [](const PartDesc& a, const PartDesc& b) { return a.L > b.L; });
  nparts = (int)parts.size();
  nseps = (int)seps.size();
  last_part.assign(nsys, -1);
  for (int i = 0; i < nparts; ++i)
    if (!(parts[i].flags & HAS_RIGHT)) last_part[parts[i].sys] = i;
  Lmax = nparts ? parts[0].L : 0;
  active_fwd.assign(std::max(Lmax, 1), 0);
  for (int t = 0; t < Lmax; ++t) {
    int c = 0;
    while (c < nparts && parts[c].L > t) ++c;
    active_fwd[t] = c;
  }
  active_back.assign(std::max(Lmax, 1), 0);
  for (int s = 0; s + 1 < Lmax; ++s) {
    int c = 0;
    while (c < nparts && parts[c].L >= s + 2) ++c;
    active_back[s] = c;
  }
  // Both z sweeps in one persistent launch when every subsystem's cluster is
  // resident at once (a second wave would serialise whole sweeps); with many
  // subsystems the per-step launches keep the GPU busier.  DM_SOLVE_SWEEP=0
  // keeps the per-step kernels (for comparisons).
  {
    const char* e = std::getenv("DM_SOLVE_SWEEP");
    sweep_cs = (e && e[0] == '0') ? 0 : sweep_cluster_choice(f32 ? 4 : 8, max_m, max_r, nparts);
    sweep = sweep_cs > 0;
  }
  compute_costs();
  return DM_OK;
}

// Algorithmic flops and bytes of every launch (see Cost).
void Level::compute_costs() {
  const double es = f32 ? 4.0 : 8.0;
  c_inv.assign(std::max(Lmax, 1), Cost());
  c_fwd.assign(std::max(Lmax, 1), Cost());
  c_back.assign(std::max(Lmax, 1), Cost());
  c_fwds.assign(std::max(Lmax, 1), Cost());
  c_backs.assign(std::max(Lmax, 1), Cost());
  c_fwdA.assign(std::max(Lmax, 1), Cost());
  c_fwdA0.assign(std::max(Lmax, 1), Cost());
  c_fwdB.assign(std::max(Lmax, 1), Cost());
  c_cvt = Cost();
  c_asm_h = c_asm_f = c_backsub = c_resid = c_axpy = c_sepcopy = Cost();
  std::vector<double> chain(std::max(Lmax, 1), 0.0);
  for (const PartDesc& p : parts) {
    const double m2 = (double)p.m * p.m, m3 = 2.0 * m2 * p.m, mr = (double)p.m * p.r, m2r = 2.0 * m2 * p.r;
    const bool hl = p.flags & HAS_LEFT, hr = p.flags & HAS_RIGHT;
    for (int t = 0; t < p.L; ++t) {
      if (t < p.L - 1) chain[t] += 2 * m3;
      else if (hr) chain[t] += m3;
      Cost& ci = c_inv[t];
      ci.flops += m3;
      ci.bytes += (t == 0 ? 8.0 : es) * m2 + es * m2;
      Cost& cf = c_fwd[t];
      if (t < p.L - 1) { cf.flops += 2 * m3; cf.bytes += es * m2 * 3 + 24.0 * m2; }
      else if (hr) { cf.flops += m3; cf.bytes += es * m2 * 2 + 8.0 * m2; }
      if (hl) { cf.flops += (t == 0 ? m3 : 2 * m3); cf.bytes += 8.0 * m2 + es * m2 * (t == 0 ? 1 : 2) + (hl && t + 1 < p.L ? 0 : 0); }
      {
        // the same products split as the tensor-core step kernels launch them:
        // A = G_t [C_t | Y_t], B = A_{t+1} [Acal_t | Bcal_t]
        Cost& ca = c_fwdA[t];
        if (t < p.L - 1 || hr) {
          ca.flops += m3;
          ca.bytes += es * m2 * 2 + 3 * es * m2;
          c_fwdA0[t].flops += m3;
          c_fwdA0[t].bytes += es * m2 * 2 + 3 * es * m2;
        }
        if (hl) { ca.flops += m3; ca.bytes += es * m2 * 2 + 2 * es * m2; }
        if (t < p.L - 1) {
          Cost& cb = c_fwdB[t];
          cb.flops += m3;
          cb.bytes += es * m2 * 2 + 2 * es * m2;
          if (hl) { cb.flops += m3; cb.bytes += es * m2 + es * m2; }
        }
      }
      Cost& cs = c_fwds[t];
      cs.flops += (t == 0 ? m2r : 2 * m2r);
      cs.bytes += es * m2 + (t ? 8.0 * m2 + es * mr : 0) + 8.0 * mr + es * mr;
      if (t + 1 < p.L) {
        const int s = p.L - 2 - t;
        Cost& cb = c_back[s];
        if (hl || hr) cb.bytes += es * m2;
        if (hl) { cb.flops += m3; cb.bytes += 3 * es * m2; }
        if (hr) { cb.flops += m3; cb.bytes += 2 * es * m2; }
        Cost& cbs = c_backs[s];
        cbs.flops += m2r;
        cbs.bytes += es * m2 + 3 * es * mr;
      }
      const int ns = (hl ? 1 : 0) + (hr ? 1 : 0);
      c_backsub.flops += ns * m2r;
      c_backsub.bytes += ns * es * m2 + es * mr + 8.0 * mr;
    }
  }
  c_cvt.bytes = (double)nblk * (3 * 8.0 + 3 * 4.0);  // A, B, C read as float64, their copies written
  fwd_chain_frac.assign(std::max(Lmax, 1), 1.0);
  for (int t = 0; t < Lmax; ++t) fwd_chain_frac[t] = c_fwd[t].flops > 0 ? chain[t] / c_fwd[t].flops : 1.0;
  for (const SepDesc& d : seps) {
    const double m2 = (double)d.m * d.m, m3 = 2.0 * m2 * d.m, mr = (double)d.m * d.r, m2r = 2.0 * m2 * d.r;
    const int extra = ((d.flags & HAS_HA) ? 1 : 0) + ((d.flags & HAS_HC) ? 1 : 0);
    c_asm_h.flops += (2 + extra) * m3;
    c_asm_h.bytes += 24.0 * m2 + (2 + extra) * (8.0 + 0.0) * m2 + (2 + extra) * es * m2;
    c_asm_f.flops += 2 * m2r;
    c_asm_f.bytes += 16.0 * m2 + 8.0 * mr * 2 + 2 * es * mr;
    c_sepcopy.bytes += 16.0 * mr;
  }
  for (const SysDesc& d : sysd) {
    const double m2 = (double)d.m * d.m, mr = (double)d.m * d.r;
    c_resid.flops += d.N * 6.0 * m2 * d.r;
    c_resid.bytes += d.N * (24.0 * m2 + 24.0 * mr);
    c_axpy.flops += d.N * 2.0 * mr;
    c_axpy.bytes += d.N * 24.0 * mr;
  }
}

// Device bytes of the tensor-core step kernels' operand copies (4 bytes per
// element in both modes: float32, or bf16 hi + lo): B32, A, C^T (+ Acal for
// split bf16) over all blocks, and the rolling buffers (G for split bf16,
// Acal^T, Y^T, two slots each of ZL^T, ZR^T) per subsystem.
static size_t tc2_bytes(int mode, long long nblk, int nparts, int m) {
  const size_t mm = (size_t)m * m;
  return (size_t)nblk * 4 * (mode == 1 ? 4 : 3) + (size_t)nparts * mm * 4 * (mode == 1 ? 7 : 6);
}

static bool uniform_m(const std::vector<SysSpec>& spec, int m) {
  for (const SysSpec& sp : spec)
    if (sp.m != m) return false;
  return true;
}

static bool tc2_wanted(const Level& L) {
  const char* e = std::getenv("DM_TC_STEP");
  return L.tc_mode >= 0 && !(e && e[0] == '0') && uniform_m(L.spec, L.max_m) && tc2_eligible(L.max_m);
}

// Float64 products by digit slicing on the tensor cores: float64 levels
// with one block size m % 8 == 0, m <= 256, unless the plan asked for the
// FP64 pipe (DM_PLAN_FP64_FMA) or DM_FP64_PRODUCTS=fma is set.
static bool oz_wanted(const Level& L) {
  const char* e = std::getenv("DM_FP64_PRODUCTS");
  return !L.f32 && !L.fp64_fma && !(e && std::strcmp(e, "fma") == 0) && uniform_m(L.spec, L.max_m) &&
         oz_eligible(L.max_m);
}

static size_t oz_bytes(long long nblk, int nparts, int nseps, int m) {
  const size_t mm = (size_t)m * m, sl = (size_t)oz_slice_blocks_bytes(m), nb = nblk / mm, np = std::max(1, nparts);
  return (3 * nb + 7 * np + 5 * (size_t)nseps) * (sl + m * sizeof(int)) + np * mm * sizeof(double) +
         np * ((size_t)2 * 9 * m * 32 * 2 + 3 * m * sizeof(int));
}

// The supplementary blocks of a sliced level as digit-sliced tensor-core
// products, unless DM_FP64_ASSEMBLY=fma (the float64 kernel).  Measured at
// m = 256 on GB300: see the assembly kernel's figures in the design notes.
static bool oz_asm_wanted() {
  const char* e = std::getenv("DM_FP64_ASSEMBLY");
  return !(e && std::strcmp(e, "fma") == 0);
}

// The float64 block inverse of a sliced level: blocked Gauss-Jordan with the
// trailing updates on the tensor cores, unless DM_FP64_INVERSE=cluster (the
// column-by-column kernel).  Measured at m = 256 on GB300: faster for every
// launch size, 64 blocks per launch (the top level) 1.45 vs 2.5 ms, and the
// supplementary levels' 1-12 blocks per launch 9.2 vs 10.9 ms per factor.
static bool gj_wanted(const Level& L) {
  const char* e = std::getenv("DM_FP64_INVERSE");
  return !L.inv_column && !(e && std::strcmp(e, "cluster") == 0);
}

size_t Level::bytes_needed() const {
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  size_t b = 3 * nblk * sizeof(double);     // A, B, C
  if (tc2_wanted(*this)) b += tc2_bytes(tc_mode, nblk, nparts, max_m);
  else if (oz_wanted(*this)) b += oz_bytes(nblk, nparts, nseps, max_m);
  else if (tc_mode >= 0) b += 3 * nblk * sizeof(float);
  b += 4 * nblk * es;                       // G, Acal, ZL, ZR
  b += nvec * es;                           // z
  b += 2 * nvec * sizeof(double);           // F, X
  b += parts.size() * sizeof(PartDesc) + seps.size() * sizeof(SepDesc) + sysd.size() * sizeof(SysDesc);
  b += nsys * sizeof(int);
  if (supp) b += supp->bytes_needed();
  return b;
}

int Level::allocate() {
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(DM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    owned.push_back(*p);
    return DM_OK;
  };
  int rc;
#define DM_ALLOC(ptr, bytes)                                    \
  if ((rc = alloc(reinterpret_cast<void**>(&(ptr)), (bytes)))) \
    return rc;
  // the top level's A, B, C copies are allocated at the first copying factor
  // (ensure_inputs); deeper levels own their assembled blocks from the start
  if (!lazy_inputs) {
    DM_ALLOC(A, nblk * sizeof(double));
    DM_ALLOC(B, nblk * sizeof(double));
    DM_ALLOC(C, nblk * sizeof(double));
  }
  DM_ALLOC(G, nblk * es);
  DM_ALLOC(Acal, nblk * es);
  DM_ALLOC(ZL, nblk * es);
  DM_ALLOC(ZR, nblk * es);
  DM_ALLOC(z, nvec * es);
  DM_ALLOC(F, nvec * sizeof(double));
  DM_ALLOC(X, nvec * sizeof(double));
  DM_ALLOC(d_parts, std::max<size_t>(1, parts.size()) * sizeof(PartDesc));
  DM_ALLOC(d_seps, std::max<size_t>(1, seps.size()) * sizeof(SepDesc));
  DM_ALLOC(d_sys, std::max<size_t>(1, sysd.size()) * sizeof(SysDesc));
  DM_ALLOC(status, std::max(1, nsys) * sizeof(int));
  DM_ALLOC(d_err, sizeof(int));
  if (tc_mode >= 0 && tc2_wanted(*this)) {
    // operand copies and tensor maps of the tensor-core step kernels
    Tc2Level& T = tc2;
    const int m = max_m, mode = tc_mode, np = std::max(1, nparts), parts_ = mode == 1 ? 2 : 1;
    const long long mm = (long long)m * m, nb = nblk / mm;
    const size_t blk4 = (size_t)mm * 4;  // bytes of one block copy (both modes)
    T.mode = mode;
    DM_ALLOC(B32, nblk * sizeof(float));
    if (mode == 0) {
      DM_ALLOC(A32, nblk * sizeof(float));
      T.A = A32;
    } else {
      DM_ALLOC(T.A, nb * blk4);
      DM_ALLOC(T.Acal, nb * blk4);
      DM_ALLOC(T.G, np * blk4);
    }
    DM_ALLOC(T.CT, nb * blk4);
    DM_ALLOC(T.AcalT, np * blk4);
    DM_ALLOC(T.YT, np * blk4);
    DM_ALLOC(T.ZLT, 2 * np * blk4);
    DM_ALLOC(T.ZRT, 2 * np * blk4);
    T.capA = T.capCT = T.capAcal = nb;
    T.capG = T.capAcalT = T.capYT = np;
    T.capZLT = T.capZRT = 2 * np;
    const int nt = tc2_ntile(m);
    const void* lbase[3] = {mode == 0 ? G : T.G, T.A, mode == 0 ? Acal : T.Acal};
    const long long lblk[3] = {mode == 0 ? nb : T.capG * parts_, T.capA * parts_, mode == 0 ? nb : T.capAcal * parts_};
    const void* rbase[5] = {T.CT, T.YT, T.AcalT, T.ZLT, T.ZRT};
    const long long rblk[5] = {T.capCT * parts_, T.capYT * parts_, T.capAcalT * parts_, T.capZLT * parts_,
                               T.capZRT * parts_};
    bool ok = tc2_map_bytes() == 128;
    for (int i = 0; ok && i < 3; ++i) ok = tc2_make_map(mode, lbase[i], lblk[i], m, 128, T.maps[i]);
    for (int i = 0; ok && i < 5; ++i) ok = tc2_make_map(mode, rbase[i], rblk[i], m, nt, T.maps[3 + i]);
    if (!ok) return set_error(DM_ECUDA, "tensor map creation for the tensor-core step kernels failed (m = %d)", m);
    T.on = true;
  } else if (oz_wanted(*this)) {
    // digit slices, exponents and tensor maps of the float64 tensor-core products
    OzLevel& Z = oz;
    const int m = max_m, np = std::max(1, nparts);
    const long long mm = (long long)m * m, nb = nblk / mm;
    const size_t sl = (size_t)oz_slice_blocks_bytes(m), ex = (size_t)m * sizeof(int);
    DM_ALLOC(Z.A, nb * sl);
    DM_ALLOC(Z.CT, nb * sl);
    DM_ALLOC(Z.Acal, nb * sl);
    DM_ALLOC(Z.G, np * sl);
    DM_ALLOC(Z.AcalT, np * sl);
    DM_ALLOC(Z.YT, np * sl);
    DM_ALLOC(Z.ZLT, 2 * np * sl);
    DM_ALLOC(Z.ZRT, 2 * np * sl);
    DM_ALLOC(Z.eA, nb * ex);
    DM_ALLOC(Z.eCT, nb * ex);
    DM_ALLOC(Z.eAcal, nb * ex);
    DM_ALLOC(Z.eG, np * ex);
    DM_ALLOC(Z.eAcalT, np * ex);
    DM_ALLOC(Z.eYT, np * ex);
    DM_ALLOC(Z.eZLT, 2 * np * ex);
    DM_ALLOC(Z.eZRT, 2 * np * ex);
    DM_ALLOC(Z.Y, np * mm * sizeof(double));
    const void* lbase[3] = {Z.G, Z.A, Z.Acal};
    const long long lblk[3] = {np, nb, nb};
    const void* rbase[5] = {Z.CT, Z.YT, Z.AcalT, Z.ZLT, Z.ZRT};
    const long long rblk[5] = {nb, np, np, 2 * np, 2 * np};
    bool ok = true;
    for (int i = 0; ok && i < 3; ++i) ok = oz_make_map(lbase[i], lblk[i], m, oz_box_rows_left(), Z.maps[i]);
    for (int i = 0; ok && i < 5; ++i) ok = oz_make_map(rbase[i], rblk[i], m, oz_box_rows_right(), Z.maps[3 + i]);
    if (!ok) return set_error(DM_ECUDA, "tensor map creation for the float64 slice products failed (m = %d)", m);
    Z.on = true;
    if (gj_wanted(*this)) {
      const size_t pb = (size_t)9 * m * 32 * 2;
      DM_ALLOC(Z.U, np * pb);
      DM_ALLOC(Z.V, np * pb);
      DM_ALLOC(Z.eU, np * ex);
      DM_ALLOC(Z.eV, np * ex);
      DM_ALLOC(Z.piv, np * ex);
      ok = oz_make_map(Z.U, np, m, oz_box_rows_left(), Z.gj_maps[0], 32) &&
           oz_make_map(Z.V, np, m, oz_box_rows_gj(), Z.gj_maps[1], 32);
      if (!ok) return set_error(DM_ECUDA, "tensor map creation for the blocked inversion failed (m = %d)", m);
      Z.gj = true;
    }
    const char* eb = std::getenv("DM_BANDED");
    if (!(eb && std::strcmp(eb, "0") == 0)) {
      DM_ALLOC(Z.band, sizeof(int));
      cudaMemset(Z.band, 0x7f, sizeof(int));  // "not banded" until a factorisation finds out
      if (cudaHostAlloc(reinterpret_cast<void**>(&Z.band_host), sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return set_error(DM_ENOMEM, "cudaHostAlloc of 4 bytes failed");
      }
      *Z.band_host = kBandMax + 1;
    }
    if (nseps > 0 && oz_asm_wanted()) {
      OzAsm& a = Z.as;
      DM_ALLOC(a.Cq, nseps * sl);
      DM_ALLOC(a.S, 4LL * nseps * sl);
      DM_ALLOC(a.eCq, nseps * ex);
      DM_ALLOC(a.eS, 4LL * nseps * ex);
      ok = oz_make_map(a.Cq, nseps, m, oz_box_rows_left(), a.maps[0]) &&
           oz_make_map(a.S, 4LL * nseps, m, oz_box_rows_right(), a.maps[1]);
      if (!ok) return set_error(DM_ECUDA, "tensor map creation for the sliced assembly failed (m = %d)", m);
      Z.asm_on = true;
    }
  } else if (tc_mode >= 0) {
    DM_ALLOC(A32, nblk * sizeof(float));
    DM_ALLOC(B32, nblk * sizeof(float));
    DM_ALLOC(C32, nblk * sizeof(float));
    // TF32 sweeps stream G, A32, Acal by TMA when every system has the same m
    if (tc_mode == 0 && uniform_m(spec, max_m) && tma_maps_bytes() <= (int)sizeof(tmaps))
      has_tma = make_tma_maps(static_cast<float*>(G), A32, static_cast<float*>(Acal), nblk / max_m, max_m, tmaps);
  }
#undef DM_ALLOC
  if (!parts.empty()) DM_CUDA(cudaMemcpy(d_parts, parts.data(), parts.size() * sizeof(PartDesc), cudaMemcpyHostToDevice));
  if (!seps.empty()) DM_CUDA(cudaMemcpy(d_seps, seps.data(), seps.size() * sizeof(SepDesc), cudaMemcpyHostToDevice));
  DM_CUDA(cudaMemcpy(d_sys, sysd.data(), sysd.size() * sizeof(SysDesc), cudaMemcpyHostToDevice));
  if (supp) {
    rc = supp->allocate();
    if (rc) return rc;
    // corner blocks of the supplementary systems that no assembly writes
    DM_CUDA(cudaMemset(supp->A, 0, supp->nblk * sizeof(double)));
    DM_CUDA(cudaMemset(supp->C, 0, supp->nblk * sizeof(double)));
  }
  return DM_OK;
}

int Level::ensure_inputs() {
  if (A) return DM_OK;
  void* p[3] = {nullptr, nullptr, nullptr};
  for (int i = 0; i < 3; ++i) {
    cudaError_t e = cudaMalloc(&p[i], std::max<size_t>(16, nblk * sizeof(double)));
    if (e != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < i; ++j) cudaFree(p[j]);
      return set_error(DM_ENOMEM, "cudaMalloc of the %zu-byte input copies failed: %s", nblk * sizeof(double),
                       cudaGetErrorString(e));
    }
  }
  for (int i = 0; i < 3; ++i) owned.push_back(p[i]);
  A = static_cast<double*>(p[0]);
  B = static_cast<double*>(p[1]);
  C = static_cast<double*>(p[2]);
  return DM_OK;
}

void Level::release(void* p) {
  for (size_t i = 0; i < owned.size(); ++i)
    if (owned[i] == p) {
      cudaFree(p);
      owned.erase(owned.begin() + i);
      return;
    }
}

Level::~Level() {
  for (void* p : owned) cudaFree(p);
  if (oz.band_host) cudaFreeHost(oz.band_host);
}

// ---------------------------------------------------------------------------
// Profiler
const char* const kClassNames[K_NCLASS] = {
    "inv", "fwd_factor", "back_factor", "assemble_h", "fwd_solve", "back_solve", "assemble_f",
    "backsub", "sep_copy", "residual", "axpy_norms", "sweep_solve", "tc_convert", "inv_panel", "inv_update",
    "banded"};

cudaEvent_t Prof::take() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Prof::begin(cudaStream_t st, cudaEvent_t* e0) {
  *e0 = nullptr;
  if (!on) return;
  *e0 = take();
  cudaEventRecord(*e0, st);
}

void Prof::end(cudaStream_t st, cudaEvent_t e0, int cls, double fl, double by, int kernels) {
  const bool launched = kernels > 0;
  launches += kernels;
  if (!on || !e0) return;
  if (!launched) {
    pool.push_back(e0);
    return;
  }
  cudaEvent_t e1 = take();
  cudaEventRecord(e1, st);
  recs.push_back(Rec{cls + K_NCLASS * std::min(depth, kDepths - 1), e0, e1, fl, by});
}

int Prof::collect() {
  for (Rec& r : recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess) {
      cudaGetLastError();
      t = 0.f;
    }
    n[r.cls] += 1;
    ms[r.cls] += t;
    flops[r.cls] += r.flops;
    bytes[r.cls] += r.bytes;
    pool.push_back(r.e0);
    pool.push_back(r.e1);
  }
  recs.clear();
  return DM_OK;
}

void Prof::reset() {
  collect();
  for (int i = 0; i < K_NCLASS * kDepths; ++i) n[i] = 0, ms[i] = flops[i] = bytes[i] = 0.0;
}

Prof::~Prof() {
  for (Rec& r : recs) pool.push_back(r.e0), pool.push_back(r.e1);
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

// One profiled call that launches `nk` kernels (when active > 0).
#define DM_LAUNCH_K(pf, st, cls, cost, active, nk, call)                         \
  do {                                                                           \
    cudaEvent_t e0_;                                                             \
    (pf).begin((st), &e0_);                                                      \
    call;                                                                        \
    (pf).end((st), e0_, (cls), (cost).flops, (cost).bytes, (active) > 0 ? (nk) : 0); \
  } while (0)
#define DM_LAUNCH(pf, st, cls, cost, active, call) DM_LAUNCH_K(pf, st, cls, cost, active, 1, call)

// Forward and backward sweeps of a float32 level on the tensor-core step
// kernels (dm_tc2.cu): operand copies of A, B, C^T and Y_0 = A_first^T, then
// per step the inversion, (split bf16) the copy of G_t, launch A = G_t [C_t |
// Y_t] and launch B = A_{t+1} [Acal_t | Bcal_t]; then the backward steps.
static void factor_level_tc2(Level& L, cudaStream_t st, Prof& pf) {
  Tc2Level& T = L.tc2;
  const int m = L.max_m, mode = T.mode;
  const long long nb = L.nblk / ((long long)m * m);
  float* G = static_cast<float*>(L.G);
  Tc2Out out;
  out.B32 = L.B32;
  out.G = G;
  out.Acal = static_cast<float*>(L.Acal);
  out.ZL = static_cast<float*>(L.ZL);
  out.ZR = static_cast<float*>(L.ZR);
  out.acal_l = T.Acal;
  out.acalT = T.AcalT;
  out.yT = T.YT;
  out.zlT = T.ZLT;
  out.zrT = T.ZRT;
  out.cap_acal_l = T.capAcal;
  out.cap_acalT = T.capAcalT;
  out.cap_yT = T.capYT;
  out.cap_zlT = T.capZLT;
  out.cap_zrT = T.capZRT;
  alignas(64) unsigned char maps[3][3][128];
  const int sel[3][3] = {{0, 3, 4}, {1, 5, 6}, {2, 6, 7}};  // left, right 0, right 1 of kinds 0, 1, 2
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) std::memcpy(maps[k][i], T.maps[sel[k][i]], 128);
  const int lo[3][3] = {{(int)T.capG, (int)T.capCT, (int)T.capYT},
                        {(int)T.capA, (int)T.capAcalT, (int)T.capZLT},
                        {(int)T.capAcal, (int)T.capZLT, (int)T.capZRT}};
  auto convert_inputs = [&] {
    launch_to_f32(L.B, L.B32, L.nblk, st);
    if (mode == 0) launch_to_f32(L.A, L.A32, L.nblk, st);
    else launch_tc2_convert(1, L.A, nullptr, nullptr, (int)nb, 0, m, false, T.A, T.capA, st);
    launch_tc2_convert(mode, L.C, nullptr, nullptr, (int)nb, 0, m, true, T.CT, T.capCT, st);
    launch_tc2_convert(mode, L.A, nullptr, L.d_parts, L.nparts, 0, m, true, T.YT, T.capYT, st);
  };
  DM_LAUNCH_K(pf, st, K_TC_CONVERT, L.c_cvt, 1, 4, convert_inputs());
  for (int t = 0; t < L.Lmax; ++t) {
    const int np = L.active_fwd[t];
    DM_LAUNCH(pf, st, K_INV, L.c_inv[t], np, launch_inv<float>(L.d_parts, np, t, L.B, G, L.status, L.max_m, st));
    if (mode == 1) {
      Cost c;
      c.bytes = 8.0 * np * m * m;
      DM_LAUNCH(pf, st, K_TC_CONVERT, c, np,
                launch_tc2_convert(1, nullptr, G, L.d_parts, np, t, m, false, T.G, T.capG, st));
    }
    DM_LAUNCH(pf, st, K_FWD_FACTOR, L.c_fwdA[t], np,
              launch_tc2_step(mode, 0, L.d_parts, np, t, m, lo[0], out, maps[0], L.d_err, st));
    const int nbk = L.active_back[t];
    DM_LAUNCH(pf, st, K_FWD_FACTOR, L.c_fwdB[t], nbk,
              launch_tc2_step(mode, 1, L.d_parts, nbk, t, m, lo[1], out, maps[1], L.d_err, st));
  }
  for (int s = 0; s + 1 < L.Lmax; ++s)
    DM_LAUNCH(pf, st, K_BACK_FACTOR, L.c_back[s], L.active_back[s],
              launch_tc2_step(mode, 2, L.d_parts, L.active_back[s], s, m, lo[2], out, maps[2], L.d_err, st));
}

// Forward and backward sweeps of a float64 level with its block products on
// the tensor cores by digit slicing (dm_oz.cu): slices of A (rows), C^T and
// Y_0 = A_first^T (columns), then per step the float64 inversion, the row
// slices of G_t, launch A = G_t [C_t | Y_t], slices of its results (Acal_t
// rows and columns, Bcal_t columns, the right spike's seed), launch B =
// A_{t+1} [Acal_t | Bcal_t] and the column slices of Y_{t+1}; then the
// backward steps, each followed by the column slices of its spikes.
static void factor_level_oz(Level& L, cudaStream_t st, Prof& pf) {
  OzLevel& Z = L.oz;
  const int m = L.max_m;
  const long long nb = L.nblk / ((long long)m * m);
  double* G = static_cast<double*>(L.G);
  OzOut out{};
  out.B = L.B;
  out.G = G;
  out.Acal = static_cast<double*>(L.Acal);
  out.ZL = static_cast<double*>(L.ZL);
  out.ZR = static_cast<double*>(L.ZR);
  out.Y = Z.Y;
  out.band = Z.band;
  // banded A and C as the previous factorisation found them (profiling costs
  // only: the kernels read the flag this factorisation's slicing sets)
  const int wb = Z.band ? *Z.band_host : kBandMax + 1;
  const bool banded_h = wb <= kBandMax;
  auto band_cost = [&](int units, int products) {
    Cost c;
    if (banded_h) {
      c.flops = (double)units * products * 2.0 * m * m * (2 * wb + 1);
      c.bytes = (double)units * products * (16.0 + 8.0) * m * m;
    }
    return c;
  };
  alignas(64) unsigned char maps[3][3][128];
  const int sel[3][3] = {{0, 3, 4}, {1, 5, 6}, {2, 6, 7}};
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i) std::memcpy(maps[k][i], Z.maps[sel[k][i]], 128);
  const int* lexp[3] = {Z.eG, Z.eA, Z.eAcal};
  const int* r0exp[3] = {Z.eCT, Z.eAcalT, Z.eZLT};
  const int* r1exp[3] = {Z.eYT, Z.eZLT, Z.eZRT};
  auto job = [](const double* src, void* dst, int* e, int kind) { return OzSliceJob{src, dst, e, kind}; };
  auto slice_inputs = [&] {
    if (Z.band) {
      cudaMemsetAsync(Z.band, 0, sizeof(int), st);
      launch_band_detect(L.A, L.C, L.nblk, m, Z.band, st);
    }
    launch_oz_slice_all(false, L.A, (int)nb, m, Z.A, Z.eA, Z.band, st);
    launch_oz_slice_all(true, L.C, (int)nb, m, Z.CT, Z.eCT, Z.band, st);
    if (Z.band) cudaMemcpyAsync(Z.band_host, Z.band, sizeof(int), cudaMemcpyDeviceToHost, st);
    OzSliceJobs j0;
    j0.job[0] = job(L.A, Z.YT, Z.eYT, 8);
    launch_oz_slice_jobs(L.d_parts, L.nparts, 0, m, j0, 1, st);
  };
  Cost cslice = L.c_cvt;
  DM_LAUNCH_K(pf, st, K_TC_CONVERT, cslice, 1, Z.band ? 4 : 3, slice_inputs());
  Cost cs;
  cs.bytes = 26.0 * m * m;  // one block: float64 read, nine bf16 slices written
  for (int t = 0; t < L.Lmax; ++t) {
    const int np = L.active_fwd[t], nbk = L.active_back[t];
    if (Z.gj) {
      // the blocked inversion, its phases profiled apart: the float64 panels
      // (2 m kw^2 flops per block), the tensor-core trailing updates (2 m (m -
      // kw) kw), the copy of B_0 and the finishing pass, which also writes
      // G_t's row slices
      Cost cb, cf;
      cb.bytes = np * 16.0 * m * m;           // B_0 read, written to G
      cf.bytes = np * (16.0 + 18.0) * m * m;  // G_t read and written, nine bf16 slices written
      if (t == 0) DM_LAUNCH(pf, st, K_INV, cb, np, launch_gj_begin(L.d_parts, np, t, m, L.B, G, st));
      for (int k0 = 0; k0 < m; k0 += 32) {
        const double kw = std::min(32, m - k0);
        Cost cp, cu;
        cp.flops = np * 2.0 * m * kw * kw;
        cp.bytes = np * (16.0 * m * kw + 18.0 * 32.0 * 2 * m + 8.0 * kw * m);
        cu.flops = np * 2.0 * m * (m - kw) * kw;
        cu.bytes = np * (16.0 * m * (m - kw) + 18.0 * 32.0 * 2 * m);
        DM_LAUNCH(pf, st, K_INV_PANEL, cp, np,
                  launch_gj_panel(L.d_parts, np, t, m, k0 / 32, G, Z.piv, Z.U, Z.eU, Z.V, Z.eV, L.status, st));
        if (m > 32)
          DM_LAUNCH(pf, st, K_INV_UPDATE, cu, np,
                    launch_gj_update(L.d_parts, np, t, m, k0 / 32, G, Z.eU, Z.eV, Z.gj_maps, L.d_err, st));
      }
      DM_LAUNCH(pf, st, K_INV, cf, np, launch_gj_finish(L.d_parts, np, t, m, G, Z.piv, Z.G, Z.eG, st));
    } else {
      DM_LAUNCH(pf, st, K_INV, L.c_inv[t], np, launch_inv<double>(L.d_parts, np, t, L.B, G, L.status, L.max_m, st));
      OzSliceJobs jg;
      jg.job[0] = job(G, Z.G, Z.eG, 0);
      Cost c0 = cs;
      c0.bytes *= np;
      DM_LAUNCH(pf, st, K_TC_CONVERT, c0, np, launch_oz_slice_jobs(L.d_parts, np, t, m, jg, 1, st));
    }
    Cost ca = L.c_fwdA[t];
    if (banded_h) ca.flops -= L.c_fwdA0[t].flops, ca.bytes -= L.c_fwdA0[t].bytes;
    DM_LAUNCH(pf, st, K_FWD_FACTOR, ca, np,
              launch_oz_step(0, L.d_parts, np, t, m, out, lexp[0], r0exp[0], r1exp[0], maps[0], L.d_err, st));
    if (Z.band)  // G_t C_t when C is banded (the tiles above skip it then)
      DM_LAUNCH(pf, st, K_BANDED, band_cost(np, 1), np,
                launch_band_gc(L.d_parts, np, t, m, G, L.C, out.Acal, out.ZR, Z.band, st));
    OzSliceJobs ja;
    ja.band = Z.band;
    ja.job[0] = job(out.Acal, Z.Acal, Z.eAcal, 1);
    ja.job[1] = job(out.Acal, Z.AcalT, Z.eAcalT, 2);
    ja.job[2] = job(out.ZL, Z.ZLT, Z.eZLT, 3);
    ja.job[3] = job(out.ZR, Z.ZRT, Z.eZRT, 4);
    Cost c1 = cs;
    c1.bytes *= 4.0 * np;
    DM_LAUNCH(pf, st, K_TC_CONVERT, c1, np, launch_oz_slice_jobs(L.d_parts, np, t, m, ja, 4, st));
    DM_LAUNCH(pf, st, K_FWD_FACTOR, banded_h ? Cost() : L.c_fwdB[t], nbk,
              launch_oz_step(1, L.d_parts, nbk, t, m, out, lexp[1], r0exp[1], r1exp[1], maps[1], L.d_err, st));
    if (Z.band)  // both products of launch B when A is banded
      DM_LAUNCH(pf, st, K_BANDED, band_cost(nbk, 2), nbk,
                launch_band_b(L.d_parts, nbk, t, m, L.A, L.B, out.Acal, out.ZL, G, Z.Y, Z.band, st));
    OzSliceJobs jy;
    jy.job[0] = job(Z.Y, Z.YT, Z.eYT, 5);
    Cost c2 = cs;
    c2.bytes *= nbk;
    DM_LAUNCH(pf, st, K_TC_CONVERT, c2, nbk, launch_oz_slice_jobs(L.d_parts, nbk, t, m, jy, 1, st));
  }
  for (int s = 0; s + 1 < L.Lmax; ++s) {
    const int nbk = L.active_back[s];
    DM_LAUNCH(pf, st, K_BACK_FACTOR, L.c_back[s], nbk,
              launch_oz_step(2, L.d_parts, nbk, s, m, out, lexp[2], r0exp[2], r1exp[2], maps[2], L.d_err, st));
    OzSliceJobs jb;
    jb.job[0] = job(out.ZL, Z.ZLT, Z.eZLT, 6);
    jb.job[1] = job(out.ZR, Z.ZRT, Z.eZRT, 7);
    Cost c3 = cs;
    c3.bytes *= 2.0 * nbk;
    DM_LAUNCH(pf, st, K_TC_CONVERT, c3, nbk, launch_oz_slice_jobs(L.d_parts, nbk, s, m, jb, 2, st));
  }
}

// Forward and backward spike sweeps, assembly, and the factorisation of the
// supplementary level (recursively).  A, B, C must hold the level's blocks.
template <typename T>
static void factor_level_t(Level& L, cudaStream_t st, Prof& pf, Aux* aux) {
  T* G = static_cast<T*>(L.G);
  T* Ac = static_cast<T*>(L.Acal);
  T* ZL = static_cast<T*>(L.ZL);
  T* ZR = static_cast<T*>(L.ZR);
  // With a side stream, the left-spike tiles of step t (type 1) run there,
  // overlapping the next inversion, which depends only on the type-0 tiles.
  if constexpr (std::is_same<T, double>::value) {
    if (L.oz.on) {
      factor_level_oz(L, st, pf);
      if (L.supp && L.oz.asm_on) {
        const bool bh = L.oz.band && *L.oz.band_host <= kBandMax;
        DM_LAUNCH_K(pf, st, K_ASSEMBLE_H, bh ? Cost() : L.c_asm_h, L.nseps, 3,
                    launch_oz_assemble(L.d_seps, L.nseps, L.max_m, L.B, L.C, ZL, ZR, L.supp->A, L.supp->B, L.supp->C,
                                       L.oz.as, L.oz.eA, L.oz.maps[1], L.d_err, L.oz.band, st));
        if (L.oz.band) {  // the supplementary blocks when A and C are banded
          Cost cb;
          if (bh) {
            cb.flops = (double)L.nseps * 4 * 2.0 * L.max_m * L.max_m * (2 * *L.oz.band_host + 1);
            cb.bytes = (double)L.nseps * 4 * 24.0 * L.max_m * L.max_m;
          }
          DM_LAUNCH(pf, st, K_BANDED, cb, L.nseps,
                    launch_band_h(L.d_seps, L.nseps, L.max_m, L.A, L.B, L.C, ZL, ZR, L.supp->A, L.supp->B,
                                  L.supp->C, L.oz.band, st));
        }
      }
      else if (L.supp)
        DM_LAUNCH(pf, st, K_ASSEMBLE_H, L.c_asm_h, L.nseps,
                  launch_assemble_h<T>(L.d_seps, L.nseps, L.max_m, L.A, L.B, L.C, ZL, ZR, L.supp->A, L.supp->B,
                                       L.supp->C, st));
      return;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    if (L.tc2.on) {
      factor_level_tc2(L, st, pf);
      if (L.supp)
        DM_LAUNCH(pf, st, K_ASSEMBLE_H, L.c_asm_h, L.nseps,
                  launch_assemble_h<T>(L.d_seps, L.nseps, L.max_m, L.A, L.B, L.C, ZL, ZR, L.supp->A, L.supp->B,
                                       L.supp->C, st));
      return;
    }
  }
  const bool split = aux && aux->st;
  cudaStream_t sb = split ? aux->st : st;
  if (L.tc_mode >= 0)
    DM_LAUNCH_K(pf, st, K_TC_CONVERT, L.c_cvt, 1, 3,
                (launch_to_f32(L.A, L.A32, L.nblk, st), launch_to_f32(L.B, L.B32, L.nblk, st),
                 launch_to_f32(L.C, L.C32, L.nblk, st)));
  // block products on the tensor cores (float32 levels with a tensor mode) or CUDA cores
  auto fwd = [&](int np, int t, cudaStream_t s, int lo, int hi) {
    if constexpr (std::is_same<T, float>::value) {
      if (L.tc_mode >= 0) {
        launch_fwd_factor_tc(L.tc_mode, L.d_parts, np, t, L.max_m, L.A32, L.B32, L.C32, G, Ac, ZL, ZR, L.d_err, s,
                             lo, hi, L.has_tma ? L.tmaps : nullptr);
        return;
      }
    }
    launch_fwd_factor<T>(L.d_parts, np, t, L.max_m, L.A, L.B, L.C, G, Ac, ZL, ZR, s, lo, hi);
  };
  auto back = [&](int np, int s) {
    if constexpr (std::is_same<T, float>::value) {
      if (L.tc_mode >= 0) {
        launch_back_factor_tc(L.tc_mode, L.d_parts, np, s, L.max_m, Ac, ZL, ZR, L.d_err, st,
                              L.has_tma ? L.tmaps : nullptr);
        return;
      }
    }
    launch_back_factor<T>(L.d_parts, np, s, L.max_m, Ac, ZL, ZR, st);
  };
  if (split) {
    cudaEventRecord(aux->ev_main, st);
    cudaStreamWaitEvent(sb, aux->ev_main, 0);
  }
  for (int t = 0; t < L.Lmax; ++t) {
    const int np = L.active_fwd[t];
    DM_LAUNCH(pf, st, K_INV, L.c_inv[t], np, launch_inv<T>(L.d_parts, np, t, L.B, G, L.status, L.max_m, st));
    if (split) {
      cudaEventRecord(aux->ev_main, st);
      cudaStreamWaitEvent(sb, aux->ev_main, 0);
      Cost c0 = L.c_fwd[t], c1 = L.c_fwd[t];
      c0.flops *= L.fwd_chain_frac[t];
      c0.bytes *= L.fwd_chain_frac[t];
      c1.flops -= c0.flops;
      c1.bytes -= c0.bytes;
      DM_LAUNCH(pf, st, K_FWD_FACTOR, c0, np, fwd(np, t, st, 0, 1));
      DM_LAUNCH(pf, sb, K_FWD_FACTOR, c1, np, fwd(np, t, sb, 1, 2));
    } else {
      DM_LAUNCH(pf, st, K_FWD_FACTOR, L.c_fwd[t], np, fwd(np, t, st, 0, 2));
    }
  }
  if (split) {
    cudaEventRecord(aux->ev_aux, sb);
    cudaStreamWaitEvent(st, aux->ev_aux, 0);
  }
  for (int s = 0; s + 1 < L.Lmax; ++s)
    DM_LAUNCH(pf, st, K_BACK_FACTOR, L.c_back[s], L.active_back[s], back(L.active_back[s], s));
  if (L.supp)
    DM_LAUNCH(pf, st, K_ASSEMBLE_H, L.c_asm_h, L.nseps,
              launch_assemble_h<T>(L.d_seps, L.nseps, L.max_m, L.A, L.B, L.C, ZL, ZR, L.supp->A, L.supp->B,
                                   L.supp->C, st));
}

void factor_level(Level& L, cudaStream_t st, Prof& pf, Aux* aux) {
  cudaMemsetAsync(L.status, 0x7f, std::max(1, L.nsys) * sizeof(int), st);
  cudaMemsetAsync(L.d_err, 0, sizeof(int), st);
  pf.depth = L.depth;
  if (L.f32)
    factor_level_t<float>(L, st, pf, aux);
  else
    factor_level_t<double>(L, st, pf, aux);
  if (L.supp) factor_level(*L.supp, st, pf, aux);
  pf.depth = L.depth;
}

// Solve with resident factors: F -> X for every system of the level.
template <typename T>
static void solve_level_t(Level& L, const double* F, double* X, cudaStream_t st, Prof& pf) {
  T* z = static_cast<T*>(L.z);
  const T* G = static_cast<const T*>(L.G);
  const T* Ac = static_cast<const T*>(L.Acal);
  if (L.sweep) {
    Cost c;
    for (int t = 0; t < L.Lmax; ++t) c.flops += L.c_fwds[t].flops + L.c_backs[t].flops,
                                     c.bytes += L.c_fwds[t].bytes + L.c_backs[t].bytes;
    DM_LAUNCH(pf, st, K_SWEEP_SOLVE, c, L.nparts,
              launch_sweep_solve<T>(L.d_parts, L.nparts, L.sweep_cs, L.max_m, L.max_r, L.A, G, Ac, F, z, st));
  } else {
    for (int t = 0; t < L.Lmax; ++t)
      DM_LAUNCH(pf, st, K_FWD_SOLVE, L.c_fwds[t], L.active_fwd[t],
                launch_fwd_solve<T>(L.d_parts, L.active_fwd[t], t, L.max_m, L.max_r, L.A, G, F, z, st));
    for (int s = 0; s + 1 < L.Lmax; ++s)
      DM_LAUNCH(pf, st, K_BACK_SOLVE, L.c_backs[s], L.active_back[s],
                launch_back_solve<T>(L.d_parts, L.active_back[s], s, L.max_m, L.max_r, Ac, z, st));
  }
  if (L.supp) {
    DM_LAUNCH(pf, st, K_ASSEMBLE_F, L.c_asm_f, L.nseps,
              launch_assemble_f<T>(L.d_seps, L.nseps, L.max_m, L.max_r, L.A, L.C, F, z, L.supp->F, st));
    solve_level(*L.supp, L.supp->F, L.supp->X, st, pf);
    pf.depth = L.depth;
  }
  DM_LAUNCH(pf, st, K_BACKSUB, L.c_backsub, L.nparts,
            launch_backsub<T>(L.d_parts, L.nparts, L.Lmax, L.max_m, L.max_r, static_cast<const T*>(L.ZL),
                              static_cast<const T*>(L.ZR), z, L.supp ? L.supp->X : nullptr, X, st));
  if (L.supp)
    DM_LAUNCH(pf, st, K_SEP_COPY, L.c_sepcopy, L.nseps,
              launch_sep_copy(L.d_seps, L.nseps, L.max_m, L.max_r, L.supp->X, X, st));
}

void solve_level(Level& L, const double* F, double* X, cudaStream_t st, Prof& pf) {
  pf.depth = L.depth;
  if (L.f32)
    solve_level_t<float>(L, F, X, st, pf);
  else
    solve_level_t<double>(L, F, X, st, pf);
}

// first failing block row per system (host check after a factorisation)
static int check_status(Level& L, cudaStream_t st, int depth) {
  std::vector<int> h(std::max(1, L.nsys));
  int herr = 0;
  DM_CUDA(cudaMemcpyAsync(h.data(), L.status, h.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  DM_CUDA(cudaMemcpyAsync(&herr, L.d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DM_CUDA(cudaStreamSynchronize(st));
  if (herr) return set_error(DM_ETIMEOUT, "a tensor-core wait expired at level %d", depth);
  for (int s = 0; s < L.nsys; ++s)
    if (h[s] != 0x7f7f7f7f)
      return set_error(DM_ESINGULAR, "singular pivot: level %d, system %d, block row %d (0-based)", depth, s,
                       h[s] - 1);
  if (L.supp) return check_status(*L.supp, st, depth + 1);
  return DM_OK;
}

// algorithmic flops (2 per multiply-add) of the level's factor and solve kernels
void level_flops(const Level& L, double* ffac, double* fsol) {
  double f = 0, g = 0;
  for (const PartDesc& p : L.parts) {
    const double m3 = 2.0 * p.m * (double)p.m * p.m, m2r = 2.0 * p.m * (double)p.m * p.r;
    const bool hl = p.flags & HAS_LEFT, hr = p.flags & HAS_RIGHT;
    f += p.L * m3;                                   // inversions
    f += (p.L - 1) * m3 * 2 + (hr ? m3 : 0);         // Acal and D, right-spike bottom block
    if (hl) f += p.L * m3 + (p.L - 1) * m3;          // left spike forward
    if (hl) f += (p.L - 1) * m3;                     // left spike backward
    if (hr) f += (p.L - 1) * m3;                     // right spike backward
    g += p.L * m2r + (p.L - 1) * m2r + (p.L - 1) * m2r;  // z forward and backward
    g += ((hl ? 1 : 0) + (hr ? 1 : 0)) * p.L * m2r;       // back-substitution
  }
  for (const SepDesc& s : L.seps) {
    const double m3 = 2.0 * s.m * (double)s.m * s.m, m2r = 2.0 * s.m * (double)s.m * s.r;
    f += 2 * m3 + ((s.flags & HAS_HA) ? m3 : 0) + ((s.flags & HAS_HC) ? m3 : 0);
    g += 2 * m2r;
  }
  if (L.supp) {
    double a, b;
    level_flops(*L.supp, &a, &b);
    f += a;
    g += b;
  }
  *ffac = f;
  *fsol = g;
}

// ---------------------------------------------------------------------------
bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copy between device memory and page-locked host memory by a kernel that
// reads (or writes) the host buffer through its device mapping: on a
// coherent CPU-GPU link this runs at the link's bandwidth (measured about
// 210 GB/s on GB300), where the copy engines reached about 25 GB/s.
__global__ void k_copy_mapped(uint4* __restrict__ dst, const uint4* __restrict__ src, long long n16) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
}

// Device address of page-locked, mapped host memory (nullptr otherwise).
static void* mapped_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

static int copy_mapped(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  const size_t n16 = bytes / 16, tail = bytes - n16 * 16;
  if (n16) {
    const int grid = (int)std::min<size_t>((n16 + 255) / 256, 152 * 8);
    k_copy_mapped<<<grid, 256, 0, st>>>(static_cast<uint4*>(dst), static_cast<const uint4*>(src), (long long)n16);
    DM_CUDA(cudaGetLastError());
  }
  if (tail)
    DM_CUDA(cudaMemcpyAsync(static_cast<char*>(dst) + n16 * 16, static_cast<const char*>(src) + n16 * 16, tail,
                            cudaMemcpyDefault, st));
  return DM_OK;
}

static bool aligned16(const void* a, const void* b) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return DM_OK;
  if (is_device_ptr(src)) {
    DM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
    return DM_OK;
  }
  void* ms = mapped_host(src);
  if (ms && aligned16(dst, ms)) return copy_mapped(dst, ms, bytes, st);
  DM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
  return DM_OK;
}

int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return DM_OK;
  if (is_device_ptr(dst)) {
    DM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
    return DM_OK;
  }
  void* md = mapped_host(dst);
  if (md && aligned16(md, src)) return copy_mapped(md, src, bytes, st);
  DM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
  return DM_OK;
}

template <typename F>
int Plan::run(GraphCache& g, F&& body) {
  cudaStream_t st = stream;
  if (prof.on || !use_graphs || g.broken || g.uses == 0) {
    const long long l0 = prof.launches;
    body();
    if (g.uses == 0) g.launches = prof.launches - l0;
    ++g.uses;
    DM_CUDA(cudaGetLastError());
    return DM_OK;
  }
  if (!g.exec) {
    const long long l0 = prof.launches;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      g.broken = true;
      return run(g, body);
    }
    body();
    prof.launches = l0;  // the capture itself launches nothing
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &gr);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, gr, 0);
    if (e == cudaSuccess) {
      // a replay launches exactly the graph's kernel nodes (a call that
      // issues several kernels counted as one in the eager run)
      size_t nn = 0;
      if (cudaGraphGetNodes(gr, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(gr, nodes.data(), &nn) == cudaSuccess) {
          long long k = 0;
          for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++k;
          }
          g.launches = k;
        }
      }
      cudaGetLastError();
    }
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g.exec = nullptr;
      g.broken = true;
      return run(g, body);
    }
  }
  DM_CUDA(cudaGraphLaunch(g.exec, st));
  prof.launches += g.launches;
  ++g.uses;
  return DM_OK;
}

int Plan::init(const std::vector<SysSpec>& specs, int prec) {
  precision = prec;
  DM_CUDA(cudaGetDevice(&device));
  top.lazy_inputs = true;
  top.fp64_fma = !specs.empty() && (specs[0].flags & DM_PLAN_FP64_FMA) != 0;
  top.inv_column = !specs.empty() && (specs[0].flags & DM_PLAN_FP64_INV_COLUMN) != 0;
  int rc = top.build(specs, prec != DM_FP64, prec == DM_TF32 ? 0 : (prec == DM_BF16X3 ? 1 : -1));
  if (rc) return rc;
  {
    // admission: refuse cleanly, before allocating anything, when the device
    // lacks the plan's footprint plus a reserve
    size_t free_b = 0, total_b = 0;
    DM_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t need = top.bytes_needed() - 3 * top.nblk * sizeof(double) + 2 * top.nvec * sizeof(double);
    const size_t reserve = std::min<size_t>(total_b / 64, size_t(1) << 30);
    if (need + reserve > free_b)
      return set_error(DM_ENOMEM, "admission refused: plan needs %zu bytes, %zu free (reserve %zu)", need, free_b,
                       reserve);
  }
  DM_CUDA(cudaStreamCreateWithFlags(&own_stream, cudaStreamNonBlocking));
  stream = own_stream;
  DM_CUDA(cudaStreamCreateWithFlags(&aux.st, cudaStreamNonBlocking));
  DM_CUDA(cudaEventCreateWithFlags(&aux.ev_main, cudaEventDisableTiming));
  DM_CUDA(cudaEventCreateWithFlags(&aux.ev_aux, cudaEventDisableTiming));
  rc = top.allocate();
  if (rc) return rc;
  auto alloc = [&](void** p, size_t bytes) -> int {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(DM_ENOMEM, "cudaMalloc(%zu bytes) failed", bytes);
    }
    return DM_OK;
  };
  if ((rc = alloc((void**)&R, top.nvec * sizeof(double)))) return rc;
  if ((rc = alloc((void**)&Dx, top.nvec * sizeof(double)))) return rc;
  if ((rc = alloc((void**)&nrm, (size_t)std::max(1, top.nsys) * 4 * kMaxR * sizeof(double)))) return rc;
  {
    long long rows = 0;
    for (const SysDesc& d : top.sysd) rows += (long long)d.N * d.m;
    if ((rc = alloc((void**)&rowhi, (size_t)std::max(1ll, rows) * sizeof(unsigned)))) return rc;
    if ((rc = alloc((void**)&colhi, (size_t)std::max(1, top.nrows) * 16 * sizeof(unsigned)))) return rc;
  }
  h_nrm.assign((size_t)std::max(1, top.nsys) * 4 * kMaxR, 0.0);
  relres.assign(std::max(1, top.nsys), 0.0);
  {
    // mixed precision refines with many residuals: tensor cores by default;
    // DM_RESIDUAL=fp64 / sliced overrides (for comparisons)
    int mode = prec == DM_FP64 ? DM_RESIDUAL_FP64 : DM_RESIDUAL_AUTO;
    const char* e = std::getenv("DM_RESIDUAL");
    if (e && std::string(e) == "fp64") mode = DM_RESIDUAL_FP64;
    if (e && std::string(e) == "sliced") mode = DM_RESIDUAL_SLICED;
    if (e && std::string(e) == "auto") mode = DM_RESIDUAL_AUTO;
    if ((rc = set_residual_mode(mode))) return rc;
  }
  level_flops(top, &factor_flops, &solve_flops);
  device_bytes = top.bytes_needed() - 3 * top.nblk * sizeof(double) + 2 * top.nvec * sizeof(double);
  return DM_OK;
}

Plan::~Plan() {
  for (void* p : cbuf) cudaFree(p);
  if (R) cudaFree(R);
  if (Dx) cudaFree(Dx);
  if (nrm) cudaFree(nrm);
  if (rowhi) cudaFree(rowhi);
  if (colhi) cudaFree(colhi);
  reset_graphs();
  if (own_stream) cudaStreamDestroy(own_stream);
  if (aux.st) cudaStreamDestroy(aux.st);
  if (aux.ev_main) cudaEventDestroy(aux.ev_main);
  if (aux.ev_aux) cudaEventDestroy(aux.ev_aux);
}

void Plan::reset_graphs() {
  for (GraphCache* g : {&g_factor, &g_solve, &g_iter_first, &g_iter_next}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    *g = GraphCache();
  }
}

int Plan::factor(const double* A, const double* B, const double* C) {
  cudaStream_t st = stream;
  int rc;
  if (borrow) {
    if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C))
      return set_error(DM_EINVAL, "a plan that borrows its inputs needs device pointers for A, B, C");
    if (A != bA || B != bB || C != bC) {  // captured graphs hold the old addresses
      reset_graphs();
      bA = A, bB = B, bC = C;
    }
    top.A = const_cast<double*>(A);
    top.B = const_cast<double*>(B);
    top.C = const_cast<double*>(C);
  } else {
    if ((rc = top.ensure_inputs())) return rc;
    if ((rc = copy_in(top.A, A, top.nblk * sizeof(double), st))) return rc;
    if ((rc = copy_in(top.B, B, top.nblk * sizeof(double), st))) return rc;
    if ((rc = copy_in(top.C, C, top.nblk * sizeof(double), st))) return rc;
  }
  rc = run(g_factor, [&] {
    factor_level(top, stream, prof, overlap ? &aux : nullptr);
    row_scales();
  });
  if (rc) return rc;
  rc = check_status(top, st, 0);
  factored = (rc == DM_OK);
  return rc;
}

// per-system max over columns of sqrt(num/den) from the device norm array
static double col_ratio(const std::vector<double>& h, int s, int r, int num, int den) {
  double worst = 0.0;
  for (int c = 0; c < r; ++c) {
    const double a = h[(size_t)s * 4 * kMaxR + num * kMaxR + c];
    const double b = h[(size_t)s * 4 * kMaxR + den * kMaxR + c];
    const double q = b > 0 ? std::sqrt(a / b) : std::sqrt(a);
    worst = std::max(worst, q);
  }
  return worst;
}

double Plan::column_relres(int c0, int nc) const {
  double worst = 0.0;
  for (int c = c0; c < c0 + nc && c < kMaxR; ++c) {
    const double a = h_nrm[c], b = h_nrm[kMaxR + c];
    worst = std::max(worst, b > 0 ? std::sqrt(a / b) : std::sqrt(a));
  }
  return worst;
}

// Residual mode: the tensor-core residual for every system it fits (m <= 128,
// nrhs <= 16; SLICED) or for those where it is faster (AUTO), float64 CUDA
// cores for the others (or for all in FP64 mode).
int Plan::set_residual_mode(int mode) {
  if (mode != DM_RESIDUAL_FP64 && mode != DM_RESIDUAL_SLICED && mode != DM_RESIDUAL_AUTO)
    return set_error(DM_EINVAL, "unknown residual mode %d", mode);
  resid_mode = mode;
  top.nres_tc = 0;
  top.c_resid_tc = Cost();
  for (SysDesc& d : top.sysd) {
    const bool fits = residual_sliced_fits(d.m, d.r);
    const bool faster = (long long)d.m * d.m * d.r >= (1ll << 17);
    d.sliced = (fits && (mode == DM_RESIDUAL_SLICED || (mode == DM_RESIDUAL_AUTO && faster))) ? 1 : 0;
    if (d.sliced) {
      const double m2 = (double)d.m * d.m, mr = (double)d.m * d.r;
      ++top.nres_tc;
      top.c_resid_tc.flops += d.N * 6.0 * m2 * d.r;
      top.c_resid_tc.bytes += d.N * (24.0 * m2 + 24.0 * mr);
    }
  }
  if (top.d_sys && !top.sysd.empty())
    DM_CUDA(cudaMemcpy(top.d_sys, top.sysd.data(), top.sysd.size() * sizeof(SysDesc), cudaMemcpyHostToDevice));
  reset_graphs();
  if (factored) {
    row_scales();
    DM_CUDA(cudaStreamSynchronize(stream));
  }
  return DM_OK;
}

void Plan::residual(const double* x_dev, const double* b_dev, double* r_dev) {
  Cost c64 = top.c_resid;
  c64.flops -= top.c_resid_tc.flops;
  c64.bytes -= top.c_resid_tc.bytes;
  if (top.oz.band && *top.oz.band_host <= kBandMax) {
    // banded A, C: 2 m^2 r (B) + 4 (2w + 1) m r flops and B plus the bands read per row
    const double m = top.max_m, w = *top.oz.band_host, f = (2.0 * m * m + 4.0 * (2 * w + 1) * m) / (6.0 * m * m);
    c64.flops *= f;
    c64.bytes *= (m * m + 2 * (2 * w + 1) * m + 3 * m) / (3.0 * m * m + 3 * m);
  }
  if (top.nsys > top.nres_tc)
    DM_LAUNCH(prof, stream, K_RESIDUAL, c64, top.nsys - top.nres_tc,
              launch_residual(top.d_sys, top.nsys, top.nrows, top.max_m, top.max_r, top.A, top.B, top.C, x_dev,
                              b_dev, r_dev, nrm, stream, top.oz.band));
  if (top.nres_tc > 0) {
    DM_LAUNCH(prof, stream, K_RESIDUAL, Cost(), top.nres_tc,
              launch_col_scales(top.d_sys, top.nsys, top.nrows, x_dev, colhi, stream));
    DM_LAUNCH(prof, stream, K_RESIDUAL, top.c_resid_tc, top.nres_tc,
              launch_residual_sliced(top.d_sys, top.nsys, top.nrows, top.A, top.B, top.C, x_dev, b_dev, r_dev, nrm,
                                     rowhi, colhi, top.d_err, stream));
  }
}

void Plan::row_scales() {
  if (top.nres_tc > 0)
    DM_LAUNCH(prof, stream, K_RESIDUAL, Cost(), top.nres_tc,
              launch_row_scales(top.d_sys, top.nsys, top.nrows, top.A, top.B, top.C, rowhi, stream));
}

// after a synchronisation: a tensor-core residual whose bounded wait expired
int Plan::check_residual_error() {
  if (top.nres_tc == 0) return DM_OK;
  int herr = 0;
  DM_CUDA(cudaMemcpyAsync(&herr, top.d_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  DM_CUDA(cudaStreamSynchronize(stream));
  if (herr) return set_error(DM_ETIMEOUT, "a tensor-core residual wait expired");
  return DM_OK;
}

int Plan::solve_device(const double* b_dev, double* x_dev) {
  cudaStream_t st = stream;
  const size_t nb = (size_t)std::max(1, top.nsys) * 4 * kMaxR * sizeof(double);
  if (precision == DM_FP64) {
    auto body = [&] {
      solve_level(top, b_dev, x_dev, stream, prof);
      cudaMemsetAsync(nrm, 0, nb, stream);
      residual(x_dev, b_dev, R);
    };
    int rc0 = (b_dev == top.F && x_dev == top.X) ? run(g_solve, body) : (body(), DM_OK);
    if (rc0) return rc0;
    DM_CUDA(cudaGetLastError());
    DM_CUDA(cudaMemcpyAsync(h_nrm.data(), nrm, nb, cudaMemcpyDeviceToHost, st));
    DM_CUDA(cudaStreamSynchronize(st));
    if ((rc0 = check_residual_error())) return rc0;
    last_iters = 1;
    last_corr = 0.0;
    for (int s = 0; s < top.nsys; ++s) relres[s] = col_ratio(h_nrm, s, top.spec[s].r, 0, 1);
    return DM_OK;
  }
  // iterative refinement: x_0 = 0, r_0 = b; x_{i+1} = x_i + M^{-1} r_i with
  // M^{-1} the float32-factor DM solve; r in float64.
  DM_CUDA(cudaMemsetAsync(x_dev, 0, top.nvec * sizeof(double), st));
  const double* rhs = b_dev;
  int rc = DM_ENOTCONV;
  int it = 0;
  double corr = 0.0;
  for (it = 1; it <= max_iters; ++it) {
    auto body = [&] {
      solve_level(top, rhs, Dx, stream, prof);
      cudaMemsetAsync(nrm, 0, nb, stream);
      DM_LAUNCH(prof, stream, K_AXPY, top.c_axpy, top.nsys,
                launch_axpy_norms(top.d_sys, top.nsys, top.nrows, top.max_m, top.max_r, Dx, x_dev, nrm, stream));
      residual(x_dev, b_dev, R);
    };
    int rc0 = (b_dev == top.F && x_dev == top.X) ? run(it == 1 ? g_iter_first : g_iter_next, body) : (body(), DM_OK);
    if (rc0) return rc0;
    DM_CUDA(cudaGetLastError());
    DM_CUDA(cudaMemcpyAsync(h_nrm.data(), nrm, nb, cudaMemcpyDeviceToHost, st));
    DM_CUDA(cudaStreamSynchronize(st));
    if ((rc0 = check_residual_error())) return rc0;
    rhs = R;
    corr = 0.0;
    bool bad = false;
    for (int s = 0; s < top.nsys; ++s) {
      const double c = col_ratio(h_nrm, s, top.spec[s].r, 2, 3);
      corr = std::max(corr, c);
      relres[s] = col_ratio(h_nrm, s, top.spec[s].r, 0, 1);
      if (!std::isfinite(c) || !std::isfinite(relres[s])) bad = true;
    }
    if (bad) {
      rc = set_error(DM_ENOTCONV, "refinement diverged (non-finite correction) at iteration %d", it);
      break;
    }
    if (corr <= tol) {
      rc = DM_OK;
      break;
    }
  }
  last_iters = std::min(it, max_iters);
  last_corr = corr;
  if (rc == DM_ENOTCONV && g_last_error.find("refinement") == std::string::npos)
    set_error(DM_ENOTCONV, "refinement stopped after %d iterations: ||dx||/||x|| = %.3e > tol %.1e",
              last_iters, corr, tol);
  return rc;
}

int Plan::solve(const double* b, double* x, double* relres_out) {
  if (!factored) return set_error(DM_ESTATE, "dm_solve before a successful dm_factor");
  cudaStream_t st = stream;
  int rc;
  const size_t vb = top.nvec * sizeof(double);
  if ((rc = copy_in(top.F, b, vb, st))) return rc;
  rc = solve_device(top.F, top.X);
  if (rc != DM_OK && rc != DM_ENOTCONV) return rc;
  int rc2 = copy_out(x, top.X, vb, st);
  if (rc2) return rc2;
  DM_CUDA(cudaStreamSynchronize(st));
  if (relres_out)
    for (int s = 0; s < top.nsys; ++s) relres_out[s] = relres[s];
  return rc;
}

// Last block row only (the application case: b is zero except its last block
// row, only x_N is wanted).  Every z^k vanishes but the last subsystem's,
// whose forward sweep is one step (z_{L-1} = G_{L-1} b_N); its backward sweep
// gives z^{P}[first] for the one non-zero supplementary right-hand side
// fh_{P-1} = -C_q z^{P}[first] (Eq. e2311); after the supplementary solve,
// x_N = z_{L-1} - ZL_{L-1} h_{P-1} (Eq. endSolution).
int Plan::solve_last(const double* b_last, double* x_last) {
  if (!factored) return set_error(DM_ESTATE, "dm_solve_last before a successful dm_factor");
  if (precision != DM_FP64) return set_error(DM_EINVAL, "dm_solve_last needs a float64 plan (no refinement)");
  if (top.nsys != 1) return set_error(DM_EINVAL, "dm_solve_last needs a single-system plan");
  cudaStream_t st = stream;
  const SysSpec& sp = top.spec[0];
  const long long mr = (long long)sp.m * sp.r;
  const int li = top.last_part[0];
  const PartDesc& lp = top.parts[li];
  const PartDesc* dlp = top.d_parts + li;
  DM_CUDA(cudaMemsetAsync(top.F, 0, top.nvec * sizeof(double), st));
  DM_CUDA(cudaMemsetAsync(top.z, 0, top.nvec * sizeof(double), st));
  int rc = copy_in(top.F + (long long)(sp.N - 1) * mr, b_last, mr * sizeof(double), st);
  if (rc) return rc;
  double* z = static_cast<double*>(top.z);
  launch_fwd_solve<double>(dlp, 1, lp.L - 1, top.max_m, top.max_r, top.A, static_cast<const double*>(top.G),
                           top.F, z, st);
  for (int s = 0; s + 1 < lp.L; ++s)
    launch_back_solve<double>(dlp, 1, s, top.max_m, top.max_r, static_cast<const double*>(top.Acal), z, st);
  if (top.supp) {
    Level& S = *top.supp;
    DM_CUDA(cudaMemsetAsync(S.F, 0, S.nvec * sizeof(double), st));
    launch_assemble_f<double>(top.d_seps + (top.nseps - 1), 1, top.max_m, top.max_r, top.A, top.C, top.F, z, S.F, st);
    solve_level(S, S.F, S.X, st, prof);
  }
  launch_backsub<double>(dlp, 1, lp.L, top.max_m, top.max_r, static_cast<const double*>(top.ZL),
                         static_cast<const double*>(top.ZR), z, top.supp ? top.supp->X : nullptr, top.X, st);
  DM_CUDA(cudaGetLastError());
  rc = copy_out(x_last, top.X + (long long)(sp.N - 1) * mr, mr * sizeof(double), st);
  if (rc) return rc;
  DM_CUDA(cudaStreamSynchronize(st));
  return DM_OK;
}

// ---------------------------------------------------------------------------
// partition plan and tuner seeds (Section 2, Section 5)
void partition_plan(int N, int P, std::vector<int>& starts, std::vector<int>& lens, std::vector<int>& seps) {
  starts.clear();
  lens.clear();
  seps.clear();
  const int rows = N - (P - 1);
  const int base = rows / P, extra = rows % P;
  int r = 0;
  for (int k = 0; k < P; ++k) {
    const int L = base + (k < extra ? 1 : 0);
    starts.push_back(r);
    lens.push_back(L);
    r += L;
    if (k < P - 1) seps.push_back(r++);
  }
}

// Subsystem sizes: equal (remainder to the lowest subsystems), or with
// DM_PLAN_EQUAL_TIME equal operation counts per subsystem (Section 5.1, from
// Table 2: first N_1 = a1 N_k + 1/4, last N_M = a2 N_k + b2, middle N_k).
void partition_lengths(int N, int P, int m, int r, int flags, std::vector<int>& lens) {
  std::vector<int> st, sp;
  partition_plan(N, P, st, lens, sp);
  if (!(flags & DM_PLAN_EQUAL_TIME) || P < 2) return;
  const double n3 = (double)m * m * m, n2l = (double)m * m * r;
  const double c = 7.0 * n3 + 5.0 * n2l;
  const double a1 = c / (4.0 * n3 + 4.0 * n2l), b1 = 0.25;
  const double a2 = c / (6.0 * n3 + 4.0 * n2l), b2 = (3.0 * n3 + n2l) / (6.0 * n3 + 4.0 * n2l);
  const int rows = N - P + 1;
  const double nk = (rows - b1 - b2) / (a1 + a2 + P - 2);
  const int n1 = (int)std::floor(a1 * nk + b1 + 0.5), nm = (int)std::floor(a2 * nk + b2 + 0.5);
  const int mid = rows - n1 - nm;
  if (n1 < 1 || nm < 1 || (P > 2 && mid < P - 2) || (P == 2 && mid != 0)) {
    if (P == 2 && n1 >= 1 && rows - n1 >= 1) lens = {n1, rows - n1};
    return;  // else keep equal sizes
  }
  lens.assign(P, 0);
  lens[0] = n1;
  lens[P - 1] = nm;
  if (P > 2) {
    const int base = mid / (P - 2), extra = mid % (P - 2);
    for (int k = 0; k < P - 2; ++k) lens[1 + k] = base + (k < extra ? 1 : 0);
  }
}

// DM inside the subsystems (Section 4.2.2): M subsystems of the equal
// partition, each split into J sub-subsystems by the same rule; the M J
// sub-subsystem lengths in order (an inner separator between the
// sub-subsystems of one subsystem, the outer separators between subsystems).
void nested_lengths(int N, int M, int J, std::vector<int>& lens) {
  std::vector<int> st, Lk, sp, st2, Li, sp2;
  partition_plan(N, M, st, Lk, sp);
  lens.clear();
  for (int k = 0; k < M; ++k) {
    partition_plan(Lk[k], J, st2, Li, sp2);
    lens.insert(lens.end(), Li.begin(), Li.end());
  }
}

// Eq. (MAXSpeedP): P* = sqrt((N+1)/3 (5 + 2/(1 + l/n))), clamped to 1..(N+1)/2.
int tuner_seed_p(int N, int m, int r) {
  const double c = 5.0 + 2.0 / (1.0 + (double)r / m);
  int P = (int)std::lround(std::sqrt((N + 1) / 3.0 * c));
  P = std::max(1, std::min(P, (N + 1) / 2));
  return P;
}

// Eq. (SuppMatrM) with its boundary case m = P/3 when (P - m)/m < 2, clamped so
// that each of the Ms supplementary rows' subsystems keeps at least one row.
int supp_partitions(int Ms, int P, int r, int m) {
  const double c = 5.0 + 2.0 / (1.0 + (double)r / m);
  double p2 = std::sqrt(P / 3.0 * c);
  if ((P - p2) / p2 < 2.0) p2 = P / 3.0;
  int q = (int)std::lround(p2);
  q = std::min(q, (Ms + 1) / 2);
  return std::max(q, 1);
}

int make_spec(int N, int m, int r, int P, int levels, SysSpec* out) {
  if (N < 1 || m < 1 || r < 1) return set_error(DM_EINVAL, "N, m, nrhs must be >= 1 (got %d, %d, %d)", N, m, r);
  if (m > kMaxM) return set_error(DM_EINVAL, "block size m = %d exceeds the limit %d", m, kMaxM);
  if (r > kMaxR) return set_error(DM_EINVAL, "nrhs = %d exceeds the limit %d", r, kMaxR);
  if (P < 0 || levels < 0) return set_error(DM_EINVAL, "P and levels must be >= 0");
  if (P == 0) P = tuner_seed_p(N, m, r);
  if (P > 1 && 2 * P - 1 > N)
    return set_error(DM_EINVAL, "P = %d too large for N = %d: every subsystem needs >= 1 row (P <= (N+1)/2)", P, N);
  if (levels == 0) {
    // Section 5.2.1: DM on the supplementary system pays from P >= 21.  On the
    // GPU a level's block Thomas chain is latency-bound (one block at a time),
    // so a third level pays as soon as the second has P2 >= 8 subsystems
    // (measured: 2-10 % per step on the PDE-shaped and conditioned workloads).
    levels = (P >= 21) ? 2 : 1;
    if (levels == 2 && supp_partitions(P - 1, P, r, m) >= 8) levels = 3;
  }
  SysSpec s;
  s.N = N;
  s.m = m;
  s.r = r;
  s.P = P;
  s.levels = levels;
  s.P2 = 1;
  if (P > 1 && levels > 1) s.P2 = supp_partitions(P - 1, P, r, m);
  if (s.P2 <= 1) s.levels = (P > 1 ? std::min(levels, 1) : levels), s.P2 = 1;
  if (P == 1) s.levels = 1;
  *out = s;
  return DM_OK;
}

}  // namespace dm

// ===========================================================================
// extern "C" entry points
using namespace dm;

extern "C" {

const char* dm_last_error(void) { return g_last_error.c_str(); }

int dm_plan(dm_plan_t* out, int N, int m, int nrhs, int P, int levels, int precision) {
  return dm_plan_ex(out, N, m, nrhs, P, levels, precision, 0);
}

int dm_partition_sizes(int N, int m, int nrhs, int P, int flags, int* lengths) {
  if (!lengths) return set_error(DM_EINVAL, "NULL lengths");
  if (flags & ~(DM_PLAN_EQUAL_TIME | DM_PLAN_FP64_FMA | DM_PLAN_FP64_INV_COLUMN))
    return set_error(DM_EINVAL, "unknown plan flags 0x%x", flags);
  SysSpec s;
  int rc = make_spec(N, m, nrhs, P, 1, &s);
  if (rc) return rc;
  std::vector<int> L;
  partition_lengths(N, s.P, m, nrhs, flags, L);
  for (int k = 0; k < s.P; ++k) lengths[k] = L[k];
  return DM_OK;
}

int dm_plan_ex(dm_plan_t* out, int N, int m, int nrhs, int P, int levels, int precision, int flags) {
  if (!out) return set_error(DM_EINVAL, "out is NULL");
  if (flags & ~(DM_PLAN_EQUAL_TIME | DM_PLAN_FP64_FMA | DM_PLAN_FP64_INV_COLUMN))
    return set_error(DM_EINVAL, "unknown plan flags 0x%x", flags);
  if (precision != DM_FP64 && precision != DM_FP32 && precision != DM_TF32 && precision != DM_BF16X3)
    return set_error(DM_EINVAL, "unknown precision %d", precision);
  if ((precision == DM_TF32 || precision == DM_BF16X3) && m > kMaxMTensor)
    return set_error(DM_EINVAL, "tensor-core precisions support m <= %d", kMaxMTensor);
  if (P == 0 && levels == 0) {  // the measured choice, if any, with its kernel variant
    int tf = 0;
    if (tuned_lookup(N, m, nrhs, precision, &P, &levels, &tf) && !(flags & (DM_PLAN_FP64_FMA | DM_PLAN_FP64_INV_COLUMN)))
      flags |= tf;
  }
  SysSpec s;
  int rc = make_spec(N, m, nrhs, P, levels, &s);
  if (rc) return rc;
  s.flags = flags;
  std::unique_ptr<dm_plan_s> p(new dm_plan_s());
  rc = p->plan.init(std::vector<SysSpec>{s}, precision);
  if (rc) return rc;
  *out = p.release();
  return DM_OK;
}

int dm_plan_inside(dm_plan_t* out, int N, int m, int nrhs, int M, int J, int outer_levels, int precision) {
  if (!out) return set_error(DM_EINVAL, "out is NULL");
  if (precision != DM_FP64 && precision != DM_FP32 && precision != DM_TF32 && precision != DM_BF16X3)
    return set_error(DM_EINVAL, "unknown precision %d", precision);
  if ((precision == DM_TF32 || precision == DM_BF16X3) && m > kMaxMTensor)
    return set_error(DM_EINVAL, "tensor-core precisions support m <= %d", kMaxMTensor);
  if (N < 1 || m < 1 || nrhs < 1 || m > kMaxM || nrhs > kMaxR)
    return set_error(DM_EINVAL, "invalid sizes N = %d, m = %d, nrhs = %d", N, m, nrhs);
  if (M < 1 || J < 2 || (outer_levels != 1 && outer_levels != 2))
    return set_error(DM_EINVAL, "dm_plan_inside needs M >= 1, J >= 2, outer_levels 1 or 2");
  if (M > 1 && 2 * M - 1 > N) return set_error(DM_EINVAL, "M = %d too large for N = %d", M, N);
  {
    std::vector<int> st, Lk, sp;
    partition_plan(N, M, st, Lk, sp);
    const int Lmin = *std::min_element(Lk.begin(), Lk.end());
    if (2 * J - 1 > Lmin)
      return set_error(DM_EINVAL, "J = %d too large: the shortest subsystem has %d rows (needs >= 2J - 1)", J, Lmin);
  }
  SysSpec s;
  s.N = N;
  s.m = m;
  s.r = nrhs;
  s.P = M * J;
  s.J = J;
  s.P2 = M;
  s.levels = M > 1 ? 1 + outer_levels : 2;
  std::unique_ptr<dm_plan_s> p(new dm_plan_s());
  int rc = p->plan.init(std::vector<SysSpec>{s}, precision);
  if (rc) return rc;
  *out = p.release();
  return DM_OK;
}

int dm_plan_batch(dm_plan_t* out, int count, const int* N, const int* m, const int* nrhs, int precision) {
  if (!out || count < 1 || !N || !m || !nrhs) return set_error(DM_EINVAL, "invalid batch arguments");
  if (precision != DM_FP64 && precision != DM_FP32 && precision != DM_TF32 && precision != DM_BF16X3)
    return set_error(DM_EINVAL, "unknown precision %d", precision);
  std::vector<SysSpec> specs(count);
  for (int s = 0; s < count; ++s) {
    if ((precision == DM_TF32 || precision == DM_BF16X3) && m[s] > kMaxMTensor)
      return set_error(DM_EINVAL, "tensor-core precisions support m <= %d", kMaxMTensor);
    int rc = make_spec(N[s], m[s], nrhs[s], 0, 0, &specs[s]);
    if (rc) return rc;
  }
  std::unique_ptr<dm_plan_s> p(new dm_plan_s());
  int rc = p->plan.init(specs, precision);
  if (rc) return rc;
  *out = p.release();
  return DM_OK;
}

int dm_plan_tune(int N, int m, int nrhs, int* P, int* levels, int* P2) {
  if (!P || !levels || !P2) return set_error(DM_EINVAL, "NULL argument to dm_plan_tune");
  SysSpec s;
  int rc = make_spec(N, m, nrhs, *P, *levels, &s);
  if (rc) return rc;
  *P = s.P;
  *levels = s.levels;
  *P2 = s.P2;
  return DM_OK;
}

int dm_factor(dm_plan_t plan, const double* A, const double* B, const double* C) {
  if (!plan || !A || !B || !C) return set_error(DM_EINVAL, "NULL argument to dm_factor");
  return plan->plan.factor(A, B, C);
}

int dm_solve(dm_plan_t plan, const double* b, double* x, double* relres_out) {
  if (!plan || !b || !x) return set_error(DM_EINVAL, "NULL argument to dm_solve");
  return plan->plan.solve(b, x, relres_out);
}

int dm_solve_last(dm_plan_t plan, const double* b_last, double* x_last) {
  if (!plan || !b_last || !x_last) return set_error(DM_EINVAL, "NULL argument to dm_solve_last");
  return plan->plan.solve_last(b_last, x_last);
}

int dm_set_stream(dm_plan_t plan, void* cuda_stream) {
  if (!plan) return set_error(DM_EINVAL, "NULL plan");
  plan->plan.stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : plan->plan.own_stream;
  return DM_OK;
}

int dm_set_side_stream(dm_plan_t plan, int enable) {
  if (!plan) return set_error(DM_EINVAL, "NULL plan");
  if (plan->plan.overlap != (enable != 0)) plan->plan.reset_graphs();
  plan->plan.overlap = enable != 0;
  return DM_OK;
}

int dm_set_borrow_inputs(dm_plan_t plan, int enable) {
  if (!plan) return set_error(DM_EINVAL, "NULL plan");
  Plan& p = plan->plan;
  if (!enable) return p.borrow ? set_error(DM_ESTATE, "borrowing cannot be switched off") : DM_OK;
  if (p.borrow) return DM_OK;
  if (p.top.A) {
    p.top.release(p.top.A);
    p.top.release(p.top.B);
    p.top.release(p.top.C);
    p.top.A = p.top.B = p.top.C = nullptr;
  }
  p.borrow = true;
  p.factored = false;
  return DM_OK;
}

int dm_set_refinement(dm_plan_t plan, double tol, int max_iters) {
  if (!plan || !(tol > 0) || max_iters < 1) return set_error(DM_EINVAL, "invalid refinement settings");
  plan->plan.tol = tol;
  plan->plan.max_iters = max_iters;
  return DM_OK;
}

int dm_plan_query(dm_plan_t plan, dm_plan_info* info) {
  if (!plan || !info) return set_error(DM_EINVAL, "NULL argument to dm_plan_query");
  const Plan& p = plan->plan;
  const SysSpec& s = p.top.spec[0];
  info->N = s.N;
  info->m = s.m;
  info->nrhs = s.r;
  info->P = s.P;
  info->levels = s.levels;
  info->P2 = s.P2;
  info->precision = p.precision;
  info->count = p.top.nsys;
  info->last_iters = p.last_iters;
  info->max_rows = p.top.Lmax;
  info->device_bytes = p.device_bytes;
  info->last_relres = 0;
  for (int i = 0; i < p.top.nsys; ++i) info->last_relres = std::max(info->last_relres, p.relres[i]);
  info->last_correction = p.last_corr;
  info->factor_flops = p.factor_flops;
  info->solve_flops = p.solve_flops;
  info->residual_mode = p.resid_mode;
  info->residual_tc_systems = p.top.nres_tc;
  info->J = s.J;
  return DM_OK;
}

int dm_set_residual(dm_plan_t plan, int mode) {
  if (!plan) return set_error(DM_EINVAL, "NULL plan");
  serve_drain(plan);
  return plan->plan.set_residual_mode(mode);
}

int dm_residual(dm_plan_t plan, const double* x, const double* b, double* r, double* relres_out) {
  if (!plan || !x || !b || !r) return set_error(DM_EINVAL, "NULL argument to dm_residual");
  Plan& p = plan->plan;
  if (!p.factored) return set_error(DM_ESTATE, "dm_residual before a successful dm_factor");
  const size_t vb = p.top.nvec * sizeof(double);
  const size_t nb = (size_t)std::max(1, p.top.nsys) * 4 * kMaxR * sizeof(double);
  int rc;
  if ((rc = copy_in(p.Dx, x, vb, p.stream))) return rc;
  if ((rc = copy_in(p.top.F, b, vb, p.stream))) return rc;
  DM_CUDA(cudaMemsetAsync(p.nrm, 0, nb, p.stream));
  p.residual(p.Dx, p.top.F, p.R);
  DM_CUDA(cudaGetLastError());
  if ((rc = copy_out(r, p.R, vb, p.stream))) return rc;
  DM_CUDA(cudaMemcpyAsync(p.h_nrm.data(), p.nrm, nb, cudaMemcpyDeviceToHost, p.stream));
  DM_CUDA(cudaStreamSynchronize(p.stream));
  if ((rc = p.check_residual_error())) return rc;
  if (relres_out) {
    double worst = 0.0;
    for (int s = 0; s < p.top.nsys; ++s) worst = std::max(worst, col_ratio(p.h_nrm, s, p.top.spec[s].r, 0, 1));
    *relres_out = worst;
  }
  return DM_OK;
}

int dm_profile(dm_plan_t plan, int enable, dm_profile_entry* out, int max_entries, int* n_entries) {
  if (!plan) return set_error(DM_EINVAL, "NULL plan");
  Prof& pf = plan->plan.prof;
  if (out && max_entries > 0) {
    pf.collect();
    int k = 0;
    for (int c = 0; c < K_NCLASS * Prof::kDepths && k < max_entries; ++c) {
      if (pf.n[c] == 0) continue;
      dm_profile_entry& e = out[k++];
      std::memset(e.name, 0, sizeof e.name);
      const int d = c / K_NCLASS;
      if (d == 0)
        std::snprintf(e.name, sizeof e.name, "%s", kClassNames[c % K_NCLASS]);
      else
        std::snprintf(e.name, sizeof e.name, "%s@%d", kClassNames[c % K_NCLASS], d);
      e.launches = pf.n[c];
      e.ms = pf.ms[c];
      e.flops = pf.flops[c];
      e.bytes = pf.bytes[c];
    }
    if (n_entries) *n_entries = k;
  } else if (n_entries) {
    *n_entries = 0;
  }
  pf.reset();
  pf.on = enable != 0;
  return DM_OK;
}

long long dm_launch_count(dm_plan_t plan) { return plan ? plan->plan.prof.launches : -1; }

void dm_destroy(dm_plan_t plan) {
  if (!plan) return;
  serve_drain(plan);  // queued or running serving requests finish first
  delete plan;
}

}  // extern "C"

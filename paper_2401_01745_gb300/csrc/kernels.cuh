// CUDA kernels of the emRKC step (Algorithm 3) and of the power iteration
// (Algorithm 5), templated on the ionic model and on the precision mode.
//
// Data layout in HBM (structure of arrays, leading dimension ld = n rounded
// up to a multiple of 128):
//   V            double[ld]                 (every mode)
//   z block      Z[(N-1) * ld], row k = variable k+1 (Z = double or float)
//   L            sliced ELL, 32-row slices, slot-major inside a slice so that
//                a warp's loads of one slot are contiguous (Ell in launch.h)
// One thread owns one node; all per-node loads and stores are coalesced.
#pragma once

#include <cstdint>
#include <utility>
#include <type_traits>

#include <cuda/atomic>

#include "launch.h"
#include "models.cuh"
#include "rkc_coeffs.h"
#include "dual.cuh"

namespace emrkc {

// ---------------------------------------------------------------------------
// Sparse rows.

// Loads of data that may have been written earlier in the same launch by
// another SM (the persistent batched and fused-step kernels) go through L2
// only (ld.cg): L1 is not coherent across SMs.  Single-step kernels use
// read-only loads (ldm) or plain loads (ldp).
template <bool CG, typename T>
__device__ __forceinline__ T ldm(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return __ldg(p);
}
template <bool CG, typename T>
__device__ __forceinline__ T ldp(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// FP64: sum_k L_ik x_k over the stored row (diagonal included).
template <bool CG = false>
__device__ __forceinline__ double ell_dot64(const Ell& A, int64_t i, const double* __restrict__ x) {
  const int64_t b = i >> 5;
  const int w = __ldg(A.width + b);
  int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
  double acc = 0.0;
  for (int k = 0; k < w; ++k, p += 32) acc += __ldg(A.val + p) * ldm<CG>(x + __ldg(A.col + p));
  return acc;
}

// Mixed: sum_{k != i} L_ik (x_k - x_i) in FP32 (row sums of L vanish, so
// this equals (L x)_i; differences keep the FP32 sum well conditioned).
template <bool CG = false>
__device__ __forceinline__ float ell_diff32(const Ell& A, int64_t i, const float* __restrict__ x) {
  const int64_t b = i >> 5;
  const int w = __ldg(A.width + b);
  int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
  const float xi = ldm<CG>(x + i);
  float acc = 0.0f;
  for (int k = 0; k < w; ++k, p += 32) acc += __ldg(A.val32 + p) * (ldm<CG>(x + __ldg(A.col + p)) - xi);
  return acc;
}

// Split form of ell_diff32 for rows of at most W stored entries: ell_row
// loads the row's columns and values, ell_gather_x issues every neighbour
// load up front (into registers), ell_reduce sums them later, so the loads
// can be in flight while the caller does other work.  Same sum, same order.
template <int W>
__device__ __forceinline__ int ell_row(const Ell& A, int64_t i, int32_t (&c)[W], float (&lv)[W]) {
  const int64_t b = i >> 5;
  const int w = __ldg(A.width + b);
  const int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
#pragma unroll
  for (int k = 0; k < W; ++k) {
    if (k < w) {
      c[k] = __ldg(A.col + p + 32 * k);
      lv[k] = __ldg(A.val32 + p + 32 * k);
    }
  }
  return w;
}

template <int W, bool CG = false>
__device__ __forceinline__ void ell_gather_x(const int32_t (&c)[W], int w, const float* __restrict__ x,
                                             float (&xv)[W]) {
#pragma unroll
  for (int k = 0; k < W; ++k)
    if (k < w) xv[k] = ldm<CG>(x + c[k]);
}

template <int W>
__device__ __forceinline__ float ell_reduce(const float (&xv)[W], const float (&lv)[W], int w, float xi) {
  float acc = 0.0f;
#pragma unroll
  for (int k = 0; k < W; ++k)
    if (k < w) acc += lv[k] * (xv[k] - xi);
  return acc;
}

// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-serialisation attribute may start while its predecessor in the
// stream drains; it must wait (griddepcontrol.wait) before touching memory the
// predecessor writes.  Each step kernel lets its own dependent start early.
// Both instructions are no-ops for kernels launched without the attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Step epilogue: non-finite flag and activation time (first upward crossing
// of the threshold, linear interpolation between the step's end points).
__device__ __forceinline__ void step_epilogue(int64_t i, double Vn, double Vnew, double* act, double t_n,
                                              double dt, double th, int* flags) {
  if (!isfinite(Vnew)) atomicOr(flags, 1);
  if (act != nullptr) {
    const double a0 = act[i];
    if (isnan(a0) && Vn < th && Vnew >= th) act[i] = t_n + dt * (th - Vn) / (Vnew - Vn);
  }
}

// Mixed path: V is carried as the unevaluated sum hi + lo of two floats
// (48 significand bits) and updated with error-free transformations, so the
// V accumulation never uses the FP64 pipe.  ff_add is Knuth's TwoSum of
// (hi, inc) followed by Dekker's FastTwoSum renormalisation; __fadd_rn /
// __fsub_rn keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void ff_add(float hi, float lo, float inc, float& ohi, float& olo) {
  const float s = __fadd_rn(hi, inc);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(inc, bp));
  const float l = __fadd_rn(lo, e);
  const float h = __fadd_rn(s, l);
  olo = __fsub_rn(l, __fsub_rn(h, s));
  ohi = h;
}

// Epilogue of the mixed path on the hi parts (the crossing branch is rare).
__device__ __forceinline__ void step_epilogue_ff(int64_t i, float Vn, float Vnew, double* act, double t_n,
                                                 double dt, float th, int* flags) {
  if (!isfinite(Vnew)) atomicOr(flags, 1);
  if (act != nullptr && Vn < th && Vnew >= th) {
    if (isnan(act[i])) act[i] = t_n + dt * (double)((th - Vn) / (Vnew - Vn));
  }
}

// Mixed path (FP32), one node of outer stage j: the exponential step of the
// gates (Algorithm 3, Exponential_Euler), f_S at the gates y_E, and the z
// rows of g_j = nu g_{j-1} + kappa g_{j-2} + mu dt f_bar with f_bar =
// (y_E - y)/eta on the gates and c_m g_S on z_S (HAS_M2: j >= 2).  Each gate's
// row is written as soon as its increment dz = y_E - y = (e^{eta Lambda} - 1)
// (z - z_inf) is known, so that only y_E and z_S stay live through f_S.
// Returns F = (I_stim - I_ion) / C_m.
template <class Model, bool HAS_M2, bool CG>
__device__ __forceinline__ float stage_rows_mixed(const StageArgs& a, const int64_t i, const float V, const float* z,
                                                  const bool stim) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  const int64_t ld = a.ld;
  const float* __restrict__ Zm2 = static_cast<const float*>(a.Zm2);
  float* __restrict__ Zout = static_cast<float*>(a.Zout);
  const float mudt_eta = a.f_mudt * a.f_inv_eta;
  float zE1[NE > 0 ? NE : 1];
  Model::gating_each(V, z, z + NE, [&](int k, float lam, float zinf) {
    const float dz = Math<float>::em1(a.f_eta * lam) * (z[k] - zinf);
    zE1[k] = z[k] + dz;
    const float mfbar = mudt_eta * dz;
    float out;
    if constexpr (HAS_M2) out = a.f_nu * z[k] + a.f_kappa * ldm<CG>(Zm2 + k * ld + i) + mfbar;
    else out = z[k] + mfbar;
    Zout[k * ld + i] = out;
  });
  float Iion;
  float gS[NS > 0 ? NS : 1];
  Model::currents(V, zE1, z + NE, Iion, gS);
  if constexpr (NS > 0) {
#pragma unroll
    for (int k = NE; k < NZ; ++k) {
      const float mfbar = a.f_mudt * (a.f_cm * gS[k - NE]);
      float out;
      if constexpr (HAS_M2) out = a.f_nu * z[k] + a.f_kappa * ldm<CG>(Zm2 + k * ld + i) + mfbar;
      else out = z[k] + mfbar;
      Zout[k * ld + i] = out;
    }
  }
  const float Istim = stim ? a.f_stim : 0.0f;
  return (Istim - Iion) * a.f_inv_Cm;
}

// ---------------------------------------------------------------------------
// Outer stage j (FP64 path): exponential Euler of the gates (Algorithm 3,
// Exponential_Euler), frozen forcing f_S(t_j, y_E), first inner RKC stage and
// the z-part of g_j = nu g_{j-1} + kappa g_{j-2} + mu dt f_bar, where
// f_bar = ((y_E - y)/eta on the gates, c_m g_S on z_S, (u_m - V)/eta on V).
// CG: loads through L2 only (the fused step kernel, which rewrites the
// buffers within its launch).
template <class Model, bool HAS_M2, bool CG>
__device__ __forceinline__ void stage_node_fp64(const StageArgs& a, const Ell& A, const int64_t i) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  using M = Math<double>;
  const int64_t ld = a.ld;
  const double* __restrict__ Zm1 = static_cast<const double*>(a.Zm1);
  const double* __restrict__ Zm2 = static_cast<const double*>(a.Zm2);
  double* __restrict__ Zout = static_cast<double*>(a.Zout);

  const double V = ldp<CG>(a.Vm1 + i);
  double z[NZ > 0 ? NZ : 1];
#pragma unroll
  for (int k = 0; k < NZ; ++k) z[k] = ldp<CG>(Zm1 + k * ld + i);

  double zE1[NE > 0 ? NE : 1];
  if constexpr (NE > 0) {
    double lam[NE], zinf[NE];
    Model::gating(V, z, z + NE, lam, zinf);
#pragma unroll
    for (int k = 0; k < NE; ++k) zE1[k] = z[k] + M::em1(a.eta * lam[k]) * (z[k] - zinf[k]);
  }
  double Iion;
  double gS[NS > 0 ? NS : 1];
  Model::currents(V, zE1, z + NE, Iion, gS);
  const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
  const double F = (Istim - Iion) * a.inv_Cm;

  if constexpr (NZ > 0) {
#pragma unroll
    for (int k = 0; k < NZ; ++k) {
      const double fbar = (k < NE) ? (zE1[k < NE ? k : 0] - z[k]) * a.inv_eta : a.cm_inner * gS[k >= NE ? k - NE : 0];
      double out;
      if constexpr (HAS_M2) out = a.nu * z[k] + a.kappa * ldp<CG>(Zm2 + k * ld + i) + a.mu_dt * fbar;
      else out = z[k] + a.mu_dt * fbar;
      Zout[k * ld + i] = out;
    }
  }
  const double LV = ell_dot64<CG>(A, i, a.Vm1);
  if (a.Vn_copy != nullptr) a.Vn_copy[i] = V;
  if (a.m == 1) {
    const double fbarV = a.mu1 * (LV + F);  // (u_1 - V)/eta with u_1 = V + mu'_1 eta (L V + F)
    double Vnew;
    if constexpr (HAS_M2) Vnew = a.nu * V + a.kappa * ldp<CG>(a.Vm2 + i) + a.mu_dt * fbarV;
    else Vnew = V + a.mu_dt * fbarV;
    a.Vout[i] = Vnew;
    if (a.final_stage) step_epilogue(i, ldp<CG>(a.Vn + i), Vnew, a.act, a.t_n, a.dt, a.threshold, a.flags);
  } else {
    a.U1[i] = V + a.mu1_eta * (LV + F);
    static_cast<double*>(a.F)[i] = F;
  }
}

template <class Model, bool HAS_M2>
__global__ void __launch_bounds__(128) stage_kernel_fp64(const StageArgs a, const Ell A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  stage_node_fp64<Model, HAS_M2, false>(a, A, i);
}

// Outer stage j (mixed path): as above with z, the ionic model, the gating
// exponentials and L V in FP32 (on the FP32 mirror of V); V itself is only
// updated in FP64 (m == 1).  For m >= 2 the inner stages carry the FP32
// increments delta_k = u_k - V_{j-1}; this kernel writes delta_1, L V and F.
// The node's work after its V and z have been loaded (by the caller, possibly
// one node ahead).
// SPLIT: rows of at most 8 entries (checked at run time) have their
// neighbour gathers issued before the ionic model.  ROW: the caller holds
// the row (rc, rv: rw <= 8 entries, as ell_row returns them).
template <class Model, bool HAS_M2, bool CG, bool SPLIT = false, bool ROW = false>
__device__ __forceinline__ void stage_node_mixed_with(const StageArgs& a, const Ell& A, const int64_t i, const float V,
                                                      const float* z, const int32_t* rc = nullptr,
                                                      const float* rv = nullptr, const int rw = 0) {
  // the neighbour gathers go out before the ionic model, so their latency
  // overlaps it; the row's values are read after it
  const bool split = SPLIT && a.ell_wmax <= 8;
  float xv[8];
  int w = 0;
  int64_t p = 0;
  if constexpr (ROW) {
    w = rw;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < w) xv[k] = ldm<CG>(a.V32m1 + rc[k]);
  } else if (split) {
    const int64_t b = i >> 5;
    w = __ldg(A.width + b);
    p = __ldg(A.slice_ptr + b) + (i & 31);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < w) xv[k] = ldm<CG>(a.V32m1 + __ldg(A.col + p + 32 * k));
  }
  const float F = stage_rows_mixed<Model, HAS_M2, CG>(a, i, V, z, a.mask != nullptr && a.mask[i]);
  float LV = 0.0f;
  if constexpr (ROW) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < w) LV += rv[k] * (xv[k] - V);
  } else if (split) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < w) LV += __ldg(A.val32 + p + 32 * k) * (xv[k] - V);
  } else {
    LV = ell_diff32<CG>(A, i, a.V32m1);
  }
  if (a.Vn32_copy != nullptr) a.Vn32_copy[i] = V;
  if (a.m == 1) {
    // V_j = V_{j-1} + kappa (V_{j-2} - V_{j-1}) + mu dt f_bar  (nu + kappa = 1)
    const float fbarV = a.f_mu1 * (LV + F);
    const float lo1 = ldm<CG>(a.Vlo_m1 + i);
    float inc = a.f_mudt * fbarV;
    if constexpr (HAS_M2) inc += a.f_kappa * ((ldm<CG>(a.Vhi_m2 + i) - V) + (ldm<CG>(a.Vlo_m2 + i) - lo1));
    float hi, lo;
    ff_add(V, lo1, inc, hi, lo);
    a.V32out[i] = hi;
    a.Vlo_out[i] = lo;
    if (a.final_stage) step_epilogue_ff(i, ldm<CG>(a.Vn32 + i), hi, a.act, a.t_n, a.dt, a.f_th, a.flags);
  } else {
    a.D1[i] = a.f_mu1eta * (LV + F);
    if (a.LV != nullptr) a.LV[i] = LV + F;  // kept for inner stages k >= 4 only
  }
}

template <class Model, bool HAS_M2, bool CG = false, bool SPLIT = false>
__device__ __forceinline__ void stage_node_mixed(const StageArgs& a, const Ell& A, const int64_t i) {
  constexpr int NZ = Model::NE + Model::NS;
  const float* __restrict__ Zm1 = static_cast<const float*>(a.Zm1);
  const float V = ldm<CG>(a.V32m1 + i);
  float z[NZ > 0 ? NZ : 1];
#pragma unroll
  for (int k = 0; k < NZ; ++k) z[k] = ldm<CG>(Zm1 + k * a.ld + i);
  stage_node_mixed_with<Model, HAS_M2, CG, SPLIT>(a, A, i, V, z);
}

template <class Model, bool HAS_M2>
__global__ void __launch_bounds__(128) stage_kernel_mixed(const StageArgs a, const Ell A) {
  pdl_trigger();
  pdl_wait();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  stage_node_mixed<Model, HAS_M2, false, true>(a, A, i);
}

// ---------------------------------------------------------------------------
// Persistent, bulk-copy variant of the mixed stage kernel.
//
// A CTA of 128 threads owns tiles of 128 consecutive nodes (tile, tile + G,
// tile + 2G, ...).  One elected thread copies a tile's inputs (the NZ rows of
// z, V hi and the stimulus mask: contiguous 512-byte / 128-byte segments of
// the SoA arrays, and the tile's four sliced-ELL slices when rows have at
// most kTmaStageEllWidth entries) into a shared-memory stage buffer with
// cp.async.bulk completing on an mbarrier; the slices' offsets and widths go
// to shared memory with them.  One buffer per CTA by default (more CTAs per
// SM), two on request (the next tile's copy overlaps the current tile).
// The first tile's ELL slices are requested before griddepcontrol.wait, L
// being constant.  Each node issues its neighbour gathers (ordinary
// read-only loads) before its ionic model.  Waits are bounded: after
// kTmaSpinLimit polls a CTA records bit 1 in flags, waits (bounded) for its
// copies in flight and returns.
constexpr int kTmaTile = 128;
constexpr int kTmaStageEllWidth = 8;  // rows of at most this many entries are staged too
constexpr long long kTmaSpinLimit = 1ll << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// add to the expected transaction bytes of the current phase without arriving
__device__ __forceinline__ void mbar_expect_tx_only(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory bytes of one pipeline stage for NZ z rows and rows of at most
// wmax stored entries: z rows, V hi, mask, then the tile's sliced-ELL column
// indices and values (4 slices of 32 rows).
__host__ __device__ constexpr int tma_fixed_bytes(int nz) {
  return (nz * kTmaTile + kTmaTile) * 4 + kTmaTile;
}
__host__ __device__ constexpr int tma_stage_bytes(int nz, int wmax) {
  return tma_fixed_bytes(nz) + (wmax <= kTmaStageEllWidth ? 2 * 4 * wmax * 32 * 4 : 0);
}
// one stage buffer, with the ELL slices staged (ell != 0) or read from global
__host__ __device__ constexpr int tma_smem_bytes(int nz, int wmax, int ell) {
  return ell ? tma_stage_bytes(nz, wmax) : tma_fixed_bytes(nz);
}
// prefetching variant: one state region and two ELL buffers
__host__ __device__ constexpr int tma_pf_smem_bytes(int nz, int wmax) {
  return tma_fixed_bytes(nz) + 2 * (2 * 4 * wmax * 32 * 4);
}

// The outputs of one node of a mixed outer stage from its inputs in
// registers: z, V hi, the stimulus bit, and the neighbour values xv of a
// staged row (w entries at base + 32 k of the staged values sval), or
// sval = nullptr to take the row from global memory.
template <class Model, bool HAS_M2>
__device__ __forceinline__ void stage_node_core(const StageArgs& a, const Ell& A, const int64_t i,
                                                const float (&z)[(Model::NE + Model::NS) > 0 ? Model::NE + Model::NS : 1],
                                                const float V, const unsigned char mk,
                                                const float (&xv)[kTmaStageEllWidth], const int w, const float* sval,
                                                const int base) {
  const float F = stage_rows_mixed<Model, HAS_M2, false>(a, i, V, z, mk != 0);
  // sparse row: slot k of row i at base + 32 k in the staged tile
  float LV = 0.0f;
  if (sval == nullptr) {
    LV = ell_diff32<false>(A, i, a.V32m1);
  } else {
#pragma unroll
    for (int k = 0; k < kTmaStageEllWidth; ++k)
      if (k < w) LV += sval[base + 32 * k] * (xv[k] - V);
  }
  if (a.Vn32_copy != nullptr) a.Vn32_copy[i] = V;
  if (a.m == 1) {
    const float fbarV = a.f_mu1 * (LV + F);
    const float lo1 = __ldg(a.Vlo_m1 + i);
    float inc = a.f_mudt * fbarV;
    if constexpr (HAS_M2) inc += a.f_kappa * ((__ldg(a.Vhi_m2 + i) - V) + (__ldg(a.Vlo_m2 + i) - lo1));
    float hi, lo;
    ff_add(V, lo1, inc, hi, lo);
    a.V32out[i] = hi;
    a.Vlo_out[i] = lo;
    if (a.final_stage) step_epilogue_ff(i, __ldg(a.Vn32 + i), hi, a.act, a.t_n, a.dt, a.f_th, a.flags);
  } else {
    a.D1[i] = a.f_mu1eta * (LV + F);
    if (a.LV != nullptr) a.LV[i] = LV + F;  // kept for inner stages k >= 4 only
  }
}

// One node of an outer stage (mixed path) from a shared-memory stage buffer
// holding the tile's z rows, V hi and stimulus mask (kTmaTile entries each):
// the body of the bulk-copy stage kernel.  scol/sval/base/w locate the row in
// a staged sliced-ELL tile, or scol = nullptr to read the row from global.
template <class Model, bool HAS_M2>
__device__ __forceinline__ void stage_node_staged(const StageArgs& a, const Ell& A, const int64_t i, const int tid,
                                                  const float* sz, const int32_t* scol, const float* sval,
                                                  const int base, const int w) {
  constexpr int NZ = Model::NE + Model::NS;
  float z[NZ > 0 ? NZ : 1];
#pragma unroll
  for (int k = 0; k < NZ; ++k) z[k] = sz[k * kTmaTile + tid];
  const float V = sz[NZ * kTmaTile + tid];
  const unsigned char mk = reinterpret_cast<const unsigned char*>(sz + (NZ + 1) * kTmaTile)[tid];
  // neighbour values of the staged row first: the gathers are in flight
  // while the ionic model runs
  float xv[kTmaStageEllWidth];
  if (scol != nullptr) {
#pragma unroll
    for (int k = 0; k < kTmaStageEllWidth; ++k)
      if (k < w) xv[k] = __ldg(a.V32m1 + scol[base + 32 * k]);
  }
  stage_node_core<Model, HAS_M2>(a, A, i, z, V, mk, xv, w, scol != nullptr ? sval : nullptr, base);
}

template <class Model, bool HAS_M2>
__global__ void __launch_bounds__(kTmaTile) stage_kernel_mixed_tma(const StageArgs a, const Ell A) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  constexpr int FB = tma_fixed_bytes(NZ);
  const bool stage_ell = a.tma_ell && a.ell_wmax <= kTmaStageEllWidth;
  const int SB = stage_ell ? tma_stage_bytes(NZ, a.ell_wmax) : FB;
  // stage buffers per CTA: 1 or 2 (mode 3 belongs to the prefetching kernel;
  // rows it cannot stage come here with one buffer)
  const int nb = (a.tma_nbuf == 2) ? 2 : 1;
  const int64_t nslices = A.n_slices;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ int s_abort;
  // per stage buffer: offset (in entries) of each 32-row slice of the tile in
  // the staged ELL block, and its width; written with the tile's copies
  __shared__ int s_roff[2][kTmaTile / 32];
  __shared__ int s_rw[2][kTmaTile / 32];
  const int tid = threadIdx.x;
  const int64_t ntiles = (a.n + kTmaTile - 1) / kTmaTile;
  const int64_t G = gridDim.x;
  const unsigned bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
  const unsigned stage_base = smem_u32(tma_smem);

  // A tile's copies in two parts on the buffer's barrier: the ELL slices (L is
  // constant, so this part may be issued before the predecessor kernel has
  // finished) and the state (z rows, V hi, mask), whose arrival closes the phase.
  auto issue_ell = [&](int64_t tile, int buf) {
    if (!stage_ell) return;
    const unsigned bar = buf ? bar1 : bar0;
    const unsigned dst = stage_base + buf * SB;
    const int64_t s0 = tile * (kTmaTile / 32);
    const int64_t s1 = (s0 + kTmaTile / 32 < nslices) ? s0 + kTmaTile / 32 : nslices;
    const int64_t e0 = __ldg(A.slice_ptr + s0), e1 = __ldg(A.slice_ptr + s1);
#pragma unroll
    for (int q = 0; q < kTmaTile / 32; ++q) {
      const bool in = s0 + q < s1;
      s_roff[buf][q] = in ? (int)(__ldg(A.slice_ptr + s0 + q) - e0) : 0;
      s_rw[buf][q] = in ? __ldg(A.width + s0 + q) : 0;
    }
    const unsigned ell_bytes = (unsigned)((e1 - e0) * 4);
    if (ell_bytes == 0) return;
    const unsigned half = (unsigned)(4 * a.ell_wmax * 32 * 4);
    mbar_expect_tx_only(bar, 2u * ell_bytes);
    bulk_g2s(dst + FB, A.col + e0, ell_bytes, bar);
    bulk_g2s(dst + FB + half, A.val32 + e0, ell_bytes, bar);
  };
  auto issue_state = [&](int64_t tile, int buf) {
    const unsigned bar = buf ? bar1 : bar0;
    const unsigned dst = stage_base + buf * SB;
    const int64_t off = tile * kTmaTile;
    mbar_expect_tx(bar, (unsigned)FB);
    const float* Zm1 = static_cast<const float*>(a.Zm1);
#pragma unroll 1
    for (int k = 0; k < NZ; ++k) bulk_g2s(dst + k * kTmaTile * 4, Zm1 + k * a.ld + off, kTmaTile * 4, bar);
    bulk_g2s(dst + NZ * kTmaTile * 4, a.V32m1 + off, kTmaTile * 4, bar);
    bulk_g2s(dst + (NZ + 1) * kTmaTile * 4, a.mask + off, kTmaTile, bar);
  };

  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();
  pdl_trigger();
  // the stage copies the mask with the rest: a solver without stimulus has no
  // mask array, so this variant is only launched with one
  const bool run = a.mask != nullptr;
  const int64_t first = blockIdx.x;
  if (tid == 0 && run) {
    if (first < ntiles) issue_ell(first, 0);
    if (nb == 2 && first + G < ntiles) issue_ell(first + G, 1);
  }
  pdl_wait();
  if (!run) return;
  if (tid == 0) {
    if (first < ntiles) issue_state(first, 0);
    if (nb == 2 && first + G < ntiles) issue_state(first + G, 1);
  }
  unsigned phase[2] = {0u, 0u};
  int it = 0;
  for (int64_t tile = first; tile < ntiles; tile += G, ++it) {
    const int buf = (nb == 2) ? (it & 1) : 0;
    const unsigned bar = buf ? bar1 : bar0;
    long long spins = 0;
    bool ok = true;
    while (!mbar_try_wait(bar, phase[buf])) {
      if (++spins > kTmaSpinLimit) {
        atomicOr(a.flags, 2);
        s_abort = 1;
        ok = false;
        break;
      }
    }
    if (ok) phase[buf] ^= 1u;
    __syncthreads();
    if (s_abort) break;
    const float* sz = reinterpret_cast<const float*>(tma_smem + buf * SB);
    const int64_t i = tile * kTmaTile + tid;
    if (i < a.n) {
      const int32_t* scol = nullptr;
      const float* sval = nullptr;
      int base = 0, w = 0;
      if (stage_ell) {
        base = s_roff[buf][tid >> 5] + (tid & 31);
        w = s_rw[buf][tid >> 5];
        scol = reinterpret_cast<const int32_t*>(tma_smem + buf * SB + FB);
        sval = reinterpret_cast<const float*>(tma_smem + buf * SB + FB + 4 * a.ell_wmax * 32 * 4);
      }
      stage_node_staged<Model, HAS_M2>(a, A, i, tid, sz, scol, sval, base, w);
    }
    __syncthreads();  // every thread is done with this stage buffer
    if (tid == 0 && tile + nb * G < ntiles) {
      fence_proxy_async();
      issue_ell(tile + nb * G, buf);
      issue_state(tile + nb * G, buf);
    }
  }
  // on abort: give copies already in flight a bounded chance to land (a
  // buffer whose wait gave up, and the other one if its tile was issued)
  if (s_abort && tid == 0) {
    for (int b = 0; b < nb; ++b) {
      long long spins = 0;
      while (!mbar_try_wait(b ? bar1 : bar0, phase[b]) && ++spins < kTmaSpinLimit) {
      }
    }
  }
}

// Bulk-copy stage kernel with the next tile prefetched during compute (rows
// of at most kTmaStageEllWidth entries only).  Shared memory: one state
// region (z rows, V hi, mask) and two ELL buffers.  Each thread first moves
// its node's state from shared memory into registers and issues its
// neighbour gathers; after a CTA barrier the state region is free, and the
// elected thread requests the next tile's state and ELL slices (into the
// other ELL buffer) while all threads compute the current tile.  So one
// tile is always in flight per CTA at the shared-memory cost of one state
// buffer.  Waits are bounded as in stage_kernel_mixed_tma.
template <class Model, bool HAS_M2>
__global__ void __launch_bounds__(kTmaTile) stage_kernel_mixed_tma_pf(const StageArgs a, const Ell A) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  constexpr int FB = tma_fixed_bytes(NZ);
  const int EB = 2 * 4 * a.ell_wmax * 32 * 4;  // one ELL buffer: columns, then values
  const int64_t nslices = A.n_slices;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ int s_abort;
  __shared__ int s_roff[2][kTmaTile / 32];
  __shared__ int s_rw[2][kTmaTile / 32];
  const int tid = threadIdx.x;
  const int64_t ntiles = (a.n + kTmaTile - 1) / kTmaTile;
  const int64_t G = gridDim.x;
  const unsigned bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
  const unsigned base_s = smem_u32(tma_smem);

  auto issue_ell = [&](int64_t tile, int e) {
    const unsigned bar = e ? bar1 : bar0;
    const unsigned dst = base_s + FB + e * EB;
    const int64_t s0 = tile * (kTmaTile / 32);
    const int64_t s1 = (s0 + kTmaTile / 32 < nslices) ? s0 + kTmaTile / 32 : nslices;
    const int64_t e0 = __ldg(A.slice_ptr + s0), e1 = __ldg(A.slice_ptr + s1);
#pragma unroll
    for (int q = 0; q < kTmaTile / 32; ++q) {
      const bool in = s0 + q < s1;
      s_roff[e][q] = in ? (int)(__ldg(A.slice_ptr + s0 + q) - e0) : 0;
      s_rw[e][q] = in ? __ldg(A.width + s0 + q) : 0;
    }
    const unsigned ell_bytes = (unsigned)((e1 - e0) * 4);
    if (ell_bytes == 0) return;
    mbar_expect_tx_only(bar, 2u * ell_bytes);
    bulk_g2s(dst, A.col + e0, ell_bytes, bar);
    bulk_g2s(dst + (unsigned)(EB / 2), A.val32 + e0, ell_bytes, bar);
  };
  auto issue_state = [&](int64_t tile, int e) {
    const unsigned bar = e ? bar1 : bar0;
    const int64_t off = tile * kTmaTile;
    mbar_expect_tx(bar, (unsigned)FB);
    const float* Zm1 = static_cast<const float*>(a.Zm1);
#pragma unroll 1
    for (int k = 0; k < NZ; ++k) bulk_g2s(base_s + k * kTmaTile * 4, Zm1 + k * a.ld + off, kTmaTile * 4, bar);
    bulk_g2s(base_s + NZ * kTmaTile * 4, a.V32m1 + off, kTmaTile * 4, bar);
    bulk_g2s(base_s + (NZ + 1) * kTmaTile * 4, a.mask + off, kTmaTile, bar);
  };

  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();
  pdl_trigger();
  const bool run = a.mask != nullptr;  // the mask is copied with the state
  const int64_t first = blockIdx.x;
  if (tid == 0 && run && first < ntiles) issue_ell(first, 0);
  pdl_wait();
  if (!run) return;
  if (tid == 0 && first < ntiles) issue_state(first, 0);
  unsigned phase[2] = {0u, 0u};
  const float* sz = reinterpret_cast<const float*>(tma_smem);
  int it = 0;
  for (int64_t tile = first; tile < ntiles; tile += G, ++it) {
    const int e = it & 1;
    const unsigned bar = e ? bar1 : bar0;
    long long spins = 0;
    bool ok = true;
    while (!mbar_try_wait(bar, phase[e])) {
      if (++spins > kTmaSpinLimit) {
        atomicOr(a.flags, 2);
        s_abort = 1;
        ok = false;
        break;
      }
    }
    if (ok) phase[e] ^= 1u;
    __syncthreads();
    if (s_abort) break;
    // inputs of this thread's node into registers; gathers issued
    const int64_t i = tile * kTmaTile + tid;
    const bool live = i < a.n;
    float z[NZ > 0 ? NZ : 1];
    float V = 0.0f;
    unsigned char mk = 0;
    float xv[kTmaStageEllWidth];
    const int base = s_roff[e][tid >> 5] + (tid & 31);
    const int w = s_rw[e][tid >> 5];
    const int32_t* scol = reinterpret_cast<const int32_t*>(tma_smem + FB + e * EB);
    const float* sval = reinterpret_cast<const float*>(tma_smem + FB + e * EB + EB / 2);
    if (live) {
#pragma unroll
      for (int k = 0; k < NZ; ++k) z[k] = sz[k * kTmaTile + tid];
      V = sz[NZ * kTmaTile + tid];
      mk = reinterpret_cast<const unsigned char*>(sz + (NZ + 1) * kTmaTile)[tid];
#pragma unroll
      for (int k = 0; k < kTmaStageEllWidth; ++k)
        if (k < w) xv[k] = __ldg(a.V32m1 + scol[base + 32 * k]);
    }
    __syncthreads();  // the state region and the other ELL buffer are free
    if (tid == 0 && tile + G < ntiles) {
      fence_proxy_async();
      issue_ell(tile + G, e ^ 1);
      issue_state(tile + G, e ^ 1);
    }
    if (live) stage_node_core<Model, HAS_M2>(a, A, i, z, V, mk, xv, w, sval, base);
  }
  // on abort: give copies already in flight a bounded chance to land
  if (s_abort && tid == 0) {
    for (int b = 0; b < 2; ++b) {
      long long spins = 0;
      while (!mbar_try_wait(b ? bar1 : bar0, phase[b]) && ++spins < kTmaSpinLimit) {
      }
    }
  }
}

// Inner RKC stage k >= 2 (FP64 path), Algorithm 1 applied to f_u = f_F + frozen f_S.
template <bool CG>
__device__ __forceinline__ void inner_node_fp64(const InnerArgs& a, const Ell& A, const int64_t i) {
  const double Lu = ell_dot64<CG>(A, i, a.u1);
  const double F = ldp<CG>(static_cast<const double*>(a.F) + i);
  const double uk = a.nu * ldp<CG>(a.u1 + i) + a.kappa * ldp<CG>(a.u2 + i) + a.mu_eta * (Lu + F);
  if (!a.last) {
    a.uk[i] = uk;
    return;
  }
  const double V1 = ldp<CG>(a.Vm1 + i);
  const double fbar = (uk - V1) * a.inv_eta;
  double Vnew;
  if (a.Vm2 != nullptr) Vnew = a.onu * V1 + a.okappa * ldp<CG>(a.Vm2 + i) + a.omu_dt * fbar;
  else Vnew = V1 + a.omu_dt * fbar;
  a.Vout[i] = Vnew;
  if (a.final_stage) step_epilogue(i, ldp<CG>(a.Vn + i), Vnew, a.act, a.t_n, a.dt, a.threshold, a.flags);
}

static __global__ void __launch_bounds__(256) inner_kernel_fp64(const InnerArgs a, const Ell A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  inner_node_fp64<false>(a, A, i);
}

// Inner RKC stage k >= 2 (mixed path) on the FP32 increments:
// delta_k = nu'_k delta_{k-1} + kappa'_k delta_{k-2} + mu'_k eta (L V + L delta_{k-1} + F)
// (nu'_k + kappa'_k = 1 makes this the u-recurrence shifted by V); the last
// stage forms f_bar_V = delta_m / eta and updates the float-float V.
// L V_{j-1} + F of the node: delta_1 / (mu'_1 eta) while delta_1 is still one
// of the two increments at hand (k = 2: delta_{k-1}, k = 3: delta_{k-2}), else
// the value the stage kernel stored.
template <bool CG>
__device__ __forceinline__ float inner_lf(const InnerArgs& a, int64_t i, float d1, float d2) {
  if (a.lf_src == 1) return d1 * a.f_inv_mu1eta;
  if (a.lf_src == 2) return d2 * a.f_inv_mu1eta;
  return ldm<CG>(a.LV + i);
}

template <bool CG = false>
__device__ __forceinline__ void inner_node_mixed(const InnerArgs& a, const Ell& A, const int64_t i) {
  const float Ld = ell_diff32<CG>(A, i, a.d1);
  const float d1 = ldm<CG>(a.d1 + i);
  const float d2 = (a.d2 != nullptr) ? ldm<CG>(a.d2 + i) : 0.0f;
  float dk = a.f_nu * d1 + a.f_mueta * (inner_lf<CG>(a, i, d1, d2) + Ld);
  if (a.d2 != nullptr) dk += a.f_kappa * d2;
  if (!a.last) {
    a.dk[i] = dk;
    return;
  }
  const float hi1 = ldm<CG>(a.Vhi1 + i), lo1 = ldm<CG>(a.Vlo1 + i);
  float inc = a.f_omu_dt * (dk * a.f_inv_eta);
  if (a.Vhi2 != nullptr) inc += a.f_okappa * ((ldm<CG>(a.Vhi2 + i) - hi1) + (ldm<CG>(a.Vlo2 + i) - lo1));
  float hi, lo;
  ff_add(hi1, lo1, inc, hi, lo);
  a.V32out[i] = hi;
  a.Vlo_out[i] = lo;
  if (a.final_stage) step_epilogue_ff(i, ldm<CG>(a.Vn32 + i), hi, a.act, a.t_n, a.dt, a.f_th, a.flags);
}

static __global__ void __launch_bounds__(256) inner_kernel_mixed(const InnerArgs a, const Ell A) {
  pdl_trigger();
  pdl_wait();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  inner_node_mixed<false>(a, A, i);
}

// Same stage with the row's loads issued up front (rows of at most W entries);
// c, lv, w: the row of L, already loaded (ell_row).
template <int W, bool CG = false>
__device__ __forceinline__ void inner_node_mixed_row(const InnerArgs& a, const int64_t i, const int32_t (&c)[W],
                                                     const float (&lv)[W], const int w) {
  float xv[W];
  ell_gather_x<W, CG>(c, w, a.d1, xv);
  const float d1 = ldm<CG>(a.d1 + i);
  const float d2 = (a.d2 != nullptr) ? ldm<CG>(a.d2 + i) : 0.0f;
  const float LF = inner_lf<CG>(a, i, d1, d2);
  float lo1 = 0.0f, hi1 = 0.0f, hi2 = 0.0f, lo2 = 0.0f;
  if (a.last) {
    hi1 = ldm<CG>(a.Vhi1 + i);
    lo1 = ldm<CG>(a.Vlo1 + i);
    if (a.Vhi2 != nullptr) {
      hi2 = ldm<CG>(a.Vhi2 + i);
      lo2 = ldm<CG>(a.Vlo2 + i);
    }
  }
  const float Ld = ell_reduce<W>(xv, lv, w, d1);
  float dk = a.f_nu * d1 + a.f_mueta * (LF + Ld);
  if (a.d2 != nullptr) dk += a.f_kappa * d2;
  if (!a.last) {
    a.dk[i] = dk;
    return;
  }
  float inc = a.f_omu_dt * (dk * a.f_inv_eta);
  if (a.Vhi2 != nullptr) inc += a.f_okappa * ((hi2 - hi1) + (lo2 - lo1));
  float hi, lo;
  ff_add(hi1, lo1, inc, hi, lo);
  a.V32out[i] = hi;
  a.Vlo_out[i] = lo;
  if (a.final_stage) step_epilogue_ff(i, ldm<CG>(a.Vn32 + i), hi, a.act, a.t_n, a.dt, a.f_th, a.flags);
}

template <int W>
__global__ void __launch_bounds__(256, 8) inner_kernel_mixed_w(const InnerArgs a, const Ell A) {
  pdl_trigger();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // L is constant: load the row while the kernel that writes delta_1 drains
  int32_t c[W];
  float lv[W];
  const int w = (i < a.n) ? ell_row<W>(A, i, c, lv) : 0;
  pdl_wait();
  if (i >= a.n) return;
  inner_node_mixed_row<W, false>(a, i, c, lv, w);
}

// ---------------------------------------------------------------------------
// Deterministic reduction: warp shuffles, then one partial per block, then
// the last block to arrive (ticket counter) sums the partials in index order.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = (threadIdx.x < (blockDim.x >> 5)) ? sh[l] : 0.0;
  if (w == 0) t = warp_sum(t);
  return t;  // valid in thread 0
}

__device__ __forceinline__ void reduce_finish(double v, const ReduceScratch& rs, int slot) {
  __shared__ double sh[32];
  __shared__ int is_last;
  const double bsum = block_sum(v, sh);
  if (threadIdx.x == 0) {
    rs.partials[blockIdx.x] = bsum;
    __threadfence();
    const unsigned int tk = atomicAdd(rs.ticket, 1u);
    is_last = (tk == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double acc = 0.0;
  const volatile double* p = rs.partials;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) acc += p[k];
  const double total = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    rs.result[slot] = total;
    *rs.ticket = 0u;
    __threadfence();
  }
}

// Grid-wide barrier of a cooperative launch (all CTAs co-resident).  Bounded:
// after spin_limit polls it records bit 4 in flags and returns false; a CTA
// also returns false once another one has given up.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* flags, long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> gen(bar[1]);
    cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(bar[0]);
    const unsigned int my = gen.load(cuda::memory_order_acquire);
    s_ok = 1;
    __threadfence();  // the CTA's writes (ordered by the bar.sync above) before the arrival
    if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == gridDim.x - 1) {
      cnt.store(0u, cuda::memory_order_relaxed);
      gen.store(my + 1u, cuda::memory_order_release);
    } else {
      long long k = 0;
      while (gen.load(cuda::memory_order_acquire) == my) {
        if (++k > spin_limit) {
          atomicOr(flags, 4);
          s_ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (s_ok && (cuda::atomic_ref<int, cuda::thread_scope_device>(*flags).load(cuda::memory_order_relaxed) & 4))
      s_ok = 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// FP32 block sum (valid in thread 0), for per-thread sums of the mixed path.
__device__ __forceinline__ float block_sum_f(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  float t = (threadIdx.x < (blockDim.x >> 5)) ? sh[l] : 0.0f;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// Sum of column c (stride 4) of nb per-CTA partials, in the same fixed order
// in every CTA, so that every CTA takes the same scalar.  One warp adds them
// (lane l takes partials l, l + 32, ..., then a shuffle tree) and shares the
// sum: FP64 arithmetic is narrow on GB300, so the other warps do none of it.
__device__ __forceinline__ double sum_partials(const double* part, int nb, int c, double* sh) {
  (void)sh;
  __shared__ double s_w;
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int k = threadIdx.x; k < nb; k += 32) v += __ldcg(part + 4 * k + c);
    v = warp_sum(v);
    if (threadIdx.x == 0) s_w = v;
  }
  __syncthreads();
  const double r = s_w;
  __syncthreads();
  return r;
}

inline int reduce_grid(int64_t count) {
  int64_t g = (count + kReduceBlock - 1) / kReduceBlock;
  if (g < 1) g = 1;
  if (g > kReduceMaxBlocks) g = kReduceMaxBlocks;
  return (int)g;
}

// Power iteration on f_F (Algorithm 5): v_new = f_F(V + q v_old) - f_F(V), ||v_new||^2.
template <bool MIXED>
__global__ void __launch_bounds__(kReduceBlock) powerF_kernel(const PowerFArgs a, const Ell A,
                                                              const ReduceScratch rs) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    double fz, fy;
    if constexpr (MIXED) {
      // f_F is linear: f_F(V + q v) - f_F(V) = q L v, formed in FP32 on the
      // off-diagonal matrix (no cancellation)
      const int64_t b = i >> 5;
      const int w = __ldg(A.width + b);
      int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
      const float vi = (float)a.v_old[i];
      float acc32 = 0.0f;
      for (int k = 0; k < w; ++k, p += 32) acc32 += __ldg(A.val32 + p) * ((float)a.v_old[__ldg(A.col + p)] - vi);
      fz = a.q * (double)acc32;
      fy = 0.0;
    } else {
      const int64_t b = i >> 5;
      const int w = A.width[b];
      int64_t p = A.slice_ptr[b] + (i & 31);
      fz = 0.0;
      fy = 0.0;
      for (int k = 0; k < w; ++k, p += 32) {
        const int32_t c = A.col[p];
        fz += A.val[p] * (a.V[c] + a.q * a.v_old[c]);
        fy += A.val[p] * a.V[c];
      }
    }
    const double w = fz - fy;
    a.v_new[i] = w;
    acc += w * w;
  }
  reduce_finish(acc, rs, a.slot);
}

// f_S at a full state (FP64 model); writes the N rows of f_S into out.
template <class ModelD>
__device__ __forceinline__ void fS_full(const double* y, double Istim, double Cm, double* out) {
  constexpr int NE = ModelD::NE, NS = ModelD::NS;
  double I;
  double gS[NS > 0 ? NS : 1];
  ModelD::currents(y[0], y + 1, y + 1 + NE, I, gS);
  out[0] = (Istim - I) / Cm;
#pragma unroll
  for (int k = 0; k < NE; ++k) out[1 + k] = 0.0;
#pragma unroll
  for (int k = 0; k < NS; ++k) out[1 + NE + k] = gS[k];
}

template <class ModelD, typename Z>
__device__ __forceinline__ void load_state_d(const PowerSArgs& a, int64_t i, double* y) {
  constexpr int N = 1 + ModelD::NE + ModelD::NS;
  const Z* Zs = static_cast<const Z*>(a.Z);
  y[0] = a.V[i];
#pragma unroll
  for (int k = 1; k < N; ++k) y[k] = (double)Zs[(k - 1) * a.ld + i];
}

// Power iteration on f_S: v_new = f_S(y + q v_old) - f_S(y) over the full state.
template <class ModelD, typename Z>
__global__ void __launch_bounds__(kReduceBlock) powerS_kernel(const PowerSArgs a, const ReduceScratch rs) {
  constexpr int N = 1 + ModelD::NE + ModelD::NS;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    double y[N], f[N];
    load_state_d<ModelD, Z>(a, i, y);
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] = y[k] + a.q * a.v_old[k * a.ld + i];
    const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
    fS_full<ModelD>(y, Istim, a.Cm, f);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double w = f[k] - a.fy[k * a.ld + i];
      a.v_new[k * a.ld + i] = w;
      acc += w * w;
    }
  }
  reduce_finish(acc, rs, a.slot);
}

// Mixed path: v_new = q J(y) v with J v from dual numbers (see dual.cuh); f_S
// has no gate rows (they belong to f_E), so only V and z_S rows are nonzero.
template <class ModelDu, typename Z>
__global__ void __launch_bounds__(kReduceBlock) powerS_dual_kernel(const PowerSArgs a, const ReduceScratch rs) {
  constexpr int NE = ModelDu::NE, NS = ModelDu::NS, N = 1 + NE + NS;
  double acc = 0.0;
  const Z* Zs = static_cast<const Z*>(a.Z);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    Dual y[N];
    y[0] = Dual((float)a.V[i], (float)a.v_old[i]);
#pragma unroll
    for (int k = 1; k < N; ++k) y[k] = Dual((float)Zs[(k - 1) * a.ld + i], (float)a.v_old[k * a.ld + i]);
    Dual I;
    Dual gS[NS > 0 ? NS : 1];
    ModelDu::currents(y[0], y + 1, y + 1 + NE, I, gS);
    const double w0 = a.q * (double)(-I.d * (float)(1.0 / a.Cm));
    a.v_new[i] = w0;
    acc += w0 * w0;
#pragma unroll
    for (int k = 0; k < NE; ++k) a.v_new[(1 + k) * a.ld + i] = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const double w = a.q * (double)gS[k].d;
      a.v_new[(1 + NE + k) * a.ld + i] = w;
      acc += w * w;
    }
  }
  reduce_finish(acc, rs, a.slot);
}

template <class ModelD, typename Z>
__global__ void __launch_bounds__(kReduceBlock) fS_kernel(const PowerSArgs a, double* out) {
  constexpr int N = 1 + ModelD::NE + ModelD::NS;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    double y[N], f[N];
    load_state_d<ModelD, Z>(a, i, y);
    const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
    fS_full<ModelD>(y, Istim, a.Cm, f);
#pragma unroll
    for (int k = 0; k < N; ++k) out[k * a.ld + i] = f[k];
  }
}

template <typename Z>
__global__ void __launch_bounds__(kReduceBlock) state_sumsq_kernel(int64_t n, int64_t ld, int nz, const double* V,
                                                                   const Z* Zb, const ReduceScratch rs, int slot) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = V[i];
    acc += v * v;
    for (int k = 0; k < nz; ++k) {
      const double z = (double)Zb[k * ld + i];
      acc += z * z;
    }
  }
  reduce_finish(acc, rs, slot);
}

template <typename Z>
__global__ void convert_kernel(int64_t count, const void* src, double* dst, int to_double) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    if (to_double) dst[i] = (double)static_cast<const Z*>(src)[i];
    else static_cast<Z*>(const_cast<void*>(src))[i] = (Z)dst[i];
  }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers shared by the per-precision translation units.
inline unsigned blocks_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// Barrier between the phases of power_fused_kernel.  CLUSTER: the grid is
// one thread-block cluster, and the hardware cluster barrier (release /
// acquire at cluster scope, which covers the partial sums in global memory)
// replaces the atomic grid barrier; for problems small enough that one
// cluster holds them, the iteration is then bound by its loads, not by
// device-scope atomics.
template <bool CLUSTER>
__device__ __forceinline__ bool power_barrier(const PowerFusedArgs& a) {
  if constexpr (CLUSTER) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    return true;
  } else {
    return grid_barrier(a.bar, a.flags, a.spin_limit);
  }
}

// Algorithm 5 for rho_F and rho_S in one persistent launch (a cooperative
// grid, or one thread-block cluster for small problems): the iteration
// loops run on the device (every CTA takes the same scalars from the same
// partial sums, so all take the same branches) and the host reads the two
// estimates once.  FP64 path: the differences f(y + q v) - f(y) of Algorithm
// 5; mixed path: q J v (q L v for f_F, dual numbers for f_S).  Iterates
// ping-pong between two buffers per estimate; out[4], out[5] say which holds
// the last one.
struct PowerResult {
  double rhoF = 0, rhoS = 0;
  int itF = 0, itS = 0;
  int lastF = 0, lastS = 0;  // iterate buffer (0 or 1) holding the last iterate
  bool ok = false;           // false: a grid barrier gave up (flags bit 1 set)
};

// Hardware barrier of the whole cluster (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// A double in the shared memory of CTA `rank` of this cluster, at the
// address of `local` in this CTA (distributed shared memory).
__device__ __forceinline__ double ld_cluster_f64(const double* local, unsigned rank) {
  const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(local));
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(r) : "memory");
  return v;
}

// The body of the launch: every thread of every CTA returns the same result.
// CLUSTER: the per-CTA partial sums stay in each CTA's shared memory and are
// read across the cluster after the barrier; otherwise they go through
// global memory.  Same values, same order of addition.
template <class MD, class MDu, typename Z, bool MIXED, bool CLUSTER>
__device__ __forceinline__ PowerResult power_fused_body(const PowerFusedArgs& a, const Ell& A) {
  constexpr int NE = MD::NE, NS = MD::NS, N = 1 + NE + NS;
  PowerResult res;
  // Mixed path: iterates, per-thread and per-CTA sums in FP32 (GB300's FP64
  // pipe is a small fraction of its FP32 rate); the grid sums and the
  // scalars of Algorithm 5 in FP64.  FP64 path: everything in FP64.
  using VT = typename std::conditional<MIXED, float, double>::type;
  __shared__ double sh[32];
  __shared__ float shf[32];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int G = gridDim.x;
  const Z* Zs = static_cast<const Z*>(a.Z);
  VT* const vF[2] = {reinterpret_cast<VT*>(a.vF[0]), reinterpret_cast<VT*>(a.vF[1])};
  VT* const vS[2] = {reinterpret_cast<VT*>(a.vS[0]), reinterpret_cast<VT*>(a.vS[1])};
  int par = 0;
  auto part = [&](int p) { return a.part + (size_t)p * 4 * G; };
  __shared__ double s_cpart[2][4];  // CLUSTER: this CTA's partials (two parities)
  __shared__ double s_csum[4];
  // grid sums of the first cnt columns of the partials of parity par, the
  // same in every CTA (lane k adds CTA k's partial; G <= 32 here)
  auto gather = [&](int cnt, double* out) {
    if constexpr (CLUSTER) {
      if (threadIdx.x < 32) {
        for (int c = 0; c < cnt; ++c) {
          double v = (threadIdx.x < (unsigned)G) ? ld_cluster_f64(&s_cpart[par][c], threadIdx.x) : 0.0;
          v = warp_sum(v);
          if (threadIdx.x == 0) s_csum[c] = v;
        }
      }
      __syncthreads();
      for (int c = 0; c < cnt; ++c) out[c] = s_csum[c];
      __syncthreads();
    } else {
      for (int c = 0; c < cnt; ++c) out[c] = sum_partials(part(par), G, c, sh);
    }
  };
  // block sums of the first cnt values into this CTA's partials (FP32 sums
  // of FP32 per-thread sums on the mixed path)
  auto bsum = [&](VT v) -> double {
    if constexpr (MIXED) return (double)block_sum_f(v, shf);
    else return block_sum(v, sh);
  };
  auto publish = [&](int cnt, VT v0, VT v1, VT v2, VT v3) {
    const double t0 = bsum(v0);
    const double t1 = cnt > 1 ? bsum(v1) : 0.0;
    const double t2 = cnt > 2 ? bsum(v2) : 0.0;
    const double t3 = cnt > 3 ? bsum(v3) : 0.0;
    if (threadIdx.x == 0) {
      if constexpr (CLUSTER) {
        s_cpart[par][0] = t0;
        s_cpart[par][1] = t1;
        s_cpart[par][2] = t2;
        s_cpart[par][3] = t3;
      } else {
        double* p = part(par) + 4 * blockIdx.x;
        p[0] = t0;
        p[1] = t1;
        p[2] = t2;
        p[3] = t3;
      }
    }
  };
  // norms of y and of the start iterates; f_S(y) for the FP64 differences
  {
    VT s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int64_t i = i0; i < a.n; i += stride) {
      VT y[N];
      if constexpr (MIXED) y[0] = a.Vhi[i];
      else y[0] = a.V[i];
#pragma unroll
      for (int k = 1; k < N; ++k) y[k] = (VT)Zs[(k - 1) * a.ld + i];
      s0 += y[0] * y[0];
      s1 += vF[0][i] * vF[0][i];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        s2 += y[k] * y[k];
        const VT v = vS[0][k * a.ld + i];
        s3 += v * v;
      }
      if constexpr (!MIXED) {
        double f[N];
        const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
        fS_full<MD>(y, Istim, a.Cm, f);
#pragma unroll
        for (int k = 0; k < N; ++k) a.fy[k * a.ld + i] = f[k];
      }
    }
    publish(4, s0, s1, s2, s3);
  }
  if (!power_barrier<CLUSTER>(a)) return res;
  // The scalars of Algorithm 5 (norms, q, rho, the stopping test) are
  // computed by thread 0 and shared: they are FP64, and GB300's FP64 pipe is
  // narrow, so the other threads must not repeat them.
  __shared__ double s_q, s_rho, s_delta, s_tol;
  __shared__ int s_go, s_it, s_maxit;
  // squared norms of y_F, v_F, y_S, v_S (the same value in every thread)
  double nsum[4];
  gather(4, nsum);
  par ^= 1;

  // one power iteration per loop trip: v_new = f(y + q v) - f(y) (FP64 path)
  // or q J v (mixed path), rho = |v_new| / delta, until the relative change
  // of rho is below tol or max_iter iterations
  // no initial guess (warm value 0): the cold-start tolerance and cap
  // Mixed path: these scalars in FP32 too (its iterates are FP32, and one
  // thread's FP64 square roots and divisions cost about 0.4 us each on
  // GB300's narrow FP64 pipe); FP64 path: in FP64.
  auto start = [&](double ny2, double nv2, double warm) {
    if (threadIdx.x == 0) {
      s_rho = warm;
      s_it = 0;
      s_tol = warm == 0.0 ? a.tol_cold : a.tol;
      s_maxit = warm == 0.0 ? a.max_iter_cold : a.max_iter;
      if constexpr (MIXED) {
        const float ny = sqrtf((float)ny2), nv = sqrtf((float)nv2), e = (float)a.eps;
        const float delta = ny > 0.0f ? ny * e : e;
        s_delta = delta;
        if (nv == 0.0f) {
          s_rho = 0.0;
          s_go = 0;
        } else {
          s_q = delta / nv;
          s_go = (fabs(warm) >= s_tol * warm && s_maxit > 0) ? 1 : 0;
        }
      } else {
        const double ny = sqrt(ny2), nv = sqrt(nv2);
        s_delta = ny > 0.0 ? ny * a.eps : a.eps;
        if (nv == 0.0) {
          s_rho = 0.0;
          s_go = 0;
        } else {
          s_q = s_delta / nv;
          s_go = (fabs(warm) >= s_tol * warm && s_maxit > 0) ? 1 : 0;
        }
      }
    }
    __syncthreads();
  };
  auto advance = [&](double nv2) {
    if (threadIdx.x == 0) {
      ++s_it;
      if constexpr (MIXED) {
        const float nv = sqrtf((float)nv2);
        if (nv == 0.0f) {
          s_rho = 0.0;
          s_go = 0;
        } else {
          const float rho_old = (float)s_rho, delta = (float)s_delta;
          const float rho = nv / delta;
          s_q = delta / nv;
          s_rho = rho;
          s_go = (fabsf(rho - rho_old) >= (float)s_tol * rho && s_it < s_maxit) ? 1 : 0;
        }
      } else {
        const double nv = sqrt(nv2);
        if (nv == 0.0) {
          s_rho = 0.0;
          s_go = 0;
        } else {
          const double rho_old = s_rho;
          s_q = s_delta / nv;
          s_rho = nv / s_delta;
          s_go = (fabs(s_rho - rho_old) >= s_tol * s_rho && s_it < s_maxit) ? 1 : 0;
        }
      }
    }
    __syncthreads();
  };

  // rho_F on the V block
  int curF = 0;
  start(nsum[0], nsum[1], a.rhoF_warm);
  while (s_go) {
    const double q = s_q;
    const VT* vo = vF[curF];
    VT* vn = vF[curF ^ 1];
    VT acc = 0;
    const float qf = (float)q;
    if constexpr (MIXED) {
      if (a.ell_wmax <= 8) {
        // rows of at most 8 entries: the row's columns and values, then all
        // of its gathers, are issued at once (three dependent loads per node
        // instead of two per entry); same sum in the same order
#pragma unroll 2
        for (int64_t i = i0; i < a.n; i += stride) {
          int32_t c[8];
          float lv[8], xv[8];
          const int w = ell_row<8>(A, i, c, lv);
          ell_gather_x<8, true>(c, w, vo, xv);
          const float wv = qf * ell_reduce<8>(xv, lv, w, __ldcg(vo + i));
          vn[i] = wv;
          acc += wv * wv;
        }
      } else {
        for (int64_t i = i0; i < a.n; i += stride) {
          const int64_t b = i >> 5;
          const int w = __ldg(A.width + b);
          int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
          // q L v in FP32: f_F is linear, so f_F(V + q v) - f_F(V) = q L v
          const float vi = __ldcg(vo + i);
          float s32 = 0.0f;
          for (int k = 0; k < w; ++k, p += 32) s32 += __ldg(A.val32 + p) * (__ldcg(vo + __ldg(A.col + p)) - vi);
          const float wv = qf * s32;
          vn[i] = wv;
          acc += wv * wv;
        }
      }
    } else {
      for (int64_t i = i0; i < a.n; i += stride) {
        const int64_t b = i >> 5;
        const int w = __ldg(A.width + b);
        int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
        double fz = 0.0, fy = 0.0;
        for (int k = 0; k < w; ++k, p += 32) {
          const int32_t c = __ldg(A.col + p);
          fz += __ldg(A.val + p) * (a.V[c] + q * __ldcg(vo + c));
          fy += __ldg(A.val + p) * a.V[c];
        }
        const double wv = fz - fy;
        vn[i] = wv;
        acc += wv * wv;
      }
    }
    publish(1, acc, 0, 0, 0);
    if (!power_barrier<CLUSTER>(a)) return res;
    double nv2;
    gather(1, &nv2);
    par ^= 1;
    curF ^= 1;
    advance(nv2);
  }
  const double rhoF = s_rho;
  const int itF = s_it;
  __syncthreads();

  // rho_S on the full state
  int curS = 0;
  start(nsum[2], nsum[3], a.rhoS_warm);
  while (s_go) {
    const double q = s_q;
    const VT* vo = vS[curS];
    VT* vn = vS[curS ^ 1];
    VT acc = 0;
    const float qf = (float)q;
    const float inv_Cm = a.f_inv_Cm;
    for (int64_t i = i0; i < a.n; i += stride) {
      if constexpr (MIXED) {
        // q J v by forward-mode dual numbers in FP32
        Dual y[N];
        y[0] = Dual(a.Vhi[i], vo[i]);
#pragma unroll
        for (int k = 1; k < N; ++k) y[k] = Dual((float)Zs[(k - 1) * a.ld + i], vo[k * a.ld + i]);
        Dual I;
        Dual gS[NS > 0 ? NS : 1];
        MDu::currents(y[0], y + 1, y + 1 + NE, I, gS);
        const float w0 = qf * (-I.d * inv_Cm);
        vn[i] = w0;
        acc += w0 * w0;
#pragma unroll
        for (int k = 0; k < NE; ++k) vn[(1 + k) * a.ld + i] = 0.0f;
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const float w = qf * gS[k].d;
          vn[(1 + NE + k) * a.ld + i] = w;
          acc += w * w;
        }
      } else {
        double y[N], f[N];
        y[0] = a.V[i];
#pragma unroll
        for (int k = 1; k < N; ++k) y[k] = (double)Zs[(k - 1) * a.ld + i];
#pragma unroll
        for (int k = 0; k < N; ++k) y[k] = y[k] + q * vo[k * a.ld + i];
        const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
        fS_full<MD>(y, Istim, a.Cm, f);
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const double w = f[k] - a.fy[k * a.ld + i];
          vn[k * a.ld + i] = w;
          acc += w * w;
        }
      }
    }
    publish(1, acc, 0, 0, 0);
    if (!power_barrier<CLUSTER>(a)) return res;
    double nv2;
    gather(1, &nv2);
    par ^= 1;
    curS ^= 1;
    advance(nv2);
  }
  res.rhoF = rhoF;
  res.rhoS = s_rho;
  res.itF = itF;
  res.itS = s_it;
  res.lastF = curF;
  res.lastS = curS;
  res.ok = true;
  return res;
}

template <class MD, class MDu, typename Z, bool MIXED, bool CLUSTER = false>
__global__ void __launch_bounds__(kReduceBlock) power_fused_kernel(const PowerFusedArgs a, const Ell A) {
  const PowerResult r = power_fused_body<MD, MDu, Z, MIXED, CLUSTER>(a, A);
  // no CTA leaves while another may still read its shared memory
  if constexpr (CLUSTER) cluster_sync_all();
  if (r.ok && blockIdx.x == 0 && threadIdx.x == 0) {
    a.out[0] = r.rhoF;
    a.out[1] = r.rhoS;
    a.out[2] = (double)r.itF;
    a.out[3] = (double)r.itS;
    a.out[4] = (double)r.lastF;
    a.out[5] = (double)r.lastS;
  }
}

// ---------------------------------------------------------------------------
// Device-resident emRKC step for problems that one thread-block cluster
// holds: Algorithm 5 when due (the body above), Algorithm 1 (rkc_stages,
// rkc_coeffs) from the resulting radii, then the s outer stages and the
// m - 1 inner stages of each (Algorithm 3) with the per-node functions of
// the single-step kernels, phases separated by the hardware cluster
// barrier (release / acquire at cluster scope).  Buffers rewritten within
// the launch after being read are loaded through L2, the others may come
// through L1 (the rule of the batched kernel).  g_j goes to buffer
// (b0 + r j) mod 3 with r = 2 when s = 2 (mod 3), else r = 1, so that
// g_s = y_{n+1} lands in buffer (b0 + 1) mod 3 as the host expects; when
// s = 0 (mod 3) it lands in b0 and is copied over after the last stage.  The
// host never reads s, m or rho during a step: they are kept in
// FusedStepState.

// Largest CTA of the fused step: 512 threads for the light models, 256 for
// TTP06 (its registers); the launch uses the smallest multiple of 32 that
// gives every node its own thread, up to this bound.
template <class MR>
struct FusedBlock {
  static constexpr int value = (MR::NE + MR::NS > 3) ? 256 : 512;
};

template <class MD, class MR, class MDu, typename Z, bool MIXED>
__global__ void __launch_bounds__(FusedBlock<MR>::value, 1) step_fused_kernel(const FusedStepArgs a, const Ell A) {
  constexpr int NZ = MR::NE + MR::NS;
  __shared__ double s_co[4][kFusedMaxStages + 1];  // outer mu, nu, kappa, c
  __shared__ double s_ci[4][kFusedMaxStages + 1];  // inner mu', nu', kappa', c'
  __shared__ double s_eta;
  __shared__ int s_S, s_M;
  // the scalars of every phase of the step (outer stage j at j - 1, inner
  // stage k at k - 2), computed once per step, one thread per phase, with
  // multiplications only (GB300's FP64 pipe is narrow, and a division or
  // square root in one thread costs about 0.4 us)
  __shared__ double s_sd[kFusedMaxStages][10];
  __shared__ float s_sf[kFusedMaxStages][12];
  __shared__ double s_id[kFusedMaxStages][3];
  __shared__ float s_if[kFusedMaxStages][3];
  // launched with programmatic dependent launch: the next step's cluster
  // may be made resident now, and this one waits for the previous step
  pdl_trigger();
  pdl_wait();
  FusedStepState* const st = a.state;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;

  // ---- spectral radii: given, estimated now (Algorithm 5), or the last
  // estimates; the safety factor and the rho_S floor as on the host path
  double rF = 0.0, rS = 0.0;
  if (!a.fixed) {
    rF = st->rhoF_raw;
    rS = st->rhoS_raw;
    if (a.due) {
      PowerFusedArgs pa = a.pw;
      const int cF = st->curF, cS = st->curS;
      if (cF) {
        double* t = pa.vF[0];
        pa.vF[0] = pa.vF[1];
        pa.vF[1] = t;
      }
      if (cS) {
        double* t = pa.vS[0];
        pa.vS[0] = pa.vS[1];
        pa.vS[1] = t;
      }
      pa.rhoF_warm = rF;
      pa.rhoS_warm = rS;
      pa.stim = (a.mask != nullptr && a.t_on <= a.t_n && a.t_n <= a.t_off) ? a.amp : 0.0;
      // every CTA has read the state before the body's first barrier, so
      // the lead thread may rewrite it afterwards
      const PowerResult r = power_fused_body<MD, MDu, Z, MIXED, true>(pa, A);
      rF = r.rhoF;
      rS = r.rhoS;
      if (lead) {
        st->rhoF_raw = rF;
        st->rhoS_raw = rS;
        st->curF = cF ^ r.lastF;
        st->curS = cS ^ r.lastS;
        st->itF = r.itF;
        st->itS = r.itS;
        st->total_it += r.itF + r.itS;
      }
    } else if (lead) {
      st->itF = st->itS = 0;
    }
  } else if (lead) {
    st->itF = st->itS = 0;
  }

  // ---- Algorithm 1: stage counts (the same in every CTA), coefficients
  // from the host's tables
  const int L = rkc_table_len(kFusedMaxStages);
  const double* __restrict__ inv_ls = a.ctab + 4 * L;                        // 1 / (beta s^2)
  const double* __restrict__ inv_mu1 = a.ctab + 4 * L + kFusedMaxStages + 1;  // 1 / mu_1 of s
  if (threadIdx.x == 0) {
    const double rhoF = a.fixed ? a.rho_F_fixed : a.safety * rF;
    const double rhoS = a.fixed ? a.rho_S_fixed : fmax(a.safety * rS, a.rho_S_min);
    const int S = rkc_stages_mul(a.dt * rhoS, a.beta);
    const double eta = S <= kFusedMaxStages ? a.two_dt * inv_ls[S] : 0.0;
    const int M = S <= kFusedMaxStages ? rkc_stages_mul(eta * rhoF, a.beta) : 0;
    s_S = S;
    s_M = M;
    s_eta = eta;
    if (lead) {
      st->rhoF = rhoF;
      st->rhoS = rhoS;
      st->s = S;
      st->m = M;
      st->eta = eta;
    }
  }
  __syncthreads();
  const int S = s_S, M = s_M;
  if (S > kFusedMaxStages || M > kFusedMaxStages) {
    if (lead) atomicOr(a.flags, 16);
    cluster_sync_all();  // the power iteration's shared-memory reads are done
    return;
  }
  for (int q = threadIdx.x; q < 4 * (S + 1); q += blockDim.x)
    s_co[q / (S + 1)][q % (S + 1)] = a.ctab[(q / (S + 1)) * L + rkc_table_row(S) + q % (S + 1)];
  for (int q = threadIdx.x; q < 4 * (M + 1); q += blockDim.x)
    s_ci[q / (M + 1)][q % (M + 1)] = a.ctab[(q / (M + 1)) * L + rkc_table_row(M) + q % (M + 1)];
  __syncthreads();
  // every phase's scalars at once
  for (int j = threadIdx.x + 1; j <= S; j += blockDim.x) {
    const double eta = s_eta, mu1 = s_ci[0][1];
    const double inv_eta = a.beta * (double)S * (double)S * a.inv_two_dt;
    const double nu = j >= 2 ? s_co[1][j] : 1.0, kappa = j >= 2 ? s_co[2][j] : 0.0, mu_dt = s_co[0][j] * a.dt;
    const double ts = __dadd_rn(a.t_n, __dmul_rn(s_co[3][j - 1], a.dt));
    const double stim = (a.mask != nullptr && a.t_on <= ts && ts <= a.t_off) ? a.amp : 0.0;
    double* sd = s_sd[j - 1];
    float* sf = s_sf[j - 1];
    sd[0] = nu;
    sd[1] = kappa;
    sd[2] = mu_dt;
    sd[3] = eta;
    sd[4] = s_ci[3][M];
    sd[5] = mu1 * eta;
    sd[6] = stim;
    sd[7] = a.inv_Cm;
    sd[8] = inv_eta;
    sd[9] = mu1;
    sf[0] = (float)nu;
    sf[1] = (float)kappa;
    sf[2] = (float)mu_dt;
    sf[3] = (float)inv_eta;
    sf[4] = (float)sd[4];
    sf[5] = (float)mu1;
    sf[6] = (float)sd[5];
    sf[7] = (float)eta;
    sf[8] = (float)stim;
    sf[9] = (float)a.inv_Cm;
    sf[10] = (float)a.threshold;
    sf[11] = (float)(inv_eta * inv_mu1[M]);
  }
  for (int k = threadIdx.x + 2; k <= M; k += blockDim.x) {
    const double mu_eta = s_ci[0][k] * s_eta;
    s_id[k - 2][0] = s_ci[1][k];
    s_id[k - 2][1] = s_ci[2][k];
    s_id[k - 2][2] = mu_eta;
    s_if[k - 2][0] = (float)s_ci[1][k];
    s_if[k - 2][1] = (float)s_ci[2][k];
    s_if[k - 2][2] = (float)mu_eta;
  }
  __syncthreads();

  // ---- the s outer stages, each followed by its m - 1 inner stages
  // Mixed path with one node per thread and rows of at most 8 entries: the
  // thread's row of L is loaded once and kept in registers for every stage.
  const bool row_pre = MIXED && a.n <= stride && a.ell_wmax <= 8;
  int32_t rc[8];
  float rv[8];
  int rw = 0;
  if (row_pre && i0 < a.n) rw = ell_row<8>(A, i0, rc, rv);
  const int b0 = a.b0;
  const int rot = (S % 3 == 2) ? 2 : 1;
  // L1 may serve the stage loads when no buffer is rewritten after being
  // read in this launch: with s <= 2 each state buffer is written once, the
  // increment buffers once only when m <= 3 and s = 1 (the power iteration's
  // own buffers are always loaded through L2)
  const bool l2 = S >= 3 || M >= 4 || (S >= 2 && M >= 2);
  for (int j = 1; j <= S; ++j) {
    const int bm1 = (b0 + rot * (j - 1)) % 3, bm2 = (b0 + rot * (j + 1)) % 3, bo = (b0 + rot * j) % 3;
    const double* sd = s_sd[j - 1];
    const float* sf = s_sf[j - 1];
    StageArgs sa;
    sa.n = a.n;
    sa.ld = a.ld;
    sa.Zm1 = a.Z[bm1];
    sa.Zm2 = j >= 2 ? a.Z[bm2] : nullptr;
    sa.Zout = a.Z[bo];
    sa.nu = sd[0];
    sa.kappa = sd[1];
    sa.mu_dt = sd[2];
    sa.eta = sd[3];
    sa.cm_inner = sd[4];
    sa.mu1_eta = sd[5];
    sa.m = M;
    sa.F = a.F;
    sa.mask = a.mask;
    sa.stim = sd[6];
    sa.Cm = a.Cm;
    sa.inv_Cm = sd[7];
    sa.final_stage = (j == S && M == 1) ? 1 : 0;
    sa.act = a.act;
    sa.t_n = a.t_n;
    sa.dt = a.dt;
    sa.threshold = a.threshold;
    sa.flags = a.flags;
    sa.inv_eta = sd[8];
    sa.mu1 = sd[9];
    if constexpr (MIXED) {
      sa.V32m1 = a.Vhi[bm1];
      sa.V32out = a.Vhi[bo];
      sa.Vlo_m1 = a.Vlo[bm1];
      sa.Vhi_m2 = j >= 2 ? a.Vhi[bm2] : nullptr;
      sa.Vlo_m2 = j >= 2 ? a.Vlo[bm2] : nullptr;
      sa.Vlo_out = a.Vlo[bo];
      sa.Vn32 = (S <= 2) ? a.Vhi[b0] : a.Vn32;
      sa.Vn32_copy = (j == 1 && S >= 3) ? a.Vn32 : nullptr;
      sa.f_th = sf[10];
      sa.D1 = a.D[0];
      sa.LV = (M >= 4) ? a.LV : nullptr;
      sa.f_nu = sf[0];
      sa.f_kappa = sf[1];
      sa.f_mudt = sf[2];
      sa.f_inv_eta = sf[3];
      sa.f_cm = sf[4];
      sa.f_mu1 = sf[5];
      sa.f_mu1eta = sf[6];
      sa.f_eta = sf[7];
      sa.f_stim = sf[8];
      sa.f_inv_Cm = sf[9];
      sa.ell_wmax = a.ell_wmax;
      auto nodes = [&](auto cg_tag) {
        constexpr bool CG = decltype(cg_tag)::value;
        if (row_pre) {
          if (i0 < a.n) {
            const float* __restrict__ Zm1 = static_cast<const float*>(sa.Zm1);
            const float V = ldm<CG>(sa.V32m1 + i0);
            float z[NZ > 0 ? NZ : 1];
#pragma unroll
            for (int k = 0; k < NZ; ++k) z[k] = ldm<CG>(Zm1 + k * a.ld + i0);
            if (j >= 2) stage_node_mixed_with<MR, true, CG, false, true>(sa, A, i0, V, z, rc, rv, rw);
            else stage_node_mixed_with<MR, false, CG, false, true>(sa, A, i0, V, z, rc, rv, rw);
          }
        } else {
          for (int64_t i = i0; i < a.n; i += stride) {
            if (j >= 2) stage_node_mixed<MR, true, CG>(sa, A, i);
            else stage_node_mixed<MR, false, CG>(sa, A, i);
          }
        }
      };
      if (l2) nodes(std::true_type{});
      else nodes(std::false_type{});
    } else {
      sa.Vm1 = a.V[bm1];
      sa.Vm2 = j >= 2 ? a.V[bm2] : nullptr;
      sa.Vout = a.V[bo];
      sa.U1 = a.U[0];
      sa.Vn = (S <= 2) ? a.V[b0] : a.Vn;
      sa.Vn_copy = (j == 1 && S >= 3) ? a.Vn : nullptr;
      auto nodes = [&](auto cg_tag) {
        constexpr bool CG = decltype(cg_tag)::value;
        for (int64_t i = i0; i < a.n; i += stride) {
          if (j >= 2) stage_node_fp64<MR, true, CG>(sa, A, i);
          else stage_node_fp64<MR, false, CG>(sa, A, i);
        }
      };
      if (l2) nodes(std::true_type{});
      else nodes(std::false_type{});
    }
    cluster_sync_all();
    for (int k = 2; k <= M; ++k) {
      const double* id = s_id[k - 2];
      const float* ifl = s_if[k - 2];
      InnerArgs ib;
      ib.n = a.n;
      ib.F = a.F;
      ib.nu = id[0];
      ib.kappa = id[1];
      ib.mu_eta = id[2];
      ib.last = (k == M) ? 1 : 0;
      ib.onu = sa.nu;
      ib.okappa = sa.kappa;
      ib.omu_dt = sa.mu_dt;
      ib.eta = sa.eta;
      ib.final_stage = (j == S && k == M) ? 1 : 0;
      ib.act = a.act;
      ib.t_n = a.t_n;
      ib.dt = a.dt;
      ib.threshold = a.threshold;
      ib.flags = a.flags;
      ib.inv_eta = sa.inv_eta;
      if constexpr (MIXED) {
        ib.d1 = a.D[(k - 2) % 3];
        ib.d2 = (k == 2) ? nullptr : a.D[(k - 3) % 3];
        ib.dk = a.D[(k - 1) % 3];
        ib.LV = a.LV;
        ib.lf_src = (M >= 4) ? 0 : (k == 2 ? 1 : 2);
        ib.f_inv_mu1eta = sf[11];
        ib.V32out = a.Vhi[bo];
        ib.Vhi1 = a.Vhi[bm1];
        ib.Vlo1 = a.Vlo[bm1];
        ib.Vhi2 = j >= 2 ? a.Vhi[bm2] : nullptr;
        ib.Vlo2 = j >= 2 ? a.Vlo[bm2] : nullptr;
        ib.Vlo_out = a.Vlo[bo];
        ib.Vn32 = sa.Vn32;
        ib.f_okappa = sa.f_kappa;
        ib.f_omu_dt = sa.f_mudt;
        ib.f_th = sa.f_th;
        ib.f_nu = ifl[0];
        ib.f_kappa = ifl[1];
        ib.f_mueta = ifl[2];
        ib.f_inv_eta = sa.f_inv_eta;
        auto nodes = [&](auto cg_tag) {
          constexpr bool CG = decltype(cg_tag)::value;
          if (row_pre) {
            if (i0 < a.n) inner_node_mixed_row<8, CG>(ib, i0, rc, rv, rw);
          } else {
            for (int64_t i = i0; i < a.n; i += stride) inner_node_mixed<CG>(ib, A, i);
          }
        };
        if (l2) nodes(std::true_type{});
        else nodes(std::false_type{});
      } else {
        ib.u1 = a.U[(k - 2) % 3];
        ib.u2 = (k == 2) ? a.V[bm1] : a.U[(k - 3) % 3];
        ib.uk = a.U[(k - 1) % 3];
        ib.Vm1 = a.V[bm1];
        ib.Vm2 = j >= 2 ? a.V[bm2] : nullptr;
        ib.Vout = a.V[bo];
        ib.Vn = sa.Vn;
        if (l2) {
          for (int64_t i = i0; i < a.n; i += stride) inner_node_fp64<true>(ib, A, i);
        } else {
          for (int64_t i = i0; i < a.n; i += stride) inner_node_fp64<false>(ib, A, i);
        }
      }
      cluster_sync_all();
    }
  }
  // s = 0 (mod 3): y_{n+1} is in b0; move it to (b0 + 1) mod 3
  if (S % 3 == 0) {
    const int bd = (b0 + 1) % 3;
    const Z* __restrict__ zs = static_cast<const Z*>(a.Z[b0]);
    Z* __restrict__ zd = static_cast<Z*>(a.Z[bd]);
    for (int64_t i = i0; i < a.n; i += stride) {
      if constexpr (MIXED) {
        a.Vhi[bd][i] = __ldcg(a.Vhi[b0] + i);
        a.Vlo[bd][i] = __ldcg(a.Vlo[b0] + i);
      } else {
        a.V[bd][i] = __ldcg(a.V[b0] + i);
      }
#pragma unroll
      for (int k = 0; k < NZ; ++k) zd[k * a.ld + i] = __ldcg(zs + k * a.ld + i);
    }
  }
}

// Launch with the programmatic-serialisation attribute when pdl is set.
template <typename... KArgs, typename... Args>
inline void launch_k(bool pdl, void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                     Args&&... args) {
  if (!pdl) {
    k<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

template <class MD, class MR, typename R, typename Z, bool MIXED, class MDu = MD>
struct Kernels {
  static void stage(const StageArgs& a, const Ell& A, int has_m2, cudaStream_t st) {
    if (a.n == 0) return;
    const unsigned g = blocks_for(a.n, 128);
    if constexpr (MIXED) {
      const bool pdl = a.pdl != 0;
      if (a.mask != nullptr && a.tma_grid > 0 && a.tma_nbuf == 3 && a.tma_ell && a.ell_wmax <= kTmaStageEllWidth) {
        const int smem = tma_pf_smem_bytes(MR::NE + MR::NS, a.ell_wmax);
        const int64_t ntiles = (a.n + kTmaTile - 1) / kTmaTile;
        const unsigned g2 = (unsigned)std::min<int64_t>(a.tma_grid, ntiles);
        if (has_m2) launch_k(pdl, stage_kernel_mixed_tma_pf<MR, true>, g2, kTmaTile, smem, st, a, A);
        else launch_k(pdl, stage_kernel_mixed_tma_pf<MR, false>, g2, kTmaTile, smem, st, a, A);
      } else if (a.mask != nullptr && a.tma_grid > 0) {
        const int smem = (a.tma_nbuf == 3 ? 1 : a.tma_nbuf) * tma_smem_bytes(MR::NE + MR::NS, a.ell_wmax, a.tma_ell);
        // no more CTAs than tiles (small problems)
        const int64_t ntiles = (a.n + kTmaTile - 1) / kTmaTile;
        const unsigned g2 = (unsigned)std::min<int64_t>(a.tma_grid, ntiles);
        if (has_m2) launch_k(pdl, stage_kernel_mixed_tma<MR, true>, g2, kTmaTile, smem, st, a, A);
        else launch_k(pdl, stage_kernel_mixed_tma<MR, false>, g2, kTmaTile, smem, st, a, A);
      } else if (has_m2) {
        launch_k(pdl, stage_kernel_mixed<MR, true>, g, 128, 0, st, a, A);
      } else {
        launch_k(pdl, stage_kernel_mixed<MR, false>, g, 128, 0, st, a, A);
      }
    } else {
      if (has_m2) stage_kernel_fp64<MR, true><<<g, 128, 0, st>>>(a, A);
      else stage_kernel_fp64<MR, false><<<g, 128, 0, st>>>(a, A);
    }
  }
  static void inner(const InnerArgs& a, const Ell& A, cudaStream_t st) {
    if (a.n == 0) return;
    if constexpr (MIXED) {
      const bool pdl = a.pdl != 0;
      if (a.ell_wmax <= 8) launch_k(pdl, inner_kernel_mixed_w<8>, blocks_for(a.n, 256), 256, 0, st, a, A);
      else launch_k(pdl, inner_kernel_mixed, blocks_for(a.n, 256), 256, 0, st, a, A);
    }
    else inner_kernel_fp64<<<blocks_for(a.n, 256), 256, 0, st>>>(a, A);
  }
  static void power_F(const PowerFArgs& a, const Ell& A, const ReduceScratch& rs, cudaStream_t st) {
    powerF_kernel<MIXED><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, A, rs);
  }
  static void power_S(const PowerSArgs& a, const ReduceScratch& rs, cudaStream_t st) {
    if constexpr (MIXED) powerS_dual_kernel<MDu, Z><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, rs);
    else powerS_kernel<MD, Z><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, rs);
  }
  // grid > 0: cooperative launch of that many CTAs (at most) with the atomic
  // grid barrier; grid < 0: one cluster of -grid CTAs with the hardware
  // cluster barrier.
  static cudaError_t power_fused(const PowerFusedArgs& a, const Ell& A, int grid, cudaStream_t st) {
    PowerFusedArgs ac = a;
    Ell Ac = A;
    if (grid < 0) {
      cudaLaunchConfig_t cfg = {};
      // the device-resident step's CTA size where it fits (the smallest
      // multiple of 32 that gives every node a thread): the same launch
      // shape adds the norms' partial sums in the same order in both
      const int64_t per = (a.n + (-grid) - 1) / (-grid);
      const int block = (int)std::min<int64_t>(kReduceBlock, std::max<int64_t>(32, (per + 31) / 32 * 32));
      cfg.gridDim = dim3(-grid);
      cfg.blockDim = dim3(block);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = -grid;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, power_fused_kernel<MD, MDu, Z, MIXED, true>, ac, Ac);
    }
    cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    void* args[] = {&ac, &Ac};
    const int64_t need = (a.n + kReduceBlock - 1) / kReduceBlock;
    const int g = (int)std::min<int64_t>(grid, std::max<int64_t>(need, 1));
    return cudaLaunchCooperativeKernel((const void*)power_fused_kernel<MD, MDu, Z, MIXED>, dim3(g),
                                       dim3(kReduceBlock), args, 0, st);
  }
  // CTAs of one cluster for the single-cluster variant: 16 where the device
  // takes clusters of 16 (non-portable size), else 8, else 0
  static int power_cluster_size(int device) {
    (void)device;
    auto k = power_fused_kernel<MD, MDu, Z, MIXED, true>;
    for (int cl : {16, 8}) {
      if (cl > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(kReduceBlock);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) == cudaSuccess && nclusters > 0) return cl;
      cudaGetLastError();
    }
    return 0;
  }
  static cudaError_t step_fused(const FusedStepArgs& a, const Ell& A, int cluster, cudaStream_t st) {
    FusedStepArgs ac = a;
    Ell Ac = A;
    const int64_t per = (a.n + cluster - 1) / cluster;
    const int block = (int)std::min<int64_t>(FusedBlock<MR>::value, std::max<int64_t>(32, (per + 31) / 32 * 32));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(block);
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, step_fused_kernel<MD, MR, MDu, Z, MIXED>, ac, Ac);
  }
  // CTAs of the fused step's cluster: 16 where the device allows a
  // non-portable cluster of that size, else 8, else 0 (no fused step)
  static int step_fused_cluster_size(int device) {
    (void)device;
    auto k = step_fused_kernel<MD, MR, MDu, Z, MIXED>;
    for (int cl : {16, 8}) {
      if (cl > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(FusedBlock<MR>::value);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) == cudaSuccess && nclusters > 0) return cl;
      cudaGetLastError();
    }
    return 0;
  }
  static int step_fused_block(void) { return FusedBlock<MR>::value; }
  static int power_fused_grid(int device) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, power_fused_kernel<MD, MDu, Z, MIXED>, kReduceBlock, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return per_sm * sms;
  }
  static void fS_eval(const PowerSArgs& a, double* out, cudaStream_t st) {
    if (a.n == 0) return;
    fS_kernel<MD, Z><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, out);
  }
  static void state_sumsq(int64_t n, int64_t ld, int nz, const double* V, const void* Zb, const ReduceScratch& rs,
                          int slot, cudaStream_t st) {
    state_sumsq_kernel<Z><<<reduce_grid(n), kReduceBlock, 0, st>>>(n, ld, nz, V, static_cast<const Z*>(Zb), rs,
                                                                    slot);
  }
  static void convert_z(int64_t count, const void* src, double* dst, int to_double, cudaStream_t st) {
    if (count == 0) return;
    unsigned g = blocks_for(count, 256);
    if (g > 4096) g = 4096;
    convert_kernel<Z><<<g, 256, 0, st>>>(count, src, dst, to_double);
  }
  // CTAs of the persistent bulk-copy stage kernel: all SMs x resident CTAs
  static int tma_grid(int device, int wmax, int nbuf, int ell) {
    if constexpr (!MIXED) {
      return 0;
    } else {
      int per_sm = 0, sms = 0;
      if (nbuf == 3 && ell && wmax <= kTmaStageEllWidth) {
        const int smem = tma_pf_smem_bytes(MR::NE + MR::NS, wmax);
        cudaFuncSetAttribute(stage_kernel_mixed_tma_pf<MR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(stage_kernel_mixed_tma_pf<MR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel_mixed_tma_pf<MR, false>, kTmaTile, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        return per_sm * sms;
      }
      const int smem = (nbuf == 3 ? 1 : nbuf) * tma_smem_bytes(MR::NE + MR::NS, wmax, ell);
      cudaFuncSetAttribute(stage_kernel_mixed_tma<MR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      cudaFuncSetAttribute(stage_kernel_mixed_tma<MR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel_mixed_tma<MR, false>, kTmaTile, smem);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
      return per_sm * sms;
    }
  }
  static void fill(KernelSet* ks, int model) {
    ks->model = model;
    ks->nE = MR::NE;
    ks->nS = MR::NS;
    ks->N = 1 + MR::NE + MR::NS;
    ks->stage = &stage;
    ks->inner = &inner;
    ks->power_F = &power_F;
    ks->power_S = &power_S;
    ks->fS_eval = &fS_eval;
    ks->state_sumsq = &state_sumsq;
    ks->convert_z = &convert_z;
    ks->tma_grid = &tma_grid;
    ks->power_fused = &power_fused;
    ks->power_fused_grid = &power_fused_grid;
    ks->power_cluster_size = &power_cluster_size;
    ks->step_fused = &step_fused;
    ks->step_fused_cluster_size = &step_fused_cluster_size;
    ks->step_fused_block = &step_fused_block;
  }
};

}  // namespace emrkc

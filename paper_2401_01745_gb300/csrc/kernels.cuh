// CUDA kernels of the emRKC step (Algorithm 3) and of the power iteration
// (Algorithm 5), templated on the ionic model and on the precision mode.
//
// Data layout in HBM (structure of arrays, leading dimension ld = n rounded
// up to a multiple of 64):
//   V            double[ld]                 (every mode)
//   z block      Z[(N-1) * ld], row k = variable k+1 (Z = double or float)
//   L            sliced ELL, 32-row slices, slot-major inside a slice so that
//                a warp's loads of one slot are contiguous (Ell in launch.h)
// One thread owns one node; all per-node loads and stores are coalesced.
#pragma once

#include <cstdint>

#include "launch.h"
#include "models.cuh"

namespace emrkc {

// ---------------------------------------------------------------------------
// Sparse rows.

// FP64: sum_k L_ik x_k over the stored row (diagonal included).
__device__ __forceinline__ double ell_dot64(const Ell& A, int64_t i, const double* __restrict__ x) {
  const int64_t b = i >> 5;
  const int w = __ldg(A.width + b);
  int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
  double acc = 0.0;
  for (int k = 0; k < w; ++k, p += 32) acc += __ldg(A.val + p) * __ldg(x + __ldg(A.col + p));
  return acc;
}

// Mixed: sum_{k != i} L_ik (x_k - x_i) in FP32 (row sums of L vanish, so
// this equals (L x)_i; differences keep the FP32 sum well conditioned).
__device__ __forceinline__ float ell_diff32(const Ell& A, int64_t i, const double* __restrict__ x) {
  const int64_t b = i >> 5;
  const int w = __ldg(A.width + b);
  int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
  const float xi = (float)__ldg(x + i);
  float acc = 0.0f;
  for (int k = 0; k < w; ++k, p += 32) acc += __ldg(A.val32 + p) * ((float)__ldg(x + __ldg(A.col + p)) - xi);
  return acc;
}

// FP64 evaluation with the off-diagonal FP32 matrix (power iteration in mixed mode).
__device__ __forceinline__ double ell_diff64(const Ell& A, int64_t i, const double* __restrict__ x,
                                             const double* __restrict__ v, double q) {
  const int64_t b = i >> 5;
  const int w = __ldg(A.width + b);
  int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
  const double xi = v ? x[i] + q * v[i] : x[i];
  double acc = 0.0;
  for (int k = 0; k < w; ++k, p += 32) {
    const int32_t c = __ldg(A.col + p);
    const double xc = v ? x[c] + q * v[c] : x[c];
    acc += (double)__ldg(A.val32 + p) * (xc - xi);
  }
  return acc;
}

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

// ---------------------------------------------------------------------------
// Outer stage j: exponential Euler of the gates (Algorithm 3, Exponential_Euler),
// frozen forcing f_S(t_j, y_E), first inner RKC stage and the z-part of g_j.
template <class Model, typename R, typename Z, bool MIXED, bool HAS_M2>
__global__ void __launch_bounds__(128) stage_kernel(const StageArgs a, const Ell A) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  using M = Math<R>;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t ld = a.ld;
  const Z* __restrict__ Zm1 = static_cast<const Z*>(a.Zm1);
  const Z* __restrict__ Zm2 = static_cast<const Z*>(a.Zm2);
  Z* __restrict__ Zout = static_cast<Z*>(a.Zout);

  const double V = a.Vm1[i];
  R z[NZ > 0 ? NZ : 1];
#pragma unroll
  for (int k = 0; k < NZ; ++k) z[k] = (R)Zm1[k * ld + i];

  // y_E = y + (e^{eta Lambda} - I)(y - y_inf) on the gates
  R zE1[NE > 0 ? NE : 1];
  if constexpr (NE > 0) {
    R lam[NE], zinf[NE];
    Model::gating((R)V, z, z + NE, lam, zinf);
#pragma unroll
    for (int k = 0; k < NE; ++k) zE1[k] = z[k] + M::em1((R)a.eta * lam[k]) * (z[k] - zinf[k]);
  }
  // f_S(t_j, y_E): V-row and g_S
  R Iion;
  R gS[NS > 0 ? NS : 1];
  Model::currents((R)V, zE1, z + NE, Iion, gS);
  const R Istim = (a.mask != nullptr && a.mask[i]) ? (R)a.stim : R(0);
  R F;
  if constexpr (MIXED) F = (Istim - Iion) * (R)a.inv_Cm;
  else F = (Istim - Iion) / (R)a.Cm;

  // z-part of g_j = nu g_{j-1} + kappa g_{j-2} + mu dt f_bar, with
  // f_bar = ((y_E - y)/eta on the gates, c_m g_S on z_S)
  if constexpr (NZ > 0) {
    const R nu = (R)a.nu, kap = (R)a.kappa, mudt = (R)a.mu_dt;
#pragma unroll
    for (int k = 0; k < NZ; ++k) {
      R fbar;
      if (k < NE) {
        if constexpr (MIXED) fbar = (zE1[k < NE ? k : 0] - z[k]) * (R)(1.0 / a.eta);
        else fbar = (zE1[k < NE ? k : 0] - z[k]) / (R)a.eta;
      } else {
        fbar = (R)a.cm_inner * gS[k >= NE ? k - NE : 0];
      }
      R out;
      if constexpr (HAS_M2) out = nu * z[k] + kap * (R)Zm2[k * ld + i] + mudt * fbar;
      else out = z[k] + mudt * fbar;
      Zout[k * ld + i] = (Z)out;
    }
  }

  // first inner stage needs L V_{j-1}
  double LV;
  if constexpr (MIXED) LV = (double)ell_diff32(A, i, a.Vm1);
  else LV = ell_dot64(A, i, a.Vm1);

  if (a.Vn_copy != nullptr) a.Vn_copy[i] = V;
  if (a.m == 1) {
    double fbarV;
    if constexpr (MIXED) {
      fbarV = (double)((float)(a.mu1_eta / a.eta) * ((float)LV + F));
    } else {
      const double u1 = V + a.mu1_eta * (LV + (double)F);
      fbarV = (u1 - V) / a.eta;
    }
    double Vnew;
    if constexpr (HAS_M2) Vnew = a.nu * V + a.kappa * a.Vm2[i] + a.mu_dt * fbarV;
    else Vnew = V + a.mu_dt * fbarV;
    a.Vout[i] = Vnew;
    if (a.final_stage) step_epilogue(i, a.Vn[i], Vnew, a.act, a.t_n, a.dt, a.threshold, a.flags);
  } else {
    a.U1[i] = V + a.mu1_eta * (LV + (double)F);
    static_cast<R*>(a.F)[i] = F;
  }
}

// Inner RKC stage k >= 2 (Algorithm 1 applied to f_u = f_F + frozen f_S).
template <typename R, bool MIXED>
__global__ void __launch_bounds__(256) inner_kernel(const InnerArgs a, const Ell A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  double Lu;
  if constexpr (MIXED) Lu = (double)ell_diff32(A, i, a.u1);
  else Lu = ell_dot64(A, i, a.u1);
  const double F = (double)static_cast<const R*>(a.F)[i];
  const double uk = a.nu * a.u1[i] + a.kappa * a.u2[i] + a.mu_eta * (Lu + F);
  if (!a.last) {
    a.uk[i] = uk;
    return;
  }
  const double V1 = a.Vm1[i];
  double fbar;
  if constexpr (MIXED) fbar = (uk - V1) * (1.0 / a.eta);
  else fbar = (uk - V1) / a.eta;
  double Vnew;
  if (a.Vm2 != nullptr) Vnew = a.onu * V1 + a.okappa * a.Vm2[i] + a.omu_dt * fbar;
  else Vnew = V1 + a.omu_dt * fbar;
  a.Vout[i] = Vnew;
  if (a.final_stage) step_epilogue(i, a.Vn[i], Vnew, a.act, a.t_n, a.dt, a.threshold, a.flags);
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
      fz = ell_diff64(A, i, a.V, a.v_old, a.q);
      fy = ell_diff64(A, i, a.V, nullptr, 0.0);
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

template <class MD, class MR, typename R, typename Z, bool MIXED>
struct Kernels {
  static void stage(const StageArgs& a, const Ell& A, int has_m2, cudaStream_t st) {
    if (a.n == 0) return;
    if (has_m2)
      stage_kernel<MR, R, Z, MIXED, true><<<blocks_for(a.n, 128), 128, 0, st>>>(a, A);
    else
      stage_kernel<MR, R, Z, MIXED, false><<<blocks_for(a.n, 128), 128, 0, st>>>(a, A);
  }
  static void inner(const InnerArgs& a, const Ell& A, cudaStream_t st) {
    if (a.n == 0) return;
    inner_kernel<R, MIXED><<<blocks_for(a.n, 256), 256, 0, st>>>(a, A);
  }
  static void power_F(const PowerFArgs& a, const Ell& A, const ReduceScratch& rs, cudaStream_t st) {
    powerF_kernel<MIXED><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, A, rs);
  }
  static void power_S(const PowerSArgs& a, const ReduceScratch& rs, cudaStream_t st) {
    powerS_kernel<MD, Z><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, rs);
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
  }
};

}  // namespace emrkc

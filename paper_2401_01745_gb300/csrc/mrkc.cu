// mRKC (Algorithm 2) for the monodomain system with the stiffest-gate split
// of Sec. 3.3, FP64:
//   f~_F(y) = f_F(y) + f_E^1(y),   f~_S(t, y) = f_S(t, y) + f_E^2(y),
// where f_E^1 is the exponential-type right-hand side Lambda_k (z_k - z_inf,k)
// of the single stiffest gate k = kStiff (the sodium activation m of HH and
// TTP06, z_E[0]; the one gate of the passive model) and f_E^2 that of every
// other gate.  There is no exponential step: every gate is integrated by the
// RKC iterations.
//
// One outer stage j runs the inner RKC iteration over u' = f~_F(u) +
// f~_S(t_j, g_{j-1}) on [0, eta], u(0) = g_{j-1}.  Only V and z_k feel f~_F;
// every other component sees a constant forcing, which the inner RKC
// integrates exactly (c_m = 1), so its averaged force is f~_S itself.  The
// stage kernel evaluates f~_S, writes those components of g_j and the first
// inner stage of (V, z_k); the inner kernels run stages 2..m on (V, z_k), the
// gate rate evaluated at the inner V; the last one forms the (V, z_k) part of
// g_j.
#include "kernels.cuh"

namespace emrkc {

template <class Model>
struct Stiff {
  static constexpr int k = Model::NE > 0 ? 0 : -1;
};

template <class Model, bool HAS_M2>
__global__ void __launch_bounds__(128) mrkc_stage_kernel(const MrkcArgs a, const Ell A) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  constexpr int KS = Stiff<Model>::k;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t ld = a.ld;
  const double V = a.Vm1[i];
  double z[NZ > 0 ? NZ : 1];
#pragma unroll
  for (int k = 0; k < NZ; ++k) z[k] = a.Zm1[k * ld + i];
  double lam[NE > 0 ? NE : 1], zinf[NE > 0 ? NE : 1];
  if constexpr (NE > 0) Model::gating(V, z, z + NE, lam, zinf);
  double Iion;
  double gS[NS > 0 ? NS : 1];
  Model::currents(V, z, z + NE, Iion, gS);
  const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
  const double F = (Istim - Iion) * a.inv_Cm;
  // components with constant inner forcing: f_bar = f~_S
#pragma unroll
  for (int k = 0; k < NZ; ++k) {
    if (k == KS) continue;
    const double fbar = (k < NE) ? lam[k < NE ? k : 0] * (z[k] - zinf[k < NE ? k : 0]) : gS[k >= NE ? k - NE : 0];
    double out;
    if constexpr (HAS_M2) out = a.nu * z[k] + a.kappa * a.Zm2[k * ld + i] + a.mu_dt * fbar;
    else out = z[k] + a.mu_dt * fbar;
    a.Zout[k * ld + i] = out;
  }
  const double LV = ell_dot64(A, i, a.Vm1);
  double fm = 0.0;
  if constexpr (KS >= 0) fm = lam[KS] * (z[KS] - zinf[KS]);
  if (a.m == 1) {
    // (u_1 - y)/eta = mu~_1 (f~_F(y) + f~_S(y)) on V and z_k
    const double fbarV = a.mu1 * (LV + F);
    double Vnew;
    if constexpr (HAS_M2) Vnew = a.nu * V + a.kappa * a.Vm2[i] + a.mu_dt * fbarV;
    else Vnew = V + a.mu_dt * fbarV;
    a.Vout[i] = Vnew;
    if constexpr (KS >= 0) {
      const double fbarm = a.mu1 * fm;
      double out;
      if constexpr (HAS_M2) out = a.nu * z[KS] + a.kappa * a.Zm2[KS * ld + i] + a.mu_dt * fbarm;
      else out = z[KS] + a.mu_dt * fbarm;
      a.Zout[KS * ld + i] = out;
    }
    if (a.final_stage) step_epilogue(i, a.Vn[i], Vnew, a.act, a.t_n, a.dt, a.threshold, a.flags);
  } else {
    a.uVk[i] = V + a.mu1_eta * (LV + F);
    if constexpr (KS >= 0) a.umk[i] = z[KS] + a.mu1_eta * fm;
    a.F[i] = F;
  }
}

// Inner RKC stage k >= 2 on (V, z_k): u_k = nu u_{k-1} + kappa u_{k-2} +
// mu eta (f~_F(u_{k-1}) + f~_S(y)); f~_S(y) is F on V and 0 on z_k.
template <class Model>
__global__ void __launch_bounds__(128) mrkc_inner_kernel(const MrkcArgs a, const Ell A) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  constexpr int KS = Stiff<Model>::k;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const int64_t ld = a.ld;
  const double uV = a.uV1[i];
  const double Lu = ell_dot64(A, i, a.uV1);
  const double uVk = a.inu * uV + a.ikappa * a.uV2[i] + a.imu_eta * (Lu + a.F[i]);
  double umk = 0.0;
  if constexpr (KS >= 0) {
    // the gate's rate at the inner V (the other arguments from y = g_{j-1})
    double z[NZ];
#pragma unroll
    for (int k = 0; k < NZ; ++k) z[k] = a.Zm1[k * ld + i];
    const double um = a.um1[i];
    z[KS] = um;
    double lam[NE], zinf[NE];
    Model::gating(uV, z, z + NE, lam, zinf);
    umk = a.inu * um + a.ikappa * a.um2[i] + a.imu_eta * (lam[KS] * (um - zinf[KS]));
  }
  if (!a.last) {
    a.uVk[i] = uVk;
    if constexpr (KS >= 0) a.umk[i] = umk;
    return;
  }
  const double V1 = a.Vm1[i];
  const double fbarV = (uVk - V1) * a.inv_eta;
  double Vnew;
  if (a.Vm2 != nullptr) Vnew = a.nu * V1 + a.kappa * a.Vm2[i] + a.mu_dt * fbarV;
  else Vnew = V1 + a.mu_dt * fbarV;
  a.Vout[i] = Vnew;
  if constexpr (KS >= 0) {
    const double m1 = a.Zm1[KS * ld + i];
    const double fbarm = (umk - m1) * a.inv_eta;
    double out;
    if (a.Zm2 != nullptr) out = a.nu * m1 + a.kappa * a.Zm2[KS * ld + i] + a.mu_dt * fbarm;
    else out = m1 + a.mu_dt * fbarm;
    a.Zout[KS * ld + i] = out;
  }
  if (a.final_stage) step_epilogue(i, a.Vn[i], Vnew, a.act, a.t_n, a.dt, a.threshold, a.flags);
}

// Algorithm 5 on f~_F over the block (V, z_k): v_new = f~_F(y + q v) - f~_F(y)
// with v = (v_V, v_k) in two rows of ld.
template <class Model>
__global__ void __launch_bounds__(kReduceBlock) mrkc_powerF_kernel(const MrkcPowerArgs a, const Ell A,
                                                                   const ReduceScratch rs) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  constexpr int KS = Stiff<Model>::k;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i >> 5;
    const int w = A.width[b];
    int64_t p = A.slice_ptr[b] + (i & 31);
    double fz = 0.0, fy = 0.0;
    for (int k = 0; k < w; ++k, p += 32) {
      const int32_t c = A.col[p];
      fz += A.val[p] * (a.V[c] + a.q * a.v_old[c]);
      fy += A.val[p] * a.V[c];
    }
    const double w0 = fz - fy;
    double w1 = 0.0;
    if constexpr (KS >= 0) {
      double z[NZ];
#pragma unroll
      for (int k = 0; k < NZ; ++k) z[k] = a.Z[k * a.ld + i];
      const double V = a.V[i];
      double lam[NE], zinf[NE];
      Model::gating(V, z, z + NE, lam, zinf);
      const double f0 = lam[KS] * (z[KS] - zinf[KS]);
      const double Vq = V + a.q * a.v_old[i];
      z[KS] = z[KS] + a.q * a.v_old[a.ld + i];
      Model::gating(Vq, z, z + NE, lam, zinf);
      w1 = lam[KS] * (z[KS] - zinf[KS]) - f0;
    }
    a.v_new[i] = w0;
    a.v_new[a.ld + i] = w1;
    acc += w0 * w0 + w1 * w1;
  }
  reduce_finish(acc, rs, a.slot);
}

// f~_S at a full state: f_S plus the exponential-type rows of every gate but k.
template <class Model>
__device__ __forceinline__ void fS_tilde(const double* y, double Istim, double Cm, double* out) {
  constexpr int NE = Model::NE, NS = Model::NS;
  constexpr int KS = Stiff<Model>::k;
  double I;
  double gS[NS > 0 ? NS : 1];
  Model::currents(y[0], y + 1, y + 1 + NE, I, gS);
  out[0] = (Istim - I) / Cm;
  if constexpr (NE > 0) {
    double lam[NE], zinf[NE];
    Model::gating(y[0], y + 1, y + 1 + NE, lam, zinf);
#pragma unroll
    for (int k = 0; k < NE; ++k) out[1 + k] = (k == KS) ? 0.0 : lam[k] * (y[1 + k] - zinf[k]);
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) out[1 + NE + k] = gS[k];
}

template <class Model>
__device__ __forceinline__ void load_state64(const PowerSArgs& a, int64_t i, double* y) {
  constexpr int N = 1 + Model::NE + Model::NS;
  const double* Zs = static_cast<const double*>(a.Z);
  y[0] = a.V[i];
#pragma unroll
  for (int k = 1; k < N; ++k) y[k] = Zs[(k - 1) * a.ld + i];
}

template <class Model>
__global__ void __launch_bounds__(kReduceBlock) mrkc_powerS_kernel(const PowerSArgs a, const ReduceScratch rs) {
  constexpr int N = 1 + Model::NE + Model::NS;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    double y[N], f[N];
    load_state64<Model>(a, i, y);
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] = y[k] + a.q * a.v_old[k * a.ld + i];
    const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
    fS_tilde<Model>(y, Istim, a.Cm, f);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const double w = f[k] - a.fy[k * a.ld + i];
      a.v_new[k * a.ld + i] = w;
      acc += w * w;
    }
  }
  reduce_finish(acc, rs, a.slot);
}

template <class Model>
__global__ void __launch_bounds__(kReduceBlock) mrkc_fS_kernel(const PowerSArgs a, double* out) {
  constexpr int N = 1 + Model::NE + Model::NS;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    double y[N], f[N];
    load_state64<Model>(a, i, y);
    const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
    fS_tilde<Model>(y, Istim, a.Cm, f);
#pragma unroll
    for (int k = 0; k < N; ++k) out[k * a.ld + i] = f[k];
  }
}

template <class Model>
struct MrkcLaunch {
  static void stage(const MrkcArgs& a, const Ell& A, bool has_m2, cudaStream_t st) {
    if (a.n == 0) return;
    const unsigned g = blocks_for(a.n, 128);
    if (has_m2) mrkc_stage_kernel<Model, true><<<g, 128, 0, st>>>(a, A);
    else mrkc_stage_kernel<Model, false><<<g, 128, 0, st>>>(a, A);
  }
  static void inner(const MrkcArgs& a, const Ell& A, cudaStream_t st) {
    if (a.n == 0) return;
    mrkc_inner_kernel<Model><<<blocks_for(a.n, 128), 128, 0, st>>>(a, A);
  }
  static void power_F(const MrkcPowerArgs& a, const Ell& A, const ReduceScratch& rs, cudaStream_t st) {
    mrkc_powerF_kernel<Model><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, A, rs);
  }
  static void power_S(const PowerSArgs& a, const ReduceScratch& rs, cudaStream_t st) {
    mrkc_powerS_kernel<Model><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, rs);
  }
  static void fS(const PowerSArgs& a, double* out, cudaStream_t st) {
    if (a.n == 0) return;
    mrkc_fS_kernel<Model><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, out);
  }
  static void fill(MrkcKernels* k) {
    k->stage = &stage;
    k->inner = &inner;
    k->power_F = &power_F;
    k->power_S = &power_S;
    k->fS = &fS;
    k->stiff_gate = Stiff<Model>::k;
  }
};

bool get_kernels_mrkc(int model, MrkcKernels* k) {
  switch (model) {
    case 0: MrkcLaunch<ModelNone<double>>::fill(k); return true;
    case 1: MrkcLaunch<ModelPassive<double>>::fill(k); return true;
    case 2: MrkcLaunch<ModelHH<double>>::fill(k); return true;
    case 3: MrkcLaunch<ModelTTP06<double>>::fill(k); return true;
    default: return false;
  }
}

}  // namespace emrkc

// The comparison integrators of Sec. 5, FP64:
//
//  EXEX-RL (Sec. 5, the fine-step reference solver): one fused kernel per
//    step -- exponential Euler of the gates with V frozen, explicit Euler of
//    z_S, then explicit Euler of V with the diffusion SpMV.
//  IMEX-RL (Algorithm 4): the same ionic update, then the implicit diffusion
//    step (Cm M + dt K / chi) V_{n+1} = Cm M V_n + dt M (I_stim - I_ion),
//    solved on the device by Jacobi-preconditioned conjugate gradients in one
//    persistent cooperative launch.
//
// With L = -(chi Cm M)^-1 K (the stored matrix) the system is B x = c with
// B = I - dt L and c = V_n + dt (I_stim - I_ion) / Cm.  B is self-adjoint in
// the lumped-mass inner product <u, v>_M = sum_i M_i u_i v_i (M B = M + dt K /
// (chi Cm) is symmetric), so CG runs in that inner product with the Jacobi
// preconditioner P = diag(B) = 1 - dt L_ii; this is CG on the symmetric
// system M B x = M c with its diagonal as preconditioner.  The solve stops
// when ||r||_M <= rtol ||c||_M or after max_iter iterations, warm started
// from x_0 = V_n.

#include "kernels.cuh"

namespace emrkc {

// ---------------------------------------------------------------------------
// Ionic half of Algorithm 4 at one node: z_E by exponential Euler over dt
// with V frozen, z_S by explicit Euler with the updated gates, I_ion with
// both updated.  Returns F = (I_stim - I_ion) / Cm and writes the new z.
template <class Model>
__device__ __forceinline__ double rl_ionic(const RlArgs& a, int64_t i, double V) {
  constexpr int NE = Model::NE, NS = Model::NS, NZ = NE + NS;
  using M = Math<double>;
  const int64_t ld = a.ld;
  double z[NZ > 0 ? NZ : 1];
#pragma unroll
  for (int k = 0; k < NZ; ++k) z[k] = a.Z[k * ld + i];
  double zE1[NE > 0 ? NE : 1];
  if constexpr (NE > 0) {
    double lam[NE], zinf[NE];
    Model::gating(V, z, z + NE, lam, zinf);
#pragma unroll
    for (int k = 0; k < NE; ++k) zE1[k] = z[k] + M::em1(a.dt * lam[k]) * (z[k] - zinf[k]);
  }
  double Iion;
  double gS[NS > 0 ? NS : 1];
  double zS1[NS > 0 ? NS : 1];
  Model::currents(V, zE1, z + NE, Iion, gS);
  if constexpr (NS > 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) zS1[k] = z[NE + k] + a.dt * gS[k];
    double gS_unused[NS];
    Model::currents(V, zE1, zS1, Iion, gS_unused);
  }
#pragma unroll
  for (int k = 0; k < NE; ++k) a.Zout[k * ld + i] = zE1[k];
#pragma unroll
  for (int k = 0; k < NS; ++k) a.Zout[(NE + k) * ld + i] = zS1[k];
  const double Istim = (a.mask != nullptr && a.mask[i]) ? a.stim : 0.0;
  return (Istim - Iion) * a.inv_Cm;
}

// (L x)_i and L_ii from the FP64 sliced ELL (the diagonal is stored).
__device__ __forceinline__ double ell_dot_diag(const Ell& A, int64_t i, const double* __restrict__ x, double& dii) {
  const int64_t b = i >> 5;
  const int w = __ldg(A.width + b);
  int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
  double acc = 0.0, d = 0.0;
  for (int k = 0; k < w; ++k, p += 32) {
    const int32_t c = __ldg(A.col + p);
    const double v = __ldg(A.val + p);
    acc += v * __ldg(x + c);
    if (c == i) d += v;
  }
  dii = d;
  return acc;
}

// EXEX-RL: V_{n+1} = V_n + dt (L V_n + (I_stim - I_ion(V_n, z_E,n+1, z_S,n+1)) / Cm).
template <class Model>
__global__ void __launch_bounds__(128) exex_rl_kernel(const RlArgs a, const Ell A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const double V = a.V[i];
  const double F = rl_ionic<Model>(a, i, V);
  const double Vnew = V + a.dt * (ell_dot64(A, i, a.V) + F);
  a.Vout[i] = Vnew;
  step_epilogue(i, V, Vnew, a.act, a.t_n, a.dt, a.threshold, a.flags);
}

// IMEX-RL, ionic half and PCG set-up: x_0 = V_n, r_0 = c - B x_0 =
// dt (F + L V_n), z_0 = P^-1 r_0.  Per-CTA partial sums of <r_0, z_0>_M,
// <r_0, r_0>_M and <c, c>_M go to part0[4 b + 0..2]; the PCG launch adds them.
template <class Model>
__global__ void __launch_bounds__(kReduceBlock) imex_rl_setup_kernel(const RlArgs a, const Ell A) {
  __shared__ double sh[32];
  double rz = 0.0, rr = 0.0, cc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double V = a.V[i];
    const double F = rl_ionic<Model>(a, i, V);
    double Lii;
    const double LV = ell_dot_diag(A, i, a.V, Lii);
    const double c = V + a.dt * F;
    const double r = a.dt * (F + LV);
    const double pinv = 1.0 / (1.0 - a.dt * Lii);
    const double z = pinv * r;
    const double m = a.mass[i];
    a.Vout[i] = V;
    a.r[i] = r;
    a.zr[i] = z;
    a.pinv[i] = pinv;
    rz += m * r * z;
    rr += m * r * r;
    cc += m * c * c;
  }
  const double t0 = block_sum(rz, sh);
  const double t1 = block_sum(rr, sh);
  const double t2 = block_sum(cc, sh);
  if (threadIdx.x == 0) {
    a.part0[4 * blockIdx.x + 0] = t0;
    a.part0[4 * blockIdx.x + 1] = t1;
    a.part0[4 * blockIdx.x + 2] = t2;
  }
}

// The PCG iterations of the implicit diffusion step, one cooperative launch.
// Loads of vectors written by other CTAs within the launch go through L2.
__global__ void __launch_bounds__(kPcgBlock) imex_pcg_kernel(const PcgArgs a, const Ell A) {
  __shared__ double sh[32];
  const double cc = sum_partials(a.part0, a.n_part0, 2, sh);
  const double rtol2_cc = a.rtol * a.rtol * cc;
  double rz = sum_partials(a.part0, a.n_part0, 0, sh);
  double rr = sum_partials(a.part0, a.n_part0, 1, sh);
  double rz_prev = 1.0;
  int it = 0;
  const double* p_old = a.p1;
  double* p_new = a.p0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  while (it < a.max_iter && rr > rtol2_cc) {
    const double beta = (it == 0) ? 0.0 : rz / rz_prev;
    // q = B p_new with p_new = z + beta p_old, gathered on the fly; <p, q>_M
    double pq = 0.0;
    for (int64_t i = i0; i < a.n; i += stride) {
      const int64_t b = i >> 5;
      const int w = __ldg(A.width + b);
      int64_t p = __ldg(A.slice_ptr + b) + (i & 31);
      double acc = 0.0;
      for (int k = 0; k < w; ++k, p += 32) {
        const int32_t c = __ldg(A.col + p);
        const double pc = (it == 0) ? __ldcg(a.zr + c) : __ldcg(a.zr + c) + beta * __ldcg(p_old + c);
        acc += __ldg(A.val + p) * pc;
      }
      const double pi = (it == 0) ? __ldcg(a.zr + i) : __ldcg(a.zr + i) + beta * __ldcg(p_old + i);
      const double q = pi - a.dt * acc;
      p_new[i] = pi;
      a.q[i] = q;
      pq += a.mass[i] * pi * q;
    }
    {
      const double t = block_sum(pq, sh);
      if (threadIdx.x == 0) a.part[4 * blockIdx.x + 0] = t;
    }
    if (!grid_barrier(a.bar, a.flags, a.spin_limit)) return;
    const double alpha = rz / sum_partials(a.part, gridDim.x, 0, sh);
    // x += alpha p; r -= alpha q; z = P^-1 r; <r, z>_M, <r, r>_M
    double s_rz = 0.0, s_rr = 0.0;
    for (int64_t i = i0; i < a.n; i += stride) {
      const double pi = p_new[i];
      a.x[i] += alpha * pi;
      const double r = a.r[i] - alpha * a.q[i];
      const double z = a.pinv[i] * r;
      a.r[i] = r;
      a.zr[i] = z;
      const double m = a.mass[i];
      s_rz += m * r * z;
      s_rr += m * r * r;
    }
    {
      const double t1 = block_sum(s_rz, sh);
      const double t2 = block_sum(s_rr, sh);
      if (threadIdx.x == 0) {
        a.part[4 * blockIdx.x + 1] = t1;
        a.part[4 * blockIdx.x + 2] = t2;
      }
    }
    if (!grid_barrier(a.bar, a.flags, a.spin_limit)) return;
    rz_prev = rz;
    rz = sum_partials(a.part, gridDim.x, 1, sh);
    rr = sum_partials(a.part, gridDim.x, 2, sh);
    const double* t = p_new;
    p_new = const_cast<double*>(p_old);
    p_old = t;
    ++it;
  }
  // epilogue: activation times and the non-finite flag on (V_n, V_{n+1})
  for (int64_t i = i0; i < a.n; i += stride) step_epilogue(i, a.Vn[i], a.x[i], a.act, a.t_n, a.dt, a.threshold, a.flags);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.iters[0] = (unsigned long long)it;
    a.iters[1] += (unsigned long long)it;
    a.res[0] = rr;
    a.res[1] = cc;
  }
}

template <class Model>
static void launch_exex(const RlArgs& a, const Ell& A, cudaStream_t st) {
  if (a.n == 0) return;
  exex_rl_kernel<Model><<<blocks_for(a.n, 128), 128, 0, st>>>(a, A);
}

template <class Model>
static void launch_imex_setup(const RlArgs& a, const Ell& A, int grid, cudaStream_t st) {
  imex_rl_setup_kernel<Model><<<grid, kReduceBlock, 0, st>>>(a, A);
}

int rl_exex_step(int model, const RlArgs& a, const Ell& A, cudaStream_t st) {
  switch (model) {
    case 0: launch_exex<ModelNone<double>>(a, A, st); break;
    case 1: launch_exex<ModelPassive<double>>(a, A, st); break;
    case 2: launch_exex<ModelHH<double>>(a, A, st); break;
    case 3: launch_exex<ModelTTP06<double>>(a, A, st); break;
    default: return -1;
  }
  return 0;
}

int rl_imex_setup_grid(int64_t n) { return reduce_grid(n); }

int rl_imex_setup(int model, const RlArgs& a, const Ell& A, cudaStream_t st) {
  const int g = reduce_grid(a.n);
  switch (model) {
    case 0: launch_imex_setup<ModelNone<double>>(a, A, g, st); break;
    case 1: launch_imex_setup<ModelPassive<double>>(a, A, g, st); break;
    case 2: launch_imex_setup<ModelHH<double>>(a, A, g, st); break;
    case 3: launch_imex_setup<ModelTTP06<double>>(a, A, g, st); break;
    default: return -1;
  }
  return 0;
}

int pcg_grid(int device) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, imex_pcg_kernel, kPcgBlock, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}

cudaError_t rl_imex_pcg(const PcgArgs& a, const Ell& A, int grid, cudaStream_t st) {
  const int64_t need = (a.n + kPcgBlock - 1) / kPcgBlock;
  int g = (int)std::min<int64_t>(grid, std::max<int64_t>(need, 1));
  PcgArgs ac = a;
  Ell Ac = A;
  void* args[] = {&ac, &Ac};
  return cudaLaunchCooperativeKernel((const void*)imex_pcg_kernel, dim3(g), dim3(kPcgBlock), args, 0, st);
}

}  // namespace emrkc

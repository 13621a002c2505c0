// Host runtime of the emRKC solver: the C ABI of include/emrkc.h.
//
// Per step (Algorithm 3):
//   rho policy -> power iteration (Algorithm 5, device kernels + host loop)
//   s = get_stages(dt, rho_S), eta = 2 dt / l_s, m = get_stages(eta, rho_F)
//   for j = 1..s: stage kernel (exponential Euler, f_S, first inner stage,
//                 z-part of g_j), then inner kernels k = 2..m (SpMV stages;
//                 the last one writes the V-part of g_j)
// Three rotating state buffers hold g_{j-2}, g_{j-1}, g_j (Sec. 3.1); three
// rotating V-sized buffers hold the inner stages u_{k-2}, u_{k-1}, u_k.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "emrkc.h"
#include "launch.h"
#include "solver_internal.h"

using namespace emrkc;

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace {

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

void free_all(emrkc_solver* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  s->harvest();
  void* ptrs[] = {s->d_slice_ptr, s->d_width, s->d_col, s->d_val, s->d_val32, s->d_V[0], s->d_V[1], s->d_V[2],
                  s->d_Z[0], s->d_Z[1], s->d_Z[2], s->d_U[0], s->d_U[1], s->d_U[2], s->d_F, s->d_mask, s->d_vF,
                  s->d_vF2, s->d_vS, s->d_vS2, s->d_fy, s->d_act, s->d_Vn, s->d_tmp, s->d_rest,
                  s->rs.partials, s->rs.ticket, s->rs.result, s->d_V32[0], s->d_V32[1], s->d_V32[2],
                  s->d_D[0], s->d_D[1], s->d_D[2], s->d_LV, s->d_Vlo[0], s->d_Vlo[1], s->d_Vlo[2],
                  s->d_Vn32, s->d_mass, s->d_cg[0], s->d_cg[1], s->d_cg[2], s->d_cg[3], s->d_cg[4],
                  s->d_cg[5], s->d_part, s->d_bar, s->d_iters, s->d_res, s->d_Um[0], s->d_Um[1], s->d_Um[2],
                  s->d_ppart, s->d_pbar, s->d_mask_alt, s->d_stage[0], s->d_stage[1], s->d_fstate,
                  s->d_ctab};
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  if (s->h2d_stream) cudaStreamSynchronize(s->h2d_stream);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  cudaEvent_t evs[] = {s->ev_mask_free[0], s->ev_mask_free[1], s->ev_mask_ready, s->ev_stage_ready[0],
                       s->ev_stage_ready[1], s->ev_stage_free[0], s->ev_stage_free[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  if (s->h2d_stream) cudaStreamDestroy(s->h2d_stream);
  if (s->h_pin) cudaFreeHost(s->h_pin);
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

// Read back reduction results [first, first+count) and the flags word in one
// copy: the flags live right after the 16 result slots (kFlagsSlot).
int read_results(emrkc_solver* s, int first, int count) {
  (void)count;
  cudaError_t e = cudaMemcpyAsync(s->h_pin + first, s->rs.result + first, (kFlagsSlot + 1 - first) * sizeof(double),
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "copy of reduction results");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "stream synchronisation");
  return EMRKC_OK;
}

int check_flags(emrkc_solver* s) {
  int flags = 0;
  std::memcpy(&flags, s->h_pin + kFlagsSlot, sizeof(int));
  if (flags & 1) {
    int zero = 0;
    cudaMemcpyAsync(s->d_flags, &zero, sizeof(int), cudaMemcpyHostToDevice, s->stream);
    cudaStreamSynchronize(s->stream);
    return s->fail(EMRKC_ERR_NONFINITE, "non-finite transmembrane potential produced by a step");
  }
  if (flags & 4) {
    int zero = 0;
    cudaMemcpyAsync(s->d_flags, &zero, sizeof(int), cudaMemcpyHostToDevice, s->stream);
    cudaStreamSynchronize(s->stream);
    return s->fail(EMRKC_ERR_TIMEOUT, "a grid barrier of the CG solve gave up");
  }
  if (flags & 16) {
    int zero = 0;
    cudaMemcpyAsync(s->d_flags, &zero, sizeof(int), cudaMemcpyHostToDevice, s->stream);
    cudaStreamSynchronize(s->stream);
    return s->fail(EMRKC_ERR_STATE, "a device-resident step needed more than 128 outer or inner stages");
  }
  return EMRKC_OK;
}

// Host copies of the device-resident step's state: rho estimates, iteration
// counts, the last stage counts, and which power-iteration buffer holds the
// last iterate (the host's pointers are swapped to match, the device's
// indices reset).  A no-op unless a device-resident step ran since the
// last call.
int fused_pull(emrkc_solver* s) {
  if (!s->fcluster || !s->fstate_stale) return EMRKC_OK;
  cudaError_t e = cudaMemcpyAsync(&s->h_fstate, s->d_fstate, sizeof(FusedStepState), cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "device step state");
  FusedStepState& h = s->h_fstate;
  s->rhoF_raw = h.rhoF_raw;
  s->rhoS_raw = h.rhoS_raw;
  s->itF = h.itF;
  s->itS = h.itS;
  s->total_it = h.total_it;
  s->last_s = h.s;
  s->last_m = h.m;
  s->last_eta = h.eta;
  s->last_rhoF = h.rhoF;
  s->last_rhoS = h.rhoS;
  if (h.curF) std::swap(s->d_vF, s->d_vF2);
  if (h.curS) std::swap(s->d_vS, s->d_vS2);
  h.curF = h.curS = 0;
  e = cudaMemcpyAsync(s->d_fstate, &h, sizeof(FusedStepState), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "device step state");
  s->fstate_stale = false;
  return EMRKC_OK;
}

// The host's rho estimates and counts into the device state (after a
// power iteration run from the host).
int fused_push(emrkc_solver* s) {
  if (!s->fcluster) return EMRKC_OK;
  FusedStepState& h = s->h_fstate;
  h.rhoF_raw = s->rhoF_raw;
  h.rhoS_raw = s->rhoS_raw;
  h.itF = s->itF;
  h.itS = s->itS;
  h.total_it = s->total_it;
  h.curF = h.curS = 0;
  cudaError_t e = cudaMemcpyAsync(s->d_fstate, &h, sizeof(FusedStepState), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "device step state");
  return EMRKC_OK;
}

// Mixed path: write V = hi + lo of the current state into the double buffer.
void materialise_V(emrkc_solver* s) {
  if (s->d_V32[s->cur]) launch_ff_join(s->d_V32[s->cur], s->d_Vlo[s->cur], s->d_V[s->cur], s->n, s->stream);
}

// Stopping test of Algorithm 5: a call with no initial guess (rho still 0)
// is a cold start from the arbitrary start vector and takes the tighter
// tolerance; warm-started calls take the App. A tolerance.
double pow_tol_for(const emrkc_solver* s, double rho_warm) {
  return rho_warm == 0.0 ? s->opt.pow_tol_cold : s->opt.pow_tol;
}
int pow_max_iter_for(const emrkc_solver* s, double rho_warm) {
  return rho_warm == 0.0 ? s->opt.pow_max_iter_cold : s->opt.pow_max_iter;
}

double stim_at(const emrkc_solver* s, double t) {
  return (s->d_mask != nullptr && s->t_on <= t && t <= s->t_off) ? s->amp : 0.0;
}

// Algorithm 5 on f_F (V block only); for mRKC on f~_F over (V, z_k).
int power_F(emrkc_solver* s) {
  materialise_V(s);
  double* V = s->d_V[s->cur];
  const bool mrkc = s->method == EMRKC_METHOD_MRKC;
  const int ks = s->mk.stiff_gate;
  const double* zk = (mrkc && ks >= 0) ? static_cast<const double*>(s->d_Z[s->cur]) + (size_t)ks * s->ld : nullptr;
  s->launch(EMRKC_PHASE_OTHER, [&] { launch_sumsq(s->n, V, s->rs, 0, s->stream); });
  s->launch(EMRKC_PHASE_OTHER, [&] {
    launch_sumsq(mrkc ? 2 * s->ld : s->n, s->d_vF, s->rs, 1, s->stream);
  });
  if (zk) s->launch(EMRKC_PHASE_OTHER, [&] { launch_sumsq(s->n, zk, s->rs, 4, s->stream); });
  int rc = read_results(s, 0, zk ? 5 : 2);
  if (rc) return rc;
  if ((rc = check_flags(s))) return rc;
  const double ny = std::sqrt(s->h_pin[0] + (zk ? s->h_pin[4] : 0.0));
  double nv = std::sqrt(s->h_pin[1]);
  const double delta = ny > 0.0 ? ny * s->opt.pow_eps : s->opt.pow_eps;
  int it = 0;
  double rho = s->rhoF_raw;
  if (nv == 0.0) {
    s->rhoF_raw = 0.0;
    s->itF = 0;
    return EMRKC_OK;
  }
  const double tol = pow_tol_for(s, rho);
  const int max_iter = pow_max_iter_for(s, rho);
  double q = delta / nv, rho_old = 0.0;
  while (std::fabs(rho - rho_old) >= tol * rho && it < max_iter) {
    rho_old = rho;
    if (mrkc) {
      MrkcPowerArgs a;
      a.n = s->n;
      a.ld = s->ld;
      a.V = V;
      a.Z = static_cast<const double*>(s->d_Z[s->cur]);
      a.v_old = s->d_vF;
      a.v_new = s->d_vF2;
      a.q = q;
      a.slot = 2;
      s->launch(EMRKC_PHASE_POWER_F, [&] { s->mk.power_F(a, s->ell, s->rs, s->stream); });
    } else {
      PowerFArgs a;
      a.n = s->n;
      a.V = V;
      a.v_old = s->d_vF;
      a.v_new = s->d_vF2;
      a.q = q;
      a.slot = 2;
      s->launch(EMRKC_PHASE_POWER_F, [&] { s->ks.power_F(a, s->ell, s->rs, s->stream); });
    }
    if ((rc = read_results(s, 2, 1))) return rc;
    std::swap(s->d_vF, s->d_vF2);
    ++it;
    nv = std::sqrt(s->h_pin[2]);
    if (nv == 0.0) {
      rho = 0.0;
      break;
    }
    q = delta / nv;
    rho = nv / delta;
  }
  s->rhoF_raw = rho;
  s->itF = it;
  s->total_it += it;
  return EMRKC_OK;
}

// Algorithm 5 on f_S (full state), evaluated in FP64.
int power_S(emrkc_solver* s) {
  materialise_V(s);
  double* V = s->d_V[s->cur];
  const int64_t rows = s->N;
  PowerSArgs a;
  a.n = s->n;
  a.ld = s->ld;
  a.V = V;
  a.Z = s->d_Z[s->cur];
  a.mask = s->d_mask;
  a.stim = stim_at(s, s->t);
  a.Cm = s->Cm;
  s->launch(EMRKC_PHASE_OTHER, [&] { s->ks.state_sumsq(s->n, s->ld, s->N - 1, V, s->d_Z[s->cur], s->rs, 0, s->stream); });
  s->launch(EMRKC_PHASE_OTHER, [&] { launch_sumsq(rows * s->ld, s->d_vS, s->rs, 1, s->stream); });
  const bool mrkc = s->method == EMRKC_METHOD_MRKC;  // f~_S = f_S + f_E^2
  // f_S(y) for the differences of Algorithm 5 (the mixed path forms J v directly)
  if (mrkc || s->precision != EMRKC_PREC_MIXED) {
    s->launch(EMRKC_PHASE_OTHER, [&] {
      if (mrkc) s->mk.fS(a, s->d_fy, s->stream);
      else s->ks.fS_eval(a, s->d_fy, s->stream);
    });
  }
  int rc = read_results(s, 0, 2);
  if (rc) return rc;
  if ((rc = check_flags(s))) return rc;
  const double ny = std::sqrt(s->h_pin[0]);
  double nv = std::sqrt(s->h_pin[1]);
  const double delta = ny > 0.0 ? ny * s->opt.pow_eps : s->opt.pow_eps;
  int it = 0;
  double rho = s->rhoS_raw;
  if (nv == 0.0) {
    s->rhoS_raw = 0.0;
    s->itS = 0;
    return EMRKC_OK;
  }
  const double tol = pow_tol_for(s, rho);
  const int max_iter = pow_max_iter_for(s, rho);
  double q = delta / nv, rho_old = 0.0;
  while (std::fabs(rho - rho_old) >= tol * rho && it < max_iter) {
    rho_old = rho;
    a.v_old = s->d_vS;
    a.v_new = s->d_vS2;
    a.fy = s->d_fy;
    a.q = q;
    a.slot = 3;
    s->launch(EMRKC_PHASE_POWER_S, [&] {
      if (mrkc) s->mk.power_S(a, s->rs, s->stream);
      else s->ks.power_S(a, s->rs, s->stream);
    });
    if ((rc = read_results(s, 3, 1))) return rc;
    std::swap(s->d_vS, s->d_vS2);
    ++it;
    nv = std::sqrt(s->h_pin[3]);
    if (nv == 0.0) {
      rho = 0.0;
      break;
    }
    q = delta / nv;
    rho = nv / delta;
  }
  s->rhoS_raw = rho;
  s->itS = it;
  s->total_it += it;
  return EMRKC_OK;
}

// EXEX-RL and IMEX-RL (Algorithm 4), FP64; state buffers cur -> cur + 1.
int do_step_rl(emrkc_solver* s, double dt) {
  const int b0 = s->cur, b1 = (s->cur + 1) % 3;
  RlArgs a;
  a.n = s->n;
  a.ld = s->ld;
  a.V = s->d_V[b0];
  a.Z = static_cast<const double*>(s->d_Z[b0]);
  a.Vout = s->d_V[b1];
  a.Zout = static_cast<double*>(s->d_Z[b1]);
  a.mask = s->d_mask;
  a.stim = stim_at(s, s->t);
  a.inv_Cm = 1.0 / s->Cm;
  a.dt = dt;
  a.act = s->act_on ? s->d_act : nullptr;
  a.t_n = s->t;
  a.threshold = s->opt.act_threshold;
  a.flags = s->d_flags;
  if (s->method == EMRKC_METHOD_EXEX_RL) {
    s->launch(EMRKC_PHASE_STAGE, [&] { rl_exex_step(s->model, a, s->ell, s->stream); });
  } else {
    a.mass = s->d_mass;
    a.r = s->d_cg[0];
    a.zr = s->d_cg[1];
    a.pinv = s->d_cg[5];
    a.part0 = s->d_part;
    s->launch(EMRKC_PHASE_STAGE, [&] { rl_imex_setup(s->model, a, s->ell, s->stream); });
    PcgArgs c;
    c.n = s->n;
    c.dt = dt;
    c.rtol = s->opt.lin_rtol;
    c.max_iter = s->opt.lin_max_iter;
    c.spin_limit = 1ll << 26;
    c.mass = s->d_mass;
    c.pinv = s->d_cg[5];
    c.Vn = s->d_V[b0];
    c.x = s->d_V[b1];
    c.r = s->d_cg[0];
    c.zr = s->d_cg[1];
    c.q = s->d_cg[2];
    c.p0 = s->d_cg[3];
    c.p1 = s->d_cg[4];
    c.part0 = s->d_part;
    c.n_part0 = rl_imex_setup_grid(s->n);
    c.part = s->d_part + 4 * kReduceMaxBlocks;
    c.res = s->d_res;
    c.bar = s->d_bar;
    c.iters = s->d_iters;
    c.flags = s->d_flags;
    c.act = a.act;
    c.t_n = s->t;
    c.threshold = s->opt.act_threshold;
    cudaError_t e = cudaMemsetAsync(s->d_bar, 0, 2 * sizeof(unsigned int), s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "barrier reset");
    s->launch(EMRKC_PHASE_INNER, [&] { e = rl_imex_pcg(c, s->ell, s->pcg_grid, s->stream); });
    if (e != cudaSuccess) return s->cuda_fail(e, "cooperative CG launch");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return s->cuda_fail(e, "kernel launch");
  s->cur = b1;
  s->t += dt;
  s->steps += 1;
  s->last_s = s->last_m = 0;
  s->last_eta = 0.0;
  return EMRKC_OK;
}

// Algorithm 5 for rho_F and rho_S in one cooperative launch (emRKC): the
// iteration loops run on the device; one read of the results.
int power_fused(emrkc_solver* s) {
  PowerFusedArgs a;
  a.n = s->n;
  a.ld = s->ld;
  a.V = s->d_V[s->cur];
  a.Vhi = s->d_V32[s->cur];  // mixed path: the kernel reads hi + lo (no join launch)
  a.Vlo = s->d_Vlo[s->cur];
  a.Z = s->d_Z[s->cur];
  a.vF[0] = s->d_vF;
  a.vF[1] = s->d_vF2;
  a.vS[0] = s->d_vS;
  a.vS[1] = s->d_vS2;
  a.fy = s->d_fy;
  a.mask = s->d_mask;
  a.stim = stim_at(s, s->t);
  a.Cm = s->Cm;
  a.f_inv_Cm = (float)(1.0 / s->Cm);
  a.ell_wmax = s->ell_wmax;
  a.eps = s->opt.pow_eps;
  a.tol = s->opt.pow_tol;
  a.max_iter = s->opt.pow_max_iter;
  a.tol_cold = s->opt.pow_tol_cold;
  a.max_iter_cold = s->opt.pow_max_iter_cold;
  a.rhoF_warm = s->rhoF_raw;
  a.rhoS_warm = s->rhoS_raw;
  a.part = s->d_ppart;
  a.bar = s->d_pbar;
  a.flags = s->d_flags;
  a.spin_limit = 1ll << 26;
  a.out = s->rs.result;
  // problems one cluster holds (at most 4 nodes per thread) take the
  // single-cluster variant; the others the cooperative grid
  const int grid = (s->pcluster > 0 && s->n <= (int64_t)4 * s->pcluster * kReduceBlock) ? -s->pcluster
                                                                                         : s->pfused_grid;
  cudaError_t e = cudaSuccess;
  s->launch(EMRKC_PHASE_POWER_S, [&] { e = s->ks.power_fused(a, s->ell, grid, s->stream); });
  if (e != cudaSuccess) return s->cuda_fail(e, "power-iteration launch");
  int rc = read_results(s, 0, 6);
  if (rc) return rc;
  if ((rc = check_flags(s))) return rc;
  s->rhoF_raw = s->h_pin[0];
  s->rhoS_raw = s->h_pin[1];
  s->itF = (int)s->h_pin[2];
  s->itS = (int)s->h_pin[3];
  s->total_it += s->itF + s->itS;
  if (s->h_pin[4] != 0.0) std::swap(s->d_vF, s->d_vF2);
  if (s->h_pin[5] != 0.0) std::swap(s->d_vS, s->d_vS2);
  return EMRKC_OK;
}

// Both spectral radii now: one cooperative launch for emRKC, the host-driven
// loops for mRKC (whose f~_F and f~_S have their own kernels).
int update_rho_now(emrkc_solver* s) {
  int rc = fused_pull(s);
  if (rc) return rc;
  if (s->method == EMRKC_METHOD_EMRKC && s->pfused_grid > 0) {
    rc = power_fused(s);
  } else {
    rc = power_F(s);
    if (!rc) rc = power_S(s);
  }
  if (!rc) rc = fused_push(s);
  return rc;
}

// rho policy shared by emRKC and mRKC: (rho_F, rho_S) with the safety factor
int step_rho(emrkc_solver* s, double* rhoF, double* rhoS) {
  int rc;
  s->itF = s->itS = 0;
  if (s->opt.rho_every == EMRKC_RHO_FIXED) {
    *rhoF = s->opt.rho_F;
    *rhoS = s->opt.rho_S;
    return EMRKC_OK;
  }
  const bool due = (s->opt.rho_every == EMRKC_RHO_ONCE) ? !s->rho_done : (s->steps % s->opt.rho_every == 0);
  if (due) {
    if ((rc = update_rho_now(s))) return rc;
    s->rho_done = true;
  }
  *rhoF = s->opt.safety * s->rhoF_raw;
  *rhoS = std::max(s->opt.safety * s->rhoS_raw, s->opt.rho_S_min);
  return EMRKC_OK;
}

// mRKC (Algorithm 2), FP64.
int do_step_mrkc(emrkc_solver* s, double dt) {
  double rhoF, rhoS;
  int rc = step_rho(s, &rhoF, &rhoS);
  if (rc) return rc;
  double l_s = 0.0;
  const int S = stages_for(dt, rhoS, s->opt.eps, &l_s);
  const double eta = 2.0 * dt / l_s;
  const int Mi = stages_for(eta, rhoF, s->opt.eps, nullptr);
  const Coeffs co = s->coeffs(S);
  const Coeffs ci = s->coeffs(Mi);
  const int b0 = s->cur;
  const int ks = s->mk.stiff_gate;
  // V_n for the activation test: buffer b0 survives the step while S <= 2
  const double* Vn = (S <= 2) ? s->d_V[b0] : s->d_Vn;
  if (S >= 3) cudaMemcpyAsync(s->d_Vn, s->d_V[b0], s->n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
  for (int j = 1; j <= S; ++j) {
    const int bm1 = (b0 + j - 1) % 3, bm2 = (b0 + j - 2 + 3) % 3, bo = (b0 + j) % 3;
    MrkcArgs a;
    a.n = s->n;
    a.ld = s->ld;
    a.Vm1 = s->d_V[bm1];
    a.Zm1 = static_cast<const double*>(s->d_Z[bm1]);
    a.Vm2 = j >= 2 ? s->d_V[bm2] : nullptr;
    a.Zm2 = j >= 2 ? static_cast<const double*>(s->d_Z[bm2]) : nullptr;
    a.Vout = s->d_V[bo];
    a.Zout = static_cast<double*>(s->d_Z[bo]);
    a.nu = j >= 2 ? co.nu[j] : 1.0;
    a.kappa = j >= 2 ? co.kappa[j] : 0.0;
    a.mu_dt = co.mu[j] * dt;
    a.eta = eta;
    a.inv_eta = 1.0 / eta;
    a.m = Mi;
    a.mu1 = ci.mu[1];
    a.mu1_eta = ci.mu[1] * eta;
    a.uVk = s->d_U[0];
    a.umk = s->d_Um[0];
    a.F = static_cast<double*>(s->d_F);
    a.mask = s->d_mask;
    a.stim = stim_at(s, s->t + co.c[j - 1] * dt);
    a.inv_Cm = 1.0 / s->Cm;
    a.final_stage = (j == S && Mi == 1) ? 1 : 0;
    a.Vn = Vn;
    a.act = s->act_on ? s->d_act : nullptr;
    a.t_n = s->t;
    a.dt = dt;
    a.threshold = s->opt.act_threshold;
    a.flags = s->d_flags;
    s->launch(EMRKC_PHASE_STAGE, [&] { s->mk.stage(a, s->ell, j >= 2, s->stream); });
    const double* zk0 = ks >= 0 ? a.Zm1 + (size_t)ks * s->ld : nullptr;
    for (int k = 2; k <= Mi; ++k) {
      MrkcArgs b = a;
      b.uV1 = s->d_U[(k - 2) % 3];
      b.um1 = s->d_Um[(k - 2) % 3];
      b.uV2 = (k == 2) ? s->d_V[bm1] : s->d_U[(k - 3) % 3];
      b.um2 = (k == 2) ? zk0 : s->d_Um[(k - 3) % 3];
      b.uVk = s->d_U[(k - 1) % 3];
      b.umk = s->d_Um[(k - 1) % 3];
      b.inu = ci.nu[k];
      b.ikappa = ci.kappa[k];
      b.imu_eta = ci.mu[k] * eta;
      b.last = (k == Mi) ? 1 : 0;
      b.final_stage = (j == S && k == Mi) ? 1 : 0;
      s->launch(EMRKC_PHASE_INNER, [&] { s->mk.inner(b, s->ell, s->stream); });
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return s->cuda_fail(e, "kernel launch");
  s->cur = (b0 + S) % 3;
  s->t += dt;
  s->steps += 1;
  s->last_s = S;
  s->last_m = Mi;
  s->last_eta = eta;
  s->last_rhoF = rhoF;
  s->last_rhoS = rhoS;
  return EMRKC_OK;
}

// One emRKC step as one launch of the device-resident step kernel: the
// rho policy's decision (due / fixed) is the host's, the estimates, stage
// counts and coefficients are the kernel's; y_{n+1} lands in (cur + 1) mod 3.
int do_step_fused(emrkc_solver* s, double dt) {
  FusedStepArgs a;
  a.n = s->n;
  a.ld = s->ld;
  a.b0 = s->cur;
  for (int b = 0; b < 3; ++b) {
    a.V[b] = s->d_V[b];
    a.Z[b] = s->d_Z[b];
    a.Vhi[b] = s->d_V32[b];
    a.Vlo[b] = s->d_Vlo[b];
    a.U[b] = s->d_U[b];
    a.D[b] = s->d_D[b];
  }
  a.F = s->d_F;
  a.LV = s->d_LV;
  a.Vn = s->d_Vn;
  a.Vn32 = s->d_Vn32;
  a.mask = s->d_mask;
  a.amp = s->amp;
  a.t_on = s->t_on;
  a.t_off = s->t_off;
  a.Cm = s->Cm;
  a.t_n = s->t;
  a.dt = dt;
  a.threshold = s->opt.act_threshold;
  a.act = s->act_on ? s->d_act : nullptr;
  a.flags = s->d_flags;
  a.eps = s->opt.eps;
  a.ell_wmax = s->ell_wmax;
  a.safety = s->opt.safety;
  a.rho_S_min = s->opt.rho_S_min;
  if (s->opt.rho_every == EMRKC_RHO_FIXED) {
    a.fixed = 1;
    a.rho_F_fixed = s->opt.rho_F;
    a.rho_S_fixed = s->opt.rho_S;
  } else {
    a.due = (s->opt.rho_every == EMRKC_RHO_ONCE) ? !s->rho_done : (s->steps % s->opt.rho_every == 0);
  }
  PowerFusedArgs& p = a.pw;
  p.n = s->n;
  p.ld = s->ld;
  p.V = s->d_V[s->cur];
  p.Vhi = s->d_V32[s->cur];
  p.Vlo = s->d_Vlo[s->cur];
  p.Z = s->d_Z[s->cur];
  p.vF[0] = s->d_vF;
  p.vF[1] = s->d_vF2;
  p.vS[0] = s->d_vS;
  p.vS[1] = s->d_vS2;
  p.fy = s->d_fy;
  p.mask = s->d_mask;
  p.Cm = s->Cm;
  p.f_inv_Cm = (float)(1.0 / s->Cm);
  p.ell_wmax = s->ell_wmax;
  p.eps = s->opt.pow_eps;
  p.tol = s->opt.pow_tol;
  p.max_iter = s->opt.pow_max_iter;
  p.tol_cold = s->opt.pow_tol_cold;
  p.max_iter_cold = s->opt.pow_max_iter_cold;
  p.part = s->d_ppart;
  p.flags = s->d_flags;
  a.state = s->d_fstate;
  a.ctab = s->d_ctab;
  a.beta = 2.0 - 4.0 * s->opt.eps / 3.0;
  a.two_dt = 2.0 * dt;
  a.inv_two_dt = 1.0 / (2.0 * dt);
  a.inv_Cm = 1.0 / s->Cm;
  cudaError_t e = cudaSuccess;
  s->launch(EMRKC_PHASE_STAGE, [&] { e = s->ks.step_fused(a, s->ell, s->fcluster, s->stream); });
  if (e != cudaSuccess) return s->cuda_fail(e, "device-resident step launch");
  if (a.due) s->rho_done = true;
  s->cur = (s->cur + 1) % 3;
  s->t += dt;
  s->steps += 1;
  s->fstate_stale = true;
  return EMRKC_OK;
}

int do_step(emrkc_solver* s, double dt) {
  if (s->method == EMRKC_METHOD_EXEX_RL || s->method == EMRKC_METHOD_IMEX_RL) return do_step_rl(s, dt);
  if (s->method == EMRKC_METHOD_MRKC) return do_step_mrkc(s, dt);
  if (s->fcluster > 0) {
    // fixed radii whose stage counts exceed the device-resident step's
    // limit take the host-driven step (estimated radii cannot be checked
    // before the launch: the kernel then flags the step, bit 4)
    bool fits = true;
    if (s->opt.rho_every == EMRKC_RHO_FIXED) {
      double l_s = 0.0;
      const int S = stages_for(dt, s->opt.rho_S, s->opt.eps, &l_s);
      const int Mi = stages_for(2.0 * dt / l_s, s->opt.rho_F, s->opt.eps, nullptr);
      fits = S <= kFusedMaxStages && Mi <= kFusedMaxStages;
    }
    if (fits) return do_step_fused(s, dt);
    const int rc = fused_pull(s);
    if (rc) return rc;
  }
  double rhoF, rhoS;
  int rc = step_rho(s, &rhoF, &rhoS);
  if (rc) return rc;
  // Algorithm 1 in the device-resident step's own expressions (stage counts
  // by comparison, eta and its reciprocals by multiplication), so that both
  // step forms take the same coefficients to the last bit
  const double beta = 2.0 - 4.0 * s->opt.eps / 3.0;
  const int S = rkc_stages_mul(dt * rhoS, beta);
  const double eta = (2.0 * dt) * (1.0 / (beta * (double)S * (double)S));
  const int Mi = rkc_stages_mul(eta * rhoF, beta);
  // a radius that is not finite (or beyond any useful stage count) gives
  // 1 << 24 stages: refuse the step instead of launching them
  if (S >= (1 << 24) || Mi >= (1 << 24))
    return s->fail(EMRKC_ERR_STATE, "spectral radius estimate not finite or too large for a step");
  const double inv_eta = beta * (double)S * (double)S * (1.0 / (2.0 * dt));
  const Coeffs co = s->coeffs(S);
  const Coeffs ci = s->coeffs(Mi);
  const float f_inv_mu1eta = (float)(inv_eta * (1.0 / ci.mu[1]));
  const int b0 = s->cur;
  // V_n for the activation test: buffer b0 survives the step while S <= 2
  // (stage j writes buffer b0 + j); a copy is kept for S >= 3
  const double* Vn = (S <= 2) ? s->d_V[b0] : s->d_Vn;
  for (int j = 1; j <= S; ++j) {
    const int bm1 = (b0 + j - 1) % 3, bm2 = (b0 + j - 2 + 3) % 3, bo = (b0 + j) % 3;
    StageArgs a;
    a.n = s->n;
    a.ld = s->ld;
    a.Vm1 = s->d_V[bm1];
    a.Zm1 = s->d_Z[bm1];
    a.Vm2 = j >= 2 ? s->d_V[bm2] : nullptr;
    a.Zm2 = j >= 2 ? s->d_Z[bm2] : nullptr;
    a.Vout = s->d_V[bo];
    a.Zout = s->d_Z[bo];
    a.nu = j >= 2 ? co.nu[j] : 1.0;
    a.kappa = j >= 2 ? co.kappa[j] : 0.0;
    a.mu_dt = co.mu[j] * dt;
    a.eta = eta;
    a.cm_inner = ci.c[Mi];
    a.mu1_eta = ci.mu[1] * eta;
    a.m = Mi;
    a.U1 = s->d_U[0];
    a.F = s->d_F;
    a.mask = s->d_mask;
    a.stim = stim_at(s, s->t + co.c[j - 1] * dt);
    a.Cm = s->Cm;
    a.inv_Cm = 1.0 / s->Cm;
    a.final_stage = (j == S && Mi == 1) ? 1 : 0;
    a.Vn = Vn;
    a.act = s->act_on ? s->d_act : nullptr;
    a.t_n = s->t;
    a.dt = dt;
    a.threshold = s->opt.act_threshold;
    a.flags = s->d_flags;
    a.Vn_copy = (j == 1 && S >= 3) ? s->d_Vn : nullptr;
    a.inv_eta = inv_eta;
    a.mu1 = ci.mu[1];
    a.V32m1 = s->d_V32[bm1];
    a.V32out = s->d_V32[bo];
    a.Vlo_m1 = s->d_Vlo[bm1];
    a.Vhi_m2 = j >= 2 ? s->d_V32[bm2] : nullptr;
    a.Vlo_m2 = j >= 2 ? s->d_Vlo[bm2] : nullptr;
    a.Vlo_out = s->d_Vlo[bo];
    a.Vn32 = (S <= 2) ? s->d_V32[b0] : s->d_Vn32;
    a.Vn32_copy = (j == 1 && S >= 3) ? s->d_Vn32 : nullptr;
    a.f_th = (float)s->opt.act_threshold;
    a.D1 = s->d_D[0];
    a.LV = (Mi >= 4) ? s->d_LV : nullptr;  // L V + F, kept for inner stages k >= 4
    a.f_nu = (float)a.nu;
    a.f_kappa = (float)a.kappa;
    a.f_mudt = (float)a.mu_dt;
    a.f_inv_eta = (float)inv_eta;
    a.f_cm = (float)a.cm_inner;
    a.f_mu1 = (float)ci.mu[1];
    a.f_mu1eta = (float)(ci.mu[1] * eta);
    a.f_eta = (float)eta;
    a.f_stim = (float)a.stim;
    a.f_inv_Cm = (float)(1.0 / s->Cm);
    a.tma_grid = s->tma_grid;
    a.tma_nbuf = s->tma_nbuf;
    a.tma_ell = s->tma_ell;
    a.pdl = s->pdl;
    a.ell_wmax = s->ell_wmax;
    s->launch(EMRKC_PHASE_STAGE, [&] { s->ks.stage(a, s->ell, j >= 2, s->stream); });
    for (int k = 2; k <= Mi; ++k) {
      InnerArgs b;
      b.n = s->n;
      b.u1 = (k - 1 == 0) ? s->d_V[bm1] : s->d_U[(k - 2) % 3];
      b.u2 = (k - 2 == 0) ? s->d_V[bm1] : s->d_U[(k - 3) % 3];
      b.uk = s->d_U[(k - 1) % 3];
      b.F = s->d_F;
      b.nu = ci.nu[k];
      b.kappa = ci.kappa[k];
      b.mu_eta = ci.mu[k] * eta;
      b.last = (k == Mi) ? 1 : 0;
      b.Vm1 = s->d_V[bm1];
      b.Vm2 = j >= 2 ? s->d_V[bm2] : nullptr;
      b.Vout = s->d_V[bo];
      b.onu = a.nu;
      b.okappa = a.kappa;
      b.omu_dt = a.mu_dt;
      b.eta = eta;
      b.final_stage = (j == S && k == Mi) ? 1 : 0;
      b.Vn = Vn;
      b.act = a.act;
      b.t_n = s->t;
      b.dt = dt;
      b.threshold = s->opt.act_threshold;
      b.flags = s->d_flags;
      b.inv_eta = inv_eta;
      b.d1 = s->d_D[(k - 2) % 3];
      b.d2 = (k - 2 == 0) ? nullptr : s->d_D[(k - 3) % 3];
      b.dk = s->d_D[(k - 1) % 3];
      b.LV = s->d_LV;
      b.lf_src = (Mi >= 4) ? 0 : (k == 2 ? 1 : 2);
      b.f_inv_mu1eta = f_inv_mu1eta;
      b.V32out = s->d_V32[bo];
      b.Vhi1 = s->d_V32[bm1];
      b.Vlo1 = s->d_Vlo[bm1];
      b.Vhi2 = j >= 2 ? s->d_V32[bm2] : nullptr;
      b.Vlo2 = j >= 2 ? s->d_Vlo[bm2] : nullptr;
      b.Vlo_out = s->d_Vlo[bo];
      b.Vn32 = a.Vn32;
      b.f_okappa = (float)a.kappa;
      b.f_omu_dt = (float)a.mu_dt;
      b.f_th = a.f_th;
      b.f_nu = (float)ci.nu[k];
      b.f_kappa = (float)ci.kappa[k];
      b.f_mueta = (float)(ci.mu[k] * eta);
      b.f_inv_eta = (float)inv_eta;
      b.ell_wmax = s->ell_wmax;
      b.pdl = s->pdl;
      s->launch(EMRKC_PHASE_INNER, [&] { s->ks.inner(b, s->ell, s->stream); });
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return s->cuda_fail(e, "kernel launch");
  s->cur = (b0 + S) % 3;
  s->t += dt;
  s->steps += 1;
  s->last_s = S;
  s->last_m = Mi;
  s->last_eta = eta;
  s->last_rhoF = rhoF;
  s->last_rhoS = rhoS;
  return EMRKC_OK;
}

int sync_and_check(emrkc_solver* s) {
  cudaError_t e = cudaMemcpyAsync(s->h_pin + kFlagsSlot, s->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "copy of flags");
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "stream synchronisation");
  return check_flags(s);
}

// Build the device matrices from the CSR input.
int build_matrix(emrkc_solver* s, const emrkc_matrix* m) {
  const int64_t n = m->n;
  const bool mixed = s->precision == EMRKC_PREC_MIXED;
  // L = -(chi Cm M)^-1 K row by row; entries at or below 1e-14 |K_ii| off the
  // diagonal are dropped, the diagonal is dropped in the mixed path (its
  // rows sum to zero).  Two passes over the CSR rows (count, then fill the
  // sliced ELL in CSR order), parallel over rows and slices.
  auto keep = [&](int64_t i, int64_t p, double drop) {
    const int32_t c = m->col[p];
    if (c != i && std::fabs(m->K[p]) <= drop) return false;
    if (mixed && c == i) return false;
    return true;
  };
  auto drop_of = [&](int64_t i) {
    double kii = 0.0;
    for (int64_t p = m->row_ptr[i]; p < m->row_ptr[i + 1]; ++p)
      if (m->col[p] == i) kii += m->K[p];
    return 1e-14 * std::fabs(kii);
  };
  std::vector<int32_t> cnt(n, 0);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double drop = drop_of(i);
    int c = 0;
    for (int64_t p = m->row_ptr[i]; p < m->row_ptr[i + 1]; ++p) c += keep(i, p, drop) ? 1 : 0;
    cnt[i] = c;
  }
  const int64_t ns = (n + 31) / 32;
  std::vector<int64_t> sptr(ns + 1, 0);
  std::vector<int32_t> width(ns, 0);
  for (int64_t b = 0; b < ns; ++b) {
    int w = 0;
    for (int64_t i = b * 32; i < std::min<int64_t>(n, b * 32 + 32); ++i) w = std::max<int>(w, cnt[i]);
    width[b] = w;
    sptr[b + 1] = sptr[b] + (int64_t)w * 32;
  }
  const int64_t total = sptr[ns];
  s->mat_slots = total;
  s->ell_wmax = 0;
  for (int64_t b = 0; b < ns; ++b) s->ell_wmax = std::max<int>(s->ell_wmax, width[b]);
  s->mat_entries = 0;
  for (int64_t i = 0; i < n; ++i) s->mat_entries += cnt[i];
  std::vector<int32_t> col(std::max<int64_t>(total, 1), 0);
  std::vector<double> val(mixed ? 0 : std::max<int64_t>(total, 1), 0.0);
  std::vector<float> val32(mixed ? std::max<int64_t>(total, 1) : 0, 0.0f);
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < ns; ++b) {
    for (int l = 0; l < 32; ++l) {
      const int64_t i = b * 32 + l;
      const int32_t pad_col = (int32_t)std::min<int64_t>(i, n - 1);
      int k = 0;
      if (i < n) {
        const double drop = drop_of(i);
        const double scale = -1.0 / (s->chi * s->Cm * m->lumped_mass[i]);
        for (int64_t q = m->row_ptr[i]; q < m->row_ptr[i + 1]; ++q) {
          if (!keep(i, q, drop)) continue;
          const int64_t p = sptr[b] + (int64_t)k * 32 + l;
          col[p] = m->col[q];
          if (mixed) val32[p] = (float)(m->K[q] * scale);
          else val[p] = m->K[q] * scale;
          ++k;
        }
      }
      for (; k < width[b]; ++k) col[sptr[b] + (int64_t)k * 32 + l] = pad_col;
    }
  }
  cudaError_t e;
  if ((e = dalloc(&s->d_slice_ptr, ns + 1)) != cudaSuccess) return s->fail(EMRKC_ERR_OOM, "device allocation (matrix)");
  if ((e = dalloc(&s->d_width, ns)) != cudaSuccess) return s->fail(EMRKC_ERR_OOM, "device allocation (matrix)");
  if ((e = dalloc(&s->d_col, col.size())) != cudaSuccess) return s->fail(EMRKC_ERR_OOM, "device allocation (matrix)");
  cudaMemcpy(s->d_slice_ptr, sptr.data(), sptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (ns) cudaMemcpy(s->d_width, width.data(), width.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  cudaMemcpy(s->d_col, col.data(), col.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (mixed) {
    if ((e = dalloc(&s->d_val32, val32.size())) != cudaSuccess) return s->fail(EMRKC_ERR_OOM, "device allocation (matrix)");
    cudaMemcpy(s->d_val32, val32.data(), val32.size() * sizeof(float), cudaMemcpyHostToDevice);
  } else {
    if ((e = dalloc(&s->d_val, val.size())) != cudaSuccess) return s->fail(EMRKC_ERR_OOM, "device allocation (matrix)");
    cudaMemcpy(s->d_val, val.data(), val.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return s->cuda_fail(e, "matrix upload");
  s->ell.n = n;
  s->ell.n_slices = ns;
  s->ell.slice_ptr = s->d_slice_ptr;
  s->ell.width = s->d_width;
  s->ell.col = s->d_col;
  s->ell.val = s->d_val;
  s->ell.val32 = s->d_val32;
  return EMRKC_OK;
}

int validate_matrix(const emrkc_matrix* m, std::string* why) {
  if (!m || m->n <= 0 || m->nnz < 0 || !m->row_ptr || (m->nnz > 0 && (!m->col || !m->K)) || !m->lumped_mass) {
    *why = "matrix: null pointer or non-positive size";
    return EMRKC_ERR_ARG;
  }
  if (m->n > (int64_t)INT32_MAX - 64) {
    *why = "matrix: more than 2^31 - 64 rows";
    return EMRKC_ERR_ARG;
  }
  if (m->row_ptr[0] != 0 || m->row_ptr[m->n] != m->nnz) {
    *why = "matrix: row_ptr[0] must be 0 and row_ptr[n] must equal nnz";
    return EMRKC_ERR_ARG;
  }
  for (int64_t i = 0; i < m->n; ++i) {
    if (m->row_ptr[i + 1] < m->row_ptr[i]) {
      *why = "matrix: row_ptr is not monotone";
      return EMRKC_ERR_ARG;
    }
    if (!(m->lumped_mass[i] > 0.0) || !std::isfinite(m->lumped_mass[i])) {
      *why = "matrix: lumped mass must be positive and finite";
      return EMRKC_ERR_ARG;
    }
  }
  int64_t bad_col = 0, bad_val = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad_col, bad_val)
  for (int64_t p = 0; p < m->nnz; ++p) {
    bad_col += (m->col[p] < 0 || m->col[p] >= m->n) ? 1 : 0;
    bad_val += std::isfinite(m->K[p]) ? 0 : 1;
  }
  if (bad_col) {
    *why = "matrix: column index out of range";
    return EMRKC_ERR_ARG;
  }
  if (bad_val) {
    *why = "matrix: non-finite entry";
    return EMRKC_ERR_ARG;
  }
  return EMRKC_OK;
}

int state_copy(emrkc_solver* s, int var, double* buf, int64_t len, bool to_host, bool dev_ptr) {
  if (!s) return EMRKC_ERR_ARG;
  cudaSetDevice(s->device);
  if (!buf) return s->fail(EMRKC_ERR_ARG, "null buffer");
  if (var < -1 || var >= s->N) return s->fail(EMRKC_ERR_ARG, "variable index out of range");
  const int64_t need = (var == -1) ? (int64_t)s->N * s->n : s->n;
  if (len != need) return s->fail(EMRKC_ERR_STATE, "buffer length does not match the state size");
  const cudaMemcpyKind kind = dev_ptr ? cudaMemcpyDeviceToDevice
                                      : (to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
  const size_t row = (size_t)s->n * sizeof(double), pitch_b = (size_t)s->n * sizeof(double);
  cudaError_t e = cudaSuccess;
  // V (mixed path: materialise hi + lo as double first)
  if (var <= 0 && to_host) materialise_V(s);
  if (var <= 0) {
    e = to_host ? cudaMemcpyAsync(buf, s->d_V[s->cur], row, kind, s->stream)
                : cudaMemcpyAsync(s->d_V[s->cur], buf, row, kind, s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "state copy");
  }
  // z rows first..last (z index = var - 1), as one pitched copy
  const int zfirst = (var == -1) ? 0 : var - 1;
  const int zrows = (var == -1) ? s->N - 1 : (var >= 1 ? 1 : 0);
  if (zrows > 0) {
    double* hb = buf + ((var == -1) ? s->n : 0);
    const size_t dpitch = (size_t)s->ld * sizeof(double);
    if (s->zsize == 8) {
      double* zr = (double*)s->zrow(s->cur, zfirst);
      e = to_host ? cudaMemcpy2DAsync(hb, pitch_b, zr, dpitch, row, zrows, kind, s->stream)
                  : cudaMemcpy2DAsync(zr, dpitch, hb, pitch_b, row, zrows, kind, s->stream);
    } else {
      void* zr = s->zrow(s->cur, zfirst);
      const int64_t count = (int64_t)zrows * s->ld;
      if (to_host) {
        s->ks.convert_z(count, zr, s->d_tmp, 1, s->stream);
        e = cudaMemcpy2DAsync(hb, pitch_b, s->d_tmp, dpitch, row, zrows, kind, s->stream);
      } else {
        e = cudaMemcpy2DAsync(s->d_tmp, dpitch, hb, pitch_b, row, zrows, kind, s->stream);
        if (e == cudaSuccess) s->ks.convert_z(count, zr, s->d_tmp, 0, s->stream);
      }
    }
    if (e != cudaSuccess) return s->cuda_fail(e, "state copy");
  }
  if (!to_host && var <= 0 && s->d_V32[s->cur])
    launch_ff_split(s->d_V[s->cur], s->d_V32[s->cur], s->d_Vlo[s->cur], s->n, s->stream);
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "state copy");
  return EMRKC_OK;
}

}  // namespace

namespace emrkc {
int solver_update_rho(emrkc_solver* s) {
  int rc = update_rho_now(s);
  if (!rc) s->rho_done = true;
  return rc;
}
void solver_materialise_V(emrkc_solver* s) { materialise_V(s); }

}  // namespace emrkc

extern "C" {

int emrkc_default_options(emrkc_options* o) {
  if (!o) return EMRKC_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->precision = EMRKC_PREC_FP64;
  o->rho_every = 1;
  o->rho_F = 0.0;
  o->rho_S = 0.0;
  o->eps = 0.05;
  o->safety = 1.05;
  o->pow_tol = 1e-2;
  o->pow_eps = 1e-8;
  o->pow_max_iter = 50;
  o->seed = 0;
  o->act_threshold = -20.0;
  o->cuda_stream = nullptr;
  o->device = 0;
  o->profile = 0;
  o->use_graphs = 1;
  o->rho_S_min = 0.0;
  o->method = EMRKC_METHOD_EMRKC;
  o->lin_rtol = 1e-10;
  o->lin_max_iter = 1000;
  o->pow_tol_cold = 1e-4;
  o->pow_max_iter_cold = 1000;
  return EMRKC_OK;
}

int emrkc_num_vars(int model) {
  const auto r = rest_state(model);
  return r.empty() ? -1 : (int)r.size();
}

int emrkc_num_gates(int model) {
  switch (model) {
    case EMRKC_MODEL_NONE: return 0;
    case EMRKC_MODEL_PASSIVE: return 1;
    case EMRKC_MODEL_HH: return 3;
    case EMRKC_MODEL_TTP06_EPI: return 12;
    default: return -1;
  }
}

int emrkc_rkc_stages(double dt, double rho, double eps, int* s, double* l_s) {
  if (!s) return EMRKC_ERR_ARG;
  if (!(dt >= 0.0) || !(rho >= 0.0) || !(eps >= 0.0) || !std::isfinite(dt) || !std::isfinite(rho) ||
      !std::isfinite(eps) || !(eps < 1.5))
    return EMRKC_ERR_ARG;
  if (!(dt * rho < 1e15)) return EMRKC_ERR_ARG;
  *s = emrkc::stages_for(dt, rho, eps, l_s);
  return EMRKC_OK;
}

int emrkc_rkc_coeffs(int s, double eps, double* mu, double* nu, double* kappa, double* c) {
  if (s < 1 || s > (1 << 20) || !(eps >= 0.0) || !std::isfinite(eps) || !mu || !nu || !kappa || !c)
    return EMRKC_ERR_ARG;
  emrkc::rkc_coeffs(s, eps, mu, nu, kappa, c);
  return EMRKC_OK;
}

int emrkc_create(const emrkc_matrix* mat, const emrkc_tissue* tissue, int ionic_model, const emrkc_stimulus* stim,
                 const emrkc_options* opt, emrkc_solver** out) {
  if (!out) {
    g_create_error = "out is NULL";
    return EMRKC_ERR_ARG;
  }
  *out = nullptr;
  std::string why;
  int rc = validate_matrix(mat, &why);
  if (rc) {
    g_create_error = why;
    return rc;
  }
  if (!tissue || !(tissue->chi > 0) || !(tissue->Cm > 0)) {
    g_create_error = "tissue: chi and Cm must be positive";
    return EMRKC_ERR_ARG;
  }
  if (emrkc_num_vars(ionic_model) < 0) {
    g_create_error = "unknown ionic model";
    return EMRKC_ERR_ARG;
  }
  emrkc_options o;
  if (opt) o = *opt;
  else emrkc_default_options(&o);
  if (o.precision != EMRKC_PREC_FP64 && o.precision != EMRKC_PREC_MIXED) {
    g_create_error = "unknown precision mode";
    return EMRKC_ERR_ARG;
  }
  if (o.rho_every < EMRKC_RHO_FIXED || !(o.eps > 0) || !(o.safety > 0) || !(o.pow_tol > 0) || !(o.pow_eps > 0) ||
      o.pow_max_iter < 1 || !(o.pow_tol_cold > 0) || o.pow_max_iter_cold < 1) {
    g_create_error = "options: invalid rho policy or power-iteration parameters";
    return EMRKC_ERR_ARG;
  }
  if (!(o.rho_S_min >= 0) || !std::isfinite(o.rho_S_min)) {
    g_create_error = "options: rho_S_min must be finite and >= 0";
    return EMRKC_ERR_ARG;
  }
  if (o.method < EMRKC_METHOD_EMRKC || o.method > EMRKC_METHOD_MRKC) {
    g_create_error = "options: unknown method";
    return EMRKC_ERR_ARG;
  }
  if (o.method != EMRKC_METHOD_EMRKC && o.precision != EMRKC_PREC_FP64) {
    g_create_error = "options: mRKC, EXEX-RL and IMEX-RL run in FP64 only";
    return EMRKC_ERR_ARG;
  }
  if (o.method == EMRKC_METHOD_IMEX_RL && (!(o.lin_rtol >= 0) || o.lin_max_iter < 0)) {
    g_create_error = "options: lin_rtol must be >= 0 and lin_max_iter >= 0";
    return EMRKC_ERR_ARG;
  }
  if (o.rho_every == EMRKC_RHO_FIXED && (!(o.rho_F >= 0) || !(o.rho_S >= 0))) {
    g_create_error = "options: fixed rho values must be >= 0";
    return EMRKC_ERR_ARG;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev <= o.device || o.device < 0) {
    g_create_error = std::string("no usable CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "ordinal");
    return EMRKC_ERR_CUDA;
  }
  auto* s = new emrkc_solver();
  s->opt = o;
  s->device = o.device;
  cudaSetDevice(s->device);
  s->model = ionic_model;
  s->precision = o.precision;
  s->method = o.method;
  const bool ok = (s->precision == EMRKC_PREC_FP64) ? get_kernels_fp64(ionic_model, &s->ks)
                                                    : get_kernels_mixed(ionic_model, &s->ks);
  if (ok && o.method == EMRKC_METHOD_MRKC && !get_kernels_mrkc(ionic_model, &s->mk)) {
    g_create_error = "no mRKC kernels for this model";
    delete s;
    return EMRKC_ERR_ARG;
  }
  if (!ok) {
    g_create_error = "no kernels for this model";
    delete s;
    return EMRKC_ERR_ARG;
  }
  s->N = s->ks.N;
  s->nE = s->ks.nE;
  s->nS = s->ks.nS;
  s->zsize = s->precision == EMRKC_PREC_FP64 ? 8 : 4;
  s->rsize = s->zsize;
  s->n = mat->n;
  // ld: multiple of 128 so that every 128-node tile of every SoA row lies in
  // the allocation and starts on a 512-byte boundary (bulk-copy alignment)
  s->ld = (mat->n + 127) / 128 * 128;
  s->chi = tissue->chi;
  s->Cm = tissue->Cm;
  s->act_on = !std::isnan(o.act_threshold);
  auto bail = [&](int code, const std::string& msg) {
    g_create_error = msg.empty() ? s->err : msg;
    free_all(s);
    delete s;
    return code;
  };
  if (o.cuda_stream) {
    s->stream = (cudaStream_t)o.cuda_stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(EMRKC_ERR_CUDA, std::string("stream creation: ") + cudaGetErrorString(e));
    s->own_stream = true;
  }
  if ((rc = build_matrix(s, mat))) return bail(rc, "");
  if (s->precision == EMRKC_PREC_MIXED && s->ks.tma_grid) {
    const char* no_tma = std::getenv("EMRKC_NO_TMA");
    if (!(no_tma && no_tma[0] == '1')) {
      const char* nbuf = std::getenv("EMRKC_TMA_NBUF");
      const char* ell = std::getenv("EMRKC_TMA_ELL");
      // default 3: one state region and two ELL buffers, the next tile
      // prefetched during compute; 1 or 2: whole-tile stage buffers
      if (nbuf && (nbuf[0] == '1' || nbuf[0] == '2')) s->tma_nbuf = nbuf[0] - '0';
      if (ell && ell[0] == '0') s->tma_ell = 0;
      s->tma_grid = s->ks.tma_grid(s->device, s->ell_wmax, s->tma_nbuf, s->tma_ell);
    }
    const char* no_pdl = std::getenv("EMRKC_NO_PDL");
    s->pdl = (no_pdl && no_pdl[0] == '1') ? 0 : 1;
  }
  const int64_t ld = s->ld, nz = s->N - 1;
  bool fail = false;
  for (int b = 0; b < 3; ++b) {
    fail |= dalloc(&s->d_V[b], ld) != cudaSuccess;
    fail |= cudaMalloc(&s->d_Z[b], std::max<int64_t>(nz * ld, 1) * s->zsize) != cudaSuccess;
    fail |= dalloc(&s->d_U[b], ld) != cudaSuccess;
  }
  fail |= cudaMalloc(&s->d_F, ld * s->rsize) != cudaSuccess;
  if (s->precision == EMRKC_PREC_MIXED) {
    for (int b = 0; b < 3; ++b) {
      fail |= dalloc(&s->d_V32[b], ld) != cudaSuccess;
      fail |= dalloc(&s->d_Vlo[b], ld) != cudaSuccess;
      fail |= dalloc(&s->d_D[b], ld) != cudaSuccess;
    }
    fail |= dalloc(&s->d_LV, ld) != cudaSuccess;
    fail |= dalloc(&s->d_Vn32, ld) != cudaSuccess;
  }
  // the f_F iterate: V only, or (V, z_k) for mRKC
  const int64_t rowsF = (s->method == EMRKC_METHOD_MRKC) ? 2 : 1;
  fail |= dalloc(&s->d_vF, rowsF * ld) != cudaSuccess;
  fail |= dalloc(&s->d_vF2, rowsF * ld) != cudaSuccess;
  if (s->method == EMRKC_METHOD_MRKC)
    for (int b = 0; b < 3; ++b) fail |= dalloc(&s->d_Um[b], ld) != cudaSuccess;
  fail |= dalloc(&s->d_vS, (int64_t)s->N * ld) != cudaSuccess;
  fail |= dalloc(&s->d_vS2, (int64_t)s->N * ld) != cudaSuccess;
  fail |= dalloc(&s->d_fy, (int64_t)s->N * ld) != cudaSuccess;
  fail |= dalloc(&s->d_act, ld) != cudaSuccess;
  fail |= dalloc(&s->d_Vn, ld) != cudaSuccess;
  fail |= dalloc(&s->d_tmp, (int64_t)std::max(1, s->N - 1) * ld) != cudaSuccess;
  fail |= dalloc(&s->d_rest, 64) != cudaSuccess;
  if (s->method == EMRKC_METHOD_EMRKC) {
    s->pfused_grid = s->ks.power_fused_grid(s->device);
    s->pcluster = s->ks.power_cluster_size ? s->ks.power_cluster_size(s->device) : 0;
    const char* no_cluster = std::getenv("EMRKC_NO_CLUSTER");
    if (no_cluster && no_cluster[0] == '1') s->pcluster = 0;
    // device-resident steps for problems one cluster holds (at most 4 nodes
    // per thread), by default for mixed precision with rho estimated every
    // step: there the step saves the host round trip of every power
    // iteration.  With rho known after the first step the host-driven step
    // is faster (its stage kernels, chained by programmatic dependent launch,
    // take about 3 us each against about 5 us for a stage inside the
    // cluster), and FP64 is bound by the FP64 pipe, which the separate
    // launches spread over more SMs than one cluster has.
    // EMRKC_FUSED_STEP=0 / 1 turns the device-resident step off / on.
    const char* fused_env = std::getenv("EMRKC_FUSED_STEP");
    const bool want = fused_env && (fused_env[0] == '0' || fused_env[0] == '1')
                          ? fused_env[0] == '1'
                          : (s->precision == EMRKC_PREC_MIXED && o.rho_every == 1);
    if (want && s->pcluster > 0 && s->pfused_grid >= 16 && s->ks.step_fused_cluster_size) {
      const int cl = s->ks.step_fused_cluster_size(s->device);
      if (cl > 0 && s->n <= (int64_t)4 * cl * s->ks.step_fused_block()) s->fcluster = cl;
    }
    if (s->pfused_grid > 0) {
      fail |= dalloc(&s->d_ppart, 8 * (int64_t)s->pfused_grid) != cudaSuccess;
      fail |= dalloc(&s->d_pbar, 2) != cudaSuccess;
    }
    if (s->fcluster > 0) {
      if (cudaMalloc(&s->d_fstate, sizeof(FusedStepState)) != cudaSuccess) {
        s->d_fstate = nullptr;
        fail = true;
      } else {
        fail |= cudaMemsetAsync(s->d_fstate, 0, sizeof(FusedStepState), s->stream) != cudaSuccess;
      }
      // Algorithm 1's coefficients for every stage count the fused step
      // can take, with 1 / (beta s^2) and 1 / mu_1 (rkc_coeffs.h layout)
      const int L = rkc_table_len(kFusedMaxStages);
      std::vector<double> tab(rkc_table_doubles(kFusedMaxStages), 0.0);
      const double beta = 2.0 - 4.0 * s->opt.eps / 3.0;
      for (int sc = 1; sc <= kFusedMaxStages; ++sc) {
        const int r = rkc_table_row(sc);
        rkc_coeffs(sc, s->opt.eps, &tab[r], &tab[L + r], &tab[2 * L + r], &tab[3 * L + r]);
        tab[4 * L + sc] = 1.0 / (beta * (double)sc * (double)sc);
        tab[4 * L + kFusedMaxStages + 1 + sc] = 1.0 / tab[r + 1];
      }
      if (cudaMalloc(&s->d_ctab, tab.size() * sizeof(double)) != cudaSuccess) {
        s->d_ctab = nullptr;
        fail = true;
      } else {
        fail |= cudaMemcpy(s->d_ctab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess;
      }
    }
  }
  fail |= dalloc(&s->rs.partials, kReduceMaxBlocks) != cudaSuccess;
  fail |= dalloc(&s->rs.ticket, 4) != cudaSuccess;
  // 16 result slots, then the flags words (kFlagsSlot): one copy reads both
  fail |= dalloc(&s->rs.result, kFlagsSlot + 2) != cudaSuccess;
  if (s->rs.result) s->d_flags = reinterpret_cast<int*>(s->rs.result + kFlagsSlot);
  if (s->method == EMRKC_METHOD_IMEX_RL) {
    s->pcg_grid = pcg_grid(s->device);
    fail |= s->pcg_grid <= 0;
    fail |= dalloc(&s->d_mass, ld) != cudaSuccess;
    for (int k = 0; k < 6; ++k) fail |= dalloc(&s->d_cg[k], ld) != cudaSuccess;
    fail |= dalloc(&s->d_part, 4 * (int64_t)(kReduceMaxBlocks + std::max(s->pcg_grid, 1))) != cudaSuccess;
    fail |= dalloc(&s->d_bar, 2) != cudaSuccess;
    fail |= dalloc(&s->d_iters, 2) != cudaSuccess;
    fail |= dalloc(&s->d_res, 2) != cudaSuccess;
  }
  if (fail) return bail(EMRKC_ERR_OOM, "device allocation failed");
  if (s->d_mass) {
    cudaMemsetAsync(s->d_mass, 0, ld * sizeof(double), s->stream);
    cudaMemcpyAsync(s->d_mass, mat->lumped_mass, s->n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    for (int k = 0; k < 6; ++k) cudaMemsetAsync(s->d_cg[k], 0, ld * sizeof(double), s->stream);
    cudaMemsetAsync(s->d_bar, 0, 2 * sizeof(unsigned int), s->stream);
    cudaMemsetAsync(s->d_iters, 0, 2 * sizeof(unsigned long long), s->stream);
    cudaMemsetAsync(s->d_res, 0, 2 * sizeof(double), s->stream);
  }
  if ((e = cudaMallocHost(&s->h_pin, 32 * sizeof(double))) != cudaSuccess) return bail(EMRKC_ERR_OOM, "pinned allocation failed");
  std::memset(s->h_pin, 0, 32 * sizeof(double));
  if (stim) {
    // amplitude and window are kept without a mask too: they apply to a mask
    // given later (emrkc_batch_set_stimulus_async)
    s->amp = stim->amplitude;
    s->t_on = stim->t_on;
    s->t_off = stim->t_off;
  }
  if (stim && stim->node_mask) {
    if ((e = dalloc(&s->d_mask, ld)) != cudaSuccess) return bail(EMRKC_ERR_OOM, "device allocation failed");
    cudaMemsetAsync(s->d_mask, 0, ld, s->stream);
    cudaMemcpyAsync(s->d_mask, stim->node_mask, s->n, cudaMemcpyHostToDevice, s->stream);
  }
  cudaMemsetAsync(s->d_flags, 0, 4 * sizeof(int), s->stream);
  cudaMemsetAsync(s->rs.ticket, 0, 4 * sizeof(unsigned int), s->stream);
  cudaMemsetAsync(s->rs.result, 0, 16 * sizeof(double), s->stream);
  for (int b = 0; b < 3; ++b) cudaMemsetAsync(s->d_U[b], 0, ld * sizeof(double), s->stream);
  // power-iteration iterates: the kernels write rows [0, n) only and the norms
  // run over whole rows, so the padding must hold zeros in both buffers
  cudaMemsetAsync(s->d_vF2, 0, rowsF * ld * sizeof(double), s->stream);
  cudaMemsetAsync(s->d_vS2, 0, (size_t)s->N * ld * sizeof(double), s->stream);
  cudaMemsetAsync(s->d_fy, 0, (size_t)s->N * ld * sizeof(double), s->stream);
  // rest state in every buffer
  const auto rest = rest_state(ionic_model);
  cudaMemcpy(s->d_rest, rest.data(), rest.size() * sizeof(double), cudaMemcpyHostToDevice);
  for (int b = 0; b < 3; ++b) {
    launch_fill(s->d_V[b], ld, rest[0], s->stream);
    if (s->d_V32[b]) launch_ff_split(s->d_V[b], s->d_V32[b], s->d_Vlo[b], ld, s->stream);
    if (nz > 0) launch_fill_rows(s->d_Z[b], (int)s->zsize, s->n, ld, (int)nz, s->d_rest + 1, s->stream);
  }
  launch_fill(s->d_act, ld, std::nan(""), s->stream);
  launch_start_vector(o.seed, s->n, ld, (int)rowsF, s->d_vF, s->stream);
  launch_start_vector(~o.seed, s->n, ld, s->N, s->d_vS, s->stream);
  if (s->precision == EMRKC_PREC_MIXED && s->method == EMRKC_METHOD_EMRKC && s->pfused_grid > 0) {
    // the fused power iteration of the mixed path keeps its iterates in FP32:
    // the start vectors rounded into the spare buffers, which become current
    s->ks.convert_z(rowsF * ld, s->d_vF2, s->d_vF, 0, s->stream);
    s->ks.convert_z((int64_t)s->N * ld, s->d_vS2, s->d_vS, 0, s->stream);
    std::swap(s->d_vF, s->d_vF2);
    std::swap(s->d_vS, s->d_vS2);
  }
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
    return bail(EMRKC_ERR_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
  if ((e = cudaGetLastError()) != cudaSuccess)
    return bail(EMRKC_ERR_CUDA, std::string("initialisation: ") + cudaGetErrorString(e));
  *out = s;
  return EMRKC_OK;
}

int emrkc_step(emrkc_solver* s, double dt) {
  if (!s) return EMRKC_ERR_ARG;
  if (!(dt > 0) || !std::isfinite(dt)) return s->fail(EMRKC_ERR_ARG, "dt must be positive and finite");
  cudaSetDevice(s->device);
  return do_step(s, dt);
}

int emrkc_run(emrkc_solver* s, double T, double dt) {
  if (!s) return EMRKC_ERR_ARG;
  if (!(dt > 0) || !(T >= 0) || !std::isfinite(T) || !std::isfinite(dt))
    return s->fail(EMRKC_ERR_ARG, "T and dt must be finite, dt > 0, T >= 0");
  const double r = T / dt;
  const int64_t steps = (int64_t)std::llround(r);
  if (std::fabs((double)steps * dt - T) > 1e-9 * std::max(1.0, std::fabs(T)))
    return s->fail(EMRKC_ERR_ARG, "T is not an integer multiple of dt");
  cudaSetDevice(s->device);
  for (int64_t k = 0; k < steps; ++k) {
    int rc = do_step(s, dt);
    if (rc) return rc;
  }
  return sync_and_check(s);
}

int emrkc_sync(emrkc_solver* s) {
  if (!s) return EMRKC_ERR_ARG;
  cudaSetDevice(s->device);
  for (cudaStream_t cs : {s->copy_stream, s->h2d_stream}) {
    if (!cs) continue;
    const cudaError_t e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return s->cuda_fail(e, "copy stream synchronisation");
  }
  int rc = sync_and_check(s);
  s->harvest();
  return rc;
}

int emrkc_get_state(emrkc_solver* s, int var, double* host_out, int64_t len) {
  return state_copy(s, var, host_out, len, true, false);
}

int emrkc_set_state(emrkc_solver* s, int var, const double* host_in, int64_t len) {
  return state_copy(s, var, const_cast<double*>(host_in), len, false, false);
}

int emrkc_get_state_device(emrkc_solver* s, int var, double* dev_out, int64_t len) {
  return state_copy(s, var, dev_out, len, true, true);
}

int emrkc_set_state_device(emrkc_solver* s, int var, const double* dev_in, int64_t len) {
  return state_copy(s, var, const_cast<double*>(dev_in), len, false, true);
}

int emrkc_get_activation_times(emrkc_solver* s, double* host_out, int64_t n) {
  if (!s) return EMRKC_ERR_ARG;
  if (!host_out) return s->fail(EMRKC_ERR_ARG, "null buffer");
  if (n != s->n) return s->fail(EMRKC_ERR_STATE, "length must equal the number of nodes");
  cudaSetDevice(s->device);
  cudaError_t e = cudaMemcpyAsync(host_out, s->d_act, s->n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return s->cuda_fail(e, "activation copy");
  return EMRKC_OK;
}

int emrkc_estimate_rho(emrkc_solver* s, double* rho_F, double* rho_S, int* it_F, int* it_S) {
  if (!s) return EMRKC_ERR_ARG;
  cudaSetDevice(s->device);
  s->itF = s->itS = 0;
  int rc = update_rho_now(s);
  if (rc) return rc;
  if (rho_F) *rho_F = s->rhoF_raw;
  if (rho_S) *rho_S = s->rhoS_raw;
  if (it_F) *it_F = s->itF;
  if (it_S) *it_S = s->itS;
  return EMRKC_OK;
}

int emrkc_set_stimulus(emrkc_solver* s, const uint8_t* node_mask, int64_t n, double amplitude, double t_on,
                       double t_off) {
  if (!s) return EMRKC_ERR_ARG;
  if (n != s->n) return s->fail(EMRKC_ERR_ARG, "mask length does not match the node count");
  if (!std::isfinite(amplitude) || std::isnan(t_on) || std::isnan(t_off))
    return s->fail(EMRKC_ERR_ARG, "stimulus amplitude and window must be numbers");
  cudaSetDevice(s->device);
  if (!node_mask) {
    // no stimulus: an empty window keeps the kernels' mask reads harmless
    s->amp = 0.0;
    s->t_on = 0.0;
    s->t_off = -1.0;
    return EMRKC_OK;
  }
  cudaError_t e;
  if (!s->d_mask) {
    if ((e = dalloc(&s->d_mask, s->ld)) != cudaSuccess) return s->fail(EMRKC_ERR_OOM, "device allocation failed");
    if ((e = cudaMemsetAsync(s->d_mask, 0, s->ld, s->stream)) != cudaSuccess) return s->cuda_fail(e, "mask clear");
  }
  // synchronous with respect to the caller's buffer: it may be reused at once
  if ((e = cudaMemcpyAsync(s->d_mask, node_mask, s->n, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
    return s->cuda_fail(e, "mask copy");
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return s->cuda_fail(e, "mask copy");
  s->amp = amplitude;
  s->t_on = t_on;
  s->t_off = t_off;
  return EMRKC_OK;
}

namespace {
// Two copy streams, one per direction, so that a mask upload never queues
// behind a state download (each direction has its own copy engine).
int ensure_copy_stream(emrkc_solver* s) {
  if (s->copy_stream) return EMRKC_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&s->h2d_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    s->h2d_stream = nullptr;
    return s->cuda_fail(e, "copy stream creation");
  }
  e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    s->copy_stream = nullptr;
    return s->cuda_fail(e, "copy stream creation");
  }
  cudaEvent_t* evs[] = {&s->ev_mask_free[0], &s->ev_mask_free[1], &s->ev_mask_ready, &s->ev_stage_ready[0],
                        &s->ev_stage_ready[1], &s->ev_stage_free[0], &s->ev_stage_free[1]};
  for (cudaEvent_t* ev : evs) {
    if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
      return s->cuda_fail(e, "event creation");
  }
  return EMRKC_OK;
}
}  // namespace

int emrkc_set_stimulus_async(emrkc_solver* s, const uint8_t* node_mask, int64_t n, double amplitude, double t_on,
                             double t_off) {
  if (!s) return EMRKC_ERR_ARG;
  if (n != s->n) return s->fail(EMRKC_ERR_ARG, "mask length does not match the node count");
  if (!std::isfinite(amplitude) || std::isnan(t_on) || std::isnan(t_off))
    return s->fail(EMRKC_ERR_ARG, "stimulus amplitude and window must be numbers");
  cudaSetDevice(s->device);
  if (!node_mask) return emrkc_set_stimulus(s, nullptr, n, amplitude, t_on, t_off);
  int rc = ensure_copy_stream(s);
  if (rc) return rc;
  cudaError_t e;
  if (!s->d_mask || !s->d_mask_alt) {
    // first use: both buffers zeroed (the padding of the last tile is read)
    for (uint8_t** m : {&s->d_mask, &s->d_mask_alt}) {
      if (*m) continue;
      if ((e = dalloc(m, s->ld)) != cudaSuccess) return s->fail(EMRKC_ERR_OOM, "device allocation failed");
      if ((e = cudaMemsetAsync(*m, 0, s->ld, s->stream)) != cudaSuccess) return s->cuda_fail(e, "mask clear");
    }
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return s->cuda_fail(e, "mask clear");
  }
  const int ti = s->mask_idx ^ 1;
  uint8_t* tgt = s->d_mask_alt;
  // the copy waits until no enqueued step reads the target buffer any more
  if (s->mask_free_rec[ti] && (e = cudaStreamWaitEvent(s->h2d_stream, s->ev_mask_free[ti], 0)) != cudaSuccess)
    return s->cuda_fail(e, "mask copy ordering");
  if ((e = cudaMemcpyAsync(tgt, node_mask, s->n, cudaMemcpyHostToDevice, s->h2d_stream)) != cudaSuccess)
    return s->cuda_fail(e, "mask copy");
  if ((e = cudaEventRecord(s->ev_mask_ready, s->h2d_stream)) != cudaSuccess) return s->cuda_fail(e, "mask copy");
  // steps enqueued from now on read the new buffer, after its copy
  if ((e = cudaStreamWaitEvent(s->stream, s->ev_mask_ready, 0)) != cudaSuccess)
    return s->cuda_fail(e, "mask copy ordering");
  if ((e = cudaEventRecord(s->ev_mask_free[s->mask_idx], s->stream)) != cudaSuccess)
    return s->cuda_fail(e, "mask copy ordering");
  s->mask_free_rec[s->mask_idx] = true;
  s->d_mask_alt = s->d_mask;
  s->d_mask = tgt;
  s->mask_idx = ti;
  s->amp = amplitude;
  s->t_on = t_on;
  s->t_off = t_off;
  return EMRKC_OK;
}

int emrkc_get_state_async(emrkc_solver* s, int var, double* host_out, int64_t len) {
  if (!s) return EMRKC_ERR_ARG;
  if (!host_out) return s->fail(EMRKC_ERR_ARG, "null buffer");
  if (var < 0 || var >= s->N) return s->fail(EMRKC_ERR_ARG, "variable index out of range (one variable)");
  if (len != s->n) return s->fail(EMRKC_ERR_STATE, "buffer length must equal the number of nodes");
  cudaSetDevice(s->device);
  int rc = ensure_copy_stream(s);
  if (rc) return rc;
  cudaError_t e;
  const int k = s->stage_k;
  if (!s->d_stage[k] && (e = dalloc(&s->d_stage[k], s->ld)) != cudaSuccess)
    return s->fail(EMRKC_ERR_OOM, "device allocation failed");
  // the staging buffer is refilled only after its previous copy-out
  if (s->stage_used[k] && (e = cudaStreamWaitEvent(s->stream, s->ev_stage_free[k], 0)) != cudaSuccess)
    return s->cuda_fail(e, "state copy ordering");
  const size_t row = (size_t)s->n * sizeof(double);
  if (var == 0) {
    if (s->d_V32[s->cur]) {
      launch_ff_join(s->d_V32[s->cur], s->d_Vlo[s->cur], s->d_stage[k], s->n, s->stream);
      e = cudaGetLastError();
    } else {
      e = cudaMemcpyAsync(s->d_stage[k], s->d_V[s->cur], row, cudaMemcpyDeviceToDevice, s->stream);
    }
  } else if (s->zsize == 8) {
    e = cudaMemcpyAsync(s->d_stage[k], s->zrow(s->cur, var - 1), row, cudaMemcpyDeviceToDevice, s->stream);
  } else {
    s->ks.convert_z(s->n, s->zrow(s->cur, var - 1), s->d_stage[k], 1, s->stream);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return s->cuda_fail(e, "state staging");
  if ((e = cudaEventRecord(s->ev_stage_ready[k], s->stream)) != cudaSuccess) return s->cuda_fail(e, "state staging");
  if ((e = cudaStreamWaitEvent(s->copy_stream, s->ev_stage_ready[k], 0)) != cudaSuccess)
    return s->cuda_fail(e, "state copy ordering");
  if ((e = cudaMemcpyAsync(host_out, s->d_stage[k], row, cudaMemcpyDeviceToHost, s->copy_stream)) != cudaSuccess)
    return s->cuda_fail(e, "state copy");
  if ((e = cudaEventRecord(s->ev_stage_free[k], s->copy_stream)) != cudaSuccess) return s->cuda_fail(e, "state copy");
  s->stage_used[k] = true;
  s->stage_k = k ^ 1;
  return EMRKC_OK;
}

int emrkc_set_time(emrkc_solver* s, double t, int64_t steps) {
  if (!s) return EMRKC_ERR_ARG;
  if (!std::isfinite(t) || steps < 0) return s->fail(EMRKC_ERR_ARG, "invalid time or step count");
  s->t = t;
  s->steps = steps;
  return EMRKC_OK;
}

int emrkc_get_stats(emrkc_solver* s, emrkc_stats* out) {
  if (!s || !out) return EMRKC_ERR_ARG;
  cudaSetDevice(s->device);
  int rc = fused_pull(s);
  if (rc) return rc;
  s->harvest();
  std::memset(out, 0, sizeof(*out));
  out->t = s->t;
  out->steps = s->steps;
  out->s = s->last_s;
  out->m = s->last_m;
  out->eta = s->last_eta;
  out->rho_F = s->last_rhoF;
  out->rho_S = s->last_rhoS;
  out->pow_iters_F = s->itF;
  out->pow_iters_S = s->itS;
  out->total_pow_iters = s->total_it;
  out->launches = s->launches;
  out->matrix_entries = s->mat_entries;
  out->matrix_slots = s->mat_slots;
  for (int k = 0; k < EMRKC_NUM_PHASES; ++k) {
    out->phase_ms[k] = s->phase_ms[k];
    out->phase_launches[k] = s->phase_launches[k];
  }
  if (s->d_iters) {
    unsigned long long it[2] = {0, 0};
    double res[2] = {0, 0};
    cudaStreamSynchronize(s->stream);
    cudaMemcpy(it, s->d_iters, sizeof(it), cudaMemcpyDeviceToHost);
    cudaMemcpy(res, s->d_res, sizeof(res), cudaMemcpyDeviceToHost);
    out->lin_iters = (int)it[0];
    out->total_lin_iters = (int64_t)it[1];
    out->lin_residual = res[1] > 0 ? std::sqrt(res[0] / res[1]) : 0.0;
  }
  return EMRKC_OK;
}

const char* emrkc_last_error(const emrkc_solver* s) {
  if (!s) return g_create_error.c_str();
  return s->err.c_str();
}

int emrkc_estimate_rho_F_noalloc(emrkc_solver* s, double* d_v, double* d_w, int64_t n, double rho_warm,
                                 double* rho_out, int* it_out) {
  if (!s) return EMRKC_ERR_ARG;
  if (!d_v || !d_w || !rho_out) return s->fail(EMRKC_ERR_ARG, "null pointer");
  if (n != s->n) return s->fail(EMRKC_ERR_ARG, "vector length must equal the number of nodes");
  if (s->method != EMRKC_METHOD_EMRKC)
    return s->fail(EMRKC_ERR_ARG, "the allocation-free estimate is for emRKC solvers (f_F on V) only");
  if (!(rho_warm >= 0.0) || !std::isfinite(rho_warm)) return s->fail(EMRKC_ERR_ARG, "rho_warm must be >= 0");
  cudaSetDevice(s->device);
  ReduceScratch rs;
  const char* why = "";
  if (noalloc_scratch(s->device, s->stream, &rs, &why) != 0) return s->fail(EMRKC_ERR_CUDA, why);
  materialise_V(s);
  const double* V = s->d_V[s->cur];
  const bool mixed = s->precision == EMRKC_PREC_MIXED;
  double res[2] = {0.0, 0.0};
  auto read = [&](int first, int count) -> int {
    cudaError_t e = cudaMemcpyAsync(res, rs.result + first, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "allocation-free power iteration");
    return EMRKC_OK;
  };
  noalloc_sumsq(n, V, rs, 0, s->stream);
  noalloc_sumsq(n, d_v, rs, 1, s->stream);
  if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return s->cuda_fail(e, "allocation-free power iteration");
  int rc = read(0, 2);
  if (rc) return rc;
  const double ny = std::sqrt(res[0]);
  double nv = std::sqrt(res[1]);
  const double delta = ny > 0.0 ? ny * s->opt.pow_eps : s->opt.pow_eps;
  double rho = rho_warm;
  int it = 0;
  if (nv == 0.0) {
    *rho_out = 0.0;
    if (it_out) *it_out = 0;
    return EMRKC_OK;
  }
  double* cur = d_v;
  double* nxt = d_w;
  const double tol = pow_tol_for(s, rho);
  const int max_iter = pow_max_iter_for(s, rho);
  double q = delta / nv, rho_old = 0.0;
  while (std::fabs(rho - rho_old) >= tol * rho && it < max_iter) {
    rho_old = rho;
    PowerFArgs a;
    a.n = n;
    a.V = V;
    a.v_old = cur;
    a.v_new = nxt;
    a.q = q;
    a.slot = 2;
    noalloc_power_F(a, s->ell, mixed, rs, s->stream);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return s->cuda_fail(e, "allocation-free power iteration");
    if ((rc = read(2, 1))) return rc;
    std::swap(cur, nxt);
    ++it;
    nv = std::sqrt(res[0]);
    if (nv == 0.0) {
      rho = 0.0;
      break;
    }
    q = delta / nv;
    rho = nv / delta;
  }
  if (cur != d_v) {
    cudaError_t e = cudaMemcpyAsync(d_v, cur, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return s->cuda_fail(e, "allocation-free power iteration");
  }
  *rho_out = rho;
  if (it_out) *it_out = it;
  return EMRKC_OK;
}

void emrkc_destroy(emrkc_solver* s) {
  if (!s) return;
  free_all(s);
  delete s;
}

}  // extern "C"

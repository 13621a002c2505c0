// Internal definitions shared by the host runtime units (solver.cpp,
// batch_host.cpp): the solver object, the host RKC coefficients (Algorithm 1)
// and the rest states of the ionic models.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "emrkc.h"
#include "launch.h"
#include "rkc_coeffs.h"

namespace emrkc {

// ---- Algorithm 1 (FP64): the shared definition of rkc_coeffs.h -------------
inline int stages_for(double dt, double rho, double eps, double* l_s) { return rkc_stages(dt, rho, eps, l_s); }

struct Coeffs {
  std::vector<double> mu, nu, kappa, c;
};

inline Coeffs make_coeffs(int s, double eps) {
  Coeffs co;
  co.mu.assign(s + 1, 0.0);
  co.nu.assign(s + 1, 0.0);
  co.kappa.assign(s + 1, 0.0);
  co.c.assign(s + 1, 0.0);
  rkc_coeffs(s, eps, co.mu.data(), co.nu.data(), co.kappa.data(), co.c.data());
  return co;
}


// Rest states (Sec. 5: "provided by the ionic model's definition").
inline std::vector<double> rest_state(int model) {
  switch (model) {
    case EMRKC_MODEL_NONE:
      return {0.0};
    case EMRKC_MODEL_PASSIVE:
      return {0.0, 1.0, 1.0};
    case EMRKC_MODEL_HH: {
      // gates at z_inf(V_rest), rates at v = 0
      const double am = 2.5 / std::expm1(2.5), bm = 4.0;
      const double ah = 0.07, bh = 1.0 / (std::exp(3.0) + 1.0);
      const double an = 0.1 * 1.0 / std::expm1(1.0), bn = 0.125;
      return {-75.0, am / (am + bm), ah / (ah + bh), an / (an + bn)};
    }
    case EMRKC_MODEL_TTP06_EPI:
      // V; m h j xr1 xr2 xs r s d f f2 fCass; Rbar Ki Nai Cai CaSR CaSS
      return {-85.23, 0.00172, 0.7444,  0.7045, 0.00621, 0.4712, 0.0095,   2.42e-8, 0.999998, 3.373e-5,
              0.7888, 0.9755,  0.9953,  0.9073, 136.89,  8.604,  0.000126, 3.64,    0.00036};
    default:
      return {};
  }
}

// slot of rs.result (in doubles) where the flags words start
constexpr int kFlagsSlot = 16;

struct Timing {
  int cls;
  cudaEvent_t a, b;
};


}  // namespace emrkc

struct emrkc_solver {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  emrkc_options opt{};
  int model = 0, N = 1, nE = 0, nS = 0, precision = 0;
  size_t zsize = 8;   // bytes per stored z value
  size_t rsize = 8;   // bytes per forcing value (compute type)
  int64_t n = 0, ld = 0;
  emrkc::KernelSet ks{};
  emrkc::Ell ell{};
  // device buffers
  int64_t* d_slice_ptr = nullptr;
  int32_t* d_width = nullptr;
  int32_t* d_col = nullptr;
  double* d_val = nullptr;
  float* d_val32 = nullptr;
  double* d_V[3] = {nullptr, nullptr, nullptr};
  void* d_Z[3] = {nullptr, nullptr, nullptr};
  double* d_U[3] = {nullptr, nullptr, nullptr};
  float* d_V32[3] = {nullptr, nullptr, nullptr};  // mixed: hi part of V per state buffer
  float* d_Vlo[3] = {nullptr, nullptr, nullptr};  // mixed: lo part of V (V = hi + lo)
  float* d_Vn32 = nullptr;                         // mixed: hi of V_n when s >= 2
  float* d_D[3] = {nullptr, nullptr, nullptr};    // mixed: inner increments delta_k
  float* d_LV = nullptr;                          // mixed: L V_{j-1}
  void* d_F = nullptr;
  uint8_t* d_mask = nullptr;
  // pipelined host I/O: a copy stream, a second mask buffer (the one no
  // enqueued step reads) and two staging buffers for state reads
  cudaStream_t copy_stream = nullptr;  // device-to-host copies (state reads)
  cudaStream_t h2d_stream = nullptr;   // host-to-device copies (stimulus masks)
  uint8_t* d_mask_alt = nullptr;
  int mask_idx = 0;                       // which of the two mask buffers d_mask is
  bool mask_free_rec[2] = {false, false};
  cudaEvent_t ev_mask_free[2] = {nullptr, nullptr};  // main stream: last use of mask buffer k
  cudaEvent_t ev_mask_ready = nullptr;                 // h2d stream: mask copy done
  double* d_stage[2] = {nullptr, nullptr};
  bool stage_used[2] = {false, false};
  int stage_k = 0;
  cudaEvent_t ev_stage_ready[2] = {nullptr, nullptr};  // main stream: staging buffer k filled
  cudaEvent_t ev_stage_free[2] = {nullptr, nullptr};   // copy stream: staging buffer k copied out
  double* d_vF = nullptr;
  double* d_vF2 = nullptr;
  double* d_vS = nullptr;
  double* d_vS2 = nullptr;
  double* d_fy = nullptr;
  double* d_act = nullptr;
  double* d_Vn = nullptr;
  double* d_tmp = nullptr;
  double* d_rest = nullptr;
  int* d_flags = nullptr;
  emrkc::ReduceScratch rs{};
  double* h_pin = nullptr;  // pinned: [0..7] results, [8] flags
  int cur = 0;
  double amp = 0, t_on = 0, t_off = -1, chi = 1, Cm = 1;
  double rhoF_raw = 0, rhoS_raw = 0;
  bool rho_done = false;
  double t = 0;
  int64_t steps = 0;
  int last_s = 0, last_m = 0;
  double last_eta = 0, last_rhoF = 0, last_rhoS = 0;
  int itF = 0, itS = 0;
  int64_t total_it = 0, launches = 0;
  int64_t mat_entries = 0, mat_slots = 0;
  int tma_grid = 0;  // persistent bulk-copy stage kernel grid (mixed path), 0 = off
  int tma_nbuf = 3;  // its stage buffers per CTA (3: state region + two ELL buffers, prefetching)
  int tma_ell = 1;   // it stages the ELL slices of a tile
  int pdl = 0;             // mixed path: programmatic dependent launch of the step kernels
  // Algorithm 5 in one cooperative launch (emRKC)
  int pfused_grid = 0;
  int pcluster = 0;  // CTAs of the single-cluster power iteration (0: not available)
  double* d_ppart = nullptr;      // 2 x 4 x grid partial sums
  unsigned int* d_pbar = nullptr; // grid barrier
  // EXEX-RL / IMEX-RL (rl_methods.cu)
  int method = 0;
  double* d_mass = nullptr;     // lumped mass (IMEX-RL)
  double* d_cg[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // r, z, q, p0, p1, P^-1
  double* d_part = nullptr;     // CG partial sums: 4 per CTA, set-up then solve
  unsigned int* d_bar = nullptr;        // grid barrier of the CG launch
  unsigned long long* d_iters = nullptr;  // CG iterations: last, total
  double* d_res = nullptr;      // final <r, r>_M, <c, c>_M
  int pcg_grid = 0;
  // mRKC (mrkc.cu)
  emrkc::MrkcKernels mk{};
  double* d_Um[3] = {nullptr, nullptr, nullptr};  // inner stages, stiff-gate part
  int ell_wmax = 0;  // widest sliced-ELL slice
  // device-resident step (emRKC on problems one cluster holds): cluster
  // size (0: off), the device state, its host copy, and whether the host's
  // rho, iteration and stage-count fields are behind the device's
  int fcluster = 0;
  emrkc::FusedStepState* d_fstate = nullptr;
  double* d_ctab = nullptr;  // Algorithm 1 tables of the fused step (rkc_coeffs.h layout)
  emrkc::FusedStepState h_fstate{};
  bool fstate_stale = false;
  bool act_on = false;
  double phase_ms[EMRKC_NUM_PHASES] = {0};
  int64_t phase_launches[EMRKC_NUM_PHASES] = {0};
  std::vector<emrkc::Timing> pending;
  std::vector<cudaEvent_t> event_pool;
  std::map<int, emrkc::Coeffs> coeff_cache;
  std::string err;

  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return EMRKC_ERR_CUDA;
  }
  const emrkc::Coeffs& coeffs(int s) {
    auto it = coeff_cache.find(s);
    if (it == coeff_cache.end()) it = coeff_cache.emplace(s, emrkc::make_coeffs(s, opt.eps)).first;
    return it->second;
  }
  cudaEvent_t get_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // Bracket one kernel launch with events when profiling.
  template <class Fn>
  void launch(int cls, Fn&& fn) {
    if (opt.profile) {
      emrkc::Timing tm{cls, get_event(), get_event()};
      cudaEventRecord(tm.a, stream);
      fn();
      cudaEventRecord(tm.b, stream);
      pending.push_back(tm);
    } else {
      fn();
    }
    ++launches;
    ++phase_launches[cls];
  }
  void harvest() {
    for (auto& tm : pending) {
      float ms = 0.f;
      cudaEventSynchronize(tm.b);
      cudaEventElapsedTime(&ms, tm.a, tm.b);
      phase_ms[tm.cls] += ms;
      event_pool.push_back(tm.a);
      event_pool.push_back(tm.b);
    }
    pending.clear();
  }
  void* zrow(int buf, int k) const { return (char*)d_Z[buf] + (size_t)k * ld * zsize; }
};


// Runtime helpers implemented in solver.cpp and used by the batch runtime.
namespace emrkc {
int solver_update_rho(emrkc_solver* s);   // Algorithm 5 for rho_F and rho_S now
void solver_materialise_V(emrkc_solver* s);
}  // namespace emrkc

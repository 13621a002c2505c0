// Internal interface between the host runtime (solver.cpp) and the CUDA
// kernels (kernels_fp64.cu, kernels_mixed.cu).  Plain structs of device
// pointers and scalars; no CUDA types leak into the host runtime beyond
// cudaStream_t.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace emrkc {

// Sliced ELL: slices of 32 consecutive rows; slice b stores width[b]
// entries per row at slice_ptr[b] + k*32 + (row % 32), k < width[b].
// Padding entries have col = the row itself and val = 0.
struct Ell {
  int64_t n = 0;
  int64_t n_slices = 0;
  const int64_t* slice_ptr = nullptr;
  const int32_t* width = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;  // FP64 mode: L including the diagonal
  const float* val32 = nullptr; // mixed mode: off-diagonal L only
};

// Deterministic two-level reduction scratch: per-block partial sums, a
// ticket counter and result slots.
struct ReduceScratch {
  double* partials = nullptr;   // >= kReduceMaxBlocks entries
  unsigned int* ticket = nullptr;
  double* result = nullptr;     // result slots (device)
};
constexpr int kReduceBlock = 256;
constexpr int kReduceMaxBlocks = 1024;

// One outer stage j of the emRKC step (Algorithm 3): exponential Euler of
// the gates at g_{j-1}, f_S at y_E, the first inner RKC stage (needs one
// SpMV of V_{j-1}) and the z-part of g_j.
struct StageArgs {
  int64_t n = 0, ld = 0;
  const double* Vm1 = nullptr;  // V of g_{j-1}
  const void* Zm1 = nullptr;    // z block of g_{j-1} ((N-1) x ld, Z type)
  const double* Vm2 = nullptr;  // g_{j-2} (j >= 2 only)
  const void* Zm2 = nullptr;
  double* Vout = nullptr;       // V of g_j (written when m == 1)
  void* Zout = nullptr;         // z block of g_j
  double nu = 1, kappa = 0, mu_dt = 0;  // outer coefficients of stage j
  double eta = 0;               // inner step
  double cm_inner = 1;          // c_m of the inner iteration
  double mu1_eta = 0;           // mu'_1 * eta (inner first stage)
  int m = 1;                    // inner stage count
  double* U1 = nullptr;         // u_1 of the inner iteration (m >= 2)
  void* F = nullptr;            // frozen forcing (I_stim - I_ion)/Cm (m >= 2; R type)
  const uint8_t* mask = nullptr;
  double stim = 0;              // stimulus amplitude at this stage's time
  double inv_Cm = 1, Cm = 1;
  // epilogue of the last kernel of a step
  int final_stage = 0;
  const double* Vn = nullptr;   // V at the start of the step
  double* act = nullptr;        // activation times (nullptr: off)
  double t_n = 0, dt = 0, threshold = -20;
  int* flags = nullptr;         // bit 0: non-finite V
  double* Vn_copy = nullptr;    // if set: store V_n (first stage when s >= 2)
  // precomputed reciprocals / products (no divisions in the kernels)
  double inv_eta = 1, mu_dt_over_eta = 0, mu1 = 1;
  // mixed mode: FP32 mirror of V, FP32 increments delta_k = u_k - V_{j-1}
  const float* V32m1 = nullptr;
  float* V32out = nullptr;      // written with Vout (m == 1)
  float* D1 = nullptr;          // delta_1 = mu'_1 eta (L V + F)   (m >= 2)
  float* LV = nullptr;          // L V_{j-1}, reused by the inner stages (m >= 2)
  float f_nu = 1, f_kappa = 0, f_mudt = 0, f_inv_eta = 1, f_cm = 1, f_mu1 = 1, f_mu1eta = 0;
  float f_eta = 0, f_stim = 0, f_inv_Cm = 1;
  // mixed mode: V is the unevaluated sum hi + lo of two floats (V32 = hi)
  const float* Vlo_m1 = nullptr;
  const float* Vhi_m2 = nullptr;
  const float* Vlo_m2 = nullptr;
  float* Vlo_out = nullptr;
  const float* Vn32 = nullptr;  // hi of V_n (epilogue)
  float* Vn32_copy = nullptr;   // store hi of V_n (first stage when s >= 2)
  float f_th = -20;
  int tma_grid = 0;             // > 0: persistent bulk-copy variant with this grid
  int tma_nbuf = 3;             // bulk-copy variant: 1 or 2 whole-tile stage buffers per CTA, or 3 = one
                                // state region + two ELL buffers with the next tile prefetched
  int tma_ell = 1;              // bulk-copy variant stages the tile's ELL slices (1) or reads them (0)
  int pdl = 0;                  // 1: programmatic dependent launch
  int ell_wmax = 1 << 30;       // widest sliced-ELL slice (selects unrolled row variants)
};

// Inner RKC stage k >= 2 over f_u(u) = L u + F:
// u_k = nu'_k u_{k-1} + kappa'_k u_{k-2} + mu'_k eta (L u_{k-1} + F).
// When last: f_bar_V = (u_m - V_{j-1})/eta and V_j = nu V_{j-1} + kappa V_{j-2} + mu dt f_bar_V.
struct InnerArgs {
  int64_t n = 0;
  const double* u1 = nullptr;   // u_{k-1}
  const double* u2 = nullptr;   // u_{k-2}
  double* uk = nullptr;         // u_k (when not last)
  const void* F = nullptr;
  double nu = 0, kappa = 0, mu_eta = 0;
  int last = 0;
  const double* Vm1 = nullptr;
  const double* Vm2 = nullptr;
  double* Vout = nullptr;
  double onu = 1, okappa = 0, omu_dt = 0, eta = 1;
  int final_stage = 0;
  const double* Vn = nullptr;
  double* act = nullptr;
  double t_n = 0, dt = 0, threshold = -20;
  int* flags = nullptr;
  double inv_eta = 1;
  // mixed mode: delta_k = nu'_k delta_{k-1} + kappa'_k delta_{k-2} + mu'_k eta (LV + L delta_{k-1} + F)
  const float* d1 = nullptr;    // delta_{k-1}
  const float* d2 = nullptr;    // delta_{k-2} (nullptr: delta_0 = 0)
  float* dk = nullptr;          // delta_k (when not last)
  const float* LV = nullptr;
  float* V32out = nullptr;
  float f_nu = 0, f_kappa = 0, f_mueta = 0, f_inv_eta = 1;
  const float* Vhi1 = nullptr;  // V_{j-1} as hi + lo
  const float* Vlo1 = nullptr;
  const float* Vhi2 = nullptr;  // V_{j-2} (nullptr when j == 1)
  const float* Vlo2 = nullptr;
  float* Vlo_out = nullptr;     // V32out holds hi
  const float* Vn32 = nullptr;
  float f_okappa = 0, f_omu_dt = 0, f_th = -20;
  int ell_wmax = 1 << 30;       // widest sliced-ELL slice (selects unrolled row variants)
  int pdl = 0;                  // 1: programmatic dependent launch
  // mixed path: L V_{j-1} + F as delta_1 / (mu'_1 eta) from d1 (1) or d2 (2),
  // or from the array LV (0, inner stages k >= 4)
  int lf_src = 0;
  float f_inv_mu1eta = 0.0f;
};

// Power iteration (Algorithm 5) kernels.
struct PowerFArgs {
  int64_t n = 0;
  const double* V = nullptr;
  const double* v_old = nullptr;
  double* v_new = nullptr;
  double q = 0;
  int slot = 0;  // result slot for the sum of squares of v_new
};

struct PowerSArgs {
  int64_t n = 0, ld = 0;
  const double* V = nullptr;
  const void* Z = nullptr;      // state z block (Z type)
  const double* v_old = nullptr;  // N x ld
  double* v_new = nullptr;        // N x ld
  const double* fy = nullptr;     // f_S(y), N x ld
  double q = 0;
  const uint8_t* mask = nullptr;
  double stim = 0, Cm = 1;
  int slot = 0;
};

// Algorithm 5 for rho_F and rho_S in one cooperative launch.
struct PowerFusedArgs {
  int64_t n = 0, ld = 0;
  const double* V = nullptr;
  const float* Vhi = nullptr;          // mixed path: V = hi + lo (then V is not read)
  const float* Vlo = nullptr;
  const void* Z = nullptr;
  double* vF[2] = {nullptr, nullptr};  // iterate on V: current in [0] at entry
  double* vS[2] = {nullptr, nullptr};  // iterate on the full state (N x ld)
  double* fy = nullptr;                // FP64 path: f_S(y), N x ld
  const uint8_t* mask = nullptr;
  double stim = 0, Cm = 1;
  float f_inv_Cm = 1;                  // (float)(1 / Cm)
  int ell_wmax = 1 << 30;              // widest sliced-ELL slice (rows of <= 8: split row loads)
  double eps = 1e-8, tol = 1e-2;
  int max_iter = 50;
  double tol_cold = 1e-4;        // a start with warm value 0 (no initial guess)
  int max_iter_cold = 1000;
  double rhoF_warm = 0, rhoS_warm = 0;
  double* part = nullptr;              // 2 x 4 x grid partial sums
  unsigned int* bar = nullptr;         // grid barrier
  int* flags = nullptr;
  long long spin_limit = 0;
  double* out = nullptr;               // rho_F, rho_S, it_F, it_S, last buffer of v_F, of v_S
};

// Device-resident emRKC step for problems one thread-block cluster holds:
// Algorithm 5 (when due), Algorithm 1 and every outer and inner stage of
// Algorithm 3 in one launch, with no host round trip.  The state below
// lives in device memory and carries the power iteration from step to step.
struct FusedStepState {
  double rhoF_raw = 0, rhoS_raw = 0;  // last estimates (warm start of Algorithm 5)
  double rhoF = 0, rhoS = 0, eta = 0; // values the last step used (safety factor, floor)
  int curF = 0, curS = 0;             // iterate buffer holding the last iterate (1: the second)
  int s = 0, m = 0, itF = 0, itS = 0; // last step's stage counts and power iterations
  long long total_it = 0;
};
constexpr int kFusedMaxStages = 128;  // s and m of one fused step (flags bit 4 beyond)

struct FusedStepArgs {
  int64_t n = 0, ld = 0;
  int b0 = 0;                          // state buffer of y_n; y_{n+1} goes to (b0 + 1) mod 3
  double* V[3] = {nullptr, nullptr, nullptr};  // FP64 path
  void* Z[3] = {nullptr, nullptr, nullptr};    // z blocks ((N-1) x ld, Z type)
  float* Vhi[3] = {nullptr, nullptr, nullptr}; // mixed path: V = hi + lo
  float* Vlo[3] = {nullptr, nullptr, nullptr};
  double* U[3] = {nullptr, nullptr, nullptr};  // FP64 inner iterates
  float* D[3] = {nullptr, nullptr, nullptr};   // mixed inner increments
  void* F = nullptr;                   // frozen forcing (R type)
  float* LV = nullptr;                 // mixed: L V + F for inner stages k >= 4
  double* Vn = nullptr;                // FP64: copy of V_n when s >= 3
  float* Vn32 = nullptr;               // mixed: copy of V_n hi when s >= 3
  const uint8_t* mask = nullptr;
  double amp = 0, t_on = 0, t_off = -1;
  double Cm = 1;
  double t_n = 0, dt = 0, threshold = -20;
  double* act = nullptr;
  int* flags = nullptr;                // bit 0: non-finite V; bit 4: s or m above kFusedMaxStages
  double eps = 0.05;                   // RKC damping
  int ell_wmax = 1 << 30;              // widest sliced-ELL slice (rows kept in registers when <= 8)
  int due = 0;                         // 1: Algorithm 5 before the step
  int fixed = 0;                       // 1: rho_F_fixed, rho_S_fixed as given (no estimate)
  double rho_F_fixed = 0, rho_S_fixed = 0;
  double safety = 1.05, rho_S_min = 0;
  PowerFusedArgs pw;                   // Algorithm 5: vF, vS in buffer order, scratch, tolerances
  FusedStepState* state = nullptr;
  // Algorithm 1 without FP64 divisions on the device: the coefficient
  // tables of rkc_coeffs.h for s = 1 .. kFusedMaxStages, and host-side
  // reciprocals
  const double* ctab = nullptr;
  double beta = 2.0, two_dt = 0, inv_two_dt = 0, inv_Cm = 1;
};

struct Launchers;  // per precision mode

// Kernel launchers, implemented per precision (FP64 / mixed) and per model.
struct KernelSet {
  int model = 0;
  int N = 1, nE = 0, nS = 0;
  void (*stage)(const StageArgs&, const Ell&, int has_m2, cudaStream_t) = nullptr;
  void (*inner)(const InnerArgs&, const Ell&, cudaStream_t) = nullptr;
  void (*power_F)(const PowerFArgs&, const Ell&, const ReduceScratch&, cudaStream_t) = nullptr;
  void (*power_S)(const PowerSArgs&, const ReduceScratch&, cudaStream_t) = nullptr;
  void (*fS_eval)(const PowerSArgs&, double* out, cudaStream_t) = nullptr;  // fy = f_S(y)
  void (*state_sumsq)(int64_t n, int64_t ld, int nz, const double* V, const void* Z,
                      const ReduceScratch&, int slot, cudaStream_t) = nullptr;
  void (*convert_z)(int64_t count, const void* src, double* dst, int to_double, cudaStream_t) = nullptr;
  int (*tma_grid)(int device, int wmax, int nbuf, int ell) = nullptr;  // grid of the persistent stage kernel (0: not used)
  cudaError_t (*power_fused)(const PowerFusedArgs&, const Ell&, int grid, cudaStream_t) = nullptr;
  int (*power_fused_grid)(int device) = nullptr;
  int (*power_cluster_size)(int device) = nullptr;  // CTAs of the single-cluster variant (0: unavailable)
  cudaError_t (*step_fused)(const FusedStepArgs&, const Ell&, int cluster, cudaStream_t) = nullptr;
  int (*step_fused_cluster_size)(int device) = nullptr;  // CTAs of the fused step's cluster (0: unavailable)
  int (*step_fused_block)(void) = nullptr;                // largest CTA of the fused step
};

// mRKC (mrkc.cu, FP64): one outer stage (stage kernel, inner stage 1) or
// one inner stage k >= 2 on the block (V, z_k) of the stiffest gate k.
struct MrkcArgs {
  int64_t n = 0, ld = 0;
  const double* Vm1 = nullptr;   // g_{j-1}
  const double* Zm1 = nullptr;
  const double* Vm2 = nullptr;   // g_{j-2} (nullptr for j = 1)
  const double* Zm2 = nullptr;
  double* Vout = nullptr;        // g_j
  double* Zout = nullptr;
  double nu = 1, kappa = 0, mu_dt = 0;   // outer coefficients of stage j
  double eta = 0, inv_eta = 0;
  int m = 1;                     // inner stages
  double mu1 = 0, mu1_eta = 0;   // inner stage 1
  double inu = 0, ikappa = 0, imu_eta = 0;  // inner stage k >= 2
  const double* uV1 = nullptr;   // u_{k-1}, u_{k-2} (V and z_k parts)
  const double* uV2 = nullptr;
  const double* um1 = nullptr;
  const double* um2 = nullptr;
  double* uVk = nullptr;         // u_k
  double* umk = nullptr;
  int last = 0;
  double* F = nullptr;           // frozen V forcing of f~_S
  const uint8_t* mask = nullptr;
  double stim = 0, inv_Cm = 1;
  int final_stage = 0;
  const double* Vn = nullptr;
  double* act = nullptr;
  double t_n = 0, dt = 0, threshold = 0;
  int* flags = nullptr;
};

struct MrkcPowerArgs {
  int64_t n = 0, ld = 0;
  const double* V = nullptr;
  const double* Z = nullptr;     // z block of the state (FP64)
  const double* v_old = nullptr; // 2 x ld: (v_V, v_k)
  double* v_new = nullptr;
  double q = 0;
  int slot = 0;
};

struct MrkcKernels {
  void (*stage)(const MrkcArgs&, const Ell&, bool has_m2, cudaStream_t) = nullptr;
  void (*inner)(const MrkcArgs&, const Ell&, cudaStream_t) = nullptr;
  void (*power_F)(const MrkcPowerArgs&, const Ell&, const ReduceScratch&, cudaStream_t) = nullptr;
  void (*power_S)(const PowerSArgs&, const ReduceScratch&, cudaStream_t) = nullptr;
  void (*fS)(const PowerSArgs&, double*, cudaStream_t) = nullptr;
  int stiff_gate = -1;           // index into z_E of the gate in f~_F, -1: none
};
bool get_kernels_mrkc(int model, MrkcKernels* k);

// EXEX-RL / IMEX-RL steps (rl_methods.cu, FP64).  One step reads the state
// buffer (V, Z) and writes (Vout, Zout).
struct RlArgs {
  int64_t n = 0, ld = 0;
  const double* V = nullptr;
  const double* Z = nullptr;     // NZ rows of ld
  double* Vout = nullptr;        // EXEX: V_{n+1}; IMEX: x_0 = V_n
  double* Zout = nullptr;
  const uint8_t* mask = nullptr;
  double stim = 0, inv_Cm = 1, dt = 0;
  double* act = nullptr;
  double t_n = 0, threshold = 0;
  int* flags = nullptr;
  // IMEX set-up
  const double* mass = nullptr;  // lumped mass M_i
  double* r = nullptr;
  double* zr = nullptr;
  double* pinv = nullptr;        // 1 / (1 - dt L_ii)
  double* part0 = nullptr;       // 4 per set-up CTA
};

constexpr int kPcgBlock = 256;

struct PcgArgs {
  int64_t n = 0;
  double dt = 0, rtol = 0;
  int max_iter = 0;
  long long spin_limit = 0;
  const double* mass = nullptr;
  const double* pinv = nullptr;
  const double* Vn = nullptr;
  double* x = nullptr;
  double* r = nullptr;
  double* zr = nullptr;
  double* q = nullptr;
  double* p0 = nullptr;
  double* p1 = nullptr;
  double* part = nullptr;         // 4 per CTA of the PCG launch
  const double* part0 = nullptr;  // set-up partials
  int n_part0 = 0;
  double* res = nullptr;          // out: [0] final <r, r>_M, [1] <c, c>_M
  unsigned int* bar = nullptr;    // grid barrier: [0] arrivals, [1] generation
  unsigned long long* iters = nullptr;  // [0] last solve, [1] running total
  int* flags = nullptr;
  double* act = nullptr;
  double t_n = 0, threshold = 0;
};

int rl_exex_step(int model, const RlArgs& a, const Ell& A, cudaStream_t st);
int rl_imex_setup(int model, const RlArgs& a, const Ell& A, cudaStream_t st);
int rl_imex_setup_grid(int64_t n);
int pcg_grid(int device);
cudaError_t rl_imex_pcg(const PcgArgs& a, const Ell& A, int grid, cudaStream_t st);

// Float-float V of the mixed path: split a double into hi + lo, and join.
void launch_ff_split(const double* v, float* hi, float* lo, int64_t count, cudaStream_t st);
void launch_ff_join(const float* hi, const float* lo, double* v, int64_t count, cudaStream_t st);

// Defined in kernels_fp64.cu / kernels_mixed.cu.
bool get_kernels_fp64(int model, KernelSet* ks);
bool get_kernels_mixed(int model, KernelSet* ks);

// Precision-independent kernels (kernels_fp64.cu).
void launch_sumsq(int64_t count, const double* x, const ReduceScratch& rs, int slot, cudaStream_t st);
void launch_start_vector(uint64_t key, int64_t n, int64_t ld, int rows, double* v, cudaStream_t st);
void launch_fill(double* x, int64_t count, double value, cudaStream_t st);
void launch_fill_rows(void* z, int zsize, int64_t n, int64_t ld, int rows, const double* values,
                      cudaStream_t st);

// ---- Batched persistent step (batch.cu, batch_host.cpp) -------------------
constexpr int kBatchMaxStages = 32;  // s, m <= 32 for a batched instance
constexpr int kBatchMaxPhases = 64;  // s * m <= 64

// One instance of the batch as the persistent kernel sees it (device table).
// All buffers belong to the instance's own mixed-precision solver.
struct BatchInst {
  int model = 0, s = 1, m = 1, P = 1;  // P = s * m phases per step
  int cur = 0, ntiles = 0;
  int wmax = 0;  // widest sliced-ELL slice
  int64_t n = 0, ld = 0;
  float* Vhi[3] = {nullptr, nullptr, nullptr};
  float* Vlo[3] = {nullptr, nullptr, nullptr};
  float* Z[3] = {nullptr, nullptr, nullptr};
  float* D[3] = {nullptr, nullptr, nullptr};
  float* LV = nullptr;
  float* F = nullptr;
  float* Vn32 = nullptr;
  const uint8_t* mask = nullptr;
  double* act = nullptr;
  int* flags = nullptr;
  Ell ell{};
  double t = 0, dt = 0, amp = 0, t_on = 0, t_off = -1;
  int64_t steps = 0;
  float f_th = -20, f_inv_Cm = 1, f_eta = 0, f_inv_eta = 1, f_cm = 1, f_mu1 = 1, f_mu1eta = 0, f_inv_mu1eta = 0;
  double o_c[kBatchMaxStages + 1];      // outer stage times c_j
  float o_nu[kBatchMaxStages + 1];      // outer nu_j (1 for j = 1)
  float o_kappa[kBatchMaxStages + 1];   // outer kappa_j (0 for j = 1)
  float o_mudt[kBatchMaxStages + 1];    // outer mu_j dt
  float i_nu[kBatchMaxStages + 1];      // inner nu'_k
  float i_kappa[kBatchMaxStages + 1];   // inner kappa'_k
  float i_mueta[kBatchMaxStages + 1];   // inner mu'_k eta
};

// Work item: (instance, phase, tile), phase-major order.
struct BatchCtl {
  BatchInst* inst = nullptr;
  const uint64_t* items = nullptr;
  unsigned int n_items = 0;
  int tile = 1024;                 // nodes per work item
  unsigned int* ticket = nullptr;  // next item to take
  unsigned int* done = nullptr;    // [instance * kBatchMaxPhases + phase] completed tiles
  int* err = nullptr;              // bit 1: a dependency wait gave up
  long long spin_limit = 1 << 24;  // iterations of a dependency wait before giving up
  int dry = 0;                     // 1: no bookkeeping, no activation writes (autotuning)
};
inline uint64_t batch_item(int inst, int phase, int tile) {
  return ((uint64_t)(uint32_t)inst << 40) | ((uint64_t)(uint32_t)phase << 32) | (uint32_t)tile;
}
// tps: resident threads per SM the persistent kernel is compiled for (1024,
// 1536 or 2048)
void launch_batch_step(const BatchCtl& c, int grid, int block, int tps, cudaStream_t st);
int batch_blocks_per_sm(int block, int tps);
// Whole-batch host I/O: V of every instance (current state buffer, joined to
// double) into out[off[k] ...]; node masks from src[off[k] ...] into each
// instance's mask buffer.  ni instances, off has ni + 1 entries.
void launch_batch_join_V(const BatchInst* inst, const int64_t* off, int ni, double* out, cudaStream_t st);
void launch_batch_join_V32(const BatchInst* inst, const int64_t* off, int ni, float* out, cudaStream_t st);
void launch_batch_scatter_mask(uint8_t* const* masks, const int64_t* off, int ni, const uint8_t* src,
                               cudaStream_t st);
// out[k] = the flag word of instance k (bit 0: non-finite V), ni instances.
void launch_batch_gather_flags(const BatchInst* inst, int ni, int* out, cudaStream_t st);

// Allocation-free power iteration on f_F (noalloc.cu): static device scratch.
int noalloc_scratch(int device, cudaStream_t st, ReduceScratch* out, const char** why);
void noalloc_sumsq(int64_t count, const double* x, const ReduceScratch& rs, int slot, cudaStream_t st);
void noalloc_power_F(const PowerFArgs& a, const Ell& A, bool mixed, const ReduceScratch& rs, cudaStream_t st);

}  // namespace emrkc

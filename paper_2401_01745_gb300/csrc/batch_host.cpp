// Host runtime of the batched persistent step (emrkc_batch_* in emrkc.h).
//
// Each instance is an ordinary mixed-precision solver (it owns its buffers);
// the batch keeps a device table of the instances (BatchInst), a phase-major
// work list and per-instance phase counters, and replays
//   memset(done) -> memset(ticket) -> persistent kernel
// as one CUDA graph per step.  The plan (stage counts, coefficients, work
// list) is rebuilt when instances join or leave or dt changes; instance time
// and buffer rotation advance on the device and are mirrored on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "emrkc.h"
#include "launch.h"
#include "solver_internal.h"

using namespace emrkc;

namespace {

thread_local std::string g_batch_create_error;

struct Member {
  int id = 0;
  emrkc_solver* s = nullptr;
  bool rho_ready = false;
  int S = 0, M = 0;
};

}  // namespace

struct emrkc_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  emrkc_options opt{};
  std::vector<Member> members;
  int next_id = 1;
  bool dirty = true;
  double plan_dt = -1.0;
  std::vector<BatchInst> h_inst;
  BatchInst* d_inst = nullptr;
  size_t inst_cap = 0;
  uint64_t* d_items = nullptr;
  size_t items_cap = 0;
  unsigned int n_items = 0;
  unsigned int* d_ticket = nullptr;
  unsigned int* d_done = nullptr;
  size_t done_cap = 0;
  int* d_err = nullptr;
  int tile = 1024, block = 128, grid = 0;
  int sched = 0;  // order of the work list (rebuild)
  int tps = 1536; // resident threads per SM of the persistent kernel (register budget)
  long long spin_limit = 1 << 24;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  std::string err;
  // membership version (bumped by add / remove); the I/O tables follow it
  int64_t version = 0;
  // pipelined whole-batch host I/O: one copy stream per direction, two
  // staging buffers per direction, per-instance offsets into the
  // concatenated host arrays (member order) and mask pointers
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  int64_t io_version = -1, io_total = 0;
  int64_t* d_off = nullptr;
  size_t off_cap = 0;
  uint8_t** d_masks = nullptr;
  size_t masks_cap = 0;
  uint8_t* d_mstage[2] = {nullptr, nullptr};
  size_t mstage_cap[2] = {0, 0};
  double* d_vstage[2] = {nullptr, nullptr};
  size_t vstage_cap[2] = {0, 0};
  cudaEvent_t ev_mready[2] = {nullptr, nullptr}, ev_mfree[2] = {nullptr, nullptr};
  cudaEvent_t ev_vready[2] = {nullptr, nullptr}, ev_vfree[2] = {nullptr, nullptr};
  bool mfree_rec[2] = {false, false}, vfree_rec[2] = {false, false};
  int mk = 0, vk = 0;
  // kernel timing (emrkc_batch_set_profile): CUDA events around each
  // persistent launch on the batch's stream, read at emrkc_batch_sync
  bool profile = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending, prof_pool;
  double kernel_ms = 0.0;
  int64_t kernel_launches = 0;
  // every instance's flag word gathered into one device array and read with
  // one copy at emrkc_batch_sync
  int* d_flagv = nullptr;
  int* h_flagv = nullptr;
  size_t flagv_cap = 0;

  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return EMRKC_ERR_CUDA;
  }
  Member* find(int id) {
    for (auto& m : members)
      if (m.id == id) return &m;
    return nullptr;
  }
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  void harvest() {
    for (auto& pr : prof_pending) {
      float ms = 0.f;
      cudaEventSynchronize(pr.second);
      cudaEventElapsedTime(&ms, pr.first, pr.second);
      kernel_ms += ms;
      ++kernel_launches;
      prof_pool.push_back(pr);
    }
    prof_pending.clear();
  }
};

namespace {

template <class T>
cudaError_t grow(T** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  size_t c = std::max<size_t>(need, 1);
  c = c + c / 4;
  cudaError_t e = cudaMalloc((void**)p, c * sizeof(T));
  *cap = (e == cudaSuccess) ? c : 0;
  return e;
}

BatchCtl make_ctl(emrkc_batch* b, int dry) {
  BatchCtl c;
  c.inst = b->d_inst;
  c.items = b->d_items;
  c.n_items = b->n_items;
  c.tile = b->tile;
  c.ticket = b->d_ticket;
  c.done = b->d_done;
  c.err = b->d_err;
  c.dry = dry;
  c.spin_limit = b->spin_limit;
  return c;
}

// Fill the device table entry of one instance for step size dt.
int fill_inst(emrkc_batch* b, Member& mb, double dt, BatchInst* I) {
  emrkc_solver* s = mb.s;
  double rhoF, rhoS;
  if (s->opt.rho_every == EMRKC_RHO_FIXED) {
    rhoF = s->opt.rho_F;
    rhoS = s->opt.rho_S;
  } else {
    if (!mb.rho_ready) {
      int rc = solver_update_rho(s);
      if (rc) return b->fail(rc, std::string("power iteration: ") + s->err);
      mb.rho_ready = true;
    }
    rhoF = s->opt.safety * s->rhoF_raw;
    rhoS = std::max(s->opt.safety * s->rhoS_raw, s->opt.rho_S_min);
  }
  double l_s = 0.0;
  const int S = stages_for(dt, rhoS, s->opt.eps, &l_s);
  const double eta = 2.0 * dt / l_s;
  const int Mi = stages_for(eta, rhoF, s->opt.eps, nullptr);
  if (S > kBatchMaxStages || Mi > kBatchMaxStages || S * Mi > kBatchMaxPhases)
    return b->fail(EMRKC_ERR_ARG, "stage counts beyond the batch limits (s, m <= 32, s*m <= 64)");
  const Coeffs& co = s->coeffs(S);
  const Coeffs& ci = s->coeffs(Mi);
  *I = BatchInst();
  I->model = s->model;
  I->s = S;
  I->m = Mi;
  I->P = S * Mi;
  I->cur = s->cur;
  I->n = s->n;
  I->ld = s->ld;
  I->ntiles = (int)((s->n + b->tile - 1) / b->tile);
  I->wmax = s->ell_wmax;
  for (int k = 0; k < 3; ++k) {
    I->Vhi[k] = s->d_V32[k];
    I->Vlo[k] = s->d_Vlo[k];
    I->Z[k] = static_cast<float*>(s->d_Z[k]);
    I->D[k] = s->d_D[k];
  }
  I->LV = s->d_LV;
  I->F = static_cast<float*>(s->d_F);
  I->Vn32 = s->d_Vn32;
  I->mask = s->d_mask;
  I->act = s->act_on ? s->d_act : nullptr;
  I->flags = s->d_flags;
  I->ell = s->ell;
  I->t = s->t;
  I->dt = dt;
  I->amp = s->amp;
  I->t_on = s->t_on;
  I->t_off = s->t_off;
  I->steps = s->steps;
  I->f_th = (float)s->opt.act_threshold;
  I->f_inv_Cm = (float)(1.0 / s->Cm);
  I->f_eta = (float)eta;
  I->f_inv_eta = (float)(1.0 / eta);
  I->f_cm = (float)ci.c[Mi];
  I->f_mu1 = (float)ci.mu[1];
  I->f_mu1eta = (float)(ci.mu[1] * eta);
  I->f_inv_mu1eta = (float)(1.0 / (ci.mu[1] * eta));
  for (int j = 0; j <= S; ++j) {
    I->o_c[j] = co.c[j];
    I->o_nu[j] = j >= 2 ? (float)co.nu[j] : 1.0f;
    I->o_kappa[j] = j >= 2 ? (float)co.kappa[j] : 0.0f;
    I->o_mudt[j] = j >= 1 ? (float)(co.mu[j] * dt) : 0.0f;
  }
  for (int k = 0; k <= Mi; ++k) {
    I->i_nu[k] = (float)ci.nu[k];
    I->i_kappa[k] = (float)ci.kappa[k];
    I->i_mueta[k] = (float)(ci.mu[k] * eta);
  }
  mb.S = S;
  mb.M = Mi;
  return EMRKC_OK;
}

int rebuild(emrkc_batch* b, double dt) {
  b->drop_graph();
  const size_t ni = b->members.size();
  b->h_inst.assign(ni, BatchInst());
  int maxP = 0;
  for (size_t i = 0; i < ni; ++i) {
    int rc = fill_inst(b, b->members[i], dt, &b->h_inst[i]);
    if (rc) return rc;
    maxP = std::max(maxP, b->h_inst[i].P);
  }
  // Skewed order: an instance's phase p is emitted only after `lag` tiles of
  // other work have been emitted since its phase p - 1, so that compute-heavy
  // stage tiles of some instances run beside memory-bound SpMV tiles of
  // others and a dependent tile rarely waits.  Every item still follows all
  // items it depends on (deadlock-free in-order consumption).
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  b->grid = std::max(1, sms * std::max(1, batch_blocks_per_sm(b->block, b->tps)));
  // Schedule 0 emits an instance's whole phase at once (the first ready
  // instance in index order); schedules 1 and 2 emit at most 16 or 4 tiles of
  // an instance before moving on to the next ready instance (cyclically), so
  // that tiles of different instances, models and phases interleave finely.
  std::vector<uint64_t> items;
  {
    const int64_t lag = 2 * (int64_t)std::max(b->grid, 1);
    const int chunk = b->sched == 1 ? 16 : b->sched == 2 ? 4 : (1 << 30);
    std::vector<int> next(ni, 0), tnext(ni, 0);
    std::vector<int64_t> ready(ni, 0);
    size_t left = ni;
    int64_t now = 0;
    size_t cursor = 0;
    while (left > 0) {
      int best = -1;
      if (b->sched == 0) {
        for (size_t i = 0; i < ni; ++i) {
          if (next[i] >= b->h_inst[i].P) continue;
          if (best < 0 || ready[i] < ready[best]) best = (int)i;
          if (ready[i] <= now) {
            best = (int)i;
            break;
          }
        }
      } else {
        for (size_t q = 0; q < ni; ++q) {
          const size_t i = (cursor + q) % ni;
          if (next[i] >= b->h_inst[i].P) continue;
          if (best < 0 || ready[i] < ready[best]) best = (int)i;
          if (ready[i] <= now) {
            best = (int)i;
            break;
          }
        }
        cursor = (size_t)best + 1;
      }
      const int p = next[best];
      const int nt = b->h_inst[best].ntiles;
      const int t1 = std::min(nt, tnext[best] + chunk);
      for (int t = tnext[best]; t < t1; ++t) items.push_back(batch_item(best, p, t));
      now = std::max(now, ready[best]) + (t1 - tnext[best]);
      tnext[best] = t1;
      if (t1 == nt) {
        tnext[best] = 0;
        ready[best] = now + lag;
        if (++next[best] >= b->h_inst[best].P) --left;
      }
    }
  }
  if (items.size() >= 0xffffffffull) return b->fail(EMRKC_ERR_ARG, "too many work items");
  b->n_items = (unsigned int)items.size();
  cudaError_t e;
  if ((e = grow(&b->d_inst, &b->inst_cap, ni)) != cudaSuccess) return b->fail(EMRKC_ERR_OOM, "batch table");
  if ((e = grow(&b->d_items, &b->items_cap, items.size())) != cudaSuccess) return b->fail(EMRKC_ERR_OOM, "batch items");
  if ((e = grow(&b->d_done, &b->done_cap, std::max<size_t>(ni, 1) * kBatchMaxPhases)) != cudaSuccess)
    return b->fail(EMRKC_ERR_OOM, "batch counters");
  if (ni) e = cudaMemcpyAsync(b->d_inst, b->h_inst.data(), ni * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return b->cuda_fail(e, "batch plan upload");
  b->plan_dt = dt;
  b->dirty = false;
  return EMRKC_OK;
}

// Enqueue one step: counters reset + persistent launch (as a graph if enabled).
int enqueue_step(emrkc_batch* b, int dry) {
  const size_t ni = b->members.size();
  if (ni == 0 || b->n_items == 0) return EMRKC_OK;
  cudaError_t e;
  if (!dry && b->opt.use_graphs && !b->profile) {
    if (!b->exec) {
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return b->cuda_fail(e, "graph capture");
      cudaMemsetAsync(b->d_done, 0, ni * kBatchMaxPhases * sizeof(unsigned int), b->stream);
      cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned int), b->stream);
      launch_batch_step(make_ctl(b, 0), b->grid, b->block, b->tps, b->stream);
      e = cudaStreamEndCapture(b->stream, &b->graph);
      if (e != cudaSuccess) return b->cuda_fail(e, "graph capture");
      e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      if (e != cudaSuccess) return b->cuda_fail(e, "graph instantiation");
    }
    e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return b->cuda_fail(e, "graph launch");
  } else {
    cudaMemsetAsync(b->d_done, 0, ni * kBatchMaxPhases * sizeof(unsigned int), b->stream);
    cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned int), b->stream);
    std::pair<cudaEvent_t, cudaEvent_t> pr{nullptr, nullptr};
    if (b->profile && !dry) {
      if (!b->prof_pool.empty()) {
        pr = b->prof_pool.back();
        b->prof_pool.pop_back();
      } else if ((e = cudaEventCreate(&pr.first)) != cudaSuccess || (e = cudaEventCreate(&pr.second)) != cudaSuccess) {
        return b->cuda_fail(e, "event creation");
      }
      cudaEventRecord(pr.first, b->stream);
    }
    launch_batch_step(make_ctl(b, dry), b->grid, b->block, b->tps, b->stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return b->cuda_fail(e, "batch launch");
    if (pr.second) {
      cudaEventRecord(pr.second, b->stream);
      b->prof_pending.push_back(pr);
    }
  }
  ++b->launches;
  return EMRKC_OK;
}

int64_t solver_bytes(const emrkc_solver* s) {
  const int64_t ld = s->ld, N = s->N;
  int64_t bytes = 0;
  bytes += 3 * ld * 8 + 3 * std::max<int64_t>(N - 1, 1) * ld * (int64_t)s->zsize + 3 * ld * 8;  // V, z, U
  bytes += ld * (int64_t)s->rsize;                                                                // F
  bytes += 2 * ld * 8 + 3 * N * ld * 8;                                                           // power iteration
  bytes += 2 * ld * 8 + std::max<int64_t>(N - 1, 1) * ld * 8 + 64 * 8 + 16;                       // act, Vn, tmp, rest, flags
  if (s->precision == EMRKC_PREC_MIXED) bytes += 10 * ld * 4;                                     // V hi/lo, delta, LV, Vn32
  bytes += s->mat_slots * (4 + (s->precision == EMRKC_PREC_MIXED ? 4 : 8)) + (s->ell.n_slices + 1) * 12;
  if (s->d_mask) bytes += s->n;
  return bytes;
}

}  // namespace

extern "C" {

int64_t emrkc_instance_bytes(int64_t n, double nnz_per_row, int model) {
  const int N = emrkc_num_vars(model);
  if (N < 1 || n <= 0) return -1;
  const int64_t ld = (n + 127) / 128 * 128;
  int64_t bytes = 3 * ld * 8 + 3 * std::max(N - 1, 1) * ld * 4 + 3 * ld * 8 + ld * 4;
  bytes += 2 * ld * 8 + 3 * (int64_t)N * ld * 8;
  bytes += 2 * ld * 8 + std::max(N - 1, 1) * ld * 8 + 64 * 8 + 16;
  bytes += 10 * ld * 4;
  bytes += (int64_t)std::ceil(nnz_per_row * (double)ld) * 8 + (ld / 32 + 1) * 12 + n;
  return bytes;
}

int emrkc_batch_create(const emrkc_options* opt, emrkc_batch** out) {
  if (!out) {
    g_batch_create_error = "out is NULL";
    return EMRKC_ERR_ARG;
  }
  *out = nullptr;
  emrkc_options o;
  if (opt) o = *opt;
  else emrkc_default_options(&o);
  if (o.rho_every != EMRKC_RHO_ONCE && o.rho_every != EMRKC_RHO_FIXED) {
    g_batch_create_error = "a batch supports the rho policies ONCE and FIXED";
    return EMRKC_ERR_ARG;
  }
  o.precision = EMRKC_PREC_MIXED;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || o.device < 0 || o.device >= ndev) {
    g_batch_create_error = "no usable CUDA device";
    return EMRKC_ERR_CUDA;
  }
  auto* b = new emrkc_batch();
  b->opt = o;
  b->device = o.device;
  cudaSetDevice(b->device);
  if (o.cuda_stream) {
    b->stream = (cudaStream_t)o.cuda_stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) {
      g_batch_create_error = "stream creation failed";
      delete b;
      return EMRKC_ERR_CUDA;
    }
    b->own_stream = true;
  }
  b->opt.cuda_stream = b->stream;
  if (cudaMalloc(&b->d_ticket, sizeof(unsigned int)) != cudaSuccess || cudaMalloc(&b->d_err, sizeof(int)) != cudaSuccess) {
    g_batch_create_error = "device allocation failed";
    emrkc_batch_destroy(b);
    return EMRKC_ERR_OOM;
  }
  cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
  cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned int), b->stream);
  cudaStreamSynchronize(b->stream);
  *out = b;
  return EMRKC_OK;
}

int emrkc_batch_add(emrkc_batch* b, const emrkc_matrix* mat, const emrkc_tissue* tissue, int model,
                    const emrkc_stimulus* stim, const emrkc_options* inst_opt, int* id_out) {
  if (!b) return EMRKC_ERR_ARG;
  cudaSetDevice(b->device);
  emrkc_options o = b->opt;
  if (inst_opt) {
    o = *inst_opt;
    o.precision = EMRKC_PREC_MIXED;
    o.cuda_stream = b->stream;
    o.device = b->device;
    o.profile = 0;
  }
  if (o.rho_every != EMRKC_RHO_ONCE && o.rho_every != EMRKC_RHO_FIXED)
    return b->fail(EMRKC_ERR_ARG, "a batched instance supports the rho policies ONCE and FIXED");
  emrkc_solver* s = nullptr;
  int rc = emrkc_create(mat, tissue, model, stim, &o, &s);
  if (rc) return b->fail(rc, std::string("instance: ") + emrkc_last_error(nullptr));
  Member mb;
  mb.id = b->next_id++;
  mb.s = s;
  b->members.push_back(mb);
  b->dirty = true;
  ++b->version;
  if (id_out) *id_out = mb.id;
  return EMRKC_OK;
}

int emrkc_batch_remove(emrkc_batch* b, int id) {
  if (!b) return EMRKC_ERR_ARG;
  cudaSetDevice(b->device);
  for (size_t i = 0; i < b->members.size(); ++i) {
    if (b->members[i].id == id) {
      cudaStreamSynchronize(b->stream);
      emrkc_destroy(b->members[i].s);
      b->members.erase(b->members.begin() + (long)i);
      b->dirty = true;
      ++b->version;
      return EMRKC_OK;
    }
  }
  return b->fail(EMRKC_ERR_ARG, "unknown instance id");
}

int emrkc_batch_step(emrkc_batch* b, double dt) {
  if (!b) return EMRKC_ERR_ARG;
  if (!(dt > 0) || !std::isfinite(dt)) return b->fail(EMRKC_ERR_ARG, "dt must be positive and finite");
  cudaSetDevice(b->device);
  if (b->dirty || dt != b->plan_dt) {
    int rc = rebuild(b, dt);
    if (rc) return rc;
  }
  int rc = enqueue_step(b, 0);
  if (rc) return rc;
  for (size_t i = 0; i < b->members.size(); ++i) {
    Member& mb = b->members[i];
    emrkc_solver* s = mb.s;
    s->cur = (s->cur + mb.S) % 3;
    s->t += dt;
    s->steps += 1;
    s->last_s = mb.S;
    s->last_m = mb.M;
    BatchInst& I = b->h_inst[i];
    I.cur = s->cur;
    I.t = s->t;
    I.steps = s->steps;
  }
  return EMRKC_OK;
}

int emrkc_batch_sync(emrkc_batch* b) {
  if (!b) return EMRKC_ERR_ARG;
  cudaSetDevice(b->device);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return b->cuda_fail(e, "stream synchronisation");
  int err = 0;
  e = cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return b->cuda_fail(e, "error flag");
  if (err) return b->fail(EMRKC_ERR_TIMEOUT, "a dependency wait of the persistent kernel gave up");
  for (cudaStream_t cs : {b->h2d_stream, b->d2h_stream}) {
    if (cs && (e = cudaStreamSynchronize(cs)) != cudaSuccess) return b->cuda_fail(e, "copy stream synchronisation");
  }
  b->harvest();
  const size_t ni = b->members.size();
  if (ni > 0 && !b->dirty && b->h_inst.size() == ni) {
    // the device table lists every member: one gather of the flag words and
    // one copy instead of a copy and a synchronisation per instance
    if (b->flagv_cap < ni) {
      if (b->d_flagv) cudaFree(b->d_flagv);
      if (b->h_flagv) cudaFreeHost(b->h_flagv);
      b->d_flagv = nullptr;
      b->h_flagv = nullptr;
      b->flagv_cap = 0;
      if (cudaMalloc(&b->d_flagv, ni * sizeof(int)) != cudaSuccess ||
          cudaMallocHost(&b->h_flagv, ni * sizeof(int)) != cudaSuccess)
        return b->fail(EMRKC_ERR_OOM, "flag array allocation failed");
      b->flagv_cap = ni;
    }
    launch_batch_gather_flags(b->d_inst, (int)ni, b->d_flagv, b->stream);
    if ((e = cudaGetLastError()) != cudaSuccess) return b->cuda_fail(e, "flag gather");
    if ((e = cudaMemcpyAsync(b->h_flagv, b->d_flagv, ni * sizeof(int), cudaMemcpyDeviceToHost, b->stream)) !=
        cudaSuccess)
      return b->cuda_fail(e, "copy of flags");
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return b->cuda_fail(e, "stream synchronisation");
    for (size_t i = 0; i < ni; ++i) {
      if (b->h_flagv[i] == 0) continue;
      // the instance's own check reads, reports and clears its flag word
      Member& mb = b->members[i];
      int rc = emrkc_sync(mb.s);
      if (rc == EMRKC_ERR_NONFINITE) return b->fail(rc, "instance " + std::to_string(mb.id) + ": non-finite V");
      if (rc) return b->fail(rc, mb.s->err);
    }
    return EMRKC_OK;
  }
  for (auto& mb : b->members) {
    int rc = emrkc_sync(mb.s);
    if (rc == EMRKC_ERR_NONFINITE) return b->fail(rc, "instance " + std::to_string(mb.id) + ": non-finite V");
    if (rc) return b->fail(rc, mb.s->err);
  }
  return EMRKC_OK;
}

int emrkc_batch_get_state(emrkc_batch* b, int id, int var, double* host_out, int64_t len) {
  if (!b) return EMRKC_ERR_ARG;
  Member* mb = b->find(id);
  if (!mb) return b->fail(EMRKC_ERR_ARG, "unknown instance id");
  int rc = emrkc_get_state(mb->s, var, host_out, len);
  if (rc) return b->fail(rc, mb->s->err);
  return EMRKC_OK;
}

int emrkc_batch_set_state(emrkc_batch* b, int id, int var, const double* host_in, int64_t len) {
  if (!b) return EMRKC_ERR_ARG;
  Member* mb = b->find(id);
  if (!mb) return b->fail(EMRKC_ERR_ARG, "unknown instance id");
  int rc = emrkc_set_state(mb->s, var, host_in, len);
  if (rc) return b->fail(rc, mb->s->err);
  return EMRKC_OK;
}

int emrkc_batch_get_activation_times(emrkc_batch* b, int id, double* host_out, int64_t n) {
  if (!b) return EMRKC_ERR_ARG;
  Member* mb = b->find(id);
  if (!mb) return b->fail(EMRKC_ERR_ARG, "unknown instance id");
  int rc = emrkc_get_activation_times(mb->s, host_out, n);
  if (rc) return b->fail(rc, mb->s->err);
  return EMRKC_OK;
}

int emrkc_batch_get_info(emrkc_batch* b, int id, emrkc_batch_info* out) {
  if (!b || !out) return EMRKC_ERR_ARG;
  Member* mb = b->find(id);
  if (!mb) return b->fail(EMRKC_ERR_ARG, "unknown instance id");
  out->n = mb->s->n;
  out->N = mb->s->N;
  out->model = mb->s->model;
  out->s = mb->S;
  out->m = mb->M;
  out->t = mb->s->t;
  out->steps = mb->s->steps;
  out->device_bytes = solver_bytes(mb->s);
  return EMRKC_OK;
}

int emrkc_batch_get_stats(emrkc_batch* b, emrkc_batch_stats* out) {
  if (!b || !out) return EMRKC_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->instances = (int)b->members.size();
  for (auto& mb : b->members) {
    out->total_nodes += mb.s->n;
    out->device_bytes += solver_bytes(mb.s);
  }
  out->device_bytes += (int64_t)(b->inst_cap * sizeof(BatchInst) + b->items_cap * 8 + b->done_cap * 4 + 8);
  out->items = b->n_items;
  out->tile = b->tile;
  out->block = b->block;
  out->grid = b->grid;
  out->launches = b->launches;
  out->schedule = b->sched;
  out->threads_per_sm = b->tps;
  return EMRKC_OK;
}

int emrkc_batch_set_config(emrkc_batch* b, int tile, int block) {
  if (!b) return EMRKC_ERR_ARG;
  if (tile < 256 || tile > 8192 || (tile & (tile - 1)) != 0 || (block != 128 && block != 256))
    return b->fail(EMRKC_ERR_ARG, "tile must be a power of two in [256, 8192] and block 128 or 256");
  if (tile != b->tile || block != b->block) {
    b->tile = tile;
    b->block = block;
    b->dirty = true;
  }
  return EMRKC_OK;
}

int emrkc_batch_set_occupancy(emrkc_batch* b, int threads_per_sm) {
  if (!b) return EMRKC_ERR_ARG;
  if (threads_per_sm != 1024 && threads_per_sm != 1536 && threads_per_sm != 2048)
    return b->fail(EMRKC_ERR_ARG, "threads per SM must be 1024, 1536 or 2048");
  if (threads_per_sm != b->tps) {
    b->tps = threads_per_sm;
    b->dirty = true;
  }
  return EMRKC_OK;
}

int emrkc_batch_set_schedule(emrkc_batch* b, int schedule) {
  if (!b) return EMRKC_ERR_ARG;
  if (schedule < 0 || schedule > 2) return b->fail(EMRKC_ERR_ARG, "schedule must be 0, 1 or 2");
  if (schedule != b->sched) {
    b->sched = schedule;
    b->dirty = true;
  }
  return EMRKC_OK;
}

int emrkc_batch_autotune(emrkc_batch* b, double dt, int reps, int* tile_out, int* block_out, double* ms_out) {
  if (!b) return EMRKC_ERR_ARG;
  if (!(dt > 0) || reps < 1) return b->fail(EMRKC_ERR_ARG, "dt > 0 and reps >= 1 required");
  cudaSetDevice(b->device);
  if (b->members.empty()) return b->fail(EMRKC_ERR_STATE, "empty batch");
  int rc = rebuild(b, dt);
  if (rc) return rc;
  for (auto& mb : b->members)
    if (mb.S >= 3) return b->fail(EMRKC_ERR_STATE, "an instance has s >= 3: dry steps would overwrite its state");
  const int tiles[] = {512, 1024, 2048, 4096, 8192};
  const int blocks[] = {128, 256};
  const int scheds[] = {0, 1, 2};
  const int tpss[] = {1024, 1536, 2048};
  const int keep_tile = b->tile, keep_block = b->block, keep_sched = b->sched, keep_tps = b->tps;
  int best_tile = keep_tile, best_block = keep_block, best_sched = keep_sched, best_tps = keep_tps;
  double best = 1e300;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int tp : tpss) {
    for (int sc : scheds) {
      for (int tl : tiles) {
        for (int bl : blocks) {
          b->tile = tl;
          b->block = bl;
          b->sched = sc;
          b->tps = tp;
          if ((rc = rebuild(b, dt))) break;
          if ((rc = enqueue_step(b, 1))) break;
          cudaEventRecord(e0, b->stream);
          for (int r = 0; r < reps && !rc; ++r) rc = enqueue_step(b, 1);
          cudaEventRecord(e1, b->stream);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          const double per = ms / reps;
          if (per < best) {
            best = per;
            best_tile = tl;
            best_block = bl;
            best_sched = sc;
            best_tps = tp;
          }
        }
        if (rc) break;
      }
      if (rc) break;
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tile = best_tile;
  b->block = best_block;
  b->sched = best_sched;
  b->tps = best_tps;
  b->dirty = true;
  if (rc) {
    b->tile = keep_tile;
    b->block = keep_block;
    b->sched = keep_sched;
    b->tps = keep_tps;
    return rc;
  }
  int err = 0;
  cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (err) return b->fail(EMRKC_ERR_TIMEOUT, "a dependency wait gave up during autotuning");
  if (tile_out) *tile_out = best_tile;
  if (block_out) *block_out = best_block;
  if (ms_out) *ms_out = best;
  return EMRKC_OK;
}

int emrkc_batch_set_spin_limit(emrkc_batch* b, int64_t limit) {
  if (!b) return EMRKC_ERR_ARG;
  if (limit < 0) return b->fail(EMRKC_ERR_ARG, "limit must be >= 0");
  b->spin_limit = limit;
  b->drop_graph();
  return EMRKC_OK;
}

namespace {
// Copy streams, events and the per-instance tables of the whole-batch host
// I/O, (re)built when instances joined or left since the last call.
int io_prepare(emrkc_batch* b) {
  cudaError_t e;
  if (!b->h2d_stream) {
    if ((e = cudaStreamCreateWithFlags(&b->h2d_stream, cudaStreamNonBlocking)) != cudaSuccess) {
      b->h2d_stream = nullptr;
      return b->cuda_fail(e, "copy stream creation");
    }
    if ((e = cudaStreamCreateWithFlags(&b->d2h_stream, cudaStreamNonBlocking)) != cudaSuccess) {
      b->d2h_stream = nullptr;
      return b->cuda_fail(e, "copy stream creation");
    }
    cudaEvent_t* evs[] = {&b->ev_mready[0], &b->ev_mready[1], &b->ev_mfree[0], &b->ev_mfree[1],
                          &b->ev_vready[0], &b->ev_vready[1], &b->ev_vfree[0], &b->ev_vfree[1]};
    for (cudaEvent_t* ev : evs)
      if ((e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
        return b->cuda_fail(e, "event creation");
  }
  if (b->io_version == b->version) return EMRKC_OK;
  const size_t ni = b->members.size();
  std::vector<int64_t> off(ni + 1, 0);
  std::vector<uint8_t*> masks(ni, nullptr);
  for (size_t i = 0; i < ni; ++i) {
    emrkc_solver* s = b->members[i].s;
    off[i + 1] = off[i] + s->n;
    if (!s->d_mask) {
      // an instance created without a stimulus gets a zeroed mask buffer
      // (ld bytes: the padding of its last tile is read)
      if ((e = cudaMalloc((void**)&s->d_mask, (size_t)s->ld)) != cudaSuccess) {
        s->d_mask = nullptr;
        return b->fail(EMRKC_ERR_OOM, "device allocation failed");
      }
      if ((e = cudaMemsetAsync(s->d_mask, 0, (size_t)s->ld, b->stream)) != cudaSuccess)
        return b->cuda_fail(e, "mask clear");
      b->dirty = true;  // the plan picks up the new mask pointer
    }
    masks[i] = s->d_mask;
  }
  // the tables are rewritten only after every enqueued use of them
  if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return b->cuda_fail(e, "stream synchronisation");
  if ((e = grow(&b->d_off, &b->off_cap, ni + 1)) != cudaSuccess) return b->fail(EMRKC_ERR_OOM, "batch I/O table");
  if ((e = grow(&b->d_masks, &b->masks_cap, std::max<size_t>(ni, 1))) != cudaSuccess)
    return b->fail(EMRKC_ERR_OOM, "batch I/O table");
  if ((e = cudaMemcpy(b->d_off, off.data(), (ni + 1) * sizeof(int64_t), cudaMemcpyHostToDevice)) != cudaSuccess)
    return b->cuda_fail(e, "batch I/O table upload");
  if (ni && (e = cudaMemcpy(b->d_masks, masks.data(), ni * sizeof(uint8_t*), cudaMemcpyHostToDevice)) != cudaSuccess)
    return b->cuda_fail(e, "batch I/O table upload");
  b->io_total = off[ni];
  b->io_version = b->version;
  return EMRKC_OK;
}
}  // namespace

int emrkc_batch_set_stimulus_async(emrkc_batch* b, const uint8_t* host_masks, int64_t len) {
  if (!b) return EMRKC_ERR_ARG;
  if (!host_masks) return b->fail(EMRKC_ERR_ARG, "null buffer");
  cudaSetDevice(b->device);
  int rc = io_prepare(b);
  if (rc) return rc;
  if (len != b->io_total) return b->fail(EMRKC_ERR_STATE, "buffer length must equal the batch's total node count");
  if (b->members.empty()) return EMRKC_OK;
  cudaError_t e;
  const int k = b->mk;
  if ((e = grow(&b->d_mstage[k], &b->mstage_cap[k], (size_t)len)) != cudaSuccess)
    return b->fail(EMRKC_ERR_OOM, "device allocation failed");
  // the staging buffer is overwritten only after the scatter that read it
  if (b->mfree_rec[k] && (e = cudaStreamWaitEvent(b->h2d_stream, b->ev_mfree[k], 0)) != cudaSuccess)
    return b->cuda_fail(e, "mask copy ordering");
  if ((e = cudaMemcpyAsync(b->d_mstage[k], host_masks, (size_t)len, cudaMemcpyHostToDevice, b->h2d_stream)) !=
      cudaSuccess)
    return b->cuda_fail(e, "mask copy");
  if ((e = cudaEventRecord(b->ev_mready[k], b->h2d_stream)) != cudaSuccess) return b->cuda_fail(e, "mask copy");
  // steps enqueued after this call read the new masks: the scatter runs on
  // the batch's stream after the copy and after every step enqueued so far
  if ((e = cudaStreamWaitEvent(b->stream, b->ev_mready[k], 0)) != cudaSuccess)
    return b->cuda_fail(e, "mask copy ordering");
  launch_batch_scatter_mask(b->d_masks, b->d_off, (int)b->members.size(), b->d_mstage[k], b->stream);
  if ((e = cudaGetLastError()) != cudaSuccess) return b->cuda_fail(e, "mask scatter");
  if ((e = cudaEventRecord(b->ev_mfree[k], b->stream)) != cudaSuccess) return b->cuda_fail(e, "mask scatter");
  b->mfree_rec[k] = true;
  b->mk = k ^ 1;
  return EMRKC_OK;
}

namespace {
// V of every instance into host_out (doubles, or floats when f32) through a
// staging buffer: the join on the batch's stream, the copy on the
// device-to-host stream (the two staging buffers rotate).
int get_V_async(emrkc_batch* b, void* host_out, int64_t len, bool f32) {
  if (!b) return EMRKC_ERR_ARG;
  if (!host_out) return b->fail(EMRKC_ERR_ARG, "null buffer");
  cudaSetDevice(b->device);
  if (b->dirty || b->n_items == 0)
    return b->fail(EMRKC_ERR_STATE, "step the batch once after instances joined or left");
  int rc = io_prepare(b);
  if (rc) return rc;
  if (len != b->io_total) return b->fail(EMRKC_ERR_STATE, "buffer length must equal the batch's total node count");
  cudaError_t e;
  const int k = b->vk;
  if ((e = grow(&b->d_vstage[k], &b->vstage_cap[k], (size_t)len)) != cudaSuccess)
    return b->fail(EMRKC_ERR_OOM, "device allocation failed");
  // the staging buffer is refilled only after its previous copy-out
  if (b->vfree_rec[k] && (e = cudaStreamWaitEvent(b->stream, b->ev_vfree[k], 0)) != cudaSuccess)
    return b->cuda_fail(e, "state copy ordering");
  const int ni = (int)b->members.size();
  if (f32) launch_batch_join_V32(b->d_inst, b->d_off, ni, reinterpret_cast<float*>(b->d_vstage[k]), b->stream);
  else launch_batch_join_V(b->d_inst, b->d_off, ni, b->d_vstage[k], b->stream);
  if ((e = cudaGetLastError()) != cudaSuccess) return b->cuda_fail(e, "state staging");
  if ((e = cudaEventRecord(b->ev_vready[k], b->stream)) != cudaSuccess) return b->cuda_fail(e, "state staging");
  if ((e = cudaStreamWaitEvent(b->d2h_stream, b->ev_vready[k], 0)) != cudaSuccess)
    return b->cuda_fail(e, "state copy ordering");
  const size_t bytes = (size_t)len * (f32 ? sizeof(float) : sizeof(double));
  if ((e = cudaMemcpyAsync(host_out, b->d_vstage[k], bytes, cudaMemcpyDeviceToHost, b->d2h_stream)) != cudaSuccess)
    return b->cuda_fail(e, "state copy");
  if ((e = cudaEventRecord(b->ev_vfree[k], b->d2h_stream)) != cudaSuccess) return b->cuda_fail(e, "state copy");
  b->vfree_rec[k] = true;
  b->vk = k ^ 1;
  return EMRKC_OK;
}
}  // namespace

int emrkc_batch_get_V_async(emrkc_batch* b, double* host_out, int64_t len) {
  return get_V_async(b, host_out, len, false);
}

int emrkc_batch_get_V32_async(emrkc_batch* b, float* host_out, int64_t len) {
  return get_V_async(b, host_out, len, true);
}

int emrkc_batch_ids(const emrkc_batch* b, int* ids_out, int cap) {
  if (!b) return -1;
  const int ni = (int)b->members.size();
  if (ids_out)
    for (int i = 0; i < ni && i < cap; ++i) ids_out[i] = b->members[i].id;
  return ni;
}

int emrkc_batch_set_profile(emrkc_batch* b, int on) {
  if (!b) return EMRKC_ERR_ARG;
  b->profile = on != 0;
  b->drop_graph();
  return EMRKC_OK;
}

int emrkc_batch_get_kernel_time(emrkc_batch* b, double* ms_out, int64_t* launches_out) {
  if (!b) return EMRKC_ERR_ARG;
  cudaSetDevice(b->device);
  b->harvest();
  if (ms_out) *ms_out = b->kernel_ms;
  if (launches_out) *launches_out = b->kernel_launches;
  return EMRKC_OK;
}

const char* emrkc_batch_last_error(const emrkc_batch* b) {
  if (!b) return g_batch_create_error.c_str();
  return b->err.c_str();
}

void emrkc_batch_destroy(emrkc_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& mb : b->members) emrkc_destroy(mb.s);
  b->members.clear();
  b->drop_graph();
  for (cudaStream_t cs : {b->h2d_stream, b->d2h_stream})
    if (cs) cudaStreamSynchronize(cs);
  b->harvest();
  for (auto& pr : b->prof_pool) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  void* ptrs[] = {b->d_inst,       b->d_items,      b->d_ticket,     b->d_done,       b->d_err,
                  b->d_off,        b->d_masks,      b->d_mstage[0],  b->d_mstage[1],  b->d_vstage[0],
                  b->d_vstage[1],  b->d_flagv};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_flagv) cudaFreeHost(b->h_flagv);
  cudaEvent_t evs[] = {b->ev_mready[0], b->ev_mready[1], b->ev_mfree[0], b->ev_mfree[1],
                       b->ev_vready[0], b->ev_vready[1], b->ev_vfree[0], b->ev_vfree[1]};
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  for (cudaStream_t cs : {b->h2d_stream, b->d2h_stream})
    if (cs) cudaStreamDestroy(cs);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"

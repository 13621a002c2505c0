// Batched persistent emRKC step: many independent monodomain instances of
// different sizes, ionic models and stage counts (s, m) advance one step in
// ONE launch.
//
// Work is a phase-major list of items (instance, phase, tile); phase p of an
// instance is stage j = p / m + 1 with inner stage k = p % m + 1 (k = 1: the
// fused stage work, k >= 2: an inner SpMV stage).  Persistent CTAs take items
// in list order from an atomic ticket, one item ahead.  An item of phase p > 0 waits until all
// tiles of phase p - 1 of its instance are done (per-instance counters).
// Because items are taken in order and an item only waits on items earlier in
// the list, every awaited item is already held by a running CTA: the schedule
// cannot deadlock, whatever the grid size.  Waits are still bounded: after
// spin_limit polls the kernel records an error and every CTA returns.
//
// The per-node arithmetic is the mixed-precision stage / inner code of the
// single-instance kernels (stage_node_mixed, inner_node_mixed); see
// batch_stage_rows for when loads may go through L1.
#include <cuda/atomic>

#include "kernels.cuh"

namespace emrkc {

// Which loads may use the non-coherent (L1) path.  L1 holds no line of a
// buffer from an earlier launch, so a load can go through L1 unless this
// launch rewrites a buffer after reading it.  The three state buffers rotate
// with period 3 over the s outer stages: with s <= 2 each is written at most
// once.  The three increment buffers rotate over the m inner stages and are
// written again by every outer stage: they are written at most once only
// when m <= 3 and s = 1 (with m = 1 they are not used).  So L1 serves
// instances with s <= 2 and m = 1, or s = 1 and m <= 3; the others load data
// produced within the launch through L2 (ld.cg).
// Light models (at most 3 z rows): V and z of the thread's next node are
// loaded before the current node's work, one node ahead.
__device__ __forceinline__ bool batch_loads_l2(int s, int m) { return s >= 3 || m >= 4 || (s >= 2 && m >= 2); }

template <class Model, bool HAS_M2, bool CG>
__device__ __forceinline__ void light_rows(const StageArgs& a, const Ell& A, int64_t r0, int64_t r1) {
  constexpr int NZ = Model::NE + Model::NS;
  const float* __restrict__ Zm1 = static_cast<const float*>(a.Zm1);
  const int64_t B = blockDim.x, ld = a.ld;
  int64_t i = r0 + threadIdx.x;
  if (i >= r1) return;
  float Vn = ldm<CG>(a.V32m1 + i);
  float zn[NZ > 0 ? NZ : 1];
#pragma unroll
  for (int k = 0; k < NZ; ++k) zn[k] = ldm<CG>(Zm1 + k * ld + i);
  for (; i < r1; i += B) {
    const float V = Vn;
    float z[NZ > 0 ? NZ : 1];
#pragma unroll
    for (int k = 0; k < NZ; ++k) z[k] = zn[k];
    if (i + B < r1) {
      Vn = ldm<CG>(a.V32m1 + i + B);
#pragma unroll
      for (int k = 0; k < NZ; ++k) zn[k] = ldm<CG>(Zm1 + k * ld + i + B);
    }
    stage_node_mixed_with<Model, HAS_M2, CG>(a, A, i, V, z);
  }
}

template <class Model>
__device__ __forceinline__ void batch_stage_rows(const StageArgs& a, const Ell& A, int64_t r0, int64_t r1, bool has_m2,
                                                 bool cg) {
  if constexpr (Model::NE + Model::NS <= 3) {
    if (has_m2) {
      if (cg) light_rows<Model, true, true>(a, A, r0, r1);
      else light_rows<Model, true, false>(a, A, r0, r1);
    } else {
      light_rows<Model, false, false>(a, A, r0, r1);
    }
    return;
  }
  if (has_m2) {
    if (cg) {
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) stage_node_mixed<Model, true, true>(a, A, i);
    } else {
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) stage_node_mixed<Model, true, false>(a, A, i);
    }
  } else {
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) stage_node_mixed<Model, false, false>(a, A, i);
  }
}

// TPS: resident threads per SM the kernel is compiled for (1024, 1536 or
// 2048: a register budget of 64, 40 or 32 per thread).  The items are bound
// by the latency of their global loads and gain from more resident warps;
// the two smaller budgets spill some registers to local memory (mostly L1
// hits).  The autotuner chooses.
template <int BLOCK, int TPS>
__global__ void __launch_bounds__(BLOCK, TPS / BLOCK) batch_step_kernel(const BatchCtl c) {
  __shared__ unsigned int s_item;
  __shared__ int s_abort;
  // Thread 0 takes the next ticket while the CTA works on the current item
  // (its value is first used one item later, so the atomic's round trip is
  // hidden).  A CTA processes its tickets in increasing order, so the
  // smallest unfinished item is always the current item of some CTA: the
  // in-order argument above still holds.
  unsigned int next_ticket = 0;
  if (threadIdx.x == 0) next_ticket = atomicAdd(c.ticket, 1u);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_abort = 0;
      // stop early if another CTA gave up on a wait
      if (cuda::atomic_ref<int, cuda::thread_scope_device>(*c.err).load(cuda::memory_order_relaxed) != 0) {
        s_item = 0xffffffffu;
      } else {
        s_item = next_ticket;
        next_ticket = atomicAdd(c.ticket, 1u);
      }
    }
    __syncthreads();
    const unsigned int it = s_item;
    if (it >= c.n_items) return;
    const uint64_t d = c.items[it];
    const int ii = (int)(d >> 40);
    const int p = (int)((d >> 32) & 0xffu);
    const int tile = (int)(d & 0xffffffffu);
    BatchInst* I = c.inst + ii;
    if (p > 0) {
      if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(c.done[ii * kBatchMaxPhases + p - 1]);
        const unsigned int need = (unsigned int)I->ntiles;
        long long k = 0;
        while (cnt.load(cuda::memory_order_acquire) < need) {
          if (++k > c.spin_limit) {
            atomicOr(c.err, 2);
            s_abort = 1;
            break;
          }
          __nanosleep(100);
        }
      }
      __syncthreads();
      if (s_abort) return;
    }
    const int s = I->s, m = I->m, cur = I->cur;
    const int j = p / m + 1, k = p % m + 1;
    const int bm1 = (cur + j - 1) % 3, bm2 = (cur + j + 1) % 3, bo = (cur + j) % 3;
    const int64_t r0 = (int64_t)tile * c.tile;
    const int64_t r1 = (r0 + c.tile < I->n) ? r0 + c.tile : I->n;
    // V_n hi for the activation test: its own buffer survives the step while
    // s <= 2 (stage j writes buffer cur + j); a copy is kept for s >= 3
    float* const Vn32 = (s <= 2) ? I->Vhi[cur] : I->Vn32;
    double* const act = c.dry ? nullptr : I->act;
    if (k == 1) {
      StageArgs a;
      a.n = I->n;
      a.ld = I->ld;
      a.Zm1 = I->Z[bm1];
      a.Zm2 = j >= 2 ? I->Z[bm2] : nullptr;
      a.Zout = I->Z[bo];
      a.m = m;
      a.F = I->F;
      a.mask = I->mask;
      const double ts = __dadd_rn(I->t, __dmul_rn(I->o_c[j - 1], I->dt));
      a.f_stim = (I->mask != nullptr && I->t_on <= ts && ts <= I->t_off) ? (float)I->amp : 0.0f;
      a.f_inv_Cm = I->f_inv_Cm;
      a.final_stage = (j == s && m == 1) ? 1 : 0;
      a.Vn32 = Vn32;
      a.act = act;
      a.t_n = I->t;
      a.dt = I->dt;
      a.f_th = I->f_th;
      a.flags = I->flags;
      a.Vn32_copy = (j == 1 && s >= 3) ? I->Vn32 : nullptr;
      a.V32m1 = I->Vhi[bm1];
      a.Vlo_m1 = I->Vlo[bm1];
      a.Vhi_m2 = j >= 2 ? I->Vhi[bm2] : nullptr;
      a.Vlo_m2 = j >= 2 ? I->Vlo[bm2] : nullptr;
      a.V32out = I->Vhi[bo];
      a.Vlo_out = I->Vlo[bo];
      a.D1 = I->D[0];
      a.LV = (m >= 4) ? I->LV : nullptr;
      a.f_nu = I->o_nu[j];
      a.f_kappa = I->o_kappa[j];
      a.f_mudt = I->o_mudt[j];
      a.f_inv_eta = I->f_inv_eta;
      a.f_cm = I->f_cm;
      a.f_mu1 = I->f_mu1;
      a.f_mu1eta = I->f_mu1eta;
      a.f_eta = I->f_eta;
      a.ell_wmax = I->wmax;
      const bool has_m2 = j >= 2;
      const bool cg = batch_loads_l2(s, m);
      switch (I->model) {
        case 0: batch_stage_rows<ModelNone<float>>(a, I->ell, r0, r1, has_m2, cg); break;
        case 1: batch_stage_rows<ModelPassive<float>>(a, I->ell, r0, r1, has_m2, cg); break;
        case 2: batch_stage_rows<ModelHH<float>>(a, I->ell, r0, r1, has_m2, cg); break;
        default: batch_stage_rows<ModelTTP06<float>>(a, I->ell, r0, r1, has_m2, cg); break;
      }
    } else {
      InnerArgs b;
      b.n = I->n;
      b.F = I->F;
      b.last = (k == m) ? 1 : 0;
      b.final_stage = (j == s && k == m) ? 1 : 0;
      b.Vn32 = Vn32;
      b.act = act;
      b.t_n = I->t;
      b.dt = I->dt;
      b.f_th = I->f_th;
      b.flags = I->flags;
      b.d1 = I->D[(k - 2) % 3];
      b.d2 = (k == 2) ? nullptr : I->D[(k - 3) % 3];
      b.dk = I->D[(k - 1) % 3];
      b.LV = I->LV;
      b.lf_src = (m >= 4) ? 0 : (k == 2 ? 1 : 2);
      b.f_inv_mu1eta = I->f_inv_mu1eta;
      b.V32out = I->Vhi[bo];
      b.Vhi1 = I->Vhi[bm1];
      b.Vlo1 = I->Vlo[bm1];
      b.Vhi2 = j >= 2 ? I->Vhi[bm2] : nullptr;
      b.Vlo2 = j >= 2 ? I->Vlo[bm2] : nullptr;
      b.Vlo_out = I->Vlo[bo];
      b.f_nu = I->i_nu[k];
      b.f_kappa = I->i_kappa[k];
      b.f_mueta = I->i_mueta[k];
      b.f_inv_eta = I->f_inv_eta;
      b.f_okappa = I->o_kappa[j];
      b.f_omu_dt = I->o_mudt[j];
      if (batch_loads_l2(s, m)) {
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) inner_node_mixed<true>(b, I->ell, i);
      } else {
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) inner_node_mixed<false>(b, I->ell, i);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(c.done[ii * kBatchMaxPhases + p]);
      const unsigned int prev = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
      // the last tile of the last phase advances the instance: y_{n+1} = g_s
      if (p == I->P - 1 && prev + 1 == (unsigned int)I->ntiles && !c.dry) {
        I->cur = (cur + s) % 3;
        I->t = I->t + I->dt;
        I->steps = I->steps + 1;
      }
    }
  }
}

// ---- Pipelined host I/O of a whole batch ---------------------------------
// Instance k (blockIdx.y) owns entries [off[k], off[k + 1]) of the batch's
// concatenated host arrays.  The join reads V = hi + lo of the instance's
// current state buffer from the device table, which the persistent kernel of
// the preceding step has advanced (same stream).
__global__ void __launch_bounds__(256) batch_join_V_kernel(const BatchInst* __restrict__ inst,
                                                          const int64_t* __restrict__ off, double* __restrict__ out) {
  const BatchInst* I = inst + blockIdx.y;
  const int cur = I->cur;
  const float* __restrict__ hi = I->Vhi[cur];
  const float* __restrict__ lo = I->Vlo[cur];
  const int64_t n = I->n;
  double* __restrict__ o = out + off[blockIdx.y];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (double)hi[i] + (double)lo[i];
}

// The same with V rounded to FP32: the hi part (|lo| is at most half an ulp
// of hi, so hi is V's nearest float).
__global__ void __launch_bounds__(256) batch_join_V32_kernel(const BatchInst* __restrict__ inst,
                                                            const int64_t* __restrict__ off, float* __restrict__ out) {
  const BatchInst* I = inst + blockIdx.y;
  const float* __restrict__ hi = I->Vhi[I->cur];
  const int64_t n = I->n;
  float* __restrict__ o = out + off[blockIdx.y];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = hi[i];
}

__global__ void __launch_bounds__(256) batch_scatter_mask_kernel(uint8_t* const* __restrict__ masks,
                                                                const int64_t* __restrict__ off,
                                                                const uint8_t* __restrict__ src) {
  uint8_t* __restrict__ dst = masks[blockIdx.y];
  const int64_t o = off[blockIdx.y], n = off[blockIdx.y + 1] - o;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[o + i];
}

__global__ void __launch_bounds__(256) batch_gather_flags_kernel(const BatchInst* __restrict__ inst, int ni,
                                                                int* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < ni) out[k] = *inst[k].flags;
}

void launch_batch_gather_flags(const BatchInst* inst, int ni, int* out, cudaStream_t st) {
  if (ni <= 0) return;
  batch_gather_flags_kernel<<<(unsigned)((ni + 255) / 256), 256, 0, st>>>(inst, ni, out);
}

void launch_batch_join_V(const BatchInst* inst, const int64_t* off, int ni, double* out, cudaStream_t st) {
  if (ni <= 0) return;
  batch_join_V_kernel<<<dim3(128, (unsigned)ni), 256, 0, st>>>(inst, off, out);
}

void launch_batch_join_V32(const BatchInst* inst, const int64_t* off, int ni, float* out, cudaStream_t st) {
  if (ni <= 0) return;
  batch_join_V32_kernel<<<dim3(128, (unsigned)ni), 256, 0, st>>>(inst, off, out);
}

void launch_batch_scatter_mask(uint8_t* const* masks, const int64_t* off, int ni, const uint8_t* src,
                               cudaStream_t st) {
  if (ni <= 0) return;
  batch_scatter_mask_kernel<<<dim3(64, (unsigned)ni), 256, 0, st>>>(masks, off, src);
}

namespace {
template <int BLOCK>
void launch_tps(const BatchCtl& c, int grid, int tps, cudaStream_t st) {
  if (tps == 2048) batch_step_kernel<BLOCK, 2048><<<grid, BLOCK, 0, st>>>(c);
  else if (tps == 1536) batch_step_kernel<BLOCK, 1536><<<grid, BLOCK, 0, st>>>(c);
  else batch_step_kernel<BLOCK, 1024><<<grid, BLOCK, 0, st>>>(c);
}
template <int BLOCK>
int blocks_tps(int tps) {
  int nb = 0;
  if (tps == 2048) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_step_kernel<BLOCK, 2048>, BLOCK, 0);
  else if (tps == 1536) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_step_kernel<BLOCK, 1536>, BLOCK, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_step_kernel<BLOCK, 1024>, BLOCK, 0);
  return nb;
}
}  // namespace

void launch_batch_step(const BatchCtl& c, int grid, int block, int tps, cudaStream_t st) {
  if (block == 256) launch_tps<256>(c, grid, tps, st);
  else launch_tps<128>(c, grid, tps, st);
}

int batch_blocks_per_sm(int block, int tps) {
  return block == 256 ? blocks_tps<256>(tps) : blocks_tps<128>(tps);
}

}  // namespace emrkc

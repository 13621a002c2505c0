// Allocation-free variant of the f_F power iteration (emrkc_estimate_rho_F_noalloc).
//
// Callers that cannot allocate device memory while they run -- a host that
// has handed every byte of the GPU to its own allocator, or a time-critical
// loop that must not call cudaMalloc (it may synchronise the device) -- still
// need the reduction scratch of the power iteration: per-block partial sums,
// a ticket counter and result slots.  Here that scratch is one file-scope
// device array of fixed size, which every GPU that loads the library holds
// until the process exits.  The kernels are the same templates as the
// solver's own power iteration, so results are identical.
#include <cstdio>
#include <mutex>

#include "kernels.cuh"

namespace emrkc {

// Layout: [0, 8 KiB) partial sums (one per block, at most kReduceMaxBlocks),
// then 8 result slots, then the ticket counter.
constexpr size_t kNoAllocPartialBytes = (size_t)kReduceMaxBlocks * sizeof(double);
constexpr size_t kNoAllocResultOffset = kNoAllocPartialBytes;
constexpr size_t kNoAllocTicketOffset = kNoAllocResultOffset + 8 * sizeof(double);
constexpr size_t kNoAllocBytes = kNoAllocTicketOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
struct DeviceScratch {
  bool ready = false;
  ReduceScratch rs{};
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

static __global__ void __launch_bounds__(kReduceBlock) noalloc_sumsq_kernel(int64_t count, const double* x,
                                                                            const ReduceScratch rs, int slot) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    acc += v * v;
  }
  reduce_finish(acc, rs, slot);
}
}  // namespace

// Device address of the static scratch on the current device (which must be
// `device`).  The first call per device looks the symbol up with
// cudaGetSymbolAddress and zeroes the ticket counter; later calls reuse the
// address, which stays valid while the device's primary context lives (a
// cudaDeviceReset while the library is in use would leave it stale).
// The reductions launch at most kReduceMaxBlocks blocks (grid-stride loops
// cover any n), one partial sum each, which is what the array holds.
static_assert(kNoAllocPartialBytes >= (size_t)kReduceMaxBlocks * sizeof(double), "one partial per block");
int noalloc_scratch(int device, cudaStream_t st, ReduceScratch* out, const char** why) {
  if (device < 0 || device >= kMaxDevices) {
    *why = "device ordinal beyond the allocation-free scratch table";
    return 1;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  DeviceScratch& d = g_scratch[device];
  if (!d.ready) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      *why = "cudaGetSymbolAddress of the static scratch failed";
      return 2;
    }
    ReduceScratch rs;
    rs.partials = static_cast<double*>(ptr);
    rs.result = reinterpret_cast<double*>(static_cast<unsigned char*>(ptr) + kNoAllocResultOffset);
    rs.ticket = reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(ptr) + kNoAllocTicketOffset);
    // the ticket must start at zero; the reduction's last block resets it
    e = cudaMemsetAsync(rs.ticket, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      *why = "clearing the static scratch failed";
      return 2;
    }
    d.rs = rs;
    d.ready = true;
  }
  *out = d.rs;
  return 0;
}

void noalloc_sumsq(int64_t count, const double* x, const ReduceScratch& rs, int slot, cudaStream_t st) {
  noalloc_sumsq_kernel<<<reduce_grid(count), kReduceBlock, 0, st>>>(count, x, rs, slot);
}

void noalloc_power_F(const PowerFArgs& a, const Ell& A, bool mixed, const ReduceScratch& rs, cudaStream_t st) {
  if (mixed) powerF_kernel<true><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, A, rs);
  else powerF_kernel<false><<<reduce_grid(a.n), kReduceBlock, 0, st>>>(a, A, rs);
}

}  // namespace emrkc

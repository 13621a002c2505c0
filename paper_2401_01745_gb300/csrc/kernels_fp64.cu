// FP64 instantiations of the emRKC kernels, plus precision-independent
// helper kernels (start vectors, fills, plain sums of squares).
#include "kernels.cuh"

namespace emrkc {

bool get_kernels_fp64(int model, KernelSet* ks) {
  switch (model) {
    case 0: Kernels<ModelNone<double>, ModelNone<double>, double, double, false>::fill(ks, model); return true;
    case 1: Kernels<ModelPassive<double>, ModelPassive<double>, double, double, false>::fill(ks, model); return true;
    case 2: Kernels<ModelHH<double>, ModelHH<double>, double, double, false>::fill(ks, model); return true;
    case 3: Kernels<ModelTTP06<double>, ModelTTP06<double>, double, double, false>::fill(ks, model); return true;
    default: return false;
  }
}

__global__ void __launch_bounds__(kReduceBlock) sumsq_kernel(int64_t count, const double* x, const ReduceScratch rs,
                                                             int slot) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    acc += v * v;
  }
  reduce_finish(acc, rs, slot);
}

void launch_sumsq(int64_t count, const double* x, const ReduceScratch& rs, int slot, cudaStream_t st) {
  sumsq_kernel<<<reduce_grid(count), kReduceBlock, 0, st>>>(count, x, rs, slot);
}

// SplitMix64 (Steele, Lea, Flood 2014): golden-ratio increment, then two
// xor-shift-multiply rounds and a final xor-shift.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Start vector of the power iteration: v[r*ld + i] = u01(splitmix64(key ^ (r*n + i))) - 0.5
// for i < n, 0 in the padding.
__global__ void start_vector_kernel(uint64_t key, int64_t n, int64_t ld, int rows, double* v) {
  const int64_t total = (int64_t)rows * ld;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / ld, i = idx - r * ld;
    if (i >= n) {
      v[idx] = 0.0;
    } else {
      const uint64_t k = (uint64_t)(r * n + i);
      v[idx] = (double)(splitmix64(key ^ k) >> 11) * 0x1.0p-53 - 0.5;
    }
  }
}

void launch_start_vector(uint64_t key, int64_t n, int64_t ld, int rows, double* v, cudaStream_t st) {
  const int64_t total = (int64_t)rows * ld;
  if (total == 0) return;
  unsigned g = blocks_for(total, 256);
  if (g > 8192) g = 8192;
  start_vector_kernel<<<g, 256, 0, st>>>(key, n, ld, rows, v);
}

__global__ void fill_kernel(double* x, int64_t count, double value) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = value;
}

void launch_fill(double* x, int64_t count, double value, cudaStream_t st) {
  if (count == 0) return;
  unsigned g = blocks_for(count, 256);
  if (g > 8192) g = 8192;
  fill_kernel<<<g, 256, 0, st>>>(x, count, value);
}

// Set rows 0..rows-1 of an SoA block (element size zsize = 4 or 8) to per-row values.
__global__ void fill_rows_kernel(void* z, int zsize, int64_t n, int64_t ld, int rows, const double* values) {
  const int64_t total = (int64_t)rows * ld;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / ld, i = idx - r * ld;
    const double val = (i < n) ? values[r] : 0.0;
    if (zsize == 8) static_cast<double*>(z)[idx] = val;
    else static_cast<float*>(z)[idx] = (float)val;
  }
}

void launch_fill_rows(void* z, int zsize, int64_t n, int64_t ld, int rows, const double* values, cudaStream_t st) {
  const int64_t total = (int64_t)rows * ld;
  if (total == 0) return;
  unsigned g = blocks_for(total, 256);
  if (g > 8192) g = 8192;
  fill_rows_kernel<<<g, 256, 0, st>>>(z, zsize, n, ld, rows, values);
}

__global__ void ff_split_kernel(const double* v, float* hi, float* lo, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[i];
    const float h = (float)x;
    hi[i] = h;
    lo[i] = (float)(x - (double)h);
  }
}

__global__ void ff_join_kernel(const float* hi, const float* lo, double* v, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (double)hi[i] + (double)lo[i];
}

void launch_ff_split(const double* v, float* hi, float* lo, int64_t count, cudaStream_t st) {
  if (count == 0) return;
  unsigned g = blocks_for(count, 256);
  if (g > 8192) g = 8192;
  ff_split_kernel<<<g, 256, 0, st>>>(v, hi, lo, count);
}

void launch_ff_join(const float* hi, const float* lo, double* v, int64_t count, cudaStream_t st) {
  if (count == 0) return;
  unsigned g = blocks_for(count, 256);
  if (g > 8192) g = 8192;
  ff_join_kernel<<<g, 256, 0, st>>>(hi, lo, v, count);
}

}  // namespace emrkc

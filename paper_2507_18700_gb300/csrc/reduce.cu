// FP64 reductions of the VMC estimators (Sec. III): energy mean and variance,
// per-sample gradient weights, and the sum of per-block partial gradients.
#include "kernels.h"

namespace nqs {

// stats = [mean E_loc, mean(E_loc^2) - mean^2, M]; one block, fixed order.
__global__ void energy_stats_kernel(const float* __restrict__ eloc, int64_t B, double* stats) {
  __shared__ double s1[1024], s2[1024];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
    const double e = (double)eloc[i];
    a += e;
    b += e * e;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      s1[threadIdx.x] += s1[threadIdx.x + off];
      s2[threadIdx.x] += s2[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double M = (double)B;
    const double mean = s1[0] / M;
    stats[0] = mean;
    stats[1] = s2[0] / M - mean * mean;
    stats[2] = M;
  }
}

// sums = [sum E_loc, sum E_loc^2, B]: one rank's share of the statistics of
// a data-parallel step, in the fixed order of energy_stats_kernel.
__global__ void energy_sums_kernel(const float* __restrict__ eloc, int64_t B, double* sums) {
  __shared__ double s1[1024], s2[1024];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
    const double e = (double)eloc[i];
    a += e;
    b += e * e;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      s1[threadIdx.x] += s1[threadIdx.x + off];
      s2[threadIdx.x] += s2[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[0] = s1[0];
    sums[1] = s2[0];
    sums[2] = (double)B;
  }
}

// stats = [mean, mean(E^2) - mean^2, M] from sums = [sum E, sum E^2, M] of all ranks.
__global__ void stats_from_sums_kernel(const double* __restrict__ sums, double* stats) {
  const double M = sums[2];
  const double mean = sums[0] / M;
  stats[0] = mean;
  stats[1] = sums[1] / M - mean * mean;
  stats[2] = M;
}

// w_b = 2 (E_loc,b - mean) / M
__global__ void vmc_weights_kernel(const float* __restrict__ eloc, const double* __restrict__ stats,
                                   int64_t B, float* __restrict__ w) {
  const double mean = stats[0], M = stats[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (float)(2.0 * ((double)eloc[i] - mean) / M);
}

// grad[p] = sum_r partial[r][p] in a fixed order, written as T (float, or
// double for gradients that are summed over ranks).  The accumulators are
// unevaluated pairs hi + lo of FP32 words updated with Knuth's two-sum (s =
// hi + x exactly equals s_rounded + e), so that each keeps about 48
// significant bits, like an FP64 sum of FP32 terms, while running on the FP32
// pipe (GB300's FP64 rate is a small fraction of it: with FP64 adds and
// conversions this reduction took ~44 us for 304 rows x 34 k columns).
// A block sums 32 columns: 8 row groups (r = g mod 8) per column, each with 4
// independent accumulators, then the 8 group sums in a fixed tree in FP64.
struct Fsum {
  float hi, lo;
};
__device__ __forceinline__ void fsum_add(Fsum& a, float x) {
  const float s = a.hi + x;
  const float bp = s - a.hi;
  const float e = (a.hi - (s - bp)) + (x - bp);   // two-sum: a.hi + x = s + e exactly
  a.hi = s;
  a.lo += e;
}
__device__ __forceinline__ double fsum_value(const Fsum& a) { return (double)a.hi + (double)a.lo; }

template <typename T>
__global__ void __launch_bounds__(256) reduce_partials_kernel(const float* __restrict__ partial, int rows, int P,
                                                              int64_t ld, T* __restrict__ grad) {
  __shared__ double red[8][33];
  const int col = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + col;
  Fsum a0{0.0f, 0.0f}, a1{0.0f, 0.0f}, a2{0.0f, 0.0f}, a3{0.0f, 0.0f};
  if (p < P) {
    int r = g;
    for (; r + 24 < rows; r += 32) {
      fsum_add(a0, partial[(size_t)r * ld + p]);
      fsum_add(a1, partial[(size_t)(r + 8) * ld + p]);
      fsum_add(a2, partial[(size_t)(r + 16) * ld + p]);
      fsum_add(a3, partial[(size_t)(r + 24) * ld + p]);
    }
    for (; r < rows; r += 8) fsum_add(a0, partial[(size_t)r * ld + p]);
  }
  red[g][col] = (fsum_value(a0) + fsum_value(a1)) + (fsum_value(a2) + fsum_value(a3));
  __syncthreads();
  if (g == 0 && p < P) {
    const double s = ((red[0][col] + red[1][col]) + (red[2][col] + red[3][col])) +
                     ((red[4][col] + red[5][col]) + (red[6][col] + red[7][col]));
    grad[p] = (T)s;
  }
}

cudaError_t energy_stats(const float* eloc, int64_t B, double* stats, cudaStream_t st) {
  energy_stats_kernel<<<1, 1024, 0, st>>>(eloc, B, stats);
  return cudaGetLastError();
}

cudaError_t energy_sums(const float* eloc, int64_t B, double* sums, cudaStream_t st) {
  energy_sums_kernel<<<1, 1024, 0, st>>>(eloc, B, sums);
  return cudaGetLastError();
}

cudaError_t stats_from_sums(const double* sums, double* stats, cudaStream_t st) {
  stats_from_sums_kernel<<<1, 1, 0, st>>>(sums, stats);
  return cudaGetLastError();
}

cudaError_t vmc_weights(const float* eloc, const double* stats, int64_t B, float* w, cudaStream_t st) {
  int64_t blocks = (B + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  vmc_weights_kernel<<<(unsigned)blocks, 256, 0, st>>>(eloc, stats, B, w);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t reduce_cols(const float* partial, int rows, int ncols, int64_t ld, T* grad, cudaStream_t st) {
  const int blocks = (ncols + 31) / 32;
  if (blocks < 1) return cudaSuccess;
  reduce_partials_kernel<T><<<blocks, 256, 0, st>>>(partial, rows, ncols, ld, grad);
  return cudaGetLastError();
}

cudaError_t reduce_partials_cols(const float* partial, int rows, int ncols, int64_t ld, float* grad,
                                 cudaStream_t st) {
  return reduce_cols(partial, rows, ncols, ld, grad, st);
}
cudaError_t reduce_partials_cols(const float* partial, int rows, int ncols, int64_t ld, double* grad,
                                 cudaStream_t st) {
  return reduce_cols(partial, rows, ncols, ld, grad, st);
}

// acc[p] += grad of the partial rows (FP64): the checkpointed gradient sums
// its segments' partial rows this way.
__global__ void add_f64_kernel(const double* __restrict__ x, double* __restrict__ acc, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc[i] += x[i];
}
__global__ void f64_to_f32_kernel(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

cudaError_t reduce_partials(const float* partial, int rows, int P, float* grad, cudaStream_t st) {
  return reduce_partials_cols(partial, rows, P, P, grad, st);
}

cudaError_t reduce_partials_acc(const float* partial, int rows, int P, double* acc, cudaStream_t st) {
  // the segment's sum goes to the P doubles after acc, then is added in
  double* seg = acc + P;
  cudaError_t e = reduce_partials_cols(partial, rows, P, P, seg, st);
  if (e != cudaSuccess) return e;
  const int blocks = (P + 255) / 256 < 1024 ? (P + 255) / 256 : 1024;
  add_f64_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(seg, acc, P);
  return cudaGetLastError();
}

cudaError_t f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  f64_to_f32_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}
cudaError_t reduce_partials(const float* partial, int rows, int P, double* grad, cudaStream_t st) {
  return reduce_partials_cols(partial, rows, P, P, grad, st);
}

}  // namespace nqs

// Training-loop kernels around the VMC step (Sec. II B, Sec. III and the
// hyperparameter appendix): the Adam update with the paper's learning-rate
// schedules, a device step counter shared with the sampler (so a captured CUDA
// graph of whole steps draws fresh samples and advances the schedule on every
// replay), a per-step log of the energy statistics, and the FP64 accumulation
// of the final-evaluation mode.
#include "kernels.h"

namespace nqs {

namespace {

// Learning rate at training step t (0-based), Tab. III: constant; a step from
// lr0 to lr1 at t_switch (1D Adaptive: 5e-3 then 5e-4 from step 25,000);
// lr0 / (1 + (t - t_switch) / decay) from t_switch on and lr0 before it (2D
// Static with t_switch = 0; 2D Adaptive with t_switch = 100,000, the reading
// of its garbled formula in which the floor term switches the decay on for
// the second half of training).
__device__ __forceinline__ double lr_at(const LrSchedule& s, int64_t t) {
  if (s.kind == 1) return t < s.t_switch ? s.lr0 : s.lr1;
  if (s.kind == 2) return t < s.t_switch ? s.lr0 : s.lr0 / (1.0 + (double)(t - s.t_switch) / s.decay);
  return s.lr0;
}

// Adam (Kingma and Ba 2014, Algorithm 1) on the flat parameters: with the
// update number k = t + 1,
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   theta -= lr(t) * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps).
// Moments and parameters stay FP32; the bias corrections and the step size
// are formed in FP64 once per thread.
template <typename G>
__global__ void adam_kernel(const G* __restrict__ grad, float* __restrict__ params, float* __restrict__ m,
                            float* __restrict__ v, int64_t P, AdamArgs a, const uint64_t* __restrict__ t_dev) {
  const int64_t t = (int64_t)(t_dev ? *t_dev : a.t);
  const double k = (double)(t + 1);
  const double c1 = 1.0 - pow(a.beta1, k), c2 = 1.0 - pow(a.beta2, k);
  const float lr = (float)lr_at(a.sched, t);
  // 1 - beta formed in FP64: 1 - float(0.999) would be off by 1.3e-5 relative
  const float b1 = (float)a.beta1, b2 = (float)a.beta2, eps = (float)a.eps;
  const float omb1 = (float)(1.0 - a.beta1), omb2 = (float)(1.0 - a.beta2);
  const float ic1 = (float)(1.0 / c1), ic2 = (float)(1.0 / c2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = (float)grad[i];
    const float mi = fmaf(b1, m[i], omb1 * g);
    const float vi = fmaf(b2, v[i], omb2 * g * g);
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi * ic1) / (sqrtf(vi * ic2) + eps);
  }
}

__global__ void step_incr_kernel(uint64_t* t_dev) { *t_dev += 1; }

// log[t mod cap] = (t, stats[0], stats[1], stats[2]) with t the device step.
__global__ void record_stats_kernel(const double* __restrict__ stats, double* __restrict__ log, int64_t cap,
                                    const uint64_t* __restrict__ t_dev) {
  const uint64_t t = *t_dev;
  double* row = log + 4 * (int64_t)(t % (uint64_t)cap);
  row[0] = (double)t;
  row[1] = stats[0];
  row[2] = stats[1];
  row[3] = stats[2];
}

// sums += [sum E, sum E^2, B] of one chunk (fixed order within the chunk).
__global__ void energy_sums_acc_kernel(const float* __restrict__ eloc, int64_t B, double* sums) {
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
    sums[0] += s1[0];
    sums[1] += s2[0];
    sums[2] += (double)B;
  }
}

// stats = [mean, variance (1/M), M, standard error of the mean sqrt(var / M),
// error of the variance var sqrt(2 / (M - 1)) for Gaussian local energies
// (Tab. I caption)].
__global__ void eval_stats_kernel(const double* __restrict__ sums, double* stats) {
  const double M = sums[2];
  const double mean = sums[0] / M;
  const double var = sums[1] / M - mean * mean;
  stats[0] = mean;
  stats[1] = var;
  stats[2] = M;
  stats[3] = sqrt(var / M);
  stats[4] = M > 1.0 ? var * sqrt(2.0 / (M - 1.0)) : 0.0;
}

__global__ void status_merge_kernel(const WsHeader* from, WsHeader* into) {
  if (from->status != 0) atomicCAS(&into->status, 0, from->status);
}

}  // namespace

cudaError_t status_merge(const WsHeader* from, WsHeader* into, cudaStream_t st) {
  status_merge_kernel<<<1, 1, 0, st>>>(from, into);
  return cudaGetLastError();
}

cudaError_t adam_update(const float* grad32, const double* grad64, float* params, float* m, float* v, int64_t P,
                        const AdamArgs& a, uint64_t* t_dev, cudaStream_t st) {
  int64_t blocks = (P + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  if (grad64)
    adam_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(grad64, params, m, v, P, a, t_dev);
  else
    adam_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(grad32, params, m, v, P, a, t_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !t_dev) return e;
  step_incr_kernel<<<1, 1, 0, st>>>(t_dev);
  return cudaGetLastError();
}

cudaError_t step_increment(uint64_t* t_dev, cudaStream_t st) {
  step_incr_kernel<<<1, 1, 0, st>>>(t_dev);
  return cudaGetLastError();
}

cudaError_t record_stats(const double* stats, double* log, int64_t cap, const uint64_t* t_dev, cudaStream_t st) {
  record_stats_kernel<<<1, 1, 0, st>>>(stats, log, cap, t_dev);
  return cudaGetLastError();
}

cudaError_t energy_sums_acc(const float* eloc, int64_t B, double* sums, cudaStream_t st) {
  energy_sums_acc_kernel<<<1, 1024, 0, st>>>(eloc, B, sums);
  return cudaGetLastError();
}

cudaError_t eval_stats(const double* sums, double* stats, cudaStream_t st) {
  eval_stats_kernel<<<1, 1, 0, st>>>(sums, stats);
  return cudaGetLastError();
}

}  // namespace nqs

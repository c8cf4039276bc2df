// Grouped VMC step for a batch of 1D GRU replicas of uneven hidden size,
// field and batch (the Adaptive schedule's model family, Sec. II B): every
// phase of the step -- weight packing, sampling, cached-path readout,
// prefix-cached TFIM chains, local energies, FP64 statistics, the reverse
// sweep and the partial-gradient reduction -- is one launch over all
// replicas.  Blocks of the per-replica phases pick their replica from
// prefix tables; the chain launch is persistent: each CTA starts on the
// replica its share of the work points to and then drains the other
// replicas' queues.  The replica table is a kernel argument (no device copy),
// so the whole step can be captured in a CUDA graph; with a device-side step
// counter every replay draws fresh samples.
#include <algorithm>

#include "gru1d_body.cuh"

namespace nqs {

namespace {

constexpr int kMaxRep = NQS_MAX_REPLICAS;
constexpr int kFwdNT = 128, kChainNT = 256, kBpttNT = 256;

struct Rep {
  int d, N, P;
  int64_t B;
  uint64_t seed;
  float J, Gamma;
  const float* params;
  float* img;
  uint8_t* sigma;
  float* logpsi;
  float* hcache;
  float* eloc;
  float* grad;
  double* stats;
  float* dlog;
  float* delta;
  float* partial;
  float* w;
  unsigned long long* counter;
};

struct RepTable {
  int R;
  uint64_t step;
  const uint64_t* step_dev;       // nullable: device-side step counter
  int fwd_begin[kMaxRep + 1];     // block ranges of the per-replica launches
  int bptt_begin[kMaxRep + 1];
  int chain_begin[kMaxRep + 1];   // CTA ranges of the persistent chain launch
  Rep r[kMaxRep];
};

__device__ __forceinline__ int find_rep(const int* begin, int R, int blk) {
  int r = 0;
  while (r + 1 < R && blk >= begin[r + 1]) ++r;
  return r;
}

// Tile geometry of the grouped launches (uniform thread counts).
template <int D> struct G1 {
  static constexpr int F_RPT = D >= 64 ? 2 : 4;
  static constexpr int C_RPT = D >= 128 ? 2 : 4;
  static constexpr int B_RPT = 2;
  static constexpr bool WSMEM = D <= 64;
  static constexpr int TU = Geo<D>::TU;
  static constexpr int F_R = (kFwdNT / TU) * F_RPT;
  static constexpr int C_R = (kChainNT / TU) * C_RPT;
  static constexpr int B_NRG = kBpttNT / TU;
  static constexpr int B_R = B_NRG * B_RPT;
  static constexpr size_t F_SMEM = sizeof(float) * (img1_small(D) + (WSMEM ? 3 * D * D : 0) + 2 * F_R * Geo<D>::DP);
  static constexpr size_t C_SMEM = sizeof(float) * (img1_small(D) + (WSMEM ? 3 * D * D : 0) + 2 * C_R * Geo<D>::DP);
  static constexpr size_t B_SMEM = sizeof(float) * (img1_small(D) + (WSMEM ? 6 * D * D : 0) + B_R * Geo<D>::DP +
                                                    B_R * (3 * D + 4) + B_NRG * (kSmallGrads * D + 2));
};

__global__ void grouped_pack_kernel(RepTable t) {
  const Rep& r = t.r[blockIdx.y];
  const int D = r.d;
  const Off1 o = off1(D);
  const int small = img1_small(D), total = img1_floats(D), D3 = 3 * D;
  const float* p = r.params;
  for (int q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < total; q0 += gridDim.x * blockDim.x) {
    float v = 0.0f;
    const int q = q0;
    if (q < 6 * D) {
      const int s = q / D3, g = (q % D3) / D, u = q % D;
      v = g == 0 ? p[o.Wg + u * (D + 2) + D + s] : g == 1 ? p[o.Wr + u * (D + 2) + D + s] : p[o.Win + u * 2 + s];
    } else if (q < 10 * D) {
      v = p[o.bg + (q - 6 * D)];
    } else if (q < 12 * D) {
      v = p[o.U + (q - 10 * D)];
    } else if (q < small) {
      v = (q - 12 * D) < 2 ? p[o.c + q - 12 * D] : 0.0f;
    } else {
      int w = q - small, k, g, u;
      if (w < D3 * D) {
        k = w / D3; g = (w % D3) / D; u = w % D;
      } else {
        w -= D3 * D;
        g = w / (D * D); u = (w / D) % D; k = w % D;
      }
      v = g == 0 ? p[o.Wg + u * (D + 2) + k] : g == 1 ? p[o.Wr + u * (D + 2) + k] : p[o.Wh + u * D + k];
    }
    r.img[q0] = v;
  }
}

__global__ void __launch_bounds__(kFwdNT) grouped_sample_kernel(RepTable t) {
  const int ri = find_rep(t.fwd_begin, t.R, blockIdx.x);
  const Rep& r = t.r[ri];
  Fwd1Args a{};
  a.B = r.B;
  a.N = r.N;
  a.sigma_out = r.sigma;
  a.seed = r.seed;
  a.step = t.step_dev ? *t.step_dev : t.step;
  a.logpsi = r.logpsi;
  a.hcache = r.hcache;
  const int blk = blockIdx.x - t.fwd_begin[ri];
  switch (r.d) {
    case 16: gru1d_forward_body<16, G1<16>::F_RPT, kFwdNT, true, G1<16>::WSMEM>(r.img, a, blk); break;
    case 32: gru1d_forward_body<32, G1<32>::F_RPT, kFwdNT, true, G1<32>::WSMEM>(r.img, a, blk); break;
    case 64: gru1d_forward_body<64, G1<64>::F_RPT, kFwdNT, true, G1<64>::WSMEM>(r.img, a, blk); break;
    case 128: gru1d_forward_body<128, G1<128>::F_RPT, kFwdNT, true, G1<128>::WSMEM>(r.img, a, blk); break;
  }
}

// Logit differences of every cached state (one warp per (sample, site)).
__global__ void grouped_readout_kernel(RepTable t) {
  const Rep& r = t.r[blockIdx.y];
  dlog_rows(r.img, r.hcache, r.dlog, r.B * r.N, r.d, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
            ((int64_t)gridDim.x * blockDim.x) >> 5);
}

__global__ void __launch_bounds__(kChainNT) grouped_chains_kernel(RepTable t) {
  const int first = find_rep(t.chain_begin, t.R, blockIdx.x);
  for (int k = 0; k < t.R; ++k) {
    const Rep& r = t.r[(first + k) % t.R];
    Chain1Args a{};
    a.B = r.B;
    a.N = r.N;
    a.sigma = r.sigma;
    a.hcache = r.hcache;
    a.dlog = r.dlog;
    a.delta = r.delta;
    a.counter = r.counter;
    switch (r.d) {
      case 16: tfim_chains1d_body<16, G1<16>::C_RPT, kChainNT, G1<16>::WSMEM>(r.img, a); break;
      case 32: tfim_chains1d_body<32, G1<32>::C_RPT, kChainNT, G1<32>::WSMEM>(r.img, a); break;
      case 64: tfim_chains1d_body<64, G1<64>::C_RPT, kChainNT, G1<64>::WSMEM>(r.img, a); break;
      case 128: tfim_chains1d_body<128, G1<128>::C_RPT, kChainNT, G1<128>::WSMEM>(r.img, a); break;
    }
    __syncthreads();   // shared memory is reloaded for the next replica
  }
}

// Local energies (one warp per sample), then the statistics and the
// per-sample gradient weights of each replica (one block per replica).
__global__ void grouped_eloc_kernel(RepTable t) {
  const Rep& r = t.r[blockIdx.y];
  const int lane = threadIdx.x & 31, N = r.N;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < r.B;
       b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float diag = 0.0f, off = 0.0f;
    for (int n = lane; n < N; n += 32) {
      const int s = r.sigma[b * N + n] ? 1 : 0;
      if (n + 1 < N) diag += (s == (r.sigma[b * N + n + 1] ? 1 : 0)) ? 1.0f : -1.0f;
      float dl;
      if (n + 1 < N) {
        dl = r.delta[b * N + n];
      } else {
        const float d = r.dlog[b * N + n];
        dl = 0.5f * (s == 0 ? -d : d);
      }
      off += expf(dl);
    }
    diag = group_sum<32>(diag);
    off = group_sum<32>(off);
    if (lane == 0) r.eloc[b] = -r.J * diag - r.Gamma * off;
  }
}

__global__ void grouped_stats_kernel(RepTable t) {
  __shared__ double s1[1024], s2[1024];
  const Rep& r = t.r[blockIdx.x];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < r.B; i += blockDim.x) {
    const double e = (double)r.eloc[i];
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
  const double M = (double)r.B, mean = s1[0] / M;
  if (threadIdx.x == 0) {
    r.stats[0] = mean;
    r.stats[1] = s2[0] / M - mean * mean;
    r.stats[2] = M;
  }
  for (int64_t i = threadIdx.x; i < r.B; i += blockDim.x) r.w[i] = (float)(2.0 * ((double)r.eloc[i] - mean) / M);
}

__global__ void __launch_bounds__(kBpttNT) grouped_bptt_kernel(RepTable t) {
  const int ri = find_rep(t.bptt_begin, t.R, blockIdx.x);
  const Rep& r = t.r[ri];
  Bptt1Args a{};
  a.B = r.B;
  a.N = r.N;
  a.P = r.P;
  a.sigma = r.sigma;
  a.hcache = r.hcache;
  a.weights = r.w;
  a.partial = r.partial;
  const int blk = blockIdx.x - t.bptt_begin[ri];
  switch (r.d) {
    case 16: gru1d_bptt_body<16, 2, kBpttNT, G1<16>::WSMEM, true>(r.img, a, blk); break;
    case 32: gru1d_bptt_body<32, 2, kBpttNT, G1<32>::WSMEM, true>(r.img, a, blk); break;
    case 64: gru1d_bptt_body<64, 2, kBpttNT, G1<64>::WSMEM, true>(r.img, a, blk); break;
    case 128: gru1d_bptt_body<128, 2, kBpttNT, G1<128>::WSMEM, false>(r.img, a, blk); break;
  }
}

__global__ void grouped_reduce_kernel(RepTable t) {
  const Rep& r = t.r[blockIdx.y];
  const int rows = t.bptt_begin[blockIdx.y + 1] - t.bptt_begin[blockIdx.y];
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < r.P; p += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < rows; ++q) s += (double)r.partial[(size_t)q * r.P + p];
    r.grad[p] = (float)s;
  }
}

__global__ void advance_step_kernel(uint64_t* step) { *step += 1; }

int sm_count_b() {
  static int sms = 0;
  if (!sms) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      sms = n;
    else
      sms = 152;
  }
  return sms;
}

size_t fwd_rows(int d) {
  switch (d) { case 16: return G1<16>::F_R; case 32: return G1<32>::F_R; case 64: return G1<64>::F_R; case 128: return G1<128>::F_R; }
  return 1;
}
size_t bptt_rows(int d) {
  switch (d) { case 16: return G1<16>::B_R; case 32: return G1<32>::B_R; case 64: return G1<64>::B_R; case 128: return G1<128>::B_R; }
  return 1;
}

}  // namespace

bool batched_supported_d(int d) { return d == 16 || d == 32 || d == 64 || d == 128; }
int batched_bptt_blocks(int d, int64_t B) { return (int)((B + (int64_t)bptt_rows(d) - 1) / (int64_t)bptt_rows(d)); }

size_t batched_max_smem(int which) {
  size_t m = 0;
  const size_t f[4] = {G1<16>::F_SMEM, G1<32>::F_SMEM, G1<64>::F_SMEM, G1<128>::F_SMEM};
  const size_t c[4] = {G1<16>::C_SMEM, G1<32>::C_SMEM, G1<64>::C_SMEM, G1<128>::C_SMEM};
  const size_t b[4] = {G1<16>::B_SMEM, G1<32>::B_SMEM, G1<64>::B_SMEM, G1<128>::B_SMEM};
  for (int i = 0; i < 4; ++i) m = std::max(m, which == 0 ? f[i] : which == 1 ? c[i] : b[i]);
  return m;
}

cudaError_t batched_step(const BatchRep* reps, int R, uint64_t step, const uint64_t* step_dev, uint64_t* step_inc,
                         cudaStream_t st) {
  RepTable t{};
  t.R = R;
  t.step = step;
  t.step_dev = step_dev;
  int fwd = 0, bptt = 0;
  double work_total = 0.0, work[kMaxRep];
  int64_t max_rows = 0;
  for (int i = 0; i < R; ++i) {
    const BatchRep& s = reps[i];
    Rep& r = t.r[i];
    r.d = s.d; r.N = s.N; r.P = s.P; r.B = s.B; r.seed = s.seed; r.J = s.J; r.Gamma = s.Gamma;
    r.params = s.params; r.img = s.img; r.sigma = s.sigma; r.logpsi = s.logpsi; r.hcache = s.hcache;
    r.eloc = s.eloc; r.grad = s.grad; r.stats = s.stats; r.dlog = s.dlog; r.delta = s.delta;
    r.partial = s.partial; r.w = s.w; r.counter = s.counter;
    t.fwd_begin[i] = fwd;
    fwd += (int)((s.B + (int64_t)fwd_rows(s.d) - 1) / (int64_t)fwd_rows(s.d));
    t.bptt_begin[i] = bptt;
    bptt += batched_bptt_blocks(s.d, s.B);
    work[i] = (double)s.B * s.N * (s.N - 1) * (3.0 * s.d * s.d + 2.0 * s.d);
    work_total += work[i];
    max_rows = std::max<int64_t>(max_rows, s.B * (int64_t)s.N);
  }
  t.fwd_begin[R] = fwd;
  t.bptt_begin[R] = bptt;
  const int chain_grid = sm_count_b();
  double acc = 0.0;
  for (int i = 0; i < R; ++i) {
    t.chain_begin[i] = (int)(acc / work_total * chain_grid + 0.5);
    acc += work[i];
  }
  t.chain_begin[R] = chain_grid;
  cudaError_t e;
  // packing
  grouped_pack_kernel<<<dim3(64, R), 256, 0, st>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // sampling
  const size_t fs = batched_max_smem(0);
  if ((e = cudaFuncSetAttribute(grouped_sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs)) != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  grouped_sample_kernel<<<fwd, kFwdNT, fs, st>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // local energies: readout, chains, energies
  grouped_readout_kernel<<<dim3((unsigned)std::min<int64_t>((max_rows * 32 + 255) / 256, 4096), R), 256, 0, st>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(reps[0].counter, 0, sizeof(unsigned long long) * R, st)) != cudaSuccess) return e;
  const size_t cs = batched_max_smem(1);
  if ((e = cudaFuncSetAttribute(grouped_chains_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs)) != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  grouped_chains_kernel<<<chain_grid, kChainNT, cs, st>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int64_t maxB = 1;
  for (int i = 0; i < R; ++i) maxB = std::max(maxB, reps[i].B);
  grouped_eloc_kernel<<<dim3((unsigned)std::min<int64_t>((maxB * 32 + 255) / 256, 4096), R), 256, 0, st>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  grouped_stats_kernel<<<R, 1024, 0, st>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // gradient
  size_t pbytes = 0;
  for (int i = 0; i < R; ++i) pbytes = std::max(pbytes, (size_t)((char*)reps[i].partial - (char*)reps[0].partial) +
                                                            (size_t)batched_bptt_blocks(reps[i].d, reps[i].B) * reps[i].P * 4);
  if ((e = cudaMemsetAsync(reps[0].partial, 0, pbytes, st)) != cudaSuccess) return e;
  const size_t bs = batched_max_smem(2);
  if ((e = cudaFuncSetAttribute(grouped_bptt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs)) != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  grouped_bptt_kernel<<<bptt, kBpttNT, bs, st>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  grouped_reduce_kernel<<<dim3(64, R), 256, 0, st>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (step_inc) {
    advance_step_kernel<<<1, 1, 0, st>>>(step_inc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nqs

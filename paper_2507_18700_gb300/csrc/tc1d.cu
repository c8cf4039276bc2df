// BF16 tensor-core path of the 1D GRU wave function (App. A) for sm_103a:
// sampling, teacher-forced log psi and the prefix-cached TFIM chains, with the
// gate GEMM h x [W_g | W_r | W_h] on tcgen05 (BF16 operands, FP32 accumulate
// in TMEM) and the FP32 recurrent state in registers.
//
// A CTA runs GROUPS independent tiles of 128 rows; tile g uses warps 4g..4g+3,
// one thread per row (= TMEM lane), and TMEM columns [256 g, 256 g + 3D).  Per
// cell step a tile: writes its rows' h (BF16) into its A operand in shared
// memory; one thread issues D/16 MMAs (M = 128, N = 3D, K = 16) against the
// weight operand kept in shared memory and commits them to the tile's
// mbarrier; after the wait every thread reads its row's 3D accumulators from
// TMEM, applies the gates, updates h in FP32 and the readout, and runs the
// row logic (draw / teacher forcing / chain bookkeeping).  Two tiles per CTA
// let one tile's MMA overlap the other tile's epilogue.
#include "kernels.h"
#include "tc.cuh"

namespace nqs {

namespace {

constexpr uint32_t kWaitLimit = 1u << 26;   // mbarrier polls before giving up (seconds)

// Row-major [3D][D] gate weights as a K-major BF16 operand (see tc.cuh).
__global__ void pack1d_tc_kernel(const float* __restrict__ p, uint8_t* __restrict__ wimg, int D) {
  const int total = 3 * D * D;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int n = t / D, k = t % D, g = n / D, u = n % D;
    const int Wg = 0, Wr = D * (D + 2), Wh = 2 * D * (D + 2);
    const float v = g == 0 ? p[Wg + u * (D + 2) + k] : g == 1 ? p[Wr + u * (D + 2) + k] : p[Wh + u * D + k];
    *reinterpret_cast<__nv_bfloat16*>(wimg + tc::kmajor_offset(n, k, D)) = __float2bfloat16_rn(v);
  }
}

// Gate nonlinearities of the BF16 path: one hardware tanh (MUFU.TANH,
// relative error ~2^-11, below the 2^-9 rounding of the BF16 GEMM operands)
// per gate; sigmoid(x) = (1 + tanh(x/2)) / 2.
__device__ __forceinline__ float hw_tanh(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float fast_sigmoid(float x) { return fmaf(0.5f, hw_tanh(0.5f * x), 0.5f); }
__device__ __forceinline__ float fast_tanh(float x) { return hw_tanh(x); }

// Shared-memory carve-up (bytes from a 1024-aligned base).
template <int D, int GROUPS>
struct Smem {
  static constexpr int kB = 0;                                   // weights, 3D x D bf16
  static constexpr int kA = kB + 3 * D * D * 2;                  // GROUPS x 128 x D bf16
  static constexpr int kSmall = kA + GROUPS * 128 * D * 2;       // 12D+4 floats
  static constexpr int kBar = (kSmall + (12 * D + 4) * 4 + 15) / 16 * 16;
  static constexpr int kSlot = kBar + 8 * GROUPS;
  static constexpr int kUsed = kSlot + 16;
  // one CTA per SM for the persistent chain launch (TMEM holds two tiles)
  static constexpr int kBytes = 1024 + (GROUPS == 2 ? (kUsed > 120 * 1024 ? kUsed : 120 * 1024) : kUsed);
};

template <int D, int MODE, int GROUPS>
__global__ void __launch_bounds__(128 * GROUPS, 1)
tc1d_engine_kernel(const float* __restrict__ img, const uint8_t* __restrict__ wimg, Tc1Args a) {
  using S = Smem<D, GROUPS>;
  constexpr int NT = 128 * GROUPS;
  constexpr int N3 = 3 * D;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  uint8_t* sB = sm + S::kB;
  float* small = reinterpret_cast<float*>(sm + S::kSmall);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);

  // ---- prologue: operands and constants into shared memory, TMEM, barriers ----
  for (int i = threadIdx.x; i < N3 * D * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sB)[i] = reinterpret_cast<const uint4*>(wimg)[i];
  for (int i = threadIdx.x; i < (12 * D + 4) / 4; i += NT)
    reinterpret_cast<float4*>(small)[i] = reinterpret_cast<const float4*>(img)[i];
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    for (int g = 0; g < GROUPS; ++g) tc::mbar_init(&mbar[g], 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, GROUPS == 2 ? 512 : 256);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;

  const int g = threadIdx.x / 128, m = threadIdx.x % 128, lane = threadIdx.x & 31;
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16) + (uint32_t)(g * 256);
  uint8_t* sA = sm + S::kA + g * 128 * D * 2;
  const float* Ws = small;
  const float* Bs = small + 6 * D;
  const float* Us = small + 10 * D;
  const float c0 = small[12 * D], c1 = small[12 * D + 1];
  const int N = a.N;
  const int64_t B = a.B;

  float h[D];
#pragma unroll
  for (int u = 0; u < D; ++u) h[u] = 0.0f;
  int64_t b = 0;
  int t = 0, s_in = -1, f = 0;
  float acc = 0.0f;            // log psi sum, or Delta of the chain
  bool active = false;

  const uint64_t total = MODE == 2 ? (uint64_t)B * (uint64_t)(N - 1) : 0;
  // Warp-aggregated work-queue pull: one atomic per warp; returns job or -1.
  auto pull = [&](bool need) -> long long {
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    if (!mask) return -1;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(a.counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!need) return -1;
    const unsigned long long j = base + __popc(mask & ((1u << lane) - 1u));
    return j < total ? (long long)j : -1;
  };
  auto load_h = [&](const float* src) {
#pragma unroll
    for (int q = 0; q < D / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(src)[q];
      h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
    }
  };
  auto start_job = [&](long long j) {
    if (j < 0) { active = false; return; }
    b = (int64_t)((unsigned long long)j % (unsigned long long)B);
    f = (int)((unsigned long long)j / (unsigned long long)B);
    const int sf = a.sigma[b * N + f] ? 1 : 0;
    const float df = a.dlog[b * N + f];
    t = f + 1;
    s_in = 1 - sf;
    acc = 0.5f * (sf == 0 ? -df : df);
    active = true;
    load_h(a.hcache + (b * N + f) * D);
  };

  if constexpr (MODE == 2) {
    start_job(pull(true));
  } else {
    b = ((int64_t)blockIdx.x * GROUPS + g) * 128 + m;
    active = b < B;
  }

  uint32_t phase = 0;
  bool timed_out = false;
  for (;;) {
    // ---- (a) this row's h as BF16 into the A operand ----
#pragma unroll
    for (int kc = 0; kc < D / 8; ++kc) {
      __nv_bfloat162 p0 = __floats2bfloat162_rn(h[8 * kc + 0], h[8 * kc + 1]);
      __nv_bfloat162 p1 = __floats2bfloat162_rn(h[8 * kc + 2], h[8 * kc + 3]);
      __nv_bfloat162 p2 = __floats2bfloat162_rn(h[8 * kc + 4], h[8 * kc + 5]);
      __nv_bfloat162 p3 = __floats2bfloat162_rn(h[8 * kc + 6], h[8 * kc + 7]);
      uint4 v;
      v.x = *reinterpret_cast<uint32_t*>(&p0);
      v.y = *reinterpret_cast<uint32_t*>(&p1);
      v.z = *reinterpret_cast<uint32_t*>(&p2);
      v.w = *reinterpret_cast<uint32_t*>(&p3);
      *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, 8 * kc, D)) = v;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    const bool any = tc::group_barrier_or(active && !timed_out, 1 + g, 128);
    if (!any) break;
    tc::fence_after_sync();
    // ---- (b) one thread issues the tile's MMAs ----
    if (m == 0) {
      constexpr uint32_t idesc = tc::make_idesc_bf16(128, N3);
#pragma unroll
      for (int k = 0; k < D / 16; ++k) {
        const uint64_t da = tc::make_desc(tc::smem_addr(sA) + k * 256, 128, (D / 8) * 128);
        const uint64_t db = tc::make_desc(tc::smem_addr(sB) + k * 256, 128, (D / 8) * 128);
        tc::mma_bf16(tbase + (uint32_t)(g * 256), da, db, idesc, k > 0);
      }
      tc::mma_commit(&mbar[g]);
    }
    // ---- (c) row inputs of this step, fetched while the MMA runs ----
    int s_t = 0;
    float dl = 0.0f, uni = 0.0f;
    if (active) {
      if constexpr (MODE == 0) {
        uni = a.uniforms ? a.uniforms[b * N + t] : sampling_uniform(a.seed, a.step, (uint32_t)b, (uint32_t)t);
      } else {
        s_t = a.sigma[b * N + t] ? 1 : 0;
        if constexpr (MODE == 2) dl = a.dlog[b * N + t];
      }
    }
    // ---- (d) wait for the accumulator ----
    if (!tc::mbar_wait(&mbar[g], phase, kWaitLimit)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    phase ^= 1;
    tc::fence_after_sync();
    // ---- (e) gates and FP32 state update ----
    const float* Wsel = Ws + (s_in > 0 ? 3 * D : 0);
    const float on = s_in >= 0 ? 1.0f : 0.0f;
    float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
    for (int c = 0; c < D / 16; ++c) {
      float au[16], ar[16], ah[16];
      tc::tmem_ld16(trow + c * 16, au);
      tc::tmem_ld16(trow + D + c * 16, ar);
      tc::tmem_ld16(trow + 2 * D + c * 16, ah);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int u = c * 16 + q;
        const float ug = fast_sigmoid(au[q] + Bs[u] + on * Wsel[u]);
        const float rg = fast_sigmoid(ar[q] + Bs[D + u] + on * Wsel[D + u]);
        const float cc = fast_tanh(fmaf(rg, ah[q] + Bs[2 * D + u], Bs[3 * D + u] + on * Wsel[2 * D + u]));
        h[u] = fmaf(ug, cc - h[u], h[u]);
        z0 = fmaf(Us[u], h[u], z0);
        z1 = fmaf(Us[D + u], h[u], z1);
      }
    }
    // ---- (f) row logic ----
    bool need = false;
    if (active && !timed_out) {
      const float d = (z0 + c0) - (z1 + c1);
      if constexpr (MODE == 2) {
        acc += 0.5f * (log_prob(s_t, d) - log_prob(s_t, dl));
        s_in = s_t;
        if (++t == N) {
          a.delta[b * N + f] = acc;
          need = true;
        }
      } else {
        int s = s_t;
        if constexpr (MODE == 0) {
          s = uni < sigmoid_acc(d) ? 0 : 1;
          a.sigma_out[b * N + t] = (uint8_t)s;
        }
        acc += log_prob(s, d);
        if (a.hcache) {
          float4* dst = reinterpret_cast<float4*>(a.hcache + (b * N + t) * D);
#pragma unroll
          for (int q = 0; q < D / 4; ++q) dst[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
        }
        s_in = s;
        if (++t == N) {
          const float lp = 0.5f * acc;
          a.logpsi[b] = lp;
          if (!isfinite(lp)) flag_status(a.hdr, NQS_ENONFINITE);
          active = false;
        }
      }
    }
    if constexpr (MODE == 2) {
      const long long j = pull(need);
      if (need) start_job(j);
    }
  }
  // ---- epilogue: free TMEM once both tiles are done ----
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, GROUPS == 2 ? 512 : 256);
}

// ----------------------------------------------------------------------------
// Reverse sweep on the tensor cores.  One CTA = one tile of 128 samples, one
// thread per sample; sites n = N-1 .. 0.  Per site:
//   X  = [h_{n-1} | 1 | onehot(s_{n-1}) | 0]  (BF16, 80 columns, row per sample)
//   MMA_f: acc_f = X[:, :D] W3^T            recompute the gate pre-activations
//   epilogue: gates, h_n, readout, dz = c_b (onehot - softmax), dh, and
//             G = [du_a | dr_a | dq | dc_a]  (BF16, 4D columns)
//   MMA_b: acc_b = G[:, :3D] W3               (dh_{n-1} through the gates)
//   MMA_w: acc_w += G^T X                     (weight, bias and one-hot-column
//                                              gradients; G and X read as
//                                              MN-major operands)
//   carry = dh direct + acc_b.
// acc_w stays in TMEM for the whole sweep; readout gradients (U, c) come from
// dz written per (sample, site) and are reduced by a separate kernel.
// ----------------------------------------------------------------------------
constexpr int kXCols = 80;

template <int D>
struct BSmem {
  static constexpr int GW = 4 * D >= 128 ? 4 * D : 128;  // G row width (>= one M = 128 operand)
  static constexpr int kW3 = 0;                         // [3D x D] bf16, K-major
  static constexpr int kWt = kW3 + 3 * D * D * 2;       // [D x 3D] bf16, K-major
  static constexpr int kX = kWt + 3 * D * D * 2;        // [128 x 80] bf16
  static constexpr int kG = kX + 128 * kXCols * 2;      // [128 x GW] bf16
  static constexpr int kSmall = kG + 128 * GW * 2;      // 12D + 4 floats
  static constexpr int kBar = (kSmall + (12 * D + 4) * 4 + 15) / 16 * 16;
  static constexpr int kSlot = kBar + 16;
  static constexpr int kBytes = 1024 + kSlot + 16;
  // TMEM columns
  static constexpr int cF = 0, cB = 3 * D, cW0 = 3 * D + D, cW1 = cW0 + kXCols;
  static_assert(cW1 + kXCols <= 512, "TMEM budget");
};

__device__ __forceinline__ void st_bf16x8(uint8_t* dst, const float* v) {
  __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 p1 = __floats2bfloat162_rn(v[2], v[3]);
  __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]);
  __nv_bfloat162 p3 = __floats2bfloat162_rn(v[6], v[7]);
  uint4 q;
  q.x = *reinterpret_cast<uint32_t*>(&p0);
  q.y = *reinterpret_cast<uint32_t*>(&p1);
  q.z = *reinterpret_cast<uint32_t*>(&p2);
  q.w = *reinterpret_cast<uint32_t*>(&p3);
  *reinterpret_cast<uint4*>(dst) = q;
}

template <int D>
__global__ void __launch_bounds__(128, 1)
tc1d_bptt_kernel(const float* __restrict__ img, const uint8_t* __restrict__ w3img, const uint8_t* __restrict__ wtimg,
                 TcBpttArgs a) {
  using S = BSmem<D>;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  uint8_t* sW3 = sm + S::kW3;
  uint8_t* sWt = sm + S::kWt;
  uint8_t* sX = sm + S::kX;
  uint8_t* sG = sm + S::kG;
  float* small = reinterpret_cast<float*>(sm + S::kSmall);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < 3 * D * D * 2 / 16; i += 128) {
    reinterpret_cast<uint4*>(sW3)[i] = reinterpret_cast<const uint4*>(w3img)[i];
    reinterpret_cast<uint4*>(sWt)[i] = reinterpret_cast<const uint4*>(wtimg)[i];
  }
  for (int i = threadIdx.x; i < (12 * D + 4) / 4; i += 128)
    reinterpret_cast<float4*>(small)[i] = reinterpret_cast<const float4*>(img)[i];
  for (int i = threadIdx.x; i < 128 * S::GW * 2 / 16; i += 128) reinterpret_cast<uint4*>(sG)[i] = make_uint4(0, 0, 0, 0);
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int m = threadIdx.x;
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16);
  const float* Ws = small;
  const float* Bs = small + 6 * D;
  const float* Us = small + 10 * D;
  const float c0 = small[12 * D], c1 = small[12 * D + 1];
  const int N = a.N;
  const int64_t b = (int64_t)blockIdx.x * 128 + m;
  const bool valid = b < a.B;
  const float coef = valid ? 0.5f * a.weights[b] : 0.0f;
  float carry[D];
#pragma unroll
  for (int u = 0; u < D; ++u) carry[u] = 0.0f;
  uint32_t ph_f = 0, ph_b = 0;
  bool timed_out = false;
  constexpr uint32_t idesc_f = tc::make_idesc_bf16(128, 3 * D);
  constexpr uint32_t idesc_b = tc::make_idesc_bf16(128, D);
  constexpr uint32_t idesc_w = tc::make_idesc_bf16(128, kXCols) | (1u << 15) | (1u << 16);
  // 16 values of h_{n-1} of this sample (zero at the first site / past the batch)
  auto load_hp16 = [&](int n, int c, float (&v)[16]) {
    if (valid && n > 0) {
      const float4* src = reinterpret_cast<const float4*>(a.hcache + (b * N + n - 1) * D + 16 * c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 t = src[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = 0.0f;
    }
  };

  for (int n = N - 1; n >= 0; --n) {
    // ---- X row: [h_{n-1} | 1 | onehot(s_{n-1}) | 0] ----
    int s_in = -1, s_n = 0;
    if (valid) {
      s_n = a.sigma[b * N + n] ? 1 : 0;
      if (n > 0) s_in = a.sigma[b * N + n - 1] ? 1 : 0;
    }
#pragma unroll
    for (int c = 0; c < D / 16; ++c) {
      float hp[16];
      load_hp16(n, c, hp);
      st_bf16x8(sX + tc::kmajor_offset(m, 16 * c, kXCols), hp);
      st_bf16x8(sX + tc::kmajor_offset(m, 16 * c + 8, kXCols), hp + 8);
    }
    {
      float ext[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) ext[q] = 0.0f;
      ext[0] = 1.0f;
      if (s_in >= 0) ext[1 + s_in] = 1.0f;
      st_bf16x8(sX + tc::kmajor_offset(m, D, kXCols), ext);
      st_bf16x8(sX + tc::kmajor_offset(m, D + 8, kXCols), ext + 8);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (m == 0) {
#pragma unroll
      for (int k = 0; k < D / 16; ++k) {
        const uint64_t da = tc::make_desc(tc::smem_addr(sX) + k * 256, 128, (kXCols / 8) * 128);
        const uint64_t db = tc::make_desc(tc::smem_addr(sW3) + k * 256, 128, (D / 8) * 128);
        tc::mma_bf16(tbase + S::cF, da, db, idesc_f, k > 0);
      }
      tc::mma_commit(&mbar[0]);
    }
    if (!tc::mbar_wait(&mbar[0], ph_f, kWaitLimit)) { timed_out = true; flag_status(a.hdr, NQS_ETIMEOUT); }
    ph_f ^= 1;
    tc::fence_after_sync();
    const float* Wsel = Ws + (s_in > 0 ? 3 * D : 0);
    const float on = s_in >= 0 ? 1.0f : 0.0f;
    // ---- pass 1: recompute h_n for the readout ----
    float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
    for (int c = 0; c < D / 16; ++c) {
      float au[16], ar[16], ah[16], hp[16];
      tc::tmem_ld16(trow + S::cF + c * 16, au);
      tc::tmem_ld16(trow + S::cF + D + c * 16, ar);
      tc::tmem_ld16(trow + S::cF + 2 * D + c * 16, ah);
      load_hp16(n, c, hp);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int u = c * 16 + q;
        const float ug = fast_sigmoid(au[q] + Bs[u] + on * Wsel[u]);
        const float rg = fast_sigmoid(ar[q] + Bs[D + u] + on * Wsel[D + u]);
        const float cg = fast_tanh(fmaf(rg, ah[q] + Bs[2 * D + u], Bs[3 * D + u] + on * Wsel[2 * D + u]));
        const float hn = fmaf(ug, cg - hp[q], hp[q]);
        z0 = fmaf(Us[u], hn, z0);
        z1 = fmaf(Us[D + u], hn, z1);
      }
    }
    const float d = (z0 + c0) - (z1 + c1);
    const float dz0 = coef * ((s_n == 0 ? 1.0f : 0.0f) - sigmoid_acc(d));
    if (valid) a.dz[b * N + n] = dz0;
    // ---- pass 2: gates again, backward through the cell, G = [du_a | dr_a | dq | dc_a] ----
#pragma unroll
    for (int c = 0; c < D / 16; ++c) {
      float au[16], ar[16], ah[16], hp[16];
      tc::tmem_ld16(trow + S::cF + c * 16, au);
      tc::tmem_ld16(trow + S::cF + D + c * 16, ar);
      tc::tmem_ld16(trow + S::cF + 2 * D + c * 16, ah);
      load_hp16(n, c, hp);
      tc::tmem_wait_ld();
      float gbuf[4][16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int u = c * 16 + q;
        const float ug = fast_sigmoid(au[q] + Bs[u] + on * Wsel[u]);
        const float rg = fast_sigmoid(ar[q] + Bs[D + u] + on * Wsel[D + u]);
        const float qv = ah[q] + Bs[2 * D + u];
        const float cg = fast_tanh(fmaf(rg, qv, Bs[3 * D + u] + on * Wsel[2 * D + u]));
        const float dh = dz0 * (Us[u] - Us[D + u]) + carry[u];
        const float dc = dh * ug;
        const float du = dh * (cg - hp[q]);
        carry[u] = dh * (1.0f - ug);                     // direct path; acc_b adds the rest
        const float dac = dc * (1.0f - cg * cg);
        gbuf[0][q] = du * ug * (1.0f - ug);
        gbuf[1][q] = dac * qv * rg * (1.0f - rg);
        gbuf[2][q] = dac * rg;
        gbuf[3][q] = dac;
      }
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        st_bf16x8(sG + tc::kmajor_offset(m, g * D + 16 * c, S::GW), gbuf[g]);
        st_bf16x8(sG + tc::kmajor_offset(m, g * D + 16 * c + 8, S::GW), gbuf[g] + 8);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (m == 0) {
      // dh_{n-1} += G[:, :3D] W3   (K-major: LBO = 128 B along K, SBO = row-group stride)
#pragma unroll
      for (int k = 0; k < 3 * D / 16; ++k) {
        const uint64_t da = tc::make_desc(tc::smem_addr(sG) + k * 256, 128, (S::GW / 8) * 128);
        const uint64_t db = tc::make_desc(tc::smem_addr(sWt) + k * 256, 128, (3 * D / 8) * 128);
        tc::mma_bf16(tbase + S::cB, da, db, idesc_b, k > 0);
      }
      // acc_w += G^T X over the 128 samples of this site, halves of 128 gate rows.
      // Both operands MN-major: LBO = stride of 8-sample groups along K (the
      // buffer's row-group stride), SBO = 128 B between 8-column groups along
      // M / N.  One K = 16 step covers two sample groups.
#pragma unroll
      for (int half = 0; half < S::GW / 128; ++half) {
#pragma unroll
        for (int k = 0; k < 128 / 16; ++k) {
          const uint64_t da = tc::make_desc(tc::smem_addr(sG) + half * 16 * 128 + k * 2 * (S::GW / 8) * 128,
                                            (S::GW / 8) * 128, 128);
          const uint64_t db = tc::make_desc(tc::smem_addr(sX) + k * 2 * (kXCols / 8) * 128, (kXCols / 8) * 128, 128);
          tc::mma_bf16(tbase + (half ? S::cW1 : S::cW0), da, db, idesc_w, (n < N - 1) || k > 0);
        }
      }
      tc::mma_commit(&mbar[1]);
    }
    if (!tc::mbar_wait(&mbar[1], ph_b, kWaitLimit)) { timed_out = true; flag_status(a.hdr, NQS_ETIMEOUT); }
    ph_b ^= 1;
    tc::fence_after_sync();
#pragma unroll
    for (int c = 0; c < D / 16; ++c) {
      float v[16];
      tc::tmem_ld16(trow + S::cB + c * 16, v);
      tc::tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 16; ++q) carry[c * 16 + q] += v[q];
    }
    if (timed_out) break;
  }
  // ---- this CTA's weight, bias and one-hot-column gradients from acc_w ----
  const int Wg = 0, Wr = D * (D + 2), Wh = 2 * D * (D + 2), Win = Wh + D * D;
  const int bg = Win + 2 * D, br = bg + D, bh = br + D, bin = bh + D;
  float* part = a.partial + (size_t)blockIdx.x * a.P;
#pragma unroll 1
  for (int half = 0; half < S::GW / 128; ++half) {
    const int gu = half * 128 + m;
    if (gu < 4 * D) {
      const int g = gu / D, u = gu % D;
#pragma unroll 1
      for (int c = 0; c < kXCols; c += 16) {
        float v[16];
        tc::tmem_ld16(trow + (half ? S::cW1 : S::cW0) + c, v);
        tc::tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int k = c + q;
          if (k < D) {
            if (g == 0) part[Wg + u * (D + 2) + k] = v[q];
            else if (g == 1) part[Wr + u * (D + 2) + k] = v[q];
            else if (g == 2) part[Wh + u * D + k] = v[q];
          } else if (k == D) {
            part[(g == 0 ? bg : g == 1 ? br : g == 2 ? bh : bin) + u] = v[q];
          } else if (k <= D + 2) {
            const int s = k - D - 1;
            if (g == 0) part[Wg + u * (D + 2) + D + s] = v[q];
            else if (g == 1) part[Wr + u * (D + 2) + D + s] = v[q];
            else if (g == 3) part[Win + u * 2 + s] = v[q];
          }
        }
      }
    } else {
      // keep the warp's collective TMEM loads aligned
#pragma unroll 1
      for (int c = 0; c < kXCols; c += 16) {
        float v[16];
        tc::tmem_ld16(trow + (half ? S::cW1 : S::cW0) + c, v);
        tc::tmem_wait_ld();
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 512);
}

// Readout gradients: dU[0][u] = sum_{b,n} dz h_n[u], dU[1] = -dU[0], dc0 = sum dz,
// dc1 = -dc0; one partial row per block.
template <int D>
__global__ void tc1d_readout_grad_kernel(const float* __restrict__ hcache, const float* __restrict__ dz,
                                         int64_t rows, float* __restrict__ partial, int P, int part_row0) {
  __shared__ float red[256];
  const int Uoff = 3 * D * D + 10 * D, coff = Uoff + 2 * D;   // U and c of the flat 1D layout
  float* part = partial + (size_t)(part_row0 + blockIdx.x) * P;
  // thread t accumulates unit t % D over rows t / D, t / D + 256 / D, ...
  constexpr int RPB = 256 / D;
  const int u = threadIdx.x % D, r0 = threadIdx.x / D;
  float acc = 0.0f, accc = 0.0f;
  for (int64_t r = (int64_t)blockIdx.x * RPB + r0; r < rows; r += (int64_t)gridDim.x * RPB) {
    const float z = dz[r];
    acc = fmaf(z, hcache[r * D + u], acc);
    if (u == 0) accc += z;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < D) {
    float s = 0.0f;
    for (int q = 0; q < RPB; ++q) s += red[q * D + threadIdx.x];
    part[Uoff + threadIdx.x] = s;
    part[Uoff + D + threadIdx.x] = -s;
  }
  __syncthreads();
  red[threadIdx.x] = accc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int q = 0; q < RPB; ++q) s += red[q * D];
    part[coff] = s;
    part[coff + 1] = -s;
  }
}

// Gate weights as the B operand of MMA_b: [D rows (k) x 3D (gate, unit)].
__global__ void pack1d_tc_t_kernel(const float* __restrict__ p, uint8_t* __restrict__ wt, int D) {
  const int total = 3 * D * D;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int k = t / (3 * D), gu = t % (3 * D), g = gu / D, u = gu % D;
    const int Wg = 0, Wr = D * (D + 2), Wh = 2 * D * (D + 2);
    const float v = g == 0 ? p[Wg + u * (D + 2) + k] : g == 1 ? p[Wr + u * (D + 2) + k] : p[Wh + u * D + k];
    *reinterpret_cast<__nv_bfloat16*>(wt + tc::kmajor_offset(k, gu, 3 * D)) = __float2bfloat16_rn(v);
  }
}

int sm_count_tc() {
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

template <int D, int MODE, int GROUPS>
cudaError_t launch_tc(const Tc1Args& a, const float* img, const uint8_t* wimg, cudaStream_t st) {
  using S = Smem<D, GROUPS>;
  auto k = tc1d_engine_kernel<D, MODE, GROUPS>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  int64_t grid;
  if (MODE == 2) {
    const int64_t jobs = a.B * (int64_t)(a.N - 1);
    grid = sm_count_tc();
    const int64_t need = (jobs + 255) / 256;
    if (grid > need) grid = need;
  } else {
    grid = (a.B + 128 * GROUPS - 1) / (128 * GROUPS);
  }
  if (grid < 1) grid = 1;
  k<<<(unsigned)grid, 128 * GROUPS, S::kBytes, st>>>(img, wimg, a);
  return cudaGetLastError();
}

template <int D>
cudaError_t dispatch_mode(const Tc1Args& a, const float* img, const uint8_t* wimg, int mode, cudaStream_t st) {
  switch (mode) {
    case 0: return launch_tc<D, 0, 1>(a, img, wimg, st);
    case 1: return launch_tc<D, 1, 1>(a, img, wimg, st);
    case 2: return launch_tc<D, 2, 2>(a, img, wimg, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int tc1d_supported(int D) { return D == 16 || D == 32 || D == 64; }

constexpr int kReadoutGradBlocks = 64;
int tc1d_bptt_partial_rows(int64_t B) { return (int)((B + 127) / 128) + kReadoutGradBlocks; }

template <int D>
cudaError_t launch_tc_bptt(const TcBpttArgs& a, const float* img, const uint8_t* w3, const uint8_t* wt, cudaStream_t st) {
  using S = BSmem<D>;
  auto k = tc1d_bptt_kernel<D>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  const int grid = (int)((a.B + 127) / 128);
  k<<<grid, 128, S::kBytes, st>>>(img, w3, wt, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tc1d_readout_grad_kernel<D><<<kReadoutGradBlocks, 256, 0, st>>>(a.hcache, a.dz, a.B * (int64_t)a.N, a.partial, a.P,
                                                                   grid);
  return cudaGetLastError();
}

cudaError_t tc1d_pack_t(const float* params, uint8_t* wt, int D, cudaStream_t st) {
  const int total = 3 * D * D;
  pack1d_tc_t_kernel<<<(total + 255) / 256, 256, 0, st>>>(params, wt, D);
  return cudaGetLastError();
}

cudaError_t tc1d_bptt(const TcBpttArgs& a, const float* img, const uint8_t* w3, const uint8_t* wt, int D,
                      cudaStream_t st) {
  switch (D) {
    case 16: return launch_tc_bptt<16>(a, img, w3, wt, st);
    case 32: return launch_tc_bptt<32>(a, img, w3, wt, st);
    case 64: return launch_tc_bptt<64>(a, img, w3, wt, st);
  }
  return cudaErrorInvalidValue;
}
size_t tc1d_wimg_bytes(int D) { return (size_t)3 * D * D * 2; }

cudaError_t tc1d_pack(const float* params, uint8_t* wimg, int D, cudaStream_t st) {
  const int total = 3 * D * D;
  pack1d_tc_kernel<<<(total + 255) / 256, 256, 0, st>>>(params, wimg, D);
  return cudaGetLastError();
}

cudaError_t tc1d_run(const Tc1Args& a, const float* img, const uint8_t* wimg, int D, int mode, cudaStream_t st) {
  switch (D) {
    case 16: return dispatch_mode<16>(a, img, wimg, mode, st);
    case 32: return dispatch_mode<32>(a, img, wimg, mode, st);
    case 64: return dispatch_mode<64>(a, img, wimg, mode, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nqs

// BF16 tensor-core reverse sweep of the 1D GRU wave function (App. A) at d_h =
// 128: d/dtheta sum_b w_b log psi_b (log psi = 1/2 sum_n log p(s_n | s_<n)).
//
// The d_h <= 64 sweep (tc1d.cu) keeps the weight gradient in TMEM beside the
// recurrent product and both weight operands in shared memory; at d_h = 128
// neither fits.  Here the sweep is split in four passes:
//  1. tape pass, every (sample, site n) cell in parallel (tiles of 128
//     samples at one site): the forward's gate pre-activations from the
//     cached h_{n-1} with the engine's own BF16 weight operand and FP32 x_in
//     table (so u, r, q, the candidate c and x_in are those of the forward),
//     the five factors with which the cell backward is linear in dh,
//       k0 = (c - h_{n-1}) u (1 - u)   (gradient of the u pre-activation)
//       k3 = u (1 - c^2)               (of the candidate's pre-activation)
//       k2 = k3 r                      (of q = W_h h_{n-1} + b_h)
//       k1 = k2 q (1 - r)              (of the r pre-activation)
//       k4 = 1 - u                     (the direct path to h_{n-1})
//     (FP16), the readout gradient gd_n = w_b (onehot_0(s_n) - p_0(h_n)) / 2,
//     and the weight-gradient operands X_n = [h_{n-1} | 1 | onehot(s_{n-1})]
//     (BF16, operand-tape layout of tc_wgrad.cuh);
//  2. sequential sweep, one CTA per tile of 128 samples, n = N-1 .. 0:
//       dh = gd_n (U_0 - U_1) + carry,  G = dh [k0 | k1 | k2 | k3]  (BF16),
//       carry = G[:, :3D] W3 + dh k4
//     with W3 = [W_g ; W_r ; W_h] restricted to the h_{n-1} columns (true,
//     not halved) resident in shared memory; G goes to the G tape;
//  3. weight gradients dW = G^T X over every cell (tcw::wgrad_kernel<128>:
//     four 128-row blocks u, r, q, c against [h_{n-1} | extras]), readout
//     gradients dU, dc from gd and the cached h_n;
//  4. the final reduction into the flat gradient.
#include <cuda_fp16.h>

#include "kernels.h"
#include "tc.cuh"
#include "tc_wgrad.cuh"

namespace nqs {

namespace {

using namespace tcw;

constexpr int D = 128, KA = D + 16;                // engine operand columns: [h | 1 1 | onehot x2 | 0]
constexpr int kThreads = 512;                      // 4 threads per row, 32 units each
constexpr int kWgSplits = 38;                      // 4 tiles x 38 cell ranges = 152 units
constexpr int kRoBlocks = 304;
// flat layout (App. A; nqs.h): W_g [d, d+2], W_r [d, d+2], W_h [d, d], W_in [d, 2], b_g, b_r, b_h, b_in, U [2, d], c [2]
constexpr int oWg = 0, oWr = D * (D + 2), oWh = 2 * D * (D + 2), oWin = oWh + D * D, obg = oWin + 2 * D,
              obr = obg + D, obh = obr + D, obin = obh + D, oU = obin + D, oc = oU + 2 * D, kP = oc + 2;

__device__ __forceinline__ float hw_tanh1(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void tld8_1(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  tc::tmem_wait_ld();
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    asm volatile("" : "+r"(r[q]));
    v[q] = __uint_as_float(r[q]);
  }
}
__device__ __forceinline__ void ld8(const float* p, float (&v)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ uint4 pack8_f16(const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __half2 p = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
    w[q] = *reinterpret_cast<uint32_t*>(&p);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void unpack8_f16(uint4 q, float (&v)[8]) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

// W3 operand of the sweep: K-major [D rows (h_{n-1} units) x 3D columns (u, r,
// q gate units)], element (n, k) = W_blk(k / D)[k % D][n] with W_g, W_r, W_h.
__global__ void pack_w3_kernel(const float* __restrict__ p, uint8_t* __restrict__ w3) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < D * 3 * D; t += gridDim.x * blockDim.x) {
    const int n = t / (3 * D), k = t % (3 * D), g = k / D, u = k % D;
    const float v = g == 0 ? p[oWg + u * (D + 2) + n] : g == 1 ? p[oWr + u * (D + 2) + n] : p[oWh + u * D + n];
    *reinterpret_cast<__nv_bfloat16*>(w3 + tc::kmajor_offset(n, k, 3 * D)) = __float2bfloat16_rn(v);
  }
}

struct T1Args {
  int64_t B, Bp;
  int N;
  const uint8_t* sigma;
  const float* hcache;
  const float* weights;
  const float* params;
  __half* tape_k;            // [cells, 5, D]
  float* gd;                 // [cells]
  uint8_t* x1a;              // X tape, h_{n-1} (one tile of 128 columns)
  uint8_t* x1c;              // X tape, [1 | onehot(s_{n-1}) | 0] (16 columns)
  WsHeader* hdr;
};

struct T1S {
  static constexpr uint32_t kW = 0;                                  // [3D x KA] bf16 (the engine's u, r, q rows)
  static constexpr uint32_t kA = kW + 3 * D * KA * 2;                // [128 x KA] bf16
  static constexpr uint32_t kXin = kA + 128 * KA * 2;                // [3][D] x_in table: no input, s = 0, s = 1
  static constexpr uint32_t kUd = kXin + 3 * D * 4;                  // D + 4 floats: U_0 - U_1, c_0 - c_1
  static constexpr uint32_t kZ = kUd + (D + 4) * 4;                  // 4 x 128 floats: readout partials
  static constexpr uint32_t kBar = kZ + 512 * 4;                     // MMA, drain
  static constexpr uint32_t kSlot = kBar + 16;
  static constexpr uint32_t kBytes = 1024 + kSlot + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
};

__global__ void __launch_bounds__(kThreads, 1) tc1d128_tape_kernel(const uint8_t* __restrict__ wimg, T1Args a) {
  using S = T1S;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;
  uint8_t* sW = sm + S::kW;
  uint8_t* sA = sm + S::kA;
  float* sXin = reinterpret_cast<float*>(sm + S::kXin);
  float* sUd = reinterpret_cast<float*>(sm + S::kUd);
  float* sZ = reinterpret_cast<float*>(sm + S::kZ);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < 3 * D * KA * 2 / 16; i += kThreads)
    reinterpret_cast<uint4*>(sW)[i] = reinterpret_cast<const uint4*>(wimg)[i];
  const float* p = a.params;
  for (int i = threadIdx.x; i < 3 * D; i += kThreads) {   // x_in = b_in + W_in onehot(s), as the engine forms it
    const int sv = i / D - 1, u = i % D;
    sXin[i] = p[obin + u] + (sv >= 0 ? p[oWin + u * 2 + sv] : 0.0f);
  }
  for (int i = threadIdx.x; i < D; i += kThreads) sUd[i] = p[oU + i] - p[oU + D + i];
  if (threadIdx.x == 0) {
    sUd[D] = p[oc] - p[oc + 1];
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 512);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, part = warp >> 2, quarter = warp & 3;
  const int m = quarter * 32 + lane, u0 = 32 * part;
  const uint32_t trow = tbase + ((uint32_t)(quarter * 32) << 16);
  const int N = a.N;
  const int64_t B = a.B, nbt = a.Bp / 128, ntile = (int64_t)N * nbt, nkb = a.Bp * N / 16;
  const uint32_t one = 0x3F80u;
  uint32_t ph = 0;
  bool timed_out = false;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int n = (int)(tile / nbt);
    const int64_t b = (tile % nbt) * 128 + m;
    const bool valid = b < B;
    const int64_t cell = (int64_t)n * a.Bp + b;
    const float* hp = valid && n > 0 ? a.hcache + (b * N + n - 1) * D : nullptr;   // h_{n-1} (h_0 = 0)
    const int s_in = valid && n > 0 ? (a.sigma[b * N + n - 1] ? 1 : 0) : -1;       // no input at n = 0
    // ---- A row [bf16(h_{n-1}) | 1 1 | onehot(s) x2 | 0] and the X tape ----
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[8];
      if (hp) ld8(hp + u0 + 8 * c, v);
      else
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = 0.0f;
      const uint4 pk = pack8_bf16(v);
      *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, u0 + 8 * c, KA)) = pk;
      *reinterpret_cast<uint4*>(a.x1a + tape_off(cell, u0 + 8 * c, 128, nkb)) = pk;
    }
    if (part == 0) {
      const uint32_t oh = s_in < 0 ? 0u : (s_in == 0 ? one : (one << 16));
      *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, D, KA)) = make_uint4(one | (one << 16), oh, oh, 0u);
      *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, D + 8, KA)) = make_uint4(0u, 0u, 0u, 0u);
      const float xe[8] = {1.0f, s_in == 0 ? 1.0f : 0.0f, s_in == 1 ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      *reinterpret_cast<uint4*>(a.x1c + tape_off(cell, 0, 16, nkb)) = pack8_bf16(xe);
      *reinterpret_cast<uint4*>(a.x1c + tape_off(cell, 8, 16, nkb)) = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
      // u, r rows [0, 256) -> TMEM [0, 256); q rows [256, 384) -> [256, 384)
      constexpr uint32_t i256 = tc::make_idesc_bf16(128, 256), i128 = tc::make_idesc_bf16(128, 128);
      constexpr uint32_t sbo = (KA / 8) * 128;
#pragma unroll
      for (int k = 0; k < KA / 16; ++k) {
        const uint64_t da = tc::make_desc(tc::smem_addr(sA) + k * 256, 128, sbo);
        tc::mma_bf16(tbase, da, tc::make_desc(tc::smem_addr(sW) + k * 256, 128, sbo), i256, k > 0);
        tc::mma_bf16(tbase + 256, da, tc::make_desc(tc::smem_addr(sW) + 32 * sbo + k * 256, 128, sbo), i128, k > 0);
      }
      tc::mma_commit(&mbar[0]);
    }
    // readout of h_n (the cache) while the MMA runs: this slice's partial of (U_0 - U_1) h_n
    float zp = 0.0f;
    const float* hn = valid ? a.hcache + (b * N + n) * D + u0 : nullptr;
    if (hn) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v[8];
        ld8(hn + 8 * c, v);
#pragma unroll
        for (int q = 0; q < 8; ++q) zp = fmaf(sUd[u0 + 8 * c + q], v[q], zp);
      }
    }
    sZ[part * 128 + m] = zp;
    if (!tc::mbar_wait(&mbar[0], ph, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    ph ^= 1;
    tc::fence_after_sync();
    // ---- the factors k0..k4 of this slice's units ----
    const float* xin = sXin + (s_in + 1) * D;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int u = u0 + 8 * c;
      float au[8], ar[8], aq[8], hprev[8];
      tld8_1(trow + u, au);
      tld8_1(trow + D + u, ar);
      tld8_1(trow + 2 * D + u, aq);
      if (hp) ld8(hp + u, hprev);
      else
#pragma unroll
        for (int q = 0; q < 8; ++q) hprev[q] = 0.0f;
      float k0[8], k1[8], k2[8], k3[8], k4[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float ug = fmaf(0.5f, hw_tanh1(au[q]), 0.5f);
        const float rg = fmaf(0.5f, hw_tanh1(ar[q]), 0.5f);
        const float cc = hw_tanh1(fmaf(rg, aq[q], xin[u + q]));
        k0[q] = (cc - hprev[q]) * ug * (1.0f - ug);
        k3[q] = ug * (1.0f - cc * cc);
        k2[q] = k3[q] * rg;
        k1[q] = k2[q] * aq[q] * (1.0f - rg);
        k4[q] = 1.0f - ug;
      }
      __half* dst = a.tape_k + cell * (5 * D) + u;
      *reinterpret_cast<uint4*>(dst) = pack8_f16(k0);
      *reinterpret_cast<uint4*>(dst + D) = pack8_f16(k1);
      *reinterpret_cast<uint4*>(dst + 2 * D) = pack8_f16(k2);
      *reinterpret_cast<uint4*>(dst + 3 * D) = pack8_f16(k3);
      *reinterpret_cast<uint4*>(dst + 4 * D) = pack8_f16(k4);
    }
    tc::fence_before_sync();
    __syncthreads();                                   // readout partials complete; A and TMEM free again
    tc::fence_after_sync();
    if (part == 0) {
      float g = 0.0f;
      if (valid) {
        const float d = (sZ[m] + sZ[128 + m]) + (sZ[256 + m] + sZ[384 + m]) + sUd[D];
        const int s = a.sigma[b * N + n] ? 1 : 0;
        g = 0.5f * a.weights[b] * ((s == 0 ? 1.0f : 0.0f) - 1.0f / (1.0f + expf(-d)));
      }
      a.gd[cell] = g;
    }
  }
  tc::fence_before_sync();
  if (__syncthreads_or(timed_out) && threadIdx.x == 0) tc::drain_mmas(&mbar[1], tc::kDefaultWaitPolls);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 512);
}

struct S1Args {
  int64_t B, Bp;
  int N;
  const float* params;
  const __half* tape_k;
  const float* gd;
  uint8_t* g1;               // G tape: [dh k0 | dh k1 | dh k2 | dh k3] in four tiles of 128 columns
  WsHeader* hdr;
};

struct S1S {
  static constexpr uint32_t kW3 = 0;                                 // [D x 3D] bf16
  static constexpr uint32_t kA = kW3 + D * 3 * D * 2;                // [128 x 3D] bf16: G[:, :3D]
  static constexpr uint32_t kUd = kA + 128 * 3 * D * 2;              // D floats: U_0 - U_1
  static constexpr uint32_t kBar = kUd + D * 4;                      // MMA, drain
  static constexpr uint32_t kSlot = kBar + 16;
  static constexpr uint32_t kBytes = 1024 + kSlot + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
};

__global__ void __launch_bounds__(kThreads, 1) tc1d128_sweep_kernel(const uint8_t* __restrict__ w3, S1Args a) {
  using S = S1S;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;
  uint8_t* sW3 = sm + S::kW3;
  uint8_t* sA = sm + S::kA;
  float* sUd = reinterpret_cast<float*>(sm + S::kUd);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < D * 3 * D * 2 / 16; i += kThreads)
    reinterpret_cast<uint4*>(sW3)[i] = reinterpret_cast<const uint4*>(w3)[i];
  for (int i = threadIdx.x; i < D; i += kThreads) sUd[i] = a.params[oU + i] - a.params[oU + D + i];
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 128);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, part = warp >> 2, quarter = warp & 3;
  const int m = quarter * 32 + lane, u0 = 32 * part;
  const uint32_t trow = tbase + ((uint32_t)(quarter * 32) << 16);
  const int N = a.N;
  const int64_t b = (int64_t)blockIdx.x * 128 + m;     // rows past B: zero readout gradients, zero carries
  const int64_t nkb = a.Bp * N / 16;
  float carry[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) carry[j] = 0.0f;
  uint32_t ph = 0;
  bool timed_out = false;
  for (int n = N - 1; n >= 0; --n) {
    const int64_t cell = (int64_t)n * a.Bp + b;
    const float g = a.gd[cell];
    const __half* kt = a.tape_k + cell * (5 * D) + u0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int u = u0 + 8 * c;
      float k0[8], k1[8], k2[8], k3[8], k4[8], dh[8];
      unpack8_f16(*reinterpret_cast<const uint4*>(kt + 8 * c), k0);
      unpack8_f16(*reinterpret_cast<const uint4*>(kt + D + 8 * c), k1);
      unpack8_f16(*reinterpret_cast<const uint4*>(kt + 2 * D + 8 * c), k2);
      unpack8_f16(*reinterpret_cast<const uint4*>(kt + 3 * D + 8 * c), k3);
      unpack8_f16(*reinterpret_cast<const uint4*>(kt + 4 * D + 8 * c), k4);
      float gu[8], gr[8], gq[8], gc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        dh[q] = fmaf(g, sUd[u + q], carry[8 * c + q]);
        gu[q] = dh[q] * k0[q];
        gr[q] = dh[q] * k1[q];
        gq[q] = dh[q] * k2[q];
        gc[q] = dh[q] * k3[q];
        carry[8 * c + q] = dh[q] * k4[q];               // the direct path; the gate paths are added below
      }
      const uint4 pu = pack8_bf16(gu), pr = pack8_bf16(gr), pq = pack8_bf16(gq), pc = pack8_bf16(gc);
      *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, u, 3 * D)) = pu;
      *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, D + u, 3 * D)) = pr;
      *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, 2 * D + u, 3 * D)) = pq;
      *reinterpret_cast<uint4*>(a.g1 + tape_off(cell, u, 128, nkb)) = pu;
      *reinterpret_cast<uint4*>(a.g1 + tape_off(cell, D + u, 128, nkb)) = pr;
      *reinterpret_cast<uint4*>(a.g1 + tape_off(cell, 2 * D + u, 128, nkb)) = pq;
      *reinterpret_cast<uint4*>(a.g1 + tape_off(cell, 3 * D + u, 128, nkb)) = pc;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
      // dh_{n-1} through the gates: G[:, :3D] W3, N = D
      constexpr uint32_t idesc = tc::make_idesc_bf16(128, D);
      constexpr uint32_t sbo = (3 * D / 8) * 128;
#pragma unroll
      for (int k = 0; k < 3 * D / 16; ++k)
        tc::mma_bf16(tbase, tc::make_desc(tc::smem_addr(sA) + k * 256, 128, sbo),
                     tc::make_desc(tc::smem_addr(sW3) + k * 256, 128, sbo), idesc, k > 0);
      tc::mma_commit(&mbar[0]);
    }
    if (!tc::mbar_wait(&mbar[0], ph, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    ph ^= 1;
    tc::fence_after_sync();
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float v[8];
      tld8_1(trow + u0 + 8 * c, v);
#pragma unroll
      for (int q = 0; q < 8; ++q) carry[8 * c + q] += v[q];
    }
    tc::fence_before_sync();
    __syncthreads();                                   // TMEM read and the A operand free for the next site
    tc::fence_after_sync();
  }
  tc::fence_before_sync();
  if (__syncthreads_or(timed_out) && threadIdx.x == 0) tc::drain_mmas(&mbar[1], tc::kDefaultWaitPolls);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 128);
}

// dU[0] = sum_cells gd h_n, dU[1] = -dU[0], dc = (sum gd, -sum gd): per block a
// fixed range of cells in order; thread k < D sums column k, thread D the gd.
__global__ void __launch_bounds__(160) tc1d128_readout_kernel(const float* __restrict__ hcache,
                                                            const float* __restrict__ gd, int64_t B, int64_t Bp,
                                                            int N, float* __restrict__ part) {
  const int64_t ncell = Bp * N, per = (ncell + gridDim.x - 1) / gridDim.x, c0 = blockIdx.x * per;
  const int64_t c1 = c0 + per < ncell ? c0 + per : ncell;
  const int k = threadIdx.x;
  if (k > D) return;
  float acc = 0.0f;
  for (int64_t c = c0; c < c1; ++c) {
    const int64_t n = c / Bp, b = c % Bp;
    if (b < B) acc = fmaf(gd[c], k < D ? hcache[(b * N + n) * D + k] : 1.0f, acc);
  }
  part[(size_t)blockIdx.x * (D + 1) + k] = acc;
}

// Every flat parameter from the GEMM units' sums (cell ranges in order) and
// the readout blocks' sums.  GEMM tiles: 0 u (W_g, b_g), 1 r (W_r, b_r),
// 2 q (W_h, b_h), 3 c (W_in, b_in); output columns [h_{n-1} (D) | 1 | onehot(s)].
__global__ void tc1d128_final_kernel(const float* __restrict__ wg, int splits, const float* __restrict__ ro, int nro,
                                     float* __restrict__ grad) {
  constexpr int kCols = WgS<128>::kCols;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kP) return;
  int tile = -1, row = 0, col = 0;
  float sign = 1.0f;
  if (i < oWh) {                                   // W_g, W_r [d, d + 2]
    tile = i < oWr ? 0 : 1;
    const int r0 = i - (tile == 0 ? oWg : oWr);
    row = r0 / (D + 2);
    const int cc = r0 % (D + 2);
    col = cc < D ? cc : D + 1 + (cc - D);
  } else if (i < oWin) {                           // W_h [d, d]
    tile = 2;
    row = (i - oWh) / D;
    col = (i - oWh) % D;
  } else if (i < obg) {                            // W_in [d, 2]
    tile = 3;
    row = (i - oWin) / 2;
    col = D + 1 + (i - oWin) % 2;
  } else if (i < oU) {                             // b_g, b_r, b_h, b_in: the ones column
    tile = (i - obg) / D;
    row = (i - obg) % D;
    col = D;
  }
  float s = 0.0f;
  if (tile >= 0) {
    for (int sp = 0; sp < splits; ++sp) s += wg[(((size_t)tile * splits + sp) * 128 + row) * kCols + col];
  } else {                                         // U [2, d], c [2]
    const int k = i < oc ? (i - oU) % D : D;
    sign = (i < oc ? (i - oU) / D : i - oc) == 0 ? 1.0f : -1.0f;
    for (int q = 0; q < nro; ++q) s += ro[(size_t)q * (D + 1) + k];
  }
  grad[i] = sign * s;
}

struct Grad128Layout {
  size_t w3, tape_k, gd, g1, x1a, x1c, wg, ro, total;
};

Grad128Layout grad128_layout(int64_t B, int N) {
  const size_t Bp = (size_t)((B + 127) / 128 * 128), cells = Bp * (size_t)N;
  Grad128Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off += (bytes + 255) / 256 * 256; return at; };
  L.w3 = take((size_t)D * 3 * D * 2);
  L.tape_k = take(cells * 5 * D * 2);
  L.gd = take(cells * 4);
  L.g1 = take(cells * 4 * D * 2);
  L.x1a = take(cells * D * 2);
  L.x1c = take(cells * 16 * 2);
  L.wg = take((size_t)4 * kWgSplits * 128 * WgS<128>::kCols * 4);
  L.ro = take((size_t)kRoBlocks * (D + 1) * 4);
  L.total = off;
  return L;
}

int sm_count_1d128() {
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

}  // namespace

size_t tc1d128_grad_bytes(int64_t B, int N) { return grad128_layout(B, N).total; }

cudaError_t tc1d128_grad(const Tc1WGrad& g, const uint8_t* wimg, float* grad, cudaStream_t st) {
  const Grad128Layout L = grad128_layout(g.B, g.N);
  uint8_t* w = g.scratch;
  const int64_t Bp = (g.B + 127) / 128 * 128, nkb = Bp * g.N / 16;
  cudaError_t e;
  uint8_t* w3 = w + L.w3;
  pack_w3_kernel<<<(D * 3 * D + 255) / 256, 256, 0, st>>>(g.params, w3);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 1. tape pass
  T1Args t{};
  t.B = g.B;
  t.Bp = Bp;
  t.N = g.N;
  t.sigma = g.sigma;
  t.hcache = g.hcache;
  t.weights = g.weights;
  t.params = g.params;
  t.tape_k = reinterpret_cast<__half*>(w + L.tape_k);
  t.gd = reinterpret_cast<float*>(w + L.gd);
  t.x1a = w + L.x1a;
  t.x1c = w + L.x1c;
  t.hdr = g.hdr;
  if ((e = cudaFuncSetAttribute(tc1d128_tape_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, T1S::kBytes)) !=
      cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  const int64_t ntile = (Bp / 128) * g.N;
  const int64_t tgrid = ntile < sm_count_1d128() ? ntile : sm_count_1d128();
  if (tgrid > 0) {
    tc1d128_tape_kernel<<<(unsigned)tgrid, kThreads, T1S::kBytes, st>>>(wimg, t);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 2. sequential sweep
  S1Args s{};
  s.B = g.B;
  s.Bp = Bp;
  s.N = g.N;
  s.params = g.params;
  s.tape_k = t.tape_k;
  s.gd = t.gd;
  s.g1 = w + L.g1;
  s.hdr = g.hdr;
  if ((e = cudaFuncSetAttribute(tc1d128_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, S1S::kBytes)) !=
      cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  if (Bp > 0) {
    tc1d128_sweep_kernel<<<(unsigned)(Bp / 128), kThreads, S1S::kBytes, st>>>(w3, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 3. weight gradients and the readout gradients
  WgArgs wg{};
  for (int q = 0; q < 4; ++q) {
    wg.tiles[q].A = s.g1 + (size_t)q * nkb * 4096;
    wg.tiles[q].Bm = t.x1a;
    wg.tiles[q].Bx = t.x1c;
  }
  wg.nkb = nkb;
  wg.splits = kWgSplits;
  wg.out = reinterpret_cast<float*>(w + L.wg);
  wg.hdr = g.hdr;
  if ((e = launch_wgrad<128>(wg, 4, st)) != cudaSuccess) return e;
  float* ro = reinterpret_cast<float*>(w + L.ro);
  tc1d128_readout_kernel<<<kRoBlocks, 160, 0, st>>>(g.hcache, t.gd, g.B, Bp, g.N, ro);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 4. the flat gradient
  tc1d128_final_kernel<<<(kP + 255) / 256, 256, 0, st>>>(wg.out, kWgSplits, ro, kRoBlocks, grad);
  return cudaGetLastError();
}

cudaError_t tc1d128_set_wait_polls(uint32_t polls) {
  return cudaMemcpyToSymbol(tc::g_wait_polls, &polls, sizeof(polls));
}

}  // namespace nqs

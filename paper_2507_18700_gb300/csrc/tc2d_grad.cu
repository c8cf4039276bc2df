// BF16 tensor-core reverse sweep of the 2D GRU wave function with its GLU head
// (App. A): d/dtheta sum_b w_b log psi_b over the zig-zag order (Sec. II),
// with the zero-magnetisation mask, for d_h in {32, 64} and N <= 256.
//
// Phase 1a, tc2d_tape_kernel, parallel over (tile of 128 samples, position
// t): from the cached states, everything that does not depend on the
// incoming gradient --
//   MMA1: [hi(h') | extras | lo(h')] x W1^T   (the forward's gate pre-activations)
//   MMA2: [hi(h)  | extras | lo(h)]  x W2^T   (the forward's GLU pre-activations)
//   GLU:  y, the logit difference d, dz = c_b (onehot(s) - p0) (0 at a
//         forced site of the mask), G2 = [dy W_1-path | dy W_2-path]
//   MMA_g: dh_glu = G2 W2                     (W2 read as an MN-major operand)
// and the three factors with which the cell backward through
// h = u h~ + (1 - u) U_mix h' is linear in dh: G1 = dh [kW | kg | km].
// dh_glu (FP32) and the factors (FP16) go to a sample-minor tape; G2, dz and
// y go to the images of phases 2 and 3.
// Phase 1b, tc2d_bsweep_kernel, sequential over t = N-1 .. 0 for a tile of
// 128 samples: dh = dh_glu + the carries of the horizontal and vertical
// successors, G1 = dh [kW | kg | km] (BF16, also written as an image),
//   MMA_b: dh' = G1 W1          (W1 read as an MN-major operand)
// dh' splits into the horizontal predecessor's carry (registers) and the
// vertical predecessor's (a per-sample column carry buffer in global memory).
// The forward images hold W_g and W_2 halved (their sigmoids are one tanh);
// G1 and G2 carry those blocks doubled, so both products are exact.
// Phase 2, tc2d_wgrad_kernel: split-K over the (tile, site) images, a CTA
// accumulates dW1 += G1^T X1 and dW2 += G2^T X2 in TMEM (X1 = [h' | 1 |
// one-hots], X2 = [h | 1], built from the cache; both operands MN-major), so
// the ones and one-hot columns give the bias and one-hot-weight gradients.
// Phase 3, tc2d_readout_grad_kernel: dU_out and dc from dz and y.
#include <cuda_fp16.h>

#include "tc2d_common.cuh"

namespace nqs {

namespace {

using namespace tc2dh;

template <int D>
struct G2S {
  static constexpr int K1 = 2 * D + 16, K2 = D + 16;       // weight image columns (as in the forward)
  static constexpr int KA1 = K1 + 2 * D, KA2 = K2 + D;     // A operand columns: [hi | extras | lo]
  static constexpr int GW1 = 4 * D >= 128 ? 4 * D : 128;  // G1 image width (whole 128-row M halves)
  static constexpr int GW2 = 2 * D >= 128 ? 2 * D : 128;  // G2 image width
  static constexpr int kW1 = 0;                            // [3D x K1] bf16
  static constexpr int kW2 = kW1 + 3 * D * K1 * 2;         // [2D x K2] bf16
  static constexpr int kA1 = kW2 + 2 * D * K2 * 2;         // [128 x KA1]; G1 [128 x 3D] aliases it
  static constexpr int kA2 = kA1 + 128 * KA1 * 2;          // [128 x KA2]; G2 [128 x 2D] aliases it
  static constexpr int kAux = kA2 + 128 * KA2 * 2;         // D + 4 floats: U_0 - U_1, c_0 - c_1
  static constexpr int kBar = kAux + (D + 4) * 4;          // 4 mbarrier slots: MMA1+2, MMA_g, -, drain
  static constexpr int kSlot = kBar + 32;
  static constexpr int kBytes = 1024 + kSlot + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
  // TMEM columns: MMA1 [0, 3D), MMA2 and later MMA_b [3D, 5D), MMA_g [5D, 6D)
  static constexpr uint32_t c1 = 0, c2 = 3 * D, cg = 5 * D;
  static_assert(6 * D <= 512, "TMEM budget");
};

struct Sweep2Args {
  int64_t B;
  int Lx, Ly, N, sz0;
  const uint8_t* sigma;
  const float* hcache;
  const float* weights;
  float* ccarry;             // [B, Lx, d] vertical carries
  uint8_t* g1img;            // [tiles, N] images of 128 x GW1 bf16 (padding columns never read back)
  uint8_t* g2img;            // [tiles, N] images of 128 x GW2 bf16 (padding columns never read back)
  float* yimg;               // [tiles, N, d, 128]
  float* dzimg;              // [tiles, N, 128]
  float* tape_h;             // [N][d / 4][B][4] f32: dlog psi / dh through the GLU
  uint8_t* tape_k;           // [N][3][d / 8][B][8] f16: cell-backward factors
  WsHeader* hdr;
};

// 16 values of an FP32 row (16-byte aligned) or zeros
__device__ __forceinline__ void ld16(const float* src, bool ok, float (&v)[16]) {
  if (ok) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 x = reinterpret_cast<const float4*>(src)[q];
      v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = 0.0f;
  }
}

__device__ __forceinline__ void st_bf16_8(uint8_t* dst, const float* v) {
  *reinterpret_cast<uint4*>(dst) = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                              pack_bf16(v[6], v[7]));
}

__device__ __forceinline__ uint4 pack_h8(const float* v) {
  __half2 p0 = __floats2half2_rn(v[0], v[1]);
  __half2 p1 = __floats2half2_rn(v[2], v[3]);
  __half2 p2 = __floats2half2_rn(v[4], v[5]);
  __half2 p3 = __floats2half2_rn(v[6], v[7]);
  return make_uint4(*reinterpret_cast<uint32_t*>(&p0), *reinterpret_cast<uint32_t*>(&p1),
                    *reinterpret_cast<uint32_t*>(&p2), *reinterpret_cast<uint32_t*>(&p3));
}

__device__ __forceinline__ void unpack_h8(uint4 q, float* v) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[i]));
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

// 16-byte cp.async of `bytes` (16 or 0, the rest zero-filled)
__device__ __forceinline__ void cp_async16_z2(void* smem, const void* gmem, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n"
               :
               : "r"(tc::smem_addr(smem)), "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_arrive_noinc2(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" : : "r"(tc::smem_addr(bar)) : "memory");
}

// Tape groups (16 bytes) of sample b at position t: 4 floats of dh_glu, or 8
// halves of factor vector c.
__device__ __forceinline__ int64_t t2h_group(int64_t B, int t, int g4, int64_t b, int D) {
  return ((int64_t)t * (D / 4) + g4) * B + b;
}
__device__ __forceinline__ int64_t t2k_group(int64_t B, int t, int c, int g8, int64_t b, int D) {
  return (((int64_t)t * 3 + c) * (D / 8) + g8) * B + b;
}

// ----------------------------------------------------------------------------
// Phase 1a, the tape: parallel over (tile of 128 samples, position t).  One
// CTA per SM walks runs of consecutive positions of one tile; per cell it
// recomputes the forward pre-activations (MMA1, MMA2 with the hi / lo
// operands, as in the forward), the GLU forward and backward (dz, y, G2; the
// images for the weight gradients), dh_glu = G2 W2 (MMA_g), and the three
// factors of the cell backward, which is linear in dh:
//   G1 = [da_W | 2 da_g | d(U_mix h')] = dh [kW | kg | km],
//   kW = u (1 - c^2),  kg = (c - U_mix h') (1 - tanh^2(a_g)) / 2,  km = 1 - u.
// ----------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(128, 1)
tc2d_tape_kernel(const uint8_t* __restrict__ w1img, const uint8_t* __restrict__ w2img, const float* __restrict__ aux,
                 Sweep2Args a, int sites_per_run, int runs_per_tile) {
  using S = G2S<D>;
  constexpr int K1 = S::K1, K2 = S::K2, KA1 = S::KA1, KA2 = S::KA2;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sW1 = sm + S::kW1;
  uint8_t* sW2 = sm + S::kW2;
  uint8_t* sA1 = sm + S::kA1;
  uint8_t* sA2 = sm + S::kA2;
  float* sAux = reinterpret_cast<float*>(sm + S::kAux);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < 3 * D * K1 * 2 / 16; i += 128)
    reinterpret_cast<uint4*>(sW1)[i] = reinterpret_cast<const uint4*>(w1img)[i];
  for (int i = threadIdx.x; i < 2 * D * K2 * 2 / 16; i += 128)
    reinterpret_cast<uint4*>(sW2)[i] = reinterpret_cast<const uint4*>(w2img)[i];
  for (int i = threadIdx.x; i < D + 1; i += 128) sAux[i] = aux[i];
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) tc::mbar_init(&mbar[q], 1);
    tc::mbar_init(&mbar[3], 1);              // drain (MMA issuer: thread 0)
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int m = threadIdx.x;
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16);
  const int Lx = a.Lx, N = a.N;
  const int64_t B = a.B;
  const float dc = sAux[D];
  const int64_t runs = (B + 127) / 128 * runs_per_tile;
  uint32_t phases = 0;
  bool timed_out = false;
  const uint32_t one = 0x3F80u;
  auto wait = [&](int q) {
    if (!tc::mbar_wait(&mbar[q], (phases >> q) & 1u, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    phases ^= 1u << q;
    tc::fence_after_sync();
  };
  auto sync_tc = [&]() {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  uint4* th = reinterpret_cast<uint4*>(a.tape_h);
  uint4* tk = reinterpret_cast<uint4*>(a.tape_k);
  for (int64_t run = blockIdx.x; run < runs; run += gridDim.x) {
    const int64_t tile = run / runs_per_tile;
    const int t0 = (int)(run % runs_per_tile) * sites_per_run;
    const int t1 = t0 + sites_per_run < N ? t0 + sites_per_run : N;
    if (t0 >= t1) continue;                  // uniform
    const int64_t b = tile * 128 + m;
    const bool valid = b < B;
    const float coef = valid ? 0.5f * a.weights[b] : 0.0f;
    const uint8_t* sg = a.sigma + (valid ? b : 0) * N;
    const float* hc = a.hcache + (valid ? b : 0) * (int64_t)N * D;
    int n_up = 0;                            // up spins before position t
    if (valid)
      for (int t = 0; t < t0; ++t) {
        const Pz q = zpos(t, Lx);
        n_up += sg[q.j * Lx + q.i] ? 0 : 1;
      }
    for (int t = t0; t < t1; ++t) {
      const Pz p = zpos(t, Lx);
      const int k = p.j * Lx + p.i;
      const int s_k = valid ? (sg[k] ? 1 : 0) : 0;
      const int s_h = p.r > 0 ? (valid ? (sg[p.j * Lx + zhor(p)] ? 1 : 0) : 0) : -1;
      const int s_v = p.j > 0 ? (valid ? (sg[(p.j - 1) * Lx + p.i] ? 1 : 0) : 0) : -1;
      // ---- A1 = [hi(h_hor) hi(h_ver) | extras | lo(h_hor) lo(h_ver)], A2 = [hi(h) | 1 1 | lo(h)] ----
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const bool ok = valid && (half == 0 ? p.r > 0 : p.j > 0);
        const float* src =
            hc + (int64_t)(half == 0 ? p.j * Lx + (p.r > 0 ? zhor(p) : 0) : (p.j > 0 ? (p.j - 1) * Lx + p.i : 0)) * D;
        // all loads of the state first (interleaved with the shared stores
        // they would serialise), then its hi / lo rows
        float v[D];
#pragma unroll
        for (int c = 0; c < D / 16; ++c) ld16(src + 16 * c, ok, *reinterpret_cast<float(*)[16]>(v + 16 * c));
#pragma unroll
        for (int c = 0; c < D / 8; ++c)
          st_split8(sA1 + tc::kmajor_offset(m, half * D + 8 * c, KA1), sA1 + tc::kmajor_offset(m, K1 + half * D + 8 * c, KA1),
                    v + 8 * c);
      }
      {
        const uint32_t oh = s_h < 0 ? 0u : (s_h == 0 ? one : (one << 16));
        const uint32_t ov = s_v < 0 ? 0u : (s_v == 0 ? one : (one << 16));
        *reinterpret_cast<uint4*>(sA1 + tc::kmajor_offset(m, 2 * D, KA1)) = make_uint4(one | (one << 16), oh, ov, oh);
        *reinterpret_cast<uint4*>(sA1 + tc::kmajor_offset(m, 2 * D + 8, KA1)) = make_uint4(ov, 0u, 0u, 0u);
      }
      {
        float v[D];
#pragma unroll
        for (int c = 0; c < D / 16; ++c) ld16(hc + (int64_t)k * D + 16 * c, valid, *reinterpret_cast<float(*)[16]>(v + 16 * c));
#pragma unroll
        for (int c = 0; c < D / 8; ++c)
          st_split8(sA2 + tc::kmajor_offset(m, 8 * c, KA2), sA2 + tc::kmajor_offset(m, K2 + 8 * c, KA2), v + 8 * c);
      }
      *reinterpret_cast<uint4*>(sA2 + tc::kmajor_offset(m, D, KA2)) = make_uint4(one | (one << 16), 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(sA2 + tc::kmajor_offset(m, D + 8, KA2)) = make_uint4(0u, 0u, 0u, 0u);
      sync_tc();
      // ---- MMA1, MMA2: the forward pre-activations ----
      if (m == 0) {
        constexpr uint32_t i1 = tc::make_idesc_bf16(128, 3 * D), i2 = tc::make_idesc_bf16(128, 2 * D);
#pragma unroll
        for (int c = 0; c < KA1 / 16; ++c) {
          const int kb = c < K1 / 16 ? c : c - K1 / 16;
          tc::mma_bf16(tbase + S::c1, tc::make_desc(tc::smem_addr(sA1) + c * 256, 128, (KA1 / 8) * 128),
                       tc::make_desc(tc::smem_addr(sW1) + kb * 256, 128, (K1 / 8) * 128), i1, c > 0);
        }
#pragma unroll
        for (int c = 0; c < KA2 / 16; ++c) {
          const int kb = c < K2 / 16 ? c : c - K2 / 16;
          tc::mma_bf16(tbase + S::c2, tc::make_desc(tc::smem_addr(sA2) + c * 256, 128, (KA2 / 8) * 128),
                       tc::make_desc(tc::smem_addr(sW2) + kb * 256, 128, (K2 / 8) * 128), i2, c > 0);
        }
        tc::mma_commit(&mbar[0]);
      }
      wait(0);
      // ---- GLU forward: the logit difference (the engine's readout order) and dz ----
      float zc[D / 16];
#pragma unroll
      for (int c = 0; c < D / 16; ++c) zc[c] = 0.0f;
#pragma unroll
      for (int c = 0; c < D / 8; ++c) {
        uint32_t a1[8], a2[8];
        tld8(trow + S::c2 + 8 * c, a1);
        tld8(trow + S::c2 + D + 8 * c, a2);
        tc::tmem_wait_ld();
        tie(a1);
        tie(a2);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          zc[c / 2] = fmaf(sAux[8 * c + q],
                           __uint_as_float(a1[q]) * fmaf(0.5f, hw_tanh2(__uint_as_float(a2[q])), 0.5f), zc[c / 2]);
      }
#pragma unroll
      for (int w = 1; w < D / 16; w *= 2)
#pragma unroll
        for (int c = 0; c + w < D / 16; c += 2 * w) zc[c] += zc[c + w];
      const float z = zc[0];
      const bool forced = a.sz0 && (n_up >= (N >> 1) || (t - n_up) >= (N >> 1));
      const float dz = (forced || !valid) ? 0.0f : coef * ((s_k == 0 ? 1.0f : 0.0f) - sigmoid_acc(z + dc));
      n_up += (s_k == 0);
      const int64_t img = tile * N + t;
      a.dzimg[img * 128 + m] = dz;
      // ---- GLU backward: G2 = [da_1 | 2 da_2], y for the readout gradient ----
      uint8_t* g2g = a.g2img + (size_t)img * 128 * S::GW2 * 2;
#pragma unroll
      for (int c = 0; c < D / 8; ++c) {
        uint32_t a1[8], a2[8];
        tld8(trow + S::c2 + 8 * c, a1);
        tld8(trow + S::c2 + D + 8 * c, a2);
        tc::tmem_wait_ld();
        tie(a1);
        tie(a2);
        float g1v[8], g2v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int v = 8 * c + q;
          const float x1 = __uint_as_float(a1[q]);
          const float th = hw_tanh2(__uint_as_float(a2[q]));
          const float sg2 = fmaf(0.5f, th, 0.5f);
          const float dy = dz * sAux[v];
          g1v[q] = dy * sg2;                                   // d a_1
          g2v[q] = 2.0f * dy * x1 * (0.25f * fmaf(-th, th, 1.0f));   // 2 d a_2 (W_2 halved in the image)
          a.yimg[(img * D + v) * 128 + m] = x1 * sg2;
        }
        st_bf16_8(sA2 + tc::kmajor_offset(m, 8 * c, 2 * D), g1v);
        st_bf16_8(sA2 + tc::kmajor_offset(m, D + 8 * c, 2 * D), g2v);
        st_bf16_8(g2g + tc::kmajor_offset(m, 8 * c, S::GW2), g1v);
        st_bf16_8(g2g + tc::kmajor_offset(m, D + 8 * c, S::GW2), g2v);
      }
      sync_tc();
      // ---- MMA_g: dh (from the GLU) = G2 W2 ----
      if (m == 0) {
        constexpr uint32_t ig = tc::make_idesc_bf16(128, D) | (1u << 16);   // B MN-major
#pragma unroll
        for (int c = 0; c < 2 * D / 16; ++c)
          tc::mma_bf16(tbase + S::cg, tc::make_desc(tc::smem_addr(sA2) + c * 256, 128, (2 * D / 8) * 128),
                       tc::make_desc(tc::smem_addr(sW2) + c * 2 * (K2 / 8) * 128, (K2 / 8) * 128, 128), ig, c > 0);
        tc::mma_commit(&mbar[1]);
      }
      // ---- the cell factors, under MMA_g ----
#pragma unroll
      for (int c = 0; c < D / 8; ++c) {
        uint32_t aw[8], ag[8], au[8];
        tld8(trow + S::c1 + 8 * c, aw);
        tld8(trow + S::c1 + D + 8 * c, ag);
        tld8(trow + S::c1 + 2 * D + 8 * c, au);
        tc::tmem_wait_ld();
        tie(aw);
        tie(ag);
        tie(au);
        float kw[8], kg[8], km[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float cc_ = hw_tanh2(__uint_as_float(aw[q]));
          const float tg = hw_tanh2(__uint_as_float(ag[q]));
          const float ug = fmaf(0.5f, tg, 0.5f);
          kw[q] = ug * fmaf(-cc_, cc_, 1.0f);                               // u (1 - c^2)
          kg[q] = (cc_ - __uint_as_float(au[q])) * (0.5f * fmaf(-tg, tg, 1.0f));   // 2 (c - mix) u (1 - u)
          km[q] = 0.5f - 0.5f * tg;                                         // 1 - u
        }
        if (valid) {
          tk[t2k_group(B, t, 0, c, b, D)] = pack_h8(kw);
          tk[t2k_group(B, t, 1, c, b, D)] = pack_h8(kg);
          tk[t2k_group(B, t, 2, c, b, D)] = pack_h8(km);
        }
      }
      wait(1);
#pragma unroll
      for (int c = 0; c < D / 8; ++c) {
        uint32_t gh[8];
        tld8(trow + S::cg + 8 * c, gh);
        tc::tmem_wait_ld();
        tie(gh);
        if (valid) {
          th[t2h_group(B, t, 2 * c, b, D)] = make_uint4(gh[0], gh[1], gh[2], gh[3]);
          th[t2h_group(B, t, 2 * c + 1, b, D)] = make_uint4(gh[4], gh[5], gh[6], gh[7]);
        }
      }
      // TMEM and the operand tiles are free for the next cell
      tc::fence_before_sync();
      if (__syncthreads_or(timed_out)) { timed_out = true; break; }
      tc::fence_after_sync();
    }
    if (timed_out) break;                   // uniform
  }
  tc::fence_before_sync();
  // after a wait that gave up, TMEM is freed only once the MMAs have drained
  if (__syncthreads_or(timed_out) && threadIdx.x == 0) tc::drain_mmas(&mbar[3], kWait2);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 512);
}

// ----------------------------------------------------------------------------
// Phase 1b, the sequential sweep: one CTA per tile of 128 samples, SPLIT
// threads per sample on D / SPLIT units each, positions N-1 .. 0.  Per cell
//   dh = dh_glu + carry (horizontal successor) + cv (vertical successor)
//   G1 = dh [kW | kg | km] (BF16; also the image for the weight gradients)
//   MMA_b: dh' = G1 W1 (W1 read as an MN-major operand; three K chains, one
//          per gate block, summed on read)
// dh' splits into the horizontal predecessor's carry (registers) and the
// vertical predecessor's (a per-sample column carry in global memory, which
// only the thread owning those units reads and writes).  The tape of the
// next cell arrives by cp.async while a cell runs.
// ----------------------------------------------------------------------------
template <int D, int SPLIT, int ROWS>
struct B2S {
  static constexpr int K1 = 2 * D + 16;                    // W1 image columns
  static constexpr int GW1 = 4 * D >= 128 ? 4 * D : 128;  // G1 image width
  static constexpr int RQ = ROWS / 32;                     // TMEM lane quarters holding distinct samples
  static constexpr int NS = (4 / RQ) * SPLIT;              // unit slices per sample
  static constexpr int DU = D / NS;                        // units per thread
  static constexpr int NG = D / 4 + 3 * D / 8;             // 16-byte tape groups per sample
  static constexpr int CS = D + 4;                         // exchange row stride (floats)
  static constexpr int kW1 = 0;                            // [3D x K1] bf16
  static constexpr int kA1 = kW1 + 3 * D * K1 * 2;         // [128 x 3D] bf16 (G1; rows past ROWS unused)
  static constexpr int kT = kA1 + 128 * 3 * D * 2;         // [NG][ROWS] x 16 B tape of one cell
  static constexpr int kC = kT + NG * ROWS * 16;           // 2 x [ROWS x CS] f32 (ROWS < 128)
  static constexpr int kBar = kC + (ROWS < 128 ? 2 * ROWS * CS * 4 : 0);   // 4 mbarriers (the last: drain)
  static constexpr int kSlot = kBar + 32;
  static constexpr int kBytes = 1024 + kSlot + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
  static_assert(6 * D <= 512, "TMEM budget");
  static_assert(DU >= 8 && DU % 8 == 0 && ROWS % 32 == 0 && ROWS <= 128, "tile shape");
};

// Thread -> (sample, unit slice): warp w is in TMEM lane quarter q = w % 4;
// quarters q % RQ hold distinct samples s = 32 (q % RQ) + lane and split its
// units with the SPLIT warps of a quarter into NS slices.  With ROWS < 128
// the quarters that own the samples' lanes pass dh' on through shared memory.
template <int D, int SPLIT, int ROWS>
__global__ void __launch_bounds__(128 * SPLIT, 1)
tc2d_bsweep_kernel(const uint8_t* __restrict__ w1img, Sweep2Args a) {
  using S = B2S<D, SPLIT, ROWS>;
  constexpr int NT = 128 * SPLIT, DU = S::DU, K1 = S::K1, RQ = S::RQ, CS = S::CS;
  constexpr bool XCH = ROWS < 128;         // carries exchanged through shared memory
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sW1 = sm + S::kW1;
  uint8_t* sA1 = sm + S::kA1;
  uint8_t* sT = sm + S::kT;
  float* sCh = reinterpret_cast<float*>(sm + S::kC);
  float* sCv = sCh + ROWS * CS;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < 3 * D * K1 * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sW1)[i] = reinterpret_cast<const uint4*>(w1img)[i];
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);              // MMA_b, horizontal half, done
    tc::mbar_init(&mbar[1], NT);             // tape of the cell in place
    tc::mbar_init(&mbar[2], 1);              // MMA_b, vertical half, done
    tc::mbar_init(&mbar[3], 1);              // drain (MMA issuer: thread 0)
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int lane = threadIdx.x & 31, wt = threadIdx.x >> 5, q4 = wt % 4, p = wt / 4;
  const int s = 32 * (q4 % RQ) + lane;     // sample row of the tile (and its TMEM lane)
  const int u0 = ((q4 / RQ) * SPLIT + p) * DU;
  const bool owner = q4 < RQ;              // this warp's TMEM lanes are its samples'
  constexpr int CW = D / SPLIT;            // columns an owner moves in an exchange
  const uint32_t trow = tbase + ((uint32_t)(32 * q4) << 16);
  const int Lx = a.Lx, Ly = a.Ly, N = a.N;
  const int64_t B = a.B;
  const int64_t b = (int64_t)blockIdx.x * ROWS + s;
  const bool valid = b < B;
  // the G1 image of the 128-sample tile holding this sample
  const int64_t itile = ((int64_t)blockIdx.x * ROWS) / 128;
  const int irow = (int)(((int64_t)blockIdx.x * ROWS) % 128) + s;
  float* ccb = a.ccarry + (valid ? b : 0) * (int64_t)Lx * D;
  // tape groups: dh_glu group g at th_b + t GH + g B, factor vector c group g
  // at tk_b + (3 t + c) GK + g B
  const int64_t GH = (int64_t)(D / 4) * B, GK = (int64_t)(D / 8) * B;
  const uint4* th_b = reinterpret_cast<const uint4*>(a.tape_h) + (valid ? b + (int64_t)(u0 / 4) * B : 0);
  const uint4* tk_b = reinterpret_cast<const uint4*>(a.tape_k) + (valid ? b + (int64_t)(u0 / 8) * B : 0);
  uint32_t phases = 0;
  bool timed_out = false;
  auto wait = [&](int q) {
    if (!tc::mbar_wait(&mbar[q], (phases >> q) & 1u, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    phases ^= 1u << q;
    tc::fence_after_sync();
  };
  auto sync = [&]() {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  };
  // this thread's groups of the tape at position t (zeros past the batch)
  auto fetch = [&](int t) {
    const uint32_t n = valid ? 16u : 0u;
    const uint4* h = th_b + (valid ? t * GH : 0);
    const uint4* k = tk_b + (valid ? 3 * t * GK : 0);
#pragma unroll
    for (int g = 0; g < DU / 4; ++g)
      cp_async16_z2(sT + ((u0 / 4 + g) * ROWS + s) * 16, h + (valid ? g * B : 0), n);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int g = 0; g < DU / 8; ++g)
        cp_async16_z2(sT + ((D / 4 + c * (D / 8) + u0 / 8 + g) * ROWS + s) * 16, k + (valid ? c * GK + g * B : 0), n);
    cp_arrive_noinc2(&mbar[1]);
  };
  // dh' = G1 W1 in six accumulators: three K chains (one per gate block) for
  // each of its halves, the horizontal predecessor's [0, D) (needed at once)
  // and the vertical predecessor's [D, 2D) (needed a row later; its MMAs run
  // under the next cell)
  auto tmem_sum3 = [&](int col, float (&v)[8]) {
    uint32_t r0[8], r1[8], r2[8];
    tld8(trow + col, r0);
    tld8(trow + D + col, r1);
    tld8(trow + 2 * D + col, r2);
    tc::tmem_wait_ld();
    tie(r0);
    tie(r1);
    tie(r2);
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = (__uint_as_float(r0[i]) + __uint_as_float(r1[i])) + __uint_as_float(r2[i]);
  };
  float carry[DU], cv[DU];                 // dh' of the horizontal and the vertical successor
#pragma unroll
  for (int u = 0; u < DU; ++u) carry[u] = cv[u] = 0.0f;   // the last cell has no successors
  fetch(N - 1);
  for (int t = N - 1; t >= 0; --t) {
    const Pz pz = zpos(t, Lx);
    wait(1);
    // this thread's tape groups into registers; the buffer then takes the
    // next cell's tape, whose copy runs under the rest of this cell
    uint4 th4[DU / 4], tk4[3][DU / 8];
#pragma unroll
    for (int g = 0; g < DU / 4; ++g) th4[g] = *reinterpret_cast<const uint4*>(sT + ((u0 / 4 + g) * ROWS + s) * 16);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int g = 0; g < DU / 8; ++g)
        tk4[c][g] = *reinterpret_cast<const uint4*>(sT + ((D / 4 + c * (D / 8) + u0 / 8 + g) * ROWS + s) * 16);
    if (t > 0) fetch(t - 1);
    if (t < N - 1) {
      // the vertical half of cell t + 1: G1 is free again, and its dh' goes
      // to the column carry of (i, j - 1), or straight into this cell when
      // this cell is that predecessor
      const Pz p1 = zpos(t + 1, Lx);
      const bool here = pz.j < Ly - 1 && zsnake(pz.i, pz.j + 1, Lx) == t + 1;   // uniform
      if (!XCH) {
        wait(2);
#pragma unroll
        for (int c = 0; c < DU / 8; ++c) {
          float hv[8];
          tmem_sum3(3 * D + u0 + 8 * c, hv);
          if (valid && p1.j > 0) {
            float4* dst = reinterpret_cast<float4*>(ccb + p1.i * D + u0 + 8 * c);
            dst[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
            dst[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
          }
          if (here) {
#pragma unroll
            for (int i = 0; i < 8; ++i) cv[8 * c + i] = hv[i];
          }
        }
      } else {
        if (owner) {
          wait(2);
#pragma unroll
          for (int c = 0; c < CW / 8; ++c) {
            float hv[8];
            tmem_sum3(3 * D + p * CW + 8 * c, hv);
            if (valid && p1.j > 0) {
              float4* dst = reinterpret_cast<float4*>(ccb + p1.i * D + p * CW + 8 * c);
              dst[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
              dst[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
            }
            if (here) {
              float4* dst = reinterpret_cast<float4*>(sCv + s * CS + p * CW + 8 * c);
              dst[0] = make_float4(hv[0], hv[1], hv[2], hv[3]);
              dst[1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
            }
          }
        }
        // G1 is rewritten below (the MMAs have read it), and the column
        // carries and the exchange are published
        sync();
        if (here) {
#pragma unroll
          for (int c = 0; c < DU / 4; ++c) {
            const float4 x = reinterpret_cast<const float4*>(sCv + s * CS + u0)[c];
            cv[4 * c] = x.x; cv[4 * c + 1] = x.y; cv[4 * c + 2] = x.z; cv[4 * c + 3] = x.w;
          }
        }
      }
    }
    // ---- G1 = dh [kW | kg | km], 8 units at a time ----
    uint8_t* g1g = a.g1img + (size_t)(itile * N + t) * 128 * S::GW1 * 2;
#pragma unroll
    for (int sc = 0; sc < DU / 8; ++sc) {
      const int cu = u0 + 8 * sc;
      float hg[8], kw[8], kg[8], km[8];
      {
        const uint4 x0 = th4[2 * sc], x1 = th4[2 * sc + 1];
        hg[0] = __uint_as_float(x0.x); hg[1] = __uint_as_float(x0.y); hg[2] = __uint_as_float(x0.z);
        hg[3] = __uint_as_float(x0.w); hg[4] = __uint_as_float(x1.x); hg[5] = __uint_as_float(x1.y);
        hg[6] = __uint_as_float(x1.z); hg[7] = __uint_as_float(x1.w);
      }
      unpack_h8(tk4[0][sc], kw);
      unpack_h8(tk4[1][sc], kg);
      unpack_h8(tk4[2][sc], km);
      float gw[8], gg[8], gm[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int j = 8 * sc + i;
        const float dh = hg[i] + carry[j] + cv[j];
        gw[i] = dh * kw[i];
        gg[i] = dh * kg[i];
        gm[i] = dh * km[i];
      }
      st_bf16_8(sA1 + tc::kmajor_offset(s, cu, 3 * D), gw);
      st_bf16_8(sA1 + tc::kmajor_offset(s, D + cu, 3 * D), gg);
      st_bf16_8(sA1 + tc::kmajor_offset(s, 2 * D + cu, 3 * D), gm);
      // the image for the weight gradients (its padding columns 3D .. GW1 are
      // never written: they only feed accumulator rows that are not read)
      st_bf16_8(g1g + tc::kmajor_offset(irow, cu, S::GW1), gw);
      st_bf16_8(g1g + tc::kmajor_offset(irow, D + cu, S::GW1), gg);
      st_bf16_8(g1g + tc::kmajor_offset(irow, 2 * D + cu, S::GW1), gm);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    if (__syncthreads_or(timed_out)) { timed_out = true; break; }
    tc::fence_after_sync();
    // ---- MMA_b: the horizontal half, then the vertical half ----
    if (threadIdx.x == 0) {
      constexpr uint32_t ib = tc::make_idesc_bf16(128, D) | (1u << 16);   // B MN-major, N = D
#pragma unroll
      for (int half = 0; half < 2; ++half) {
#pragma unroll
        for (int kk = 0; kk < D / 16; ++kk)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const int c = j * (D / 16) + kk;
            tc::mma_bf16(tbase + half * 3 * D + j * D,
                         tc::make_desc(tc::smem_addr(sA1) + c * 256, 128, (3 * D / 8) * 128),
                         tc::make_desc(tc::smem_addr(sW1) + c * 2 * (K1 / 8) * 128 + half * (D / 8) * 128,
                                       (K1 / 8) * 128, 128),
                         ib, kk > 0);
          }
        tc::mma_commit(&mbar[half ? 2 : 0]);
      }
    }
    // the vertical carry into cell t - 1 from global memory (written when its
    // vertical successor's MMAs completed, published by the barrier above),
    // unless that successor is this cell (then it is taken at the next cell)
    const Pz pq = zpos(t > 0 ? t - 1 : 0, Lx);
    const bool from_mem = valid && t > 0 && pq.j < Ly - 1 && zsnake(pq.i, pq.j + 1, Lx) != t;
    float cv1[DU];
    if (from_mem) {
#pragma unroll
      for (int c = 0; c < DU / 4; ++c) {
        const float4 x = reinterpret_cast<const float4*>(ccb + pq.i * D + u0)[c];
        cv1[4 * c] = x.x; cv1[4 * c + 1] = x.y; cv1[4 * c + 2] = x.z; cv1[4 * c + 3] = x.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < DU; ++c) cv1[c] = 0.0f;
    }
    // ---- the horizontal predecessor's carry (t - 1 in the same row) ----
    if (!XCH) {
      wait(0);
#pragma unroll
      for (int c = 0; c < DU / 8; ++c) {
        float hh[8];
        tmem_sum3(u0 + 8 * c, hh);
#pragma unroll
        for (int i = 0; i < 8; ++i) carry[8 * c + i] = pz.r > 0 ? hh[i] : 0.0f;
      }
    } else {
      if (owner) {
        wait(0);
#pragma unroll
        for (int c = 0; c < CW / 8; ++c) {
          float hh[8];
          tmem_sum3(p * CW + 8 * c, hh);
          float4* dst = reinterpret_cast<float4*>(sCh + s * CS + p * CW + 8 * c);
          dst[0] = make_float4(hh[0], hh[1], hh[2], hh[3]);
          dst[1] = make_float4(hh[4], hh[5], hh[6], hh[7]);
        }
      }
      sync();
#pragma unroll
      for (int c = 0; c < DU / 4; ++c) {
        const float4 x = reinterpret_cast<const float4*>(sCh + s * CS + u0)[c];
        carry[4 * c] = pz.r > 0 ? x.x : 0.0f;
        carry[4 * c + 1] = pz.r > 0 ? x.y : 0.0f;
        carry[4 * c + 2] = pz.r > 0 ? x.z : 0.0f;
        carry[4 * c + 3] = pz.r > 0 ? x.w : 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < DU; ++u) cv[u] = cv1[u];
  }
  if (!timed_out && (!XCH || owner)) wait(2);   // the last vertical half, before TMEM is freed
  asm volatile("cp.async.wait_all;\n" ::: "memory");   // copies in flight after a timeout
  tc::fence_before_sync();
  // after a wait that gave up, TMEM is freed only once the MMAs have drained
  if (__syncthreads_or(timed_out) && threadIdx.x == 0) tc::drain_mmas(&mbar[3], kWait2);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 512);
}

// ----------------------------------------------------------------------------
// Phase 2: weight gradients from the G images, split over CTAs by image.
// ----------------------------------------------------------------------------
template <int D>
struct W2S {
  static constexpr int K1 = 2 * D + 16, K2 = D + 16;
  static constexpr int GW1 = G2S<D>::GW1, GW2 = G2S<D>::GW2;
  static constexpr int H1 = GW1 / 128;                     // 128-row halves of the gate rows of W1
  static constexpr int kG1 = 0;                            // [128 x GW1] bf16
  static constexpr int kG2 = kG1 + 128 * GW1 * 2;          // [128 x GW2] bf16
  static constexpr int kX1 = kG2 + 128 * GW2 * 2;          // [128 x K1] bf16
  static constexpr int kX2 = kX1 + 128 * K1 * 2;           // [128 x K2] bf16
  static constexpr int kBar = kX2 + 128 * K2 * 2;          // 2 mbarriers: MMA, drain
  static constexpr int kSlot = kBar + 16;
  static constexpr int kBytes = 1024 + kSlot + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
  static constexpr uint32_t cW1 = 0, cW2 = H1 * K1;        // TMEM accumulators
  static_assert(H1 * K1 + K2 <= 512, "TMEM budget");
};

struct Wgrad2Args {
  int64_t B;
  int Lx, N, P, tiles;
  const uint8_t* sigma;
  const float* hcache;
  const uint8_t* g1img;
  const uint8_t* g2img;
  float* partial;            // one row per CTA
  WsHeader* hdr;
};

template <int D>
__global__ void __launch_bounds__(128, 1) tc2d_wgrad_kernel(Wgrad2Args a) {
  using S = W2S<D>;
  constexpr int K1 = S::K1, K2 = S::K2, GW1 = S::GW1, GW2 = S::GW2;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sG1 = sm + S::kG1;
  uint8_t* sG2 = sm + S::kG2;
  uint8_t* sX1 = sm + S::kX1;
  uint8_t* sX2 = sm + S::kX2;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);              // drain (MMA issuer: thread 0)
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int m = threadIdx.x;
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16);
  const int Lx = a.Lx, N = a.N;
  const int64_t nimg = (int64_t)a.tiles * N;
  const int64_t i0 = nimg * blockIdx.x / gridDim.x, i1 = nimg * (blockIdx.x + 1) / gridDim.x;
  const uint32_t one = 0x3F80u;
  uint32_t ph = 0;
  bool timed_out = false;
  for (int64_t im = i0; im < i1 && !timed_out; ++im) {
    const int64_t tile = im / N;
    const int t = (int)(im % N);
    const int64_t b = tile * 128 + m;
    const bool valid = b < a.B;
    const Pz p = zpos(t, Lx);
    const uint8_t* sg = a.sigma + (valid ? b : 0) * N;
    const float* hc = a.hcache + (valid ? b : 0) * (int64_t)N * D;
    // G images (this thread copies a 1/128 share of each), asynchronously:
    // they land while the X operands are built
    const uint4* g1 = reinterpret_cast<const uint4*>(a.g1img + (size_t)im * 128 * GW1 * 2);
    const uint4* g2 = reinterpret_cast<const uint4*>(a.g2img + (size_t)im * 128 * GW2 * 2);
    for (int q = m; q < 128 * GW1 * 2 / 16; q += 128) cp_async16_cg(reinterpret_cast<uint4*>(sG1) + q, g1 + q);
    for (int q = m; q < 128 * GW2 * 2 / 16; q += 128) cp_async16_cg(reinterpret_cast<uint4*>(sG2) + q, g2 + q);
    cp_commit_2d();
    // X1 = [h_hor | h_ver | 1 1 | onehot(s_hor) onehot(s_ver) x2 | 0], X2 = [h | 1 1 | 0]
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const bool ok = valid && (half == 0 ? p.r > 0 : p.j > 0);
      const float* src = hc + (int64_t)(half == 0 ? p.j * Lx + (p.r > 0 ? zhor(p) : 0) : (p.j > 0 ? (p.j - 1) * Lx + p.i : 0)) * D;
      // all loads of the state first (interleaved with the shared stores
      // they would serialise), then the BF16 rows
      float v[D];
#pragma unroll
      for (int c = 0; c < D / 16; ++c) ld16(src + 16 * c, ok, *reinterpret_cast<float(*)[16]>(v + 16 * c));
#pragma unroll
      for (int c = 0; c < D / 8; ++c) st_bf16_8(sX1 + tc::kmajor_offset(m, half * D + 8 * c, K1), v + 8 * c);
    }
    {
      const int s_h = p.r > 0 ? (valid ? (sg[p.j * Lx + zhor(p)] ? 1 : 0) : 0) : -1;
      const int s_v = p.j > 0 ? (valid ? (sg[(p.j - 1) * Lx + p.i] ? 1 : 0) : 0) : -1;
      const uint32_t oh = s_h < 0 ? 0u : (s_h == 0 ? one : (one << 16));
      const uint32_t ov = s_v < 0 ? 0u : (s_v == 0 ? one : (one << 16));
      *reinterpret_cast<uint4*>(sX1 + tc::kmajor_offset(m, 2 * D, K1)) = make_uint4(one | (one << 16), oh, ov, oh);
      *reinterpret_cast<uint4*>(sX1 + tc::kmajor_offset(m, 2 * D + 8, K1)) = make_uint4(ov, 0u, 0u, 0u);
    }
    {
      float v[D];
#pragma unroll
      for (int c = 0; c < D / 16; ++c)
        ld16(hc + (int64_t)(p.j * Lx + p.i) * D + 16 * c, valid, *reinterpret_cast<float(*)[16]>(v + 16 * c));
#pragma unroll
      for (int c = 0; c < D / 8; ++c) st_bf16_8(sX2 + tc::kmajor_offset(m, 8 * c, K2), v + 8 * c);
    }
    *reinterpret_cast<uint4*>(sX2 + tc::kmajor_offset(m, D, K2)) = make_uint4(one | (one << 16), 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(sX2 + tc::kmajor_offset(m, D + 8, K2)) = make_uint4(0u, 0u, 0u, 0u);
    cp_wait_2d();
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (m == 0) {
      // both operands MN-major: rows = the tile's 128 samples (K), columns = gate rows (M) / inputs (N)
      constexpr uint32_t iw1 = tc::make_idesc_bf16(128, K1) | (1u << 15) | (1u << 16);
      constexpr uint32_t iw2 = tc::make_idesc_bf16(128, K2) | (1u << 15) | (1u << 16);
      const uint32_t acc0 = im > i0 ? 1u : 0u;
#pragma unroll
      for (int h = 0; h < S::H1; ++h)
#pragma unroll
        for (int c = 0; c < 128 / 16; ++c)
          tc::mma_bf16(tbase + S::cW1 + h * K1,
                       tc::make_desc(tc::smem_addr(sG1) + h * 16 * 128 + c * 2 * (GW1 / 8) * 128, (GW1 / 8) * 128, 128),
                       tc::make_desc(tc::smem_addr(sX1) + c * 2 * (K1 / 8) * 128, (K1 / 8) * 128, 128), iw1,
                       acc0 | (c > 0));
#pragma unroll
      for (int c = 0; c < 128 / 16; ++c)
        tc::mma_bf16(tbase + S::cW2, tc::make_desc(tc::smem_addr(sG2) + c * 2 * (GW2 / 8) * 128, (GW2 / 8) * 128, 128),
                     tc::make_desc(tc::smem_addr(sX2) + c * 2 * (K2 / 8) * 128, (K2 / 8) * 128, 128), iw2,
                     acc0 | (c > 0));
      tc::mma_commit(&mbar[0]);
    }
    if (!tc::mbar_wait(&mbar[0], ph, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    ph ^= 1;
    tc::fence_after_sync();
    // the shared images are rewritten for the next image; a wait that gave up
    // anywhere ends the loop for every thread (the drain below)
    if (__syncthreads_or(timed_out)) timed_out = true;
  }
  tc::fence_before_sync();
  if (timed_out && threadIdx.x == 0) tc::drain_mmas(&mbar[1], kWait2);
  __syncthreads();
  tc::fence_after_sync();
  // ---- this CTA's partial gradient row (flat 2D layout, App. A; nqs.h) ----
  const int W2c = 2 * D + 4;
  const int oW = 0, oWg = D * W2c, oU = 2 * D * W2c, ob = oU + 2 * D * D, obg = ob + D, oW1 = obg + D,
            ob1 = oW1 + D * D, oW2 = ob1 + D, ob2 = oW2 + D * D;
  float* part = a.partial + (size_t)blockIdx.x * a.P;
  if (i1 > i0) {
#pragma unroll 1
    for (int h = 0; h < S::H1; ++h) {
      const int gu = h * 128 + m, g = gu / D, u = gu % D;
#pragma unroll 1
      for (int c0 = 0; c0 < K1; c0 += 16) {
        float v[16];
        tc::tmem_ld16(trow + S::cW1 + h * K1 + c0, v);
        tc::tmem_wait_ld();
        if (gu >= 3 * D) continue;
        const float sc = g == 1 ? 0.5f : 1.0f;   // G1 carries 2 d a_g
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int k = c0 + q;
          const float x = sc * v[q];
          if (k < 2 * D) {
            part[(g == 0 ? oW + u * W2c : g == 1 ? oWg + u * W2c : oU + u * 2 * D) + k] = x;
          } else if (g < 2) {
            if (k == 2 * D) part[(g == 0 ? ob : obg) + u] = x;
            else if (k >= 2 * D + 2 && k < 2 * D + 6) part[(g == 0 ? oW : oWg) + u * W2c + 2 * D + (k - 2 * D - 2)] = x;
          }
        }
      }
    }
    {
      const int g = m / D, v = m % D;
#pragma unroll 1
      for (int c0 = 0; c0 < K2; c0 += 16) {
        float w[16];
        tc::tmem_ld16(trow + S::cW2 + c0, w);
        tc::tmem_wait_ld();
        if (m >= 2 * D) continue;
        const float sc = g == 1 ? 0.5f : 1.0f;   // G2 carries 2 d a_2
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int k = c0 + q;
          if (k < D) part[(g == 0 ? oW1 : oW2) + v * D + k] = sc * w[q];
          else if (k == D) part[(g == 0 ? ob1 : ob2) + v] = sc * w[q];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 512);
}

// Phase 3: dU_out[0][v] = sum dz y_v, dU_out[1] = -dU_out[0], dc_0 = sum dz,
// dc_1 = -dc_0; one partial row per block, images split over the blocks.
template <int D>
__global__ void __launch_bounds__(128) tc2d_readout_grad_kernel(const float* __restrict__ yimg,
                                                              const float* __restrict__ dzimg, int64_t nimg,
                                                              float* __restrict__ partial, int P, int row0) {
  __shared__ float red[4][D + 1];
  const int m = threadIdx.x, lane = m & 31, warp = m >> 5;
  const int64_t i0 = nimg * blockIdx.x / gridDim.x, i1 = nimg * (blockIdx.x + 1) / gridDim.x;
  float acc[D];
#pragma unroll
  for (int v = 0; v < D; ++v) acc[v] = 0.0f;
  float accd = 0.0f;
  for (int64_t im = i0; im < i1; ++im) {
    const float z = dzimg[im * 128 + m];
    accd += z;
#pragma unroll
    for (int v = 0; v < D; ++v) acc[v] = fmaf(z, yimg[(im * D + v) * 128 + m], acc[v]);
  }
#pragma unroll
  for (int v = 0; v < D; ++v) {
    float x = acc[v];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[warp][v] = x;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) accd += __shfl_xor_sync(0xffffffffu, accd, off);
  if (lane == 0) red[warp][D] = accd;
  __syncthreads();
  const int W2c = 2 * D + 4;
  const int oUo = 2 * D * W2c + 2 * D * D + 2 * D + 2 * D * D + 2 * D, oc = oUo + 2 * D;
  float* part = partial + (size_t)(row0 + blockIdx.x) * P;
  for (int v = m; v <= D; v += 128) {
    const float s = (red[0][v] + red[1][v]) + (red[2][v] + red[3][v]);
    if (v < D) {
      part[oUo + v] = s;
      part[oUo + D + v] = -s;
    } else {
      part[oc] = s;
      part[oc + 1] = -s;
    }
  }
}

int sm_count_g() {
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

constexpr int kReadout2Blocks = 152;

template <int D, int SPLIT, int ROWS>
cudaError_t launch_bsweep(int64_t B, const uint8_t* w1, const Sweep2Args& s, cudaStream_t st) {
  using S = B2S<D, SPLIT, ROWS>;
  auto k = tc2d_bsweep_kernel<D, SPLIT, ROWS>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  // whole 128-sample tiles, so that every row of the weight-gradient images
  // is written (zeros past the batch)
  k<<<(unsigned)((B + 127) / 128 * (128 / ROWS)), 128 * SPLIT, S::kBytes, st>>>(w1, s);
  return cudaGetLastError();
}

template <int D>
cudaError_t run_grad(const Tc2Grad& g, const uint8_t* wimg, cudaStream_t st) {
  const int tiles = (int)((g.B + 127) / 128);
  const int64_t nimg = (int64_t)tiles * g.N;
  const uint8_t* w1 = wimg;
  const uint8_t* w2 = w1 + (size_t)3 * D * (2 * D + 16) * 2;
  const float* aux = reinterpret_cast<const float*>(w2 + (size_t)2 * D * (D + 16) * 2);
  Sweep2Args s{};
  s.B = g.B;
  s.Lx = g.Lx;
  s.Ly = g.Ly;
  s.N = g.N;
  s.sz0 = g.sz0;
  s.sigma = g.sigma;
  s.hcache = g.hcache;
  s.weights = g.weights;
  s.ccarry = g.ccarry;
  s.g1img = g.g1img;
  s.g2img = g.g2img;
  s.yimg = g.yimg;
  s.dzimg = g.dzimg;
  s.tape_h = g.tape_h;
  s.tape_k = g.tape_k;
  s.hdr = g.hdr;
  // the tape: one CTA per SM, runs of consecutive positions of one tile
  const int sms = sm_count_g();
  const int runs_per_tile = tiles >= sms ? 1 : sms / tiles;
  const int sites_per_run = (g.N + runs_per_tile - 1) / runs_per_tile;
  int64_t tgrid = (int64_t)tiles * runs_per_tile;
  if (tgrid > sms) tgrid = sms;
  auto kt = tc2d_tape_kernel<D>;
  cudaError_t e = cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, G2S<D>::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  kt<<<(unsigned)tgrid, 128, G2S<D>::kBytes, st>>>(w1, w2, aux, s, sites_per_run, runs_per_tile);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the sequential sweep: 32-sample tiles (the four TMEM lane quarters split
  // the units) while the batch leaves SMs idle, else 128-sample tiles; a
  // pinned tile variant selects 128 (variant 0) or 32 (any other)
  const int pin = tc1d_pinned_variant();
  if (pin >= 0 ? pin > 0 : g.B <= 32LL * sms) e = launch_bsweep<D, (D >= 64 ? 2 : 1), 32>(g.B, w1, s, st);
  else e = launch_bsweep<D, D / 16, 128>(g.B, w1, s, st);
  if (e != cudaSuccess) return e;
  Wgrad2Args w{};
  w.B = g.B;
  w.Lx = g.Lx;
  w.N = g.N;
  w.P = g.P;
  w.tiles = tiles;
  w.sigma = g.sigma;
  w.hcache = g.hcache;
  w.g1img = g.g1img;
  w.g2img = g.g2img;
  w.partial = g.partial;
  w.hdr = g.hdr;
  auto kw = tc2d_wgrad_kernel<D>;
  if ((e = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, W2S<D>::kBytes)) != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  const int gw = tc2d_wgrad_grid(g.B, g.N);
  kw<<<gw, 128, W2S<D>::kBytes, st>>>(w);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  tc2d_readout_grad_kernel<D><<<kReadout2Blocks, 128, 0, st>>>(g.yimg, g.dzimg, nimg, g.partial, g.P, gw);
  return cudaGetLastError();
}

}  // namespace

int tc2d_wgrad_grid(int64_t B, int N) {
  const int64_t nimg = (B + 127) / 128 * N;
  const int64_t g = sm_count_g();
  return (int)(nimg < g ? nimg : g);
}

int tc2d_grad_partial_rows(int64_t B, int N) { return tc2d_wgrad_grid(B, N) + kReadout2Blocks; }

size_t tc2d_grad_image_bytes(int64_t B, int N, int D, int which) {
  const int64_t nimg = (B + 127) / 128 * N;
  const int gw1 = 4 * D >= 128 ? 4 * D : 128, gw2 = 2 * D >= 128 ? 2 * D : 128;
  switch (which) {
    case 0: return (size_t)nimg * 128 * gw1 * 2;          // G1 images
    case 1: return (size_t)nimg * 128 * gw2 * 2;          // G2 images
    case 2: return (size_t)nimg * D * 128 * 4;             // y
    case 3: return (size_t)nimg * 128 * 4;                 // dz
    case 4: return (size_t)B * N * D * 4;                  // tape: dh through the GLU
    default: return (size_t)B * N * 3 * D * 2;             // tape: cell-backward factors
  }
}

cudaError_t tc2d_grad(const Tc2Grad& g, const uint8_t* wimg, int D, cudaStream_t st) {
  switch (D) {
    case 32: return run_grad<32>(g, wimg, st);
    case 64: return run_grad<64>(g, wimg, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nqs

namespace nqs {
cudaError_t tc2d_grad_set_wait_polls(uint32_t polls) {
  return cudaMemcpyToSymbol(tc::g_wait_polls, &polls, sizeof(polls));
}
}  // namespace nqs

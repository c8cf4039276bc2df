// BF16 tensor-core path of the 1D GRU wave function (App. A) for sm_103a:
// sampling, teacher-forced log psi, the prefix-cached TFIM chains and the
// reverse sweep, with the gate GEMM [h | 1 | onehot(s)] x W^T on tcgen05 (BF16
// operands, FP32 accumulate in TMEM; biases and one-hot weights folded into
// 16 extra K columns as BF16 hi / lo pairs) and the FP32 recurrent state in
// registers.
//
// Engine (tc1d_engine_kernel): a CTA runs GROUPS tiles of 128 TMEM lanes;
// tile g uses warps 4g.. with SPLIT threads per row (a warp reads only its own
// 32-lane quarter of TMEM).  Per cell step a tile writes its rows' h (BF16)
// into its A operand in shared memory; one thread issues (D + 16) / 16 MMAs
// (M = 128, N = 4D = the u / r / q / x_in pre-activations, K = 16) against
// the weight operand kept in shared memory and commits them to the tile's
// mbarrier; after the wait every thread reads its row's accumulators from
// TMEM, applies the gates, updates h in FP32 and the readout, and runs the
// row logic (draw / teacher forcing / chain bookkeeping).  Chains ping-pong
// two tiles per CTA, so one tile's MMA and row logic run under the other's
// MUFU-bound epilogue; sampling and teacher forcing of a small batch use 64-
// or 32-row tiles, at d_h = 64 with each A row in all four lane quarters.
//
// Reverse sweep: a parallel tape kernel (the carry-independent factors of the
// cell backward) and a sequential kernel (MMA_b, MMA_w and the carries);
// their comment block below gives the details.  The autotuner at the end
// picks the tile variant of each kernel per shape.
#include <map>
#include <mutex>
#include <tuple>

#include <cuda_fp16.h>

#include "kernels.h"
#include "tc.cuh"

namespace nqs {

namespace {

constexpr uint32_t kWaitLimit = tc::kDefaultWaitPolls;   // the drain's bound
// ping-pong: sub-chunks of the epilogue left when the token is passed (0 =
// after the last); measured on the TFIM N = 100, d_h = 64, B = 4096 step:
// 1.782 ms with 0, 1.764 ms with 1, 1.798 ms with 2
constexpr int kPPEarly = 1;

// Gate weights with the biases and one-hot input columns folded in, as a
// K-major BF16 operand of 4D rows x (D + 16) columns (see tc.cuh).  Biases and
// input weights enter as a BF16 pair hi + lo (hi = bf16(v), lo = bf16(v - hi)),
// so they keep about 16 significant bits.  Against an A row
// [h | 1 | 1 | onehot(s) | onehot(s) | 0] the four row blocks give
//   a_u = W_g [h; s] + b_g,  a_r = W_r [h; s] + b_r,  q = W_h h + b_h,
//   x_in = W_in s + b_in,
// so the epilogue needs no bias or input terms.  The u and r rows are scaled
// by 1/2 (exact in BF16), so each sigmoid gate is one tanh and one FMA.
__device__ __forceinline__ float bf16_hi(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__global__ void pack1d_tc_kernel(const float* __restrict__ p, uint8_t* __restrict__ wimg, int D) {
  const int KA = D + 16, total = 4 * D * KA;
  const int Wg = 0, Wr = D * (D + 2), Wh = 2 * D * (D + 2), Win = Wh + D * D;
  const int bg = Win + 2 * D, br = bg + D, bh = br + D, bin = bh + D;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int n = t / KA, k = t % KA, g = n / D, u = n % D;
    float v = 0.0f;
    if (k < D) {
      v = g == 0 ? p[Wg + u * (D + 2) + k] : g == 1 ? p[Wr + u * (D + 2) + k] : g == 2 ? p[Wh + u * D + k] : 0.0f;
    } else if (k < D + 6) {
      // extra columns: [b hi | b lo | w0 hi | w1 hi | w0 lo | w1 lo]
      const int e = k - D;
      const float bias = p[(g == 0 ? bg : g == 1 ? br : g == 2 ? bh : bin) + u];
      float w0 = 0.0f, w1 = 0.0f;
      if (g == 0 || g == 1) {
        const int W = g == 0 ? Wg : Wr;
        w0 = p[W + u * (D + 2) + D];
        w1 = p[W + u * (D + 2) + D + 1];
      } else if (g == 3) {
        w0 = p[Win + u * 2];
        w1 = p[Win + u * 2 + 1];
      }
      const float x = e < 2 ? bias : (e == 2 || e == 4) ? w0 : w1;
      v = e < 2 ? (e == 0 ? bf16_hi(x) : x - bf16_hi(x)) : (e < 4 ? bf16_hi(x) : x - bf16_hi(x));
    }
    if (g < 2) v *= 0.5f;   // u, r rows hold half the pre-activation: sigmoid(x) = (1 + tanh(x / 2)) / 2
    *reinterpret_cast<__nv_bfloat16*>(wimg + tc::kmajor_offset(n, k, KA)) = __float2bfloat16_rn(v);
  }
}

// 16-byte asynchronous global -> shared copies (the chain's next cached state).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" : : "r"(tc::smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The arrival on an mbarrier that takes place when all of this thread's
// earlier cp.async copies have landed (counted against the barrier's
// expected arrivals: no increment).
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" : : "r"(tc::smem_addr(bar)) : "memory");
}

// 8 consecutive TMEM columns of this thread's lane, and the wait that makes
// them usable: the empty asm statements after the wait tie every loaded
// register to it, so no use of the values can be scheduled above the wait.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}
// Shared-memory vector load kept inside the loop (a loop-invariant load of
// the readout weights would otherwise be hoisted into registers and spill).
__device__ __forceinline__ float4 lds4(const float* p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];\n"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(tc::smem_addr(p)));
  return v;
}
__device__ __forceinline__ void tmem_wait_regs(float (&v)[4][8]) {
  tc::tmem_wait_ld();
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int q = 0; q < 8; ++q) asm volatile("" : "+f"(v[b][q]));
}

// Gate nonlinearities of the BF16 path: one hardware tanh (MUFU.TANH,
// relative error ~2^-11, below the 2^-9 rounding of the BF16 GEMM operands)
// per gate; sigmoid(x) = (1 + tanh(x/2)) / 2.
__device__ __forceinline__ float hw_tanh(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// softplus(x) = max(x, 0) + log(1 + e^-|x|) with the hardware exp2 / log2
// approximations (the argument of the log lies in (1, 2]): absolute error
// below 1e-6, against logit errors of ~1e-3 from the BF16 operands; used for
// the chains' log-probability differences, -log p(s | d) = softplus(-+d).
__device__ __forceinline__ float softplus_hw(float x) {
  return fmaxf(x, 0.0f) + __logf(1.0f + __expf(-fabsf(x)));
}

// Shared-memory carve-up (bytes from a 1024-aligned base).
template <int D, int GROUPS, int SPLIT>
struct Smem {
  static constexpr int KA = D + 16;                              // A columns: [h | 1 1 | onehot x2 | 0]
  // d_h = 128: the x_in block (W_in s + b_in depends on the input spin only)
  // comes from a 3 x D FP32 table instead of the MMA, so the weight operand
  // keeps 3D rows and the accumulators 3D columns (the 4D rows would not fit
  // shared memory beside the A operand and the staging buffer)
  static constexpr bool XT = D >= 128;
  static constexpr int kRowsB = (XT ? 3 : 4) * D;                // weight operand rows
  static constexpr int kTmemCols = GROUPS * 4 * D <= 256 ? 256 : 512;
  static constexpr int kB = 0;                                   // weights, kRowsB x KA bf16
  static constexpr int kA = kB + kRowsB * KA * 2;                // GROUPS x 128 x KA bf16
  static constexpr int kDU = kA + GROUPS * 128 * KA * 2;        // D floats: U[0] - U[1]
  static constexpr int kZ = kDU + D * 4;                         // GROUPS x SPLIT x 128 floats
  static constexpr int kJob = kZ + GROUPS * SPLIT * 128 * 4;     // GROUPS x 128 long long
  static constexpr int HS = D + 4;                               // staging row stride (floats; conflict-free float4)
  static constexpr int kStage = kJob + GROUPS * 128 * 8;         // GROUPS x 128 x HS floats: next chain state
                                                                 // (chains) or the new states (cache stores)
  static constexpr int kXin = kStage + GROUPS * 128 * HS * 4;    // XT: x_in table [no input | s = 0 | s = 1][D]
  static constexpr int kBar = (kXin + (XT ? 3 * D * 4 : 0) + 15) / 16 * 16;   // GROUPS MMA + 1 drain
  static constexpr int kSlot = kBar + 8 * (GROUPS + 1);
  static constexpr int kFlags = kSlot + 16;                      // ping-pong idle flags, one int per tile
  static constexpr int kUsed = kFlags + 16;
  // one CTA per SM for the persistent chain launch (TMEM holds two tiles)
  static constexpr int kBytes = 1024 + (GROUPS == 2 ? (kUsed > 120 * 1024 ? kUsed : 120 * 1024) : kUsed);
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
};

// Tile threads: SPLIT threads per row, in different warps (a warp reads only
// its own 32-lane quarter of TMEM): warp w of a tile serves rows 32 (w % 4) ..
// + 31 and hidden units [(w / 4) D / SPLIT, (w / 4 + 1) D / SPLIT).  With REP
// = 4 (sampling / teacher forcing on 32-sample tiles) every sample's A row is
// written into all four lane quarters (the MMA's 128 rows are computed
// anyway), and the quarters' warps take a quarter of the units each, so the
// MUFU-bound epilogue of a small tile runs on all four sub-partitions.
template <int D, int MODE, int GROUPS, int SPLIT, int REP = 1>
__global__ void __launch_bounds__(128 * GROUPS * SPLIT, 1)
tc1d_engine_kernel(const float* __restrict__ img, const uint8_t* __restrict__ wimg, Tc1Args a) {
  using S = Smem<D, GROUPS, SPLIT>;
  static_assert(REP == 1 || (REP == 4 && MODE != 2 && GROUPS == 1), "replicated rows: sampling / teacher forcing");
  constexpr int TT = 128 * SPLIT;          // threads per tile
  constexpr int NT = TT * GROUPS;
  constexpr int N4 = 4 * D, KA = S::KA;
  constexpr int NSL = REP * SPLIT;         // unit slices per row
  constexpr int RS = 128 / REP;            // rows per tile with REP
  constexpr int DU = D / NSL;              // hidden units per thread
  static_assert(DU % 16 == 0, "at least 16 units per thread");
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sB = sm + S::kB;
  float* dUs = reinterpret_cast<float*>(sm + S::kDU);
  float* zbuf = reinterpret_cast<float*>(sm + S::kZ);
  long long* jobbuf = reinterpret_cast<long long*>(sm + S::kJob);
  float* stage = reinterpret_cast<float*>(sm + S::kStage);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  volatile int* idle_flag = reinterpret_cast<volatile int*>(sm + S::kFlags);

  // ---- prologue: operands and constants into shared memory, TMEM, barriers ----
  for (int i = threadIdx.x; i < S::kRowsB * KA * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sB)[i] = reinterpret_cast<const uint4*>(wimg)[i];
  // readout: only the logit difference d = (U_0 - U_1) h + c_0 - c_1 is used
  for (int i = threadIdx.x; i < D; i += NT) dUs[i] = img[10 * D + i] - img[11 * D + i];
  float* xin = reinterpret_cast<float*>(sm + S::kXin);
  if constexpr (S::XT) {
    // x_in = b_in + W_in onehot(s) in FP32 (image: Ws[s][2D + u] = W_in[u][s], Bs[3D + u] = b_in[u])
    for (int i = threadIdx.x; i < 3 * D; i += NT) {
      const int sv = i / D - 1, u = i % D;
      xin[i] = img[6 * D + 3 * D + u] + (sv >= 0 ? img[sv * 3 * D + 2 * D + u] : 0.0f);
    }
  }
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    for (int g = 0; g < GROUPS; ++g) tc::mbar_init(&mbar[g], 1);
    tc::mbar_init(&mbar[GROUPS], GROUPS);    // drain: one arrival per tile's MMA issuer
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 2) idle_flag[threadIdx.x] = 0;
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, S::kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;

  const int g = threadIdx.x / TT, tt = threadIdx.x % TT, lane = threadIdx.x & 31;
  const int wt = tt / 32, m = (wt % 4) * 32 + lane;          // m: this thread's A row and TMEM lane
  const int r = REP == 4 ? lane : m;                          // r: its sample row in the tile
  const int part = REP == 4 ? (wt % 4) * SPLIT + wt / 4 : wt / 4;   // its unit slice (0: side effects)
  const int u0 = part * DU;
  // sampling / teacher forcing with 64- or 32-row tiles: warps whose 32 rows
  // lie past the tile's rows skip the A rows, the epilogue and the cache
  // stores (they still take part in every barrier)
  const bool wact = MODE == 2 || GROUPS == 2 || REP == 4 || (m & ~31) < a.rows;
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16) + (uint32_t)(g * 256);
  const uint32_t bar_main = 1 + g, bar_x = 1 + GROUPS + g;
  uint8_t* sA = sm + S::kA + g * 128 * KA * 2;
  float* zb = zbuf + g * SPLIT * 128;
  long long* jb = jobbuf + g * 128;
  float* stg = stage + (g * 128 + r) * S::HS + u0;   // this thread's units of the row's staged state
  const float dc = img[12 * D] - img[12 * D + 1];
  const int N = a.N;
  const int64_t B = a.B;

  float h[DU];
#pragma unroll
  for (int u = 0; u < DU; ++u) h[u] = 0.0f;
  int64_t b = 0;
  int t = 0, s_in = -1, f = 0;
  float acc = 0.0f;            // log psi sum, or Delta of the chain
  bool active = false;
  long long nxt = -1;          // chains: prefetched next job (-1: none)
  bool pending = false;        // chains: prefetch requested for the current job

  const uint64_t total = MODE == 2 ? (uint64_t)B * (uint64_t)(N - 1) : 0;
  // Job hand-out (chains): the part-0 warps pull, one atomic per warp, and
  // publish the job of each row in shared memory for the other parts.
  auto pull_publish = [&](bool need) {
    if (part == 0) {
      const unsigned mask = __ballot_sync(0xffffffffu, need);
      long long j = -1;
      if (mask) {
        const int leader = __ffs(mask) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(a.counter, (unsigned long long)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        const unsigned long long jj = base + __popc(mask & ((1u << lane) - 1u));
        if constexpr (MODE == 2) {
          if (need && jj < total) j = (long long)jj;
        }
      }
      if (need) jb[m] = j;
    }
  };
  auto job_src = [&](long long j) -> const float* {
    const int64_t bj = (int64_t)((unsigned long long)j % (unsigned long long)B);
    const int fj = (int)((unsigned long long)j / (unsigned long long)B);
    return a.hcache + (bj * N + fj) * D + u0;
  };
  // start job j; its cached state comes from `src` (global or the staging slot)
  auto start_job = [&](long long j, const float* src) {
    if (j < 0) { active = false; return; }
    b = (int64_t)((unsigned long long)j % (unsigned long long)B);
    f = (int)((unsigned long long)j / (unsigned long long)B);
    const int sf = a.sigma[b * N + f] ? 1 : 0;
    const float df = a.dlog[b * N + f];
    t = f + 1;
    s_in = 1 - sf;
    acc = 0.5f * (sf == 0 ? -df : df);
    active = true;
    pending = false;
#pragma unroll
    for (int q = 0; q < DU / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(src)[q];
      h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
    }
  };

  if constexpr (MODE == 2) {
    pull_publish(true);
    tc::group_barrier(bar_x, TT);
    const long long j = jb[m];
    if (j >= 0) start_job(j, job_src(j));
  } else {
    b = ((int64_t)blockIdx.x * GROUPS + g) * a.rows + r;
    active = r < a.rows && b < B;
  }

  // Ping-pong (two tiles): the tiles take turns in the MUFU-bound epilogue,
  // so one tile's MMA and row logic run under the other's epilogue.  Tile g
  // waits for the other tile's token (named barrier) before its epilogue and
  // passes its own token after it: E0(0), E1(0), E0(1), E1(1), ...  Each token
  // carries the sender's idle flag (no active rows, permanent); a tile that
  // is idle keeps taking turns without work until both are idle, and the
  // exit rule below leaves no token unconsumed.
  constexpr bool PP = GROUPS == 2;
  const uint32_t pp_wait = g == 0 ? 6 : 5, pp_sig = g == 0 ? 5 : 6;
  bool prev_idle = false;      // the idle flag this tile sent with its last token
  int pstep = 0;

  uint32_t phase = 0;
  bool timed_out = false;
  for (;;) {
    // ---- (a) A row: this thread's units of h as BF16 (+ the constant and input columns by part 0) ----
#pragma unroll
    for (int kc = 0; kc < DU / 8; ++kc) {
      __nv_bfloat162 p0 = __floats2bfloat162_rn(h[8 * kc + 0], h[8 * kc + 1]);
      __nv_bfloat162 p1 = __floats2bfloat162_rn(h[8 * kc + 2], h[8 * kc + 3]);
      __nv_bfloat162 p2 = __floats2bfloat162_rn(h[8 * kc + 4], h[8 * kc + 5]);
      __nv_bfloat162 p3 = __floats2bfloat162_rn(h[8 * kc + 6], h[8 * kc + 7]);
      uint4 v;
      v.x = *reinterpret_cast<uint32_t*>(&p0);
      v.y = *reinterpret_cast<uint32_t*>(&p1);
      v.z = *reinterpret_cast<uint32_t*>(&p2);
      v.w = *reinterpret_cast<uint32_t*>(&p3);
      if (wact) {
#pragma unroll
        for (int c4 = 0; c4 < REP; ++c4)
          *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(REP == 4 ? r + 32 * c4 : m, u0 + 8 * kc, KA)) = v;
      }
    }
    if (part == 0 && wact) {
      // bf16 1.0 = 0x3F80: [1 | 1 | s_in == 0 | s_in == 1 | s_in == 0 | s_in == 1 | 0 0]
      const uint32_t one = 0x3F80u;
      const uint32_t oh = (s_in == 0 ? one : 0u) | ((s_in == 1 ? one : 0u) << 16);
      uint4 v;
      v.x = one | (one << 16);
      v.y = oh;
      v.z = oh;
      v.w = 0u;
#pragma unroll
      for (int c4 = 0; c4 < REP; ++c4) {
        const int row = REP == 4 ? r + 32 * c4 : m;
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, D, KA)) = v;
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, D + 8, KA)) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    const bool any = tc::group_barrier_or(active && !timed_out, bar_main, TT);
    if (!PP && !any) break;
    tc::fence_after_sync();
    // ---- (b) one thread issues the tile's MMAs ----
    if (any && tt == 0) {
      if constexpr (S::XT) {
        // 3D = 384 gate rows: u and r (N = 256) and q (N = 128) as two MMAs per K step
        constexpr uint32_t idesc0 = tc::make_idesc_bf16(128, 256), idesc1 = tc::make_idesc_bf16(128, D);
        constexpr uint32_t row256 = (256 / 8) * (KA / 8) * 128;   // byte offset of weight row 256
#pragma unroll
        for (int k = 0; k < KA / 16; ++k) {
          const uint64_t da = tc::make_desc(tc::smem_addr(sA) + k * 256, 128, (KA / 8) * 128);
          const uint64_t db0 = tc::make_desc(tc::smem_addr(sB) + k * 256, 128, (KA / 8) * 128);
          const uint64_t db1 = tc::make_desc(tc::smem_addr(sB) + row256 + k * 256, 128, (KA / 8) * 128);
          tc::mma_bf16(tbase, da, db0, idesc0, k > 0);
          tc::mma_bf16(tbase + 256u, da, db1, idesc1, k > 0);
        }
      } else {
        constexpr uint32_t idesc = tc::make_idesc_bf16(128, N4);
#pragma unroll
        for (int k = 0; k < KA / 16; ++k) {
          const uint64_t da = tc::make_desc(tc::smem_addr(sA) + k * 256, 128, (KA / 8) * 128);
          const uint64_t db = tc::make_desc(tc::smem_addr(sB) + k * 256, 128, (KA / 8) * 128);
          tc::mma_bf16(tbase + (uint32_t)(g * 256), da, db, idesc, k > 0);
        }
      }
      tc::mma_commit(&mbar[g]);
    }
    // ---- (c) row inputs of this step, fetched while the MMA runs ----
    int s_t = 0;
    float dl = 0.0f, uni = 0.0f;
    if (active) {
      if constexpr (MODE == 0) {
        uni = a.uniforms ? a.uniforms[b * N + t] : sampling_uniform(a.seed, a.step_dev ? *a.step_dev : a.step, (uint32_t)(a.b0 + b), (uint32_t)t);
      } else {
        s_t = a.sigma[b * N + t] ? 1 : 0;
        if constexpr (MODE == 2) dl = a.dlog[b * N + t];
      }
    }
    // ---- (d) wait for the accumulator ----
    if (any) {
      if (!tc::mbar_wait(&mbar[g], phase, wlim)) {
        timed_out = true;
        flag_status(a.hdr, NQS_ETIMEOUT);
      }
      phase ^= 1;
      tc::fence_after_sync();
    }
    // the first accumulator columns are loaded before the hand-off wait
    float bufA[4][8], bufB[4][8];
    auto issue = [&](int sc, float (&bf)[4][8]) {
      const int cu = u0 + sc * 8;
      tmem_ld8(trow + cu, bf[0]);
      tmem_ld8(trow + D + cu, bf[1]);
      tmem_ld8(trow + 2 * D + cu, bf[2]);
      if constexpr (S::XT) {
        const float* xr = xin + (s_in + 1) * D + cu;
        const float4 x0 = lds4(xr), x1 = lds4(xr + 4);
        bf[3][0] = x0.x; bf[3][1] = x0.y; bf[3][2] = x0.z; bf[3][3] = x0.w;
        bf[3][4] = x1.x; bf[3][5] = x1.y; bf[3][6] = x1.z; bf[3][7] = x1.w;
      } else {
        tmem_ld8(trow + 3 * D + cu, bf[3]);
      }
    };
    if (any && wact) issue(0, bufA);
    if constexpr (PP) {
      bool oth = false;        // the other tile's idle flag from its last token
      if (g == 1 || pstep > 0) {
        tc::group_barrier(pp_wait, 2 * TT);
        oth = idle_flag[1 - g] != 0;
      }
      // both idle and the other tile saw this tile idle: it has left, no token
      if (oth && prev_idle) break;
      // both idle: the other tile waits for one more token, then leaves
      if (!any && oth) {
        if (tt == 0) idle_flag[g] = 1;
        tc::group_arrive(pp_sig, 2 * TT);
        break;
      }
    }
    // ---- (e) gates and FP32 state update of this thread's units ----
    // Accumulator columns come in 8-unit sub-chunks, double-buffered, and the
    // gate math is software-pipelined: the u / r gates of sub-chunk c + 1
    // (stage A) are computed together with the candidate and state update of
    // sub-chunk c (stage B), so the MUFU always has independent work.
    // Readout: sequential sums over 16-unit chunks, chunks combined by a fixed
    // pairwise tree, so every SPLIT gives bitwise the same logits.
    float zc[DU / 16];
#pragma unroll
    for (int c = 0; c < DU / 16; ++c) zc[c] = 0.0f;
    if (any && wact) {
      constexpr int NS = DU / 8;
      // stage A: tu = tanh(a_u / 2 pre-scaled), ag = r * q + x_in
      auto stage_a = [&](float (&bf)[4][8], float (&tu)[8], float (&ag)[8]) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          tu[q] = hw_tanh(bf[0][q]);
          const float rg = fmaf(0.5f, hw_tanh(bf[1][q]), 0.5f);
          ag[q] = fmaf(rg, bf[2][q], bf[3][q]);
        }
      };
      float tuA[8], agA[8], tuB[8], agB[8];
      tmem_wait_regs(bufA);
      if (NS > 1) issue(1, bufB);
      stage_a(bufA, tuA, agA);
      float s0 = 0.0f;
#pragma unroll
      for (int sc = 0; sc < NS; ++sc) {
        float (&tu)[8] = (sc & 1) ? tuB : tuA;
        float (&ag)[8] = (sc & 1) ? agB : agA;
        if (sc + 1 < NS) {
          float (&nb)[4][8] = ((sc + 1) & 1) ? bufB : bufA;
          float (&fb)[4][8] = ((sc + 1) & 1) ? bufA : bufB;   // consumed by stage A of sc
          tmem_wait_regs(nb);
          if (sc + 2 < NS) issue(sc + 2, fb);
          stage_a(nb, (sc & 1) ? tuA : tuB, (sc & 1) ? agA : agB);
        }
        float Ud[8];
        {
          const float4 a0 = lds4(dUs + u0 + sc * 8), a1 = lds4(dUs + u0 + sc * 8 + 4);
          Ud[0] = a0.x; Ud[1] = a0.y; Ud[2] = a0.z; Ud[3] = a0.w;
          Ud[4] = a1.x; Ud[5] = a1.y; Ud[6] = a1.z; Ud[7] = a1.w;
        }
        // stage B
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = sc * 8 + q;
          const float cc = hw_tanh(ag[q]);
          const float ug = fmaf(0.5f, tu[q], 0.5f);
          h[j] = fmaf(ug, cc - h[j], h[j]);
          s0 = fmaf(Ud[q], h[j], s0);
        }
        if (sc & 1) {
          zc[sc / 2] = s0;
          s0 = 0.0f;
        }
        if constexpr (PP) {
          // pass the token kPPEarly sub-chunks before the end: the other
          // tile's first loads and gates overlap this tile's last ones
          if (sc == (NS > kPPEarly ? NS - 1 - kPPEarly : NS - 1)) {
            if (tt == 0) idle_flag[g] = 0;
            tc::group_arrive(pp_sig, 2 * TT);
            prev_idle = false;
          }
        }
      }
    }
#pragma unroll
    for (int w = 1; w < DU / 16; w *= 2)
#pragma unroll
      for (int c = 0; c + w < DU / 16; c += 2 * w) zc[c] += zc[c + w];
    float z = zc[0];
    if constexpr (PP) {
      if (!any) {             // idle: pass the token with the idle flag
        if (tt == 0) idle_flag[g] = 1;
        tc::group_arrive(pp_sig, 2 * TT);
        prev_idle = true;
      }
    }
    if constexpr (NSL > 1) {
      zb[part * RS + r] = z;
      tc::group_barrier(bar_x, TT);
      float pz[NSL];
#pragma unroll
      for (int p = 0; p < NSL; ++p) pz[p] = zb[p * RS + r];
#pragma unroll
      for (int w = 1; w < NSL; w *= 2)
#pragma unroll
        for (int p = 0; p + w < NSL; p += 2 * w) pz[p] += pz[p + w];
      z = pz[0];
    }
    // ---- (f) row logic (identical in every part; side effects by part 0) ----
    bool fin = false;
    if (active && !timed_out) {
      const float d = z + dc;
      if constexpr (MODE == 2) {
        acc += 0.5f * (softplus_hw(s_t == 0 ? -dl : dl) - softplus_hw(s_t == 0 ? -d : d));   // log p(d) - log p(dl)
        s_in = s_t;
        if (++t == N) {
          if (part == 0) a.delta[b * N + f] = acc;
          fin = true;
        }
      } else {
        int s = s_t;
        if constexpr (MODE == 0) {
          s = uni < sigmoid_acc(d) ? 0 : 1;
          if (part == 0) a.sigma_out[b * N + t] = (uint8_t)s;
        }
        acc += log_prob(s, d);
        s_in = s;
        if (++t == N) {
          const float lp = 0.5f * acc;
          if (part == 0) {
            a.logpsi[b] = lp;
            if (!isfinite(lp)) flag_status(a.hdr, NQS_ENONFINITE);
          }
          active = false;
        }
      }
    }
    if constexpr (MODE != 2) {
      // cache store of this step's states, coalesced: every thread stages its
      // units of h, then each warp writes its 32 rows as whole row segments
      // (all rows of a tile are at the same site, pstep)
      if (a.hcache && any && wact) {
#pragma unroll
        for (int q = 0; q < DU / 4; ++q)
          reinterpret_cast<float4*>(stg)[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
        __syncwarp();
        constexpr int L = DU / 4, RPI = 32 / L;   // lanes per row segment, rows per store
        const int lr = lane / L, lq = lane % L, m0 = REP == 4 ? 0 : (wt % 4) * 32;
        const int64_t b0 = ((int64_t)blockIdx.x * GROUPS + g) * a.rows;
#pragma unroll 4
        for (int i = 0; i < 32; i += RPI) {
          const int mr = m0 + i + lr;
          const int64_t br = b0 + mr;
          if (mr < a.rows && br < B)
            reinterpret_cast<float4*>(a.hcache + (br * N + pstep) * D + u0)[lq] =
                reinterpret_cast<const float4*>(stage + (g * 128 + mr) * S::HS + u0)[lq];
        }
        __syncwarp();
      }
    }
    if constexpr (MODE == 2) {
      // A finished chain takes its prefetched successor (a prefetch that found
      // the queue empty retires the row); a chain that finished without a
      // prefetch pulls its successor now.  A chain with one step left pulls
      // the next job and starts copying its cached state to shared memory.
      bool need = false;
      if (fin) {
        if (!pending) {
          need = true;
        } else if (nxt >= 0) {
          cp_async_wait_all();
          start_job(nxt, stg);
        } else {
          active = false;
        }
        nxt = -1;
      }
      const bool want = active && !timed_out && !pending && t == N - 1;
      pull_publish(need || want);
      tc::group_barrier(bar_x, TT);
      if (need) {
        const long long j = jb[m];
        start_job(j, j >= 0 ? job_src(j) : nullptr);
      } else if (want) {
        pending = true;
        nxt = jb[m];
        if (nxt >= 0) {
          const float* src = job_src(nxt);
#pragma unroll
          for (int q = 0; q < DU / 4; ++q) cp_async16(stg + 4 * q, src + 4 * q);
          cp_async_commit();
        }
      }
    } else if constexpr (NSL > 1) {
      tc::group_barrier(bar_x, TT);   // zbuf is rewritten next step
    }
    ++pstep;
  }
  cp_async_wait_all();
  // ---- epilogue: free TMEM once both tiles are done (and, after a wait that
  // gave up, once their MMAs have drained) ----
  tc::fence_before_sync();
  if (__syncthreads_or(timed_out) && tt == 0) tc::drain_mmas(&mbar[GROUPS], kWaitLimit);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, S::kTmemCols);
}

// ----------------------------------------------------------------------------
// Reverse sweep on the tensor cores, in two launches.
//
// (1) tc1d_tape_kernel, parallel over (tile of 128 samples, site n): every
// part of the cell backward that does not depend on the incoming gradient.
// From the cached states it builds X_n = [h_{n-1} | 1 1 | onehot(s_{n-1}) x2
// | 0] (BF16), recomputes acc_f = X_n Wf^T with the engine's folded weights
// (the u / r / q / x_in pre-activations, bitwise those of the forward) and
// writes per (sample, site):
//   e_n = onehot_0(s_n) - p_0, p_0 the softmax of the readout of h_n (FP32;
//         the readout gradient is dz_n = c_b e_n);
//   x_n = BF16 h_{n-1}, the state part of X_n;
//   k_n = five factors (FP16, 5 x D) with which the cell backward is linear
//         in dh = dlog psi / dh_n:  G = [du_a | dr_a | dq | dc_a] = dh [k0 |
//         k1 | k2 | k3] and the direct path dh k4, where (u, r gates, c the
//         candidate, q its recurrent pre-activation)
//           k0 = (c - h_{n-1}) u (1 - u),  k3 = u (1 - c^2),  k2 = k3 r,
//           k1 = k2 q (1 - r),             k4 = 1 - u.
// The tape is sample-minor in 8-unit groups ([n][vector][unit / 8][b][8]),
// so that warps of consecutive samples read and write it in whole lines.
// One CTA per SM walks a run of consecutive sites of one sample tile; the
// cached state rows come in by coalesced cp.async into three shared-memory
// buffers (h_{n-1}, h_n, and h_{n+1} in flight).
//
// (2) tc1d_bptt_kernel, one CTA per tile of ROWS samples, sites N-1 .. 0:
//   dh = dz_n (U_0 - U_1) + carry,  G = dh k_n (BF16),  carry = dh k4
//   MMA_b: acc_b = G[:, :3D] W3             (dh_{n-1} through the gates)
//   MMA_w: acc_w += G^T X_n                 (weight, bias and one-hot-column
//                                           gradients; G and X MN-major)
//   carry += acc_b.
// Only this chain is sequential.  All four TMEM lane quarters' warps work on
// every tile: with ROWS < 128 the quarters split the hidden units, and the
// quarters that hold the samples' TMEM lanes pass acc_b on through shared
// memory.  The tape of later sites and the next X operand are copied in with
// cp.async while a site runs, and MMA_w runs under the next site's
// elementwise work.  acc_w stays in TMEM for the whole sweep; the readout
// gradients (U, c) come from dz and the cache and are reduced by a separate
// kernel.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint4 pack_bf16x8(const float* v) {
  __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 p1 = __floats2bfloat162_rn(v[2], v[3]);
  __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]);
  __nv_bfloat162 p3 = __floats2bfloat162_rn(v[6], v[7]);
  return make_uint4(*reinterpret_cast<uint32_t*>(&p0), *reinterpret_cast<uint32_t*>(&p1),
                    *reinterpret_cast<uint32_t*>(&p2), *reinterpret_cast<uint32_t*>(&p3));
}

__device__ __forceinline__ uint4 pack_f16x8(const float* v) {
  __half2 p0 = __floats2half2_rn(v[0], v[1]);
  __half2 p1 = __floats2half2_rn(v[2], v[3]);
  __half2 p2 = __floats2half2_rn(v[4], v[5]);
  __half2 p3 = __floats2half2_rn(v[6], v[7]);
  return make_uint4(*reinterpret_cast<uint32_t*>(&p0), *reinterpret_cast<uint32_t*>(&p1),
                    *reinterpret_cast<uint32_t*>(&p2), *reinterpret_cast<uint32_t*>(&p3));
}

__device__ __forceinline__ void unpack_f16x8(uint4 q, float* v) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
    const float2 f = __half22float2(h);
    v[2 * i] = f.x;
    v[2 * i + 1] = f.y;
  }
}

__device__ __forceinline__ void st_bf16x8(uint8_t* dst, const float* v) {
  *reinterpret_cast<uint4*>(dst) = pack_bf16x8(v);
}

// 16-byte cp.async that copies `bytes` (16 or 0) and zero-fills the rest.
__device__ __forceinline__ void cp_async16_zf(void* smem, const void* gmem, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n"
               :
               : "r"(tc::smem_addr(smem)), "l"(gmem), "r"(bytes)
               : "memory");
}

// Spin byte load kept in place (issued one site ahead of its use).
__device__ __forceinline__ uint32_t ldg_u8(const uint8_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc.u8 %0, [%1];\n" : "=r"(v) : "l"(p));
  return v;
}

// Tape element offsets (in 16-byte groups of 8 units) of sample b, site n.
__device__ __forceinline__ int64_t tape_k_group(int64_t B, int n, int c, int g, int64_t b, int D) {
  return (((int64_t)n * 5 + c) * (D / 8) + g) * B + b;
}
__device__ __forceinline__ int64_t tape_x_group(int64_t B, int n, int g, int64_t b, int D) {
  return ((int64_t)n * (D / 8) + g) * B + b;
}

template <int D>
struct TpS {
  static constexpr int SPLIT = D / 16;                    // threads per row (16 units each)
  static constexpr int NT = 128 * SPLIT;
  static constexpr int KA = D + 16;                       // X columns
  static constexpr int HS = D + 4;                        // state row stride (floats): 16-byte
                                                          // accesses of 8 consecutive rows hit distinct banks
  static constexpr int kWf = 0;                           // [4D x KA] bf16, K-major (folded)
  static constexpr int kA = kWf + 4 * D * KA * 2;         // [128 x KA] bf16
  static constexpr int kH = kA + 128 * KA * 2;            // 3 x [128 x HS] f32 state rows
  static constexpr int kDU = kH + 3 * 128 * HS * 4;       // D floats: U[0] - U[1]
  static constexpr int kZ = kDU + D * 4;                  // SPLIT x 128 floats (readout exchange)
  static constexpr int kBar = kZ + SPLIT * 128 * 4;       // 5 mbarriers: MMA, 3 state buffers, drain
  static constexpr int kSlot = kBar + 40;
  static constexpr int kBytes = 1024 + kSlot + 16;
  static constexpr int kCols = 4 * D;                     // 64, 128 or 256 columns
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
};

template <int D>
__global__ void __launch_bounds__(TpS<D>::NT, 1)
tc1d_tape_kernel(const float* __restrict__ img, const uint8_t* __restrict__ wfimg, TcBpttArgs a, int sites_per_run,
                 int runs_per_tile, int part_row0) {
  using S = TpS<D>;
  constexpr int SPLIT = S::SPLIT, NT = S::NT, KA = S::KA, HS = S::HS, DU = D / SPLIT;
  static_assert(DU == 16, "16 units per thread");
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sWf = sm + S::kWf;
  uint8_t* sA = sm + S::kA;
  float* sH = reinterpret_cast<float*>(sm + S::kH);
  float* dU = reinterpret_cast<float*>(sm + S::kDU);
  float* zb = reinterpret_cast<float*>(sm + S::kZ);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < 4 * D * KA * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sWf)[i] = reinterpret_cast<const uint4*>(wfimg)[i];
  for (int i = threadIdx.x; i < D; i += NT) dU[i] = img[10 * D + i] - img[11 * D + i];
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);                           // MMA done
    for (int k = 1; k < 4; ++k) tc::mbar_init(&mbar[k], NT);   // state buffer k - 1 filled
    tc::mbar_init(&mbar[4], 1);                           // drain (MMA issuer: thread 0)
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, S::kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int lane = threadIdx.x & 31, wt = threadIdx.x >> 5, part = wt / 4, m = (wt % 4) * 32 + lane;
  const int u0 = part * DU;
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16);
  const float dc = img[12 * D] - img[12 * D + 1];
  const int N = a.N;
  const int64_t B = a.B;
  const int64_t runs = (B + 127) / 128 * runs_per_tile;
  constexpr uint32_t idesc = tc::make_idesc_bf16(128, 4 * D);
  uint32_t phases = 0;                     // bit k: the phase of mbar[k] waited for next
  bool timed_out = false;
  auto wait = [&](int k) {
    if (!tc::mbar_wait(&mbar[k], (phases >> k) & 1u, wlim)) { timed_out = true; flag_status(a.hdr, NQS_ETIMEOUT); }
    phases ^= 1u << k;
  };
  // readout gradients of this thread's rows: dU_0[u] += dz_n h_n[u], dc_0 += dz_n
  float gU[DU];
#pragma unroll
  for (int u = 0; u < DU; ++u) gU[u] = 0.0f;
  float gc = 0.0f;
  // state rows h_n of the tile's 128 samples into buffer k, 16 bytes per copy,
  // consecutive threads on consecutive pieces of a row (zeros for n outside
  // [0, N) or samples past the batch)
  auto load_rows = [&](int64_t bt, int n, int k) {
    float* dst = sH + k * 128 * HS;
    constexpr int PR = D / 4;              // pieces per row
    for (int q = threadIdx.x; q < 128 * PR; q += NT) {
      const int row = q / PR, pc = q % PR;
      const int64_t b = bt * 128 + row;
      const bool ok = b < B && n >= 0 && n < N;
      const float* src = ok ? a.hcache + (b * N + n) * D + 4 * pc : a.hcache;
      cp_async16_zf(dst + row * HS + 4 * pc, src, ok ? 16u : 0u);
    }
    cp_async_arrive_noinc(&mbar[1 + k]);
  };
  for (int64_t run = blockIdx.x; run < runs; run += gridDim.x) {
    const int64_t bt = run / runs_per_tile;
    const int n0 = (int)(run % runs_per_tile) * sites_per_run;
    const int n1 = n0 + sites_per_run < N ? n0 + sites_per_run : N;
    if (n0 >= n1) continue;                 // uniform
    // h_{n} sits in buffer (n - n0 + 1) % 3
    load_rows(bt, n0 - 1, 0);
    load_rows(bt, n0, 1);
    wait(1);
    const int64_t b = bt * 128 + m;
    const bool valid = b < B;
    const float coef = valid ? 0.5f * a.weights[b] : 0.0f;
    for (int n = n0; n < n1; ++n) {
      const int kp = (n - n0) % 3, kn = (n - n0 + 1) % 3;
      if (n + 1 < n1) load_rows(bt, n + 1, (n - n0 + 2) % 3);
      wait(1 + kn);
      const float* hp = sH + (kp * 128 + m) * HS + u0;
      const float* hn = sH + (kn * 128 + m) * HS + u0;
      // ---- X_n row (also the tape's x_n) ----
#pragma unroll
      for (int c = 0; c < DU / 8; ++c) {
        float v[8];
        const float4 x0 = reinterpret_cast<const float4*>(hp)[2 * c];
        const float4 x1 = reinterpret_cast<const float4*>(hp)[2 * c + 1];
        v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w; v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
        const uint4 q = pack_bf16x8(v);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, u0 + 8 * c, KA)) = q;
        if (valid) reinterpret_cast<uint4*>(a.tape_x)[tape_x_group(B, n, (u0 >> 3) + c, b, D)] = q;
      }
      if (part == 0) {
        const int s_in = (valid && n > 0) ? (a.sigma[b * N + n - 1] ? 1 : 0) : -1;
        const uint32_t one = 0x3F80u;
        const uint32_t oh = (s_in == 0 ? one : 0u) | ((s_in == 1 ? one : 0u) << 16);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, D, KA)) = make_uint4(one | (one << 16), oh, oh, 0u);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, D + 8, KA)) = make_uint4(0u, 0u, 0u, 0u);
      }
      // ---- readout of h_n: 16-unit chunk sums in order, parts by a fixed
      // pairwise tree, as in the forward pass ----
      float z = 0.0f;
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 h4 = reinterpret_cast<const float4*>(hn)[q4];
        const float4 w4 = reinterpret_cast<const float4*>(dU + u0)[q4];
        z = fmaf(w4.x, h4.x, z);
        z = fmaf(w4.y, h4.y, z);
        z = fmaf(w4.z, h4.z, z);
        z = fmaf(w4.w, h4.w, z);
      }
      if constexpr (SPLIT > 1) zb[part * 128 + m] = z;
      tc::fence_async_smem();
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
      if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < KA / 16; ++k) {
          const uint64_t da = tc::make_desc(tc::smem_addr(sA) + k * 256, 128, (KA / 8) * 128);
          const uint64_t db = tc::make_desc(tc::smem_addr(sWf) + k * 256, 128, (KA / 8) * 128);
          tc::mma_bf16(tbase, da, db, idesc, k > 0);
        }
        tc::mma_commit(&mbar[0]);
      }
      if constexpr (SPLIT > 1) {
        float pz[SPLIT];
#pragma unroll
        for (int p = 0; p < SPLIT; ++p) pz[p] = zb[p * 128 + m];
#pragma unroll
        for (int w = 1; w < SPLIT; w *= 2)
#pragma unroll
          for (int p = 0; p + w < SPLIT; p += 2 * w) pz[p] += pz[p + w];
        z = pz[0];
      }
      {
        const int s_n = valid ? (a.sigma[b * N + n] ? 1 : 0) : 0;
        const float e = (s_n == 0 ? 1.0f : 0.0f) - sigmoid_acc(z + dc);
        if (valid && part == 0) a.tape_e[(int64_t)n * B + b] = e;
        const float dz = coef * e;
#pragma unroll
        for (int q4 = 0; q4 < DU / 4; ++q4) {
          const float4 h4 = reinterpret_cast<const float4*>(hn)[q4];
          gU[4 * q4] = fmaf(dz, h4.x, gU[4 * q4]);
          gU[4 * q4 + 1] = fmaf(dz, h4.y, gU[4 * q4 + 1]);
          gU[4 * q4 + 2] = fmaf(dz, h4.z, gU[4 * q4 + 2]);
          gU[4 * q4 + 3] = fmaf(dz, h4.w, gU[4 * q4 + 3]);
        }
        gc += dz;
      }
      wait(0);
      tc::fence_after_sync();
      // ---- the five factors, 8 units at a time ----
#pragma unroll
      for (int sc = 0; sc < DU / 8; ++sc) {
        const int cu = u0 + 8 * sc;
        float acc[4][8];
        tmem_ld8(trow + cu, acc[0]);
        tmem_ld8(trow + D + cu, acc[1]);
        tmem_ld8(trow + 2 * D + cu, acc[2]);
        tmem_ld8(trow + 3 * D + cu, acc[3]);
        tmem_wait_regs(acc);
        float hv[8];
        {
          const float4 x0 = reinterpret_cast<const float4*>(hp)[2 * sc];
          const float4 x1 = reinterpret_cast<const float4*>(hp)[2 * sc + 1];
          hv[0] = x0.x; hv[1] = x0.y; hv[2] = x0.z; hv[3] = x0.w; hv[4] = x1.x; hv[5] = x1.y; hv[6] = x1.z; hv[7] = x1.w;
        }
        float k0[8], k1[8], k2[8], k3[8], k4[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float tu = hw_tanh(acc[0][q]), tr = hw_tanh(acc[1][q]);
          const float ug = fmaf(0.5f, tu, 0.5f), rg = fmaf(0.5f, tr, 0.5f);
          const float cg = hw_tanh(fmaf(rg, acc[2][q], acc[3][q]));
          k3[q] = ug * fmaf(-cg, cg, 1.0f);                      // u (1 - c^2)
          k2[q] = k3[q] * rg;
          k1[q] = k2[q] * acc[2][q] * (0.5f - 0.5f * tr);        // q (1 - r)
          k0[q] = (cg - hv[q]) * (0.25f * fmaf(-tu, tu, 1.0f));  // u (1 - u) = (1 - tanh^2) / 4
          k4[q] = 0.5f - 0.5f * tu;                              // 1 - u
        }
        if (valid) {
          uint4* kt = reinterpret_cast<uint4*>(a.tape_k);
          const int g = cu >> 3;
          kt[tape_k_group(B, n, 0, g, b, D)] = pack_f16x8(k0);
          kt[tape_k_group(B, n, 1, g, b, D)] = pack_f16x8(k1);
          kt[tape_k_group(B, n, 2, g, b, D)] = pack_f16x8(k2);
          kt[tape_k_group(B, n, 3, g, b, D)] = pack_f16x8(k3);
          kt[tape_k_group(B, n, 4, g, b, D)] = pack_f16x8(k4);
        }
      }
      // TMEM, the A tile, the readout exchange and buffer kp are free again
      tc::fence_before_sync();
      if (__syncthreads_or(timed_out)) { timed_out = true; break; }
      tc::fence_after_sync();
    }
    if (timed_out) break;                   // uniform
    // the run's last prefetch was not issued (n + 1 == n1): every buffer's
    // fills have been waited for, so the next run starts from a clean state
  }
  cp_async_wait_all();
  tc::fence_before_sync();
  // after a wait that gave up, TMEM is freed only once the MMAs have drained
  if (__syncthreads_or(timed_out) && threadIdx.x == 0) tc::drain_mmas(&mbar[4], kWaitLimit);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, S::kCols);
  // ---- this CTA's readout gradients: rows summed in a fixed order into one
  // partial row (U_1 and c_1 get the negatives: the softmax of two logits) ----
  float* red = sH;                         // [128 x HS] (the state buffers are free)
#pragma unroll
  for (int q4 = 0; q4 < DU / 4; ++q4)
    reinterpret_cast<float4*>(red + m * HS + u0)[q4] = make_float4(gU[4 * q4], gU[4 * q4 + 1], gU[4 * q4 + 2], gU[4 * q4 + 3]);
  if (part == 0) red[m * HS + D] = gc;
  __syncthreads();
  float* part_g = a.partial + (size_t)(part_row0 + blockIdx.x) * a.P;
  const int Uoff = 3 * D * D + 10 * D, coff = Uoff + 2 * D;   // U and c of the flat 1D layout
  for (int u = threadIdx.x; u <= D; u += NT) {
    float acc = 0.0f;
    for (int r = 0; r < 128; ++r) acc += red[r * HS + u];
    if (u < D) {
      part_g[Uoff + u] = acc;
      part_g[Uoff + D + u] = -acc;
    } else {
      part_g[coff] = acc;
      part_g[coff + 1] = -acc;
    }
  }
}

template <int D, int SPLIT, int ROWS>
struct BSmem {
  static constexpr int KA = D + 16;                       // X columns
  static constexpr int GW = 4 * D >= 128 ? 4 * D : 128;  // G row width (>= one M = 128 operand)
  static constexpr int RQ = ROWS / 32;                    // lane quarters holding distinct samples
  static constexpr int NS = (4 / RQ) * SPLIT;             // unit slices per sample
  static constexpr int DU = D / NS;                       // units per thread
  static constexpr int NB = ROWS <= 64 ? 2 : 1;           // tape buffers
  static constexpr int KB = 5 * D * ROWS * 2;             // tape buffer: [5][D/8][ROWS][8] fp16
  static constexpr int CS = D + 4;                        // acc_b exchange row stride (floats)
  static constexpr int kWt = 0;                           // [D x 3D] bf16, K-major
  static constexpr int kX = kWt + 3 * D * D * 2;          // 2 x [128 x KA] bf16
  static constexpr int kG = kX + 2 * 128 * KA * 2;        // [128 x GW] bf16
  static constexpr int kK = kG + 128 * GW * 2;            // NB tape buffers
  static constexpr int kC = kK + NB * KB;                 // [ROWS x CS] f32 (ROWS < 128)
  static constexpr int kDU = kC + (ROWS < 128 ? ROWS * CS * 4 : 0);   // D floats: U[0] - U[1]
  static constexpr int kBar = kDU + D * 4;                // 7 mbarriers (the last: drain)
  static constexpr int kSlot = kBar + 56;
  static constexpr int kBytes = 1024 + kSlot + 16;
  // TMEM columns: acc_b in three accumulators (one per gate block of G, so
  // that the K steps form three independent chains), acc_w in two halves
  static constexpr int cB = 0, cW0 = 3 * D, cW1 = 3 * D + KA;
  static constexpr int kCols = cW1 + KA <= 128 ? 128 : cW1 + KA <= 256 ? 256 : 512;
  static_assert(cW1 + KA <= kCols, "TMEM budget");
  static_assert(DU >= 8 && DU % 8 == 0 && ROWS % 32 == 0 && ROWS <= 128, "tile shape");
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
};

template <int D, int SPLIT, int ROWS>
__global__ void __launch_bounds__(128 * SPLIT, 1)
tc1d_bptt_kernel(const float* __restrict__ img, const uint8_t* __restrict__ wtimg, TcBpttArgs a) {
  using S = BSmem<D, SPLIT, ROWS>;
  constexpr int NT = 128 * SPLIT;
  constexpr int KA = S::KA, NB = S::NB, RQ = S::RQ, DU = S::DU, CS = S::CS;
  constexpr int DG = D / 8;                // 8-unit groups per state
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sWt = sm + S::kWt;
  uint8_t* sX = sm + S::kX;
  uint8_t* sG = sm + S::kG;
  uint8_t* sK = sm + S::kK;
  float* sC = reinterpret_cast<float*>(sm + S::kC);
  float* dU = reinterpret_cast<float*>(sm + S::kDU);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < 3 * D * D * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sWt)[i] = reinterpret_cast<const uint4*>(wtimg)[i];
  for (int i = threadIdx.x; i < D; i += NT) dU[i] = img[10 * D + i] - img[11 * D + i];
  for (int i = threadIdx.x; i < 128 * S::GW * 2 / 16; i += NT) reinterpret_cast<uint4*>(sG)[i] = make_uint4(0, 0, 0, 0);
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);              // MMA_b done
    tc::mbar_init(&mbar[1], 1);              // MMA_w done
    for (int k = 2; k < 6; ++k) tc::mbar_init(&mbar[k], NT);   // tape buffers 0, 1 and X buffers 0, 1 filled
    tc::mbar_init(&mbar[6], 2);              // drain: MMA issuers threads 0 and 32
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, S::kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  // thread -> (sample, unit slice): warp w is in TMEM lane quarter q = w % 4;
  // quarters q % RQ hold distinct samples s = 32 (q % RQ) + lane, and the
  // 4 / RQ quarters over a sample with the SPLIT warps of a quarter split
  // its units into NS slices of DU
  const int lane = threadIdx.x & 31, wt = threadIdx.x >> 5, q = wt % 4, p = wt / 4;
  const int s = 32 * (q % RQ) + lane;
  const int sl = (q / RQ) * SPLIT + p;
  const int u0 = sl * DU;
  const uint32_t tq = tbase + ((uint32_t)(32 * q) << 16);   // this warp's TMEM lanes
  const int N = a.N;
  const int64_t B = a.B;
  const int64_t b = (int64_t)blockIdx.x * ROWS + s;
  const bool valid = b < B;
  const float coef = valid ? 0.5f * a.weights[b] : 0.0f;
  bool timed_out = false;
  uint32_t phases = 0;                     // bit k: the phase of mbar[k] this thread waits for next
  auto wait = [&](int k) {
    if (!tc::mbar_wait(&mbar[k], (phases >> k) & 1u, wlim)) { timed_out = true; flag_status(a.hdr, NQS_ETIMEOUT); }
    phases ^= 1u << k;
  };
  // tape factors k_n of this thread's units into tape buffer kb (zeros past
  // the batch: G = 0 there).  Global groups of sample b: site n, vector c,
  // 8-unit group g at kt_b + n (5 DG B) + c (DG B) + g B.
  const uint4* kt_b = reinterpret_cast<const uint4*>(a.tape_k) + (valid ? b + (int64_t)(u0 >> 3) * B : 0);
  const uint4* xt_b = reinterpret_cast<const uint4*>(a.tape_x) + (valid ? b + (int64_t)(u0 >> 3) * B : 0);
  const int64_t vstride = (int64_t)DG * B;
  const uint32_t cpb = valid ? 16u : 0u;
  auto fetch_k = [&](int n, int kb) {
    uint8_t* dst = sK + kb * S::KB + ((u0 >> 3) * ROWS + s) * 16;
    const uint4* src = kt_b + (valid ? (int64_t)n * 5 * vstride : 0);
#pragma unroll
    for (int c = 0; c < 5; ++c) {
#pragma unroll
      for (int g = 0; g < DU / 8; ++g) cp_async16_zf(dst + (c * DG + g) * ROWS * 16, src + (valid ? g * B : 0), cpb);
      if (valid) src += vstride;
    }
    cp_async_arrive_noinc(&mbar[2 + kb]);
  };
  // X_n = [x_n | 1 1 | onehot(s_{n-1}) x2 | 0] into X buffer xb; s_in is
  // s_{n-1} (-1: none), loaded one site ahead
  auto fetch_x = [&](int n, int xb, int s_in) {
    uint8_t* xs = sX + xb * (128 * KA * 2);
    const uint4* src = xt_b + (valid ? (int64_t)n * vstride : 0);
#pragma unroll
    for (int g = 0; g < DU / 8; ++g)
      cp_async16_zf(xs + tc::kmajor_offset(s, u0 + 8 * g, KA), src + (valid ? g * B : 0), cpb);
    if (sl == 0) {
      const uint32_t one = 0x3F80u;
      const uint32_t oh = (s_in == 0 ? one : 0u) | ((s_in == 1 ? one : 0u) << 16);
      *reinterpret_cast<uint4*>(xs + tc::kmajor_offset(s, D, KA)) = make_uint4(one | (one << 16), oh, oh, 0u);
      *reinterpret_cast<uint4*>(xs + tc::kmajor_offset(s, D + 8, KA)) = make_uint4(0u, 0u, 0u, 0u);
    }
    cp_async_arrive_noinc(&mbar[4 + xb]);
  };
  float carry[DU];
#pragma unroll
  for (int u = 0; u < DU; ++u) carry[u] = 0.0f;

  constexpr uint32_t idesc_b = tc::make_idesc_bf16(128, D);
  constexpr uint32_t idesc_w = tc::make_idesc_bf16(128, KA) | (1u << 15) | (1u << 16);
  fetch_k(N - 1, (N - 1) % NB);
  if (NB == 2 && N > 1) fetch_k(N - 2, (N - 2) % NB);
  fetch_x(N - 1, (N - 1) & 1, (valid && N > 1) ? (ldg_u8(a.sigma + b * N + N - 2) ? 1 : 0) : -1);
  float e_cur = valid ? a.tape_e[(int64_t)(N - 1) * B + b] : 0.0f;
  uint32_t s_pre = (valid && N > 2) ? ldg_u8(a.sigma + b * N + N - 3) : 0u;   // s_{n-2} at site n

  for (int n = N - 1; n >= 0; --n) {
    const int xb = n & 1, kb = n % NB;
    // MMA_w of site n + 1 has read G and X buffer xb ^ 1
    if (n < N - 1) {
      wait(1);
      tc::fence_after_sync();
    }
    if (n > 0) fetch_x(n - 1, xb ^ 1, (valid && n > 1) ? (s_pre ? 1 : 0) : -1);
    s_pre = (valid && n > 2) ? ldg_u8(a.sigma + b * N + n - 3) : 0u;
    const float e_next = (valid && n > 0) ? a.tape_e[(int64_t)(n - 1) * B + b] : 0.0f;
    wait(2 + kb);
    const float dz0 = coef * e_cur;
    // ---- G = dh k_n, carry = dh k4, 8 units at a time ----
    const uint8_t* kr = sK + kb * S::KB + s * 16;
#pragma unroll
    for (int sc = 0; sc < DU / 8; ++sc) {
      const int cu = u0 + 8 * sc, gg = cu >> 3;
      float k0[8], k1[8], k2[8], k3[8], k4[8], w[8];
      unpack_f16x8(*reinterpret_cast<const uint4*>(kr + (0 * DG + gg) * ROWS * 16), k0);
      unpack_f16x8(*reinterpret_cast<const uint4*>(kr + (1 * DG + gg) * ROWS * 16), k1);
      unpack_f16x8(*reinterpret_cast<const uint4*>(kr + (2 * DG + gg) * ROWS * 16), k2);
      unpack_f16x8(*reinterpret_cast<const uint4*>(kr + (3 * DG + gg) * ROWS * 16), k3);
      unpack_f16x8(*reinterpret_cast<const uint4*>(kr + (4 * DG + gg) * ROWS * 16), k4);
      {
        const float4 w0 = reinterpret_cast<const float4*>(dU + cu)[0];
        const float4 w1 = reinterpret_cast<const float4*>(dU + cu)[1];
        w[0] = w0.x; w[1] = w0.y; w[2] = w0.z; w[3] = w0.w; w[4] = w1.x; w[5] = w1.y; w[6] = w1.z; w[7] = w1.w;
      }
      float g0[8], g1[8], g2[8], g3[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int j = 8 * sc + i;
        const float dh = fmaf(dz0, w[i], carry[j]);
        g0[i] = dh * k0[i];
        g1[i] = dh * k1[i];
        g2[i] = dh * k2[i];
        g3[i] = dh * k3[i];
        carry[j] = dh * k4[i];                           // direct path; acc_b adds the rest
      }
      st_bf16x8(sG + tc::kmajor_offset(s, cu, S::GW), g0);
      st_bf16x8(sG + tc::kmajor_offset(s, D + cu, S::GW), g1);
      st_bf16x8(sG + tc::kmajor_offset(s, 2 * D + cu, S::GW), g2);
      st_bf16x8(sG + tc::kmajor_offset(s, 3 * D + cu, S::GW), g3);
    }
    // this thread has read its part of tape buffer kb: it takes site n - NB
    if (n - NB >= 0) fetch_k(n - NB, kb);
    wait(4 + xb);                          // X_n is in place
    e_cur = e_next;
    tc::fence_async_smem();
    tc::fence_before_sync();
    // a wait that ran out anywhere in the CTA ends the sweep for every thread here
    if (__syncthreads_or(timed_out)) { timed_out = true; break; }
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
      // dh_{n-1} = G[:, :3D] W3 as three K chains, one per gate block j
      // (acc_b^j = G_j W3_j; K-major: LBO = 128 B along K, SBO = row-group
      // stride), issued interleaved so that the chains overlap
#pragma unroll
      for (int kk = 0; kk < D / 16; ++kk)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int k = j * (D / 16) + kk;
          const uint64_t da = tc::make_desc(tc::smem_addr(sG) + k * 256, 128, (S::GW / 8) * 128);
          const uint64_t db = tc::make_desc(tc::smem_addr(sWt) + k * 256, 128, (3 * D / 8) * 128);
          tc::mma_bf16(tbase + S::cB + j * D, da, db, idesc_b, kk > 0);
        }
      tc::mma_commit(&mbar[0]);
    } else if (threadIdx.x == 32) {
      // acc_w += G^T X_n over the tile's ROWS samples, halves of 128 gate
      // rows, issued by a second warp alongside MMA_b.  Both operands
      // MN-major: LBO = stride of 8-sample groups along K (the buffer's
      // row-group stride), SBO = 128 B between 8-column groups along M / N.
      // One K = 16 step covers two sample groups.
      const uint32_t xs = tc::smem_addr(sX) + xb * (128 * KA * 2);
#pragma unroll
      for (int half = 0; half < S::GW / 128; ++half) {
#pragma unroll
        for (int k = 0; k < ROWS / 16; ++k) {
          const uint64_t da = tc::make_desc(tc::smem_addr(sG) + half * 16 * 128 + k * 2 * (S::GW / 8) * 128,
                                            (S::GW / 8) * 128, 128);
          const uint64_t db = tc::make_desc(xs + k * 2 * (KA / 8) * 128, (KA / 8) * 128, 128);
          tc::mma_bf16(tbase + (half ? S::cW1 : S::cW0), da, db, idesc_w, (n < N - 1) || k > 0);
        }
      }
      tc::mma_commit(&mbar[1]);
    }
    // ---- carry += acc_b ----
    if constexpr (ROWS == 128) {
      wait(0);
      tc::fence_after_sync();
#pragma unroll
      for (int c = 0; c < DU / 8; ++c) {
        float v0[8], v1[8], v2[8];
        tmem_ld8(tq + S::cB + u0 + 8 * c, v0);
        tmem_ld8(tq + S::cB + D + u0 + 8 * c, v1);
        tmem_ld8(tq + S::cB + 2 * D + u0 + 8 * c, v2);
        tc::tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          asm volatile("" : "+f"(v0[i]), "+f"(v1[i]), "+f"(v2[i]));
          carry[8 * c + i] += (v0[i] + v1[i]) + v2[i];
        }
      }
    } else {
      // the quarters holding the samples' lanes pass acc_b on through shared memory
      if (q < RQ) {
        wait(0);
        tc::fence_after_sync();
        constexpr int CW = D / SPLIT;      // columns per warp of the quarter
#pragma unroll
        for (int c = 0; c < CW / 8; ++c) {
          float v0[8], v1[8], v2[8];
          tmem_ld8(tq + S::cB + p * CW + 8 * c, v0);
          tmem_ld8(tq + S::cB + D + p * CW + 8 * c, v1);
          tmem_ld8(tq + S::cB + 2 * D + p * CW + 8 * c, v2);
          tc::tmem_wait_ld();
          float v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            asm volatile("" : "+f"(v0[i]), "+f"(v1[i]), "+f"(v2[i]));
            v[i] = (v0[i] + v1[i]) + v2[i];
          }
          float4* dst = reinterpret_cast<float4*>(sC + s * CS + p * CW + 8 * c);
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
      tc::fence_before_sync();
      __syncthreads();
      tc::fence_after_sync();
#pragma unroll
      for (int c = 0; c < DU / 4; ++c) {
        const float4 x = reinterpret_cast<const float4*>(sC + s * CS + u0)[c];
        carry[4 * c] += x.x;
        carry[4 * c + 1] += x.y;
        carry[4 * c + 2] += x.z;
        carry[4 * c + 3] += x.w;
      }
    }
  }
  // the last MMA_w, before acc_w is read; copies still in flight (after a
  // timeout) land before the CTA leaves
  if (threadIdx.x == 0 && !timed_out) wait(1);
  cp_async_wait_all();
  tc::fence_before_sync();
  // after a wait that gave up, acc_w is read and TMEM freed only once every
  // MMA_b and MMA_w has drained
  if (__syncthreads_or(timed_out) && (threadIdx.x == 0 || threadIdx.x == 32))
    tc::drain_mmas(&mbar[6], kWaitLimit);
  __syncthreads();
  tc::fence_after_sync();
  // ---- this CTA's weight, bias and one-hot-column gradients from acc_w (warps 0-3) ----
  // X columns: k < D: h; D: bias; D + 2, D + 3: one-hot weights (D + 1, D + 4 .. are duplicates / zero)
  const int Wg = 0, Wr = D * (D + 2), Wh = 2 * D * (D + 2), Win = Wh + D * D;
  const int bg = Win + 2 * D, br = bg + D, bh = br + D, bin = bh + D;
  float* part_g = a.partial + (size_t)blockIdx.x * a.P;
  if (p == 0) {
    const int m = 32 * q + lane;           // gate row (TMEM lane) of this thread
#pragma unroll 1
    for (int half = 0; half < S::GW / 128; ++half) {
      const int gu = half * 128 + m;
      const int g = gu / D, u = gu % D;
#pragma unroll 1
      for (int c = 0; c < KA; c += 16) {
        float v[16];
        tc::tmem_ld16(tq + (half ? S::cW1 : S::cW0) + c, v);
        tc::tmem_wait_ld();
        if (gu >= 4 * D) continue;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = c + i;
          if (k < D) {
            if (g == 0) part_g[Wg + u * (D + 2) + k] = v[i];
            else if (g == 1) part_g[Wr + u * (D + 2) + k] = v[i];
            else if (g == 2) part_g[Wh + u * D + k] = v[i];
          } else if (k == D) {
            part_g[(g == 0 ? bg : g == 1 ? br : g == 2 ? bh : bin) + u] = v[i];
          } else if (k == D + 2 || k == D + 3) {
            const int si = k - D - 2;
            if (g == 0) part_g[Wg + u * (D + 2) + D + si] = v[i];
            else if (g == 1) part_g[Wr + u * (D + 2) + D + si] = v[i];
            else if (g == 3) part_g[Win + u * 2 + si] = v[i];
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, S::kCols);
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

template <int D, int MODE, int GROUPS, int SPLIT, int REP = 1>
cudaError_t launch_tc(const Tc1Args& a, const float* img, const uint8_t* wimg, cudaStream_t st) {
  using S = Smem<D, GROUPS, SPLIT>;
  auto k = tc1d_engine_kernel<D, MODE, GROUPS, SPLIT, REP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  int64_t grid;
  if (MODE == 2) {
    const int64_t jobs = a.B * (int64_t)(a.N - 1);
    grid = sm_count_tc();
    const int64_t need = (jobs + 128 * GROUPS - 1) / (128 * GROUPS);
    if (grid > need) grid = need;
  } else {
    grid = (a.B + (int64_t)a.rows * GROUPS - 1) / ((int64_t)a.rows * GROUPS);
  }
  if (grid < 1) grid = 1;
  k<<<(unsigned)grid, 128 * GROUPS * SPLIT, S::kBytes, st>>>(img, wimg, a);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Autotuner: each kernel has a few tile variants (threads per row).  The first
// call for a (kernel, d_h, N, B) key that is not inside a stream capture runs
// every variant twice on the call's own inputs, times the second run with
// CUDA events (this synchronises the stream once) and caches the fastest; the
// outputs of the final launch are those of the chosen variant (every variant
// computes the same values).  Inside a capture, or with tuning off, the cached
// choice or the first variant is used.
// ----------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, long long>, int> g_tune;
bool g_tune_on = true;
int g_force = -1;            // >= 0: every kernel uses this variant (the last one it has if fewer)

template <typename Launch, typename Prep>
cudaError_t tuned_launch(int kind, int D, int N, int64_t B, int nvar, Launch launch, Prep prep, cudaStream_t st) {
  const auto key = std::make_tuple(kind, D, N, (long long)B);
  int choice = -1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (g_force >= 0) {
      choice = g_force < nvar ? g_force : nvar - 1;
    } else {
      auto it = g_tune.find(key);
      if (it != g_tune.end()) choice = it->second;
    }
  }
  cudaError_t e;
  if (choice < 0) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) { cudaGetLastError(); cap = cudaStreamCaptureStatusActive; }
    if (!g_tune_on || nvar == 1 || cap != cudaStreamCaptureStatusNone) {
      choice = 0;
    } else {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      float best = 1e30f;
      for (int v = 0; v < nvar; ++v) {
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          if ((e = prep()) != cudaSuccess) return e;
          cudaEventRecord(e0, st);
          if ((e = launch(v)) != cudaSuccess) return e;
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          cudaEventElapsedTime(&ms, e0, e1);
        }
        if (ms < best) { best = ms; choice = v; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune[key] = choice;
    }
  }
  if ((e = prep()) != cudaSuccess) return e;
  return launch(choice);
}

template <int D>
cudaError_t dispatch_mode(const Tc1Args& a, const float* img, const uint8_t* wimg, int mode, cudaStream_t st) {
  auto none = []() { return cudaSuccess; };
  if constexpr (D == 128) {
    // one tile per CTA (its 3D accumulator columns take TMEM's 512), 2 or 4
    // threads per row (64 or 32 units each); chains without ping-pong
    if (mode == 2) {
      auto reset = [&]() { return cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st); };
      Tc1Args c = a;
      c.rows = 128;
      auto run = [&](int v) {
        return v == 1 ? launch_tc<D, 2, 1, 4>(c, img, wimg, st) : launch_tc<D, 2, 1, 2>(c, img, wimg, st);
      };
      return tuned_launch(2, D, a.N, a.B, 2, run, reset, st);
    }
    auto run = [&](int v) {
      Tc1Args b = a;
      b.rows = 128 >> (v / 2);
      if (mode == 0) return v % 2 ? launch_tc<D, 0, 1, 4>(b, img, wimg, st) : launch_tc<D, 0, 1, 2>(b, img, wimg, st);
      return v % 2 ? launch_tc<D, 1, 1, 4>(b, img, wimg, st) : launch_tc<D, 1, 1, 2>(b, img, wimg, st);
    };
    return tuned_launch(mode, D, a.N, a.B, 6, run, none, st);
  } else {
    if (mode == 2) {
      // chains: 1 or 2 threads per row (the work counter is reset before every run)
      auto reset = [&]() { return cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st); };
      Tc1Args c = a;
      c.rows = 128;
      auto run = [&](int v) {
        if (v == 1 && D >= 32) return launch_tc<D, 2, 2, (D >= 32 ? 2 : 1)>(c, img, wimg, st);
        return launch_tc<D, 2, 2, 1>(c, img, wimg, st);
      };
      return tuned_launch(2, D, a.N, a.B, D >= 32 ? 2 : 1, run, reset, st);
    }
    // sampling / teacher forcing: 1, 2 or 4 threads per row, times 128, 64 or
    // 32 rows per tile (partly filled tiles put more SMs on a small batch); at
    // d_h = 64 the 32-row tile has its A rows in all four lane quarters instead
    const int ns = D >= 64 ? 3 : (D >= 32 ? 2 : 1);
    auto run = [&](int v) {
      Tc1Args b = a;
      b.rows = 128 >> (v / ns);
      const int sv = v % ns;
      if constexpr (D == 64) {
        if (v >= 2 * ns) {
          b.rows = 32;
          return mode == 0 ? launch_tc<D, 0, 1, 1, 4>(b, img, wimg, st) : launch_tc<D, 1, 1, 1, 4>(b, img, wimg, st);
        }
      }
      if (mode == 0) {
        if (sv == 2 && D >= 64) return launch_tc<D, 0, 1, (D >= 64 ? 4 : 1)>(b, img, wimg, st);
        if (sv == 1 && D >= 32) return launch_tc<D, 0, 1, (D >= 32 ? 2 : 1)>(b, img, wimg, st);
        return launch_tc<D, 0, 1, 1>(b, img, wimg, st);
      }
      if (sv == 2 && D >= 64) return launch_tc<D, 1, 1, (D >= 64 ? 4 : 1)>(b, img, wimg, st);
      if (sv == 1 && D >= 32) return launch_tc<D, 1, 1, (D >= 32 ? 2 : 1)>(b, img, wimg, st);
      return launch_tc<D, 1, 1, 1>(b, img, wimg, st);
    };
    return tuned_launch(mode, D, a.N, a.B, D == 64 ? 2 * ns + 1 : 3 * ns, run, none, st);
  }
}

}  // namespace

int tc1d_supported(int D) { return D == 16 || D == 32 || D == 64 || D == 128; }

void tc1d_set_autotune(int on) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_on = on != 0;
  if (!on) g_tune.clear();
}

void tc1d_set_variant(int v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_force = v < 0 ? -1 : v;
}

int tc1d_pinned_variant() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return g_force;
}

// rows of per-CTA partial gradients: the reverse sweep's CTAs (at most one per
// 32 samples) and then the tape kernel's CTAs (readout gradients)
constexpr int kTapeRows = 304;
int bptt_sweep_rows(int64_t B) { return (int)((B + 31) / 32); }
int tc1d_bptt_partial_rows(int64_t B) { return bptt_sweep_rows(B) + kTapeRows; }
size_t tc1d_tape_bytes(int64_t B, int N, int D, int which) {
  const size_t BN = (size_t)B * (size_t)N;
  return which == 0 ? BN * sizeof(float) : which == 1 ? BN * D * 2 : BN * 5 * D * 2;
}

template <int D, int SPLIT, int ROWS>
cudaError_t launch_tc_bptt_v(const TcBpttArgs& a, const float* img, const uint8_t* wt, cudaStream_t st) {
  using S = BSmem<D, SPLIT, ROWS>;
  auto k = tc1d_bptt_kernel<D, SPLIT, ROWS>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  const int grid = (int)((a.B + ROWS - 1) / ROWS);
  k<<<grid, 128 * SPLIT, S::kBytes, st>>>(img, wt, a);
  return cudaGetLastError();
}

// Reverse-sweep variants (rows per tile, threads per row) with at least 8
// units per thread; the autotuner picks one.
template <int D>
constexpr int bptt_variants() { return D == 64 ? 8 : D == 32 ? 5 : 3; }

template <int D>
cudaError_t launch_tc_bptt_n(const TcBpttArgs& a, const float* img, const uint8_t* wt, int v, cudaStream_t st) {
  if constexpr (D == 64) {
    switch (v) {
      case 0: return launch_tc_bptt_v<64, 1, 128>(a, img, wt, st);
      case 1: return launch_tc_bptt_v<64, 2, 128>(a, img, wt, st);
      case 2: return launch_tc_bptt_v<64, 4, 128>(a, img, wt, st);
      case 3: return launch_tc_bptt_v<64, 1, 64>(a, img, wt, st);
      case 4: return launch_tc_bptt_v<64, 2, 64>(a, img, wt, st);
      case 5: return launch_tc_bptt_v<64, 4, 64>(a, img, wt, st);
      case 6: return launch_tc_bptt_v<64, 1, 32>(a, img, wt, st);
      default: return launch_tc_bptt_v<64, 2, 32>(a, img, wt, st);
    }
  } else if constexpr (D == 32) {
    switch (v) {
      case 0: return launch_tc_bptt_v<32, 1, 128>(a, img, wt, st);
      case 1: return launch_tc_bptt_v<32, 2, 128>(a, img, wt, st);
      case 2: return launch_tc_bptt_v<32, 1, 64>(a, img, wt, st);
      case 3: return launch_tc_bptt_v<32, 2, 64>(a, img, wt, st);
      default: return launch_tc_bptt_v<32, 1, 32>(a, img, wt, st);
    }
  } else {
    switch (v) {
      case 0: return launch_tc_bptt_v<D, 1, 128>(a, img, wt, st);
      case 1: return launch_tc_bptt_v<D, 2, 128>(a, img, wt, st);
      default: return launch_tc_bptt_v<D, 1, 64>(a, img, wt, st);
    }
  }
}

// The tape: one CTA per SM, each on runs of consecutive sites of one sample
// tile (a run reads each cached state row once, plus one row before it).
struct TapeGrid {
  int grid, sites_per_run, runs_per_tile;
};
TapeGrid tape_grid(int64_t B, int N) {
  const int64_t tiles = (B + 127) / 128;
  const int sms = sm_count_tc();
  TapeGrid t;
  t.runs_per_tile = tiles >= sms ? 1 : (int)(sms / tiles);
  t.sites_per_run = (N + t.runs_per_tile - 1) / t.runs_per_tile;
  int64_t grid = tiles * t.runs_per_tile;
  if (grid > sms) grid = sms;
  if (grid > kTapeRows) grid = kTapeRows;
  t.grid = grid < 1 ? 1 : (int)grid;
  return t;
}

template <int D>
cudaError_t launch_tape(const TcBpttArgs& a, const float* img, const uint8_t* w3, cudaStream_t st) {
  using S = TpS<D>;
  auto k = tc1d_tape_kernel<D>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  const TapeGrid t = tape_grid(a.B, a.N);
  k<<<(unsigned)t.grid, S::NT, S::kBytes, st>>>(img, w3, a, t.sites_per_run, t.runs_per_tile, bptt_sweep_rows(a.B));
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_tc_bptt(const TcBpttArgs& a, const float* img, const uint8_t* w3, const uint8_t* wt, cudaStream_t st) {
  // reverse sweep: 1, 2 or 4 threads per row, times 128, 64 or 32 rows per
  // tile, picked by the autotuner (fewer rows put more SMs on the sequential
  // sweep of a small batch).  A run writes one partial row per CTA (at most
  // B/32 rows) and the reduction sums all rows, so the sweep's rows are
  // cleared before every run: an autotuning trial with fewer rows per tile
  // leaves rows that a final run with more rows per tile would not overwrite.
  // The tape launch comes first; the sweep only reads it.
  cudaError_t e = launch_tape<D>(a, img, w3, st);
  if (e != cudaSuccess) return e;
  auto run = [&](int v) { return launch_tc_bptt_n<D>(a, img, wt, v, st); };
  const int rows_max = bptt_sweep_rows(a.B);
  auto clear = [&]() {
    return cudaMemsetAsync(a.partial, 0, (size_t)rows_max * a.P * sizeof(float), st);
  };
  return tuned_launch(3, D, a.N, a.B, bptt_variants<D>(), run, clear, st);
}

// Partial rows: the sweep's rows (cleared before the sweep, so rows past the
// chosen variant's CTAs are zero) carry the weight, bias and one-hot-column
// gradients, columns [0, U); the tape CTAs' rows carry the readout gradients,
// columns [U, P).  Each block of columns is summed over its own rows.
template <typename T>
static cudaError_t bptt_reduce(const TcBpttArgs& a, int D, T* grad, cudaStream_t st) {
  const int rows = bptt_sweep_rows(a.B);
  const int Uoff = 3 * D * D + 10 * D;
  cudaError_t e = reduce_partials_cols(a.partial, rows, Uoff, a.P, grad, st);
  if (e != cudaSuccess) return e;
  return reduce_partials_cols(a.partial + (size_t)rows * a.P + Uoff, tape_grid(a.B, a.N).grid, a.P - Uoff, a.P,
                              grad + Uoff, st);
}
cudaError_t tc1d_bptt_reduce(const TcBpttArgs& a, int D, float* grad, cudaStream_t st) {
  return bptt_reduce(a, D, grad, st);
}
cudaError_t tc1d_bptt_reduce(const TcBpttArgs& a, int D, double* grad, cudaStream_t st) {
  return bptt_reduce(a, D, grad, st);
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
size_t tc1d_wimg_bytes(int D) { return (size_t)4 * D * (D + 16) * 2; }

cudaError_t tc1d_pack(const float* params, uint8_t* wimg, int D, cudaStream_t st) {
  const int total = 4 * D * (D + 16);
  pack1d_tc_kernel<<<(total + 255) / 256, 256, 0, st>>>(params, wimg, D);
  return cudaGetLastError();
}

cudaError_t tc1d_run(const Tc1Args& a, const float* img, const uint8_t* wimg, int D, int mode, cudaStream_t st) {
  switch (D) {
    case 16: return dispatch_mode<16>(a, img, wimg, mode, st);
    case 32: return dispatch_mode<32>(a, img, wimg, mode, st);
    case 64: return dispatch_mode<64>(a, img, wimg, mode, st);
    case 128: return dispatch_mode<128>(a, img, wimg, mode, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nqs

namespace nqs {
uint32_t tc_default_wait_polls() { return tc::kDefaultWaitPolls; }
cudaError_t tc1d_set_wait_polls(uint32_t polls) { return cudaMemcpyToSymbol(tc::g_wait_polls, &polls, sizeof(polls)); }
}  // namespace nqs

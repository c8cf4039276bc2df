// Pieces shared by the streamed-weight BF16 reverse sweeps (tc2d_wide.cu,
// tc1d_grad128.cu): bulk asynchronous copies, the layout of the per-cell
// operand tapes, and the weight-gradient GEMM over them.
//
// A weight gradient is a sum over every (sample, position) cell of an outer
// product: dW = sum_cells G_cell X_cell^T, G the gradients of a block of
// pre-activations and X the cell's inputs.  The reverse sweeps write G and X
// to tapes in which each block of 16 cells and each tile of columns is one
// contiguous MN-major BF16 operand (rows = cells = the GEMM's K), so the GEMM
// streams whole blocks with one bulk copy each and feeds them to tcgen05
// with both operands MN-major.
#pragma once

#include <cuda_bf16.h>

#include "kernels.h"
#include "tc.cuh"

namespace nqs {
namespace tcw {
namespace {

// Bulk asynchronous copy global -> shared, completing on an mbarrier's
// transaction count (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" : : "r"(tc::smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               :
               : "r"(tc::smem_addr(dst)), "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
               : "memory");
}

// Byte offset of element (cell c, column v) in an operand tape: columns split
// into tiles of TW, cells into blocks of 16; each (tile, block) is one
// contiguous MN-major [16 x TW] BF16 operand (rows = cells = K, LBO = (TW / 8)
// * 128, SBO = 128).  v is a multiple of 8 (a 16-byte piece of one cell).
__device__ __forceinline__ size_t tape_off(int64_t c, int v, int TW, int64_t nkb) {
  const int tile = v / TW, vv = v % TW, r = (int)(c & 15);
  return ((size_t)tile * nkb + (size_t)(c >> 4)) * (size_t)(16 * TW * 2) + (size_t)((r >> 3) * (TW / 8) * 128) +
         (size_t)((vv >> 3) * 128) + (size_t)((r & 7) * 16);
}
__device__ __forceinline__ uint4 pack8_bf16(const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    w[q] = *reinterpret_cast<uint32_t*>(&p);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// One output tile: D[128 x (TWB + 16)] = sum over the cell blocks of A^T [Bm | Bx],
// A a 128-column tile of a G tape, Bm a TWB-column tile of an X tape and Bx
// (nullable) its 16 extra columns [1 | one-hots | 0].
struct WgTile {
  const uint8_t* A;
  const uint8_t* Bm;
  const uint8_t* Bx;
};
constexpr int kWgMaxTiles = 16, kWgRing = 8;
struct WgArgs {
  WgTile tiles[kWgMaxTiles];
  int64_t nkb;               // 16-cell blocks
  int splits;                // cell ranges per tile: work unit = tile * splits + range
  float* out;                // [units][128][TWB + 16] FP32 sums
  WsHeader* hdr;
};

template <int TWB>
struct WgS {
  static constexpr uint32_t kABytes = 4096, kBBytes = 16 * TWB * 2, kXBytes = 512;
  static constexpr uint32_t kSlot = kABytes + kBBytes + kXBytes;
  static constexpr int kCols = TWB + 16;
  static constexpr uint32_t kTmemCols = kCols <= 256 ? 256 : 512;
  static constexpr uint32_t kBar = kWgRing * kSlot;                    // full[R], empty[R], done, drain
  static constexpr uint32_t kMisc = kBar + (2 * kWgRing + 2) * 8;
  static constexpr uint32_t kBytes = 1024 + kMisc + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
};

// One work unit per CTA: one thread streams the unit's blocks through an
// 8-slot ring (bulk copies, full / empty mbarriers) and issues one or two
// MMAs per block (M = 128, N = TWB and 16, K = 16 cells); all four warps then
// move the FP32 sums from TMEM to the unit's output rows.
template <int TWB>
__global__ void __launch_bounds__(128, 1) wgrad_kernel(WgArgs a) {
  using S = WgS<TWB>;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;
  uint8_t* ring = sm;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint64_t* empty = full + kWgRing;
  uint64_t* done = empty + kWgRing;
  uint64_t* drain = done + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kMisc);
  const int unit = blockIdx.x, split = unit % a.splits;
  const WgTile tl = a.tiles[unit / a.splits];
  const int64_t kps = (a.nkb + a.splits - 1) / a.splits, kb0 = (int64_t)split * kps;
  const int64_t kb1 = kb0 + kps < a.nkb ? kb0 + kps : a.nkb;
  const int64_t nk = kb1 > kb0 ? kb1 - kb0 : 0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < kWgRing; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(drain, 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, S::kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  bool timed_out = false;
  if (threadIdx.x == 0 && nk > 0) {
    // both operands MN-major: rows = 16 cells (K), columns = 128 G rows (M) or inputs (N)
    constexpr uint32_t im = tc::make_idesc_bf16(128, TWB) | (1u << 15) | (1u << 16);
    constexpr uint32_t ix = tc::make_idesc_bf16(128, 16) | (1u << 15) | (1u << 16);
    const uint32_t r_addr = tc::smem_addr(ring);
    const uint32_t bytes = S::kABytes + S::kBBytes + (tl.Bx ? S::kXBytes : 0);
    int64_t s_cons = 0, s_fill = 0;
    bool dead = false;
    auto fill = [&]() {
      if (dead || s_fill >= nk) return;
      const int64_t s = s_fill;
      const uint32_t slot = (uint32_t)(s % kWgRing);
      if (s >= kWgRing && !tc::mbar_wait(&empty[slot], (uint32_t)((s / kWgRing) - 1) & 1, wlim)) {
        dead = true;
        return;
      }
      uint8_t* d = ring + slot * S::kSlot;
      const int64_t kb = kb0 + s;
      mbar_expect_tx(&full[slot], bytes);
      bulk_g2s(d, tl.A + (size_t)kb * S::kABytes, S::kABytes, &full[slot]);
      bulk_g2s(d + S::kABytes, tl.Bm + (size_t)kb * S::kBBytes, S::kBBytes, &full[slot]);
      if (tl.Bx) bulk_g2s(d + S::kABytes + S::kBBytes, tl.Bx + (size_t)kb * S::kXBytes, S::kXBytes, &full[slot]);
      ++s_fill;
    };
    for (int q = 0; q < kWgRing; ++q) fill();
    while (!dead && s_cons < nk) {
      const int64_t s = s_cons;
      const uint32_t slot = (uint32_t)(s % kWgRing);
      if (!tc::mbar_wait(&full[slot], (uint32_t)(s / kWgRing) & 1, wlim)) {
        dead = true;
        break;
      }
      tc::fence_after_sync();
      const uint32_t sa = r_addr + slot * S::kSlot;
      const uint32_t accf = s > 0 ? 1u : 0u;
      const uint64_t da = tc::make_desc(sa, 2048, 128);
      tc::mma_bf16(tbase, da, tc::make_desc(sa + S::kABytes, (TWB / 8) * 128, 128), im, accf);
      if (tl.Bx) tc::mma_bf16(tbase + TWB, da, tc::make_desc(sa + S::kABytes + S::kBBytes, 256, 128), ix, accf);
      tc::mma_commit(&empty[slot]);
      ++s_cons;
      while (!dead && s_fill < nk && s_fill < s_cons + kWgRing - 1) fill();
    }
    tc::mma_commit(done);
    if (dead) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    // no copy may still be landing when the CTA exits
    for (int64_t s = s_cons; s < s_fill; ++s)
      tc::mbar_wait(&full[(uint32_t)(s % kWgRing)], (uint32_t)(s / kWgRing) & 1, tc::kDefaultWaitPolls);
  }
  __syncwarp();
  if (nk > 0 && !tc::mbar_wait(done, 0, wlim)) {
    timed_out = true;
    flag_status(a.hdr, NQS_ETIMEOUT);
  }
  tc::fence_after_sync();
  // lane m of the accumulator = output row m
  const int w = threadIdx.x >> 5, m = threadIdx.x;
  const uint32_t trow = tbase + ((uint32_t)(w * 32) << 16);
  float* out = a.out + ((size_t)unit * 128 + m) * S::kCols;
  const int ncol = tl.Bx ? S::kCols : TWB;
  for (int c = 0; c < ncol; c += 8) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(trow + c));
    tc::tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < 8; ++q) asm volatile("" : "+r"(r[q]));
    float4 v0 = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
    float4 v1 = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]), __uint_as_float(r[7]));
    if (nk == 0 || timed_out) v0 = v1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    reinterpret_cast<float4*>(out + c)[0] = v0;
    reinterpret_cast<float4*>(out + c)[1] = v1;
  }
  tc::fence_before_sync();
  if (__syncthreads_or(timed_out) && threadIdx.x == 0) tc::drain_mmas(drain, tc::kDefaultWaitPolls);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, S::kTmemCols);
}

template <int TWB>
cudaError_t launch_wgrad(const WgArgs& a, int ntiles, cudaStream_t st) {
  auto k = wgrad_kernel<TWB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, WgS<TWB>::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  k<<<ntiles * a.splits, 128, WgS<TWB>::kBytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace
}  // namespace tcw
}  // namespace nqs

// Helpers shared by the BF16 tensor-core 2D kernels (tc2d.cu, tc2d_grad.cu):
// hi / lo BF16 splitting of FP32 states, tcgen05 loads, cp.async, zig-zag
// geometry (Sec. II, Fig. 1(b)) and the zero-magnetisation mask.
#pragma once

#include "kernels.h"
#include "tc.cuh"

namespace nqs {
namespace tc2dh {

constexpr uint32_t kWait2 = tc::kDefaultWaitPolls;   // the drain's bound (mbarrier polls)

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float hw_tanh2(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&p);
}
// hi and lo BF16 pairs of two values: hi = bf16(v), lo = bf16(v - hi)
__device__ __forceinline__ void split_bf16(float a, float b, uint32_t& hi, uint32_t& lo) {
  hi = pack_bf16(a, b);
  lo = pack_bf16(a - bf16_round(a), b - bf16_round(b));
}
// 8 values as hi / lo 16-byte rows of an operand
__device__ __forceinline__ void st_split8(uint8_t* dhi, uint8_t* dlo, const float* v) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) split_bf16(v[2 * q], v[2 * q + 1], h[q], l[q]);
  *reinterpret_cast<uint4*>(dhi) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(dlo) = make_uint4(l[0], l[1], l[2], l[3]);
}
__device__ __forceinline__ void cp_async16_2d(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" : : "r"(tc::smem_addr(smem)), "l"(gmem) : "memory");
}
// L2-only variant (the source may have been written by this thread earlier in the kernel)
__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" : : "r"(tc::smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit_2d() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_2d() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ float ldg_f32_v(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];\n" : "=f"(v) : "l"(p));
  return v;
}

// 8 consecutive 32-bit TMEM columns of this thread's lane (warp-collective).
__device__ __forceinline__ void tld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
// 16 consecutive 32-bit TMEM columns of this thread's lane (warp-collective).
__device__ __forceinline__ void tld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Ties loaded registers to the preceding wait: no use is scheduled above it.
template <int NW>
__device__ __forceinline__ void tie(uint32_t (&r)[NW]) {
#pragma unroll
  for (int q = 0; q < NW; ++q) asm volatile("" : "+r"(r[q]));
}

// Zig-zag geometry (Sec. II, Fig. 1(b)), as in the FP32 path.
struct Pz {
  int i, j, r;
};
__device__ __forceinline__ Pz zpos(int t, int Lx) {
  Pz p;
  p.j = t / Lx;
  p.r = t - p.j * Lx;
  p.i = (p.j & 1) ? Lx - 1 - p.r : p.r;
  return p;
}
__device__ __forceinline__ int zhor(const Pz& p) { return (p.j & 1) ? p.i + 1 : p.i - 1; }
__device__ __forceinline__ int zsnake(int i, int j, int Lx) { return j * Lx + ((j & 1) ? Lx - 1 - i : i); }

// A configuration of up to 64 NW spins as a bit mask (bit k = spin of lattice site k).
// The word is chosen by selects, not by a runtime index, so the mask stays in
// registers.
template <int NW>
__device__ __forceinline__ int mbit(const uint64_t (&m)[NW], int k) {
  uint64_t w = m[0];
#pragma unroll
  for (int i = 1; i < NW; ++i) w = (k >> 6) == i ? m[i] : w;
  return (int)((w >> (k & 63)) & 1ull);
}
template <int NW>
__device__ __forceinline__ void mset(uint64_t (&m)[NW], int k, int s) {
  const uint64_t b = 1ull << (k & 63);
#pragma unroll
  for (int i = 0; i < NW; ++i)
    if ((k >> 6) == i) m[i] = s ? (m[i] | b) : (m[i] & ~b);
}

// Heisenberg chain job: one antiparallel (sample, bond) pair with the start
// values of its chain taken from the cached-path tables.
// The bond travels in the record (no dependent load of the bond table when a
// chain starts): rank_pa_a = rank | pa << 10 | site a << 18 (pa = the earlier
// zig-zag position of the bond, at site a; rank < 1024, pa, a < 256 for N <=
// 256), nup_b = nup0 | site b << 16.
template <int NW>
struct JobT {
  int b, rank_pa_a;
  float acc0;          // 1/2 [log p_pa(s_new) - log p_pa(s_old)]
  int nup_b;           // up spins before pa+1 on the exchanged configuration | site b << 16
  uint64_t mask[NW];   // exchanged configuration, bit k = spin of lattice site k
};
__host__ __device__ __forceinline__ int job_rank(int rpa) { return rpa & 1023; }
__host__ __device__ __forceinline__ int job_pa(int rpa) { return (rpa >> 10) & 255; }
__host__ __device__ __forceinline__ int job_site_a(int rpa) { return (rpa >> 18) & 255; }
__host__ __device__ __forceinline__ int job_nup(int nb) { return nb & 0xffff; }
__host__ __device__ __forceinline__ int job_site_b(int nb) { return (nb >> 16) & 255; }
static_assert(sizeof(JobT<2>) == 32 && sizeof(JobT<4>) == 48, "job records of 32 / 48 bytes");

// Zero-magnetisation mask (forced outcomes have log p = 0 / -inf).
__device__ __forceinline__ float lp_masked(int s, float d, int n_up, int n_done, int N, bool sz0) {
  if (sz0) {
    const int half = N >> 1;
    if (n_up >= half) return s == 1 ? 0.0f : -INFINITY;
    if (n_done - n_up >= half) return s == 0 ? 0.0f : -INFINITY;
  }
  return log_prob(s, d);
}

}  // namespace tc2dh
}  // namespace nqs

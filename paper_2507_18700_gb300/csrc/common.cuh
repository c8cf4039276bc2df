// Shared device helpers of libnqs: Philox4x32-10, the two-outcome softmax in
// log form, the workspace header and launch-side error handling.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nqs.h"

namespace nqs {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): per round
// (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
// c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), key bumped by (W0, W1).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = mulhi32(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = mulhi32(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Top 24 bits of a word as a uniform in [0, 1): exact in float32.
__device__ __forceinline__ float word_to_uniform(uint32_t x) {
  return (float)(x >> 8) * 5.9604644775390625e-08f;
}

// Sampling uniform of (seed, step, sample b, sampling position n).
__device__ __forceinline__ float sampling_uniform(uint64_t seed, uint64_t step, uint32_t b,
                                                  uint32_t n) {
  const uint4 x = philox4x32_10(make_uint4(n, b, (uint32_t)step, (uint32_t)(step >> 32)),
                                (uint32_t)seed, (uint32_t)(seed >> 32));
  return word_to_uniform(x.x);
}

// ---------------------------------------------------------------------------
// Two-outcome softmax (Eq. 3) in terms of the logit difference d = z0 - z1:
// log p(0) = -softplus(-d), log p(1) = -softplus(d).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float softplusf(float x) {
  return fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x)));
}
__device__ __forceinline__ float log_prob(int s, float d) {
  return -softplusf(s == 0 ? -d : d);
}
__device__ __forceinline__ float sigmoid_acc(float x) { return 1.0f / (1.0f + expf(-x)); }

// ---------------------------------------------------------------------------
// Workspace header: first 256 bytes of every workspace.
// ---------------------------------------------------------------------------
struct WsHeader {
  int32_t status;                  // nqs_status recorded by kernels (0 = OK)
  int32_t pad0;
  unsigned long long job_counter;  // persistent-kernel work queue
  unsigned long long pad[30];
};
static_assert(sizeof(WsHeader) == 256, "header must be 256 bytes");

__device__ __forceinline__ void flag_status(WsHeader* hdr, int code) {
  if (hdr) atomicCAS(&hdr->status, 0, code);
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace nqs

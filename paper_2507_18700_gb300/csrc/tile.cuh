// Register-tiled FP32 building blocks shared by the 1D and 2D recurrent kernels.
//
// Thread geometry of a "row tile": a CTA of NT threads owns R rows (samples or
// connected-configuration chains).  Lanes are grouped TU at a time; the TU
// lanes of a group share RPT rows and split the D hidden units, UPT = D/TU
// units each.  All rows of a tile advance one cell step per iteration, so one
// weight fetch from shared memory feeds RPT rows.
#pragma once

#include "common.cuh"

namespace nqs {

template <int D>
struct Geo {
  static constexpr int TU = D < 16 ? D : 16;   // lanes per row group
  static constexpr int UPT = D / TU;           // hidden units per lane
  static constexpr int RGW = 32 / TU;          // row groups per warp
  static constexpr int DP = D + 4;             // padded row stride of h tiles (floats)
};

// Load / store UPT consecutive floats (16-byte aligned when UPT % 4 == 0).
// The pointer is deliberately not __restrict__: these helpers also read
// buffers that the same kernel rewrites (column buffers, carries), which
// must not go through the non-coherent read-only cache path.
template <int UPT>
__device__ __forceinline__ void ld_units(const float* p, float (&v)[UPT]) {
  if constexpr (UPT % 4 == 0) {
#pragma unroll
    for (int q = 0; q < UPT / 4; ++q) {
      const float4 t = reinterpret_cast<const float4*>(p)[q];
      v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
  } else if constexpr (UPT == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int q = 0; q < UPT; ++q) v[q] = p[q];
  }
}

template <int UPT>
__device__ __forceinline__ void st_units(float* p, const float (&v)[UPT]) {
  if constexpr (UPT % 4 == 0) {
#pragma unroll
    for (int q = 0; q < UPT / 4; ++q)
      reinterpret_cast<float4*>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else if constexpr (UPT == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int q = 0; q < UPT; ++q) p[q] = v[q];
  }
}

// acc[i][g][j] += sum_{k<K} A[(r0+i)*lda + k] * Wt[k*ldw + g*gstride + u0 + j]
// A rows in shared memory (16-byte aligned rows, K % 4 == 0); Wt k-major.
template <int K, int RPT, int NG, int UPT>
__device__ __forceinline__ void tile_gemm(const float* __restrict__ A, int lda, int r0,
                                          const float* __restrict__ Wt, int ldw, int gstride,
                                          int u0, float (&acc)[RPT][NG][UPT]) {
#pragma unroll 2
  for (int k = 0; k < K; k += 4) {
    float4 hv[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) hv[i] = *reinterpret_cast<const float4*>(A + (r0 + i) * lda + k);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const float* wrow = Wt + (k + kk) * ldw + u0;
      float w[NG][UPT];
#pragma unroll
      for (int g = 0; g < NG; ++g) ld_units<UPT>(wrow + g * gstride, w[g]);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const float a = kk == 0 ? hv[i].x : kk == 1 ? hv[i].y : kk == 2 ? hv[i].z : hv[i].w;
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int j = 0; j < UPT; ++j) acc[i][g][j] = fmaf(a, w[g][j], acc[i][g][j]);
      }
    }
  }
}

// Sum over the TU lanes of a row group (lanes are contiguous, TU a power of 2).
template <int TU>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int off = TU / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Copy n floats (n % 4 == 0, both 16-byte aligned) global -> shared by the whole CTA.
__device__ __forceinline__ void cta_copy4(float* __restrict__ dst, const float* __restrict__ src, int n) {
  const float4* s = reinterpret_cast<const float4*>(src);
  float4* d = reinterpret_cast<float4*>(dst);
  for (int t = threadIdx.x; t < n / 4; t += blockDim.x) d[t] = s[t];
}

}  // namespace nqs

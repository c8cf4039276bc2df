// Hidden-dimension growth (Sec. II B, Fig. 2(b)): embed a trained small RNN
// into a larger one.  Old entries keep their indices; every hidden-input
// column group is [old units | new units] followed by the one-hot columns;
// entries without a counterpart are eps * z, z standard normal from Philox
// keyed by (seed, tensor index, row, column) through Box-Muller.
#include "kernels.h"

namespace nqs {

namespace {
constexpr uint32_t kGrowTag = 0x6E717367u;

struct TensorShape { int rows, cols; };

// Shape of tensor t of the flat layout for hidden size D and GLU width M.
__device__ TensorShape tensor_shape(int cell, int t, int D, int M) {
  if (cell == NQS_GRU1D) {
    switch (t) {
      case 0: case 1: return {D, D + 2};
      case 2: return {D, D};
      case 3: return {D, 2};
      case 4: case 5: case 6: case 7: return {D, 1};
      case 8: case 10: return {2, D};     // U; cRNN U_phi
      default: return {2, 1};            // c; cRNN c_phi
    }
  }
  switch (t) {
    case 0: case 1: return {D, 2 * D + 4};
    case 2: return {D, 2 * D};
    case 3: case 4: return {D, 1};
    case 5: return {M, D};
    case 6: return {M, 1};
    case 7: return {M, D};
    case 8: return {M, 1};
    case 9: return {2, M};
    default: return {2, 1};
  }
}

// Old (row, col) of big entry (r, c) of tensor t, or row = -1 if it is new.
__device__ void old_index(int cell, int t, int r, int c, int d, int m, int D, int M, int& orow, int& ocol) {
  orow = -1;
  ocol = -1;
  auto hcol = [&](int cc) -> int { return cc < d ? cc : -1; };
  if (cell == NQS_GRU1D) {
    switch (t) {
      case 0: case 1:
        if (r < d) ocol = c < D ? hcol(c) : d + (c - D);
        break;
      case 2: if (r < d) ocol = hcol(c); break;
      case 3: case 4: case 5: case 6: case 7: if (r < d) ocol = c; break;
      case 8: case 10: ocol = hcol(c); break;
      default: ocol = c; break;
    }
  } else {
    switch (t) {
      case 0: case 1:
        if (r < d) {
          if (c < D) ocol = hcol(c);
          else if (c < 2 * D) ocol = (c - D) < d ? d + (c - D) : -1;
          else ocol = 2 * d + (c - 2 * D);
        }
        break;
      case 2:
        if (r < d) ocol = c < D ? hcol(c) : ((c - D) < d ? d + (c - D) : -1);
        break;
      case 3: case 4: if (r < d) ocol = c; break;
      case 5: case 7: if (r < m) ocol = hcol(c); break;
      case 6: case 8: if (r < m) ocol = c; break;
      case 9: ocol = c < m ? c : -1; break;
      default: ocol = c; break;
    }
  }
  if (ocol >= 0) orow = r;
}

__global__ void grow_kernel(int cell, int phase, int d, int m, int D, int M, const float* __restrict__ ps,
                            float* __restrict__ pb, uint32_t k0, uint32_t k1, float eps) {
  const int ntens = cell == NQS_GRU1D ? (phase ? 12 : 10) : 11;   // cRNN: U_phi, c_phi after c
  // offsets of every tensor in both layouts
  int offb = 0, offs = 0;
  for (int t = 0; t < ntens; ++t) {
    const TensorShape sb = tensor_shape(cell, t, D, M);
    const TensorShape ss = tensor_shape(cell, t, d, m);
    const int nb = sb.rows * sb.cols;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb; e += gridDim.x * blockDim.x) {
      const int r = e / sb.cols, c = e % sb.cols;
      int orow, ocol;
      old_index(cell, t, r, c, d, m, D, M, orow, ocol);
      float v;
      if (orow >= 0) {
        v = ps[offs + orow * ss.cols + ocol];
      } else {
        const uint4 x = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)r, (uint32_t)t, kGrowTag), k0, k1);
        const float u1 = word_to_uniform(x.x) + 5.9604644775390625e-08f;  // (0, 1]
        const float u2 = word_to_uniform(x.y);                            // [0, 1)
        v = eps * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
      }
      pb[offb + e] = v;
    }
    offb += nb;
    offs += ss.rows * ss.cols;
  }
}
}  // namespace

cudaError_t grow_params(int cell, int phase, int d, int m, int D, int M, const float* p_small, float* p_big,
                        uint64_t seed, float eps, cudaStream_t st) {
  grow_kernel<<<256, 256, 0, st>>>(cell, phase, d, m, D, M, p_small, p_big, (uint32_t)seed,
                                   (uint32_t)(seed >> 32), eps);
  return cudaGetLastError();
}

}  // namespace nqs

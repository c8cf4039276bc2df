// FP32 kernels of the 2D GRU wave function with its GLU head (App. A) on the
// CUDA cores: zig-zag sampling / teacher forcing, and the prefix-cached
// Heisenberg local energy (Eq. heisenberg, Marshall-rotated, Sec. III B).
//
// Zig-zag order (Sec. II, Fig. 1(b)): position t = j*Lx + r is row j, column
// i = r (j even) or Lx-1-r (j odd).  Cell (i, j) reads its horizontal
// neighbour i - (-1)^j of the same row (the previous position, absent at the
// first cell of a row) and its vertical neighbour (i, j-1) (absent in row 0).
// Every row slot keeps a column buffer colbuf[slot][i][:] holding the latest
// hidden state of column i, so both neighbours are colbuf entries.
#include "kernels.h"
#include "tile.cuh"

namespace nqs {

struct Off2 {
  int W, Wg, Umix, b, bg, W1, b1, W2, b2, Uo, c, P;
};
__host__ __device__ inline Off2 off2(int D, int M) {
  Off2 o;
  o.W = 0;
  o.Wg = o.W + D * (2 * D + 4);
  o.Umix = o.Wg + D * (2 * D + 4);
  o.b = o.Umix + D * 2 * D;
  o.bg = o.b + D;
  o.W1 = o.bg + D;
  o.b1 = o.W1 + M * D;
  o.W2 = o.b1 + M;
  o.b2 = o.W2 + M * D;
  o.Uo = o.b2 + M;
  o.c = o.Uo + 2 * M;
  o.P = o.c + 2;
  return o;
}

// Packed image (floats), M = D:
//   small: Ws[4][2D] (one-hot column q of W (first D) and W_g (next D)),
//          Bs[2][D] (b, b_g), B2[2][D] (b_1, b_2), Uo[2][D], c0 c1 0 0   (14D + 4)
//   Wt1[2D][3D]:  Wt1[k][g*D+u] = W / W_g / U_mix [u][k]   (k < 2D)
//   Wt2[D][2D]:   Wt2[k][g*D+v] = W_1 / W_2 [v][k]
//   Wn1[3D][2D]:  the same numbers as Wt1, row-major by (gate, unit)
//   Wn2[2D][D]:   the same numbers as Wt2, row-major by (gate, unit)
__host__ __device__ inline int img2_small(int D) { return 14 * D + 4; }
__host__ __device__ inline int img2_fwd(int D) { return img2_small(D) + 6 * D * D + 2 * D * D; }
__host__ __device__ inline int img2_floats(int D) { return img2_fwd(D) + 8 * D * D; }

__global__ void pack2d_kernel(const float* __restrict__ p, float* __restrict__ img, int D) {
  const Off2 o = off2(D, D);
  const int small = img2_small(D), total = img2_floats(D);
  const int W2 = 2 * D + 4;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    float v = 0.0f;
    if (t < 8 * D) {
      const int q = t / (2 * D), g = (t % (2 * D)) / D, u = t % D;
      v = p[(g == 0 ? o.W : o.Wg) + u * W2 + 2 * D + q];
    } else if (t < 10 * D) {
      v = p[o.b + (t - 8 * D)];                       // b, b_g contiguous
    } else if (t < 12 * D) {
      const int q = t - 10 * D;
      v = q < D ? p[o.b1 + q] : p[o.b2 + q - D];
    } else if (t < 14 * D) {
      v = p[o.Uo + (t - 12 * D)];
    } else if (t < small) {
      const int q = t - 14 * D;
      v = q < 2 ? p[o.c + q] : 0.0f;
    } else {
      int q = t - small;
      if (q < 6 * D * D) {                            // Wt1
        const int k = q / (3 * D), g = (q % (3 * D)) / D, u = q % D;
        v = g == 0 ? p[o.W + u * W2 + k] : g == 1 ? p[o.Wg + u * W2 + k] : p[o.Umix + u * 2 * D + k];
      } else if ((q -= 6 * D * D) < 2 * D * D) {      // Wt2
        const int k = q / (2 * D), g = (q % (2 * D)) / D, u = q % D;
        v = p[(g == 0 ? o.W1 : o.W2) + u * D + k];
      } else if ((q -= 2 * D * D) < 6 * D * D) {      // Wn1
        const int gu = q / (2 * D), k = q % (2 * D), g = gu / D, u = gu % D;
        v = g == 0 ? p[o.W + u * W2 + k] : g == 1 ? p[o.Wg + u * W2 + k] : p[o.Umix + u * 2 * D + k];
      } else {                                        // Wn2
        q -= 6 * D * D;
        const int gu = q / D, k = q % D, g = gu / D, u = gu % D;
        v = p[(g == 0 ? o.W1 : o.W2) + u * D + k];
      }
    }
    img[t] = v;
  }
}

// Zig-zag geometry.
struct Pos {
  int i, j, r;
};
__device__ __forceinline__ Pos pos_of(int t, int Lx) {
  Pos p;
  p.j = t / Lx;
  p.r = t - p.j * Lx;
  p.i = (p.j & 1) ? Lx - 1 - p.r : p.r;
  return p;
}
__device__ __forceinline__ int hor_col(const Pos& p) { return (p.j & 1) ? p.i + 1 : p.i - 1; }
__device__ __forceinline__ int snake_pos(int i, int j, int Lx) { return j * Lx + ((j & 1) ? Lx - 1 - i : i); }

// Masked log-probabilities of the two outcomes (zero-magnetisation mask).
__device__ __forceinline__ float masked_lp(int s, float d, int n_up, int n_done, int N, bool sz0) {
  if (sz0) {
    const int half = N >> 1;
    if (n_up >= half) return s == 1 ? 0.0f : -INFINITY;
    if (n_done - n_up >= half) return s == 0 ? 0.0f : -INFINITY;
  }
  return log_prob(s, d);
}

// ----------------------------------------------------------------------------
// Bond table: nearest-neighbour bonds of the open Lx x Ly lattice with
// (lattice a, lattice b, zig-zag position of a, of b), pa < pb, sorted by pa
// (longest chains first).  One block.
// ----------------------------------------------------------------------------
template <bool SH>
__global__ void bonds2d_kernel(int Lx, int Ly, int4* __restrict__ out) {
  // bond k: sites (a, b), zig-zag positions (pa, pb) with pa < pb; ranked by
  // (pa, k) against every bond's pa, kept in shared memory (SH) or recomputed
  // (lattices whose keys do not fit)
  extern __shared__ int key[];
  const int nh = (Lx - 1) * Ly, nb = nh + Lx * (Ly - 1);
  auto bond = [&](int k, int& a, int& b, int& pa, int& pb) {
    if (k < nh) {
      const int j = k / (Lx - 1), i = k % (Lx - 1);
      a = j * Lx + i;
      b = a + 1;
    } else {
      const int q = k - nh, j = q / Lx, i = q % Lx;
      a = j * Lx + i;
      b = a + Lx;
    }
    pa = snake_pos(a % Lx, a / Lx, Lx);
    pb = snake_pos(b % Lx, b / Lx, Lx);
    if (pa > pb) {
      int t = pa; pa = pb; pb = t;
      t = a; a = b; b = t;
    }
  };
  if constexpr (SH) {
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
      int a, b, pa, pb;
      bond(k, a, b, pa, pb);
      key[k] = pa;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    int a, b, pa, pb;
    bond(k, a, b, pa, pb);
    int rank = 0;
    for (int q = 0; q < nb; ++q) {
      int qa = 0, qb = 0, qpa = 0, qpb = 0;
      if constexpr (SH) {
        qpa = key[q];
      } else {
        bond(q, qa, qb, qpa, qpb);
      }
      rank += (qpa < pa) || (qpa == pa && q < k);
    }
    out[rank] = make_int4(a, b, pa, pb);
  }
}

// ----------------------------------------------------------------------------
// Row-slot recurrent engine.  MODE 0: sampling, 1: teacher forcing (one job =
// one sample, positions 0..N-1), 2: Heisenberg chains (one job = one
// antiparallel bond of one sample, positions pa+1..N-1 on the exchanged
// configuration, restarted from the cached states).
// ----------------------------------------------------------------------------
template <int D, int RPT, int NT, int MODE, bool WSMEM>
__global__ void __launch_bounds__(NT) gru2d_engine_kernel(const float* __restrict__ img, Eng2Args a) {
  using G = Geo<D>;
  constexpr int TU = G::TU, UPT = G::UPT;
  constexpr int NRG = NT / TU, R = NRG * RPT;
  constexpr int AP = 2 * D + 4, HP = D + 4;
  extern __shared__ __align__(16) float sm[];
  float* small = sm;
  const float* Wt1 = WSMEM ? sm + img2_small(D) : img + img2_small(D);
  const float* Wt2 = Wt1 + 6 * D * D;
  float* Atile = sm + img2_small(D) + (WSMEM ? 8 * D * D : 0);
  float* Htile = Atile + R * AP;
  cta_copy4(sm, img, img2_small(D) + (WSMEM ? 8 * D * D : 0));
  __syncthreads();   // the copied constants are read below by every warp

  const int lane = threadIdx.x & 31, ug = lane % TU;
  const unsigned gmask = (TU == 32 ? 0xffffffffu : ((1u << TU) - 1u) << (lane - ug));
  const int rg = threadIdx.x / TU, r0 = rg * RPT, u0 = ug * UPT;
  const int Lx = a.Lx, N = a.N;
  const int64_t B = a.B;
  const float* Ws = small;
  const float* Bs = small + 8 * D;
  const float* B2 = small + 10 * D;
  const float* Uo = small + 12 * D;
  const float c0 = small[14 * D], c1 = small[14 * D + 1];

  int64_t jb[RPT];
  int t[RPT], n_up[RPT], bsa[RPT], bsb[RPT], bk[RPT];
  float acc_lp[RPT];
  bool act[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    jb[i] = 0; t[i] = 0; n_up[i] = 0; bsa[i] = -1; bsb[i] = -1; bk[i] = 0; acc_lp[i] = 0.0f; act[i] = false;
  }
  const uint64_t total = MODE == 2 ? (uint64_t)B * (uint64_t)a.nbonds : 0;

  auto slot_col = [&](int i, int col) -> float* {
    const int64_t slot = (int64_t)blockIdx.x * R + r0 + i;
    return a.colbuf + (slot * Lx + col) * D;
  };
  // spin of lattice site k of the row's (possibly exchanged) configuration
  auto spin = [&](int i, int k) -> int {
    if constexpr (MODE == 0) {
      return a.sigma_out[jb[i] * N + k];
    } else if constexpr (MODE == 1) {
      return a.sigma_in[jb[i] * N + k] ? 1 : 0;
    } else {
      const int kk = k == bsa[i] ? bsb[i] : k == bsb[i] ? bsa[i] : k;
      return a.sigma_in[jb[i] * N + kk] ? 1 : 0;
    }
  };

  // ---- job setup (collective within the row group) ----
  auto start_chain = [&](int i) {
    for (;;) {
      unsigned long long j = 0;
      if (ug == 0) j = atomicAdd(a.counter, 1ull);
      j = __shfl_sync(gmask, j, lane - ug);
      if (j >= total) { act[i] = false; return; }  // queue drained
      const int rank = (int)(j / (unsigned long long)B);
      const int64_t b = (int64_t)(j % (unsigned long long)B);
      const int4 bond = a.bonds[rank];
      const int sa = a.sigma_in[b * N + bond.x] ? 1 : 0;
      const int sb = a.sigma_in[b * N + bond.y] ? 1 : 0;
      if (sa == sb) continue;                     // parallel bond: diagonal only
      jb[i] = b; bsa[i] = bond.x; bsb[i] = bond.y; bk[i] = rank;
      const int pa = bond.z;
      t[i] = pa + 1;
      act[i] = true;
      // bond.x sits at position pa and takes the partner's spin; the prefix before pa is unchanged
      const int s_new = sb;
      acc_lp[i] = 0.5f * (a.lp_tab[(b * N + pa) * 2 + s_new] - a.lp_tab[(b * N + pa) * 2 + sa]);
      n_up[i] = a.nup_tab[b * N + pa] + (s_new == 0 ? 1 : 0);
      // column buffer: latest original state of every column at positions <= pa
      const Pos pp = pos_of(pa, Lx);
      for (int col = 0; col < Lx; ++col) {
        const int jr = snake_pos(col, pp.j, Lx) <= pa ? pp.j : pp.j - 1;
        float hv[UPT];
        if (jr >= 0) {
          ld_units<UPT>(a.hcache + (b * N + jr * Lx + col) * D + u0, hv);
        } else {
#pragma unroll
          for (int q = 0; q < UPT; ++q) hv[q] = 0.0f;
        }
        st_units<UPT>(slot_col(i, col) + u0, hv);
      }
      return;
    }
  };

  // initial jobs
  int64_t next_sample = 0;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    if constexpr (MODE == 2) {
      act[i] = false;
      bsa[i] = bsb[i] = -1;
      start_chain(i);
    } else {
      jb[i] = (int64_t)blockIdx.x * R + r0 + i;
      act[i] = jb[i] < B;
      t[i] = 0; n_up[i] = 0; acc_lp[i] = 0.0f; bsa[i] = bsb[i] = -1; bk[i] = 0;
    }
  }
  (void)next_sample;

  for (;;) {
    bool any = false;
#pragma unroll
    for (int i = 0; i < RPT; ++i) any |= act[i];
    if (!__syncthreads_or(any)) break;
    // ---- stage A = [h_hor | h_ver] of every row ----
    int s_h[RPT], s_v[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      float hv[UPT], vv[UPT];
#pragma unroll
      for (int q = 0; q < UPT; ++q) { hv[q] = 0.0f; vv[q] = 0.0f; }
      s_h[i] = -1; s_v[i] = -1;
      if (act[i]) {
        const Pos p = pos_of(t[i], Lx);
        if (p.r > 0) {
          const int ih = hor_col(p);
          ld_units<UPT>(slot_col(i, ih) + u0, hv);
          s_h[i] = spin(i, p.j * Lx + ih);
        }
        if (p.j > 0) {
          ld_units<UPT>(slot_col(i, p.i) + u0, vv);
          s_v[i] = spin(i, (p.j - 1) * Lx + p.i);
        }
      }
      st_units<UPT>(Atile + row * AP + u0, hv);
      st_units<UPT>(Atile + row * AP + D + u0, vv);
    }
    __syncthreads();
    // ---- GEMM1 [h_hor | h_ver] x [W | W_g | U_mix] and the cell ----
    {
      float acc[RPT][3][UPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int g = 0; g < 3; ++g)
#pragma unroll
          for (int j = 0; j < UPT; ++j) acc[i][g][j] = 0.0f;
      tile_gemm<2 * D, RPT, 3, UPT>(Atile, AP, r0, Wt1, 3 * D, D, u0, acc);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int row = r0 + i;
        float hn[UPT];
#pragma unroll
        for (int j = 0; j < UPT; ++j) {
          const int u = u0 + j;
          float av = acc[i][0][j] + Bs[u];
          float gv = acc[i][1][j] + Bs[D + u];
          if (s_h[i] >= 0) { av += Ws[s_h[i] * 2 * D + u]; gv += Ws[s_h[i] * 2 * D + D + u]; }
          if (s_v[i] >= 0) { av += Ws[(2 + s_v[i]) * 2 * D + u]; gv += Ws[(2 + s_v[i]) * 2 * D + D + u]; }
          const float cc = tanhf(av);
          const float uu = sigmoid_acc(gv);
          const float mix = acc[i][2][j];
          hn[j] = fmaf(uu, cc - mix, mix);
        }
        st_units<UPT>(Htile + row * HP + u0, hn);
        if (act[i]) {
          const Pos p = pos_of(t[i], Lx);
          st_units<UPT>(slot_col(i, p.i) + u0, hn);
          if (MODE != 2 && a.hcache) st_units<UPT>(a.hcache + (jb[i] * N + p.j * Lx + p.i) * D + u0, hn);
        }
      }
    }
    __syncthreads();
    // ---- GEMM2 h x [W_1 | W_2], GLU, readout, and the per-row logic ----
    {
      float acc[RPT][2][UPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
          for (int j = 0; j < UPT; ++j) acc[i][g][j] = 0.0f;
      tile_gemm<D, RPT, 2, UPT>(Htile, HP, r0, Wt2, 2 * D, D, u0, acc);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
        for (int j = 0; j < UPT; ++j) {
          const int v = u0 + j;
          const float gl = (acc[i][0][j] + B2[v]) * sigmoid_acc(acc[i][1][j] + B2[D + v]);
          z0 = fmaf(Uo[v], gl, z0);
          z1 = fmaf(Uo[D + v], gl, z1);
        }
        z0 = group_sum<TU>(z0);
        z1 = group_sum<TU>(z1);
        bool fin = false;
        if (act[i]) {
          const float d = (z0 + c0) - (z1 + c1);
          const Pos p = pos_of(t[i], Lx);
          const int k = p.j * Lx + p.i;
          int s;
          if constexpr (MODE == 0) {
            const bool forced_dn = a.sz0 && n_up[i] >= (N >> 1);
            const bool forced_up = a.sz0 && (t[i] - n_up[i]) >= (N >> 1);
            const float u = a.uniforms ? a.uniforms[jb[i] * N + t[i]]
                                       : sampling_uniform(a.seed, a.step_dev ? *a.step_dev : a.step, (uint32_t)(a.b0 + jb[i]), (uint32_t)t[i]);
            s = forced_dn ? 1 : forced_up ? 0 : (u < sigmoid_acc(d) ? 0 : 1);
            if (ug == 0) a.sigma_out[jb[i] * N + k] = (uint8_t)s;
          } else {
            s = spin(i, k);
          }
          const float lp = masked_lp(s, d, n_up[i], t[i], N, a.sz0);
          if constexpr (MODE == 2) {
            acc_lp[i] += 0.5f * (lp - a.lp_tab[(jb[i] * N + t[i]) * 2 + (a.sigma_in[jb[i] * N + k] ? 1 : 0)]);
          } else {
            acc_lp[i] += lp;
          }
          n_up[i] += (s == 0);
          if (++t[i] == N) {
            fin = true;
            if (ug == 0) {
              if constexpr (MODE == 2) {
                a.delta[jb[i] * a.nbonds + bk[i]] = acc_lp[i];
              } else {
                const float lpsi = 0.5f * acc_lp[i];
                a.logpsi[jb[i]] = lpsi;
                if (!isfinite(lpsi)) flag_status(a.hdr, NQS_ENONFINITE);
              }
            }
          }
        }
        if constexpr (MODE == 2) {
          if (fin) start_chain(i);
        } else {
          if (fin) act[i] = false;
        }
      }
    }
  }
}

// Per-sample scan of the cached path: masked log-probabilities of both
// outcomes at every position and the count of up spins before it.  One warp
// per sample; the GLU and readout of each cached state are warp-parallel.
__global__ void prep2d_kernel(const float* __restrict__ img, const float* __restrict__ hcache,
                              const uint8_t* __restrict__ sigma, float* __restrict__ lp_tab,
                              int* __restrict__ nup_tab, int64_t B, int Lx, int N, int D, int sz0) {
  const float* Wt2 = img + img2_small(D) + 6 * D * D;
  const float* B2 = img + 10 * D;
  const float* Uo = img + 12 * D;
  const float c0 = img[14 * D], c1 = img[14 * D + 1];
  const int lane = threadIdx.x & 31;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < B;
       b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int n_up = 0;
    for (int t = 0; t < N; ++t) {
      const Pos p = pos_of(t, Lx);
      const int k = p.j * Lx + p.i;
      const float* h = hcache + (b * N + k) * D;
      float z0 = 0.0f, z1 = 0.0f;
      for (int v = lane; v < D; v += 32) {
        float y1 = B2[v], y2 = B2[D + v];
        for (int q = 0; q < D; ++q) {
          const float hq = h[q];
          y1 = fmaf(Wt2[q * 2 * D + v], hq, y1);
          y2 = fmaf(Wt2[q * 2 * D + D + v], hq, y2);
        }
        const float gl = y1 * sigmoid_acc(y2);
        z0 = fmaf(Uo[v], gl, z0);
        z1 = fmaf(Uo[D + v], gl, z1);
      }
      z0 = group_sum<32>(z0);
      z1 = group_sum<32>(z1);
      const float d = (z0 + c0) - (z1 + c1);
      if (lane == 0) {
        lp_tab[(b * N + t) * 2 + 0] = masked_lp(0, d, n_up, t, N, sz0);
        lp_tab[(b * N + t) * 2 + 1] = masked_lp(1, d, n_up, t, N, sz0);
        nup_tab[b * N + t] = n_up;
      }
      n_up += sigma[b * N + k] ? 0 : 1;
    }
  }
}

// E_loc = sum over bonds: +J/4 (parallel) or -J/4 + x exp(Delta) (antiparallel).
__global__ void heis_eloc_kernel(const uint8_t* __restrict__ sigma, const int4* __restrict__ bonds,
                                 const float* __restrict__ delta, float* __restrict__ eloc, int64_t B,
                                 int N, int nb, float J, float x, WsHeader* hdr) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < B;
       b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float e = 0.0f;
    for (int k = lane; k < nb; k += 32) {
      const int4 bd = bonds[k];
      const bool par = (sigma[b * N + bd.x] != 0) == (sigma[b * N + bd.y] != 0);
      e += par ? 0.25f * J : -0.25f * J + x * expf(delta[b * nb + k]);
    }
    e = group_sum<32>(e);
    if (lane == 0) {
      eloc[b] = e;
      if (!isfinite(e)) flag_status(hdr, NQS_ENONFINITE);
    }
  }
}

// ----------------------------------------------------------------------------
// Reverse sweep over the zig-zag order: d/dtheta sum_b w_b log psi_b.  One row
// per sample; positions t = N-1 .. 0.  Cached states give each cell's inputs;
// the cell and the GLU are recomputed.  dh of a cell collects the GLU/readout
// term, the horizontal successor's term (carried in registers) and the
// vertical successor's term (per-column carry buffer ccarry[b][i]).  Weight
// gradients of the large matrices are accumulated into this CTA's partial
// gradient in global memory; the small ones in shared memory.
// ----------------------------------------------------------------------------
constexpr int kSmall2 = 14;  // b b_g Wsh0 Wsh1 Wsv0 Wsv1 Wgsh0 Wgsh1 Wgsv0 Wgsv1 b1 b2 Uo0 Uo1

// part[base + u*ld + k] += sum_r G[r*gs + goff + u] * A[r*as + k], u < D, k < K.
// Lanes split the units (UPT each) and the k range; each lane sweeps its k
// columns in chunks of at most 8 so the accumulators stay in registers.
template <int D, int K, int NT, int R>
__device__ __forceinline__ void accum_outer(float* part, int base, int ld, const float* Gs, int gs, int goff,
                                            const float* As, int as) {
  constexpr int TU = Geo<D>::TU, UPT = Geo<D>::UPT;
  constexpr int KG = NT / TU, KPT = K / KG;
  static_assert(KPT * KG == K, "bad outer tiling");
  constexpr int KCMAX = UPT >= 16 ? 4 : 8;
  constexpr int KC = KPT < KCMAX ? KPT : KCMAX;
  const int ug = threadIdx.x % TU, kg = threadIdx.x / TU;
  const int u0 = ug * UPT;
#pragma unroll 1
  for (int c = 0; c < KPT / KC; ++c) {
    const int k0 = kg * KPT + c * KC;
    float acc[UPT][KC];
#pragma unroll
    for (int j = 0; j < UPT; ++j)
#pragma unroll
      for (int q = 0; q < KC; ++q) acc[j][q] = 0.0f;
    for (int r = 0; r < R; ++r) {
      float gv[UPT], av[KC];
      ld_units<UPT>(Gs + r * gs + goff + u0, gv);
      ld_units<KC>(As + r * as + k0, av);
#pragma unroll
      for (int j = 0; j < UPT; ++j)
#pragma unroll
        for (int q = 0; q < KC; ++q) acc[j][q] = fmaf(gv[j], av[q], acc[j][q]);
    }
#pragma unroll
    for (int j = 0; j < UPT; ++j)
#pragma unroll
      for (int q = 0; q < KC; ++q) part[base + (u0 + j) * ld + k0 + q] += acc[j][q];
  }
}

template <int D, int RPT, int NT, bool GSACC>
__global__ void __launch_bounds__(NT) gru2d_bptt_kernel(const float* __restrict__ img, Bptt2Args a) {
  using G = Geo<D>;
  constexpr int TU = G::TU, UPT = G::UPT;
  constexpr int NRG = NT / TU, R = NRG * RPT;
  constexpr int AP = 2 * D + 4, HP = D + 4, YP = 2 * D + 4, GP = 3 * D + 4;
  extern __shared__ __align__(16) float sm[];
  float* small = sm;
  float* Atile = sm + img2_small(D);        // [R][AP]  [h_hor | h_ver]
  float* Htile = Atile + R * AP;            // [R][HP]  h
  float* DY = Htile + R * HP;               // [R][YP]  [dy1 | dy2]
  float* GG = DY + R * YP;                  // [R][GP]  [da | dg | dmix]
  // per-row-group small-gradient accumulators [NRG][kSmall2][D]: shared
  // memory, or (large d_h) this CTA's slice of a global scratch area
  float* cacc = GG + R * GP;                // [NRG][2]
  float* sacc = GSACC ? a.sacc + (size_t)blockIdx.x * NRG * kSmall2 * D : cacc + 2 * NRG;
  const float* Wt1 = img + img2_small(D);
  const float* Wt2 = Wt1 + 6 * D * D;
  const float* Wn1 = Wt2 + 2 * D * D;
  const float* Wn2 = Wn1 + 6 * D * D;
  cta_copy4(sm, img, img2_small(D));
  for (int q = threadIdx.x; q < 2 * NRG; q += NT) cacc[q] = 0.0f;
  if (!GSACC)
    for (int q = threadIdx.x; q < NRG * kSmall2 * D; q += NT) sacc[q] = 0.0f;
  __syncthreads();   // the copied constants are read below by every warp

  const int lane = threadIdx.x & 31, ug = lane % TU;
  const int rg = threadIdx.x / TU, r0 = rg * RPT, u0 = ug * UPT;
  const int Lx = a.Lx, N = a.N;
  const float* Ws = small;
  const float* Bs = small + 8 * D;
  const float* B2 = small + 10 * D;
  const float* Uo = small + 12 * D;
  const float c0 = small[14 * D], c1 = small[14 * D + 1];
  const Off2 o = off2(D, D);
  float* part = a.partial + (size_t)blockIdx.x * a.P;

  int64_t bb[RPT];
  float coef[RPT];
  int n_up[RPT];       // up spins before the current position
  float carry_h[RPT][UPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    bb[i] = (int64_t)blockIdx.x * R + r0 + i;
    const bool valid = bb[i] < a.B;
    coef[i] = valid ? 0.5f * a.weights[bb[i]] : 0.0f;
    int cnt = 0;
    if (valid)
      for (int k = 0; k < N; ++k) cnt += a.sigma[bb[i] * N + k] ? 0 : 1;
    n_up[i] = cnt;
#pragma unroll
    for (int j = 0; j < UPT; ++j) carry_h[i][j] = 0.0f;
    if (valid)
      for (int col = 0; col < Lx; ++col) {
        float z[UPT];
#pragma unroll
        for (int q = 0; q < UPT; ++q) z[q] = 0.0f;
        st_units<UPT>(a.ccarry + (bb[i] * Lx + col) * D + u0, z);
      }
  }

  for (int t = N - 1; t >= 0; --t) {
    const Pos p = pos_of(t, Lx);
    const int k = p.j * Lx + p.i;
    const int ih = hor_col(p);
    // ---- (1) stage the cell inputs from the cache ----
    int s_h[RPT], s_v[RPT], s_k[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      const bool valid = bb[i] < a.B;
      float hv[UPT], vv[UPT];
#pragma unroll
      for (int q = 0; q < UPT; ++q) { hv[q] = 0.0f; vv[q] = 0.0f; }
      s_h[i] = -1; s_v[i] = -1; s_k[i] = 0;
      if (valid) {
        s_k[i] = a.sigma[bb[i] * N + k] ? 1 : 0;
        n_up[i] -= (s_k[i] == 0);
        if (p.r > 0) {
          ld_units<UPT>(a.hcache + (bb[i] * N + p.j * Lx + ih) * D + u0, hv);
          s_h[i] = a.sigma[bb[i] * N + p.j * Lx + ih] ? 1 : 0;
        }
        if (p.j > 0) {
          ld_units<UPT>(a.hcache + (bb[i] * N + (p.j - 1) * Lx + p.i) * D + u0, vv);
          s_v[i] = a.sigma[bb[i] * N + (p.j - 1) * Lx + p.i] ? 1 : 0;
        }
      }
      st_units<UPT>(Atile + row * AP + u0, hv);
      st_units<UPT>(Atile + row * AP + D + u0, vv);
    }
    __syncthreads();
    // ---- (2) recompute the cell ----
    float cc[RPT][UPT], uu[RPT][UPT], mx[RPT][UPT];
    {
      float acc[RPT][3][UPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int g = 0; g < 3; ++g)
#pragma unroll
          for (int j = 0; j < UPT; ++j) acc[i][g][j] = 0.0f;
      tile_gemm<2 * D, RPT, 3, UPT>(Atile, AP, r0, Wt1, 3 * D, D, u0, acc);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        float hn[UPT];
#pragma unroll
        for (int j = 0; j < UPT; ++j) {
          const int u = u0 + j;
          float av = acc[i][0][j] + Bs[u];
          float gv = acc[i][1][j] + Bs[D + u];
          if (s_h[i] >= 0) { av += Ws[s_h[i] * 2 * D + u]; gv += Ws[s_h[i] * 2 * D + D + u]; }
          if (s_v[i] >= 0) { av += Ws[(2 + s_v[i]) * 2 * D + u]; gv += Ws[(2 + s_v[i]) * 2 * D + D + u]; }
          cc[i][j] = tanhf(av);
          uu[i][j] = sigmoid_acc(gv);
          mx[i][j] = acc[i][2][j];
          hn[j] = fmaf(uu[i][j], cc[i][j] - mx[i][j], mx[i][j]);
        }
        st_units<UPT>(Htile + (r0 + i) * HP + u0, hn);
      }
    }
    __syncthreads();
    // ---- (3) recompute the GLU and readout; back through them ----
    // small gradients go straight to this thread's own accumulator slots
    auto sacc_add = [&](int q, int u, float v) { sacc[(rg * kSmall2 + q) * D + u] += v; };
    float dcs = 0.0f;
    {
      float acc[RPT][2][UPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i)
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
          for (int j = 0; j < UPT; ++j) acc[i][g][j] = 0.0f;
      tile_gemm<D, RPT, 2, UPT>(Htile, HP, r0, Wt2, 2 * D, D, u0, acc);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        float y1[UPT], s2[UPT], gl[UPT];
        float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
        for (int j = 0; j < UPT; ++j) {
          const int v = u0 + j;
          y1[j] = acc[i][0][j] + B2[v];
          s2[j] = sigmoid_acc(acc[i][1][j] + B2[D + v]);
          gl[j] = y1[j] * s2[j];
          z0 = fmaf(Uo[v], gl[j], z0);
          z1 = fmaf(Uo[D + v], gl[j], z1);
        }
        z0 = group_sum<TU>(z0);
        z1 = group_sum<TU>(z1);
        const float d = (z0 + c0) - (z1 + c1);
        bool forced = false;
        if (a.sz0) {
          const int half = N >> 1;
          forced = n_up[i] >= half || (t - n_up[i]) >= half;
        }
        const float dz0 = forced ? 0.0f : coef[i] * ((s_k[i] == 0 ? 1.0f : 0.0f) - sigmoid_acc(d));
        dcs += dz0;
        float dy[2][UPT];
#pragma unroll
        for (int j = 0; j < UPT; ++j) {
          const int v = u0 + j;
          const float dgl = dz0 * (Uo[v] - Uo[D + v]);
          dy[0][j] = dgl * s2[j];
          dy[1][j] = dgl * y1[j] * s2[j] * (1.0f - s2[j]);
          sacc_add(10, v, dy[0][j]);
          sacc_add(11, v, dy[1][j]);
          sacc_add(12, v, dz0 * gl[j]);
          sacc_add(13, v, -dz0 * gl[j]);
        }
        st_units<UPT>(DY + (r0 + i) * YP + u0, dy[0]);
        st_units<UPT>(DY + (r0 + i) * YP + D + u0, dy[1]);
      }
    }
    __syncthreads();
    // ---- (4) dh and the cell's backward; dW_1, dW_2 ----
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      const bool valid = bb[i] < a.B;
      float dh[UPT];
#pragma unroll
      for (int j = 0; j < UPT; ++j) dh[j] = carry_h[i][j];
      if (valid) {
        float cv[UPT];
        ld_units<UPT>(a.ccarry + (bb[i] * Lx + p.i) * D + u0, cv);
#pragma unroll
        for (int j = 0; j < UPT; ++j) dh[j] += cv[j];
      }
#pragma unroll 2
      for (int gv = 0; gv < 2 * D; gv += 4) {
        const float4 y = *reinterpret_cast<const float4*>(DY + row * YP + gv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float w[UPT];
          ld_units<UPT>(Wn2 + (gv + q) * D + u0, w);
          const float yq = q == 0 ? y.x : q == 1 ? y.y : q == 2 ? y.z : y.w;
#pragma unroll
          for (int j = 0; j < UPT; ++j) dh[j] = fmaf(yq, w[j], dh[j]);
        }
      }
      float gg[3][UPT];
#pragma unroll
      for (int j = 0; j < UPT; ++j) {
        const float dc = dh[j] * uu[i][j];
        const float du = dh[j] * (cc[i][j] - mx[i][j]);
        gg[2][j] = dh[j] * (1.0f - uu[i][j]);                  // d mix
        gg[0][j] = dc * (1.0f - cc[i][j] * cc[i][j]);           // d a
        gg[1][j] = du * uu[i][j] * (1.0f - uu[i][j]);           // d g
        const int u = u0 + j;
        sacc_add(0, u, gg[0][j]);
        sacc_add(1, u, gg[1][j]);
        if (s_h[i] >= 0) { sacc_add(2 + s_h[i], u, gg[0][j]); sacc_add(6 + s_h[i], u, gg[1][j]); }
        if (s_v[i] >= 0) { sacc_add(4 + s_v[i], u, gg[0][j]); sacc_add(8 + s_v[i], u, gg[1][j]); }
      }
#pragma unroll
      for (int g = 0; g < 3; ++g) st_units<UPT>(GG + row * GP + g * D + u0, gg[g]);
    }
    if (ug == 0) { cacc[rg * 2] += dcs; cacc[rg * 2 + 1] -= dcs; }
    accum_outer<D, D, NT, R>(part, o.W1, D, DY, YP, 0, Htile, HP);
    accum_outer<D, D, NT, R>(part, o.W2, D, DY, YP, D, Htile, HP);
    __syncthreads();
    // ---- (5) dA = G Wn1 -> carries; dW, dW_g, dU_mix ----
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      float dhor[UPT], dver[UPT];
#pragma unroll
      for (int j = 0; j < UPT; ++j) { dhor[j] = 0.0f; dver[j] = 0.0f; }
#pragma unroll 2
      for (int gu = 0; gu < 3 * D; gu += 4) {
        const float4 gv = *reinterpret_cast<const float4*>(GG + row * GP + gu);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float w1[UPT], w2[UPT];
          ld_units<UPT>(Wn1 + (gu + q) * 2 * D + u0, w1);
          ld_units<UPT>(Wn1 + (gu + q) * 2 * D + D + u0, w2);
          const float gq = q == 0 ? gv.x : q == 1 ? gv.y : q == 2 ? gv.z : gv.w;
#pragma unroll
          for (int j = 0; j < UPT; ++j) {
            dhor[j] = fmaf(gq, w1[j], dhor[j]);
            dver[j] = fmaf(gq, w2[j], dver[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < UPT; ++j) carry_h[i][j] = p.r > 0 ? dhor[j] : 0.0f;
      if (bb[i] < a.B) {
        if (p.j == 0) {
#pragma unroll
          for (int j = 0; j < UPT; ++j) dver[j] = 0.0f;
        }
        st_units<UPT>(a.ccarry + (bb[i] * Lx + p.i) * D + u0, dver);
      }
    }
    accum_outer<D, 2 * D, NT, R>(part, o.W, 2 * D + 4, GG, GP, 0, Atile, AP);
    accum_outer<D, 2 * D, NT, R>(part, o.Wg, 2 * D + 4, GG, GP, D, Atile, AP);
    accum_outer<D, 2 * D, NT, R>(part, o.Umix, 2 * D, GG, GP, 2 * D, Atile, AP);
    __syncthreads();
  }

  // small gradients of this CTA
  for (int u = threadIdx.x; u < D; u += NT) {
    float v[kSmall2];
#pragma unroll
    for (int q = 0; q < kSmall2; ++q) {
      float s = 0.0f;
      for (int r = 0; r < NRG; ++r) s += sacc[(r * kSmall2 + q) * D + u];
      v[q] = s;
    }
    const int W2s = 2 * D + 4;
    part[o.b + u] += v[0];
    part[o.bg + u] += v[1];
    for (int q = 0; q < 4; ++q) {
      part[o.W + u * W2s + 2 * D + q] += v[2 + q];
      part[o.Wg + u * W2s + 2 * D + q] += v[6 + q];
    }
    part[o.b1 + u] += v[10];
    part[o.b2 + u] += v[11];
    part[o.Uo + u] += v[12];
    part[o.Uo + D + u] += v[13];
  }
  if (threadIdx.x < 2) {
    float s = 0.0f;
    for (int r = 0; r < NRG; ++r) s += cacc[r * 2 + threadIdx.x];
    part[o.c + threadIdx.x] += s;
  }
}

// ----------------------------------------------------------------------------
// Host launchers.
// ----------------------------------------------------------------------------
namespace {

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      sms = n;
    else
      sms = 152;   // no device visible: size for a GB300
  }
  return sms;
}

template <int D> struct Tune2 {
  static constexpr int F_RPT = 1, F_NT = D >= 16 ? 256 : 64;   // forward: R = 16 or 8
  static constexpr int C_RPT = 2, C_NT = D >= 16 ? 256 : 64;   // chains: R = 32 or 16
  static constexpr bool WSMEM = D <= 64;
};

// Rows per CTA and grid of the engine: one row per sample for sampling and
// teacher forcing; for chains a persistent grid of SMs x resident CTAs, the
// residency estimated from the shared-memory footprint (no device query).
template <int D, int MODE>
constexpr int engine_rows() {
  using T = Tune2<D>;
  return (((MODE == 2) ? T::C_NT : T::F_NT) / Geo<D>::TU) * ((MODE == 2) ? T::C_RPT : T::F_RPT);
}
template <int D, int MODE>
int64_t engine_grid(int64_t B) {
  using T = Tune2<D>;
  constexpr int R = engine_rows<D, MODE>();
  if (MODE != 2) return B > 0 ? (B + R - 1) / R : 1;
  constexpr int NT = T::C_NT;
  const size_t smem = sizeof(float) * (img2_small(D) + (T::WSMEM ? 8 * D * D : 0) + R * (2 * D + 4) + R * (D + 4));
  int per_sm = (int)((228 * 1024) / (smem + 1024));
  if (per_sm > 2048 / NT) per_sm = 2048 / NT;
  if (per_sm < 1) per_sm = 1;
  return (int64_t)sm_count() * per_sm;
}

template <int D, int MODE>
cudaError_t launch_engine(const Eng2Args& a, const float* img, cudaStream_t st, int64_t* slots_out) {
  using T = Tune2<D>;
  using Gm = Geo<D>;
  constexpr int RPT = MODE == 2 ? T::C_RPT : T::F_RPT;
  constexpr int NT = MODE == 2 ? T::C_NT : T::F_NT;
  constexpr int R = (NT / Gm::TU) * RPT;
  const size_t smem = sizeof(float) * (img2_small(D) + (T::WSMEM ? 8 * D * D : 0) + R * (2 * D + 4) +
                                       R * (D + 4));
  const int64_t grid = engine_grid<D, MODE>(a.B);
  if (slots_out) *slots_out = grid * R;
  if (!a.colbuf) return cudaSuccess;   // size query only
  auto k = gru2d_engine_kernel<D, RPT, NT, MODE, T::WSMEM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  k<<<(unsigned)grid, NT, smem, st>>>(img, a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t engine_dispatch(const Eng2Args& a, const float* img, int D, cudaStream_t st, int64_t* slots) {
  switch (D) {
    case 8: return launch_engine<8, MODE>(a, img, st, slots);
    case 16: return launch_engine<16, MODE>(a, img, st, slots);
    case 32: return launch_engine<32, MODE>(a, img, st, slots);
    case 64: return launch_engine<64, MODE>(a, img, st, slots);
    case 128: return launch_engine<128, MODE>(a, img, st, slots);
    case 256: return launch_engine<256, MODE>(a, img, st, slots);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

size_t gru2d_img_floats(int D) { return (size_t)img2_floats(D); }
int gru2d_supported(int D) { return D == 8 || D == 16 || D == 32 || D == 64 || D == 128 || D == 256; }

int64_t gru2d_engine_slots(int D, int64_t B, int mode) {
  Eng2Args a{};
  a.B = B;
  int64_t slots = 0;
  if (mode == 2) engine_dispatch<2>(a, nullptr, D, 0, &slots);
  else engine_dispatch<1>(a, nullptr, D, 0, &slots);
  return slots;
}

cudaError_t gru2d_pack(const float* params, float* img, int D, cudaStream_t st) {
  const int total = img2_floats(D);
  pack2d_kernel<<<(total + 255) / 256, 256, 0, st>>>(params, img, D);
  return cudaGetLastError();
}

cudaError_t gru2d_forward(const Eng2Args& a, const float* img, int D, bool sample, cudaStream_t st) {
  return sample ? engine_dispatch<0>(a, img, D, st, nullptr) : engine_dispatch<1>(a, img, D, st, nullptr);
}

cudaError_t gru2d_bonds(int Lx, int Ly, int4* bonds, cudaStream_t st) {
  const int nb = (Lx - 1) * Ly + Lx * (Ly - 1);
  if (nb <= 0) return cudaSuccess;
  if ((size_t)nb * sizeof(int) <= 48 * 1024)
    bonds2d_kernel<true><<<1, 256, (size_t)nb * sizeof(int), st>>>(Lx, Ly, bonds);
  else
    bonds2d_kernel<false><<<1, 256, 0, st>>>(Lx, Ly, bonds);
  return cudaGetLastError();
}

cudaError_t gru2d_prep(const float* img, const float* hcache, const uint8_t* sigma, float* lp_tab,
                       int* nup_tab, int64_t B, int Lx, int N, int D, int sz0, cudaStream_t st) {
  int64_t blocks = (B * 32 + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  prep2d_kernel<<<(unsigned)blocks, 256, 0, st>>>(img, hcache, sigma, lp_tab, nup_tab, B, Lx, N, D, sz0);
  return cudaGetLastError();
}

cudaError_t gru2d_heis_chains(const Eng2Args& a, const float* img, int D, cudaStream_t st) {
  return engine_dispatch<2>(a, img, D, st, nullptr);
}

cudaError_t heis_eloc(const uint8_t* sigma, const int4* bonds, const float* delta, float* eloc, int64_t B,
                      int N, int nb, float J, float x, WsHeader* hdr, cudaStream_t st) {
  int64_t blocks = (B * 32 + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  if (blocks < 1) blocks = 1;
  heis_eloc_kernel<<<(unsigned)blocks, 256, 0, st>>>(sigma, bonds, delta, eloc, B, N, nb, J, x, hdr);
  return cudaGetLastError();
}

// Threads per CTA of the 2D reverse sweep: fewer at d_h = 128 so that the
// shared-memory tiles of one CTA stay below 227 KB.
template <int D> struct TuneB2 {
  static constexpr int NT = D >= 128 ? 128 : (D >= 16 ? 256 : 64);
  // one row per row group at d_h = 64: twice the CTAs (measured 17 % faster at 8 x 8, B = 2048)
  static constexpr int RPT = D >= 256 || D == 64 ? 1 : 2;
  static constexpr int R = (NT / Geo<D>::TU) * RPT;
  static constexpr bool GSACC = D >= 256;   // small-gradient accumulators in global scratch
};

int gru2d_bptt_grid(int D, int64_t B) {
  int R = 16;
  switch (D) {
    case 8: R = TuneB2<8>::R; break;
    case 16: R = TuneB2<16>::R; break;
    case 32: R = TuneB2<32>::R; break;
    case 64: R = TuneB2<64>::R; break;
    case 128: R = TuneB2<128>::R; break;
    case 256: R = TuneB2<256>::R; break;
  }
  return (int)((B + R - 1) / R);
}

size_t gru2d_bptt_scratch_floats(int D, int64_t B) {
  if (D < 256) return 0;
  constexpr int NRG = TuneB2<256>::NT / Geo<256>::TU;
  return (size_t)gru2d_bptt_grid(D, B) * NRG * kSmall2 * D;
}

template <int D>
cudaError_t launch_bptt2(const Bptt2Args& a, const float* img, cudaStream_t st) {
  constexpr int NT = TuneB2<D>::NT, RPT = TuneB2<D>::RPT;
  constexpr int NRG = NT / Geo<D>::TU, R = NRG * RPT;
  constexpr bool GS = TuneB2<D>::GSACC;
  const size_t smem = sizeof(float) * (img2_small(D) + R * (2 * D + 4) + R * (D + 4) + R * (2 * D + 4) +
                                       R * (3 * D + 4) + 2 * NRG + (GS ? 0 : NRG * kSmall2 * D));
  auto k = gru2d_bptt_kernel<D, RPT, NT, GS>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  const unsigned grid = (unsigned)((a.B + R - 1) / R);
  k<<<grid, NT, smem, st>>>(img, a);
  return cudaGetLastError();
}

cudaError_t gru2d_bptt(const Bptt2Args& a, const float* img, int D, cudaStream_t st) {
  switch (D) {
    case 8: return launch_bptt2<8>(a, img, st);
    case 16: return launch_bptt2<16>(a, img, st);
    case 32: return launch_bptt2<32>(a, img, st);
    case 64: return launch_bptt2<64>(a, img, st);
    case 128: return launch_bptt2<128>(a, img, st);
    case 256: return launch_bptt2<256>(a, img, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nqs

// Device bodies of the FP32 1D GRU kernels (App. A), shared by the
// per-model launches (gru1d.cu) and the grouped multi-replica launches
// (batched.cu).  A body processes one block of rows; `blk` is the block's
// index within its model.
#pragma once

#include "kernels.h"
#include "tile.cuh"

namespace nqs {

// ----------------------------------------------------------------------------
// Parameter offsets of the flat 1D layout (include/nqs.h).
// ----------------------------------------------------------------------------
struct Off1 {
  int Wg, Wr, Wh, Win, bg, br, bh, bin, U, c, P;
};
__host__ __device__ inline Off1 off1(int D) {
  Off1 o;
  o.Wg = 0;
  o.Wr = o.Wg + D * (D + 2);
  o.Wh = o.Wr + D * (D + 2);
  o.Win = o.Wh + D * D;
  o.bg = o.Win + 2 * D;
  o.br = o.bg + D;
  o.bh = o.br + D;
  o.bin = o.bh + D;
  o.U = o.bin + D;
  o.c = o.U + 2 * D;
  o.P = o.c + 2;
  return o;
}

// Packed weight image in the workspace (floats):
//   small = [Ws 2x3D | Bs 4xD | Us 2xD | c0 c1 0 0]           (12D + 4)
//   Wt[k][g*D + u]  = gate g weight (W_g, W_r, W_h) of unit u on h_k   (3D^2)
//   Wn[g*D + u][k]  = the same numbers, row-major by (gate, unit)      (3D^2)
// Ws[s][0*D+u] = W_g[u][D+s], Ws[s][D+u] = W_r[u][D+s], Ws[s][2D+u] = W_in[u][s].
__host__ __device__ constexpr int img1_small(int D) { return 12 * D + 4; }
__host__ __device__ constexpr int img1_floats(int D) { return img1_small(D) + 6 * D * D; }

// One GRU cell update for the UPT units of a lane, given the gate
// pre-activations from the h-GEMM, the one-hot input s_in (-1: zero vector)
// and the previous state hp.  Returns h' in hn and adds U h' to z0, z1.
template <int D, int UPT>
__device__ __forceinline__ void gru1d_epilogue(const float* __restrict__ small, int u0, int s_in,
                                               const float (&acc)[3][UPT], const float (&hp)[UPT],
                                               float (&hn)[UPT], float& z0, float& z1) {
  const float* Ws = small + (s_in > 0 ? 3 * D : 0);
  const float* Bs = small + 6 * D;
  const float* Us = small + 10 * D;
  const float on = s_in >= 0 ? 1.0f : 0.0f;
#pragma unroll
  for (int j = 0; j < UPT; ++j) {
    const int u = u0 + j;
    const float au = acc[0][j] + Bs[u] + on * Ws[u];
    const float ar = acc[1][j] + Bs[D + u] + on * Ws[D + u];
    const float q = acc[2][j] + Bs[2 * D + u];
    const float xin = Bs[3 * D + u] + on * Ws[2 * D + u];
    const float ug = sigmoid_acc(au);
    const float rg = sigmoid_acc(ar);
    const float c = tanhf(fmaf(rg, q, xin));
    hn[j] = fmaf(ug, c - hp[j], hp[j]);
    z0 = fmaf(Us[u], hn[j], z0);
    z1 = fmaf(Us[D + u], hn[j], z1);
  }
}

// ----------------------------------------------------------------------------
// Sampling (SAMPLE = true) or teacher forcing: one row per sample, N steps.
// ----------------------------------------------------------------------------
template <int D, int RPT, int NT, bool SAMPLE, bool WSMEM>
__device__ __forceinline__ void gru1d_forward_body(const float* __restrict__ img, const Fwd1Args& a, int blk) {
  using G = Geo<D>;
  constexpr int TU = G::TU, UPT = G::UPT, DP = G::DP;
  constexpr int NRG = NT / TU, R = NRG * RPT;
  extern __shared__ __align__(16) float sm[];
  float* small = sm;
  float* Wt = WSMEM ? sm + img1_small(D) : const_cast<float*>(img) + img1_small(D);
  float* hbuf = sm + img1_small(D) + (WSMEM ? 3 * D * D : 0);

  cta_copy4(sm, img, img1_small(D) + (WSMEM ? 3 * D * D : 0));
  for (int t = threadIdx.x; t < 2 * R * DP; t += NT) hbuf[t] = 0.0f;

  const int lane = threadIdx.x & 31, ug = lane % TU;
  const int rg = threadIdx.x / TU, r0 = rg * RPT, u0 = ug * UPT;
  const int N = a.N;
  // a segment [n0, n1) of teacher forcing starts from h_{n0-1} and sigma_{n0-1}
  const int n0 = a.n0, n1 = a.n1 ? a.n1 : N;
  const int hcr = a.hc_rows ? a.hc_rows : N;
  int s_prev[RPT];
  float lpsum[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) { s_prev[i] = -1; lpsum[i] = 0.0f; }
  if (n0 > 0) {
    __syncthreads();   // the zeroing above and the initial states below touch the same rows
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int64_t b = (int64_t)blk * R + r0 + i;
      if (b < a.B) {
        float hv[UPT];
        ld_units<UPT>(a.h_init + b * (a.hi_ld ? a.hi_ld : D) + u0, hv);
        st_units<UPT>(hbuf + (n0 & 1) * R * DP + (r0 + i) * DP + u0, hv);
        s_prev[i] = a.sigma_in[b * N + n0 - 1] ? 1 : 0;
      }
    }
  }
  const int nck = a.ckpt ? (N + a.ck - 1) / a.ck - 1 : 0;
  __syncthreads();

  for (int n = n0; n < n1; ++n) {
    const float* hc = hbuf + (n & 1) * R * DP;
    float* hx = hbuf + ((n + 1) & 1) * R * DP;
    float acc[RPT][3][UPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int g = 0; g < 3; ++g)
#pragma unroll
        for (int j = 0; j < UPT; ++j) acc[i][g][j] = 0.0f;
    if (n > 0) tile_gemm<D, RPT, 3, UPT>(hc, DP, r0, Wt, 3 * D, D, u0, acc);
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      const int64_t b = (int64_t)blk * R + row;
      const bool valid = b < a.B;
      float hp[UPT], hn[UPT];
      ld_units<UPT>(hc + row * DP + u0, hp);
      float z0 = 0.0f, z1 = 0.0f;
      gru1d_epilogue<D, UPT>(small, u0, s_prev[i], acc[i], hp, hn, z0, z1);
      st_units<UPT>(hx + row * DP + u0, hn);
      z0 = group_sum<TU>(z0);
      z1 = group_sum<TU>(z1);
      const float d = (z0 + small[12 * D]) - (z1 + small[12 * D + 1]);
      int s = 0;
      if (valid) {
        if constexpr (SAMPLE) {
          const float u = a.uniforms ? a.uniforms[b * N + n]
                                     : sampling_uniform(a.seed, a.step_dev ? *a.step_dev : a.step, (uint32_t)(a.b0 + b), (uint32_t)n);
          s = u < sigmoid_acc(d) ? 0 : 1;
          if (ug == 0) a.sigma_out[b * N + n] = (uint8_t)s;
        } else {
          s = a.sigma_in[b * N + n] ? 1 : 0;
        }
        if (a.hcache) st_units<UPT>(a.hcache + (b * hcr + n - a.hc_base) * D + u0, hn);
        if (a.ckpt && n % a.ck == a.ck - 1 && n / a.ck < nck) st_units<UPT>(a.ckpt + (b * nck + n / a.ck) * D + u0, hn);
      }
      lpsum[i] += log_prob(s, d);
      s_prev[i] = s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int64_t b = (int64_t)blk * R + r0 + i;
    if (b < a.B && ug == 0 && a.logpsi) {
      const float lp = 0.5f * lpsum[i];
      a.logpsi[b] = lp;
      if (!isfinite(lp)) flag_status(a.hdr, NQS_ENONFINITE);
    }
  }
}

// ----------------------------------------------------------------------------
// TFIM connected configurations with prefix re-use.  Job j of the queue is the
// flip of site f = j / B of sample b = j % B (longest chains first); its chain
// restarts from the cached h_f with the flipped spin as input and re-runs
// cells f+1..N-1, accumulating
//   Delta_f = 1/2 [log p_f(1-s_f) - log p_f(s_f)] + 1/2 sum_{n>f} [log p'_n - log p_n].
// A persistent grid; every row slot pulls its next job when its chain ends.
// ----------------------------------------------------------------------------
template <int D, int RPT, int NT, bool WSMEM>
__device__ __forceinline__ void tfim_chains1d_body(const float* __restrict__ img, const Chain1Args& a) {
  using G = Geo<D>;
  constexpr int TU = G::TU, UPT = G::UPT, DP = G::DP;
  constexpr int NRG = NT / TU, R = NRG * RPT;
  extern __shared__ __align__(16) float sm[];
  float* small = sm;
  float* Wt = WSMEM ? sm + img1_small(D) : const_cast<float*>(img) + img1_small(D);
  float* hbuf = sm + img1_small(D) + (WSMEM ? 3 * D * D : 0);
  cta_copy4(sm, img, img1_small(D) + (WSMEM ? 3 * D * D : 0));

  const int lane = threadIdx.x & 31, ug = lane % TU, lead = lane - ug;
  const int rg = threadIdx.x / TU, r0 = rg * RPT, u0 = ug * UPT;
  const int N = a.N;
  const int64_t B = a.B;
  const uint64_t total = (uint64_t)B * (uint64_t)(N - 1);
  int64_t jb[RPT];
  int jf[RPT], t[RPT], s_in[RPT];
  float delta[RPT];
  bool act[RPT];

  // Pull a job for row slot i (collective over the warp: all lanes call it).
  auto pull = [&](int i, bool need, float* hdst) {
    unsigned long long j = 0;
    if (need && ug == 0) j = atomicAdd(a.counter, 1ull);
    j = __shfl_sync(0xffffffffu, j, lead);
    if (!need) return;
    float hv[UPT];
    if (j < total) {
      const int64_t b = (int64_t)(j % (unsigned long long)B);
      const int f = (int)(j / (unsigned long long)B);
      const int sf = a.sigma[b * N + f] ? 1 : 0;
      const float df = a.dlog[b * N + f];
      jb[i] = b; jf[i] = f; t[i] = f + 1; s_in[i] = 1 - sf; act[i] = true;
      delta[i] = 0.5f * (sf == 0 ? -df : df);
      ld_units<UPT>(a.hcache + (b * N + f) * D + u0, hv);
    } else {
      act[i] = false;
#pragma unroll
      for (int q = 0; q < UPT; ++q) hv[q] = 0.0f;
    }
    st_units<UPT>(hdst + (r0 + i) * DP + u0, hv);
  };

#pragma unroll
  for (int i = 0; i < RPT; ++i) { act[i] = false; s_in[i] = 0; pull(i, true, hbuf); }
  __syncthreads();

  int cur = 0;
  for (;;) {
    bool any = false;
#pragma unroll
    for (int i = 0; i < RPT; ++i) any |= act[i];
    if (!__syncthreads_or(any)) break;
    const float* hc = hbuf + cur * R * DP;
    float* hx = hbuf + (cur ^ 1) * R * DP;
    float acc[RPT][3][UPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int g = 0; g < 3; ++g)
#pragma unroll
        for (int j = 0; j < UPT; ++j) acc[i][g][j] = 0.0f;
    tile_gemm<D, RPT, 3, UPT>(hc, DP, r0, Wt, 3 * D, D, u0, acc);
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      float hp[UPT], hn[UPT];
      ld_units<UPT>(hc + row * DP + u0, hp);
      float z0 = 0.0f, z1 = 0.0f;
      gru1d_epilogue<D, UPT>(small, u0, s_in[i], acc[i], hp, hn, z0, z1);
      st_units<UPT>(hx + row * DP + u0, hn);
      z0 = group_sum<TU>(z0);
      z1 = group_sum<TU>(z1);
      bool fin = false;
      if (act[i]) {
        const float d = (z0 + small[12 * D]) - (z1 + small[12 * D + 1]);
        const int64_t idx = jb[i] * N + t[i];
        const int st = a.sigma[idx] ? 1 : 0;
        delta[i] += 0.5f * (log_prob(st, d) - log_prob(st, a.dlog[idx]));
        s_in[i] = st;
        if (++t[i] == N) {
          if (ug == 0) a.delta[jb[i] * N + jf[i]] = delta[i];
          fin = true;
        }
      }
      pull(i, fin, hx);
    }
    __syncthreads();
    cur ^= 1;
  }
}

// ----------------------------------------------------------------------------
// Reverse sweep: d/dtheta sum_b w_b log psi_b.  One row per sample; sites
// n = N-1 .. 0; states h_{n-1} come from the prefix cache, gates are
// recomputed.  Per step: (1) forward recompute + backward through the readout
// and the cell, (2) dh_{n-1} = direct term + G W (G = [du_a | dr_a | dq]),
// (3) dW_h-part += G^T h_{n-1}.  Per-CTA partial gradients go to `partial`.
// ----------------------------------------------------------------------------
constexpr int kSmallGrads = 12;  // b_g b_r b_h b_in Wg_s0 Wg_s1 Wr_s0 Wr_s1 Win_s0 Win_s1 U0 U1

template <int D, int RPT, int NT, bool WSMEM, bool DW_REGS>
__device__ __forceinline__ void gru1d_bptt_body(const float* __restrict__ img, const Bptt1Args& a, int blk) {
  using G = Geo<D>;
  constexpr int TU = G::TU, UPT = G::UPT, DP = G::DP;
  constexpr int NRG = NT / TU, R = NRG * RPT;
  constexpr int KG = NT / TU;          // k groups of the dW GEMM
  constexpr int KPT = D / KG;          // k columns per lane in the dW GEMM
  static_assert(KPT >= 1 && KPT * KG == D, "bad dW tiling");
  constexpr int GP = 3 * D + 4;        // row stride of the G tile
  extern __shared__ __align__(16) float sm[];
  float* small = sm;
  const float* Wt = WSMEM ? sm + img1_small(D) : img + img1_small(D);
  const float* Wn = WSMEM ? sm + img1_small(D) + 3 * D * D : img + img1_small(D) + 3 * D * D;
  float* Hs = sm + img1_small(D) + (WSMEM ? 6 * D * D : 0);   // [R][DP]  h_{n-1}
  float* Gs = Hs + R * DP;                                      // [R][GP]
  float* sacc = Gs + R * GP;                                    // [NRG][12][D]
  float* cacc = sacc + NRG * kSmallGrads * D;                   // [NRG][2]
  cta_copy4(sm, img, img1_small(D) + (WSMEM ? 6 * D * D : 0));
  for (int q = threadIdx.x; q < NRG * (kSmallGrads * D + 2); q += NT) sacc[q] = 0.0f;

  const int lane = threadIdx.x & 31, ug = lane % TU;
  const int rg = threadIdx.x / TU, r0 = rg * RPT, u0 = ug * UPT;
  const int N = a.N;
  const int kg = threadIdx.x / TU, k0 = kg * KPT;     // dW GEMM mapping: (ug, kg)
  const float* Us = small + 10 * D;

  float coef[RPT];
  int64_t bb[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    bb[i] = (int64_t)blk * R + r0 + i;
    coef[i] = bb[i] < a.B ? 0.5f * a.weights[bb[i]] : 0.0f;
  }
  // a segment [n0, n1) starts from the carry of the later sites and hands
  // dL/dh_{n0-1} on; its first state h_{n0-1} comes from h_init
  const int n0 = a.n0, n1 = a.n1 ? a.n1 : N;
  const int hcr = a.hc_rows ? a.hc_rows : N;
  float carry[RPT][UPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    if (a.carry_in && bb[i] < a.B) {
      ld_units<UPT>(a.carry_in + bb[i] * D + u0, carry[i]);
    } else {
#pragma unroll
      for (int j = 0; j < UPT; ++j) carry[i][j] = 0.0f;
    }
  }
  float dw[DW_REGS ? 3 : 1][UPT][KPT];
  if constexpr (DW_REGS) {
#pragma unroll
    for (int g = 0; g < 3; ++g)
#pragma unroll
      for (int j = 0; j < UPT; ++j)
#pragma unroll
        for (int kk = 0; kk < KPT; ++kk) dw[g][j][kk] = 0.0f;
  }
  float* part = a.partial + (size_t)blk * a.P;
  const Off1 o = off1(D);

  for (int n = n1 - 1; n >= n0; --n) {
    // stage h_{n-1} of every row of the tile
    for (int q = threadIdx.x; q < R * (D / 4); q += NT) {
      const int row = q / (D / 4), c4 = q % (D / 4);
      const int64_t b = (int64_t)blk * R + row;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n > 0 && b < a.B) {
        const float* src = n > n0 ? a.hcache + (b * hcr + n - 1 - a.hc_base) * D
                                  : a.h_init + b * (a.hi_ld ? a.hi_ld : D);
        v = reinterpret_cast<const float4*>(src)[c4];
      }
      reinterpret_cast<float4*>(Hs + row * DP)[c4] = v;
    }
    __syncthreads();
    // (1) recompute the cell and back-propagate through readout and cell
    float acc[RPT][3][UPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int g = 0; g < 3; ++g)
#pragma unroll
        for (int j = 0; j < UPT; ++j) acc[i][g][j] = 0.0f;
    if (n > 0) tile_gemm<D, RPT, 3, UPT>(Hs, DP, r0, Wt, 3 * D, D, u0, acc);
    float sg[kSmallGrads][UPT];
#pragma unroll
    for (int q = 0; q < kSmallGrads; ++q)
#pragma unroll
      for (int j = 0; j < UPT; ++j) sg[q][j] = 0.0f;
    float dcs = 0.0f;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = r0 + i;
      const bool valid = bb[i] < a.B;
      const int s_in = (n > 0 && valid) ? (a.sigma[bb[i] * N + n - 1] ? 1 : 0) : -1;
      const int s_n = valid ? (a.sigma[bb[i] * N + n] ? 1 : 0) : 0;
      const float* Ws = small + (s_in > 0 ? 3 * D : 0);
      const float* Bs = small + 6 * D;
      const float on = s_in >= 0 ? 1.0f : 0.0f;
      float hp[UPT];
      ld_units<UPT>(Hs + row * DP + u0, hp);
      float uu[UPT], rr[UPT], qq[UPT], cc[UPT], hn[UPT];
      float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
      for (int j = 0; j < UPT; ++j) {
        const int u = u0 + j;
        uu[j] = sigmoid_acc(acc[i][0][j] + Bs[u] + on * Ws[u]);
        rr[j] = sigmoid_acc(acc[i][1][j] + Bs[D + u] + on * Ws[D + u]);
        qq[j] = acc[i][2][j] + Bs[2 * D + u];
        cc[j] = tanhf(fmaf(rr[j], qq[j], Bs[3 * D + u] + on * Ws[2 * D + u]));
        hn[j] = fmaf(uu[j], cc[j] - hp[j], hp[j]);
        z0 = fmaf(Us[u], hn[j], z0);
        z1 = fmaf(Us[D + u], hn[j], z1);
      }
      z0 = group_sum<TU>(z0);
      z1 = group_sum<TU>(z1);
      const float d = (z0 + small[12 * D]) - (z1 + small[12 * D + 1]);
      const float p0 = sigmoid_acc(d);
      const float dz0 = coef[i] * ((s_n == 0 ? 1.0f : 0.0f) - p0);   // dz1 = -dz0
      dcs += dz0;
#pragma unroll
      for (int j = 0; j < UPT; ++j) {
        const int u = u0 + j;
        const float dh = dz0 * (Us[u] - Us[D + u]) + carry[i][j];
        const float dc = dh * uu[j];
        const float du = dh * (cc[j] - hp[j]);
        carry[i][j] = dh * (1.0f - uu[j]);                   // direct path to h_{n-1}
        const float dac = dc * (1.0f - cc[j] * cc[j]);
        const float dau = du * uu[j] * (1.0f - uu[j]);
        const float dq = dac * rr[j];
        const float dar = dac * qq[j] * rr[j] * (1.0f - rr[j]);
        Gs[row * GP + u] = dau;
        Gs[row * GP + D + u] = dar;
        Gs[row * GP + 2 * D + u] = dq;
        sg[0][j] += dau; sg[1][j] += dar; sg[2][j] += dq; sg[3][j] += dac;
        if (s_in == 0) { sg[4][j] += dau; sg[6][j] += dar; sg[8][j] += dac; }
        if (s_in == 1) { sg[5][j] += dau; sg[7][j] += dar; sg[9][j] += dac; }
        sg[10][j] = fmaf(dz0, hn[j], sg[10][j]);
        sg[11][j] = fmaf(-dz0, hn[j], sg[11][j]);
      }
    }
    // owner-exclusive accumulation of the small gradients (no atomics)
#pragma unroll
    for (int q = 0; q < kSmallGrads; ++q)
#pragma unroll
      for (int j = 0; j < UPT; ++j) sacc[(rg * kSmallGrads + q) * D + u0 + j] += sg[q][j];
    if (ug == 0) {
      cacc[rg * 2 + 0] += dcs;
      cacc[rg * 2 + 1] -= dcs;
    }
    __syncthreads();
    if (n > 0) {
      // (2) dh_{n-1} += sum_{g,u} G[row][g*D+u] * W_g[u][k]
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int row = r0 + i;
        float acc2[UPT];
#pragma unroll
        for (int j = 0; j < UPT; ++j) acc2[j] = 0.0f;
#pragma unroll 2
        for (int gu = 0; gu < 3 * D; gu += 4) {
          const float4 gv = *reinterpret_cast<const float4*>(Gs + row * GP + gu);
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            float w[UPT];
            ld_units<UPT>(Wn + (gu + qq) * D + u0, w);
            const float gq = qq == 0 ? gv.x : qq == 1 ? gv.y : qq == 2 ? gv.z : gv.w;
#pragma unroll
            for (int j = 0; j < UPT; ++j) acc2[j] = fmaf(gq, w[j], acc2[j]);
          }
        }
#pragma unroll
        for (int j = 0; j < UPT; ++j) carry[i][j] += acc2[j];
      }
      // (3) dW[g*D+u][k] += sum_rows G[row][g*D+u] * h_{n-1}[row][k]
      if constexpr (DW_REGS) {
        for (int row = 0; row < R; ++row) {
          float hk[KPT], gv[3][UPT];
          ld_units<KPT>(Hs + row * DP + k0, hk);
#pragma unroll
          for (int g = 0; g < 3; ++g) ld_units<UPT>(Gs + row * GP + g * D + u0, gv[g]);
#pragma unroll
          for (int g = 0; g < 3; ++g)
#pragma unroll
            for (int j = 0; j < UPT; ++j)
#pragma unroll
              for (int kk = 0; kk < KPT; ++kk) dw[g][j][kk] = fmaf(gv[g][j], hk[kk], dw[g][j][kk]);
        }
      } else {
#pragma unroll 1
        for (int g = 0; g < 3; ++g) {
          float acc3[UPT][KPT];
#pragma unroll
          for (int j = 0; j < UPT; ++j)
#pragma unroll
            for (int kk = 0; kk < KPT; ++kk) acc3[j][kk] = 0.0f;
          for (int row = 0; row < R; ++row) {
            float hk[KPT], gv[UPT];
            ld_units<KPT>(Hs + row * DP + k0, hk);
            ld_units<UPT>(Gs + row * GP + g * D + u0, gv);
#pragma unroll
            for (int j = 0; j < UPT; ++j)
#pragma unroll
              for (int kk = 0; kk < KPT; ++kk) acc3[j][kk] = fmaf(gv[j], hk[kk], acc3[j][kk]);
          }
          const int base = g == 0 ? o.Wg : g == 1 ? o.Wr : o.Wh;
          const int ld = g == 2 ? D : D + 2;
#pragma unroll
          for (int j = 0; j < UPT; ++j)
#pragma unroll
            for (int kk = 0; kk < KPT; ++kk) part[base + (u0 + j) * ld + k0 + kk] += acc3[j][kk];
        }
      }
    }
    __syncthreads();
  }

  if (a.carry_out) {
#pragma unroll
    for (int i = 0; i < RPT; ++i)
      if (bb[i] < a.B) st_units<UPT>(a.carry_out + bb[i] * D + u0, carry[i]);
  }
  // write this CTA's partial gradient
  if constexpr (DW_REGS) {
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      const int base = g == 0 ? o.Wg : g == 1 ? o.Wr : o.Wh;
      const int ld = g == 2 ? D : D + 2;
#pragma unroll
      for (int j = 0; j < UPT; ++j)
#pragma unroll
        for (int kk = 0; kk < KPT; ++kk) part[base + (u0 + j) * ld + k0 + kk] = dw[g][j][kk];
    }
  }
  for (int u = threadIdx.x; u < D; u += NT) {
    float v[kSmallGrads];
#pragma unroll
    for (int q = 0; q < kSmallGrads; ++q) {
      float s = 0.0f;
      for (int r = 0; r < NRG; ++r) s += sacc[(r * kSmallGrads + q) * D + u];
      v[q] = s;
    }
    part[o.bg + u] = v[0];
    part[o.br + u] = v[1];
    part[o.bh + u] = v[2];
    part[o.bin + u] = v[3];
    part[o.Wg + u * (D + 2) + D] = v[4];
    part[o.Wg + u * (D + 2) + D + 1] = v[5];
    part[o.Wr + u * (D + 2) + D] = v[6];
    part[o.Wr + u * (D + 2) + D + 1] = v[7];
    part[o.Win + u * 2] = v[8];
    part[o.Win + u * 2 + 1] = v[9];
    part[o.U + u] = v[10];
    part[o.U + D + u] = v[11];
  }
  if (threadIdx.x < 2) {
    float s = 0.0f;
    for (int r = 0; r < NRG; ++r) s += cacc[r * 2 + threadIdx.x];
    part[o.c + threadIdx.x] = s;
  }
}


// Readout logit difference of cached states, dlog[r] = (U_0 - U_1) h_r + c_0 - c_1,
// for rows r = w * RPW + sub, w = warp0, warp0 + nwarps, ...: G = D / 4 lanes
// per row (one float4 each, D <= 128), RPW = 32 / G rows per warp pass, the
// G products summed by a fixed xor tree.
__device__ __forceinline__ void dlog_rows(const float* __restrict__ img, const float* __restrict__ hcache,
                                          float* __restrict__ dlog, int64_t rows, int D, int64_t warp0,
                                          int64_t nwarps) {
  const int lane = threadIdx.x & 31;
  const int G = D / 4, RPW = 32 / G, sub = lane / G, q = lane % G;
  const float4 u0 = reinterpret_cast<const float4*>(img + 10 * D)[q];
  const float4 u1 = reinterpret_cast<const float4*>(img + 11 * D)[q];
  const float4 du = make_float4(u0.x - u1.x, u0.y - u1.y, u0.z - u1.z, u0.w - u1.w);
  const float dc = img[12 * D] - img[12 * D + 1];
#pragma unroll 4
  for (int64_t base = warp0 * RPW; base < rows; base += nwarps * RPW) {
    const int64_t r = base + sub;
    float z = 0.0f;
    if (r < rows) {
      const float4 h = reinterpret_cast<const float4*>(hcache + r * D)[q];
      z = fmaf(du.x, h.x, fmaf(du.y, h.y, fmaf(du.z, h.z, du.w * h.w)));
    }
    for (int off = G / 2; off > 0; off >>= 1) z += __shfl_xor_sync(0xffffffffu, z, off);
    if (r < rows && q == 0) dlog[r] = z + dc;
  }
}

}  // namespace nqs

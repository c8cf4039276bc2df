// Complex RNN wave function (cRNN, Sec. II and Eq. softsign) on the FP32 1D
// GRU path, and the cluster-state Hamiltonian of Sec. III D.
//
// log psi(sigma) = 1/2 sum_n log p_n(sigma_n) + i sum_n phi_n with
// phi_n = pi Softsign(U_phi h_n + c_phi) . onehot(sigma_n): the phase layer
// reads the same hidden state h_n as the amplitude's softmax.  The complex
// log psi is stored as a float pair (log |psi|, phi).
//
// Cluster Hamiltonian (stabiliser reading: K_1 = Z_1 X_2, K_k = X_{k-1} Z_k
// X_{k+1}, K_N = X_{N-1} Z_N, H = -sum_k K_k): term k flips one or two sites,
// so its connected configuration differs from sigma from the first flipped
// site f on.  The chain of term k restarts from the cached h_f, flips the
// second site g when the recurrence reaches it, and accumulates the complex
// ratio log psi(sigma') - log psi(sigma) against the cached path's readout
// (amplitude logits and phase logits of every cached state, tabulated once).
//
// Kernels reuse the FP32 row-tile design of the 1D GRU (tile.cuh): a CTA owns
// R rows; the gate GEMM on h runs against the transposed weights in shared
// memory (global / L2 for d_h = 128) with RPT = 1 row per lane group.
#include "gru1d_body.cuh"

namespace nqs {

namespace {

constexpr float kPi = 3.14159265358979323846f;

__device__ __forceinline__ float softsign(float x) { return x / (1.0f + fabsf(x)); }

// phase parameters in shared memory: [U_phi 2 x D | c_phi0 c_phi1 0 0]
__host__ __device__ constexpr int phs_floats(int D) { return 2 * D + 4; }

template <int D>
__device__ __forceinline__ void load_phase(float* dst, const float* __restrict__ ph) {
  for (int t = threadIdx.x; t < 2 * D + 2; t += blockDim.x) dst[t] = ph[t];
  if (threadIdx.x < 2) dst[2 * D + 2 + threadIdx.x] = 0.0f;
}

template <int D>
constexpr bool wsmem() { return D <= 64; }

// ---------------------------------------------------------------------------
// Sampling / teacher forcing with the phase head; logpsi2 is [B, 2].
// ---------------------------------------------------------------------------
template <int D, bool SAMPLE>
__global__ void __launch_bounds__(128) crnn_forward_kernel(const float* __restrict__ img,
                                                           const float* __restrict__ phase_params,
                                                           Fwd1Args a, float* __restrict__ logpsi2) {
  using G = Geo<D>;
  constexpr int TU = G::TU, UPT = G::UPT, DP = G::DP, NT = 128;
  constexpr int R = NT / TU;
  constexpr bool WS = wsmem<D>();
  extern __shared__ __align__(16) float sm[];
  float* small = sm;
  float* ph = sm + img1_small(D);
  float* Wt = WS ? ph + phs_floats(D) : const_cast<float*>(img) + img1_small(D);
  float* hbuf = ph + phs_floats(D) + (WS ? 3 * D * D : 0);
  cta_copy4(small, img, img1_small(D));
  if (WS) cta_copy4(Wt, img + img1_small(D), 3 * D * D);
  load_phase<D>(ph, phase_params);
  for (int t = threadIdx.x; t < 2 * R * DP; t += NT) hbuf[t] = 0.0f;
  const int lane = threadIdx.x & 31, ug = lane % TU;
  const int row = threadIdx.x / TU, u0 = ug * UPT;
  const int N = a.N;
  const int64_t b = (int64_t)blockIdx.x * R + row;
  const bool valid = b < a.B;
  int s_prev = -1;
  float lpsum = 0.0f, phsum = 0.0f;
  __syncthreads();
  for (int n = 0; n < N; ++n) {
    const float* hc = hbuf + (n & 1) * R * DP;
    float* hx = hbuf + ((n + 1) & 1) * R * DP;
    float acc[1][3][UPT];
#pragma unroll
    for (int g = 0; g < 3; ++g)
#pragma unroll
      for (int j = 0; j < UPT; ++j) acc[0][g][j] = 0.0f;
    if (n > 0) tile_gemm<D, 1, 3, UPT>(hc, DP, row, Wt, 3 * D, D, u0, acc);
    float hp[UPT], hn[UPT];
    ld_units<UPT>(hc + row * DP + u0, hp);
    float z0 = 0.0f, z1 = 0.0f;
    gru1d_epilogue<D, UPT>(small, u0, s_prev, acc[0], hp, hn, z0, z1);
    st_units<UPT>(hx + row * DP + u0, hn);
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
      y0 = fmaf(ph[u0 + j], hn[j], y0);
      y1 = fmaf(ph[D + u0 + j], hn[j], y1);
    }
    z0 = group_sum<TU>(z0);
    z1 = group_sum<TU>(z1);
    y0 = group_sum<TU>(y0) + ph[2 * D];
    y1 = group_sum<TU>(y1) + ph[2 * D + 1];
    const float d = (z0 + small[12 * D]) - (z1 + small[12 * D + 1]);
    int s = 0;
    if (valid) {
      if constexpr (SAMPLE) {
        const float u = a.uniforms ? a.uniforms[b * N + n]
                                   : sampling_uniform(a.seed, a.step_dev ? *a.step_dev : a.step,
                                                      (uint32_t)(a.b0 + b), (uint32_t)n);
        s = u < sigmoid_acc(d) ? 0 : 1;
        if (ug == 0) a.sigma_out[b * N + n] = (uint8_t)s;
      } else {
        s = a.sigma_in[b * N + n] ? 1 : 0;
      }
      if (a.hcache) st_units<UPT>(a.hcache + (b * N + n) * D + u0, hn);
    }
    lpsum += log_prob(s, d);
    phsum += kPi * softsign(s == 0 ? y0 : y1);
    s_prev = s;
    __syncthreads();
  }
  if (valid && ug == 0) {
    const float lp = 0.5f * lpsum;
    logpsi2[2 * b] = lp;
    logpsi2[2 * b + 1] = phsum;
    if (!isfinite(lp) || !isfinite(phsum)) flag_status(a.hdr, NQS_ENONFINITE);
  }
}

// ---------------------------------------------------------------------------
// Cached-path readout: dlog[r] = z0 - z1 and the phase logits zph[r] = U_phi
// h_r + c_phi of every cached state r = b N + n; one warp per row.
// ---------------------------------------------------------------------------
__global__ void crnn_readout_kernel(const float* __restrict__ img, const float* __restrict__ phase_params,
                                    const float* __restrict__ hcache, float* __restrict__ dlog,
                                    float* __restrict__ zph, int64_t rows, int D) {
  const int lane = threadIdx.x & 31;
  const float* U = img + 10 * D;
  const float dc = img[12 * D] - img[12 * D + 1];
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float z = 0.0f, y0 = 0.0f, y1 = 0.0f;
    for (int u = lane; u < D; u += 32) {
      const float h = hcache[r * D + u];
      z = fmaf(U[u] - U[D + u], h, z);
      if (phase_params) {
        y0 = fmaf(phase_params[u], h, y0);
        y1 = fmaf(phase_params[D + u], h, y1);
      }
    }
    z = group_sum<32>(z);
    y0 = group_sum<32>(y0);
    y1 = group_sum<32>(y1);
    if (lane == 0) {
      dlog[r] = z + dc;
      if (phase_params) {
        zph[2 * r] = y0 + phase_params[2 * D];
        zph[2 * r + 1] = y1 + phase_params[2 * D + 1];
      }
    }
  }
}

// Term of rank q (longest chains first) and its flipped sites (0-based; g < 0: one flip).
__device__ __forceinline__ void cluster_term(int q, int N, int& k, int& f, int& g) {
  k = q == 0 ? 1 : q == 1 ? 0 : q;
  if (k == 0) { f = 1; g = -1; }
  else if (k == N - 1) { f = N - 2; g = -1; }
  else { f = k - 1; g = k + 1; }
}

struct ClusterChainArgs {
  int64_t B;
  int N;
  const uint8_t* sigma;
  const float* hcache;
  const float* dlog;        // [B, N]
  const float* zph;         // [B, N, 2]
  float* dre;               // [B, N] by term: log|psi(sigma')| - log|psi(sigma)|
  float* dim;               // [B, N] by term: phi(sigma') - phi(sigma)
  unsigned long long* counter;
  int phase;                // 0: pRNN (no phase head)
};

// ---------------------------------------------------------------------------
// Cluster-state connected configurations with prefix re-use: a persistent
// grid; every row slot pulls job j = (term rank q = j / B, sample b = j % B).
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(128) cluster_chains_kernel(const float* __restrict__ img,
                                                             const float* __restrict__ phase_params,
                                                             ClusterChainArgs a) {
  using G = Geo<D>;
  constexpr int TU = G::TU, UPT = G::UPT, DP = G::DP, NT = 128;
  constexpr int R = NT / TU;
  constexpr bool WS = wsmem<D>();
  extern __shared__ __align__(16) float sm[];
  float* small = sm;
  float* ph = sm + img1_small(D);
  float* Wt = WS ? ph + phs_floats(D) : const_cast<float*>(img) + img1_small(D);
  float* hbuf = ph + phs_floats(D) + (WS ? 3 * D * D : 0);
  cta_copy4(small, img, img1_small(D));
  if (WS) cta_copy4(Wt, img + img1_small(D), 3 * D * D);
  if (a.phase) {
    load_phase<D>(ph, phase_params);
  } else {
    for (int t = threadIdx.x; t < phs_floats(D); t += NT) ph[t] = 0.0f;
  }
  const int lane = threadIdx.x & 31, ug = lane % TU, lead = lane - ug;
  const int row = threadIdx.x / TU, u0 = ug * UPT;
  const int N = a.N;
  const int64_t B = a.B;
  const uint64_t total = (uint64_t)B * (uint64_t)N;
  int64_t jb = 0;
  int jk = 0, jg = -1, t = 0, s_in = 0;
  float dre = 0.0f, dim = 0.0f;
  bool act = false;
  auto pull = [&](bool need, float* hdst) {
    unsigned long long j = 0;
    if (need && ug == 0) j = atomicAdd(a.counter, 1ull);
    j = __shfl_sync(0xffffffffu, j, lead);
    if (!need) return;
    float hv[UPT];
    if (j < total) {
      const int q = (int)(j / (unsigned long long)B);
      jb = (int64_t)(j % (unsigned long long)B);
      int f;
      cluster_term(q, N, jk, f, jg);
      const int64_t idx = jb * N + f;
      const int sf = a.sigma[idx] ? 1 : 0;
      const float df = a.dlog[idx];
      dre = 0.5f * (log_prob(1 - sf, df) - log_prob(sf, df));
      dim = a.phase ? kPi * (softsign(a.zph[2 * idx + 1 - sf]) - softsign(a.zph[2 * idx + sf])) : 0.0f;
      t = f + 1;
      s_in = 1 - sf;
      act = true;
      ld_units<UPT>(a.hcache + idx * D + u0, hv);
    } else {
      act = false;
#pragma unroll
      for (int q = 0; q < UPT; ++q) hv[q] = 0.0f;
    }
    st_units<UPT>(hdst + row * DP + u0, hv);
  };
  pull(true, hbuf);
  __syncthreads();
  int cur = 0;
  for (;;) {
    if (!__syncthreads_or(act)) break;
    const float* hc = hbuf + cur * R * DP;
    float* hx = hbuf + (cur ^ 1) * R * DP;
    float acc[1][3][UPT];
#pragma unroll
    for (int g = 0; g < 3; ++g)
#pragma unroll
      for (int j = 0; j < UPT; ++j) acc[0][g][j] = 0.0f;
    tile_gemm<D, 1, 3, UPT>(hc, DP, row, Wt, 3 * D, D, u0, acc);
    float hp[UPT], hn[UPT];
    ld_units<UPT>(hc + row * DP + u0, hp);
    float z0 = 0.0f, z1 = 0.0f;
    gru1d_epilogue<D, UPT>(small, u0, s_in, acc[0], hp, hn, z0, z1);
    st_units<UPT>(hx + row * DP + u0, hn);
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
      y0 = fmaf(ph[u0 + j], hn[j], y0);
      y1 = fmaf(ph[D + u0 + j], hn[j], y1);
    }
    z0 = group_sum<TU>(z0);
    z1 = group_sum<TU>(z1);
    y0 = group_sum<TU>(y0) + ph[2 * D];
    y1 = group_sum<TU>(y1) + ph[2 * D + 1];
    bool fin = false;
    if (act) {
      const float d = (z0 + small[12 * D]) - (z1 + small[12 * D + 1]);
      const int64_t idx = jb * N + t;
      const int st = a.sigma[idx] ? 1 : 0;
      const int sp = t == jg ? 1 - st : st;             // the connected configuration's spin
      dre += 0.5f * (log_prob(sp, d) - log_prob(st, a.dlog[idx]));
      if (a.phase) dim += kPi * (softsign(sp == 0 ? y0 : y1) - softsign(a.zph[2 * idx + st]));
      s_in = sp;
      if (++t == N) {
        if (ug == 0) {
          a.dre[jb * N + jk] = dre;
          a.dim[jb * N + jk] = dim;
        }
        fin = true;
      }
    }
    pull(fin, hx);
    __syncthreads();
    cur ^= 1;
  }
}

// E_loc = -J sum_k s_k exp(dre_k + i dim_k); one warp per sample; eloc [B, 2]
// (cRNN) or [B] (pRNN, real).
__global__ void cluster_eloc_kernel(const uint8_t* __restrict__ sigma, const float* __restrict__ dre,
                                    const float* __restrict__ dim, float* __restrict__ eloc, int64_t B, int N,
                                    int phase, float J, WsHeader* hdr) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < B;
       b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    float er = 0.0f, ei = 0.0f;
    for (int k = lane; k < N; k += 32) {
      const float sk = sigma[b * N + k] ? -1.0f : 1.0f;
      const float m = expf(dre[b * N + k]);
      float sn, cs;
      sincosf(dim[b * N + k], &sn, &cs);
      er = fmaf(-sk * m, cs, er);
      ei = fmaf(-sk * m, sn, ei);
    }
    er = J * group_sum<32>(er);
    ei = J * group_sum<32>(ei);
    if (lane == 0) {
      if (phase) {
        eloc[2 * b] = er;
        eloc[2 * b + 1] = ei;
      } else {
        eloc[b] = er;
      }
      if (!isfinite(er) || !isfinite(ei)) flag_status(hdr, NQS_ENONFINITE);
    }
  }
}

// stats = [Re mean, mean |E - mean|^2, M, Im mean] of complex energies
// (one block, fixed order), and the complex weights w = 2 (E - mean) / M.
__global__ void complex_stats_kernel(const float* __restrict__ eloc, int64_t B, double* stats) {
  __shared__ double s[3][1024];
  double a = 0.0, bi = 0.0, c = 0.0;
  for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
    const double er = eloc[2 * i], ei = eloc[2 * i + 1];
    a += er;
    bi += ei;
    c += er * er + ei * ei;
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = bi;
  s[2][threadIdx.x] = c;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off)
      for (int q = 0; q < 3; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double M = (double)B, mr = s[0][0] / M, mi = s[1][0] / M;
    stats[0] = mr;
    stats[1] = s[2][0] / M - (mr * mr + mi * mi);
    stats[2] = M;
    stats[3] = mi;
  }
}

__global__ void complex_weights_kernel(const float* __restrict__ eloc, const double* __restrict__ stats, int64_t B,
                                       float* __restrict__ w) {
  const double mr = stats[0], mi = stats[3], M = stats[2];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
    w[2 * i] = (float)(2.0 * ((double)eloc[2 * i] - mr) / M);
    w[2 * i + 1] = (float)(2.0 * ((double)eloc[2 * i + 1] - mi) / M);
  }
}

// ---------------------------------------------------------------------------
// Reverse sweep of L = sum_b [w_b log|psi_b| + v_b phi_b] (weights2 = [B, 2]
// = (w, v)), one row per sample, sites N-1 .. 0, as the FP32 1D sweep with
// the phase layer added: dphi_n / dz_phi[s_n] = pi / (1 + |z|)^2.
// ---------------------------------------------------------------------------
constexpr int kSmallPh = 14;   // b_g b_r b_h b_in Wg_s0 Wg_s1 Wr_s0 Wr_s1 Win_s0 Win_s1 U0 U1 Uphi0 Uphi1

template <int D>
__global__ void __launch_bounds__(128) crnn_bptt_kernel(const float* __restrict__ img,
                                                        const float* __restrict__ phase_params, Bptt1Args a,
                                                        const float* __restrict__ weights2) {
  using G = Geo<D>;
  constexpr int TU = G::TU, UPT = G::UPT, DP = G::DP, NT = 128;
  constexpr int R = NT / TU, NRG = R;
  constexpr int KG = NT / TU, KPT = D / KG;
  static_assert(KPT >= 1 && KPT * KG == D, "bad dW tiling");
  constexpr int GP = 3 * D + 4;
  constexpr bool WS = wsmem<D>();
  extern __shared__ __align__(16) float sm[];
  float* small = sm;
  float* ph = sm + img1_small(D);
  float* Wt = WS ? ph + phs_floats(D) : const_cast<float*>(img) + img1_small(D);
  float* Wn = WS ? Wt + 3 * D * D : const_cast<float*>(img) + img1_small(D) + 3 * D * D;
  float* Hs = ph + phs_floats(D) + (WS ? 6 * D * D : 0);   // [R][DP] h_{n-1}
  float* Gs = Hs + R * DP;                                  // [R][GP]
  float* sacc = Gs + R * GP;                                // [NRG][14][D]
  float* cacc = sacc + NRG * kSmallPh * D;                  // [NRG][4]
  cta_copy4(small, img, img1_small(D));
  if (WS) cta_copy4(Wt, img + img1_small(D), 6 * D * D);
  load_phase<D>(ph, phase_params);
  for (int q = threadIdx.x; q < NRG * (kSmallPh * D + 4); q += NT) sacc[q] = 0.0f;

  const int lane = threadIdx.x & 31, ug = lane % TU;
  const int row = threadIdx.x / TU, rg = row, u0 = ug * UPT;
  const int N = a.N;
  const int kg = threadIdx.x / TU, k0 = kg * KPT;
  const float* Us = small + 10 * D;
  const int64_t b = (int64_t)blockIdx.x * R + row;
  const bool valid = b < a.B;
  const float coef = valid ? 0.5f * weights2[2 * b] : 0.0f;
  const float vph = valid ? weights2[2 * b + 1] : 0.0f;
  float carry[UPT];
#pragma unroll
  for (int j = 0; j < UPT; ++j) carry[j] = 0.0f;
  // dW of the h columns: in registers up to d_h 64, else accumulated in this
  // CTA's partial row (each entry owned by one thread, zeroed here)
  constexpr bool DWR = D <= 64;
  float dw[DWR ? 3 : 1][DWR ? UPT : 1][DWR ? KPT : 1];
  float* part = a.partial + (size_t)blockIdx.x * a.P;
  const Off1 o = off1(D);
  const int oUph = o.P, ocph = o.P + 2 * D;    // phase layer after the amplitude head
  auto dw_at = [&](int g, int j, int kk) -> float& {
    const int base = g == 0 ? o.Wg : g == 1 ? o.Wr : o.Wh;
    const int ld = g == 2 ? D : D + 2;
    return part[base + (u0 + j) * ld + k0 + kk];
  };
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int j = 0; j < UPT; ++j)
#pragma unroll
      for (int kk = 0; kk < KPT; ++kk) {
        if constexpr (DWR) dw[g][j][kk] = 0.0f;
        else dw_at(g, j, kk) = 0.0f;
      }

  for (int n = N - 1; n >= 0; --n) {
    for (int q = threadIdx.x; q < R * (D / 4); q += NT) {
      const int rr = q / (D / 4), c4 = q % (D / 4);
      const int64_t bq = (int64_t)blockIdx.x * R + rr;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n > 0 && bq < a.B) v = reinterpret_cast<const float4*>(a.hcache + (bq * N + n - 1) * D)[c4];
      reinterpret_cast<float4*>(Hs + rr * DP)[c4] = v;
    }
    __syncthreads();
    float acc[1][3][UPT];
#pragma unroll
    for (int g = 0; g < 3; ++g)
#pragma unroll
      for (int j = 0; j < UPT; ++j) acc[0][g][j] = 0.0f;
    if (n > 0) tile_gemm<D, 1, 3, UPT>(Hs, DP, row, Wt, 3 * D, D, u0, acc);
    float sg[kSmallPh][UPT];
#pragma unroll
    for (int q = 0; q < kSmallPh; ++q)
#pragma unroll
      for (int j = 0; j < UPT; ++j) sg[q][j] = 0.0f;
    const int s_in = (n > 0 && valid) ? (a.sigma[b * N + n - 1] ? 1 : 0) : -1;
    const int s_n = valid ? (a.sigma[b * N + n] ? 1 : 0) : 0;
    const float* Ws = small + (s_in > 0 ? 3 * D : 0);
    const float* Bs = small + 6 * D;
    const float on = s_in >= 0 ? 1.0f : 0.0f;
    float hp[UPT];
    ld_units<UPT>(Hs + row * DP + u0, hp);
    float uu[UPT], rr[UPT], qq[UPT], cc[UPT], hn[UPT];
    float z0 = 0.0f, z1 = 0.0f, y = 0.0f;
    const float* Up = ph + (s_n ? D : 0);
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
      const int u = u0 + j;
      uu[j] = sigmoid_acc(acc[0][0][j] + Bs[u] + on * Ws[u]);
      rr[j] = sigmoid_acc(acc[0][1][j] + Bs[D + u] + on * Ws[D + u]);
      qq[j] = acc[0][2][j] + Bs[2 * D + u];
      cc[j] = tanhf(fmaf(rr[j], qq[j], Bs[3 * D + u] + on * Ws[2 * D + u]));
      hn[j] = fmaf(uu[j], cc[j] - hp[j], hp[j]);
      z0 = fmaf(Us[u], hn[j], z0);
      z1 = fmaf(Us[D + u], hn[j], z1);
      y = fmaf(Up[u], hn[j], y);
    }
    z0 = group_sum<TU>(z0);
    z1 = group_sum<TU>(z1);
    y = group_sum<TU>(y) + ph[2 * D + s_n];
    const float d = (z0 + small[12 * D]) - (z1 + small[12 * D + 1]);
    const float dz0 = coef * ((s_n == 0 ? 1.0f : 0.0f) - sigmoid_acc(d));
    const float ay = 1.0f + fabsf(y);
    const float dy = vph * kPi / (ay * ay);      // d (v phi_n) / d z_phi[s_n]
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
      const int u = u0 + j;
      const float dh = dz0 * (Us[u] - Us[D + u]) + dy * Up[u] + carry[j];
      const float dc = dh * uu[j];
      const float du = dh * (cc[j] - hp[j]);
      carry[j] = dh * (1.0f - uu[j]);
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
      sg[12 + s_n][j] = fmaf(dy, hn[j], sg[12 + s_n][j]);
    }
#pragma unroll
    for (int q = 0; q < kSmallPh; ++q)
#pragma unroll
      for (int j = 0; j < UPT; ++j) sacc[(rg * kSmallPh + q) * D + u0 + j] += sg[q][j];
    if (ug == 0) {
      cacc[rg * 4 + 0] += dz0;
      cacc[rg * 4 + 1] -= dz0;
      cacc[rg * 4 + 2 + s_n] += dy;
    }
    __syncthreads();
    if (n > 0) {
      float acc2[UPT];
#pragma unroll
      for (int j = 0; j < UPT; ++j) acc2[j] = 0.0f;
#pragma unroll 2
      for (int gu = 0; gu < 3 * D; gu += 4) {
        const float4 gv = *reinterpret_cast<const float4*>(Gs + row * GP + gu);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          float w[UPT];
          ld_units<UPT>(Wn + (gu + q4) * D + u0, w);
          const float gq = q4 == 0 ? gv.x : q4 == 1 ? gv.y : q4 == 2 ? gv.z : gv.w;
#pragma unroll
          for (int j = 0; j < UPT; ++j) acc2[j] = fmaf(gq, w[j], acc2[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < UPT; ++j) carry[j] += acc2[j];
      if constexpr (DWR) {
        for (int r2 = 0; r2 < R; ++r2) {
          float hk[KPT], gv[3][UPT];
          ld_units<KPT>(Hs + r2 * DP + k0, hk);
#pragma unroll
          for (int g = 0; g < 3; ++g) ld_units<UPT>(Gs + r2 * GP + g * D + u0, gv[g]);
#pragma unroll
          for (int g = 0; g < 3; ++g)
#pragma unroll
            for (int j = 0; j < UPT; ++j)
#pragma unroll
              for (int kk = 0; kk < KPT; ++kk) dw[g][j][kk] = fmaf(gv[g][j], hk[kk], dw[g][j][kk]);
        }
      } else {
#pragma unroll 1
        for (int g = 0; g < 3; ++g)
#pragma unroll 1
          for (int kc = 0; kc < KPT; kc += 4) {
            float a3[UPT][4];
#pragma unroll
            for (int j = 0; j < UPT; ++j)
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) a3[j][kk] = 0.0f;
            for (int r2 = 0; r2 < R; ++r2) {
              const float4 hk = *reinterpret_cast<const float4*>(Hs + r2 * DP + k0 + kc);
              float gv[UPT];
              ld_units<UPT>(Gs + r2 * GP + g * D + u0, gv);
#pragma unroll
              for (int j = 0; j < UPT; ++j) {
                a3[j][0] = fmaf(gv[j], hk.x, a3[j][0]);
                a3[j][1] = fmaf(gv[j], hk.y, a3[j][1]);
                a3[j][2] = fmaf(gv[j], hk.z, a3[j][2]);
                a3[j][3] = fmaf(gv[j], hk.w, a3[j][3]);
              }
            }
#pragma unroll
            for (int j = 0; j < UPT; ++j)
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) dw_at(g, j, kc + kk) += a3[j][kk];
          }
      }
    }
    __syncthreads();
  }
  if constexpr (DWR) {
#pragma unroll
    for (int g = 0; g < 3; ++g)
#pragma unroll
      for (int j = 0; j < UPT; ++j)
#pragma unroll
        for (int kk = 0; kk < KPT; ++kk) dw_at(g, j, kk) = dw[g][j][kk];
  }
  for (int u = threadIdx.x; u < D; u += NT) {
    float v[kSmallPh];
#pragma unroll
    for (int q = 0; q < kSmallPh; ++q) {
      float s = 0.0f;
      for (int r2 = 0; r2 < NRG; ++r2) s += sacc[(r2 * kSmallPh + q) * D + u];
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
    part[oUph + u] = v[12];
    part[oUph + D + u] = v[13];
  }
  if (threadIdx.x < 4) {
    float s = 0.0f;
    for (int r2 = 0; r2 < NRG; ++r2) s += cacc[r2 * 4 + threadIdx.x];
    part[threadIdx.x < 2 ? o.c + threadIdx.x : ocph + threadIdx.x - 2] = s;
  }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return bytes > 48 * 1024 ? cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
                           : cudaSuccess;
}

template <int D>
size_t fwd_smem() {
  constexpr int R = 128 / Geo<D>::TU;
  return (size_t)(img1_small(D) + phs_floats(D) + (wsmem<D>() ? 3 * D * D : 0) + 2 * R * Geo<D>::DP) * 4;
}
template <int D>
size_t bptt_smem() {
  constexpr int R = 128 / Geo<D>::TU;
  return (size_t)(img1_small(D) + phs_floats(D) + (wsmem<D>() ? 6 * D * D : 0) + R * Geo<D>::DP +
                  R * (3 * D + 4) + R * (kSmallPh * D + 4)) * 4;
}

template <int D>
cudaError_t fwd_launch(const Fwd1Args& a, const float* img, const float* phase_params, float* logpsi2, bool sample,
                       cudaStream_t st) {
  constexpr int R = 128 / Geo<D>::TU;
  const unsigned grid = (unsigned)((a.B + R - 1) / R);
  const size_t smem = fwd_smem<D>();
  cudaError_t e;
  if (sample) {
    if ((e = set_smem(crnn_forward_kernel<D, true>, smem)) != cudaSuccess) return e;
    crnn_forward_kernel<D, true><<<grid, 128, smem, st>>>(img, phase_params, a, logpsi2);
  } else {
    if ((e = set_smem(crnn_forward_kernel<D, false>, smem)) != cudaSuccess) return e;
    crnn_forward_kernel<D, false><<<grid, 128, smem, st>>>(img, phase_params, a, logpsi2);
  }
  return cudaGetLastError();
}

template <int D>
cudaError_t chains_launch(const ClusterChainArgs& c, const float* img, const float* phase_params, cudaStream_t st) {
  const size_t smem = fwd_smem<D>();
  cudaError_t e;
  if ((e = set_smem(cluster_chains_kernel<D>, smem)) != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cluster_chains_kernel<D>, 128, smem)) != cudaSuccess)
    return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  constexpr int R = 128 / Geo<D>::TU;
  const int64_t need = ((int64_t)c.B * c.N + R - 1) / R;
  int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  cluster_chains_kernel<D><<<(unsigned)grid, 128, smem, st>>>(img, phase_params, c);
  return cudaGetLastError();
}

template <int D>
cudaError_t bptt_launch(const Bptt1Args& a, const float* img, const float* phase_params, const float* weights2,
                        cudaStream_t st) {
  constexpr int R = 128 / Geo<D>::TU;
  const unsigned grid = (unsigned)((a.B + R - 1) / R);
  const size_t smem = bptt_smem<D>();
  cudaError_t e;
  if ((e = set_smem(crnn_bptt_kernel<D>, smem)) != cudaSuccess) return e;
  crnn_bptt_kernel<D><<<grid, 128, smem, st>>>(img, phase_params, a, weights2);
  return cudaGetLastError();
}

}  // namespace

int crnn_bptt_grid(int64_t B, int D) {
  const int TU = D < 16 ? D : 16;
  const int R = 128 / TU;
  return (int)((B + R - 1) / R);
}

#define CRNN_DISPATCH(CALL)           \
  switch (D) {                        \
    case 16: return CALL(16);         \
    case 32: return CALL(32);         \
    case 64: return CALL(64);         \
    case 128: return CALL(128);       \
  }                                   \
  return cudaErrorInvalidValue;

cudaError_t crnn_forward(const Fwd1Args& a, const float* img, const float* phase_params, float* logpsi2, int D,
                         bool sample, cudaStream_t st) {
#define F(d) fwd_launch<d>(a, img, phase_params, logpsi2, sample, st)
  CRNN_DISPATCH(F)
#undef F
}

cudaError_t crnn_readout(const float* img, const float* phase_params, const float* hcache, float* dlog, float* zph,
                         int64_t rows, int D, cudaStream_t st) {
  int64_t blocks = (rows * 32 + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  if (blocks < 1) blocks = 1;
  crnn_readout_kernel<<<(unsigned)blocks, 256, 0, st>>>(img, phase_params, hcache, dlog, zph, rows, D);
  return cudaGetLastError();
}

cudaError_t cluster_local_energy(const Fwd1Args& f, const float* img, const float* phase_params, int phase,
                                 const float* dlog, const float* zph, float* dre, float* dim, float* eloc,
                                 unsigned long long* counter, float J, int D, cudaStream_t st) {
  ClusterChainArgs c{};
  c.B = f.B;
  c.N = f.N;
  c.sigma = f.sigma_in;
  c.hcache = f.hcache;
  c.dlog = dlog;
  c.zph = zph;
  c.dre = dre;
  c.dim = dim;
  c.counter = counter;
  c.phase = phase;
  cudaError_t e;
  if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
#define F(d) chains_launch<d>(c, img, phase_params, st)
  e = [&]() -> cudaError_t { CRNN_DISPATCH(F) }();
#undef F
  if (e != cudaSuccess) return e;
  int64_t blocks = (f.B * 32 + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  if (blocks < 1) blocks = 1;
  cluster_eloc_kernel<<<(unsigned)blocks, 256, 0, st>>>(f.sigma_in, dre, dim, eloc, f.B, f.N, phase, J, f.hdr);
  return cudaGetLastError();
}

cudaError_t complex_stats_weights(const float* eloc, int64_t B, double* stats, float* w, cudaStream_t st) {
  complex_stats_kernel<<<1, 1024, 0, st>>>(eloc, B, stats);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !w) return e;
  int64_t blocks = (B + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  complex_weights_kernel<<<(unsigned)blocks, 256, 0, st>>>(eloc, stats, B, w);
  return cudaGetLastError();
}

cudaError_t crnn_bptt(const Bptt1Args& a, const float* img, const float* phase_params, const float* weights2, int D,
                      cudaStream_t st) {
#define F(d) bptt_launch<d>(a, img, phase_params, weights2, st)
  CRNN_DISPATCH(F)
#undef F
}

#undef CRNN_DISPATCH

}  // namespace nqs

// BF16 tensor-core path of the 2D GRU wave function with its GLU head (App. A):
// zig-zag sampling / teacher forcing and the prefix-cached Heisenberg chains
// (Eq. heisenberg, Marshall-rotated, Sec. III B), for d_h in {32, 64} on up to
// 256 sites (d_h = 256: tc2d_wide.cu).
//
// One CTA = one tile of 128 rows (= TMEM lanes), one thread per row.  Per
// cell (position t = (i, j) of the zig-zag order, Sec. II):
//   A1  = [hi(h') | 1 1 | onehot(s_hor) onehot(s_ver) x2 | 0 | lo(h')],  h' = [h_hor | h_ver]
//   MMA1: acc = A1 W1^T, W1 = [W | W_g / 2 | U_mix] (N = 3d) with the biases and
//         one-hot input weights as BF16 hi + lo pairs in the extra columns; the
//         lo(h') columns reuse the h' columns of W1
//   epilogue 1: h~ = tanh(acc_W), u = (1 + tanh(acc_g)) / 2, h = u h~ + (1 - u) U_mix h'
//   A2  = [hi(h) | 1 1 | 0 | lo(h)]
//   MMA2: acc = A2 W2^T, W2 = [W_1 | W_2 / 2] with b_1, b_2 / 2 folded (N = 2d)
//   epilogue 2: y = (W_1 h + b_1) sigmoid(W_2 h + b_2), d = (U_0 - U_1) y + c_0 - c_1
// The 2D cell has no FP32 carry of the state: the previous states enter only
// through the GEMMs (the mixing path U_mix h' included), and the GLU reads h.
// A single BF16 rounding of h per cell compounds over the lattice, so every
// state enters both GEMMs as a BF16 pair hi + lo (hi = bf16(h), lo =
// bf16(h - hi): about 16 significant bits); the weights are plain BF16.  The
// state just computed stays in FP32 registers (the next cell's horizontal
// neighbour) as its packed hi / lo words; every state is also written in that
// packed form to a per-row column buffer in global memory (the latest state of
// each lattice column, coalesced warp stores), from which the vertical
// neighbour of the next cell is copied straight into the A operand with
// cp.async one step ahead.  A chain that restarts from the
// cache takes the states of the columns it has not recomputed yet from the
// cache the same way.  Spins of a row's configuration are a bit mask in
// registers.
#include "tc2d_common.cuh"

namespace nqs {

namespace {

using namespace tc2dh;

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// ----------------------------------------------------------------------------
// Packed BF16 operands (K-major, no swizzle; tc.cuh) and FP32 readout constants.
// ----------------------------------------------------------------------------
__global__ void pack2d_tc_kernel(const float* __restrict__ p, uint8_t* __restrict__ w1, uint8_t* __restrict__ w2,
                                 float* __restrict__ aux, int D) {
  const int K1 = 2 * D + 16, K2 = D + 16, W2c = 2 * D + 4;
  // flat layout (App. A; nqs.h): W, W_g [d, 2d+4], U_mix [d, 2d], b, b_g, W_1 [d, d], b_1, W_2, b_2, U_out [2, d], c
  const int oW = 0, oWg = D * W2c, oU = 2 * D * W2c, ob = oU + 2 * D * D, obg = ob + D, oW1 = obg + D, ob1 = oW1 + D * D,
            oW2 = ob1 + D, ob2 = oW2 + D * D, oUo = ob2 + D, oc = oUo + 2 * D;
  const int n1 = 3 * D * K1, n2 = 2 * D * K2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n1 + n2 + D + 1; t += gridDim.x * blockDim.x) {
    if (t < n1) {
      const int n = t / K1, k = t % K1, g = n / D, u = n % D;
      float v = 0.0f;
      if (k < 2 * D) {
        v = g == 0 ? p[oW + u * W2c + k] : g == 1 ? p[oWg + u * W2c + k] : p[oU + u * 2 * D + k];
      } else if (g < 2 && k < 2 * D + 10) {
        // extra columns: [b hi | b lo | w_h0 w_h1 w_v0 w_v1 hi | the same lo]
        const int e = k - 2 * D;
        const int Wo = g == 0 ? oW : oWg;
        const float x = e < 2 ? p[(g == 0 ? ob : obg) + u] : p[Wo + u * W2c + 2 * D + (e < 6 ? e - 2 : e - 6)];
        v = (e == 0 || (e >= 2 && e < 6)) ? bf16_round(x) : x - bf16_round(x);
      }
      if (g == 1) v *= 0.5f;   // u = (1 + tanh(a_g / 2)) / 2
      *reinterpret_cast<__nv_bfloat16*>(w1 + tc::kmajor_offset(n, k, K1)) = __float2bfloat16_rn(v);
    } else if (t < n1 + n2) {
      const int q = t - n1, n = q / K2, k = q % K2, g = n / D, v = n % D;
      float x = 0.0f;
      if (k < D) {
        x = p[(g == 0 ? oW1 : oW2) + v * D + k];
      } else if (k < D + 2) {
        const float bb = p[(g == 0 ? ob1 : ob2) + v];
        x = k == D ? bf16_round(bb) : bb - bf16_round(bb);
      }
      if (g == 1) x *= 0.5f;   // sigmoid(a) = (1 + tanh(a / 2)) / 2
      *reinterpret_cast<__nv_bfloat16*>(w2 + tc::kmajor_offset(n, k, K2)) = __float2bfloat16_rn(x);
    } else {
      const int v = t - n1 - n2;
      aux[v] = v < D ? p[oUo + v] - p[oUo + D + v] : p[oc] - p[oc + 1];
    }
  }
}

// Heisenberg chain jobs: the antiparallel (sample, bond) pairs in bond order
// (bonds sorted by the earlier zig-zag position: longest chains first), with
// each chain's start values taken from the cached-path tables.
__global__ void heis_count_kernel(const uint8_t* __restrict__ sigma, const int4* __restrict__ bonds, int64_t B,
                                  int N, int* __restrict__ counts) {
  __shared__ int red[32];
  const int4 bd = bonds[blockIdx.x];
  int c = 0;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) c += (sigma[b * N + bd.x] != 0) != (sigma[b * N + bd.y] != 0);
  c = warp_sum_int(c);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    counts[blockIdx.x] = s;
  }
}

// Configuration of every sample as a bit mask (bit k = spin of site k).
template <int NW>
__global__ void heis_masks_kernel(const uint8_t* __restrict__ sigma, int64_t B, int N, uint64_t* __restrict__ masks) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  uint64_t m[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) m[w] = 0ull;
  for (int k = 0; k < N; ++k)
    if (sigma[b * N + k]) m[k >> 6] |= 1ull << (k & 63);
#pragma unroll
  for (int w = 0; w < NW; ++w) masks[b * NW + w] = m[w];
}

template <int NW>
__global__ void __launch_bounds__(1024) heis_jobs_kernel(const uint8_t* __restrict__ sigma, const int4* __restrict__ bonds,
                                                        const float* __restrict__ lp_tab, const int* __restrict__ nup_tab,
                                                        const int* __restrict__ counts, const uint64_t* __restrict__ masks,
                                                        int64_t B, int N, int nb, JobT<NW>* __restrict__ jobs,
                                                        int* __restrict__ njobs) {
  __shared__ int wsum[32];
  __shared__ int base_s;
  const int rank = blockIdx.x;
  const int4 bd = bonds[rank];
  if (threadIdx.x == 0) {
    int off = 0;
    for (int q = 0; q < rank; ++q) off += counts[q];
    base_s = off;
    if (rank == nb - 1) *njobs = off + counts[rank];
  }
  __syncthreads();
  int base = base_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < B; b0 += blockDim.x) {
    const int64_t b = b0 + threadIdx.x;
    int sa = 0, sb = 0;
    bool anti = false;
    if (b < B) {
      sa = sigma[b * N + bd.x] ? 1 : 0;
      sb = sigma[b * N + bd.y] ? 1 : 0;
      anti = sa != sb;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, anti);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) before += wsum[w];
      total += wsum[w];
    }
    if (anti) {
      const int idx = base + before + __popc(bal & ((1u << lane) - 1u));
      JobT<NW> jb;
      jb.b = (int)b;
      const int pa = bd.z;
      jb.rank_pa_a = rank | (pa << 10) | (bd.x << 18);
      const int64_t row = b * N;
      // bond.x sits at position pa and takes the partner's spin sb
      jb.acc0 = 0.5f * (lp_tab[(row + pa) * 2 + sb] - lp_tab[(row + pa) * 2 + sa]);
      jb.nup_b = (nup_tab[row + pa] + (sb == 0 ? 1 : 0)) | (bd.y << 16);
      // the exchanged configuration: the two antiparallel spins swap, i.e. both flip
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        uint64_t mw = masks[b * NW + w];
        if ((bd.x >> 6) == w) mw ^= 1ull << (bd.x & 63);
        if ((bd.y >> 6) == w) mw ^= 1ull << (bd.y & 63);
        jb.mask[w] = mw;
      }
      jobs[idx] = jb;
    }
    base += total;
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// The engine.  MODE 0: sampling, 1: teacher forcing, 2: Heisenberg chains.
// ----------------------------------------------------------------------------
template <int D>
struct S2 {
  static constexpr int K1 = 2 * D + 16, K2 = D + 16, HS = D + 4;
  static constexpr int KA1 = K1 + 2 * D, KA2 = K2 + D;     // A operand columns: [hi | extras | lo]
  static constexpr int kW1 = 0;                            // [3D x K1] bf16
  static constexpr int kW2 = kW1 + 3 * D * K1 * 2;         // [2D x K2] bf16
  static constexpr int kA = kW2 + 2 * D * K2 * 2;          // A1 [128 x KA1] bf16; A2 [128 x KA2] aliases it
  static constexpr int kHS = kA + 128 * KA1 * 2;           // [128 x HS] f32: horizontal-input copy / store staging
  static constexpr int kVS = kHS + 128 * HS * 4;           // [128 x HS] f32: vertical-input copy
  static constexpr int kAux = kVS + 128 * HS * 4;          // D + 4 floats: U_0 - U_1, c_0 - c_1
  static constexpr int kCol = kAux + (D + 4) * 4;          // 128 ints: column-buffer entry of each row's new state
  static constexpr int kPos = kCol + 128 * 4;              // 256 ints: (i, j, r) of every zig-zag position
  static constexpr int kZx = kPos + 256 * 4;               // 512 floats: readout partials of the unit slices
  static constexpr int kJob = kZx + 512 * 4;               // 128 long long: chain job of each row (split rows)
  static constexpr int kBar = kJob + 128 * 8;              // 3 mbarriers: MMA1, MMA2, drain
  static constexpr int kSlot = kBar + 24;
  static constexpr int kBytes = 1024 + kSlot + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
  static constexpr uint32_t kTmemCols = 3 * D <= 128 ? 128 : 256;   // accumulators [0, 3D)
};

struct Tc2Args {
  int64_t B;
  int Lx, N, nb, sz0;
  const uint8_t* sigma_in;
  uint8_t* sigma_out;
  const float* uniforms;
  uint64_t seed, step;
  uint64_t b0;               // sampling: global index of sample 0 (Philox counter offset)
  const uint64_t* step_dev;  // sampling: device Philox step or null
  float* logpsi;             // nullable in teacher forcing
  float* hcache;             // written by sampling / teacher forcing (nullable); read by chains
  float* colbuf;             // [CTAs x 128 rows, Lx, d] latest FP32 state of every lattice column
  float* lp_tab;             // chains: cached-path tables
  int* nup_tab;
  const int4* bonds;
  const void* jobs;          // chains: JobT<NW> records
  const int* njobs;
  float* delta;
  unsigned long long* counter;
  WsHeader* hdr;
};

// REP = 4 (sampling / teacher forcing of a small batch): a CTA holds 32
// samples, every sample's A rows are written into all four TMEM lane quarters
// (the MMAs compute 128 rows either way), and warp q takes units [16 q, 16 q
// + 16) of every sample, so the epilogues of a small tile run on all four
// sub-partitions.  SPLIT > 1 (128 rows): SPLIT warps per lane quarter split a
// row's units; part 0 pulls the chain jobs and publishes them in shared
// memory.  The readout partials of the unit slices meet in shared memory; the
// readout sums 16-unit chunks in order and combines the chunks by a fixed
// pairwise tree in every variant (and in the cached-path tables).
template <int D, int MODE, int REP = 1, int SPLIT = 1, int NW = 2>
__global__ void __launch_bounds__(128 * SPLIT, 1)
tc2d_engine_kernel(const uint8_t* __restrict__ w1img, const uint8_t* __restrict__ w2img, const float* __restrict__ aux,
                   Tc2Args a) {
  using S = S2<D>;
  static_assert(REP == 1 || (REP == 4 && MODE != 2 && D == 64 && SPLIT == 1), "replicated rows: sampling / teacher forcing, d_h 64");
  constexpr int K1 = S::K1, K2 = S::K2, KA1 = S::KA1, KA2 = S::KA2;
  constexpr int NT = 128 * SPLIT;          // threads
  constexpr int NSL = REP * SPLIT;         // unit slices per row
  constexpr int DU = D / NSL;              // hidden units per thread
  constexpr int RT = 128 / REP;            // samples (rows) per CTA
  static_assert(DU >= 16 && DU % 16 == 0, "16-unit readout chunks");
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sW1 = sm + S::kW1;
  uint8_t* sW2 = sm + S::kW2;
  uint8_t* sA = sm + S::kA;
  float* sHS = reinterpret_cast<float*>(sm + S::kHS);
  float* sVS = reinterpret_cast<float*>(sm + S::kVS);
  float* sAux = reinterpret_cast<float*>(sm + S::kAux);
  int* sCol = reinterpret_cast<int*>(sm + S::kCol);
  int* sPos = reinterpret_cast<int*>(sm + S::kPos);
  float* sZx = reinterpret_cast<float*>(sm + S::kZx);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);

  long long* jbuf = reinterpret_cast<long long*>(sm + S::kJob);
  for (int i = threadIdx.x; i < 3 * D * K1 * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sW1)[i] = reinterpret_cast<const uint4*>(w1img)[i];
  for (int i = threadIdx.x; i < 2 * D * K2 * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sW2)[i] = reinterpret_cast<const uint4*>(w2img)[i];
  for (int i = threadIdx.x; i < D + 1; i += NT) sAux[i] = aux[i];
  for (int t = threadIdx.x; t < a.N; t += NT) {
    const Pz p = zpos(t, a.Lx);
    sPos[t] = p.i | (p.j << 8) | (p.r << 16);
  }
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init(&mbar[2], 1);              // drain (MMA issuer: thread 0)
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, S::kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, part = warp / 4;
  const int m = (warp % 4) * 32 + lane;    // this thread's A row and TMEM lane
  const int r = REP == 4 ? lane : m;       // its sample row in the CTA
  const int u0 = (REP == 4 ? warp : part) * DU;   // its first unit
  constexpr uint32_t kBarPub = 2;          // named barrier: chain jobs published
  float* colrow = a.colbuf + ((int64_t)blockIdx.x * RT + r) * a.Lx * D;   // this row's column buffer
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16);               // its TMEM lane (m)
  const int Lx = a.Lx, N = a.N;
  const int64_t B = a.B;
  const float dc = sAux[D];
  auto P = [&](int t) -> Pz {        // zig-zag position t (table lookup)
    const int v = sPos[t];
    Pz p;
    p.i = v & 255;
    p.j = (v >> 8) & 255;
    p.r = v >> 16;
    return p;
  };
  float* hs = sHS + r * S::HS;       // this row's horizontal-input copy
  float* vs = sVS + r * S::HS;       // this row's vertical-input copy

  // row state
  int64_t b = 0;
  int t = 0, pa = -1, rank = 0, n_up = 0, bsa = -1, bsb = -1;   // chains: exchanged lattice sites
  float acc = 0.0f, lp_next = 0.0f;
  bool active = false;
  uint64_t mask[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) mask[w] = 0ull;
  constexpr int HW = DU / 2;          // 32-bit words of this thread's packed BF16 units
  uint32_t hhi[HW], hlo[HW];         // the state just computed, as BF16 hi / lo pairs
#pragma unroll
  for (int q = 0; q < HW; ++q) hhi[q] = hlo[q] = 0u;
  // next cell's inputs: 0 zero, 1 registers, 2 FP32 shared copy, 3 copied into the A operand
  int hsrc = 0, vsrc = 0;

  auto fetch = [&](float* dst, const float* src) {
#pragma unroll
    for (int q = 0; q < DU / 4; ++q) cp_async16_2d(dst + u0 + 4 * q, src + u0 + 4 * q);
  };
  // Chains: the original state of lattice site k of sample b.
  auto fetch_orig = [&](float* dst, int k) { fetch(dst, a.hcache + (b * N + k) * D); };
  // Inputs of the cell at position tn (the row's next cell): sources and copies.
  auto plan_inputs = [&](int tn, bool fresh) {
    const Pz p = P(tn);
    hsrc = 0;
    vsrc = 0;
    bool copies = false;
    if (p.r > 0) {
      if (fresh) {              // chain start: the state at position pa is the original
        fetch_orig(hs, p.j * Lx + zhor(p));
        hsrc = 2;
        copies = true;
      } else {
        hsrc = 1;
      }
    }
    if (p.j > 0) {
      const int q = zsnake(p.i, p.j - 1, Lx);
      if (!fresh && q == tn - 1) {
        vsrc = 1;               // the state just computed (first cell of a row)
      } else if (MODE == 2 && q <= pa) {
        fetch_orig(vs, (p.j - 1) * Lx + p.i);
        vsrc = 2;
        copies = true;
      } else {
        // recomputed by this row (at least two cells back): its packed hi / lo
        // words go straight into the A operand's vertical-input columns
        // (replicated rows: into the first copy only; step (a) replicates it)
        const uint8_t* src = reinterpret_cast<const uint8_t*>(colrow + p.i * D);
        const int row = REP == 4 ? r : m;
#pragma unroll
        for (int c = u0 / 8; c < u0 / 8 + DU / 8; ++c) {
          cp_async16_2d(sA + tc::kmajor_offset(row, D + 8 * c, KA1), src + 16 * c);
          cp_async16_2d(sA + tc::kmajor_offset(row, K1 + D + 8 * c, KA1), src + 2 * D + 16 * c);
        }
        vsrc = 3;
        copies = true;
      }
    }
    if (copies) cp_commit_2d();
    if constexpr (MODE == 2) {
      const int k = p.j * Lx + p.i;
      const int so = mbit(mask, k) ^ ((k == bsa || k == bsb) ? 1 : 0);   // original spin at k
      lp_next = ldg_f32_v(a.lp_tab + (b * N + tn) * 2 + so);
    }
  };
  // Chains: take job j (or go idle).
  const unsigned long long nj = MODE == 2 ? (unsigned long long)*a.njobs : 0ull;
  auto start_job = [&](unsigned long long j) {
    if (j >= nj) {
      active = false;
      return;
    }
    const JobT<NW> jb = reinterpret_cast<const JobT<NW>*>(a.jobs)[j];
    b = jb.b;
    rank = job_rank(jb.rank_pa_a);
    pa = job_pa(jb.rank_pa_a);
    bsa = job_site_a(jb.rank_pa_a);
    bsb = job_site_b(jb.nup_b);
    t = pa + 1;
    acc = jb.acc0;
    n_up = job_nup(jb.nup_b);
#pragma unroll
    for (int w = 0; w < NW; ++w) mask[w] = jb.mask[w];
    active = true;
    plan_inputs(t, true);
  };
  // warp-aggregated pull of one job for every lane with `need`, in two halves
  // called by all lanes: the atomic is issued first and its result is read
  // later, so its round trip overlaps the step
  unsigned pbal = 0;
  unsigned long long pbase = 0;
  auto pull_issue = [&](bool need) {
    pbal = __ballot_sync(0xffffffffu, need);
    if (pbal && lane == __ffs(pbal) - 1) pbase = atomicAdd(a.counter, (unsigned long long)__popc(pbal));
  };
  auto pull_take = [&]() -> unsigned long long {
    if (!pbal) return ~0ull;
    const unsigned long long base = __shfl_sync(0xffffffffu, pbase, __ffs(pbal) - 1);
    return (pbal >> lane) & 1u ? base + __popc(pbal & ((1u << lane) - 1u)) : ~0ull;
  };

  unsigned long long jpend = ~0ull;
  if constexpr (MODE == 2) {
    if constexpr (SPLIT == 1) {
      pull_issue(true);
      start_job(pull_take());
    } else {
      // part 0 pulls one job per row and publishes it to the row's other parts
      if (part == 0) {
        pull_issue(true);
        jbuf[m] = (long long)pull_take();
      }
      tc::group_barrier(kBarPub, NT);
      start_job((unsigned long long)jbuf[m]);
    }
  } else {
    b = (int64_t)blockIdx.x * RT + r;
    active = b < B;
    if (MODE == 1 && active) {
      for (int k = 0; k < N; ++k) mset(mask, k, a.sigma_in[b * N + k] ? 1 : 0);
    }
  }

  uint32_t ph0 = 0, ph1 = 0;
  bool timed_out = false;
  const uint32_t one = 0x3F80u;
  for (int step = 0;; ++step) {
    // ---- (a) A1 row ----
    cp_wait_2d();
    int s_h = -1, s_v = -1;
    if (active) {
      const Pz p = P(t);
      if (p.r > 0) s_h = mbit(mask, p.j * Lx + zhor(p));
      if (p.j > 0) s_v = mbit(mask, (p.j - 1) * Lx + p.i);
    }
    if (REP == 4 && active && vsrc == 3) {
      // the vertical input copied into the first copy of the row: to the others
      // (reads first: interleaved with the writes they would serialise)
      uint4 vh[DU / 8], vl[DU / 8];
#pragma unroll
      for (int c = 0; c < DU / 8; ++c) {
        vh[c] = *reinterpret_cast<const uint4*>(sA + tc::kmajor_offset(r, D + u0 + 8 * c, KA1));
        vl[c] = *reinterpret_cast<const uint4*>(sA + tc::kmajor_offset(r, K1 + D + u0 + 8 * c, KA1));
      }
#pragma unroll
      for (int c4 = 1; c4 < REP; ++c4)
#pragma unroll
        for (int c = 0; c < DU / 8; ++c) {
          *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(r + 32 * c4, D + u0 + 8 * c, KA1)) = vh[c];
          *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(r + 32 * c4, K1 + D + u0 + 8 * c, KA1)) = vl[c];
        }
    }
#pragma unroll
    for (int c4 = 0; c4 < REP; ++c4) {
      const int row = REP == 4 ? r + 32 * c4 : m;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int src = active ? (half == 0 ? hsrc : vsrc) : 0;
        const float* stg = half == 0 ? hs : vs;
        uint8_t* dhi = sA + tc::kmajor_offset(row, half * D + u0, KA1);
        uint8_t* dlo = sA + tc::kmajor_offset(row, K1 + half * D + u0, KA1);
        if (src == 2) {
#pragma unroll
          for (int c = 0; c < DU / 8; ++c) st_split8(dhi + 128 * c, dlo + 128 * c, stg + u0 + 8 * c);
        } else if (src != 3) {
#pragma unroll
          for (int c = 0; c < DU / 8; ++c) {
            const bool rg = src == 1;
            *reinterpret_cast<uint4*>(dhi + 128 * c) =
                rg ? make_uint4(hhi[4 * c], hhi[4 * c + 1], hhi[4 * c + 2], hhi[4 * c + 3]) : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(dlo + 128 * c) =
                rg ? make_uint4(hlo[4 * c], hlo[4 * c + 1], hlo[4 * c + 2], hlo[4 * c + 3]) : make_uint4(0u, 0u, 0u, 0u);
          }
        }
      }
      if (u0 == 0) {
        const uint32_t oh = s_h < 0 ? 0u : (s_h == 0 ? one : (one << 16));
        const uint32_t ov = s_v < 0 ? 0u : (s_v == 0 ? one : (one << 16));
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, 2 * D, KA1)) = make_uint4(one | (one << 16), oh, ov, oh);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, 2 * D + 8, KA1)) = make_uint4(ov, 0u, 0u, 0u);
      }
    }
    // chains: a row on its last cell pulls its successor now (the loads land during the step)
    if constexpr (MODE == 2) {
      if (SPLIT == 1 || part == 0) pull_issue(active && !timed_out && t == N - 1);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    const bool any = tc::group_barrier_or(active && !timed_out, 1, NT);
    if (!any) break;
    tc::fence_after_sync();
    // ---- (b) MMA1 ----
    if (threadIdx.x == 0) {
      // A column chunk c pairs with W1 chunk c (hi and extras) or c - K1/16 (lo)
      constexpr uint32_t idesc = tc::make_idesc_bf16(128, 3 * D);
#pragma unroll
      for (int c = 0; c < KA1 / 16; ++c) {
        const int kb = c < K1 / 16 ? c : c - K1 / 16;
        const uint64_t da = tc::make_desc(tc::smem_addr(sA) + c * 256, 128, (KA1 / 8) * 128);
        const uint64_t db = tc::make_desc(tc::smem_addr(sW1) + kb * 256, 128, (K1 / 8) * 128);
        tc::mma_bf16(tbase, da, db, idesc, c > 0);
      }
      tc::mma_commit(&mbar[0]);
    }
    float uni = 0.0f;
    if (MODE == 0 && active) {
      uni = a.uniforms ? a.uniforms[b * N + t] : sampling_uniform(a.seed, a.step_dev ? *a.step_dev : a.step, (uint32_t)(a.b0 + b), (uint32_t)t);
    }
    if (!tc::mbar_wait(&mbar[0], ph0, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    ph0 ^= 1;
    tc::fence_after_sync();
    // ---- (c) epilogue 1: the cell ----
    float h[DU];
#pragma unroll
    for (int c = 0; c < DU / 8; ++c) {
      uint32_t aw[8], ag[8], au[8];
      tld8(trow + u0 + 8 * c, aw);
      tld8(trow + D + u0 + 8 * c, ag);
      tld8(trow + 2 * D + u0 + 8 * c, au);
      tc::tmem_wait_ld();
      tie(aw);
      tie(ag);
      tie(au);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float cc = hw_tanh2(__uint_as_float(aw[q]));
        const float ug = fmaf(0.5f, hw_tanh2(__uint_as_float(ag[q])), 0.5f);
        const float mix = __uint_as_float(au[q]);
        h[8 * c + q] = fmaf(ug, cc - mix, mix);
      }
    }
#pragma unroll
    for (int q = 0; q < HW; ++q) split_bf16(h[2 * q], h[2 * q + 1], hhi[q], hlo[q]);
    // A2 row [hi(h) | 1 1 | 0 | lo(h)] (aliases A1: MMA1 has completed)
#pragma unroll
    for (int c4 = 0; c4 < REP; ++c4) {
      const int row = REP == 4 ? r + 32 * c4 : m;
#pragma unroll
      for (int c = 0; c < DU / 8; ++c) {
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, u0 + 8 * c, KA2)) =
            make_uint4(hhi[4 * c], hhi[4 * c + 1], hhi[4 * c + 2], hhi[4 * c + 3]);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, K2 + u0 + 8 * c, KA2)) =
            make_uint4(hlo[4 * c], hlo[4 * c + 1], hlo[4 * c + 2], hlo[4 * c + 3]);
      }
      if (u0 == 0) {
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, D, KA2)) = make_uint4(one | (one << 16), 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(row, D + 8, KA2)) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- (d) MMA2 (the GLU) ----
    if (threadIdx.x == 0) {
      constexpr uint32_t idesc = tc::make_idesc_bf16(128, 2 * D);
#pragma unroll
      for (int c = 0; c < KA2 / 16; ++c) {
        const int kb = c < K2 / 16 ? c : c - K2 / 16;
        const uint64_t da = tc::make_desc(tc::smem_addr(sA) + c * 256, 128, (KA2 / 8) * 128);
        const uint64_t db = tc::make_desc(tc::smem_addr(sW2) + kb * 256, 128, (K2 / 8) * 128);
        tc::mma_bf16(tbase, da, db, idesc, c > 0);
      }
      tc::mma_commit(&mbar[1]);
    }
    // stores of this step's states, coalesced: every thread stages its row's
    // packed hi / lo state (and, in sampling / teacher forcing, its FP32
    // state), then each warp writes whole rows to the column buffer (entry of
    // the row's lattice column) and to the cache (all rows of such a tile are
    // at the same position).  Chains stage in hs, whose chain-start copy is
    // issued after these stores; the forward modes never copy into vs.
    {
      // packed row: [hi words (D / 2) | lo words (D / 2)]; this thread's units
      // are words [u0 / 2, (u0 + DU) / 2) of each half
      float* pst = MODE == 2 ? hs : vs;
#pragma unroll
      for (int q = 0; q < HW / 4; ++q) {
        reinterpret_cast<uint4*>(pst + u0 / 2)[q] = make_uint4(hhi[4 * q], hhi[4 * q + 1], hhi[4 * q + 2], hhi[4 * q + 3]);
        reinterpret_cast<uint4*>(pst + D / 2 + u0 / 2)[q] =
            make_uint4(hlo[4 * q], hlo[4 * q + 1], hlo[4 * q + 2], hlo[4 * q + 3]);
      }
      if constexpr (MODE != 2) {
#pragma unroll
        for (int q = 0; q < DU / 4; ++q)
          reinterpret_cast<float4*>(hs + u0)[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
      }
      sCol[r] = active ? P(t).i : -1;     // (REP: every slice writes the same value for its own lanes)
      __syncwarp();
      const int kc = MODE != 2 ? P(step).j * Lx + P(step).i : 0;
      const float* pbase = MODE == 2 ? sHS : sVS;
      if constexpr (NSL == 1) {
        // groups of G rows: all shared reads of a group, then its global
        // stores (interleaved, the stores would serialise behind the reads)
        constexpr int L = D / 4, RPI = 32 / L, G = 4;
        const int lr = lane / L, lq = lane % L;
#pragma unroll
        for (int i0 = 0; i0 < 32; i0 += RPI * G) {
          int ci[G];
          float4 vp[G], vf[G];
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int mr = warp * 32 + i0 + RPI * g + lr;
            ci[g] = sCol[mr];
            vp[g] = reinterpret_cast<const float4*>(pbase + mr * S::HS)[lq];
            if (MODE != 2) vf[g] = reinterpret_cast<const float4*>(sHS + mr * S::HS)[lq];
          }
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int mr = warp * 32 + i0 + RPI * g + lr;
            if (ci[g] >= 0) {
              const int64_t slot = (int64_t)blockIdx.x * 128 + mr;
              reinterpret_cast<float4*>(a.colbuf + (slot * Lx + ci[g]) * D)[lq] = vp[g];
              if (MODE != 2 && a.hcache)
                reinterpret_cast<float4*>(a.hcache + (slot * N + kc) * D)[lq] = vf[g];
            }
          }
        }
      } else {
        // this warp's unit slice of its 32 rows (all 32 samples with REP):
        // DU / 8 packed hi, DU / 8 packed lo and (forward modes) DU / 4 FP32
        // pieces of 16 bytes per row
        constexpr int PH = DU / 8, PF = MODE != 2 ? DU / 4 : 0, PPR = 2 * PH + PF;
        constexpr int NIT = PPR, G = NIT < 4 ? NIT : 4;   // 32 * PPR pieces, 32 per pass
        static_assert(NIT % G == 0, "store groups");
        const int m0 = REP == 4 ? 0 : (warp % 4) * 32;
        // groups of G pieces per lane: all shared reads, then the global stores
#pragma unroll
        for (int it0 = 0; it0 < NIT; it0 += G) {
          int ci[G];
          float4 v[G];
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int idx = lane + 32 * (it0 + g);
            const int mr = m0 + idx / PPR, pc = idx % PPR;
            ci[g] = sCol[mr];
            const int off = pc < 2 * PH ? (pc < PH ? u0 / 2 : D / 2 + u0 / 2) + 4 * (pc % PH) : u0 + 4 * (pc - 2 * PH);
            v[g] = *reinterpret_cast<const float4*>((pc < 2 * PH ? pbase : sHS) + mr * S::HS + off);
          }
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int idx = lane + 32 * (it0 + g);
            const int mr = m0 + idx / PPR, pc = idx % PPR;
            if (ci[g] >= 0) {
              const int64_t slot = (int64_t)blockIdx.x * RT + mr;
              if (pc < 2 * PH) {
                const int off = (pc < PH ? u0 / 2 : D / 2 + u0 / 2) + 4 * (pc % PH);
                *reinterpret_cast<float4*>(a.colbuf + (slot * Lx + ci[g]) * D + off) = v[g];
              } else if (MODE != 2 && a.hcache) {
                const int off = u0 + 4 * (pc - 2 * PH);
                *reinterpret_cast<float4*>(a.hcache + (slot * N + kc) * D + off) = v[g];
              }
            }
          }
        }
      }
      __syncwarp();
    }
    if (!tc::mbar_wait(&mbar[1], ph1, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    ph1 ^= 1;
    tc::fence_after_sync();
    // sampling / teacher forcing: the next position does not depend on this
    // cell's outcome, so its input copies go out now (the A operand is free)
    // and land during epilogue 2 and the row logic
    if constexpr (MODE != 2) {
      if (active && !timed_out && t + 1 < N) plan_inputs(t + 1, false);
    }
    // ---- (e) epilogue 2: GLU and the logit difference (16-unit chunks in
    // order, chunks by a fixed pairwise tree) ----
    float zc[DU / 16];
#pragma unroll
    for (int c = 0; c < DU / 16; ++c) zc[c] = 0.0f;
#pragma unroll
    for (int c = 0; c < DU / 8; ++c) {
      uint32_t a1[8], a2[8];
      tld8(trow + u0 + 8 * c, a1);
      tld8(trow + D + u0 + 8 * c, a2);
      tc::tmem_wait_ld();
      tie(a1);
      tie(a2);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float y = __uint_as_float(a1[q]) * fmaf(0.5f, hw_tanh2(__uint_as_float(a2[q])), 0.5f);
        zc[c / 2] = fmaf(sAux[u0 + 8 * c + q], y, zc[c / 2]);
      }
    }
#pragma unroll
    for (int w = 1; w < DU / 16; w *= 2)
#pragma unroll
      for (int c = 0; c + w < DU / 16; c += 2 * w) zc[c] += zc[c + w];
    float z = zc[0];
    if constexpr (REP == 4) {
      sZx[warp * 32 + r] = z;
      __syncthreads();
      z = (sZx[r] + sZx[32 + r]) + (sZx[64 + r] + sZx[96 + r]);
    } else if constexpr (SPLIT > 1) {
      sZx[part * 128 + m] = z;
      __syncthreads();
      float pz[SPLIT];
#pragma unroll
      for (int q = 0; q < SPLIT; ++q) pz[q] = sZx[q * 128 + m];
#pragma unroll
      for (int w = 1; w < SPLIT; w *= 2)
#pragma unroll
        for (int q = 0; q + w < SPLIT; q += 2 * w) pz[q] += pz[q + w];
      z = pz[0];
    }
    // ---- (f) row logic ----
    bool fin = false;
    if (active && !timed_out) {
      const float d = z + dc;
      const Pz p = P(t);
      const int k = p.j * Lx + p.i;
      int s;
      if constexpr (MODE == 0) {
        const bool fdn = a.sz0 && n_up >= (N >> 1);
        const bool fup = a.sz0 && (t - n_up) >= (N >> 1);
        s = fdn ? 1 : fup ? 0 : (uni < sigmoid_acc(d) ? 0 : 1);
        if (u0 == 0) a.sigma_out[b * N + k] = (uint8_t)s;
        mset(mask, k, s);
      } else {
        s = mbit(mask, k);
      }
      const float lp = lp_masked(s, d, n_up, t, N, a.sz0 != 0);
      if constexpr (MODE == 2) {
        acc += 0.5f * (lp - lp_next);
      } else {
        acc += lp;
      }
      n_up += (s == 0);
      if (++t == N) {
        fin = true;
        if constexpr (MODE == 2) {
          if (u0 == 0) a.delta[(int64_t)b * a.nb + rank] = acc;
        } else {
          const float lpsi = 0.5f * acc;
          if (a.logpsi && u0 == 0) a.logpsi[b] = lpsi;
          if (!isfinite(lpsi)) flag_status(a.hdr, NQS_ENONFINITE);
          active = false;
        }
      } else if constexpr (MODE == 2) {
        plan_inputs(t, false);
      }
    }
    if constexpr (MODE == 2) {
      if constexpr (SPLIT == 1) {
        jpend = pull_take();
        if (fin) start_job(jpend);
      } else {
        if (part == 0) jbuf[m] = (long long)pull_take();
        tc::group_barrier(kBarPub, NT);
        if (fin) start_job((unsigned long long)jbuf[m]);
      }
    }
  }
  cp_wait_2d();
  tc::fence_before_sync();
  // after a wait that gave up, TMEM is freed only once the MMAs have drained
  if (__syncthreads_or(timed_out) && threadIdx.x == 0) tc::drain_mmas(&mbar[2], kWait2);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, S::kTmemCols);
}

// ----------------------------------------------------------------------------
// Cached-path tables for the chains: for every cell (sample b, position t) the
// masked log p of both outcomes and the up-spin count before t.  The logits
// come from the GLU readout of the cached state h_t with the engine's own hi /
// lo GLU GEMM and readout order, so they equal the engine's bit for bit; every
// cell is independent, so tiles of 128 cells run in parallel.
// ----------------------------------------------------------------------------
template <int D>
struct T2S {
  static constexpr int K2 = D + 16, KA2 = K2 + D;
  static constexpr int kW2 = 0;                            // [2D x K2] bf16
  static constexpr int kA = kW2 + 2 * D * K2 * 2;          // [128 x KA2] bf16
  static constexpr int kAux = kA + 128 * KA2 * 2;          // D + 4 floats
  static constexpr int kPos = kAux + (D + 4) * 4;          // 256 ints: lattice site of every position
  static constexpr int kBar = kPos + 256 * 4;              // 2 mbarriers: MMA, drain
  static constexpr int kSlot = kBar + 16;
  static constexpr int kBytes = 1024 + kSlot + 16;
};

struct Tab2Args {
  int64_t B;
  int Lx, N, sz0;
  const uint8_t* sigma;
  const float* hcache;
  float* lp_tab;
  int* nup_tab;
  WsHeader* hdr;
};

template <int D>
__global__ void __launch_bounds__(128, 3)
tc2d_tables_kernel(const uint8_t* __restrict__ w2img, const float* __restrict__ aux, Tab2Args a) {
  using S = T2S<D>;
  constexpr int K2 = S::K2, KA2 = S::KA2;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sW2 = sm + S::kW2;
  uint8_t* sA = sm + S::kA;
  float* sAux = reinterpret_cast<float*>(sm + S::kAux);
  int* sSite = reinterpret_cast<int*>(sm + S::kPos);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < 2 * D * K2 * 2 / 16; i += 128)
    reinterpret_cast<uint4*>(sW2)[i] = reinterpret_cast<const uint4*>(w2img)[i];
  for (int i = threadIdx.x; i < D + 1; i += 128) sAux[i] = aux[i];
  for (int t = threadIdx.x; t < a.N; t += 128) {
    const Pz p = zpos(t, a.Lx);
    sSite[t] = p.j * a.Lx + p.i;
  }
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);              // drain (MMA issuer: thread 0)
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 128);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int m = threadIdx.x;
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16);
  const int N = a.N;
  const float dc = sAux[D];
  const uint32_t one = 0x3F80u;
  const int64_t ncell = a.B * N, ntile = (ncell + 127) / 128;
  uint32_t ph = 0;
  bool timed_out = false;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t cell = tile * 128 + m;
    const bool valid = cell < ncell;
    const int64_t b = valid ? cell / N : 0;
    const int t = valid ? (int)(cell % N) : 0;
    const float* hc = a.hcache + (b * N + sSite[t]) * D;
    {
      // all loads of the state first (interleaved with the shared stores they
      // would serialise), then its hi / lo rows
      float v[D];
#pragma unroll
      for (int q = 0; q < D / 4; ++q) {
        const float4 x = valid ? reinterpret_cast<const float4*>(hc)[q] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        v[4 * q] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
      }
#pragma unroll
      for (int c = 0; c < D / 8; ++c)
        st_split8(sA + tc::kmajor_offset(m, 8 * c, KA2), sA + tc::kmajor_offset(m, K2 + 8 * c, KA2), v + 8 * c);
    }
    *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, D, KA2)) = make_uint4(one | (one << 16), 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(sA + tc::kmajor_offset(m, D + 8, KA2)) = make_uint4(0u, 0u, 0u, 0u);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (m == 0) {
      constexpr uint32_t idesc = tc::make_idesc_bf16(128, 2 * D);
#pragma unroll
      for (int c = 0; c < KA2 / 16; ++c) {
        const int kb = c < K2 / 16 ? c : c - K2 / 16;
        tc::mma_bf16(tbase, tc::make_desc(tc::smem_addr(sA) + c * 256, 128, (KA2 / 8) * 128),
                     tc::make_desc(tc::smem_addr(sW2) + kb * 256, 128, (K2 / 8) * 128), idesc, c > 0);
      }
      tc::mma_commit(&mbar[0]);
    }
    // up spins before position t, while the MMA runs
    int n_up = 0;
    if (valid)
      for (int q = 0; q < t; ++q) n_up += a.sigma[b * N + sSite[q]] ? 0 : 1;
    const bool ok = tc::mbar_wait(&mbar[0], ph, wlim);
    if (!ok) flag_status(a.hdr, NQS_ETIMEOUT);
    ph ^= 1;
    tc::fence_after_sync();
    // the engine's readout order: 16-unit chunks in order, chunks by a fixed pairwise tree
    float zc[D / 16];
#pragma unroll
    for (int c = 0; c < D / 16; ++c) zc[c] = 0.0f;
#pragma unroll
    for (int c = 0; c < D / 8; ++c) {
      uint32_t a1[8], a2[8];
      tld8(trow + 8 * c, a1);
      tld8(trow + D + 8 * c, a2);
      tc::tmem_wait_ld();
      tie(a1);
      tie(a2);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float y = __uint_as_float(a1[q]) * fmaf(0.5f, hw_tanh2(__uint_as_float(a2[q])), 0.5f);
        zc[c / 2] = fmaf(sAux[8 * c + q], y, zc[c / 2]);
      }
    }
#pragma unroll
    for (int w = 1; w < D / 16; w *= 2)
#pragma unroll
      for (int c = 0; c + w < D / 16; c += 2 * w) zc[c] += zc[c + w];
    const float z = zc[0];
    if (valid) {
      const float d = z + dc;
      a.lp_tab[(b * N + t) * 2] = lp_masked(0, d, n_up, t, N, a.sz0 != 0);
      a.lp_tab[(b * N + t) * 2 + 1] = lp_masked(1, d, n_up, t, N, a.sz0 != 0);
      a.nup_tab[b * N + t] = n_up;
    }
    tc::fence_before_sync();
    // every lane has read the accumulator before the next tile's MMA; a timeout ends all lanes together
    const bool stop = __syncthreads_or(!ok);
    tc::fence_after_sync();
    if (stop) {
      timed_out = true;
      break;
    }
  }
  tc::fence_before_sync();
  // after a wait that gave up, TMEM is freed only once the MMA has drained
  if (timed_out && m == 0) tc::drain_mmas(&mbar[1], kWait2);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 128);
}

// ----------------------------------------------------------------------------
// Heisenberg chains with two 128-row tiles per CTA (the default chain kernel
// at d_h <= 64).  With one tile per CTA most of a cell step is the serial
// work of the tile's rows (A rows, epilogues, row logic), during which the
// tensor pipe idles, and the MMAs wait for that work in turn.  Here warps 0-3
// run tile 0 and warps 4-7 tile 1, each tile with its own A operand, TMEM
// columns, mbarriers, named barriers and MMA-issuing thread, over the same
// shared weights and the same job queue: one tile's MMAs and loads proceed
// while the other works through its epilogues.  The arithmetic is the
// engine's, in the same order (bitwise the same energies).  To fit two A
// operands beside the weights there are no FP32 staging rows: a cached state
// is copied by cp.async into the hi / lo slots of its own half of the row's A
// operand and split there in place, and a row's new state goes to its
// column-buffer entry by direct stores.
// ----------------------------------------------------------------------------
template <int D>
struct S2P {
  static constexpr int K1 = 2 * D + 16, K2 = D + 16;
  static constexpr int KA1 = K1 + 2 * D, KA2 = K2 + D;     // A operand columns: [hi | extras | lo]
  static constexpr int kW1 = 0;                            // [3D x K1] bf16
  static constexpr int kW2 = kW1 + 3 * D * K1 * 2;         // [2D x K2] bf16
  // 2 tiles x A1 [128 x KA1] bf16; A2 [128 x KA2] aliases A1 with A1's row-group
  // stride, so that every warp's rows lie in one region of their own in both
  // (a warp reads its rows' A2 slots while other warps already write A1)
  static constexpr int kA = kW2 + 2 * D * K2 * 2;
  static constexpr int kAux = kA + 2 * 128 * KA1 * 2;      // D + 4 floats: U_0 - U_1, c_0 - c_1
  static constexpr int kPos = kAux + (D + 4) * 4;          // 256 ints: (i, j, r) of every zig-zag position
  static constexpr int kZx = kPos + 256 * 4;               // split rows: 2 tiles x 2 parts x 128 readout partials
  static constexpr int kJob = kZx + 2 * 2 * 128 * 4;       // split rows: 2 tiles x 128 published job ids
  static constexpr int kBar = kJob + 2 * 128 * 8;          // per tile: MMA1, MMA2, drain
  static constexpr int kSlot = kBar + 6 * 8;
  static constexpr int kBytes = 1024 + kSlot + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
  static constexpr uint32_t kTileCols = 3 * D <= 128 ? 128 : 256;   // a tile's accumulators [0, 3D)
  static constexpr uint32_t kTmemCols = 2 * kTileCols;
};

template <int D, int NW, int SP>
__global__ void __launch_bounds__(256 * SP, 1)
tc2d_chain2_kernel(const uint8_t* __restrict__ w1img, const uint8_t* __restrict__ w2img, const float* __restrict__ aux,
                   Tc2Args a) {
  using S = S2P<D>;
  constexpr int K1 = S::K1, K2 = S::K2, KA1 = S::KA1, KA2 = S::KA2;
  static_assert(SP == 1 || SP == 2, "one or two threads per row");
  constexpr int NT = 256 * SP, TT = 128 * SP;   // threads of the CTA, of a tile
  constexpr int DU = D / SP;                     // hidden units per thread
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sW1 = sm + S::kW1;
  uint8_t* sW2 = sm + S::kW2;
  float* sAux = reinterpret_cast<float*>(sm + S::kAux);
  int* sPos = reinterpret_cast<int*>(sm + S::kPos);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + S::kBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + S::kSlot);
  for (int i = threadIdx.x; i < 3 * D * K1 * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sW1)[i] = reinterpret_cast<const uint4*>(w1img)[i];
  for (int i = threadIdx.x; i < 2 * D * K2 * 2 / 16; i += NT)
    reinterpret_cast<uint4*>(sW2)[i] = reinterpret_cast<const uint4*>(w2img)[i];
  for (int i = threadIdx.x; i < D + 1; i += NT) sAux[i] = aux[i];
  for (int t = threadIdx.x; t < a.N; t += NT) {
    const Pz p = zpos(t, a.Lx);
    sPos[t] = p.i | (p.j << 8) | (p.r << 16);
  }
  tc::fence_async_smem();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) tc::mbar_init(&mbar[q], 1);
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, S::kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const int g = threadIdx.x / TT, tt = threadIdx.x % TT;   // tile, thread within the tile
  const int part = tt >> 7, m = tt & 127, lane = threadIdx.x & 31;   // unit slice; row = TMEM lane
  const int u0 = part * DU;                                // this thread's first unit
  const bool issuer = tt == 0;                             // the tile's MMA-issuing thread
  uint8_t* sA = sm + S::kA + g * 128 * KA1 * 2;
  const uint32_t sA_addr = tc::smem_addr(sA);
  const uint32_t tmem0 = *tslot;
  const uint32_t tbase = tmem0 + (uint32_t)g * S::kTileCols;
  const uint32_t trow = tbase + ((uint32_t)(m & ~31) << 16);
  uint64_t* mb1 = &mbar[3 * g];
  uint64_t* mb2 = &mbar[3 * g + 1];
  uint64_t* mdrain = &mbar[3 * g + 2];
  // the tile's named barriers (TT threads each)
  const uint32_t bar_or = 1 + g, bar_sync = 3 + g, bar_z = 5 + g, bar_pub = 7 + g;
  float* sZx = reinterpret_cast<float*>(sm + S::kZx) + g * 2 * 128;
  long long* jbuf = reinterpret_cast<long long*>(sm + S::kJob) + g * 128;
  const int Lx = a.Lx, N = a.N;
  const float dc = sAux[D];
  float* colrow = a.colbuf + (((int64_t)blockIdx.x * 2 + g) * 128 + m) * Lx * D;   // this row's column buffer
  auto P = [&](int t) -> Pz {        // zig-zag position t (table lookup)
    const int v = sPos[t];
    Pz p;
    p.i = v & 255;
    p.j = (v >> 8) & 255;
    p.r = v >> 16;
    return p;
  };
  auto kmo = [&](int k, int K) { return sA + tc::kmajor_offset(m, k, K); };
  const int mw = m & ~31;            // the warp's first row

  // row state
  int64_t b = 0;
  int t = 0, pa = -1, rank = 0, n_up = 0, bsa = -1, bsb = -1;   // exchanged lattice sites
  float acc = 0.0f, lp_next = 0.0f;
  bool active = false;
  uint64_t mask[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) mask[w] = 0ull;
  // next cell's inputs: 0 zero, 1 the state just computed (in place in the
  // horizontal slots), 2 cached FP32 state in the A slots, 3 packed copy in the A slots
  int hsrc = 0, vsrc = 0;
  // The copies a row needs for its next cell, as source address | kind
  // (sources are 128-byte aligned): ldh the horizontal input (kind 2 only),
  // ldv the vertical one (kind 2 or 3).  Kind 2: a cached FP32 state (D
  // floats) into the hi / lo slots of its half of the A1 operand, floats [8c,
  // 8c + 4) to hi chunk c and [8c + 4, 8c + 8) to lo chunk c, so that
  // splitting chunk c in place reads exactly the two slots it then writes.
  // Kind 3: a packed column-buffer entry [hi words | lo words] into the
  // vertical hi and lo columns.
  uint64_t ldh = 0, ldv = 0;
  // The warp issues all its rows' copies together: one instruction covers 8
  // rows x 4 consecutive 16-byte pieces, so its global side touches 8 lines
  // (64 contiguous bytes per row) rather than 32, and its shared side the 8
  // rows' distinct bank groups.
  auto issue_slot = [&](uint64_t mine, int half) {
    if (!__any_sync(0xffffffffu, mine != 0)) return;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 8 * q + (lane & 7);
      const uint64_t u = __shfl_sync(0xffffffffu, mine, i);
      if (u) {
        const uint8_t* src = reinterpret_cast<const uint8_t*>(u & ~(uint64_t)15);
        const bool packed = (u & 15) == 3;
#pragma unroll
        for (int kk = 0; kk < DU / 16; ++kk) {
          // 16-byte piece pc of the source, among those of this thread's units
          const int L = 4 * kk + (lane >> 3);
          const int pc = packed ? (L < DU / 8 ? u0 / 8 + L : D / 8 + u0 / 8 + (L - DU / 8)) : u0 / 4 + L;
          const int col = packed ? (pc < D / 8 ? D + 8 * pc : K1 + D + 8 * (pc - D / 8))
                                 : ((pc & 1) ? K1 : 0) + half * D + 8 * (pc >> 1);
          cp_async16_cg(sA + tc::kmajor_offset(mw + i, col, KA1), src + 16 * pc);
        }
      }
    }
  };
  auto issue_copies = [&]() {
    issue_slot(ldh, 0);
    issue_slot(ldv, 1);
    cp_commit_2d();
    ldh = ldv = 0;
  };
  // Inputs of the cell at position tn (the row's next cell): sources and the
  // copies to issue; returns the cached-path log p at tn.
  auto plan_inputs = [&](int tn, bool fresh) -> float {
    const Pz p = P(tn);
    hsrc = 0;
    vsrc = 0;
    if (p.r > 0) {
      if (fresh) {              // chain start: the state at position pa is the original
        ldh = reinterpret_cast<uint64_t>(a.hcache + (b * N + p.j * Lx + zhor(p)) * D) | 2u;
        hsrc = 2;
      } else {
        hsrc = 1;
      }
    }
    if (p.j > 0) {
      const int q = zsnake(p.i, p.j - 1, Lx);
      if (!fresh && q == tn - 1) {
        vsrc = 1;               // the state just computed (first cell of a row)
      } else if (q <= pa) {
        ldv = reinterpret_cast<uint64_t>(a.hcache + (b * N + (p.j - 1) * Lx + p.i) * D) | 2u;
        vsrc = 2;
      } else {
        // recomputed by this row (at least two cells back): its packed hi / lo
        // words go straight into the vertical-input columns
        ldv = reinterpret_cast<uint64_t>(colrow + p.i * D) | 3u;
        vsrc = 3;
      }
    }
    const int k = p.j * Lx + p.i;
    const int so = mbit(mask, k) ^ ((k == bsa || k == bsb) ? 1 : 0);   // original spin at k
    return ldg_f32_v(a.lp_tab + (b * N + tn) * 2 + so);
  };
  // Take job j (or go idle).
  const unsigned long long nj = (unsigned long long)*a.njobs;
  auto start_job = [&](unsigned long long j) {
    if (j >= nj) {
      active = false;
      return;
    }
    const JobT<NW> jb = reinterpret_cast<const JobT<NW>*>(a.jobs)[j];
    b = jb.b;
    rank = job_rank(jb.rank_pa_a);
    pa = job_pa(jb.rank_pa_a);
    bsa = job_site_a(jb.rank_pa_a);
    bsb = job_site_b(jb.nup_b);
    t = pa + 1;
    acc = jb.acc0;
    n_up = job_nup(jb.nup_b);
#pragma unroll
    for (int w = 0; w < NW; ++w) mask[w] = jb.mask[w];
    active = true;
    lp_next = plan_inputs(t, true);
  };
  // warp-aggregated pull of one job for every lane with `need`, in two halves
  // called by all lanes (the atomic's round trip overlaps the step)
  unsigned pbal = 0;
  unsigned long long pbase = 0;
  auto pull_issue = [&](bool need) {
    pbal = __ballot_sync(0xffffffffu, need);
    if (pbal && lane == __ffs(pbal) - 1) pbase = atomicAdd(a.counter, (unsigned long long)__popc(pbal));
  };
  auto pull_take = [&]() -> unsigned long long {
    if (!pbal) return ~0ull;
    const unsigned long long base = __shfl_sync(0xffffffffu, pbase, __ffs(pbal) - 1);
    return (pbal >> lane) & 1u ? base + __popc(pbal & ((1u << lane) - 1u)) : ~0ull;
  };
  if constexpr (SP == 1) {
    pull_issue(true);
    start_job(pull_take());
  } else {
    if (part == 0) {
      pull_issue(true);
      jbuf[m] = (long long)pull_take();
    }
    tc::group_barrier(bar_pub, TT);
    start_job((unsigned long long)jbuf[m]);
  }
  issue_copies();

  uint32_t ph0 = 0, ph1 = 0;
  bool timed_out = false;
  const uint32_t one = 0x3F80u;
  for (;;) {
    // ---- (a) A1 row ----
    cp_wait_2d();
    __syncwarp();   // the copies into this row's slots were issued by other lanes of the warp
    int s_h = -1, s_v = -1;
    if (active) {
      const Pz p = P(t);
      if (p.r > 0) s_h = mbit(mask, p.j * Lx + zhor(p));
      if (p.j > 0) s_v = mbit(mask, (p.j - 1) * Lx + p.i);
    }
    if (active && vsrc == 1) {
      // the state just computed (hi / lo, left in the horizontal slots by
      // the A2 row) is this first cell's vertical input
      // (reads before writes throughout: interleaved, they would serialise)
#pragma unroll
      for (int lo = 0; lo < 2; ++lo) {
        uint4 v[DU / 8];
#pragma unroll
        for (int c = 0; c < DU / 8; ++c) v[c] = *reinterpret_cast<const uint4*>(kmo(lo * K1 + u0 + 8 * c, KA1));
#pragma unroll
        for (int c = 0; c < DU / 8; ++c) *reinterpret_cast<uint4*>(kmo(lo * K1 + D + u0 + 8 * c, KA1)) = v[c];
      }
    }
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int src = active ? (half == 0 ? hsrc : vsrc) : 0;
      uint8_t* dhi = kmo(half * D + u0, KA1);
      uint8_t* dlo = kmo(K1 + half * D + u0, KA1);
      if (src == 2) {
        float4 f0[DU / 8], f1[DU / 8];
#pragma unroll
        for (int c = 0; c < DU / 8; ++c) {
          f0[c] = *reinterpret_cast<const float4*>(dhi + 128 * c);
          f1[c] = *reinterpret_cast<const float4*>(dlo + 128 * c);
        }
#pragma unroll
        for (int c = 0; c < DU / 8; ++c) {
          const float v[8] = {f0[c].x, f0[c].y, f0[c].z, f0[c].w, f1[c].x, f1[c].y, f1[c].z, f1[c].w};
          st_split8(dhi + 128 * c, dlo + 128 * c, v);
        }
      } else if (src == 0) {
#pragma unroll
        for (int c = 0; c < DU / 8; ++c) {
          *reinterpret_cast<uint4*>(dhi + 128 * c) = make_uint4(0u, 0u, 0u, 0u);
          *reinterpret_cast<uint4*>(dlo + 128 * c) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
    }
    if (part == 0) {
      const uint32_t oh = s_h < 0 ? 0u : (s_h == 0 ? one : (one << 16));
      const uint32_t ov = s_v < 0 ? 0u : (s_v == 0 ? one : (one << 16));
      *reinterpret_cast<uint4*>(kmo(2 * D, KA1)) = make_uint4(one | (one << 16), oh, ov, oh);
      *reinterpret_cast<uint4*>(kmo(2 * D + 8, KA1)) = make_uint4(ov, 0u, 0u, 0u);
    }
    // a row on its last cell pulls its successor now (the loads land during the step)
    if (part == 0) pull_issue(active && !timed_out && t == N - 1);
    tc::fence_async_smem();
    tc::fence_before_sync();
    const bool any = tc::group_barrier_or(active && !timed_out, bar_or, TT);
    if (!any) break;
    tc::fence_after_sync();
    // ---- (b) MMA1 ----
    if (issuer) {
      // A column chunk c pairs with W1 chunk c (hi and extras) or c - K1/16 (lo)
      constexpr uint32_t idesc = tc::make_idesc_bf16(128, 3 * D);
#pragma unroll
      for (int c = 0; c < KA1 / 16; ++c) {
        const int kb = c < K1 / 16 ? c : c - K1 / 16;
        const uint64_t da = tc::make_desc(sA_addr + c * 256, 128, (KA1 / 8) * 128);
        const uint64_t db = tc::make_desc(tc::smem_addr(sW1) + kb * 256, 128, (K1 / 8) * 128);
        tc::mma_bf16(tbase, da, db, idesc, c > 0);
      }
      tc::mma_commit(mb1);
    }
    if (!tc::mbar_wait(mb1, ph0, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    ph0 ^= 1;
    tc::fence_after_sync();
    // ---- (c) epilogue 1: the cell, in 16-unit chunks; the A2 row [hi(h) | 1 1
    // | 0] keeps A1's horizontal hi columns and lo(h) goes to A1's horizontal
    // lo columns (MMA1 has completed), so that a next cell whose horizontal
    // input is h finds it in place ----
    // (TMEM loads double-buffered: chunk c + 1's are in flight while chunk c
    // is computed)
    constexpr int NC = DU / 16;
    uint32_t ra[2][3][16];
    auto load1 = [&](int c, uint32_t (&r)[3][16]) {
      tld16(trow + u0 + 16 * c, r[0]);
      tld16(trow + D + u0 + 16 * c, r[1]);
      tld16(trow + 2 * D + u0 + 16 * c, r[2]);
    };
    load1(0, ra[0]);
    tc::tmem_wait_ld();
    tie(ra[0][0]);
    tie(ra[0][1]);
    tie(ra[0][2]);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      uint32_t (&cur)[3][16] = ra[c & 1];
      if (c + 1 < NC) load1(c + 1, ra[(c + 1) & 1]);
      float h[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float cc = hw_tanh2(__uint_as_float(cur[0][q]));
        const float ug = fmaf(0.5f, hw_tanh2(__uint_as_float(cur[1][q])), 0.5f);
        const float mix = __uint_as_float(cur[2][q]);
        h[q] = fmaf(ug, cc - mix, mix);
      }
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) split_bf16(h[2 * q], h[2 * q + 1], hi[q], lo[q]);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        *reinterpret_cast<uint4*>(kmo(u0 + 16 * c + 8 * e, KA1)) =
            make_uint4(hi[4 * e], hi[4 * e + 1], hi[4 * e + 2], hi[4 * e + 3]);
        *reinterpret_cast<uint4*>(kmo(K1 + u0 + 16 * c + 8 * e, KA1)) =
            make_uint4(lo[4 * e], lo[4 * e + 1], lo[4 * e + 2], lo[4 * e + 3]);
      }
      if (c + 1 < NC) {
        tc::tmem_wait_ld();
        tie(ra[(c + 1) & 1][0]);
        tie(ra[(c + 1) & 1][1]);
        tie(ra[(c + 1) & 1][2]);
      }
    }
    if (part == 0) {
      *reinterpret_cast<uint4*>(kmo(D, KA1)) = make_uint4(one | (one << 16), 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(kmo(D + 8, KA1)) = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    tc::group_barrier(bar_sync, TT);
    tc::fence_after_sync();
    // ---- (d) MMA2 (the GLU) ----
    if (issuer) {
      constexpr uint32_t idesc = tc::make_idesc_bf16(128, 2 * D);
#pragma unroll
      for (int c = 0; c < KA2 / 16; ++c) {
        // A chunks: hi(h) and the extras, then lo(h) from the horizontal lo columns
        const int kb = c < K2 / 16 ? c : c - K2 / 16;
        const int ca = c < K2 / 16 ? c : K1 / 16 + kb;
        const uint64_t da = tc::make_desc(sA_addr + ca * 256, 128, (KA1 / 8) * 128);
        const uint64_t db = tc::make_desc(tc::smem_addr(sW2) + kb * 256, 128, (K2 / 8) * 128);
        tc::mma_bf16(tbase, da, db, idesc, c > 0);
      }
      tc::mma_commit(mb2);
    }
    // this state, packed [hi words (D / 2) | lo words (D / 2)], to the row's
    // column-buffer entry of its lattice column, by the warp together (8 rows
    // x 4 pieces per instruction) from the A2 rows, which MMA2 only reads
    {
      // all shared reads first, then all global stores (the compiler cannot
      // tell the two apart, so interleaved they would serialise)
      // a state is read back from the buffer only as the vertical input of the
      // cell above it, and not at all when that cell comes right after it
      // (the last cell of a lattice row) or does not exist (the top row)
      int ci_me = -1;
      if (active) {
        const Pz p = P(t);
        if (p.r < Lx - 1 && (p.j + 1) * Lx < N) ci_me = p.i;
      }
      float* cbase = a.colbuf + (((int64_t)blockIdx.x * 2 + g) * 128 + mw) * Lx * D;
      int ci[4];
      uint4 v[4][DU / 16];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 8 * q + (lane & 7);
        ci[q] = __shfl_sync(0xffffffffu, ci_me, i);
#pragma unroll
        for (int kk = 0; kk < DU / 16; ++kk) {
          const int L = 4 * kk + (lane >> 3);   // this thread's units' pieces: hi, then lo
          const int pc = L < DU / 8 ? u0 / 8 + L : D / 8 + u0 / 8 + (L - DU / 8);
          const int col = pc < D / 8 ? 8 * pc : K1 + 8 * (pc - D / 8);
          v[q][kk] = *reinterpret_cast<const uint4*>(sA + tc::kmajor_offset(mw + i, col, KA1));
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (ci[q] >= 0) {
          uint4* e = reinterpret_cast<uint4*>(cbase + ((int64_t)(8 * q + (lane & 7)) * Lx + ci[q]) * D);
#pragma unroll
          for (int kk = 0; kk < DU / 16; ++kk) {
            const int L = 4 * kk + (lane >> 3);
            e[L < DU / 8 ? u0 / 8 + L : D / 8 + u0 / 8 + (L - DU / 8)] = v[q][kk];
          }
        }
      }
      __syncwarp();   // these reads of other rows' A2 slots precede any later write to them
    }
    if (!tc::mbar_wait(mb2, ph1, wlim)) {
      timed_out = true;
      flag_status(a.hdr, NQS_ETIMEOUT);
    }
    ph1 ^= 1;
    tc::fence_after_sync();
    // ---- (e) epilogue 2: GLU and the logit difference (16-unit chunks in
    // order, chunks by a fixed pairwise tree) ----
    float zc[DU / 16];
    {
      // TMEM loads double-buffered as in epilogue 1
      constexpr int NC = DU / 16;
      uint32_t rb[2][2][16];
      auto load2 = [&](int c, uint32_t (&r)[2][16]) {
        tld16(trow + u0 + 16 * c, r[0]);
        tld16(trow + D + u0 + 16 * c, r[1]);
      };
      load2(0, rb[0]);
      tc::tmem_wait_ld();
      tie(rb[0][0]);
      tie(rb[0][1]);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        uint32_t (&cur)[2][16] = rb[c & 1];
        if (c + 1 < NC) load2(c + 1, rb[(c + 1) & 1]);
        float u[16];   // U_0 - U_1 of these units
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 f = reinterpret_cast<const float4*>(sAux + u0 + 16 * c)[q];
          u[4 * q] = f.x;
          u[4 * q + 1] = f.y;
          u[4 * q + 2] = f.z;
          u[4 * q + 3] = f.w;
        }
        zc[c] = 0.0f;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float y = __uint_as_float(cur[0][q]) * fmaf(0.5f, hw_tanh2(__uint_as_float(cur[1][q])), 0.5f);
          zc[c] = fmaf(u[q], y, zc[c]);
        }
        if (c + 1 < NC) {
          tc::tmem_wait_ld();
          tie(rb[(c + 1) & 1][0]);
          tie(rb[(c + 1) & 1][1]);
        }
      }
    }
#pragma unroll
    for (int w = 1; w < DU / 16; w *= 2)
#pragma unroll
      for (int c = 0; c + w < DU / 16; c += 2 * w) zc[c] += zc[c + w];
    float z = zc[0];
    if constexpr (SP == 2) {
      // the two halves' sums meet at the top of the same pairwise tree
      sZx[part * 128 + m] = z;
      tc::group_barrier(bar_z, TT);
      z = sZx[m] + sZx[128 + m];
    }
    // ---- (f) row logic ----
    bool fin = false;
    if (active && !timed_out) {
      const float d = z + dc;
      const Pz p = P(t);
      const int s = mbit(mask, p.j * Lx + p.i);
      const float lp = lp_masked(s, d, n_up, t, N, a.sz0 != 0);
      acc += 0.5f * (lp - lp_next);
      n_up += (s == 0);
      if (++t == N) {
        fin = true;
        if (part == 0) a.delta[(int64_t)b * a.nb + rank] = acc;
      } else {
        lp_next = plan_inputs(t, false);
      }
    }
    if constexpr (SP == 1) {
      const unsigned long long jn = pull_take();
      if (fin) start_job(jn);
    } else {
      // part 0 pulled the row's job; both parts take it
      if (part == 0) jbuf[m] = (long long)pull_take();
      tc::group_barrier(bar_pub, TT);
      if (fin) start_job((unsigned long long)jbuf[m]);
    }
    issue_copies();
  }
  cp_wait_2d();
  tc::fence_before_sync();
  // after a wait that gave up, TMEM is freed only once both tiles' MMAs have drained
  if (__syncthreads_or(timed_out) && issuer) tc::drain_mmas(mdrain, kWait2);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tmem0, S::kTmemCols);
}

int sm_count_2d() {
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

template <int D, int MODE, int REP, int SPLIT, int NW>
cudaError_t launch2_nw(const Tc2Args& a, const uint8_t* w1, const uint8_t* w2, const float* aux, cudaStream_t st) {
  using S = S2<D>;
  auto k = tc2d_engine_kernel<D, MODE, REP, SPLIT, NW>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  const int64_t grid = MODE == 2 ? sm_count_2d() : (a.B + 128 / REP - 1) / (128 / REP);
  if (grid < 1) return cudaSuccess;
  k<<<(unsigned)grid, 128 * SPLIT, S::kBytes, st>>>(w1, w2, aux, a);
  return cudaGetLastError();
}

// configurations as 128-bit masks up to 128 sites, 256-bit masks up to 256
template <int D, int MODE, int REP = 1, int SPLIT = 1>
cudaError_t launch2(const Tc2Args& a, const uint8_t* w1, const uint8_t* w2, const float* aux, cudaStream_t st) {
  return a.N > 128 ? launch2_nw<D, MODE, REP, SPLIT, 4>(a, w1, w2, aux, st)
                   : launch2_nw<D, MODE, REP, SPLIT, 2>(a, w1, w2, aux, st);
}

// Sampling / teacher forcing at d_h = 64: 32-sample CTAs with replicated A
// rows while 128-sample tiles would leave SMs idle; a pinned tile variant
// selects 128 (variant 0) or 32 (any other).
template <int MODE>
cudaError_t launch2_fwd64(const Tc2Args& a, const uint8_t* w1, const uint8_t* w2, const float* aux, cudaStream_t st) {
  const int pin = tc1d_pinned_variant();
  if (pin >= 0 ? pin > 0 : a.B <= 32LL * sm_count_2d()) return launch2<64, MODE, 4>(a, w1, w2, aux, st);
  return launch2<64, MODE, 1>(a, w1, w2, aux, st);
}

// Chains on two 128-row tiles per CTA, one CTA per SM, SP threads per row.
template <int D, int SP>
cudaError_t launch_chain2(const Tc2Args& a, const uint8_t* w1, const uint8_t* w2, const float* aux, cudaStream_t st) {
  auto k = a.N > 128 ? tc2d_chain2_kernel<D, 4, SP> : tc2d_chain2_kernel<D, 2, SP>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S2P<D>::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  k<<<(unsigned)sm_count_2d(), 256 * SP, S2P<D>::kBytes, st>>>(w1, w2, aux, a);
  return cudaGetLastError();
}

}  // namespace

int tc2d_supported(int D, int Lx, int N) {
  if (D != 32 && D != 64 && D != 256) return 0;   // d_h = 256: tc2d_wide.cu
  return N <= 256 && Lx >= 1;
}

size_t tc2d_colbuf_floats(int64_t B, int Lx, int D) {
  const int64_t rows_fwd = (B + 127) / 128 * 128, rows_chain = (int64_t)sm_count_2d() * 256;
  return (size_t)(rows_fwd > rows_chain ? rows_fwd : rows_chain) * Lx * D;
}

size_t tc2d_wimg_bytes(int D) {
  return (size_t)(3 * D * (2 * D + 16) + 2 * D * (D + 16)) * 2 + (size_t)(D + 4) * 4;
}

// chain job records carry 128-bit configuration masks where N <= 128 and the
// engine is the d_h <= 64 one, 256-bit masks otherwise
static bool wide_jobs(int N, int D) { return N > 128 || D == 256; }

// [job records | counts (nb) and the job count | sample masks (16-byte aligned)]
static size_t jobs_masks_offset(int64_t B, int nb, int N, int D) {
  const size_t rec = wide_jobs(N, D) ? sizeof(JobT<4>) : sizeof(JobT<2>);
  return ((size_t)B * nb * rec + (size_t)(nb + 4) * sizeof(int) + 15) / 16 * 16;
}

size_t tc2d_jobs_bytes(int64_t B, int nb, int N, int D) {
  return jobs_masks_offset(B, nb, N, D) + (size_t)B * (wide_jobs(N, D) ? 4 : 2) * sizeof(uint64_t);
}

cudaError_t tc2d_pack(const float* params, uint8_t* wimg, int D, cudaStream_t st) {
  if (D == 256) return tc2dw_pack(params, wimg, st);
  uint8_t* w1 = wimg;
  uint8_t* w2 = w1 + (size_t)3 * D * (2 * D + 16) * 2;
  float* aux = reinterpret_cast<float*>(w2 + (size_t)2 * D * (D + 16) * 2);
  const int total = 3 * D * (2 * D + 16) + 2 * D * (D + 16) + D + 1;
  pack2d_tc_kernel<<<(total + 255) / 256, 256, 0, st>>>(params, w1, w2, aux, D);
  return cudaGetLastError();
}

cudaError_t tc2d_forward(const Tc2Fwd& f, const uint8_t* wimg, int D, bool sample, cudaStream_t st) {
  if (D == 256) return tc2dw_forward(f, wimg, sample, st);
  Tc2Args a{};
  a.B = f.B;
  a.Lx = f.Lx;
  a.N = f.N;
  a.sz0 = f.sz0;
  a.sigma_in = f.sigma_in;
  a.sigma_out = f.sigma_out;
  a.uniforms = f.uniforms;
  a.seed = f.seed;
  a.step = f.step;
  a.b0 = f.b0;
  a.step_dev = f.step_dev;
  a.logpsi = f.logpsi;
  a.hcache = f.hcache;
  a.colbuf = f.colbuf;
  a.lp_tab = f.lp_tab;
  a.nup_tab = f.nup_tab;
  a.hdr = f.hdr;
  const uint8_t* w1 = wimg;
  const uint8_t* w2 = w1 + (size_t)3 * D * (2 * D + 16) * 2;
  const float* aux = reinterpret_cast<const float*>(w2 + (size_t)2 * D * (D + 16) * 2);
  switch (D) {
    case 32: return sample ? launch2<32, 0>(a, w1, w2, aux, st) : launch2<32, 1>(a, w1, w2, aux, st);
    case 64: return sample ? launch2_fwd64<0>(a, w1, w2, aux, st) : launch2_fwd64<1>(a, w1, w2, aux, st);
  }
  return cudaErrorInvalidValue;
}

template <int D>
cudaError_t launch_tables(const Tab2Args& a, const uint8_t* w2, const float* aux, cudaStream_t st) {
  auto k = tc2d_tables_kernel<D>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, T2S<D>::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  // three CTAs per SM (60 KB of shared memory, 128 TMEM columns each at d_h
  // 64), so that one tile's loads and MMA overlap the others' epilogues
  const int64_t ntile = (a.B * a.N + 127) / 128;
  const int64_t grid = ntile < 3 * sm_count_2d() ? ntile : 3 * sm_count_2d();
  if (grid < 1) return cudaSuccess;
  k<<<(unsigned)grid, 128, T2S<D>::kBytes, st>>>(w2, aux, a);
  return cudaGetLastError();
}

cudaError_t tc2d_tables(const Tc2Fwd& f, const uint8_t* wimg, int D, cudaStream_t st) {
  if (D == 256) return tc2dw_tables(f, wimg, st);
  Tab2Args a{};
  a.B = f.B;
  a.Lx = f.Lx;
  a.N = f.N;
  a.sz0 = f.sz0;
  a.sigma = f.sigma_in;
  a.hcache = f.hcache;
  a.lp_tab = f.lp_tab;
  a.nup_tab = f.nup_tab;
  a.hdr = f.hdr;
  const uint8_t* w2 = wimg + (size_t)3 * D * (2 * D + 16) * 2;
  const float* aux = reinterpret_cast<const float*>(w2 + (size_t)2 * D * (D + 16) * 2);
  switch (D) {
    case 32: return launch_tables<32>(a, w2, aux, st);
    case 64: return launch_tables<64>(a, w2, aux, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tc2d_heis_chains(const Tc2Chains& c, const uint8_t* wimg, int D, cudaStream_t st) {
  // jobs: antiparallel (sample, bond) pairs in bond order, with their start values
  uint8_t* jb = c.jobs_ws;
  const bool wide = wide_jobs(c.N, D);
  const size_t rec = wide ? sizeof(JobT<4>) : sizeof(JobT<2>);
  int* counts = reinterpret_cast<int*>(jb + (size_t)c.B * c.nb * rec);
  int* njobs = counts + c.nb;
  uint64_t* masks = reinterpret_cast<uint64_t*>(jb + jobs_masks_offset(c.B, c.nb, c.N, D));
  heis_count_kernel<<<c.nb, 256, 0, st>>>(c.sigma, c.bonds, c.B, c.N, counts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned mblocks = (unsigned)((c.B + 255) / 256);
  if (!wide) {
    if (mblocks) heis_masks_kernel<2><<<mblocks, 256, 0, st>>>(c.sigma, c.B, c.N, masks);
    heis_jobs_kernel<2><<<c.nb, 1024, 0, st>>>(c.sigma, c.bonds, c.lp_tab, c.nup_tab, counts, masks, c.B, c.N, c.nb,
                                                reinterpret_cast<JobT<2>*>(jb), njobs);
  } else {
    if (mblocks) heis_masks_kernel<4><<<mblocks, 256, 0, st>>>(c.sigma, c.B, c.N, masks);
    heis_jobs_kernel<4><<<c.nb, 1024, 0, st>>>(c.sigma, c.bonds, c.lp_tab, c.nup_tab, counts, masks, c.B, c.N, c.nb,
                                                reinterpret_cast<JobT<4>*>(jb), njobs);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c.counter, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
  if (D == 256) return tc2dw_chains(c, wimg, jb, njobs, st);
  const void* jobs = jb;
  Tc2Args a{};
  a.B = c.B;
  a.Lx = c.Lx;
  a.N = c.N;
  a.nb = c.nb;
  a.sz0 = c.sz0;
  a.hcache = const_cast<float*>(c.hcache);
  a.colbuf = c.colbuf;
  a.lp_tab = const_cast<float*>(c.lp_tab);
  a.bonds = c.bonds;
  a.jobs = jobs;
  a.njobs = njobs;
  a.delta = c.delta;
  a.counter = c.counter;
  a.hdr = c.hdr;
  const uint8_t* w1 = wimg;
  const uint8_t* w2 = w1 + (size_t)3 * D * (2 * D + 16) * 2;
  const float* aux = reinterpret_cast<const float*>(w2 + (size_t)2 * D * (D + 16) * 2);
  // default: two 128-row tiles per CTA with one thread per row (measured at 8
  // x 8, d_h = 64, B = 2048: local energy 0.945 ms, against 1.036 ms with two
  // threads per row, whose extra barriers outweigh the halved epilogues, and
  // 1.29 ms on one tile).  Pinned tile variants: 0 the one-tile engine with
  // one thread per row, 1 the one-tile engine with 16 units per thread (2
  // threads per row at d_h = 32, 4 at 64), 2 two tiles with one thread per
  // row, 3 two tiles with two.  All give bitwise the same energies.
  const int pin = tc1d_pinned_variant();
  switch (D) {
    case 32:
      if (pin < 0 || pin == 2) return launch_chain2<32, 1>(a, w1, w2, aux, st);
      if (pin == 3) return launch_chain2<32, 2>(a, w1, w2, aux, st);
      return pin >= 1 ? launch2<32, 2, 1, 2>(a, w1, w2, aux, st) : launch2<32, 2>(a, w1, w2, aux, st);
    case 64:
      if (pin < 0 || pin == 2) return launch_chain2<64, 1>(a, w1, w2, aux, st);
      if (pin == 3) return launch_chain2<64, 2>(a, w1, w2, aux, st);
      return pin >= 1 ? launch2<64, 2, 1, 4>(a, w1, w2, aux, st) : launch2<64, 2>(a, w1, w2, aux, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace nqs

namespace nqs {
cudaError_t tc2d_set_wait_polls(uint32_t polls) { return cudaMemcpyToSymbol(tc::g_wait_polls, &polls, sizeof(polls)); }
}  // namespace nqs

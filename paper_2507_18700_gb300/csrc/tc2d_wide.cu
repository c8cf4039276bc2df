// BF16 tensor-core path of the 2D GRU + GLU wave function (App. A) at d_h =
// 256: zig-zag sampling, teacher forcing, the cached-path tables and the
// prefix-cached Heisenberg chains (Eq. heisenberg, Marshall-rotated, Sec.
// III B) on lattices of up to 256 sites (the 16 x 16 lattice of Sec. III B).
//
// The cell arithmetic is that of tc2d.cu: states enter the GEMMs as BF16
// pairs hi + lo, the weights are BF16 with the biases and one-hot input
// weights folded into 16 extra columns, accumulation is FP32, and the
// epilogues and the readout order are the same.  What changes is the size:
// the weights (1.09 MB of BF16) do not fit in shared memory, and the 3 d_h =
// 768 gate accumulators of a 128-row tile do not fit in TMEM (512 columns).
//
//  * Weights stream from global memory (L2-resident: every CTA reads the same
//    1.09 MB) as a fixed sequence of "slabs": 16 K columns of all B rows of
//    one MMA phase (12 or 16 KB, already in the K-major core-matrix layout).
//    One issuing thread copies slabs with bulk asynchronous copies into a
//    five-slot ring in shared memory and runs ahead of its MMAs across phase
//    and cell boundaries (the sequence does not depend on the data); slot
//    reuse waits on the commit of the MMAs that read the slot.
//  * The gates run in two chunks of 128 units (N = 384: the W, W_g / 2 and
//    U_mix rows of those units, accumulators in TMEM columns [0, 384)), each
//    over the horizontal and the vertical input.  The A operand (128 rows x
//    [hi(h) | extras | lo(h)], 135 KB) holds one input state at a time:
//        h_hor: chunk 0 | h_ver: chunk 0, chunk 1 | h_hor: chunk 1 | h: GLU
//    so a cell stages its vertical input once and its horizontal input
//    twice, and the state it computes (chunk 0 kept in registers until the
//    A operand is free) is the GLU's input and, in place, the next cell's
//    horizontal input.  The GLU (N = 512) then fills all of TMEM.
//  * 16 worker warps, four per TMEM lane quarter, hold a row each in four
//    slices (32 units of each gate chunk, 64 GLU units); they stage the
//    inputs, run the epilogues and the row logic.  Warp 16 issues the copies
//    and the MMAs and meets the workers at named barriers.
// States leave the cell as packed hi / lo words in a per-row column buffer
// (the latest state of each lattice column) and, in sampling / teacher
// forcing, as FP32 in the prefix cache.
#include <cuda_fp16.h>

#include "tc2d_common.cuh"
#include "tc_wgrad.cuh"

namespace nqs {

namespace {

using namespace tc2dh;
using namespace tcw;

constexpr int WD = 256;                            // d_h
constexpr int WKA = 2 * WD + 16;                   // A operand columns: [hi(h) | extras | lo(h)]
constexpr int WEX = WD;                            // first extra column
constexpr int WLO = WD + 16;                       // first lo column
constexpr uint32_t kSboA = (WKA / 8) * 128;        // A: bytes between 8-row groups
constexpr int kGateRows = 384, kGluRows = 512;     // B rows of a gate / GLU slab
constexpr uint32_t kGateSlab = kGateRows * 32;     // 16 BF16 K columns of every B row
constexpr uint32_t kGluSlab = kGluRows * 32;
constexpr int kNHor = 17, kNVer = 16, kNGlu = 17;  // slabs per phase (horizontal and GLU: + the extras slab)
constexpr int kGateSlabs = 2 * kNHor + 2 * kNVer;  // 66
constexpr int kCellSlabs = kGateSlabs + kNGlu;     // 83
constexpr size_t kOffGlu = (size_t)kGateSlabs * kGateSlab;
constexpr size_t kOffAux = kOffGlu + (size_t)kNGlu * kGluSlab;
// backward image: the sweep's transposed gate weights (48 slabs of [512 h'
// columns x 16 gate units]) and the GLU's transposed weights (32 slabs of
// [256 h units x 16 GLU units]), true (not halved) W_g and W_2
constexpr uint32_t kW1tSlab = 512 * 32, kGlutSlab = 256 * 32;
constexpr int kNW1t = 48, kNGlut = 32;
constexpr size_t kOffGlut = (size_t)kNW1t * kW1tSlab;
constexpr size_t kBwdImg = kOffGlut + (size_t)kNGlut * kGlutSlab;
constexpr int kTapeSlabs = kCellSlabs + kNGlut;    // 115 slabs per tape-pass tile
constexpr int kRing = 5;                           // ring slots
constexpr uint32_t kSlotBytes = 16384;
constexpr int kWorkers = 512;
constexpr int kSync = kWorkers + 32;               // threads at the named barriers: workers + issuer warp
constexpr int kThreads = kWorkers + 64;            // + the producer warp (copies only)
constexpr uint32_t kBarAll = 1, kBarGo = 2, kBarW = 3;   // named barriers
constexpr uint32_t kIdesc256 = tc::make_idesc_bf16(128, 256);
constexpr uint32_t kIdesc128 = tc::make_idesc_bf16(128, 128);
static_assert(kGluSlab <= kSlotBytes && kGateSlab <= kSlotBytes, "slab fits a slot");

// ----------------------------------------------------------------------------
// Weight image: the slabs of one cell in the order the MMAs use them, then the
// FP32 readout constants.  Slab q (element (n, k) at kmajor_offset(n, k, 16)):
//   [0, 17)   chunk 0 (units 0-127) on h_hor: W columns [16 q, 16 q + 16), then the extras
//   [17, 33)  chunk 0 on h_ver
//   [33, 49)  chunk 1 (units 128-255) on h_ver
//   [49, 66)  chunk 1 on h_hor, then the extras
//   [66, 83)  GLU: W_1 / W_2 columns, then the extras
// Gate slab rows: [W | W_g / 2 | U_mix] rows of the chunk's 128 units; extra
// columns [b hi | b lo | w_h0 w_h1 w_v0 w_v1 hi | the same lo] (W, W_g rows; U_mix
// rows have none).  GLU slab rows: [W_1 | W_2 / 2], extras [b hi | b lo].
// ----------------------------------------------------------------------------
__global__ void pack_wide_kernel(const float* __restrict__ p, uint8_t* __restrict__ img) {
  constexpr int D = WD, W2c = 2 * D + 4;
  // flat layout (App. A; nqs.h): W, W_g [d, 2d+4], U_mix [d, 2d], b, b_g, W_1 [d, d], b_1, W_2, b_2, U_out [2, d], c
  const int oW = 0, oWg = D * W2c, oU = 2 * D * W2c, ob = oU + 2 * D * D, obg = ob + D, oW1 = obg + D, ob1 = oW1 + D * D,
            oW2 = ob1 + D, ob2 = oW2 + D * D, oUo = ob2 + D, oc = oUo + 2 * D;
  const int ng = kGateSlabs * kGateRows * 16, nl = kNGlu * kGluRows * 16;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ng + nl + D + 1; t += gridDim.x * blockDim.x) {
    if (t < ng) {
      const int q = t / (kGateRows * 16), e = t % (kGateRows * 16), n = e / 16, k = e % 16;
      const int chunk = q < 33 ? 0 : 1;
      const bool ver = q >= 17 && q < 49;
      const int kk = q < 17 ? q : q < 33 ? q - 17 : q < 49 ? q - 33 : q - 49;
      const int g = n / 128, u = chunk * 128 + n % 128;
      float v = 0.0f;
      if (kk < 16) {
        const int col = (ver ? D : 0) + 16 * kk + k;
        v = g == 0 ? p[oW + u * W2c + col] : g == 1 ? p[oWg + u * W2c + col] : p[oU + u * 2 * D + col];
      } else if (g < 2 && k < 10) {
        const int Wo = g == 0 ? oW : oWg;
        const float x = k < 2 ? p[(g == 0 ? ob : obg) + u] : p[Wo + u * W2c + 2 * D + (k < 6 ? k - 2 : k - 6)];
        v = (k == 0 || (k >= 2 && k < 6)) ? bf16_round(x) : x - bf16_round(x);
      }
      if (g == 1) v *= 0.5f;   // u = (1 + tanh(a_g / 2)) / 2
      *reinterpret_cast<__nv_bfloat16*>(img + (size_t)q * kGateSlab + tc::kmajor_offset(n, k, 16)) = __float2bfloat16_rn(v);
    } else if (t < ng + nl) {
      const int r = t - ng, q = r / (kGluRows * 16), e = r % (kGluRows * 16), n = e / 16, k = e % 16;
      const int g = n / 256, v = n % 256;
      float x = 0.0f;
      if (q < 16) {
        x = p[(g == 0 ? oW1 : oW2) + v * D + 16 * q + k];
      } else if (k < 2) {
        const float bb = p[(g == 0 ? ob1 : ob2) + v];
        x = k == 0 ? bf16_round(bb) : bb - bf16_round(bb);
      }
      if (g == 1) x *= 0.5f;   // sigmoid(a) = (1 + tanh(a / 2)) / 2
      *reinterpret_cast<__nv_bfloat16*>(img + kOffGlu + (size_t)q * kGluSlab + tc::kmajor_offset(n, k, 16)) =
          __float2bfloat16_rn(x);
    } else {
      const int v = t - ng - nl;
      float* aux = reinterpret_cast<float*>(img + kOffAux);
      aux[v] = v < D ? p[oUo + v] - p[oUo + D + v] : p[oc] - p[oc + 1];
    }
  }
}

// up spins before every zig-zag position (the tables' n_up), one thread per sample
__global__ void nup_prefix_kernel(const uint8_t* __restrict__ sigma, int64_t B, int Lx, int N, int* __restrict__ nup) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int n = 0;
  for (int t = 0; t < N; ++t) {
    nup[b * N + t] = n;
    const Pz p = zpos(t, Lx);
    n += sigma[b * N + p.j * Lx + p.i] ? 0 : 1;
  }
}

struct SW {
  static constexpr uint32_t kA = 0;                                  // [128 x WKA] bf16
  static constexpr uint32_t kRingOff = kA + 128 * WKA * 2;           // kRing x 16 KB
  static constexpr uint32_t kAux = kRingOff + kRing * kSlotBytes;    // WD + 4 floats: U_0 - U_1, c_0 - c_1
  static constexpr uint32_t kPos = kAux + (WD + 4) * 4;              // 256 ints: (i, j, r) of every position
  static constexpr uint32_t kZx = kPos + 256 * 4;                    // 4 x 128 floats: readout partials
  static constexpr uint32_t kJob = kZx + 512 * 4;                    // 128 long long: published chain jobs
  static constexpr uint32_t kBar = kJob + 128 * 8;                   // full[kRing], empty[kRing], done, drain
  static constexpr uint32_t kMisc = kBar + (2 * kRing + 2) * 8;      // TMEM slot, abort flag
  static constexpr uint32_t kBytes = 1024 + kMisc + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
};

// The producer warp's loop (lane 0): copy slab s into ring slot s % kRing as
// soon as the MMAs that read the slot's previous slab have committed to
// empty[slot], running up to kRing slabs ahead of the issuer, until the
// issuer raises *stop; then wait for the copies issued beyond the issuer's
// last consumed slab (*cons), so that none lands after the CTA has exited.
// src(s, ptr, bytes) names slab s of the kernel's sequence.
template <typename Src>
__device__ void produce_slabs(uint8_t* ring, uint64_t* full, uint64_t* empty, volatile int* stop,
                              volatile uint32_t* cons, volatile int* abort_flag, WsHeader* hdr, uint32_t wlim,
                              bool& timed_out, Src src) {
  uint32_t s = 0;
  for (;; ++s) {
    const uint32_t slot = s % kRing;
    if (s >= (uint32_t)kRing) {
      const uint32_t par = ((s / kRing) - 1) & 1;
      bool got = false;
      for (uint32_t it = 0; it < wlim; ++it) {
        if (tc::mbar_wait(&empty[slot], par, 1)) {
          got = true;
          break;
        }
        if (*stop) break;
      }
      if (!got) {
        if (!*stop) {
          timed_out = true;
          *abort_flag = 1;
          flag_status(hdr, NQS_ETIMEOUT);
        }
        break;
      }
    }
    if (*stop) break;
    const uint8_t* ptr;
    uint32_t bytes;
    src(s, ptr, bytes);
    mbar_expect_tx(&full[slot], bytes);
    bulk_g2s(ring + slot * kSlotBytes, ptr, bytes, &full[slot]);
  }
  // the issuer publishes its count before it raises *stop (bounded wait:
  // after a timeout here the issuer still finishes its loop)
  for (uint32_t it = 0; it < (1u << 22) && !*stop; ++it) __nanosleep(1000);
  const uint32_t c0 = *cons;
  for (uint32_t q = c0; q < s; ++q) tc::mbar_wait(&full[q % kRing], (q / kRing) & 1, tc::kDefaultWaitPolls);
}

struct WArgs {
  int64_t B;
  int Lx, N, nb, sz0;
  const uint8_t* sigma_in;
  uint8_t* sigma_out;
  const float* uniforms;
  uint64_t seed, step;
  uint64_t b0;               // sampling: global index of sample 0 (Philox counter offset)
  const uint64_t* step_dev;  // sampling: device Philox step or null
  float* logpsi;             // nullable in teacher forcing
  float* hcache;             // written by sampling / teacher forcing (nullable); read by tables and chains
  float* colbuf;             // [CTAs x 128 rows, Lx, d] latest packed hi / lo state of every lattice column
  float* lp_tab;             // written by the tables, read by the chains
  const int* nup_tab;
  const int4* bonds;
  const JobT<4>* jobs;
  const int* njobs;
  float* delta;
  unsigned long long* counter;
  WsHeader* hdr;
  // tape pass of the reverse sweep (MODE 4) over positions [t0, t1); cells
  // c = (t - t0) * Bp + b
  int t0, t1;
  const uint8_t* img2;       // backward image (its GLU slabs)
  const float* wts;          // [B] per-sample weights w_b of sum_b w_b log psi_b
  int64_t Bp;                // B rounded up to a whole tile of 128
  __half* tape_f;            // [cells, 3, D] FP16 factors u (1 - h~^2), (h~ - U_mix h') u (1 - u), 1 - u
  float* tape_dh;            // [cells, D] dh_glu
  uint8_t* x1a;              // operand tapes (tape_off layout): h_hor, h_ver, [1 | one-hots] ...
  uint8_t* x1b;
  uint8_t* x1c;
  uint8_t* g2;               // ... [dy_1 | dy_2] (GLU pre-activation gradients), [h], [1]
  uint8_t* x2a;
  uint8_t* x2c;
  __nv_bfloat16* ytape;      // [cells, D] GLU outputs
  float* gd;                 // [cells] d(sum w log psi) / d(logit difference)
};

// MODE 0: sampling, 1: teacher forcing, 2: Heisenberg chains, 3: cached-path
// tables, 4: tape pass of the reverse sweep (every (sample, position) cell in
// parallel: gate factors, GLU backward, weight-gradient operands).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) tc2dw_kernel(const uint8_t* __restrict__ img, WArgs a) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sA = sm + SW::kA;
  uint8_t* ring = sm + SW::kRingOff;
  float* sAux = reinterpret_cast<float*>(sm + SW::kAux);
  int* sPos = reinterpret_cast<int*>(sm + SW::kPos);
  float* sZx = reinterpret_cast<float*>(sm + SW::kZx);
  long long* jbuf = reinterpret_cast<long long*>(sm + SW::kJob);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + SW::kBar);
  uint64_t* empty = full + kRing;
  uint64_t* done = empty + kRing;
  uint64_t* drain = done + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + SW::kMisc);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + SW::kMisc + 4);
  volatile int* s_stop = reinterpret_cast<volatile int*>(sm + SW::kMisc + 8);          // issuer done
  volatile uint32_t* s_consf = reinterpret_cast<volatile uint32_t*>(sm + SW::kMisc + 12);   // its slab count

  const float* aux = reinterpret_cast<const float*>(img + kOffAux);
  for (int i = threadIdx.x; i < WD + 1; i += kThreads) sAux[i] = aux[i];
  for (int t = threadIdx.x; t < a.N; t += kThreads) {
    const Pz p = zpos(t, a.Lx);
    sPos[t] = p.i | (p.j << 8) | (p.r << 16);
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < kRing; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(drain, 1);
    *s_abort = 0;
    *s_stop = 0;
    *s_consf = 0;
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool timed_out = false;

  if (warp == kWorkers / 32 + 1) {
    // ======================== producer warp ========================
    if (lane == 0)
      produce_slabs(ring, full, empty, s_stop, s_consf, s_abort, a.hdr, wlim, timed_out,
                    [&](uint32_t s, const uint8_t*& src, uint32_t& bytes) {
                      if constexpr (MODE == 3) {
                        src = img + kOffGlu + (size_t)(s % kNGlu) * kGluSlab;
                        bytes = kGluSlab;
                      } else {
                        if (MODE == 4 && s % kTapeSlabs >= (uint32_t)kCellSlabs) {
                          src = a.img2 + kOffGlut + (size_t)(s % kTapeSlabs - kCellSlabs) * kGlutSlab;
                          bytes = kGlutSlab;
                          return;
                        }
                        const uint32_t q = s % (MODE == 4 ? kTapeSlabs : kCellSlabs);
                        src = q < (uint32_t)kGateSlabs ? img + (size_t)q * kGateSlab
                                                       : img + kOffGlu + (size_t)(q - kGateSlabs) * kGluSlab;
                        bytes = q < (uint32_t)kGateSlabs ? kGateSlab : kGluSlab;
                      }
                    });
    __syncwarp();
  } else if (warp == kWorkers / 32) {
    // ======================== issuer warp ========================
    const bool leader = lane == 0;
    const uint32_t a_addr = tc::smem_addr(sA), r_addr = tc::smem_addr(ring);
    uint32_t s_cons = 0;               // slabs consumed by MMAs (leader)
    bool dead = false;                 // a wait gave up: no more MMAs
    auto die = [&]() {
      dead = true;
      timed_out = true;
      *s_abort = 1;
      flag_status(a.hdr, NQS_ETIMEOUT);
    };
    // one slab: wait for its copy, issue its MMAs, release the slot to the producer
    auto consume = [&](auto&& mmas) {
      if (dead) return;
      const uint32_t s = s_cons, slot = s % kRing;
      if (!tc::mbar_wait(&full[slot], (s / kRing) & 1, wlim)) {
        die();
        return;
      }
      tc::fence_after_sync();
      mmas(r_addr + slot * kSlotBytes);
      tc::mma_commit(&empty[slot]);
      ++s_cons;
    };
    // end of a phase: its completion to the workers
    auto end_phase = [&]() { tc::mma_commit(done); };
    auto desc_a = [&](int col) { return tc::make_desc(a_addr + (uint32_t)col * 16, 128, kSboA); };
    // gate slab: rows [0, 256) -> TMEM [0, 256), rows [256, 384) -> [256, 384)
    auto mma_gate = [&](uint32_t sa, int col, bool lo, uint32_t accf) {
      const uint64_t b0 = tc::make_desc(sa, 128, 256), b1 = tc::make_desc(sa + 8192, 128, 256);
      tc::mma_bf16(tbase, desc_a(col), b0, kIdesc256, accf);
      tc::mma_bf16(tbase + 256, desc_a(col), b1, kIdesc128, accf);
      if (lo) {
        tc::mma_bf16(tbase, desc_a(WLO + col), b0, kIdesc256, 1);
        tc::mma_bf16(tbase + 256, desc_a(WLO + col), b1, kIdesc128, 1);
      }
    };
    // GLU slab: rows [0, 256) -> TMEM [0, 256), rows [256, 512) -> [256, 512)
    auto mma_glu = [&](uint32_t sa, int col, bool lo, uint32_t accf) {
      const uint64_t b0 = tc::make_desc(sa, 128, 256), b1 = tc::make_desc(sa + 8192, 128, 256);
      tc::mma_bf16(tbase, desc_a(col), b0, kIdesc256, accf);
      tc::mma_bf16(tbase + 256, desc_a(col), b1, kIdesc256, accf);
      if (lo) {
        tc::mma_bf16(tbase, desc_a(WLO + col), b0, kIdesc256, 1);
        tc::mma_bf16(tbase + 256, desc_a(WLO + col), b1, kIdesc256, 1);
      }
    };
    auto phase_hor = [&](bool first) {   // 16 slabs on hi / lo, then the extras
      for (int i = 0; i < kNHor; ++i)
        consume([&](uint32_t sa) {
          if (i < 16) mma_gate(sa, 16 * i, true, (first && i == 0) ? 0u : 1u);
          else mma_gate(sa, WEX, false, 1u);
        });
      end_phase();
    };
    auto phase_ver = [&](bool first) {
      for (int i = 0; i < kNVer; ++i)
        consume([&](uint32_t sa) { mma_gate(sa, 16 * i, true, (first && i == 0) ? 0u : 1u); });
      end_phase();
    };
    auto phase_glu = [&]() {
      for (int i = 0; i < kNGlu; ++i)
        consume([&](uint32_t sa) {
          if (i < 16) mma_glu(sa, 16 * i, true, i == 0 ? 0u : 1u);
          else mma_glu(sa, WEX, false, 1u);
        });
      end_phase();
    };
    // GLU backward (tape pass): dh_glu = [dy_1 | dy_2] [W_1 ; W_2] over A
    // columns [0, 512) (single BF16), N = 256 -> TMEM [0, 256)
    auto phase_glub = [&]() {
      for (int i = 0; i < kNGlut; ++i)
        consume([&](uint32_t sa) {
          tc::mma_bf16(tbase, desc_a(16 * i), tc::make_desc(sa, 128, 256), kIdesc256, i == 0 ? 0u : 1u);
        });
      end_phase();
    };
    auto go = [&]() {                  // the workers' inputs / TMEM reads are done
      __syncwarp();
      tc::group_barrier(kBarGo, kSync);
      tc::fence_after_sync();
    };
    for (;;) {
      const bool any = tc::group_barrier_or(false, kBarAll, kSync);
      if (!any) break;
      tc::fence_after_sync();
      if constexpr (MODE == 3) {
        if (leader) phase_glu();
      } else {
        if (leader) phase_hor(true);    // chunk 0, h_hor
        go();
        if (leader) phase_ver(false);   // chunk 0, h_ver
        go();
        if (leader) phase_ver(true);    // chunk 1, h_ver
        go();
        if (leader) phase_hor(false);   // chunk 1, h_hor
        go();
        if (leader) phase_glu();
        if constexpr (MODE == 4) {
          go();
          if (leader) phase_glub();
        }
      }
      __syncwarp();
    }
    // the producer waits for its copies past this count, then exits
    if (leader) {
      *s_consf = s_cons;
      __threadfence_block();
      *s_stop = 1;
    }
    __syncwarp();
  } else {
    // ======================== worker warps ========================
    const int part = warp >> 2, quarter = warp & 3;
    const int m = quarter * 32 + lane;                                  // row = TMEM lane
    const uint32_t trow = tbase + ((uint32_t)(quarter * 32) << 16);
    const int Lx = a.Lx, N = a.N;
    const int64_t B = a.B;
    const float dc = sAux[WD];
    const uint32_t one = 0x3F80u;
    auto P = [&](int t) -> Pz {        // zig-zag position t (table lookup)
      const int v = sPos[t];
      Pz p;
      p.i = v & 255;
      p.j = (v >> 8) & 255;
      p.r = v >> 16;
      return p;
    };
    auto kmo = [&](int k) { return sA + tc::kmajor_offset(m, k, WKA); };
    // this thread's units: gate chunk c -> 128 c + 32 part + [0, 32); GLU -> 64 part + [0, 64)
    auto stage_zero = [&]() {
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = 128 * c + 32 * part + 8 * q;
          *reinterpret_cast<uint4*>(kmo(u)) = make_uint4(0u, 0u, 0u, 0u);
          *reinterpret_cast<uint4*>(kmo(WLO + u)) = make_uint4(0u, 0u, 0u, 0u);
        }
    };
    auto stage_f32 = [&](const float* src) {   // FP32 state (the prefix cache)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = 128 * c + 32 * part + 8 * q;
          const float4 x0 = *reinterpret_cast<const float4*>(src + u);
          const float4 x1 = *reinterpret_cast<const float4*>(src + u + 4);
          const float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
          st_split8(kmo(u), kmo(WLO + u), v);
        }
    };
    auto stage_packed = [&](const float* entry) {   // packed [hi words | lo words] column-buffer entry
      const uint8_t* e = reinterpret_cast<const uint8_t*>(entry);
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = 128 * c + 32 * part + 8 * q;
          cp_async16_cg(kmo(u), e + 2 * u);
          cp_async16_cg(kmo(WLO + u), e + 2 * WD + 2 * u);
        }
      cp_commit_2d();
    };
    auto glu_extras = [&]() {
      *reinterpret_cast<uint4*>(kmo(WEX)) = make_uint4(one | (one << 16), 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(kmo(WEX + 8)) = make_uint4(0u, 0u, 0u, 0u);
    };
    // GLU epilogue and readout: 16-unit chunks in order, chunks by a fixed
    // pairwise tree (within the slice, then over the four slices)
    // (yout: this slice's 64 GLU outputs as BF16, the tape pass)
    auto glu_readout = [&](__nv_bfloat16* yout) -> float {
      float zc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8) {
        uint32_t a1[8], a2[8];
        const int col = 64 * part + 8 * c8;
        tld8(trow + col, a1);
        tld8(trow + 256 + col, a2);
        tc::tmem_wait_ld();
        tie(a1);
        tie(a2);
        float y[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          y[q] = __uint_as_float(a1[q]) * fmaf(0.5f, hw_tanh2(__uint_as_float(a2[q])), 0.5f);
          zc[c8 >> 1] = fmaf(sAux[col + q], y[q], zc[c8 >> 1]);
        }
        if (yout) *reinterpret_cast<uint4*>(yout + col) = pack8_bf16(y);
      }
      sZx[part * 128 + m] = (zc[0] + zc[1]) + (zc[2] + zc[3]);
      tc::fence_before_sync();
      tc::group_barrier(kBarW, kWorkers);
      return (sZx[m] + sZx[128 + m]) + (sZx[256 + m] + sZx[384 + m]);
    };
    uint32_t pd = 0;                   // parity of the next completion on `done`
    auto wait_done = [&]() {
      if (!tc::mbar_wait(done, pd, wlim)) {
        timed_out = true;
        *s_abort = 1;
        flag_status(a.hdr, NQS_ETIMEOUT);
      }
      pd ^= 1;
      tc::fence_after_sync();
    };
    auto to_issuer = [&]() {           // inputs staged / TMEM read: the next phase may start
      cp_wait_2d();
      tc::fence_async_smem();
      tc::fence_before_sync();
      tc::group_arrive(kBarGo, kSync);
    };

    if constexpr (MODE == 4) {
      // ---- tape pass of the reverse sweep: tiles of 128 samples at one position ----
      const int nbt = (int)(a.Bp / 128), npos = a.t1 - a.t0;
      const int64_t ntile = (int64_t)npos * nbt, nkb = a.Bp * npos / 16;
      // an FP32 state (null: zeros) into the A operand and, if xt, its BF16
      // rounding into an operand tape of width 256
      auto stage_x = [&](const float* src, uint8_t* xt, int64_t cell) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int u = 128 * c + 32 * part + 8 * q;
            float v[8];
            if (src) {
              const float4 x0 = *reinterpret_cast<const float4*>(src + u);
              const float4 x1 = *reinterpret_cast<const float4*>(src + u + 4);
              v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
              v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
            } else {
#pragma unroll
              for (int e = 0; e < 8; ++e) v[e] = 0.0f;
            }
            st_split8(kmo(u), kmo(WLO + u), v);
            if (xt) *reinterpret_cast<uint4*>(xt + tape_off(cell, u, 256, nkb)) = pack8_bf16(v);
          }
      };
      // chunk c's factors of the cell backward through h = u h~ + (1 - u) U_mix h':
      // dh [u (1 - h~^2) | (h~ - U_mix h') u (1 - u) | 1 - u] are the
      // gradients of the three pre-activation blocks
      auto factors = [&](int c, int64_t cell) {
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          uint32_t aw[8], ag[8], au[8];
          const int col = 32 * part + 8 * q4;
          tld8(trow + col, aw);
          tld8(trow + 128 + col, ag);
          tld8(trow + 256 + col, au);
          tc::tmem_wait_ld();
          tie(aw);
          tie(ag);
          tie(au);
          __half2 f1[4], f2[4], f3[4];
#pragma unroll
          for (int q = 0; q < 8; q += 2) {
            float g1[2], g2[2], g3[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float cc = hw_tanh2(__uint_as_float(aw[q + e]));
              const float ug = fmaf(0.5f, hw_tanh2(__uint_as_float(ag[q + e])), 0.5f);
              const float mix = __uint_as_float(au[q + e]);
              g1[e] = ug * (1.0f - cc * cc);
              g2[e] = (cc - mix) * ug * (1.0f - ug);
              g3[e] = 1.0f - ug;
            }
            f1[q / 2] = __floats2half2_rn(g1[0], g1[1]);
            f2[q / 2] = __floats2half2_rn(g2[0], g2[1]);
            f3[q / 2] = __floats2half2_rn(g3[0], g3[1]);
          }
          __half* dst = a.tape_f + cell * (3 * WD) + 128 * c + col;
          *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(f1);
          *reinterpret_cast<uint4*>(dst + WD) = *reinterpret_cast<const uint4*>(f2);
          *reinterpret_cast<uint4*>(dst + 2 * WD) = *reinterpret_cast<const uint4*>(f3);
        }
      };
      for (int64_t tile = blockIdx.x;; tile += gridDim.x) {
        const bool has = tile < ntile;                  // the same for every row of the CTA
        const int t = has ? a.t0 + (int)(tile / nbt) : a.t0;
        const int64_t b = has ? (tile % nbt) * 128 + m : 0;
        const bool valid = has && b < B;                // rows past B: zeros in, zeros out
        const int64_t cell = (int64_t)(t - a.t0) * a.Bp + b;
        const Pz p = P(t);
        const float* src_h = valid && p.r > 0 ? a.hcache + (b * N + p.j * Lx + zhor(p)) * WD : nullptr;
        const float* src_v = valid && p.j > 0 ? a.hcache + (b * N + (p.j - 1) * Lx + p.i) * WD : nullptr;
        const float* src_c = valid ? a.hcache + (b * N + p.j * Lx + p.i) * WD : nullptr;
        if (has) {
          stage_x(src_h, a.x1a, cell);
          if (part == 0) {
            const int s_h = valid && p.r > 0 ? (a.sigma_in[b * N + p.j * Lx + zhor(p)] ? 1 : 0) : -1;
            const int s_v = valid && p.j > 0 ? (a.sigma_in[b * N + (p.j - 1) * Lx + p.i] ? 1 : 0) : -1;
            const uint32_t oh = s_h < 0 ? 0u : (s_h == 0 ? one : (one << 16));
            const uint32_t ov = s_v < 0 ? 0u : (s_v == 0 ? one : (one << 16));
            *reinterpret_cast<uint4*>(kmo(WEX)) = make_uint4(one | (one << 16), oh, ov, oh);
            *reinterpret_cast<uint4*>(kmo(WEX + 8)) = make_uint4(ov, 0u, 0u, 0u);
            // the extra columns of the gate weight gradient: [1 | onehot(s_hor) | onehot(s_ver) | 0]
            const float xe[8] = {1.0f, s_h == 0 ? 1.0f : 0.0f, s_h == 1 ? 1.0f : 0.0f, s_v == 0 ? 1.0f : 0.0f,
                                 s_v == 1 ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f};
            *reinterpret_cast<uint4*>(a.x1c + tape_off(cell, 0, 16, nkb)) = pack8_bf16(xe);
            *reinterpret_cast<uint4*>(a.x1c + tape_off(cell, 8, 16, nkb)) = make_uint4(0u, 0u, 0u, 0u);
          }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (!tc::group_barrier_or(has && !*s_abort, kBarAll, kSync)) break;
        wait_done();                                    // chunk 0 on h_hor
        stage_x(src_v, a.x1b, cell);
        to_issuer();
        wait_done();                                    // chunk 0 complete
        factors(0, cell);
        to_issuer();
        wait_done();                                    // chunk 1 on h_ver
        stage_x(src_h, nullptr, cell);
        to_issuer();
        wait_done();                                    // chunk 1 complete
        factors(1, cell);
        stage_x(src_c, a.x2a, cell);                    // the cell's own state: the GLU's input
        if (part == 0) {
          glu_extras();
          const float xe[8] = {1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
          *reinterpret_cast<uint4*>(a.x2c + tape_off(cell, 0, 16, nkb)) = pack8_bf16(xe);
          *reinterpret_cast<uint4*>(a.x2c + tape_off(cell, 8, 16, nkb)) = make_uint4(0u, 0u, 0u, 0u);
        }
        to_issuer();
        wait_done();                                    // GLU
        const float z = glu_readout(a.ytape + cell * WD);
        // gradient of sum_b w_b log psi_b (log psi = 1/2 sum_t log p) with
        // respect to the logit difference d; 0 at a site the mask forces
        float gdv = 0.0f;
        if (valid && !timed_out) {
          const int s = a.sigma_in[b * N + p.j * Lx + p.i] ? 1 : 0;
          const int nu = a.nup_tab[b * N + t];
          const bool forced = a.sz0 && (nu >= (N >> 1) || t - nu >= (N >> 1));
          if (!forced) gdv = 0.5f * a.wts[b] * ((s == 0 ? 1.0f : 0.0f) - sigmoid_acc(z + dc));
        }
        if (part == 0) a.gd[cell] = gdv;
        // [dy_1 | dy_2] = dy [sigmoid(a_2) | y_1 sigmoid'(a_2)], dy = (U_0 - U_1) gdv,
        // into the A operand (single BF16) and the G2 tape
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
          uint32_t a1[8], a2[8];
          const int col = 64 * part + 8 * c8;
          tld8(trow + col, a1);
          tld8(trow + 256 + col, a2);
          tc::tmem_wait_ld();
          tie(a1);
          tie(a2);
          float d1[8], d2[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float sg = fmaf(0.5f, hw_tanh2(__uint_as_float(a2[q])), 0.5f);
            const float dy = sAux[col + q] * gdv;
            d1[q] = dy * sg;
            d2[q] = dy * __uint_as_float(a1[q]) * sg * (1.0f - sg);
          }
          const uint4 p1 = pack8_bf16(d1), p2 = pack8_bf16(d2);
          *reinterpret_cast<uint4*>(kmo(col)) = p1;
          *reinterpret_cast<uint4*>(kmo(256 + col)) = p2;
          *reinterpret_cast<uint4*>(a.g2 + tape_off(cell, col, 128, nkb)) = p1;
          *reinterpret_cast<uint4*>(a.g2 + tape_off(cell, 256 + col, 128, nkb)) = p2;
        }
        to_issuer();
        wait_done();                                    // GLU backward: dh_glu
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
          uint32_t r[8];
          const int col = 64 * part + 8 * c8;
          tld8(trow + col, r);
          tc::tmem_wait_ld();
          tie(r);
          float* dst = a.tape_dh + cell * WD + col;
          reinterpret_cast<float4*>(dst)[0] =
              make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
          reinterpret_cast<float4*>(dst)[1] =
              make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]), __uint_as_float(r[7]));
        }
        tc::fence_before_sync();
      }
    } else if constexpr (MODE == 3) {
      // ---- cached-path tables: every (sample, position) cell is a row ----
      const int64_t ncell = B * N, ntile = (ncell + 127) / 128;
      for (int64_t tile = blockIdx.x;; tile += gridDim.x) {
        const int64_t cell = tile * 128 + m;
        const bool valid = tile < ntile && cell < ncell;
        int64_t b = 0;
        int t = 0;
        if (valid) {
          b = cell / N;
          t = (int)(cell % N);
          const Pz p = P(t);
          stage_f32(a.hcache + (b * N + p.j * Lx + p.i) * WD);
          if (part == 0) glu_extras();
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        const bool any = tc::group_barrier_or(valid && !*s_abort, kBarAll, kSync);
        if (!any) break;
        wait_done();
        const float z = glu_readout(nullptr);
        if (valid && part == 0 && !timed_out) {
          const float d = z + dc;
          const int nu = a.nup_tab[b * N + t];
          a.lp_tab[(b * N + t) * 2] = lp_masked(0, d, nu, t, N, a.sz0 != 0);
          a.lp_tab[(b * N + t) * 2 + 1] = lp_masked(1, d, nu, t, N, a.sz0 != 0);
        }
      }
    } else {
      // row state
      int64_t b = 0;
      int t = 0, pa = -1, rank = 0, n_up = 0, bsa = -1, bsb = -1;
      float acc = 0.0f, lp_next = 0.0f;
      bool active = false, fresh = false;
      uint64_t mask[4] = {0ull, 0ull, 0ull, 0ull};
      int hsrc = 0, vsrc = 0;          // 0 zero, 1 previous state (A / column buffer), 2 cached FP32 state, 3 column buffer
      const int64_t slot_row = (int64_t)blockIdx.x * 128 + m;
      float* colrow = a.colbuf + slot_row * Lx * WD;   // this row's column buffer

      auto plan = [&]() {              // input sources of the cell at position t
        const Pz p = P(t);
        hsrc = p.r == 0 ? 0 : (MODE == 2 && fresh) ? 2 : 1;
        vsrc = p.j == 0 ? 0 : (MODE == 2 && zsnake(p.i, p.j - 1, Lx) <= pa) ? 2 : 3;
        if constexpr (MODE == 2) {
          const int k = p.j * Lx + p.i;
          const int so = mbit(mask, k) ^ ((k == bsa || k == bsb) ? 1 : 0);   // original spin at k
          lp_next = ldg_f32_v(a.lp_tab + (b * N + t) * 2 + so);
        }
      };
      auto stage_hor = [&](bool restage) {
        const Pz p = P(t);
        if (hsrc == 0) stage_zero();
        else if (hsrc == 2) stage_f32(a.hcache + (b * N + p.j * Lx + zhor(p)) * WD);
        else if (restage) stage_packed(colrow + zhor(p) * WD);
        // hsrc == 1 at the start of a cell: the A operand holds the previous state
      };
      auto stage_ver = [&]() {
        const Pz p = P(t);
        if (vsrc == 0) stage_zero();
        else if (vsrc == 2) stage_f32(a.hcache + (b * N + (p.j - 1) * Lx + p.i) * WD);
        else stage_packed(colrow + p.i * WD);
      };
      auto gate_extras = [&]() {
        const Pz p = P(t);
        const int s_h = p.r > 0 ? mbit(mask, p.j * Lx + zhor(p)) : -1;
        const int s_v = p.j > 0 ? mbit(mask, (p.j - 1) * Lx + p.i) : -1;
        const uint32_t oh = s_h < 0 ? 0u : (s_h == 0 ? one : (one << 16));
        const uint32_t ov = s_v < 0 ? 0u : (s_v == 0 ? one : (one << 16));
        *reinterpret_cast<uint4*>(kmo(WEX)) = make_uint4(one | (one << 16), oh, ov, oh);
        *reinterpret_cast<uint4*>(kmo(WEX + 8)) = make_uint4(ov, 0u, 0u, 0u);
      };
      // gate epilogue of chunk c: h~ = tanh(a_W), u = (1 + tanh(a_g)) / 2, h = u h~ + (1 - u) U_mix h'
      auto gate_epilogue = [&](float (&h)[32]) {
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          uint32_t aw[8], ag[8], au[8];
          const int col = 32 * part + 8 * q4;
          tld8(trow + col, aw);
          tld8(trow + 128 + col, ag);
          tld8(trow + 256 + col, au);
          tc::tmem_wait_ld();
          tie(aw);
          tie(ag);
          tie(au);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float cc = hw_tanh2(__uint_as_float(aw[q]));
            const float ug = fmaf(0.5f, hw_tanh2(__uint_as_float(ag[q])), 0.5f);
            const float mix = __uint_as_float(au[q]);
            h[8 * q4 + q] = fmaf(ug, cc - mix, mix);
          }
        }
      };
      // the state's 32 units of chunk c: packed words to the column buffer
      // (entry of lattice column i) and, forward modes, FP32 to the cache
      auto store_state = [&](int c, const float (&h)[32], const uint32_t (&hi)[16], const uint32_t (&lo)[16]) {
        const Pz p = P(t);
        const int u = 128 * c + 32 * part;
        uint8_t* e = reinterpret_cast<uint8_t*>(colrow + p.i * WD);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          *reinterpret_cast<uint4*>(e + 2 * u + 16 * q) = make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
          *reinterpret_cast<uint4*>(e + 2 * WD + 2 * u + 16 * q) =
              make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
        }
        if (MODE != 2 && a.hcache) {
          float* dst = a.hcache + (b * N + p.j * Lx + p.i) * WD + u;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
        }
      };
      auto write_a = [&](int c, const uint32_t (&hi)[16], const uint32_t (&lo)[16]) {
        const int u = 128 * c + 32 * part;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          *reinterpret_cast<uint4*>(kmo(u + 8 * q)) = make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
          *reinterpret_cast<uint4*>(kmo(WLO + u + 8 * q)) =
              make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
        }
      };

      // Chains: take job j (or go idle).
      const unsigned long long nj = MODE == 2 ? (unsigned long long)*a.njobs : 0ull;
      auto start_job = [&](unsigned long long j) {
        if (j >= nj) {
          active = false;
          return;
        }
        const JobT<4> jb = a.jobs[j];
        b = jb.b;
        rank = job_rank(jb.rank_pa_a);
        pa = job_pa(jb.rank_pa_a);
        bsa = job_site_a(jb.rank_pa_a);
        bsb = job_site_b(jb.nup_b);
        t = pa + 1;
        acc = jb.acc0;
        n_up = job_nup(jb.nup_b);
#pragma unroll
        for (int w = 0; w < 4; ++w) mask[w] = jb.mask[w];
        active = true;
        fresh = true;
        plan();
      };
      // warp-aggregated pull of one job for every lane with `need` (part 0 warps)
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

      if constexpr (MODE == 2) {
        if (part == 0) {
          pull_issue(true);
          jbuf[m] = (long long)pull_take();
        }
        tc::group_barrier(kBarW, kWorkers);
        start_job((unsigned long long)jbuf[m]);
      } else {
        b = (int64_t)blockIdx.x * 128 + m;
        active = b < B;
        if (MODE == 1 && active)
          for (int k = 0; k < N; ++k) mset(mask, k, a.sigma_in[b * N + k] ? 1 : 0);
        plan();
      }

      for (;;) {
        // ---- (a) horizontal input and extras ----
        if (active) {
          stage_hor(false);
          if (part == 0) gate_extras();
        }
        if constexpr (MODE == 2) {
          if (part == 0) pull_issue(active && !timed_out && t == N - 1);   // a row on its last cell pulls now
        }
        cp_wait_2d();
        tc::fence_async_smem();
        tc::fence_before_sync();
        const bool any = tc::group_barrier_or(active && !*s_abort, kBarAll, kSync);
        if (!any) break;
        float uni = 0.0f;
        if (MODE == 0 && active)
          uni = a.uniforms ? a.uniforms[b * N + t]
                           : sampling_uniform(a.seed, a.step_dev ? *a.step_dev : a.step, (uint32_t)(a.b0 + b), (uint32_t)t);
        // ---- (b) chunk 0 on h_hor done: stage h_ver ----
        wait_done();
        if (active) stage_ver();
        to_issuer();
        // ---- (c) chunk 0 complete: its units of the new state ----
        wait_done();
        float h[32];
        uint32_t h0hi[16], h0lo[16];
        gate_epilogue(h);
#pragma unroll
        for (int q = 0; q < 16; ++q) split_bf16(h[2 * q], h[2 * q + 1], h0hi[q], h0lo[q]);
        if (active) store_state(0, h, h0hi, h0lo);
        to_issuer();
        // ---- (d) chunk 1 on h_ver done: stage h_hor again ----
        wait_done();
        if (active) stage_hor(true);
        to_issuer();
        // ---- (e) chunk 1 complete: the new state into the A operand ----
        wait_done();
        {
          uint32_t h1hi[16], h1lo[16];
          gate_epilogue(h);
#pragma unroll
          for (int q = 0; q < 16; ++q) split_bf16(h[2 * q], h[2 * q + 1], h1hi[q], h1lo[q]);
          if (active) store_state(1, h, h1hi, h1lo);
          write_a(0, h0hi, h0lo);
          write_a(1, h1hi, h1lo);
          if (part == 0) glu_extras();
        }
        to_issuer();
        // ---- (f) GLU and the logit difference ----
        wait_done();
        const float z = glu_readout(nullptr);
        // ---- (g) row logic (every slice of a row runs it; slice 0 writes) ----
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
            if (part == 0) a.sigma_out[b * N + k] = (uint8_t)s;
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
              if (part == 0) a.delta[b * a.nb + rank] = acc;
            } else {
              const float lpsi = 0.5f * acc;
              if (a.logpsi && part == 0) a.logpsi[b] = lpsi;
              if (!isfinite(lpsi)) flag_status(a.hdr, NQS_ENONFINITE);
              active = false;
            }
          } else {
            fresh = false;
            plan();
          }
        }
        if constexpr (MODE == 2) {
          if (part == 0) jbuf[m] = (long long)pull_take();
          tc::group_barrier(kBarW, kWorkers);
          if (fin) start_job((unsigned long long)jbuf[m]);
        }
      }
    }
    cp_wait_2d();
  }
  tc::fence_before_sync();
  // after a wait that gave up, TMEM is freed only once the MMAs have drained
  if (__syncthreads_or(timed_out) && threadIdx.x == kWorkers) tc::drain_mmas(drain, kWait2);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 512);
}

template <int MODE>
cudaError_t launch_w(const WArgs& a, const uint8_t* img, int64_t grid, cudaStream_t st) {
  auto k = tc2dw_kernel<MODE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SW::kBytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  if (grid < 1) return cudaSuccess;
  k<<<(unsigned)grid, kThreads, SW::kBytes, st>>>(img, a);
  return cudaGetLastError();
}

int sm_count_w() {
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


// ----------------------------------------------------------------------------
// Reverse sweep at d_h = 256: d/dtheta sum_b w_b log psi_b (App. A cell and GLU,
// zig-zag order of Sec. II), in four passes:
//  1. tape pass (tc2dw_kernel<4>, every (sample, position) cell in parallel):
//     from the cached states the forward's gates give the three factors with
//     which the cell backward is linear in dh; the GLU forward gives y and the
//     logit difference, hence gd = d(sum w log psi)/dd = w_b (onehot_0(s) -
//     p0) / 2, dy = (U_0 - U_1) gd and [dy_1 | dy_2]; the GLU backward
//     [dy_1 | dy_2] [W_1 ; W_2] is dh_glu.  The cell's inputs h_hor, h_ver,
//     [1 | one-hots], its state h and [dy_1 | dy_2] go to the operand tapes of
//     the weight-gradient GEMMs.
//  2. sequential sweep (tc2dw_sweep_kernel, t = N-1 .. 0 for a tile of 128
//     samples): dh = dh_glu + the horizontal successor's and the vertical
//     successor's carries, G1 = dh [f1 | f2 | f3] (BF16, to the G1 tape and the
//     A operand, in six chunks of 128 gate units), dh' = G1 [W ; W_g ; U_mix]
//     (N = 512: the horizontal and the vertical predecessor's carries);
//  3. weight-gradient GEMMs (tcw::wgrad_kernel): dW1 = G1^T [h_hor | h_ver |
//     1 | one-hots] and dW2 = G2^T [h | 1] summed over every cell, split over
//     cell ranges, both operands MN-major blocks of 16 cells streamed by bulk
//     copies; dU_out and dc from gd and y (tc2dw_readout_kernel);
//  4. the final reduction into the flat gradient (tc2dw_final_kernel).
// ----------------------------------------------------------------------------

// Backward image.  W1t slab q (q = 0..47): gate block g = q / 16 (W, W_g, U_mix,
// true values), gate units 16 (q % 16) + k; element (n, k) = block[unit][n] for
// the 512 h' columns n.  GLU-t slab q (0..31): element (n, k) = W_1[16 q + k][n]
// (q < 16) or W_2[16 (q - 16) + k][n], n < 256.
__global__ void pack_wide_bwd_kernel(const float* __restrict__ p, uint8_t* __restrict__ img2) {
  constexpr int D = WD, W2c = 2 * D + 4;
  const int oW = 0, oWg = D * W2c, oU = 2 * D * W2c, ob = oU + 2 * D * D, obg = ob + D, oW1 = obg + D, ob1 = oW1 + D * D,
            oW2 = ob1 + D;
  const int n1 = kNW1t * 512 * 16, n2 = kNGlut * 256 * 16;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n1 + n2; t += gridDim.x * blockDim.x) {
    if (t < n1) {
      const int q = t / (512 * 16), e = t % (512 * 16), n = e / 16, k = e % 16;
      const int g = q / 16, u = 16 * (q % 16) + k;
      const float v = g == 0 ? p[oW + u * W2c + n] : g == 1 ? p[oWg + u * W2c + n] : p[oU + u * 2 * D + n];
      *reinterpret_cast<__nv_bfloat16*>(img2 + (size_t)q * kW1tSlab + tc::kmajor_offset(n, k, 16)) =
          __float2bfloat16_rn(v);
    } else {
      const int r = t - n1, q = r / (256 * 16), e = r % (256 * 16), n = e / 16, k = e % 16;
      const float v = q < 16 ? p[oW1 + (16 * q + k) * D + n] : p[oW2 + (16 * (q - 16) + k) * D + n];
      *reinterpret_cast<__nv_bfloat16*>(img2 + kOffGlut + (size_t)q * kGlutSlab + tc::kmajor_offset(n, k, 16)) =
          __float2bfloat16_rn(v);
    }
  }
}

struct SwArgs {
  int64_t B, Bp;
  int Lx, N;
  int t0, t1;                // positions of this launch, swept t1 - 1 down to t0; cells (t - t0) * Bp + b
  const __half* tape_f;      // [cells, 3, D]
  const float* tape_dh;      // [cells, D]
  float* carry_h;            // [Bp, D] the horizontal successor's dh' share
  float* carry_v;            // [Bp, Lx, D] the vertical successor's dh' share, per lattice column
  uint8_t* g1;               // G1 tape: [dh_W | dh_g | dh_mix] in six tiles of 128 columns
  WsHeader* hdr;
};

struct SS {
  static constexpr uint32_t kA = 0;                                  // 4 x [128 x 128] bf16 chunk slots
  static constexpr uint32_t kRingOff = kA + 4 * 128 * 128 * 2;       // kRing x 16 KB
  static constexpr uint32_t kPos = kRingOff + kRing * kSlotBytes;    // 256 ints
  static constexpr uint32_t kBar = kPos + 256 * 4;                   // full[kRing], empty[kRing], done, drain
  static constexpr uint32_t kMisc = kBar + (2 * kRing + 2) * 8;      // TMEM slot, abort flag
  static constexpr uint32_t kBytes = 1024 + kMisc + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
};

__global__ void __launch_bounds__(kThreads, 1) tc2dw_sweep_kernel(const uint8_t* __restrict__ w1t, SwArgs a) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024 - (tc::smem_addr(smraw) & 1023)) & 1023);
  const uint32_t wlim = tc::g_wait_polls;   // bound of the waits that may give up
  uint8_t* sA = sm + SS::kA;
  uint8_t* ring = sm + SS::kRingOff;
  int* sPos = reinterpret_cast<int*>(sm + SS::kPos);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + SS::kBar);
  uint64_t* empty = full + kRing;
  uint64_t* done = empty + kRing;
  uint64_t* drain = done + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + SS::kMisc);
  volatile int* s_abort = reinterpret_cast<volatile int*>(sm + SS::kMisc + 4);
  volatile int* s_stop = reinterpret_cast<volatile int*>(sm + SS::kMisc + 8);
  volatile uint32_t* s_consf = reinterpret_cast<volatile uint32_t*>(sm + SS::kMisc + 12);
  const int N = a.N, Lx = a.Lx, Ly = a.N / a.Lx;
  for (int t = threadIdx.x; t < N; t += kThreads) {
    const Pz p = zpos(t, Lx);
    sPos[t] = p.i | (p.j << 8) | (p.r << 16);
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < kRing; ++q) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&empty[q], 1);
    }
    tc::mbar_init(done, 1);
    tc::mbar_init(drain, 1);
    *s_abort = 0;
    *s_stop = 0;
    *s_consf = 0;
    tc::mbar_fence_init();
  }
  if (threadIdx.x < 32) tc::tmem_alloc(tslot, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool timed_out = false;
  auto P = [&](int t) -> Pz {
    const int v = sPos[t];
    Pz p;
    p.i = v & 255;
    p.j = (v >> 8) & 255;
    p.r = v >> 16;
    return p;
  };

  if (warp == kWorkers / 32 + 1) {
    // ======================== producer warp ========================
    if (lane == 0)
      produce_slabs(ring, full, empty, s_stop, s_consf, s_abort, a.hdr, wlim, timed_out,
                    [&](uint32_t s, const uint8_t*& src, uint32_t& bytes) {
                      src = w1t + (size_t)(s % kNW1t) * kW1tSlab;
                      bytes = kW1tSlab;
                    });
    __syncwarp();
  } else if (warp == kWorkers / 32) {
    // ======================== issuer warp ========================
    // per step, six chunks of 128 gate units (W, W_g, U_mix blocks, two
    // halves each), 8 slabs of [512 h' columns x 16 units] per chunk; chunk q
    // reads A slot q % 4
    const bool leader = lane == 0;
    const uint32_t a_addr = tc::smem_addr(sA), r_addr = tc::smem_addr(ring);
    uint32_t s_cons = 0;
    bool dead = false;
    auto die = [&]() {
      dead = true;
      timed_out = true;
      *s_abort = 1;
      flag_status(a.hdr, NQS_ETIMEOUT);
    };
    auto chunk = [&](int q) {
      for (int kk = 0; kk < 8; ++kk) {
        if (dead) return;
        const uint32_t s = s_cons, slot = s % kRing;
        if (!tc::mbar_wait(&full[slot], (s / kRing) & 1, wlim)) {
          die();
          return;
        }
        tc::fence_after_sync();
        const uint32_t sa = r_addr + slot * kSlotBytes;
        const uint64_t da = tc::make_desc(a_addr + (uint32_t)(q % 4) * 32768u + 256u * kk, 128, 2048);
        const uint32_t accf = (q == 0 && kk == 0) ? 0u : 1u;
        tc::mma_bf16(tbase, da, tc::make_desc(sa, 128, 256), kIdesc256, accf);
        tc::mma_bf16(tbase + 256, da, tc::make_desc(sa + 8192, 128, 256), kIdesc256, accf);
        tc::mma_commit(&empty[slot]);
        ++s_cons;
      }
    };
    auto go = [&]() {
      __syncwarp();
      tc::group_barrier(kBarGo, kSync);
      tc::fence_after_sync();
    };
    for (int step = 0; step < a.t1 - a.t0; ++step) {
      go();                            // dh' of the previous step read, chunks 0-3 written
      if (leader) {
        chunk(0);
        chunk(1);
        tc::mma_commit(done);          // slots 0, 1 free again
        chunk(2);
        chunk(3);
        tc::mma_commit(done);
      }
      go();                            // chunks 4, 5 written
      if (leader) {
        chunk(4);
        chunk(5);
        tc::mma_commit(done);          // dh' complete
      }
      __syncwarp();
    }
    if (leader) {
      *s_consf = s_cons;
      __threadfence_block();
      *s_stop = 1;
    }
    __syncwarp();
  } else {
    // ======================== worker warps ========================
    const int part = warp >> 2, quarter = warp & 3;
    const int m = quarter * 32 + lane;                         // sample row = TMEM lane
    const uint32_t trow = tbase + ((uint32_t)(quarter * 32) << 16);
    const int64_t b = (int64_t)blockIdx.x * 128 + m;           // rows past B carry zeros
    const int h = part >> 1, cb = 64 * (part & 1);             // this slice's chunk half and column base
    const int64_t nkb = a.Bp * (a.t1 - a.t0) / 16;
    uint32_t pd = 0;
    auto wait_done = [&]() {
      if (!tc::mbar_wait(done, pd, wlim)) {
        timed_out = true;
        *s_abort = 1;
        flag_status(a.hdr, NQS_ETIMEOUT);
      }
      pd ^= 1;
      tc::fence_after_sync();
    };
    auto to_issuer = [&]() {
      tc::fence_async_smem();
      tc::fence_before_sync();
      tc::group_arrive(kBarGo, kSync);
    };
    auto slot_row = [&](int slot, int col) { return sA + slot * 32768 + tc::kmajor_offset(m, col, 128); };
    for (int step = 0; step < a.t1 - a.t0; ++step) {
      const int t = a.t1 - 1 - step;
      const Pz p = P(t);
      const int64_t cell = (int64_t)(t - a.t0) * a.Bp + b;
      const bool has_h = t + 1 < N && P(t + 1).r > 0;         // horizontal successor in this lattice row
      const bool has_v = p.j + 1 < Ly;                        // vertical successor (i, j + 1)
      const float* ch = a.carry_h + b * WD;
      const float* cv = a.carry_v + (b * Lx + p.i) * WD;
      uint32_t dmp[32];                                        // dh_mix chunk, packed BF16
#pragma unroll
      for (int g8 = 0; g8 < 8; ++g8) {
        const int u0 = 64 * part + 8 * g8;
        float dh[8];
        {
          const float4 x0 = *reinterpret_cast<const float4*>(a.tape_dh + cell * WD + u0);
          const float4 x1 = *reinterpret_cast<const float4*>(a.tape_dh + cell * WD + u0 + 4);
          dh[0] = x0.x; dh[1] = x0.y; dh[2] = x0.z; dh[3] = x0.w;
          dh[4] = x1.x; dh[5] = x1.y; dh[6] = x1.z; dh[7] = x1.w;
        }
        if (has_h) {
          const float4 x0 = *reinterpret_cast<const float4*>(ch + u0);
          const float4 x1 = *reinterpret_cast<const float4*>(ch + u0 + 4);
          dh[0] += x0.x; dh[1] += x0.y; dh[2] += x0.z; dh[3] += x0.w;
          dh[4] += x1.x; dh[5] += x1.y; dh[6] += x1.z; dh[7] += x1.w;
        }
        if (has_v) {
          const float4 x0 = *reinterpret_cast<const float4*>(cv + u0);
          const float4 x1 = *reinterpret_cast<const float4*>(cv + u0 + 4);
          dh[0] += x0.x; dh[1] += x0.y; dh[2] += x0.z; dh[3] += x0.w;
          dh[4] += x1.x; dh[5] += x1.y; dh[6] += x1.z; dh[7] += x1.w;
        }
        const __half* f = a.tape_f + cell * (3 * WD) + u0;
        const uint4 r1 = *reinterpret_cast<const uint4*>(f);
        const uint4 r2 = *reinterpret_cast<const uint4*>(f + WD);
        const uint4 r3 = *reinterpret_cast<const uint4*>(f + 2 * WD);
        const __half2* f1 = reinterpret_cast<const __half2*>(&r1);
        const __half2* f2 = reinterpret_cast<const __half2*>(&r2);
        const __half2* f3 = reinterpret_cast<const __half2*>(&r3);
        float gw[8], gg[8], gm[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 a1 = __half22float2(f1[q]), a2 = __half22float2(f2[q]), a3 = __half22float2(f3[q]);
          gw[2 * q] = dh[2 * q] * a1.x;
          gw[2 * q + 1] = dh[2 * q + 1] * a1.y;
          gg[2 * q] = dh[2 * q] * a2.x;
          gg[2 * q + 1] = dh[2 * q + 1] * a2.y;
          gm[2 * q] = dh[2 * q] * a3.x;
          gm[2 * q + 1] = dh[2 * q + 1] * a3.y;
        }
        const uint4 pw = pack8_bf16(gw), pg = pack8_bf16(gg), pm = pack8_bf16(gm);
        *reinterpret_cast<uint4*>(slot_row(h, cb + 8 * g8)) = pw;
        *reinterpret_cast<uint4*>(slot_row(2 + h, cb + 8 * g8)) = pg;
        dmp[4 * g8] = pm.x;
        dmp[4 * g8 + 1] = pm.y;
        dmp[4 * g8 + 2] = pm.z;
        dmp[4 * g8 + 3] = pm.w;
        *reinterpret_cast<uint4*>(a.g1 + tape_off(cell, u0, 128, nkb)) = pw;
        *reinterpret_cast<uint4*>(a.g1 + tape_off(cell, WD + u0, 128, nkb)) = pg;
        *reinterpret_cast<uint4*>(a.g1 + tape_off(cell, 2 * WD + u0, 128, nkb)) = pm;
      }
      to_issuer();
      wait_done();                                             // chunks 0, 1 done: their slots are free
#pragma unroll
      for (int g8 = 0; g8 < 8; ++g8)
        *reinterpret_cast<uint4*>(slot_row(h, cb + 8 * g8)) =
            make_uint4(dmp[4 * g8], dmp[4 * g8 + 1], dmp[4 * g8 + 2], dmp[4 * g8 + 3]);
      to_issuer();
      wait_done();                                             // chunks 2, 3
      wait_done();                                             // chunks 4, 5: dh' in TMEM
      // dh' = [horizontal predecessor's share | vertical predecessor's share]
#pragma unroll
      for (int g8 = 0; g8 < 8; ++g8) {
        const int u0 = 64 * part + 8 * g8;
        uint32_t rh[8], rv[8];
        tld8(trow + u0, rh);
        tld8(trow + 256 + u0, rv);
        tc::tmem_wait_ld();
        tie(rh);
        tie(rv);
        float* dh_ = a.carry_h + b * WD + u0;
        float* dv_ = a.carry_v + (b * Lx + p.i) * WD + u0;
        reinterpret_cast<float4*>(dh_)[0] =
            make_float4(__uint_as_float(rh[0]), __uint_as_float(rh[1]), __uint_as_float(rh[2]), __uint_as_float(rh[3]));
        reinterpret_cast<float4*>(dh_)[1] =
            make_float4(__uint_as_float(rh[4]), __uint_as_float(rh[5]), __uint_as_float(rh[6]), __uint_as_float(rh[7]));
        reinterpret_cast<float4*>(dv_)[0] =
            make_float4(__uint_as_float(rv[0]), __uint_as_float(rv[1]), __uint_as_float(rv[2]), __uint_as_float(rv[3]));
        reinterpret_cast<float4*>(dv_)[1] =
            make_float4(__uint_as_float(rv[4]), __uint_as_float(rv[5]), __uint_as_float(rv[6]), __uint_as_float(rv[7]));
      }
    }
  }
  tc::fence_before_sync();
  if (__syncthreads_or(timed_out) && threadIdx.x == kWorkers) tc::drain_mmas(drain, kWait2);
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tbase, 512);
}

// Weight-gradient GEMMs (tcw::wgrad_kernel<256>).  Output tiles: GEMM1 (G1^T
// X1) t = 0..11: M-tile t / 2 of the 768 gate rows against h_hor (+ the 16
// extra columns) for even t, h_ver for odd t; GEMM2 (G2^T X2) t = 12..15:
// M-tile t - 12 of the 512 GLU rows against h (+ extras).  A work unit is one
// tile over one of kWgSplits ranges of 16-cell blocks.
constexpr int kWgTiles = 16, kWgCols = tcw::WgS<256>::kCols;

// dU_out[0] = sum_cells gd y, dU_out[1] = -dU_out[0], dc = (sum gd, -sum gd):
// per block, a fixed range of cells in order; thread k < 256 sums column k,
// thread 256 the gd themselves.
constexpr int kRoBlocks = 304;
__global__ void __launch_bounds__(288) tc2dw_readout_kernel(const __nv_bfloat16* __restrict__ y,
                                                          const float* __restrict__ gd, int64_t ncell,
                                                          float* __restrict__ part) {
  const int64_t per = (ncell + gridDim.x - 1) / gridDim.x, c0 = blockIdx.x * per;
  const int64_t c1 = c0 + per < ncell ? c0 + per : ncell;
  const int k = threadIdx.x;
  if (k > WD) return;
  float acc = 0.0f;
  for (int64_t c = c0; c < c1; ++c) acc = fmaf(gd[c], k < WD ? __bfloat162float(y[c * WD + k]) : 1.0f, acc);
  part[(size_t)blockIdx.x * (WD + 1) + k] = acc;
}

// Every flat parameter (App. A layout) from the GEMM units' sums (segments of
// positions in order, splits in order within each) and the readout blocks'
// sums.
__global__ void tc2dw_final_kernel(const float* __restrict__ wg, int splits, int nseg, const float* __restrict__ ro,
                                   int nro, float* __restrict__ grad) {
  constexpr int D = WD, W2c = 2 * D + 4;
  const int oWg = D * W2c, oU = 2 * D * W2c, ob = oU + 2 * D * D, obg = ob + D, oW1 = obg + D, ob1 = oW1 + D * D,
            oW2 = ob1 + D, ob2 = oW2 + D * D, oUo = ob2 + D, oc = oUo + 2 * D, P = oc + 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  int tile = -1, row = 0, col = 0;
  float sign = 1.0f;
  if (i < ob) {                                  // W, W_g [d, 2d + 4], U_mix [d, 2d]
    const int g = i < oWg ? 0 : i < oU ? 1 : 2;
    const int w = g < 2 ? W2c : 2 * D, r = (i - (g == 0 ? 0 : g == 1 ? oWg : oU)) / w,
              cc = (i - (g == 0 ? 0 : g == 1 ? oWg : oU)) % w;
    const int gr = g * D + r;                    // gate row of G1
    tile = 2 * (gr / 128) + (cc >= D && cc < 2 * D ? 1 : 0);
    row = gr % 128;
    col = cc < D ? cc : cc < 2 * D ? cc - D : 256 + 1 + (cc - 2 * D);
  } else if (i < oW1) {                          // b, b_g: the extra column 0
    const int g = i < obg ? 0 : 1, gr = g * D + (i - (g == 0 ? ob : obg));
    tile = 2 * (gr / 128);
    row = gr % 128;
    col = 256;
  } else if (i < oUo) {                          // W_1, b_1, W_2, b_2
    const int g = i < oW2 ? 0 : 1, base = g == 0 ? oW1 : oW2, r0 = i - base;
    const bool bias = r0 >= D * D;
    const int v = bias ? r0 - D * D : r0 / D;
    const int gr = g * D + v;
    tile = 12 + gr / 128;
    row = gr % 128;
    col = bias ? 256 : r0 % D;
  }
  float s = 0.0f;
  if (tile >= 0) {
    const size_t seg_stride = (size_t)kWgTiles * splits * 128 * kWgCols;
    for (int sg = 0; sg < nseg; ++sg)
      for (int sp = 0; sp < splits; ++sp)
        s += wg[sg * seg_stride + (((size_t)tile * splits + sp) * 128 + row) * kWgCols + col];
  } else {                                       // U_out [2, d], c [2]
    const int k = i < oc ? (i - oUo) % D : D;
    sign = (i < oc ? (i - oUo) / D : i - oc) == 0 ? 1.0f : -1.0f;
    for (int q = 0; q < nro; ++q) s += ro[(size_t)q * (WD + 1) + k];
  }
  grad[i] = sign * s;
}

}  // namespace

cudaError_t tc2dw_pack(const float* params, uint8_t* wimg, cudaStream_t st) {
  const int total = kGateSlabs * kGateRows * 16 + kNGlu * kGluRows * 16 + WD + 1;
  pack_wide_kernel<<<(total + 255) / 256, 256, 0, st>>>(params, wimg);
  return cudaGetLastError();
}

cudaError_t tc2dw_forward(const Tc2Fwd& f, const uint8_t* wimg, bool sample, cudaStream_t st) {
  WArgs a{};
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
  a.hdr = f.hdr;
  const int64_t grid = (f.B + 127) / 128;
  return sample ? launch_w<0>(a, wimg, grid, st) : launch_w<1>(a, wimg, grid, st);
}

cudaError_t tc2dw_tables(const Tc2Fwd& f, const uint8_t* wimg, cudaStream_t st) {
  if (f.B > 0) {
    nup_prefix_kernel<<<(unsigned)((f.B + 127) / 128), 128, 0, st>>>(f.sigma_in, f.B, f.Lx, f.N, f.nup_tab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  WArgs a{};
  a.B = f.B;
  a.Lx = f.Lx;
  a.N = f.N;
  a.sz0 = f.sz0;
  a.hcache = f.hcache;
  a.lp_tab = f.lp_tab;
  a.nup_tab = f.nup_tab;
  a.hdr = f.hdr;
  const int64_t ntile = (f.B * f.N + 127) / 128;
  return launch_w<3>(a, wimg, ntile < sm_count_w() ? ntile : sm_count_w(), st);
}

cudaError_t tc2dw_chains(const Tc2Chains& c, const uint8_t* wimg, const uint8_t* jobs, const int* njobs, cudaStream_t st) {
  WArgs a{};
  a.B = c.B;
  a.Lx = c.Lx;
  a.N = c.N;
  a.nb = c.nb;
  a.sz0 = c.sz0;
  a.hcache = const_cast<float*>(c.hcache);
  a.colbuf = c.colbuf;
  a.lp_tab = const_cast<float*>(c.lp_tab);
  a.bonds = c.bonds;
  a.jobs = reinterpret_cast<const JobT<4>*>(jobs);
  a.njobs = njobs;
  a.delta = c.delta;
  a.counter = c.counter;
  a.hdr = c.hdr;
  return launch_w<2>(a, wimg, sm_count_w(), st);
}

namespace {
constexpr int kWgSplits = 9;   // 16 tiles x 9 cell ranges: 144 units, one wave on 152 SMs

struct WideGradLayout {
  size_t img2, nup, tape_f, tape_dh, g1, x1a, x1b, x1c, g2, x2a, x2c, y, gd, carry_h, carry_v, wg, ro, total;
};

// Positions per pass of the reverse sweep: all N, or seg (> 0) at a time.
int wide_seg_positions(int N, int seg) { return seg > 0 && seg < N ? seg : N; }

// The tapes hold one pass's cells; the weight-gradient and readout partial
// sums are kept per pass.
WideGradLayout wide_grad_layout(int64_t B, int Lx, int N, int seg) {
  const int S = wide_seg_positions(N, seg), nseg = (N + S - 1) / S;
  const size_t Bp = (size_t)((B + 127) / 128 * 128), cells = Bp * (size_t)S;
  WideGradLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off += (bytes + 255) / 256 * 256; return at; };
  L.img2 = take(kBwdImg);
  L.nup = take((size_t)B * N * 4);
  L.tape_f = take(cells * 3 * WD * 2);
  L.tape_dh = take(cells * WD * 4);
  L.g1 = take(cells * 3 * WD * 2);
  L.x1a = take(cells * WD * 2);
  L.x1b = take(cells * WD * 2);
  L.x1c = take(cells * 16 * 2);
  L.g2 = take(cells * 2 * WD * 2);
  L.x2a = take(cells * WD * 2);
  L.x2c = take(cells * 16 * 2);
  L.y = take(cells * WD * 2);
  L.gd = take(cells * 4);
  L.carry_h = take(Bp * WD * 4);
  L.carry_v = take(Bp * (size_t)Lx * WD * 4);
  L.wg = take((size_t)nseg * kWgTiles * kWgSplits * 128 * kWgCols * 4);
  L.ro = take((size_t)nseg * kRoBlocks * (WD + 1) * 4);
  L.total = off;
  return L;
}
}  // namespace

size_t tc2dw_grad_bytes(int64_t B, int Lx, int N, int seg) { return wide_grad_layout(B, Lx, N, seg).total; }

cudaError_t tc2dw_grad(const Tc2WGrad& g, const uint8_t* wimg, float* grad, cudaStream_t st) {
  const WideGradLayout L = wide_grad_layout(g.B, g.Lx, g.N, g.seg);
  uint8_t* w = g.scratch;
  const int S = wide_seg_positions(g.N, g.seg), nseg = (g.N + S - 1) / S;
  const int64_t Bp = (g.B + 127) / 128 * 128;
  uint8_t* img2 = w + L.img2;
  cudaError_t e;
  const int nbwd = kNW1t * 512 * 16 + kNGlut * 256 * 16;
  pack_wide_bwd_kernel<<<(nbwd + 255) / 256, 256, 0, st>>>(g.params, img2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int* nup = reinterpret_cast<int*>(w + L.nup);
  if (g.B > 0) {
    nup_prefix_kernel<<<(unsigned)((g.B + 127) / 128), 128, 0, st>>>(g.sigma, g.B, g.Lx, g.N, nup);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  WArgs a{};
  a.B = g.B;
  a.Lx = g.Lx;
  a.N = g.N;
  a.sz0 = g.sz0;
  a.sigma_in = g.sigma;
  a.hcache = const_cast<float*>(g.hcache);
  a.nup_tab = nup;
  a.hdr = g.hdr;
  a.img2 = img2;
  a.wts = g.weights;
  a.Bp = Bp;
  a.tape_f = reinterpret_cast<__half*>(w + L.tape_f);
  a.tape_dh = reinterpret_cast<float*>(w + L.tape_dh);
  a.x1a = w + L.x1a;
  a.x1b = w + L.x1b;
  a.x1c = w + L.x1c;
  a.g2 = w + L.g2;
  a.x2a = w + L.x2a;
  a.x2c = w + L.x2c;
  a.ytape = reinterpret_cast<__nv_bfloat16*>(w + L.y);
  a.gd = reinterpret_cast<float*>(w + L.gd);
  SwArgs sw{};
  sw.B = g.B;
  sw.Bp = Bp;
  sw.Lx = g.Lx;
  sw.N = g.N;
  sw.tape_f = a.tape_f;
  sw.tape_dh = a.tape_dh;
  sw.carry_h = reinterpret_cast<float*>(w + L.carry_h);
  sw.carry_v = reinterpret_cast<float*>(w + L.carry_v);
  sw.g1 = w + L.g1;
  sw.hdr = g.hdr;
  if ((e = cudaFuncSetAttribute(tc2dw_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SS::kBytes)) !=
      cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  float* wgbuf = reinterpret_cast<float*>(w + L.wg);
  float* ro = reinterpret_cast<float*>(w + L.ro);
  // passes over positions [t0, t1), last first: the sweep's carries (in
  // global memory) run on from one pass into the next
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int t0 = sg * S, t1 = t0 + S < g.N ? t0 + S : g.N;
    const int64_t cells = Bp * (t1 - t0), nkb = cells / 16;
    // 1. tape pass
    a.t0 = t0;
    a.t1 = t1;
    const int64_t ntile = (int64_t)(t1 - t0) * (Bp / 128);
    if ((e = launch_w<4>(a, wimg, ntile < sm_count_w() ? ntile : sm_count_w(), st)) != cudaSuccess) return e;
    // 2. sequential sweep
    sw.t0 = t0;
    sw.t1 = t1;
    if (Bp > 0) {
      tc2dw_sweep_kernel<<<(unsigned)(Bp / 128), kThreads, SS::kBytes, st>>>(img2, sw);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // 3. weight-gradient GEMMs and the readout gradients of this pass's cells
    WgArgs wg{};
    for (int t = 0; t < kWgTiles; ++t) {
      const bool first = t < 12;
      const int mt = first ? t / 2 : t - 12, nt = first ? t % 2 : 0;
      wg.tiles[t].A = (first ? sw.g1 : a.g2) + (size_t)mt * nkb * 4096;
      wg.tiles[t].Bm = first ? (nt == 0 ? a.x1a : a.x1b) : a.x2a;
      wg.tiles[t].Bx = first ? (nt == 0 ? a.x1c : nullptr) : a.x2c;
    }
    wg.nkb = nkb;
    wg.splits = kWgSplits;
    wg.out = wgbuf + (size_t)sg * kWgTiles * kWgSplits * 128 * kWgCols;
    wg.hdr = g.hdr;
    if ((e = launch_wgrad<256>(wg, kWgTiles, st)) != cudaSuccess) return e;
    tc2dw_readout_kernel<<<kRoBlocks, 288, 0, st>>>(a.ytape, a.gd, cells, ro + (size_t)sg * kRoBlocks * (WD + 1));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 4. the flat gradient
  constexpr int D = WD;
  const int P = 6 * D * D + 10 * D + 2 * D * D + 4 * D + 2;
  tc2dw_final_kernel<<<(P + 255) / 256, 256, 0, st>>>(wgbuf, kWgSplits, nseg, ro, nseg * kRoBlocks, grad);
  return cudaGetLastError();
}

cudaError_t tc2dw_set_wait_polls(uint32_t polls) { return cudaMemcpyToSymbol(tc::g_wait_polls, &polls, sizeof(polls)); }

}  // namespace nqs

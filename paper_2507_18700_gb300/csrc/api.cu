// C-ABI entry points of libnqs (include/nqs.h): argument checks on the host,
// workspace carving, and kernel dispatch.  Nothing here allocates memory.
#include <cstring>

#include "kernels.h"

using namespace nqs;

namespace {

struct Dims {
  int cell, Lx, Ly, N, d, m, sz0, precision, phase;
  size_t P;
};

bool valid_hidden(int cell, int d) { return cell == NQS_GRU2D ? gru2d_supported(d) : gru1d_supported(d); }

nqs_status check_desc(const nqs_model_desc* desc, Dims* out) {
  if (!desc) return NQS_EINVAL;
  Dims d{};
  d.cell = desc->cell;
  d.Lx = desc->Lx;
  d.Ly = desc->Ly;
  d.d = desc->d_h;
  d.m = desc->d_model == 0 ? desc->d_h : desc->d_model;
  d.sz0 = desc->sz0;
  d.phase = desc->phase;
  d.precision = desc->precision;
  if (d.cell != NQS_GRU1D && d.cell != NQS_GRU2D) return NQS_EINVAL;
  if (d.precision != NQS_FP32 && d.precision != NQS_BF16) return NQS_EINVAL;
  if (d.sz0 != 0 && d.sz0 != 1) return NQS_EINVAL;
  if (d.phase != 0 && d.phase != 1) return NQS_EINVAL;
  if (d.Lx < 1 || d.Ly < 1 || (int64_t)d.Lx * d.Ly > (1 << 20)) return NQS_ESHAPE;
  d.N = d.Lx * d.Ly;
  if (!valid_hidden(d.cell, d.d)) return NQS_ESHAPE;
  if (d.cell == NQS_GRU1D && d.Ly != 1) return NQS_ESHAPE;
  if (d.cell == NQS_GRU2D && d.m != d.d) return NQS_ESHAPE;
  if (d.sz0 && (d.N % 2)) return NQS_ESHAPE;
  if (d.cell == NQS_GRU1D)
    d.P = 3 * (size_t)d.d * d.d + 12 * (size_t)d.d + 2 + (d.phase ? 2 * (size_t)d.d + 2 : 0);
  else
    d.P = 6 * (size_t)d.d * d.d + 10 * (size_t)d.d + 2 * (size_t)d.m * d.d + 4 * (size_t)d.m + 2;
  if (out) *out = d;
  return NQS_OK;
}

// Paths built so far: FP32 1D GRU (no mask), FP32 2D GRU, the BF16
// tensor-core 1D GRU for d_h in {16, 32, 64, 128} and the BF16 tensor-core 2D
// GRU for d_h in {32, 64, 256} with N <= 256 (configurations as 128- or
// 256-bit masks).
nqs_status check_built(const Dims& d) {
  if (d.cell == NQS_GRU1D && d.sz0) return NQS_EUNSUPPORTED;
  // the cRNN phase head: FP32 1D GRU, d_h >= 16
  if (d.phase && (d.cell != NQS_GRU1D || d.precision != NQS_FP32 || d.d < 16)) return NQS_EUNSUPPORTED;
  if (d.precision == NQS_BF16) {
    const bool ok = d.cell == NQS_GRU1D ? tc1d_supported(d.d) != 0 : tc2d_supported(d.d, d.Lx, d.N) != 0;
    if (!ok) return NQS_EUNSUPPORTED;
  }
  return NQS_OK;
}

bool use_tc(const Dims& d) { return d.precision == NQS_BF16 && d.cell == NQS_GRU1D; }
// the 1D BF16 reverse sweep: weight gradients in TMEM for d_h <= 64 (tc1d.cu),
// through operand tapes and a separate GEMM at d_h = 128 (tc1d_grad128.cu)
bool use_tc_grad(const Dims& d) { return use_tc(d) && d.d <= 64; }
bool use_tc128_grad(const Dims& d) { return use_tc(d) && d.d == 128; }
// flat offset of the cRNN phase layer [U_phi | c_phi] (after the amplitude parameters)
size_t phase_offset(const Dims& d) { return 3 * (size_t)d.d * d.d + 12 * (size_t)d.d + 2; }
bool use_tc2d(const Dims& d) { return d.precision == NQS_BF16 && d.cell == NQS_GRU2D; }
// the 2D BF16 reverse sweep: weights in shared memory for d_h <= 64
// (tc2d_grad.cu), streamed for d_h = 256 (tc2d_wide.cu)
bool use_tc2d_grad(const Dims& d) { return use_tc2d(d) && d.d <= 64; }
bool use_tc2dw_grad(const Dims& d) { return use_tc2d(d) && d.d == 256; }

// Positions per pass of the d_h = 256 2D reverse sweep (0: one pass).
int g_sweep_seg = 0;

int n_bonds(const Dims& d) { return (d.Lx - 1) * d.Ly + d.Lx * (d.Ly - 1); }

// Workspace layout: [header | packed weights | per-op buffers], 256-aligned.
struct Layout {
  size_t img, w, w2, a, b, c, e, f, g, h, i, j, total;
};

Layout layout(const Dims& d, int64_t B, int op) {
  Layout L{};
  size_t off = sizeof(WsHeader);
  const bool two = d.cell == NQS_GRU2D;
  L.img = off;
  off += align256((two ? gru2d_img_floats(d.d) : gru1d_img_floats(d.d)) * sizeof(float));
  if (use_tc(d)) {
    L.w = off;
    off += align256(tc1d_wimg_bytes(d.d));
    L.w2 = off;                                   // transposed image for the reverse sweep
    off += align256(tc1d_wimg_bytes(d.d));
  }
  if (use_tc2d(d)) {
    L.w = off;
    off += align256(tc2d_wimg_bytes(d.d));
  }
  const size_t BN = (size_t)B * (size_t)d.N;
  auto take = [&](size_t bytes) { const size_t at = off; off += align256(bytes); return at; };
  switch (op) {
    case NQS_OP_SAMPLE:
    case NQS_OP_LOGPSI:
      if (two) L.a = take((use_tc2d(d) ? tc2d_colbuf_floats(B, d.Lx, d.d)
                                        : (size_t)gru2d_engine_slots(d.d, B, 1) * d.Lx * d.d) * sizeof(float));  // colbuf
      break;
    case NQS_OP_LOCAL_ENERGY:
      if (!two) {
        L.a = take(BN * sizeof(float));        // dlog
        L.b = take(BN * sizeof(float));        // delta (cluster: its real part)
        L.c = take(BN * 2 * sizeof(float));    // cluster: phase logits of the cached path
        L.e = take(BN * sizeof(float));        // cluster: imaginary part of delta
      } else {
        L.a = take((use_tc2d(d) ? tc2d_colbuf_floats(B, d.Lx, d.d)
                                : (size_t)gru2d_engine_slots(d.d, B, 2) * d.Lx * d.d) * sizeof(float));  // colbuf
        L.b = take((size_t)n_bonds(d) * 16);                  // bond table
        L.c = take(BN * 2 * sizeof(float));                   // lp_tab
        L.e = take(BN * sizeof(int));                         // nup_tab
        L.f = take((size_t)B * n_bonds(d) * sizeof(float));   // delta
        if (use_tc2d(d)) L.g = take(tc2d_jobs_bytes(B, n_bonds(d), d.N, d.d));   // chain jobs
      }
      break;
    case NQS_OP_LOGPSI_GRAD:
    case NQS_OP_VMC_GRAD: {
      if (use_tc128_grad(d)) {
        L.a = take(d.P * sizeof(float));                       // the flat FP32 gradient
        L.b = take((size_t)B * sizeof(float));                 // weights
        L.c = take(tc1d128_grad_bytes(B, d.N));                // tapes of the reverse sweep
        break;
      }
      if (use_tc2dw_grad(d)) {
        L.a = take(d.P * sizeof(float));                       // the flat FP32 gradient
        L.b = take((size_t)B * sizeof(float));                 // weights
        L.c = take(tc2dw_grad_bytes(B, d.Lx, d.N, g_sweep_seg));   // tapes of the reverse sweep
        break;
      }
      if (use_tc2d_grad(d)) {
        L.a = take((size_t)tc2d_grad_partial_rows(B, d.N) * d.P * sizeof(float));  // partial gradients
        L.b = take((size_t)B * sizeof(float));                                     // weights
        L.c = take((size_t)B * d.Lx * d.d * sizeof(float));                        // vertical carries
        L.e = take(tc2d_grad_image_bytes(B, d.N, d.d, 0));                         // G1 images
        L.f = take(tc2d_grad_image_bytes(B, d.N, d.d, 1));                         // G2 images
        L.g = take(tc2d_grad_image_bytes(B, d.N, d.d, 2));                         // GLU outputs
        L.h = take(tc2d_grad_image_bytes(B, d.N, d.d, 3));                         // readout gradients
        L.i = take(tc2d_grad_image_bytes(B, d.N, d.d, 4));                         // tape: dh_glu
        L.j = take(tc2d_grad_image_bytes(B, d.N, d.d, 5));                         // tape: factors
        break;
      }
      if (use_tc_grad(d)) {
        L.a = take((size_t)tc1d_bptt_partial_rows(B) * d.P * sizeof(float));  // partial gradients
        L.b = take((size_t)B * sizeof(float));                                 // weights
        L.e = take(tc1d_tape_bytes(B, d.N, d.d, 0));                            // tape: e
        L.f = take(tc1d_tape_bytes(B, d.N, d.d, 1));                            // tape: BF16 states
        L.g = take(tc1d_tape_bytes(B, d.N, d.d, 2));                            // tape: backward factors
        break;
      }
      const size_t grid = (size_t)(two ? gru2d_bptt_grid(d.d, B)
                                       : d.phase ? crnn_bptt_grid(B, d.d) : gru1d_bptt_grid(d.d, B));
      L.a = take(grid * d.P * sizeof(float));               // partial gradients
      L.b = take((size_t)B * 2 * sizeof(float));             // weights (complex for the cRNN)
      if (two) L.c = take((size_t)B * d.Lx * d.d * sizeof(float));  // vertical carries
      if (two) L.e = take(gru2d_bptt_scratch_floats(d.d, B) * sizeof(float));  // small-gradient scratch
      break;
    }
    default:
      break;
  }
  L.total = off;
  return L;
}

// params and hcache are read (and hcache written) in 16-byte pieces
bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

nqs_status check_ws(void* ws, size_t ws_bytes, const Layout& L) {
  if (!ws) return NQS_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return NQS_EWORKSPACE;
  if (ws_bytes < L.total) return NQS_EWORKSPACE;
  return NQS_OK;
}

inline nqs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? NQS_OK : NQS_ECUDA; }

// Every call starts by clearing the workspace status word, so after a call the
// word holds what that call's kernels recorded.
inline bool reset_status(void* ws, cudaStream_t st) {
  return cudaMemsetAsync(&static_cast<WsHeader*>(ws)->status, 0, sizeof(int32_t), st) == cudaSuccess;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

}  // namespace

namespace nqs {
// The descriptor checks of every workspace call, for the other entry points.
nqs_status desc_status(const nqs_model_desc* desc) { return check_desc(desc, nullptr); }
}  // namespace nqs

// The gradient reverse sweep behind nqs_logpsi_grad, nqs_vmc_grad and
// nqs_vmc_grad_global; T is the type of the reduced gradient (float or double).
template <typename T>
static nqs_status grad_common(const Dims& d, const Layout& L, const float* params,
                              const uint8_t* sigma, const float* hcache, const float* weights,
                              int64_t B, T* grad, void* ws, cudaStream_t st) {
  float* img = at<float>(ws, L.img);
  float* partial = at<float>(ws, L.a);
  if (d.phase) {
    // cRNN: weights are [B, 2] = (w for log |psi|, v for phi)
    const int grid = crnn_bptt_grid(B, d.d);
    if (gru1d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Bptt1Args a{};
    a.B = B;
    a.N = d.N;
    a.P = (int)d.P;
    a.sigma = sigma;
    a.hcache = hcache;
    a.weights = weights;
    a.partial = partial;
    if (crnn_bptt(a, img, params + phase_offset(d), weights, d.d, st) != cudaSuccess) return NQS_ECUDA;
    return cuda_status(reduce_partials(partial, grid, (int)d.P, grad, st));
  }
  if (use_tc_grad(d)) {
    uint8_t* w3 = at<uint8_t>(ws, L.w);
    uint8_t* wt = at<uint8_t>(ws, L.w2);
    if (gru1d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    if (tc1d_pack(params, w3, d.d, st) != cudaSuccess) return NQS_ECUDA;
    if (tc1d_pack_t(params, wt, d.d, st) != cudaSuccess) return NQS_ECUDA;
    TcBpttArgs t{};
    t.B = B;
    t.N = d.N;
    t.P = (int)d.P;
    t.sigma = sigma;
    t.hcache = hcache;
    t.weights = weights;
    t.partial = partial;
    t.tape_e = at<float>(ws, L.e);
    t.tape_x = at<uint8_t>(ws, L.f);
    t.tape_k = at<uint8_t>(ws, L.g);
    t.hdr = static_cast<WsHeader*>(ws);
    if (tc1d_bptt(t, img, w3, wt, d.d, st) != cudaSuccess) return NQS_ECUDA;
    return cuda_status(tc1d_bptt_reduce(t, d.d, grad, st));
  }
  if (use_tc128_grad(d)) {
    uint8_t* wimg = at<uint8_t>(ws, L.w);
    if (tc1d_pack(params, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Tc1WGrad g{};
    g.B = B;
    g.N = d.N;
    g.sigma = sigma;
    g.hcache = hcache;
    g.weights = weights;
    g.params = params;
    g.scratch = at<uint8_t>(ws, L.c);
    g.hdr = static_cast<WsHeader*>(ws);
    if (tc1d128_grad(g, wimg, partial, st) != cudaSuccess) return NQS_ECUDA;
    return cuda_status(reduce_partials(partial, 1, (int)d.P, grad, st));
  }
  if (use_tc2dw_grad(d)) {
    uint8_t* wimg = at<uint8_t>(ws, L.w);
    if (tc2d_pack(params, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Tc2WGrad g{};
    g.B = B;
    g.Lx = d.Lx;
    g.N = d.N;
    g.sz0 = d.sz0;
    g.sigma = sigma;
    g.hcache = hcache;
    g.weights = weights;
    g.params = params;
    g.scratch = at<uint8_t>(ws, L.c);
    g.hdr = static_cast<WsHeader*>(ws);
    g.seg = g_sweep_seg;
    if (tc2dw_grad(g, wimg, partial, st) != cudaSuccess) return NQS_ECUDA;
    return cuda_status(reduce_partials(partial, 1, (int)d.P, grad, st));
  }
  if (use_tc2d_grad(d)) {
    uint8_t* wimg = at<uint8_t>(ws, L.w);
    const int rows = tc2d_grad_partial_rows(B, d.N);
    if (tc2d_pack(params, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
    if (cudaMemsetAsync(partial, 0, (size_t)rows * d.P * sizeof(float), st) != cudaSuccess) return NQS_ECUDA;
    Tc2Grad g{};
    g.B = B;
    g.Lx = d.Lx;
    g.Ly = d.Ly;
    g.N = d.N;
    g.P = (int)d.P;
    g.sz0 = d.sz0;
    g.sigma = sigma;
    g.hcache = hcache;
    g.weights = weights;
    g.ccarry = at<float>(ws, L.c);
    g.g1img = at<uint8_t>(ws, L.e);
    g.g2img = at<uint8_t>(ws, L.f);
    g.yimg = at<float>(ws, L.g);
    g.dzimg = at<float>(ws, L.h);
    g.tape_h = at<float>(ws, L.i);
    g.tape_k = at<uint8_t>(ws, L.j);
    g.partial = partial;
    g.hdr = static_cast<WsHeader*>(ws);
    if (tc2d_grad(g, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
    return cuda_status(reduce_partials(partial, rows, (int)d.P, grad, st));
  }
  if (d.cell == NQS_GRU2D) {
    const int grid = gru2d_bptt_grid(d.d, B);
    if (gru2d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    if (cudaMemsetAsync(partial, 0, (size_t)grid * d.P * sizeof(float), st) != cudaSuccess)
      return NQS_ECUDA;
    Bptt2Args a{};
    a.B = B;
    a.Lx = d.Lx;
    a.N = d.N;
    a.P = (int)d.P;
    a.sz0 = d.sz0;
    a.sigma = sigma;
    a.hcache = hcache;
    a.weights = weights;
    a.ccarry = at<float>(ws, L.c);
    a.partial = partial;
    a.sacc = at<float>(ws, L.e);
    const size_t scratch = gru2d_bptt_scratch_floats(d.d, B);
    if (scratch && cudaMemsetAsync(a.sacc, 0, scratch * sizeof(float), st) != cudaSuccess) return NQS_ECUDA;
    if (gru2d_bptt(a, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    return cuda_status(reduce_partials(partial, grid, (int)d.P, grad, st));
  }
  const int grid = gru1d_bptt_grid(d.d, B);
  if (gru1d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
  if (cudaMemsetAsync(partial, 0, (size_t)grid * d.P * sizeof(float), st) != cudaSuccess)
    return NQS_ECUDA;
  Bptt1Args a{};
  a.B = B;
  a.N = d.N;
  a.P = (int)d.P;
  a.sigma = sigma;
  a.hcache = hcache;
  a.weights = weights;
  a.partial = partial;
  if (gru1d_bptt(a, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
  return cuda_status(reduce_partials(partial, grid, (int)d.P, grad, st));
}

extern "C" {

void nqs_set_autotune(int on) { tc1d_set_autotune(on); }
void nqs_set_tile_variant(int variant) { tc1d_set_variant(variant); }

void nqs_set_sweep_segment(int32_t positions) { g_sweep_seg = positions > 0 ? positions : 0; }

size_t nqs_param_count(const nqs_model_desc* desc) {
  Dims d;
  if (check_desc(desc, &d) != NQS_OK) return 0;
  return d.P;
}

size_t nqs_workspace_bytes(const nqs_model_desc* desc, const nqs_ham_desc* ham, int64_t B, int op) {
  Dims d;
  if (check_desc(desc, &d) != NQS_OK || B < 0) return 0;
  if (op < NQS_OP_SAMPLE || op > NQS_OP_VMC_GRAD) return 0;
  if (op == NQS_OP_LOCAL_ENERGY && !ham) return 0;
  return layout(d, B, op).total;
}

const char* nqs_status_string(nqs_status s) {
  switch (s) {
    case NQS_OK: return "NQS_OK";
    case NQS_EINVAL: return "NQS_EINVAL: invalid argument";
    case NQS_ESHAPE: return "NQS_ESHAPE: unsupported shape";
    case NQS_EWORKSPACE: return "NQS_EWORKSPACE: workspace missing, misaligned or too small";
    case NQS_ECUDA: return "NQS_ECUDA: CUDA runtime error";
    case NQS_ETIMEOUT: return "NQS_ETIMEOUT: device wait timed out";
    case NQS_ENONFINITE: return "NQS_ENONFINITE: non-finite value on the device";
    case NQS_EUNSUPPORTED: return "NQS_EUNSUPPORTED: combination not built";
  }
  return "NQS: unknown status";
}

nqs_status nqs_workspace_status(void* ws, int32_t* device_status, void* stream) {
  if (!ws || !device_status) return NQS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* hdr = static_cast<WsHeader*>(ws);
  int32_t v = 0;
  if (cudaMemcpyAsync(&v, &hdr->status, sizeof(v), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return NQS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return NQS_ECUDA;
  if (cudaMemsetAsync(&hdr->status, 0, sizeof(int32_t), st) != cudaSuccess) return NQS_ECUDA;
  *device_status = v;
  return NQS_OK;
}

nqs_status nqs_grow_hidden(const nqs_model_desc* small, const float* p_small,
                           const nqs_model_desc* big, float* p_big, uint64_t seed, float eps,
                           void* stream) {
  Dims s, b;
  nqs_status r = check_desc(small, &s);
  if (r != NQS_OK) return r;
  if ((r = check_desc(big, &b)) != NQS_OK) return r;
  if (!p_small || !p_big) return NQS_EINVAL;
  if (s.cell != b.cell || s.Lx != b.Lx || s.Ly != b.Ly) return NQS_ESHAPE;
  if (b.d < s.d || b.m < s.m) return NQS_ESHAPE;
  if (!(eps >= 0.0f)) return NQS_EINVAL;
  if (s.phase != b.phase) return NQS_ESHAPE;
  return cuda_status(grow_params(s.cell, s.phase, s.d, s.m, b.d, b.m, p_small, p_big, seed, eps,
                                 static_cast<cudaStream_t>(stream)));
}

static nqs_status forward_common(const nqs_model_desc* desc, const float* params, int64_t B,
                                 bool sample, uint64_t seed, uint64_t step, const uint64_t* step_dev,
                                 uint64_t b0, const float* uniforms,
                                 const uint8_t* sigma_in, uint8_t* sigma_out, float* logpsi,
                                 float* hcache, void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  nqs_status r = check_desc(desc, &d);
  if (r != NQS_OK) return r;
  if ((r = check_built(d)) != NQS_OK) return r;
  if (B < 0) return NQS_EINVAL;
  // the Philox counter holds the global sample index in 32 bits
  if (sample && (b0 > ((uint64_t)1 << 32) || (uint64_t)B > ((uint64_t)1 << 32) - b0)) return NQS_EINVAL;
  if (!params || misaligned(params) || misaligned(hcache)) return NQS_EINVAL;
  const Layout L = layout(d, B, sample ? NQS_OP_SAMPLE : NQS_OP_LOGPSI);
  if ((r = check_ws(ws, ws_bytes, L)) != NQS_OK) return r;
  if (B == 0) return NQS_OK;  // empty batch: outputs are empty, pointers may be null
  if (!logpsi || (sample ? !sigma_out : !sigma_in)) return NQS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  float* img = at<float>(ws, L.img);
  if (d.phase) {
    // cRNN: logpsi is [B, 2] = (log |psi|, phi)
    if (gru1d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Fwd1Args a{};
    a.B = B;
    a.N = d.N;
    a.sigma_in = sigma_in;
    a.sigma_out = sigma_out;
    a.uniforms = uniforms;
    a.seed = seed;
    a.step = step;
    a.b0 = b0;
    a.step_dev = step_dev;
    a.hcache = hcache;
    a.hdr = static_cast<WsHeader*>(ws);
    return cuda_status(crnn_forward(a, img, params + phase_offset(d), logpsi, d.d, sample, st));
  }
  if (use_tc2d(d)) {
    uint8_t* wimg = at<uint8_t>(ws, L.w);
    if (tc2d_pack(params, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Tc2Fwd f{};
    f.B = B;
    f.Lx = d.Lx;
    f.N = d.N;
    f.sz0 = d.sz0;
    f.sigma_in = sigma_in;
    f.sigma_out = sigma_out;
    f.uniforms = uniforms;
    f.seed = seed;
    f.step = step;
    f.b0 = b0;
    f.step_dev = step_dev;
    f.logpsi = logpsi;
    f.hcache = hcache;
    f.colbuf = at<float>(ws, L.a);
    f.hdr = static_cast<WsHeader*>(ws);
    return cuda_status(tc2d_forward(f, wimg, d.d, sample, st));
  }
  if (d.cell == NQS_GRU2D) {
    if (gru2d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Eng2Args a{};
    a.B = B;
    a.Lx = d.Lx;
    a.N = d.N;
    a.sz0 = d.sz0;
    a.sigma_in = sigma_in;
    a.sigma_out = sigma_out;
    a.uniforms = uniforms;
    a.seed = seed;
    a.step = step;
    a.b0 = b0;
    a.step_dev = step_dev;
    a.logpsi = logpsi;
    a.hcache = hcache;
    a.colbuf = at<float>(ws, L.a);
    a.hdr = static_cast<WsHeader*>(ws);
    return cuda_status(gru2d_forward(a, img, d.d, sample, st));
  }
  cudaError_t e = gru1d_pack(params, img, d.d, st);
  if (e != cudaSuccess) return NQS_ECUDA;
  if (use_tc(d)) {
    uint8_t* wimg = at<uint8_t>(ws, L.w);
    if (tc1d_pack(params, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Tc1Args t{};
    t.B = B;
    t.N = d.N;
    t.sigma = sigma_in;
    t.sigma_out = sigma_out;
    t.uniforms = uniforms;
    t.seed = seed;
    t.step = step;
    t.b0 = b0;
    t.step_dev = step_dev;
    t.logpsi = logpsi;
    t.hcache = hcache;
    t.hdr = static_cast<WsHeader*>(ws);
    return cuda_status(tc1d_run(t, img, wimg, d.d, sample ? 0 : 1, st));
  }
  Fwd1Args a{};
  a.B = B;
  a.N = d.N;
  a.sigma_in = sigma_in;
  a.sigma_out = sigma_out;
  a.uniforms = uniforms;
  a.seed = seed;
  a.step = step;
  a.b0 = b0;
  a.step_dev = step_dev;
  a.logpsi = logpsi;
  a.hcache = hcache;
  a.hdr = static_cast<WsHeader*>(ws);
  return cuda_status(gru1d_forward(a, img, d.d, sample, st));
}

nqs_status nqs_sample(const nqs_model_desc* desc, const float* params, int64_t B, uint64_t seed,
                      uint64_t step, const uint64_t* step_dev, uint64_t sample_offset, const float* uniforms,
                      uint8_t* sigma, float* logpsi, float* hcache, void* ws, size_t ws_bytes, void* stream) {
  return forward_common(desc, params, B, true, seed, step, step_dev, sample_offset, uniforms, nullptr, sigma,
                        logpsi, hcache, ws, ws_bytes, stream);
}

nqs_status nqs_logpsi(const nqs_model_desc* desc, const float* params, const uint8_t* sigma,
                      int64_t B, float* logpsi, float* hcache, void* ws, size_t ws_bytes,
                      void* stream) {
  return forward_common(desc, params, B, false, 0, 0, nullptr, 0, nullptr, sigma, nullptr, logpsi, hcache, ws,
                        ws_bytes, stream);
}

nqs_status nqs_local_energy(const nqs_model_desc* desc, const float* params,
                            const nqs_ham_desc* ham, const uint8_t* sigma, const float* hcache,
                            int64_t B, float* eloc, void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  nqs_status r = check_desc(desc, &d);
  if (r != NQS_OK) return r;
  if ((r = check_built(d)) != NQS_OK) return r;
  if (!ham || !params || B < 0) return NQS_EINVAL;
  if (B > 0 && (!sigma || !hcache || !eloc)) return NQS_EINVAL;
  if (misaligned(params) || misaligned(hcache)) return NQS_EINVAL;
  if (ham->kind != NQS_TFIM && ham->kind != NQS_HEISENBERG && ham->kind != NQS_LRTFIM && ham->kind != NQS_CLUSTER)
    return NQS_EINVAL;
  if (ham->kind == NQS_LRTFIM && !(ham->alpha >= 0.0)) return NQS_EINVAL;
  if ((ham->kind == NQS_TFIM || ham->kind == NQS_LRTFIM || ham->kind == NQS_CLUSTER) && d.cell != NQS_GRU1D)
    return NQS_EUNSUPPORTED;
  // the phase head is built with the cluster Hamiltonian, which runs on the FP32 path
  if (d.phase && ham->kind != NQS_CLUSTER) return NQS_EUNSUPPORTED;
  if (ham->kind == NQS_CLUSTER && d.precision != NQS_FP32) return NQS_EUNSUPPORTED;
  if (ham->kind == NQS_CLUSTER && d.N < 3) return NQS_ESHAPE;
  if (ham->kind == NQS_CLUSTER && d.d < 16) return NQS_EUNSUPPORTED;
  if (ham->kind == NQS_HEISENBERG && d.cell != NQS_GRU2D) return NQS_EUNSUPPORTED;
  if (ham->kind == NQS_HEISENBERG && (d.Lx < 2 && d.Ly < 2)) return NQS_ESHAPE;
  const Layout L = layout(d, B, NQS_OP_LOCAL_ENERGY);
  if ((r = check_ws(ws, ws_bytes, L)) != NQS_OK) return r;
  if (B == 0) return NQS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  WsHeader* hdr = static_cast<WsHeader*>(ws);
  float* img = at<float>(ws, L.img);
  if (ham->kind == NQS_CLUSTER) {
    // cRNN: eloc is [B, 2] (complex); pRNN: [B] (real ratios)
    if (gru1d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    const float* php = d.phase ? params + phase_offset(d) : nullptr;
    float* dlog = at<float>(ws, L.a);
    float* dre = at<float>(ws, L.b);
    float* zph = at<float>(ws, L.c);
    float* dim = at<float>(ws, L.e);
    if (crnn_readout(img, php, hcache, dlog, zph, B * d.N, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Fwd1Args f{};
    f.B = B;
    f.N = d.N;
    f.sigma_in = sigma;
    f.hcache = const_cast<float*>(hcache);
    f.hdr = hdr;
    return cuda_status(cluster_local_energy(f, img, php, d.phase, dlog, zph, dre, dim, eloc, &hdr->job_counter,
                                            (float)ham->J, d.d, st));
  }
  if (ham->kind == NQS_HEISENBERG) {
    const int nb = n_bonds(d);
    int4* bonds = at<int4>(ws, L.b);
    float* lp_tab = at<float>(ws, L.c);
    int* nup_tab = at<int>(ws, L.e);
    float* delta = at<float>(ws, L.f);
    const float x = ham->marshall ? -0.5f * (float)ham->J : 0.5f * (float)ham->J;
    if (use_tc2d(d)) {
      // cached-path tables from the cache with the chains' own BF16 readout,
      // then the chains over the antiparallel bonds
      uint8_t* wimg = at<uint8_t>(ws, L.w);
      if (tc2d_pack(params, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
      if (gru2d_bonds(d.Lx, d.Ly, bonds, st) != cudaSuccess) return NQS_ECUDA;
      Tc2Fwd f{};
      f.B = B;
      f.Lx = d.Lx;
      f.N = d.N;
      f.sz0 = d.sz0;
      f.sigma_in = sigma;
      f.hcache = const_cast<float*>(hcache);
      f.lp_tab = lp_tab;
      f.nup_tab = nup_tab;
      f.hdr = hdr;
      if (tc2d_tables(f, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
      Tc2Chains c{};
      c.B = B;
      c.Lx = d.Lx;
      c.N = d.N;
      c.nb = nb;
      c.sz0 = d.sz0;
      c.sigma = sigma;
      c.hcache = hcache;
      c.lp_tab = lp_tab;
      c.nup_tab = nup_tab;
      c.bonds = bonds;
      c.delta = delta;
      c.colbuf = at<float>(ws, L.a);
      c.jobs_ws = at<uint8_t>(ws, L.g);
      c.counter = &hdr->job_counter;
      c.hdr = hdr;
      if (tc2d_heis_chains(c, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
      return cuda_status(heis_eloc(sigma, bonds, delta, eloc, B, d.N, nb, (float)ham->J, x, hdr, st));
    }
    if (gru2d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    if (gru2d_bonds(d.Lx, d.Ly, bonds, st) != cudaSuccess) return NQS_ECUDA;
    if (gru2d_prep(img, hcache, sigma, lp_tab, nup_tab, B, d.Lx, d.N, d.d, d.sz0, st) != cudaSuccess)
      return NQS_ECUDA;
    if (cudaMemsetAsync(&hdr->job_counter, 0, sizeof(hdr->job_counter), st) != cudaSuccess)
      return NQS_ECUDA;
    Eng2Args c{};
    c.B = B;
    c.Lx = d.Lx;
    c.N = d.N;
    c.nbonds = nb;
    c.sz0 = d.sz0;
    c.sigma_in = sigma;
    c.hcache = const_cast<float*>(hcache);
    c.colbuf = at<float>(ws, L.a);
    c.lp_tab = lp_tab;
    c.nup_tab = nup_tab;
    c.bonds = bonds;
    c.delta = delta;
    c.counter = &hdr->job_counter;
    c.hdr = hdr;
    if (gru2d_heis_chains(c, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    return cuda_status(heis_eloc(sigma, bonds, delta, eloc, B, d.N, nb, (float)ham->J, x, hdr, st));
  }
  float* dlog = at<float>(ws, L.a);
  float* delta = at<float>(ws, L.b);
  if (gru1d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
  if (gru1d_readout(img, hcache, dlog, B * d.N, d.d, st) != cudaSuccess) return NQS_ECUDA;
  if (cudaMemsetAsync(&hdr->job_counter, 0, sizeof(hdr->job_counter), st) != cudaSuccess)
    return NQS_ECUDA;
  if (use_tc(d)) {
    uint8_t* wimg = at<uint8_t>(ws, L.w);
    if (tc1d_pack(params, wimg, d.d, st) != cudaSuccess) return NQS_ECUDA;
    Tc1Args t{};
    t.B = B;
    t.N = d.N;
    t.sigma = sigma;
    t.hcache = const_cast<float*>(hcache);
    t.dlog = dlog;
    t.delta = delta;
    t.counter = &hdr->job_counter;
    t.hdr = hdr;
    if (tc1d_run(t, img, wimg, d.d, 2, st) != cudaSuccess) return NQS_ECUDA;
  } else {
    Chain1Args c{};
    c.B = B;
    c.N = d.N;
    c.sigma = sigma;
    c.hcache = hcache;
    c.dlog = dlog;
    c.delta = delta;
    c.counter = &hdr->job_counter;
    if (gru1d_tfim_chains(c, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
  }
  if (ham->kind == NQS_LRTFIM)
    return cuda_status(lrtfim_eloc(sigma, dlog, delta, eloc, B, d.N, ham->J, ham->h, ham->alpha, hdr, st));
  return cuda_status(tfim_eloc(sigma, dlog, delta, eloc, B, d.N, (float)ham->J, (float)ham->h, hdr, st));
}


nqs_status nqs_logpsi_grad(const nqs_model_desc* desc, const float* params, const uint8_t* sigma,
                           const float* hcache, const float* weights, int64_t B, float* grad,
                           void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  nqs_status r = check_desc(desc, &d);
  if (r != NQS_OK) return r;
  if ((r = check_built(d)) != NQS_OK) return r;
  if (!params || !grad || B < 0) return NQS_EINVAL;
  if (B > 0 && (!sigma || !hcache || !weights)) return NQS_EINVAL;
  if (misaligned(params) || misaligned(hcache)) return NQS_EINVAL;
  const Layout L = layout(d, B, NQS_OP_LOGPSI_GRAD);
  if ((r = check_ws(ws, ws_bytes, L)) != NQS_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  if (B == 0) return cuda_status(cudaMemsetAsync(grad, 0, d.P * sizeof(float), st));
  return grad_common(d, L, params, sigma, hcache, weights, B, grad, ws, st);
}

nqs_status nqs_vmc_grad(const nqs_model_desc* desc, const float* params, const uint8_t* sigma,
                        const float* hcache, const float* eloc, int64_t B, float* grad,
                        double* stats, void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  nqs_status r = check_desc(desc, &d);
  if (r != NQS_OK) return r;
  if ((r = check_built(d)) != NQS_OK) return r;
  if (!params || !sigma || !hcache || !eloc || !grad || !stats || B < 1) return NQS_EINVAL;
  if (misaligned(params) || misaligned(hcache)) return NQS_EINVAL;
  const Layout L = layout(d, B, NQS_OP_VMC_GRAD);
  if ((r = check_ws(ws, ws_bytes, L)) != NQS_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  float* w = at<float>(ws, L.b);
  if (d.phase) {
    // complex local energies: stats [Re mean, variance, M, Im mean], w = 2 (E - mean) / M
    if (complex_stats_weights(eloc, B, stats, w, st) != cudaSuccess) return NQS_ECUDA;
    return grad_common(d, L, params, sigma, hcache, w, B, grad, ws, st);
  }
  if (energy_stats(eloc, B, stats, st) != cudaSuccess) return NQS_ECUDA;
  if (vmc_weights(eloc, stats, B, w, st) != cudaSuccess) return NQS_ECUDA;
  return grad_common(d, L, params, sigma, hcache, w, B, grad, ws, st);
}


nqs_status nqs_energy_sums(const float* eloc, int64_t B, double* sums, void* stream) {
  if (!sums || B < 0 || (B > 0 && !eloc)) return NQS_EINVAL;
  return cuda_status(energy_sums(eloc, B, sums, static_cast<cudaStream_t>(stream)));
}

nqs_status nqs_vmc_grad_global(const nqs_model_desc* desc, const float* params, const uint8_t* sigma,
                               const float* hcache, const float* eloc, int64_t B, const double* sums,
                               double* grad, double* stats, void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  nqs_status r = check_desc(desc, &d);
  if (r != NQS_OK) return r;
  if ((r = check_built(d)) != NQS_OK) return r;
  if (d.phase) return NQS_EUNSUPPORTED;
  if (!params || !sums || !grad || !stats || B < 0) return NQS_EINVAL;
  if (B > 0 && (!sigma || !hcache || !eloc)) return NQS_EINVAL;
  if (misaligned(params) || misaligned(hcache)) return NQS_EINVAL;
  const Layout L = layout(d, B, NQS_OP_VMC_GRAD);
  if ((r = check_ws(ws, ws_bytes, L)) != NQS_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  if (stats_from_sums(sums, stats, st) != cudaSuccess) return NQS_ECUDA;
  if (B == 0) return cuda_status(cudaMemsetAsync(grad, 0, d.P * sizeof(double), st));
  float* w = at<float>(ws, L.b);
  if (vmc_weights(eloc, stats, B, w, st) != cudaSuccess) return NQS_ECUDA;
  return grad_common(d, L, params, sigma, hcache, w, B, grad, ws, st);
}

nqs_status nqs_set_wait_limit(int64_t polls) {
  const uint32_t v = polls < 0 ? tc_default_wait_polls() : (uint32_t)(polls > 0xFFFFFFFFll ? 0xFFFFFFFFll : polls);
  if (tc1d_set_wait_polls(v) != cudaSuccess || tc2d_set_wait_polls(v) != cudaSuccess || tc2dw_set_wait_polls(v) != cudaSuccess || tc1d128_set_wait_polls(v) != cudaSuccess ||
      tc2d_grad_set_wait_polls(v) != cudaSuccess)
    return NQS_ECUDA;
  return NQS_OK;
}

// ---------------------------------------------------------------------------
// Checkpointed teacher forcing and gradient (FP32 1D GRU).
// ---------------------------------------------------------------------------
namespace {
nqs_status check_ckpt(const nqs_model_desc* desc, int64_t B, int32_t k, Dims* d) {
  nqs_status r = check_desc(desc, d);
  if (r != NQS_OK) return r;
  if ((r = check_built(*d)) != NQS_OK) return r;
  if (d->cell != NQS_GRU1D || d->precision != NQS_FP32 || d->phase) return NQS_EUNSUPPORTED;
  if (B < 0 || k < 1) return NQS_EINVAL;
  return NQS_OK;
}
int n_ckpt(const Dims& d, int32_t k) { return (d.N + k - 1) / k - 1; }
struct CkptLayout {
  size_t img, seg, ca, cb, partial, acc, total;
};
CkptLayout ckpt_layout(const Dims& d, int64_t B, int32_t k) {
  CkptLayout L{};
  size_t off = sizeof(WsHeader);
  auto take = [&](size_t bytes) { const size_t at = off; off += align256(bytes); return at; };
  L.img = take(gru1d_img_floats(d.d) * sizeof(float));
  L.seg = take((size_t)B * k * d.d * sizeof(float));          // one segment's recomputed states
  L.ca = take((size_t)B * d.d * sizeof(float));               // carries between segments
  L.cb = take((size_t)B * d.d * sizeof(float));
  L.partial = take((size_t)gru1d_bptt_grid(d.d, B) * d.P * sizeof(float));
  L.acc = take(2 * d.P * sizeof(double));
  L.total = off;
  return L;
}
}  // namespace

size_t nqs_ckpt_floats(const nqs_model_desc* desc, int64_t B, int32_t k) {
  Dims d;
  if (check_ckpt(desc, B, k, &d) != NQS_OK) return 0;
  return (size_t)B * n_ckpt(d, k) * d.d;
}

size_t nqs_ckpt_workspace_bytes(const nqs_model_desc* desc, int64_t B, int32_t k) {
  Dims d;
  if (check_ckpt(desc, B, k, &d) != NQS_OK) return 0;
  return ckpt_layout(d, B, k).total;
}

nqs_status nqs_logpsi_ckpt(const nqs_model_desc* desc, const float* params, const uint8_t* sigma, int64_t B,
                           int32_t k, float* logpsi, float* ckpt, void* ws, size_t ws_bytes, void* stream) {
  Dims d;
  nqs_status r = check_ckpt(desc, B, k, &d);
  if (r != NQS_OK) return r;
  if (!params || misaligned(params) || misaligned(ckpt)) return NQS_EINVAL;
  if (B > 0 && (!sigma || !logpsi || (n_ckpt(d, k) > 0 && !ckpt))) return NQS_EINVAL;
  const CkptLayout L = ckpt_layout(d, B, k);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < L.img + align256(gru1d_img_floats(d.d) * 4))
    return NQS_EWORKSPACE;
  if (B == 0) return NQS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  float* img = at<float>(ws, L.img);
  if (gru1d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
  Fwd1Args a{};
  a.B = B;
  a.N = d.N;
  a.sigma_in = sigma;
  a.logpsi = logpsi;
  a.hdr = static_cast<WsHeader*>(ws);
  a.ckpt = n_ckpt(d, k) > 0 ? ckpt : nullptr;
  a.ck = k;
  return cuda_status(gru1d_forward(a, img, d.d, false, st));
}

nqs_status nqs_logpsi_grad_ckpt(const nqs_model_desc* desc, const float* params, const uint8_t* sigma, int64_t B,
                                int32_t k, const float* ckpt, const float* weights, float* grad, void* ws,
                                size_t ws_bytes, void* stream) {
  Dims d;
  nqs_status r = check_ckpt(desc, B, k, &d);
  if (r != NQS_OK) return r;
  if (!params || !grad || misaligned(params) || misaligned(ckpt)) return NQS_EINVAL;
  if (B > 0 && (!sigma || !weights || (n_ckpt(d, k) > 0 && !ckpt))) return NQS_EINVAL;
  const CkptLayout L = ckpt_layout(d, B, k);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < L.total) return NQS_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  if (B == 0) return cuda_status(cudaMemsetAsync(grad, 0, d.P * sizeof(float), st));
  float* img = at<float>(ws, L.img);
  float* seg = at<float>(ws, L.seg);
  float* carry[2] = {at<float>(ws, L.ca), at<float>(ws, L.cb)};
  float* partial = at<float>(ws, L.partial);
  double* acc = at<double>(ws, L.acc);
  if (gru1d_pack(params, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
  if (cudaMemsetAsync(acc, 0, d.P * sizeof(double), st) != cudaSuccess) return NQS_ECUDA;
  const int nseg = n_ckpt(d, k) + 1;
  const int grid = gru1d_bptt_grid(d.d, B);
  const int64_t ld = (int64_t)n_ckpt(d, k) * d.d;
  for (int s = nseg - 1; s >= 0; --s) {
    const int n0 = s * k, n1 = n0 + k < d.N ? n0 + k : d.N;
    const float* h0 = s > 0 ? ckpt + (size_t)(s - 1) * d.d : nullptr;
    // (1) recompute the segment's states from its checkpoint
    Fwd1Args f{};
    f.B = B;
    f.N = d.N;
    f.sigma_in = sigma;
    f.hcache = seg;
    f.hdr = static_cast<WsHeader*>(ws);
    f.n0 = n0;
    f.n1 = n1;
    f.h_init = h0;
    f.hi_ld = ld;
    f.hc_rows = k;
    f.hc_base = n0;
    if (gru1d_forward(f, img, d.d, false, st) != cudaSuccess) return NQS_ECUDA;
    // (2) the reverse sweep over the segment, carrying dL/dh across segments
    if (cudaMemsetAsync(partial, 0, (size_t)grid * d.P * sizeof(float), st) != cudaSuccess) return NQS_ECUDA;
    Bptt1Args b{};
    b.B = B;
    b.N = d.N;
    b.P = (int)d.P;
    b.sigma = sigma;
    b.hcache = seg;
    b.weights = weights;
    b.partial = partial;
    b.n0 = n0;
    b.n1 = n1;
    b.h_init = h0;
    b.hi_ld = ld;
    b.hc_rows = k;
    b.hc_base = n0;
    b.carry_in = s == nseg - 1 ? nullptr : carry[(s + 1) & 1];
    b.carry_out = s > 0 ? carry[s & 1] : nullptr;
    if (gru1d_bptt(b, img, d.d, st) != cudaSuccess) return NQS_ECUDA;
    if (reduce_partials_acc(partial, grid, (int)d.P, acc, st) != cudaSuccess) return NQS_ECUDA;
  }
  return cuda_status(f64_to_f32(acc, grad, (int64_t)d.P, st));
}

// ---------------------------------------------------------------------------
// Training loop and final evaluation.
// ---------------------------------------------------------------------------
static bool valid_schedule(const nqs_lr_schedule* s) {
  if (!s || s->kind < NQS_LR_CONSTANT || s->kind > NQS_LR_INVERSE) return false;
  if (!(s->lr0 >= 0.0) || (s->kind == NQS_LR_STEP && !(s->lr1 >= 0.0))) return false;
  if (s->kind == NQS_LR_INVERSE && !(s->decay > 0.0)) return false;
  return s->t_switch >= 0;
}

nqs_status nqs_adam_step(const float* grad, const double* grad64, float* params, float* m, float* v, int64_t P,
                         const nqs_adam_desc* adam, const nqs_lr_schedule* sched, uint64_t t, uint64_t* t_dev,
                         void* stream) {
  if ((grad == nullptr) == (grad64 == nullptr)) return NQS_EINVAL;
  if (!params || !m || !v || P < 1 || !adam || !valid_schedule(sched)) return NQS_EINVAL;
  if (!(adam->beta1 >= 0.0 && adam->beta1 < 1.0 && adam->beta2 >= 0.0 && adam->beta2 < 1.0 && adam->eps > 0.0))
    return NQS_EINVAL;
  AdamArgs a{};
  a.beta1 = adam->beta1;
  a.beta2 = adam->beta2;
  a.eps = adam->eps;
  a.t = (int64_t)t;
  a.sched.kind = sched->kind - NQS_LR_CONSTANT;
  a.sched.lr0 = sched->lr0;
  a.sched.lr1 = sched->lr1;
  a.sched.t_switch = sched->t_switch;
  a.sched.decay = sched->decay;
  return cuda_status(adam_update(grad, grad64, params, m, v, P, a, t_dev, static_cast<cudaStream_t>(stream)));
}

nqs_status nqs_record_stats(const double* stats, double* log, int64_t cap, const uint64_t* t_dev, void* stream) {
  if (!stats || !log || cap < 1 || !t_dev) return NQS_EINVAL;
  return cuda_status(record_stats(stats, log, cap, t_dev, static_cast<cudaStream_t>(stream)));
}

namespace {
struct EvalLayout {
  size_t sums, sigma, logpsi, hcache, eloc, inner, inner_bytes, total;
};
EvalLayout eval_layout(const Dims& d, const nqs_ham_desc* ham, int64_t chunk) {
  EvalLayout L{};
  size_t off = sizeof(WsHeader);
  L.sums = off;
  off += 256;
  L.sigma = off;
  off += align256((size_t)chunk * d.N);
  L.logpsi = off;
  off += align256((size_t)chunk * sizeof(float));
  L.hcache = off;
  off += align256((size_t)chunk * d.N * d.d * sizeof(float));
  L.eloc = off;
  off += align256((size_t)chunk * sizeof(float));
  L.inner = off;
  const Layout ls = layout(d, chunk, NQS_OP_SAMPLE), le = layout(d, chunk, NQS_OP_LOCAL_ENERGY);
  L.inner_bytes = ls.total > le.total ? ls.total : le.total;
  L.total = off + L.inner_bytes;
  (void)ham;
  return L;
}
}  // namespace

size_t nqs_evaluate_workspace_bytes(const nqs_model_desc* desc, const nqs_ham_desc* ham, int64_t chunk) {
  Dims d;
  if (check_desc(desc, &d) != NQS_OK || !ham || chunk < 1) return 0;
  return eval_layout(d, ham, chunk).total;
}

nqs_status nqs_evaluate(const nqs_model_desc* desc, const float* params, const nqs_ham_desc* ham, int64_t M,
                        int64_t chunk, uint64_t seed, uint64_t step, double* stats, void* ws, size_t ws_bytes,
                        void* stream) {
  Dims d;
  nqs_status r = check_desc(desc, &d);
  if (r != NQS_OK) return r;
  if ((r = check_built(d)) != NQS_OK) return r;
  if (d.phase || ham == nullptr || ham->kind == NQS_CLUSTER) return ham ? NQS_EUNSUPPORTED : NQS_EINVAL;
  if (!params || !ham || !stats || M < 1 || chunk < 1 || (uint64_t)M > ((uint64_t)1 << 32)) return NQS_EINVAL;
  if (misaligned(params)) return NQS_EINVAL;
  if (chunk > M) chunk = M;
  const EvalLayout L = eval_layout(d, ham, chunk);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < L.total) return NQS_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  double* sums = at<double>(ws, L.sums);
  if (cudaMemsetAsync(sums, 0, 3 * sizeof(double), st) != cudaSuccess) return NQS_ECUDA;
  uint8_t* sigma = at<uint8_t>(ws, L.sigma);
  float* logpsi = at<float>(ws, L.logpsi);
  float* hcache = at<float>(ws, L.hcache);
  float* eloc = at<float>(ws, L.eloc);
  void* inner = at<void>(ws, L.inner);
  for (int64_t off = 0; off < M; off += chunk) {
    const int64_t B = M - off < chunk ? M - off : chunk;
    if ((r = nqs_sample(desc, params, B, seed, step, nullptr, (uint64_t)off, nullptr, sigma, logpsi, hcache, inner,
                        L.inner_bytes, stream)) != NQS_OK)
      return r;
    if (status_merge(static_cast<const WsHeader*>(inner), static_cast<WsHeader*>(ws), st) != cudaSuccess)
      return NQS_ECUDA;
    if ((r = nqs_local_energy(desc, params, ham, sigma, hcache, B, eloc, inner, L.inner_bytes, stream)) != NQS_OK)
      return r;
    if (status_merge(static_cast<const WsHeader*>(inner), static_cast<WsHeader*>(ws), st) != cudaSuccess)
      return NQS_ECUDA;
    if (energy_sums_acc(eloc, B, sums, st) != cudaSuccess) return NQS_ECUDA;
  }
  return cuda_status(eval_stats(sums, stats, st));
}

// ---------------------------------------------------------------------------
// Batched step over replicas.
// ---------------------------------------------------------------------------
static nqs_status check_replicas(int R, const nqs_replica* reps, Dims* dims) {
  if (R < 1 || R > NQS_MAX_REPLICAS || !reps) return NQS_EINVAL;
  for (int i = 0; i < R; ++i) {
    const nqs_replica& r = reps[i];
    nqs_status s = check_desc(&r.desc, &dims[i]);
    if (s != NQS_OK) return s;
    if (dims[i].cell != NQS_GRU1D || dims[i].sz0 || dims[i].phase) return NQS_EUNSUPPORTED;
    if (dims[i].precision == NQS_FP32 ? !batched_supported_d(dims[i].d) : !tc1d_supported(dims[i].d))
      return NQS_EUNSUPPORTED;
    if (r.ham.kind != NQS_TFIM)
      return r.ham.kind == NQS_HEISENBERG || r.ham.kind == NQS_LRTFIM ? NQS_EUNSUPPORTED : NQS_EINVAL;
    if (r.B < 1) return NQS_EINVAL;
  }
  return NQS_OK;
}

// FP32 replicas run as grouped launches over all of them (their counters and
// partial rows contiguous, in replica order); BF16 replicas run the
// tensor-core calls of one model each, one after the other, in a shared
// inner workspace.
struct BatchLayout {
  size_t counters, img[NQS_MAX_REPLICAS], dlog[NQS_MAX_REPLICAS], delta[NQS_MAX_REPLICAS],
      w[NQS_MAX_REPLICAS], partial[NQS_MAX_REPLICAS], inner, inner_bytes, total;
};

static BatchLayout batch_layout(int R, const nqs_replica* reps, const Dims* dims) {
  BatchLayout L{};
  size_t off = sizeof(WsHeader);
  L.counters = off;
  off += align256((size_t)R * sizeof(unsigned long long));
  for (int i = 0; i < R; ++i) {
    if (dims[i].precision != NQS_FP32) continue;
    const size_t BN = (size_t)reps[i].B * dims[i].N;
    L.img[i] = off; off += align256(gru1d_img_floats(dims[i].d) * sizeof(float));
    L.dlog[i] = off; off += align256(BN * sizeof(float));
    L.delta[i] = off; off += align256(BN * sizeof(float));
    L.w[i] = off; off += align256((size_t)reps[i].B * sizeof(float));
  }
  for (int i = 0; i < R; ++i) {   // contiguous, first FP32 replica first
    if (dims[i].precision != NQS_FP32) continue;
    L.partial[i] = off;
    off += align256((size_t)batched_bptt_blocks(dims[i].d, reps[i].B) * dims[i].P * sizeof(float));
  }
  for (int i = 0; i < R; ++i) {
    if (dims[i].precision == NQS_FP32) continue;
    for (int op : {NQS_OP_SAMPLE, NQS_OP_LOCAL_ENERGY, NQS_OP_VMC_GRAD}) {
      const size_t b = layout(dims[i], reps[i].B, op).total;
      if (b > L.inner_bytes) L.inner_bytes = b;
    }
  }
  L.inner = off;
  off += align256(L.inner_bytes);
  L.total = off;
  return L;
}

size_t nqs_vmc_step_batched_workspace_bytes(int R, const nqs_replica* reps) {
  Dims dims[NQS_MAX_REPLICAS];
  if (check_replicas(R, reps, dims) != NQS_OK) return 0;
  return batch_layout(R, reps, dims).total;
}

nqs_status nqs_vmc_step_batched(int R, const nqs_replica* reps, uint64_t step, uint64_t* step_dev,
                                void* ws, size_t ws_bytes, void* stream) {
  Dims dims[NQS_MAX_REPLICAS];
  nqs_status r = check_replicas(R, reps, dims);
  if (r != NQS_OK) return r;
  for (int i = 0; i < R; ++i) {
    const nqs_replica& p = reps[i];
    if (!p.params || !p.sigma || !p.logpsi || !p.hcache || !p.eloc || !p.grad || !p.stats) return NQS_EINVAL;
    if (misaligned(p.params) || misaligned(p.hcache)) return NQS_EINVAL;
  }
  const BatchLayout L = batch_layout(R, reps, dims);
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 || ws_bytes < L.total) return NQS_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!reset_status(ws, st)) return NQS_ECUDA;
  // BF16 replicas first (they read the step before the grouped launches advance it)
  void* inner = at<void>(ws, L.inner);
  WsHeader* hdr = static_cast<WsHeader*>(ws);
  int nf = 0;
  for (int i = 0; i < R; ++i) {
    const nqs_replica& p = reps[i];
    if (dims[i].precision == NQS_FP32) {
      ++nf;
      continue;
    }
    if ((r = nqs_sample(&p.desc, p.params, p.B, p.seed, step, step_dev, 0, nullptr, p.sigma, p.logpsi, p.hcache,
                        inner, L.inner_bytes, stream)) != NQS_OK)
      return r;
    if (status_merge(static_cast<const WsHeader*>(inner), hdr, st) != cudaSuccess) return NQS_ECUDA;
    if ((r = nqs_local_energy(&p.desc, p.params, &p.ham, p.sigma, p.hcache, p.B, p.eloc, inner, L.inner_bytes,
                              stream)) != NQS_OK)
      return r;
    if (status_merge(static_cast<const WsHeader*>(inner), hdr, st) != cudaSuccess) return NQS_ECUDA;
    if ((r = nqs_vmc_grad(&p.desc, p.params, p.sigma, p.hcache, p.eloc, p.B, p.grad, p.stats, inner,
                          L.inner_bytes, stream)) != NQS_OK)
      return r;
    if (status_merge(static_cast<const WsHeader*>(inner), hdr, st) != cudaSuccess) return NQS_ECUDA;
  }
  if (nf == 0) return step_dev ? cuda_status(step_increment(step_dev, st)) : NQS_OK;
  BatchRep br[NQS_MAX_REPLICAS];
  int nb = 0;
  for (int i = 0; i < R; ++i) {
    const nqs_replica& p = reps[i];
    if (dims[i].precision != NQS_FP32) continue;
    BatchRep& b = br[nb++];
    b.d = dims[i].d;
    b.N = dims[i].N;
    b.P = (int)dims[i].P;
    b.B = p.B;
    b.seed = p.seed;
    b.J = (float)p.ham.J;
    b.Gamma = (float)p.ham.h;
    b.params = p.params;
    b.img = at<float>(ws, L.img[i]);
    b.sigma = p.sigma;
    b.logpsi = p.logpsi;
    b.hcache = p.hcache;
    b.eloc = p.eloc;
    b.grad = p.grad;
    b.stats = p.stats;
    b.dlog = at<float>(ws, L.dlog[i]);
    b.delta = at<float>(ws, L.delta[i]);
    b.partial = at<float>(ws, L.partial[i]);
    b.w = at<float>(ws, L.w[i]);
    b.counter = at<unsigned long long>(ws, L.counters) + (nb - 1);
  }
  return cuda_status(batched_step(br, nb, step, step_dev, step_dev, st));
}

}  // extern "C"

// nqs_local_energy_static: the local-energy call for callers that cannot
// allocate device memory.  Its scratch (packed weights, per-site logit
// differences, per-flip log-amplitude ratios and the work-queue counter) lives
// in one fixed device array of this library instead of a caller workspace.
#include <mutex>

#include "kernels.h"

namespace nqs {
namespace {

constexpr size_t kStaticScratchBytes = NQS_STATIC_SCRATCH_BYTES;

// Every GPU that loads the library holds this array until the process exits.
// Its name is a host-side stand-in in host code: only the address returned by
// cudaGetSymbolAddress (per device) may be handed to a kernel.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
nqs_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NQS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return NQS_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return NQS_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return NQS_OK;
}

}  // namespace
}  // namespace nqs

using namespace nqs;

extern "C" nqs_status nqs_local_energy_static(const nqs_model_desc* desc, const float* params,
                                              const nqs_ham_desc* ham, const uint8_t* sigma,
                                              const float* hcache, int64_t B, float* eloc,
                                              void* stream) {
  // a bad descriptor gets the status nqs_local_energy gives it; a valid one
  // outside this call's single path gets NQS_EUNSUPPORTED
  const nqs_status ds = desc_status(desc);
  if (ds != NQS_OK) return ds;
  if (!ham || !params || B < 0) return NQS_EINVAL;
  if (ham->kind != NQS_TFIM && ham->kind != NQS_HEISENBERG && ham->kind != NQS_LRTFIM) return NQS_EINVAL;
  if (desc->cell != NQS_GRU1D || desc->precision != NQS_FP32 || desc->sz0 != 0 || desc->phase != 0 ||
      ham->kind != NQS_TFIM)
    return NQS_EUNSUPPORTED;
  const int D = desc->d_h, N = desc->Lx;
  if (B > 0 && (!sigma || !hcache || !eloc)) return NQS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(params) | reinterpret_cast<uintptr_t>(hcache)) & 15) return NQS_EINVAL;
  // scratch layout: [header | packed weights | dlog B*N | delta B*N]
  const size_t img_off = sizeof(WsHeader);
  const size_t dlog_off = img_off + align256(gru1d_img_floats(D) * sizeof(float));
  const size_t bn_bytes = align256((size_t)B * (size_t)N * sizeof(float));
  const size_t delta_off = dlog_off + bn_bytes;
  if ((size_t)B > ((size_t)1 << 40) / (size_t)N || delta_off + bn_bytes > kStaticScratchBytes)
    return NQS_EWORKSPACE;
  if (B == 0) return NQS_OK;
  void* base = nullptr;
  nqs_status r = scratch_address(&base);
  if (r != NQS_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* hdr = static_cast<WsHeader*>(base);
  char* b = static_cast<char*>(base);
  float* img = reinterpret_cast<float*>(b + img_off);
  float* dlog = reinterpret_cast<float*>(b + dlog_off);
  float* delta = reinterpret_cast<float*>(b + delta_off);
  // the array keeps the previous call's contents: reset the status word and the queue counter
  if (cudaMemsetAsync(hdr, 0, 16, st) != cudaSuccess) return NQS_ECUDA;
  if (gru1d_pack(params, img, D, st) != cudaSuccess) return NQS_ECUDA;
  if (gru1d_readout(img, hcache, dlog, B * N, D, st) != cudaSuccess) return NQS_ECUDA;
  Chain1Args c{};
  c.B = B;
  c.N = N;
  c.sigma = sigma;
  c.hcache = hcache;
  c.dlog = dlog;
  c.delta = delta;
  c.counter = &hdr->job_counter;
  if (gru1d_tfim_chains(c, img, D, st) != cudaSuccess) return NQS_ECUDA;
  // no status word is reported by this call (the caller cannot read the
  // array), so the energy kernel gets none: a non-finite energy is only seen
  // in eloc itself
  return tfim_eloc(sigma, dlog, delta, eloc, B, N, (float)ham->J, (float)ham->h, nullptr, st) == cudaSuccess
             ? NQS_OK
             : NQS_ECUDA;
}

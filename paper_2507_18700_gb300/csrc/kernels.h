// Internal launcher interface between the C-ABI layer (api.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace nqs {

// NQS_OK for a valid model descriptor, else the status every workspace call
// returns for it (api.cu).
nqs_status desc_status(const nqs_model_desc* desc);

struct Fwd1Args {
  int64_t B;
  int N;
  const uint8_t* sigma_in;   // teacher forcing
  uint8_t* sigma_out;        // sampling
  const float* uniforms;     // sampling, nullable
  uint64_t seed, step;
  uint64_t b0;               // sampling: global index of sample 0 (Philox counter offset)
  const uint64_t* step_dev;  // sampling: device Philox step (read on the device) or null: step
  float* logpsi;             // nullable for a segment (n0 > 0 or n1 < N)
  float* hcache;             // nullable
  WsHeader* hdr;
  // segments (FP32 1D teacher forcing, checkpointed gradient); zero = whole chain
  int n0, n1;                // sites [n0, n1) of this call (n1 = 0: N)
  const float* h_init;       // h_{n0-1} of sample b at h_init + b * hi_ld (n0 > 0)
  int64_t hi_ld;             // floats between samples in h_init (0: d)
  int hc_rows, hc_base;      // cache row of site n: b * hc_rows + n - hc_base (hc_rows = 0: N)
  float* ckpt;               // nullable: h_{(j+1) ck - 1} -> ckpt[b, j], j < ceil(N / ck) - 1
  int ck;
};

struct Chain1Args {
  int64_t B;
  int N;
  const uint8_t* sigma;
  const float* hcache;
  const float* dlog;         // [B, N] logit differences of the sampled path
  float* delta;              // [B, N] log-amplitude ratio per flipped site
  unsigned long long* counter;
};

struct Bptt1Args {
  int64_t B;
  int N;
  int P;
  const uint8_t* sigma;
  const float* hcache;
  const float* weights;      // [B] dL/dlogpsi
  float* partial;            // [grid, P]
  // segments (checkpointed gradient); zero = whole chain
  int n0, n1;                // sites [n0, n1) (n1 = 0: N)
  const float* h_init;       // h_{n0-1} of sample b at h_init + b * hi_ld (n0 > 0)
  int64_t hi_ld;
  int hc_rows, hc_base;      // cache row of site n: b * hc_rows + n - hc_base (hc_rows = 0: N)
  const float* carry_in;     // [B, d] dL/dh_{n1-1} from the later sites, or null
  float* carry_out;          // [B, d] dL/dh_{n0-1} (n0 > 0), or null
};

int gru1d_supported(int D);
size_t gru1d_img_floats(int D);
int gru1d_bptt_grid(int D, int64_t B);
cudaError_t gru1d_pack(const float* params, float* img, int D, cudaStream_t st);
cudaError_t gru1d_forward(const Fwd1Args& a, const float* img, int D, bool sample, cudaStream_t st);
cudaError_t gru1d_readout(const float* img, const float* hcache, float* dlog, int64_t rows, int D,
                          cudaStream_t st);
cudaError_t gru1d_tfim_chains(const Chain1Args& a, const float* img, int D, cudaStream_t st);
cudaError_t tfim_eloc(const uint8_t* sigma, const float* dlog, const float* delta, float* eloc,
                      int64_t B, int N, float J, float Gamma, WsHeader* hdr, cudaStream_t st);
// long-range TFIM energies (FP64 diagonal) from the same chain outputs
cudaError_t lrtfim_eloc(const uint8_t* sigma, const float* dlog, const float* delta, float* eloc, int64_t B,
                        int N, double J, double Gamma, double alpha, WsHeader* hdr, cudaStream_t st);
cudaError_t gru1d_bptt(const Bptt1Args& a, const float* img, int D, cudaStream_t st);
// acc[p] += sum of the partial rows (FP64), for gradients accumulated over
// segments; acc has 2 P doubles (the second half is scratch)
cudaError_t reduce_partials_acc(const float* partial, int rows, int P, double* acc, cudaStream_t st);
cudaError_t f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t st);

struct Eng2Args {
  int64_t B;
  int Lx, N, nbonds, sz0;
  const uint8_t* sigma_in;   // teacher forcing / chains
  uint8_t* sigma_out;        // sampling
  const float* uniforms;     // sampling, nullable
  uint64_t seed, step;
  uint64_t b0;               // sampling: global index of sample 0 (Philox counter offset)
  const uint64_t* step_dev;  // sampling: device Philox step (read on the device) or null: step
  float* logpsi;             // sampling / teacher forcing
  float* hcache;             // written by sampling / teacher forcing, read by chains
  float* colbuf;             // [slots, Lx, d] column buffers
  const float* lp_tab;       // chains: [B, N, 2] masked log p of both outcomes on the cached path
  const int* nup_tab;        // chains: [B, N] up spins before each position
  const int4* bonds;         // chains: sorted bond table
  float* delta;              // chains: [B, nbonds]
  unsigned long long* counter;
  WsHeader* hdr;
};

struct Bptt2Args {
  int64_t B;
  int Lx, N, P, sz0;
  const uint8_t* sigma;
  const float* hcache;
  const float* weights;
  float* ccarry;             // [B, Lx, d] vertical carries
  float* partial;            // [grid, P]
  float* sacc;               // large d_h: [grid, row groups, 14, d] small-gradient scratch (zeroed)
};

// BF16 tensor-core 2D path (tc2d.cu)
struct Tc2Fwd {
  int64_t B;
  int Lx, N, sz0;
  const uint8_t* sigma_in;   // teacher forcing
  uint8_t* sigma_out;        // sampling
  const float* uniforms;     // nullable
  uint64_t seed, step;
  uint64_t b0;               // sampling: global index of sample 0 (Philox counter offset)
  const uint64_t* step_dev;  // sampling: device Philox step (read on the device) or null: step
  float* logpsi;             // nullable in teacher forcing
  float* hcache;             // nullable
  float* colbuf;             // tc2d_colbuf_floats(B, Lx, d)
  float* lp_tab;             // tables: [B, N, 2] masked log p of both outcomes
  int* nup_tab;              // tables: [B, N] up spins before each position
  WsHeader* hdr;
};
struct Tc2Chains {
  int64_t B;
  int Lx, N, nb, sz0;
  const uint8_t* sigma;
  const float* hcache;
  const float* lp_tab;
  const int* nup_tab;
  const int4* bonds;
  float* delta;              // [B, nb]
  float* colbuf;             // tc2d_colbuf_floats(B, Lx, d)
  uint8_t* jobs_ws;          // tc2d_jobs_bytes(B, nb, N, d)
  unsigned long long* counter;
  WsHeader* hdr;
};
int tc2d_supported(int D, int Lx, int N);
size_t tc2d_wimg_bytes(int D);
size_t tc2d_jobs_bytes(int64_t B, int nb, int N, int D);
size_t tc2d_colbuf_floats(int64_t B, int Lx, int D);
cudaError_t tc2d_pack(const float* params, uint8_t* wimg, int D, cudaStream_t st);
cudaError_t tc2d_forward(const Tc2Fwd& f, const uint8_t* wimg, int D, bool sample, cudaStream_t st);
// cached-path tables (lp_tab, nup_tab) from sigma_in and hcache of f, all cells in parallel
cudaError_t tc2d_tables(const Tc2Fwd& f, const uint8_t* wimg, int D, cudaStream_t st);
cudaError_t tc2d_heis_chains(const Tc2Chains& c, const uint8_t* wimg, int D, cudaStream_t st);
// d_h = 256 (tc2d_wide.cu), reached through the tc2d_* calls above: the
// weights stream from global memory through a shared-memory ring; the image
// has the same size as tc2d_wimg_bytes(256) in another layout
cudaError_t tc2dw_pack(const float* params, uint8_t* wimg, cudaStream_t st);
cudaError_t tc2dw_forward(const Tc2Fwd& f, const uint8_t* wimg, bool sample, cudaStream_t st);
cudaError_t tc2dw_tables(const Tc2Fwd& f, const uint8_t* wimg, cudaStream_t st);
cudaError_t tc2dw_chains(const Tc2Chains& c, const uint8_t* wimg, const uint8_t* jobs, const int* njobs, cudaStream_t st);
cudaError_t tc2dw_set_wait_polls(uint32_t polls);
// d_h = 256 BF16 reverse sweep (tc2d_wide.cu): tape pass, sequential sweep,
// weight-gradient GEMMs, readout gradients; writes grad [P] directly
struct Tc2WGrad {
  int64_t B;
  int Lx, N, sz0;
  const uint8_t* sigma;
  const float* hcache;
  const float* weights;      // [B] w_b of sum_b w_b log psi_b
  const float* params;
  uint8_t* scratch;          // tc2dw_grad_bytes(B, Lx, N, seg), 256-byte aligned
  WsHeader* hdr;
  int seg;                   // positions per pass of the reverse sweep (<= 0 or >= N: one pass)
};
size_t tc2dw_grad_bytes(int64_t B, int Lx, int N, int seg);
// d_h = 128 BF16 reverse sweep of the 1D GRU (tc1d_grad128.cu): tape pass,
// sequential sweep, weight-gradient GEMMs, readout gradients; writes grad [P]
struct Tc1WGrad {
  int64_t B;
  int N;
  const uint8_t* sigma;
  const float* hcache;
  const float* weights;      // [B] w_b of sum_b w_b log psi_b
  const float* params;
  uint8_t* scratch;          // tc1d128_grad_bytes(B, N), 256-byte aligned
  WsHeader* hdr;
};
size_t tc1d128_grad_bytes(int64_t B, int N);
cudaError_t tc1d128_grad(const Tc1WGrad& g, const uint8_t* wimg, float* grad, cudaStream_t st);
cudaError_t tc1d128_set_wait_polls(uint32_t polls);
cudaError_t tc2dw_grad(const Tc2WGrad& g, const uint8_t* wimg, float* grad, cudaStream_t st);

// BF16 tensor-core 2D reverse sweep (tc2d_grad.cu)
struct Tc2Grad {
  int64_t B;
  int Lx, Ly, N, P, sz0;
  const uint8_t* sigma;
  const float* hcache;
  const float* weights;
  float* ccarry;             // [B, Lx, d] vertical carries
  uint8_t* g1img;            // tc2d_grad_image_bytes(.., 0)
  uint8_t* g2img;            // tc2d_grad_image_bytes(.., 1)
  float* yimg;               // tc2d_grad_image_bytes(.., 2)
  float* dzimg;              // tc2d_grad_image_bytes(.., 3)
  float* tape_h;             // tc2d_grad_image_bytes(.., 4)
  uint8_t* tape_k;           // tc2d_grad_image_bytes(.., 5)
  float* partial;            // [tc2d_grad_partial_rows(B, N), P], zeroed
  WsHeader* hdr;
};
int tc2d_wgrad_grid(int64_t B, int N);
int tc2d_grad_partial_rows(int64_t B, int N);
size_t tc2d_grad_image_bytes(int64_t B, int N, int D, int which);
cudaError_t tc2d_grad(const Tc2Grad& g, const uint8_t* wimg, int D, cudaStream_t st);

size_t gru2d_img_floats(int D);
int gru2d_supported(int D);
size_t gru2d_bptt_scratch_floats(int D, int64_t B);
int64_t gru2d_engine_slots(int D, int64_t B, int mode);
int gru2d_bptt_grid(int D, int64_t B);
cudaError_t gru2d_pack(const float* params, float* img, int D, cudaStream_t st);
cudaError_t gru2d_forward(const Eng2Args& a, const float* img, int D, bool sample, cudaStream_t st);
cudaError_t gru2d_bonds(int Lx, int Ly, int4* bonds, cudaStream_t st);
cudaError_t gru2d_prep(const float* img, const float* hcache, const uint8_t* sigma, float* lp_tab,
                       int* nup_tab, int64_t B, int Lx, int N, int D, int sz0, cudaStream_t st);
cudaError_t gru2d_heis_chains(const Eng2Args& a, const float* img, int D, cudaStream_t st);
cudaError_t heis_eloc(const uint8_t* sigma, const int4* bonds, const float* delta, float* eloc, int64_t B,
                      int N, int nb, float J, float x, WsHeader* hdr, cudaStream_t st);
cudaError_t gru2d_bptt(const Bptt2Args& a, const float* img, int D, cudaStream_t st);

struct Tc1Args {
  int64_t B;
  int N;
  const uint8_t* sigma;      // teacher forcing / chains
  uint8_t* sigma_out;        // sampling
  const float* uniforms;     // sampling, nullable
  uint64_t seed, step;
  uint64_t b0;               // sampling: global index of sample 0 (Philox counter offset)
  const uint64_t* step_dev;  // sampling: device Philox step (read on the device) or null: step
  float* logpsi;
  float* hcache;             // written by sampling / teacher forcing (nullable), read by chains
  const float* dlog;         // chains
  float* delta;              // chains
  unsigned long long* counter;
  WsHeader* hdr;
  int rows;                  // sampling / teacher forcing: rows per 128-lane tile (128, 64 or 32; set by the launcher)
};

struct TcBpttArgs {
  int64_t B;
  int N, P;
  const uint8_t* sigma;
  const float* hcache;
  const float* weights;
  float* partial;            // [tc1d_bptt_partial_rows(B), P], zeroed
  float* tape_e;             // [B, N] onehot_0(s_n) - p_0(h_n)
  uint8_t* tape_x;           // [B, N, d] bf16 h_{n-1}
  uint8_t* tape_k;           // [B, N, 5, d] fp16 cell-backward factors
  WsHeader* hdr;
};

int tc1d_supported(int D);
void tc1d_set_autotune(int on);
void tc1d_set_variant(int v);
int tc1d_pinned_variant();   // the pinned tile variant, -1 if none
int tc1d_bptt_partial_rows(int64_t B);
size_t tc1d_tape_bytes(int64_t B, int N, int D, int which);   // which: 0 e, 1 x, 2 k
cudaError_t tc1d_pack_t(const float* params, uint8_t* wt, int D, cudaStream_t st);
cudaError_t tc1d_bptt(const TcBpttArgs& a, const float* img, const uint8_t* w3, const uint8_t* wt, int D,
                      cudaStream_t st);
// grad = the FP64 sum of the partial rows tc1d_bptt wrote
cudaError_t tc1d_bptt_reduce(const TcBpttArgs& a, int D, float* grad, cudaStream_t st);
cudaError_t tc1d_bptt_reduce(const TcBpttArgs& a, int D, double* grad, cudaStream_t st);
size_t tc1d_wimg_bytes(int D);
cudaError_t tc1d_pack(const float* params, uint8_t* wimg, int D, cudaStream_t st);
// mode 0: sampling, 1: teacher forcing, 2: TFIM chains
cudaError_t tc1d_run(const Tc1Args& a, const float* img, const uint8_t* wimg, int D, int mode, cudaStream_t st);

// grouped multi-replica step (batched.cu)
struct BatchRep {
  int d, N, P;
  int64_t B;
  uint64_t seed;
  float J, Gamma;
  const float* params;
  float* img;
  uint8_t* sigma;
  float* logpsi;
  float* hcache;
  float* eloc;
  float* grad;
  double* stats;
  float* dlog;
  float* delta;
  float* partial;   // replicas' partials are contiguous, replica 0 first
  float* w;
  unsigned long long* counter;   // replicas' counters are contiguous, replica 0 first
};
bool batched_supported_d(int d);
int batched_bptt_blocks(int d, int64_t B);
cudaError_t batched_step(const BatchRep* reps, int R, uint64_t step, const uint64_t* step_dev, uint64_t* step_inc,
                         cudaStream_t st);

// reductions (reduce.cu)
cudaError_t energy_stats(const float* eloc, int64_t B, double* stats, cudaStream_t st);
cudaError_t vmc_weights(const float* eloc, const double* stats, int64_t B, float* w, cudaStream_t st);
// sums = [sum E, sum E^2, B] of one rank; stats = [mean, variance, M] from the sums of all ranks
cudaError_t energy_sums(const float* eloc, int64_t B, double* sums, cudaStream_t st);
cudaError_t stats_from_sums(const double* sums, double* stats, cudaStream_t st);
cudaError_t reduce_partials(const float* partial, int rows, int P, float* grad, cudaStream_t st);
cudaError_t reduce_partials(const float* partial, int rows, int P, double* grad, cudaStream_t st);
// grad[0 .. ncols) = FP64 sum over `rows` rows (stride ld floats) of partial
cudaError_t reduce_partials_cols(const float* partial, int rows, int ncols, int64_t ld, float* grad,
                                 cudaStream_t st);
cudaError_t reduce_partials_cols(const float* partial, int rows, int ncols, int64_t ld, double* grad,
                                 cudaStream_t st);

// cRNN (phase head) and the cluster Hamiltonian on the FP32 1D path (crnn.cu);
// phase_params points at [U_phi | c_phi] after the amplitude parameters;
// logpsi2, eloc and weights2 are [B, 2] float pairs (real, imaginary)
int crnn_bptt_grid(int64_t B, int D);
cudaError_t crnn_forward(const Fwd1Args& a, const float* img, const float* phase_params, float* logpsi2, int D,
                         bool sample, cudaStream_t st);
// dlog [rows] and, when phase_params is non-null, the phase logits zph [rows, 2]
cudaError_t crnn_readout(const float* img, const float* phase_params, const float* hcache, float* dlog, float* zph,
                         int64_t rows, int D, cudaStream_t st);
// chains and energies of the cluster Hamiltonian (f: B, N, sigma_in, hcache, hdr)
cudaError_t cluster_local_energy(const Fwd1Args& f, const float* img, const float* phase_params, int phase,
                                 const float* dlog, const float* zph, float* dre, float* dim, float* eloc,
                                 unsigned long long* counter, float J, int D, cudaStream_t st);
// stats = [Re mean, mean |E - mean|^2, M, Im mean] and w = 2 (E - mean) / M (nullable)
cudaError_t complex_stats_weights(const float* eloc, int64_t B, double* stats, float* w, cudaStream_t st);
cudaError_t crnn_bptt(const Bptt1Args& a, const float* img, const float* phase_params, const float* weights2, int D,
                      cudaStream_t st);

// training loop and final evaluation (train.cu)
struct LrSchedule {
  int kind;            // 0 constant, 1 step at t_switch, 2 inverse decay from t_switch
  double lr0, lr1;
  int64_t t_switch;
  double decay;
};
struct AdamArgs {
  double beta1, beta2, eps;
  int64_t t;           // step when no device counter is given
  LrSchedule sched;
};
// Adam update from grad32 or grad64 (one of them non-null); t_dev (nullable)
// holds the step and is incremented after the update
cudaError_t adam_update(const float* grad32, const double* grad64, float* params, float* m, float* v, int64_t P,
                        const AdamArgs& a, uint64_t* t_dev, cudaStream_t st);
cudaError_t record_stats(const double* stats, double* log, int64_t cap, const uint64_t* t_dev, cudaStream_t st);
cudaError_t step_increment(uint64_t* t_dev, cudaStream_t st);
cudaError_t energy_sums_acc(const float* eloc, int64_t B, double* sums, cudaStream_t st);
cudaError_t eval_stats(const double* sums, double* stats, cudaStream_t st);
cudaError_t status_merge(const WsHeader* from, WsHeader* into, cudaStream_t st);

// bound of the tensor-core waits that may give up, per translation unit
uint32_t tc_default_wait_polls();
cudaError_t tc1d_set_wait_polls(uint32_t polls);
cudaError_t tc2d_set_wait_polls(uint32_t polls);
cudaError_t tc2d_grad_set_wait_polls(uint32_t polls);

// growth (grow.cu)
cudaError_t grow_params(int cell, int phase, int d, int m, int D, int Mm, const float* p_small, float* p_big,
                        uint64_t seed, float eps, cudaStream_t st);

}  // namespace nqs

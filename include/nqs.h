/*
 * libnqs -- C ABI of the GB300 (sm_103a) hot path of variational Monte Carlo
 * with recurrent-neural-network wave functions ("Adaptive Neural Quantum
 * States: A Recurrent Neural Network Perspective", arXiv 2507.18700).
 *
 * The library evaluates, for one set of RNN weights, the per-step work of VMC:
 * autoregressive sampling, teacher-forced log psi, local energies with
 * prefix-cached connected configurations, the VMC gradient (a hand-written
 * reverse sweep) and the hidden-dimension growth step.
 *
 * Conventions used by every call
 * ------------------------------
 * - Spins sigma in {0, 1}; 0 is spin up (sigma^z = +1).  The one-hot input of
 *   a spin is e_sigma and "no input" (the first site; a 2D neighbour outside
 *   the lattice) is the zero vector, with h = 0 (Sec. II, Eq. 2).
 * - Configurations are uint8 arrays [B, N] in lattice order: index j*Lx + i
 *   for column i, row j (1D: Ly = 1).
 * - Sampling order: 1D left to right; 2D zig-zag, row 0 left to right, odd
 *   rows right to left; the 2D cell reads the horizontal neighbour
 *   i - (-1)^j of its own row and the vertical neighbour (i, j-1)
 *   (Sec. II and Fig. 1(b)).
 * - log psi = 1/2 sum_n log p_n(sigma_n): positive RNN wave function, psi =
 *   sqrt(P) (Sec. II), with the two-outcome softmax of Eq. (3).
 * - Optional zero-magnetisation mask (sz0): once N/2 spins of the prefix are
 *   up the remaining ones are down with probability 1, and vice versa.
 *
 * Flat float32 parameter layout (row-major tensors, in this order)
 * ----------------------------------------------------------------
 * NQS_GRU1D (App. A, 1D GRU), d = d_h:
 *   W_g[d, d+2]  W_r[d, d+2]  W_h[d, d]  W_in[d, 2]
 *   b_g[d]  b_r[d]  b_h[d]  b_in[d]  U[2, d]  c[2]
 *   and, for a cRNN (phase = 1), U_phi[2, d]  c_phi[2]
 *   (columns of W_g, W_r: [h_{n-1} | one-hot sigma_{n-1}])
 *   u = sigmoid(W_g[h;s] + b_g), r = sigmoid(W_r[h;s] + b_r),
 *   h~ = tanh(r * (W_h h + b_h) + W_in s + b_in), h' = (1 - u) h + u h~.
 * NQS_GRU2D (App. A, 2D GRU with GLU head), d = d_h, m = d_model:
 *   W[d, 2d+4]  W_g[d, 2d+4]  U_mix[d, 2d]  b[d]  b_g[d]
 *   W_1[m, d]  b_1[m]  W_2[m, d]  b_2[m]  U_out[2, m]  c[2]
 *   (columns of W, W_g: [h_hor | h_ver | s_hor | s_ver])
 *   h~ = tanh(W[h';s'] + b), u = sigmoid(W_g[h';s'] + b_g),
 *   h = u h~ + (1 - u) U_mix h', y = (W_1 h + b_1) * sigmoid(W_2 h + b_2),
 *   logits = U_out y + c.
 *
 * Ownership, streams and errors
 * -----------------------------
 * - The caller owns every buffer: params, inputs, outputs and the workspace
 *   (size from nqs_workspace_bytes, 256-byte aligned).  Pointers named
 *   "device" must be device (or managed) memory of the current device.
 *   params and hcache are accessed in 16-byte pieces and must be 16-byte
 *   aligned (NQS_EINVAL otherwise).  The library allocates no memory.
 * - Every call only enqueues work on `stream` (a cudaStream_t; NULL is the
 *   legacy default stream) and returns; results are ready when the stream is.
 * - Arguments are checked on the host before anything is enqueued; a bad
 *   argument returns an error and enqueues nothing.  The library never aborts.
 * - A kernel that meets a non-finite log psi or local energy records
 *   NQS_ENONFINITE, and a tensor-core wait that gives up records
 *   NQS_ETIMEOUT, in the workspace status word (the first int32 of the
 *   workspace).  Every call clears that word when it starts, so after the
 *   call's work has drained nqs_workspace_status returns what that call
 *   recorded.
 */
#ifndef NQS_H
#define NQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NQS_OK = 0,
  NQS_EINVAL = 1,        /* null pointer, bad enum, bad size */
  NQS_ESHAPE = 2,        /* unsupported lattice / hidden size combination */
  NQS_EWORKSPACE = 3,    /* workspace missing, misaligned or too small */
  NQS_ECUDA = 4,         /* a CUDA runtime call failed */
  NQS_ETIMEOUT = 5,      /* a device wait gave up (recorded in the workspace) */
  NQS_ENONFINITE = 6,    /* non-finite value met on the device (workspace) */
  NQS_EUNSUPPORTED = 7   /* valid but not built (e.g. model/Hamiltonian pair) */
} nqs_status;

enum { NQS_GRU1D = 1, NQS_GRU2D = 2 };
enum { NQS_FP32 = 0, NQS_BF16 = 1 };
enum { NQS_TFIM = 1, NQS_HEISENBERG = 2, NQS_LRTFIM = 3, NQS_CLUSTER = 4 };
enum {
  NQS_OP_SAMPLE = 1,
  NQS_OP_LOGPSI = 2,
  NQS_OP_LOCAL_ENERGY = 3,
  NQS_OP_LOGPSI_GRAD = 4,
  NQS_OP_VMC_GRAD = 5
};

typedef struct {
  int32_t cell;       /* NQS_GRU1D | NQS_GRU2D */
  int32_t Lx, Ly;     /* N = Lx * Ly; 1D: Ly = 1 */
  int32_t d_h;        /* hidden size: 8, 16, 32, 64, 128 (and 256 for NQS_GRU2D) */
  int32_t d_model;    /* 2D GLU width; must equal d_h (App. A) ; 0 means d_h */
  int32_t sz0;        /* 1: zero-magnetisation mask (needs N even) */
  int32_t precision;  /* NQS_FP32 | NQS_BF16: BF16 runs the 1D cell GEMMs of
                         sampling, teacher forcing, the local-energy chains and
                         the reverse sweep on the tensor cores (BF16 operands,
                         FP32 accumulation and FP32 state; d_h in {16, 32, 64,
                         128}), and the 2D cell and GLU GEMMs of sampling,
                         teacher forcing, the Heisenberg chains and the
                         reverse sweep (d_h in {32, 64, 256}, N <= 256); other
                         shapes return NQS_EUNSUPPORTED */
  int32_t phase;      /* 1: complex RNN (cRNN, Sec. II and Eq. softsign): a phase
                         layer z_phi = U_phi h_n + c_phi after the amplitude head,
                         phi_n = pi Softsign(z_phi) . onehot(sigma_n), log psi =
                         1/2 sum log p_n + i sum phi_n.  Built for NQS_GRU1D,
                         NQS_FP32, d_h >= 16, with NQS_CLUSTER.  Every log psi,
                         local energy and gradient weight of a cRNN is a float
                         pair (real, imaginary): logpsi [B, 2], eloc [B, 2],
                         weights [B, 2]; vmc stats [4] */
} nqs_model_desc;

typedef struct {
  int32_t kind;       /* NQS_TFIM | NQS_LRTFIM | NQS_CLUSTER (1D GRU) | NQS_HEISENBERG (2D GRU) */
  int32_t marshall;   /* Heisenberg: 1 = Marshall-rotated exchange (-J/2) */
  double J;           /* coupling J */
  double h;           /* TFIM / long-range TFIM transverse field Gamma (ignored for Heisenberg) */
  double alpha;       /* long-range TFIM: coupling J / |i - j|^alpha, alpha >= 0 (may be +inf) */
} nqs_ham_desc;

/* Number of float32 parameters of the flat layout above; 0 if desc is invalid. */
size_t nqs_param_count(const nqs_model_desc* desc);

/* Workspace bytes that `op` (NQS_OP_*) needs for B samples; 0 if invalid.
 * ham may be NULL except for NQS_OP_LOCAL_ENERGY. */
size_t nqs_workspace_bytes(const nqs_model_desc* desc, const nqs_ham_desc* ham,
                           int64_t B, int op);

/* Hidden-dimension growth, Sec. II B and Fig. 2(b): embed the parameters of the
 * trained model `small` into the larger model `big` (same cell and lattice,
 * d_h(big) >= d_h(small)).  Old blocks keep their indices; every hidden-input
 * column group is laid out [old units | new units] followed by the one-hot
 * columns; every entry without a counterpart in `small` is eps * z, z a
 * standard normal from Philox4x32-10 keyed by (seed, tensor index in the
 * layout, row, column) through Box-Muller.
 *   p_small  device, nqs_param_count(small) floats (read)
 *   p_big    device, nqs_param_count(big) floats (written)            */
nqs_status nqs_grow_hidden(const nqs_model_desc* small, const float* p_small,
                           const nqs_model_desc* big, float* p_big,
                           uint64_t seed, float eps, void* stream);

/* Exact autoregressive ("perfect") sampling, Sec. II and Eq. (1)-(3): B
 * independent configurations, site by site in sampling order;
 * sigma_n = 0 iff u_n < p_n(sigma_n = 0).
 *   uniforms device [B, N] float in [0,1) indexed by sampling position, or
 *            NULL: u_n of sample b is drawn from Philox4x32-10 with key = seed
 *            and counter = (n, sample_offset + b, step & 0xffffffff,
 *            step >> 32), u = (x0>>8)/2^24
 *   step_dev device uint64 or NULL: when given, the Philox step is read from
 *            it on the device instead of `step` (a captured CUDA graph of a
 *            training step then draws fresh samples on every replay;
 *            nqs_adam_step advances the counter)
 *   sample_offset  global index of this call's first sample: ranks that each
 *            draw B samples of one step pass rank * B, so the union of their
 *            samples is bitwise the one-rank batch (sample_offset + B <= 2^32,
 *            NQS_EINVAL otherwise)
 *   sigma    device [B, N] uint8 (written, lattice order)
 *   logpsi   device [B] float (written)
 *   hcache   device [B, N, d_h] float or NULL: hidden state h_n used for the
 *            conditional of site n (lattice order) -- the prefix cache that
 *            nqs_local_energy and the gradient calls read.            */
nqs_status nqs_sample(const nqs_model_desc* desc, const float* params, int64_t B,
                      uint64_t seed, uint64_t step, const uint64_t* step_dev,
                      uint64_t sample_offset, const float* uniforms, uint8_t* sigma,
                      float* logpsi, float* hcache, void* ws, size_t ws_bytes, void* stream);

/* Teacher-forced log psi(sigma) = 1/2 sum_n log p_n(sigma_n) (Eq. 1, pRNN).
 *   sigma  device [B, N] uint8 (read); logpsi device [B] float (written);
 *   hcache device [B, N, d_h] float or NULL (written, as in nqs_sample). */
nqs_status nqs_logpsi(const nqs_model_desc* desc, const float* params,
                      const uint8_t* sigma, int64_t B, float* logpsi, float* hcache,
                      void* ws, size_t ws_bytes, void* stream);

/* Local energies E_loc(sigma) = sum_sigma' H[sigma, sigma'] psi(sigma')/psi(sigma):
 *   NQS_CLUSTER (the cluster state of Sec. III D, open chain, GRU1D, FP32,
 *     N >= 3, d_h >= 16): H = -J sum_k K_k with the stabilisers K_1 = Z_1 X_2,
 *     K_k = X_{k-1} Z_k X_{k+1}, K_N = X_{N-1} Z_N (the paper's boundary
 *     terms read as the cluster state's stabilisers; ground energy -J N):
 *     E_loc = -J sum_k s_k psi(sigma^(k))/psi(sigma), complex [B, 2] for a
 *     cRNN, real [B] for a positive RNN; a term flipping two sites restarts
 *     from the cached state at the first and flips the second on the way;
 *   NQS_TFIM (Eq. tfim, open chain, GRU1D):
 *     -J sum s_i s_{i+1} - h sum_i psi(flip_i sigma)/psi(sigma);
 *   NQS_LRTFIM (the long-range TFIM of Sec. III C, open chain, GRU1D):
 *     -J sum_{i<j} s_i s_j / |i - j|^alpha - h sum_i psi(flip_i sigma)/psi(sigma)
 *     (the O(N^2) diagonal summed in FP64 per sample; the flips run the
 *     prefix-cached chains of the TFIM);
 *   NQS_HEISENBERG (Eq. heisenberg, open square lattice, GRU2D, Pauli/4):
 *     per bond +J/4 (parallel) or -J/4 + x exp(Delta) (antiparallel), with
 *     x = -J/2 when marshall = 1 (Marshall rotation, Sec. III B), +J/2 otherwise.
 * Each ratio is exp(Delta) with Delta accumulated from the first changed
 * site on, restarting the recurrence from the cached hidden states.
 *   sigma  device [B, N] uint8; hcache device [B, N, d_h] float from
 *          nqs_sample/nqs_logpsi with the same params (required);
 *   eloc   device [B] float (written).                                   */
nqs_status nqs_local_energy(const nqs_model_desc* desc, const float* params,
                            const nqs_ham_desc* ham, const uint8_t* sigma,
                            const float* hcache, int64_t B, float* eloc,
                            void* ws, size_t ws_bytes, void* stream);

/* Gradient of L = sum_b w_b log psi(sigma_b) (cRNN: weights [B, 2] = (w, v)
 * and L = sum_b [w_b log |psi_b| + v_b phi_b] = sum_b Re(conj(w_b + i v_b)
 * log psi_b)) with respect to the flat
 * parameters, by a reverse sweep over the unrolled recurrence.  In the 1D
 * BF16 path a parallel pass first stores, per (sample, site), the factors
 * with which the cell backward is linear in the incoming gradient (FP16,
 * with the direct path's 1 - u kept to FP16 relative precision); the
 * sequential sweep then only multiplies and runs the BF16 MMAs.
 *   weights device [B] float; hcache as above (required);
 *   grad    device [P] float (written; per-block partials are summed in FP64). */
nqs_status nqs_logpsi_grad(const nqs_model_desc* desc, const float* params,
                           const uint8_t* sigma, const float* hcache,
                           const float* weights, int64_t B, float* grad,
                           void* ws, size_t ws_bytes, void* stream);

/* VMC step statistics and gradient (Sec. III; the paper follows Hibat-Allah
 * et al. 2020 and prints no formula -- the estimator used is
 *   g = (2/M) sum_b (E_loc,b - mean E_loc) d log psi(sigma_b)/d theta,
 * with E_loc held constant; for a cRNN, g = (2/M) sum_b Re[(E_loc,b -
 * mean)^* d log psi_b], eloc [B, 2] and stats [4] = Re mean, mean |E -
 * mean|^2, M, Im mean).
 *   eloc  device [B] float (read); grad device [P] float (written);
 *   stats device [3] double (written): mean E_loc, variance (1/M), M.  */
nqs_status nqs_vmc_grad(const nqs_model_desc* desc, const float* params,
                        const uint8_t* sigma, const float* hcache,
                        const float* eloc, int64_t B, float* grad, double* stats,
                        void* ws, size_t ws_bytes, void* stream);

/* Hidden-state checkpointing for the gradient (FP32 1D GRU, positive RNN):
 * the forward keeps only every k-th state and the reverse sweep recomputes
 * each segment of k sites from its checkpoint (k ~ sqrt(N) keeps
 * O(sqrt(N)) states per sample instead of the N of the prefix cache, at the
 * cost of one more forward).  The gradient equals nqs_logpsi_grad's up to the
 * FP32 rounding of the per-block partial sums (the segments' partial rows are
 * summed in FP64).
 *   ckpt      device [B, ceil(N/k) - 1, d_h] float: ckpt[b, j] = h_{(j+1)k - 1},
 *             the state that produced the conditional of site (j+1)k - 1
 *             (nqs_ckpt_floats gives the size; may be NULL when k >= N)
 *   logpsi    device [B] float (written); weights device [B]; grad device [P]
 *   ws        nqs_ckpt_workspace_bytes(desc, B, k) bytes (one segment's
 *             states, two carries, per-block partial rows, 2 P doubles)
 * Other models return NQS_EUNSUPPORTED. */
size_t nqs_ckpt_floats(const nqs_model_desc* desc, int64_t B, int32_t k);
size_t nqs_ckpt_workspace_bytes(const nqs_model_desc* desc, int64_t B, int32_t k);
nqs_status nqs_logpsi_ckpt(const nqs_model_desc* desc, const float* params, const uint8_t* sigma,
                           int64_t B, int32_t k, float* logpsi, float* ckpt, void* ws, size_t ws_bytes,
                           void* stream);
nqs_status nqs_logpsi_grad_ckpt(const nqs_model_desc* desc, const float* params, const uint8_t* sigma,
                                int64_t B, int32_t k, const float* ckpt, const float* weights, float* grad,
                                void* ws, size_t ws_bytes, void* stream);

/* Data-parallel VMC step over ranks (Sec. III; samples are independent, so
 * each rank draws and evaluates its own share of the batch with replicated
 * weights).  The step's only exchange is the energy statistics that centre
 * the gradient weights and the sum of the ranks' gradients:
 *   1. nqs_energy_sums on each rank: sums = [sum E_loc, sum E_loc^2, B]
 *      (device [3] double, written);
 *   2. the caller sums `sums` over ranks (an all-reduce of 3 doubles);
 *   3. nqs_vmc_grad_global on each rank with the global sums: writes
 *      stats = [mean, variance (1/M), M] of all ranks and this rank's share
 *        grad = sum_{b in this rank} 2 (E_loc,b - mean) / M d log psi_b / d theta
 *      (device [P] double, FP64 sum of the per-block partials);
 *   4. the caller sums `grad` over ranks (an all-reduce of P doubles).
 * With one rank, stats equal nqs_vmc_grad's bitwise and grad equals its
 * gradient before the rounding to float. */
nqs_status nqs_energy_sums(const float* eloc, int64_t B, double* sums, void* stream);
nqs_status nqs_vmc_grad_global(const nqs_model_desc* desc, const float* params,
                               const uint8_t* sigma, const float* hcache, const float* eloc,
                               int64_t B, const double* sums, double* grad, double* stats,
                               void* ws, size_t ws_bytes, void* stream);

/* Training loop (Sec. II B, Sec. III; hyperparameters of Tab. III).
 *
 * Learning-rate schedules, with t the 0-based training step:
 *   NQS_LR_CONSTANT  lr0
 *   NQS_LR_STEP      lr0 for t < t_switch, lr1 from t_switch on (1D TFIM
 *                    Adaptive: 5e-3, then 5e-4 from step 25,000)
 *   NQS_LR_INVERSE   lr0 for t < t_switch, lr0 / (1 + (t - t_switch) / decay)
 *                    from t_switch on (2D Heisenberg Static: t_switch = 0,
 *                    decay = 5000; 2D Adaptive: t_switch = 100,000, reading
 *                    the table's floor term as the switch to the decay in the
 *                    second half of training) */
enum { NQS_LR_CONSTANT = 1, NQS_LR_STEP = 2, NQS_LR_INVERSE = 3 };
typedef struct {
  int32_t kind;       /* NQS_LR_* */
  int32_t reserved;
  double lr0, lr1;
  int64_t t_switch;
  double decay;
} nqs_lr_schedule;

/* Adam hyperparameters (Kingma and Ba 2014): beta1, beta2 in [0, 1), eps > 0. */
typedef struct {
  double beta1, beta2, eps;
} nqs_adam_desc;

/* One Adam update of the flat parameters (Adam is the paper's optimiser,
 * Sec. III and the hyperparameter appendix):
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,  k = t + 1,
 *   params -= lr(t) (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps).
 *   grad     device [P] float, or grad64 device [P] double (exactly one of
 *            them non-NULL; grad64 takes the rank-summed gradient of
 *            nqs_vmc_grad_global)
 *   params, m, v  device [P] float (updated in place); m = v = 0 before the
 *            first update.  On growth the moments are embedded like the
 *            parameters: nqs_grow_hidden with eps = 0 (the appendix carries
 *            parameters and momentum states over to the larger model).
 *   t_dev    device uint64 step counter or NULL (then t is used): read for
 *            the update and incremented after it, so the step of a captured
 *            graph advances on every replay; nqs_sample may read the same
 *            counter as its Philox step. */
nqs_status nqs_adam_step(const float* grad, const double* grad64, float* params, float* m, float* v,
                         int64_t P, const nqs_adam_desc* adam, const nqs_lr_schedule* sched,
                         uint64_t t, uint64_t* t_dev, void* stream);

/* log[t mod cap] = (t, stats[0], stats[1], stats[2]) with t = *t_dev: a
 * per-step record of the energy statistics of a captured training step
 * (log: device [cap, 4] double). */
nqs_status nqs_record_stats(const double* stats, double* log, int64_t cap, const uint64_t* t_dev,
                            void* stream);

/* Final evaluation (Sec. III A, Tab. I and Tab. II: energies and variances
 * from 10^6 samples after training): M samples drawn in chunks of `chunk`
 * (global sample indices 0 .. M - 1 of the Philox stream (seed, step), so the
 * result does not depend on the chunk size beyond FP64 rounding), their local
 * energies, and FP64 statistics:
 *   stats  device [5] double (written): mean E_loc, variance (1/M), M,
 *          standard error of the mean sqrt(var / M), and the error of the
 *          variance var sqrt(2 / (M - 1)) for Gaussian local energies (the
 *          error bar of Tab. I);
 *   ws     nqs_evaluate_workspace_bytes(desc, ham, chunk) bytes (it holds one
 *          chunk's configurations and prefix cache); its status word is the
 *          first status any chunk recorded.  M <= 2^32. */
size_t nqs_evaluate_workspace_bytes(const nqs_model_desc* desc, const nqs_ham_desc* ham, int64_t chunk);
nqs_status nqs_evaluate(const nqs_model_desc* desc, const float* params, const nqs_ham_desc* ham,
                        int64_t M, int64_t chunk, uint64_t seed, uint64_t step, double* stats,
                        void* ws, size_t ws_bytes, void* stream);

/* One replica of a batched VMC step. */
#define NQS_MAX_REPLICAS 16
typedef struct {
  nqs_model_desc desc;   /* NQS_GRU1D, sz0 = 0, phase = 0, d_h in {16, 32, 64, 128};
                            NQS_FP32 replicas run as grouped launches over all
                            of them, NQS_BF16 replicas the tensor-core calls of
                            one model each (autotuned tiles) */
  nqs_ham_desc ham;      /* NQS_TFIM */
  int64_t B;             /* samples of this replica, >= 1 */
  uint64_t seed;         /* Philox key of this replica's sampling */
  const float* params;   /* device [P] (read) */
  uint8_t* sigma;        /* device [B, N] (written) */
  float* logpsi;         /* device [B] (written) */
  float* hcache;         /* device [B, N, d_h] (written) */
  float* eloc;           /* device [B] (written) */
  float* grad;           /* device [P] (written) */
  double* stats;         /* device [3] (written): mean E_loc, variance, M */
} nqs_replica;

/* Workspace bytes of nqs_vmc_step_batched for these replicas; 0 if invalid. */
size_t nqs_vmc_step_batched_workspace_bytes(int R, const nqs_replica* reps);

/* A whole VMC step (nqs_sample + nqs_local_energy + nqs_vmc_grad) for R
 * replicas of uneven hidden size, field, batch and chain length -- the model
 * family of the Adaptive schedule (Sec. II B), e.g. one model per growth
 * stage and field.  For the FP32 replicas every phase is one launch over all
 * of them (the chain phase is persistent and balances the replicas' work),
 * and the replica table travels as a kernel argument; the BF16 replicas run
 * first, each through the single-model tensor-core calls on the same stream
 * and Philox step.  The call can be captured in a CUDA graph (after a first
 * call outside the capture, which tunes the BF16 tiles).
 *   reps      host array of R replicas (1 <= R <= NQS_MAX_REPLICAS)
 *   step      Philox step of the sampling when step_dev is NULL
 *   step_dev  device counter or NULL: when given, the step is read from it on
 *             the device and incremented at the end of the call, so every
 *             replay of a captured graph draws fresh samples.            */
nqs_status nqs_vmc_step_batched(int R, const nqs_replica* reps, uint64_t step, uint64_t* step_dev,
                                void* ws, size_t ws_bytes, void* stream);

/* Local energies for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a library convenience.  Some callers
 * cannot call cudaMalloc -- a plugin whose host application owns every device
 * allocation, code running where an allocation would stall a latency-critical
 * loop, or a thin foreign-language binding with no device allocator.  This
 * call computes exactly what nqs_local_energy computes for the 1D TFIM with
 * the FP32 GRU, but takes no workspace: its scratch is one fixed device array
 * of NQS_STATIC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library keeps until the process exits.  The call itself allocates
 * nothing.
 *   - Capacity: the array holds a 256-byte header, the packed weights and two
 *     float arrays of B*N entries; larger B*N returns NQS_EWORKSPACE (about
 *     2 million B*N entries at d_h = 64) and enqueues nothing.
 *   - The first call on a device looks up the array's device address with
 *     that device current (cudaGetSymbolAddress); make that first call before
 *     any stream capture.
 *   - Every call on a device shares the one array and it keeps the previous
 *     call's contents (the call resets what must start at zero).  Calls whose
 *     work overlaps on the GPU (other streams, other host threads) race on it:
 *     serialise them, e.g. on one stream.
 *   - The looked-up address is kept per device number for the process: use
 *     the device's primary context (the runtime's default) and do not call
 *     cudaDeviceReset between calls.
 *   - No device-side status is reported (there is no workspace status word to
 *     read): a non-finite local energy shows only in eloc.
 * Arguments as nqs_local_energy, with the same status for an invalid
 * descriptor; a valid one must be NQS_GRU1D with NQS_FP32 and no mask, and ham
 * NQS_TFIM, otherwise NQS_EUNSUPPORTED. */
#define NQS_STATIC_SCRATCH_BYTES ((size_t)16 << 20)
nqs_status nqs_local_energy_static(const nqs_model_desc* desc, const float* params,
                                   const nqs_ham_desc* ham, const uint8_t* sigma,
                                   const float* hcache, int64_t B, float* eloc, void* stream);

/* Autotuning of the tensor-core kernels' tile shapes (threads per row), on by
 * default: the first call for a new (kernel, d_h, N, B) that is not inside a
 * stream capture times every variant on its own inputs (synchronising the
 * stream once) and caches the fastest for the process; make that first call
 * before capturing a graph.  on = 0 turns tuning off and clears the cache
 * (the first variant is then used). */
void nqs_set_autotune(int on);

/* Pin the tile variant of every tensor-core kernel: variant >= 0 selects
 * that variant (a kernel with fewer variants takes its last one), bypassing
 * the autotuner and its cache; variant < 0 returns to normal selection.
 * 1D: variants differ in threads per row (1, 2, 4) and, for sampling,
 * teacher forcing and the reverse sweep, in rows per 128-lane tile (128, or
 * 64 or 32 to put more SMs on a small batch; at d_h = 64 the 32-row sampling
 * / teacher-forcing tile writes each A row into all four lane quarters).
 * 2D (d_h 64 where noted): variant 0 selects 128-sample tiles with one
 * thread per row everywhere; any other variant selects 32-sample tiles with
 * replicated A rows for sampling / teacher forcing (d_h 64) and 32-sample
 * tiles for the sequential reverse sweep.  The 2D chains (d_h 32 / 64) run
 * by default on two 128-row tiles per CTA with one thread per row; variant 0
 * selects one tile with one thread per row, 1 one tile with 16 units per
 * thread (2 or 4 threads per row), 2 the default, 3 two tiles with two
 * threads per row.  Per-sample results (samples, log psi, cache,
 * local energies) are bitwise the same in every variant; the gradient, a sum
 * over samples grouped by tile, is bitwise the same for the same rows per tile
 * and equal to rounding otherwise (2D: bitwise the same).  This is for timing
 * and testing them one by one. */
void nqs_set_tile_variant(int variant);

/* Positions per pass of the reverse sweep of the 2D GRU at d_h = 256 in BF16
 * (NQS_OP_LOGPSI_GRAD, NQS_OP_VMC_GRAD; App. A).  0 (the default) sweeps all
 * N positions in one pass; k > 0 sweeps passes of k positions, the last pass
 * first, with the backward carries running on from pass to pass, so that the
 * per-cell tapes of the sweep (about 7.2 KB per sample and position) need
 * workspace for B k cells instead of B N.  The prefix cache is still read at
 * every position.  The gradient equals the one-pass gradient to rounding (its
 * weight-gradient sums are grouped by pass).  nqs_workspace_bytes follows the
 * setting, and the gradient calls check their workspace against it (set it
 * before sizing the workspace).  Process-wide; other shapes ignore it. */
void nqs_set_sweep_segment(int32_t positions);

/* Bound, in polls, of every tensor-core wait that may give up (default 2^26
 * polls, about a second); polls < 0 restores the default.  It exists to
 * exercise the NQS_ETIMEOUT path: with 0 every such wait gives up at once,
 * the kernels record NQS_ETIMEOUT, finish early with garbage outputs, and
 * free their tensor memory only after every MMA they issued has drained
 * (that drain keeps the default bound).  Applies to the current device, for
 * the whole process; do not change it while kernels of this library run. */
nqs_status nqs_set_wait_limit(int64_t polls);

/* Copy the workspace status word to *device_status (an nqs_status) after
 * waiting for `stream`; clears it.  This call blocks the host. */
nqs_status nqs_workspace_status(void* ws, int32_t* device_status, void* stream);

/* Human-readable name of a status code (static storage). */
const char* nqs_status_string(nqs_status status);

#ifdef __cplusplus
}
#endif

#endif /* NQS_H */

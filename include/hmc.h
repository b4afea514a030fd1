/*
 * hmc.h -- C ABI of the GB300 subset-HMC library (libhmc.so).
 *
 * The library runs the hot path of the hybrid VI-HMC method of arXiv
 * 2507.14652: full-batch Hamiltonian Monte Carlo over a selected subset
 * Theta_s of a network's parameters, the rest Theta_~s held at caller-supplied
 * values (Sec. 3.2 and Algorithm 2).  Every step runs in CUDA kernels on one GPU.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * Parameter order: for each Linear layer in order, W[out][in] row-major, then
 *   b[out] if the layer has a bias.  A DeepONet lists all branch layers, then
 *   all trunk layers, then its scalar output bias b0.  P = total count.
 * Subset: subset_mask[P] (1 = sampled).  The sampled entries, in ascending
 *   parameter index, form the position vector q of length k.
 * Energy (Sec. 2.2, constants Z and normalisers dropped):
 *   U(q) = sum over data terms (F(x) - y)^2 / (2 sigma^2) + sum_j q_j^2 / (2 alpha^2)
 *   with sigma = noise_sigma (Gaussian likelihood over the full batch) and
 *   alpha = prior_sigma (N(0, alpha^2) prior on the sampled parameters only).
 * Kinetic energy K(p) = p.p / 2 (mass matrix M = I); H = U + K.
 * Precision of q, p, grad and samples: double for HMC_PREC_FP64, float for
 *   every other precision.  U and dH are always double.
 * Pointers: every array argument may be host or device memory (detected with
 *   cudaPointerGetAttributes).  Device arrays must be contiguous, row-major
 *   and stay owned by the caller.  Work is queued on the handle's stream;
 *   when an output is host memory the call copies it back and synchronises
 *   before returning, otherwise it returns without waiting.
 * Errors: every call returns an hmc_status; hmc_last_error() gives the
 *   message of the last failure on the calling thread.  No call aborts, throws
 *   across the ABI or traps on the device.
 */
#ifndef HMC_H
#define HMC_H

#ifdef __cplusplus
extern "C" {
#endif

#define HMC_MAX_LAYERS 16
#define HMC_MAX_SPLITS 64

/* Symbols of the C ABI are exported even when the library hides everything else. */
#if defined(__GNUC__)
#define HMC_API __attribute__((visibility("default")))
#else
#define HMC_API
#endif

typedef struct hmc_handle_s *hmc_handle;

typedef enum {
    HMC_OK = 0,
    HMC_ERR_ARG = 1,          /* invalid argument (sizes, spec, pointers) */
    HMC_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    HMC_ERR_OOM = 3,          /* device allocation failed */
    HMC_ERR_NONFINITE = 4,    /* U was NaN or +-Inf (outputs are still written) */
    HMC_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
    HMC_ERR_UNSUPPORTED = 6   /* a valid request the library does not implement */
} hmc_status;

typedef enum { HMC_ACT_IDENTITY = 0, HMC_ACT_TANH = 1, HMC_ACT_SIN = 2 } hmc_act;

/* Arithmetic of the network evaluation.  FP64 and FP32 run plain CUDA-core
 * kernels.  BF16 runs the wide layers on tcgen05 tensor cores (bf16 operands,
 * fp32 accumulation) with fp32 positions/momenta and fp64 energy sums.  FP16 is the
 * same tensor-core path with fp16 operands: the same bytes and tensor rate, 11
 * significant bits against bf16's 8, so the leapfrog's forces are about eight times
 * more accurate (the output deltas are scaled by a power of two near 1/sigma to stay
 * inside fp16's range, and the gradient sums are scaled back in fp32).
 * HMC_PREC_TF32 is reserved: creating a handle with it returns HMC_ERR_UNSUPPORTED. */
typedef enum {
    HMC_PREC_FP64 = 0,
    HMC_PREC_FP32 = 1,
    HMC_PREC_TF32 = 2,
    HMC_PREC_BF16 = 3,
    HMC_PREC_FP16 = 4
} hmc_prec;

/* HMC_NET_DEEPONET: n_u input functions evaluated at n_y query points shared by all
 * of them.  HMC_NET_DEEPONET_UNALIGNED: every input function with its own n_y query
 * points (FP64 and FP32 only). */
typedef enum { HMC_NET_MLP = 0, HMC_NET_DEEPONET = 1, HMC_NET_DEEPONET_UNALIGNED = 2 } hmc_net_kind;

/* One feed-forward stack: widths[0] inputs, widths[n_layers] outputs;
 * act[l] and has_bias[l] for Linear layer l. */
typedef struct {
    int n_layers;
    int widths[HMC_MAX_LAYERS + 1];
    int act[HMC_MAX_LAYERS];
    int has_bias[HMC_MAX_LAYERS];
} hmc_mlp_spec;

/* An MLP (kind = HMC_NET_MLP, uses `net`) or a DeepONet (uses `branch` and
 * `trunk`, whose output widths must match; output = <branch(u), trunk(y)> + b0,
 * Sec. 4.2 and App. A). */
typedef struct {
    int kind;
    hmc_mlp_spec net;
    hmc_mlp_spec branch;
    hmc_mlp_spec trunk;
    int deeponet_out_bias;   /* 1 = scalar b0 present */
    int prec;                /* hmc_prec */
} hmc_net_spec;

/* Training set, FP64 (or FP32, see dtype), host or device.  MLP: x[n][dx], y[n][dout].
 * DeepONet (aligned): u[n_u][du] input functions, yq[n_y][dy] query points
 * shared by all functions, t[n_u][n_y] targets.  Unaligned DeepONet: yq[n_u][n_y][dy],
 * the n_y query points of each function.  Unused fields are ignored.
 * An empty training set (n = 0, or n_u = 0 or n_y = 0) is allowed: the likelihood is 1
 * and U(q) = |q|^2 / (2 alpha^2), so the sampler draws from the prior (Sec. 2.2); the
 * array pointers may then be NULL.  Split handles need at least n_splits data rows. */
typedef struct {
    const void *x; long n; int dx;
    const void *y;
    const void *u; long n_u; int du;
    const void *yq; long n_y; int dy;
    const void *t;
    int dtype;               /* hmc_data_dtype of every array above (0, the zero value: FP64) */
} hmc_data;

/* Element type of the training-set arrays.  The handle converts them once, at creation,
 * to the engine's working precision, so the type has no cost on the sampling path. */
typedef enum { HMC_DATA_F64 = 0, HMC_DATA_F32 = 1 } hmc_data_dtype;

/*
 * Create a sampler for one problem (Algorithm 2 after its subset is fixed).
 *   spec          network and precision
 *   data          training set (copied to the device and converted)
 *   prior_sigma   alpha > 0, noise_sigma = sigma > 0
 *   subset_mask   [P] bytes, 1 = sampled (the set Theta_s); k = its popcount, k >= 1
 *   frozen_params [P] doubles; entries off the subset are held fixed (Theta_~s = mu_~s)
 *   n_chains      C >= 1 independent chains, batched inside every launch
 *   cuda_stream   cudaStream_t to queue all work on (NULL = legacy default stream)
 * The handle copies everything it needs; the caller may free its arrays on return.
 */
HMC_API hmc_status hmc_create(hmc_handle *out, const hmc_net_spec *spec, const hmc_data *data,
                      double prior_sigma, double noise_sigma,
                      const unsigned char *subset_mask, const double *frozen_params,
                      int n_chains, void *cuda_stream);

/*
 * Create one handle over n_problems independent problems (each with its own
 * spec, data, sigmas, mask and frozen vector, all with n_chains chains).  The problems
 * run side by side: in an HMC_PREC_BF16 or HMC_PREC_FP16 batch, the tensor-core MLP
 * problems that share a kernel shape (padded hidden width, input width) form a group
 * whose gradient takes one launch per kernel and layer slot for all of them (a job
 * table walked by each kernel, every problem on its own buffers, results identical to
 * separate launches); groups and the remaining problems run on up to 16 stream lanes
 * (concurrent branches of the captured trajectory graph) that join again; the kicks,
 * drifts and the Metropolis step cover all problems in single launches.  State vectors of a batch handle are
 * packed per problem: q = [problem][chain][k_problem]; U, accepted and dH are
 * [problem][chain] per trajectory.  Momenta of problem p use Philox stream p.
 * In an HMC_PREC_BF16 or HMC_PREC_FP16 batch, a problem whose network the tensor-core
 * kernels do not cover (a hidden width above 256, a sine activation, say) runs on the FP32
 * CUDA-core engine instead; its positions are float like the others'.  Hidden widths up to
 * 128 run on the tensor cores padded to 128 with zero units, wider ones padded to 256.
 */
HMC_API hmc_status hmc_create_batch(hmc_handle *out, int n_problems, const hmc_net_spec *specs,
                            const hmc_data *data, const double *prior_sigma,
                            const double *noise_sigma, const unsigned char *const *subset_masks,
                            const double *const *frozen_params, int n_chains, void *cuda_stream);

/*
 * Create a sampler for one problem whose trajectories use the symmetric split
 * integrator over n_splits data batches (the split HMC Sec. 4.2.3 runs for its
 * full-HMC comparisons) instead of the full-batch leapfrog.  Arguments as
 * hmc_create, plus
 *   n_splits   M in [1, HMC_MAX_SPLITS] and at most the number of data rows R
 *              (MLP: data points; DeepONet: input functions, each with all its
 *              queries).  Batch m holds rows [floor(m R / M), floor((m + 1) R / M)).
 * The Hamiltonian is split as H = sum_m [U_m(q) + K(p)/M], U_m the likelihood of
 * batch m plus 1/M of the prior.  One step of size eps is the forward sweep
 * m = 1..M of {p -= eps/2 grad U_m(q); q += eps/(2M) p} followed by the backward
 * sweep m = M..1 of {q += eps/(2M) p; p -= eps/2 grad U_m(q)}: symplectic and
 * reversible, so the Metropolis test on H = U + K stays exact; M = 1 is the
 * leapfrog.  A step costs 2M - 1 batch gradients (about two full ones); each
 * batch's activations take 1/M of the full batch's device memory.
 * On such a handle hmc_leapfrog, hmc_sample and hmc_adapt_step_size integrate
 * with this scheme; hmc_energy_grad returns the full U and grad U (sums over the
 * batches).  Everything else is as for hmc_create.
 */
HMC_API hmc_status hmc_create_split(hmc_handle *out, const hmc_net_spec *spec, const hmc_data *data,
                                    double prior_sigma, double noise_sigma, const unsigned char *subset_mask,
                                    const double *frozen_params, int n_chains, int n_splits,
                                    void *cuda_stream);

/*
 * Create a sampler for one problem whose potential and force are evaluated in passes over
 * the data rows, rows_per_pass (>= 1) rows at a time (MLP: data points; DeepONet: input
 * functions, each with all its queries), so the device holds one pass's activations.
 * U and grad U are sums over the data terms (Sec. 2.2, the full-batch potential of
 * Sec. 3.3), so the passes' sums give them exactly (up to the order of the additions):
 * pass m holds rows [floor(m R / M), floor((m + 1) R / M)) of the R rows, M =
 * ceil(R / rows_per_pass), plus 1/M of the prior.  Every buffer that grows with the rows
 * is shared by the passes, which run one after another on the handle's stream (a DeepONet
 * pass evaluates the trunk net again, on all queries).  Trajectories use the full-batch
 * leapfrog, as for hmc_create; everything else is as for hmc_create.
 * hmc_create itself falls back to passes when the whole batch's buffers do not fit in
 * device memory (it halves the rows of a pass until the handle fits); hmc_num_passes
 * reports the passes a handle uses.
 */
HMC_API hmc_status hmc_create_chunked(hmc_handle *out, const hmc_net_spec *spec, const hmc_data *data,
                                      double prior_sigma, double noise_sigma, const unsigned char *subset_mask,
                                      const double *frozen_params, int n_chains, long rows_per_pass,
                                      void *cuda_stream);

/* Passes over the data rows per evaluation (1 unless the handle is chunked), or -1. */
HMC_API int hmc_num_passes(hmc_handle h);

/* k (for a batch: the sum of k over problems), or -1 for a bad handle. */
HMC_API long hmc_subset_size(hmc_handle h);

/* P (for a batch: the sum over problems), or -1 for a bad handle. */
HMC_API long hmc_param_count(hmc_handle h);

/* Number of chains C, or -1. */
HMC_API int hmc_num_chains(hmc_handle h);

/*
 * U and grad U for every chain (Sec. 2.2 potential; its gradient is the force of
 * Hamilton's equations).  q [C][k] (batch: packed per problem) in the handle's
 * position precision; U [C] doubles; grad [C][k] or NULL.  Returns
 * HMC_ERR_NONFINITE (after writing the outputs) when U is a host array and some
 * U is not finite.
 */
HMC_API hmc_status hmc_energy_grad(hmc_handle h, const void *q, double *U, void *grad);

/*
 * L leapfrog steps of size eps in place on (q, p) [C][k] (Sec. 2.2):
 *   p -= eps/2 grad U(q); repeat L times { q += eps p; p -= eps grad U(q) }, the
 *   last kick being eps/2.  L >= 0.
 */
HMC_API hmc_status hmc_leapfrog(hmc_handle h, void *q, void *p, double eps, int L);

/*
 * n_samples HMC trajectories per chain starting from q0 [C][k] (Algorithm 1 on
 * the subset, as in Algorithm 2).  Trajectory t = first_traj + i draws
 * p ~ N(0, I) from Philox4x64-10 keyed by seed (bit-identical to the reference
 * generator), integrates L leapfrog steps of size eps, and accepts iff
 * log u < H(q, p) - H(q*, p*) with u ~ U(0, 1] from the same generator (a
 * non-finite difference rejects).  Outputs (any may be NULL):
 *   samples  [n][C][k]  the chain state after each trajectory (repeats on rejection)
 *   accepted [n][C]     1 = accepted
 *   dH       [n][C]     H(q*, p*) - H(q, p)
 *   q_last   [C][k]     final state
 * Restarting from q_last with first_traj advanced by n continues the same chains.
 */
HMC_API hmc_status hmc_sample(hmc_handle h, const void *q0, double eps, int L, long n_samples,
                      unsigned long long seed, long first_traj,
                      void *samples, unsigned char *accepted, double *dH, void *q_last);

/*
 * hmc_sample with a step size per problem: eps [n_problems] doubles (host or device,
 * each finite and > 0; one entry for a single-problem handle), problem p's trajectories
 * integrating with eps[p].  Independent problems of a batch differ in their data and
 * networks, so a common step that suits one can reject everything on another
 * (hmc_adapt_step_size returns such per-problem steps).  Everything else as hmc_sample.
 */
HMC_API hmc_status hmc_sample_steps(hmc_handle h, const void *q0, const double *eps, int L, long n_samples,
                                    unsigned long long seed, long first_traj,
                                    void *samples, unsigned char *accepted, double *dH, void *q_last);

/*
 * Step-size adaptation for the warm-up (the paper tunes eps to about 80% acceptance;
 * Sec. 4.2.3): runs n_warmup trajectories of L steps from q, one at a time, and adapts
 * each problem's log eps by dual averaging (Hoffman and Gelman 2014, Sec. 3.2) so that
 * the mean over the problem's chains of the Metropolis acceptance probability
 * min(1, exp(-dH)) approaches target_accept; a non-finite dH counts as 0.
 *   q [C][k]        in: start state; out: state after the warm-up (device or host)
 *   eps0            initial step of every problem; the shrinkage point is log(10 eps0)
 *   seed, first_traj  Philox stream and trajectory index of the first warm-up
 *                   trajectory; continue sampling with first_traj + n_warmup
 *   eps_out         [n_problems] host doubles: each problem's averaged step after the
 *                   last update (one double for a single-problem handle); pass them to
 *                   hmc_sample_steps
 * The step sizes are device state: every warm-up trajectory replays the same captured
 * trajectory graph (the one hmc_sample uses for this L and seed), and each update runs
 * on the device right after its trajectory, so the warm-up waits for the GPU once, at
 * the end.  Errors as hmc_sample.
 */
HMC_API hmc_status hmc_adapt_step_size(hmc_handle h, void *q, int L, double eps0, long n_warmup,
                               double target_accept, unsigned long long seed, long first_traj,
                               double *eps_out);

/*
 * Sensitivities of the network output to each parameter around the VI mean (Sec. 3.1,
 * the equation defining S_i^2; the step before the sampler in Algorithm 2):
 *   S2[i] = sd[i]^2 / N_d * sum over the data terms of (dF/dtheta_i)^2 at theta = mu,
 * the data terms being the MLP outputs F_o(x_n) (N_d = n * d_out) or the DeepONet
 * outputs S_jk = <B_j, T_k> + b0 over all (input function, query) pairs
 * (N_d = n_u * n_y).
 *   spec        network; spec->prec chooses the arithmetic: HMC_PREC_FP64 runs in
 *               double, any other precision in float with double column sums
 *   data        inputs x (MLP) or u and yq (DeepONet); targets are not read
 *   mu, sd [P]  VI means and standard deviations (double), parameter order as above
 *   S2 [P]      output (double)
 *   cuda_stream where the work is queued; the call returns once S2 is written
 * Cost: one forward pass, d_out (MLP) or p (DeepONet) reverse passes batched as GEMMs,
 * and per layer one GEMM of the squared activations with the squared adjoints.
 */
HMC_API hmc_status hmc_sensitivity(const hmc_net_spec *spec, const hmc_data *data, const double *mu,
                                   const double *sd, double *S2, void *cuda_stream);

/*
 * The truncation of the parameter set (Sec. 3.1, the equation defining N-hat, and the
 * subsets of Sec. 3.2): with the parameters ranked by S2 from most to least sensitive
 * (equal values: lower index first),
 *   N_hat = max{ N_T : sum of the first N_T S2 / sum of all S2 <= tau },
 * and the sampled subset Theta_s is the first N_hat of the ranking.  Sums are FP64,
 * in rank order; an all-zero S2 gives N_hat = 0.
 *   S2 [P]        sensitivities (double, non-negative and finite; else HMC_ERR_ARG)
 *   tau           the variance share to keep
 *   mask [P]      output: 1 for Theta_s (the subset_mask of hmc_create), else 0
 *   n_hat         output (host): N_hat
 *   order [P]     output, may be NULL: parameter indices in rank order (int64)
 * The ranking is a stable radix sort, so it is exact and reproducible.
 */
HMC_API hmc_status hmc_select_subset(const double *S2, long P, double tau, unsigned char *mask, long *n_hat,
                                     long long *order, void *cuda_stream);

/*
 * Posterior predictive (Sec. 4.2.1): the network's outputs on new inputs for every
 * sample, reduced over the samples to
 *   mean = (1/S) sum_s F_s   and   std = sqrt((1/S) sum_s (F_s - mean)^2)
 * per output, and optionally the mean relative L2 error of the mean against targets,
 *   rel_l2 = (1/N) sum_i ||Y_i - mean_i||_2 / ||Y_i||_2,
 * over the N = n_u input functions of a DeepONet (each over its n_y queries), or with
 * N = 1 over all outputs of an MLP.
 *   h          a single-problem handle (hmc_create or hmc_create_split): its network,
 *              frozen vector and subset
 *   samples    [n_samples][k] positions in the handle's precision (e.g. the samples
 *              array of hmc_sample, whose [n][C][k] is n*C samples)
 *   inputs     new inputs: x, n, dx (MLP) or u, n_u, du, yq, n_y, dy (DeepONet); the
 *              targets y or t are read only when rel_l2 is not NULL
 *   mean, std  outputs [n][d_out] (MLP) or [n_u][n_y] (DeepONet), double
 *   rel_l2     output (host double) or NULL
 * Runs in the handle's arithmetic (double for HMC_PREC_FP64, float otherwise; the
 * reduction over samples in double, samples in order) and returns when done.
 */
HMC_API hmc_status hmc_predict(hmc_handle h, const void *samples, long n_samples, const hmc_data *inputs,
                               double *mean, double *std, double *rel_l2);

/*
 * Wait for the work queued on the handle and report whether a device-side wait gave up
 * since the last check.  The tensor-core kernels bound every wait on a barrier (2 s); one
 * that runs out records it in the engine's error flag, stops its kernel early and leaves
 * the context usable, so the results of the calls since the last check cannot be trusted.
 * Returns HMC_ERR_TIMEOUT then (and clears the record), HMC_OK otherwise.
 */
HMC_API hmc_status hmc_check(hmc_handle h);

/* Free the handle and all its device memory. NULL is accepted. */
HMC_API hmc_status hmc_destroy(hmc_handle h);

/*
 * U and grad U of an FP32 MLP for C chains without any device allocation.
 * The paper has no counterpart.  It is for callers that cannot call cudaMalloc:
 * a plug-in inside another framework whose memory pool owns the whole device (a
 * cudaMalloc of its own would fail, or steal memory the pool has promised), or a
 * real-time loop that may not block in the driver's allocator.  It runs the same
 * CUDA-core kernels as hmc_energy_grad with HMC_PREC_FP32, without a handle.
 *   net          the MLP (widths, activations, biases); parameter order as above
 *   x [n][dx], y [n][dout], frozen [P], subset_idx [k] (strictly ascending int32
 *   parameter indices of the sampled entries), q [C][k]: device arrays owned by
 *   the caller
 *   U [C] (double) and grad [C][k] (float, may be NULL): device outputs
 *   cuda_stream  where the work is queued; the call returns without waiting
 * Every intermediate lives in one fixed 16 MiB array inside the library's device
 * image, held by every GPU that loads the library until the process exits.
 * Problems whose intermediates exceed it are rejected with HMC_ERR_ARG and a
 * message giving the limit.  All calls share that array and each call overwrites
 * it (what must start at zero is cleared by the call itself), so calls that
 * overlap on the GPU race; serialise them.  subset_idx is checked on the device:
 * an entry outside [0, P) or not above the one before it is never used to
 * address memory, and every U (and grad) of that call is set to NaN instead.
 * The first call on a device also looks up the array's device address (a host-side
 * query of the driver, once per device, with that device current).
 */
HMC_API hmc_status hmc_energy_grad_noalloc(const hmc_mlp_spec *net, const float *x, const float *y, long n,
                                           const float *frozen, const int *subset_idx, long k,
                                           double prior_sigma, double noise_sigma, int n_chains,
                                           const float *q, double *U, float *grad, void *cuda_stream);

/* Message of the last failed call on this thread ("" if none).  Owned by the library. */
HMC_API const char *hmc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HMC_H */

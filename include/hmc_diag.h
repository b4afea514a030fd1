/*
 * hmc_diag.h -- diagnostic entry points of libhmc.so, used by the tests to
 * check the device random-number stream bit by bit against an independent
 * implementation.  They allocate, compute on the legacy default stream and
 * copy the result into the host array before returning.
 */
#ifndef HMC_DIAG_H
#define HMC_DIAG_H

#include "hmc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x64-10 (Salmon et al., SC'11) of n counters ctr[n][4] under keys
 * key[n][2]; out_host[n][4] receives the output words. */
HMC_API hmc_status hmc_diag_philox(const unsigned long long *ctr, const unsigned long long *key, long n,
                           unsigned long long *out_host);

/* Momentum components 0..k-1 of (problem, chain, traj) exactly as hmc_sample
 * draws them (p ~ N(0, I), Algorithm 1), as doubles in out_host[k]. */
HMC_API hmc_status hmc_diag_momenta(unsigned long long seed, unsigned long long problem, unsigned long long chain,
                            unsigned long long traj, long k, double *out_host);

/* log u of the Metropolis uniform (Algorithm 1) for chains 0..n_chain-1 and
 * trajectories 0..n_traj-1: out_host[chain][traj]. */
HMC_API hmc_status hmc_diag_log_uniform(unsigned long long seed, unsigned long long problem, long n_chain, long n_traj,
                                double *out_host);

/* Kernel nodes in the captured graph of one trajectory of the last hmc_sample
 * call (the launches one trajectory costs), or -1 for a bad handle. */
HMC_API long hmc_diag_graph_kernels(hmc_handle h);

/* How many trajectory graphs the handle has captured so far (a new one only when L or
 * the seed changes), or -1 for a bad handle. */
HMC_API long hmc_diag_graph_captures(hmc_handle h);

/* The step sizes of the last hmc_adapt_step_size call on h, out_host[n][problems][2]:
 * entry [m - 1][p][0] is the step trajectory m + 1 of problem p was given (exp of the
 * dual-averaging iterate after update m) and [m - 1][p][1] the averaged step after
 * update m, for m = 1..n (n at most that call's n_warmup). */
HMC_API hmc_status hmc_diag_adapt_trace(hmc_handle h, double *out_host, long n);

/* The device dual-averaging update of hmc_adapt_step_size (Hoffman and Gelman 2014,
 * Sec. 3.2) run on given energy errors dH[n][nseg] (host or device) of one problem with
 * nseg chains instead of trajectories: update m takes row m - 1.  out_host[n][2] as
 * hmc_diag_adapt_trace. */
HMC_API hmc_status hmc_diag_dual_averaging(const double *dH, long n, int nseg, double eps0, double target,
                                           double *out_host);

/* The tanh the FP16 tensor-core engine applies in its epilogues, on n device floats
 * x -> y; synchronises before returning. */
HMC_API hmc_status hmc_diag_tanh16(const float *x, float *y, long n);

/* Device memory the library's buffers hold right now, in bytes (every handle together). */
HMC_API long hmc_diag_device_bytes(void);

/* Cap the library's device buffers at `bytes` in total (<= 0 lifts the cap): an allocation
 * that would exceed it fails with HMC_ERR_OOM as cudaMalloc would on a full device.  Lets
 * a test drive hmc_create's fallback to passes over the rows without filling the GPU. */
HMC_API void hmc_diag_set_memory_cap(long bytes);

/* Whether batch handles created from now on run their tensor-core MLP problems as grouped
 * launches (on by default): problems whose engines share a kernel shape (padded width,
 * input width, kernel family), two or more of them, take one launch per kernel and layer
 * slot together instead of one per problem, with the same results bit for bit.  Off,
 * every problem launches its own kernels on the batch's concurrent lanes. */
HMC_API void hmc_diag_set_grouping(int on);

/* The groups of a batch handle, one line each (problems, width, launches per gradient),
 * NUL-terminated in buf (truncated to n bytes; buf may be NULL).  Returns the number of
 * groups, or -1 for a bad handle. */
HMC_API long hmc_diag_groups(hmc_handle h, char *buf, long n);

/* The energy the Metropolis test uses, for states q [C][k] (device or host; U [C] host
 * or device doubles): on the tensor-core engines the accurate forward pass with
 * hi/lo activations, elsewhere the energy of hmc_energy_grad. */
HMC_API hmc_status hmc_diag_metropolis_energy(hmc_handle h, const void *q, double *U);

/* What each problem's engine autotuned at creation (tile shapes and grids, with the
 * measured candidates), one line per problem, NUL-terminated in buf (truncated to n
 * bytes).  Returns the length of the full text. */
HMC_API long hmc_diag_tuning(hmc_handle h, char *buf, long n);

/* Run one bounded wait out on purpose: a one-thread kernel waits limit_ns (1 us .. 0.1 s)
 * on a shared-memory barrier that nothing arrives at, then records the timeout in the
 * error flag of the handle's first engine that keeps one (the tensor-core engines), as a
 * kernel whose pipeline stalled would.  No GPU fault or hang is involved.  The next
 * hmc_check returns HMC_ERR_TIMEOUT.  HMC_ERR_UNSUPPORTED when no engine keeps a flag. */
HMC_API hmc_status hmc_diag_expire_wait(hmc_handle h, long limit_ns);

typedef struct {
    char name[48];      /* kernel kind */
    double ms_total;    /* summed CUDA-event time over all its launches */
    long launches;
} hmc_kernel_time;

/* Run hmc_energy_grad on device states q reps times, synchronously, with a CUDA
 * event pair around every kernel launch on the stream it is launched on; the
 * timed evaluations are replayed from a CUDA graph so that the kernels run back
 * to back as in a trajectory.  Per-kind totals go to out[0..n-1]; the return
 * value is n, or minus an hmc_status on failure. */
HMC_API int hmc_diag_profile_energy_grad(hmc_handle h, const void *q, int reps, hmc_kernel_time *out,
                                         int max_out);

/* One batched BF16 tensor-core GEMM on the library's tcgen05 pipeline (TMA ->
 * shared memory -> tcgen05.mma -> TMEM -> registers), FP32 result:
 *   C[b][m][n] = sum_k A(m, k) B(n, k),  b < batch.
 * A is [batch][M][K] (a_mn = 0, K-major) or [batch][K][M] (a_mn = 1);
 * B is [batch][N][K] (b_mn = 0) or [batch][K][N] (b_mn = 1); all device pointers,
 * bf16, row-major.  N must be 64, 128, 192 or 256; M and K multiples of 8.
 * Synchronises the device before returning. */
HMC_API hmc_status hmc_diag_umma_gemm(int M, int N, int K, int batch, int a_mn, int b_mn, const void *A,
                                      const void *B, float *C);

#ifdef __cplusplus
}
#endif

#endif /* HMC_DIAG_H */

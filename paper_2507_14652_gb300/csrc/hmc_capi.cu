// hmc_capi.cu -- the C ABI (include/hmc.h): handles, argument checks, and the
// trajectory kernels that implement Algorithm 1 on the sampled subset
// (Algorithm 2): momentum draw, leapfrog kicks/drifts with the scatter of q into
// the network, kinetic energy and the Metropolis step.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "hmc_internal.cuh"
#include "k_rng.cuh"
#include "hmc_diag.h"

namespace hmc {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

// Whether new batch handles group their tensor-core problems (hmc_diag_set_grouping).
std::atomic<bool> g_grouping{true};

// Bytes held by DevBufs, and the cap hmc_diag_set_memory_cap may put on them.
std::atomic<size_t> g_devbuf_bytes{0};
std::atomic<size_t> g_devbuf_cap{~size_t(0)};

static void devbuf_free(void *&ptr, size_t n, bool own)
{
    if (ptr && own) {
        cudaFree(ptr);
        g_devbuf_bytes -= n;
    }
    ptr = nullptr;
}

void DevBuf::alloc(size_t bytes)
{
    devbuf_free(ptr, n, own);
    own = true;
    n = 0;
    if (bytes == 0) return;
    if (g_devbuf_bytes + bytes > g_devbuf_cap) {
        set_error("device allocation of %zu bytes exceeds the memory cap of %zu bytes", bytes, (size_t)g_devbuf_cap);
        throw Fail{HMC_ERR_OOM};
    }
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        ptr = nullptr;
        set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
        throw Fail{e == cudaErrorMemoryAllocation ? HMC_ERR_OOM : HMC_ERR_CUDA};
    }
    n = bytes;
    g_devbuf_bytes += bytes;
}

DevBuf::~DevBuf() { devbuf_free(ptr, n, own); }

void DevBuf::view(void *p, size_t bytes)
{
    devbuf_free(ptr, n, own);
    ptr = p;
    n = bytes;
    own = false;
}

void RowArena::take(DevBuf &dst, size_t bytes)
{
    if (next == slots.size()) slots.emplace_back(new DevBuf(bytes));
    DevBuf &s = *slots[next++];
    if (s.n < bytes) {
        set_error("internal: a chunk engine asked for more row memory than the first (largest) chunk");
        throw Fail{HMC_ERR_CUDA};
    }
    dst.view(s.ptr, bytes);
}

Profiler *&active_profiler()
{
    static thread_local Profiler *p = nullptr;
    return p;
}

ProfScope::ProfScope(const char *name, cudaStream_t st) : p(active_profiler()), s(st)
{
    if (!p) return;
    Profiler::Rec r{name, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecordWithFlags(r.a, s, cudaEventRecordExternal);   // a real record node when captured
    p->recs.push_back(r);
    i = p->recs.size() - 1;
}

ProfScope::~ProfScope()
{
    if (p) cudaEventRecordWithFlags(p->recs[i].b, s, cudaEventRecordExternal);
}

void build_net_desc(NetDesc &nd, const hmc_mlp_spec &s, long base, const std::vector<long> &idx)
{
    nd.L = s.n_layers;
    long off = base;
    for (int l = 0; l <= nd.L; ++l) nd.w[l] = s.widths[l];
    for (int l = 0; l < nd.L; ++l) {
        nd.act[l] = s.act[l];
        nd.bias[l] = s.has_bias[l] ? 1 : 0;
        nd.woff[l] = off;
        off += (long)nd.w[l + 1] * nd.w[l];
        nd.boff[l] = -1;
        if (nd.bias[l]) {
            nd.boff[l] = off;
            off += nd.w[l + 1];
        }
    }
    nd.base = base;
    nd.P = off - base;
    nd.any_sampled = false;
    nd.lmin = nd.L;
    for (int l = 0; l < nd.L; ++l) {
        long lo = nd.woff[l];
        long hi = nd.woff[l] + (long)nd.w[l + 1] * nd.w[l] + (nd.bias[l] ? nd.w[l + 1] : 0);
        auto it = std::lower_bound(idx.begin(), idx.end(), lo);
        if (it != idx.end() && *it < hi) {
            if (!nd.any_sampled) nd.lmin = l;
            nd.any_sampled = true;
        }
    }
    if (!nd.any_sampled) nd.lmin = nd.L;
}

// ---------------------------------------------------------------------------
// Trajectory kernels.  One block per (problem, chain) segment.
// ---------------------------------------------------------------------------

struct TrajState {
    long long traj;
    long long slot;
    void *samples;            // outputs of the current hmc_sample call (device; may be null)
    unsigned char *accepted;
    double *dH;
    // dual averaging of log eps during a warm-up (Hoffman and Gelman 2014, Sec. 3.2): the
    // updates so far; each problem's Hbar and log eps-bar are in the handle's da array
    long long da_m;
};

// The kick and drift of one launch for problem pi: eps / kick_div and eps / drift_div (a
// divisor of 0 means no kick, or no drift), eps read from the handle's per-problem step
// sizes in device memory when eps_p is set (captured trajectories, so that a new step
// size needs no new graph), else the literal eps for every problem.
struct Step {
    const double *eps_p;   // [problems]
    double eps;
    double kick_div, drift_div;
};

__device__ __forceinline__ double step_eps(const Step &s, int pi) { return s.eps_p ? s.eps_p[pi] : s.eps; }
__device__ __forceinline__ double step_kick(const Step &s, int pi)
{
    return s.kick_div != 0.0 ? step_eps(s, pi) / s.kick_div : 0.0;
}
__device__ __forceinline__ double step_drift(const Step &s, int pi)
{
    return s.drift_div != 0.0 ? step_eps(s, pi) / s.drift_div : 0.0;
}

// Write q into the network buffer b at offset o of chain c (bf16 or fp16 hi/lo pair, or plain).
template <typename T>
__device__ __forceinline__ void scatter_at(const ScatterPlan &sc, long c, int b, long off, T q)
{
    const long o = c * sc.cstride[b] + off;
    if (sc.kind16[b] == 1) {
        const __nv_bfloat16 hi = __float2bfloat16_rn((float)q);
        reinterpret_cast<__nv_bfloat16 *>(sc.base[b])[o] = hi;
        if (sc.base_lo[b])
            reinterpret_cast<__nv_bfloat16 *>(sc.base_lo[b])[o] = __float2bfloat16_rn((float)q - __bfloat162float(hi));
    } else if (sc.kind16[b] == 2) {
        const __half hi = __float2half_rn((float)q);
        reinterpret_cast<__half *>(sc.base[b])[o] = hi;
        if (sc.base_lo[b]) reinterpret_cast<__half *>(sc.base_lo[b])[o] = __float2half_rn((float)q - __half2float(hi));
    } else {
        reinterpret_cast<T *>(sc.base[b])[o] = q;
    }
}

template <typename T>
__device__ __forceinline__ void scatter_one(const ScatterPlan &sc, long c, long j, T q)
{
    scatter_at<T>(sc, c, sc.buf_id ? (int)sc.buf_id[j] : 0, (long)sc.off[j], q);
}

__device__ __forceinline__ double seg_sum(double v, double *sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sm[i];
    __syncthreads();
    return r;
}

// The trajectory kernels run on a (blocks per chain) x (problem, chain) grid; each
// block owns TRAJ_ELEMS consecutive coordinates of one chain.  Sums over a chain are
// per-block partials added in a fixed order, so results do not depend on scheduling.
constexpr int TRAJ_THREADS = 256;
constexpr int TRAJ_ELEMS = 4 * TRAJ_THREADS;

__device__ __forceinline__ void load_seg(SegDesc &dst, const SegDesc *src)
{
    const int *a = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(SegDesc) / 4); i += blockDim.x) d[i] = a[i];
    __syncthreads();
}

// p ~ N(0, I); partial sums of p.p; first half kick p -= eps/2 g; first drift q* = q + drift p
// (drift = eps for the leapfrog); scatter q*.  stp gives the kick eps/2 and the drift.
template <typename T>
__global__ void __launch_bounds__(TRAJ_THREADS) k_traj_begin(const SegDesc *segs, int C, int nblk, const T *q_cur,
                                                             const T *g_cur, T *q_prop, T *p, double *K0p,
                                                             Step stp, uint64_t seed, const TrajState *st)
{
    __shared__ __align__(16) unsigned char sd_raw[sizeof(SegDesc)];
    SegDesc &sd = *reinterpret_cast<SegDesc *>(sd_raw);
    __shared__ double sm[8];
    pdl_wait();
    pdl_trigger();
    const int s = blockIdx.y, pi = s / C, c = s % C;
    load_seg(sd, &segs[pi]);
    const long j0 = (long)blockIdx.x * TRAJ_ELEMS;
    double kin = 0.0;
    if (j0 < sd.k) {
        const long base = sd.qoff + (long)c * sd.k;
        const uint64_t traj = (uint64_t)st->traj;
        const T h = (T)step_kick(stp, pi), e = (T)step_drift(stp, pi);
        const long blk = j0 / 4 + threadIdx.x;
        if (blk * 4 < sd.k) {
            double z[4];
            momenta4(seed, (uint64_t)sd.problem, (uint64_t)c, traj, (uint64_t)blk, z);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const long j = blk * 4 + t;
                if (j >= sd.k) break;
                T pj = (T)z[t];
                kin += (double)pj * (double)pj;
                pj = pj - h * g_cur[base + j];
                const T qj = q_cur[base + j] + e * pj;
                p[base + j] = pj;
                q_prop[base + j] = qj;
                scatter_one<T>(sd.sc, c, j, qj);
            }
        }
    }
    const double tot = seg_sum(kin, sm);
    if (threadIdx.x == 0) K0p[(long)s * nblk + blockIdx.x] = tot;
}

// p -= kick g; q += drift p; scatter q.
template <typename T>
__global__ void __launch_bounds__(TRAJ_THREADS) k_kick_drift(const SegDesc *segs, int C, const T *g, T *p, T *q,
                                                             Step stp)
{
    __shared__ __align__(16) unsigned char sd_raw[sizeof(SegDesc)];
    SegDesc &sd = *reinterpret_cast<SegDesc *>(sd_raw);
    pdl_wait();
    pdl_trigger();
    const int s = blockIdx.y, pi = s / C, c = s % C;
    load_seg(sd, &segs[pi]);
    const long base = sd.qoff + (long)c * sd.k;
    const bool kick = stp.kick_div != 0.0, drift = stp.drift_div != 0.0;
    const T kk = (T)step_kick(stp, pi), dd = (T)step_drift(stp, pi);
    const long j0 = (long)blockIdx.x * TRAJ_ELEMS;
    // every load of the thread's four coordinates first, then the dependent updates
    T pv[4], gv[4], qv[4];
    int bv[4];
    long ov[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const long j = j0 + threadIdx.x + (long)t * TRAJ_THREADS;
        pv[t] = gv[t] = qv[t] = (T)0;
        bv[t] = 0;
        ov[t] = 0;
        if (j < sd.k) {
            pv[t] = p[base + j];
            if (kick) gv[t] = g[base + j];
            if (drift) {
                qv[t] = q[base + j];
                bv[t] = sd.sc.buf_id ? (int)sd.sc.buf_id[j] : 0;
                ov[t] = (long)sd.sc.off[j];
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const long j = j0 + threadIdx.x + (long)t * TRAJ_THREADS;
        if (j >= sd.k) break;
        T pj = pv[t];
        if (kick) pj = pj - kk * gv[t];
        p[base + j] = pj;
        if (drift) {
            const T qj = qv[t] + dd * pj;
            q[base + j] = qj;
            scatter_at<T>(sd.sc, c, bv[t], ov[t], qj);
        }
    }
}

// Last half kick (p itself is not needed afterwards) and partial sums of p.p.
template <typename T>
__global__ void __launch_bounds__(TRAJ_THREADS) k_traj_kinetic(const SegDesc *segs, int C, int nblk, const T *p,
                                                               const T *g_prop, double *K1p, Step stp)
{
    __shared__ double sm[8];
    pdl_wait();
    pdl_trigger();
    const int s = blockIdx.y, pi = s / C, c = s % C;
    const long k = segs[pi].k;
    const long base = segs[pi].qoff + (long)c * k;
    const T h = (T)step_kick(stp, pi);
    const long j0 = (long)blockIdx.x * TRAJ_ELEMS;
    double kin = 0.0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const long j = j0 + threadIdx.x + (long)t * TRAJ_THREADS;
        if (j >= k) break;
        const T pj = p[base + j] - h * g_prop[base + j];
        kin += (double)pj * (double)pj;
    }
    const double tot = seg_sum(kin, sm);
    if (threadIdx.x == 0) K1p[(long)s * nblk + blockIdx.x] = tot;
}

// Metropolis step.  Every block of a chain recomputes the same decision from the same
// fixed-order sums (H0 = U + K0, H1 = U* + K1, accept iff log u < H0 - H1), then
// copies its slice of the state; block 0 records the outputs.
template <typename T>
__global__ void __launch_bounds__(TRAJ_THREADS) k_traj_accept(const SegDesc *segs, int C, int nblk, int nseg,
                                                              long S_total, T *q_cur, T *g_cur, const double *U_cur,
                                                              const T *q_prop, const T *g_prop, const double *U_prop,
                                                              const double *K0p, const double *K1p, uint64_t seed,
                                                              const TrajState *st, int *acc_int)
{
    __shared__ int s_acc;
    pdl_wait();
    pdl_trigger();
    const int s = blockIdx.y, pi = s / C, c = s % C;
    const long k = segs[pi].k;
    const long base = segs[pi].qoff + (long)c * k;
    const long long slot = st->slot;
    if (threadIdx.x == 0) {
        double K0 = 0.0, K1 = 0.0;
        for (int i = 0; i < nblk; ++i) {
            K0 += K0p[(long)s * nblk + i];
            K1 += K1p[(long)s * nblk + i];
        }
        const double H0 = U_cur[s] + 0.5 * K0;
        const double H1 = U_prop[s] + 0.5 * K1;
        const double lu = mh_log_uniform(seed, (uint64_t)segs[pi].problem, (uint64_t)c, (uint64_t)st->traj);
        const int a = lu < H0 - H1;
        s_acc = a;
        if (blockIdx.x == 0) {
            acc_int[s] = a;
            if (st->accepted) st->accepted[slot * nseg + s] = (unsigned char)a;
            if (st->dH) st->dH[slot * nseg + s] = H1 - H0;
        }
    }
    __syncthreads();
    const int a = s_acc;
    T *samples = static_cast<T *>(st->samples);
    const long j0 = (long)blockIdx.x * TRAJ_ELEMS;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const long j = j0 + threadIdx.x + (long)t * TRAJ_THREADS;
        if (j >= k) break;
        T qj = q_cur[base + j];
        if (a) {
            qj = q_prop[base + j];
            q_cur[base + j] = qj;
            g_cur[base + j] = g_prop[base + j];
        }
        if (samples) samples[slot * S_total + base + j] = qj;
    }
}

// After every block has decided: commit U of accepted chains, advance the counters.
__global__ void k_traj_advance(TrajState *st, int nseg, const int *acc_int, double *U_cur, const double *U_prop)
{
    pdl_wait();
    pdl_trigger();
    for (int s = threadIdx.x; s < nseg; s += blockDim.x)
        if (acc_int[s]) U_cur[s] = U_prop[s];
    if (threadIdx.x == 0) {
        st->traj += 1;
        st->slot += 1;
    }
}

// New trajectory counters and outputs; every problem's step set to eps_src[i] (device
// array) or to eps, and its dual-averaging state cleared.
__global__ void k_set_state(TrajState *st, long long traj, long long slot, void *samples, unsigned char *acc,
                            double *dH, double *eps_prob, double *da, int nprob, const double *eps_src, double eps)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->traj = traj;
        st->slot = slot;
        st->samples = samples;
        st->accepted = acc;
        st->dH = dH;
        st->da_m = 0;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nprob; i += gridDim.x * blockDim.x) {
        eps_prob[i] = eps_src ? eps_src[i] : eps;
        da[2 * i] = 0.0;
        da[2 * i + 1] = 0.0;
    }
}

// One dual-averaging update (Hoffman and Gelman 2014, Sec. 3.2, their Algorithm 5
// without the NUTS parts) of every problem's step after trajectory slot - 1 of a warm-up.
// A warp per problem: the statistic is the mean over the problem's C chains of
// min(1, exp(-dH)) (a non-finite dH counts as 0), strided over the lanes and summed in a
// fixed butterfly; the new step goes to eps_prob[pi] for the next trajectory.
// trace[2 (m - 1) nprob + 2 pi] = exp(log eps_m), [... + 1] = exp(log eps-bar_m).
__global__ void __launch_bounds__(256) k_dual_avg(TrajState *st, double *eps_prob, double *da, int nprob, int C,
                                                  double target, double mu, double gamma, double t0, double kappa,
                                                  double *trace)
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const long long m = st->da_m + 1;
    const double *dh = st->dH + (st->slot - 1) * (long long)nprob * C;
    for (int pi = threadIdx.x >> 5; pi < nprob; pi += nw) {
        double a = 0.0;
        for (int c = lane; c < C; c += 32) {
            const double v = dh[(long)pi * C + c];
            a += isfinite(v) ? fmin(1.0, exp(-v)) : 0.0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) {
            const double abar = a / (double)C;
            const double w = 1.0 / ((double)m + t0);
            const double hbar = (1.0 - w) * da[2 * pi] + w * (target - abar);
            const double log_eps = mu - sqrt((double)m) / gamma * hbar;
            const double eta = pow((double)m, -kappa);
            const double lbar = eta * log_eps + (1.0 - eta) * da[2 * pi + 1];
            da[2 * pi] = hbar;
            da[2 * pi + 1] = lbar;
            eps_prob[pi] = exp(log_eps);
            if (trace) {
                trace[2 * ((m - 1) * nprob + pi)] = exp(log_eps);
                trace[2 * ((m - 1) * nprob + pi) + 1] = exp(lbar);
            }
        }
    }
    __syncthreads();   // every warp has read m
    if (threadIdx.x == 0) st->da_m = m;
}

__global__ void k_rewind_slot(TrajState *st) { st->slot = 0; }
__global__ void k_advance_slot(TrajState *st) { st->slot += 1; }

__global__ void k_debug_momenta(uint64_t seed, uint64_t problem, uint64_t chain, uint64_t traj, long k, double *out)
{
    for (long blk = (long)blockIdx.x * blockDim.x + threadIdx.x; blk * 4 < k; blk += (long)gridDim.x * blockDim.x) {
        double z[4];
        momenta4(seed, problem, chain, traj, (uint64_t)blk, z);
        for (int t = 0; t < 4; ++t)
            if (blk * 4 + t < k) out[blk * 4 + t] = z[t];
    }
}

__global__ void k_debug_logu(uint64_t seed, uint64_t problem, long n_chain, long n_traj, double *out)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_chain * n_traj; i += (long)gridDim.x * blockDim.x)
        out[i] = mh_log_uniform(seed, problem, (uint64_t)(i / n_traj), (uint64_t)(i % n_traj));
}

__global__ void k_debug_philox(const uint64_t *ctr, const uint64_t *key, long n, uint64_t *out)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        uint64_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
        philox4x64_10(c, key[2 * i], key[2 * i + 1]);
        for (int t = 0; t < 4; ++t) out[4 * i + t] = c[t];
    }
}

__global__ void k_nonfinite_count(const double *U, int n, int *out)
{
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) bad += isfinite(U[i]) ? 0 : 1;
    atomicAdd(out, bad);
}

// U[c] = sum over batches m (in order) of U_split[m][c].
__global__ void k_split_energy_sum(const double *U_split, int M, int C, double *U)
{
    pdl_wait();
    pdl_trigger();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        double u = 0.0;
        for (int m = 0; m < M; ++m) u += U_split[(long)m * C + c];
        U[c] = u;
    }
}

// g += d, elementwise over n entries.
template <typename T> __global__ void k_accumulate(T *g, const T *d, long n)
{
    pdl_wait();
    pdl_trigger();
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        g[i] = g[i] + d[i];
}

}  // namespace hmc

using namespace hmc;

struct hmc_handle_s {
    int prec = 0;
    int C = 0;
    int nprob = 0;
    size_t elem = 4;
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // batches: each problem's gradient runs on its own stream between a fork and a join
    // event, so the problems overlap on the GPU (and become parallel graph branches)
    std::vector<cudaStream_t> lanes;
    // batches of tensor-core MLPs: problems of one kernel shape run as grouped launches
    // (grouped[i]: problem i belongs to one of the groups)
    std::vector<std::unique_ptr<EngineGroup>> groups;
    std::vector<bool> grouped;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    std::vector<std::unique_ptr<Problem>> probs;
    std::vector<std::unique_ptr<Engine>> engines;
    // split handles (hmc_create_split): one problem whose data rows are cut into
    // nsplit batches, engines[m] holding batch m with 1/nsplit of the prior
    int nsplit = 1;
    // chunked handles (hmc_create_chunked): the same per-batch engines, integrated by the
    // full-batch leapfrog with U and grad U summed over the batches, which share one
    // arena of row buffers
    bool chunked = false;
    std::unique_ptr<RowArena> arena;
    DevBuf U_split, g_tmp;
    std::vector<long> qoff;
    long k_total = 0, P_total = 0, S_total = 0;
    DevBuf q_cur, g_cur, q_prop, p, g_prop, U_cur, U_prop, K0p, K1p, acc_int, segs, state, scratch;
    int traj_nblk = 1;   // blocks per chain in the trajectory kernels
    // staging buffers for host arguments, kept across calls (allocating and freeing device
    // memory on every call would synchronise the device twice per call)
    std::vector<std::unique_ptr<DevBuf>> stage;
    size_t stage_used = 0;
    // one trajectory as an executable graph, reused while (L, seed) stay the same
    cudaGraphExec_t traj_exec = nullptr;
    int traj_L = -1;
    unsigned long long traj_seed = 0;
    long traj_kernels = 0;     // kernel nodes in that graph
    long traj_captures = 0;    // graphs captured so far
    DevBuf adapt_trace;        // [n][problems][2] step sizes of the last warm-up (hmc_diag_adapt_trace)
    DevBuf eps_prob;           // [problems] step sizes the captured trajectories read
    DevBuf da_state;           // [problems][2] dual averaging: Hbar, log eps-bar
    long adapt_n = 0;
    ~hmc_handle_s()
    {
        if (traj_exec) cudaGraphExecDestroy(traj_exec);
        for (cudaStream_t l : lanes) cudaStreamDestroy(l);
        for (cudaEvent_t e : ev_join) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
};

namespace {

bool is_device_ptr(const void *ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void check_mlp_spec(const hmc_mlp_spec &s, const char *what)
{
    HMC_REQUIRE(s.n_layers >= 1 && s.n_layers <= HMC_MAX_LAYERS, "%s: n_layers must be in [1, %d]", what,
                HMC_MAX_LAYERS);
    for (int l = 0; l <= s.n_layers; ++l)
        HMC_REQUIRE(s.widths[l] >= 1 && s.widths[l] <= (1 << 20), "%s: widths[%d] = %d is out of range", what, l,
                    s.widths[l]);
    for (int l = 0; l < s.n_layers; ++l)
        HMC_REQUIRE(s.act[l] >= HMC_ACT_IDENTITY && s.act[l] <= HMC_ACT_SIN, "%s: act[%d] = %d is invalid", what, l,
                    s.act[l]);
}

template <typename V> std::vector<V> fetch(const V *src, long n, const char *what)
{
    HMC_REQUIRE(n == 0 || src != nullptr, "%s is NULL", what);
    std::vector<V> v((size_t)n);
    if (n > 0) HMC_CK(cudaMemcpy(v.data(), src, sizeof(V) * (size_t)n, cudaMemcpyDefault));
    return v;
}

// A training-set array of element type `dtype` (hmc_data_dtype), host or device, as doubles.
std::vector<double> fetch_data(const void *src, long n, int dtype, const char *what)
{
    HMC_REQUIRE(dtype == HMC_DATA_F64 || dtype == HMC_DATA_F32, "%s: unknown dtype %d", what, dtype);
    if (dtype == HMC_DATA_F64) return fetch(static_cast<const double *>(src), n, what);
    const std::vector<float> f = fetch(static_cast<const float *>(src), n, what);
    return std::vector<double>(f.begin(), f.end());
}

std::unique_ptr<Problem> build_problem(const hmc_net_spec &spec, const hmc_data &d, double alpha, double sigma,
                                       const unsigned char *mask, const double *frozen, int C)
{
    HMC_REQUIRE(spec.kind == HMC_NET_MLP || spec.kind == HMC_NET_DEEPONET || spec.kind == HMC_NET_DEEPONET_UNALIGNED,
                "unknown net kind %d", spec.kind);
    HMC_REQUIRE(alpha > 0 && sigma > 0 && std::isfinite(alpha) && std::isfinite(sigma),
                "prior_sigma and noise_sigma must be positive and finite");
    auto p = std::make_unique<Problem>();
    p->kind = spec.kind;
    p->C = C;
    p->alpha = alpha;
    p->sigma = sigma;
    long P = 0;
    if (spec.kind == HMC_NET_MLP) {
        check_mlp_spec(spec.net, "net");
        HMC_REQUIRE(d.n >= 0 && d.dx == spec.net.widths[0], "data.dx (%d) must equal widths[0] (%d)", d.dx,
                    spec.net.widths[0]);
        for (int l = 0; l < spec.net.n_layers; ++l)
            P += (long)spec.net.widths[l + 1] * spec.net.widths[l] + (spec.net.has_bias[l] ? spec.net.widths[l + 1] : 0);
    } else {
        check_mlp_spec(spec.branch, "branch");
        check_mlp_spec(spec.trunk, "trunk");
        HMC_REQUIRE(spec.branch.widths[spec.branch.n_layers] == spec.trunk.widths[spec.trunk.n_layers],
                    "branch and trunk output widths differ");
        HMC_REQUIRE(d.n_u >= 0 && d.n_y >= 0 && d.du == spec.branch.widths[0] && d.dy == spec.trunk.widths[0],
                    "DeepONet data dimensions do not match the spec");
        for (const hmc_mlp_spec *s : {&spec.branch, &spec.trunk})
            for (int l = 0; l < s->n_layers; ++l)
                P += (long)s->widths[l + 1] * s->widths[l] + (s->has_bias[l] ? s->widths[l + 1] : 0);
        P += spec.deeponet_out_bias ? 1 : 0;
    }
    HMC_REQUIRE(P < (1L << 31), "too many parameters (%ld)", P);
    p->P = P;
    auto m = fetch(mask, P, "subset_mask");
    p->frozen = fetch(frozen, P, "frozen_params");
    for (long i = 0; i < P; ++i)
        if (m[i]) p->idx.push_back(i);
    p->k = (long)p->idx.size();
    HMC_REQUIRE(p->k >= 1, "subset_mask selects no parameter");
    if (spec.kind == HMC_NET_MLP) {
        build_net_desc(p->net, spec.net, 0, p->idx);
        p->n = d.n;
        p->dx = d.dx;
        p->dout = spec.net.widths[spec.net.n_layers];
        p->x = fetch_data(d.x, d.n * d.dx, d.dtype, "data.x");
        p->y = fetch_data(d.y, d.n * p->dout, d.dtype, "data.y");
    } else {
        build_net_desc(p->branch, spec.branch, 0, p->idx);
        build_net_desc(p->trunk, spec.trunk, p->branch.P, p->idx);
        p->out_bias = spec.deeponet_out_bias ? 1 : 0;
        p->b0_off = p->out_bias ? p->branch.P + p->trunk.P : -1;
        p->n_u = d.n_u;
        p->n_y = d.n_y;
        p->du = d.du;
        p->dy = d.dy;
        p->u = fetch_data(d.u, d.n_u * d.du, d.dtype, "data.u");
        const long nq = spec.kind == HMC_NET_DEEPONET_UNALIGNED ? d.n_u * d.n_y : d.n_y;
        p->yq = fetch_data(d.yq, nq * d.dy, d.dtype, "data.yq");
        p->t = fetch_data(d.t, d.n_u * d.n_y, d.dtype, "data.t");
    }
    return p;
}

void join_in(hmc_handle h)
{
    HMC_CK(cudaEventRecord(h->ev_in, h->user_stream));
    HMC_CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
}

void join_out(hmc_handle h)
{
    HMC_CK(cudaEventRecord(h->ev_out, h->stream));
    HMC_CK(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
}

// Run fn(problem, stream) for every problem.  Batches fork onto the handle's lanes
// (problem i on lane i mod lanes) and join back on the handle's stream, so the
// problems overlap on the GPU and a captured trajectory has one branch per lane.
template <typename F> void for_each_problem(hmc_handle h, F &&fn)
{
    if (h->nprob == 1) {
        fn(0, h->stream);
        return;
    }
    HMC_CK(cudaEventRecord(h->ev_fork, h->stream));
    for (cudaStream_t l : h->lanes) HMC_CK(cudaStreamWaitEvent(l, h->ev_fork, 0));
    for (int i = 0; i < h->nprob; ++i) fn(i, h->lanes[i % h->lanes.size()]);
    for (size_t j = 0; j < h->lanes.size(); ++j) {
        HMC_CK(cudaEventRecord(h->ev_join[j], h->lanes[j]));
        HMC_CK(cudaStreamWaitEvent(h->stream, h->ev_join[j], 0));
    }
}

void split_energy_grad_full(hmc_handle h, const void *q, double *U, void *g);

void energy_grad_all(hmc_handle h, void *q, double *U, void *g, bool scattered)
{
    if (h->nsplit > 1) {
        split_energy_grad_full(h, q, U, g);
        return;
    }
    if (!h->groups.empty()) {   // each group on a lane of its own, the other problems after them
        HMC_CK(cudaEventRecord(h->ev_fork, h->stream));
        for (cudaStream_t l : h->lanes) HMC_CK(cudaStreamWaitEvent(l, h->ev_fork, 0));
        size_t lane = 0;
        for (auto &gr : h->groups) gr->energy_grad(q, U, g, scattered, h->lanes[lane++ % h->lanes.size()]);
        for (int i = 0; i < h->nprob; ++i) {
            if (h->grouped[i]) continue;
            char *qb = static_cast<char *>(q) + h->qoff[i] * h->elem;
            char *gb = g ? static_cast<char *>(g) + h->qoff[i] * h->elem : nullptr;
            h->engines[i]->energy_grad(qb, U + (long)i * h->C, gb, scattered, h->lanes[lane++ % h->lanes.size()]);
        }
        for (size_t j = 0; j < h->lanes.size(); ++j) {
            HMC_CK(cudaEventRecord(h->ev_join[j], h->lanes[j]));
            HMC_CK(cudaStreamWaitEvent(h->stream, h->ev_join[j], 0));
        }
        return;
    }
    for_each_problem(h, [&](int i, cudaStream_t s) {
        char *qb = static_cast<char *>(q) + h->qoff[i] * h->elem;
        char *gb = g ? static_cast<char *>(g) + h->qoff[i] * h->elem : nullptr;
        h->engines[i]->energy_grad(qb, U + (long)i * h->C, gb, scattered, s);
    });
}

// Overwrite U with the accurate energy where an engine's energy_grad U is a
// reduced-precision one (q already scattered by the preceding energy_grad_all).
void split_energy(hmc_handle h, int m, const void *q);
void split_sum(hmc_handle h, double *U);

void accurate_energy_all(hmc_handle h, void *q, double *U)
{
    if (h->nsplit > 1) {
        bool any = false;
        for (auto &e : h->engines) any = any || e->has_accurate_energy();
        if (!any) return;
        for (int m = 0; m < h->nsplit; ++m) split_energy(h, m, q);
        split_sum(h, U);
        return;
    }
    bool any = false;
    for (auto &e : h->engines) any = any || e->has_accurate_energy();
    if (!any) return;
    for_each_problem(h, [&](int i, cudaStream_t s) {
        Engine *e = h->engines[i].get();
        if (!e->has_accurate_energy()) return;
        char *qb = static_cast<char *>(q) + h->qoff[i] * h->elem;
        e->accurate_energy(qb, U + (long)i * h->C, s);
    });
}

// A device view of a user array: the pointer itself when it is device memory,
// otherwise a staging buffer (copied in when `in`).
void *dev_view(hmc_handle h, const void *user, size_t bytes, bool in, bool *staged)
{
    *staged = false;
    if (!user) return nullptr;
    if (is_device_ptr(user)) return const_cast<void *>(user);
    if (h->stage_used == h->stage.size()) h->stage.emplace_back(new DevBuf());
    std::unique_ptr<DevBuf> &buf = h->stage[h->stage_used++];
    if (buf->n < bytes) buf.reset(new DevBuf(bytes));
    void *d = buf->ptr;
    if (in) HMC_CK(cudaMemcpyAsync(d, user, bytes, cudaMemcpyHostToDevice, h->stream));
    *staged = true;
    return d;
}

void kick_drift(hmc_handle h, void *q, void *p, const void *g, Step stp)
{
    const int nseg = h->nprob * h->C;
    const SegDesc *sd = h->segs.as<SegDesc>();
    const dim3 grid(h->traj_nblk, nseg);
    if (h->prec == HMC_PREC_FP64)
        launch_pdl(k_kick_drift<double>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, (const double *)g,
                   (double *)p, (double *)q, stp);
    else
        launch_pdl(k_kick_drift<float>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, (const float *)g,
                   (float *)p, (float *)q, stp);
    HMC_LAUNCH_CK();
}

// ---- symmetric split integrator (split handles) ----------------------------------
// H = sum_m [U_m + K/M] with U_m the likelihood of data batch m plus 1/M of the prior
// (engine m).  One step of size eps: for m = 1..M { p -= eps/2 grad U_m; q += eps/(2M) p }
// then for m = M..1 { q += eps/(2M) p; p -= eps/2 grad U_m }.  The launches below fuse
// each kick with the drift after it, and the last kick of a step (batch 1) with the
// first kick of the next, so a step costs 2M - 1 batch gradients.

// grad U_m(q) into g and U_m into U_split[m]; engine m scatters q itself.
void split_grad(hmc_handle h, int m, const void *q, void *g)
{
    h->engines[m]->energy_grad(q, h->U_split.as<double>() + (long)m * h->C, g, false, h->stream);
}

// U_m(q) only, the accurate one where the engine has it.
void split_energy(hmc_handle h, int m, const void *q)
{
    Engine *e = h->engines[m].get();
    double *Um = h->U_split.as<double>() + (long)m * h->C;
    if (e->has_accurate_energy()) {
        e->scatter(q, h->stream);
        e->accurate_energy(q, Um, h->stream);
    } else {
        e->energy_grad(q, Um, nullptr, false, h->stream);
    }
}

void split_sum(hmc_handle h, double *U)
{
    launch_pdl(k_split_energy_sum, dim3((h->C + 255) / 256), dim3(256), 0, h->stream, h->U_split.as<double>(),
               h->nsplit, h->C, U);
    HMC_LAUNCH_CK();
}

// U and grad U of the whole data set: the sums over the batches.
void split_energy_grad_full(hmc_handle h, const void *q, double *U, void *g)
{
    const long n = h->S_total;
    for (int m = 0; m < h->nsplit; ++m) {
        if (!g) {
            h->engines[m]->energy_grad(q, h->U_split.as<double>() + (long)m * h->C, nullptr, false, h->stream);
            continue;
        }
        split_grad(h, m, q, m == 0 ? g : h->g_tmp.ptr);
        if (m == 0) continue;
        const dim3 grid((unsigned)std::min<long>((n + 255) / 256, 4096));
        if (h->prec == HMC_PREC_FP64)
            launch_pdl(k_accumulate<double>, grid, dim3(256), 0, h->stream, (double *)g, h->g_tmp.as<double>(), n);
        else
            launch_pdl(k_accumulate<float>, grid, dim3(256), 0, h->stream, (float *)g, h->g_tmp.as<float>(), n);
        HMC_LAUNCH_CK();
    }
    split_sum(h, U);
}

// The Metropolis energy sum_m U_m(q) into U, and grad U_1(q) (batch 1) into g1.
void split_start(hmc_handle h, const void *q, double *U, void *g1)
{
    for (int m = h->nsplit - 1; m >= 1; --m) split_energy(h, m, q);
    split_grad(h, 0, q, g1);
    if (h->engines[0]->has_accurate_energy())
        h->engines[0]->accurate_energy(q, h->U_split.as<double>(), h->stream);
    split_sum(h, U);
}

// L split steps on (q, p).  On entry p has had the first half kick with grad U_1 and q
// its first drift; on exit g1 = grad U_1(q_end) and U_split[0] = U_1(q_end), and the
// final half kick is still to be applied.  The step is *eps_p when eps_p is set (a
// captured trajectory), else eps; the drifts are eps/(2M) (eps/M where two meet).
void split_steps(hmc_handle h, void *q, void *p, void *g1, const double *eps_p, double eps, int L)
{
    const int M = h->nsplit;
    const double dd = 2.0 * M, d0 = M == 1 ? 1.0 : dd;
    for (int s = 1; s <= L; ++s) {
        for (int m = 1; m < M; ++m) {   // forward sweep, batches 2..M
            split_grad(h, m, q, h->g_tmp.ptr);
            kick_drift(h, q, p, h->g_tmp.ptr, Step{eps_p, eps, 2.0, m < M - 1 ? dd : (double)M});
        }
        for (int m = M - 1; m >= 1; --m) {   // backward sweep, batches M..2
            split_grad(h, m, q, h->g_tmp.ptr);
            kick_drift(h, q, p, h->g_tmp.ptr, Step{eps_p, eps, 2.0, dd});
        }
        split_grad(h, 0, q, g1);
        if (s < L) kick_drift(h, q, p, g1, Step{eps_p, eps, 1.0, d0});
    }
}

// The step size of a captured trajectory is read from the device state (TrajState::eps),
// so one graph serves every step size.
template <typename T> void enqueue_split_trajectory(hmc_handle h, int L, uint64_t seed)
{
    const int nseg = h->C, nblk = h->traj_nblk, M = h->nsplit;
    const SegDesc *sd = h->segs.as<SegDesc>();
    TrajState *st = h->state.as<TrajState>();
    const double *ep = h->eps_prob.as<double>();
    const dim3 grid(nblk, nseg);
    launch_pdl(k_traj_begin<T>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, nblk, h->q_cur.as<T>(),
               h->g_cur.as<T>(), h->q_prop.as<T>(), h->p.as<T>(), h->K0p.as<double>(),
               Step{ep, 0.0, 2.0, M == 1 ? 1.0 : 2.0 * M}, seed, st);
    HMC_LAUNCH_CK();
    split_steps(h, h->q_prop.ptr, h->p.ptr, h->g_prop.ptr, ep, 0.0, L);
    // H1: the other batches' energies at the end point (batch 1's came with its gradient)
    for (int m = M - 1; m >= 1; --m) split_energy(h, m, h->q_prop.ptr);
    if (h->engines[0]->has_accurate_energy())
        h->engines[0]->accurate_energy(h->q_prop.ptr, h->U_split.as<double>(), h->stream);
    split_sum(h, h->U_prop.as<double>());
    launch_pdl(k_traj_kinetic<T>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, nblk, h->p.as<T>(),
               h->g_prop.as<T>(), h->K1p.as<double>(), Step{ep, 0.0, 2.0, 0.0});
    HMC_LAUNCH_CK();
    launch_pdl(k_traj_accept<T>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, nblk, nseg, h->S_total,
               h->q_cur.as<T>(), h->g_cur.as<T>(), h->U_cur.as<double>(), h->q_prop.as<T>(), h->g_prop.as<T>(),
               h->U_prop.as<double>(), h->K0p.as<double>(), h->K1p.as<double>(), seed, st, h->acc_int.as<int>());
    HMC_LAUNCH_CK();
    launch_pdl(k_traj_advance, dim3(1), dim3(256), 0, h->stream, st, nseg, h->acc_int.as<int>(),
               h->U_cur.as<double>(), h->U_prop.as<double>());
    HMC_LAUNCH_CK();
}

template <typename T> void enqueue_trajectory(hmc_handle h, int L, uint64_t seed)
{
    if (h->nsplit > 1 && !h->chunked) {
        enqueue_split_trajectory<T>(h, L, seed);
        return;
    }
    const int nseg = h->nprob * h->C, nblk = h->traj_nblk;
    const SegDesc *sd = h->segs.as<SegDesc>();
    TrajState *st = h->state.as<TrajState>();
    const double *ep = h->eps_prob.as<double>();
    const dim3 grid(nblk, nseg);
    launch_pdl(k_traj_begin<T>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, nblk, h->q_cur.as<T>(),
               h->g_cur.as<T>(), h->q_prop.as<T>(), h->p.as<T>(), h->K0p.as<double>(), Step{ep, 0.0, 2.0, 1.0}, seed,
               st);
    HMC_LAUNCH_CK();
    for (int s = 1; s <= L; ++s) {
        energy_grad_all(h, h->q_prop.ptr, h->U_prop.as<double>(), h->g_prop.ptr, true);
        if (s == L) accurate_energy_all(h, h->q_prop.ptr, h->U_prop.as<double>());   // H1 for the Metropolis test
        if (s < L) {
            launch_pdl(k_kick_drift<T>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, h->g_prop.as<T>(),
                       h->p.as<T>(), h->q_prop.as<T>(), Step{ep, 0.0, 1.0, 1.0});
            HMC_LAUNCH_CK();
        }
    }
    launch_pdl(k_traj_kinetic<T>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, nblk, h->p.as<T>(),
               h->g_prop.as<T>(), h->K1p.as<double>(), Step{ep, 0.0, 2.0, 0.0});
    HMC_LAUNCH_CK();
    launch_pdl(k_traj_accept<T>, grid, dim3(TRAJ_THREADS), 0, h->stream, sd, h->C, nblk, nseg, h->S_total,
               h->q_cur.as<T>(), h->g_cur.as<T>(), h->U_cur.as<double>(), h->q_prop.as<T>(), h->g_prop.as<T>(),
               h->U_prop.as<double>(), h->K0p.as<double>(), h->K1p.as<double>(), seed, st, h->acc_int.as<int>());
    HMC_LAUNCH_CK();
    launch_pdl(k_traj_advance, dim3(1), dim3(256), 0, h->stream, st, nseg, h->acc_int.as<int>(),
               h->U_cur.as<double>(), h->U_prop.as<double>());
    HMC_LAUNCH_CK();
}

// in_batch: inside a BF16 batch, a network the tensor-core kernels do not cover (a hidden
// width above 256, say) runs on the FP32 CUDA-core engine, which
// keeps the batch's float positions and is the more accurate of the two.
Engine *make_engine(Problem &p, int prec, int C, bool in_batch = false)
{
    if (prec == HMC_PREC_TF32) {
        set_error("HMC_PREC_TF32 is not implemented");
        throw Fail{HMC_ERR_UNSUPPORTED};
    }
    // no data terms: the potential is the prior alone, in every precision
    const bool no_data = p.kind == HMC_NET_MLP ? p.n == 0 : (p.n_u == 0 || p.n_y == 0);
    if (no_data) return make_prior_engine(p, prec, C);
    if (prec == HMC_PREC_FP64) return make_simt_engine_f64(p, C);
    if (prec == HMC_PREC_FP32) return make_simt_engine_f32(p, C);
    if (prec == HMC_PREC_BF16 || prec == HMC_PREC_FP16) {
        std::string why;
        const bool don = p.kind != HMC_NET_MLP;
        if (!(don ? don_engine_supports(p, &why) : umma_engine_supports(p, &why))) {
            if (in_batch) return make_simt_engine_f32(p, C);
            set_error("%s tensor-core path does not support this network: %s",
                      prec == HMC_PREC_BF16 ? "BF16" : "FP16", why.c_str());
            throw Fail{HMC_ERR_UNSUPPORTED};
        }
        if (prec == HMC_PREC_FP16) return don ? make_don_engine_f16(p, C) : make_umma_engine_f16(p, C);
        return don ? make_don_engine_bf16(p, C) : make_umma_engine_bf16(p, C);
    }
    set_error("unknown precision %d", prec);
    throw Fail{HMC_ERR_ARG};
}

// Data batch m of M (rows [floor(m R / M), floor((m + 1) R / M)) of the R data rows:
// MLP points, or DeepONet input functions with all their queries), with 1/M of the
// prior: alpha scaled by sqrt(M) makes its q^2 / (2 alpha^2) term 1/M of the whole.
std::unique_ptr<Problem> batch_problem(const Problem &full, int M, int m)
{
    auto p = std::make_unique<Problem>(full);
    p->engine = nullptr;
    p->alpha = full.alpha * std::sqrt((double)M);
    const long R = full.kind == HMC_NET_MLP ? full.n : full.n_u;
    const long r0 = (long)((__int128)R * m / M), r1 = (long)((__int128)R * (m + 1) / M);
    auto rows = [&](const std::vector<double> &v, long width) {
        return std::vector<double>(v.begin() + r0 * width, v.begin() + r1 * width);
    };
    if (full.kind == HMC_NET_MLP) {
        p->n = r1 - r0;
        p->x = rows(full.x, full.dx);
        p->y = rows(full.y, full.dout);
    } else {
        p->n_u = r1 - r0;
        p->u = rows(full.u, full.du);
        p->t = rows(full.t, full.n_y);
        if (full.kind == HMC_NET_DEEPONET_UNALIGNED) p->yq = rows(full.yq, full.n_y * full.dy);
    }
    return p;
}

hmc_status create_impl(hmc_handle *out, int nprob, const hmc_net_spec *specs, const hmc_data *data,
                       const double *alpha, const double *sigma, const unsigned char *const *masks,
                       const double *const *frozen, int C, void *stream, int nsplit = 1, bool chunked = false)
{
    HMC_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    HMC_REQUIRE(nprob >= 1, "n_problems must be >= 1");
    HMC_REQUIRE(specs && data && alpha && sigma && masks && frozen, "NULL argument");
    HMC_REQUIRE(C >= 1 && C <= 65535, "n_chains must be in [1, 65535]");
    const int prec = specs[0].prec;
    HMC_REQUIRE(prec >= HMC_PREC_FP64 && prec <= HMC_PREC_FP16, "unknown precision %d", prec);
    for (int i = 0; i < nprob; ++i) HMC_REQUIRE(specs[i].prec == prec, "all problems of a batch share one precision");
    std::unique_ptr<hmc_handle_s> h(new hmc_handle_s);
    h->prec = prec;
    h->C = C;
    h->nprob = nprob;
    h->elem = prec == HMC_PREC_FP64 ? 8 : 4;
    h->user_stream = static_cast<cudaStream_t>(stream);
    int dev = 0;
    HMC_CK(cudaGetDevice(&dev));
    HMC_CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    HMC_CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    HMC_CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    if (nprob > 1) {   // up to 16 concurrent problem lanes
        HMC_CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        const int nl = std::min(nprob, 16);
        h->lanes.resize(nl, nullptr);
        h->ev_join.resize(nl, nullptr);
        for (int j = 0; j < nl; ++j) {
            HMC_CK(cudaStreamCreateWithFlags(&h->lanes[j], cudaStreamNonBlocking));
            HMC_CK(cudaEventCreateWithFlags(&h->ev_join[j], cudaEventDisableTiming));
        }
    }
    HMC_REQUIRE(nsplit >= 1 && nsplit <= (chunked ? (1 << 20) : HMC_MAX_SPLITS), "n_splits must be in [1, %d]",
                HMC_MAX_SPLITS);
    HMC_REQUIRE(nsplit == 1 || nprob == 1, "a split handle holds one problem");
    h->nsplit = nsplit;
    h->chunked = chunked && nsplit > 1;
    if (nsplit > 1) {
        auto full = build_problem(specs[0], data[0], alpha[0], sigma[0], masks[0], frozen[0], C);
        const long R = full->kind == HMC_NET_MLP ? full->n : full->n_u;
        HMC_REQUIRE(R >= nsplit, "n_splits (%d) exceeds the number of data rows (%ld)", nsplit, R);
        if (h->chunked) h->arena.reset(new RowArena());
        // chunk engines take their row buffers from the arena: the largest chunk comes first
        std::vector<int> order(nsplit);
        for (int m = 0; m < nsplit; ++m) order[m] = m;
        auto rows = [&](int m) { return (long)((__int128)R * (m + 1) / nsplit) - (long)((__int128)R * m / nsplit); };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rows(a) > rows(b); });
        h->probs.resize(nsplit);
        h->engines.resize(nsplit);
        for (int m : order) {
            h->probs[m] = batch_problem(*full, nsplit, m);
            Problem &p = *h->probs[m];
            p.arena = h->arena.get();
            if (p.arena) p.arena->begin();
            Engine *e = make_engine(p, prec, C);
            h->engines[m].reset(e);
            p.engine = e;
        }
        h->qoff.push_back(0);
        h->k_total = full->k;
        h->P_total = full->P;
        h->U_split.alloc(sizeof(double) * nsplit * C);
        h->g_tmp.alloc(h->elem * (size_t)full->k * C);
    } else {
        for (int i = 0; i < nprob; ++i) {
            h->probs.push_back(build_problem(specs[i], data[i], alpha[i], sigma[i], masks[i], frozen[i], C));
            Problem &p = *h->probs.back();
            p.batch_member = nprob > 1;
            Engine *e = make_engine(p, prec, C, nprob > 1);
            h->engines.emplace_back(e);
            p.engine = e;
            h->qoff.push_back(h->k_total * C);
            h->k_total += p.k;
            h->P_total += p.P;
        }
        if (nprob > 1 && g_grouping && (prec == HMC_PREC_BF16 || prec == HMC_PREC_FP16)) {
            std::vector<Engine *> es;
            std::vector<long> uoff;
            for (int i = 0; i < nprob; ++i) {
                es.push_back(h->engines[i].get());
                uoff.push_back((long)i * C);
            }
            h->groups = prec == HMC_PREC_FP16 ? make_umma_groups_f16(es, h->qoff, uoff, h->grouped)
                                              : make_umma_groups_bf16(es, h->qoff, uoff, h->grouped);
        }
    }
    h->S_total = h->k_total * C;
    const size_t sb = h->elem * (size_t)h->S_total;
    h->q_cur.alloc(sb);
    h->g_cur.alloc(sb);
    h->q_prop.alloc(sb);
    h->p.alloc(sb);
    h->g_prop.alloc(sb);
    const size_t nseg = (size_t)nprob * C;
    h->U_cur.alloc(sizeof(double) * nseg);
    h->U_prop.alloc(sizeof(double) * nseg);
    long kmax = 1;
    for (auto &pr : h->probs) kmax = std::max(kmax, pr->k);
    h->traj_nblk = (int)((kmax + TRAJ_ELEMS - 1) / TRAJ_ELEMS);
    h->K0p.alloc(sizeof(double) * nseg * h->traj_nblk);
    h->K1p.alloc(sizeof(double) * nseg * h->traj_nblk);
    h->acc_int.alloc(sizeof(int) * nseg);
    h->scratch.alloc(sizeof(int) * 4);
    h->state.alloc(sizeof(TrajState));
    h->eps_prob.alloc(sizeof(double) * nprob);
    h->da_state.alloc(sizeof(double) * 2 * nprob);
    std::vector<SegDesc> sd(nprob);
    for (int i = 0; i < nprob; ++i) {
        sd[i].qoff = h->qoff[i];
        sd[i].k = (int)h->probs[i]->k;
        sd[i].problem = i;
        sd[i].sc = h->engines[i]->scatter_plan();
    }
    h->segs.alloc(sizeof(SegDesc) * nprob);
    HMC_CK(cudaMemcpy(h->segs.ptr, sd.data(), sizeof(SegDesc) * nprob, cudaMemcpyHostToDevice));
    HMC_CK(cudaDeviceSynchronize());
    *out = h.release();
    return HMC_OK;
}

template <typename F> hmc_status guarded(F &&f)
{
    try {
        return f();
    } catch (const Fail &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return HMC_ERR_OOM;
    } catch (...) {
        set_error("unexpected internal error");
        return HMC_ERR_CUDA;
    }
}

}  // namespace

extern "C" {

hmc_status hmc_create(hmc_handle *out, const hmc_net_spec *spec, const hmc_data *data, double prior_sigma,
                      double noise_sigma, const unsigned char *subset_mask, const double *frozen_params,
                      int n_chains, void *cuda_stream)
{
    g_err.clear();
    hmc_status st = guarded([&] {
        return create_impl(out, 1, spec, data, &prior_sigma, &noise_sigma, &subset_mask, &frozen_params, n_chains,
                           cuda_stream);
    });
    if (st != HMC_ERR_OOM || !spec || !data) return st;
    // the whole batch's row buffers do not fit: evaluate the rows in passes, halving the
    // rows of a pass until the handle fits (the energy and its gradient are sums over rows)
    const long R = spec->kind == HMC_NET_MLP ? data->n : data->n_u;
    for (long M = 2; M <= R && st == HMC_ERR_OOM; M *= 2) {
        cudaGetLastError();   // the failed allocation's error is not sticky; clear it
        g_err.clear();
        st = guarded([&] {
            return create_impl(out, 1, spec, data, &prior_sigma, &noise_sigma, &subset_mask, &frozen_params,
                               n_chains, cuda_stream, (int)M, true);
        });
    }
    return st;
}

hmc_status hmc_create_chunked(hmc_handle *out, const hmc_net_spec *spec, const hmc_data *data, double prior_sigma,
                              double noise_sigma, const unsigned char *subset_mask, const double *frozen_params,
                              int n_chains, long rows_per_pass, void *cuda_stream)
{
    g_err.clear();
    return guarded([&] {
        HMC_REQUIRE(spec && data, "NULL argument");
        HMC_REQUIRE(rows_per_pass >= 1, "rows_per_pass must be >= 1");
        const long R = spec->kind == HMC_NET_MLP ? data->n : data->n_u;
        const long M = std::max<long>(1, (R + rows_per_pass - 1) / rows_per_pass);
        HMC_REQUIRE(M <= (1 << 20), "too many passes (%ld)", M);
        return create_impl(out, 1, spec, data, &prior_sigma, &noise_sigma, &subset_mask, &frozen_params, n_chains,
                           cuda_stream, (int)M, true);
    });
}

int hmc_num_passes(hmc_handle h) { return h ? (h->chunked ? h->nsplit : 1) : -1; }

void hmc_diag_set_memory_cap(long bytes) { g_devbuf_cap = bytes > 0 ? (size_t)bytes : ~size_t(0); }

long hmc_diag_device_bytes(void) { return (long)g_devbuf_bytes.load(); }

void hmc_diag_set_grouping(int on) { g_grouping = on != 0; }

long hmc_diag_groups(hmc_handle h, char *buf, long n)
{
    if (!h) return -1;
    std::string t;
    for (auto &g : h->groups) t += g->describe() + "\n";
    if (buf && n > 0) {
        const long m = std::min<long>(n - 1, (long)t.size());
        memcpy(buf, t.data(), m);
        buf[m] = 0;
    }
    return (long)h->groups.size();
}

hmc_status hmc_create_split(hmc_handle *out, const hmc_net_spec *spec, const hmc_data *data, double prior_sigma,
                            double noise_sigma, const unsigned char *subset_mask, const double *frozen_params,
                            int n_chains, int n_splits, void *cuda_stream)
{
    g_err.clear();
    return guarded([&] {
        return create_impl(out, 1, spec, data, &prior_sigma, &noise_sigma, &subset_mask, &frozen_params, n_chains,
                           cuda_stream, n_splits);
    });
}

hmc_status hmc_create_batch(hmc_handle *out, int n_problems, const hmc_net_spec *specs, const hmc_data *data,
                            const double *prior_sigma, const double *noise_sigma,
                            const unsigned char *const *subset_masks, const double *const *frozen_params,
                            int n_chains, void *cuda_stream)
{
    g_err.clear();
    return guarded([&] {
        return create_impl(out, n_problems, specs, data, prior_sigma, noise_sigma, subset_masks, frozen_params,
                           n_chains, cuda_stream);
    });
}

hmc_status hmc_sensitivity(const hmc_net_spec *spec, const hmc_data *data, const double *mu, const double *sd,
                           double *S2, void *cuda_stream)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(spec && data && mu && sd && S2, "NULL argument");
        if (spec->kind == HMC_NET_DEEPONET_UNALIGNED) {   // each function would need its own Gram matrix
            set_error("hmc_sensitivity does not cover DeepONets with per-function query points");
            throw Fail{HMC_ERR_UNSUPPORTED};
        }
        HMC_REQUIRE(spec->kind == HMC_NET_MLP || spec->kind == HMC_NET_DEEPONET, "unknown net kind %d", spec->kind);
        SensProblem pr;
        pr.kind = spec->kind;
        const std::vector<long> none;
        if (spec->kind == HMC_NET_MLP) {
            check_mlp_spec(spec->net, "net");
            HMC_REQUIRE(data->n >= 1 && data->dx == spec->net.widths[0], "data.n must be >= 1 and data.dx = widths[0]");
            build_net_desc(pr.net, spec->net, 0, none);
            pr.P = pr.net.P;
            pr.n = data->n;
            pr.x = fetch_data(data->x, data->n * data->dx, data->dtype, "data.x");
        } else {
            check_mlp_spec(spec->branch, "branch");
            check_mlp_spec(spec->trunk, "trunk");
            HMC_REQUIRE(spec->branch.widths[spec->branch.n_layers] == spec->trunk.widths[spec->trunk.n_layers],
                        "branch and trunk output widths differ");
            HMC_REQUIRE(data->n_u >= 1 && data->n_y >= 1 && data->du == spec->branch.widths[0] &&
                            data->dy == spec->trunk.widths[0],
                        "DeepONet data dimensions do not match the spec");
            build_net_desc(pr.branch, spec->branch, 0, none);
            build_net_desc(pr.trunk, spec->trunk, pr.branch.P, none);
            pr.out_bias = spec->deeponet_out_bias ? 1 : 0;
            pr.P = pr.branch.P + pr.trunk.P + pr.out_bias;
            pr.n_u = data->n_u;
            pr.n_y = data->n_y;
            pr.u = fetch_data(data->u, data->n_u * data->du, data->dtype, "data.u");
            pr.yq = fetch_data(data->yq, data->n_y * data->dy, data->dtype, "data.yq");
        }
        HMC_REQUIRE(pr.P < (1L << 31), "too many parameters (%ld)", pr.P);
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        const size_t pb = sizeof(double) * (size_t)pr.P;
        DevBuf dmu, dsd, ds2;
        const double *m = mu, *d = sd;
        double *o = S2;
        if (!is_device_ptr(mu)) {
            dmu.alloc(pb);
            HMC_CK(cudaMemcpy(dmu.ptr, mu, pb, cudaMemcpyHostToDevice));
            m = dmu.as<double>();
        }
        if (!is_device_ptr(sd)) {
            dsd.alloc(pb);
            HMC_CK(cudaMemcpy(dsd.ptr, sd, pb, cudaMemcpyHostToDevice));
            d = dsd.as<double>();
        }
        const bool host_out = !is_device_ptr(S2);
        if (host_out) {
            ds2.alloc(pb);
            o = ds2.as<double>();
        }
        sensitivity_run(pr, spec->prec, m, d, o, st);
        if (host_out) HMC_CK(cudaMemcpy(S2, o, pb, cudaMemcpyDeviceToHost));
        return HMC_OK;
    });
}

hmc_status hmc_select_subset(const double *S2, long P, double tau, unsigned char *mask, long *n_hat,
                             long long *order, void *cuda_stream)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(S2 && mask && n_hat, "NULL argument");
        HMC_REQUIRE(P >= 1 && P < (1L << 31), "P must be in [1, 2^31)");
        HMC_REQUIRE(std::isfinite(tau), "tau must be finite");
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        DevBuf ds2, dm, dord;
        const double *s2 = S2;
        if (!is_device_ptr(S2)) {
            ds2.alloc(sizeof(double) * P);
            HMC_CK(cudaMemcpy(ds2.ptr, S2, sizeof(double) * P, cudaMemcpyHostToDevice));
            s2 = ds2.as<double>();
        }
        const bool host_mask = !is_device_ptr(mask), host_ord = order && !is_device_ptr(order);
        unsigned char *m = mask;
        long long *od = order;
        if (host_mask) {
            dm.alloc(P);
            m = dm.as<unsigned char>();
        }
        if (host_ord) {
            dord.alloc(sizeof(long long) * P);
            od = dord.as<long long>();
        }
        *n_hat = select_subset_run(s2, P, tau, m, od, st);
        if (host_mask) HMC_CK(cudaMemcpy(mask, m, P, cudaMemcpyDeviceToHost));
        if (host_ord) HMC_CK(cudaMemcpy(order, od, sizeof(long long) * P, cudaMemcpyDeviceToHost));
        return HMC_OK;
    });
}

hmc_status hmc_predict(hmc_handle h, const void *samples, long n_samples, const hmc_data *inputs, double *mean,
                       double *std_out, double *rel_l2)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h && samples && inputs && mean && std_out, "NULL argument");
        HMC_REQUIRE(h->nprob == 1, "hmc_predict takes a single-problem handle");
        if (h->probs[0]->kind == HMC_NET_DEEPONET_UNALIGNED) {
            set_error("hmc_predict does not cover DeepONets with per-function query points");
            throw Fail{HMC_ERR_UNSUPPORTED};
        }
        HMC_REQUIRE(n_samples >= 1, "n_samples must be >= 1");
        const Problem &p = *h->probs[0];
        PredictInput in;
        in.kind = p.kind;
        in.net = p.net;
        in.branch = p.branch;
        in.trunk = p.trunk;
        in.out_bias = p.out_bias;
        in.P = p.P;
        in.frozen = p.frozen;
        in.idx = p.idx;
        long nout;
        if (p.kind == HMC_NET_MLP) {
            HMC_REQUIRE(inputs->n >= 1 && inputs->dx == p.dx, "inputs: n must be >= 1 and dx = %d", p.dx);
            in.n = inputs->n;
            nout = in.n * p.dout;
            in.x = fetch_data(inputs->x, in.n * p.dx, inputs->dtype, "inputs.x");
            if (rel_l2) in.targets = fetch_data(inputs->y, nout, inputs->dtype, "inputs.y (targets for rel_l2)");
        } else {
            HMC_REQUIRE(inputs->n_u >= 1 && inputs->n_y >= 1 && inputs->du == p.du && inputs->dy == p.dy,
                        "inputs: DeepONet dimensions do not match the handle's");
            in.n_u = inputs->n_u;
            in.n_y = inputs->n_y;
            nout = in.n_u * in.n_y;
            in.u = fetch_data(inputs->u, in.n_u * p.du, inputs->dtype, "inputs.u");
            in.yq = fetch_data(inputs->yq, in.n_y * p.dy, inputs->dtype, "inputs.yq");
            if (rel_l2) in.targets = fetch_data(inputs->t, nout, inputs->dtype, "inputs.t (targets for rel_l2)");
        }
        h->stage_used = 0;
        join_in(h);
        bool ss, sm, sv;
        const void *ds = dev_view(h, samples, h->elem * (size_t)n_samples * p.k, true, &ss);
        double *dm = static_cast<double *>(dev_view(h, mean, sizeof(double) * nout, false, &sm));
        double *dv = static_cast<double *>(dev_view(h, std_out, sizeof(double) * nout, false, &sv));
        predict_run(in, h->prec, ds, n_samples, dm, dv, rel_l2, h->stream);
        if (sm) HMC_CK(cudaMemcpy(mean, dm, sizeof(double) * nout, cudaMemcpyDeviceToHost));
        if (sv) HMC_CK(cudaMemcpy(std_out, dv, sizeof(double) * nout, cudaMemcpyDeviceToHost));
        join_out(h);
        return HMC_OK;
    });
}

long hmc_subset_size(hmc_handle h) { return h ? h->k_total : -1; }
long hmc_param_count(hmc_handle h) { return h ? h->P_total : -1; }
int hmc_num_chains(hmc_handle h) { return h ? h->C : -1; }

hmc_status hmc_energy_grad(hmc_handle h, const void *q, double *U, void *grad)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h && q && U, "NULL argument");
        h->stage_used = 0;
        join_in(h);
        bool sq, su, sg;
        const size_t sb = h->elem * (size_t)h->S_total;
        void *dq = dev_view(h, q, sb, true, &sq);
        double *dU = static_cast<double *>(dev_view(h, U, sizeof(double) * h->nprob * h->C, false, &su));
        void *dg = dev_view(h, grad, sb, false, &sg);
        energy_grad_all(h, dq, dU, dg, false);
        if (sg) HMC_CK(cudaMemcpyAsync(grad, dg, sb, cudaMemcpyDeviceToHost, h->stream));
        if (su) HMC_CK(cudaMemcpyAsync(U, dU, sizeof(double) * h->nprob * h->C, cudaMemcpyDeviceToHost, h->stream));
        join_out(h);
        if (su || sg || sq) HMC_CK(cudaStreamSynchronize(h->stream));
        if (su) {
            for (int i = 0; i < h->nprob * h->C; ++i)
                if (!std::isfinite(U[i])) {
                    set_error("U is not finite for (problem, chain) %d", i);
                    return HMC_ERR_NONFINITE;
                }
        }
        return HMC_OK;
    });
}

hmc_status hmc_leapfrog(hmc_handle h, void *q, void *p, double eps, int L)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h && q && p, "NULL argument");
        HMC_REQUIRE(L >= 0 && std::isfinite(eps), "L must be >= 0 and eps finite");
        h->stage_used = 0;
        join_in(h);
        const size_t sb = h->elem * (size_t)h->S_total;
        bool sq, sp;
        void *dq = dev_view(h, q, sb, true, &sq);
        void *dp = dev_view(h, p, sb, true, &sp);
        if (L > 0 && h->nsplit > 1 && !h->chunked) {
            split_grad(h, 0, dq, h->g_prop.ptr);
            kick_drift(h, dq, dp, h->g_prop.ptr, Step{nullptr, eps, 2.0, 2.0 * h->nsplit});
            split_steps(h, dq, dp, h->g_prop.ptr, nullptr, eps, L);
            kick_drift(h, dq, dp, h->g_prop.ptr, Step{nullptr, eps, 2.0, 0.0});
        } else if (L > 0) {
            energy_grad_all(h, dq, h->U_prop.as<double>(), h->g_prop.ptr, false);
            kick_drift(h, dq, dp, h->g_prop.ptr, Step{nullptr, eps, 2.0, 1.0});
            for (int s = 1; s <= L; ++s) {
                energy_grad_all(h, dq, h->U_prop.as<double>(), h->g_prop.ptr, true);
                if (s < L) kick_drift(h, dq, dp, h->g_prop.ptr, Step{nullptr, eps, 1.0, 1.0});
                else kick_drift(h, dq, dp, h->g_prop.ptr, Step{nullptr, eps, 2.0, 0.0});
            }
        }
        if (sq) HMC_CK(cudaMemcpyAsync(q, dq, sb, cudaMemcpyDeviceToHost, h->stream));
        if (sp) HMC_CK(cudaMemcpyAsync(p, dp, sb, cudaMemcpyDeviceToHost, h->stream));
        join_out(h);
        if (sq || sp) HMC_CK(cudaStreamSynchronize(h->stream));
        return HMC_OK;
    });
}

// The executable graph of one trajectory, captured once per (L, seed) and reused; the
// step size lives in the device state, so it does not enter the graph.
void ensure_trajectory_graph(hmc_handle h, int L, unsigned long long seed)
{
    if (h->traj_exec && h->traj_L == L && h->traj_seed == seed) return;
    if (h->traj_exec) {
        cudaGraphExecDestroy(h->traj_exec);
        h->traj_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    HMC_CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    try {
        if (h->prec == HMC_PREC_FP64) enqueue_trajectory<double>(h, L, seed);
        else enqueue_trajectory<float>(h, L, seed);
    } catch (...) {
        cudaStreamEndCapture(h->stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
    }
    HMC_CK(cudaStreamEndCapture(h->stream, &graph));
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    long nk = 0;
    if (nn) {
        cudaGraphGetNodes(graph, nodes.data(), &nn);
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
        }
    }
    cudaError_t e = cudaGraphInstantiate(&h->traj_exec, graph, 0);
    cudaGraphDestroy(graph);
    HMC_CK(e);
    h->traj_L = L;
    h->traj_seed = seed;
    h->traj_kernels = nk;
    ++h->traj_captures;
}

// hmc_sample (one step for every problem) and hmc_sample_steps (eps_each: a step per
// problem, host or device).
hmc_status sample_impl(hmc_handle h, const void *q0, double eps, bool each, const double *eps_each, int L,
                       long n_samples, unsigned long long seed, long first_traj, void *samples,
                       unsigned char *accepted, double *dH, void *q_last)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h && q0 && (eps_each || !each), "NULL argument");
        HMC_REQUIRE(L >= 1 && n_samples >= 0 && first_traj >= 0, "need L >= 1, n_samples >= 0, first_traj >= 0");
        h->stage_used = 0;
        const double *deps = nullptr;
        std::vector<double> e;
        if (each) {
            e.resize(h->nprob);
            HMC_CK(cudaMemcpy(e.data(), eps_each, sizeof(double) * h->nprob, cudaMemcpyDefault));
            for (double v : e) HMC_REQUIRE(std::isfinite(v) && v > 0, "every step size must be finite and > 0");
            bool staged;
            deps = static_cast<const double *>(dev_view(h, e.data(), sizeof(double) * h->nprob, true, &staged));
        } else {
            HMC_REQUIRE(std::isfinite(eps) && eps > 0, "need eps > 0");
        }
        join_in(h);
        const size_t sb = h->elem * (size_t)h->S_total;
        const long nseg = (long)h->nprob * h->C;
        bool s0, ss, sa, sd, sl;
        void *dq0 = dev_view(h, q0, sb, true, &s0);
        HMC_CK(cudaMemcpyAsync(h->q_cur.ptr, dq0, sb, cudaMemcpyDeviceToDevice, h->stream));
        void *ds = dev_view(h, samples, sb * (size_t)n_samples, false, &ss);
        unsigned char *da = static_cast<unsigned char *>(dev_view(h, accepted, (size_t)nseg * n_samples, false, &sa));
        double *ddh = static_cast<double *>(dev_view(h, dH, sizeof(double) * nseg * n_samples, false, &sd));
        void *dl = dev_view(h, q_last, sb, false, &sl);
        if (h->nsplit > 1 && !h->chunked) {   // U for H0 and grad U of the first batch for the first kick
            split_start(h, h->q_cur.ptr, h->U_cur.as<double>(), h->g_cur.ptr);
        } else {
            energy_grad_all(h, h->q_cur.ptr, h->U_cur.as<double>(), h->g_cur.ptr, false);
            accurate_energy_all(h, h->q_cur.ptr, h->U_cur.as<double>());   // H0 of the first trajectory
        }
        k_set_state<<<1, 256, 0, h->stream>>>(h->state.as<TrajState>(), first_traj, 0, ds, da, ddh,
                                               h->eps_prob.as<double>(), h->da_state.as<double>(), h->nprob, deps, eps);
        HMC_LAUNCH_CK();
        if (n_samples > 0) {
            ensure_trajectory_graph(h, L, seed);
            for (long i = 0; i < n_samples; ++i) HMC_CK(cudaGraphLaunch(h->traj_exec, h->stream));
        }
        if (dl) HMC_CK(cudaMemcpyAsync(dl, h->q_cur.ptr, sb, cudaMemcpyDeviceToDevice, h->stream));
        if (ss) HMC_CK(cudaMemcpyAsync(samples, ds, sb * (size_t)n_samples, cudaMemcpyDeviceToHost, h->stream));
        if (sa) HMC_CK(cudaMemcpyAsync(accepted, da, (size_t)nseg * n_samples, cudaMemcpyDeviceToHost, h->stream));
        if (sd) HMC_CK(cudaMemcpyAsync(dH, ddh, sizeof(double) * nseg * n_samples, cudaMemcpyDeviceToHost, h->stream));
        if (sl) HMC_CK(cudaMemcpyAsync(q_last, dl, sb, cudaMemcpyDeviceToHost, h->stream));
        join_out(h);
        if (s0 || ss || sa || sd || sl || deps) HMC_CK(cudaStreamSynchronize(h->stream));
        return HMC_OK;
    });
}

hmc_status hmc_sample(hmc_handle h, const void *q0, double eps, int L, long n_samples, unsigned long long seed,
                      long first_traj, void *samples, unsigned char *accepted, double *dH, void *q_last)
{
    return sample_impl(h, q0, eps, false, nullptr, L, n_samples, seed, first_traj, samples, accepted, dH, q_last);
}

hmc_status hmc_sample_steps(hmc_handle h, const void *q0, const double *eps, int L, long n_samples,
                            unsigned long long seed, long first_traj, void *samples, unsigned char *accepted,
                            double *dH, void *q_last)
{
    return sample_impl(h, q0, 0.0, true, eps, L, n_samples, seed, first_traj, samples, accepted, dH, q_last);
}

hmc_status hmc_adapt_step_size(hmc_handle h, void *q, int L, double eps0, long n_warmup, double target_accept,
                               unsigned long long seed, long first_traj, double *eps_out)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h && q && eps_out, "NULL argument");
        HMC_REQUIRE(L >= 1 && n_warmup >= 1 && first_traj >= 0 && std::isfinite(eps0) && eps0 > 0,
                    "need L >= 1, n_warmup >= 1, eps0 > 0, first_traj >= 0");
        HMC_REQUIRE(target_accept > 0.0 && target_accept < 1.0, "target_accept must lie in (0, 1)");
        h->stage_used = 0;
        join_in(h);
        const long nseg = (long)h->nprob * h->C;
        const size_t sb = h->elem * (size_t)h->S_total;
        bool sq;
        void *dq = dev_view(h, q, sb, true, &sq);
        const size_t trace_bytes = sizeof(double) * 2 * (size_t)n_warmup * h->nprob;
        if (h->adapt_trace.n < trace_bytes) h->adapt_trace.alloc(trace_bytes);
        DevBuf dh_dev(sizeof(double) * nseg);
        TrajState *st = h->state.as<TrajState>();
        HMC_CK(cudaMemcpyAsync(h->q_cur.ptr, dq, sb, cudaMemcpyDeviceToDevice, h->stream));
        if (h->nsplit > 1 && !h->chunked) {
            split_start(h, h->q_cur.ptr, h->U_cur.as<double>(), h->g_cur.ptr);
        } else {
            energy_grad_all(h, h->q_cur.ptr, h->U_cur.as<double>(), h->g_cur.ptr, false);
            accurate_energy_all(h, h->q_cur.ptr, h->U_cur.as<double>());
        }
        k_set_state<<<1, 256, 0, h->stream>>>(st, first_traj, 0, nullptr, nullptr, dh_dev.as<double>(),
                                               h->eps_prob.as<double>(), h->da_state.as<double>(), h->nprob, nullptr,
                                               eps0);
        HMC_LAUNCH_CK();
        ensure_trajectory_graph(h, L, seed);
        // Dual averaging of log eps (Hoffman and Gelman 2014, Sec. 3.2), each problem's
        // step towards a mean Metropolis acceptance probability `target_accept` over its
        // chains; shrinkage towards log(10 eps0), gamma = 0.05, t0 = 10, kappa = 0.75.  Each
        // update runs on the device after its trajectory and sets the next trajectory's
        // steps in device memory, so the warm-up replays one captured graph without host
        // round trips.  The returned steps are the averaged iterates.
        const double mu = std::log(10.0 * eps0), gamma = 0.05, t0 = 10.0, kappa = 0.75;
        for (long m = 1; m <= n_warmup; ++m) {
            HMC_CK(cudaGraphLaunch(h->traj_exec, h->stream));
            k_dual_avg<<<1, 256, 0, h->stream>>>(st, h->eps_prob.as<double>(), h->da_state.as<double>(), h->nprob,
                                                 h->C, target_accept, mu, gamma, t0, kappa,
                                                 h->adapt_trace.as<double>());
            HMC_LAUNCH_CK();
            k_rewind_slot<<<1, 1, 0, h->stream>>>(st);   // every trajectory's dH goes to slot 0
            HMC_LAUNCH_CK();
        }
        std::vector<double> da(2 * (size_t)h->nprob);
        HMC_CK(cudaMemcpyAsync(da.data(), h->da_state.ptr, sizeof(double) * da.size(), cudaMemcpyDeviceToHost,
                               h->stream));
        HMC_CK(cudaMemcpyAsync(dq, h->q_cur.ptr, sb, cudaMemcpyDeviceToDevice, h->stream));
        if (sq) HMC_CK(cudaMemcpyAsync(q, dq, sb, cudaMemcpyDeviceToHost, h->stream));
        join_out(h);
        HMC_CK(cudaStreamSynchronize(h->stream));
        h->adapt_n = n_warmup;
        for (int i = 0; i < h->nprob; ++i) eps_out[i] = std::exp(da[2 * (size_t)i + 1]);
        return HMC_OK;
    });
}

hmc_status hmc_diag_adapt_trace(hmc_handle h, double *out_host, long n)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h && out_host, "NULL argument");
        HMC_REQUIRE(n >= 0 && n <= h->adapt_n, "n (%ld) exceeds the last warm-up's %ld updates", n, h->adapt_n);
        HMC_CK(cudaStreamSynchronize(h->stream));
        if (n > 0)
            HMC_CK(cudaMemcpy(out_host, h->adapt_trace.ptr, sizeof(double) * 2 * (size_t)n * h->nprob,
                              cudaMemcpyDeviceToHost));
        return HMC_OK;
    });
}

hmc_status hmc_diag_dual_averaging(const double *dH, long n, int nseg, double eps0, double target, double *out_host)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(dH && out_host && n >= 1 && nseg >= 1 && eps0 > 0 && std::isfinite(eps0), "bad argument");
        HMC_REQUIRE(target > 0.0 && target < 1.0, "target must lie in (0, 1)");
        // one problem with nseg chains
        DevBuf st(sizeof(TrajState)), d(sizeof(double) * (size_t)n * nseg), tr(sizeof(double) * 2 * (size_t)n);
        DevBuf ep(sizeof(double)), da(2 * sizeof(double));
        HMC_CK(cudaMemcpy(d.ptr, dH, d.n, cudaMemcpyDefault));
        k_set_state<<<1, 32>>>(st.as<TrajState>(), 0, 0, nullptr, nullptr, d.as<double>(), ep.as<double>(),
                               da.as<double>(), 1, nullptr, eps0);
        HMC_LAUNCH_CK();
        const double mu = std::log(10.0 * eps0);
        for (long m = 1; m <= n; ++m) {
            k_advance_slot<<<1, 1>>>(st.as<TrajState>());   // as a trajectory would: dH row m - 1
            HMC_LAUNCH_CK();
            k_dual_avg<<<1, 256>>>(st.as<TrajState>(), ep.as<double>(), da.as<double>(), 1, nseg, target, mu, 0.05,
                                   10.0, 0.75, tr.as<double>());
            HMC_LAUNCH_CK();
        }
        HMC_CK(cudaMemcpy(out_host, tr.ptr, tr.n, cudaMemcpyDeviceToHost));
        return HMC_OK;
    });
}

hmc_status hmc_destroy(hmc_handle h)
{
    g_err.clear();
    if (!h) return HMC_OK;
    return guarded([&]() -> hmc_status {
        cudaStreamSynchronize(h->stream);
        h->engines.clear();
        h->probs.clear();
        h->stage_used = 0;
        cudaStream_t s = h->stream;
        cudaEvent_t a = h->ev_in, b = h->ev_out;
        delete h;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaStreamDestroy(s);
        return HMC_OK;
    });
}

const char *hmc_last_error(void) { return g_err.c_str(); }

hmc_status hmc_check(hmc_handle h)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h, "NULL argument");
        HMC_CK(cudaStreamSynchronize(h->stream));
        bool timed_out = false;
        for (auto &e : h->engines) {
            int *f = e->error_flag();
            if (!f) continue;
            int v = 0;
            HMC_CK(cudaMemcpy(&v, f, sizeof(int), cudaMemcpyDeviceToHost));
            if (v) {
                timed_out = true;
                HMC_CK(cudaMemset(f, 0, sizeof(int)));
            }
        }
        if (timed_out) {
            set_error("a bounded device-side wait gave up since the last check: results since then are not valid");
            return HMC_ERR_TIMEOUT;
        }
        return HMC_OK;
    });
}

hmc_status hmc_diag_expire_wait(hmc_handle h, long limit_ns)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h, "NULL argument");
        HMC_REQUIRE(limit_ns >= 1000 && limit_ns <= 100000000, "limit_ns must be in [1e3, 1e8]");
        for (auto &e : h->engines) {
            int *f = e->error_flag();
            if (!f) continue;
            expire_wait_run(f, limit_ns, h->stream);
            return HMC_OK;
        }
        set_error("no engine of this handle keeps a device error flag");
        return HMC_ERR_UNSUPPORTED;
    });
}

long hmc_diag_graph_kernels(hmc_handle h) { return h ? h->traj_kernels : -1; }

long hmc_diag_graph_captures(hmc_handle h) { return h ? h->traj_captures : -1; }

long hmc_diag_tuning(hmc_handle h, char *buf, long n)
{
    if (!h) return -1;
    std::string t;
    for (size_t i = 0; i < h->engines.size(); ++i)
        t += (h->nsplit > 1 ? "batch " : "problem ") + std::to_string(i) + ": " + h->engines[i]->tuning() + "\n";
    if (buf && n > 0) {
        const size_t m = std::min<size_t>((size_t)n - 1, t.size());
        memcpy(buf, t.data(), m);
        buf[m] = 0;
    }
    return (long)t.size();
}

hmc_status hmc_diag_metropolis_energy(hmc_handle h, const void *q, double *U)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(h && q && U, "NULL argument");
        h->stage_used = 0;
        join_in(h);
        bool sq, su;
        const size_t sb = h->elem * (size_t)h->S_total;
        void *dq = dev_view(h, q, sb, true, &sq);
        double *dU = static_cast<double *>(dev_view(h, U, sizeof(double) * h->nprob * h->C, false, &su));
        energy_grad_all(h, dq, dU, h->g_prop.ptr, false);
        accurate_energy_all(h, dq, dU);
        if (su) HMC_CK(cudaMemcpyAsync(U, dU, sizeof(double) * h->nprob * h->C, cudaMemcpyDeviceToHost, h->stream));
        join_out(h);
        if (sq || su) HMC_CK(cudaStreamSynchronize(h->stream));
        return HMC_OK;
    });
}

int hmc_diag_profile_energy_grad(hmc_handle h, const void *q, int reps, hmc_kernel_time *out, int max_out)
{
    g_err.clear();
    Profiler prof;
    int n = 0;
    cudaGraphExec_t exec = nullptr;
    hmc_status st = guarded([&]() -> hmc_status {
        HMC_REQUIRE(h && q && out && reps >= 1 && max_out >= 1, "bad argument");
        HMC_REQUIRE(is_device_ptr(q), "q must be device memory");
        join_in(h);
        HMC_CK(cudaStreamSynchronize(h->stream));
        // one untimed evaluation, then `reps` timed ones replayed from a graph so that the
        // GPU runs them back to back (the host never starves it between launches)
        energy_grad_all(h, const_cast<void *>(q), h->U_prop.as<double>(), h->g_prop.ptr, false);
        cudaGraph_t graph = nullptr;
        HMC_CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        active_profiler() = &prof;
        try {
            for (int r = 0; r < reps; ++r)
                energy_grad_all(h, const_cast<void *>(q), h->U_prop.as<double>(), h->g_prop.ptr, false);
        } catch (...) {
            active_profiler() = nullptr;
            cudaStreamEndCapture(h->stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        active_profiler() = nullptr;
        HMC_CK(cudaStreamEndCapture(h->stream, &graph));
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        HMC_CK(e);
        HMC_CK(cudaGraphLaunch(exec, h->stream));
        HMC_CK(cudaStreamSynchronize(h->stream));
        for (auto &r : prof.recs) {
            float ms = 0.0f;
            HMC_CK(cudaEventElapsedTime(&ms, r.a, r.b));
            int k = 0;
            while (k < n && strncmp(out[k].name, r.name, sizeof(out[k].name) - 1) != 0) ++k;
            if (k == n) {
                if (n == max_out) continue;
                memset(&out[n], 0, sizeof(out[n]));
                strncpy(out[n].name, r.name, sizeof(out[n].name) - 1);
                ++n;
            }
            out[k].ms_total += ms;
            out[k].launches += 1;
        }
        join_out(h);
        return HMC_OK;
    });
    if (exec) cudaGraphExecDestroy(exec);
    for (auto &r : prof.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    return st == HMC_OK ? n : -(int)st;
}

// --- diagnostics (include/hmc_diag.h) ---------------------------------------

hmc_status hmc_diag_momenta(unsigned long long seed, unsigned long long problem, unsigned long long chain,
                            unsigned long long traj, long k, double *out_host)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(out_host && k >= 0, "bad argument");
        DevBuf d(sizeof(double) * std::max<long>(k, 1));
        k_debug_momenta<<<64, 256>>>(seed, problem, chain, traj, k, d.as<double>());
        HMC_LAUNCH_CK();
        HMC_CK(cudaMemcpy(out_host, d.ptr, sizeof(double) * k, cudaMemcpyDeviceToHost));
        return HMC_OK;
    });
}

hmc_status hmc_diag_log_uniform(unsigned long long seed, unsigned long long problem, long n_chain, long n_traj,
                                double *out_host)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(out_host && n_chain >= 0 && n_traj >= 0, "bad argument");
        DevBuf d(sizeof(double) * std::max<long>(n_chain * n_traj, 1));
        k_debug_logu<<<64, 256>>>(seed, problem, n_chain, n_traj, d.as<double>());
        HMC_LAUNCH_CK();
        HMC_CK(cudaMemcpy(out_host, d.ptr, sizeof(double) * n_chain * n_traj, cudaMemcpyDeviceToHost));
        return HMC_OK;
    });
}

hmc_status hmc_diag_philox(const unsigned long long *ctr, const unsigned long long *key, long n,
                           unsigned long long *out_host)
{
    g_err.clear();
    return guarded([&]() -> hmc_status {
        HMC_REQUIRE(ctr && key && out_host && n >= 0, "bad argument");
        DevBuf dc(32 * std::max<long>(n, 1)), dk(16 * std::max<long>(n, 1)), dout(32 * std::max<long>(n, 1));
        HMC_CK(cudaMemcpy(dc.ptr, ctr, 32 * n, cudaMemcpyHostToDevice));
        HMC_CK(cudaMemcpy(dk.ptr, key, 16 * n, cudaMemcpyHostToDevice));
        k_debug_philox<<<64, 256>>>(dc.as<uint64_t>(), dk.as<uint64_t>(), n, dout.as<uint64_t>());
        HMC_LAUNCH_CK();
        HMC_CK(cudaMemcpy(out_host, dout.ptr, 32 * n, cudaMemcpyDeviceToHost));
        return HMC_OK;
    });
}

}  // extern "C"

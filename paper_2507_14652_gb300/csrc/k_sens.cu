// k_sens.cu -- sensitivities of the network output to each parameter around the VI
// mean, and the truncation of the parameter set that follows from them (Sec. 3.1).
//
// S_i^2 = sd_i^2 / N_d * sum over data terms of (dF/dtheta_i)^2 at theta = mu.
// For a weight W_l[a][b] the derivative of one output is delta[a] A_{l-1}[b], with
// delta the reverse-mode adjoint of that output at layer l's pre-activation, so
//   sum over terms of (dF/dW_l[a][b])^2 = sum_n E_l[n][a] A_{l-1}[n][b]^2,
//   E_l[n][a] = sum over the terms of row n of delta[a]^2,
// a GEMM of E_l^T with the squared activations; a bias takes the column sums of E_l.
// An MLP's terms of row n are its d_out outputs: one reverse pass per output seed.
// A DeepONet's terms of branch row j are S_jk = <B_j, T_k> + b0 over all queries k,
// whose branch derivative is sum_c (dB_jc/dtheta) T_kc; squared and summed over k it
// is the quadratic form D G_T D^T with G_T = T^T T (p x p), D the adjoints of the p
// branch outputs.  So E = sum_c D_c (G D)_c, with p seeds; the trunk uses G_B = B^T B.
//
// The truncation ranks the parameters by S2 (descending, ties to the lower index)
// with a stable LSD radix sort on 64-bit keys, takes the FP64 prefix sums in rank
// order and keeps the ranks before the first prefix whose share of the total
// exceeds tau.
#include <algorithm>
#include <memory>
#include <vector>

#include "hmc_internal.cuh"

namespace hmc {
namespace {

#include "simt_kernels.cuh"

// D[c][n][a] = slope[n][a] if a == c else 0: the adjoint of output c at the last layer.
template <typename T>
__global__ void k_seed(const T *slope, long rows, int w, int nseeds, T *D)
{
    const long nx = rows * w;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nx * nseeds; i += (long)gridDim.x * blockDim.x) {
        const long c = i / nx, x = i % nx;
        D[i] = ((x % w) == c) ? slope[x] : T(0);
    }
}

// E[x] = sum_c D[c][x] * Q[c][x] (Q = D when null), summed in double.
template <typename T>
__global__ void k_seed_energy(const T *D, const T *Q, int nseeds, long nx, T *E)
{
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += (long)gridDim.x * blockDim.x) {
        double e = 0.0;
        for (int c = 0; c < nseeds; ++c) {
            const double d = (double)D[(long)c * nx + x];
            e += d * (double)(Q ? Q[(long)c * nx + x] : D[(long)c * nx + x]);
        }
        E[x] = (T)e;
    }
}

template <typename T>
__global__ void k_square(const T *A, long n, T *out)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = A[i] * A[i];
}

// S2[off + i] = sd[off + i]^2 * scale * src[i]
template <typename T>
__global__ void k_scale_out(const T *src, long n, const double *sd, long off, double scale, double *S2)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double s = sd[off + i];
        S2[off + i] = s * s * scale * (double)src[i];
    }
}

// S2[off + a] = sd[off + a]^2 * scale * sum_n E[n][a]  (FP64 column sums, fixed order)
template <typename T>
__global__ void k_colsum_scale(const T *E, long rows, int w, const double *sd, long off, double scale, double *S2)
{
    __shared__ double sm[8][33];
    const int col = blockIdx.x * 32 + threadIdx.x;
    double s = 0.0;
    if (col < w)
        for (long r = threadIdx.y; r < rows; r += 8) s += (double)E[r * w + col];
    sm[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && col < w) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += sm[i][threadIdx.x];
        const double d = sd[off + col];
        S2[off + col] = d * d * scale * t;
    }
}

template <typename T>
__global__ void k_to_t(const double *src, long n, T *dst)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// The DeepONet output bias: dS_jk/db0 = 1 for every term, so S2 = sd^2.
__global__ void k_scale_b0(const double *sd, long off, double *S2)
{
    const double d = sd[off];
    S2[off] = d * d;
}

inline dim3 grid_1d(long n)
{
    return dim3((unsigned)std::max<long>(1, std::min<long>((n + 255) / 256, 8192)));
}

// One feed-forward net at the VI mean: its forward pass on `rows` inputs, and the
// reverse passes of `nseeds` output seeds that give its parameters' S2.
template <typename T> struct SensNet {
    const NetDesc &nd;
    long rows;
    std::vector<std::unique_ptr<DevBuf>> A, S;   // A[0] = inputs; A[l], S[l] for l = 1..L

    SensNet(const NetDesc &d, long r) : nd(d), rows(r) {}

    void forward(const std::vector<double> &x, const T *theta, cudaStream_t s)
    {
        A.resize(nd.L + 1);
        S.resize(nd.L + 1);
        std::vector<T> xt(x.begin(), x.end());
        A[0].reset(new DevBuf(sizeof(T) * std::max<size_t>(xt.size(), 1)));
        if (!xt.empty())
            HMC_CK(cudaMemcpyAsync(A[0]->ptr, xt.data(), sizeof(T) * xt.size(), cudaMemcpyHostToDevice, s));
        HMC_CK(cudaStreamSynchronize(s));
        for (int l = 0; l < nd.L; ++l) {
            const int wi = nd.w[l], wo = nd.w[l + 1];
            A[l + 1].reset(new DevBuf(sizeof(T) * std::max<long>(rows * wo, 1)));
            S[l + 1].reset(new DevBuf(sizeof(T) * std::max<long>(rows * wo, 1)));
            // Z = A W^T + b (M = rows, N = wo, K = wi)
            GemmArgs<T> ga{(int)rows, wo, wi, A[l]->as<T>(), wi, 1, 0, theta + nd.woff[l], 1, wi, 0};
            EpiArgs<T> ea{EPI_ACT, A[l + 1]->as<T>(), wo, 1, 0, nd.boff[l] >= 0 ? theta + nd.boff[l] : nullptr, 1, 0,
                          nd.act[l], S[l + 1]->as<T>()};
            launch_gemm(ga, ea, 1, s);
        }
    }

    const T *out() const { return A[nd.L]->as<T>(); }

    // S2 of every parameter of this net.  G [nseeds][nseeds] (null: identity) weighs the
    // seeds' adjoints; scale = 1/N_d.
    void sens(const T *theta, int nseeds, const T *G, double scale, const double *sd, double *S2, cudaStream_t s)
    {
        const int L = nd.L;
        long wmax = 1;
        for (int l = 1; l <= L; ++l) wmax = std::max<long>(wmax, nd.w[l]);
        long win = 1, wprod = 1;   // widest layer input, largest weight matrix
        for (int l = 0; l < L; ++l) {
            win = std::max<long>(win, nd.w[l]);
            wprod = std::max<long>(wprod, (long)nd.w[l] * nd.w[l + 1]);
        }
        HMC_REQUIRE(rows * wmax < (1L << 30) && rows < (1L << 31), "layer too large for the sensitivity pass");
        const size_t big = sizeof(T) * std::max<long>((long)nseeds * rows * wmax, 1);
        DevBuf D0(big), D1(big), Q(G ? big : sizeof(T)), E(sizeof(T) * std::max<long>(rows * wmax, 1));
        DevBuf Asq(sizeof(T) * std::max<long>(rows * win, 1)), SW(sizeof(T) * wprod);
        T *D = D0.as<T>(), *Dn = D1.as<T>();
        {
            const int w = nd.w[L];
            k_seed<T><<<grid_1d((long)nseeds * rows * w), 256, 0, s>>>(S[L]->as<T>(), rows, w, nseeds, D);
            HMC_LAUNCH_CK();
        }
        for (int l = L; l >= 1; --l) {
            const int wo = nd.w[l], wi = nd.w[l - 1];
            const long nx = rows * wo;
            if (G) {   // Q[c][x] = sum_c' G[c][c'] D[c'][x]
                GemmArgs<T> ga{nseeds, (int)nx, nseeds, G, nseeds, 1, 0, D, nx, 1, 0};
                EpiArgs<T> ea{EPI_STORE, Q.as<T>(), nx, 1, 0, nullptr, 0, 0, 0, nullptr};
                launch_gemm(ga, ea, 1, s);
            }
            k_seed_energy<T><<<grid_1d(nx), 256, 0, s>>>(D, G ? Q.as<T>() : nullptr, nseeds, nx, E.as<T>());
            HMC_LAUNCH_CK();
            // weights: SW[a][b] = sum_n E[n][a] A_{l-1}[n][b]^2 (M = wo, N = wi, K = rows)
            k_square<T><<<grid_1d(rows * wi), 256, 0, s>>>(A[l - 1]->as<T>(), rows * wi, Asq.as<T>());
            HMC_LAUNCH_CK();
            {
                GemmArgs<T> ga{wo, wi, (int)rows, E.as<T>(), 1, wo, 0, Asq.as<T>(), wi, 1, 0};
                EpiArgs<T> ea{EPI_STORE, SW.as<T>(), wi, 1, 0, nullptr, 0, 0, 0, nullptr};
                launch_gemm(ga, ea, 1, s);
            }
            k_scale_out<T><<<grid_1d((long)wo * wi), 256, 0, s>>>(SW.as<T>(), (long)wo * wi, sd, nd.woff[l - 1],
                                                                   scale, S2);
            HMC_LAUNCH_CK();
            if (nd.boff[l - 1] >= 0) {
                k_colsum_scale<T><<<dim3((wo + 31) / 32), dim3(32, 8), 0, s>>>(E.as<T>(), rows, wo, sd,
                                                                              nd.boff[l - 1], scale, S2);
                HMC_LAUNCH_CK();
            }
            if (l > 1) {   // D_{l-1}[c] = (D_l[c] W_l) * act'(Z_{l-1})  (M = rows, N = wi, K = wo)
                GemmArgs<T> ga{(int)rows, wi, wo, D, wo, 1, nx, theta + nd.woff[l - 1], wi, 1, 0};
                EpiArgs<T> ea{EPI_SCALE, Dn, wi, 1, rows * wi, nullptr, 0, 0, 0, S[l - 1]->as<T>()};
                ea.slope_b = 0;
                launch_gemm(ga, ea, nseeds, s);
                std::swap(D, Dn);
            }
        }
        HMC_CK(cudaStreamSynchronize(s));   // before the work buffers are freed
    }
};

template <typename T>
void sensitivity_t(const SensProblem &pr, const double *mu, const double *sd, double *S2, cudaStream_t s)
{
    const long P = pr.P;
    DevBuf theta(sizeof(T) * std::max<long>(P, 1));
    k_to_t<T><<<grid_1d(P), 256, 0, s>>>(mu, P, theta.as<T>());
    HMC_LAUNCH_CK();
    const T *th = theta.as<T>();
    if (pr.kind == HMC_NET_MLP) {
        SensNet<T> net(pr.net, pr.n);
        net.forward(pr.x, th, s);
        const double scale = 1.0 / ((double)pr.n * pr.net.w[pr.net.L]);
        net.sens(th, pr.net.w[pr.net.L], nullptr, scale, sd, S2, s);
    } else {
        SensNet<T> br(pr.branch, pr.n_u), tr(pr.trunk, pr.n_y);
        br.forward(pr.u, th, s);
        tr.forward(pr.yq, th, s);
        const int p = pr.branch.w[pr.branch.L];
        DevBuf GT(sizeof(T) * p * p), GB(sizeof(T) * p * p);
        // G_T = T^T T and G_B = B^T B (M = N = p, K = rows)
        for (int which = 0; which < 2; ++which) {
            const T *X = which == 0 ? tr.out() : br.out();
            const long rows = which == 0 ? pr.n_y : pr.n_u;
            GemmArgs<T> ga{p, p, (int)rows, X, 1, p, 0, X, p, 1, 0};
            EpiArgs<T> ea{EPI_STORE, (which == 0 ? GT : GB).as<T>(), p, 1, 0, nullptr, 0, 0, 0, nullptr};
            launch_gemm(ga, ea, 1, s);
        }
        const double scale = 1.0 / ((double)pr.n_u * pr.n_y);
        br.sens(th, p, GT.as<T>(), scale, sd, S2, s);
        tr.sens(th, p, GB.as<T>(), scale, sd, S2, s);
        if (pr.out_bias) {   // dS_jk/db0 = 1 for every term
            k_scale_b0<<<1, 1, 0, s>>>(sd, P - 1, S2);
            HMC_LAUNCH_CK();
        }
    }
    HMC_CK(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// Truncation: stable LSD radix sort of (key, index) with 8-bit digits.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;   // one element per thread per tile
constexpr int RS_BINS = 256;

// Keys ascending = S2 descending: for non-negative doubles the bit pattern grows with
// the value, so its complement falls.  A negative or NaN S2 raises the error flag.
__global__ void k_keys(const double *S2, long P, unsigned long long *key, long long *idx, int *err)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long)gridDim.x * blockDim.x) {
        const double v = S2[i];
        if (!(v >= 0.0) || isinf(v)) atomicExch(err, 1);
        key[i] = ~(unsigned long long)__double_as_longlong(v + 0.0);   // -0 -> +0
        idx[i] = i;
    }
}

// hist[d * nblk + blk] = number of elements of tile blk whose digit is d.
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const unsigned long long *key, long P, int shift, int nblk,
                                                        unsigned *hist)
{
    __shared__ unsigned h[RS_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long i = (long)blockIdx.x * RS_THREADS + threadIdx.x;
    if (i < P) atomicAdd(&h[(key[i] >> shift) & 0xff], 1u);
    __syncthreads();
    hist[(long)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of n counts in place, one block, in order.
__global__ void __launch_bounds__(1024) k_rs_scan(unsigned *v, long n)
{
    __shared__ unsigned s[1024];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long base = 0; base < n; base += 1024) {
        const long i = base + threadIdx.x;
        const unsigned x = i < n ? v[i] : 0u;
        s[threadIdx.x] = x;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const unsigned t = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0u;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) v[i] = carry + s[threadIdx.x] - x;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

// Stable scatter: an element goes to its digit's tile offset plus its rank among the
// tile's elements of the same digit that precede it.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const unsigned long long *key, const long long *idx,
                                                           long P, int shift, int nblk, const unsigned *off,
                                                           unsigned long long *key_out, long long *idx_out)
{
    __shared__ unsigned wcnt[RS_THREADS / 32][RS_BINS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (RS_THREADS / 32) * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const long i = (long)blockIdx.x * RS_THREADS + threadIdx.x;
    const bool valid = i < P;
    const unsigned long long k = valid ? key[i] : 0ull;
    const unsigned d = valid ? (unsigned)((k >> shift) & 0xff) : RS_BINS;   // RS_BINS: no digit
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank_w = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank_w == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
        unsigned before = 0;
        for (int w2 = 0; w2 < warp; ++w2) before += wcnt[w2][d];
        const unsigned pos = off[(long)d * nblk + blockIdx.x] + before + rank_w;
        key_out[pos] = k;
        idx_out[pos] = idx[i];
    }
}

// Block-wise inclusive FP64 prefix sums of S2 in rank order; block totals to bsum.
constexpr int PS_THREADS = 1024;
__global__ void __launch_bounds__(PS_THREADS) k_prefix_local(const double *S2, const long long *order, long P,
                                                             double *cum, double *bsum)
{
    __shared__ double s[PS_THREADS];
    const long i = (long)blockIdx.x * PS_THREADS + threadIdx.x;
    s[threadIdx.x] = i < P ? S2[order[i]] : 0.0;
    __syncthreads();
    for (int o = 1; o < PS_THREADS; o <<= 1) {
        const double t = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0.0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < P) cum[i] = s[threadIdx.x];
    if (threadIdx.x == PS_THREADS - 1) bsum[blockIdx.x] = s[PS_THREADS - 1];
}

// Exclusive scan of the block totals (one thread, in order) and the grand total.
__global__ void k_prefix_blocks(double *bsum, long nb, double *total)
{
    double c = 0.0;
    for (long b = 0; b < nb; ++b) {
        const double t = bsum[b];
        bsum[b] = c;
        c += t;
    }
    *total = c;
}

// First rank whose prefix share exceeds tau (atomicMin over ranks).
__global__ void k_cut(const double *cum, const double *bsum, long P, const double *total, double tau,
                      unsigned long long *first)
{
    const double tot = *total;
    for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < P; r += (long)gridDim.x * blockDim.x) {
        const double c = cum[r] + bsum[r / PS_THREADS];
        if (!(tot > 0.0) || c / tot > tau) atomicMin(first, (unsigned long long)r);
    }
}

__global__ void k_mask(const long long *order, long P, const unsigned long long *first, unsigned char *mask,
                       long long *nhat)
{
    const long n = (long)*first;
    for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < P; r += (long)gridDim.x * blockDim.x)
        mask[order[r]] = r < n ? 1 : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *nhat = n;
}

}  // namespace

void sensitivity_run(const SensProblem &pr, int prec, const double *mu, const double *sd, double *S2,
                     cudaStream_t s)
{
    if (prec == HMC_PREC_FP64) sensitivity_t<double>(pr, mu, sd, S2, s);
    else sensitivity_t<float>(pr, mu, sd, S2, s);
}

long select_subset_run(const double *S2, long P, double tau, unsigned char *mask, long long *order_out,
                       cudaStream_t s)
{
    HMC_REQUIRE(P >= 1 && P < (1L << 31), "P must be in [1, 2^31)");
    const int nblk = (int)((P + RS_THREADS - 1) / RS_THREADS);
    DevBuf k0(8 * P), k1(8 * P), i0(8 * P), i1(8 * P), hist(sizeof(unsigned) * RS_BINS * (size_t)nblk),
        err(sizeof(int)), cum(8 * P), bsum(8 * ((P + PS_THREADS - 1) / PS_THREADS)), total(8), first(8), nhat(8);
    HMC_CK(cudaMemsetAsync(err.ptr, 0, sizeof(int), s));
    k_keys<<<grid_1d(P), 256, 0, s>>>(S2, P, k0.as<unsigned long long>(), i0.as<long long>(), err.as<int>());
    HMC_LAUNCH_CK();
    unsigned long long *ka = k0.as<unsigned long long>(), *kb = k1.as<unsigned long long>();
    long long *ia = i0.as<long long>(), *ib = i1.as<long long>();
    for (int shift = 0; shift < 64; shift += 8) {
        k_rs_hist<<<nblk, RS_THREADS, 0, s>>>(ka, P, shift, nblk, hist.as<unsigned>());
        HMC_LAUNCH_CK();
        k_rs_scan<<<1, 1024, 0, s>>>(hist.as<unsigned>(), (long)RS_BINS * nblk);
        HMC_LAUNCH_CK();
        k_rs_scatter<<<nblk, RS_THREADS, 0, s>>>(ka, ia, P, shift, nblk, hist.as<unsigned>(), kb, ib);
        HMC_LAUNCH_CK();
        std::swap(ka, kb);
        std::swap(ia, ib);
    }
    const long nb = (P + PS_THREADS - 1) / PS_THREADS;
    k_prefix_local<<<(unsigned)nb, PS_THREADS, 0, s>>>(S2, ia, P, cum.as<double>(), bsum.as<double>());
    HMC_LAUNCH_CK();
    k_prefix_blocks<<<1, 1, 0, s>>>(bsum.as<double>(), nb, total.as<double>());
    HMC_LAUNCH_CK();
    const unsigned long long none = (unsigned long long)P;
    HMC_CK(cudaMemcpyAsync(first.ptr, &none, 8, cudaMemcpyHostToDevice, s));
    k_cut<<<grid_1d(P), 256, 0, s>>>(cum.as<double>(), bsum.as<double>(), P, total.as<double>(), tau,
                                     first.as<unsigned long long>());
    HMC_LAUNCH_CK();
    k_mask<<<grid_1d(P), 256, 0, s>>>(ia, P, first.as<unsigned long long>(), mask, nhat.as<long long>());
    HMC_LAUNCH_CK();
    if (order_out) HMC_CK(cudaMemcpyAsync(order_out, ia, 8 * P, cudaMemcpyDeviceToDevice, s));
    int e = 0;
    long long n = 0;
    HMC_CK(cudaMemcpyAsync(&e, err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    HMC_CK(cudaMemcpyAsync(&n, nhat.ptr, 8, cudaMemcpyDeviceToHost, s));
    HMC_CK(cudaStreamSynchronize(s));
    HMC_REQUIRE(e == 0, "S2 holds a negative, infinite or NaN value");
    return (long)n;
}

}  // namespace hmc

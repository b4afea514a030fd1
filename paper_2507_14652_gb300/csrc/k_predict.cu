// k_predict.cu -- the posterior predictive (Sec. 4.2.1): the network's outputs on new
// inputs for every posterior sample, reduced over the samples to a mean and a
// standard deviation per output, and the mean relative L2 error of that mean.
//
// Samples run in batches: one theta per sample (the frozen vector with the sample
// scattered into the subset), a batched forward pass (samples in the grid's z), and a
// Welford update of the per-output running mean and sum of squared deviations in
// FP64, samples in order, so the result does not depend on the batch size.
#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "hmc_internal.cuh"

namespace hmc {
namespace {

#include "simt_kernels.cuh"

inline dim3 grid_1d(long n)
{
    return dim3((unsigned)std::max<long>(1, std::min<long>((n + 255) / 256, 8192)));
}

// thetas[c] = base for c < Cb
template <typename T>
__global__ void k_rep(const T *base, long P, int Cb, T *thetas)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < P * Cb; i += (long)gridDim.x * blockDim.x)
        thetas[i] = base[i % P];
}

// thetas[c][idx[j]] = samples[c][j]
template <typename T>
__global__ void k_scatter_samples(const T *samples, const int *idx, long k, int Cb, long P, T *thetas)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < k * Cb; i += (long)gridDim.x * blockDim.x) {
        const long c = i / k, j = i % k;
        thetas[c * P + idx[j]] = samples[i];
    }
}

// Welford over the batch, samples in order: n = done + c + 1.
template <typename T>
__global__ void k_welford(const T *F, long nout, int Cb, long done, double *mean, double *M2)
{
    for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < nout; x += (long)gridDim.x * blockDim.x) {
        double m = mean[x], q = M2[x];
        for (int c = 0; c < Cb; ++c) {
            const double f = (double)F[(long)c * nout + x];
            const double d = f - m;
            m += d / (double)(done + c + 1);
            q += d * (f - m);
        }
        mean[x] = m;
        M2[x] = q;
    }
}

__global__ void k_std(const double *M2, long n, long S, double *sd)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        sd[i] = sqrt(M2[i] / (double)S);
}

// ratio[i] = ||Y_i - Yp_i|| / ||Y_i|| for row i of length m (one block per row)
__global__ void __launch_bounds__(256) k_rel_rows(const double *Y, const double *Yp, long m, double *ratio)
{
    __shared__ double sm[8];
    const long i = blockIdx.x;
    double e = 0.0, y = 0.0;
    for (long j = threadIdx.x; j < m; j += blockDim.x) {
        const double t = Y[i * m + j], d = t - Yp[i * m + j];
        e += d * d;
        y += t * t;
    }
    const double es = block_sum<256>(e, sm);
    const double ys = block_sum<256>(y, sm);
    if (threadIdx.x == 0) ratio[i] = sqrt(es) / sqrt(ys);
}

__global__ void k_mean_of(const double *v, long n, double *out)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += v[i];
    *out = s / (double)n;
}

template <typename T> struct Batch {
    std::vector<std::unique_ptr<DevBuf>> act;
};

// Batched forward pass of one net over Cb thetas; returns the last layer's outputs.
template <typename T>
const T *forward(const NetDesc &nd, const T *X, long rows, const T *thetas, long P, int Cb, Batch<T> &b,
                 cudaStream_t s)
{
    const T *in = X;
    long in_b = 0;
    for (int l = 0; l < nd.L; ++l) {
        const int wi = nd.w[l], wo = nd.w[l + 1];
        T *out = b.act[l + 1]->template as<T>();
        GemmArgs<T> ga{(int)rows, wo, wi, in, wi, 1, in_b, thetas + nd.woff[l], 1, wi, P};
        EpiArgs<T> ea{EPI_ACT, out, wo, 1, rows * wo, nd.boff[l] >= 0 ? thetas + nd.boff[l] : nullptr, 1, P,
                      nd.act[l], nullptr};
        launch_gemm(ga, ea, Cb, s);
        in = out;
        in_b = rows * wo;
    }
    return in;
}

template <typename T> void alloc_net(const NetDesc &nd, long rows, int Cb, Batch<T> &b)
{
    b.act.resize(nd.L + 1);
    for (int l = 1; l <= nd.L; ++l) b.act[l].reset(new DevBuf(sizeof(T) * std::max<long>((long)Cb * rows * nd.w[l], 1)));
}

template <typename T> std::unique_ptr<DevBuf> upload(const std::vector<double> &v)
{
    std::vector<T> t(v.begin(), v.end());
    std::unique_ptr<DevBuf> d(new DevBuf(sizeof(T) * std::max<size_t>(t.size(), 1)));
    if (!t.empty()) HMC_CK(cudaMemcpy(d->ptr, t.data(), sizeof(T) * t.size(), cudaMemcpyHostToDevice));
    return d;
}

template <typename T>
void predict_t(const PredictInput &in, const void *samples_v, long S, double *mean, double *sd, double *rel,
               cudaStream_t s)
{
    const T *samples = static_cast<const T *>(samples_v);
    const long P = in.P, k = (long)in.idx.size();
    const bool mlp = in.kind == HMC_NET_MLP;
    const long nout = mlp ? in.n * in.net.w[in.net.L] : in.n_u * in.n_y;
    // samples per batch: about 1 GiB of thetas and activations
    long per = P;
    if (mlp) {
        for (int l = 1; l <= in.net.L; ++l) per += in.n * in.net.w[l];
    } else {
        for (int l = 1; l <= in.branch.L; ++l) per += in.n_u * in.branch.w[l];
        for (int l = 1; l <= in.trunk.L; ++l) per += in.n_y * in.trunk.w[l];
        per += nout;
    }
    const int Cb = (int)std::max<long>(1, std::min<long>({S, (1L << 30) / ((long)sizeof(T) * per), 65535}));
    auto base = upload<T>(in.frozen);
    std::vector<int> idx32(in.idx.begin(), in.idx.end());
    DevBuf idx(sizeof(int) * std::max<long>(k, 1));
    if (k) HMC_CK(cudaMemcpy(idx.ptr, idx32.data(), sizeof(int) * k, cudaMemcpyHostToDevice));
    auto X = upload<T>(mlp ? in.x : in.u), Y = upload<T>(mlp ? std::vector<double>() : in.yq);
    DevBuf thetas(sizeof(T) * (size_t)Cb * P), M2(sizeof(double) * std::max<long>(nout, 1)),
        Sout(mlp ? sizeof(T) : sizeof(T) * (size_t)Cb * nout);
    Batch<T> b1, b2;
    if (mlp) {
        alloc_net(in.net, in.n, Cb, b1);
    } else {
        alloc_net(in.branch, in.n_u, Cb, b1);
        alloc_net(in.trunk, in.n_y, Cb, b2);
    }
    HMC_CK(cudaMemsetAsync(mean, 0, sizeof(double) * nout, s));
    HMC_CK(cudaMemsetAsync(M2.ptr, 0, sizeof(double) * nout, s));
    for (long done = 0; done < S; done += Cb) {
        const int nb = (int)std::min<long>(Cb, S - done);
        k_rep<T><<<grid_1d(P * nb), 256, 0, s>>>(base->template as<T>(), P, nb, thetas.as<T>());
        HMC_LAUNCH_CK();
        if (k) {
            k_scatter_samples<T><<<grid_1d(k * nb), 256, 0, s>>>(samples + done * k, idx.as<int>(), k, nb, P,
                                                                   thetas.as<T>());
            HMC_LAUNCH_CK();
        }
        const T *F;
        if (mlp) {
            F = forward(in.net, X->template as<T>(), in.n, thetas.as<T>(), P, nb, b1, s);
        } else {
            const T *B = forward(in.branch, X->template as<T>(), in.n_u, thetas.as<T>(), P, nb, b1, s);
            const T *Tm = forward(in.trunk, Y->template as<T>(), in.n_y, thetas.as<T>(), P, nb, b2, s);
            const int p = in.branch.w[in.branch.L];
            // S = B T^T + b0 (M = n_u, N = n_y, K = p)
            GemmArgs<T> ga{(int)in.n_u, (int)in.n_y, p, B, p, 1, in.n_u * p, Tm, 1, p, in.n_y * p};
            EpiArgs<T> ea{EPI_ACT, Sout.as<T>(), in.n_y, 1, nout, in.out_bias ? thetas.as<T>() + (P - 1) : nullptr,
                          0, P, HMC_ACT_IDENTITY, nullptr};
            launch_gemm(ga, ea, nb, s);
            F = Sout.as<T>();
        }
        k_welford<T><<<grid_1d(nout), 256, 0, s>>>(F, nout, nb, done, mean, M2.as<double>());
        HMC_LAUNCH_CK();
    }
    k_std<<<grid_1d(nout), 256, 0, s>>>(M2.as<double>(), nout, S, sd);
    HMC_LAUNCH_CK();
    if (rel) {   // mean relative L2 error of the predictive mean against the targets
        const long rows = mlp ? 1 : in.n_u, m = mlp ? nout : in.n_y;
        DevBuf tgt(sizeof(double) * std::max<long>(nout, 1)), ratio(sizeof(double) * rows), out(sizeof(double));
        HMC_CK(cudaMemcpy(tgt.ptr, in.targets.data(), sizeof(double) * nout, cudaMemcpyHostToDevice));
        k_rel_rows<<<(unsigned)rows, 256, 0, s>>>(tgt.as<double>(), mean, m, ratio.as<double>());
        HMC_LAUNCH_CK();
        k_mean_of<<<1, 1, 0, s>>>(ratio.as<double>(), rows, out.as<double>());
        HMC_LAUNCH_CK();
        HMC_CK(cudaMemcpyAsync(rel, out.ptr, sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    HMC_CK(cudaStreamSynchronize(s));   // before the work buffers are freed
}

}  // namespace

void predict_run(const PredictInput &in, int prec, const void *samples, long S, double *mean, double *sd,
                 double *rel_l2, cudaStream_t s)
{
    if (prec == HMC_PREC_FP64) predict_t<double>(in, samples, S, mean, sd, rel_l2, s);
    else predict_t<float>(in, samples, S, mean, sd, rel_l2, s);
}

}  // namespace hmc

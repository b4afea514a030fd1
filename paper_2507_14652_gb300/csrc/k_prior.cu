// k_prior.cu -- the engine of a problem with no data terms (zero training points, or a
// DeepONet with no input functions or no query points).  The likelihood of an empty
// training set is 1, so the potential of Sec. 2.2 reduces to the Gaussian prior over the
// sampled subset Theta_s (Sec. 3.2; the frozen parameters add a constant that the energy
// leaves out, as it does with data):
//     U(q) = |q|^2 / (2 alpha^2),   grad U(q) = q / alpha^2.
// HMC then samples the prior itself and the leapfrog integrates a harmonic oscillator.
//
// The engine keeps the full parameter vector of every chain so that the trajectory
// kernels' scatter has a target ([C][P], q_j at index idx[j]), as every other engine does.
#include <algorithm>
#include <vector>

#include "hmc_internal.cuh"

namespace hmc {
namespace {

// One block per chain: g = q / alpha^2 and U = sum q^2 / (2 alpha^2), the sum in FP64
// in a fixed order (per-thread strided partials, then the warps in order).
template <typename T>
__global__ void __launch_bounds__(256) k_prior_energy_grad(const T *q, long k, double inv_a2, double *U, T *g)
{
    __shared__ double sm[8];
    pdl_wait();
    pdl_trigger();
    const long c = blockIdx.x;
    const T *qc = q + c * k;
    double s = 0.0;
    for (long j = threadIdx.x; j < k; j += blockDim.x) {
        const T v = qc[j];
        s += (double)v * (double)v;
        if (g) g[c * k + j] = (T)((double)v * inv_a2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w];
        U[c] = 0.5 * t * inv_a2;
    }
}

// theta[c][off[j]] = q[c][j]
template <typename T>
__global__ void k_prior_scatter(const T *q, long k, const int *off, long P, T *theta)
{
    pdl_wait();
    pdl_trigger();
    const long c = blockIdx.y;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (long)gridDim.x * blockDim.x)
        theta[c * P + off[j]] = q[c * k + j];
}

template <typename T> class PriorEngine final : public Engine {
  public:
    PriorEngine(const Problem &p, int C) : k_(p.k), P_(p.P), C_(C), inv_a2_(1.0 / (p.alpha * p.alpha))
    {
        std::vector<T> th((size_t)C * P_);
        for (int c = 0; c < C; ++c)
            for (long i = 0; i < P_; ++i) th[(size_t)c * P_ + i] = (T)p.frozen[i];
        theta_.alloc(sizeof(T) * std::max<size_t>(th.size(), 1));
        HMC_CK(cudaMemcpy(theta_.ptr, th.data(), sizeof(T) * th.size(), cudaMemcpyHostToDevice));
        std::vector<int> off(p.idx.begin(), p.idx.end());
        off_.alloc(sizeof(int) * std::max<size_t>(off.size(), 1));
        HMC_CK(cudaMemcpy(off_.ptr, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
        plan_.nbuf = 1;
        plan_.base[0] = theta_.ptr;
        plan_.cstride[0] = P_;
        plan_.off = off_.as<int>();
    }

    void energy_grad(const void *q, double *U, void *g, bool scattered, cudaStream_t s) override
    {
        if (!scattered) scatter(q, s);
        launch_pdl(k_prior_energy_grad<T>, dim3(C_), dim3(256), 0, s, static_cast<const T *>(q), k_, inv_a2_, U,
                   static_cast<T *>(g));
        HMC_LAUNCH_CK();
    }

    void scatter(const void *q, cudaStream_t s) override
    {
        const dim3 grid((unsigned)std::min<long>((k_ + 255) / 256, 1024), C_);
        launch_pdl(k_prior_scatter<T>, grid, dim3(256), 0, s, static_cast<const T *>(q), k_, off_.as<int>(), P_,
                   theta_.as<T>());
        HMC_LAUNCH_CK();
    }

    ScatterPlan scatter_plan() override { return plan_; }
    size_t bytes() const override { return theta_.n + off_.n; }

  private:
    long k_, P_;
    int C_;
    double inv_a2_;
    DevBuf theta_, off_;
    ScatterPlan plan_;
};

}  // namespace

Engine *make_prior_engine(const Problem &p, int prec, int C)
{
    if (prec == HMC_PREC_FP64) return new PriorEngine<double>(p, C);
    return new PriorEngine<float>(p, C);
}

}  // namespace hmc

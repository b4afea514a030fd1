// k_simt.cu -- CUDA-core engine for U and grad U in FP64 or FP32.
//
// Any MLP or DeepONet shape.  Per gradient evaluation (all chains batched in
// the grid's z dimension):
//   forward   A_l = act(A_{l-1} W_l^T + b_l), keeping A_l and act'(Z_l)
//   residual  r = F - y, U_lik partials sum r^2 in FP64, delta_L = r/sigma^2 * act'
//   reverse   dW_l = delta_l^T A_{l-1}, db_l = column sums of delta_l,
//             delta_{l-1} = (delta_l W_l) * act'(Z_{l-1}); it stops at the lowest
//             layer that holds a sampled parameter
//   DeepONet  S = B T^T + b0, dB = dS T, dT = dS^T B (Sec. 4.2 operator output)
//   finalize  U = sum partials / (2 sigma^2) + |q|^2/(2 alpha^2) (FP64, fixed order),
//             g_j = dU/dtheta_{idx_j} + q_j / alpha^2
// Every reduction has a fixed order, so results are bit-reproducible.
#include <cstdio>
#include <memory>

#include "hmc_internal.cuh"

namespace hmc {
namespace {

#include "simt_kernels.cuh"

// r = F - y; U partials (sum r^2, FP64); delta = r/sigma^2 * slope; sum of delta.
template <typename T>
__global__ void __launch_bounds__(256) k_residual(const T *f, long f_b, const T *y, long n_el,
                                                  const T *slope, double inv_s2, T *delta,
                                                  double *part_r2, double *part_d, int nparts)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    __shared__ double sm[8];
    const int b = blockIdx.y;
    double r2 = 0.0, ds = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += (long)gridDim.x * blockDim.x) {
        T r = f[(long)b * f_b + i] - y[i];
        double rd = (double)r;
        r2 += rd * rd;
        T d = (T)(rd * inv_s2);
        if (slope) d = d * slope[(long)b * f_b + i];
        delta[(long)b * f_b + i] = d;
        ds += (double)d;
    }
    double a = block_sum<256>(r2, sm);
    double c = block_sum<256>(ds, sm);
    if (threadIdx.x == 0) {
        part_r2[(long)b * nparts + blockIdx.x] = a;
        if (part_d) part_d[(long)b * nparts + blockIdx.x] = c;
    }
}


// The output layer and the residual in one pass (small output layers in FP64): element
// (row m, output o) of chain b, z = sum_k A[b][m][k] W[b][o][k] + bias[b][o] (k in order,
// as the GEMM sums it), f = act(z), r = f - y, delta = r / sigma^2 act'(z), and the
// block's sum of r^2 (FP64) as k_residual forms it.
template <typename T>
__global__ void __launch_bounds__(256) k_out_residual(const T *A, long a_b, int K, const T *W, const T *bias, long P,
                                                      int act, const T *y, long rows, int dout, double inv_s2,
                                                      T *delta, double *part_r2, int nparts)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    __shared__ double sm[8];
    const int b = blockIdx.y;
    const long n_el = rows * dout;
    double r2 = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += (long)gridDim.x * blockDim.x) {
        const long m = i / dout;
        const int o = (int)(i % dout);
        const T *a = A + (long)b * a_b + m * K;
        const T *w = W + (long)b * P + (long)o * K;
        T z = T(0);
        for (int k = 0; k < K; ++k) z += a[k] * w[k];
        if (bias) z += bias[(long)b * P + o];
        T f, sl;
        act_eval(act, z, f, sl);
        const T r = f - y[i];
        const double rd = (double)r;
        r2 += rd * rd;
        T d = (T)(rd * inv_s2);
        if (act != HMC_ACT_IDENTITY) d = d * sl;
        delta[(long)b * n_el + i] = d;
    }
    const double t = block_sum<256>(r2, sm);
    if (threadIdx.x == 0) part_r2[(long)b * nparts + blockIdx.x] = t;
}

template <typename T>
__global__ void k_scatter(const T *q, const int *idx, long k, T *theta, long P)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    const int b = blockIdx.y;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (long)gridDim.x * blockDim.x)
        theta[(long)b * P + idx[j]] = q[(long)b * k + j];
}

// U[b] and g[b][:] from the partials and the dense gradient G[b][P].
template <typename T>
__global__ void __launch_bounds__(256) k_finalize(const double *part_r2, const double *part_d, int nparts,
                                                  double half_inv_s2, const T *q, long k, const int *idx,
                                                  const T *G, long P, long b0_off, double inv_a2,
                                                  double *U, T *g)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    __shared__ double sm[8];
    __shared__ double s_db0;
    const int b = blockIdx.x;
    if (threadIdx.x == 0) {
        double t = 0.0;
        if (part_d)
            for (int i = 0; i < nparts; ++i) t += part_d[(long)b * nparts + i];
        s_db0 = t;
    }
    __syncthreads();
    const double db0 = s_db0;
    double pr = 0.0;
    for (long j = threadIdx.x; j < k; j += blockDim.x) {
        T qj = q[(long)b * k + j];
        pr += (double)qj * (double)qj;
        long id = idx[j];
        T gj = (id == b0_off) ? (T)db0 : G[(long)b * P + id];
        if (g) g[(long)b * k + j] = gj + qj * (T)inv_a2;
    }
    double prs = block_sum<256>(pr, sm);
    if (threadIdx.x == 0) {
        double lik = 0.0;
        for (int i = 0; i < nparts; ++i) lik += part_r2[(long)b * nparts + i];
        U[b] = lik * half_inv_s2 + 0.5 * prs * inv_a2;
    }
}


// DeepONet with per-function queries: S[c][j][k] = <B[c][j], T[c][j nq + k]> + b0.
template <typename T>
__global__ void k_rowdot(const T *B, const T *Tm, long n_u, long nq, int p, const T *b0, long P, T *S)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    const int c = blockIdx.y;
    const long n = n_u * nq;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const T *b = B + ((long)c * n_u + i / nq) * p;
        const T *t = Tm + ((long)c * n + i) * p;
        T acc = b0 ? b0[(long)c * P] : T(0);
        for (int q = 0; q < p; ++q) acc += b[q] * t[q];
        S[(long)c * n + i] = acc;
    }
}

// dB[c][j][q] = sl * sum_k dS[c][j][k] T[c][j nq + k][q]   (sl: branch output slope, or 1)
template <typename T>
__global__ void k_rowdot_dB(const T *dS, const T *Tm, long n_u, long nq, int p, const T *sl, T *dB)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    const int c = blockIdx.y;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n_u * p; i += (long)gridDim.x * blockDim.x) {
        const long j = i / p;
        const int q = (int)(i % p);
        const T *d = dS + ((long)c * n_u + j) * nq;
        const T *t = Tm + ((long)c * n_u * nq + j * nq) * p + q;
        T acc = T(0);
        for (long k = 0; k < nq; ++k) acc += d[k] * t[k * p];
        const long o = (long)c * n_u * p + i;
        dB[o] = sl ? acc * sl[o] : acc;
    }
}

// dT[c][j nq + k][q] = sl * dS[c][j][k] B[c][j][q]   (sl: trunk output slope, or 1)
template <typename T>
__global__ void k_rowdot_dT(const T *dS, const T *B, long n_u, long nq, int p, const T *sl, T *dT)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    const int c = blockIdx.y;
    const long n = n_u * nq * p;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long r = i / p;   // trunk row j nq + k
        const int q = (int)(i % p);
        const T v = dS[(long)c * n_u * nq + r] * B[((long)c * n_u + r / nq) * p + q];
        const long o = (long)c * n + i;
        dT[o] = sl ? v * sl[o] : v;
    }
}

template <typename T> struct NetBufs {
    std::vector<std::unique_ptr<DevBuf>> act, slope;   // index l = 1..L (output of layer l-1)
};

template <typename T> class SimtEngine final : public Engine {
  public:
    SimtEngine(Problem &p, int C) : p_(p), C_(C)
    {
        const long P = p.P;
        theta_.alloc(sizeof(T) * C * P);
        G_.alloc(sizeof(T) * C * P);
        idx_.alloc(sizeof(int) * std::max<long>(p.k, 1));
        std::vector<int> idx32(p.idx.begin(), p.idx.end());
        HMC_CK(cudaMemcpy(idx_.ptr, idx32.data(), sizeof(int) * p.k, cudaMemcpyHostToDevice));
        std::vector<T> th(C * P);
        for (int c = 0; c < C; ++c)
            for (long i = 0; i < P; ++i) th[c * P + i] = (T)p.frozen[i];
        HMC_CK(cudaMemcpy(theta_.ptr, th.data(), sizeof(T) * C * P, cudaMemcpyHostToDevice));
        HMC_CK(cudaMemset(G_.ptr, 0, sizeof(T) * C * P));
        if (p.kind == HMC_NET_MLP) {
            upload(x_, p.x);
            upload(y_, p.y);
            alloc_net(p.net, p.n, netb_);
            long wmax = max_width(p.net);
            row_alloc(p.arena, delta_[0], sizeof(T) * C * p.n * wmax);
            row_alloc(p.arena, delta_[1], sizeof(T) * C * p.n * wmax);
            n_el_ = p.n * p.dout;
        } else {
            upload(u_, p.u);
            upload(yq_, p.yq);
            upload(t_, p.t);
            // trunk rows: the shared queries, or every function's own
            nt_ = p.kind == HMC_NET_DEEPONET_UNALIGNED ? p.n_u * p.n_y : p.n_y;
            alloc_net(p.branch, p.n_u, brb_);
            alloc_net(p.trunk, nt_, trb_);
            const int lat = p.branch.w[p.branch.L];
            row_alloc(p.arena, S_, sizeof(T) * C * std::max<long>(p.n_u * p.n_y, 1));
            row_alloc(p.arena, dB_, sizeof(T) * C * p.n_u * lat);
            row_alloc(p.arena, dT_, sizeof(T) * C * nt_ * lat);
            long wmax = std::max(max_width(p.branch), max_width(p.trunk));
            long rows = std::max(p.n_u, nt_);
            row_alloc(p.arena, delta_[0], sizeof(T) * C * rows * wmax);
            row_alloc(p.arena, delta_[1], sizeof(T) * C * rows * wmax);
            n_el_ = p.n_u * p.n_y;
        }
        nparts_ = (int)std::min<long>(64, std::max<long>(1, (n_el_ + 255) / 256));
        part_r2_.alloc(sizeof(double) * C * nparts_);
        part_d_.alloc(sizeof(double) * C * nparts_);
        // split-K workspace of the FP32 reductions over data rows (weight gradients, dB, dT),
        // at most 256 MB; a GEMM whose partials do not fit runs unsplit
        if (sizeof(T) == 4) {
            size_t need = 0;
            auto net_need = [&](const NetDesc &nd, long rows) {
                for (int l = nd.lmin; l < nd.L; ++l)
                    need = std::max(need, gemm_ws_floats(nd.w[l + 1], nd.w[l], (int)rows, C));
            };
            if (p.kind == HMC_NET_MLP) {
                net_need(p.net, p.n);
            } else {
                const int lat = p.branch.w[p.branch.L];
                net_need(p.branch, p.n_u);
                net_need(p.trunk, nt_);
                need = std::max(need, gemm_ws_floats((int)p.n_u, lat, (int)p.n_y, C));
                need = std::max(need, gemm_ws_floats((int)p.n_y, lat, (int)p.n_u, C));
            }
            ws_floats_ = std::min<size_t>(need, (size_t)64 << 20);
            row_alloc(p.arena, ws_, sizeof(float) * ws_floats_);   // requested even when empty (arena order)
            if (ws_.own) bytes_ += ws_.n;
        }
        for (DevBuf *b : {&delta_[0], &delta_[1], &S_, &dB_, &dT_})
            if (b->own) bytes_ += b->n;
    }

    ScatterPlan scatter_plan() override
    {
        ScatterPlan sp;
        sp.nbuf = 1;
        sp.base[0] = theta_.ptr;
        sp.cstride[0] = p_.P;
        sp.kind16[0] = 0;
        sp.buf_id = nullptr;
        sp.off = idx_.as<int>();
        return sp;
    }

    size_t bytes() const override { return bytes_; }

    void scatter(const void *qv, cudaStream_t s) override
    {
        if (p_.k <= 0) return;
        dim3 grid((unsigned)std::min<long>((p_.k + 255) / 256, 1024), C_);
        launch_pdl(k_scatter<T>, grid, dim3(256), 0, s, static_cast<const T *>(qv), (const int *)idx_.as<int>(), p_.k,
                   theta_.as<T>(), p_.P);
        HMC_LAUNCH_CK();
    }

    void energy_grad(const void *qv, double *U, void *gv, bool scattered, cudaStream_t s) override
    {
        const T *q = static_cast<const T *>(qv);
        T *g = static_cast<T *>(gv);
        const long P = p_.P, k = p_.k;
        T *theta = theta_.as<T>();
        if (!scattered) scatter(qv, s);
        const double inv_s2 = 1.0 / (p_.sigma * p_.sigma);
        if (p_.kind == HMC_NET_MLP) {
            const NetDesc &nd = p_.net;
            if (sizeof(T) == 8 && p_.dout <= 8) {   // the output layer and the residual in one launch
                forward(nd, x_.as<T>(), 0, p_.n, netb_, s, nd.L - 1);
                const int l = nd.L - 1;
                const T *a = l > 0 ? netb_.act[l]->template as<T>() : x_.as<T>();
                ProfScope ps("simt_out_residual", s);
                launch_pdl(k_out_residual<T>, dim3(nparts_, C_), dim3(256), 0, s, a, l > 0 ? p_.n * nd.w[l] : 0L,
                           nd.w[l], (const T *)(theta + nd.woff[l]),
                           (const T *)(nd.boff[l] >= 0 ? theta + nd.boff[l] : nullptr), P, nd.act[l],
                           (const T *)y_.as<T>(), p_.n, p_.dout, inv_s2, delta_[0].as<T>(), part_r2_.as<double>(),
                           nparts_);
            } else {
                forward(nd, x_.as<T>(), 0, p_.n, netb_, s);
                T *f = netb_.act[nd.L]->template as<T>();
                const T *sl = nd.act[nd.L - 1] == HMC_ACT_IDENTITY ? nullptr : netb_.slope[nd.L]->template as<T>();
                residual(f, p_.n * p_.dout, y_.as<T>(), sl, inv_s2, delta_[0].as<T>(), false, s);
            }
            if (nd.any_sampled && g) backward(nd, x_.as<T>(), 0, p_.n, netb_, delta_[0].as<T>(), s);
        } else {
            const NetDesc &bn = p_.branch, &tn = p_.trunk;
            const int lat = bn.w[bn.L];
            const bool ua = p_.kind == HMC_NET_DEEPONET_UNALIGNED;
            forward(bn, u_.as<T>(), 0, p_.n_u, brb_, s);
            forward(tn, yq_.as<T>(), 0, nt_, trb_, s);
            T *Bm = brb_.act[bn.L]->template as<T>();
            T *Tm = trb_.act[tn.L]->template as<T>();
            T *S = S_.as<T>();
            const dim3 ua_grid((unsigned)std::min<long>((p_.n_u * p_.n_y * lat + 255) / 256, 4096), C_);
            if (ua) {   // S_jk = <B_j, T_jk> + b0
                launch_pdl(k_rowdot<T>, ua_grid, dim3(256), 0, s, (const T *)Bm, (const T *)Tm, p_.n_u, p_.n_y, lat,
                           (const T *)(p_.out_bias ? theta + p_.b0_off : nullptr), P, S);
                HMC_LAUNCH_CK();
            } else {   // S = B T^T + b0
                GemmArgs<T> ga{(int)p_.n_u, (int)p_.n_y, lat, Bm, lat, 1, p_.n_u * lat,
                               Tm, 1, lat, p_.n_y * lat};
                EpiArgs<T> ea{EPI_ACT, S, p_.n_y, 1, p_.n_u * p_.n_y,
                              p_.out_bias ? theta + p_.b0_off : nullptr, 0, P, HMC_ACT_IDENTITY, nullptr};
                launch_gemm(ga, ea, C_, s, ws_.template as<float>(), ws_floats_);
            }
            residual(S, p_.n_u * p_.n_y, t_.as<T>(), nullptr, inv_s2, S, true, s);
            if (ua && bn.any_sampled && g) {   // dB_j = sum_k dS_jk T_jk (times the branch output slope)
                const bool id = bn.act[bn.L - 1] == HMC_ACT_IDENTITY;
                launch_pdl(k_rowdot_dB<T>, ua_grid, dim3(256), 0, s, (const T *)S, (const T *)Tm, p_.n_u, p_.n_y, lat,
                           (const T *)(id ? nullptr : brb_.slope[bn.L]->template as<T>()), dB_.as<T>());
                HMC_LAUNCH_CK();
                backward(bn, u_.as<T>(), 0, p_.n_u, brb_, dB_.as<T>(), s);
            }
            if (ua && tn.any_sampled && g) {   // dT_jk = dS_jk B_j (times the trunk output slope)
                const bool id = tn.act[tn.L - 1] == HMC_ACT_IDENTITY;
                launch_pdl(k_rowdot_dT<T>, ua_grid, dim3(256), 0, s, (const T *)S, (const T *)Bm, p_.n_u, p_.n_y, lat,
                           (const T *)(id ? nullptr : trb_.slope[tn.L]->template as<T>()), dT_.as<T>());
                HMC_LAUNCH_CK();
                backward(tn, yq_.as<T>(), 0, nt_, trb_, dT_.as<T>(), s);
            }
            if (!ua && bn.any_sampled && g) {   // dB = dS T (times the branch output slope)
                const bool id = bn.act[bn.L - 1] == HMC_ACT_IDENTITY;
                GemmArgs<T> ga{(int)p_.n_u, lat, (int)p_.n_y, S, p_.n_y, 1, p_.n_u * p_.n_y,
                               Tm, lat, 1, p_.n_y * lat};
                EpiArgs<T> ea{id ? EPI_STORE : EPI_SCALE, dB_.as<T>(), lat, 1, p_.n_u * lat, nullptr, 0, 0, 0,
                              id ? nullptr : brb_.slope[bn.L]->template as<T>()};
                launch_gemm(ga, ea, C_, s, ws_.template as<float>(), ws_floats_);
                backward(bn, u_.as<T>(), 0, p_.n_u, brb_, dB_.as<T>(), s);
            }
            if (!ua && tn.any_sampled && g) {   // dT = dS^T B
                const bool id = tn.act[tn.L - 1] == HMC_ACT_IDENTITY;
                GemmArgs<T> ga{(int)p_.n_y, lat, (int)p_.n_u, S, 1, p_.n_y, p_.n_u * p_.n_y,
                               Bm, lat, 1, p_.n_u * lat};
                EpiArgs<T> ea{id ? EPI_STORE : EPI_SCALE, dT_.as<T>(), lat, 1, p_.n_y * lat, nullptr, 0, 0, 0,
                              id ? nullptr : trb_.slope[tn.L]->template as<T>()};
                launch_gemm(ga, ea, C_, s, ws_.template as<float>(), ws_floats_);
                backward(tn, yq_.as<T>(), 0, p_.n_y, trb_, dT_.as<T>(), s);
            }
        }
        ProfScope ps("simt_finalize", s);
        const bool don = p_.kind != HMC_NET_MLP;
        launch_pdl(k_finalize<T>, dim3(C_), dim3(256), 0, s, (const double *)part_r2_.as<double>(),
                   (const double *)(don ? part_d_.as<double>() : nullptr), nparts_, 0.5 * inv_s2, q, k,
                   (const int *)idx_.as<int>(), (const T *)G_.as<T>(), P, (long)(don && p_.out_bias ? p_.b0_off : -1),
                   1.0 / (p_.alpha * p_.alpha), U, g);
        HMC_LAUNCH_CK();
    }

  private:
    static long max_width(const NetDesc &nd)
    {
        long w = 1;
        for (int l = 0; l <= nd.L; ++l) w = std::max<long>(w, nd.w[l]);
        return w;
    }

    void upload(DevBuf &dst, const std::vector<double> &src)
    {
        std::vector<T> v(src.begin(), src.end());
        dst.alloc(sizeof(T) * std::max<size_t>(v.size(), 1));
        if (!v.empty()) HMC_CK(cudaMemcpy(dst.ptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
        bytes_ += dst.n;
    }

    void alloc_net(const NetDesc &nd, long rows, NetBufs<T> &nb)
    {
        nb.act.resize(nd.L + 1);
        nb.slope.resize(nd.L + 1);
        for (int l = 1; l <= nd.L; ++l) {
            size_t n = sizeof(T) * C_ * std::max<long>(rows * nd.w[l], 1);
            nb.act[l].reset(new DevBuf());
            nb.slope[l].reset(new DevBuf());
            row_alloc(p_.arena, *nb.act[l], n);
            row_alloc(p_.arena, *nb.slope[l], n);
            if (nb.act[l]->own) bytes_ += 2 * n;
        }
    }

    // layers 0 .. upto - 1 (all of them when upto < 0)
    void forward(const NetDesc &nd, const T *in, long in_b, long rows, NetBufs<T> &nb, cudaStream_t s, int upto = -1)
    {
        const long P = p_.P;
        T *theta = theta_.as<T>();
        const T *a = in;
        long a_b = in_b;
        for (int l = 0; l < (upto < 0 ? nd.L : upto); ++l) {
            const int wi = nd.w[l], wo = nd.w[l + 1];
            GemmArgs<T> ga{(int)rows, wo, wi, a, wi, 1, a_b, theta + nd.woff[l], 1, wi, P};
            EpiArgs<T> ea{EPI_ACT, nb.act[l + 1]->template as<T>(), wo, 1, rows * wo,
                          nd.boff[l] >= 0 ? theta + nd.boff[l] : nullptr, 1, P, nd.act[l],
                          nd.act[l] == HMC_ACT_IDENTITY ? nullptr : nb.slope[l + 1]->template as<T>()};
            launch_gemm(ga, ea, C_, s, ws_.template as<float>(), ws_floats_);
            a = nb.act[l + 1]->template as<T>();
            a_b = rows * wo;
        }
    }

    // delta_L (already multiplied by the output slope) in dL [C][rows][w_L].
    void backward(const NetDesc &nd, const T *in, long in_b, long rows, NetBufs<T> &nb, T *dL, cudaStream_t s)
    {
        const long P = p_.P;
        T *theta = theta_.as<T>();
        T *G = G_.as<T>();
        T *d = dL;
        int pp = 0;
        for (int l = nd.L - 1; l >= nd.lmin; --l) {
            const int wi = nd.w[l], wo = nd.w[l + 1];
            const T *ap = l == 0 ? in : nb.act[l]->template as<T>();
            const long ap_b = l == 0 ? in_b : rows * wi;
            // dW_l = delta_l^T A_{l-1} (and db_l = delta_l^T 1 where the kernel takes it)
            GemmArgs<T> gw{wo, wi, (int)rows, d, 1, wo, rows * wo, ap, wi, 1, ap_b};
            EpiArgs<T> ew{EPI_STORE, G + nd.woff[l], wi, 1, P, nullptr, 0, 0, 0, nullptr};
            T *rs = nd.boff[l] >= 0 ? G + nd.boff[l] : nullptr;
            // delta_{l-1} = (delta_l W_l) * act'(Z_{l-1}), when a layer below needs it
            T *nx = delta_[pp].as<T>();
            if (nx == d) nx = delta_[pp ^ 1].as<T>();
            const bool id = l > 0 && nd.act[l - 1] == HMC_ACT_IDENTITY;
            GemmArgs<T> gd{(int)rows, wi, wo, d, wo, 1, rows * wo, theta + nd.woff[l], wi, 1, P};
            EpiArgs<T> ed{id ? EPI_STORE : EPI_SCALE, nx, wi, 1, rows * wi, nullptr, 0, 0, 0,
                          id || l == 0 ? nullptr : nb.slope[l]->template as<T>()};
            // both read delta_l only: one launch where the FP64 kernels allow it
            const bool both = l > nd.lmin && launch_wgrad_and_delta(gw, ew, rs, P, gd, ed, C_, s);
            const bool db_done = both ? rs != nullptr
                                      : launch_wgrad(gw, ew, C_, s, ws_.template as<float>(), ws_floats_, rs, P) &&
                                            rs != nullptr;
            if (rs && !db_done) {
                dim3 grid((wo + 31) / 32, C_);
                ProfScope ps("simt_colsum", s);
                launch_pdl(k_colsum<T>, grid, dim3(32, 8), 0, s, (const T *)d, rows, wo, rows * wo, rs, P);
                HMC_LAUNCH_CK();
            }
            if (l > nd.lmin) {
                if (!both) launch_gemm(gd, ed, C_, s, ws_.template as<float>(), ws_floats_);
                d = nx;
                pp ^= 1;
            }
        }
    }

    void residual(const T *f, long n_el, const T *y, const T *slope, double inv_s2, T *delta, bool want_d,
                  cudaStream_t s)
    {
        dim3 grid(nparts_, C_);
        ProfScope ps("simt_residual", s);
        launch_pdl(k_residual<T>, grid, dim3(256), 0, s, f, n_el, y, n_el, slope, inv_s2, delta, part_r2_.as<double>(),
                   want_d ? part_d_.as<double>() : nullptr, nparts_);
        HMC_LAUNCH_CK();
    }

    Problem &p_;
    int C_;
    size_t bytes_ = 0;
    DevBuf theta_, G_, idx_, x_, y_, u_, yq_, t_, S_, dB_, dT_, part_r2_, part_d_, ws_;
    size_t ws_floats_ = 0;
    DevBuf delta_[2];
    NetBufs<T> netb_, brb_, trb_;
    long n_el_ = 0;
    long nt_ = 0;   // DeepONet trunk rows
    int nparts_ = 1;
};

}  // namespace

Engine *make_simt_engine_f64(Problem &p, int C) { return new SimtEngine<double>(p, C); }
Engine *make_simt_engine_f32(Problem &p, int C) { return new SimtEngine<float>(p, C); }

}  // namespace hmc

// ---------------------------------------------------------------------------
// U and grad U without any device allocation (hmc_energy_grad_noalloc).
//
// Every intermediate of the CUDA-core FP32 evaluation (per-chain parameter
// vectors, activations, slopes, deltas, the dense gradient and the energy
// partials) is carved out of one fixed array that lives in the library's
// device image.  Each GPU that loads the library holds this array until the
// process exits.  All calls share it, so calls that overlap on the GPU (two
// streams, two host threads) race and corrupt each other's results.
// ---------------------------------------------------------------------------
#include <mutex>

namespace hmc {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device.  In host code the
// array's name is only a host-side stand-in, so the address has to be asked
// for once per device, with that device current.
void *noalloc_scratch_address()
{
    int dev = 0;
    HMC_CK(cudaGetDevice(&dev));
    HMC_REQUIRE(dev >= 0 && dev < kMaxDevices, "device index %d is out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        HMC_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

__global__ void k_copy_rep(const float *src, long P, int C, float *dst)
{
    const long tot = P * (long)C;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x)
        dst[i] = src[i % P];
}

// The caller's index list is only read here: every entry that is outside [0, P) or
// not above its predecessor raises *bad and is replaced by 0, so the scatter and the
// gather that follow stay inside the scratch array whatever the caller passed.
__global__ void k_sanitize_idx(const int *idx, long k, long P, int *safe, int *bad)
{
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (long)gridDim.x * blockDim.x) {
        const int v = idx[j];
        const bool ok = v >= 0 && (long)v < P && (j == 0 || idx[j - 1] < v);
        safe[j] = ok ? v : 0;
        if (!ok) atomicOr(bad, 1);
    }
}

// A rejected index list makes every chain's U NaN (and its gradient, if asked for).
__global__ void k_poison_if_bad(const int *bad, int C, long k, double *U, float *g)
{
    if (!*bad) return;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < (long)C; i += (long)gridDim.x * blockDim.x)
        U[i] = nan;
    if (g)
        for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < (long)C * k; i += (long)gridDim.x * blockDim.x)
            g[i] = __int_as_float(0x7fc00000);
}

}  // namespace
}  // namespace hmc

extern "C" hmc_status hmc_energy_grad_noalloc(const hmc_mlp_spec *net, const float *x, const float *y, long n,
                                              const float *frozen, const int *subset_idx, long k,
                                              double prior_sigma, double noise_sigma, int n_chains,
                                              const float *q, double *U, float *grad, void *cuda_stream)
{
    using namespace hmc;
    try {
        HMC_REQUIRE(net && x && y && frozen && subset_idx && q && U, "NULL argument");
        HMC_REQUIRE(net->n_layers >= 1 && net->n_layers <= HMC_MAX_LAYERS, "n_layers must be in [1, %d]",
                    HMC_MAX_LAYERS);
        HMC_REQUIRE(n >= 1 && k >= 1 && n_chains >= 1 && n_chains <= 65535, "need n >= 1, k >= 1, 1 <= C <= 65535");
        HMC_REQUIRE(prior_sigma > 0 && noise_sigma > 0, "prior_sigma and noise_sigma must be positive");
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        const int C = n_chains, L = net->n_layers;
        // layer offsets in the parameter vector (W[out][in] then b[out], layer by layer)
        long woff[MAXL], boff[MAXL], P = 0;
        long wmax = 1;
        const long cap = (long)(kNoAllocScratchBytes / sizeof(float));   // floats the scratch array holds
        for (int l = 0; l < L; ++l) {
            HMC_REQUIRE(net->widths[l] >= 1 && net->widths[l + 1] >= 1 && net->widths[l] <= cap &&
                            net->widths[l + 1] <= cap,
                        "widths must be in [1, %ld]", cap);
            HMC_REQUIRE(net->act[l] >= HMC_ACT_IDENTITY && net->act[l] <= HMC_ACT_SIN, "bad activation");
            woff[l] = P;
            P += (long)net->widths[l + 1] * net->widths[l];
            boff[l] = -1;
            if (net->has_bias[l]) {
                boff[l] = P;
                P += net->widths[l + 1];
            }
        }
        for (int l = 0; l <= L; ++l) wmax = std::max<long>(wmax, net->widths[l]);
        HMC_REQUIRE(k <= P, "k (%ld) exceeds the parameter count (%ld)", k, P);
        // every array below is at most C * max(P, n * wmax) floats: bound the factors by
        // division first, so that no size computed afterwards can wrap around
        if (n > cap / ((long)C * wmax) || P > cap / C) {
            set_error("hmc_energy_grad_noalloc: this problem's intermediates exceed the fixed %zu-byte (16 MiB) "
                      "scratch array: use hmc_create/hmc_energy_grad instead", kNoAllocScratchBytes);
            return HMC_ERR_ARG;
        }
        const int dout = net->widths[L];
        const long n_el = n * dout;
        const int nparts = (int)std::min<long>(64, std::max<long>(1, (n_el + 255) / 256));
        // scratch layout, every block 256-byte aligned
        auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
        size_t need = 0;
        const size_t o_part = need; need += up(sizeof(double) * C * nparts);
        const size_t o_theta = need; need += up(sizeof(float) * C * P);
        const size_t o_G = need; need += up(sizeof(float) * C * P);
        size_t o_act[MAXL + 1] = {}, o_slope[MAXL + 1] = {};
        for (int l = 1; l <= L; ++l) {
            o_act[l] = need; need += up(sizeof(float) * C * n * net->widths[l]);
            o_slope[l] = need; need += up(sizeof(float) * C * n * net->widths[l]);
        }
        const size_t o_d0 = need; need += up(sizeof(float) * C * n * wmax);
        const size_t o_d1 = need; need += up(sizeof(float) * C * n * wmax);
        const size_t o_idx = need; need += up(sizeof(int) * k);
        const size_t o_bad = need; need += up(sizeof(int));
        if (need > kNoAllocScratchBytes) {
            set_error("hmc_energy_grad_noalloc needs %zu bytes of scratch for this problem; the fixed maximum is "
                      "%zu bytes (16 MiB): use hmc_create/hmc_energy_grad instead", need, kNoAllocScratchBytes);
            return HMC_ERR_ARG;
        }
        unsigned char *base = static_cast<unsigned char *>(noalloc_scratch_address());
        double *part = reinterpret_cast<double *>(base + o_part);
        float *theta = reinterpret_cast<float *>(base + o_theta);
        float *G = reinterpret_cast<float *>(base + o_G);
        float *d[2] = {reinterpret_cast<float *>(base + o_d0), reinterpret_cast<float *>(base + o_d1)};
        auto act = [&](int l) { return reinterpret_cast<float *>(base + o_act[l]); };
        auto slope = [&](int l) { return reinterpret_cast<float *>(base + o_slope[l]); };
        int *idx = reinterpret_cast<int *>(base + o_idx);
        int *bad = reinterpret_cast<int *>(base + o_bad);
        // the array keeps the previous call's contents: the flag must start at zero
        HMC_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
        k_sanitize_idx<<<(unsigned)std::min<long>((k + 255) / 256, 1024), 256, 0, s>>>(subset_idx, k, P, idx, bad);
        HMC_LAUNCH_CK();
        // the gradient buffer is read only at the sampled entries, all of which the
        // reverse pass rewrites; it is still cleared so no stale value can leak out
        HMC_CK(cudaMemsetAsync(G, 0, sizeof(float) * C * P, s));
        // theta[c] = frozen, then theta[c][idx[j]] = q[c][j]
        k_copy_rep<<<(unsigned)std::min<long>((C * P + 255) / 256, 4096), 256, 0, s>>>(frozen, P, C, theta);
        HMC_LAUNCH_CK();
        {
            dim3 grid((unsigned)std::min<long>((k + 255) / 256, 1024), C);
            k_scatter<float><<<grid, 256, 0, s>>>(q, idx, k, theta, P);
            HMC_LAUNCH_CK();
        }
        // forward
        const float *a = x;
        long a_b = 0;
        for (int l = 0; l < L; ++l) {
            const int wi = net->widths[l], wo = net->widths[l + 1];
            GemmArgs<float> ga{(int)n, wo, wi, a, wi, 1, a_b, theta + woff[l], 1, wi, P};
            EpiArgs<float> ea{EPI_ACT, act(l + 1), wo, 1, n * wo, boff[l] >= 0 ? theta + boff[l] : nullptr, 1, P,
                              net->act[l], net->act[l] == HMC_ACT_IDENTITY ? nullptr : slope(l + 1)};
            launch_gemm(ga, ea, C, s);
            a = act(l + 1);
            a_b = n * wo;
        }
        // residual and energy partials
        const double inv_s2 = 1.0 / (noise_sigma * noise_sigma);
        {
            dim3 grid(nparts, C);
            const float *sl = net->act[L - 1] == HMC_ACT_IDENTITY ? nullptr : slope(L);
            k_residual<float><<<grid, 256, 0, s>>>(act(L), n_el, y, n_el, sl, inv_s2, d[0], part, nullptr, nparts);
            HMC_LAUNCH_CK();
        }
        // reverse pass over every layer
        float *dd = d[0];
        int pp = 1;
        for (int l = L - 1; l >= 0; --l) {
            const int wi = net->widths[l], wo = net->widths[l + 1];
            const float *ap = l == 0 ? x : act(l);
            const long ap_b = l == 0 ? 0 : n * wi;
            GemmArgs<float> gw{wo, wi, (int)n, dd, 1, wo, n * wo, ap, wi, 1, ap_b};
            EpiArgs<float> ew{EPI_STORE, G + woff[l], wi, 1, P, nullptr, 0, 0, 0, nullptr};
            launch_gemm(gw, ew, C, s);
            if (boff[l] >= 0) {
                dim3 grid((wo + 31) / 32, C);
                k_colsum<float><<<grid, dim3(32, 8), 0, s>>>(dd, n, wo, n * wo, G + boff[l], P);
                HMC_LAUNCH_CK();
            }
            if (l > 0) {
                const bool id = net->act[l - 1] == HMC_ACT_IDENTITY;
                GemmArgs<float> gi{(int)n, wi, wo, dd, wo, 1, n * wo, theta + woff[l], wi, 1, P};
                EpiArgs<float> ei{id ? EPI_STORE : EPI_SCALE, d[pp], wi, 1, n * wi, nullptr, 0, 0, 0,
                                  id ? nullptr : slope(l)};
                launch_gemm(gi, ei, C, s);
                dd = d[pp];
                pp ^= 1;
            }
        }
        k_finalize<float><<<C, 256, 0, s>>>(part, nullptr, nparts, 0.5 * inv_s2, q, k, idx, G, P, -1,
                                            1.0 / (prior_sigma * prior_sigma), U, grad);
        HMC_LAUNCH_CK();
        k_poison_if_bad<<<(unsigned)std::min<long>(((long)C * k + 255) / 256, 1024), 256, 0, s>>>(bad, C, k, U, grad);
        HMC_LAUNCH_CK();
        return HMC_OK;
    } catch (const Fail &f) {
        return f.st;
    }
}

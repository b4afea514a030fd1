// simt_kernels.cuh -- CUDA-core building blocks shared by the FP64/FP32 engine and the
// sensitivity pass: batched GEMMs with fused epilogues (FP32 on 128 x 128 tiles with a
// split-K for long reductions, FP64 on 16 x 16 tiles), a fixed-order FP64 block sum and
// FP64 column sums.  Include it inside an anonymous namespace of
// namespace hmc (every translation unit keeps its own copies).
#pragma once

template <typename T> struct GemmArgs {
    int M, N, K;
    const T *A; long a_m, a_k, a_b;
    const T *B; long b_k, b_n, b_b;
};

enum { EPI_ACT = 0, EPI_SCALE = 1, EPI_STORE = 2 };

template <typename T> struct EpiArgs {
    int mode;
    T *out; long o_m, o_n, o_b;
    const T *bias; long bias_n, bias_b;
    int act;
    T *slope;   // EPI_ACT: receives act'(z); EPI_SCALE: multiplies the result (same layout as out)
    long slope_b = -1;   // EPI_SCALE: batch stride of slope (-1: that of out)
};

__device__ __forceinline__ void act_eval(int act, double z, double &a, double &s)
{
    if (act == HMC_ACT_TANH) { a = tanh(z); s = 1.0 - a * a; }
    else if (act == HMC_ACT_SIN) { a = sin(z); s = cos(z); }
    else { a = z; s = 1.0; }
}
__device__ __forceinline__ void act_eval(int act, float z, float &a, float &s)
{
    if (act == HMC_ACT_TANH) { a = tanhf(z); s = 1.0f - a * a; }
    else if (act == HMC_ACT_SIN) { a = sinf(z); s = cosf(z); }
    else { a = z; s = 1.0f; }
}

// The epilogue of output (m, n) of batch b: activation (and its slope), a scale, or a store.
template <typename T>
__device__ __forceinline__ void gemm_epilogue(const EpiArgs<T> &e, int b, long m, long n, T v)
{
    const long o = (long)b * e.o_b + m * e.o_m + n * e.o_n;
    if (e.mode == EPI_ACT) {
        const T z = v + (e.bias ? e.bias[(long)b * e.bias_b + n * e.bias_n] : T(0));
        T a, sl;
        act_eval(e.act, z, a, sl);
        e.out[o] = a;
        if (e.slope) e.slope[o] = sl;
    } else if (e.mode == EPI_SCALE) {
        const long so = (long)b * (e.slope_b < 0 ? e.o_b : e.slope_b) + m * e.o_m + n * e.o_n;
        e.out[o] = v * e.slope[so];
    } else {
        e.out[o] = v;
    }
}

// FP64: C[b](m, n) = sum_k A[b](m, k) B[b](k, n), one output per thread on 16 x 16 tiles.
// GB300's FP64 units are few, so work on padding costs real time: a 16 x 16 tile wastes
// little on the small shapes the FP64 engine serves (a 20 x 20 weight gradient filled 10%
// of a 64 x 64 tile).  Each output sums K in order, so results are reproducible.
template <typename T>
__device__ __forceinline__ void gemm16_body(const GemmArgs<T> &g, const EpiArgs<T> &e, int bx, int by, int b)
{
    __shared__ T As[16][17];
    __shared__ T Bs[16][17];
    const long m0 = (long)by * 16, n0 = (long)bx * 16;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const T *A = g.A + (long)b * g.a_b;
    const T *B = g.B + (long)b * g.b_b;
    T acc = T(0);
    for (int k0 = 0; k0 < g.K; k0 += 16) {
        {
            const long m = m0 + ty;
            const int k = k0 + tx;
            As[ty][tx] = (m < g.M && k < g.K) ? A[m * g.a_m + (long)k * g.a_k] : T(0);
            const int kb = k0 + ty;
            const long n = n0 + tx;
            Bs[ty][tx] = (kb < g.K && n < g.N) ? B[(long)kb * g.b_k + n * g.b_n] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc += As[ty][kk] * Bs[kk][tx];
        __syncthreads();
    }
    const long m = m0 + ty, n = n0 + tx;
    if (m >= g.M || n >= g.N) return;
    gemm_epilogue(e, b, m, n, acc);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm16(GemmArgs<T> g, EpiArgs<T> e)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    gemm16_body(g, e, blockIdx.x, blockIdx.y, blockIdx.z);
}

// FP64 reductions with few outputs and a long K (a small layer's weight gradient, whose K
// is the data rows): one warp per output, its lanes taking every 32nd k with two
// accumulators, then a fixed butterfly, so the result is reproducible.  On 16 x 16 tiles
// such a GEMM gets a handful of CTAs, each thread walking all of K, while most of GB300's
// FP64 units (a few per SM) stay idle.
// With rsum set, each row m also gets an extra output n = N whose B column is all ones,
// rsum[b rsum_b + m] = sum_k A(m, k) (a layer's bias gradient beside its weight gradient).
template <typename T>
__device__ __forceinline__ void gemm_dot_body(const GemmArgs<T> &g, const EpiArgs<T> &e, T *rsum, long rsum_b, int bx,
                                              int b)
{
    const int lane = threadIdx.x % 32;
    const int nc = g.N + (rsum ? 1 : 0);   // outputs per row
    const long o = (long)bx * 8 + threadIdx.x / 32;
    if (o >= (long)g.M * nc) return;   // the warp leaves together
    const long m = o / nc, n = o % nc;
    const bool ones = n == g.N;
    const T *A = g.A + (long)b * g.a_b + m * g.a_m;
    const T *B = g.B + (long)b * g.b_b + (ones ? 0 : n * g.b_n);
    auto bv = [&](int k) { return ones ? T(1) : B[(long)k * g.b_k]; };
    T acc0 = T(0), acc1 = T(0);
    int k = lane;
    for (; k + 32 < g.K; k += 64) {
        acc0 += A[(long)k * g.a_k] * bv(k);
        acc1 += A[(long)(k + 32) * g.a_k] * bv(k + 32);
    }
    if (k < g.K) acc0 += A[(long)k * g.a_k] * bv(k);
    T acc = acc0 + acc1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane != 0) return;
    if (ones) rsum[(long)b * rsum_b + m] = acc;
    else gemm_epilogue(e, b, m, n, acc);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_dot(GemmArgs<T> g, EpiArgs<T> e, T *rsum, long rsum_b)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    gemm_dot_body(g, e, rsum, rsum_b, blockIdx.x, blockIdx.y);
}

// A weight gradient one warp per output (g1, e1, rsum) and the next delta GEMM on 16 x 16
// tiles (g2, e2), which read the same delta and write different arrays, in one launch:
// blocks [0, nb1) take the former, the others the latter's tiles, nx2 of them across.
template <typename T>
__global__ void __launch_bounds__(256) k_wgrad_and_gemm16(GemmArgs<T> g1, EpiArgs<T> e1, T *rsum, long rsum_b, int nb1,
                                                          GemmArgs<T> g2, EpiArgs<T> e2, int nx2)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    const int x = blockIdx.x;
    if (x < nb1) gemm_dot_body(g1, e1, rsum, rsum_b, x, blockIdx.y);
    else gemm16_body(g2, e2, (x - nb1) % nx2, (x - nb1) / nx2, blockIdx.y);
}

// FP32: C[b](m, n) = sum_k A[b](m, k) B[b](k, n) on 128 x 128 tiles, 16-deep K stages
// double-buffered through shared memory, 8 x 8 outputs per thread (two 4-row and two
// 4-column groups 64 apart, read as float4).  With splits > 1, blockIdx.z covers
// (batch, split) and each CTA sums its own K range [sp kchunk, (sp + 1) kchunk) into the
// raw partial ws[sp][b][m][n]; k_splitk_reduce then adds the splits in order and applies
// the epilogue, so the result is the same for any batch size.
constexpr int GB_M = 128, GB_N = 128, GB_K = 16, GB_PAD = 4;


__global__ void __launch_bounds__(256) k_gemm_f32(GemmArgs<float> g, EpiArgs<float> e, float *ws, int splits,
                                                   int kchunk)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    __shared__ __align__(16) float As[2][GB_K][GB_M + GB_PAD];
    __shared__ __align__(16) float Bs[2][GB_K][GB_N + GB_PAD];
    const int b = blockIdx.z / splits, sp = blockIdx.z % splits;
    const long m0 = (long)blockIdx.y * GB_M, n0 = (long)blockIdx.x * GB_N;
    const int kbeg = sp * kchunk, kend = min(g.K, kbeg + kchunk);
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const float *A = g.A + (long)b * g.a_b;
    const float *B = g.B + (long)b * g.b_b;
    // element r of this thread's share of a stage: (k, m) of A and (k, n) of B, laid out so
    // that a warp's loads run along the operand's contiguous dimension
    const bool a_kc = g.a_k == 1, b_nc = g.b_n == 1;
    float ra[8], rb[8];
    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int el = tid + 256 * r;
            const int kk = a_kc ? (el & 15) : (el >> 7), mm = a_kc ? (el >> 4) : (el & 127);
            const long gm = m0 + mm;
            const int gk = k0 + kk;
            ra[r] = (gm < g.M && gk < kend) ? A[gm * g.a_m + (long)gk * g.a_k] : 0.0f;
            const int kb = b_nc ? (el >> 7) : (el & 15), nn = b_nc ? (el & 127) : (el >> 4);
            const long gn = n0 + nn;
            const int gkb = k0 + kb;
            rb[r] = (gn < g.N && gkb < kend) ? B[(long)gkb * g.b_k + gn * g.b_n] : 0.0f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int el = tid + 256 * r;
            As[buf][a_kc ? (el & 15) : (el >> 7)][a_kc ? (el >> 4) : (el & 127)] = ra[r];
            Bs[buf][b_nc ? (el >> 7) : (el & 15)][b_nc ? (el & 127) : (el >> 4)] = rb[r];
        }
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    int buf = 0;
    if (kbeg < kend) {
        load(kbeg);
        store(0);
    }
    __syncthreads();
    for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
        const bool more = k0 + GB_K < kend;
        if (more) load(k0 + GB_K);   // the next stage's loads are in flight during the FMAs
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const long n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
            if (n >= g.N) continue;
            if (splits > 1) ws[(((long)sp * (gridDim.z / splits) + b) * g.M + m) * g.N + n] = acc[i][j];
            else gemm_epilogue(e, b, m, n, acc[i][j]);
        }
    }
}

// Sum the split-K partials in split order and apply the epilogue.
__global__ void __launch_bounds__(256) k_splitk_reduce(const float *ws, int splits, int batch, int M, int N,
                                                        EpiArgs<float> e)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    const long per = (long)M * N, tot = per * batch;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long)gridDim.x * blockDim.x) {
        float v = 0.0f;
        for (int sp = 0; sp < splits; ++sp) v += ws[(long)sp * tot + i];
        const int b = (int)(i / per);
        const long r = i % per;
        gemm_epilogue(e, b, r / N, r % N, v);
    }
}

// K-splits of an FP32 GEMM: a reduction over many rows (the weight gradients, K = data
// rows) on few output tiles gets K ranges of about 512 (at most 64 of them), enough CTAs
// to fill the GPU; the count depends on the shape only, never on the batch.
inline int gemm_splits(int M, int N, int K)
{
    const long tiles = (long)((M + GB_M - 1) / GB_M) * ((N + GB_N - 1) / GB_N);
    if (K < 2048 || tiles >= 64) return 1;
    return (int)std::min<long>(64, (K + 511) / 512);
}

inline size_t gemm_ws_floats(int M, int N, int K, int batch)
{
    const int sp = gemm_splits(M, N, K);
    return sp > 1 ? (size_t)sp * batch * M * N : 0;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    if (l == 0) sm[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NT / 32; ++i) r += sm[i];
    __syncthreads();
    return r;   // valid in thread 0
}

// out[b][col] = sum over rows of d[b][row][col] (FP64 accumulation, fixed order).
template <typename T>
__global__ void k_colsum(const T *d, long rows, int cols, long d_b, T *out, long out_b)
{
    pdl_wait();   // under launch_pdl: the kernel before it has finished (else a no-op)
    pdl_trigger();
    __shared__ double sm[8][33];
    const int b = blockIdx.y;
    const int col = blockIdx.x * 32 + threadIdx.x;
    double s = 0.0;
    if (col < cols)
        for (long r = threadIdx.y; r < rows; r += 8) s += (double)d[(long)b * d_b + r * cols + col];
    sm[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && col < cols) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += sm[i][threadIdx.x];
        out[(long)b * out_b + col] = (T)t;
    }
}

// ws / ws_floats: split-K workspace (FP32 only; without one, or when it is too small, the
// GEMM runs unsplit).
template <typename T>
void launch_gemm(const GemmArgs<T> &g, const EpiArgs<T> &e, int batch, cudaStream_t s, float *ws = nullptr,
                 size_t ws_floats = 0)
{
    if (g.M <= 0 || g.N <= 0) return;
    if constexpr (sizeof(T) == 4) {
        int splits = gemm_splits(g.M, g.N, g.K);
        if (!ws || ws_floats < gemm_ws_floats(g.M, g.N, g.K, batch)) splits = 1;
        // K range of one split: K / splits rounded up to whole 16-deep stages
        const int kchunk = splits > 1 ? ((g.K + splits - 1) / splits + GB_K - 1) / GB_K * GB_K : std::max(g.K, 1);
        dim3 grid((g.N + GB_N - 1) / GB_N, (g.M + GB_M - 1) / GB_M, batch * splits);
        ProfScope ps("simt_gemm_f32", s);
        launch_pdl(k_gemm_f32, grid, dim3(256), 0, s, g, e, ws, splits, kchunk);
        HMC_LAUNCH_CK();
        if (splits > 1) {
            const long tot = (long)batch * g.M * g.N;
            launch_pdl(k_splitk_reduce, dim3((unsigned)std::min<long>((tot + 255) / 256, 4096)), dim3(256), 0, s,
                       (const float *)ws, splits, batch, g.M, g.N, e);
            HMC_LAUNCH_CK();
        }
    } else {
        dim3 grid((g.N + 15) / 16, (g.M + 15) / 16, batch);
        ProfScope ps("simt_gemm_f64", s);
        launch_pdl(k_gemm16<T>, grid, dim3(256), 0, s, g, e);
        HMC_LAUNCH_CK();
    }
}

// A weight gradient dW = delta^T A (K = the data rows): FP64 ones with few outputs and a
// long K take one warp per output (k_gemm_dot), and then also form the row sums of delta
// (the bias gradient) into rsum when it is set, returning true; everything else is
// launch_gemm's, and the caller sums the bias gradient itself (false).
template <typename T> bool wgrad_by_warps(const GemmArgs<T> &g)
{
    return sizeof(T) == 8 && g.M > 0 && g.N > 0 && g.K >= 128 && (long)g.M * g.N <= 1024;
}

template <typename T>
bool launch_wgrad(const GemmArgs<T> &g, const EpiArgs<T> &e, int batch, cudaStream_t s, float *ws, size_t ws_floats,
                  T *rsum = nullptr, long rsum_b = 0)
{
    if constexpr (sizeof(T) == 8) {
        if (wgrad_by_warps(g)) {
            dim3 grid((unsigned)(((long)g.M * (g.N + (rsum ? 1 : 0)) + 7) / 8), batch);
            ProfScope ps("simt_wgrad_f64", s);
            launch_pdl(k_gemm_dot<T>, grid, dim3(256), 0, s, g, e, rsum, rsum_b);
            HMC_LAUNCH_CK();
            return true;
        }
    }
    launch_gemm(g, e, batch, s, ws, ws_floats);
    return false;
}

// The weight gradient (g1, e1, rsum as for launch_wgrad) and the next delta GEMM (g2, e2)
// in one launch where both are FP64 and the first goes one warp per output; returns false
// (nothing launched) otherwise.
template <typename T>
bool launch_wgrad_and_delta(const GemmArgs<T> &g1, const EpiArgs<T> &e1, T *rsum, long rsum_b, const GemmArgs<T> &g2,
                            const EpiArgs<T> &e2, int batch, cudaStream_t s)
{
    if constexpr (sizeof(T) == 8) {
        if (wgrad_by_warps(g1) && g2.M > 0 && g2.N > 0) {
            const int nb1 = (int)(((long)g1.M * (g1.N + (rsum ? 1 : 0)) + 7) / 8);
            const int nx2 = (g2.N + 15) / 16, ny2 = (g2.M + 15) / 16;
            ProfScope ps("simt_wgrad_delta_f64", s);
            launch_pdl(k_wgrad_and_gemm16<T>, dim3((unsigned)(nb1 + nx2 * ny2), batch), dim3(256), 0, s, g1, e1, rsum,
                       rsum_b, nb1, g2, e2, nx2);
            return true;
        }
    }
    return false;
}

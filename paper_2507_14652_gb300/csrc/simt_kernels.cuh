// simt_kernels.cuh -- CUDA-core building blocks shared by the FP64/FP32 engine and the
// sensitivity pass: a batched 64x64-tile GEMM with fused epilogues, a fixed-order
// FP64 block sum and FP64 column sums.  Include it inside an anonymous namespace of
// namespace hmc (every translation unit keeps its own copies).
#pragma once

constexpr int TILE = 64;
constexpr int TK = 16;

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

// C[b](m, n) = sum_k A[b](m, k) B[b](k, n), 64x64 tile, 16-deep K steps, 4x4 per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs<T> g, EpiArgs<T> e)
{
    __shared__ T As[TK][TILE + 1];
    __shared__ T Bs[TK][TILE + 1];
    const int b = blockIdx.z;
    const long m0 = (long)blockIdx.y * TILE, n0 = (long)blockIdx.x * TILE;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const T *A = g.A + (long)b * g.a_b;
    const T *B = g.B + (long)b * g.b_b;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < g.K; k0 += TK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int el = tid + 256 * r;
            int mm, kk;
            if (g.a_k == 1) { kk = el % TK; mm = el / TK; } else { mm = el % TILE; kk = el / TILE; }
            long gm = m0 + mm; int gk = k0 + kk;
            As[kk][mm] = (gm < g.M && gk < g.K) ? A[gm * g.a_m + (long)gk * g.a_k] : T(0);
            int nn;
            if (g.b_n == 1) { nn = el % TILE; kk = el / TILE; } else { kk = el % TK; nn = el / TK; }
            long gn = n0 + nn; gk = k0 + kk;
            Bs[kk][nn] = (gn < g.N && gk < g.K) ? B[(long)gk * g.b_k + gn * g.b_n] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        long m = m0 + ty + 16 * i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            long n = n0 + tx + 16 * j;
            if (n >= g.N) continue;
            long o = (long)b * e.o_b + m * e.o_m + n * e.o_n;
            if (e.mode == EPI_ACT) {
                T z = acc[i][j] + (e.bias ? e.bias[(long)b * e.bias_b + n * e.bias_n] : T(0));
                T a, s;
                act_eval(e.act, z, a, s);
                e.out[o] = a;
                if (e.slope) e.slope[o] = s;
            } else if (e.mode == EPI_SCALE) {
                const long so = (long)b * (e.slope_b < 0 ? e.o_b : e.slope_b) + m * e.o_m + n * e.o_n;
                e.out[o] = acc[i][j] * e.slope[so];
            } else {
                e.out[o] = acc[i][j];
            }
        }
    }
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

template <typename T>
void launch_gemm(const GemmArgs<T> &g, const EpiArgs<T> &e, int batch, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0) return;
    dim3 grid((g.N + TILE - 1) / TILE, (g.M + TILE - 1) / TILE, batch);
    ProfScope ps(sizeof(T) == 8 ? "simt_gemm_f64" : "simt_gemm_f32", s);
    k_gemm<T><<<grid, 256, 0, s>>>(g, e);
    HMC_LAUNCH_CK();
}

// k_umma.cu -- tcgen05 tensor-core engine for U and grad U (BF16 operands,
// FP32 accumulation in TMEM, FP64 energy sums).
//
// Network pattern: MLP  dx -> w -> ... -> w -> 1, tanh hidden layers, identity
// output, biases everywhere, hidden width w up to 256 (padded to 128 or 256).
//
// One gradient evaluation for all C chains (rows n = data points, tiles of 128):
//   first layer   A_1 = tanh(X W_0^T + b_0)                        CUDA cores
//   hidden fwd    A_{i+1} = tanh(A_i W_i^T + b_i)                  UMMA, epilogue tanh
//                 Hidden weights are held as a bf16 pair W = W_hi + W_lo (about 16
//                 mantissa bits) and every K-slice issues two MMAs into the same
//                 accumulator, so only activations and deltas are rounded to bf16.
//   last hidden   A_{L-1} = tanh(A_{L-2} W^T + b) fused with the output layer:
//                 f = A_{L-1} w_out + b_out, r = f - y, U partial (FP64),
//                 delta_L = r / sigma^2, dW_out/db_out partials,
//                 delta_{L-1} = delta_L w_out (1 - A_{L-1}^2)   (A_{L-1} never stored)
//   hidden bwd    delta_i = (delta_{i+1} W_i) (1 - A_i^2)          UMMA, W_i read MN-major
//   first bwd     delta_1 as above, fused with dW_0 = delta_1^T X and db_0 (never stored)
//   weight grads  dW_i = delta_{i+1}^T A_i                          UMMA, both operands MN-major,
//                 split over rows, only the sampled entries leave the chip
//   finalize      U, g = sum of partials in fixed order + q / alpha^2
// Every partial sum is written to its own slot (no atomics), so the result is
// bit-reproducible.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>

#include "hmc_diag.h"
#include "hmc_internal.cuh"
#include "umma.cuh"

// The 16-bit operand type of the tensor-core GEMMs is chosen at compile time: this
// file builds the bf16 engines, and k_umma_f16.cu includes it with HMC_F16 = 1 for the
// fp16 ones (same kernels, same bytes and tensor rate; 11 significant bits against 8).
#ifndef HMC_F16
#define HMC_F16 0
#endif

namespace hmc {
namespace {

using namespace umma;

#if HMC_F16
using h16 = __half;
constexpr int H16_KIND = 2;                      // ScatterPlan::kind16 of the hidden weights
#define TM_H16 CU_TENSOR_MAP_DATA_TYPE_FLOAT16
__host__ __device__ inline h16 f_to_h16(float v) { return __float2half_rn(v); }
__host__ __device__ inline float h16_to_f(h16 v) { return __half2float(v); }
__device__ __forceinline__ uint32_t pack_h16(float a, float b) { return pack_f16(a, b); }
__device__ __forceinline__ float2 unpack_h16(uint32_t u) { return unpack_f16(u); }
__device__ __forceinline__ void mma_m16n8k16_h16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    mma_m16n8k16_f16(d, a, b0, b1);
}
__host__ __device__ constexpr uint32_t idesc_h16(int M, int N, bool a_mn, bool b_mn)
{
    return idesc_f16(M, N, a_mn, b_mn);
}
// fp16 keeps 11 significant bits, so the activations get a tanh accurate to 1e-6
__device__ __forceinline__ float act_tanh(float x) { return tanh_acc(x); }
#else
using h16 = __nv_bfloat16;
constexpr int H16_KIND = 1;
#define TM_H16 CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
__host__ __device__ inline h16 f_to_h16(float v) { return __float2bfloat16_rn(v); }
__host__ __device__ inline float h16_to_f(h16 v) { return __bfloat162float(v); }
__device__ __forceinline__ uint32_t pack_h16(float a, float b) { return pack_bf16(a, b); }
__device__ __forceinline__ float2 unpack_h16(uint32_t u) { return unpack_bf16(u); }
__device__ __forceinline__ void mma_m16n8k16_h16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    mma_m16n8k16_bf16(d, a, b0, b1);
}
__host__ __device__ constexpr uint32_t idesc_h16(int M, int N, bool a_mn, bool b_mn)
{
    return idesc_bf16(M, N, a_mn, b_mn);
}
__device__ __forceinline__ float act_tanh(float x) { return tanh_fast(x); }
#endif

// Output deltas are formed as r * dscale and every data-term gradient sum is scaled by
// gscale = (1 / sigma^2) / dscale at the end.  bf16 shares fp32's exponent range, so it
// takes dscale = 1 / sigma^2 (gscale = 1); fp16 overflows at 65504, so it takes the power
// of two nearest 1 / sigma, which keeps the deltas near the size of r / sigma.
inline double delta_scale(double sigma)
{
    return HMC_F16 ? std::ldexp(1.0, (int)std::lround(std::log2(1.0 / sigma))) : 1.0 / (sigma * sigma);
}

constexpr int BM = 128;                         // rows per tile (UMMA M)
constexpr int BK = 64;                          // K per stage (one 128-byte swizzle atom of bf16)
constexpr int STAGES = 2;
constexpr int A_STAGE_BYTES = BM * BK * 2;      // 16 KB
constexpr int B_STAGE_BYTES = 256 * BK * 2;     // 32 KB (room for N up to 256); doubled for W_hi + W_lo
constexpr int TMEM_COLS = 256;
constexpr int NTHREADS = 192;                   // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int RED_BYTES = 3 * 4 * 256 * 4 + 4 * 8 + 4 * 4 + 64;   // [3][4][256] floats, 4 doubles, 4 floats
__host__ __device__ constexpr int stage_bytes(bool wsplit) { return A_STAGE_BYTES + B_STAGE_BYTES * (wsplit ? 2 : 1); }
__host__ __device__ constexpr int smem_bytes(bool wsplit) { return 1024 + STAGES * stage_bytes(wsplit) + 256 + RED_BYTES; }

enum Mode {
    M_STORE_F32 = 0,   // out_f32 = A B^T
    M_FWD_TANH = 1,    // out = bf16(tanh(A W^T + b))
    M_FWD_OUT = 2,     // last hidden layer + scalar output layer + residual
    M_BWD_TANH = 3,    // out = bf16((A B^T) (1 - aux^2)), column sums
    M_BWD_FIRST = 4,   // as M_BWD_TANH, fused with the first layer's weight and bias sums
    M_DW = 5,          // sampled entries of A^T B
    M_FWD_LIN = 6,     // out = bf16(A W^T + b), no activation (a linear last layer)
    M_S = 7,           // operator output S = B T^T on 128 x N tiles: residual, energy, dS
    M_GEMM_BF16 = 8    // out = bf16(A B^T), column sums
};

struct Params {
    int M, N, K;           // per-batch GEMM: out[M][N] = sum_k A(m,k) B(n,k)
    int kb_per_split;      // k-blocks handled by one CTA (grid.y splits the K range)
    int ntiles;            // ceil(rows / 128) for the per-tile partial arrays
    int *err;
    // outputs / epilogue operands
    float *out_f32;                       // M_STORE_F32: [b][M][N]
    h16 *out; long out_b;       // bf16 [b][M][N]
    const float *bias; long bias_b;       // [b][N]
    const h16 *aux; long aux_b; // A_i for the tanh slope [b][M][N]
    const float *wout; long wout_b;       // output weights [b][N]
    const float *bout;                    // [b]
    const float *y;                       // targets [M]
    float inv_s2;
    float oscale;                         // M_GEMM_BF16: factor on the products (a power of two)
    double *u_part;                       // [b][ntiles]
    float *dbout_part;                    // [b][ntiles]
    float *dwout_part;                    // [b][ntiles][N]
    float *db_part;                       // [b][ntiles][N] column sums of the produced delta;
                                          // k_dw2: [split][b][M] row sums of delta, split stride db_split
    long db_split;
    const float *x; int dx;               // M_BWD_FIRST: inputs [M][dx]
    float *dw0_part;                      // [b][ntiles][N][dx]
    const int *rowptr;                    // M_DW: entries of output row o are [rowptr[o], rowptr[o+1])
    const int *ecol;                      // M_DW: column of entry j inside the layer
    const int *erow;                      // M_DW: row of entry j
    const int *epack;                     // row << 16 | column of entry j (dW gather)
    float *gw_part; long gw_split; long gw_b;   // M_DW: [split][b][k]
    // M_S computes S^T = T B^T: rows are the ny query points, columns the nu input
    // functions; targets Yt [nu][ny] (shared by the chains), dS [b][nu][ldo], per-chain
    // scalar bias b0s [b]; partials per (row tile, column tile)
    const float *Yt; int ny, nu, ldo, ntn;
    const float *b0s;
    float *db0_part;                      // [b][ntiles][ntn]
};

// One CTA of the tile kernel, block (bx, by, bz) of its problem's grid.  G: the tensor
// maps come from a grouped launch's job table in global memory.
template <int MODE, bool A_MN, bool B_MN, bool WSPLIT, bool G>
__device__ __forceinline__ void umma_body(const CUtensorMap &tmA, const CUtensorMap &tmB, const CUtensorMap &tmB2,
                                          const Params &p, int bx, int by, int bz)
{
    constexpr int STAGE_BYTES = stage_bytes(WSPLIT);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 1);
    float *red = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES + 256);   // [3][4][256]
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), accb = smem_u32(bars + 2 * STAGES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // M_S runs on a (chain, row tile, column tile) grid with the chain fastest, so the
    // chains' CTAs for one tile of the shared targets follow each other through L2
    const int m_tile = MODE == M_S ? by : bx;
    const int b = MODE == M_S ? bx : bz;
    const int n_tile = MODE == M_S ? bz : 0;
    const int split = MODE == M_S ? 0 : by;
    const int n0 = n_tile * p.N;
    const int m0 = m_tile * BM;
    const int BN = p.N;
    const int total_kb = (p.K + BK - 1) / BK;
    const int kb0 = split * p.kb_per_split;
    const int nkb = min(p.kb_per_split, total_kb - kb0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        fence_mbar_init();
        if (G) {   // thread 0 is also the TMA producer
            tensormap_acquire(&tmA);
            tensormap_acquire(&tmB);
            if (WSPLIT) tensormap_acquire(&tmB2);
        }
        prefetch_map(&tmA);
        prefetch_map(&tmB);
        if (WSPLIT) prefetch_map(&tmB2);
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            const uint32_t bbytes = (uint32_t)BN * BK * 2;
            int issued = 0;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.err)) { ok = false; break; }
                const uint32_t fb = full0 + 8 * s;
                mbar_expect_tx(fb, A_STAGE_BYTES + bbytes * (WSPLIT ? 2u : 1u));
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES), sb = sa + A_STAGE_BYTES;
                const int kc = (kb0 + i) * BK;
                if (!A_MN) {
                    tma_load_3d(sa, &tmA, kc, m0, b, fb);
                } else {
                    tma_load_3d(sa, &tmA, m0, kc, b, fb);
                    tma_load_3d(sa + 8192, &tmA, m0 + 64, kc, b, fb);
                }
                if (!B_MN) {
                    tma_load_3d(sb, &tmB, kc, n0, b, fb);
                    if (WSPLIT) tma_load_3d(sb + B_STAGE_BYTES, &tmB2, kc, n0, b, fb);
                } else {
                    for (int a = 0; a < BN / 64; ++a) {
                        tma_load_3d(sb + 8192 * a, &tmB, 64 * a, kc, b, fb);
                        if (WSPLIT) tma_load_3d(sb + B_STAGE_BYTES + 8192 * a, &tmB2, 64 * a, kc, b, fb);
                    }
                }
                ++issued;
            }
            if (!ok) {   // let the copies already in flight land before the CTA exits
                for (int i = max(0, issued - STAGES); i < issued; ++i)
                    mbar_wait(full0 + 8 * (i % STAGES), (uint32_t)(i / STAGES) & 1u, p.err, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = idesc_h16(BM, BN, A_MN, B_MN);
            for (int i = 0; i < nkb; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
                if (!mbar_wait(full0 + 8 * s, ph, p.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES), sb = sa + A_STAGE_BYTES;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint64_t ad = A_MN ? sdesc(sa + 2048 * ks, 8192, 1024) : sdesc(sa + 32 * ks, 0, 1024);
                    const uint64_t bd = B_MN ? sdesc(sb + 2048 * ks, 8192, 1024) : sdesc(sb + 32 * ks, 0, 1024);
                    mma_bf16(tmem, ad, bd, idesc, (i > 0 || ks > 0) ? 1u : 0u);
                    if (WSPLIT) {
                        const uint32_t sl = sb + B_STAGE_BYTES;
                        const uint64_t bl = B_MN ? sdesc(sl + 2048 * ks, 8192, 1024) : sdesc(sl + 32 * ks, 0, 1024);
                        mma_bf16(tmem, ad, bl, idesc, 1u);
                    }
                }
                mma_commit(empty0 + 8 * s);
            }
            mma_commit(accb);
        }
    } else {
        // ---------------- epilogue: warps 2..5, one accumulator row per thread ----------------
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        const int row = 32 * q + lane;
        const int m = m0 + row;
        const bool valid = m < p.M;
        const int et = threadIdx.x - 64;      // 0..127
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16);
        ok = mbar_wait(accb, 0, p.err);
        tc_fence_after();
        if (ok) {
            if (MODE == M_STORE_F32) {
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    float v[32];
                    tmem_ld32(taddr + c0, v);
                    if (valid) {
                        float4 *o = reinterpret_cast<float4 *>(p.out_f32 + ((long)b * p.M + m) * p.N + c0);
#pragma unroll
                        for (int j = 0; j < 8; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    }
                }
            } else if (MODE == M_FWD_TANH) {
                const float *bias = p.bias + (long)b * p.bias_b;
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    float v[32];
                    tmem_ld32(taddr + c0, v);
                    if (valid) {
                        uint32_t pk[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            pk[j] = pack_h16(act_tanh(v[2 * j] + bias[c0 + 2 * j]),
                                              act_tanh(v[2 * j + 1] + bias[c0 + 2 * j + 1]));
                        uint4 *o = reinterpret_cast<uint4 *>(p.out + (long)b * p.out_b + (long)m * p.N + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) o[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                    }
                }
            } else if (MODE == M_FWD_LIN) {
                const float *bias = p.bias + (long)b * p.bias_b;
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    float v[32];
                    tmem_ld32(taddr + c0, v);
                    if (valid) {
                        uint32_t pk[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            pk[j] = pack_h16(v[2 * j] + bias[c0 + 2 * j], v[2 * j + 1] + bias[c0 + 2 * j + 1]);
                        uint4 *o = reinterpret_cast<uint4 *>(p.out + (long)b * p.out_b + (long)m * p.N + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) o[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                    }
                }
            } else if (MODE == M_S) {
                // lane = query point y, columns = input functions u: r = S + b0 - Y[u][y] and
                // dS[u][y] = r / sigma^2 in bf16; per load and store a warp covers 32
                // consecutive y of one u.  Squares summed in FP32 per chunk, carried in FP64.
                const float b0 = p.b0s[b];
                h16 *ob = p.out + (long)b * p.out_b + m;
                const float *yb = p.Yt + m;
                double r2 = 0.0;
                float dsum = 0.0f;
                const long ny = p.ny, ldo = p.ldo;
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    float v[32];
                    tmem_ld32(taddr + c0, v);
                    const int u0 = n0 + c0;
                    if (valid && u0 + 32 <= p.nu) {   // a whole chunk: no per-column bounds
                        const float *yp = yb + (long)u0 * ny;
                        h16 *op = ob + (long)u0 * ldo;
                        float yv[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) yv[j] = __ldg(yp + j * ny);
                        float r2c = 0.0f;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float r = (v[j] + b0) - yv[j];
                            r2c += r * r;
                            const float ds = r * p.inv_s2;
                            dsum += ds;
                            op[j * ldo] = f_to_h16(ds);
                        }
                        r2 += (double)r2c;
                    } else if (valid && u0 < p.nu) {
                        float yv[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) yv[j] = u0 + j < p.nu ? __ldg(yb + (long)(u0 + j) * ny) : 0.0f;
                        float r2c = 0.0f;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (u0 + j < p.nu) {
                                const float r = (v[j] + b0) - yv[j];
                                r2c += r * r;
                                const float ds = r * p.inv_s2;
                                dsum += ds;
                                ob[(long)(u0 + j) * ldo] = f_to_h16(ds);
                            }
                        }
                        r2 += (double)r2c;
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
                    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                }
                double *rd = reinterpret_cast<double *>(red + 3 * 4 * 256);
                float *dsm = red + 3 * 4 * 256 + 8;
                if (lane == 0) {
                    rd[q] = r2;
                    dsm[q] = dsum;
                }
                named_bar_sync(1, 128);
                if (et == 0) {
                    const long o = ((long)b * p.ntiles + m_tile) * p.ntn + n_tile;
                    p.u_part[o] = rd[0] + rd[1] + rd[2] + rd[3];
                    p.db0_part[o] = dsm[0] + dsm[1] + dsm[2] + dsm[3];
                }
            } else if (MODE == M_GEMM_BF16) {
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    float v[32];
                    tmem_ld32(taddr + c0, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = valid ? v[j] * p.oscale : 0.0f;   // exact: a power of two
                    if (valid) {
                        uint32_t pk[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) pk[j] = pack_h16(v[2 * j], v[2 * j + 1]);
                        uint4 *o = reinterpret_cast<uint4 *>(p.out + (long)b * p.out_b + (long)m * p.N + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) o[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                    }
                    red[(1 * 4 + q) * 256 + c0 + lane] = reduce_scatter32(v);
                }
                named_bar_sync(1, 128);
                for (int c = et; c < BN; c += 128) {
                    const long o = ((long)b * p.ntiles + m_tile) * p.N + c;
                    p.db_part[o] = red[(1 * 4 + 0) * 256 + c] + red[(1 * 4 + 1) * 256 + c] +
                                   red[(1 * 4 + 2) * 256 + c] + red[(1 * 4 + 3) * 256 + c];
                }
            } else if (MODE == M_FWD_OUT) {
                const float *bias = p.bias + (long)b * p.bias_b;
                const float *wo = p.wout + (long)b * p.wout_b;
                float f = p.bout[b];
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    float v[32];
                    tmem_ld32(taddr + c0, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) f += act_tanh(v[j] + bias[c0 + j]) * wo[c0 + j];
                }
                const float r = valid ? f - p.y[m] : 0.0f;
                const float d = r * p.inv_s2;   // delta of the output
                double r2 = (double)r * (double)r;
                float dsum = d;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
                    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                }
                double *rd = reinterpret_cast<double *>(red + 3 * 4 * 256);   // 4 doubles after the float arrays
                float *dsm = red + 3 * 4 * 256 + 8;                           // 4 floats after the doubles
                if (lane == 0) {
                    rd[q] = r2;
                    dsm[q] = dsum;
                }
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    float v[32], dw[32], dd[32];
                    tmem_ld32(taddr + c0, v);
                    uint32_t pk[16];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float a = act_tanh(v[j] + bias[c0 + j]);
                        dw[j] = d * a;
                        dd[j] = d * wo[c0 + j] * (1.0f - a * a);
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) pk[j] = pack_h16(dd[2 * j], dd[2 * j + 1]);
                    if (valid) {
                        uint4 *o = reinterpret_cast<uint4 *>(p.out + (long)b * p.out_b + (long)m * p.N + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) o[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                    }
                    red[(0 * 4 + q) * 256 + c0 + lane] = reduce_scatter32(dw);
                    red[(1 * 4 + q) * 256 + c0 + lane] = reduce_scatter32(dd);
                }
                named_bar_sync(1, 128);
                for (int c = et; c < BN; c += 128) {
                    const long o = ((long)b * p.ntiles + m_tile) * p.N + c;
                    p.dwout_part[o] = red[(0 * 4 + 0) * 256 + c] + red[(0 * 4 + 1) * 256 + c] +
                                      red[(0 * 4 + 2) * 256 + c] + red[(0 * 4 + 3) * 256 + c];
                    p.db_part[o] = red[(1 * 4 + 0) * 256 + c] + red[(1 * 4 + 1) * 256 + c] +
                                   red[(1 * 4 + 2) * 256 + c] + red[(1 * 4 + 3) * 256 + c];
                }
                if (et == 0) {
                    p.u_part[(long)b * p.ntiles + m_tile] = rd[0] + rd[1] + rd[2] + rd[3];
                    p.dbout_part[(long)b * p.ntiles + m_tile] = dsm[0] + dsm[1] + dsm[2] + dsm[3];
                }
            } else if (MODE == M_BWD_TANH || MODE == M_BWD_FIRST) {
                const h16 *aux = p.aux + (long)b * p.aux_b + (long)(valid ? m : 0) * p.N;
                float xv[8];
#pragma unroll
                for (int d = 0; d < 8; ++d) xv[d] = (MODE == M_BWD_FIRST && valid && d < p.dx) ? p.x[(long)m * p.dx + d] : 0.0f;
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    float v[32], dd[32];
                    tmem_ld32(taddr + c0, v);
                    if (valid) {
                        const uint4 *ap = reinterpret_cast<const uint4 *>(aux + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint4 u = ap[j];
                            const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const float2 a = unpack_h16(w4[t]);
                                dd[8 * j + 2 * t] = v[8 * j + 2 * t] * (1.0f - a.x * a.x);
                                dd[8 * j + 2 * t + 1] = v[8 * j + 2 * t + 1] * (1.0f - a.y * a.y);
                            }
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) dd[j] = 0.0f;
                    }
                    if (MODE == M_BWD_TANH && valid) {
                        uint32_t pk[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) pk[j] = pack_h16(dd[2 * j], dd[2 * j + 1]);
                        uint4 *o = reinterpret_cast<uint4 *>(p.out + (long)b * p.out_b + (long)m * p.N + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) o[j] = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                    }
                    if (MODE == M_BWD_FIRST) {
                        for (int d = 0; d < p.dx; ++d) {
                            float t[32];
#pragma unroll
                            for (int j = 0; j < 32; ++j) t[j] = dd[j] * xv[d];
                            const float cs = reduce_scatter32(t);
                            // per-warp column sums of delta_1 * x_d go to dw0_part via the reduction buffer below
                            red[(2 * 4 + q) * 256 + c0 + lane] = cs;
                            named_bar_sync(1, 128);
                            if (et < 32) {
                                const int c = c0 + et;
                                const float s = red[(2 * 4 + 0) * 256 + c] + red[(2 * 4 + 1) * 256 + c] +
                                                red[(2 * 4 + 2) * 256 + c] + red[(2 * 4 + 3) * 256 + c];
                                p.dw0_part[(((long)b * p.ntiles + m_tile) * p.N + c) * p.dx + d] = s;
                            }
                            named_bar_sync(1, 128);
                        }
                    }
                    red[(1 * 4 + q) * 256 + c0 + lane] = reduce_scatter32(dd);
                }
                named_bar_sync(1, 128);
                for (int c = et; c < BN; c += 128) {
                    const long o = ((long)b * p.ntiles + m_tile) * p.N + c;
                    p.db_part[o] = red[(1 * 4 + 0) * 256 + c] + red[(1 * 4 + 1) * 256 + c] +
                                   red[(1 * 4 + 2) * 256 + c] + red[(1 * 4 + 3) * 256 + c];
                }
            } else if (MODE == M_DW) {
                // stage the fp32 tile in the (now idle) operand buffers, half of the columns at a time
                float *stg = reinterpret_cast<float *>(smem);
                const int r_end = min(m0 + BM, p.M);
                const int j0 = p.rowptr[m0], j1 = p.rowptr[r_end];
                for (int h0 = 0; h0 < BN; h0 += 128) {
                    const int hc = min(128, BN - h0);
                    for (int c0 = 0; c0 < hc; c0 += 32) {
                        float v[32];
                        tmem_ld32(taddr + h0 + c0, v);
#pragma unroll
                        for (int j = 0; j < 32; ++j) stg[row * 129 + c0 + j] = v[j];
                    }
                    named_bar_sync(1, 128);
                    for (int j = j0 + et; j < j1; j += 128) {
                        const int c = p.ecol[j] - h0;
                        if (c >= 0 && c < hc)
                            p.gw_part[(long)split * p.gw_split + (long)b * p.gw_b + j] = stg[(p.erow[j] - m0) * 129 + c];
                    }
                    named_bar_sync(1, 128);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

template <int MODE, bool A_MN, bool B_MN, bool WSPLIT>
__global__ void __launch_bounds__(NTHREADS, WSPLIT ? 1 : 2)
    k_umma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           const __grid_constant__ CUtensorMap tmB2, const __grid_constant__ Params p)
{
    umma_body<MODE, A_MN, B_MN, WSPLIT, false>(tmA, tmB, tmB2, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Grouped launches.  Several problems' launches of the same kernel become one launch
// over a linear grid: job j owns blocks [bstart, bstart + gx gy gz), and each of them
// runs the problem's own kernel body with the block index (x, y, z) it would have had
// in a launch of its own, so every problem's arithmetic, and its result bit for bit,
// is the same as in separate launches.  The job tables live in device memory, written
// once when the group is built.
// ---------------------------------------------------------------------------
struct GridJob {   // aligned as CUtensorMap requires
    CUtensorMap tm[3];
    Params p;
    int bstart, gx, gy, gz;
};

// the job whose block range holds block b (the jobs' ranges are ascending and adjacent)
template <typename J> __device__ __forceinline__ int find_job(const J *__restrict__ jobs, int njobs, long b)
{
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long)jobs[mid].bstart <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int MODE, bool A_MN, bool B_MN, bool WSPLIT>
__global__ void __launch_bounds__(NTHREADS, WSPLIT ? 1 : 2) k_umma_g(const GridJob *__restrict__ jobs, int njobs)
{
    const GridJob &J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int lb = (int)blockIdx.x - J.bstart;
    umma_body<MODE, A_MN, B_MN, WSPLIT, true>(J.tm[0], J.tm[1], J.tm[2], J.p, lb % J.gx, (lb / J.gx) % J.gy,
                                              lb / (J.gx * J.gy));
}

// ---------------------------------------------------------------------------
// Persistent layer kernel for the w x w hidden layers (w = 128 or 256).
//
// A cluster of two CTAs acts as one M = 256 tensor-core unit (tcgen05
// .cta_group::2).  Each CTA streams its own 128-row tile of the A operand
// (activations or deltas) through a 4-stage ring of 16 KB K-blocks and keeps half
// of W (its w/2 rows of the B operand, bf16 hi and lo, all K) resident while the
// chain does not change; the even CTA issues every MMA and both receive whole
// 128 x w rows of the product in their own tensor memory.  Loads of either CTA
// complete on the even CTA's barriers; MMA completions are multicast to both.
// Two TMEM accumulators alternate so the epilogue of one tile runs while the MMAs
// of the next one are in flight.
//
// Epilogue: each warp owns 32 rows (its TMEM lane quadrant) and half of the
// columns.  Row-per-thread values pass through a 2 KB swizzled staging buffer per
// warp, so global loads and stores move 8 rows x 64 contiguous bytes per
// instruction instead of 32 scattered 16-byte pieces.
// ---------------------------------------------------------------------------
enum LMode { L_FWD_TANH = 0, L_FWD_OUT = 1, L_BWD_TANH = 2, L_BWD_FIRST = 3, L_FWD_LIN = 4 };
constexpr int L_STAGES = 4;
constexpr int L_A_BYTES = BM * BK * 2;                  // one 16 KB K-block of a 128-row tile
constexpr int L_W_HALF = 64 * 1024;                     // resident half of W, hi or lo (4 K-blocks x 16 KB)
constexpr int L_STG = 2048;                             // staging bytes per epilogue warp (32 rows x 64 B)
constexpr int L_SCR_FLOATS = 4 * 256 + 8 * L_STG / 4;       // forward: [4][w] column sums + staging;
                                                             // reverse: staging, or [1 + dx][4][w] sums (dx <= 4 at w = 256)
constexpr int L_AUX = 4 * L_STG;                        // reverse: a warp's 32 x 128 slopes of a tile, in the free lo region
constexpr int L_SMEM = 1024 + 2 * L_W_HALF + L_STAGES * L_A_BYTES + 256 + L_SCR_FLOATS * 4 + 64 + 64 +
                       2 * 256 * 4 + 2 * 128 * 4;        // + bias and output weights of the chain, half-row sums
constexpr int L_THREADS = 320;                          // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
static_assert(8 * L_AUX <= L_W_HALF, "reverse-pass slope buffers fit the lo region");
static_assert(8 * L_STG / 4 + 4 * 256 <= L_SCR_FLOATS, "reverse column sums fit after the staging buffers");
// Reverse pass with the weights as a hi/lo pair (the lo region then holds W): a two-stage
// operand ring, and two of a warp's four slope chunks in flight, in a region of their own
// after the per-chain vectors, within the same L_SMEM.
constexpr int L_STAGES_RLO = 2;
constexpr int L_AUX_RLO = 2 * L_STG;
constexpr int L_AUX_OFF_RLO = 2 * L_W_HALF + L_STAGES_RLO * L_A_BYTES + 256 + L_SCR_FLOATS * 4 + 64 + 64 +
                              2 * 256 * 4 + 2 * 128 * 4;   // from the 1024-aligned base
static_assert(1024 + L_AUX_OFF_RLO + 8 * L_AUX_RLO <= L_SMEM, "reverse hi/lo layout fits the layer kernels' smem");
static_assert(L_AUX_OFF_RLO % 128 == 0, "slope buffers stay 128-byte aligned");

struct LayerParams {
    int N, W, C, ntiles, dx;
    int *err;
    h16 *out;            // [c][N][W]
    const float *bias;             // [c][W]
    const h16 *aux;      // [c][N][W]
    const float *wout, *bout, *y;  // output layer and targets
    float inv_s2;
    double *u_part;                // [c][tiles]
    float *dbout_part;             // [c][tiles]
    float *dwout_part, *db_part;   // [c][tiles][W]
    const float *x;                // [N][dx]
    float *dw0_part;               // [c][tiles][W][dx]
};

// byte offset of 16-byte piece j (0..3) of row r (0..31) in a warp's staging buffer;
// the XOR spreads both row-wise and 8-row-block accesses over all banks
__device__ __forceinline__ uint32_t stg_off(int r, int j) { return (uint32_t)(r * 64 + ((j ^ ((r >> 1) & 3)) << 4)); }

// One problem's share of a grouped launch of the layer kernel: its maps and parameters,
// and the first unit of its range in the launch's unit sequence.
struct LayerJob {   // aligned as CUtensorMap requires
    CUtensorMap tmA, tmWh, tmWl;
    LayerParams p;
    long ustart;
};

// A role's place in the unit sequence: job j, whose units start at base, with tpg tile
// pairs per chain.
struct UnitCursor {
    int j;
    long base;
    int tpg;
};

// Units: a unit is (chain, pair of consecutive tiles); CTA r takes tile 2 j + r.
// WSPLIT adds the lo part of W (forward).  The epilogue issues a tile's global
// loads (slopes, targets) before it waits for the accumulator, so their latency
// overlaps the tile's MMAs.
// G (grouped launch): the units of several problems of the same width follow each other
// (job j's from jobs[j].ustart on, utotal in all); every role tracks the job of its
// current unit, and W reloads whenever (job, chain) changes.  Otherwise tmA0, tmWh0,
// tmWl0 and p0 describe the one problem.
// WIDTH: the output features of the layer product (its columns), KD: its reduction width
// (the square hidden layers have KD = WIDTH; a net's last layer, w -> p, does not).
// L_FWD_LIN: a forward layer without activation (a DeepONet net's last layer).
template <int MODE, bool WSPLIT, int WIDTH, bool G, int KD = WIDTH>
__device__ __forceinline__ void layer_body(const CUtensorMap &tmA0, const CUtensorMap &tmWh0, const CUtensorMap &tmWl0,
                                           const LayerParams &p0, const LayerJob *__restrict__ jobs, int njobs,
                                           long utotal)
{
    constexpr bool BWD = (MODE == L_BWD_TANH || MODE == L_BWD_FIRST);
    constexpr int LN = WIDTH;                          // accumulator columns: whole rows
    constexpr int BN = WIDTH / 2;                      // rows of B (W) resident in this CTA
    constexpr int NKB = KD / 64;                       // K-blocks of the reduction
    static_assert(KD % 64 == 0 && WIDTH % 64 == 0 && (!BWD || BN % 64 == 0), "layer shape");
    constexpr int NCH = LN / 64;                       // 32-column chunks of one epilogue warp's half row
    constexpr int SLOT = LN;                           // TMEM columns per accumulator
    constexpr int TCOLS = 2 * SLOT;
    constexpr int kblk = BN * 128;                     // bytes of one resident K-block of W
    static_assert(NKB * kblk <= L_W_HALF, "resident half of W");
    // the reverse pass with hi/lo weights needs the lo region for W: its ring is two stages
    // deep and its slopes prefetch two chunks ahead in a region of their own
    constexpr bool RLO = BWD && WSPLIT;
    constexpr int STAGES = RLO ? L_STAGES_RLO : L_STAGES;
    constexpr int NAUX = RLO ? 2 : NCH;                // slope chunks in flight per epilogue warp
    static_assert(NCH % NAUX == 0, "slope chunks cycle through the buffers");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sWh = smem;
    uint8_t *sWl = smem + L_W_HALF;
    uint8_t *sA = smem + 2 * L_W_HALF;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA + STAGES * L_A_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 7);
    float *scr = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(bars) + 256);
    float *red = scr;                                                                  // column sums
    float *redb = scr + 8 * L_STG / 4;   // reverse tanh: [4][w] column sums, after the staging buffers
    uint8_t *stage0 = BWD ? reinterpret_cast<uint8_t *>(scr) : reinterpret_cast<uint8_t *>(scr + 4 * 256);
    double *dred = reinterpret_cast<double *>(scr + L_SCR_FLOATS);   // [4]
    float *fred = reinterpret_cast<float *>(dred + 4);               // [4]
    float *sbias = fred + 16;                                        // [256] bias of the current chain
    float *swo = sbias + 256;                                        // [256] output weights of the current chain
    float *fsum = swo + 256;                                         // [2][128] half-row partial dot products
    const uint32_t a_full0 = smem_u32(bars), a_empty0 = a_full0 + 8 * STAGES;
    const uint32_t w_full = a_empty0 + 8 * STAGES, w_empty = w_full + 8;
    const uint32_t acc_full0 = w_empty + 8, acc_empty0 = acc_full0 + 16;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    auto jp = [&](int j) -> const LayerParams & {
        if constexpr (G) return jobs[j].p;
        else return p0;
    };
    auto map_a = [&](int j) -> const CUtensorMap * { return G ? &jobs[j].tmA : &tmA0; };
    auto map_wh = [&](int j) -> const CUtensorMap * { return G ? &jobs[j].tmWh : &tmWh0; };
    auto map_wl = [&](int j) -> const CUtensorMap * { return G ? &jobs[j].tmWl : &tmWl0; };
    // move cursor k forward to the job holding unit u (u never decreases for one cursor)
    auto seek = [&](UnitCursor &k, long u) {
        if constexpr (G) {
            int j = k.j;
            while (j + 1 < njobs && u >= jobs[j + 1].ustart) ++j;
            if (j != k.j) k = UnitCursor{j, jobs[j].ustart, (jobs[j].p.ntiles + 1) / 2};
        }
    };
    const UnitCursor cur0{0, 0, (jp(0).ntiles + 1) / 2};
    int *const perr = jp(0).err;                       // one error flag for the whole launch
    const long U = G ? utotal : (long)p0.C * cur0.tpg;
    // (job << 32) | chain: W and the per-chain constants change with it
    auto unit_key = [](const UnitCursor &k, int c) { return ((long)k.j << 32) | (long)(unsigned)c; };
    const int ngr = gridDim.x / 2, gi = blockIdx.x / 2;
    const long u0 = U * gi / ngr, u1 = U * (gi + 1) / ngr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(a_full0 + 8 * s, 1);
            mbar_init(a_empty0 + 8 * s, 1);
        }
        mbar_init(w_full, 1);
        mbar_init(w_empty, 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(acc_full0 + 8 * s, 1);
            mbar_init(acc_empty0 + 8 * s, 16);   // one arrival per epilogue warp of the pair
        }
        fence_mbar_init();
        if (!G) {
            prefetch_map(&tmA0);
            prefetch_map(&tmWh0);
            if (WSPLIT) prefetch_map(&tmWl0);
        }
    }
    if (warp == 1) {
        tmem_alloc2(smem_u32(tmem_slot), TCOLS);
        tmem_relinquish2();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // the leader's barriers exist before the peer signals them
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait();      // the previous kernel's outputs are visible from here on
    pdl_trigger();
    // barriers that count loads and epilogue releases live in the leader CTA
    const uint32_t lead_a_full0 = mapa_shared(a_full0, 0);
    const uint32_t lead_w_full = mapa_shared(w_full, 0);
    const uint32_t lead_acc_empty0 = mapa_shared(acc_empty0, 0);

    if (warp == 0) {
        if (lane == 0) {   // TMA producer (both CTAs)
            long cur_key = -1;
            int fenced = -1;
            UnitCursor cu = cur0;
            uint32_t wph = 0;
            long kbi = 0;
            bool ok = true, w_pending = false;
            for (long u = u0; u < u1 && ok; ++u) {
                seek(cu, u);
                const int c = (int)((u - cu.base) / cu.tpg), t = (int)((u - cu.base) % cu.tpg) * 2 + (int)rank;
                const CUtensorMap *mA = map_a(cu.j), *mWh = map_wh(cu.j), *mWl = map_wl(cu.j);
                if (G && cu.j != fenced) {
                    tensormap_acquire(mA);
                    tensormap_acquire(mWh);
                    if (WSPLIT) tensormap_acquire(mWl);
                    fenced = cu.j;
                }
                const long key = unit_key(cu, c);
                if (key != cur_key) {
                    if (cur_key >= 0) {
                        if (!mbar_wait(w_empty, wph, perr)) { ok = false; break; }
                        wph ^= 1u;
                    }
                    if (leader) mbar_expect_tx(w_full, 2u * (WSPLIT ? 2u : 1u) * NKB * kblk);
                    for (int kb = 0; kb < NKB; ++kb) {
                        const uint32_t dh = smem_u32(sWh) + kb * kblk, dl = smem_u32(sWl) + kb * kblk;
                        if (!BWD) {   // B = W[f][k], K-major: this CTA's BN output features
                            tma_load_3d_pair(dh, mWh, kb * BK, (int)rank * BN, c, lead_w_full);
                            if (WSPLIT) tma_load_3d_pair(dl, mWl, kb * BK, (int)rank * BN, c, lead_w_full);
                        } else {      // B = W^T read MN-major from W[o][i]: 64-feature atoms
                            for (int a = 0; a < BN / 64; ++a) {
                                tma_load_3d_pair(dh + 8192 * a, mWh, (int)rank * BN + 64 * a, kb * BK, c, lead_w_full);
                                if (WSPLIT)
                                    tma_load_3d_pair(dl + 8192 * a, mWl, (int)rank * BN + 64 * a, kb * BK, c,
                                                     lead_w_full);
                            }
                        }
                    }
                    w_pending = true;
                    cur_key = key;
                }
                for (int kb = 0; kb < NKB; ++kb) {
                    const int s = (int)(kbi % STAGES);
                    const uint32_t ph = (uint32_t)(kbi / STAGES) & 1u;
                    if (!mbar_wait(a_empty0 + 8 * s, ph ^ 1u, perr)) { ok = false; break; }
                    if (leader) mbar_expect_tx(a_full0 + 8 * s, 2u * L_A_BYTES);
                    tma_load_3d_pair(smem_u32(sA + s * L_A_BYTES), mA, kb * BK, t * BM, c, lead_a_full0 + 8 * s);
                    ++kbi;
                }
            }
            if (!ok && leader) {   // let copies already in flight land before the CTA exits
                for (long i = std::max<long>(0, kbi - STAGES); i < kbi; ++i)
                    mbar_wait(a_full0 + 8 * (int)(i % STAGES), (uint32_t)(i / STAGES) & 1u, perr, 100000000ull);
                if (w_pending) mbar_wait(w_full, wph, perr, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {   // MMA issuer: the leader alone drives the pair
            const uint32_t idesc = idesc_h16(2 * BM, LN, false, BWD);
            long cur_key = -1;
            UnitCursor cu = cur0;
            uint32_t wph = 0;
            long kbi = 0;
            int it = 0;
            bool ok = true;
            for (long u = u0; u < u1 && ok; ++u, ++it) {
                seek(cu, u);
                const long key = unit_key(cu, (int)((u - cu.base) / cu.tpg));
                if (key != cur_key) {
                    if (!mbar_wait_cluster(w_full, wph, perr)) { ok = false; break; }
                    wph ^= 1u;
                    cur_key = key;
                }
                const int slot = it & 1;
                if (!mbar_wait(acc_empty0 + 8 * slot, ((uint32_t)(it >> 1) & 1u) ^ 1u, perr)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(slot * SLOT);
                for (int kb = 0; kb < NKB; ++kb) {
                    const int s = (int)(kbi % STAGES);
                    const uint32_t ph = (uint32_t)(kbi / STAGES) & 1u;
                    if (!mbar_wait_cluster(a_full0 + 8 * s, ph, perr)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(sA + s * L_A_BYTES);
                    const uint32_t wh = smem_u32(sWh) + kb * kblk, wl = smem_u32(sWl) + kb * kblk;
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        const uint64_t ad = sdesc(sa + 32 * ks, 0, 1024);
                        const uint64_t bh = BWD ? sdesc(wh + 2048 * ks, 8192, 1024) : sdesc(wh + 32 * ks, 0, 1024);
                        mma_bf16_pair(d_tmem, ad, bh, idesc, (kb > 0 || ks > 0) ? 1u : 0u);
                        if (WSPLIT) {
                            const uint64_t bl = BWD ? sdesc(wl + 2048 * ks, 8192, 1024) : sdesc(wl + 32 * ks, 0, 1024);
                            mma_bf16_pair(d_tmem, ad, bl, idesc, 1u);
                        }
                    }
                    mma_commit_pair(a_empty0 + 8 * s, (uint16_t)3);
                    ++kbi;
                }
                if (!ok) break;
                mma_commit_pair(acc_full0 + 8 * slot, (uint16_t)3);
                long next_key = -1;   // W stays while the next unit has the same (job, chain)
                if (u + 1 < u1) {
                    UnitCursor nx = cu;
                    seek(nx, u + 1);
                    next_key = unit_key(nx, (int)((u + 1 - nx.base) / nx.tpg));
                }
                if (next_key != key) mma_commit_pair(w_empty, (uint16_t)3);
            }
        }
    } else {
        // ---------------- epilogue warps 2..9: two per lane quadrant ----------------
        // warp e = warp - 2 owns rows 32 q .. 32 q + 31 (q = warp mod 4, the TMEM lanes it
        // may read) and the half row h = e / 4 of the columns.
        const int q = warp & 3, row = 32 * q + lane, et = threadIdx.x - 64, h = (warp - 2) >> 2;
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        const int hc0 = h * (LN / 2);          // first column of this warp's half
        uint8_t *stg = stage0 + (warp - 2) * L_STG;
        const int tr = lane >> 2, tj = lane & 3;   // transposed access: rows tr + 8 i, piece tj
        // reverse pass: the slopes of a unit's chunk ch land in abuf + (ch mod NAUX) * L_STG by
        // cp.async, one commit group per chunk, issued NAUX chunks ahead of their use (a whole
        // tile when NAUX = NCH)
        const uint32_t abuf = RLO ? smem_u32(smem + L_AUX_OFF_RLO) + (uint32_t)(warp - 2) * L_AUX_RLO
                                  : smem_u32(sWl) + (uint32_t)(warp - 2) * L_AUX;
        UnitCursor ca = cur0;   // the slope prefetch runs up to a unit ahead of the epilogue
        auto issue_aux = [&](long v, int ch) {
            if (v < u1) {
                seek(ca, v);
                const LayerParams &p = jp(ca.j);
                const int cv = (int)((v - ca.base) / ca.tpg), tv = (int)((v - ca.base) % ca.tpg) * 2 + (int)rank;
                const int rv0 = tv * BM + 32 * q;
                const h16 *src = p.aux + ((long)cv * p.N + rv0) * p.W + hc0 + 32 * ch + 8 * tj;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int rr = tr + 8 * i;
                    const bool in = rv0 + rr < p.N;
                    cp_async16(abuf + (ch % NAUX) * L_STG + stg_off(rr, tj), in ? src + (long)rr * p.W : p.aux,
                               in ? 16u : 0u);
                }
            }
            cp_async_commit();
        };
        // the chunk that follows chunk ch of unit v by NAUX chunks goes into the same buffer
        auto refill_aux = [&](long v, int ch) { issue_aux(v + (ch + NAUX) / NCH, (ch + NAUX) % NCH); };
        if (BWD)
            for (int ch = 0; ch < NAUX; ++ch) issue_aux(u0, ch);
        int it = 0;
        long loaded_key = -1;
        UnitCursor ce = cur0;
        for (long u = u0; u < u1; ++u, ++it) {
            seek(ce, u);
            const LayerParams &p = jp(ce.j);
            const int c = (int)((u - ce.base) / ce.tpg), t = (int)((u - ce.base) % ce.tpg) * 2 + (int)rank;
            const long key = unit_key(ce, c);
            const bool tile_ok = t < p.ntiles;
            const int slot = it & 1;
            const int r0 = t * BM + 32 * q;    // first data row of this warp
            const int m = r0 + row - 32 * q;
            const bool valid = m < p.N;
            const long wbase = ((long)c * p.N + r0) * p.W + hc0;   // element (r0, hc0) of [c][N][W]
            const long part = ((long)c * p.ntiles + t) * p.W;
            const float yv = (MODE == L_FWD_OUT && valid) ? p.y[m] : 0.0f;
            const float bo = MODE == L_FWD_OUT ? p.bout[c] : 0.0f;   // (loaded before the accumulator wait)
            // first-layer gradients: the B operand [X | 1] of dW0 = delta_1^T X and db0 = delta_1^T 1
            // as mma.sync fragments of this warp's 32 rows: column n < dx holds x_n, column dx
            // the ones, for rows 16 ks + 8 hf + 2 (lane % 4) + {0, 1}
            uint32_t bx[2][2] = {{0u, 0u}, {0u, 0u}};
            if (MODE == L_BWD_FIRST) {
                float vn[8];   // inputs and the ones column: dx <= 7
#pragma unroll
                for (int n = 0; n < 8; ++n)
                    vn[n] = n < p.dx ? (valid ? p.x[(long)m * p.dx + n] : 0.0f) : (n == p.dx ? 1.0f : 0.0f);
                const int g = lane >> 2, c2 = 2 * (lane & 3);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        const int r = 16 * ks + 8 * hf + c2;
                        float v0 = 0.0f, v1 = 0.0f;
#pragma unroll
                        for (int n = 0; n < 8; ++n) {
                            const float a0 = __shfl_sync(0xffffffffu, vn[n], r);
                            const float a1 = __shfl_sync(0xffffffffu, vn[n], r + 1);
                            if (g == n) {
                                v0 = a0;
                                v1 = a1;
                            }
                        }
                        bx[ks][hf] = pack_h16(v0, v1);
                    }
            }
            // per-chain constants into shared memory
            if (!BWD && key != loaded_key) {
                named_bar_sync(1, 256);
                for (int i = et; i < LN; i += 256) {
                    sbias[i] = p.bias[(long)c * p.W + i];
                    if (MODE == L_FWD_OUT) swo[i] = p.wout[(long)c * p.W + i];
                }
                named_bar_sync(1, 256);
                loaded_key = key;
            }
            // this thread's 32 packed bf16 of its row -> staging -> 8-row coalesced stores
            auto store_chunk = [&](const uint32_t (&pk)[16], int col) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    *reinterpret_cast<uint4 *>(stg + stg_off(lane, j)) =
                        make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int rr = tr + 8 * i;
                    const uint4 v = *reinterpret_cast<const uint4 *>(stg + stg_off(rr, tj));
                    if (r0 + rr < p.N) *reinterpret_cast<uint4 *>(p.out + wbase + (long)rr * p.W + col + 8 * tj) = v;
                }
                __syncwarp();
            };
            if (!mbar_wait(acc_full0 + 8 * slot, (uint32_t)(it >> 1) & 1u, perr)) break;
            tc_fence_after();
            const uint32_t taddr = tmem + lane_off + (uint32_t)(slot * SLOT + hc0);
            uint32_t rb[2][32];
            if (MODE == L_FWD_TANH || MODE == L_FWD_LIN) {
                tmem_ld32_issue(taddr, rb[0]);
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int c0 = 32 * ch;
                    tmem_ld_wait(rb[ch & 1]);
                    if (ch + 1 < NCH) tmem_ld32_issue(taddr + c0 + 32, rb[(ch + 1) & 1]);
                    uint32_t pk[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float z0 = __uint_as_float(rb[ch & 1][2 * j]) + sbias[hc0 + c0 + 2 * j];
                        const float z1 = __uint_as_float(rb[ch & 1][2 * j + 1]) + sbias[hc0 + c0 + 2 * j + 1];
                        pk[j] = MODE == L_FWD_LIN ? pack_h16(z0, z1) : pack_h16(act_tanh(z0), act_tanh(z1));
                    }
                    store_chunk(pk, c0);
                }
            } else if (BWD) {
                tmem_ld32_issue(taddr, rb[0]);
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int c0 = 32 * ch;
                    float dd[32];
                    tmem_ld_wait(rb[ch & 1]);
                    if (ch + 1 < NCH) tmem_ld32_issue(taddr + c0 + 32, rb[(ch + 1) & 1]);
                    // slopes of this chunk: exactly NAUX - 1 groups were committed after this one
                    cp_async_wait<NAUX - 1>();
                    __syncwarp();
                    uint4 av[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) av[j] = lds128(abuf + (ch % NAUX) * L_STG + stg_off(lane, j));
                    __syncwarp();   // every lane has its row: refill the chunk for the next unit
                    if (MODE != L_BWD_FIRST) refill_aux(u, ch);   // (the first layer stages in it first)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint4 uu = av[j];
                        const uint32_t w4[4] = {uu.x, uu.y, uu.z, uu.w};
#pragma unroll
                        for (int tt = 0; tt < 4; ++tt) {
                            const float2 a = unpack_h16(w4[tt]);
                            const int k = 8 * j + 2 * tt;
                            dd[k] = valid ? __uint_as_float(rb[ch & 1][k]) * (1.0f - a.x * a.x) : 0.0f;
                            dd[k + 1] = valid ? __uint_as_float(rb[ch & 1][k + 1]) * (1.0f - a.y * a.y) : 0.0f;
                        }
                    }
                    if (MODE == L_BWD_TANH) {
                        uint32_t pk[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) pk[j] = pack_h16(dd[2 * j], dd[2 * j + 1]);
                        store_chunk(pk, c0);
                        // when asked (db_part set), the column sums of the tile's deltas, the
                        // bias gradient of the layer below: this warp's 32 rows first
                        if (p.db_part) redb[q * LN + hc0 + c0 + lane] = reduce_scatter32(dd);
                    }
                    if (MODE == L_BWD_FIRST) {
                        // first-layer weight and bias gradients of this chunk's 32 columns over the
                        // warp's 32 rows: delta_1 (bf16) goes to the chunk's slope buffer, which
                        // this warp has read, and mma.sync forms delta_1^T [X | 1]
                        const uint32_t sb = abuf + (ch % NAUX) * L_STG;
                        {
                            uint32_t pk[16];
#pragma unroll
                            for (int j = 0; j < 16; ++j) pk[j] = pack_h16(dd[2 * j], dd[2 * j + 1]);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sb + stg_off(lane, j)),
                                             "r"(pk[4 * j]), "r"(pk[4 * j + 1]), "r"(pk[4 * j + 2]), "r"(pk[4 * j + 3])
                                             : "memory");
                        }
                        __syncwarp();
                        float acc[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
                        const int mi = lane >> 3;
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)        // columns 16 mt .. 16 mt + 15 of the chunk
#pragma unroll
                            for (int ks = 0; ks < 2; ++ks) {  // rows 16 ks .. 16 ks + 15 of the warp
                                uint32_t a[4];
                                ldmatrix_x4_trans(a, sb + stg_off(16 * ks + (lane & 7) + 8 * (mi >> 1), 2 * mt + (mi & 1)));
                                mma_m16n8k16_h16(acc[mt], a, bx[ks][0], bx[ks][1]);
                            }
                        __syncwarp();   // the buffer is read: refill it for the next unit
                        refill_aux(u, ch);
                        const int g = lane >> 2, c2 = 2 * (lane & 3);
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int hf = 0; hf < 2; ++hf)
#pragma unroll
                                for (int e = 0; e < 2; ++e) {
                                    const int n = c2 + e, col = hc0 + c0 + 16 * mt + 8 * hf + g;
                                    const float v = acc[mt][2 * hf + e];
                                    if (n < p.dx) red[((1 + n) * 4 + q) * LN + col] = v;
                                    else if (n == p.dx) red[(0 * 4 + q) * LN + col] = v;
                                }
                    }
                }
                if (MODE == L_BWD_TANH && p.db_part) {   // the four quadrants' sums, per tile
                    named_bar_sync(1, 256);
                    if (tile_ok)
                        for (int cc = et; cc < LN; cc += 256)
                            p.db_part[part + cc] = redb[0 * LN + cc] + redb[1 * LN + cc] + redb[2 * LN + cc] +
                                                   redb[3 * LN + cc];
                    named_bar_sync(1, 256);
                }
                if (MODE == L_BWD_FIRST) {
                    named_bar_sync(1, 256);
                    if (tile_ok) {
                        for (int cc = et; cc < LN; cc += 256) {
                            p.db_part[part + cc] = red[(0 * 4 + 0) * LN + cc] + red[(0 * 4 + 1) * LN + cc] +
                                                   red[(0 * 4 + 2) * LN + cc] + red[(0 * 4 + 3) * LN + cc];
                            for (int d = 0; d < p.dx; ++d)
                                p.dw0_part[(part + cc) * p.dx + d] =
                                    red[((1 + d) * 4 + 0) * LN + cc] + red[((1 + d) * 4 + 1) * LN + cc] +
                                    red[((1 + d) * 4 + 2) * LN + cc] + red[((1 + d) * 4 + 3) * LN + cc];
                        }
                    }
                    named_bar_sync(1, 256);
                }
            } else if (MODE == L_FWD_OUT) {
                // pass 1: the activations, written back over the accumulator so that pass 2
                // reads them instead of evaluating tanh again, and the row dot product
                float fh = 0.0f;
                tmem_ld32_issue(taddr, rb[0]);
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int c0 = 32 * ch;
                    tmem_ld_wait(rb[ch & 1]);
                    if (ch + 1 < NCH) {
                        if (ch > 0) tmem_st_wait();   // the store of chunk ch - 1 has read its registers
                        tmem_ld32_issue(taddr + c0 + 32, rb[(ch + 1) & 1]);
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float a = act_tanh(__uint_as_float(rb[ch & 1][j]) + sbias[hc0 + c0 + j]);
                        fh += a * swo[hc0 + c0 + j];
                        rb[ch & 1][j] = __float_as_uint(a);
                    }
                    tmem_st32(taddr + c0, rb[ch & 1]);
                }
                tmem_st_wait();
                // the row's dot product: both halves, in a fixed order
                fsum[h * 128 + row] = fh;
                named_bar_sync(1, 256);
                const float fo = bo + (fsum[row] + fsum[128 + row]);
                const float r = valid ? fo - yv : 0.0f;
                const float d = r * p.inv_s2;
                if (h == 0) {   // the warp's 32 squared residuals: an FP32 partial, then FP64
                    float r2 = r * r;
                    float ds = d;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
                        ds += __shfl_xor_sync(0xffffffffu, ds, o);
                    }
                    if (lane == 0) {
                        dred[q] = (double)r2;
                        fred[q] = ds;
                    }
                }
                // output-weight gradient sums d^T A over the warp's 32 rows by mma.sync: the B
                // operand is the column d (rows 16 ks + 8 hf + 2 (lane % 4) + {0, 1}, column 0)
                uint32_t bd[2][2];
                {
                    const int g = lane >> 2, c2 = 2 * (lane & 3);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                        for (int hf = 0; hf < 2; ++hf) {
                            const int rr = 16 * ks + 8 * hf + c2;
                            const float d0 = __shfl_sync(0xffffffffu, d, rr);
                            const float d1 = __shfl_sync(0xffffffffu, d, rr + 1);
                            bd[ks][hf] = g == 0 ? pack_h16(d0, d1) : 0u;
                        }
                }
                tmem_ld32_issue(taddr, rb[0]);
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int c0 = 32 * ch;
                    tmem_ld_wait(rb[ch & 1]);
                    if (ch + 1 < NCH) tmem_ld32_issue(taddr + c0 + 32, rb[(ch + 1) & 1]);
                    {   // A (bf16) through the staging buffer into mma.sync fragments
                        const uint32_t sb = smem_u32(stg);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t *w = &rb[ch & 1][8 * j];
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sb + stg_off(lane, j)),
                                         "r"(pack_h16(__uint_as_float(w[0]), __uint_as_float(w[1]))),
                                         "r"(pack_h16(__uint_as_float(w[2]), __uint_as_float(w[3]))),
                                         "r"(pack_h16(__uint_as_float(w[4]), __uint_as_float(w[5]))),
                                         "r"(pack_h16(__uint_as_float(w[6]), __uint_as_float(w[7])))
                                         : "memory");
                        }
                        __syncwarp();
                        float acc[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
                        const int mi = lane >> 3;
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int ks = 0; ks < 2; ++ks) {
                                uint32_t a4[4];
                                ldmatrix_x4_trans(a4, sb + stg_off(16 * ks + (lane & 7) + 8 * (mi >> 1), 2 * mt + (mi & 1)));
                                mma_m16n8k16_h16(acc[mt], a4, bd[ks][0], bd[ks][1]);
                            }
                        __syncwarp();   // the staging buffer is read: the deltas go through it next
                        if ((lane & 3) == 0) {   // column 0 of D: lanes 4 g hold columns g and g + 8
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                for (int hf = 0; hf < 2; ++hf)
                                    red[(0 * 4 + q) * LN + hc0 + c0 + 16 * mt + 8 * hf + (lane >> 2)] = acc[mt][2 * hf];
                        }
                    }
                    uint32_t pk[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float a0 = __uint_as_float(rb[ch & 1][2 * j]), a1 = __uint_as_float(rb[ch & 1][2 * j + 1]);
                        pk[j] = pack_h16(d * swo[hc0 + c0 + 2 * j] * (1.0f - a0 * a0),
                                          d * swo[hc0 + c0 + 2 * j + 1] * (1.0f - a1 * a1));
                    }
                    store_chunk(pk, c0);
                }
                named_bar_sync(1, 256);
                if (tile_ok) {
                    for (int cc = et; cc < LN; cc += 256)
                        p.dwout_part[part + cc] = red[(0 * 4 + 0) * LN + cc] + red[(0 * 4 + 1) * LN + cc] +
                                                  red[(0 * 4 + 2) * LN + cc] + red[(0 * 4 + 3) * LN + cc];
                    if (et == 0) {
                        p.u_part[(long)c * p.ntiles + t] = dred[0] + dred[1] + dred[2] + dred[3];
                        p.dbout_part[(long)c * p.ntiles + t] = fred[0] + fred[1] + fred[2] + fred[3];
                    }
                }
                named_bar_sync(1, 256);
            }
            // release the accumulator slot: one arrival per warp on the leader's barrier
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_remote(lead_acc_empty0 + 8 * slot);
        }
        if (BWD) cp_async_wait<0>();   // no copy into shared memory outlives the loop
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();   // neither CTA leaves while the pair may still touch its memory
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc2(tmem, TCOLS);
    }
}

template <int MODE, int WIDTH, bool SPLIT, int KD = WIDTH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(L_THREADS, 1)
    k_layer_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmWh,
                 const __grid_constant__ CUtensorMap tmWl, const __grid_constant__ LayerParams p)
{
    layer_body<MODE, SPLIT, WIDTH, false, KD>(tmA, tmWh, tmWl, p, nullptr, 1, 0);
}

// The grouped launch: the units of njobs problems (utotal in all) on one grid of CTA pairs.
template <int MODE, int WIDTH, bool SPLIT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(L_THREADS, 1)
    k_layer_pair_g(const LayerJob *__restrict__ jobs, int njobs, long utotal)
{
    const LayerJob &j0 = jobs[0];   // (the single-problem arguments, unused when grouped)
    layer_body<MODE, SPLIT, WIDTH, true>(j0.tmA, j0.tmWh, j0.tmWl, j0.p, jobs, njobs, utotal);
}

// ---------------------------------------------------------------------------
// Weight and bias gradient of a w x w hidden layer at the sampled entries.
// CTA (mh, nh) of a (row split, chain) computes the 128 x 128 block
// dW[m0 : m0+128][n0 : n0+128] = delta^T A over its rows, both operands read
// MN-major straight from their row-major [rows][w] arrays.  The CTAs with n0 = 0
// also multiply delta^T by a 16-column block of ones, which sums delta over the rows:
// the gradient of the layer's bias, from the same operand stages.  Only the sampled
// entries leave the chip.  Two CTAs fit on an SM (shared and tensor memory).
// ---------------------------------------------------------------------------
constexpr int DW_STAGES = 3;
constexpr int DW_A_BYTES = BM * BK * 2;        // 16 KB: delta, 128 output features x 64 data rows
constexpr int DW_B_BYTES = 128 * BK * 2;       // 16 KB: A_i, 128 input features x 64 data rows
constexpr int DW_STAGE = DW_A_BYTES + DW_B_BYTES;
constexpr int DW_ONES = 16 * 128;              // 16 K-major rows of 64 bf16 ones
constexpr int DW_SMEM = 1024 + DW_STAGES * DW_STAGE + DW_ONES + 256;
constexpr int DW_TCOLS = 256;                  // 128 columns of dW + 16 of row sums
constexpr int kMaxSplits = 32;                 // largest row-split count the autotuner tries

// HMC_AUTOTUNE=0 keeps the built-in heuristic choices instead of timing candidates at
// handle creation (for runs under a profiler, whose overhead would skew the timings).
bool autotune_enabled()
{
    const char *e = getenv("HMC_AUTOTUNE");
    return !(e && e[0] == '0');
}
static_assert(DW_STAGES * DW_STAGE >= 128 * 129 * 4, "the epilogue staging reuses the operand stages");

template <bool G>
__device__ __forceinline__ void dw2_body(const CUtensorMap &tmD, const CUtensorMap &tmA, const Params &p, int bx,
                                         int split, int b)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *ones = smem + DW_STAGES * DW_STAGE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(ones + DW_ONES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * DW_STAGES + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * DW_STAGES, accb = empty0 + 8 * DW_STAGES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nnh = p.N / 128;                // column blocks of dW (w / 128)
    const int m0 = (bx / nnh) * BM, n0 = (bx % nnh) * 128;
    const bool with_db = n0 == 0 && p.db_part != nullptr;
    const int total_kb = (p.K + BK - 1) / BK;
    const int kb0 = split * p.kb_per_split;
    const int nkb = min(p.kb_per_split, total_kb - kb0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < DW_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        fence_mbar_init();
        if (G) {   // thread 0 is also the TMA producer
            tensormap_acquire(&tmD);
            tensormap_acquire(&tmA);
        }
        prefetch_map(&tmD);
        prefetch_map(&tmA);
    }
    for (int i = threadIdx.x; i < DW_ONES / 4; i += blockDim.x)   // pairs of 16-bit 1.0
        reinterpret_cast<uint32_t *>(ones)[i] = pack_h16(1.0f, 1.0f);
    fence_proxy_async_smem();   // the tensor core reads what the threads wrote
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), DW_TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait();      // the reverse pass's deltas are visible from here on
    pdl_trigger();
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % DW_STAGES;
                const uint32_t ph = (uint32_t)(i / DW_STAGES) & 1u;
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.err)) { ok = false; break; }
                const uint32_t fb = full0 + 8 * s;
                mbar_expect_tx(fb, DW_STAGE);
                const uint32_t sa = smem_u32(smem + s * DW_STAGE), sb = sa + DW_A_BYTES;
                const int kc = (kb0 + i) * BK;
                for (int a = 0; a < 2; ++a) {
                    tma_load_3d(sa + 8192 * a, &tmD, m0 + 64 * a, kc, b, fb);
                    tma_load_3d(sb + 8192 * a, &tmA, n0 + 64 * a, kc, b, fb);
                }
                ++issued;
            }
            if (!ok)
                for (int i = max(0, issued - DW_STAGES); i < issued; ++i)
                    mbar_wait(full0 + 8 * (i % DW_STAGES), (uint32_t)(i / DW_STAGES) & 1u, p.err, 100000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_h16(BM, 128, true, true);
            const uint32_t idesc1 = idesc_h16(BM, 16, true, false);
            const uint32_t so = smem_u32(ones);
            for (int i = 0; i < nkb; ++i) {
                const int s = i % DW_STAGES;
                const uint32_t ph = (uint32_t)(i / DW_STAGES) & 1u;
                if (!mbar_wait(full0 + 8 * s, ph, p.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * DW_STAGE), sb = sa + DW_A_BYTES;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint64_t ad = sdesc(sa + 2048 * ks, 8192, 1024);
                    const uint32_t acc = (i > 0 || ks > 0) ? 1u : 0u;
                    mma_bf16(tmem, ad, sdesc(sb + 2048 * ks, 8192, 1024), idesc, acc);
                    if (with_db) mma_bf16(tmem + 128, ad, sdesc(so + 32 * ks, 0, 1024), idesc1, acc);
                }
                mma_commit(empty0 + 8 * s);
            }
            mma_commit(accb);
        }
    } else {
        const int q = warp & 3, row = 32 * q + lane, et = threadIdx.x - 64;
        ok = nkb > 0 && mbar_wait(accb, 0, p.err);
        tc_fence_after();
        if (ok) {
            float *stg = reinterpret_cast<float *>(smem);   // operand stages are idle now
            const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16);
            if (with_db) {   // every column of the ones product holds the row sum
                float v[32];
                tmem_ld32(taddr + 128, v);
                if (m0 + row < p.M) p.db_part[(long)split * p.db_split + (long)b * p.M + m0 + row] = v[0];
            }
            for (int c0 = 0; c0 < 128; c0 += 32) {
                float v[32];
                tmem_ld32(taddr + c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[row * 129 + c0 + j] = v[j];
            }
            named_bar_sync(1, 128);
            // eight index loads in flight per thread before any dependent access
            const int j0 = p.rowptr[m0], j1 = p.rowptr[min(m0 + BM, p.M)];
            float *dst = p.gw_part + (long)split * p.gw_split + (long)b * p.gw_b;
            for (int base = j0; base < j1; base += 128 * 8) {
                int e[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = base + et + 128 * u;
                    e[u] = j < j1 ? p.epack[j] : -1;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (e[u] < 0) continue;
                    const int c = (e[u] & 0xFFFF) - n0;
                    if (c >= 0 && c < 128) dst[base + et + 128 * u] = stg[((e[u] >> 16) - m0) * 129 + c];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, DW_TCOLS);
    }
}

__global__ void __launch_bounds__(NTHREADS, 2) k_dw2(const __grid_constant__ CUtensorMap tmD,
                                                     const __grid_constant__ CUtensorMap tmA,
                                                     const __grid_constant__ Params p)
{
    dw2_body<false>(tmD, tmA, p, blockIdx.x, blockIdx.y, blockIdx.z);
}

// grouped: tm[0] the deltas, tm[1] the activations of each job
__global__ void __launch_bounds__(NTHREADS, 2) k_dw2_g(const GridJob *__restrict__ jobs, int njobs)
{
    const GridJob &J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int lb = (int)blockIdx.x - J.bstart;
    dw2_body<true>(J.tm[0], J.tm[1], J.p, lb % J.gx, (lb / J.gx) % J.gy, lb / (J.gx * J.gy));
}

// ---------------------------------------------------------------------------
// Energy for the Metropolis test.  The trajectory's forces come from the bf16
// GEMMs; the accept/reject decision needs U(q) itself, and rounding every hidden
// activation to bf16 makes U jump by order one between nearby states (dH would
// carry that noise).  This forward pass carries the activations as bf16 hi/lo
// pairs and accumulates A_hi W_hi + A_hi W_lo + A_lo W_hi (the A_lo W_lo term is
// below 2^-16 of the product), with tanhf in the epilogue, so U follows an FP32
// forward pass.  OUT fuses the last hidden layer with the output layer and the
// residual and writes only the per-tile sums of squares (FP64).
// ---------------------------------------------------------------------------
constexpr int E3_STAGES = 2;
constexpr int E3_A = BM * BK * 2;            // 16 KB: one half of an A K-block
constexpr int E3_B = 256 * BK * 2;           // 32 KB: one half of a W K-block
constexpr int E3_STAGE = 2 * E3_A + 2 * E3_B;
constexpr int E3_SMEM = 1024 + E3_STAGES * E3_STAGE + 256 + 64;

// E3_TANH / E3_LIN: a layer whose output goes on as a hi/lo pair (tanh or linear);
// E3_OUT: the MLP's last hidden layer + scalar output + residual; E3_S: the DeepONet's
// S^T = T B^T on 128 x N tiles (N columns starting at blockIdx.y N) + residual.
enum E3Mode { E3_TANH = 0, E3_LIN = 1, E3_OUT = 2, E3_S = 3 };

struct E3Params {
    int M, N, K, ntiles;
    int *err;
    const float *bias;                   // [b][N]
    h16 *out_hi, *out_lo;      // [b][M][N]
    const float *wout, *bout, *y;        // E3_OUT: output layer [b][N], [b]; targets [M]
    double *u_part;                      // E3_OUT: [b][ntiles]; E3_S: [b][ntiles][ntn]
    const float *Yt;                     // E3_S: targets [nu][ny] (rows of S^T are the ny points)
    int nu, ntn;                         // E3_S: valid columns, column tiles
};

template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_energy3(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmWh, const __grid_constant__ CUtensorMap tmWl, const E3Params p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + E3_STAGES * E3_STAGE);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * E3_STAGES + 1);
    double *rd = reinterpret_cast<double *>(bars + 2 * E3_STAGES + 2);   // [4]
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * E3_STAGES, accb = empty0 + 8 * E3_STAGES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_tile = blockIdx.x, b = blockIdx.z, m0 = m_tile * BM;
    const int n0 = MODE == E3_S ? blockIdx.y * p.N : 0;
    const int nkb = (p.K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < E3_STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait();
    pdl_trigger();
    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = 2u * E3_A + 2u * (uint32_t)p.N * BK * 2u;
            int issued = 0;
            bool ok = true;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % E3_STAGES;
                const uint32_t ph = (uint32_t)(i / E3_STAGES) & 1u;
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, p.err)) { ok = false; break; }
                const uint32_t fb = full0 + 8 * s, sa = smem_u32(smem + s * E3_STAGE), sb = sa + 2 * E3_A;
                mbar_expect_tx(fb, bytes);
                tma_load_3d(sa, &tmAh, i * BK, m0, b, fb);
                tma_load_3d(sa + E3_A, &tmAl, i * BK, m0, b, fb);
                tma_load_3d(sb, &tmWh, i * BK, n0, b, fb);
                tma_load_3d(sb + E3_B, &tmWl, i * BK, n0, b, fb);
                ++issued;
            }
            if (!ok)
                for (int i = max(0, issued - E3_STAGES); i < issued; ++i)
                    mbar_wait(full0 + 8 * (i % E3_STAGES), (uint32_t)(i / E3_STAGES) & 1u, p.err, 100000000ull);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_h16(BM, p.N, false, false);
            for (int i = 0; i < nkb; ++i) {
                const int s = i % E3_STAGES;
                const uint32_t ph = (uint32_t)(i / E3_STAGES) & 1u;
                if (!mbar_wait(full0 + 8 * s, ph, p.err)) break;
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * E3_STAGE), sb = sa + 2 * E3_A;
#pragma unroll
                for (int ks = 0; ks < BK / 16; ++ks) {
                    const uint64_t ah = sdesc(sa + 32 * ks, 0, 1024), al = sdesc(sa + E3_A + 32 * ks, 0, 1024);
                    const uint64_t wh = sdesc(sb + 32 * ks, 0, 1024), wl = sdesc(sb + E3_B + 32 * ks, 0, 1024);
                    mma_bf16(tmem, ah, wh, idesc, (i > 0 || ks > 0) ? 1u : 0u);
                    mma_bf16(tmem, ah, wl, idesc, 1u);
                    mma_bf16(tmem, al, wh, idesc, 1u);
                }
                mma_commit(empty0 + 8 * s);
            }
            mma_commit(accb);
        }
    } else {
        const int q = warp & 3, row = 32 * q + lane, m = m0 + row, et = threadIdx.x - 64;
        const bool valid = m < p.M;
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16);
        const bool ok = mbar_wait(accb, 0, p.err);
        tc_fence_after();
        if (MODE == E3_TANH || MODE == E3_LIN) {
            const float *bias = p.bias + (long)b * p.N;
            for (int c0 = 0; ok && c0 < p.N; c0 += 32) {
                float v[32];
                tmem_ld32(taddr + c0, v);
                if (valid) {
                    uint32_t ph[16], pl[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float a0 = v[2 * j] + bias[c0 + 2 * j], a1 = v[2 * j + 1] + bias[c0 + 2 * j + 1];
                        if (MODE == E3_TANH) {
                            a0 = tanhf(a0);
                            a1 = tanhf(a1);
                        }
                        const h16 h0 = f_to_h16(a0), h1 = f_to_h16(a1);
                        ph[j] = pack_h16(h16_to_f(h0), h16_to_f(h1));
                        pl[j] = pack_h16(a0 - h16_to_f(h0), a1 - h16_to_f(h1));
                    }
                    uint4 *oh = reinterpret_cast<uint4 *>(p.out_hi + ((long)b * p.M + m) * p.N + c0);
                    uint4 *ol = reinterpret_cast<uint4 *>(p.out_lo + ((long)b * p.M + m) * p.N + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        oh[j] = make_uint4(ph[4 * j], ph[4 * j + 1], ph[4 * j + 2], ph[4 * j + 3]);
                        ol[j] = make_uint4(pl[4 * j], pl[4 * j + 1], pl[4 * j + 2], pl[4 * j + 3]);
                    }
                }
            }
        } else {
            double r2 = 0.0;
            if (MODE == E3_OUT) {
                const float *bias = p.bias + (long)b * p.N;
                const float *wo = p.wout + (long)b * p.N;
                float f = p.bout[b];
                for (int c0 = 0; ok && c0 < p.N; c0 += 32) {
                    float v[32];
                    tmem_ld32(taddr + c0, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) f += tanhf(v[j] + bias[c0 + j]) * wo[c0 + j];
                }
                const double r = valid ? (double)f - (double)p.y[m] : 0.0;
                r2 = r * r;
            } else {   // E3_S: row m is a query point, columns are input functions
                const float b0 = p.bout[b];
                const float *yb = p.Yt + m;
                for (int c0 = 0; ok && c0 < p.N; c0 += 32) {
                    float v[32];
                    tmem_ld32(taddr + c0, v);
                    const int u0 = n0 + c0;
                    if (valid && u0 + 32 <= p.nu) {   // a whole chunk: no per-column bounds
                        const long ny = p.M;
                        const float *yp = yb + (long)u0 * ny;
                        float yv[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) yv[j] = __ldg(yp + j * ny);
                        float r2c = 0.0f;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float r = (v[j] + b0) - yv[j];
                            r2c += r * r;
                        }
                        r2 += (double)r2c;
                    } else if (valid && u0 < p.nu) {
                        float r2c = 0.0f;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (u0 + j < p.nu) {
                                const float r = (v[j] + b0) - __ldg(yb + (long)(u0 + j) * p.M);
                                r2c += r * r;
                            }
                        }
                        r2 += (double)r2c;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
            if (lane == 0) rd[q] = r2;
            named_bar_sync(1, 128);
            if (et == 0) {
                const long o = MODE == E3_S ? ((long)b * p.ntiles + m_tile) * p.ntn + blockIdx.y
                                            : (long)b * p.ntiles + m_tile;
                p.u_part[o] = rd[0] + rd[1] + rd[2] + rd[3];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

template <int MODE>
void launch_energy3(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &wh, const CUtensorMap &wl,
                    const E3Params &p, dim3 grid, cudaStream_t s)
{
    static bool configured = false;
    if (!configured) {
        HMC_CK(cudaFuncSetAttribute(k_energy3<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, E3_SMEM));
        configured = true;
    }
    static const char *names[] = {"energy3_tanh", "energy3_lin", "energy3_out", "energy3_s"};
    ProfScope ps(names[MODE], s);
    launch_pdl(k_energy3<MODE>, grid, dim3(NTHREADS), E3_SMEM, s, ah, al, wh, wl, p);
}

// First layer of the accurate forward pass: A_1 = tanh(X W_0^T + b_0) in FP32, stored
// as a bf16 hi/lo pair.  Thread = (column o, slice of rows) of a (128-row tile, chain).
__global__ void __launch_bounds__(256) k_first_fwd3(const float *x, int dx, int N, int w, const float *W0,
                                                    const float *b0, h16 *A1h, h16 *A1l)
{
    __shared__ float xs[BM * 8];
    pdl_wait();
    pdl_trigger();
    const int b = blockIdx.y, n0 = blockIdx.x * BM;
    const int nr = min(BM, N - n0);
    for (int i = threadIdx.x; i < nr * dx; i += blockDim.x) xs[i] = x[(long)n0 * dx + i];
    __syncthreads();
    for (int o = threadIdx.x; o < w; o += blockDim.x) {
        float wr[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) wr[d] = d < dx ? W0[((long)b * w + o) * dx + d] : 0.0f;
        const float bo = b0[(long)b * w + o];
        const long base = ((long)b * N + n0) * w + o;
        for (int r = 0; r < nr; ++r) {
            float z = bo;
#pragma unroll
            for (int d = 0; d < 8; ++d)
                if (d < dx) z += xs[r * dx + d] * wr[d];
            const float a = tanhf(z);
            const h16 h = f_to_h16(a);
            A1h[base + (long)r * w] = h;
            A1l[base + (long)r * w] = f_to_h16(a - h16_to_f(h));
        }
    }
}

// ---------------------------------------------------------------------------
// CUDA-core kernels around the tensor-core GEMMs
// ---------------------------------------------------------------------------

// A_1[b][n][o] = tanh(sum_d X[n][d] W0[b][o][d] + b0[b][o]) in bf16.  One block per
// (128-row tile, chain); a thread keeps four adjacent rows o of W0 and b0 in registers
// and walks a slice of the tile's rows, whose inputs are staged in shared memory, so
// a warp writes 256 contiguous bytes of a row per store.  The input width DX is a
// template parameter: with a runtime width every row paid for eight predicated
// multiply-adds per output, and the kernel was bound by instruction issue.
template <int DX>
__device__ __forceinline__ void first_fwd_body(const float *x, int N, int w, const float *W0, const float *b0, h16 *A1,
                                               int bx, int b)
{
    __shared__ float xs[BM * DX];
    pdl_wait();
    pdl_trigger();
    const int n0 = bx * BM;
    const int nr = min(BM, N - n0);
    for (int i = threadIdx.x; i < nr * DX; i += blockDim.x) xs[i] = x[(long)n0 * DX + i];
    __syncthreads();
    const int quads = w / 4;                                   // w is 128 or 256 here
    const int groups = max(1, (int)blockDim.x / quads);
    const int per = (nr + groups - 1) / groups;
    for (int item = threadIdx.x; item < quads * groups; item += blockDim.x) {
        const int o0 = 4 * (item % quads), r0 = (item / quads) * per, r1 = min(nr, r0 + per);
        float wr[4][DX], bo[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            bo[c] = b0[(long)b * w + o0 + c];
#pragma unroll
            for (int d = 0; d < DX; ++d) wr[c][d] = W0[((long)b * w + o0 + c) * DX + d];
        }
        h16 *out = A1 + ((long)b * N + n0) * w + o0;
#pragma unroll 4
        for (int r = r0; r < r1; ++r) {
            float xv[DX];
#pragma unroll
            for (int d = 0; d < DX; ++d) xv[d] = xs[r * DX + d];
            float z[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                z[c] = bo[c];
#pragma unroll
                for (int d = 0; d < DX; ++d) z[c] += xv[d] * wr[c][d];
            }
            *reinterpret_cast<uint2 *>(out + (long)r * w) =
                make_uint2(pack_h16(act_tanh(z[0]), act_tanh(z[1])), pack_h16(act_tanh(z[2]), act_tanh(z[3])));
        }
    }
}

template <int DX>
__global__ void __launch_bounds__(256) k_first_fwd(const float *x, int N, int w, const float *W0, const float *b0,
                                                   h16 *A1)
{
    first_fwd_body<DX>(x, N, w, W0, b0, A1, blockIdx.x, blockIdx.y);
}

// One problem's first layer in a grouped launch: blocks [bstart, bstart + ntiles C).
struct FirstJob {
    const float *x, *W0, *b0;
    h16 *A1;
    int N, w, ntiles, bstart;
};

template <int DX> __global__ void __launch_bounds__(256) k_first_fwd_g(const FirstJob *__restrict__ jobs, int njobs)
{
    const FirstJob &J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int lb = (int)blockIdx.x - J.bstart;
    first_fwd_body<DX>(J.x, J.N, J.w, J.W0, J.b0, J.A1, lb % J.ntiles, lb / J.ntiles);
}

// The first-layer forward for an input width dx in 1..8.
void launch_first_fwd(int dx, dim3 grid, cudaStream_t s, const float *x, int N, int w, const float *W0,
                      const float *b0, h16 *A1)
{
    switch (dx) {
    case 1: launch_pdl(k_first_fwd<1>, grid, dim3(256), 0, s, x, N, w, W0, b0, A1); break;
    case 2: launch_pdl(k_first_fwd<2>, grid, dim3(256), 0, s, x, N, w, W0, b0, A1); break;
    case 3: launch_pdl(k_first_fwd<3>, grid, dim3(256), 0, s, x, N, w, W0, b0, A1); break;
    case 4: launch_pdl(k_first_fwd<4>, grid, dim3(256), 0, s, x, N, w, W0, b0, A1); break;
    case 5: launch_pdl(k_first_fwd<5>, grid, dim3(256), 0, s, x, N, w, W0, b0, A1); break;
    case 6: launch_pdl(k_first_fwd<6>, grid, dim3(256), 0, s, x, N, w, W0, b0, A1); break;
    case 7: launch_pdl(k_first_fwd<7>, grid, dim3(256), 0, s, x, N, w, W0, b0, A1); break;
    case 8: launch_pdl(k_first_fwd<8>, grid, dim3(256), 0, s, x, N, w, W0, b0, A1); break;
    default: HMC_REQUIRE(false, "first-layer input width %d is not in 1..8", dx);
    }
}

// Per-entry source of the gradient, decoded by k_finalize_bf16.
// E_GW: a weight entry gathered by a weight-gradient kernel ([split][b][k] partials);
// E_PART: anything summed from per-tile column sums, found through a DbDesc;
// E_HEAVY: an E_PART entry with many partials (per-tile sums), summed by a whole warp.
enum EntryKind { E_GW = 0, E_PART = 1, E_HEAVY = 2 };
constexpr int kHeavyPartials = 16;   // E_PART entries with at least this many partials are heavy


// Partial sums of one layer's bias gradient: entry (chain b, partial t, unit o) is at
// p[b * bstride + t * tstride + o], t < n.
struct DbDesc {
    const float *p;
    long bstride, tstride;
    int n;
};

// Marks the heavy entries in `kind` and returns their indices.
std::vector<int> mark_heavy(std::vector<int> &kind, const std::vector<int> &desc, const std::vector<DbDesc> &dbd)
{
    std::vector<int> heavy;
    for (size_t j = 0; j < kind.size(); ++j)
        if (kind[j] == E_PART && dbd[desc[j]].n >= kHeavyPartials) {
            kind[j] = E_HEAVY;
            heavy.push_back((int)j);
        }
    return heavy;
}

struct FinalArgs {
    int k, nsplit, nu;               // entries, weight-gradient splits, energy partials per chain
    const int *kind, *desc, *off;    // per entry
    const int *heavy;                // [nheavy] the E_HEAVY entries
    int nheavy, nlight;              // heavy entries; blocks of the one-thread-per-entry part
    const double *u_part;            // [b][nu]
    const float *gw_part;            // [split][b][k]
    long gw_split;
    const DbDesc *db;                // column-sum sources
    double half_inv_s2, inv_a2;
    float gscale;                    // data-term gradient scale (1 / sigma^2) / dscale
    const float *escale;             // [k] a further power of two per entry, or null
};

// grid (nlight + ceil(nheavy / 8) + 1, C): blocks 0..nlight-1 gather one entry per
// thread, the next ones one heavy entry per warp (its partials split over the lanes,
// then a fixed butterfly), and the last block of each chain computes U (fixed-order sums).
// gscale s + q / alpha^2 with the rounding steps spelled out, so that every kernel that
// inlines it (one problem's finalize, a group's) rounds alike: the compiler's own choice
// of where to fuse a multiply-add may differ between the two
__device__ __forceinline__ float grad_entry(const FinalArgs &a, float s, float qj)
{
    return __fmaf_rn(a.gscale, s, __fmul_rn(qj, (float)a.inv_a2));
}

__device__ __forceinline__ void finalize_body(const FinalArgs &a, const float *q, double *U, float *g, int bx, int gx,
                                              int b)
{
    __shared__ double sm[2][8];
    pdl_wait();
    pdl_trigger();
    if (bx == gx - 1) {   // U = likelihood + prior, block-parallel in a fixed order
        // |q|^2: eight squares at a time in FP32 (a bounded partial), accumulated in FP64;
        // this block is one SM's work, and GB300's FP64 pipe is narrow
        double pr = 0.0, lik = 0.0;
        for (int j0 = threadIdx.x; j0 < a.k; j0 += 8 * blockDim.x) {   // eight loads in flight
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * blockDim.x;
                v[u] = j < a.k ? __ldg(q + (long)b * a.k + j) : 0.0f;
            }
            pr += (double)(((v[0] * v[0] + v[1] * v[1]) + (v[2] * v[2] + v[3] * v[3])) +
                           ((v[4] * v[4] + v[5] * v[5]) + (v[6] * v[6] + v[7] * v[7])));
        }
        for (int i = threadIdx.x; i < a.nu; i += blockDim.x) lik += a.u_part[(long)b * a.nu + i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pr += __shfl_xor_sync(0xffffffffu, pr, o);
            lik += __shfl_xor_sync(0xffffffffu, lik, o);
        }
        if ((threadIdx.x & 31) == 0) {
            sm[0][threadIdx.x >> 5] = pr;
            sm[1][threadIdx.x >> 5] = lik;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0, l = 0.0;
            for (int i = 0; i < 8; ++i) {
                t += sm[0][i];
                l += sm[1][i];
            }
            U[b] = __fma_rn(l, a.half_inv_s2, __dmul_rn(__dmul_rn(0.5, t), a.inv_a2));   // (rounding as in grad_entry)
        }
        return;
    }
    if (!g) return;
    if (bx >= a.nlight) {   // heavy entries: one warp each
        const int h = (bx - a.nlight) * (int)(blockDim.x >> 5) + (int)(threadIdx.x >> 5);
        const int lane = threadIdx.x & 31;
        if (h >= a.nheavy) return;
        const int j = a.heavy[h];
        const DbDesc d = a.db[a.desc[j]];
        const float *dp = d.p + (long)b * d.bstride + a.off[j];
        float s = 0.0f;
        for (int t = lane; t < d.n; t += 32) s += __ldg(dp + (long)t * d.tstride);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (a.escale) s *= __ldg(a.escale + j);
        if (lane == 0) g[(long)b * a.k + j] = grad_entry(a, s, q[(long)b * a.k + j]);
        return;
    }
    const int j = bx * blockDim.x + threadIdx.x;
    if (j >= a.k || a.kind[j] == E_HEAVY) return;
    const float qj = q[(long)b * a.k + j];
    const float *dp;
    long stride;
    int n;
    if (a.kind[j] == E_GW) {
        dp = a.gw_part + (long)b * a.k + j, stride = a.gw_split, n = a.nsplit;
    } else {
        const DbDesc d = a.db[a.desc[j]];
        dp = d.p + (long)b * d.bstride + a.off[j], stride = d.tstride, n = d.n;
    }
    // partials added in index order, sixteen independent loads in flight per step
    float s = 0.0f;
    int t = 0;
    for (; t + 16 <= n; t += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = __ldg(dp + (long)(t + u) * stride);
#pragma unroll
        for (int u = 0; u < 16; ++u) s += v[u];
    }
    for (; t < n; ++t) s += __ldg(dp + (long)t * stride);
    if (a.escale) s *= __ldg(a.escale + j);
    g[(long)b * a.k + j] = grad_entry(a, s, qj);
}

__global__ void __launch_bounds__(256) k_finalize_bf16(FinalArgs a, const float *q, double *U, float *g)
{
    finalize_body(a, q, U, g, blockIdx.x, gridDim.x, blockIdx.y);
}

// One problem's finalize in a grouped launch: blocks [bstart, bstart + gx C); its
// coordinates start at q + qoff (and g + qoff), its energies at U + uoff.
struct FinalJob {
    FinalArgs a;
    long qoff, uoff;
    int bstart, gx;
};

__global__ void __launch_bounds__(256) k_finalize_g(const FinalJob *__restrict__ jobs, int njobs, const float *q,
                                                    double *U, float *g)
{
    const FinalJob &J = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int lb = (int)blockIdx.x - J.bstart;
    finalize_body(J.a, q + J.qoff, U + J.uoff, g ? g + J.qoff : nullptr, lb % J.gx, J.gx, lb / J.gx);
}

template <typename V>
__global__ void k_scatter_plan(const float *q, long k, ScatterPlan sc)
{
    pdl_wait();
    pdl_trigger();
    const int b = blockIdx.y;
    for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < k; j += (long)gridDim.x * blockDim.x) {
        const int bi = sc.buf_id[j];
        const long o = (long)b * sc.cstride[bi] + sc.off[j];
        const float v = q[(long)b * k + j];
        if (sc.kind16[bi]) {
            const h16 hi = f_to_h16(v);
            reinterpret_cast<h16 *>(sc.base[bi])[o] = hi;
            if (sc.base_lo[bi])
                reinterpret_cast<h16 *>(sc.base_lo[bi])[o] = f_to_h16(v - h16_to_f(hi));
        } else {
            reinterpret_cast<float *>(sc.base[bi])[o] = v;
        }
    }
}

// One bounded wait run out on purpose: a barrier that nothing arrives at, waited on
// with the same bounded wait the pipelines use, which records the timeout in *err.
__global__ void k_expire_wait(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    fence_mbar_init();
    mbar_wait(b, 0, err, limit_ns);   // phase 0 never completes
    mbar_arrive(b);                   // complete it before the CTA exits
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult qr;
        HMC_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &qr));
        if (qr != cudaDriverEntryPointSuccess || !ptr) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            throw Fail{HMC_ERR_CUDA};
        }
        fn = reinterpret_cast<EncodeTiledFn>(ptr);
    }
    return fn;
}

// bf16 tensor [outer][mid][inner] with a (box_inner x box_mid x 1) box, 128-byte swizzle.
CUtensorMap make_map(const void *base, uint64_t inner, uint64_t mid, uint64_t outer, uint32_t box_inner,
                     uint32_t box_mid)
{
    CUtensorMap m;
    memset(&m, 0, sizeof m);
    cuuint64_t dims[3] = {inner, mid, outer};
    cuuint64_t strides[2] = {inner * 2, inner * mid * 2};
    cuuint32_t box[3] = {box_inner, box_mid, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = encode_fn()(&m, TM_H16, 3, const_cast<void *>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for dims %llu x %llu x %llu box %u x %u", (int)r,
                  (unsigned long long)inner, (unsigned long long)mid, (unsigned long long)outer, box_inner, box_mid);
        throw Fail{HMC_ERR_CUDA};
    }
    return m;
}

template <int MODE, bool A_MN, bool B_MN, bool WSPLIT>
void launch_umma(const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &b2, const Params &p, dim3 grid,
                 cudaStream_t s)
{
    static bool configured = false;
    constexpr int sm = smem_bytes(WSPLIT);
    if (!configured) {
        HMC_CK(cudaFuncSetAttribute(k_umma<MODE, A_MN, B_MN, WSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        configured = true;
    }
    static const char *names[] = {"umma_store_f32", "umma_fwd_tanh", "umma_fwd_out", "umma_bwd_tanh", "umma_bwd_first",
                                  "umma_dw",        "umma_fwd_lin",  "umma_s",       "umma_gemm_bf16"};
    static_assert(MODE >= 0 && MODE < (int)(sizeof(names) / sizeof(names[0])), "profile name");
    ProfScope ps(names[MODE], s);
    k_umma<MODE, A_MN, B_MN, WSPLIT><<<grid, NTHREADS, sm, s>>>(a, b, b2, p);
    HMC_LAUNCH_CK();
}

template <int MODE, int WIDTH, bool SPLIT, int KD = WIDTH>
void launch_layer_w(const CUtensorMap &a, const CUtensorMap &wh, const CUtensorMap &wl, const LayerParams &p, int ncta,
                    cudaStream_t s)
{
    static bool configured = false;
    if (!configured) {
        HMC_CK(cudaFuncSetAttribute(k_layer_pair<MODE, WIDTH, SPLIT, KD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    L_SMEM));
        configured = true;
    }
    static const char *names[] = {"layer_fwd_tanh", "layer_fwd_out", "layer_bwd_tanh", "layer_bwd_first",
                                  "layer_fwd_lin"};
    ProfScope ps(names[MODE], s);
    launch_pdl(k_layer_pair<MODE, WIDTH, SPLIT, KD>, dim3(ncta), dim3(L_THREADS), L_SMEM, s, a, wh, wl, p);
    HMC_LAUNCH_CK();
}

// A hidden layer on CTA pairs, forward and reverse with the weights as a hi/lo pair: the
// reverse products delta W are the forces' largest rounding error with W rounded once
// (it is the same error at every leapfrog step, so it adds up along a trajectory).
template <int MODE>
void launch_layer(const CUtensorMap &a, const CUtensorMap &wh, const CUtensorMap &wl, const LayerParams &p, int ncta,
                  cudaStream_t s)
{
    constexpr bool SPLIT = true;
    if (p.W == 256) launch_layer_w<MODE, 256, SPLIT>(a, wh, wl, p, ncta, s);
    else launch_layer_w<MODE, 128, SPLIT>(a, wh, wl, p, ncta, s);
}

// A layer product of N output features over a reduction of K on the pair kernel, for the
// shape of a DeepONet net's last layer 256 -> 128: forward (N = 128, K = 256, linear) and
// the reverse through it (N = 256, K = 128).  False for a shape it has no kernel for.
bool pair_shape_ok(int mode, int N, int K)
{
    if (mode == L_FWD_LIN) return N == 128 && K == 256;
    if (mode == L_BWD_TANH) return N == 256 && K == 128;
    return false;
}

template <int MODE>
void launch_layer_nk(const CUtensorMap &a, const CUtensorMap &wh, const CUtensorMap &wl, const LayerParams &p,
                     int ncta, cudaStream_t s)
{
    if (MODE == L_FWD_LIN) launch_layer_w<L_FWD_LIN, 128, true, 256>(a, wh, wl, p, ncta, s);
    else launch_layer_w<L_BWD_TANH, 256, true, 128>(a, wh, wl, p, ncta, s);
}

void launch_dw2(const CUtensorMap &d, const CUtensorMap &a, const Params &p, dim3 grid, cudaStream_t s)
{
    static bool configured = false;
    if (!configured) {
        HMC_CK(cudaFuncSetAttribute(k_dw2, cudaFuncAttributeMaxDynamicSharedMemorySize, DW_SMEM));
        configured = true;
    }
    ProfScope ps("dw2", s);
    launch_pdl(k_dw2, grid, dim3(NTHREADS), DW_SMEM, s, d, a, p);
    HMC_LAUNCH_CK();
}

// How many CTA pairs of the layer kernel can be resident at once.
int layer_max_clusters()
{
    auto kern = k_layer_pair<L_FWD_OUT, 256, true>;
    HMC_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L_SMEM));
    int dev = 0, sms = 0;
    HMC_CK(cudaGetDevice(&dev));
    HMC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (sms / 2), 1, 1);
    cfg.blockDim = dim3(L_THREADS, 1, 1);
    cfg.dynamicSmemBytes = L_SMEM;
    int n = 0;
    HMC_CK(cudaOccupancyMaxActiveClusters(&n, kern, &cfg));
    return std::max(1, std::min(n, sms / 2));
}

int pick_splits(int total_kb, int ctas_without_split, int target)
{
    int s = std::max(1, target / std::max(1, ctas_without_split));
    return std::min(s, total_kb);
}

class UmmaGroup;

class UmmaEngine final : public Engine {
    friend class UmmaGroup;

  public:
    UmmaEngine(Problem &p, int C) : p_(p), C_(C)
    {
        const NetDesc &nd = p.net;
        L_ = nd.L;
        // hidden widths are padded to 128 (or 256 above 128) with units whose weights and
        // biases are zero: they output tanh(0) = 0, feed nothing forward and receive no
        // delta, so U and the gradient of every real parameter are unchanged.  Widths up to
        // 128 then run on the persistent pair kernel, whose CTAs each hold half of W: at
        // 64 the reverse pass's 64-feature atoms of W^T would not split between the pair
        // (the tile kernel does run 64, with one short-lived CTA per 128 rows, and in a
        // batch of many small problems that was three times slower than padding)
        wl_ = nd.w[1];
        w_ = wl_ <= 128 ? 128 : 256;
        dx_ = nd.w[0];
        N_ = p.n;
        k_ = p.k;
        ntiles_ = (int)std::max<long>(1, (N_ + BM - 1) / BM);
        int dev = 0;
        HMC_CK(cudaGetDevice(&dev));
        HMC_CK(cudaDeviceGetAttribute(&num_sms_, cudaDevAttrMultiProcessorCount, dev));
        HMC_CK(cudaMalloc(&err_, sizeof(int)));
        HMC_CK(cudaMemset(err_, 0, sizeof(int)));

        // data
        std::vector<float> xf(p.x.begin(), p.x.end()), yf(p.y.begin(), p.y.end());
        x_.alloc(sizeof(float) * std::max<size_t>(xf.size(), 1));
        y_.alloc(sizeof(float) * std::max<size_t>(yf.size(), 1));
        if (!xf.empty()) HMC_CK(cudaMemcpy(x_.ptr, xf.data(), sizeof(float) * xf.size(), cudaMemcpyHostToDevice));
        if (!yf.empty()) HMC_CK(cudaMemcpy(y_.ptr, yf.data(), sizeof(float) * yf.size(), cudaMemcpyHostToDevice));

        // parameters per chain, initialised from the frozen vector
        const int nh = L_ - 2;   // hidden w->w layers 1..L-2
        W0_.alloc(sizeof(float) * C * w_ * dx_);
        b0_.alloc(sizeof(float) * C * w_);
        Wh_.resize(nh);
        Wl_.resize(nh);
        bh_.resize(nh);
        for (int i = 0; i < nh; ++i) {
            Wh_[i].reset(new DevBuf(sizeof(h16) * C * w_ * w_));
            Wl_[i].reset(new DevBuf(sizeof(h16) * C * w_ * w_));
            bh_[i].reset(new DevBuf(sizeof(float) * C * w_));
        }
        wout_.alloc(sizeof(float) * C * w_);
        bout_.alloc(sizeof(float) * C);
        upload_rep(W0_, nd.woff[0], wl_, dx_, w_, dx_);
        upload_rep(b0_, nd.boff[0], 1, wl_, 1, w_);
        for (int i = 0; i < nh; ++i) {
            upload_rep_h16(*Wh_[i], *Wl_[i], nd.woff[i + 1], wl_, wl_, w_, w_);
            upload_rep(*bh_[i], nd.boff[i + 1], 1, wl_, 1, w_);
        }
        upload_rep(wout_, nd.woff[L_ - 1], 1, wl_, 1, w_);
        upload_rep(bout_, nd.boff[L_ - 1], 1, 1, 1, 1);

        // activations A_1..A_{L-2} and deltas delta_2..delta_{L-1}
        const size_t act_bytes = sizeof(h16) * C * std::max<long>(N_, 1) * w_;
        A_.resize(L_);   // index i = 1..L-2
        D_.resize(L_);   // index i = 2..L-1
        for (int i = 1; i <= L_ - 2; ++i) {
            A_[i].reset(new DevBuf());
            row_alloc(p.arena, *A_[i], act_bytes);
        }
        for (int i = 2; i <= L_ - 1; ++i) {
            D_[i].reset(new DevBuf());
            row_alloc(p.arena, *D_[i], act_bytes);
        }

        // partials
        u_part_.alloc(sizeof(double) * C * ntiles_);
        dbout_part_.alloc(sizeof(float) * C * ntiles_);
        dwout_part_.alloc(sizeof(float) * C * ntiles_ * w_);
        dw0_part_.alloc(sizeof(float) * C * ntiles_ * w_ * dx_);
        db_part_.resize(L_ - 1);   // biases of layers 0..L-2, per-tile column sums
        for (int l = 0; l <= L_ - 2; ++l) db_part_[l].reset(new DevBuf(sizeof(float) * C * ntiles_ * w_));
        // the persistent pair kernels keep the first layer's column sums in 20 KB (dx <= 4 at
        // w = 256) and form them from an 8-column [X | 1] block (dx <= 7)
        use_layer_ = (w_ == 128 && dx_ <= 7) || (w_ == 256 && dx_ <= 4);

        // per-entry metadata, scatter plan, per-layer CSR of the sampled hidden weights
        build_entries();

        // split of the weight-gradient GEMMs over rows: about two CTAs per SM
        const int total_kb = (int)((N_ + BK - 1) / BK);
        nsplit_ = pick_splits(total_kb, ((w_ + BM - 1) / BM) * C, 2 * num_sms_);
        nsplit2_ = pick_splits(total_kb, (w_ / 128) * (w_ / 128) * C, 2 * num_sms_);
        // the autotuner may pick any row-split count up to kMaxSplits for the persistent path
        const int max_splits = use_layer_ ? std::min(kMaxSplits, total_kb) : 1;
        nsplit_ = std::max(std::max(nsplit_, nsplit2_), max_splits);
        gw_part_.alloc(sizeof(float) * nsplit_ * C * std::max<long>(k_, 1));
        HMC_CK(cudaMemset(gw_part_.ptr, 0, gw_part_.n));
        dbw_part_.resize(L_ - 1);
        for (int l = 1; use_layer_ && l <= L_ - 2; ++l)
            dbw_part_[l].reset(new DevBuf(sizeof(float) * nsplit_ * C * w_));

        // tensor maps
        if (use_layer_) max_clusters_ = layer_max_clusters();
        for (int i = 1; i <= L_ - 2; ++i) {
            A_row_[i] = make_map(A_[i]->ptr, w_, N_, C, 64, 128);
            A_atom_[i] = make_map(A_[i]->ptr, w_, N_, C, 64, 64);
            W_fwd_[i] = make_map(Wh_[i - 1]->ptr, w_, w_, C, 64, w_);
            W_atom_[i] = make_map(Wh_[i - 1]->ptr, w_, w_, C, 64, 64);
            W_fwd_lo_[i] = make_map(Wl_[i - 1]->ptr, w_, w_, C, 64, w_);
            W_atom_lo_[i] = make_map(Wl_[i - 1]->ptr, w_, w_, C, 64, 64);
            if (use_layer_) {
                W_half_hi_[i] = make_map(Wh_[i - 1]->ptr, w_, w_, C, 64, w_ / 2);
                W_half_lo_[i] = make_map(Wl_[i - 1]->ptr, w_, w_, C, 64, w_ / 2);
            }
        }
        for (int i = 2; i <= L_ - 1; ++i) {
            D_row_[i] = make_map(D_[i]->ptr, w_, N_, C, 64, 128);
            D_atom_[i] = make_map(D_[i]->ptr, w_, N_, C, 64, 64);
        }
        if (use_layer_ && p.batch_member) {
            // in a batch the weight-gradient launch covers many problems (grouped) or runs
            // beside them (lanes), so a split is sized for its own work, 16 K-blocks (1024
            // rows) or more, not for filling the GPU alone: fewer partials to write and sum
            nsplit2_ = std::max(1, std::min(kMaxSplits, (total_kb + 15) / 16));
            tuning_ = "dw row splits " + std::to_string(nsplit2_) + " (batch member: 16 K-blocks per split)";
        } else if (use_layer_) {
            tune_dw_splits(total_kb);
        }

        // bias gradients: the first layer's from its reverse kernel (per tile); the hidden
        // layers' from the weight-gradient kernel (per row split) on the persistent path
        // descriptors 0..L-2: biases; L-1: first-layer weights; L: output weights; L+1: output bias
        std::vector<DbDesc> dbd(L_ + 2);
        for (int l = 0; l <= L_ - 2; ++l) {
            dbd[l] = DbDesc{db_part_[l]->as<float>(), (long)ntiles_ * w_, w_, ntiles_};
            if (use_layer_ && l >= 1) dbd[l] = DbDesc{dbw_part_[l]->as<float>(), w_, (long)C * w_, nsplit_eff()};
        }
        dbd[L_ - 1] = DbDesc{dw0_part_.as<float>(), (long)ntiles_ * w_ * dx_, (long)w_ * dx_, ntiles_};
        dbd[L_] = DbDesc{dwout_part_.as<float>(), (long)ntiles_ * w_, w_, ntiles_};
        dbd[L_ + 1] = DbDesc{dbout_part_.as<float>(), ntiles_, 1, ntiles_};
        db_desc_.alloc(sizeof(DbDesc) * dbd.size());
        HMC_CK(cudaMemcpy(db_desc_.ptr, dbd.data(), sizeof(DbDesc) * dbd.size(), cudaMemcpyHostToDevice));
        {   // entries with per-tile partials are summed a warp each
            const std::vector<int> heavy = mark_heavy(kind_h_, layer_h_, dbd);
            nheavy_ = (int)heavy.size();
            HMC_CK(cudaMemcpy(kind_.ptr, kind_h_.data(), sizeof(int) * kind_h_.size(), cudaMemcpyHostToDevice));
            heavy_.alloc(sizeof(int) * std::max<size_t>(heavy.size(), 1));
            if (nheavy_) HMC_CK(cudaMemcpy(heavy_.ptr, heavy.data(), sizeof(int) * heavy.size(), cudaMemcpyHostToDevice));
        }
    }

    std::string tuning() const override { return tuning_; }

    ~UmmaEngine() override
    {
        if (err_) cudaFree(err_);
        if (ev_fork_) cudaEventDestroy(ev_fork_);
        if (ev_join_) cudaEventDestroy(ev_join_);
        if (s2_) cudaStreamDestroy(s2_);
    }

    size_t bytes() const override { return 0; }

    ScatterPlan scatter_plan() override { return plan_; }
    int *error_flag() const override { return err_; }

    void scatter(const void *qv, cudaStream_t s) override
    {
        dim3 grid((unsigned)std::min<long>((k_ + 255) / 256, 1024), C_);
        ProfScope ps("scatter", s);
        launch_pdl(k_scatter_plan<float>, grid, dim3(256), 0, s, static_cast<const float *>(qv), k_, plan_);
    }

    void energy_grad(const void *qv, double *U, void *gv, bool scattered, cudaStream_t s) override
    {
        const float *q = static_cast<const float *>(qv);
        float *g = static_cast<float *>(gv);
        if (!scattered) scatter(qv, s);
        const NetDesc &nd = p_.net;
        // first layer
        {
            dim3 grid((unsigned)ntiles_, C_);
            ProfScope ps("first_fwd", s);
            launch_first_fwd(dx_, grid, s, x_.as<float>(), (int)N_, w_, W0_.as<float>(), b0_.as<float>(),
                             A_[1]->as<h16>());
        }
        if (use_layer_) {
            layers_persistent(s);
        } else {
            const dim3 row_grid(ntiles_, 1, C_);
            // hidden layers i = 1..L-3 (tanh), then layer L-2 fused with the output layer
            for (int i = 1; i <= L_ - 2; ++i) {
                const Params pp = tile_fwd_params(i);
                if (i < L_ - 2)
                    launch_umma<M_FWD_TANH, false, false, true>(A_row_[i], W_fwd_[i], W_fwd_lo_[i], pp, row_grid, s);
                else
                    launch_umma<M_FWD_OUT, false, false, true>(A_row_[i], W_fwd_[i], W_fwd_lo_[i], pp, row_grid, s);
            }
            // reverse: delta_i = (delta_{i+1} W_i) (1 - A_i^2) for i = L-2 .. 1 (down to the lowest sampled layer)
            for (int i = L_ - 2; i >= 1; --i) {
                if (i <= nd.lmin) break;   // no layer below i holds a sampled parameter
                const Params pp = tile_bwd_params(i);
                if (i > 1)
                    launch_umma<M_BWD_TANH, false, true, true>(D_row_[i + 1], W_atom_[i], W_atom_lo_[i], pp, row_grid, s);
                else
                    launch_umma<M_BWD_FIRST, false, true, true>(D_row_[i + 1], W_atom_[i], W_atom_lo_[i], pp, row_grid, s);
            }
            // weight gradients of the hidden layers at the sampled entries (the persistent path
            // launches each one next to the reverse kernel that reads the same delta)
            for (int i = 1; i <= L_ - 2; ++i) dw_layer(i, s);
        }
        const FinalArgs fa = final_args();
        {
            ProfScope ps("finalize", s);
            launch_pdl(k_finalize_bf16, dim3((unsigned)final_blocks(), C_), dim3(256), 0, s, fa, q, U, g);
            HMC_LAUNCH_CK();
        }
    }

    // ---- launch descriptions, shared by energy_grad and the grouped launches ----

    // the tile kernel's parameters for hidden layer i, forward (tanh, or fused with the
    // output layer at i = L-2) and reverse (to delta_i, or fused with the first layer's
    // gradients at i = 1)
    Params tile_fwd_params(int i) const
    {
        Params pp{};
        pp.err = err_;
        pp.ntiles = ntiles_;
        pp.M = (int)N_;
        pp.N = w_;
        pp.K = w_;
        pp.kb_per_split = (w_ + BK - 1) / BK;
        pp.bias = bh_[i - 1]->as<float>();
        pp.bias_b = w_;
        pp.out_b = N_ * (long)w_;
        if (i < L_ - 2) {
            pp.out = A_[i + 1]->as<h16>();
        } else {
            pp.out = D_[L_ - 1]->as<h16>();
            pp.wout = wout_.as<float>();
            pp.wout_b = w_;
            pp.bout = bout_.as<float>();
            pp.y = y_.as<float>();
            pp.inv_s2 = (float)delta_scale(p_.sigma);
            pp.u_part = u_part_.as<double>();
            pp.dbout_part = dbout_part_.as<float>();
            pp.dwout_part = dwout_part_.as<float>();
            pp.db_part = db_part_[L_ - 2]->as<float>();
        }
        return pp;
    }

    Params tile_bwd_params(int i) const
    {
        Params pp{};
        pp.err = err_;
        pp.ntiles = ntiles_;
        pp.M = (int)N_;
        pp.N = w_;
        pp.K = w_;
        pp.kb_per_split = (w_ + BK - 1) / BK;
        pp.aux = A_[i]->as<h16>();
        pp.aux_b = N_ * (long)w_;
        pp.db_part = db_part_[i - 1]->as<float>();
        if (i > 1) {
            pp.out = D_[i]->as<h16>();
            pp.out_b = N_ * (long)w_;
        } else {
            pp.x = x_.as<float>();
            pp.dx = dx_;
            pp.dw0_part = dw0_part_.as<float>();
        }
        return pp;
    }

    FinalArgs final_args() const
    {
        FinalArgs fa{};
        fa.k = (int)k_;
        fa.nsplit = nsplit_eff();
        fa.nu = ntiles_;
        fa.kind = kind_.as<int>();
        fa.desc = layer_.as<int>();
        fa.off = off_.as<int>();
        fa.u_part = u_part_.as<double>();
        fa.gw_part = gw_part_.as<float>();
        fa.gw_split = (long)C_ * k_;
        fa.db = db_desc_.as<const DbDesc>();
        fa.half_inv_s2 = 0.5 / (p_.sigma * p_.sigma);
        fa.gscale = (float)(1.0 / (p_.sigma * p_.sigma) / delta_scale(p_.sigma));
        fa.inv_a2 = 1.0 / (p_.alpha * p_.alpha);
        fa.heavy = heavy_.as<int>();
        fa.nheavy = nheavy_;
        fa.nlight = (int)((k_ + 255) / 256);
        return fa;
    }

    // finalize blocks per chain: the light entries, the heavy ones (a warp each), U
    int final_blocks() const { return (int)((k_ + 255) / 256) + (nheavy_ + 7) / 8 + 1; }

    bool has_accurate_energy() const override { return true; }

    // U(q) from the hi/lo-activation forward pass; the activation and delta buffers are
    // free after the gradient that preceded it: a_i's hi part goes to A_i, its lo part to D_{i+1}
    void accurate_energy(const void *qv, double *U, cudaStream_t s) override
    {
        const float *q = static_cast<const float *>(qv);
        {
            dim3 grid((unsigned)ntiles_, C_);
            ProfScope ps("first_fwd3", s);
            launch_pdl(k_first_fwd3, grid, dim3(256), 0, s, x_.as<float>(), dx_, (int)N_, w_, W0_.as<float>(),
                       b0_.as<float>(), A_[1]->as<h16>(), D_[2]->as<h16>());
        }
        for (int i = 1; i <= L_ - 2; ++i) {
            E3Params e{};
            e.M = (int)N_;
            e.N = w_;
            e.K = w_;
            e.ntiles = ntiles_;
            e.err = err_;
            e.bias = bh_[i - 1]->as<float>();
            const dim3 grid(ntiles_, 1, C_);
            if (i < L_ - 2) {
                e.out_hi = A_[i + 1]->as<h16>();
                e.out_lo = D_[i + 2]->as<h16>();
                launch_energy3<E3_TANH>(A_row_[i], D_row_[i + 1], W_fwd_[i], W_fwd_lo_[i], e, grid, s);
            } else {
                e.wout = wout_.as<float>();
                e.bout = bout_.as<float>();
                e.y = y_.as<float>();
                e.u_part = u_part_.as<double>();
                launch_energy3<E3_OUT>(A_row_[i], D_row_[i + 1], W_fwd_[i], W_fwd_lo_[i], e, grid, s);
            }
        }
        FinalArgs fa{};
        fa.k = (int)k_;
        fa.nu = ntiles_;
        fa.u_part = u_part_.as<double>();
        fa.half_inv_s2 = 0.5 / (p_.sigma * p_.sigma);
        fa.gscale = (float)(1.0 / (p_.sigma * p_.sigma) / delta_scale(p_.sigma));
        fa.inv_a2 = 1.0 / (p_.alpha * p_.alpha);
        ProfScope ps("energy3_final", s);
        launch_pdl(k_finalize_bf16, dim3(1, C_), dim3(256), 0, s, fa, q, U, (float *)nullptr);
    }

  private:
    // Autotuner for the weight-gradient grid: time each row-split count on this engine's
    // own buffers (one warm-up, three timed launches, CUDA events) and keep the fastest;
    // the choice is cached per (rows, width, chains) for the process.
    void tune_dw_splits(int total_kb)
    {
        if (!autotune_enabled()) {
            tuning_ = "dw row splits " + std::to_string(nsplit2_) + " (heuristic; autotuner off)";
            return;
        }
        int layer = -1;
        for (int i = 1; i <= L_ - 2 && layer < 0; ++i)
            if (layer_entries_[i] > 0 || bias_entries_[i] > 0) layer = i;
        if (layer < 0) return;
        static std::mutex mu;
        static std::map<std::tuple<long, int, int>, int> cache;
        const auto key = std::make_tuple(N_, w_, C_);
        {
            std::lock_guard<std::mutex> g(mu);
            auto it = cache.find(key);
            if (it != cache.end()) {
                nsplit2_ = it->second;
                tuning_ = "dw row splits " + std::to_string(nsplit2_) + " (cached)";
                return;
            }
        }
        cudaStream_t s;
        cudaEvent_t a, b;
        HMC_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        HMC_CK(cudaEventCreate(&a));
        HMC_CK(cudaEventCreate(&b));
        int best = nsplit2_;
        float best_ms = 1e30f;
        std::string log;
        for (int cand : {1, 2, 4, 8, 16, 32}) {
            if (cand > std::min(kMaxSplits, total_kb)) break;
            nsplit2_ = cand;
            dw_layer(layer, s);
            HMC_CK(cudaEventRecord(a, s));
            for (int r = 0; r < 3; ++r) dw_layer(layer, s);
            HMC_CK(cudaEventRecord(b, s));
            HMC_CK(cudaEventSynchronize(b));
            float ms = 0.0f;
            HMC_CK(cudaEventElapsedTime(&ms, a, b));
            ms /= 3.0f;
            char buf[48];
            snprintf(buf, sizeof buf, "%s%d:%.1fus", log.empty() ? "" : " ", cand, 1000.0f * ms);
            log += buf;
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        HMC_CK(cudaStreamSynchronize(s));
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaStreamDestroy(s);
        HMC_CK(cudaMemset(gw_part_.ptr, 0, gw_part_.n));
        nsplit2_ = best;
        tuning_ = "dw row splits " + std::to_string(best) + " of {" + log + "}";
        std::lock_guard<std::mutex> g(mu);
        cache[key] = best;
    }

    // weight gradient of hidden layer i (dW = delta_{i+1}^T A_i) at its sampled entries
    // The weight gradient of hidden layer i at the sampled entries (nothing when the layer
    // holds none): its kernel's parameters, grid and operand maps (deltas, activations).
    bool dw_params(int i, Params &pp, dim3 &grid, const CUtensorMap *&md, const CUtensorMap *&ma) const
    {
        if (layer_entries_[i] == 0 && !(use_layer_ && bias_entries_[i] > 0)) return false;
        pp = Params{};
        pp.err = err_;
        pp.ntiles = ntiles_;
        pp.M = w_;
        pp.N = w_;
        pp.K = (int)N_;
        const int total_kb = (int)((N_ + BK - 1) / BK);
        pp.kb_per_split = (total_kb + nsplit_ - 1) / nsplit_;
        pp.rowptr = rowptr_[i]->as<int>();
        pp.ecol = ecol_.as<int>();
        pp.erow = erow_.as<int>();
        pp.epack = epack_.as<int>();
        pp.gw_part = gw_part_.as<float>();
        pp.gw_split = (long)C_ * k_;
        pp.gw_b = k_;
        if (use_layer_) {
            pp.kb_per_split = (total_kb + nsplit2_ - 1) / nsplit2_;
            const int splits = (total_kb + pp.kb_per_split - 1) / pp.kb_per_split;
            pp.db_part = dbw_part_[i]->as<float>();
            pp.db_split = (long)C_ * w_;
            grid = dim3((w_ / 128) * (w_ / 128), splits, C_);
        } else {
            const int splits = (total_kb + pp.kb_per_split - 1) / pp.kb_per_split;
            grid = dim3((w_ + BM - 1) / BM, splits, C_);
        }
        md = &D_atom_[i + 1];
        ma = &A_atom_[i];
        return true;
    }

    void dw_layer(int i, cudaStream_t s)
    {
        Params pp;
        dim3 grid;
        const CUtensorMap *md, *ma;
        if (!dw_params(i, pp, grid, md, ma)) return;
        if (use_layer_) launch_dw2(*md, *ma, pp, grid, s);
        else launch_umma<M_DW, true, true, false>(*md, *ma, *ma, pp, grid, s);
    }

    // the persistent layer kernel's parameters for hidden layer i, forward and reverse
    LayerParams layer_fwd_params(int i) const
    {
        LayerParams lp = layer_base();
        lp.bias = bh_[i - 1]->as<float>();
        if (i < L_ - 2) {
            lp.out = A_[i + 1]->as<h16>();
        } else {
            lp.out = D_[L_ - 1]->as<h16>();
            lp.wout = wout_.as<float>();
            lp.bout = bout_.as<float>();
            lp.y = y_.as<float>();
            lp.inv_s2 = (float)delta_scale(p_.sigma);
            lp.u_part = u_part_.as<double>();
            lp.dbout_part = dbout_part_.as<float>();
            lp.dwout_part = dwout_part_.as<float>();
        }
        return lp;
    }

    LayerParams layer_bwd_params(int i) const
    {
        LayerParams lp = layer_base();
        lp.aux = A_[i]->as<h16>();
        if (i > 1) {
            lp.out = D_[i]->as<h16>();
        } else {
            lp.db_part = db_part_[0]->as<float>();
            lp.x = x_.as<float>();
            lp.dw0_part = dw0_part_.as<float>();
        }
        return lp;
    }

    LayerParams layer_base() const
    {
        LayerParams lp{};
        lp.N = (int)N_;
        lp.W = w_;
        lp.C = C_;
        lp.ntiles = ntiles_;
        lp.dx = dx_;
        lp.err = err_;
        return lp;
    }

    // (chain, tile pair) units of one layer launch
    long layer_units() const { return (long)C_ * ((ntiles_ + 1) / 2); }

    // forward and reverse hidden layers on the persistent cluster kernel
    void layers_persistent(cudaStream_t s)
    {
        const NetDesc &nd = p_.net;
        const int ncta = 2 * (int)std::min<long>(max_clusters_, layer_units());
        for (int i = 1; i <= L_ - 2; ++i) {
            const LayerParams lp = layer_fwd_params(i);
            if (i < L_ - 2) launch_layer<L_FWD_TANH>(A_row_[i], W_half_hi_[i], W_half_lo_[i], lp, ncta, s);
            else launch_layer<L_FWD_OUT>(A_row_[i], W_half_hi_[i], W_half_lo_[i], lp, ncta, s);
        }
        // reverse pass (W as a hi/lo pair, like the forward pass); the weight gradient of
        // layer i reads the same delta and activations as the reverse kernel of layer i and
        // writes nothing it reads: it runs beside it on the engine's second stream, which
        // joins back before the finalize (on one stream while a per-kernel profile runs, so
        // that each launch is timed alone)
        if (!s2_) {
            HMC_CK(cudaStreamCreateWithFlags(&s2_, cudaStreamNonBlocking));
            HMC_CK(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
            HMC_CK(cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming));
        }
        const cudaStream_t sw = active_profiler() ? s : s2_;
        for (int i = L_ - 2; i >= 1; --i) {
            if (sw != s) {
                HMC_CK(cudaEventRecord(ev_fork_, s));
                HMC_CK(cudaStreamWaitEvent(sw, ev_fork_, 0));
            }
            dw_layer(i, sw);
            if (i <= nd.lmin) break;
            const LayerParams lp = layer_bwd_params(i);
            if (i > 1) launch_layer<L_BWD_TANH>(D_row_[i + 1], W_atom_[i], W_atom_lo_[i], lp, ncta, s);
            else launch_layer<L_BWD_FIRST>(D_row_[i + 1], W_atom_[i], W_atom_lo_[i], lp, ncta, s);
        }
        if (sw != s) {
            HMC_CK(cudaEventRecord(ev_join_, sw));
            HMC_CK(cudaStreamWaitEvent(s, ev_join_, 0));
        }
    }

    int nsplit_eff() const
    {
        const int total_kb = (int)((N_ + BK - 1) / BK);
        const int ns = use_layer_ ? nsplit2_ : nsplit_;
        const int per = (total_kb + ns - 1) / ns;
        return (total_kb + per - 1) / per;
    }

    // the frozen [rows][cols] block at `off`, zero-padded to [prow][pcol], for every chain
    void upload_rep(DevBuf &dst, long off, int rows, int cols, int prow, int pcol)
    {
        const long count = (long)prow * pcol;
        std::vector<float> v(C_ * count, 0.0f);
        for (int c = 0; c < C_; ++c)
            for (int r = 0; r < rows; ++r)
                for (int i = 0; i < cols; ++i) v[c * count + (long)r * pcol + i] = (float)p_.frozen[off + (long)r * cols + i];
        HMC_CK(cudaMemcpy(dst.ptr, v.data(), sizeof(float) * v.size(), cudaMemcpyHostToDevice));
    }

    // W = hi + lo with hi = h16(W) and lo = h16(W - hi), W taken in float32, zero-padded
    void upload_rep_h16(DevBuf &hi, DevBuf &lo, long off, int rows, int cols, int prow, int pcol)
    {
        const long count = (long)prow * pcol;
        std::vector<h16> vh(C_ * count, f_to_h16(0.0f)), vl(C_ * count, f_to_h16(0.0f));
        for (int c = 0; c < C_; ++c)
            for (int r = 0; r < rows; ++r)
                for (int i = 0; i < cols; ++i) {
                    const float w = (float)p_.frozen[off + (long)r * cols + i];
                    const h16 h = f_to_h16(w);
                    vh[c * count + (long)r * pcol + i] = h;
                    vl[c * count + (long)r * pcol + i] = f_to_h16(w - h16_to_f(h));
                }
        HMC_CK(cudaMemcpy(hi.ptr, vh.data(), sizeof(h16) * vh.size(), cudaMemcpyHostToDevice));
        HMC_CK(cudaMemcpy(lo.ptr, vl.data(), sizeof(h16) * vl.size(), cudaMemcpyHostToDevice));
    }

    void build_entries()
    {
        const NetDesc &nd = p_.net;
        std::vector<int> kind(k_), layer(k_), off(k_), erow(k_, 0), ecol(k_, 0), bid(k_), boff(k_);
        std::vector<std::vector<int>> rp(L_, std::vector<int>(w_ + 1, 0));
        layer_entries_.assign(L_, 0);
        bias_entries_.assign(L_, 0);
        // scatter buffers: 0 W0, 1 b0, 2+2(i-1) W_i (bf16), 3+2(i-1) b_i, then wout, bout
        const int nh = L_ - 2;
        plan_.nbuf = 2 + 2 * nh + 2;
        HMC_REQUIRE(plan_.nbuf <= MAX_SCATTER_BUFS, "too many layers for the scatter plan");
        plan_.base[0] = W0_.ptr; plan_.cstride[0] = (long)w_ * dx_; plan_.kind16[0] = 0;
        plan_.base[1] = b0_.ptr; plan_.cstride[1] = w_; plan_.kind16[1] = 0;
        for (int i = 1; i <= nh; ++i) {
            plan_.base[2 + 2 * (i - 1)] = Wh_[i - 1]->ptr;
            plan_.cstride[2 + 2 * (i - 1)] = (long)w_ * w_;
            plan_.kind16[2 + 2 * (i - 1)] = H16_KIND;
            plan_.base_lo[2 + 2 * (i - 1)] = Wl_[i - 1]->ptr;
            plan_.base[3 + 2 * (i - 1)] = bh_[i - 1]->ptr;
            plan_.cstride[3 + 2 * (i - 1)] = w_;
            plan_.kind16[3 + 2 * (i - 1)] = 0;
        }
        plan_.base[2 + 2 * nh] = wout_.ptr; plan_.cstride[2 + 2 * nh] = w_; plan_.kind16[2 + 2 * nh] = 0;
        plan_.base[3 + 2 * nh] = bout_.ptr; plan_.cstride[3 + 2 * nh] = 1; plan_.kind16[3 + 2 * nh] = 0;
        for (long j = 0; j < k_; ++j) {
            const long id = p_.idx[j];
            int l = 0;
            while (l + 1 < L_ && id >= nd.woff[l + 1]) ++l;
            const long wend = nd.woff[l] + (long)nd.w[l + 1] * nd.w[l];
            const bool is_w = id < wend;
            const long rel = is_w ? id - nd.woff[l] : id - nd.boff[l];
            const int in = nd.w[l];
            if (l == 0) {
                kind[j] = E_PART;
                layer[j] = is_w ? L_ - 1 : 0;
                off[j] = (int)rel;   // o*dx + d, or o
                bid[j] = is_w ? 0 : 1;
                boff[j] = (int)rel;
            } else if (l == L_ - 1) {
                kind[j] = E_PART;
                layer[j] = is_w ? L_ : L_ + 1;
                off[j] = is_w ? (int)rel : 0;
                bid[j] = is_w ? 2 + 2 * nh : 3 + 2 * nh;
                boff[j] = is_w ? (int)rel : 0;
            } else {
                if (is_w) {
                    kind[j] = E_GW;
                    erow[j] = (int)(rel / in);
                    ecol[j] = (int)(rel % in);
                    rp[l][erow[j] + 1]++;
                    layer_entries_[l]++;
                    bid[j] = 2 + 2 * (l - 1);
                    boff[j] = erow[j] * w_ + ecol[j];   // in the padded [w_][w_] layout
                } else {
                    kind[j] = E_PART;
                    layer[j] = l;
                    off[j] = (int)rel;
                    bias_entries_[l]++;
                    bid[j] = 3 + 2 * (l - 1);
                    boff[j] = (int)rel;
                }
            }
        }
        // row pointers: entries are ascending in parameter index, so a layer's weight entries
        // are contiguous and sorted by (row, column); rowptr holds absolute entry indices
        rowptr_.resize(L_);
        for (int l = 1; l <= L_ - 2; ++l) {
            long first = std::lower_bound(p_.idx.begin(), p_.idx.end(), nd.woff[l]) - p_.idx.begin();
            std::vector<int> r(w_ + 1);
            r[0] = (int)first;
            for (int o = 0; o < w_; ++o) r[o + 1] = r[o] + rp[l][o + 1];
            rowptr_[l].reset(new DevBuf(sizeof(int) * (w_ + 1)));
            HMC_CK(cudaMemcpy(rowptr_[l]->ptr, r.data(), sizeof(int) * (w_ + 1), cudaMemcpyHostToDevice));
        }
        auto up = [&](DevBuf &d, const std::vector<int> &v) {
            d.alloc(sizeof(int) * std::max<size_t>(v.size(), 1));
            if (!v.empty()) HMC_CK(cudaMemcpy(d.ptr, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice));
        };
        up(kind_, kind);
        up(layer_, layer);
        up(off_, off);
        up(erow_, erow);
        up(ecol_, ecol);
        kind_h_ = kind;
        layer_h_ = layer;
        std::vector<int> epack(k_);
        for (long j = 0; j < k_; ++j) epack[j] = (erow[j] << 16) | ecol[j];
        up(epack_, epack);
        up(sc_off_, boff);
        std::vector<uint8_t> b8(bid.begin(), bid.end());
        sc_bid_.alloc(std::max<size_t>(b8.size(), 1));
        HMC_CK(cudaMemcpy(sc_bid_.ptr, b8.data(), b8.size(), cudaMemcpyHostToDevice));
        plan_.buf_id = sc_bid_.as<uint8_t>();
        plan_.off = sc_off_.as<int>();
    }

    Problem &p_;
    int C_, L_ = 0, w_ = 0, wl_ = 0, dx_ = 0, ntiles_ = 1, nsplit_ = 1, nsplit2_ = 1, num_sms_ = 148;
    long N_ = 0, k_ = 0;
    int *err_ = nullptr;
    DevBuf x_, y_, W0_, b0_, wout_, bout_, u_part_, dbout_part_, dwout_part_, dw0_part_, db_desc_, gw_part_;
    DevBuf kind_, layer_, off_, erow_, ecol_, epack_, sc_off_, sc_bid_, heavy_;
    std::vector<int> kind_h_, layer_h_;
    int nheavy_ = 0;
    std::vector<std::unique_ptr<DevBuf>> Wh_, Wl_, bh_, A_, D_, db_part_, dbw_part_, rowptr_;
    std::vector<int> layer_entries_, bias_entries_;
    CUtensorMap A_row_[MAXL], A_atom_[MAXL], W_fwd_[MAXL], W_atom_[MAXL], W_fwd_lo_[MAXL], W_atom_lo_[MAXL];
    CUtensorMap D_row_[MAXL], D_atom_[MAXL], W_half_hi_[MAXL], W_half_lo_[MAXL];
    bool use_layer_ = false;
    int max_clusters_ = 1;
    cudaStream_t s2_ = nullptr;   // the weight gradients' stream inside an evaluation
    cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
    ScatterPlan plan_;
    std::string tuning_;
};

// ---------------------------------------------------------------------------
// Grouped gradients of a batch of MLP problems (one shape class: padded width, input
// width, kernel family).  Per gradient evaluation the group issues one launch per
// kernel and layer slot for all its problems:
//   first layer                         one launch
//   hidden forward, slot s = 1..S       problem e runs its layer i = s - (S - n_e) there
//                                       (n_e hidden w x w layers), so every problem's
//                                       output-fused layer falls in the last slot
//   reverse, layer i = S..1             every problem with that layer (above its lowest
//                                       sampled layer); the first-layer reverse is the
//                                       last launch for all
//   weight gradients                    one launch over every (problem, layer) pair
//   finalize                            one launch
// Each launch walks a job table (one entry per problem) and runs each problem's own
// kernel body on its own buffers, so the group's U and grad U equal the problems'
// separate evaluations bit for bit.
// ---------------------------------------------------------------------------
class UmmaGroup final : public EngineGroup {
  public:
    UmmaGroup(const std::vector<UmmaEngine *> &es, const std::vector<long> &qoff, const std::vector<long> &uoff)
        : es_(es), qoff_(qoff), uoff_(uoff)
    {
        const UmmaEngine &e0 = *es_[0];
        w_ = e0.w_;
        dx_ = e0.dx_;
        persistent_ = e0.use_layer_;
        int S = 0;
        for (const UmmaEngine *e : es_) S = std::max(S, e->L_ - 2);
        add_first();
        for (int s = 1; s <= S; ++s) {   // forward slots, aligned on the last layer
            std::vector<std::pair<const UmmaEngine *, int>> tanh_l, out_l;
            for (const UmmaEngine *e : es_) {
                const int n = e->L_ - 2, i = s - (S - n);
                if (i >= 1) (i < n ? tanh_l : out_l).push_back({e, i});
            }
            add_layers(true, false, tanh_l);
            add_layers(true, true, out_l);
        }
        for (int i = S; i >= 1; --i) {   // reverse, by layer index
            std::vector<std::pair<const UmmaEngine *, int>> l;
            for (const UmmaEngine *e : es_)
                if (i <= e->L_ - 2 && i > e->p_.net.lmin) l.push_back({e, i});
            add_layers(false, i == 1, l);
        }
        add_dw();
        add_final();
    }

    void energy_grad(const void *qv, double *U, void *gv, bool scattered, cudaStream_t s) override
    {
        const float *q = static_cast<const float *>(qv);
        float *g = static_cast<float *>(gv);
        if (!scattered)
            for (size_t e = 0; e < es_.size(); ++e) es_[e]->scatter(q + qoff_[e], s);
        for (const Launch &l : seq_) run(l, q, U, g, s);
    }

    std::string describe() const override
    {
        return std::to_string(es_.size()) + " problems, width " + std::to_string(w_) + ", dx " + std::to_string(dx_) +
               (persistent_ ? ", persistent layer kernel" : ", tile kernel") + ": " + std::to_string(seq_.size()) +
               " launches per gradient";
    }

    size_t launches() const { return seq_.size(); }

    // engines of one class can share launches: padded width, input width, kernel family
    static std::tuple<int, int, bool> shape_class(const UmmaEngine &e) { return std::make_tuple(e.w_, e.dx_, e.use_layer_); }

  private:
    enum Kind { K_FIRST, K_LAYER, K_TILE, K_DW2, K_DWT, K_FINAL };
    struct Launch {
        Kind kind;
        int mode;          // K_LAYER: LMode; K_TILE: Mode
        int njobs;
        long work;         // K_LAYER: units; otherwise blocks
        std::shared_ptr<DevBuf> jobs;
    };

    template <typename J> std::shared_ptr<DevBuf> upload(const std::vector<J> &v)
    {
        auto d = std::make_shared<DevBuf>(sizeof(J) * v.size());
        HMC_CK(cudaMemcpy(d->ptr, v.data(), sizeof(J) * v.size(), cudaMemcpyHostToDevice));
        return d;
    }

    void add_first()
    {
        std::vector<FirstJob> v;
        int b = 0;
        for (const UmmaEngine *e : es_) {
            v.push_back(FirstJob{e->x_.as<float>(), e->W0_.as<float>(), e->b0_.as<float>(), e->A_[1]->as<h16>(),
                                 (int)e->N_, e->w_, e->ntiles_, b});
            b += e->ntiles_ * e->C_;
        }
        seq_.push_back(Launch{K_FIRST, 0, (int)v.size(), b, upload(v)});
    }

    // hidden layer i of each listed problem: forward (special: fused with the output
    // layer) or reverse (special: fused with the first layer's gradients)
    void add_layers(bool fwd, bool special, const std::vector<std::pair<const UmmaEngine *, int>> &l)
    {
        if (l.empty()) return;
        int *err = es_[0]->err_;   // one flag for the launch; hmc_check reads every engine's
        if (persistent_) {
            std::vector<LayerJob> v;
            long u = 0;
            for (auto &pr : l) {
                const UmmaEngine &e = *pr.first;
                const int i = pr.second;
                LayerJob j;
                memset(&j, 0, sizeof j);
                if (fwd) {
                    j.tmA = e.A_row_[i];
                    j.tmWh = e.W_half_hi_[i];
                    j.tmWl = e.W_half_lo_[i];
                    j.p = e.layer_fwd_params(i);
                } else {
                    j.tmA = e.D_row_[i + 1];
                    j.tmWh = e.W_atom_[i];
                    j.tmWl = e.W_atom_lo_[i];
                    j.p = e.layer_bwd_params(i);
                }
                j.p.err = err;
                j.ustart = u;
                u += e.layer_units();
                v.push_back(j);
            }
            const int mode = fwd ? (special ? L_FWD_OUT : L_FWD_TANH) : (special ? L_BWD_FIRST : L_BWD_TANH);
            seq_.push_back(Launch{K_LAYER, mode, (int)v.size(), u, upload(v)});
        } else {
            std::vector<GridJob> v;
            int b = 0;
            for (auto &pr : l) {
                const UmmaEngine &e = *pr.first;
                const int i = pr.second;
                GridJob j;
                memset(&j, 0, sizeof j);
                if (fwd) {
                    j.tm[0] = e.A_row_[i];
                    j.tm[1] = e.W_fwd_[i];
                    j.tm[2] = e.W_fwd_lo_[i];
                    j.p = e.tile_fwd_params(i);
                } else {
                    j.tm[0] = e.D_row_[i + 1];
                    j.tm[1] = e.W_atom_[i];
                    j.tm[2] = e.W_atom_lo_[i];
                    j.p = e.tile_bwd_params(i);
                }
                j.p.err = err;
                j.bstart = b;
                j.gx = e.ntiles_;
                j.gy = 1;
                j.gz = e.C_;
                b += e.ntiles_ * e.C_;
                v.push_back(j);
            }
            const int mode = fwd ? (special ? M_FWD_OUT : M_FWD_TANH) : (special ? M_BWD_FIRST : M_BWD_TANH);
            seq_.push_back(Launch{K_TILE, mode, (int)v.size(), b, upload(v)});
        }
    }

    void add_dw()
    {
        std::vector<GridJob> v;
        int b = 0;
        for (const UmmaEngine *e : es_)
            for (int i = 1; i <= e->L_ - 2; ++i) {
                Params pp;
                dim3 grid;
                const CUtensorMap *md, *ma;
                if (!e->dw_params(i, pp, grid, md, ma)) continue;
                GridJob j;
                memset(&j, 0, sizeof j);
                j.tm[0] = *md;
                j.tm[1] = *ma;
                j.tm[2] = *ma;
                j.p = pp;
                j.p.err = es_[0]->err_;
                j.bstart = b;
                j.gx = (int)grid.x;
                j.gy = (int)grid.y;
                j.gz = (int)grid.z;
                b += (int)(grid.x * grid.y * grid.z);
                v.push_back(j);
            }
        if (!v.empty()) seq_.push_back(Launch{persistent_ ? K_DW2 : K_DWT, 0, (int)v.size(), b, upload(v)});
    }

    void add_final()
    {
        std::vector<FinalJob> v;
        int b = 0;
        for (size_t k = 0; k < es_.size(); ++k) {
            const UmmaEngine &e = *es_[k];
            v.push_back(FinalJob{e.final_args(), qoff_[k], uoff_[k], b, e.final_blocks()});
            b += e.final_blocks() * e.C_;
        }
        seq_.push_back(Launch{K_FINAL, 0, (int)v.size(), b, upload(v)});
    }

    template <int MODE, int WIDTH> static void launch_layer_g(const Launch &l, int max_clusters, cudaStream_t s)
    {
        static bool configured = false;
        if (!configured) {
            HMC_CK(cudaFuncSetAttribute(k_layer_pair_g<MODE, WIDTH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        L_SMEM));
            configured = true;
        }
        static const char *names[] = {"group_layer_fwd_tanh", "group_layer_fwd_out", "group_layer_bwd_tanh",
                                      "group_layer_bwd_first"};
        ProfScope ps(names[MODE], s);
        const int ncta = 2 * (int)std::min<long>(max_clusters, l.work);
        launch_pdl(k_layer_pair_g<MODE, WIDTH, true>, dim3(ncta), dim3(L_THREADS), L_SMEM, s,
                   l.jobs->as<const LayerJob>(), l.njobs, l.work);
        HMC_LAUNCH_CK();
    }

    template <int MODE, bool A_MN, bool B_MN, bool WSPLIT> static void launch_tile_g(const Launch &l, cudaStream_t s)
    {
        static bool configured = false;
        constexpr int sm = smem_bytes(WSPLIT);
        if (!configured) {
            HMC_CK(cudaFuncSetAttribute(k_umma_g<MODE, A_MN, B_MN, WSPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        sm));
            configured = true;
        }
        ProfScope ps("group_tile", s);
        k_umma_g<MODE, A_MN, B_MN, WSPLIT><<<(unsigned)l.work, NTHREADS, sm, s>>>(l.jobs->as<const GridJob>(), l.njobs);
        HMC_LAUNCH_CK();
    }

    template <int WIDTH> void run_layer(const Launch &l, cudaStream_t s) const
    {
        const int mc = es_[0]->max_clusters_;
        switch (l.mode) {
        case L_FWD_TANH: launch_layer_g<L_FWD_TANH, WIDTH>(l, mc, s); break;
        case L_FWD_OUT: launch_layer_g<L_FWD_OUT, WIDTH>(l, mc, s); break;
        case L_BWD_TANH: launch_layer_g<L_BWD_TANH, WIDTH>(l, mc, s); break;
        default: launch_layer_g<L_BWD_FIRST, WIDTH>(l, mc, s); break;
        }
    }

    template <int DX> static void launch_first_g(const Launch &l, cudaStream_t s)
    {
        ProfScope ps("group_first_fwd", s);
        launch_pdl(k_first_fwd_g<DX>, dim3((unsigned)l.work), dim3(256), 0, s, l.jobs->as<const FirstJob>(), l.njobs);
        HMC_LAUNCH_CK();
    }

    void run(const Launch &l, const float *q, double *U, float *g, cudaStream_t s) const
    {
        switch (l.kind) {
        case K_FIRST:
            switch (dx_) {
            case 1: launch_first_g<1>(l, s); break;
            case 2: launch_first_g<2>(l, s); break;
            case 3: launch_first_g<3>(l, s); break;
            case 4: launch_first_g<4>(l, s); break;
            case 5: launch_first_g<5>(l, s); break;
            case 6: launch_first_g<6>(l, s); break;
            case 7: launch_first_g<7>(l, s); break;
            default: launch_first_g<8>(l, s); break;
            }
            break;
        case K_LAYER:
            if (w_ == 256) run_layer<256>(l, s);
            else run_layer<128>(l, s);
            break;
        case K_TILE:
            switch (l.mode) {
            case M_FWD_TANH: launch_tile_g<M_FWD_TANH, false, false, true>(l, s); break;
            case M_FWD_OUT: launch_tile_g<M_FWD_OUT, false, false, true>(l, s); break;
            case M_BWD_TANH: launch_tile_g<M_BWD_TANH, false, true, true>(l, s); break;
            default: launch_tile_g<M_BWD_FIRST, false, true, true>(l, s); break;
            }
            break;
        case K_DW2: {
            static bool configured = false;
            if (!configured) {
                HMC_CK(cudaFuncSetAttribute(k_dw2_g, cudaFuncAttributeMaxDynamicSharedMemorySize, DW_SMEM));
                configured = true;
            }
            ProfScope ps("group_dw2", s);
            launch_pdl(k_dw2_g, dim3((unsigned)l.work), dim3(NTHREADS), DW_SMEM, s, l.jobs->as<const GridJob>(),
                       l.njobs);
            HMC_LAUNCH_CK();
            break;
        }
        case K_DWT: launch_tile_g<M_DW, true, true, false>(l, s); break;
        case K_FINAL: {
            ProfScope ps("group_finalize", s);
            launch_pdl(k_finalize_g, dim3((unsigned)l.work), dim3(256), 0, s, l.jobs->as<const FinalJob>(), l.njobs, q,
                       U, g);
            HMC_LAUNCH_CK();
            break;
        }
        }
    }

    std::vector<UmmaEngine *> es_;
    std::vector<long> qoff_, uoff_;
    int w_ = 0, dx_ = 0;
    bool persistent_ = false;
    std::vector<Launch> seq_;
};

// Problems whose engines share a kernel shape, in classes of two or more.
std::vector<std::unique_ptr<EngineGroup>> make_groups(const std::vector<Engine *> &es, const std::vector<long> &qoff,
                                                      const std::vector<long> &uoff, std::vector<bool> &grouped)
{
    std::map<std::tuple<int, int, bool>, std::vector<int>> cls;
    for (size_t i = 0; i < es.size(); ++i)
        if (auto *u = dynamic_cast<UmmaEngine *>(es[i])) cls[UmmaGroup::shape_class(*u)].push_back((int)i);
    std::vector<std::unique_ptr<EngineGroup>> out;
    grouped.assign(es.size(), false);
    for (auto &kv : cls) {
        if (kv.second.size() < 2) continue;
        std::vector<UmmaEngine *> m;
        std::vector<long> qo, uo;
        for (int i : kv.second) {
            m.push_back(static_cast<UmmaEngine *>(es[i]));
            qo.push_back(qoff[i]);
            uo.push_back(uoff[i]);
            grouped[i] = true;
        }
        out.emplace_back(new UmmaGroup(m, qo, uo));
    }
    return out;
}

// ---------------------------------------------------------------------------
// DeepONet on the tensor cores (Sec. 4.2 operator output): branch and trunk MLPs
// as bf16 GEMMs with the weights as a hi/lo pair, then S = B T^T + b0 on 128 x N
// tiles whose epilogue forms the residual, the FP64 energy partials and
// dS = (S - Y) / sigma^2 in bf16; dB = dS T and dT = dS^T B are bf16 GEMMs whose
// column sums give the last layers' bias gradients; each net's reverse pass and
// its sampled weight-gradient entries use the same kernels as the MLP path.
// ---------------------------------------------------------------------------
CUtensorMap make_map_ld(const void *base, uint64_t inner, uint64_t ld, uint64_t mid, uint64_t outer,
                        uint32_t box_inner, uint32_t box_mid)
{
    CUtensorMap m;
    memset(&m, 0, sizeof m);
    cuuint64_t dims[3] = {inner, mid, outer};
    cuuint64_t strides[2] = {ld * 2, ld * mid * 2};
    cuuint32_t box[3] = {box_inner, box_mid, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = encode_fn()(&m, TM_H16, 3, const_cast<void *>(base), dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for dims %llu (ld %llu) x %llu x %llu box %u x %u", (int)r,
                  (unsigned long long)inner, (unsigned long long)ld, (unsigned long long)mid, (unsigned long long)outer,
                  box_inner, box_mid);
        throw Fail{HMC_ERR_CUDA};
    }
    return m;
}

long round_up(long v, long m) { return (v + m - 1) / m * m; }

struct DonNet {
    const NetDesc *nd = nullptr;
    int L = 0, w = 0, p = 0, dx = 0, dxp = 0, ntiles = 1, nsplit = 1, kb_split = 1;
    long R = 0;
    bool gemm_first = false;              // first layer as a GEMM on bf16 inputs (dx > 8)
    int width[MAXL + 1] = {};             // widths w_0 .. w_L
    int inld[MAXL] = {};                  // row length of W_l in memory
    int entries[MAXL] = {};               // sampled weight entries of layer l gathered by k_umma<M_DW>
    int desc0 = 0;                        // first DbDesc of this net: biases 0..L-1, then dW_0 sums
    DevBuf x32, xb, xbl, w0f, b0f, dw0;   // xbl: bf16(x - xb), the lo half of the inputs
    std::unique_ptr<DevBuf> wh[MAXL], wl[MAXL], bias[MAXL], colsum[MAXL], rowptr[MAXL];
    std::unique_ptr<DevBuf> act[MAXL + 1], del[MAXL + 1];   // A_l, D_l for l = 1..L ([C][R][w_l])
    CUtensorMap act_row[MAXL + 1], act_atom[MAXL + 1], del_row[MAXL + 1], del_atom[MAXL + 1];
    CUtensorMap w_row_h[MAXL], w_row_l[MAXL], w_atom_h[MAXL], w_atom_l[MAXL], x_row, x_atom, x_row_lo;
    // hidden w x w tanh layers (w = 128 or 256) run forward on the persistent pair kernel:
    // the halves of W (hi and lo) that each CTA of a pair keeps resident
    bool pair[MAXL] = {};
    bool pair_last = false;   // the last layer (w -> p) too, forward and reverse (pair_shape_ok)
    CUtensorMap w_half_h[MAXL], w_half_l[MAXL];
};

class DonEngine final : public Engine {
  public:
    DonEngine(Problem &p, int C) : p_(p), C_(C)
    {
        k_ = p.k;
        nu_ = p.n_u;
        ny_ = p.n_y;
        nyp_ = round_up(ny_, 8);
        int dev = 0;
        HMC_CK(cudaGetDevice(&dev));
        HMC_CK(cudaDeviceGetAttribute(&num_sms_, cudaDevAttrMultiProcessorCount, dev));
        HMC_CK(cudaStreamCreateWithFlags(&s2_, cudaStreamNonBlocking));
        HMC_CK(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
        HMC_CK(cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming));
        for (int t = 0; t < 2; ++t) {
            HMC_CK(cudaStreamCreateWithFlags(&sw_[t], cudaStreamNonBlocking));
            HMC_CK(cudaEventCreateWithFlags(&evw_fork_[t], cudaEventDisableTiming));
            HMC_CK(cudaEventCreateWithFlags(&evw_join_[t], cudaEventDisableTiming));
        }
        HMC_CK(cudaMalloc(&err_, sizeof(int)));
        HMC_CK(cudaMemset(err_, 0, sizeof(int)));
        setup_net(br_, p.branch, p.u, nu_);
        setup_net(tr_, p.trunk, p.yq, ny_);
        pl_ = br_.p;
        if (HMC_F16) {
            // fp16 overflows at 65504, and dB = dS T adds n_y products and dT = dS^T B adds
            // n_u of them: their tiles are stored times 2^-ceil(log2 n), which keeps every
            // entry within max|dS| max|T| (max|dS| max|B|); the finalize scales the two nets'
            // gradient sums back by the inverse powers of two, exactly
            auto ceil_log2 = [](long n) {
                int e = 0;
                while ((1L << e) < n) ++e;
                return e;
            };
            kb_ = (float)std::ldexp(1.0, -ceil_log2(ny_));
            kt_ = (float)std::ldexp(1.0, -ceil_log2(nu_));
        }

        // operator output: targets, dS, partials
        std::vector<float> tf(p.t.begin(), p.t.end());
        yt_.alloc(sizeof(float) * std::max<size_t>(tf.size(), 1));
        if (!tf.empty()) HMC_CK(cudaMemcpy(yt_.ptr, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice));
        row_alloc(p.arena, ds_, sizeof(h16) * C * std::max<long>(nu_, 1) * nyp_);
        HMC_CK(cudaMemset(ds_.ptr, 0, ds_.n));
        // S^T tiles: 128 query points (rows) x bs_ input functions (columns)
        bs_ = nu_ >= 256 ? 256 : (int)round_up(nu_, 32);
        nut_ = (int)std::max<long>(1, (ny_ + BM - 1) / BM);
        ntn_ = (int)std::max<long>(1, (nu_ + bs_ - 1) / bs_);
        const long max_ntn = std::max<long>(1, (nu_ + 127) / 128);   // room for the narrowest tile
        u_part_.alloc(sizeof(double) * C * nut_ * max_ntn);
        db0_part_.alloc(sizeof(float) * C * nut_ * max_ntn);
        b0v_.alloc(sizeof(float) * C);
        {
            std::vector<float> v(C, p.b0_off >= 0 ? (float)p.frozen[p.b0_off] : 0.0f);
            HMC_CK(cudaMemcpy(b0v_.ptr, v.data(), sizeof(float) * C, cudaMemcpyHostToDevice));
        }
        ds_row_ = make_map_ld(ds_.ptr, ny_, nyp_, nu_, C, 64, 128);
        ds_atom_ = make_map_ld(ds_.ptr, ny_, nyp_, nu_, C, 64, 64);
        if (nu_ > 128) tune_s_tile();
        b_col_ = make_map(br_.act[br_.L]->ptr, pl_, nu_, C, 64, bs_);

        build_entries();
        nsplit_ = std::max(br_.nsplit, tr_.nsplit);
        gw_part_.alloc(sizeof(float) * nsplit_ * C * std::max<long>(k_, 1));
        HMC_CK(cudaMemset(gw_part_.ptr, 0, gw_part_.n));   // splits a net does not use stay zero
        // accurate-energy S^T tiles: 128 query points x es_ input functions
        es_ = nu_ >= 256 ? 256 : (int)round_up(nu_, 32);
        nut_e_ = (int)std::max<long>(1, (ny_ + BM - 1) / BM);
        ntn_e_ = (int)std::max<long>(1, (nu_ + es_ - 1) / es_);
        alloc_t(u_acc_, sizeof(double) * C * nut_e_ * ntn_e_);
        b_hi_e_ = make_map(br_.act[br_.L]->ptr, pl_, nu_, C, 64, es_);
        b_lo_e_ = make_map(br_.del[br_.L]->ptr, pl_, nu_, C, 64, es_);
    }

    ~DonEngine() override
    {
        if (err_) cudaFree(err_);
        if (ev_fork_) cudaEventDestroy(ev_fork_);
        if (ev_join_) cudaEventDestroy(ev_join_);
        if (s2_) cudaStreamDestroy(s2_);
        for (int t = 0; t < 2; ++t) {
            if (evw_fork_[t]) cudaEventDestroy(evw_fork_[t]);
            if (evw_join_[t]) cudaEventDestroy(evw_join_[t]);
            if (sw_[t]) cudaStreamDestroy(sw_[t]);
        }
    }

    ScatterPlan scatter_plan() override { return plan_; }
    int *error_flag() const override { return err_; }
    size_t bytes() const override { return bytes_; }

    // The Metropolis energy (the bf16 operator output would carry order-one noise into
    // dH): branch and trunk again with hi/lo activations (their hi halves go to the
    // activation buffers, the lo halves to the delta buffers, free after the gradient),
    // then S^T = T B^T from the hi/lo outputs with only the residual's sums of squares.
    bool has_accurate_energy() const override { return true; }
    void accurate_energy(const void *qv, double *U, cudaStream_t s) override
    {
        const float *q = static_cast<const float *>(qv);
        for (DonNet *np : {&br_, &tr_}) {
            DonNet &n = *np;
            const NetDesc &nd = *n.nd;
            if (!n.gemm_first) {
                ProfScope ps("first_fwd3", s);
                launch_pdl(k_first_fwd3, dim3((unsigned)n.ntiles, C_), dim3(256), 0, s, n.x32.as<float>(), n.dx,
                           (int)n.R, n.w, n.w0f.as<float>(), n.bias[0]->as<float>(), n.act[1]->as<h16>(),
                           n.del[1]->as<h16>());
            }
            for (int l = n.gemm_first ? 0 : 1; l < n.L; ++l) {
                E3Params e{};
                e.M = (int)n.R;
                e.N = nd.w[l + 1];
                e.K = nd.w[l];
                e.ntiles = n.ntiles;
                e.err = err_;
                e.bias = n.bias[l]->as<float>();
                e.out_hi = n.act[l + 1]->as<h16>();
                e.out_lo = n.del[l + 1]->as<h16>();
                const CUtensorMap &ah = l == 0 ? n.x_row : n.act_row[l];
                const CUtensorMap &al = l == 0 ? n.x_row_lo : n.del_row[l];
                const dim3 grid(n.ntiles, 1, C_);
                if (l < n.L - 1) launch_energy3<E3_TANH>(ah, al, n.w_row_h[l], n.w_row_l[l], e, grid, s);
                else launch_energy3<E3_LIN>(ah, al, n.w_row_h[l], n.w_row_l[l], e, grid, s);
            }
        }
        E3Params e{};
        e.M = (int)ny_;
        e.N = es_;
        e.K = pl_;
        e.ntiles = nut_e_;
        e.err = err_;
        e.bout = b0v_.as<float>();
        e.Yt = yt_.as<float>();
        e.nu = (int)nu_;
        e.ntn = ntn_e_;
        e.u_part = u_acc_.as<double>();
        launch_energy3<E3_S>(tr_.act_row[tr_.L], tr_.del_row[tr_.L], b_hi_e_, b_lo_e_, e, dim3(nut_e_, ntn_e_, C_), s);
        FinalArgs fa{};
        fa.k = (int)k_;
        fa.nu = nut_e_ * ntn_e_;
        fa.u_part = u_acc_.as<double>();
        fa.half_inv_s2 = 0.5 / (p_.sigma * p_.sigma);
        fa.gscale = (float)(1.0 / (p_.sigma * p_.sigma) / delta_scale(p_.sigma));
        fa.inv_a2 = 1.0 / (p_.alpha * p_.alpha);
        ProfScope ps("energy3_final", s);
        launch_pdl(k_finalize_bf16, dim3(1, C_), dim3(256), 0, s, fa, q, U, (float *)nullptr);
    }

    void scatter(const void *qv, cudaStream_t s) override
    {
        dim3 grid((unsigned)std::min<long>((k_ + 255) / 256, 1024), C_);
        ProfScope ps("scatter", s);
        launch_pdl(k_scatter_plan<float>, grid, dim3(256), 0, s, static_cast<const float *>(qv), k_, plan_);
    }

    void energy_grad(const void *qv, double *U, void *gv, bool scattered, cudaStream_t s) override
    {
        const float *q = static_cast<const float *>(qv);
        float *g = static_cast<float *>(gv);
        if (!scattered) scatter(qv, s);
        // branch and trunk are independent up to S and again after dB and dT: the trunk's
        // work runs on the engine's second stream, joined back before S and before finalize
        const cudaStream_t st = active_profiler() ? s : s2_;   // one stream while profiling
        fork(s, st);
        forward(br_, s);
        forward(tr_, st);
        join(s, st);
        launch_s(b_col_, s);   // S = B T^T + b0, residual, energy partials and dS
        fork(s, st);
        // dB = dS T and dT = dS^T B: the deltas of the two nets' linear output layers
        {
            Params pp = base();
            pp.M = (int)nu_;
            pp.N = pl_;
            pp.K = (int)ny_;
            pp.kb_per_split = (int)((ny_ + BK - 1) / BK);
            pp.ntiles = br_.ntiles;
            pp.out = br_.del[br_.L]->as<h16>();
            pp.out_b = nu_ * pl_;
            pp.oscale = kb_;
            pp.db_part = br_.colsum[br_.L - 1]->as<float>();
            launch_umma<M_GEMM_BF16, false, true, false>(ds_row_, tr_.act_atom[tr_.L], tr_.act_atom[tr_.L], pp,
                                                          dim3(br_.ntiles, 1, C_), s);
        }
        {
            Params pp = base();
            pp.M = (int)ny_;
            pp.N = pl_;
            pp.K = (int)nu_;
            pp.kb_per_split = (int)((nu_ + BK - 1) / BK);
            pp.ntiles = tr_.ntiles;
            pp.out = tr_.del[tr_.L]->as<h16>();
            pp.out_b = ny_ * pl_;
            pp.oscale = kt_;
            pp.db_part = tr_.colsum[tr_.L - 1]->as<float>();
            launch_umma<M_GEMM_BF16, true, true, false>(ds_atom_, br_.act_atom[br_.L], br_.act_atom[br_.L], pp,
                                                         dim3(tr_.ntiles, 1, C_), st);
        }
        backward(br_, s, active_profiler() ? s : sw_[0], 0);
        backward(tr_, st, active_profiler() ? st : sw_[1], 1);
        join(s, st);
        FinalArgs fa{};
        fa.k = (int)k_;
        fa.nsplit = nsplit_;
        fa.nu = nut_ * ntn_;
        fa.kind = kind_.as<int>();
        fa.desc = desc_.as<int>();
        fa.off = off_.as<int>();
        fa.u_part = u_part_.as<double>();
        fa.gw_part = gw_part_.as<float>();
        fa.gw_split = (long)C_ * k_;
        fa.db = db_desc_.as<const DbDesc>();
        fa.half_inv_s2 = 0.5 / (p_.sigma * p_.sigma);
        fa.gscale = (float)(1.0 / (p_.sigma * p_.sigma) / delta_scale(p_.sigma));
        fa.escale = HMC_F16 ? escale_.as<float>() : nullptr;
        fa.inv_a2 = 1.0 / (p_.alpha * p_.alpha);
        fa.heavy = heavy_.as<int>();
        fa.nheavy = nheavy_;
        fa.nlight = (int)((k_ + 255) / 256);
        {
            ProfScope ps("finalize", s);
            dim3 grid((unsigned)(fa.nlight + (nheavy_ + 7) / 8 + 1), C_);
            launch_pdl(k_finalize_bf16, grid, dim3(256), 0, s, fa, q, U, g);
        }
    }

    std::string tuning() const override { return tuning_; }

  private:
    Params base() const
    {
        Params pp{};
        pp.err = err_;
        return pp;
    }

    void fork(cudaStream_t s, cudaStream_t st)
    {
        if (st == s) return;
        HMC_CK(cudaEventRecord(ev_fork_, s));
        HMC_CK(cudaStreamWaitEvent(st, ev_fork_, 0));
    }

    void join(cudaStream_t s, cudaStream_t st)
    {
        if (st == s) return;
        HMC_CK(cudaEventRecord(ev_join_, st));
        HMC_CK(cudaStreamWaitEvent(s, ev_join_, 0));
    }

    void launch_s(const CUtensorMap &bmap, cudaStream_t s)
    {
        Params pp = base();
        pp.M = (int)ny_;
        pp.N = bs_;
        pp.K = pl_;
        pp.kb_per_split = (pl_ + BK - 1) / BK;
        pp.ntiles = nut_;
        pp.Yt = yt_.as<float>();
        pp.ny = (int)ny_;
        pp.nu = (int)nu_;
        pp.ldo = (int)nyp_;
        pp.ntn = ntn_;
        pp.b0s = b0v_.as<float>();
        pp.out = ds_.as<h16>();
        pp.out_b = nu_ * nyp_;
        pp.inv_s2 = (float)delta_scale(p_.sigma);
        pp.u_part = u_part_.as<double>();
        pp.db0_part = db0_part_.as<float>();
        launch_umma<M_S, false, false, false>(tr_.act_row[tr_.L], bmap, bmap, pp, dim3(C_, nut_, ntn_), s);
    }

    // Autotuner for the operator-output tile: time S on 128- and 256-column tiles on this
    // engine's own buffers (one warm-up, three timed launches) and keep the faster one.
    void tune_s_tile()
    {
        if (!autotune_enabled()) {
            tuning_ = "S column tile " + std::to_string(bs_) + " (heuristic; autotuner off)";
            return;
        }
        cudaStream_t s;
        cudaEvent_t a, b;
        HMC_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        HMC_CK(cudaEventCreate(&a));
        HMC_CK(cudaEventCreate(&b));
        int best = bs_;
        float best_ms = 1e30f;
        std::string log;
        for (int cand : {128, 256}) {
            if (cand > round_up(nu_, 32) && cand != 128) break;
            bs_ = cand;
            ntn_ = (int)((nu_ + bs_ - 1) / bs_);
            const CUtensorMap tm = make_map(br_.act[br_.L]->ptr, pl_, nu_, C_, 64, bs_);
            launch_s(tm, s);
            HMC_CK(cudaEventRecord(a, s));
            for (int r = 0; r < 3; ++r) launch_s(tm, s);
            HMC_CK(cudaEventRecord(b, s));
            HMC_CK(cudaEventSynchronize(b));
            float ms = 0.0f;
            HMC_CK(cudaEventElapsedTime(&ms, a, b));
            ms /= 3.0f;
            char buf[48];
            snprintf(buf, sizeof buf, "%s%d:%.1fus", log.empty() ? "" : " ", cand, 1000.0f * ms);
            log += buf;
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        HMC_CK(cudaStreamSynchronize(s));
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaStreamDestroy(s);
        bs_ = best;
        ntn_ = (int)((nu_ + bs_ - 1) / bs_);
        tuning_ = "S column tile " + std::to_string(best) + " of {" + log + "}";
    }

    DevBuf *track(DevBuf *b)   // an allocated buffer
    {
        bytes_ += b->n;
        return b;
    }
    void alloc_t(DevBuf &b, size_t n)
    {
        b.alloc(n);
        bytes_ += n;
    }

    // value of parameter (layer l of net n, row o, column i) replicated over the chains
    void upload_w(DonNet &n, int l, void *hi, void *lo, bool bf16)
    {
        const NetDesc &nd = *n.nd;
        const int out = nd.w[l + 1], in = nd.w[l], ld = n.inld[l];
        const size_t per = (size_t)out * ld;
        if (bf16) {
            std::vector<h16> vh(C_ * per, f_to_h16(0.0f)), vl(C_ * per, f_to_h16(0.0f));
            for (int c = 0; c < C_; ++c)
                for (int o = 0; o < out; ++o)
                    for (int i = 0; i < in; ++i) {
                        const float w = (float)p_.frozen[nd.woff[l] + (long)o * in + i];
                        const h16 h = f_to_h16(w);
                        vh[c * per + (size_t)o * ld + i] = h;
                        vl[c * per + (size_t)o * ld + i] = f_to_h16(w - h16_to_f(h));
                    }
            HMC_CK(cudaMemcpy(hi, vh.data(), sizeof(h16) * vh.size(), cudaMemcpyHostToDevice));
            HMC_CK(cudaMemcpy(lo, vl.data(), sizeof(h16) * vl.size(), cudaMemcpyHostToDevice));
        } else {
            std::vector<float> v(C_ * per, 0.0f);
            for (int c = 0; c < C_; ++c)
                for (int o = 0; o < out; ++o)
                    for (int i = 0; i < in; ++i) v[c * per + (size_t)o * ld + i] = (float)p_.frozen[nd.woff[l] + (long)o * in + i];
            HMC_CK(cudaMemcpy(hi, v.data(), sizeof(float) * v.size(), cudaMemcpyHostToDevice));
        }
    }

    void upload_b(const NetDesc &nd, int l, void *dst)
    {
        const int out = nd.w[l + 1];
        std::vector<float> v((size_t)C_ * out);
        for (int c = 0; c < C_; ++c)
            for (int o = 0; o < out; ++o) v[(size_t)c * out + o] = (float)p_.frozen[nd.boff[l] + o];
        HMC_CK(cudaMemcpy(dst, v.data(), sizeof(float) * v.size(), cudaMemcpyHostToDevice));
    }

    void setup_net(DonNet &n, const NetDesc &nd, const std::vector<double> &xin, long R)
    {
        n.nd = &nd;
        n.L = nd.L;
        n.R = R;
        n.dx = nd.w[0];
        n.w = nd.w[1];
        n.p = nd.w[nd.L];
        for (int l = 0; l <= nd.L; ++l) n.width[l] = nd.w[l];
        n.gemm_first = n.dx > 8;
        n.dxp = n.gemm_first ? (int)round_up(n.dx, 8) : n.dx;
        n.ntiles = (int)std::max<long>(1, (R + BM - 1) / BM);
        const int C = C_;
        for (int l = 0; l < n.L; ++l) n.inld[l] = (l == 0) ? n.dxp : nd.w[l];
        // inputs
        std::vector<float> xf(xin.begin(), xin.end());
        alloc_t(n.x32, sizeof(float) * std::max<size_t>(xf.size(), 1));
        if (!xf.empty()) HMC_CK(cudaMemcpy(n.x32.ptr, xf.data(), sizeof(float) * xf.size(), cudaMemcpyHostToDevice));
        if (n.gemm_first) {   // bf16 copy per chain, rows padded to dxp
            std::vector<h16> xb((size_t)C * std::max<long>(R, 1) * n.dxp, f_to_h16(0.0f));
            std::vector<h16> xl(xb.size(), f_to_h16(0.0f));
            for (int c = 0; c < C; ++c)
                for (long r = 0; r < R; ++r)
                    for (int d = 0; d < n.dx; ++d) {
                        const float v = xf[(size_t)r * n.dx + d];
                        const h16 h = f_to_h16(v);
                        xb[((size_t)c * R + r) * n.dxp + d] = h;
                        xl[((size_t)c * R + r) * n.dxp + d] = f_to_h16(v - h16_to_f(h));
                    }
            alloc_t(n.xb, sizeof(h16) * xb.size());
            alloc_t(n.xbl, sizeof(h16) * xl.size());
            HMC_CK(cudaMemcpy(n.xb.ptr, xb.data(), sizeof(h16) * xb.size(), cudaMemcpyHostToDevice));
            HMC_CK(cudaMemcpy(n.xbl.ptr, xl.data(), sizeof(h16) * xl.size(), cudaMemcpyHostToDevice));
            n.x_row = make_map_ld(n.xb.ptr, n.dx, n.dxp, R, C, 64, 128);
            n.x_row_lo = make_map_ld(n.xbl.ptr, n.dx, n.dxp, R, C, 64, 128);
            n.x_atom = make_map_ld(n.xb.ptr, n.dx, n.dxp, R, C, 64, 64);
        }
        // parameters
        for (int l = 0; l < n.L; ++l) {
            const int out = nd.w[l + 1];
            n.bias[l].reset(track(new DevBuf(sizeof(float) * C * out)));
            upload_b(nd, l, n.bias[l]->ptr);
            if (l == 0 && !n.gemm_first) {
                alloc_t(n.w0f, sizeof(float) * C * out * n.dx);
                upload_w(n, 0, n.w0f.ptr, nullptr, false);
                continue;
            }
            const size_t wb = sizeof(h16) * C * out * n.inld[l];
            n.wh[l].reset(track(new DevBuf(wb)));
            n.wl[l].reset(track(new DevBuf(wb)));
            upload_w(n, l, n.wh[l]->ptr, n.wl[l]->ptr, true);
            const int in = nd.w[l];
            n.w_row_h[l] = make_map_ld(n.wh[l]->ptr, in, n.inld[l], out, C, 64, out);
            n.w_row_l[l] = make_map_ld(n.wl[l]->ptr, in, n.inld[l], out, C, 64, out);
            if (l >= 1) {
                n.w_atom_h[l] = make_map(n.wh[l]->ptr, in, out, C, 64, 64);
                n.w_atom_l[l] = make_map(n.wl[l]->ptr, in, out, C, 64, 64);
            }
            const bool last = l == n.L - 1 && l >= 2 && n.inld[l] == in && pair_shape_ok(L_FWD_LIN, out, in) &&
                              pair_shape_ok(L_BWD_TANH, in, out) && nd.act[l] == HMC_ACT_IDENTITY;
            if (last) {
                n.pair_last = true;
                n.w_half_h[l] = make_map(n.wh[l]->ptr, in, out, C, 64, out / 2);
                n.w_half_l[l] = make_map(n.wl[l]->ptr, in, out, C, 64, out / 2);
                if (max_clusters_ == 0) max_clusters_ = layer_max_clusters();
            }
            if (l >= 1 && l < n.L - 1 && in == out && (out == 128 || out == 256) && n.inld[l] == in &&
                nd.act[l] == HMC_ACT_TANH) {
                n.pair[l] = true;
                n.w_half_h[l] = make_map(n.wh[l]->ptr, in, out, C, 64, out / 2);
                n.w_half_l[l] = make_map(n.wl[l]->ptr, in, out, C, 64, out / 2);
                if (max_clusters_ == 0) max_clusters_ = layer_max_clusters();
            }
        }
        // activations and deltas, per-tile column sums
        for (int l = 1; l <= n.L; ++l) {
            const size_t ab = sizeof(h16) * C * std::max<long>(R, 1) * nd.w[l];
            n.act[l].reset(new DevBuf());
            n.del[l].reset(new DevBuf());
            row_alloc(p_.arena, *n.act[l], ab);
            row_alloc(p_.arena, *n.del[l], ab);
            if (!p_.arena) bytes_ += 2 * ab;
            n.act_row[l] = make_map(n.act[l]->ptr, nd.w[l], R, C, 64, 128);
            n.act_atom[l] = make_map(n.act[l]->ptr, nd.w[l], R, C, 64, 64);
            n.del_row[l] = make_map(n.del[l]->ptr, nd.w[l], R, C, 64, 128);
            n.del_atom[l] = make_map(n.del[l]->ptr, nd.w[l], R, C, 64, 64);
        }
        for (int l = 0; l < n.L; ++l)
            n.colsum[l].reset(track(new DevBuf(sizeof(float) * C * n.ntiles * nd.w[l + 1])));
        if (!n.gemm_first) alloc_t(n.dw0, sizeof(float) * C * n.ntiles * n.w * n.dx);
        const int total_kb = (int)((R + BK - 1) / BK);
        n.nsplit = pick_splits(total_kb, ((n.w + BM - 1) / BM) * C, 2 * num_sms_);
        n.kb_split = (total_kb + n.nsplit - 1) / n.nsplit;
        n.nsplit = (total_kb + n.kb_split - 1) / n.kb_split;
    }

    void forward(DonNet &n, cudaStream_t s)
    {
        const NetDesc &nd = *n.nd;
        if (!n.gemm_first) {
            dim3 grid((unsigned)n.ntiles, C_);
            ProfScope ps("first_fwd", s);
            launch_first_fwd(n.dx, grid, s, n.x32.as<float>(), (int)n.R, n.w, n.w0f.as<float>(),
                             n.bias[0]->as<float>(), n.act[1]->as<h16>());
        }
        for (int l = n.gemm_first ? 0 : 1; l < n.L; ++l) {
            Params pp = base();
            pp.M = (int)n.R;
            pp.N = nd.w[l + 1];
            pp.K = nd.w[l];
            pp.kb_per_split = (pp.K + BK - 1) / BK;
            pp.bias = n.bias[l]->as<float>();
            pp.bias_b = pp.N;
            pp.out = n.act[l + 1]->as<h16>();
            pp.out_b = n.R * pp.N;
            const CUtensorMap &a = (l == 0) ? n.x_row : n.act_row[l];
            const dim3 grid(n.ntiles, 1, C_);
            if (n.pair[l]) {   // the persistent pair kernel: (chain, tile pair) units on CTA pairs
                LayerParams lp{};
                lp.N = (int)n.R;
                lp.W = pp.N;
                lp.C = C_;
                lp.ntiles = n.ntiles;
                lp.dx = n.dx;
                lp.err = err_;
                lp.bias = pp.bias;
                lp.out = pp.out;
                const long units = (long)C_ * ((n.ntiles + 1) / 2);
                launch_layer<L_FWD_TANH>(a, n.w_half_h[l], n.w_half_l[l], lp,
                                         2 * (int)std::min<long>(max_clusters_, units), s);
            } else if (l == n.L - 1 && n.pair_last) {   // the last layer, linear, on the pair kernel
                LayerParams lp{};
                lp.N = (int)n.R;
                lp.W = pp.N;
                lp.C = C_;
                lp.ntiles = n.ntiles;
                lp.dx = n.dx;
                lp.err = err_;
                lp.bias = pp.bias;
                lp.out = pp.out;
                const long units = (long)C_ * ((n.ntiles + 1) / 2);
                launch_layer_nk<L_FWD_LIN>(a, n.w_half_h[l], n.w_half_l[l], lp, 2 * (int)std::min<long>(max_clusters_, units),
                                           s);
            } else if (l < n.L - 1)
                launch_umma<M_FWD_TANH, false, false, true>(a, n.w_row_h[l], n.w_row_l[l], pp, grid, s);
            else
                launch_umma<M_FWD_LIN, false, false, true>(a, n.w_row_h[l], n.w_row_l[l], pp, grid, s);
        }
    }

    // The reverse pass of net n on stream s.  The weight gradient of layer l reads D_{l+1}
    // and A_l, which nothing later in the pass writes, and writes only its own entries'
    // partials: it runs on the side stream sw (t: the net's fork and join events), which
    // joins s again at the end of the pass (sw == s while a per-kernel profile runs).
    void backward(DonNet &n, cudaStream_t s, cudaStream_t sw, int t)
    {
        const NetDesc &nd = *n.nd;
        const int total_kb = (int)((n.R + BK - 1) / BK);
        bool forked = false;
        for (int l = n.L - 1; l >= 0; --l) {
            // sampled entries of dW_l = D_{l+1}^T A_l
            if (n.entries[l] > 0 && (l >= 1 || n.gemm_first)) {
                if (sw != s) {
                    HMC_CK(cudaEventRecord(evw_fork_[t], s));
                    HMC_CK(cudaStreamWaitEvent(sw, evw_fork_[t], 0));
                    forked = true;
                }
                Params pp = base();
                pp.M = nd.w[l + 1];
                pp.N = (l >= 1) ? nd.w[l] : (int)round_up(n.dx, 64);
                pp.K = (int)n.R;
                pp.kb_per_split = n.kb_split;
                pp.rowptr = n.rowptr[l]->as<int>();
                pp.ecol = ecol_.as<int>();
                pp.erow = erow_.as<int>();
                pp.epack = epack_.as<int>();
                pp.gw_part = gw_part_.as<float>();
                pp.gw_split = (long)C_ * k_;
                pp.gw_b = k_;
                const int splits = (total_kb + n.kb_split - 1) / n.kb_split;
                const CUtensorMap &b = (l >= 1) ? n.act_atom[l] : n.x_atom;
                launch_umma<M_DW, true, true, false>(n.del_atom[l + 1], b, b, pp,
                                                     dim3((pp.M + BM - 1) / BM, splits, C_), sw);
            }
            if (l == 0 || l <= nd.lmin) break;   // no delta is needed below layer l
            // D_l = (D_{l+1} W_l) (1 - A_l^2); its column sums are the bias gradient of layer l-1
            Params pp = base();
            pp.M = (int)n.R;
            pp.N = nd.w[l];
            pp.K = nd.w[l + 1];
            pp.kb_per_split = (pp.K + BK - 1) / BK;
            pp.ntiles = n.ntiles;
            pp.aux = n.act[l]->as<h16>();
            pp.aux_b = n.R * pp.N;
            pp.db_part = n.colsum[l - 1]->as<float>();
            const dim3 grid(n.ntiles, 1, C_);
            // the persistent pair kernel for the w x w layers (first-layer sums of up to four
            // inputs at w = 256, seven at w = 128), with the column sums of delta_l as the
            // bias gradient
            const bool first = l == 1 && !n.gemm_first;
            const bool last = l == n.L - 1 && n.pair_last;   // through the last layer (N = w, K = p)
            if (last) {
                LayerParams lp{};
                lp.N = (int)n.R;
                lp.W = pp.N;
                lp.C = C_;
                lp.ntiles = n.ntiles;
                lp.dx = n.dx;
                lp.err = err_;
                lp.aux = pp.aux;
                lp.db_part = pp.db_part;
                lp.out = n.del[l]->as<h16>();
                const long units = (long)C_ * ((n.ntiles + 1) / 2);
                launch_layer_nk<L_BWD_TANH>(n.del_row[l + 1], n.w_atom_h[l], n.w_atom_l[l], lp,
                                            2 * (int)std::min<long>(max_clusters_, units), s);
            } else if (n.pair[l] && (!first || n.dx <= 4 || (pp.N == 128 && n.dx <= 7))) {
                LayerParams lp{};
                lp.N = (int)n.R;
                lp.W = pp.N;
                lp.C = C_;
                lp.ntiles = n.ntiles;
                lp.dx = n.dx;
                lp.err = err_;
                lp.aux = pp.aux;
                lp.db_part = pp.db_part;
                const long units = (long)C_ * ((n.ntiles + 1) / 2);
                const int ncta = 2 * (int)std::min<long>(max_clusters_, units);
                if (first) {
                    lp.x = n.x32.as<float>();
                    lp.dw0_part = n.dw0.as<float>();
                    launch_layer<L_BWD_FIRST>(n.del_row[l + 1], n.w_atom_h[l], n.w_atom_l[l], lp, ncta, s);
                } else {
                    lp.out = n.del[l]->as<h16>();
                    launch_layer<L_BWD_TANH>(n.del_row[l + 1], n.w_atom_h[l], n.w_atom_l[l], lp, ncta, s);
                }
            } else if (first) {
                pp.x = n.x32.as<float>();
                pp.dx = n.dx;
                pp.dw0_part = n.dw0.as<float>();
                launch_umma<M_BWD_FIRST, false, true, true>(n.del_row[l + 1], n.w_atom_h[l], n.w_atom_l[l], pp, grid, s);
            } else {
                pp.out = n.del[l]->as<h16>();
                pp.out_b = n.R * pp.N;
                launch_umma<M_BWD_TANH, false, true, true>(n.del_row[l + 1], n.w_atom_h[l], n.w_atom_l[l], pp, grid, s);
            }
        }
        if (forked) {
            HMC_CK(cudaEventRecord(evw_join_[t], sw));
            HMC_CK(cudaStreamWaitEvent(s, evw_join_[t], 0));
        }
    }

    // per-entry sources of the gradient, scatter plan, CSR rows of the gathered weights
    void build_entries()
    {
        std::vector<int> kind(k_), desc(k_), off(k_), erow(k_, 0), ecol(k_, 0), bid(k_), boff(k_);
        std::vector<float> esc(k_, 1.0f);   // the inverse of the output-delta factor of the entry's net
        std::vector<DbDesc> dbd;
        DonNet *nets[2] = {&br_, &tr_};
        int nb = 0;
        int wbuf[2][MAXL], bbuf[2][MAXL];
        std::vector<std::vector<int>> rp[2];
        for (int t = 0; t < 2; ++t) {
            DonNet &n = *nets[t];
            n.desc0 = (int)dbd.size();
            for (int l = 0; l < n.L; ++l)
                dbd.push_back(DbDesc{n.colsum[l]->as<float>(), (long)n.ntiles * n.width[l + 1], n.width[l + 1], n.ntiles});
            dbd.push_back(DbDesc{n.gemm_first ? nullptr : n.dw0.as<float>(), (long)n.ntiles * n.w * n.dx,
                                 (long)n.w * n.dx, n.ntiles});
            rp[t].assign(n.L, std::vector<int>());
            for (int l = 0; l < n.L; ++l) {
                rp[t][l].assign(n.width[l + 1] + 1, 0);
                const int out = n.width[l + 1];
                wbuf[t][l] = nb;
                if (l == 0 && !n.gemm_first) {
                    plan_.base[nb] = n.w0f.ptr;
                    plan_.cstride[nb] = (long)out * n.dx;
                    plan_.kind16[nb] = 0;
                } else {
                    plan_.base[nb] = n.wh[l]->ptr;
                    plan_.base_lo[nb] = n.wl[l]->ptr;
                    plan_.cstride[nb] = (long)out * n.inld[l];
                    plan_.kind16[nb] = H16_KIND;
                }
                ++nb;
                bbuf[t][l] = nb;
                plan_.base[nb] = n.bias[l]->ptr;
                plan_.cstride[nb] = out;
                plan_.kind16[nb] = 0;
                ++nb;
            }
        }
        const int b0buf = nb;
        plan_.base[nb] = b0v_.ptr;
        plan_.cstride[nb] = 1;
        plan_.kind16[nb] = 0;
        ++nb;
        HMC_REQUIRE(nb <= MAX_SCATTER_BUFS, "too many layers for the scatter plan");
        plan_.nbuf = nb;
        const int b0desc = (int)dbd.size();
        dbd.push_back(DbDesc{db0_part_.as<float>(), (long)nut_ * ntn_, 1, nut_ * ntn_});

        for (long j = 0; j < k_; ++j) {
            const long id = p_.idx[j];
            if (p_.b0_off >= 0 && id == p_.b0_off) {
                kind[j] = E_PART;
                desc[j] = b0desc;
                off[j] = 0;
                bid[j] = b0buf;
                boff[j] = 0;
                continue;
            }
            const int t = id < p_.branch.base + p_.branch.P ? 0 : 1;
            esc[j] = 1.0f / (t == 0 ? kb_ : kt_);
            DonNet &n = *nets[t];
            const NetDesc &nd = *n.nd;
            int l = 0;
            while (l + 1 < n.L && id >= nd.woff[l + 1]) ++l;
            const int in = nd.w[l];
            const bool is_w = id < nd.woff[l] + (long)nd.w[l + 1] * in;
            if (is_w) {
                const long rel = id - nd.woff[l];
                const int o = (int)(rel / in), i = (int)(rel % in);
                bid[j] = wbuf[t][l];
                boff[j] = o * n.inld[l] + i;
                if (l == 0 && !n.gemm_first) {
                    kind[j] = E_PART;
                    desc[j] = n.desc0 + n.L;
                    off[j] = o * n.dx + i;
                } else {
                    kind[j] = E_GW;
                    erow[j] = o;
                    ecol[j] = i;
                    rp[t][l][o + 1]++;
                    n.entries[l]++;
                }
            } else {
                const int rel = (int)(id - nd.boff[l]);
                kind[j] = E_PART;
                desc[j] = n.desc0 + l;
                off[j] = rel;
                bid[j] = bbuf[t][l];
                boff[j] = rel;
            }
        }
        // CSR rows: a layer's weight entries are contiguous and sorted by (row, column)
        for (int t = 0; t < 2; ++t) {
            DonNet &n = *nets[t];
            for (int l = 0; l < n.L; ++l) {
                const int out = n.width[l + 1];
                const long first = std::lower_bound(p_.idx.begin(), p_.idx.end(), n.nd->woff[l]) - p_.idx.begin();
                std::vector<int> r(out + 1);
                r[0] = (int)first;
                for (int o = 0; o < out; ++o) r[o + 1] = r[o] + rp[t][l][o + 1];
                n.rowptr[l].reset(track(new DevBuf(sizeof(int) * (out + 1))));
                HMC_CK(cudaMemcpy(n.rowptr[l]->ptr, r.data(), sizeof(int) * (out + 1), cudaMemcpyHostToDevice));
            }
        }
        auto up = [&](DevBuf &d, const std::vector<int> &v) {
            alloc_t(d, sizeof(int) * std::max<size_t>(v.size(), 1));
            if (!v.empty()) HMC_CK(cudaMemcpy(d.ptr, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice));
        };
        {   // entries with per-tile partials are summed a warp each
            const std::vector<int> heavy = mark_heavy(kind, desc, dbd);
            nheavy_ = (int)heavy.size();
            heavy_.alloc(sizeof(int) * std::max<size_t>(heavy.size(), 1));
            if (nheavy_) HMC_CK(cudaMemcpy(heavy_.ptr, heavy.data(), sizeof(int) * heavy.size(), cudaMemcpyHostToDevice));
        }
        up(kind_, kind);
        up(desc_, desc);
        up(off_, off);
        up(erow_, erow);
        up(ecol_, ecol);
        std::vector<int> epack(k_);
        for (long j = 0; j < k_; ++j) epack[j] = (erow[j] << 16) | ecol[j];
        up(epack_, epack);
        up(sc_off_, boff);
        alloc_t(escale_, sizeof(float) * std::max<size_t>(esc.size(), 1));
        if (!esc.empty()) HMC_CK(cudaMemcpy(escale_.ptr, esc.data(), sizeof(float) * esc.size(), cudaMemcpyHostToDevice));
        std::vector<uint8_t> b8(bid.begin(), bid.end());
        alloc_t(sc_bid_, std::max<size_t>(b8.size(), 1));
        HMC_CK(cudaMemcpy(sc_bid_.ptr, b8.data(), b8.size(), cudaMemcpyHostToDevice));
        plan_.buf_id = sc_bid_.as<uint8_t>();
        plan_.off = sc_off_.as<int>();
        alloc_t(db_desc_, sizeof(DbDesc) * dbd.size());
        HMC_CK(cudaMemcpy(db_desc_.ptr, dbd.data(), sizeof(DbDesc) * dbd.size(), cudaMemcpyHostToDevice));
    }

    Problem &p_;
    int C_, nut_ = 1, ntn_ = 1, bs_ = 128, pl_ = 64, nsplit_ = 1, num_sms_ = 148;
    long k_ = 0, nu_ = 0, ny_ = 0, nyp_ = 0;
    size_t bytes_ = 0;
    int *err_ = nullptr;
    DonNet br_, tr_;
    DevBuf yt_, ds_, u_part_, db0_part_, b0v_, gw_part_, db_desc_;
    DevBuf kind_, desc_, off_, erow_, ecol_, epack_, sc_off_, sc_bid_, heavy_, escale_;
    int nheavy_ = 0;
    float kb_ = 1.0f, kt_ = 1.0f;      // factors on dB and dT (powers of two; 1 for bf16)
    CUtensorMap ds_row_, ds_atom_, b_col_, b_hi_e_, b_lo_e_;
    int es_ = 256, nut_e_ = 1, ntn_e_ = 1;
    int max_clusters_ = 0;             // pair-kernel CTA pairs resident at once (0: no pair layer)
    cudaStream_t s2_ = nullptr;        // the trunk's stream inside an evaluation
    cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
    cudaStream_t sw_[2] = {nullptr, nullptr};   // the branch's and the trunk's weight gradients
    cudaEvent_t evw_fork_[2] = {nullptr, nullptr}, evw_join_[2] = {nullptr, nullptr};
    DevBuf u_acc_;
    ScatterPlan plan_;
    std::string tuning_;
};

}  // namespace

#if !HMC_F16
bool umma_engine_supports(const Problem &p, std::string *why)
{
    auto no = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    if (p.kind != HMC_NET_MLP) return no("only MLPs run on the tensor-core path (DeepONet: use FP32/FP64)");
    const NetDesc &nd = p.net;
    if (nd.L < 3) return no("need at least one hidden-to-hidden layer");
    const int w = nd.w[1];
    if (w < 1 || w > 256) return no("hidden width must be at most 256 (padded to 128 or 256)");
    for (int l = 1; l < nd.L; ++l)
        if (nd.w[l] != w) return no("all hidden layers must have the same width");
    if (nd.w[nd.L] != 1) return no("the output width must be 1");
    if (nd.w[0] < 1 || nd.w[0] > 8) return no("input width must be 1..8");
    for (int l = 0; l < nd.L - 1; ++l)
        if (nd.act[l] != HMC_ACT_TANH) return no("hidden activations must be tanh");
    if (nd.act[nd.L - 1] != HMC_ACT_IDENTITY) return no("the output activation must be the identity");
    for (int l = 0; l < nd.L; ++l)
        if (!nd.bias[l]) return no("every layer must have a bias");
    if (p.n < 1) return no("need at least one data point");
    return true;
}

#endif

#if HMC_F16
Engine *make_umma_engine_f16(Problem &p, int C) { return new UmmaEngine(p, C); }
std::vector<std::unique_ptr<EngineGroup>> make_umma_groups_f16(const std::vector<Engine *> &es,
                                                               const std::vector<long> &qoff,
                                                               const std::vector<long> &uoff, std::vector<bool> &grouped)
{
    return make_groups(es, qoff, uoff, grouped);
}
#else
Engine *make_umma_engine_bf16(Problem &p, int C) { return new UmmaEngine(p, C); }
std::vector<std::unique_ptr<EngineGroup>> make_umma_groups_bf16(const std::vector<Engine *> &es,
                                                                const std::vector<long> &qoff,
                                                                const std::vector<long> &uoff, std::vector<bool> &grouped)
{
    return make_groups(es, qoff, uoff, grouped);
}
#endif

#if !HMC_F16

bool don_engine_supports(const Problem &p, std::string *why)
{
    auto no = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    if (p.kind == HMC_NET_DEEPONET_UNALIGNED)
        return no("DeepONets with per-function query points run on the FP32/FP64 CUDA-core engines");
    if (p.kind != HMC_NET_DEEPONET) return no("not a DeepONet");
    for (const NetDesc *nd : {&p.branch, &p.trunk}) {
        if (nd->L < 2) return no("branch and trunk need a hidden layer");
        const int w = nd->w[1], pl = nd->w[nd->L];
        if (w % 64 != 0 || w > 256) return no("hidden widths must be 64, 128, 192 or 256");
        for (int l = 1; l < nd->L; ++l)
            if (nd->w[l] != w) return no("all hidden layers of a net must have the same width");
        if (pl % 64 != 0 || pl > 256) return no("the latent width must be 64, 128, 192 or 256");
        if (nd->w[0] < 1 || nd->w[0] > 256) return no("input widths must be 1..256");
        for (int l = 0; l + 1 < nd->L; ++l)
            if (nd->act[l] != HMC_ACT_TANH) return no("hidden activations must be tanh");
        if (nd->act[nd->L - 1] != HMC_ACT_IDENTITY) return no("the last layer of each net must be linear");
        for (int l = 0; l < nd->L; ++l)
            if (!nd->bias[l]) return no("every layer must have a bias");
    }
    if (p.n_u < 1 || p.n_y < 1) return no("empty data");
    return true;
}

#endif

#if HMC_F16
Engine *make_don_engine_f16(Problem &p, int C) { return new DonEngine(p, C); }
#else
Engine *make_don_engine_bf16(Problem &p, int C) { return new DonEngine(p, C); }

void expire_wait_run(int *err, long limit_ns, cudaStream_t s)
{
    k_expire_wait<<<1, 1, 0, s>>>(err, (unsigned long long)limit_ns);
    HMC_LAUNCH_CK();
}
#endif

}  // namespace hmc

#if !HMC_F16
// ---------------------------------------------------------------------------
// Diagnostic: one batched tensor-core GEMM, C[b][m][n] = sum_k A(m,k) B(n,k)
// ---------------------------------------------------------------------------
extern "C" hmc_status hmc_diag_umma_gemm(int M, int N, int K, int batch, int a_mn, int b_mn, const void *A,
                                         const void *B, float *Cout)
{
    using namespace hmc;
    try {
        HMC_REQUIRE(M >= 1 && K >= 1 && batch >= 1 && N >= 64 && N <= 256 && N % 64 == 0, "bad GEMM shape");
        HMC_REQUIRE(A && B && Cout, "NULL pointer");
        HMC_REQUIRE(K % 8 == 0 && M % 8 == 0, "row strides must be 16-byte multiples");
        CUtensorMap ma = a_mn ? make_map(A, M, K, batch, 64, 64) : make_map(A, K, M, batch, 64, 128);
        CUtensorMap mb = b_mn ? make_map(B, N, K, batch, 64, 64) : make_map(B, K, N, batch, 64, N);
        Params p{};
        p.M = M;
        p.N = N;
        p.K = K;
        p.kb_per_split = (K + BK - 1) / BK;
        p.out_f32 = Cout;
        int *err = nullptr;
        HMC_CK(cudaMalloc(&err, sizeof(int)));
        HMC_CK(cudaMemset(err, 0, sizeof(int)));
        p.err = err;
        dim3 grid((M + BM - 1) / BM, 1, batch);
        if (!a_mn && !b_mn) launch_umma<M_STORE_F32, false, false, false>(ma, mb, mb, p, grid, 0);
        else if (!a_mn && b_mn) launch_umma<M_STORE_F32, false, true, false>(ma, mb, mb, p, grid, 0);
        else if (a_mn && !b_mn) launch_umma<M_STORE_F32, true, false, false>(ma, mb, mb, p, grid, 0);
        else launch_umma<M_STORE_F32, true, true, false>(ma, mb, mb, p, grid, 0);
        HMC_CK(cudaDeviceSynchronize());
        int herr = 0;
        HMC_CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        cudaFree(err);
        if (herr) {
            set_error("a tensor-core pipeline wait timed out");
            return HMC_ERR_TIMEOUT;
        }
        return HMC_OK;
    } catch (const Fail &f) {
        return f.st;
    }
}
#endif  // !HMC_F16

#if HMC_F16
namespace hmc {
namespace {
__global__ void k_diag_tanh(const float *x, float *y, long n)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = act_tanh(x[i]);
}
}  // namespace
}  // namespace hmc

// The activation the fp16 engine applies, on n device floats (a diagnostic for its tests).
extern "C" hmc_status hmc_diag_tanh16(const float *x, float *y, long n)
{
    using namespace hmc;
    try {
        HMC_REQUIRE(x && y && n >= 0, "bad argument");
        if (n == 0) return HMC_OK;
        k_diag_tanh<<<(unsigned)std::min<long>((n + 255) / 256, 4096), 256>>>(x, y, n);
        HMC_LAUNCH_CK();
        HMC_CK(cudaDeviceSynchronize());
        return HMC_OK;
    } catch (const Fail &f) {
        return f.st;
    }
}
#endif

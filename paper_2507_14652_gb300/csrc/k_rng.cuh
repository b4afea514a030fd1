// k_rng.cuh -- counter-based momenta and Metropolis uniforms on the device.
//
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of a 64x64->128 multiply-xor S-box on a
// four-word counter with a Weyl-sequence key schedule.
//
// Gaussians by Box-Muller.  The logarithm and sin/cos are evaluated here from
// their power series with explicit round-to-nearest intrinsics (no fused
// multiply-add), so every value is fixed to the bit by IEEE-754 +, *, /, sqrt:
//   log x   : x = f 2^e, f in [sqrt(1/2), sqrt(2)), log f = 2 atanh((f-1)/(f+1)),
//             odd series of atanh through the s^25 term;
//   2 pi u  : u = m 2^-53; nearest quarter turn q found in integers, remainder
//             x = (m - q 2^51) * pi 2^-52 in [-pi/4, pi/4]; Taylor series of sin
//             through x^17 and cos through x^18, then the quadrant rotation.
// Stream layout: counter (block, chain, trajectory, 2*problem + s), key (seed, 0);
// s = 0 momenta (four components per block), s = 1 the Metropolis uniform.
#pragma once
#include <cstdint>

namespace hmc {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0;
        const uint64_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

// (0, 1] from the top 53 bits of a word.
__device__ __forceinline__ double unit53(uint64_t w)
{
    return __dmul_rn((double)((w >> 11) + 1ULL), 1.1102230246251565404236316680908203125e-16);
}

__device__ __forceinline__ double series_log(double x)
{
    const double LN2 = 0.693147180559945309417232121458176568;
    const double SQRT_HALF = 0.707106781186547524400844362104849039;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7ffULL) - 1022;
    double f = __longlong_as_double((long long)((bits & 0x000fffffffffffffULL) | 0x3fe0000000000000ULL));
    if (f < SQRT_HALF) {
        f = __dadd_rn(f, f);
        e -= 1;
    }
    const double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
    const double t = __dmul_rn(s, s);
    double p = 1.0 / 25.0;
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 23.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 21.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 19.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 17.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 15.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 13.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 11.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 9.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 7.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 5.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0 / 3.0);
    p = __dadd_rn(__dmul_rn(p, t), 1.0);
    const double lf = __dmul_rn(2.0, __dmul_rn(s, p));
    return __dadd_rn(__dmul_rn((double)e, LN2), lf);
}

__device__ __forceinline__ void series_sincos_2pi(uint64_t m, double &sn, double &cs)
{
    const double PI_2M52 = 3.14159265358979323846264338327950288 / 4503599627370496.0;
    const uint64_t q = (m + (1ULL << 50)) >> 51;
    const int64_t r = (int64_t)m - (int64_t)(q << 51);
    const double x = __dmul_rn((double)r, PI_2M52);
    const double x2 = __dmul_rn(x, x);
    double ps = 1.0 / 355687428096000.0;
    ps = __dadd_rn(__dmul_rn(ps, x2), -1.0 / 1307674368000.0);
    ps = __dadd_rn(__dmul_rn(ps, x2), 1.0 / 6227020800.0);
    ps = __dadd_rn(__dmul_rn(ps, x2), -1.0 / 39916800.0);
    ps = __dadd_rn(__dmul_rn(ps, x2), 1.0 / 362880.0);
    ps = __dadd_rn(__dmul_rn(ps, x2), -1.0 / 5040.0);
    ps = __dadd_rn(__dmul_rn(ps, x2), 1.0 / 120.0);
    ps = __dadd_rn(__dmul_rn(ps, x2), -1.0 / 6.0);
    ps = __dadd_rn(__dmul_rn(ps, x2), 1.0);
    const double sx = __dmul_rn(x, ps);
    double pc = -1.0 / 6402373705728000.0;
    pc = __dadd_rn(__dmul_rn(pc, x2), 1.0 / 20922789888000.0);
    pc = __dadd_rn(__dmul_rn(pc, x2), -1.0 / 87178291200.0);
    pc = __dadd_rn(__dmul_rn(pc, x2), 1.0 / 479001600.0);
    pc = __dadd_rn(__dmul_rn(pc, x2), -1.0 / 3628800.0);
    pc = __dadd_rn(__dmul_rn(pc, x2), 1.0 / 40320.0);
    pc = __dadd_rn(__dmul_rn(pc, x2), -1.0 / 720.0);
    pc = __dadd_rn(__dmul_rn(pc, x2), 1.0 / 24.0);
    pc = __dadd_rn(__dmul_rn(pc, x2), -1.0 / 2.0);
    pc = __dadd_rn(__dmul_rn(pc, x2), 1.0);
    const double cx = pc;
    switch ((int)(q & 3ULL)) {
    case 0: sn = sx; cs = cx; break;
    case 1: sn = cx; cs = -sx; break;
    case 2: sn = -sx; cs = -cx; break;
    default: sn = -cx; cs = sx; break;
    }
}

// The four momentum components 4*blk .. 4*blk+3 of (problem, chain, traj).
__device__ __forceinline__ void momenta4(uint64_t seed, uint64_t problem, uint64_t chain, uint64_t traj,
                                         uint64_t blk, double z[4])
{
    uint64_t c[4] = {blk, chain, traj, problem * 2ULL};
    philox4x64_10(c, seed, 0ULL);
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
        const double ua = unit53(c[2 * pr]);
        const uint64_t mb = (c[2 * pr + 1] >> 11) + 1ULL;
        const double R = __dsqrt_rn(__dmul_rn(-2.0, series_log(ua)));
        double sn, cs;
        series_sincos_2pi(mb, sn, cs);
        z[2 * pr] = __dmul_rn(R, cs);
        z[2 * pr + 1] = __dmul_rn(R, sn);
    }
}

__device__ __forceinline__ double mh_log_uniform(uint64_t seed, uint64_t problem, uint64_t chain, uint64_t traj)
{
    uint64_t c[4] = {0ULL, chain, traj, problem * 2ULL + 1ULL};
    philox4x64_10(c, seed, 0ULL);
    return series_log(unit53(c[0]));
}

}  // namespace hmc

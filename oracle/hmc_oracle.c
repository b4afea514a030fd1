/*
 * hmc_oracle.c -- plain, slow FP64 reference of the subset-HMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * What it computes (arXiv 2507.14652):
 *   - the network F_Theta: an MLP, or a DeepONet whose output is the dot
 *     product of a branch net on the input function and a trunk net on the
 *     query point plus a scalar bias (Sec. 4.2, App. A);
 *   - the potential U = -log[P(D|Theta) P(Theta)] with constants dropped
 *     (Sec. 2.2), for a Gaussian likelihood of width sigma summed over the
 *     full batch and an independent N(0, alpha^2) prior on the sampled subset
 *     Theta_s, the rest fixed at caller-supplied values (Sec. 3.2, Algorithm 2);
 *   - grad U by a hand-written reverse pass (chain rule, one data term at a
 *     time);
 *   - Hamilton's equations integrated by leapfrog (Sec. 2.2), kinetic energy
 *     K = p.p/2 for M = I;
 *   - the Metropolis step of Algorithm 1: accept when u < exp(H0 - H1), taken
 *     as log u < H0 - H1.
 *   - momenta p ~ N(0, I) from a counter-based Philox4x64-10 stream (Salmon,
 *     Moraes, Dror, Shaw, SC'11) through the Box-Muller transform, with the
 *     logarithm and sin/cos written here from their series so that the result
 *     is fixed to the bit by IEEE-754 +, *, / and sqrt alone.
 *
 * Build with -ffp-contract=off (no fused multiply-add) and without fast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LAYERS 16

enum { OR_ACT_IDENTITY = 0, OR_ACT_TANH = 1, OR_ACT_SIN = 2 };

typedef struct {
    int n_layers;
    int width[OR_MAX_LAYERS + 1];
    int act[OR_MAX_LAYERS];
    int bias[OR_MAX_LAYERS];
} or_net;

typedef struct {
    int kind;                 /* 0 = MLP, 1 = DeepONet (shared queries), 2 = DeepONet (own queries) */
    int out_bias;             /* DeepONet scalar output bias present */
    or_net net, branch, trunk;
    long n; int dx; const double *x;     /* MLP inputs  [n][dx] */
    const double *y;                     /* MLP targets [n][dout] */
    long n_u; int du; const double *u;   /* DeepONet branch inputs [n_u][du] */
    long n_y; int dy; const double *yq;  /* DeepONet trunk inputs [n_y][dy]; kind 2: [n_u][n_y][dy] */
    const double *t;                     /* DeepONet targets [n_u][n_y] */
    double noise_sigma, prior_sigma;
    const double *frozen; long P;        /* full parameter vector, values off the subset */
    const long *idx; long k;             /* ascending indices of the sampled subset */
} or_problem;

/* ------------------------------------------------------------------------ */
/* Network bookkeeping: W[out][in] row-major, then b[out], layer by layer.   */
/* ------------------------------------------------------------------------ */

long or_net_params(const or_net *nt)
{
    long p = 0;
    for (int l = 0; l < nt->n_layers; ++l)
        p += (long)nt->width[l] * nt->width[l + 1] + (nt->bias[l] ? nt->width[l + 1] : 0);
    return p;
}

long or_param_count(const or_problem *pr)
{
    if (pr->kind == 0) return or_net_params(&pr->net);
    return or_net_params(&pr->branch) + or_net_params(&pr->trunk) + (pr->out_bias ? 1 : 0);
}

static double act_value(int act, double z)
{
    if (act == OR_ACT_TANH) return tanh(z);
    if (act == OR_ACT_SIN) return sin(z);
    return z;
}

static double act_slope(int act, double z)
{
    if (act == OR_ACT_TANH) { double a = tanh(z); return 1.0 - a * a; }
    if (act == OR_ACT_SIN) return cos(z);
    return 1.0;
}

/* Per-sample activations of one net: z[l] and a[l] for l = 0..n_layers. */
typedef struct { double *buf; double *z[OR_MAX_LAYERS + 1]; double *a[OR_MAX_LAYERS + 1]; } or_tape;

static void tape_init(or_tape *tp, const or_net *nt)
{
    long tot = 0;
    for (int l = 0; l <= nt->n_layers; ++l) tot += 2L * nt->width[l];
    tp->buf = (double *)calloc((size_t)tot, sizeof(double));
    double *p = tp->buf;
    for (int l = 0; l <= nt->n_layers; ++l) {
        tp->z[l] = p; p += nt->width[l];
        tp->a[l] = p; p += nt->width[l];
    }
}

/* Forward pass for one input vector: z_l = W_l a_{l-1} + b_l, a_l = act_l(z_l). */
static void net_forward(const or_net *nt, const double *theta, const double *in, or_tape *tp)
{
    memcpy(tp->a[0], in, sizeof(double) * (size_t)nt->width[0]);
    memcpy(tp->z[0], in, sizeof(double) * (size_t)nt->width[0]);
    long off = 0;
    for (int l = 0; l < nt->n_layers; ++l) {
        int ni = nt->width[l], no = nt->width[l + 1];
        const double *W = theta + off;
        off += (long)no * ni;
        const double *b = NULL;
        if (nt->bias[l]) { b = theta + off; off += no; }
        for (int o = 0; o < no; ++o) {
            double s = 0.0;
            for (int i = 0; i < ni; ++i) s += W[(long)o * ni + i] * tp->a[l][i];
            if (b) s += b[o];
            tp->z[l + 1][o] = s;
            tp->a[l + 1][o] = act_value(nt->act[l], s);
        }
    }
}

/*
 * Reverse pass for one input vector.  dout = dL/d(a_L).  Adds dL/dtheta into
 * grad (same layout as theta).  delta_l = dL/dz_l; dW_l += delta_l a_{l-1}^T,
 * db_l += delta_l, and dL/da_{l-1} = W_l^T delta_l.
 */
static void net_backward(const or_net *nt, const double *theta, const or_tape *tp,
                         const double *dout, double *grad, double *work)
{
    int L = nt->n_layers;
    long offs_w[OR_MAX_LAYERS], offs_b[OR_MAX_LAYERS];
    long off = 0;
    int wmax = 0;
    for (int l = 0; l < L; ++l) {
        offs_w[l] = off; off += (long)nt->width[l + 1] * nt->width[l];
        offs_b[l] = -1;
        if (nt->bias[l]) { offs_b[l] = off; off += nt->width[l + 1]; }
    }
    for (int l = 0; l <= L; ++l) if (nt->width[l] > wmax) wmax = nt->width[l];
    double *delta = work, *dprev = work + wmax;
    for (int o = 0; o < nt->width[L]; ++o)
        delta[o] = dout[o] * act_slope(nt->act[L - 1], tp->z[L][o]);
    for (int l = L - 1; l >= 0; --l) {
        int ni = nt->width[l], no = nt->width[l + 1];
        const double *W = theta + offs_w[l];
        double *dW = grad + offs_w[l];
        for (int o = 0; o < no; ++o)
            for (int i = 0; i < ni; ++i) dW[(long)o * ni + i] += delta[o] * tp->a[l][i];
        if (offs_b[l] >= 0)
            for (int o = 0; o < no; ++o) grad[offs_b[l] + o] += delta[o];
        if (l > 0) {
            for (int i = 0; i < ni; ++i) {
                double s = 0.0;
                for (int o = 0; o < no; ++o) s += W[(long)o * ni + i] * delta[o];
                dprev[i] = s * act_slope(nt->act[l - 1], tp->z[l][i]);
            }
            double *tmp = delta; delta = dprev; dprev = tmp;
        }
    }
}

static int net_wmax(const or_net *nt)
{
    int w = 1;
    for (int l = 0; l <= nt->n_layers; ++l) if (nt->width[l] > w) w = nt->width[l];
    return w;
}

/* theta = frozen, then theta[idx[j]] = q[j]  (Sec. 3.2: Theta_~s fixed, Theta_s sampled) */
static double *assemble_theta(const or_problem *pr, const double *q)
{
    double *theta = (double *)malloc(sizeof(double) * (size_t)pr->P);
    memcpy(theta, pr->frozen, sizeof(double) * (size_t)pr->P);
    for (long j = 0; j < pr->k; ++j) theta[pr->idx[j]] = q[j];
    return theta;
}

/* DeepONet trunk rows: the n_y shared queries, or (kind 2) every function's own n_y queries. */
static long trunk_rows(const or_problem *pr)
{
    return pr->kind == 2 ? pr->n_u * pr->n_y : pr->n_y;
}

/* The trunk row of query j of input function i. */
static long trunk_row(const or_problem *pr, long i, long j)
{
    return pr->kind == 2 ? i * pr->n_y + j : j;
}

/* Network outputs for a full parameter vector: MLP [n][dout], DeepONet [n_u][n_y]. */
void or_forward(const or_problem *pr, const double *theta, double *f)
{
    if (pr->kind == 0) {
        const or_net *nt = &pr->net;
        int dout = nt->width[nt->n_layers];
        or_tape tp; tape_init(&tp, nt);
        for (long n = 0; n < pr->n; ++n) {
            net_forward(nt, theta, pr->x + n * pr->dx, &tp);
            for (int o = 0; o < dout; ++o) f[n * dout + o] = tp.a[nt->n_layers][o];
        }
        free(tp.buf);
        return;
    }
    const or_net *bn = &pr->branch, *tn = &pr->trunk;
    int p = bn->width[bn->n_layers];
    long pb = or_net_params(bn), pt = or_net_params(tn);
    double b0 = pr->out_bias ? theta[pb + pt] : 0.0;
    double *B = (double *)malloc(sizeof(double) * (size_t)(pr->n_u * p));
    long NT = trunk_rows(pr);
    double *T = (double *)malloc(sizeof(double) * (size_t)((NT > 0 ? NT : 1) * p));
    or_tape tb, tt; tape_init(&tb, bn); tape_init(&tt, tn);
    for (long i = 0; i < pr->n_u; ++i) {
        net_forward(bn, theta, pr->u + i * pr->du, &tb);
        memcpy(B + i * p, tb.a[bn->n_layers], sizeof(double) * (size_t)p);
    }
    for (long t = 0; t < NT; ++t) {
        net_forward(tn, theta + pb, pr->yq + t * pr->dy, &tt);
        memcpy(T + t * p, tt.a[tn->n_layers], sizeof(double) * (size_t)p);
    }
    for (long i = 0; i < pr->n_u; ++i)
        for (long j = 0; j < pr->n_y; ++j) {
            const double *Tj = T + trunk_row(pr, i, j) * p;
            double s = 0.0;
            for (int c = 0; c < p; ++c) s += B[i * p + c] * Tj[c];
            f[i * pr->n_y + j] = s + b0;
        }
    free(tb.buf); free(tt.buf); free(B); free(T);
}

/* Data rows: MLP data points, or DeepONet input functions (each with all its queries). */
long or_data_rows(const or_problem *pr)
{
    return pr->kind == 0 ? pr->n : pr->n_u;
}

/*
 * The part of U(q) and grad U(q) that comes from data rows [r0, r1), plus the
 * fraction w of the prior term, for one chain state q[k]:
 *   U_part = sum over the rows' data terms of (F - y)^2 / (2 sigma^2)
 *            + w sum_j q_j^2 / (2 alpha^2)
 * With r0 = 0, r1 = all rows and w = 1 this is U itself (or_energy_grad).
 * grad may be NULL (energy only).  Returns U_part.
 */
double or_energy_grad_rows(const or_problem *pr, const double *q, double *g, long r0, long r1, double w)
{
    double s2 = pr->noise_sigma * pr->noise_sigma;
    double a2 = pr->prior_sigma * pr->prior_sigma;
    double *theta = assemble_theta(pr, q);
    double *grad = (double *)calloc((size_t)pr->P, sizeof(double));
    double U = 0.0;

    if (pr->kind == 0) {
        const or_net *nt = &pr->net;
        int L = nt->n_layers, dout = nt->width[L];
        or_tape tp; tape_init(&tp, nt);
        int wmax = net_wmax(nt);
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * wmax));
        double *dout_v = (double *)malloc(sizeof(double) * (size_t)dout);
        for (long n = r0; n < r1; ++n) {
            net_forward(nt, theta, pr->x + n * pr->dx, &tp);
            for (int o = 0; o < dout; ++o) {
                double r = tp.a[L][o] - pr->y[n * dout + o];
                U += r * r / (2.0 * s2);
                dout_v[o] = r / s2;
            }
            net_backward(nt, theta, &tp, dout_v, grad, work);
        }
        free(work); free(dout_v); free(tp.buf);
    } else {
        const or_net *bn = &pr->branch, *tn = &pr->trunk;
        int p = bn->width[bn->n_layers];
        long pb = or_net_params(bn), pt = or_net_params(tn);
        double b0 = pr->out_bias ? theta[pb + pt] : 0.0;
        /* forward both nets, keeping every sample's tape for the reverse pass */
        /* the trunk rows these functions use: all shared queries, or their own */
        long NT = trunk_rows(pr);
        long t0 = pr->kind == 2 ? r0 * pr->n_y : 0, t1 = pr->kind == 2 ? r1 * pr->n_y : NT;
        or_tape *tb = (or_tape *)malloc(sizeof(or_tape) * (size_t)(pr->n_u > 0 ? pr->n_u : 1));
        or_tape *tt = (or_tape *)malloc(sizeof(or_tape) * (size_t)(NT > 0 ? NT : 1));
        for (long i = r0; i < r1; ++i) { tape_init(&tb[i], bn); net_forward(bn, theta, pr->u + i * pr->du, &tb[i]); }
        for (long t = t0; t < t1; ++t) { tape_init(&tt[t], tn); net_forward(tn, theta + pb, pr->yq + t * pr->dy, &tt[t]); }
        double *dB = (double *)calloc((size_t)(pr->n_u * p), sizeof(double));
        double *dT = (double *)calloc((size_t)((NT > 0 ? NT : 1) * p), sizeof(double));
        double db0 = 0.0;
        /* S_ij = <B_i, T_j> + b0;  dU/dS_ij = (S_ij - t_ij) / sigma^2 */
        for (long i = r0; i < r1; ++i) {
            const double *Bi = tb[i].a[bn->n_layers];
            for (long j = 0; j < pr->n_y; ++j) {
                long tr = trunk_row(pr, i, j);
                const double *Tj = tt[tr].a[tn->n_layers];
                double s = 0.0;
                for (int c = 0; c < p; ++c) s += Bi[c] * Tj[c];
                double r = s + b0 - pr->t[i * pr->n_y + j];
                U += r * r / (2.0 * s2);
                double dS = r / s2;
                for (int c = 0; c < p; ++c) {
                    dB[i * p + c] += dS * Tj[c];
                    dT[tr * p + c] += dS * Bi[c];
                }
                db0 += dS;
            }
        }
        int wmax = net_wmax(bn) > net_wmax(tn) ? net_wmax(bn) : net_wmax(tn);
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * wmax));
        for (long i = r0; i < r1; ++i) net_backward(bn, theta, &tb[i], dB + i * p, grad, work);
        for (long t = t0; t < t1; ++t) net_backward(tn, theta + pb, &tt[t], dT + t * p, grad + pb, work);
        if (pr->out_bias) grad[pb + pt] += db0;
        for (long i = r0; i < r1; ++i) free(tb[i].buf);
        for (long t = t0; t < t1; ++t) free(tt[t].buf);
        free(tb); free(tt); free(dB); free(dT); free(work);
    }

    /* prior on the sampled subset only: alpha-Gaussian, constants dropped */
    for (long j = 0; j < pr->k; ++j) U += w * (q[j] * q[j] / (2.0 * a2));
    if (g)
        for (long j = 0; j < pr->k; ++j) g[j] = grad[pr->idx[j]] + w * (q[j] / a2);
    free(grad);
    free(theta);
    return U;
}

/*
 * U(q) and grad U(q) for one chain state q[k].
 *   U = sum over data terms of (F - y)^2 / (2 sigma^2) + sum_j q_j^2 / (2 alpha^2)
 *   g_j = dU/dtheta_{idx_j}
 * grad may be NULL (energy only).  Returns U.
 */
double or_energy_grad(const or_problem *pr, const double *q, double *g)
{
    return or_energy_grad_rows(pr, q, g, 0, or_data_rows(pr), 1.0);
}

/* Several chain states at once (parallel over chains only; each sum keeps its order). */
void or_energy_grad_batch(const or_problem *pr, int C, const double *q, double *U, double *g, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int c = 0; c < C; ++c)
        U[c] = or_energy_grad(pr, q + (long)c * pr->k, g ? g + (long)c * pr->k : NULL);
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers                                             */
/* ------------------------------------------------------------------------ */

/* Philox4x64 with 10 rounds (Salmon et al., SC'11): multiply-xor S-box with a
 * Weyl key schedule. */
void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Top 53 bits of a word as a uniform on (0, 1]: ((w >> 11) + 1) * 2^-53. */
double or_unit_uniform(uint64_t w)
{
    return (double)((w >> 11) + 1) * 0x1p-53;
}

/* Natural log of a positive normal double.  x = f 2^e with f in [sqrt(1/2), sqrt(2)),
 * log f = 2 atanh(s), s = (f-1)/(f+1), atanh by its odd power series to s^25. */
double or_log(double x)
{
    const double LN2 = 0.69314718055994530941723212145817657;
    const double SQRT_HALF = 0.70710678118654752440084436210484904;
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int e = (int)((bits >> 52) & 0x7ff) - 1022;
    uint64_t fb = (bits & 0x000fffffffffffffULL) | 0x3fe0000000000000ULL;
    double f;
    memcpy(&f, &fb, sizeof f);
    if (f < SQRT_HALF) { f = f + f; e = e - 1; }
    double s = (f - 1.0) / (f + 1.0);
    double t = s * s;
    double p = 1.0 / 25.0;
    p = p * t + 1.0 / 23.0;
    p = p * t + 1.0 / 21.0;
    p = p * t + 1.0 / 19.0;
    p = p * t + 1.0 / 17.0;
    p = p * t + 1.0 / 15.0;
    p = p * t + 1.0 / 13.0;
    p = p * t + 1.0 / 11.0;
    p = p * t + 1.0 / 9.0;
    p = p * t + 1.0 / 7.0;
    p = p * t + 1.0 / 5.0;
    p = p * t + 1.0 / 3.0;
    p = p * t + 1.0;
    double lf = 2.0 * (s * p);
    return (double)e * LN2 + lf;
}

/* sin and cos of 2 pi u for u = m 2^-53, m in [1, 2^53].  Exact reduction to the
 * nearest quarter turn in integers, x = (4u - q) pi/2 in [-pi/4, pi/4], Taylor
 * series to x^17 (sin) and x^18 (cos). */
void or_sincos_2pi(uint64_t m, double *s_out, double *c_out)
{
    const double PI_2M52 = 3.14159265358979323846264338327950288 * 0x1p-52;
    uint64_t q = (m + (1ULL << 50)) >> 51;
    int64_t r = (int64_t)m - (int64_t)(q << 51);
    double x = (double)r * PI_2M52;
    double x2 = x * x;
    double ps = 1.0 / 355687428096000.0;
    ps = ps * x2 + -1.0 / 1307674368000.0;
    ps = ps * x2 + 1.0 / 6227020800.0;
    ps = ps * x2 + -1.0 / 39916800.0;
    ps = ps * x2 + 1.0 / 362880.0;
    ps = ps * x2 + -1.0 / 5040.0;
    ps = ps * x2 + 1.0 / 120.0;
    ps = ps * x2 + -1.0 / 6.0;
    ps = ps * x2 + 1.0;
    double sx = x * ps;
    double pc = -1.0 / 6402373705728000.0;
    pc = pc * x2 + 1.0 / 20922789888000.0;
    pc = pc * x2 + -1.0 / 87178291200.0;
    pc = pc * x2 + 1.0 / 479001600.0;
    pc = pc * x2 + -1.0 / 3628800.0;
    pc = pc * x2 + 1.0 / 40320.0;
    pc = pc * x2 + -1.0 / 720.0;
    pc = pc * x2 + 1.0 / 24.0;
    pc = pc * x2 + -1.0 / 2.0;
    pc = pc * x2 + 1.0;
    double cx = pc;
    switch (q & 3) {
    case 0: *s_out = sx; *c_out = cx; break;
    case 1: *s_out = cx; *c_out = -sx; break;
    case 2: *s_out = -sx; *c_out = -cx; break;
    default: *s_out = -cx; *c_out = sx; break;
    }
}

/*
 * Momentum component j of chain `chain` on trajectory `traj` (Algorithm 1: p ~ N(0, M), M = I).
 * One Philox block per four components: counter (j/4, chain, traj, 2*problem + 0),
 * key (seed, 0).  Words (w0,w1) give components 4b, 4b+1 and (w2,w3) give 4b+2, 4b+3
 * by Box-Muller: R = sqrt(-2 log u_a), z = R cos(2 pi u_b), R sin(2 pi u_b).
 */
double or_momentum(uint64_t seed, uint64_t problem, uint64_t chain, uint64_t traj, uint64_t j)
{
    uint64_t ctr[4] = { j >> 2, chain, traj, problem * 2 + 0 };
    uint64_t key[2] = { seed, 0 };
    uint64_t w[4];
    or_philox4x64_10(ctr, key, w);
    int pair = (int)((j & 3) >> 1);
    double ua = or_unit_uniform(w[2 * pair]);
    uint64_t mb = (w[2 * pair + 1] >> 11) + 1;
    double R = sqrt(-2.0 * or_log(ua));
    double sn, cs;
    or_sincos_2pi(mb, &sn, &cs);
    return (j & 1) ? R * sn : R * cs;
}

/* The Metropolis uniform of Algorithm 1 for (chain, traj): counter (0, chain, traj, 2*problem + 1). */
double or_mh_uniform(uint64_t seed, uint64_t problem, uint64_t chain, uint64_t traj)
{
    uint64_t ctr[4] = { 0, chain, traj, problem * 2 + 1 };
    uint64_t key[2] = { seed, 0 };
    uint64_t w[4];
    or_philox4x64_10(ctr, key, w);
    return or_unit_uniform(w[0]);
}

/* ------------------------------------------------------------------------ */
/* Integrator and sampler                                                   */
/* ------------------------------------------------------------------------ */

/*
 * Leapfrog (kick-drift-kick) for L steps of size eps, in place on q, p.
 * Uses and updates the cached energy and gradient at q: on entry *U, g hold
 * U(q), grad U(q); on exit they hold the values at the final q.
 *   p <- p - eps/2 g;  repeat L times { q <- q + eps p; g <- grad U(q);
 *                                        p <- p - eps g  (eps/2 on the last) }
 */
void or_leapfrog(const or_problem *pr, double *q, double *p, double eps, int L, double *U, double *g)
{
    long k = pr->k;
    double half = 0.5 * eps;
    if (L <= 0) return;   /* zero steps: the identity map */
    for (long j = 0; j < k; ++j) p[j] = p[j] - half * g[j];
    for (int s = 1; s <= L; ++s) {
        for (long j = 0; j < k; ++j) q[j] = q[j] + eps * p[j];
        *U = or_energy_grad(pr, q, g);
        double h = (s == L) ? half : eps;
        for (long j = 0; j < k; ++j) p[j] = p[j] - h * g[j];
    }
}

static double kinetic(const double *p, long k)
{
    double K = 0.0;
    for (long j = 0; j < k; ++j) K += p[j] * p[j];
    return 0.5 * K;
}

/*
 * HMC on the subset (Algorithm 2's sampling loop).  For each chain c and each
 * trajectory t = first_traj + i:
 *   p ~ N(0, I);  H0 = U(q) + K(p);  (q*, p*) = leapfrog(q, p);  H1 = U(q*) + K(p*)
 *   u ~ U(0, 1];  accept iff log u < H0 - H1 (a NaN difference rejects)
 *   record q (the new state if accepted, the old one otherwise), the flag and dH = H1 - H0.
 * samples [n][C][k], accepted [n][C], dH [n][C], q_last [C][k] (may be NULL).
 */
void or_sample(const or_problem *pr, const double *q0, int C, double eps, int L, long n,
               uint64_t seed, uint64_t problem, long first_traj,
               double *samples, unsigned char *accepted, double *dH, double *q_last, int nthreads)
{
    long k = pr->k;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int c = 0; c < C; ++c) {
        double *q = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *qn = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *p = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *g = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *gn = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        memcpy(q, q0 + (long)c * k, sizeof(double) * (size_t)k);
        double U = or_energy_grad(pr, q, g);
        for (long i = 0; i < n; ++i) {
            uint64_t traj = (uint64_t)(first_traj + i);
            for (long j = 0; j < k; ++j) p[j] = or_momentum(seed, problem, (uint64_t)c, traj, (uint64_t)j);
            double H0 = U + kinetic(p, k);
            memcpy(qn, q, sizeof(double) * (size_t)k);
            memcpy(gn, g, sizeof(double) * (size_t)k);
            double Un = U;
            or_leapfrog(pr, qn, p, eps, L, &Un, gn);
            double H1 = Un + kinetic(p, k);
            double lu = or_log(or_mh_uniform(seed, problem, (uint64_t)c, traj));
            int acc = lu < H0 - H1;
            if (acc) {
                memcpy(q, qn, sizeof(double) * (size_t)k);
                memcpy(g, gn, sizeof(double) * (size_t)k);
                U = Un;
            }
            if (samples) memcpy(samples + (i * C + c) * k, q, sizeof(double) * (size_t)k);
            if (accepted) accepted[i * C + c] = (unsigned char)acc;
            if (dH) dH[i * C + c] = H1 - H0;
        }
        if (q_last) memcpy(q_last + (long)c * k, q, sizeof(double) * (size_t)k);
        free(q); free(qn); free(p); free(g); free(gn);
    }
}

/* ------------------------------------------------------------------------ */
/* Symmetric split integrator over data batches                              */
/* ------------------------------------------------------------------------ */

/* Batch m of M: data rows [floor(m R / M), floor((m + 1) R / M)) of the R rows. */
void or_batch_rows(const or_problem *pr, int M, int m, long *r0, long *r1)
{
    long R = or_data_rows(pr);
    *r0 = (long)(((__int128)R * m) / M);
    *r1 = (long)(((__int128)R * (m + 1)) / M);
}

/*
 * The split Hamiltonian of symmetric split HMC (Sec. 4.2.3 uses it for the full-HMC
 * runs): H = sum_m H_m with H_m = U_m(q) + K(p)/M, where U_m holds the likelihood of
 * data batch m and 1/M of the prior.  One step of size eps is the forward sweep
 * m = 1..M of  [p <- p - eps/2 grad U_m(q);  q <- q + eps/(2M) p]  followed by the
 * backward sweep m = M..1 of  [q <- q + eps/(2M) p;  p <- p - eps/2 grad U_m(q)]:
 * a palindromic composition of exact sub-flows, so the map is symplectic and
 * reversible (the Metropolis test stays exact), of second order, and for M = 1 it is
 * the leapfrog step.  L steps, in place on q and p.
 */
void or_split_leapfrog(const or_problem *pr, int M, double *q, double *p, double eps, int L)
{
    long k = pr->k;
    double *g = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    double kick = 0.5 * eps, drift = eps / (2.0 * M), w = 1.0 / M;
    for (int s = 0; s < L; ++s) {
        for (int m = 0; m < M; ++m) {
            long r0, r1;
            or_batch_rows(pr, M, m, &r0, &r1);
            or_energy_grad_rows(pr, q, g, r0, r1, w);
            for (long j = 0; j < k; ++j) p[j] = p[j] - kick * g[j];
            for (long j = 0; j < k; ++j) q[j] = q[j] + drift * p[j];
        }
        for (int m = M - 1; m >= 0; --m) {
            long r0, r1;
            or_batch_rows(pr, M, m, &r0, &r1);
            for (long j = 0; j < k; ++j) q[j] = q[j] + drift * p[j];
            or_energy_grad_rows(pr, q, g, r0, r1, w);
            for (long j = 0; j < k; ++j) p[j] = p[j] - kick * g[j];
        }
    }
    free(g);
}

/*
 * HMC with the split integrator: as or_sample, with (q*, p*) from or_split_leapfrog
 * and H = U + K evaluated on the whole data set at both ends.
 */
void or_split_sample(const or_problem *pr, int M, const double *q0, int C, double eps, int L, long n,
                     uint64_t seed, uint64_t problem, long first_traj,
                     double *samples, unsigned char *accepted, double *dH, double *q_last, int nthreads)
{
    long k = pr->k;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int c = 0; c < C; ++c) {
        double *q = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *qn = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        double *p = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
        memcpy(q, q0 + (long)c * k, sizeof(double) * (size_t)k);
        double U = or_energy_grad(pr, q, NULL);
        for (long i = 0; i < n; ++i) {
            uint64_t traj = (uint64_t)(first_traj + i);
            for (long j = 0; j < k; ++j) p[j] = or_momentum(seed, problem, (uint64_t)c, traj, (uint64_t)j);
            double H0 = U + kinetic(p, k);
            memcpy(qn, q, sizeof(double) * (size_t)k);
            or_split_leapfrog(pr, M, qn, p, eps, L);
            double Un = or_energy_grad(pr, qn, NULL);
            double H1 = Un + kinetic(p, k);
            double lu = or_log(or_mh_uniform(seed, problem, (uint64_t)c, traj));
            int acc = lu < H0 - H1;
            if (acc) {
                memcpy(q, qn, sizeof(double) * (size_t)k);
                U = Un;
            }
            if (samples) memcpy(samples + (i * C + c) * k, q, sizeof(double) * (size_t)k);
            if (accepted) accepted[i * C + c] = (unsigned char)acc;
            if (dH) dH[i * C + c] = H1 - H0;
        }
        if (q_last) memcpy(q_last + (long)c * k, q, sizeof(double) * (size_t)k);
        free(q); free(qn); free(p);
    }
}

/* ------------------------------------------------------------------------ */
/* Sensitivities and the truncation of the parameter set (Sec. 3.1)          */
/* ------------------------------------------------------------------------ */

/*
 * The sensitivity of the network output to each parameter around the VI mean
 * (Sec. 3.1, the equation defining S_i^2): with F evaluated at theta = mu,
 *   S2[i] = sd[i]^2 / N_d * sum over the data terms of (dF/dtheta_i)^2,
 * the data terms being the outputs F_o(x_n) of an MLP (N_d = n * dout) or the
 * DeepONet outputs S_jk = <B_j, T_k> + b0 (N_d = n_u * n_y).  The derivative of
 * each data term is one reverse pass seeded with that term alone.
 */
void or_sensitivity(const or_problem *pr, const double *mu, const double *sd, double *S2)
{
    long P = or_param_count(pr);
    double *acc = (double *)calloc((size_t)P, sizeof(double));
    double *grad = (double *)malloc(sizeof(double) * (size_t)P);
    double Nd;
    if (pr->kind == 0) {
        const or_net *nt = &pr->net;
        int L = nt->n_layers, dout = nt->width[L];
        Nd = (double)pr->n * dout;
        or_tape tp; tape_init(&tp, nt);
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * net_wmax(nt)));
        double *seed = (double *)malloc(sizeof(double) * (size_t)dout);
        for (long n = 0; n < pr->n; ++n) {
            net_forward(nt, mu, pr->x + n * pr->dx, &tp);
            for (int o = 0; o < dout; ++o) {
                for (int c = 0; c < dout; ++c) seed[c] = c == o ? 1.0 : 0.0;
                memset(grad, 0, sizeof(double) * (size_t)P);
                net_backward(nt, mu, &tp, seed, grad, work);
                for (long i = 0; i < P; ++i) acc[i] += grad[i] * grad[i];
            }
        }
        free(tp.buf); free(work); free(seed);
    } else {
        const or_net *bn = &pr->branch, *tn = &pr->trunk;
        int p = bn->width[bn->n_layers];
        long pb = or_net_params(bn);
        Nd = (double)pr->n_u * pr->n_y;
        or_tape *tb = (or_tape *)malloc(sizeof(or_tape) * (size_t)(pr->n_u > 0 ? pr->n_u : 1));
        long NT = trunk_rows(pr);
        or_tape *tt = (or_tape *)malloc(sizeof(or_tape) * (size_t)(NT > 0 ? NT : 1));
        for (long j = 0; j < pr->n_u; ++j) { tape_init(&tb[j], bn); net_forward(bn, mu, pr->u + j * pr->du, &tb[j]); }
        for (long t = 0; t < NT; ++t) { tape_init(&tt[t], tn); net_forward(tn, mu + pb, pr->yq + t * pr->dy, &tt[t]); }
        int wmax = net_wmax(bn) > net_wmax(tn) ? net_wmax(bn) : net_wmax(tn);
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * wmax));
        for (long j = 0; j < pr->n_u; ++j)
            for (long k = 0; k < pr->n_y; ++k) {
                /* dS_jk/dB_j = T_k and dS_jk/dT_k = B_j; dS_jk/db0 = 1 */
                const or_tape *tk = &tt[trunk_row(pr, j, k)];
                memset(grad, 0, sizeof(double) * (size_t)P);
                net_backward(bn, mu, &tb[j], tk->a[tn->n_layers], grad, work);
                net_backward(tn, mu + pb, tk, tb[j].a[bn->n_layers], grad + pb, work);
                if (pr->out_bias) grad[P - 1] = 1.0;
                for (long i = 0; i < P; ++i) acc[i] += grad[i] * grad[i];
            }
        (void)p;
        for (long j = 0; j < pr->n_u; ++j) free(tb[j].buf);
        for (long t = 0; t < NT; ++t) free(tt[t].buf);
        free(tb); free(tt); free(work);
    }
    for (long i = 0; i < P; ++i) S2[i] = sd[i] * sd[i] / Nd * acc[i];
    free(acc); free(grad);
}

static const double *g_rank_S2;   /* key of the ordering below (single-threaded use) */

/* S2 descending; equal values by ascending parameter index. */
static int rank_cmp(const void *a, const void *b)
{
    long i = *(const long *)a, j = *(const long *)b;
    double si = g_rank_S2[i], sj = g_rank_S2[j];
    if (si > sj) return -1;
    if (si < sj) return 1;
    return (i > j) - (i < j);
}

/*
 * The truncation of Sec. 3.1 (the equation defining N-hat): with the parameters
 * ordered from most to least sensitive (ties: lower index first),
 *   N_hat = max{ N_T : sum_{r <= N_T} S2_(r) / sum_i S2_i <= tau },
 * and the sampled subset Theta_s is the first N_hat of that order (Sec. 3.2).
 * The total is summed in index order, the prefix in rank order, both in FP64.  An
 * all-zero S2 gives N_hat = 0.  mask[P] receives 1 for Theta_s; order[P] (may be
 * NULL) the ranking.  Returns N_hat.
 */
long or_truncate(const double *S2, long P, double tau, unsigned char *mask, long *order)
{
    long *ord = (long *)malloc(sizeof(long) * (size_t)(P > 0 ? P : 1));
    for (long i = 0; i < P; ++i) ord[i] = i;
    g_rank_S2 = S2;
    qsort(ord, (size_t)P, sizeof(long), rank_cmp);
    double total = 0.0;
    for (long i = 0; i < P; ++i) total += S2[i];
    long nhat = 0;
    if (total > 0.0) {
        double cum = 0.0;
        for (long r = 0; r < P; ++r) {
            cum += S2[ord[r]];
            if (cum / total <= tau) nhat = r + 1;
            else break;
        }
    }
    for (long i = 0; i < P; ++i) mask[i] = 0;
    for (long r = 0; r < nhat; ++r) mask[ord[r]] = 1;
    if (order) memcpy(order, ord, sizeof(long) * (size_t)P);
    free(ord);
    return nhat;
}

/* ------------------------------------------------------------------------ */
/* Posterior predictive (Sec. 4.2.1)                                        */
/* ------------------------------------------------------------------------ */

/*
 * The network's outputs on the problem's inputs for every posterior sample
 * q_s [S][k] (theta = frozen with the subset replaced by q_s), reduced over the
 * samples to their mean and standard deviation per output,
 *   mean = (1/S) sum_s F_s,   std = sqrt((1/S) sum_s (F_s - mean)^2),
 * two passes over the samples.  Outputs are [n][dout] (MLP) or [n_u][n_y] (DeepONet).
 */
void or_predict(const or_problem *pr, const double *samples, long S, double *mean, double *sdev)
{
    long nout = pr->kind == 0 ? pr->n * pr->net.width[pr->net.n_layers] : pr->n_u * pr->n_y;
    double *f = (double *)malloc(sizeof(double) * (size_t)(nout > 0 ? nout : 1));
    for (long i = 0; i < nout; ++i) { mean[i] = 0.0; sdev[i] = 0.0; }
    for (int pass = 0; pass < 2; ++pass)
        for (long s = 0; s < S; ++s) {
            double *theta = assemble_theta(pr, samples + s * pr->k);
            or_forward(pr, theta, f);
            for (long i = 0; i < nout; ++i) {
                if (pass == 0) mean[i] += f[i];
                else { double d = f[i] - mean[i]; sdev[i] += d * d; }
            }
            free(theta);
            if (pass == 0 && s == S - 1)
                for (long i = 0; i < nout; ++i) mean[i] /= (double)S;
        }
    for (long i = 0; i < nout; ++i) sdev[i] = sqrt(sdev[i] / (double)S);
    free(f);
}

/*
 * Mean relative L2 error of a prediction (Sec. 4.2.1): (1/N) sum_i ||Y_i - Yp_i||_2 / ||Y_i||_2
 * over N rows of length m (a DeepONet: one row per input function over its queries;
 * an MLP: the whole output as one row).
 */
double or_rel_l2(const double *Y, const double *Yp, long N, long m)
{
    double acc = 0.0;
    for (long i = 0; i < N; ++i) {
        double e = 0.0, y = 0.0;
        for (long j = 0; j < m; ++j) {
            double d = Y[i * m + j] - Yp[i * m + j];
            e += d * d;
            y += Y[i * m + j] * Y[i * m + j];
        }
        acc += sqrt(e) / sqrt(y);
    }
    return acc / (double)N;
}

/*
 * abc_oracle.c -- CPU oracle for ABC rejection sampling of the six-compartment
 * stochastic COVID-19 model (Kulkarni, Krell, Nabarro, Moritz 2020).
 *
 * TEST INFRASTRUCTURE. This file is the slow, plain, obviously-correct
 * restatement of the method that the CUDA library is checked against. Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * build, load or call it. It shares no code, header, table or helper with the
 * CUDA library, and the library never calls it.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fno-fast-math -shared -fPIC -pthread
 * (no FMA contraction: every float operation below is one IEEE-754 binary32
 * operation rounded to nearest-even, which is the exact-mode definition).
 *
 * What the paper fixes (cited by section / equation):
 *   theta = [alpha0, alpha, n, beta, gamma, delta, eta, kappa]      Sec. 2.1, Eq. 1
 *   prior U(0, [1, 100, 2, 1, 1, 1, 1, 2])                          Sec. 2.1, Eq. 2
 *   state X = [S, I, A, R, D, Ru]                                   Sec. 2.1, Eq. 3
 *   g = alpha0 + alpha / (1 + (A+R+D)^n)                            Sec. 2.1, Eq. 4
 *   init Ru=0, I0=kappa*A0, S=P-(A0+R0+D0+I0)                       Sec. 2.1 (first step)
 *   h = (g S I/P, gamma I, beta A, delta A, beta eta I)             Sec. 2.1, Eq. 5
 *   transitions ~ floor(Normal(h, .)) (Poisson approximation)       Sec. 2.1 (third step)
 *   apply S->I, I->A, A->R, A->D, I->Ru in h order                  Sec. 2.1 (fourth step)
 *   Euclidean distance of simulated vs observed [A,R,D]; accept
 *   when dist <= eps                                                Sec. 2.2, Eq. 7
 *   batched rejection over independent samples                     Sec. 3.1
 *
 * Readings where the paper is silent or ambiguous (each one is a choice the
 * CUDA library makes identically, independently written):
 *   R1 RNG: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter =
 *      (i_lo, i_hi, k, 4*stream + g). k = 0 gives the prior draw (g = 0 -> theta0..3,
 *      g = 1 -> theta4..7); k >= 1 gives days 2k-1 and 2k (g = 0,1,2 -> words w0..w11).
 *   R2 Uniform from a word: u = bits((w & 0x7FFFFF) | 0x3F800000) - (1 - 2^-24), in (0,1).
 *   R3 Normals: Box-Muller pair p = 0..4 uses (w[2p], w[2p+1]):
 *      r = sqrt(-2 ln2 * log2(u1)), z[2p] = r cos(pi*2u2), z[2p+1] = r sin(pi*2u2).
 *      Day 2k-1 uses z[0..4], day 2k uses z[5..9] (one per transition, in h order).
 *   R4 "variance sqrt(h)" read as standard deviation sqrt(h): x = h + sqrt(h) z.
 *      The literal reading (std h^(1/4)) is kept behind variance_literal.
 *   R5 n = min(max(floor(x), 0), c), floor saturating to int32, NaN -> 0, c = the
 *      source count still available (S; I; I - n(I->A); A; A - n(A->R)).
 *   R6 compartments are int32; rates are float32 from round-to-nearest int->float.
 *   R7 distance: exact uint64 sum over days 1..T of the three squared count
 *      differences (saturating at 2^63), then dist = sqrt((double)acc).
 *   R8 T = number of simulated days; observed series has T+1 columns, column 0 is
 *      the initial condition (A0, R0, D0).
 *   R9 I0 = min(max(floor(kappa * A0), 0), P - A0 - R0 - D0).
 *   R10 exact-mode log2 / exp2 / sinpi / cospi are the fixed float32 series below.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include "abc_oracle.h"

/* ------------------------------------------------------------------------- */
/* bit helpers                                                               */
/* ------------------------------------------------------------------------- */
static float f_from_bits(uint32_t b) { float f; memcpy(&f, &b, sizeof f); return f; }
static uint32_t bits_of_f(float f) { uint32_t b; memcpy(&b, &f, sizeof b); return b; }

/* ------------------------------------------------------------------------- */
/* R1: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC'11). Ten rounds; each round multiplies counter    */
/* words 0 and 2 by the two round multipliers, swaps and mixes the high      */
/* halves with words 1, 3 and the key, then bumps the key by the Weyl        */
/* constants (golden ratio, sqrt(3)-1).                                      */
/* ------------------------------------------------------------------------- */
#define PHILOX_MUL_A 0xD2511F53u
#define PHILOX_MUL_B 0xCD9E8D57u
#define PHILOX_WEYL_A 0x9E3779B9u
#define PHILOX_WEYL_B 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t pa = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
        uint64_t pb = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
        uint32_t a_hi = (uint32_t)(pa >> 32), a_lo = (uint32_t)pa;
        uint32_t b_hi = (uint32_t)(pb >> 32), b_lo = (uint32_t)pb;
        uint32_t y0 = b_hi ^ x1 ^ k0;
        uint32_t y1 = b_lo;
        uint32_t y2 = a_hi ^ x3 ^ k1;
        uint32_t y3 = a_lo;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_WEYL_A;
        k1 += PHILOX_WEYL_B;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* R1: the 4 words of block g of day-pair k for sample i. */
static void rng_block(uint64_t seed, uint32_t stream, uint64_t i, uint32_t k, uint32_t g,
                      uint32_t out[4])
{
    uint32_t ctr[4] = { (uint32_t)i, (uint32_t)(i >> 32), k, (stream << 2) | g };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    oracle_philox4x32_10(ctr, key, out);
}

/* R2: uniform in (0,1) on the lattice (2m+1) 2^-24, m = the low 23 bits of w. */
float oracle_uniform(uint32_t w)
{
    float one_plus = f_from_bits((w & 0x007FFFFFu) | 0x3F800000u);   /* 1 + m 2^-23 */
    float one_minus_half_ulp = f_from_bits(0x3F7FFFFFu);    /* 1 - 2^-24  */
    return one_plus - one_minus_half_ulp;                   /* exact      */
}

/* ------------------------------------------------------------------------- */
/* R10: exact-mode transcendentals. Each is a fixed sequence of binary32     */
/* operations; the coefficients are the correctly rounded binary32 values of */
/* the named real numbers (checked against high-precision values in tests).  */
/* ------------------------------------------------------------------------- */
static const float LN2_F = 0x1.62e430p-1f;          /* RN(ln 2)        */
static const float NEG_2LN2_F = -0x1.62e430p+0f;    /* RN(-2 ln 2)     */
static const float PI_F = 0x1.921fb6p+1f;           /* RN(pi)          */
static const float SQRT2_F = 0x1.6a09e6p+0f;        /* RN(sqrt 2)      */

/* log2 m = (2/ln2) atanh(s), s = (m-1)/(m+1): c_k = RN(2 / (k ln 2)). */
static const float LOG_C1 = 0x1.715476p+1f;
static const float LOG_C3 = 0x1.ec709ep-1f;
static const float LOG_C5 = 0x1.2776c6p-1f;
static const float LOG_C7 = 0x1.a61762p-2f;
static const float LOG_C9 = 0x1.484b14p-2f;

/* e^t Taylor coefficients RN(1/j!), j = 2..7. */
static const float EXP_C2 = 0x1.000000p-1f;
static const float EXP_C3 = 0x1.555556p-3f;
static const float EXP_C4 = 0x1.555556p-5f;
static const float EXP_C5 = 0x1.111112p-7f;
static const float EXP_C6 = 0x1.6c16c2p-10f;
static const float EXP_C7 = 0x1.a01a02p-13f;

/* sin Taylor coefficients RN((-1)^j / (2j+1)!), j = 1..4. */
static const float SIN_C3 = -0x1.555556p-3f;
static const float SIN_C5 = 0x1.111112p-7f;
static const float SIN_C7 = -0x1.a01a02p-13f;
static const float SIN_C9 = 0x1.71de3ap-19f;

/* cos Taylor coefficients RN((-1)^j / (2j)!), j = 1..5. */
static const float COS_C2 = -0x1.000000p-1f;
static const float COS_C4 = 0x1.555556p-5f;
static const float COS_C6 = -0x1.6c16c2p-10f;
static const float COS_C8 = 0x1.a01a02p-16f;
static const float COS_C10 = -0x1.27e4fcp-22f;

/* log2(x) for x a positive normal float: split x = 2^e m, fold m into
 * (sqrt(1/2), sqrt(2)], then log2 m from the odd atanh series in s. */
float oracle_log2x(float x)
{
    uint32_t b = bits_of_f(x);
    int e = (int)(b >> 23) - 127;
    float m = f_from_bits((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > SQRT2_F) {
        m = m * 0.5f;
        e = e + 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = LOG_C9;
    p = p * s2;
    p = p + LOG_C7;
    p = p * s2;
    p = p + LOG_C5;
    p = p * s2;
    p = p + LOG_C3;
    p = p * s2;
    p = p + LOG_C1;
    float frac = s * p;
    return (float)e + frac;
}

/* 2^y: y = k + f with k = rint(y), |f| <= 1/2; 2^f = e^(f ln2) by the
 * degree-7 Taylor polynomial; scale by 2^k built from its exponent bits.
 * y >= 127.5 (or NaN) gives +inf, y < -125.5 gives 0. */
float oracle_exp2x(float y)
{
    if (!(y < 127.5f)) return INFINITY;
    if (y < -125.5f) return 0.0f;
    float kf = rintf(y);
    float f = y - kf;
    float t = f * LN2_F;
    float p = EXP_C7;
    p = p * t;
    p = p + EXP_C6;
    p = p * t;
    p = p + EXP_C5;
    p = p * t;
    p = p + EXP_C4;
    p = p * t;
    p = p + EXP_C3;
    p = p * t;
    p = p + EXP_C2;
    p = p * t;
    p = p + 1.0f;
    p = p * t;
    p = p + 1.0f;
    int k = (int)kf;
    float scale = f_from_bits((uint32_t)(k + 127) << 23);
    return p * scale;
}

/* sin(pi v) and cos(pi v) for |v| <= 2^20: quarter-turn reduction
 * v = q/2 + w (exact), |w| <= 1/4, t = pi w, Taylor series in t,
 * then the quadrant q mod 4 selects and signs the pair. */
void oracle_sincospix(float v, float* sin_out, float* cos_out)
{
    float qf = rintf(v * 2.0f);
    float w = v - qf * 0.5f;
    float t = w * PI_F;
    float t2 = t * t;
    float ps = SIN_C9;
    ps = ps * t2;
    ps = ps + SIN_C7;
    ps = ps * t2;
    ps = ps + SIN_C5;
    ps = ps * t2;
    ps = ps + SIN_C3;
    ps = ps * t2;
    float sn = t * ps;
    sn = sn + t;
    float pc = COS_C10;
    pc = pc * t2;
    pc = pc + COS_C8;
    pc = pc * t2;
    pc = pc + COS_C6;
    pc = pc * t2;
    pc = pc + COS_C4;
    pc = pc * t2;
    pc = pc + COS_C2;
    pc = pc * t2;
    float cs = pc + 1.0f;
    int q = ((int)qf) & 3;
    switch (q) {
    case 0: *sin_out = sn;  *cos_out = cs;  break;
    case 1: *sin_out = cs;  *cos_out = -sn; break;
    case 2: *sin_out = -sn; *cos_out = -cs; break;
    default: *sin_out = -cs; *cos_out = sn; break;
    }
}

/* R3: one Box-Muller pair from two Philox words. */
void oracle_box_muller(uint32_t w_radius, uint32_t w_angle, float z[2])
{
    float u1 = oracle_uniform(w_radius);
    float u2 = oracle_uniform(w_angle);
    float l = oracle_log2x(u1);
    float r2 = NEG_2LN2_F * l;
    float r = sqrtf(r2);
    float v = u2 * 2.0f;
    float sv, cv;
    oracle_sincospix(v, &sv, &cv);
    z[0] = r * cv;
    z[1] = r * sv;
}

/* R1 + R3: the ten normals of day-pair k (k >= 1) of sample i. */
void oracle_day_pair_normals(uint64_t seed, uint32_t stream, uint64_t i, uint32_t k, float z[10])
{
    uint32_t w[12];
    rng_block(seed, stream, i, k, 0, w + 0);
    rng_block(seed, stream, i, k, 1, w + 4);
    rng_block(seed, stream, i, k, 2, w + 8);
    for (int p = 0; p < 5; ++p)
        oracle_box_muller(w[2 * p], w[2 * p + 1], z + 2 * p);
}

/* Sec. 2.1, Eq. 2 with R1/R2: theta_j = lo_j + (hi_j - lo_j) u_j. */
void oracle_prior_draw(const float lo[8], const float hi[8], uint64_t seed, uint32_t stream,
                       uint64_t i, float theta[8])
{
    uint32_t w[8];
    rng_block(seed, stream, i, 0, 0, w + 0);
    rng_block(seed, stream, i, 0, 1, w + 4);
    for (int j = 0; j < 8; ++j) {
        float width = hi[j] - lo[j];
        float u = oracle_uniform(w[j]);
        float scaled = width * u;
        theta[j] = lo[j] + scaled;
    }
}

/* ------------------------------------------------------------------------- */
/* The model (Sec. 2.1).                                                     */
/* ------------------------------------------------------------------------- */

/* R5: floor saturating to int32, NaN -> 0. */
static int32_t floor_to_int_sat(float x)
{
    if (x != x) return 0;
    if (x >= 2147483648.0f) return INT32_MAX;
    if (x < -2147483648.0f) return INT32_MIN;
    return (int32_t)floorf(x);
}

/* R5: transition count drawn from the continuous value x, limited by the
 * source count c still available. */
int32_t oracle_clamp_count(float x, int32_t c)
{
    int32_t n = floor_to_int_sat(x);
    if (n < 0) n = 0;
    if (n > c) n = c;
    return n;
}

/* Sec. 2.1 third step with R4: continuous draw x = h + sd(h) z. */
static float transition_value(float h, float z, int variance_literal)
{
    float sd = sqrtf(h);
    if (variance_literal) sd = sqrtf(sd);
    float dz = sd * z;
    return h + dz;
}

/* Sec. 2.1, Eq. 4: g = alpha0 + alpha / (1 + U^n), U = A + R + D,
 * U^n = 2^(n log2 U) with exact-mode log2 / exp2 and 0^n = 0. */
float oracle_infection_rate(const float theta[8], int32_t U)
{
    float pw = 0.0f;
    if (U != 0) {
        float uf = (float)U;
        float l = oracle_log2x(uf);
        float y = theta[2] * l;
        pw = oracle_exp2x(y);
    }
    float den = 1.0f + pw;
    float q = theta[1] / den;
    return theta[0] + q;
}

/* Sec. 2.1, Eq. 5: hazards from the start-of-day state. */
void oracle_hazard(const int32_t X[6], const float theta[8], int64_t P, float h[5])
{
    float S = (float)X[0], I = (float)X[1], A = (float)X[2];
    int32_t U = X[2] + X[3] + X[4];
    float g = oracle_infection_rate(theta, U);
    float inv_p = 1.0f / (float)P;
    float beta_eta = theta[3] * theta[6];
    float gs = g * S;
    float gsi = gs * I;
    h[0] = gsi * inv_p;            /* S -> I  : g S I / P    */
    h[1] = theta[4] * I;           /* I -> A  : gamma I      */
    h[2] = theta[3] * A;           /* A -> R  : beta A       */
    h[3] = theta[5] * A;           /* A -> D  : delta A      */
    h[4] = beta_eta * I;           /* I -> Ru : beta eta I   */
}

/* One day (Sec. 2.1 steps two to four) given the five normals z (h order).
 * Writes the five transition counts n (h order) and the new state. */
void oracle_step(const int32_t X[6], const float theta[8], int64_t P, const float z[5],
                 int variance_literal, int32_t n_out[5], int32_t Y[6])
{
    float h[5];
    oracle_hazard(X, theta, P, h);
    float x[5];
    for (int k = 0; k < 5; ++k) x[k] = transition_value(h[k], z[k], variance_literal);
    int32_t S = X[0], I = X[1], A = X[2], R = X[3], D = X[4], Ru = X[5];
    /* R5: clamp in h order against the source still available. */
    int32_t n_si = oracle_clamp_count(x[0], S);
    int32_t n_ia = oracle_clamp_count(x[1], I);
    int32_t n_iu = oracle_clamp_count(x[4], I - n_ia);
    int32_t n_ar = oracle_clamp_count(x[2], A);
    int32_t n_ad = oracle_clamp_count(x[3], A - n_ar);
    Y[0] = S - n_si;
    Y[1] = I + n_si - n_ia - n_iu;
    Y[2] = A + n_ia - n_ar - n_ad;
    Y[3] = R + n_ar;
    Y[4] = D + n_ad;
    Y[5] = Ru + n_iu;
    n_out[0] = n_si; n_out[1] = n_ia; n_out[2] = n_ar; n_out[3] = n_ad; n_out[4] = n_iu;
}

/* Sec. 2.1 first step with R9. Returns 0, or -1 when A0+R0+D0 > P. */
int oracle_init_state(const float theta[8], const int32_t ard0[3], int64_t P, int32_t X[6])
{
    int64_t observed0 = (int64_t)ard0[0] + ard0[1] + ard0[2];
    if (observed0 > P) return -1;
    int32_t room = (int32_t)(P - observed0);
    float kappa_a0 = theta[7] * (float)ard0[0];
    int32_t I0 = oracle_clamp_count(kappa_a0, room);
    X[0] = room - I0;
    X[1] = I0;
    X[2] = ard0[0];
    X[3] = ard0[1];
    X[4] = ard0[2];
    X[5] = 0;
    return 0;
}

/* Full trajectory traj[(T+1)][6] of sample i (RNG stream of i, given theta). */
int oracle_simulate(const float theta[8], const int32_t ard0[3], int32_t T, int64_t P,
                    uint64_t seed, uint32_t stream, uint64_t i, int variance_literal,
                    int32_t* traj)
{
    int32_t X[6];
    if (oracle_init_state(theta, ard0, P, X) != 0) return -1;
    memcpy(traj, X, sizeof X);
    float z[10];
    for (int32_t d = 1; d <= T; ++d) {
        uint32_t k = (uint32_t)((d + 1) / 2);
        if (d % 2 == 1) oracle_day_pair_normals(seed, stream, i, k, z);
        const float* zd = (d % 2 == 1) ? z : z + 5;
        int32_t n[5], Y[6];
        oracle_step(X, theta, P, zd, variance_literal, n, Y);
        memcpy(X, Y, sizeof X);
        memcpy(traj + (size_t)d * 6, X, sizeof X);
    }
    return 0;
}

/* R7: exact sum of squared differences of (A, R, D) over days 1..T.
 * observed is [3][T+1] row-major (rows A, R, D). */
uint64_t oracle_sq_distance(const int32_t* traj, const int32_t* observed, int32_t T)
{
    const uint64_t cap = (uint64_t)1 << 63;
    uint64_t acc = 0;
    for (int32_t d = 1; d <= T; ++d) {
        for (int c = 0; c < 3; ++c) {
            int64_t diff = (int64_t)traj[(size_t)d * 6 + 2 + c] - (int64_t)observed[(size_t)c * (T + 1) + d];
            uint64_t sq = (uint64_t)(diff * diff);
            acc = acc + sq;
            if (acc > cap) acc = cap;
        }
    }
    return acc;
}

double oracle_distance_from_sq(uint64_t acc) { return sqrt((double)acc); }

/* ------------------------------------------------------------------------- */
/* ABC rejection (Sec. 2.2 and Sec. 3.1), threads over contiguous ranges.   */
/* ------------------------------------------------------------------------- */
typedef struct {
    const float* lo; const float* hi; const int32_t* observed;
    int32_t T; int64_t P; double eps;
    uint64_t seed; uint32_t stream; int variance_literal;
    uint64_t begin, end;
    /* per-thread results */
    uint64_t n_acc;
    uint64_t* idx; float* theta; double* dist; uint64_t cap;
    double* dist_all; uint64_t dist_all_base;
    int status;
} abc_chunk;

static void* abc_chunk_run(void* arg)
{
    abc_chunk* c = (abc_chunk*)arg;
    int32_t T = c->T;
    int32_t* traj = (int32_t*)malloc(sizeof(int32_t) * 6 * (size_t)(T + 1));
    if (!traj) { c->status = -2; return NULL; }
    int32_t ard0[3] = { c->observed[0], c->observed[T + 1], c->observed[2 * (T + 1)] };
    for (uint64_t i = c->begin; i < c->end; ++i) {
        float th[8];
        oracle_prior_draw(c->lo, c->hi, c->seed, c->stream, i, th);
        if (oracle_simulate(th, ard0, T, c->P, c->seed, c->stream, i, c->variance_literal, traj) != 0) {
            c->status = -1;
            break;
        }
        uint64_t acc = oracle_sq_distance(traj, c->observed, T);
        double dist = oracle_distance_from_sq(acc);
        if (c->dist_all) c->dist_all[i - c->dist_all_base] = dist;
        if (dist <= c->eps) {
            if (c->n_acc < c->cap) {
                c->idx[c->n_acc] = i;
                memcpy(c->theta + 8 * c->n_acc, th, sizeof th);
                c->dist[c->n_acc] = dist;
            }
            c->n_acc++;
        }
    }
    free(traj);
    return NULL;
}

int oracle_abc(const float lo[8], const float hi[8], const int32_t* observed, int32_t T, int64_t P,
               double eps, uint64_t n_samples, uint64_t seed, uint32_t stream, uint64_t first_index,
               int variance_literal, int n_threads,
               uint64_t* idx_out, float* theta_out, double* dist_out, uint64_t capacity,
               uint64_t* n_accepted, double* dist_all)
{
    if (T < 1 || P <= 0 || P >= ((int64_t)1 << 31)) return -1;
    if (n_threads <= 0) {
        long nc = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = nc > 0 ? (int)nc : 1;
    }
    if ((uint64_t)n_threads > n_samples) n_threads = n_samples > 0 ? (int)n_samples : 1;
    abc_chunk* ch = (abc_chunk*)calloc((size_t)n_threads, sizeof(abc_chunk));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!ch || !th) { free(ch); free(th); return -2; }
    /* each thread buffers up to `capacity` accepts of its own range */
    uint64_t per = n_samples / (uint64_t)n_threads, rem = n_samples % (uint64_t)n_threads;
    uint64_t at = first_index;
    int status = 0;
    for (int t = 0; t < n_threads; ++t) {
        uint64_t len = per + ((uint64_t)t < rem ? 1 : 0);
        ch[t] = (abc_chunk){ lo, hi, observed, T, P, eps, seed, stream, variance_literal,
                             at, at + len, 0, NULL, NULL, NULL, capacity, dist_all, first_index, 0 };
        ch[t].idx = (uint64_t*)malloc(sizeof(uint64_t) * (capacity ? capacity : 1));
        ch[t].theta = (float*)malloc(sizeof(float) * 8 * (capacity ? capacity : 1));
        ch[t].dist = (double*)malloc(sizeof(double) * (capacity ? capacity : 1));
        if (!ch[t].idx || !ch[t].theta || !ch[t].dist) status = -2;
        at += len;
    }
    int started = 0;
    if (status == 0) {
        for (int t = 0; t < n_threads; ++t) {
            if (pthread_create(&th[t], NULL, abc_chunk_run, &ch[t]) != 0) { status = -2; break; }
            started++;
        }
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    /* concatenate in range order: the result is sorted by sample index */
    uint64_t total = 0;
    for (int t = 0; t < n_threads && status == 0; ++t) {
        if (ch[t].status != 0) { status = ch[t].status; break; }
        for (uint64_t a = 0; a < ch[t].n_acc && a < capacity; ++a) {
            if (total + a < capacity) {
                idx_out[total + a] = ch[t].idx[a];
                memcpy(theta_out + 8 * (total + a), ch[t].theta + 8 * a, 8 * sizeof(float));
                dist_out[total + a] = ch[t].dist[a];
            }
        }
        total += ch[t].n_acc;
    }
    for (int t = 0; t < n_threads; ++t) { free(ch[t].idx); free(ch[t].theta); free(ch[t].dist); }
    free(ch); free(th);
    if (n_accepted) *n_accepted = total;
    if (status == 0 && total > capacity) status = 1;
    return status;
}

/* ------------------------------------------------------------------------- */
/* Plain loops over the functions above, so that tests can sweep whole      */
/* input domains without one foreign call per element.                      */
/* ------------------------------------------------------------------------- */
void oracle_log2x_batch(const float* x, float* y, uint64_t n)
{
    for (uint64_t j = 0; j < n; ++j) y[j] = oracle_log2x(x[j]);
}

void oracle_exp2x_batch(const float* x, float* y, uint64_t n)
{
    for (uint64_t j = 0; j < n; ++j) y[j] = oracle_exp2x(x[j]);
}

void oracle_sincospix_batch(const float* v, float* s, float* c, uint64_t n)
{
    for (uint64_t j = 0; j < n; ++j) oracle_sincospix(v[j], s + j, c + j);
}

void oracle_uniform_batch(const uint32_t* w, float* u, uint64_t n)
{
    for (uint64_t j = 0; j < n; ++j) u[j] = oracle_uniform(w[j]);
}

/* z[n][10]: the ten normals of day-pair k for samples first .. first+n-1. */
void oracle_normals_batch(uint64_t seed, uint32_t stream, uint64_t first, uint64_t n, uint32_t k,
                          float* z)
{
    for (uint64_t j = 0; j < n; ++j) oracle_day_pair_normals(seed, stream, first + j, k, z + 10 * j);
}

/* theta[n][8]: prior draws of samples first .. first+n-1. */
void oracle_prior_batch(const float lo[8], const float hi[8], uint64_t seed, uint32_t stream,
                        uint64_t first, uint64_t n, float* theta)
{
    for (uint64_t j = 0; j < n; ++j) oracle_prior_draw(lo, hi, seed, stream, first + j, theta + 8 * j);
}

/* n[m][5], Y[m][6]: one step for each of m (state, theta, normals) triples. */
void oracle_step_batch(const int32_t* X, const float* theta, int64_t P, const float* z,
                       int variance_literal, uint64_t m, int32_t* n_out, int32_t* Y)
{
    for (uint64_t j = 0; j < m; ++j)
        oracle_step(X + 6 * j, theta + 8 * j, P, z + 5 * j, variance_literal, n_out + 5 * j, Y + 6 * j);
}

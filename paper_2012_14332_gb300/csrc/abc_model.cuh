// abc_model.cuh -- device side of one ABC sample: Philox4x32-10 words, uniforms,
// Box-Muller normals, the six-compartment model day and the distance.
//
// Paper passages (Kulkarni, Krell, Nabarro, Moritz 2020):
//   theta = [alpha0, alpha, n, beta, gamma, delta, eta, kappa]          Sec. 2.1, Eq. 1
//   prior U(lo, hi)                                                     Sec. 2.1, Eq. 2
//   X = [S, I, A, R, D, Ru]                                             Sec. 2.1, Eq. 3
//   g = alpha0 + alpha / (1 + (A+R+D)^n)                                Sec. 2.1, Eq. 4
//   Ru = 0, I0 = kappa A0, S = P - (A0 + R0 + D0 + I0)                  Sec. 2.1, first step
//   h = (g S I / P, gamma I, beta A, delta A, beta eta I)               Sec. 2.1, Eq. 5
//   counts = floor of Normal(h, h) draws (Poisson approximation)        Sec. 2.1, third step
//   S->I, I->A, A->R, A->D, I->Ru applied in h order                    Sec. 2.1, fourth step
//   Euclidean distance of simulated vs observed (A, R, D)               Sec. 2.2, Eq. 7
//
// Choices where the paper is silent (the same choices as the CPU checker,
// written independently):
//   * Counter layout: (i_lo, i_hi, k, 4*stream + g). k = 0: prior (g = 0 gives
//     theta0..3, g = 1 gives theta4..7). k >= 1: days 2k-1, 2k (g = 0, 1, 2 give
//     words w0..w11; Box-Muller pair p uses w[2p] for the radius and w[2p+1] for
//     the angle; day 2k-1 takes normals z0..z4, day 2k takes z5..z9).
//   * u = bits((w & 0x7FFFFF) | 0x3F800000) - (1 - 2^-24), exactly (2m+1) 2^-24.
//   * x = h + sqrt(h) z (standard deviation sqrt(h)); n = min(max(floor x, 0), c)
//     with floor saturating to int32 and NaN -> 0; c = source count left, in h
//     order (S; I; I - n(I->A); A; A - n(A->R)).
//   * int32 compartments, float32 rates; I0 = min(max(floor(kappa A0), 0), room).
//   * distance^2 = exact uint64 sum over days 1..T (saturating at 2^63);
//     dist = sqrt((double) distance^2).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace abcgb {

// Arithmetic mode of a kernel instance: bit 0 fast (else exact), bit 1 the
// literal reading of the transition variance (std h^(1/4), else sqrt(h)).
enum : int { kExact = 0, kFast = 1, kLiteral = 2 };
__host__ __device__ constexpr bool is_fast(int mode) { return (mode & kFast) != 0; }
__host__ __device__ constexpr bool is_literal(int mode) { return (mode & kLiteral) != 0; }

// ---------------------------------------------------------------------------
// Kernel parameters (passed by value; lives in the constant bank).
// ---------------------------------------------------------------------------
struct ModelParams {
    float lo[8];          // prior lower bounds
    float width[8];       // hi - lo, rounded to float on the host
    uint32_t rk0[10];     // Philox round keys: seed_lo + r * 0x9E3779B9
    uint32_t rk1[10];     // Philox round keys: seed_hi + r * 0xBB67AE85
    uint32_t ctr3_base;   // 4 * stream
    int32_t T;            // simulated days
    int32_t P;            // population
    float inv_p;          // 1.0f / (float)P, IEEE-rounded on the host
    int32_t room0;        // P - (A0 + R0 + D0)
    int32_t A0, R0, D0;   // initial observed compartments
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, const ModelParams& p)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t pa = (uint64_t)0xD2511F53u * c.x;
        const uint64_t pb = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t a_hi = (uint32_t)(pa >> 32), a_lo = (uint32_t)pa;
        const uint32_t b_hi = (uint32_t)(pb >> 32), b_lo = (uint32_t)pb;
        c = make_uint4(b_hi ^ c.y ^ p.rk0[r], b_lo, a_hi ^ c.w ^ p.rk1[r], a_lo);
    }
    return c;
}

// Block g of day-pair k of sample i; ctr3_base = 4 * stream.
__device__ __forceinline__ uint4 rng_block_s(const ModelParams& p, uint64_t i, uint32_t k, uint32_t ctr3_base,
                                             uint32_t g)
{
    return philox10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), k, ctr3_base | g), p);
}

__device__ __forceinline__ uint4 rng_block(const ModelParams& p, uint64_t i, uint32_t k, uint32_t g)
{
    return rng_block_s(p, i, k, p.ctr3_base, g);
}

// (2m+1) 2^-24 with m the low 23 bits of w; the subtraction is exact.
__device__ __forceinline__ float uniform01(uint32_t w)
{
    return __fsub_rn(__uint_as_float((w & 0x007FFFFFu) | 0x3F800000u), __uint_as_float(0x3F7FFFFFu));
}

// ---------------------------------------------------------------------------
// Exact mode: fixed float32 series, every operation IEEE round-to-nearest,
// no contraction. Coefficients: correctly rounded values of the named reals.
// ---------------------------------------------------------------------------
namespace exact {
constexpr float kLn2 = 0x1.62e430p-1f;         // ln 2
constexpr float kNeg2Ln2 = -0x1.62e430p+0f;    // -2 ln 2
constexpr float kPi = 0x1.921fb6p+1f;          // pi
constexpr float kSqrt2 = 0x1.6a09e6p+0f;       // sqrt 2
// log2(m) = s * sum_k c_k s^(k-1), s = (m-1)/(m+1), c_k = 2 / (k ln 2)
constexpr float kL1 = 0x1.715476p+1f, kL3 = 0x1.ec709ep-1f, kL5 = 0x1.2776c6p-1f;
constexpr float kL7 = 0x1.a61762p-2f, kL9 = 0x1.484b14p-2f;
// e^t: 1/j!, j = 2..7
constexpr float kE2 = 0x1.000000p-1f, kE3 = 0x1.555556p-3f, kE4 = 0x1.555556p-5f;
constexpr float kE5 = 0x1.111112p-7f, kE6 = 0x1.6c16c2p-10f, kE7 = 0x1.a01a02p-13f;
// sin t: (-1)^j / (2j+1)!, j = 1..4
constexpr float kS3 = -0x1.555556p-3f, kS5 = 0x1.111112p-7f, kS7 = -0x1.a01a02p-13f;
constexpr float kS9 = 0x1.71de3ap-19f;
// cos t: (-1)^j / (2j)!, j = 1..5
constexpr float kC2 = -0x1.000000p-1f, kC4 = 0x1.555556p-5f, kC6 = -0x1.6c16c2p-10f;
constexpr float kC8 = 0x1.a01a02p-16f, kC10 = -0x1.27e4fcp-22f;

__device__ __forceinline__ float madd(float a, float b, float c) { return __fadd_rn(__fmul_rn(a, b), c); }

// log2 x, x positive normal: x = 2^e m, m folded into (sqrt(1/2), sqrt 2].
__device__ __forceinline__ float log2x(float x)
{
    const uint32_t b = __float_as_uint(x);
    int e = (int)(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > kSqrt2) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float q = kL9;
    q = madd(q, s2, kL7);
    q = madd(q, s2, kL5);
    q = madd(q, s2, kL3);
    q = madd(q, s2, kL1);
    return __fadd_rn(__int2float_rn(e), __fmul_rn(s, q));
}

// 2^y = 2^k e^(f ln 2), k = rint(y); +inf for y >= 127.5 or NaN, 0 below -125.5.
__device__ __forceinline__ float exp2x(float y)
{
    if (!(y < 127.5f)) return __int_as_float(0x7F800000);
    if (y < -125.5f) return 0.0f;
    const float kf = rintf(y);
    const float t = __fmul_rn(__fsub_rn(y, kf), kLn2);
    float q = kE7;
    q = madd(q, t, kE6);
    q = madd(q, t, kE5);
    q = madd(q, t, kE4);
    q = madd(q, t, kE3);
    q = madd(q, t, kE2);
    q = madd(q, t, 1.0f);
    q = madd(q, t, 1.0f);
    const int k = __float2int_rn(kf);
    return __fmul_rn(q, __uint_as_float((uint32_t)(k + 127) << 23));
}

// sin(pi v), cos(pi v): v = q/2 + w exactly, |w| <= 1/4, series in t = pi w.
__device__ __forceinline__ void sincospix(float v, float& s_out, float& c_out)
{
    const float qf = rintf(__fmul_rn(v, 2.0f));
    const float w = __fsub_rn(v, __fmul_rn(qf, 0.5f));
    const float t = __fmul_rn(w, kPi);
    const float t2 = __fmul_rn(t, t);
    float ps = kS9;
    ps = madd(ps, t2, kS7);
    ps = madd(ps, t2, kS5);
    ps = madd(ps, t2, kS3);
    ps = __fmul_rn(ps, t2);
    const float sn = __fadd_rn(__fmul_rn(t, ps), t);
    float pc = kC10;
    pc = madd(pc, t2, kC8);
    pc = madd(pc, t2, kC6);
    pc = madd(pc, t2, kC4);
    pc = madd(pc, t2, kC2);
    pc = __fmul_rn(pc, t2);
    const float cs = __fadd_rn(pc, 1.0f);
    switch (__float2int_rn(qf) & 3) {
    case 0: s_out = sn; c_out = cs; break;
    case 1: s_out = cs; c_out = -sn; break;
    case 2: s_out = -sn; c_out = -cs; break;
    default: s_out = -cs; c_out = sn; break;
    }
}
}  // namespace exact

// ---------------------------------------------------------------------------
// Fast mode: the SFU (MUFU) approximations and FMA.
// ---------------------------------------------------------------------------
namespace fast {
// flush-to-zero forms: the sampler's inputs are never subnormal (u >= 2^-24,
// counts are integers), and .ftz spares the subnormal fix-up code.
__device__ __forceinline__ float lg2(float x) { float y; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float ex2(float x) { float y; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sqrt_a(float x) { float y; asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float rcp(float x) { float y; asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sin_a(float x) { float y; asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float cos_a(float x) { float y; asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
}  // namespace fast

// One Box-Muller pair: r = sqrt(-2 ln u1), (z0, z1) = r (cos, sin)(2 pi u2).
template <int MODE>
__device__ __forceinline__ void box_muller(uint32_t w_radius, uint32_t w_angle, float& z0, float& z1)
{
    const float u1 = uniform01(w_radius);
    if (!is_fast(MODE)) {
        const float u2 = uniform01(w_angle);
        const float r = __fsqrt_rn(__fmul_rn(exact::kNeg2Ln2, exact::log2x(u1)));
        float s, c;
        exact::sincospix(__fmul_rn(u2, 2.0f), s, c);
        z0 = __fmul_rn(r, c);
        z1 = __fmul_rn(r, s);
    } else {
        const float r = fast::sqrt_a(-0x1.62e430p+0f * fast::lg2(u1));
        // angle 2 pi u2 = 2 pi (u2 - 1/2) + pi, centred on 0 for the SFU; one FMA
        // from the word's mantissa bits b in [1, 2): u2 - 1/2 = b - (3/2 - 2^-24)
        const float b = __uint_as_float((w_angle & 0x007FFFFFu) | 0x3F800000u);
        const float a = __fmaf_rn(b, 6.28318530717958647692f, -9.42477758f);
        z0 = -r * fast::cos_a(a);
        z1 = -r * fast::sin_a(a);
    }
}

// Ten normals of day-pair k (days 2k-1 and 2k) of sample i, RNG stream ctr3_base / 4.
template <int MODE>
__device__ __forceinline__ void day_pair_normals_s(const ModelParams& p, uint64_t i, uint32_t k, uint32_t ctr3_base,
                                                   float z[10])
{
    const uint4 a = rng_block_s(p, i, k, ctr3_base, 0);
    const uint4 b = rng_block_s(p, i, k, ctr3_base, 1);
    const uint4 c = rng_block_s(p, i, k, ctr3_base, 2);
    box_muller<MODE>(a.x, a.y, z[0], z[1]);
    box_muller<MODE>(a.z, a.w, z[2], z[3]);
    box_muller<MODE>(b.x, b.y, z[4], z[5]);
    box_muller<MODE>(b.z, b.w, z[6], z[7]);
    box_muller<MODE>(c.x, c.y, z[8], z[9]);
}

template <int MODE>
__device__ __forceinline__ void day_pair_normals(const ModelParams& p, uint64_t i, uint32_t k, float z[10])
{
    day_pair_normals_s<MODE>(p, i, k, p.ctr3_base, z);
}

// Prior draw of sample i (Eq. 2): theta_j = lo_j + width_j u_j (two roundings).
__device__ __forceinline__ void prior_draw_s(const ModelParams& p, uint64_t i, uint32_t ctr3_base, float th[8])
{
    const uint4 a = rng_block_s(p, i, 0, ctr3_base, 0);
    const uint4 b = rng_block_s(p, i, 0, ctr3_base, 1);
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) th[j] = __fadd_rn(p.lo[j], __fmul_rn(p.width[j], uniform01(w[j])));
}

__device__ __forceinline__ void prior_draw(const ModelParams& p, uint64_t i, float th[8])
{
    prior_draw_s(p, i, p.ctr3_base, th);
}

// n = min(max(floor x, 0), c): cvt.rmi saturates to int32 and maps NaN to 0;
// for c >= 0, min.relu(f, c) = max(min(f, c), 0) is the same clamp.
__device__ __forceinline__ int32_t clamp_count(float x, int32_t c)
{
    int32_t n;
    asm("min.relu.s32 %0, %1, %2;" : "=r"(n) : "r"(__float2int_rd(x)), "r"(c));
    return n;
}

// ---------------------------------------------------------------------------
// The model state of one sample.
// ---------------------------------------------------------------------------
struct Theta {
    float a0, a, n, beta, gamma, delta, beta_eta, kappa;
};

// Exact mode keeps the paper's factors; fast mode folds 1/P into alpha0 and
// alpha (g/P = alpha0/P + (alpha/P) / (1 + U^n)), saving a multiply per day.
template <int MODE>
__device__ __forceinline__ Theta make_theta(const float th[8], float inv_p)
{
    Theta t;
    t.a0 = th[0]; t.a = th[1]; t.n = th[2]; t.beta = th[3]; t.gamma = th[4]; t.delta = th[5];
    t.beta_eta = __fmul_rn(th[3], th[6]);
    t.kappa = th[7];
    if (is_fast(MODE)) {
        t.a0 = th[0] * inv_p;
        t.a = th[1] * inv_p;
    }
    return t;
}

struct State {
    int32_t S, I, A, R, D, Ru;
};

// Sec. 2.1 first step: I0 = kappa A0, floored and limited by the room left
// after A0 + R0 + D0.
__device__ __forceinline__ int32_t initial_infected(const Theta& t, int32_t A0, int32_t room)
{
    return clamp_count(__fmul_rn(t.kappa, __int2float_rn(A0)), room);
}

// The initial state for a given I0: Ru = 0, S = P - (A0 + R0 + D0 + I0).
__device__ __forceinline__ State state_from(int32_t I0, int32_t A0, int32_t R0, int32_t D0, int32_t room)
{
    State x;
    x.S = room - I0; x.I = I0; x.A = A0; x.R = R0; x.D = D0; x.Ru = 0;
    return x;
}

__device__ __forceinline__ State init_state(const Theta& t, int32_t A0, int32_t R0, int32_t D0, int32_t room)
{
    return state_from(initial_infected(t, A0, room), A0, R0, D0, room);
}

// One day (Sec. 2.1 second to fourth step) with normals z[0..4] in h order.
template <int MODE>
__device__ __forceinline__ void model_day(State& x, const Theta& t, float inv_p, const float* z, int32_t* n_out = nullptr)
{
    const float Sf = __int2float_rn(x.S), If = __int2float_rn(x.I), Af = __int2float_rn(x.A);
    const int32_t U = x.A + x.R + x.D;
    float h0, h1, h2, h3, h4, v0, v1, v2, v3, v4;
    if (!is_fast(MODE)) {
        float pw = 0.0f;
        if (U != 0) pw = exact::exp2x(__fmul_rn(t.n, exact::log2x(__int2float_rn(U))));
        const float g = __fadd_rn(t.a0, __fdiv_rn(t.a, __fadd_rn(1.0f, pw)));
        h0 = __fmul_rn(__fmul_rn(__fmul_rn(g, Sf), If), inv_p);
        h1 = __fmul_rn(t.gamma, If);
        h2 = __fmul_rn(t.beta, Af);
        h3 = __fmul_rn(t.delta, Af);
        h4 = __fmul_rn(t.beta_eta, If);
        // standard deviation sqrt(h), or h^(1/4) = sqrt(sqrt(h)) under the literal reading
        auto sd = [](float h) { return is_literal(MODE) ? __fsqrt_rn(__fsqrt_rn(h)) : __fsqrt_rn(h); };
        v0 = __fadd_rn(h0, __fmul_rn(sd(h0), z[0]));
        v1 = __fadd_rn(h1, __fmul_rn(sd(h1), z[1]));
        v2 = __fadd_rn(h2, __fmul_rn(sd(h2), z[2]));
        v3 = __fadd_rn(h3, __fmul_rn(sd(h3), z[3]));
        v4 = __fadd_rn(h4, __fmul_rn(sd(h4), z[4]));
    } else {
        // U = 0: lg2 gives -inf and n (-inf) = -inf for n > 0; the clamp at -200
        // also turns n = 0 (NaN) into 2^-200 = 0, so 0^n = 0 without a branch
        const float pw = fast::ex2(fmaxf(t.n * fast::lg2(__int2float_rn(U)), -200.0f));
        const float g_over_p = __fmaf_rn(t.a, fast::rcp(1.0f + pw), t.a0);   // a0, a carry 1/P
        h0 = (g_over_p * Sf) * If;
        h1 = t.gamma * If;
        h2 = t.beta * Af;
        h3 = t.delta * Af;
        h4 = t.beta_eta * If;
        auto sd = [](float h) { return is_literal(MODE) ? fast::sqrt_a(fast::sqrt_a(h)) : fast::sqrt_a(h); };
        v0 = __fmaf_rn(sd(h0), z[0], h0);
        v1 = __fmaf_rn(sd(h1), z[1], h1);
        v2 = __fmaf_rn(sd(h2), z[2], h2);
        v3 = __fmaf_rn(sd(h3), z[3], h3);
        v4 = __fmaf_rn(sd(h4), z[4], h4);
    }
    // clamp against what is left of each source, in h order
    const int32_t n_si = clamp_count(v0, x.S);
    const int32_t n_ia = clamp_count(v1, x.I);
    const int32_t n_iu = clamp_count(v4, x.I - n_ia);
    const int32_t n_ar = clamp_count(v2, x.A);
    const int32_t n_ad = clamp_count(v3, x.A - n_ar);
    x.S -= n_si;
    x.I += n_si - n_ia - n_iu;
    x.A += n_ia - n_ar - n_ad;
    x.R += n_ar;
    x.D += n_ad;
    x.Ru += n_iu;
    if (n_out) {
        n_out[0] = n_si; n_out[1] = n_ia; n_out[2] = n_ar; n_out[3] = n_ad; n_out[4] = n_iu;
    }
}

// Distance^2 accumulation of one day when only "acc <= acc_max < 2^62" and the
// exact value of accepted samples matter. Before the day's three squares are
// added, the high word of the running sum is clamped at 2^30 (one
// instruction): the sum is then at most 2^62 + 2^32 - 1, and with three
// squares of at most (2^31 - 1)^2 each it stays below 2^64 - 2^33 + 3, so it
// never wraps. A sum that reached 2^62 keeps a high word of 2^30, so it stays
// >= 2^62 > acc_max; every partial sum of an accepted sample is <= acc_max,
// so its sum is never clamped and is exact.
__device__ __forceinline__ uint64_t add_day_sq_below62(uint64_t acc, const State& x, int4 obs)
{
    const int32_t dA = x.A - obs.x, dR = x.R - obs.y, dD = x.D - obs.z;
    const uint32_t hi = min((uint32_t)(acc >> 32), 0x40000000u);
    acc = ((uint64_t)hi << 32) | (uint32_t)acc;
    acc += (uint64_t)((int64_t)dA * dA);
    acc += (uint64_t)((int64_t)dR * dR);
    acc += (uint64_t)((int64_t)dD * dD);
    return acc;
}

// Saturating distance^2 accumulation of one day: three exact squares summed in
// uint64 (< 3 * 2^62, no wrap), then added with carry detection, capped at 2^63.
__device__ __forceinline__ uint64_t add_day_sq(uint64_t acc, const State& x, int4 obs)
{
    const int64_t dA = (int64_t)(x.A - obs.x);
    const int64_t dR = (int64_t)(x.R - obs.y);
    const int64_t dD = (int64_t)(x.D - obs.z);
    const uint64_t day = (uint64_t)(dA * dA) + (uint64_t)(dR * dR) + (uint64_t)(dD * dD);
    const uint64_t cap = 0x8000000000000000ull;
    uint64_t s = acc + day;
    s = (s < acc) ? cap : s;
    return s > cap ? cap : s;
}

// Visitor that ignores the days (distance only).
struct NoVisit {
    __device__ __forceinline__ void operator()(int32_t, const State&) const {}
};

// Simulate sample i with parameters t from the initial state, calling
// visit(d, state) after each day d and accumulating the distance against
// obs_s (int4 per day: A, R, D, 0). Returns distance^2.
template <int MODE, typename Visit>
__device__ __forceinline__ uint64_t simulate_sample(const ModelParams& p, uint64_t i, const Theta& t, State x,
                                                    const int4* __restrict__ obs_s, Visit visit)
{
    uint64_t acc = 0;
    const int32_t T = p.T;
    const uint32_t n_pairs = (uint32_t)(T + 1) >> 1;
    for (uint32_t k = 1; k <= n_pairs; ++k) {
        float z[10];
        day_pair_normals<MODE>(p, i, k, z);
        const int32_t d1 = (int32_t)(2 * k - 1);
        model_day<MODE>(x, t, p.inv_p, z);
        acc = add_day_sq(acc, x, obs_s[d1]);
        visit(d1, x);
        if (d1 < T) {
            model_day<MODE>(x, t, p.inv_p, z + 5);
            acc = add_day_sq(acc, x, obs_s[d1 + 1]);
            visit(d1 + 1, x);
        }
    }
    return acc;
}

}  // namespace abcgb

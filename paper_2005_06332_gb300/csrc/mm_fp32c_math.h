// mm_fp32c_math.h -- arithmetic of the FP32c step, host + device.
//
// Everything here is IEEE binary32 arithmetic (+, -, *, fma, correctly
// rounded reciprocal) and 32-bit integer conversions, so a host build of
// these functions gives the same bits as the GPU kernel.  No CUDA math
// library call is used: the exponential is written from its definition
// (range reduction by powers of two, Taylor series of 2^f, f in [-1/2, 1/2]).
//
// Precision plan:
//   * the state is fixed point: V = Vq * 2^-23 mV (int32), gates q * 2^-32
//     (uint32); increments are rounded once and added exactly;
//   * potential differences are taken in integers and carried exactly as
//     float pairs;
//   * the membrane and axial currents, the synaptic conductance and every
//     constant of the model (areas, axial conductances, channel densities,
//     the stimulus, the decay factor) are float pairs ("double-float", about
//     44 bits): a constant rounded to FP32 would perturb the model the same
//     way in every step, and the rhs is a sum of large terms that cancel in
//     a steady state, where FP32 rounding repeats from step to step;
//   * the rate functions, steady states and relaxation factors are computed
//     as float pairs, since their rounding biases the gate trajectories every
//     cycle;
//   * the Hines solve is FP32 on the rhs rounded once, with the diagonal split
//     into its passive part (eliminated once in FP64 at set-up, kept as a
//     pair) and the step's active conductance, eliminated in FP32 as a
//     perturbation of it.
#pragma once
#include <stdint.h>

#include <cmath>
#include <cstring>
#ifdef __CUDACC__
#define MMF_HD __host__ __device__ __forceinline__
#else
#define MMF_HD inline
#endif

namespace mmf {

struct F2 {
    float hi, lo;
};

// ------------------------------------------------------- primitive helpers

MMF_HD float fma_f(float a, float b, float c) { return fmaf(a, b, c); }

MMF_HD float rcp_rn(float x)
{
#ifdef __CUDA_ARCH__
    return __frcp_rn(x);
#else
    return 1.0f / x;
#endif
}

// An approximation of 1/x (relative error below 2^-22) for the first
// quotient of a double-float division, whose remainder step corrects it.
MMF_HD float rcp_fast(float x)
{
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return 1.0f / x;
#endif
}

MMF_HD int32_t f2i_rn(float x)
{
#ifdef __CUDA_ARCH__
    return __float2int_rn(x);
#else
    return (int32_t)std::lrintf(x);
#endif
}

MMF_HD float rint_f(float x)
{
#ifdef __CUDA_ARCH__
    return rintf(x);
#else
    return std::rintf(x);
#endif
}

// 2^n for -126 <= n <= 127.
MMF_HD float pow2i(int32_t n)
{
    const int32_t bits = (n + 127) << 23;
#ifdef __CUDA_ARCH__
    return __int_as_float(bits);
#else
    float f;
    std::memcpy(&f, &bits, sizeof(f));
    return f;
#endif
}

// ------------------------------------------------ error-free transformations

MMF_HD F2 two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

// requires |a| >= |b| (or a == 0)
MMF_HD F2 quick_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}

MMF_HD F2 two_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

// --------------------------------------------------- double-float arithmetic

MMF_HD F2 neg(F2 a) { return {-a.hi, -a.lo}; }

MMF_HD F2 add(F2 a, F2 b)
{
    const F2 s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

MMF_HD F2 add_f(F2 a, float b)
{
    const F2 s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, s.lo + a.lo);
}

MMF_HD F2 mul(F2 a, F2 b)
{
    const F2 p = two_prod(a.hi, b.hi);
    return quick_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}

MMF_HD F2 mul_f(F2 a, float b)
{
    const F2 p = two_prod(a.hi, b);
    return quick_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

// multiplication by a power of two (exact)
MMF_HD F2 scale(F2 a, float p2) { return {a.hi * p2, a.lo * p2}; }

// a / b: a first quotient from an approximate reciprocal, then one
// correction of the double-float remainder a - q b (the remainder is formed
// to double-float accuracy, so the quotient's error is the square of the
// first quotient's, below 2^-44 relative).
MMF_HD F2 div(F2 a, F2 b)
{
    const float r = rcp_fast(b.hi);
    const float q1 = a.hi * r;
    const F2 rem = add(a, neg(mul_f(b, q1)));
    return quick_two_sum(q1, rem.hi * r);
}

// ------------------------------------------------------------ exponential

constexpr double kLog2eD = 1.4426950408889634;
constexpr double kLn2D = 0.6931471805599453;
constexpr float kL2E_hi = (float)kLog2eD;
constexpr float kL2E_lo = (float)(kLog2eD - (double)kL2E_hi);
constexpr float kLN2_hi = (float)kLn2D;
constexpr float kLN2_lo = (float)(kLn2D - (double)kLN2_hi);
// Taylor coefficients of 2^f: (ln 2)^k / k!
constexpr float kP2 = (float)(kLn2D * kLn2D / 2.0);
constexpr float kP2_lo = (float)(kLn2D * kLn2D / 2.0 - (double)kP2);
constexpr float kP3 = (float)(kLn2D * kLn2D * kLn2D / 6.0);
constexpr float kP4 = (float)(kLn2D * kLn2D * kLn2D * kLn2D / 24.0);
constexpr float kP5 = (float)(kLn2D * kLn2D * kLn2D * kLn2D * kLn2D / 120.0);
constexpr float kP6 = (float)(kLn2D * kLn2D * kLn2D * kLn2D * kLn2D * kLn2D / 720.0);
constexpr float kP7 = (float)(kLn2D * kLn2D * kLn2D * kLn2D * kLn2D * kLn2D * kLn2D / 5040.0);
constexpr float kP8 = (float)(kLn2D * kLn2D * kLn2D * kLn2D * kLn2D * kLn2D * kLn2D * kLn2D / 40320.0);

// e^(x.hi + x.lo) as a double-float, |x| < 80.  x log2(e) = n + f with n an
// integer and |f| <= 1/2; 2^f = 1 + f (ln2 + P2 f + f^2 q(f)) by its Taylor
// series (truncation below 3e-10 relative).  q is evaluated in float (its
// rounding enters scaled by |f|^3 <= 1/8); u = ln2 + P2 f + f^2 q and 1 + f u
// are carried as float pairs, and the low part of f enters through
// d(2^f)/df = ln2 2^f.
MMF_HD F2 exp_df(F2 x)
{
    const float t_hi = x.hi * kL2E_hi;
    const float t_lo = fmaf(x.hi, kL2E_hi, -t_hi) + fmaf(x.hi, kL2E_lo, x.lo * kL2E_hi);
    const float n = rint_f(t_hi);
    const float f = t_hi - n;  // exact
    float q = kP8;
    q = fmaf(q, f, kP7);
    q = fmaf(q, f, kP6);
    q = fmaf(q, f, kP5);
    q = fmaf(q, f, kP4);
    q = fmaf(q, f, kP3);
    // u = ln2 + f (P2 + f q) as a pair, with P2 (as a pair) times f exact:
    // P2 f^2 is the largest term after the linear one, so its coefficient
    // must not be rounded to FP32
    const F2 p2f = add_f(two_prod(kP2, f), kP2_lo * f);
    const F2 u = add(F2{kLN2_hi, kLN2_lo}, add_f(p2f, f * f * q));
    const float u_hi = u.hi;
    const float u_lo = u.lo;
    // p = 1 + f u as a pair (1 - p_hi is exact)
    const float p_hi = fmaf(u_hi, f, 1.0f);
    float p_lo = fmaf(u_hi, f, 1.0f - p_hi) + u_lo * f;
    p_lo = fmaf(p_hi, t_lo * kLN2_hi, p_lo);
    const F2 p = quick_two_sum(p_hi, p_lo);
    int32_t ni = (int32_t)n;
    ni = ni < -120 ? -120 : (ni > 120 ? 120 : ni);
    return scale(p, pow2i(ni));
}

// x / (e^x - 1) given x and e^x, with its Bernoulli series near 0.
MMF_HD F2 xexpm1_given(F2 x, F2 ex)
{
    if (fabsf(x.hi) < 0.125f) {
        const float x2 = x.hi * x.hi;
        float s = fmaf(x2, -1.0f / 1209600.0f, 1.0f / 30240.0f);
        s = fmaf(x2, s, -1.0f / 720.0f);
        s = fmaf(x2, s, 1.0f / 12.0f);
        s = s * x2;
        const F2 r = two_sum(1.0f, -0.5f * x.hi);
        return quick_two_sum(r.hi, r.lo + (s - 0.5f * x.lo));
    }
    return div(x, add_f(ex, -1.0f));
}

MMF_HD F2 xexpm1_df(F2 x) { return xexpm1_given(x, exp_df(x)); }

// 1 - e^(-y) for y >= 0, with its series for small y.
MMF_HD F2 one_minus_exp_neg_df(F2 y)
{
    if (y.hi < 0.125f) {
        float r = fmaf(y.hi, -1.0f / 5040.0f, 1.0f / 720.0f);
        r = fmaf(-y.hi, r, 1.0f / 120.0f);
        r = fmaf(-y.hi, r, 1.0f / 24.0f);
        r = fmaf(-y.hi, r, 1.0f / 6.0f);
        r = fmaf(-y.hi, r, 0.5f);
        r = r * y.hi * y.hi;
        return add_f(y, -r);
    }
    const F2 e = exp_df(neg(y));
    return add_f(neg(e), 1.0f);
}

// ------------------------------------------------------------ fixed point

constexpr float kV2F = 1.0f / 8388608.0f;    // 2^-23 mV per unit

// (a - b) * 2^-23, one rounding (|a - b| < 2^31).
MMF_HD float vdiff(int32_t a, int32_t b) { return (float)(a - b) * kV2F; }

// (a - b) * c, c = ch + cl, as a double-float (the integer difference is
// split exactly into two floats first).
MMF_HD F2 scaled_diff(int32_t a, int32_t b, float ch, float cl)
{
    const int32_t d = a - b;
    const float dh = (float)d;
    const float dl = (float)(d - (int32_t)dh);
    const float xh = dh * ch;
    return {xh, fmaf(dh, ch, -xh) + fmaf(dh, cl, dl * ch)};
}

// (a - b) * 2^-23 exactly, as a float pair (|a - b| < 2^31).
MMF_HD F2 vdiff_df(int32_t a, int32_t b)
{
    const int32_t d = a - b;
    const float dh = (float)d;
    const float dl = (float)(d - (int32_t)dh);
    return {dh * kV2F, dl * kV2F};
}

// (vq * 2^-23) - E for E = eq * 2^-23 + eres, as a float pair.
MMF_HD F2 vminus_df(int32_t vq, int32_t eq, float eres)
{
    return add_f(vdiff_df(vq, eq), -eres);
}

// a double split into a float pair (hi the nearest float)
MMF_HD F2 split_d(double x)
{
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}

// exact value of a uint32 fixed-point gate as a double-float
MMF_HD F2 gate_df(uint32_t q)
{
    const float hi = (float)(q >> 16) * (1.0f / 65536.0f);
    const float lo = (float)(q & 0xFFFFu) * (1.0f / 4294967296.0f);
    return quick_two_sum(hi, lo);
}

MMF_HD float gate_f(uint32_t q) { return (float)q * (1.0f / 4294967296.0f); }

// q + dx * 2^32 rounded to the nearest unit (dx * 2^31 first taken in
// whole units, then the rest in half units), clamped to [0, 2^32 - 1]
MMF_HD uint32_t gate_add(uint32_t q, F2 dx)
{
    const float a = dx.hi * 2147483648.0f;
    const int32_t k1 = f2i_rn(a);
    const int32_t k2 = f2i_rn(((a - (float)k1) + dx.lo * 2147483648.0f) * 2.0f);
    const long long nq = (long long)q + 2 * (long long)k1 + (long long)k2;
    return (uint32_t)(nq < 0 ? 0 : (nq > 4294967295LL ? 4294967295LL : nq));
}

// -------------------------------------------------------------- HH kinetics

constexpr int32_t kQm40 = -40 * 8388608;
constexpr int32_t kQm65 = -65 * 8388608;
constexpr int32_t kQm55 = -55 * 8388608;

#define MMF_SPLIT(name, val)                                 \
    constexpr double name##_d = (val);                        \
    constexpr float name##_h = (float)name##_d;               \
    constexpr float name##_l = (float)(name##_d - (double)name##_h);
MMF_SPLIT(kC10, 1.0 / (10.0 * 8388608.0))
MMF_SPLIT(kC18, 1.0 / (18.0 * 8388608.0))
MMF_SPLIT(kC80, 1.0 / (80.0 * 8388608.0))
MMF_SPLIT(k007, 0.07)
MMF_SPLIT(k01, 0.1)
MMF_SPLIT(kE1, 2.718281828459045)      // e^1
MMF_SPLIT(kE25, 12.182493960703473)    // e^2.5
MMF_SPLIT(kE3, 20.085536923187668)     // e^3
#undef MMF_SPLIT

struct Rates {
    F2 am, bm, ah, bh, an, bn;
};

// Hodgkin-Huxley rates (1/ms) at V = vq * 2^-23 mV.  With u = -(V + 65),
// every exponent is u/k plus a constant: two exponentials E18 = e^{u/18}
// and E80 = e^{u/80} give all six rates (e^{u/20} = E80^4, e^{u/10} =
// E80^8; e^{-(V+40)/10} = e^{2.5} E10, e^{-(V+55)/10} = e E10,
// e^{-(V+35)/10} = e^3 E10).  Each u/k is the exact integer difference
// (Q_{-65} - vq) times 2^-23/k before its single rounding.
MMF_HD Rates hh_rates(int32_t vq)
{
    Rates r;
    const F2 E18 = exp_df(scaled_diff(kQm65, vq, kC18_h, kC18_l));
    const F2 E80 = exp_df(scaled_diff(kQm65, vq, kC80_h, kC80_l));
    F2 E20 = mul(E80, E80);
    E20 = mul(E20, E20);
    const F2 E10 = mul(E20, E20);
    r.am = xexpm1_given(scaled_diff(kQm40, vq, kC10_h, kC10_l), mul(E10, F2{kE25_h, kE25_l}));
    r.bm = scale(E18, 4.0f);
    r.ah = mul(E20, F2{k007_h, k007_l});
    r.bh = div(F2{1.0f, 0.0f}, add_f(mul(E10, F2{kE3_h, kE3_l}), 1.0f));
    r.an = mul(xexpm1_given(scaled_diff(kQm55, vq, kC10_h, kC10_l), mul(E10, F2{kE1_h, kE1_l})), F2{k01_h, k01_l});
    r.bn = scale(E80, 0.125f);
    return r;
}

// Exponential-Euler step of one gate with frozen rates a, b over dt:
// x += (x_inf - x) (1 - e^{-dt (a + b)}), x_inf = a / (a + b).
MMF_HD uint32_t gate_step(uint32_t q, F2 a, F2 b, F2 dt)
{
    const F2 s = add(a, b);
    const F2 xinf = div(a, s);
    const F2 E = one_minus_exp_neg_df(mul(s, dt));
    const F2 d = add(xinf, neg(gate_df(q)));
    return gate_add(q, mul(d, E));
}

// V^{n+1} in fixed point; returns false if dv is not finite or V leaves
// +-120 mV (the range the integer differences above assume).
MMF_HD bool v_add(int32_t vq, float dv, int32_t *out)
{
    if (!(fabsf(dv) < 240.0f)) return false;
    const long long nv = (long long)vq + (long long)f2i_rn(dv * 8388608.0f);
    if (nv > 120LL * 8388608LL || nv < -120LL * 8388608LL) return false;
    *out = (int32_t)nv;
    return true;
}

}  // namespace mmf

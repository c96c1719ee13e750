// mm_gate_table.h -- the exponential-Euler gate update of the FP32c step
// from per-interval polynomials of V (host builder + host/device evaluation).
//
// One step of a Hodgkin-Huxley gate x with frozen rates alpha(V), beta(V)
// over dt (the exponential Euler step) is
//     x <- x + (X(V) - x) E(V),   X = alpha / (alpha + beta),
//                                 E = 1 - exp(-dt (alpha + beta)),
// so for a fixed dt each gate needs two functions of V alone.  They are
// smooth on the FP32c voltage range (+-120 mV), and a polynomial of degree
// 5 per 0.5 mV interval reproduces them to about 1e-13 relative (fitted by
// interpolation at the interval's six Chebyshev points, in FP64 on the host
// when a network is created).  The evaluation keeps the polynomial's two
// leading terms as float pairs and sums the rest in FP32, whose rounding
// enters scaled by (u h / 10 mV)^2 < 1e-3: about 1e-10 relative at most and
// 1e-14 on average.  A step-repeating error in X or E biases the gate
// trajectories every cycle; this one is far below the gate's 2^-32
// resolution (and below that of a double-float exponential by its Taylor
// series).
//
// Layout: interval i (centre V_i = -120 mV + i h, h = 2^-1 mV, 0 <= i <= 480)
// has, for m, h, n in that order, X then E, each two 16-byte quads
//     (c0.hi, c0.lo, c1.hi, c1.lo), (c2, c3, c4, c5)
// the coefficients of the polynomial in u = (V - V_i) / h in [-1/2, 1/2).
// The table is 12 arrays of 481 quads (92.3 KB), quad k of every interval
// in array k: the lanes of a warp, whose compartments' V lie close together,
// then read adjacent quads of one array (a 128-byte line holds 8 intervals,
// 4 mV) instead of lines 192 B apart.  The index and u come from the
// fixed-point V exactly: w = Vq + 120 * 2^23 + 2^21, i = w >> 22,
// u = ((w mod 2^22) - 2^21) * 2^-22.
#pragma once
#include <stdint.h>

#include <cmath>

#include "mm_fp32c_math.h"

namespace mmf {

constexpr int kTabShift = 22;                         // h = 2^22 units of 2^-23 mV = 0.5 mV
constexpr int kTabIntervals = 481;                    // centres -120, -119.5, ..., 120 mV
constexpr int kTabFuncs = 6;                          // X_m, E_m, X_h, E_h, X_n, E_n
constexpr int kTabQuads = 2 * kTabFuncs;              // quads per interval = arrays
constexpr int32_t kTabBias = 120 * 8388608 + (1 << (kTabShift - 1));

#ifdef __CUDACC__
#define MMF_TAB_HD __host__ __device__ __forceinline__
#else
#define MMF_TAB_HD inline
#endif

// four floats of the table, 16-byte aligned (a float4 in device memory)
struct alignas(16) Tab4 {
    float x, y, z, w;
};

struct TabIndex {
    int32_t i;  // interval
    float u;    // position in it, [-1/2, 1/2]
};

// Interval and position of V = vq 2^-23 mV (clamped to the table's ends).
MMF_TAB_HD TabIndex tab_index(int32_t vq)
{
    const int64_t w = (int64_t)vq + kTabBias;
    TabIndex t;
    if (w < 0) {
        t.i = 0;
        t.u = -0.5f;
    } else if (w >= (int64_t)kTabIntervals << kTabShift) {
        t.i = kTabIntervals - 1;
        t.u = 0.5f;
    } else {
        t.i = (int32_t)(w >> kTabShift);
        t.u = (float)((int32_t)(w & ((1 << kTabShift) - 1)) - (1 << (kTabShift - 1))) * (1.0f / (float)(1 << kTabShift));
    }
    return t;
}

// p(u) = c0 + c1 u + u^2 (c2 + c3 u + c4 u^2 + c5 u^3) as a float pair, from
// the two quads of one function (c0, c1 pairs; c2..c5 floats).
MMF_TAB_HD F2 tab_eval(Tab4 a, Tab4 b, float u)
{
    float q = fmaf(b.w, u, b.z);
    q = fmaf(q, u, b.y);
    q = fmaf(q, u, b.x);
    const float tail = (q * u) * u;
    const F2 p1 = two_prod(a.z, u);                 // c1.hi u, exact
    const float p1lo = fmaf(a.w, u, p1.lo);
    const F2 s = two_sum(a.x, p1.hi);
    return quick_two_sum(s.hi, s.lo + ((a.y + p1lo) + tail));
}

// One exponential-Euler step of a uint32 gate from its X and E at V (the
// four quads of the gate's two functions in V's interval).
MMF_TAB_HD uint32_t tab_gate_step(uint32_t q, const Tab4 f[4], float u)
{
    const F2 X = tab_eval(f[0], f[1], u);
    const F2 E = tab_eval(f[2], f[3], u);
    return gate_add(q, mul(add(X, neg(gate_df(q))), E));
}

// ---------------------------------------------------------------- builder
// (host only: FP64 with the C library's exp and expm1)

// x / (e^x - 1), 1 at x = 0
inline double tab_xexpm1(double x) { return std::fabs(x) < 1e-8 ? 1.0 - 0.5 * x : x / std::expm1(x); }

// X and E of the three gates at V (mV) for the step dt (ms): the Hodgkin-
// Huxley rates (1/ms) of the model (alpha_m, beta_m, alpha_h, beta_h,
// alpha_n, beta_n) in FP64.
inline void tab_functions(double V, double dt, double out[kTabFuncs])
{
    const double am = tab_xexpm1(-(V + 40.0) / 10.0);
    const double bm = 4.0 * std::exp(-(V + 65.0) / 18.0);
    const double ah = 0.07 * std::exp(-(V + 65.0) / 20.0);
    const double bh = 1.0 / (1.0 + std::exp(-(V + 35.0) / 10.0));
    const double an = 0.1 * tab_xexpm1(-(V + 55.0) / 10.0);
    const double bn = 0.125 * std::exp(-(V + 65.0) / 80.0);
    const double a[3] = {am, ah, an}, b[3] = {bm, bh, bn};
    for (int g = 0; g < 3; ++g) {
        const double s = a[g] + b[g];
        out[2 * g] = a[g] / s;
        out[2 * g + 1] = -std::expm1(-dt * s);
    }
}

// Fills tab[kTabQuads * kTabIntervals] (array k, interval i at
// k * kTabIntervals + i) for the step dt.
inline void build_gate_table(double dt, Tab4 *tab)
{
    constexpr int K = 6;                    // interpolation points = degree + 1
    const double pi = 3.14159265358979323846;
    double xk[K], Tk[K][K];                 // nodes in [-1, 1], T_j(x_k)
    for (int k = 0; k < K; ++k) {
        xk[k] = std::cos(pi * (k + 0.5) / K);
        Tk[k][0] = 1.0;
        Tk[k][1] = xk[k];
        for (int j = 2; j < K; ++j) Tk[k][j] = 2.0 * xk[k] * Tk[k][j - 1] - Tk[k][j - 2];
    }
    // monomial coefficients of T_0 .. T_5 in x
    static const double Tm[K][K] = {{1, 0, 0, 0, 0, 0},   {0, 1, 0, 0, 0, 0},    {-1, 0, 2, 0, 0, 0},
                                    {0, -3, 0, 4, 0, 0},  {1, 0, -8, 0, 8, 0},   {0, 5, 0, -20, 0, 16}};
    const double h = std::ldexp(1.0, kTabShift - 23);  // interval width, mV
    for (int i = 0; i < kTabIntervals; ++i) {
        const double Vc = -120.0 + i * h;
        double f[K][kTabFuncs];
        for (int k = 0; k < K; ++k) tab_functions(Vc + 0.5 * h * xk[k], dt, f[k]);  // u = x / 2
        for (int fn = 0; fn < kTabFuncs; ++fn) {
            double cheb[K];
            for (int j = 0; j < K; ++j) {
                double s = 0.0;
                for (int k = 0; k < K; ++k) s += f[k][fn] * Tk[k][j];
                cheb[j] = (j == 0 ? 1.0 : 2.0) * s / K;
            }
            double c[K];  // in u: x = 2u, so the coefficient of u^j is 2^j times that of x^j
            for (int j = 0; j < K; ++j) {
                double s = 0.0;
                for (int l = 0; l < K; ++l) s += cheb[l] * Tm[l][j];
                c[j] = std::ldexp(s, j);
            }
            const F2 c0 = split_d(c[0]), c1 = split_d(c[1]);
            tab[(size_t)(2 * fn) * kTabIntervals + i] = Tab4{c0.hi, c0.lo, c1.hi, c1.lo};
            tab[(size_t)(2 * fn + 1) * kTabIntervals + i] = Tab4{(float)c[2], (float)c[3], (float)c[4], (float)c[5]};
        }
    }
}

}  // namespace mmf

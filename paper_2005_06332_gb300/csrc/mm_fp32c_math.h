// mm_fp32c_math.h -- arithmetic of the FP32c step, host + device.
//
// Everything here is IEEE binary32 arithmetic (+, -, *, fma) and 32-bit
// integer conversions, so a host build of these functions gives the same bits
// as the GPU kernel.  No CUDA math library call is used.
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
//   * the gates' steady states and relaxation factors, functions of V alone,
//     come from per-interval polynomials whose leading terms are float pairs
//     (mm_gate_table.h), since their rounding biases the gate trajectories
//     every cycle;
//   * the Hines solve is FP32 on the rhs rounded once, with the diagonal split
//     into its passive part (eliminated once in FP64 at set-up, kept as a
//     pair) and the step's active conductance, eliminated in FP32 as a
//     perturbation of it.
#pragma once
#include <stdint.h>

#include <cmath>
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

MMF_HD int32_t f2i_rn(float x)
{
#ifdef __CUDA_ARCH__
    return __float2int_rn(x);
#else
    return (int32_t)std::lrintf(x);
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

// ------------------------------------------------------------ fixed point

constexpr float kV2F = 1.0f / 8388608.0f;    // 2^-23 mV per unit

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

// V^{n+1} in fixed point; returns false if dv is not finite or V leaves
// +-120 mV (the range of the integer differences above and of the gate
// table, mm_gate_table.h).
MMF_HD bool v_add(int32_t vq, float dv, int32_t *out)
{
    if (!(fabsf(dv) < 240.0f)) return false;
    const long long nv = (long long)vq + (long long)f2i_rn(dv * 8388608.0f);
    if (nv > 120LL * 8388608LL || nv < -120LL * 8388608LL) return false;
    *out = (int32_t)nv;
    return true;
}

}  // namespace mmf

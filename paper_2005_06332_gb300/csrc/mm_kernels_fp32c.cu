// mm_kernels_fp32c.cu -- FP32 compensated ("FP32c") kernels (sm_103a).
//
// Same step as the FP64 kernel (HH currents, Hines assembly of Eq. 2,
// Algorithm 1 as segment waves in shared memory, exponential-Euler gates,
// synaptic decay, soma threshold test), computed in FP32 with the state kept
// exact between steps:
//   * V is an int32 fixed-point number (2^-23 mV) and each gate a uint32
//     fixed-point number (2^-32); every step adds an FP32 increment rounded
//     once, so rounding never accumulates in the state itself;
//   * differences of potentials (V - E, V_parent - V_child, V + c in the rate
//     arguments) are taken exactly in integers before the single rounding;
//   * exponential arguments are carried as an unevaluated float pair
//     (hi + lo) and exp(hi + lo) = exp(hi) (1 + lo);
//   * the soma voltage is also accumulated in FP64 and the spike crossing
//     time is computed in FP64.
#include <cuda_runtime.h>

#include "mm_internal.h"

using namespace mmk;

namespace {

constexpr double kPiD = 3.141592653589793;

struct F2 {
    float hi, lo;
};

// (a - b) * 2^-23, one rounding.
__device__ __forceinline__ float vdiff(int32_t a, int32_t b)
{
    return (float)((long long)a - (long long)b) * kVInv;
}

__device__ __forceinline__ float vminus(int32_t vq, FxPot E) { return vdiff(vq, E.q) - E.res; }

// (a - b) * c as a float pair, where c = ch + cl.
__device__ __forceinline__ F2 scaled_diff(int32_t a, int32_t b, float ch, float cl)
{
    const long long d = (long long)a - (long long)b;
    const float dh = (float)d;
    const float dl = (float)(d - (long long)dh);
    const float xh = dh * ch;
    const float xl = fmaf(dh, ch, -xh) + fmaf(dh, cl, dl * ch);
    return {xh, xl};
}

__device__ __forceinline__ float exp_pair(F2 x)
{
    const float e = expf(x.hi);
    return fmaf(e, x.lo, e);
}

// x / (e^x - 1) for x = hi + lo.
__device__ __forceinline__ float xexpm1_ratio_pair(F2 x)
{
    if (fabsf(x.hi) < 1e-4f) {
        const float v = x.hi + x.lo;
        return fmaf(v, fmaf(v, 1.0f / 12.0f, -0.5f), 1.0f);
    }
    const float E = expm1f(x.hi);
    const float den = fmaf(x.lo, E + 1.0f, E);
    return __fdiv_rn(x.hi + x.lo, den);
}

// Fixed-point potentials of the rate-function shifts (exact: integer mV).
constexpr int32_t kQm40 = -40 * 8388608;
constexpr int32_t kQm65 = -65 * 8388608;
constexpr int32_t kQm35 = -35 * 8388608;
constexpr int32_t kQm55 = -55 * 8388608;

// 2^-23 / k split into a float pair.
#define MMK_SPLIT(name, k)                                               \
    constexpr double name##_d = 1.0 / ((double)(k) * 8388608.0);         \
    constexpr float name##_h = (float)name##_d;                          \
    constexpr float name##_l = (float)(name##_d - (double)name##_h);
MMK_SPLIT(kC10, 10)
MMK_SPLIT(kC18, 18)
MMK_SPLIT(kC20, 20)
MMK_SPLIT(kC80, 80)
#undef MMK_SPLIT

struct Rates32 {
    float am, bm, ah, bh, an, bn;
};

// HH rates (1/ms) at V = vq * 2^-23 mV; every argument -(V + c)/k is formed
// as (Q_{-c} - vq) * 2^-23 / k exactly before rounding.
__device__ __forceinline__ Rates32 hh_rates32(int32_t vq)
{
    Rates32 r;
    r.am = xexpm1_ratio_pair(scaled_diff(kQm40, vq, kC10_h, kC10_l));
    r.bm = 4.0f * exp_pair(scaled_diff(kQm65, vq, kC18_h, kC18_l));
    r.ah = 0.07f * exp_pair(scaled_diff(kQm65, vq, kC20_h, kC20_l));
    r.bh = __frcp_rn(1.0f + exp_pair(scaled_diff(kQm35, vq, kC10_h, kC10_l)));
    r.an = 0.1f * xexpm1_ratio_pair(scaled_diff(kQm55, vq, kC10_h, kC10_l));
    r.bn = 0.125f * exp_pair(scaled_diff(kQm65, vq, kC80_h, kC80_l));
    return r;
}

// Exponential-Euler relaxation of a fixed-point gate: dx = (xinf - x)(1 - e^{-dt s}).
__device__ __forceinline__ uint32_t gate_step32(uint32_t q, float a, float b, float dt)
{
    const float s = a + b;
    const float xinf = __fdiv_rn(a, s);
    const float E = expm1f(-dt * s);
    const float qh = __uint2float_rn(q);
    const float ql = (float)((long long)q - (long long)qh);
    const float d = (xinf - qh * kGInv) - ql * kGInv;
    const long long nq = (long long)q + __float2ll_rn(-E * d * kGScale);
    return (uint32_t)(nq < 0 ? 0 : (nq > 4294967295LL ? 4294967295LL : nq));
}

__device__ __forceinline__ float gate_value(uint32_t q) { return __uint2float_rn(q) * kGInv; }

// ------------------------------------------------------------------ init

__device__ __forceinline__ double half_cyl_resistance_d(double Ra, double L_um, double d_um)
{
    const double rad = 0.5e-4 * d_um;
    return Ra * (0.5e-4 * L_um) / (kPiD * rad * rad) * 1e-6;
}

__device__ __forceinline__ double xexpm1_d(double x) { return fabs(x) < 1e-6 ? 1.0 - 0.5 * x : x / expm1(x); }

__global__ void init_fp32c_kernel(InitArgs a)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.C;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double L = a.L[i], d = a.diam[i];
        a.area32[i] = (float)(kPiD * d * L * 1e-8);
        const int32_t pd = a.parent_dist[i];
        double g = 0.0;
        if (pd > 0) {
            const int64_t q = i - pd;
            g = 1.0 / (half_cyl_resistance_d(a.Ra, L, d) + half_cyl_resistance_d(a.Ra, a.L[q], a.diam[q]));
        }
        a.gax32[i] = (float)g;
        const double v = a.v_init;
        a.Vq[i] = (int32_t)llrint(v * kVScaleD);
        const double am = xexpm1_d(-(v + 40.0) * 0.1), bm = 4.0 * exp(-(v + 65.0) / 18.0);
        const double ah = 0.07 * exp(-(v + 65.0) * 0.05), bh = 1.0 / (1.0 + exp(-(v + 35.0) * 0.1));
        const double an = 0.1 * xexpm1_d(-(v + 55.0) * 0.1), bn = 0.125 * exp(-(v + 65.0) * 0.0125);
        auto fx = [](double x) -> uint32_t {
            const double q = rint(x * kGScaleD);
            return (uint32_t)(q < 0.0 ? 0.0 : (q > 4294967295.0 ? 4294967295.0 : q));
        };
        a.mq[i] = fx(am / (am + bm));
        a.hq[i] = fx(ah / (ah + bh));
        a.nq[i] = fx(an / (an + bn));
    }
}

// --------------------------------------------------------------- delivery

constexpr int kMaxDClass32 = 1024;

__global__ void __launch_bounds__(256) deliver_fp32c_kernel(DeliverArgs a)
{
    __shared__ int s_pref[kMaxDClass32 + 1];
    __shared__ int s_slot[kMaxDClass32];
    const long long n = (long long)a.ctl->step_base + a.step_offset;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->queue_head = 0u;
        a.ring_cnt[n % a.R] = 0;
    }
    for (int k = threadIdx.x; k < a.n_dclass; k += blockDim.x) {
        const long long src_step = n - 1 - a.dclass[k];
        int cnt = 0, slot = 0;
        if (src_step >= 0) {
            slot = (int)(src_step % a.R);
            cnt = a.ring_cnt[slot];
        }
        s_slot[k] = slot;
        s_pref[k + 1] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_pref[0] = 0;
        for (int k = 1; k <= a.n_dclass; ++k) s_pref[k] += s_pref[k - 1];
    }
    __syncthreads();
    const int total = s_pref[a.n_dclass];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < total; u += nwarps) {
        int lo = 0, hi = a.n_dclass;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_pref[mid] <= u) lo = mid; else hi = mid;
        }
        const int src = a.ring_nrn[(long long)s_slot[lo] * a.N + (u - s_pref[lo])];
        long long b = a.out_off[src], e = a.out_off[src + 1];
        if (a.n_dclass > 1) {
            const int D = a.dclass[lo];
            long long l = b, r = e;
            while (l < r) { const long long m = (l + r) >> 1; if (a.out_dsteps[m] < D) l = m + 1; else r = m; }
            long long l2 = l, r2 = e;
            while (l2 < r2) { const long long m = (l2 + r2) >> 1; if (a.out_dsteps[m] <= D) l2 = m + 1; else r2 = m; }
            b = l;
            e = l2;
        }
        for (long long q = b + lane; q < e; q += 32) atomicAdd(&a.gsyn32[a.out_site[q]], a.out_w32[q]);
    }
}

// ------------------------------------------------------------ FP32c step

template <int NT>
__global__ void __launch_bounds__(NT) step_fp32c_kernel(StepArgs32 a)
{
    extern __shared__ float smem32[];
    float *sd = smem32;                      // diagonal; after elimination: its reciprocal
    float *sr = smem32 + a.smem_comps;       // rhs; after substitution: dV
    float *scd = sr + a.smem_comps;          // per-segment contributions to the parent
    float *scr = scd + a.smem_segs;
    __shared__ int s_item;

    const long long n = (long long)a.ctl->step_base + a.step_offset;
    const int tid = threadIdx.x;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = (int)atomicAdd(&a.ctl->queue_head, 1u);
        __syncthreads();
        const int gi = s_item;
        if (gi >= a.n_groups) break;
        const GroupRec G = a.groups[gi];
        const int64_t c0 = G.comp0;
        const int32_t *Vq = a.Vq + c0;
        const float *gax = a.gax + c0;

        // A. membrane conductance and current at (V^n, gates^n)
        for (int i = tid; i < G.ncomp; i += NT) {
            const int32_t vq = Vq[i];
            const float m = gate_value(a.mq[c0 + i]), h = gate_value(a.hq[c0 + i]), nn = gate_value(a.nq[c0 + i]);
            const float ar = a.area[c0 + i];
            const float s = ar * 1e3f;
            const float gna = a.gNa * s * (m * m * m * h);
            const float n2 = nn * nn;
            const float gk = a.gK * s * (n2 * n2);
            const float gl = a.gL * s;
            sd[i] = fmaf(ar, a.cm_dt, gna + gk + gl);
            sr[i] = -fmaf(gna, vminus(vq, a.ENa), fmaf(gk, vminus(vq, a.EK), gl * vminus(vq, a.EL)));
        }
        __syncthreads();

        // S. synaptic sites, then decay
        for (int t = tid; t < G.nsite; t += NT) {
            const int st = G.site0 + t;
            const int c = a.site_comp[st];
            const float g = a.gsyn[st];
            sd[c] += g;
            sr[c] = fmaf(-g, vminus(Vq[c], a.Esyn), sr[c]);
            a.gsyn[st] = g * a.decay;
        }
        __syncthreads();

        // B. leaves-to-root elimination with the axial terms folded in
        const SegRec *segs = a.segs + G.seg0;
        const int *woff = a.wave_off + G.wave0;
        for (int w = 0; w < G.nwave; ++w) {
            const int sb = woff[w], se = woff[w + 1];
            for (int si = sb + tid; si < se; si += NT) {
                const SegRec S = segs[si];
                const int bot = S.top + S.len - 1;
                float db = sd[bot], rb = sr[bot];
                for (int c = 0; c < S.nchild; ++c) {
                    const int cs = a.seg_child[S.child0 + c];
                    db += scd[cs];
                    rb += scr[cs];
                }
                for (int j = bot; j > S.top; --j) {
                    const float g = gax[j];
                    const float vpj = vdiff(Vq[j - 1], Vq[j]);       // V_p - V_j
                    db += g;
                    rb = fmaf(g, vpj, rb);
                    const float inv = __frcp_rn(db);
                    sd[j] = inv;
                    sr[j] = rb;
                    const float f = g * inv;
                    db = fmaf(-f, g, sd[j - 1] + g);
                    rb = fmaf(f, rb, fmaf(-g, vpj, sr[j - 1]));
                }
                const int t = S.top;
                if (S.parent >= 0) {
                    const float g = gax[t];
                    const float vpt = vdiff(Vq[S.parent], Vq[t]);
                    db += g;
                    rb = fmaf(g, vpt, rb);
                    const float inv = __frcp_rn(db);
                    sd[t] = inv;
                    sr[t] = rb;
                    const float f = g * inv;
                    scd[si] = fmaf(-f, g, g);
                    scr[si] = fmaf(f, rb, -g * vpt);
                } else {
                    rb += (float)a.stim[G.neuron0 + S.neuron];
                    const float inv = __frcp_rn(db);
                    sd[t] = inv;
                    sr[t] = rb * inv;
                }
            }
            __syncthreads();
        }

        // F. root-to-leaves substitution; the soma segment runs the FP64
        //    soma accumulator and the spike test
        for (int w = G.nwave - 1; w >= 0; --w) {
            const int sb = woff[w], se = woff[w + 1];
            for (int si = sb + tid; si < se; si += NT) {
                const SegRec S = segs[si];
                const int t = S.top;
                float x;
                if (S.parent >= 0) {
                    x = fmaf(gax[t], sr[S.parent], sr[t]) * sd[t];
                    sr[t] = x;
                } else {
                    x = sr[t];
                    const int nrn = G.neuron0 + S.neuron;
                    const double v0 = a.Vsoma[nrn], v1 = v0 + (double)x;
                    a.Vsoma[nrn] = v1;
                    if (!isfinite(v1)) atomicOr(&a.ctl->err, MMK_ERR_NUMERIC);
                    if (v0 < a.threshold && v1 >= a.threshold) {
                        const double ts = (double)n * a.dt64 + a.dt64 * (a.threshold - v0) / (v1 - v0);
                        const unsigned long long k = atomicAdd(&a.ctl->spk_count, 1ull);
                        if ((long long)k < a.spk_cap) {
                            a.spk_nrn[k] = a.user_id[nrn];
                            a.spk_t[k] = ts;
                        } else {
                            atomicOr(&a.ctl->err, MMK_ERR_OVERFLOW);
                        }
                        const int slot = (int)(n % a.R);
                        const int pos = atomicAdd(&a.ring_cnt[slot], 1);
                        a.ring_nrn[(long long)slot * a.N + pos] = nrn;
                    }
                }
                for (int j = t + 1; j < t + S.len; ++j) {
                    x = fmaf(gax[j], x, sr[j]) * sd[j];
                    sr[j] = x;
                }
            }
            __syncthreads();
        }

        // C. V^{n+1} = V^n + dV (exact in fixed point), gates at V^{n+1}
        for (int i = tid; i < G.ncomp; i += NT) {
            const float dv = sr[i];
            long long nv = (long long)Vq[i] + __float2ll_rn(dv * kVScale);
            if (!(fabsf(dv) < 256.0f) || nv > 2147483647LL || nv < -2147483647LL) {
                atomicOr(&a.ctl->err, MMK_ERR_NUMERIC);
                nv = (long long)Vq[i];
            }
            const int32_t vq = (int32_t)nv;
            a.Vq[c0 + i] = vq;
            const Rates32 r = hh_rates32(vq);
            a.mq[c0 + i] = gate_step32(a.mq[c0 + i], r.am, r.bm, a.dt);
            a.hq[c0 + i] = gate_step32(a.hq[c0 + i], r.ah, r.bh, a.dt);
            a.nq[c0 + i] = gate_step32(a.nq[c0 + i], r.an, r.bn, a.dt);
        }
    }
}

__global__ void vq_to_f64_kernel(const int32_t *vq, double *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)vq[i] / kVScaleD;
}

__global__ void gq_to_f64_kernel(const uint32_t *q, double *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (double)q[i] / kGScaleD;
}

__global__ void scatter_f32_to_f64_kernel(const float *src, const int64_t *idx, double *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[idx[i]] = (double)src[i];
}

int grid32(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

template <int NT>
int set_attr_and_occupancy(int smem, int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(step_fp32c_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, step_fp32c_kernel<NT>, NT, smem);
    return (int)e;
}

}  // namespace

int mmk_launch_step_fp32c(const StepArgs32 &a, int blocks, int threads, void *stream)
{
    const size_t smem = (size_t)(2 * a.smem_comps + 2 * a.smem_segs) * sizeof(float);
    cudaStream_t s = (cudaStream_t)stream;
    switch (threads) {
    case 128: step_fp32c_kernel<128><<<blocks, 128, smem, s>>>(a); break;
    case 256: step_fp32c_kernel<256><<<blocks, 256, smem, s>>>(a); break;
    case 512: step_fp32c_kernel<512><<<blocks, 512, smem, s>>>(a); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

int mmk_step_fp32c_blocks_per_sm(int threads, int smem_bytes, int *blocks)
{
    switch (threads) {
    case 128: return set_attr_and_occupancy<128>(smem_bytes, blocks);
    case 256: return set_attr_and_occupancy<256>(smem_bytes, blocks);
    case 512: return set_attr_and_occupancy<512>(smem_bytes, blocks);
    default: return (int)cudaErrorInvalidValue;
    }
}

int mmk_launch_init_fp32c(const InitArgs &a, void *stream)
{
    init_fp32c_kernel<<<grid32(a.C, 256), 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int mmk_launch_deliver_fp32c(const DeliverArgs &a, int blocks, void *stream)
{
    if (a.n_dclass > kMaxDClass32) return (int)cudaErrorInvalidValue;
    deliver_fp32c_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int mmk_launch_vq_to_f64(const int32_t *vq, double *dst, int64_t n, void *stream)
{
    if (n <= 0) return 0;
    vq_to_f64_kernel<<<grid32(n, 256), 256, 0, (cudaStream_t)stream>>>(vq, dst, n);
    return (int)cudaGetLastError();
}

int mmk_launch_gq_to_f64(const uint32_t *q, double *dst, int64_t n, void *stream)
{
    if (n <= 0) return 0;
    gq_to_f64_kernel<<<grid32(n, 256), 256, 0, (cudaStream_t)stream>>>(q, dst, n);
    return (int)cudaGetLastError();
}

int mmk_launch_scatter_f32_to_f64(const float *src, const int64_t *idx, double *dst, int64_t n, void *stream)
{
    if (n <= 0) return 0;
    scatter_f32_to_f64_kernel<<<grid32(n, 256), 256, 0, (cudaStream_t)stream>>>(src, idx, dst, n);
    return (int)cudaGetLastError();
}

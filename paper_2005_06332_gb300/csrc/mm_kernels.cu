// mm_kernels.cu -- FP64 kernels of the multi-morphology stepper (sm_103a).
//
// One time step n -> n+1 is two launches:
//   deliver_kernel: spikes detected round(delay/dt) + 1 steps ago raise the
//                   synaptic conductance of their target sites (the local /
//                   global spike buffers of Sec. 2 become a device ring of
//                   per-step spike lists, expanded through an outgoing CSR);
//   step_fp64:      per work item (a run of whole neurons): HH currents,
//                   assembly of the Hines system for dV (Eq. 2), the Hines
//                   solve (Algorithm 1) as segment waves in shared memory,
//                   V += dV, exponential-Euler gates, synaptic decay and the
//                   soma threshold test.
// The model is the oracle's (units um, mV, ms, nA, uS, nF); the arithmetic
// here is written independently of it.
#include <cuda_runtime.h>

#include <mutex>

#include "mm_internal.h"
#include "mm_tma.h"

using namespace mmk;

namespace {

constexpr double kPi = 3.141592653589793;

// x / (e^x - 1) and its limit near 0.
__device__ __forceinline__ double xexpm1_ratio(double x)
{
    return fabs(x) < 1e-6 ? 1.0 - 0.5 * x : x / expm1(x);
}

// HH rate constants (1/ms) at v (mV), rest -65 mV.
struct Rates {
    double am, bm, ah, bh, an, bn;
};

__device__ __forceinline__ Rates hh_rates(double v)
{
    Rates r;
    r.am = xexpm1_ratio(-(v + 40.0) * 0.1);
    r.bm = 4.0 * exp(-(v + 65.0) * (1.0 / 18.0));
    r.ah = 0.07 * exp(-(v + 65.0) * 0.05);
    r.bh = 1.0 / (1.0 + exp(-(v + 35.0) * 0.1));
    r.an = 0.1 * xexpm1_ratio(-(v + 55.0) * 0.1);
    r.bn = 0.125 * exp(-(v + 65.0) * 0.0125);
    return r;
}

// Exact relaxation of one gate over dt with frozen rates.
__device__ __forceinline__ double relax(double x, double a, double b, double dt)
{
    double s = a + b;
    double xinf = a / s;
    return xinf + (x - xinf) * exp(-dt * s);
}

__device__ __forceinline__ double half_cyl_resistance(double Ra, double L_um, double d_um)
{
    // MOhm: Ra * (L/2) / (pi d^2 / 4), lengths converted um -> cm
    double rad = 0.5e-4 * d_um;
    return Ra * (0.5e-4 * L_um) / (kPi * rad * rad) * 1e-6;
}

// ------------------------------------------------------------------ init

__global__ void init_kernel(InitArgs a)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.C;
         i += (int64_t)gridDim.x * blockDim.x) {
        double L = a.L[i], d = a.diam[i];
        a.area[i] = kPi * d * L * 1e-8;
        const int32_t pd = abs(a.parent_dist[i]);
        double g = 0.0;
        if (pd > 0) {
            const int64_t q = i - pd;
            g = 1.0 / (half_cyl_resistance(a.Ra, L, d) + half_cyl_resistance(a.Ra, a.L[q], a.diam[q]));
        }
        a.gax[i] = g;
        double v = a.v_init;
        Rates r = hh_rates(v);
        a.V[i] = v;
        a.m[i] = r.am / (r.am + r.bm);
        a.h[i] = r.ah / (r.ah + r.bh);
        a.n[i] = r.an / (r.an + r.bn);
    }
}

// --------------------------------------------------------------- delivery

constexpr int kMaxDClass = 1024;

__global__ void __launch_bounds__(256) deliver_kernel(DeliverArgs a)
{
    __shared__ int s_pref[kMaxDClass + 1];
    __shared__ int s_slot[kMaxDClass];
    const long long n = (long long)a.ctl->step_base + a.step_offset;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->queue_head = 0u;
        a.ctl->giant_head = 0u;
        a.ctl->big_head = 0u;
        a.ring_cnt[n % a.R] = 0;
    }
    for (int k = threadIdx.x; k < a.n_dclass; k += blockDim.x) {
        long long src_step = n - 1 - a.dclass[k];
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
    // groups of lanes_per_src lanes take one spike each (see the FP32c kernel)
    const int GL = a.lanes_per_src;
    const int lane = threadIdx.x & (GL - 1);
    const int ngroups = (gridDim.x * blockDim.x) / GL;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) / GL; u < total; u += ngroups) {
        int lo = 0, hi = a.n_dclass;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (s_pref[mid] <= u) lo = mid; else hi = mid;
        }
        const int src = a.ring_nrn[(long long)s_slot[lo] * a.N + (u - s_pref[lo])];
        long long b = a.out_off[src], e = a.out_off[src + 1];
        if (a.n_dclass > 1) {
            const int D = a.dclass[lo];
            long long l = b, r = e;            // first entry with dsteps >= D
            while (l < r) { long long m = (l + r) >> 1; if (a.out_dsteps[m] < D) l = m + 1; else r = m; }
            long long l2 = l, r2 = e;          // first entry with dsteps > D
            while (l2 < r2) { long long m = (l2 + r2) >> 1; if (a.out_dsteps[m] <= D) l2 = m + 1; else r2 = m; }
            b = l; e = l2;
        }
        for (long long q = b + lane; q < e; q += GL) atomicAdd(&a.gsyn[a.out_site[q]], a.out_w[q]);
    }
}

// Deterministic delivery (mm_options.deterministic_delivery): each site adds
// the weights of its synapses whose source fired round(delay/dt) + 1 steps
// ago, in ascending synapse id (the oracle's order), one thread per site;
// also the per-step resets of the work queues, of this step's spike-ring
// count and of this step's slot of the fired bitmasks (last written R steps
// ago, all of whose events are delivered).
__global__ void __launch_bounds__(256) deliver_ordered_kernel(DeliverArgs a)
{
    const long long n = (long long)a.ctl->step_base + a.step_offset;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nt = (long long)gridDim.x * blockDim.x;
    if (gt == 0) {
        a.ctl->queue_head = 0u;
        a.ctl->giant_head = 0u;
        a.ctl->big_head = 0u;
        a.ring_cnt[n % a.R] = 0;
    }
    uint32_t *slot = a.fired + (n % a.R) * a.fired_words;
    for (long long w = gt; w < a.fired_words; w += nt) slot[w] = 0u;
    for (long long st = gt; st < a.nsite; st += nt) {
        const long long e0 = a.in_off[st], e1 = a.in_off[st + 1];
        if (e0 == e1) continue;
        double g = a.gsyn[st];
        bool hit = false;
        for (long long e = e0; e < e1; ++e) {
            const long long m = n - 1 - a.in_dsteps[e];
            if (m < 0) continue;
            const int src = a.in_src[e];
            if ((a.fired[(m % a.R) * a.fired_words + (src >> 5)] >> (src & 31)) & 1u) {
                g += a.in_w[e];
                hit = true;
            }
        }
        if (hit) a.gsyn[st] = g;
    }
}

// ------------------------------------------------------------ FP64 step

template <int NT>
__global__ void __launch_bounds__(NT) step_fp64_kernel(StepArgs a)
{
    // Shared memory: the work item's tree blob (one bulk copy), then the
    // diagonal (after elimination: its reciprocal) and rhs (after
    // substitution: dV) of every compartment.
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smeta = smem_raw;
    double *sd = (double *)(smem_raw + a.smem_meta);
    double *sr = sd + a.smem_comps;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_item, s_abort;

    const long long n = (long long)a.ctl->step_base + a.step_offset;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    uint32_t parity = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const int item = (int)atomicAdd(&a.ctl->queue_head, 1u);
            s_item = item;
            s_abort = 0;
            if (item < a.n_groups) {
                const GroupRec *gp = a.groups + item;
                const uint32_t bytes = (uint32_t)gp->meta_bytes;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar, bytes);
                bulk_copy_g2s(smeta, a.meta + gp->meta_off, bytes, &bar);
            }
        }
        __syncthreads();
        const int gi = s_item;
        if (gi >= a.n_groups) break;
        const GroupRec G = a.groups[gi];
        const int64_t c0 = G.comp0;
        const double *V = a.V + c0;
        const double *gax = a.gax + c0;

        // A. membrane conductance and current at (V^n, gates^n): the
        //    compartment's own part of the diagonal and right-hand side.
        for (int i = tid; i < G.ncomp; i += NT) {
            const double v = V[i], mm = a.m[c0 + i], hh = a.h[c0 + i], nn = a.n[c0 + i];
            const double ar = a.area[c0 + i];
            const double s = ar * 1e3;
            const double gna = a.gNa * s * (mm * mm * mm * hh);
            const double n2 = nn * nn;
            const double gk = a.gK * s * (n2 * n2);
            const double gl = a.gL * s;
            sd[i] = ar * a.cm_dt + (a.g_implicit ? gna + gk + gl : 0.0);
            sr[i] = -(gna * (v - a.ENa) + gk * (v - a.EK) + gl * (v - a.EL));
        }
        if (!mbar_wait_bounded(&bar, parity)) {
            // give up on this item, but not on the copy in flight: wait for
            // it once more (bounded) so that the block never leaves while
            // the copy could still write into its shared memory
            s_abort = 1;
            mbar_wait_bounded(&bar, parity);
        }
        parity ^= 1u;
        __syncthreads();
        if (s_abort) {
            if (tid == 0) atomicOr(&a.ctl->err, MMK_ERR_TIMEOUT);
            break;
        }
        const SegP *segs = (const SegP *)smeta;
        const int16_t *kids = (const int16_t *)(segs + G.nseg);
        const int16_t *woff = kids + G.nchild;

        // S. synaptic sites: conductance into the system, then decay.
        for (int t = tid; t < G.nsite; t += NT) {
            const int st = G.site0 + t;
            const int c = a.site_comp[st];
            const double g = a.gsyn[st];
            if (a.g_implicit) sd[c] += g;
            sr[c] -= g * (V[c] - a.e_syn);
            a.gsyn[st] = g * a.decay;
        }
        __syncthreads();

        // B. leaves-to-root elimination, one segment per thread, wave by wave.
        //    The axial terms of each link (i, p(i)) are folded in as the sweep
        //    reaches i: d_i += w g, rhs_i += g (V_p - V_i) and, for the parent,
        //    d_p += w g, rhs_p += g (V_i - V_p), next to the elimination update
        //    d_p -= (a_i/d_i) c_i, rhs_p -= (a_i/d_i) rhs_i with a_i = c_i = -w g
        //    (w = gimp: 1, or 1/2 for Eq. 2 as printed).
        for (int w = 0; w < G.nwave; ++w) {
            const int sb = woff[w], se = woff[w + 1];
            for (int si = sb + tid; si < se; si += NT) {
                const SegP S = segs[si];
                const int bot = S.top + S.len - 1;
                double db = sd[bot], rb = sr[bot];
                // each child segment hangs off the bottom: from its top's
                // stored 1/d and rhs, its link terms (+g, +g (V_t - V_b)) and
                // its elimination (-g^2/d_t, +g rhs_t/d_t)
                for (int c = 0; c < S.nchild; ++c) {
                    const int t = segs[kids[S.child0 + c]].top;
                    const double g = gax[t], gi = a.gimp * g;
                    const double f = gi * sd[t];
                    db += gi - f * gi;
                    rb += g * (V[t] - V[bot]) + f * sr[t];
                }
                for (int j = bot; j > S.top; --j) {
                    const double g = gax[j], gi = a.gimp * g;
                    const double vj = V[j], vp = V[j - 1];
                    db += gi;
                    rb += g * (vp - vj);
                    const double inv = 1.0 / db;
                    sd[j] = inv;
                    sr[j] = rb;
                    const double f = gi * inv;
                    db = sd[j - 1] + gi - f * gi;
                    rb = sr[j - 1] + g * (vj - vp) + f * rb;
                }
                const int t = S.top;
                if (S.parent >= 0) {
                    const double g = gax[t];
                    db += a.gimp * g;
                    rb += g * (V[S.parent] - V[t]);
                    sd[t] = 1.0 / db;
                    sr[t] = rb;
                } else {
                    rb += a.stim[G.neuron0 + S.neuron];
                    const double inv = 1.0 / db;
                    sd[t] = inv;
                    sr[t] = rb * inv;     // dV at the soma
                }
            }
            __syncthreads();
        }

        // F. root-to-leaves substitution in the reverse wave order; the soma
        //    segment also runs the spike test.
        for (int w = G.nwave - 1; w >= 0; --w) {
            const int sb = woff[w], se = woff[w + 1];
            for (int si = sb + tid; si < se; si += NT) {
                const SegP S = segs[si];
                const int t = S.top;
                double x;
                if (S.parent >= 0) {
                    x = (sr[t] + a.gimp * gax[t] * sr[S.parent]) * sd[t];
                    sr[t] = x;
                } else {
                    x = sr[t];
                    const double v0 = V[t], v1 = v0 + x;
                    const int nrn = G.neuron0 + S.neuron;
                    if (!isfinite(v1)) atomicOr(&a.ctl->err, MMK_ERR_NUMERIC);
                    if (v0 < a.threshold && v1 >= a.threshold) {
                        const int src = soma_source(a, nrn);
                        if (src >= 0)
                            record_spike(a, src, a.user_id[nrn], 0,
                                         (double)n * a.dt + a.dt * (a.threshold - v0) / (v1 - v0), n);
                    }
                }
                for (int j = t + 1; j < t + S.len; ++j) {
                    x = (sr[j] + a.gimp * gax[j] * x) * sd[j];
                    sr[j] = x;
                }
            }
            __syncthreads();
        }

        // C. V^{n+1} = V^n + dV, the threshold test of the detection points
        //    other than somata, then exponential-Euler gates at V^{n+1}.
        for (int i = tid; i < G.ncomp; i += NT) {
            const double v0 = V[i], v = v0 + sr[i];
            a.V[c0 + i] = v;
            if (a.pt_of && v0 < a.threshold && v >= a.threshold) {
                const int p = a.pt_of[c0 + i];
                if (p >= 0) point_spike(a, p, v0, v, n, a.dt);
            }
            const Rates r = hh_rates(v);
            a.m[c0 + i] = relax(a.m[c0 + i], r.am, r.bm, a.dt);
            a.h[c0 + i] = relax(a.h[c0 + i], r.ah, r.bh, a.dt);
            a.n[c0 + i] = relax(a.n[c0 + i], r.an, r.bn, a.dt);
        }
    }
}

__global__ void advance_kernel(DevCtl *ctl, int steps) { ctl->step_base += (unsigned long long)steps; }

// Spikes of external sources into the ring slots of their steps, as if the
// step kernel had recorded them: source id N + src[i] appended to slot
// step[i] % R (and its bit in the fired mask of deterministic delivery).  A
// slot holds at most Nsrc ids: an append beyond that is undone and flagged.
__global__ void inject_kernel(int32_t *ring_nrn, int32_t *ring_cnt, int32_t R, int32_t Nsrc, int32_t N,
                              uint32_t *fired, int32_t fired_words, const int32_t *src, const int64_t *step, int64_t n,
                              DevCtl *ctl)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int slot = (int)(step[i] % R);
        const int id = N + src[i];
        const int p = atomicAdd(&ring_cnt[slot], 1);
        if (p >= Nsrc) {
            atomicSub(&ring_cnt[slot], 1);
            atomicOr(&ctl->err, MMK_ERR_OVERFLOW);
            continue;
        }
        ring_nrn[(long long)slot * Nsrc + p] = id;
        if (fired) atomicOr(&fired[(long long)slot * fired_words + (id >> 5)], 1u << (id & 31));
    }
}

__global__ void gather_f64_kernel(const double *src, const int64_t *idx, double *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[idx[i]];
}

__global__ void scatter_f64_kernel(const double *src, const int64_t *idx, double *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[idx[i]] = src[i];
}

__global__ void fill_f64_kernel(double *dst, double v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = v;
}

int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

}  // namespace

int mmk_launch_init(const InitArgs &a, void *stream)
{
    init_kernel<<<grid_for(a.C, 256), 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int mmk_launch_deliver(const DeliverArgs &a, int blocks, void *stream)
{
    if (a.n_dclass > kMaxDClass) return (int)cudaErrorInvalidValue;
    deliver_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int mmk_launch_deliver_ordered(const DeliverArgs &a, int blocks, void *stream)
{
    deliver_ordered_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

size_t mmk_step_fp64_smem(int comps, int segs, int meta_bytes)
{
    (void)segs;
    return (size_t)meta_bytes + (size_t)(2 * comps) * sizeof(double);
}

static size_t step_smem_bytes(const StepArgs &a) { return mmk_step_fp64_smem(a.smem_comps, a.smem_segs, a.smem_meta); }

int mmk_launch_step_fp64(const StepArgs &a, int blocks, int threads, void *stream)
{
    const size_t smem = step_smem_bytes(a);
    cudaStream_t s = (cudaStream_t)stream;
    switch (threads) {
    case 128:
        step_fp64_kernel<128><<<blocks, 128, smem, s>>>(a);
        break;
    case 256:
        step_fp64_kernel<256><<<blocks, 256, smem, s>>>(a);
        break;
    case 512:
        step_fp64_kernel<512><<<blocks, 512, smem, s>>>(a);
        break;
    default:
        return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

// The dynamic shared-memory limit only ever grows (see the FP32c kernels:
// several networks of one process share the kernel's attribute).
template <int NT>
static int fp64_attr_and_occupancy(int smem, int *blocks)
{
    static std::mutex mu;
    static int limit = 0;
    cudaError_t e = cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (smem > limit) {
            e = cudaFuncSetAttribute(step_fp64_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess) limit = smem;
        }
    }
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, step_fp64_kernel<NT>, NT, smem);
    return (int)e;
}

int mmk_step_fp64_blocks_per_sm(int threads, int smem_bytes, int *blocks)
{
    switch (threads) {
    case 128: return fp64_attr_and_occupancy<128>(smem_bytes, blocks);
    case 256: return fp64_attr_and_occupancy<256>(smem_bytes, blocks);
    case 512: return fp64_attr_and_occupancy<512>(smem_bytes, blocks);
    default: return (int)cudaErrorInvalidValue;
    }
}

int mmk_launch_inject(int32_t *ring_nrn, int32_t *ring_cnt, int32_t R, int32_t Nsrc, int32_t N, uint32_t *fired,
                      int32_t fired_words, const int32_t *src, const int64_t *step, int64_t n, DevCtl *ctl,
                      void *stream)
{
    if (n <= 0) return 0;
    inject_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(ring_nrn, ring_cnt, R, Nsrc, N, fired,
                                                                      fired_words, src, step, n, ctl);
    return (int)cudaGetLastError();
}

int mmk_launch_advance(DevCtl *ctl, int steps, void *stream)
{
    advance_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(ctl, steps);
    return (int)cudaGetLastError();
}

int mmk_launch_gather_f64(const double *src, const int64_t *idx, double *dst, int64_t n, void *stream)
{
    if (n <= 0) return 0;
    gather_f64_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(src, idx, dst, n);
    return (int)cudaGetLastError();
}

int mmk_launch_scatter_f64(const double *src, const int64_t *idx, double *dst, int64_t n, void *stream)
{
    if (n <= 0) return 0;
    scatter_f64_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(src, idx, dst, n);
    return (int)cudaGetLastError();
}

int mmk_launch_fill_f64(double *dst, double v, int64_t n, void *stream)
{
    if (n <= 0) return 0;
    fill_f64_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(dst, v, n);
    return (int)cudaGetLastError();
}

namespace mmk {
__global__ void bounded_wait_selftest_kernel(int *err, uint32_t max_polls)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (!mbar_wait_bounded(&bar, 0u, max_polls) && threadIdx.x == 0) atomicOr(err, MMK_ERR_TIMEOUT);
}
}  // namespace mmk

int mmk_launch_wait_selftest(int *err, unsigned int max_polls, void *stream)
{
    mmk::bounded_wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(err, max_polls);
    return (int)cudaGetLastError();
}

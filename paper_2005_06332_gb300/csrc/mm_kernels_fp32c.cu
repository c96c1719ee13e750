// mm_kernels_fp32c.cu -- FP32 compensated ("FP32c") kernels (sm_103a).
//
// Same step as the FP64 kernel (HH currents, Hines assembly of Eq. 2,
// Algorithm 1 in shared memory, exponential-Euler gates, synaptic decay, soma
// threshold test), computed in FP32 with the state kept exact between steps
// and every error that would repeat from step to step removed:
//   * V is an int32 fixed-point number (2^-23 mV) and each gate a uint32
//     fixed-point number (2^-32); every step adds an FP32 increment rounded
//     once, so rounding never accumulates in the state itself;
//   * differences of potentials (V - E, V_parent - V_child, V + c in the rate
//     arguments) are taken exactly in integers and carried as float pairs;
//   * the membrane, axial and synaptic currents are summed as float pairs
//     (mm_fp32c_math.h) from constants stored as float pairs (areas, axial
//     conductances, channel densities, weights, the decay factor), and the
//     rhs is rounded to FP32 once;
//   * the Hines diagonal is split into its passive part, eliminated once at
//     set-up in FP64 and stored as a pair, and the step's active membrane
//     and synaptic conductance, which the FP32 elimination carries as a
//     perturbation of it (the passive part alone would lose most of the
//     active conductance's digits to the capacitive and axial terms);
//   * each gate's steady state X(V) and relaxation factor E(V) for the
//     step come from a table of degree-5 polynomials per 0.5 mV interval,
//     built in FP64 for the network's dt, whose two leading terms are float
//     pairs (mm_gate_table.h; within 1e-10 relative);
//   * the soma voltage is also accumulated in FP64 and the spike crossing
//     time is computed in FP64.
#include <cuda_runtime.h>

#include <mutex>
#include <type_traits>

#include "mm_fp32c_math.h"
#include "mm_gate_table.h"
#include "mm_internal.h"
#include "mm_tma.h"

using namespace mmk;

namespace {

__device__ __forceinline__ mmf::F2 f2(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 tof2(mmf::F2 v) { return make_float2(v.hi, v.lo); }
// V - E as a float pair
__device__ __forceinline__ mmf::F2 vminus(int32_t vq, FxPot E) { return mmf::vminus_df(vq, E.q, E.res); }

// ------------------------------------------------------------------ init

__device__ __forceinline__ double xexpm1_d(double x) { return fabs(x) < 1e-6 ? 1.0 - 0.5 * x : x / expm1(x); }

// The resting state: V = v_init and every gate at its steady state there.
__global__ void init_fp32c_kernel(InitArgs a)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.C;
         i += (int64_t)gridDim.x * blockDim.x) {
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
        a.ctl->giant_head = 0u;
        a.ctl->big_head = 0u;
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
    // groups of lanes_per_src lanes take one spike each (a power of two up to
    // the warp: the sources' mean fan-out, so that sparse sources such as
    // synapse points do not leave most of a warp idle)
    const int GL = a.lanes_per_src;
    const int lane = threadIdx.x & (GL - 1);
    const int ngroups = (gridDim.x * blockDim.x) / GL;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) / GL; u < total; u += ngroups) {
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
        // the weight's high word into the site's high word; the rounding
        // error of that addition (exact, by TwoSum from the value the atomic
        // returns: the atomic rounds as the same float addition does) and
        // the weight's low word into the site's low word, so that the pair's
        // sum is every arrived weight to about 44 bits, in any order
        for (long long q = b + lane; q < e; q += GL) {
            float2 *g = a.gsyn2 + a.out_site[q];
            const float2 w = a.out_w2[q];
            const float old = atomicAdd(&g->x, w.x);
            atomicAdd(&g->y, mmf::two_sum(old, w.x).lo + w.y);
        }
    }
}

// Deterministic delivery, FP32c conductances (as deliver_ordered_kernel of
// the FP64 path: each site adds its arrived weights in ascending synapse
// id, one thread per site, as float pairs, plus the per-step resets).
__global__ void __launch_bounds__(256) deliver_ordered_fp32c_kernel(DeliverArgs a)
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
        const float2 g0 = a.gsyn2[st];
        mmf::F2 g = mmf::two_sum(g0.x, g0.y);
        bool hit = false;
        for (long long e = e0; e < e1; ++e) {
            const long long m = n - 1 - a.in_dsteps[e];
            if (m < 0) continue;
            const int src = a.in_src[e];
            if ((a.fired[(m % a.R) * a.fired_words + (src >> 5)] >> (src & 31)) & 1u) {
                g = mmf::add(g, f2(a.in_w2[e]));
                hit = true;
            }
        }
        if (hit) a.gsyn2[st] = tof2(g);
    }
}

// ------------------------------------------------------------ FP32c step

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/x to within rounding: the approximate reciprocal and one Newton step
// (its error is squared).  The Hines factors use it: their diagonals change
// little from step to step, so the approximate reciprocal's error, which
// depends on the operand's bits, would repeat in every step and bias the
// solution the same way each time.
__device__ __forceinline__ float rcp_nr(float x)
{
    const float r = rcp_approx(x);
    return fmaf(r, fmaf(-x, r, 1.f), r);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}


__device__ __forceinline__ mmf::Tab4 ld_tab(const float4 *p)
{
    const float4 v = __ldg(p);
    return {v.x, v.y, v.z, v.w};
}

// Exponential-Euler gate update at V^{n+1} of one compartment (its V is
// final for this step): X and E of each gate from the table interval of V.
__device__ __forceinline__ void gate_update(const StepArgs32 &a, int64_t c)
{
    const mmf::TabIndex t = mmf::tab_index(a.Vq[c]);
    const float4 *f = a.gtab + t.i;
    constexpr int I = mmf::kTabIntervals;
    uint32_t *const q[3] = {a.mq + c, a.hq + c, a.nq + c};
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        const mmf::Tab4 tg[4] = {ld_tab(f + (4 * g) * I), ld_tab(f + (4 * g + 1) * I), ld_tab(f + (4 * g + 2) * I),
                                 ld_tab(f + (4 * g + 3) * I)};
        *q[g] = mmf::tab_gate_step(*q[g], tg, t.u);
    }
}

// Gate updates of the compartments pc0 .. pc0 + pn - 1, in chunks of
// kGateChunk claimed by whole warps from the shared counter *next until none
// is left.
constexpr int kGateChunk = 64;

// Compartments per step of a path sweep (their operands are loaded
// together before the step's dependent chain).
constexpr int kSweepChunk = 4;

// Paths of at least this many compartments are swept by a whole warp
// (chunks per lane combined by warp scans) instead of by one lane.
constexpr int kWarpPath = 96;

__device__ __forceinline__ void gate_chunks(const StepArgs32 &a, int64_t pc0, int pn, int *next, int lane)
{
    for (;;) {
        int ch = 0;
        if (lane == 0) ch = atomicAdd(next, 1);
        ch = __shfl_sync(0xFFFFFFFFu, ch, 0);
        const int i0 = ch * kGateChunk;
        if (i0 >= pn) break;
        const int i1 = min(i0 + kGateChunk, pn);
        for (int i = i0 + lane; i < i1; i += 32) gate_update(a, pc0 + i);
    }
}


// 1024 / NT blocks per SM at most 64 registers a thread: two blocks of 512
// threads (or one of 1024) per SM, whatever the item's shared memory allows
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) step_fp32c_kernel(StepArgs32 a)
{
    // Shared memory of one work item, carved from the item's own sizes: its
    // tree blob (staged by one bulk copy), then per compartment the pair
    // (active conductance, rhs) -- after elimination the substitution
    // coefficients (f, c), after substitution (f, dV) --, the implicit axial
    // coupling to the parent and the passive eliminated diagonal (float
    // pairs, staged so that the sweeps touch only shared memory; until the
    // rhs is final the diagonal's place holds the rhs's low words); then per
    // path two words: the current
    // across its head link (a pair), later its contribution to its parent
    // compartment (active conductance, rhs) -- for the path from a soma the
    // FP64 soma voltage.  The launch provides the largest need over its
    // items.
    //
    // Warp roles: all warps run the streaming phases (A, S, C) of an item.
    // In the sweeps teams of 1, 2 or 4 warps take whole sweep bundles of the
    // item (a neuron, or several small ones), one lane per path, and
    // synchronise only among themselves; warps without a bundle, and each
    // team once its bundles are done, update the gates of the block's
    // previous item (its V^{n+1} is final since that item's phase C) in
    // chunks claimed from a shared counter, so that the arithmetic of the
    // gates fills the issue slots the latency-bound sweeps leave.
    constexpr int NS = NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smeta = smem_raw;
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_item, s_next, s_abort;  // this item, the item claimed after it
    __shared__ long long s_pc0;  // pending gate work: the previous item's compartments
    __shared__ int s_pn, s_gchunk;

    const long long n = (long long)a.ctl->step_base + a.step_offset;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        s_abort = 0;
        s_pc0 = 0;
        s_pn = 0;
        s_gchunk = 0;
        s_next = a.item0 + (int)atomicAdd(a.queue, 1u);
    }
    uint32_t parity = 0;

    for (;;) {
        __syncthreads();
        if (s_abort) break;
        if (tid == 0) {
            // items are claimed one ahead, so that the next item's
            // compartments can be pulled into L2 during this item's sweeps
            const int item = s_next;
            s_item = item;
            if (item < a.item1) {
                s_next = a.item0 + (int)atomicAdd(a.queue, 1u);
                const GroupRec *gp = a.groups + item;
                const uint32_t bytes = (uint32_t)gp->meta_bytes;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bar, bytes);
                bulk_copy_g2s(smeta, a.meta + gp->meta_off, bytes, &bar);
            }
        }
        __syncthreads();
        const int gi = s_item;
        if (gi >= a.item1) break;
        const unsigned long long t_item = (a.item_ns && tid == 0) ? global_ns() : 0ull;
        const GroupRec G = a.groups[gi];
        const int64_t c0 = G.comp0;
        const int32_t *Vq = a.Vq + c0;
        float2 *sdr = (float2 *)(smem_raw + G.meta_bytes);  // (e, rhs), then (f, c), then (f, dV)
        float *sy = (float *)sdr;                            // sy[2 i + 1]: the second member of sdr[i]
        float2 *sgp = sdr + G.ncomp;                         // implicit coupling to the parent (pair)
        float2 *sdp = sgp + G.ncomp;                         // passive eliminated diagonal (pair), staged
                                                             // once phase S is done
        float *srl = (float *)sdp;                           // until then: the low word of each rhs
        float *scd = (float *)(sdp + G.ncomp);
        float *scr = scd + G.npath;

        // A. membrane conductance and current at (V^n, gates^n), plus the
        //    axial currents of every link inside a path (both ends; a link
        //    (i-1, i) is inside a path when g_axial[i] has no sign bit), the
        //    rhs summed as a float pair; the active conductance (FP32) is the
        //    diagonal's share that changes from step to step.  Stage the
        //    couplings and the passive diagonal for the sweeps.  All reads
        //    go through the read-only path (nothing here is written by this
        //    launch before it is read), so that the loads of two iterations
        //    overlap.
#pragma unroll 2
        for (int i = tid; i < G.ncomp; i += NS) {
            const int32_t vq = __ldg(Vq + i);
            const float2 gs = __ldg(a.gax + c0 + i);
            const float gh = fabsf(gs.x);
            sgp[i] = make_float2(a.gimp * gh, a.gimp * gs.y);
            const mmf::F2 ar = f2(__ldg(a.area + c0 + i));
            const mmf::F2 m = mmf::gate_df(__ldg(a.mq + c0 + i)), h = mmf::gate_df(__ldg(a.hq + c0 + i)),
                          nn = mmf::gate_df(__ldg(a.nq + c0 + i));
            // conductances and current per unit area, then times the area
            const mmf::F2 gna = mmf::mul(f2(a.gNa), mmf::mul(mmf::mul(mmf::mul(m, m), m), h));
            const mmf::F2 n2 = mmf::mul(nn, nn);
            const mmf::F2 gk = mmf::mul(f2(a.gK), mmf::mul(n2, n2));
            const mmf::F2 iu = mmf::add(mmf::mul(gna, vminus(vq, a.ENa)),
                                        mmf::add(mmf::mul(gk, vminus(vq, a.EK)), mmf::mul(f2(a.gL), vminus(vq, a.EL))));
            mmf::F2 r = mmf::neg(mmf::mul(ar, iu));
            if (!signbit(gs.x))  // link to the parent i-1
                r = mmf::add(r, mmf::mul(mmf::F2{gh, gs.y}, mmf::vdiff_df(__ldg(Vq + i - 1), vq)));
            if (i + 1 < G.ncomp) {
                const float2 gc = __ldg(a.gax + c0 + i + 1);
                if (!signbit(gc.x))  // link to the child i+1
                    r = mmf::add(r, mmf::mul(f2(gc), mmf::vdiff_df(__ldg(Vq + i + 1), vq)));
            }
            // the active part: the membrane conductance (implicit except in
            // Eq. 2 as printed) and the constant share that stands for the
            // passive diagonal's low word
            const float eps = __ldg(&a.dp[c0 + i].y);
            sdr[i] = make_float2((a.g_implicit ? ar.hi * (gna.hi + gk.hi) : 0.f) + eps, r.hi);
            srl[i] = r.lo;
        }
        // the tree blob must have landed before the per-path work
        if (!mbar_wait_bounded(&bar, parity)) {
            // give up on this item, but not on the copy in flight: wait for
            // it once more (bounded) so that the block never leaves while
            // the copy could still write into its shared memory
            s_abort = 1;
            mbar_wait_bounded(&bar, parity);
        }
        parity ^= 1u;
        __syncthreads();
        if (s_abort) {  // the whole block leaves at the next item boundary
            if (tid == 0) atomicOr(&a.ctl->err, MMK_ERR_TIMEOUT);
            continue;
        }
        const NrnQ *nrns = (const NrnQ *)smeta;
        const PathQ *paths = (const PathQ *)(smeta + G.path_off);
        const KidQ *fold = (const KidQ *)(smeta + G.fold_off);
        const int16_t *loffs = (const int16_t *)(smeta + G.loffs_off);
        const int16_t *mcnt = (const int16_t *)(smeta + G.mcnt_off);

        // S. synaptic sites (their conductance and current, then the
        //    conductance's decay; sites are distinct compartments), then per
        //    path the current across its head link into its head (for the
        //    path from a soma: the stimulus; that path also fetches the FP64
        //    soma voltage into its slots, as two 32-bit halves), then the
        //    same currents out of the parent compartments, summed per parent
        //    in fold-list order.  Each rhs stays a float pair until then.
        for (int t = tid; t < G.nsite; t += NS) {
            const int st = G.site0 + t;
            const int c = a.site_comp[st];
            const float2 g0 = a.gsyn[st];
            const mmf::F2 g = mmf::two_sum(g0.x, g0.y);
            float2 v = sdr[c];
            if (a.g_implicit) v.x += g.hi;
            const mmf::F2 r = mmf::add(mmf::F2{v.y, srl[c]}, mmf::neg(mmf::mul(g, vminus(Vq[c], a.Esyn))));
            v.y = r.hi;
            sdr[c] = v;
            srl[c] = r.lo;
            a.gsyn[st] = tof2(mmf::mul(g, f2(a.decay)));
        }
        __syncthreads();
        for (int pi = tid; pi < G.npath; pi += NS) {
            const PathQ P = paths[pi];
            mmf::F2 t;
            if (P.parent >= 0) {
                const float2 gs = __ldg(a.gax + c0 + P.head);
                t = mmf::mul(mmf::F2{fabsf(gs.x), gs.y}, mmf::vdiff_df(Vq[P.parent], Vq[P.head]));
                scd[pi] = t.hi;
                scr[pi] = t.lo;
            } else {
                const int nrn = G.neuron0 + (P.nflag & kPathNeuron);
                t = mmf::split_d(a.stim[nrn]);
                const double v0 = a.Vsoma[nrn];
                scd[pi] = __int_as_float(__double2hiint(v0));
                scr[pi] = __int_as_float(__double2loint(v0));
            }
            const mmf::F2 r = mmf::add(mmf::F2{sdr[P.head].y, srl[P.head]}, t);
            sdr[P.head].y = r.hi;
            srl[P.head] = r.lo;
        }
        __syncthreads();
        for (int e = tid; e < G.npath; e += NS) {
            const int att = (int)(fold[e] >> 16);
            if (att >= G.ncomp) continue;  // a path from a soma (no parent)
            if (e > 0 && (int)(fold[e - 1] >> 16) == att) continue;  // not the first path of its parent
            mmf::F2 t{0.f, 0.f};
            for (int z = e; z < G.npath && (int)(fold[z] >> 16) == att; ++z) {
                const int c = (int)(fold[z] & 0xFFFFu);
                t = mmf::add(t, mmf::F2{scd[c], scr[c]});
            }
            const mmf::F2 r = mmf::add(mmf::F2{sdr[att].y, srl[att]}, mmf::neg(t));
            sdr[att].y = r.hi;
            srl[att] = r.lo;
        }
        __syncthreads();
        // every rhs is now final (its high word the nearest float): the
        // passive diagonal and the factor g^2 / d0' of the active part's
        // recurrence (taken as (g / d0') g) take the place of the low words
        for (int i = tid; i < G.ncomp; i += NS) {
            const float dh = __ldg(&a.dp[c0 + i].x);
            sdp[i] = make_float2(dh, (sgp[i].x * rcp_nr(dh)) * sgp[i].x);
        }
        __syncthreads();

        // The next item's per-compartment streams (V, gates, constants) into
        // L2, one 128-byte line per prefetch, while the sweeps run.
        {
            const int ni = s_next;
            if (ni < a.item1) {
                const int64_t nc0 = a.groups[ni].comp0, ncn = a.groups[ni].ncomp;
                auto pull = [&](const void *p, int64_t esz) {
                    const int64_t b0 = nc0 * esz, b1 = b0 + ncn * esz;
                    const int64_t l0 = b0 >> 7, nl = ((b1 + 127) >> 7) - l0;
                    for (int64_t x = tid; x < nl; x += NS)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"((const char *)p + max((l0 + x) << 7, b0)));
                };
                pull(a.Vq, 4);
                pull(a.mq, 4);
                pull(a.hq, 4);
                pull(a.nq, 4);
                pull(a.area, 8);
                pull(a.gax, 8);
                pull(a.dp, 8);
            }
        }

        // Team of each warp for the sweeps: T warps per sweep bundle (T = 1,
        // 2 or 4, as many as the item's bundles leave), the teams taking the
        // item's bundles in turn; a team synchronises on its own named
        // barrier (1 + team; 0 is the block's).
        const int nwarp = NS / 32;
        int T = nwarp / max(G.nbundle, 1);
        T = T >= 4 ? 4 : (T >= 2 ? 2 : 1);
        if (T == 2 && nwarp / 2 > 15) T = 4;
        const int team = (tid >> 5) / T, nteam = nwarp / T;
        const int tl = tid - team * T * 32;  // lane within the team
        const int TL = T * 32;
        auto team_sync = [&]() {
            if (T == 1) __syncwarp();
            else asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(TL) : "memory");
        };

        // B. leaves-to-root elimination (Algorithm 1) path by path, from the
        //    deepest level up: every compartment of a path has the one
        //    before it as its parent, so a path is one chain from its leaf
        //    up to its head (links inside a path are assembled: a = c = -g).
        //    The diagonal of compartment j after the elimination of its
        //    subtree is d'_j = d0'_j + e_j, with d0'_j the passive one
        //    (eliminated at set-up) and e_j the active conductance carried
        //    up the tree: e_{p} += (g^2/d0'_j) (1/d'_j) e_j, the exact
        //    difference of the two eliminations (g^2/d0'_j staged per
        //    compartment, so that the dependent chain is an add, the
        //    approximate reciprocal, a multiply and an FMA).  kSweepChunk compartments
        //    at a time with their operands loaded before any of their stores
        //    (indices past the head are clamped and their results dropped).
        //    The head is then eliminated into its parent compartment: a path
        //    alone on that compartment adds its contribution there itself;
        //    paths sharing one leave theirs in their slots, summed in
        //    fold-list order once the level is done.  The elimination leaves
        //    the substitution coefficients x_j = f_j x_{j-1} + c_j.
        // the head of path pi once its interior is eliminated (eh, rh: the
        // head's active conductance and rhs): for the path from a soma its
        // dV, else the head eliminated into the parent
        auto eliminate_head = [&](int pi, const PathQ &P, float eh, float rh) {
            const int h = P.head;
            const float2 dq = sdp[h];
            const float inv = rcp_nr(dq.x + eh);
            if (P.parent < 0) {  // soma: its dV
                sy[2 * h + 1] = rh * inv;
                return;
            }
            const float2 gq = sgp[h];
            const float f = fmaf(gq.x, inv, gq.y * inv);
            sdr[h] = make_float2(f, rh * inv);
            const float ce = gq.x * rcp_nr(dq.x) * f * eh, cr = f * rh;
            if (P.nflag & kPathAlone) {
                float2 v = sdr[P.parent];
                v.x += ce;
                v.y += cr;
                sdr[P.parent] = v;
            } else {
                scd[pi] = ce;
                scr[pi] = cr;
            }
        };
        auto eliminate_path = [&](int pi) {
            const PathQ P = paths[pi];
            const int h = P.head;
            int j = P.end - 1;
            const float2 v0 = sdr[j];
            float eb = v0.x, rb = v0.y;
            float eh = eb, rh = rb;
            for (; j > h; j -= kSweepChunk) {
                const int cnt = j - h;
                float gh[kSweepChunk], gl[kSweepChunk], dh[kSweepChunk], fg[kSweepChunk];
                float ep[kSweepChunk], rp[kSweepChunk];
#pragma unroll
                for (int k = 0; k < kSweepChunk; ++k) {
                    const int q = max(j - k, h + 1);
                    const float2 gq = sgp[q], dq = sdp[q], w = sdr[q - 1];
                    gh[k] = gq.x;
                    gl[k] = gq.y;
                    dh[k] = dq.x;
                    fg[k] = dq.y;
                    ep[k] = w.x;
                    rp[k] = w.y;
                }
#pragma unroll
                for (int k = 0; k < kSweepChunk; ++k) {
                    // the active conductance's recurrence (the dependent
                    // chain) takes the approximate reciprocal; the factors
                    // that the rhs and the substitution use take it refined
                    const float dd = dh[k] + eb;
                    const float r0 = rcp_approx(dd);
                    const float inv = fmaf(r0, fmaf(-dd, r0, 1.f), r0);
                    const float f = fmaf(gh[k], inv, gl[k] * inv);
                    const float c = rb * inv;
                    if (k < cnt) sdr[j - k] = make_float2(f, c);
                    rb = fmaf(f, rb, rp[k]);
                    eb = fmaf(fg[k] * r0, eb, ep[k]);
                    if (k == cnt - 1) {
                        eh = eb;
                        rh = rb;
                    }
                }
            }
            eliminate_head(pi, P, eh, rh);
        };
        // contributions of the level's paths that share a parent compartment
        // (fold entries e0 .. e1-1); a lane takes the entries that start a run
        // of equal parents
        auto fold_shared = [&](int e0, int e1) {
            for (int e = e0 + tl; e < e1; e += TL) {
                const KidQ kv = fold[e];
                const int att = (int)(kv >> 16);
                if (e > e0 && (int)(fold[e - 1] >> 16) == att) continue;
                int c = (int)(kv & 0xFFFFu);
                float ad = scd[c], ar = scr[c];
                for (int z = e + 1; z < e1; ++z) {
                    const KidQ kz = fold[z];
                    if ((int)(kz >> 16) != att) break;
                    c = (int)(kz & 0xFFFFu);
                    ad += scd[c];
                    ar += scr[c];
                }
                float2 v = sdr[att];
                v.x += ad;
                v.y += ar;
                sdr[att] = v;
            }
        };

        // F. root-to-leaves substitution path by path, one level at a time
        //    (a path's head needs its parent, on a path of the level
        //    before); the path from a soma runs the FP64 soma accumulator and
        //    the spike test
        // dV of the head of path pi: from its parent's, or for the path from
        // a soma its own, which also advances the FP64 soma accumulator and
        // runs the spike test
        auto substitute_head = [&](int pi, const PathQ &P) -> float {
            const int h = P.head;
            float x;
            const float2 vh = sdr[h];
            if (P.parent >= 0) {
                x = fmaf(vh.x, sy[2 * P.parent + 1], vh.y);
            } else {
                x = vh.y;
                const int nrn = G.neuron0 + (P.nflag & kPathNeuron);
                const double v0 = __hiloint2double(__float_as_int(scd[pi]), __float_as_int(scr[pi]));
                const double v1 = v0 + (double)x;
                a.Vsoma[nrn] = v1;
                if (!isfinite(v1)) atomicOr(&a.ctl->err, MMK_ERR_NUMERIC);
                if (v0 < a.threshold && v1 >= a.threshold) {
                    const int src = soma_source(a, nrn);
                    if (src >= 0)
                        record_spike(a, src, a.user_id[nrn], 0,
                                     (double)n * a.dt64 + a.dt64 * (a.threshold - v0) / (v1 - v0), n);
                }
            }
            return x;
        };
        auto substitute_path = [&](int pi) {
            const PathQ P = paths[pi];
            const int h = P.head;
            float x = substitute_head(pi, P);
            const float xh = x;
            // down the path, each compartment's parent is the one before
            // it: x_j = f_j x_{j-1} + c_j with the coefficients the
            // elimination left in sdr; kSweepChunk at a time, operands
            // loaded before the stores (indices past the leaf clamped, their
            // results dropped)
            for (int j = h + 1; j < P.end; j += kSweepChunk) {
                const int cnt = P.end - j;
                float r[kSweepChunk], d[kSweepChunk];
#pragma unroll
                for (int k = 0; k < kSweepChunk; ++k) {
                    const float2 w = sdr[min(j + k, P.end - 1)];
                    d[k] = w.x;
                    r[k] = w.y;
                }
#pragma unroll
                for (int k = 0; k < kSweepChunk; ++k) {
                    x = fmaf(d[k], x, r[k]);
                    if (k < cnt) sy[2 * (j + k) + 1] = x;
                }
            }
            if (P.parent >= 0) sy[2 * h + 1] = xh;  // read by the next level only
        };

        // Paths of at least kWarpPath compartments are eliminated and
        // substituted by a whole warp.  The path's interior is cut into 32
        // chunks, one per lane.  The recurrence of the active conductance,
        // e_{j-1} = E_{j-1} + (g_j / D_j) g_j e_j / (D_j + e_j) (E the
        // compartment's own share, D the passive diagonal), is the action of
        // the 2x2 matrix [[E_{j-1} + g_j^2 / D_j, E_{j-1} D_j], [1, D_j]] on
        // (e_j, 1) up to scale (all entries positive: no cancellation), and
        // the rhs recurrence r'_{j-1} = r_{j-1} + f_j r'_j and the
        // substitution x_j = f_j x_{j-1} + c_j are affine maps: each lane
        // composes its chunk, an inclusive warp scan combines the chunks,
        // and each lane runs the recurrences through its chunk from the
        // values the chunks before it leave (the same operations as the
        // serial sweep, started from scanned values).
        const int lane = tid & 31;
        auto eliminate_path_warp = [&](int pi) {
            const PathQ P = paths[pi];
            const int h = P.head, e = P.end;
            const int m = e - 1 - h;  // interior elements, t = 0 .. m-1 <-> j = e-1-t
            const int cs = (m + 31) >> 5;
            const int t0 = min(lane * cs, m), t1 = min(t0 + cs, m);
            const float2 leaf = sdr[e - 1];
            // the chunk's matrix product, rescaled as it goes (only ratios matter)
            float m00 = 1.f, m01 = 0.f, m10 = 0.f, m11 = 1.f;
            for (int tt = t0; tt < t1; ++tt) {
                const int j = e - 1 - tt;
                const float2 gq = sgp[j], dq = sdp[j];
                const float D = dq.x, En = sdr[j - 1].x;
                const float A = dq.y + En, B = En * D;
                const float n00 = fmaf(A, m00, B * m10), n01 = fmaf(A, m01, B * m11);
                const float n10 = fmaf(D, m10, m00), n11 = fmaf(D, m11, m01);
                const float s = rcp_approx(n00 + n01 + n10 + n11);
                m00 = n00 * s;
                m01 = n01 * s;
                m10 = n10 * s;
                m11 = n11 * s;
            }
            for (int off = 1; off < 32; off <<= 1) {
                const float a00 = __shfl_up_sync(0xFFFFFFFFu, m00, off), a01 = __shfl_up_sync(0xFFFFFFFFu, m01, off);
                const float a10 = __shfl_up_sync(0xFFFFFFFFu, m10, off), a11 = __shfl_up_sync(0xFFFFFFFFu, m11, off);
                if (lane >= off) {  // this lane's chunks act after the earlier ones
                    const float n00 = fmaf(m00, a00, m01 * a10), n01 = fmaf(m00, a01, m01 * a11);
                    const float n10 = fmaf(m10, a00, m11 * a10), n11 = fmaf(m10, a01, m11 * a11);
                    const float s = rcp_approx(fabsf(n00) + fabsf(n01) + fabsf(n10) + fabsf(n11));
                    m00 = n00 * s;
                    m01 = n01 * s;
                    m10 = n10 * s;
                    m11 = n11 * s;
                }
            }
            float e00 = __shfl_up_sync(0xFFFFFFFFu, m00, 1), e01 = __shfl_up_sync(0xFFFFFFFFu, m01, 1);
            float e10 = __shfl_up_sync(0xFFFFFFFFu, m10, 1), e11 = __shfl_up_sync(0xFFFFFFFFu, m11, 1);
            if (lane == 0) {
                e00 = 1.f;
                e01 = 0.f;
                e10 = 0.f;
                e11 = 1.f;
            }
            const float eb0 = fmaf(e00, leaf.x, e01) / fmaf(e10, leaf.x, e11);
            // pass 1 (reads only): the active conductance through the chunk
            // and the chunk's affine map of the rhs recurrence; the element
            // after the chunk is kept for pass 2, whose writes it may see
            float eb = eb0, A = 1.f, B = 0.f;
            float2 nb = make_float2(0.f, 0.f);
            for (int tt = t0; tt < t1; ++tt) {
                const int j = e - 1 - tt;
                const float2 gq = sgp[j], dq = sdp[j], w = sdr[j - 1];
                const float dd = dq.x + eb;
                const float r0 = rcp_approx(dd);
                const float inv = fmaf(r0, fmaf(-dd, r0, 1.f), r0);
                const float f = fmaf(gq.x, inv, gq.y * inv);
                A *= f;
                B = fmaf(f, B, w.y);
                eb = fmaf(dq.y * r0, eb, w.x);
                nb = w;
            }
            for (int off = 1; off < 32; off <<= 1) {
                const float pa = __shfl_up_sync(0xFFFFFFFFu, A, off), pb = __shfl_up_sync(0xFFFFFFFFu, B, off);
                if (lane >= off) {
                    B = fmaf(A, pb, B);
                    A *= pa;
                }
            }
            float ea = __shfl_up_sync(0xFFFFFFFFu, A, 1), ebs = __shfl_up_sync(0xFFFFFFFFu, B, 1);
            if (lane == 0) {
                ea = 1.f;
                ebs = 0.f;
            }
            // pass 2: the substitution coefficients (f_j, c_j) of the chunk
            __syncwarp();
            eb = eb0;
            float rb = fmaf(ea, leaf.y, ebs);
            for (int tt = t0; tt < t1; ++tt) {
                const int j = e - 1 - tt;
                const float2 gq = sgp[j], dq = sdp[j];
                const float2 w = tt + 1 < t1 ? sdr[j - 1] : nb;
                const float dd = dq.x + eb;
                const float r0 = rcp_approx(dd);
                const float inv = fmaf(r0, fmaf(-dd, r0, 1.f), r0);
                const float f = fmaf(gq.x, inv, gq.y * inv);
                sdr[j] = make_float2(f, rb * inv);
                rb = fmaf(f, rb, w.y);
                eb = fmaf(dq.y * r0, eb, w.x);
            }
            // the head, from the lane whose chunk ends at it
            const int lastl = (m - 1) / cs;
            const float eh = __shfl_sync(0xFFFFFFFFu, eb, lastl), rh = __shfl_sync(0xFFFFFFFFu, rb, lastl);
            __syncwarp();
            if (lane == 0) eliminate_head(pi, P, eh, rh);
            __syncwarp();
        };
        auto substitute_path_warp = [&](int pi) {
            const PathQ P = paths[pi];
            const int h = P.head, e = P.end;
            float x = 0.f;
            if (lane == 0) x = substitute_head(pi, P);
            x = __shfl_sync(0xFFFFFFFFu, x, 0);
            const int m = e - 1 - h;  // t = 0 .. m-1 <-> j = h+1+t
            const int cs = (m + 31) >> 5;
            const int t0 = min(lane * cs, m), t1 = min(t0 + cs, m);
            float A = 1.f, B = 0.f;
            for (int tt = t0; tt < t1; ++tt) {
                const float2 w = sdr[h + 1 + tt];
                A *= w.x;
                B = fmaf(w.x, B, w.y);
            }
            for (int off = 1; off < 32; off <<= 1) {
                const float pa = __shfl_up_sync(0xFFFFFFFFu, A, off), pb = __shfl_up_sync(0xFFFFFFFFu, B, off);
                if (lane >= off) {
                    B = fmaf(A, pb, B);
                    A *= pa;
                }
            }
            float ea = __shfl_up_sync(0xFFFFFFFFu, A, 1), eb = __shfl_up_sync(0xFFFFFFFFu, B, 1);
            if (lane == 0) {
                ea = 1.f;
                eb = 0.f;
            }
            float xs = fmaf(ea, x, eb);
            for (int tt = t0; tt < t1; ++tt) {
                const int j = h + 1 + tt;
                const float2 w = sdr[j];
                xs = fmaf(w.x, xs, w.y);
                sy[2 * j + 1] = xs;
            }
            __syncwarp();
            if (lane == 0 && P.parent >= 0) sy[2 * h + 1] = x;  // read by the next level only
        };
        // the number of paths at the start of a level (paths run longest
        // first) that a whole warp takes
        auto warp_paths = [&](int pb, int pe) {
            int nw = 0;
            while (pb + nw < pe && paths[pb + nw].end - paths[pb + nw].head >= kWarpPath) ++nw;
            return nw;
        };

        // B from the deepest level up, then F from the soma down; a level's
        // paths go to the team's lanes longest first.  Then gate chunks of
        // the previous item (when timing items, the gates wait until after
        // phase C, outside the timed span).
        for (int k = team; k < G.nbundle; k += nteam) {
            const NrnQ Nk = nrns[k];
            const int16_t *lo = loffs + Nk.loff0;
            const int16_t *mc = mcnt + Nk.loff0;
            for (int l = Nk.nlevel - 1; l >= 0; --l) {
                const int pb = lo[l], pe = lo[l + 1];
                const int nw = warp_paths(pb, pe);
                for (int q = tl >> 5; q < nw; q += T) eliminate_path_warp(pb + q);
                for (int pi = pb + nw + tl; pi < pe; pi += TL) eliminate_path(pi);
                team_sync();
                if (mc[l] > 0) {
                    fold_shared(pb, pb + mc[l]);
                    team_sync();
                }
            }
            for (int l = 0; l < Nk.nlevel; ++l) {
                const int pb = lo[l], pe = lo[l + 1];
                const int nw = warp_paths(pb, pe);
                for (int q = tl >> 5; q < nw; q += T) substitute_path_warp(pb + q);
                for (int pi = pb + nw + tl; pi < pe; pi += TL) substitute_path(pi);
                team_sync();
            }
        }
        if (!a.item_ns) gate_chunks(a, s_pc0, s_pn, &s_gchunk, tid & 31);
        __syncthreads();

        // C. V^{n+1} = V^n + dV (exact in fixed point), and the threshold
        //    test of the detection points other than somata
        //    (two copies of the loop, chosen by the uniform detection mode,
        //    so that soma detection runs the loop without the test)
        auto phase_c = [&](auto points) {
            for (int i = tid; i < G.ncomp; i += NS) {
                const int32_t vold = Vq[i];
                int32_t vq;
                if (!mmf::v_add(vold, sy[2 * i + 1], &vq)) {
                    atomicOr(&a.ctl->err, MMK_ERR_NUMERIC);
                    vq = vold;
                }
                a.Vq[c0 + i] = vq;
                if constexpr (decltype(points)::value) {
                    if (vold < a.thr_q && vq >= a.thr_q) {
                        const int p = a.pt_of[c0 + i];
                        if (p >= 0) point_spike(a, p, (double)vold * kVInvD, (double)vq * kVInvD, n, a.dt64);
                    }
                }
            }
        };
        if (a.pt_of) phase_c(std::true_type{});
        else phase_c(std::false_type{});
        if (a.item_ns) {  // uniform across the block
            __syncthreads();
            if (tid == 0) a.item_ns[gi] += global_ns() - t_item;
            gate_chunks(a, s_pc0, s_pn, &s_gchunk, tid & 31);
            __syncthreads();
        }
        // this item's gates are pending until the next item's sweeps (its
        // V^{n+1} is visible to the block after the barrier at the top of
        // the loop; every chunk of the previous item is done)
        if (tid == 0) {
            s_pc0 = c0;
            s_pn = G.ncomp;
            s_gchunk = 0;
        }
    }
    // the last item's gates, by the whole block
    gate_chunks(a, s_pc0, s_pn, &s_gchunk, tid & 31);
}


template <int NT>
__global__ void __launch_bounds__(NT) giant_fp32c_kernel(StepArgs32 a)
{
    // Work items too large for shared memory (giant neurons, up to the
    // int32 index range): the same path-by-path solve as step_fp32c_kernel
    // with the whole block as one team, between giant_assemble_kernel
    // (phase A of every giant compartment, spread over many blocks) and
    // giant_update_kernel (phase C and the gates, likewise).  The active
    // conductance and rhs of each compartment (after elimination f and c,
    // after substitution dV) live in a global float2 scratch, the rhs's low
    // word in a float scratch and the per-path slots in a global float4
    // scratch, so they stay in L2.  The tables are read from the item's
    // blob in global memory (32-bit records); each lane loads the next eight
    // compartments of its path while it eliminates (or substitutes) the
    // current eight.
    __shared__ int s_item;

    const long long n = (long long)a.ctl->step_base + a.step_offset;
    const int tid = threadIdx.x;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = a.item0 + (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int gi = s_item;
        if (gi >= a.item1) break;
        const unsigned long long t_item = (a.item_ns && tid == 0) ? global_ns() : 0ull;
        const GroupRec G = a.groups[gi];
        const int64_t c0 = G.comp0;
        const int32_t *Vq = a.Vq + c0;
        const float2 *gax = a.gax + c0;
        const float2 *dpp = a.dp + c0;
        float2 *dr = a.dr + G.scratch0;
        float *drl = a.drl + G.scratch0;
        float4 *pq = a.pq + G.pscratch0;
        const unsigned char *blob = a.meta + G.meta_off;
        const NrnG *nrns = (const NrnG *)blob;
        const PathG *paths = (const PathG *)(blob + G.path_off);
        const KidG *fold = (const KidG *)(blob + G.fold_off);
        const int32_t *loffs = (const int32_t *)(blob + G.loffs_off);
        const int32_t *mcnt = (const int32_t *)(blob + G.mcnt_off);

        // S. synaptic sites (then their decay; sites are distinct
        //    compartments), the current across each path's head link into
        //    its head (for the path from a soma: the stimulus), then out of
        //    the parent compartments, summed per parent in fold-list order
        //    (as in step_fp32c_kernel)
        for (int t = tid; t < G.nsite; t += NT) {
            const int st = G.site0 + t;
            const int c = a.site_comp[st];
            const float2 g0 = a.gsyn[st];
            const mmf::F2 g = mmf::two_sum(g0.x, g0.y);
            float2 v = dr[c];
            if (a.g_implicit) v.x += g.hi;
            const mmf::F2 r = mmf::add(mmf::F2{v.y, drl[c]}, mmf::neg(mmf::mul(g, vminus(Vq[c], a.Esyn))));
            v.y = r.hi;
            dr[c] = v;
            drl[c] = r.lo;
            a.gsyn[st] = tof2(mmf::mul(g, f2(a.decay)));
        }
        __syncthreads();
        for (int pi = tid; pi < G.npath; pi += NT) {
            const PathG P = paths[pi];
            mmf::F2 t;
            if (P.parent >= 0) {
                const float2 gs = gax[P.head];
                t = mmf::mul(mmf::F2{fabsf(gs.x), gs.y}, mmf::vdiff_df(Vq[P.parent], Vq[P.head]));
                pq[pi].z = t.hi;
                pq[pi].w = t.lo;
            } else {
                t = mmf::split_d(a.stim[G.neuron0 + (P.nflag & kPathNeuronG)]);
            }
            const mmf::F2 r = mmf::add(mmf::F2{dr[P.head].y, drl[P.head]}, t);
            dr[P.head].y = r.hi;
            drl[P.head] = r.lo;
        }
        __syncthreads();
        for (int e = tid; e < G.npath; e += NT) {
            const int att = fold[e].y;
            if (att < 0) continue;  // a path from a soma (no parent)
            if (e > 0 && fold[e - 1].y == att) continue;  // not the first path of its parent
            mmf::F2 t{0.f, 0.f};
            for (int z = e; z < G.npath && fold[z].y == att; ++z) {
                const float4 q = pq[fold[z].x];
                t = mmf::add(t, mmf::F2{q.z, q.w});
            }
            const mmf::F2 r = mmf::add(mmf::F2{dr[att].y, drl[att]}, mmf::neg(t));
            dr[att].y = r.hi;
            drl[att] = r.lo;
        }
        __syncthreads();

        // B. leaves-to-root elimination path by path, from the deepest level
        //    up (as in step_fp32c_kernel: passive diagonal plus the active
        //    conductance carried up the tree)
        auto eliminate_path = [&](int pi) {
            const PathG P = paths[pi];
            const int h = P.head;
            int j = P.end - 1;
            const float2 v0 = dr[j];
            float eb = v0.x, rb = v0.y, eh = eb, rh = rb;
            float g0[8], l0[8], d0[8], q0[8], e0[8], r0[8];
            float g1[8], l1[8], d1[8], q1[8], e1[8], r1[8];
            auto load = [&](int jj, float *g, float *l, float *d, float *q, float *ee, float *r) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int x = max(jj - k, h + 1);
                    const float2 gs = gax[x], w = dr[x - 1];
                    g[k] = a.gimp * fabsf(gs.x);
                    l[k] = a.gimp * gs.y;
                    d[k] = dpp[x].x;
                    q[k] = (g[k] * rcp_nr(d[k])) * g[k];
                    ee[k] = w.x;
                    r[k] = w.y;
                }
            };
            auto chain = [&](int jj, const float *g, const float *l, const float *d, const float *q,
                             const float *ee, const float *r) {
                const int cnt = jj - h;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float dd = d[k] + eb;
                    const float r0 = rcp_approx(dd);
                    const float inv = fmaf(r0, fmaf(-dd, r0, 1.f), r0);
                    const float f = fmaf(g[k], inv, l[k] * inv);
                    if (k < cnt) dr[jj - k] = make_float2(f, rb * inv);
                    rb = fmaf(f, rb, r[k]);
                    eb = fmaf(q[k] * r0, eb, ee[k]);
                    if (k == cnt - 1) {
                        eh = eb;
                        rh = rb;
                    }
                }
            };
            if (j > h) {
                load(j, g0, l0, d0, q0, e0, r0);
                for (;;) {
                    int jn = j - 8;
                    bool more = jn > h;
                    if (more) load(jn, g1, l1, d1, q1, e1, r1);
                    chain(j, g0, l0, d0, q0, e0, r0);
                    j = jn;
                    if (!more) break;
                    jn = j - 8;
                    more = jn > h;
                    if (more) load(jn, g0, l0, d0, q0, e0, r0);
                    chain(j, g1, l1, d1, q1, e1, r1);
                    j = jn;
                    if (!more) break;
                }
            }
            const float dhh = dpp[h].x;
            const float inv = rcp_nr(dhh + eh);
            if (P.parent < 0) {  // soma: its dV
                dr[h].y = rh * inv;
                return;
            }
            const float2 gs = gax[h];
            const float gh = a.gimp * fabsf(gs.x), gl = a.gimp * gs.y;
            const float f = fmaf(gh, inv, gl * inv);
            dr[h] = make_float2(f, rh * inv);
            const float ce = gh * rcp_nr(dhh) * f * eh, cr = f * rh;
            if (P.nflag & kPathAloneG) {
                float2 v = dr[P.parent];
                v.x += ce;
                v.y += cr;
                dr[P.parent] = v;
            } else {
                pq[pi].x = ce;
                pq[pi].y = cr;
            }
        };
        auto fold_shared = [&](int e0, int e1) {
            for (int e = e0 + tid; e < e1; e += NT) {
                const KidG kv = fold[e];
                if (e > e0 && fold[e - 1].y == kv.y) continue;
                float ad = pq[kv.x].x, ar = pq[kv.x].y;
                for (int z = e + 1; z < e1; ++z) {
                    const KidG kz = fold[z];
                    if (kz.y != kv.y) break;
                    ad += pq[kz.x].x;
                    ar += pq[kz.x].y;
                }
                float2 v = dr[kv.y];
                v.x += ad;
                v.y += ar;
                dr[kv.y] = v;
            }
        };
        // F. root-to-leaves substitution path by path; the path from a soma
        //    runs the FP64 soma accumulator and the spike test
        auto substitute_path = [&](int pi) {
            const PathG P = paths[pi];
            const int h = P.head;
            float x;
            if (P.parent >= 0) {
                const float2 fh = dr[h];
                x = fmaf(fh.x, dr[P.parent].y, fh.y);
            } else {
                x = dr[h].y;
                const int nrn = G.neuron0 + (P.nflag & kPathNeuronG);
                const double v0 = a.Vsoma[nrn], v1 = v0 + (double)x;
                a.Vsoma[nrn] = v1;
                if (!isfinite(v1)) atomicOr(&a.ctl->err, MMK_ERR_NUMERIC);
                if (v0 < a.threshold && v1 >= a.threshold) {
                    const int src = soma_source(a, nrn);
                    if (src >= 0)
                        record_spike(a, src, a.user_id[nrn], 0,
                                     (double)n * a.dt64 + a.dt64 * (a.threshold - v0) / (v1 - v0), n);
                }
            }
            const float xh = x;
            float f0[8], c0v[8], f1[8], c1v[8];
            auto load = [&](int jj, float *f, float *c) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float2 w = dr[min(jj + k, P.end - 1)];
                    f[k] = w.x;
                    c[k] = w.y;
                }
            };
            auto chain = [&](int jj, const float *f, const float *c) {
                const int cnt = P.end - jj;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    x = fmaf(f[k], x, c[k]);
                    if (k < cnt) dr[jj + k].y = x;
                }
            };
            int j = h + 1;
            if (j < P.end) {
                load(j, f0, c0v);
                for (;;) {
                    int jn = j + 8;
                    bool more = jn < P.end;
                    if (more) load(jn, f1, c1v);
                    chain(j, f0, c0v);
                    j = jn;
                    if (!more) break;
                    jn = j + 8;
                    more = jn < P.end;
                    if (more) load(jn, f0, c0v);
                    chain(j, f1, c1v);
                    j = jn;
                    if (!more) break;
                }
            }
            if (P.parent >= 0) dr[h].y = xh;  // read by the next level only
        };

        for (int k = 0; k < G.nbundle; ++k) {
            const NrnG Nk = nrns[k];
            const int32_t *lo = loffs + Nk.loff0;
            const int32_t *mc = mcnt + Nk.loff0;
            for (int l = Nk.nlevel - 1; l >= 0; --l) {
                const int pb = lo[l], pe = lo[l + 1];
                for (int pi = pb + tid; pi < pe; pi += NT) eliminate_path(pi);
                __syncthreads();
                if (mc[l] > 0) {
                    fold_shared(pb, pb + mc[l]);
                    __syncthreads();
                }
            }
            for (int l = 0; l < Nk.nlevel; ++l) {
                const int pe = lo[l + 1];
                for (int pi = lo[l] + tid; pi < pe; pi += NT) substitute_path(pi);
                __syncthreads();
            }
        }

        if (a.item_ns) {
            __syncthreads();
            if (tid == 0) a.item_ns[gi] += global_ns() - t_item;
        }
    }
}

// The giant items' compartments in chunks of kGiantChunk: chunk ch belongs
// to the giant item k with gchunk0[k] <= ch < gchunk0[k + 1].
constexpr int kGiantChunk = 2048;

__device__ __forceinline__ int giant_of_chunk(const StepArgs32 &a, int64_t ch)
{
    int lo = 0, hi = a.item1 - a.item0;  // gchunk0 has item1 - item0 + 1 entries
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.gchunk0[mid] <= ch) lo = mid; else hi = mid;
    }
    return lo;
}

// Phase A of every giant compartment (as in step_fp32c_kernel), into the
// global scratch (the rhs's low word into its own array).
__global__ void __launch_bounds__(256) giant_assemble_kernel(StepArgs32 a)
{
    const int64_t nch = a.gchunk0[a.item1 - a.item0];
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int k = giant_of_chunk(a, ch);
        const GroupRec &G = a.groups[a.item0 + k];
        const int64_t c0 = G.comp0;
        const int32_t *Vq = a.Vq + c0;
        const float2 *gax = a.gax + c0;
        float2 *dr = a.dr + G.scratch0;
        float *drl = a.drl + G.scratch0;
        const int i0 = (int)(ch - a.gchunk0[k]) * kGiantChunk, i1 = min(i0 + kGiantChunk, G.ncomp);
        for (int i = i0 + (int)threadIdx.x; i < i1; i += 256) {
            const int32_t vq = Vq[i];
            const float2 gs = gax[i];
            const mmf::F2 ar = f2(a.area[c0 + i]);
            const mmf::F2 m = mmf::gate_df(a.mq[c0 + i]), h = mmf::gate_df(a.hq[c0 + i]),
                          nn = mmf::gate_df(a.nq[c0 + i]);
            const mmf::F2 gna = mmf::mul(f2(a.gNa), mmf::mul(mmf::mul(mmf::mul(m, m), m), h));
            const mmf::F2 n2 = mmf::mul(nn, nn);
            const mmf::F2 gk = mmf::mul(f2(a.gK), mmf::mul(n2, n2));
            const mmf::F2 iu = mmf::add(mmf::mul(gna, vminus(vq, a.ENa)),
                                        mmf::add(mmf::mul(gk, vminus(vq, a.EK)), mmf::mul(f2(a.gL), vminus(vq, a.EL))));
            mmf::F2 r = mmf::neg(mmf::mul(ar, iu));
            if (!signbit(gs.x))  // link to the parent i-1
                r = mmf::add(r, mmf::mul(mmf::F2{fabsf(gs.x), gs.y}, mmf::vdiff_df(Vq[i - 1], vq)));
            if (i + 1 < G.ncomp) {
                const float2 gc = gax[i + 1];
                if (!signbit(gc.x))  // link to the child i+1
                    r = mmf::add(r, mmf::mul(f2(gc), mmf::vdiff_df(Vq[i + 1], vq)));
            }
            dr[i] = make_float2((a.g_implicit ? ar.hi * (gna.hi + gk.hi) : 0.f) + a.dp[c0 + i].y, r.hi);
            drl[i] = r.lo;
        }
    }
}

// Phase C (V^{n+1} = V^n + dV, exact in fixed point) and the gates at
// V^{n+1} of every giant compartment.
__global__ void __launch_bounds__(256) giant_update_kernel(StepArgs32 a)
{
    const long long n = (long long)a.ctl->step_base + a.step_offset;
    const int64_t nch = a.gchunk0[a.item1 - a.item0];
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int k = giant_of_chunk(a, ch);
        const GroupRec &G = a.groups[a.item0 + k];
        const int64_t c0 = G.comp0;
        const float2 *dr = a.dr + G.scratch0;
        const int i0 = (int)(ch - a.gchunk0[k]) * kGiantChunk, i1 = min(i0 + kGiantChunk, G.ncomp);
        for (int i = i0 + (int)threadIdx.x; i < i1; i += 256) {
            const int32_t vold = a.Vq[c0 + i];
            int32_t vq;
            if (!mmf::v_add(vold, dr[i].y, &vq)) {
                atomicOr(&a.ctl->err, MMK_ERR_NUMERIC);
                vq = vold;
            }
            a.Vq[c0 + i] = vq;
            if (a.pt_of && vold < a.thr_q && vq >= a.thr_q) {
                const int p = a.pt_of[c0 + i];
                if (p >= 0) point_spike(a, p, (double)vold * kVInvD, (double)vq * kVInvD, n, a.dt64);
            }
            gate_update(a, c0 + i);
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

__global__ void scatter_f2_to_f64_kernel(const float2 *src, const int64_t *idx, double *dst, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[idx[i]] = (double)src[i].x + (double)src[i].y;
}

int grid32(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

// The dynamic shared-memory limit is a property of the kernel, shared by
// every network of the process: it only ever grows, so that a network
// created later with smaller items does not lower it below what an earlier
// one launches with.
template <int NT>
int set_attr_and_occupancy(int smem, int *blocks)
{
    static std::mutex mu;
    static int limit = 0;
    cudaError_t e = cudaSuccess;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (smem > limit) {
            e = cudaFuncSetAttribute(step_fp32c_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess) limit = smem;
        }
    }
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, step_fp32c_kernel<NT>, NT, smem);
    return (int)e;
}

}  // namespace

int mmk_launch_giant_fp32c(const StepArgs32 &a, int blocks, void *stream)
{
    giant_fp32c_kernel<256><<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int mmk_launch_giant_assemble(const StepArgs32 &a, int chunk_blocks, void *stream)
{
    giant_assemble_kernel<<<chunk_blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int mmk_launch_giant_update(const StepArgs32 &a, int chunk_blocks, void *stream)
{
    giant_update_kernel<<<chunk_blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

int mmk_giant_chunk()
{
    return kGiantChunk;
}

int mmk_launch_step_fp32c(const StepArgs32 &a, int blocks, int threads, void *stream)
{
    const size_t smem = (size_t)a.smem_bytes;
    cudaStream_t s = (cudaStream_t)stream;
    switch (threads) {
    case 128: step_fp32c_kernel<128><<<blocks, 128, smem, s>>>(a); break;
    case 256: step_fp32c_kernel<256><<<blocks, 256, smem, s>>>(a); break;
    case 512: step_fp32c_kernel<512><<<blocks, 512, smem, s>>>(a); break;
    case 1024: step_fp32c_kernel<1024><<<blocks, 1024, smem, s>>>(a); break;
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
    case 1024: return set_attr_and_occupancy<1024>(smem_bytes, blocks);
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

int mmk_launch_deliver_ordered_fp32c(const DeliverArgs &a, int blocks, void *stream)
{
    deliver_ordered_fp32c_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
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

int mmk_launch_scatter_f2_to_f64(const float2 *src, const int64_t *idx, double *dst, int64_t n, void *stream)
{
    if (n <= 0) return 0;
    scatter_f2_to_f64_kernel<<<grid32(n, 256), 256, 0, (cudaStream_t)stream>>>(src, idx, dst, n);
    return (int)cudaGetLastError();
}

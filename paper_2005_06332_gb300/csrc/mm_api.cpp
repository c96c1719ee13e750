// mm_api.cpp -- the C-ABI of include/mm.h: network lifetime, device memory,
// step launches (direct and CUDA-graph), reads, stimulus and checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mm.h"
#include "mm_gate_table.h"
#include "mm_internal.h"
#include "mm_layout.h"

namespace {

constexpr int kStepThreads = 256;
constexpr int kDefaultGroupComps = 4096;
constexpr int kDefaultGroupComps32 = 2048;  // FP32c: 24 B of shared memory per compartment
constexpr int kMaxGroupComps = MM_FP64_MAX_NEURON_COMPS;
constexpr int kMaxGroupComps32 = 1 << 30;
constexpr int kGiantSmemLimit = 110 * 1024;  // FP32c regular class: two blocks per SM
constexpr int kBigSmemLimit = 224 * 1024;    // FP32c large class (one block per SM); above it: giant kernel
constexpr int kBigThreads = 1024;
constexpr size_t kMaxSmem = 227 * 1024;

}  // namespace

struct mm_net {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;
    // FP32c giant items run on a side stream, concurrently with the other
    // work-item classes of the same step (fork after delivery, join at the
    // end of the step)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // FP32c large class: forked onto a stream of its own after the delivery,
    // so that its blocks (the largest items) start first and the regular
    // class fills the SMs as they drain; joined at the end of the step
    cudaStream_t side2 = nullptr;
    // external spike sources (a network that is one part of a larger one)
    int32_t n_ext = 0, min_dsteps = 0;
    int32_t *inj_src = nullptr;      // device staging of mm_inject_spikes
    int64_t *inj_step = nullptr;
    int64_t inj_cap = 0;
    cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
    // pinned host staging, so that the per-step host calls copy
    // asynchronously and synchronise once: the control block (read and
    // written back), the stimulus (with the event of its last upload) and
    // a buffer for soma voltages and spike records
    mmk::DevCtl *pin_ctl = nullptr, *pin_ctl_w = nullptr;
    double *pin_stim = nullptr;
    cudaEvent_t ev_stim = nullptr;
    unsigned char *pin = nullptr;
    size_t pin_cap = 0;
    mm_allocator alloc{};
    std::vector<void *> blocks;
    std::string err;
    bool poisoned = false;

    int precision = MM_FP64;
    double dt = 0.025;
    int32_t N = 0;
    int64_t C = 0, nsite = 0, S = 0;
    int32_t R = 2;
    int32_t n_src = 0;        // spike sources: neurons, or detection points
    int detect = MM_DETECT_SOMA;
    // deterministic delivery: per step slot a bitmask of the sources that fired
    bool ordered = false;
    uint32_t *fired = nullptr;
    int32_t fired_words = 0;
    int ordered_blocks = 1;
    int64_t spk_cap = 0;
    int64_t steps_done = 0;

    mmk::StepArgs sa{};
    mmk::DeliverArgs da{};
    int step_blocks = 1, step_threads = kStepThreads, deliver_blocks = 1, giant_blocks = 1, giant_chunk_blocks = 1;
    int32_t n_giant = 0, n_small = 0, n_big = 0;
    int big_blocks = 1;
    int graph_steps = 40;
    cudaGraphExec_t gexec = nullptr;   // graph_steps steps
    cudaGraphExec_t gexec1 = nullptr;  // one step (single-step calls)

    mmk::StepArgs32 sa32{};   // regular shared-memory class
    mmk::StepArgs32 sa32b{};  // large shared-memory class
    mmk::StepArgs32 sa32g{};  // giant items

    // device arrays (FP64 path)
    double *V = nullptr, *m = nullptr, *h = nullptr, *n = nullptr;
    double *area = nullptr, *gax = nullptr, *gsyn = nullptr;
    // device arrays (FP32c path)
    int32_t *Vq = nullptr;
    uint32_t *mq = nullptr, *hq = nullptr, *nq = nullptr;
    double *Vsoma = nullptr;
    float2 *area2 = nullptr, *gax2 = nullptr, *dp2 = nullptr, *gsyn2 = nullptr;
    float2 *dr = nullptr;
    float *drl = nullptr;
    float4 *pq = nullptr;
    float4 *gtab = nullptr;           // gate table for dt (mm_gate_table.h)
    int64_t *soma_internal = nullptr, *internal_of64 = nullptr;
    // both
    double *stim = nullptr;
    double *spk_t = nullptr, *scratch = nullptr;
    int32_t *spk_nrn = nullptr, *ring_nrn = nullptr, *ring_cnt = nullptr, *user_id = nullptr;
    int32_t *spk_comp = nullptr;
    // detection points (MM_DETECT_SYNAPSE_POINTS)
    int32_t *pt_of = nullptr;
    int32_t *pt_user_nrn = nullptr, *pt_user_comp = nullptr, *soma_src = nullptr;
    int64_t *user2int = nullptr, *soma_of_user = nullptr, *site_internal = nullptr;
    mmk::DevCtl *ctl = nullptr;

    // kernel timing (events around each launch while enabled)
    bool timing = false;
    struct Pending { cudaEvent_t a, b; int kind; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    mm_kernel_times times{};

    mm_launch_info info{};

    unsigned long long *item_ns = nullptr;
    std::vector<int32_t> item_neuron0, item_nneuron;   // per work item (host copy)
    int64_t steps_at_create = 0;

    std::vector<int32_t> order;          // internal -> user
    std::vector<int32_t> internal_of;    // user -> internal
    double f_syn = 0.0;
};

namespace {

mm_status fail(mm_net *net, mm_status s, const std::string &m)
{
    if (net) {
        if (net->err.empty() || s != MM_OK) net->err = m;
        if (s == MM_ECUDA || s == MM_ENUMERIC || s == MM_ETIMEOUT) net->poisoned = true;
    }
    return s;
}

mm_status cuda_fail(mm_net *net, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(net, MM_ECUDA, m);
}

#define MM_CK(net, call)                                         \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((net), e_, #call); \
    } while (0)

#define MM_CKI(net, call)                                                        \
    do {                                                                         \
        int e_ = (call);                                                         \
        if (e_ != 0) return cuda_fail((net), (cudaError_t)e_, #call);            \
    } while (0)

void *dev_alloc(mm_net *net, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (net->alloc.alloc) {
        p = net->alloc.alloc(bytes, net->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) net->blocks.push_back(p);
    return p;
}

// Releases one block from dev_alloc (the stream must be idle).
void dev_free(mm_net *net, void *p)
{
    if (!p) return;
    auto it = std::find(net->blocks.begin(), net->blocks.end(), p);
    if (it == net->blocks.end()) return;
    net->blocks.erase(it);
    if (net->alloc.alloc) {
        if (net->alloc.release) net->alloc.release(p, net->alloc.ctx);
    } else {
        cudaFree(p);
    }
}

template <class T>
mm_status upload(mm_net *net, T **dst, const T *src, size_t count)
{
    *dst = (T *)dev_alloc(net, count * sizeof(T));
    if (!*dst) return fail(net, MM_ENOMEM, "device allocation failed");
    if (count && src) MM_CK(net, cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, net->stream));
    return MM_OK;
}

template <class T>
mm_status zeros(mm_net *net, T **dst, size_t count)
{
    *dst = (T *)dev_alloc(net, count * sizeof(T));
    if (!*dst) return fail(net, MM_ENOMEM, "device allocation failed");
    MM_CK(net, cudaMemsetAsync(*dst, 0, count * sizeof(T), net->stream));
    return MM_OK;
}

mm_status guard(mm_net *net)
{
    if (!net) return MM_EINVAL;
    if (net->poisoned) return MM_ESTATE;
    if (cudaSetDevice(net->device) != cudaSuccess) return cuda_fail(net, cudaGetLastError(), "cudaSetDevice");
    return MM_OK;
}

// Snapshot of the control block into pinned memory, enqueued on the stream
// behind everything issued so far (read it after the next synchronisation).
mm_status snap_ctl(mm_net *net)
{
    MM_CK(net, cudaMemcpyAsync(net->pin_ctl, net->ctl, sizeof(mmk::DevCtl), cudaMemcpyDeviceToHost, net->stream));
    return MM_OK;
}

// The device error word of a snapshot -> status.
mm_status ctl_status(mm_net *net, const mmk::DevCtl &c)
{
    if (c.err & mmk::MMK_ERR_NUMERIC) return fail(net, MM_ENUMERIC, "a soma voltage became NaN or infinite");
    if (c.err & mmk::MMK_ERR_TIMEOUT)
        return fail(net, MM_ETIMEOUT, "a work item's tree blob did not arrive within the kernel's wait limit");
    return MM_OK;
}

// Device error word -> status (synchronising).
mm_status check_device(mm_net *net)
{
    mm_status st = snap_ctl(net);
    if (st != MM_OK) return st;
    MM_CK(net, cudaStreamSynchronize(net->stream));
    return ctl_status(net, *net->pin_ctl);
}

// Pinned staging of at least `bytes` (contents not kept).
mm_status pinned(mm_net *net, size_t bytes)
{
    if (bytes <= net->pin_cap) return MM_OK;
    MM_CK(net, cudaStreamSynchronize(net->stream));
    if (net->pin) cudaFreeHost(net->pin);
    net->pin = nullptr;
    net->pin_cap = 0;
    const size_t cap = std::max<size_t>(bytes, 1 << 20);
    MM_CK(net, cudaMallocHost((void **)&net->pin, cap));
    net->pin_cap = cap;
    return MM_OK;
}

cudaError_t take_event(mm_net *net, cudaEvent_t *e)
{
    if (!net->event_pool.empty()) {
        *e = net->event_pool.back();
        net->event_pool.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

mm_status collect_timing(mm_net *net)
{
    for (auto &p : net->pending) {
        MM_CK(net, cudaEventSynchronize(p.b));
        float ms = 0.f;
        MM_CK(net, cudaEventElapsedTime(&ms, p.a, p.b));
        if (p.kind == 0) {
            net->times.deliver_kernel_ms += ms;
            net->times.deliver_kernel_launches++;
        } else if (p.kind == 3 || p.kind == 5 || p.kind == 6) {
            // the three kernels of the giant items; one launch per step
            net->times.giant_kernel_ms += ms;
            if (p.kind == 3) net->times.giant_kernel_launches++;
        } else if (p.kind == 4) {
            net->times.big_kernel_ms += ms;
            net->times.big_kernel_launches++;
        } else {
            net->times.step_kernel_ms += ms;
            net->times.step_kernel_launches++;
        }
        net->event_pool.push_back(p.a);
        net->event_pool.push_back(p.b);
    }
    net->pending.clear();
    return MM_OK;
}

mm_status launch_steps(mm_net *net, cudaStream_t s, int count)
{
    const bool timed = net->timing && s == net->stream;
    // Per step: delivery, then the solve of each work-item class.  FP32c
    // giant items: phase A of all their compartments (every SM), their
    // solve forked onto the side stream to run beside the shared-memory
    // classes, and after the join phase C and the gates (every SM).
    //   kinds: 0 delivery, 1 regular class, 4 large class (second side
    //          stream), 5 giant phase A, 3 giant solve (side stream), 6 giant
    //          phase C + gates, 7 join of the large class
    const bool giants = net->precision != MM_FP64 && net->n_giant > 0;
    int kinds[8], nk = 0;
    kinds[nk++] = 0;
    if (net->precision == MM_FP64) {
        kinds[nk++] = 1;
    } else {
        if (net->n_big > 0) kinds[nk++] = 4;
        if (giants) {
            kinds[nk++] = 5;
            kinds[nk++] = 3;
        }
        if (net->n_small > 0) kinds[nk++] = 1;
        if (giants) kinds[nk++] = 6;
        if (net->n_big > 0) kinds[nk++] = 7;
    }
    for (int j = 0; j < count; ++j) {
        for (int ki = 0; ki < nk; ++ki) {
            const int kind = kinds[ki];
            if (kind == 7) {  // the end of the step waits for the large class
                MM_CK(net, cudaStreamWaitEvent(s, net->ev_join2, 0));
                continue;
            }
            const bool forked = kind == 3, forked2 = kind == 4;
            cudaStream_t ks = forked ? net->side : (forked2 ? net->side2 : s);
            if (forked) {
                MM_CK(net, cudaEventRecord(net->ev_fork, s));
                MM_CK(net, cudaStreamWaitEvent(net->side, net->ev_fork, 0));
            }
            if (forked2) {
                MM_CK(net, cudaEventRecord(net->ev_fork2, s));
                MM_CK(net, cudaStreamWaitEvent(net->side2, net->ev_fork2, 0));
            }
            if (kind == 6) MM_CK(net, cudaStreamWaitEvent(s, net->ev_join, 0));
            mm_net::Pending p{nullptr, nullptr, kind};
            if (timed) {
                MM_CK(net, take_event(net, &p.a));
                MM_CK(net, take_event(net, &p.b));
                MM_CK(net, cudaEventRecord(p.a, ks));
            }
            if (kind == 0) {
                mmk::DeliverArgs da = net->da;
                da.step_offset = j;
                if (net->ordered && net->precision == MM_FP64)
                    MM_CKI(net, mmk_launch_deliver_ordered(da, net->ordered_blocks, s));
                else if (net->ordered)
                    MM_CKI(net, mmk_launch_deliver_ordered_fp32c(da, net->ordered_blocks, s));
                else if (net->precision == MM_FP64)
                    MM_CKI(net, mmk_launch_deliver(da, net->deliver_blocks, s));
                else
                    MM_CKI(net, mmk_launch_deliver_fp32c(da, net->deliver_blocks, s));
            } else if (net->precision == MM_FP64) {
                mmk::StepArgs sa = net->sa;
                sa.step_offset = j;
                MM_CKI(net, mmk_launch_step_fp64(sa, net->step_blocks, net->step_threads, s));
            } else if (kind == 1) {
                mmk::StepArgs32 sa = net->sa32;
                sa.step_offset = j;
                MM_CKI(net, mmk_launch_step_fp32c(sa, net->step_blocks, net->step_threads, s));
            } else if (kind == 4) {
                mmk::StepArgs32 sa = net->sa32b;
                sa.step_offset = j;
                MM_CKI(net, mmk_launch_step_fp32c(sa, net->big_blocks, kBigThreads, ks));
            } else {
                mmk::StepArgs32 sa = net->sa32g;
                sa.step_offset = j;
                if (kind == 5) MM_CKI(net, mmk_launch_giant_assemble(sa, net->giant_chunk_blocks, s));
                else if (kind == 3) MM_CKI(net, mmk_launch_giant_fp32c(sa, net->giant_blocks, ks));
                else MM_CKI(net, mmk_launch_giant_update(sa, net->giant_chunk_blocks, s));
            }
            if (timed) {
                MM_CK(net, cudaEventRecord(p.b, ks));
                net->pending.push_back(p);
            }
            if (forked) MM_CK(net, cudaEventRecord(net->ev_join, net->side));
            if (forked2) MM_CK(net, cudaEventRecord(net->ev_join2, net->side2));
        }
        if (timed && net->pending.size() > 4096) {
            mm_status st = collect_timing(net);
            if (st != MM_OK) return st;
        }
    }
    MM_CKI(net, mmk_launch_advance(net->ctl, count, s));
    return MM_OK;
}

// Captures `steps` steps into *exec (once).
mm_status ensure_graph(mm_net *net, int steps, cudaGraphExec_t *exec)
{
    if (*exec || steps <= 0) return MM_OK;
    cudaGraph_t graph = nullptr;
    MM_CK(net, cudaStreamBeginCapture(net->cap_stream, cudaStreamCaptureModeThreadLocal));
    mm_status st = launch_steps(net, net->cap_stream, steps);
    cudaError_t e = cudaStreamEndCapture(net->cap_stream, &graph);
    if (st != MM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(net, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return cuda_fail(net, e, "cudaGraphInstantiate");
    }
    return MM_OK;
}

void release_all(mm_net *net)
{
    if (net->gexec) cudaGraphExecDestroy(net->gexec);
    if (net->gexec1) cudaGraphExecDestroy(net->gexec1);
    net->gexec = net->gexec1 = nullptr;
    if (net->stream) cudaStreamSynchronize(net->stream);
    if (net->side) cudaStreamSynchronize(net->side);
    if (net->side2) cudaStreamSynchronize(net->side2);
    for (auto &p : net->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    net->pending.clear();
    for (cudaEvent_t e : net->event_pool) cudaEventDestroy(e);
    net->event_pool.clear();
    for (void *p : net->blocks) {
        if (net->alloc.alloc) {
            if (net->alloc.release) net->alloc.release(p, net->alloc.ctx);
        } else {
            cudaFree(p);
        }
    }
    net->blocks.clear();
    if (net->cap_stream) cudaStreamDestroy(net->cap_stream);
    if (net->side) cudaStreamDestroy(net->side);
    if (net->ev_fork) cudaEventDestroy(net->ev_fork);
    if (net->ev_join) cudaEventDestroy(net->ev_join);
    if (net->side2) cudaStreamDestroy(net->side2);
    if (net->ev_fork2) cudaEventDestroy(net->ev_fork2);
    if (net->ev_join2) cudaEventDestroy(net->ev_join2);
    if (net->ev_stim) cudaEventDestroy(net->ev_stim);
    if (net->pin_ctl) cudaFreeHost(net->pin_ctl);
    if (net->pin_stim) cudaFreeHost(net->pin_stim);
    if (net->pin) cudaFreeHost(net->pin);
    net->ev_stim = nullptr;
    net->pin_ctl = net->pin_ctl_w = nullptr;
    net->pin_stim = nullptr;
    net->pin = nullptr;
    net->pin_cap = 0;
    net->side = nullptr;
    net->ev_fork = nullptr;
    net->ev_join = nullptr;
    net->side2 = nullptr;
    net->ev_fork2 = nullptr;
    net->ev_join2 = nullptr;
    if (net->own_stream && net->stream) cudaStreamDestroy(net->stream);
    net->cap_stream = nullptr;
    net->stream = nullptr;
}

float2 split_pair(double x)
{
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

std::vector<float2> split_pairs(const std::vector<double> &v)
{
    std::vector<float2> out(v.size());
    for (size_t i = 0; i < v.size(); ++i) out[i] = split_pair(v[i]);
    return out;
}

// FP32c constants per compartment (internal order), computed in FP64 from
// the cylinders: area (cm^2), the axial conductance g to the parent (uS;
// 1 / the sum of the two half-cylinder resistances, 0 at a soma) with the
// sign bit of its high word set at path heads and somata, and the passive
// diagonal d0' of Algorithm 1's elimination (uS) as its nearest float and
// the share of the active part that stands for the rest (below):
// d0_i = C_i/dt + the leak
// conductance (backward Euler only: Eq. 2 as printed keeps the membrane
// current explicit) + the implicit share of every coupling at i, then
// d0'_p -= (w g_i)^2 / d0'_i over the children i of p, leaves first (w the
// implicit share: 1, or 1/2 for Eq. 2 as printed).
void passive_constants(const mmh::Layout &L, const mm_channel_params &ch, double dt, bool cn,
                       std::vector<float2> &area2, std::vector<float2> &gax2, std::vector<float2> &dp2)
{
    const size_t C = (size_t)L.C;
    const double pi = 3.141592653589793, w = cn ? 0.5 : 1.0;
    std::vector<double> area(C), g(C, 0.0), d(C);
    auto rhalf = [&](size_t i) {
        const double rad = 0.5e-4 * L.D[i];
        return ch.Ra * (0.5e-4 * L.L[i]) / (pi * rad * rad) * 1e-6;
    };
    for (size_t i = 0; i < C; ++i) {
        area[i] = pi * L.D[i] * L.L[i] * 1e-8;
        d[i] = ch.Cm * area[i] * 1e3 / dt + (cn ? 0.0 : ch.gL * area[i] * 1e3);
    }
    for (size_t i = 0; i < C; ++i) {
        const int32_t pd = std::abs(L.pdist[i]);
        if (pd == 0) continue;
        const size_t q = i - (size_t)pd;
        g[i] = 1.0 / (rhalf(i) + rhalf(q));
        d[i] += w * g[i];
        d[q] += w * g[i];
    }
    // parents precede their children in internal order: children first
    for (size_t i = C; i-- > 0;) {
        const int32_t pd = std::abs(L.pdist[i]);
        if (pd == 0) continue;
        const double wg = w * g[i];
        d[i - (size_t)pd] -= wg * wg / d[i];
    }
    // The sweep keeps d0' = dh + dl only through its nearest float dh: the
    // low word dl enters the active part it carries instead (e' = e + dl),
    // whose recurrence then takes dl_p - sum_c (w g_c / d0'_c)^2 dl_c once
    // per step (the children's share, at the passive coupling factor; the
    // remainder is of order (e / d0') dl, below the float rounding of d').
    std::vector<double> eps(C);
    for (size_t i = 0; i < C; ++i) eps[i] = d[i] - (double)(float)d[i];
    for (size_t i = C; i-- > 0;) {
        const int32_t pd = std::abs(L.pdist[i]);
        if (pd == 0) continue;
        const double f0 = w * g[i] / d[i];
        eps[i - (size_t)pd] -= f0 * f0 * (d[i] - (double)(float)d[i]);
    }
    area2.resize(C);
    gax2.resize(C);
    dp2.resize(C);
    for (size_t i = 0; i < C; ++i) {
        area2[i] = split_pair(area[i]);
        float2 gp = split_pair(g[i]);
        if (L.pdist[i] <= 0) gp.x = -gp.x;  // path head or soma (-0.0 at a soma)
        gax2[i] = gp;
        dp2[i] = make_float2((float)d[i], (float)eps[i]);
    }
}

mm_status build(mm_net *net, const mm_morphologies *morph, const mm_channel_params *chan, const mm_synapses *syn,
                const double *stim_nA, const mm_options *opt)
{
    net->precision = opt->precision;
    net->dt = opt->dt_ms;
    net->graph_steps = std::max(0, opt->graph_steps);
    net->device = opt->device;
    net->alloc = opt->allocator;
    if (opt->precision != MM_FP64 && opt->precision != MM_FP32C) return fail(net, MM_EINVAL, "unknown precision");
    if (opt->schedule != MM_SCHED_SIZE_SORTED && opt->schedule != MM_SCHED_COST)
        return fail(net, MM_EINVAL, "unknown schedule");
    if (opt->scheme != MM_SCHEME_BE && opt->scheme != MM_SCHEME_CN) return fail(net, MM_EINVAL, "unknown scheme");
    if (opt->detect != MM_DETECT_SOMA && opt->detect != MM_DETECT_SYNAPSE_POINTS)
        return fail(net, MM_EINVAL, "unknown detection mode");
    if (opt->deterministic_delivery != 0 && opt->deterministic_delivery != 1)
        return fail(net, MM_EINVAL, "mm_options.deterministic_delivery must be 0 or 1");
    if (opt->schedule == MM_SCHED_COST && !opt->cost) return fail(net, MM_EINVAL, "MM_SCHED_COST needs mm_options.cost");
    if (syn && !(syn->tau_ms > 0.0)) return fail(net, MM_EINVAL, "tau_ms must be > 0");
    if (opt->n_ext_sources < 0) return fail(net, MM_EINVAL, "n_ext_sources must be >= 0");
    if (opt->n_ext_sources > 0 && opt->detect != MM_DETECT_SOMA)
        return fail(net, MM_ENOTSUP, "external spike sources need MM_DETECT_SOMA");
    if (!chan) return fail(net, MM_EINVAL, "channel parameters must not be NULL");

    MM_CK(net, cudaSetDevice(net->device));
    if (opt->cuda_stream) {
        net->stream = (cudaStream_t)opt->cuda_stream;
    } else {
        MM_CK(net, cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking));
        net->own_stream = true;
    }
    MM_CK(net, cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking));
    MM_CK(net, cudaStreamCreateWithFlags(&net->side, cudaStreamNonBlocking));
    MM_CK(net, cudaEventCreateWithFlags(&net->ev_fork, cudaEventDisableTiming));
    MM_CK(net, cudaEventCreateWithFlags(&net->ev_join, cudaEventDisableTiming));
    MM_CK(net, cudaStreamCreateWithFlags(&net->side2, cudaStreamNonBlocking));
    MM_CK(net, cudaEventCreateWithFlags(&net->ev_fork2, cudaEventDisableTiming));
    MM_CK(net, cudaEventCreateWithFlags(&net->ev_join2, cudaEventDisableTiming));
    MM_CK(net, cudaEventCreateWithFlags(&net->ev_stim, cudaEventDisableTiming));
    MM_CK(net, cudaMallocHost((void **)&net->pin_ctl, 2 * sizeof(mmk::DevCtl)));
    net->pin_ctl_w = net->pin_ctl + 1;
    MM_CK(net, cudaMallocHost((void **)&net->pin_stim, (size_t)std::max(morph->n_neurons, 1) * sizeof(double)));

    // layout
    mmh::LayoutInput li{};
    li.N = morph->n_neurons;
    li.comp_offset = morph->comp_offset;
    li.parent = morph->parent;
    li.length_um = morph->length_um;
    li.diam_um = morph->diam_um;
    li.S = syn ? syn->n : 0;
    li.src = syn ? syn->src_neuron : nullptr;
    li.dst = syn ? syn->dst_neuron : nullptr;
    li.dcomp = syn ? syn->dst_comp : nullptr;
    li.w = syn ? syn->weight_uS : nullptr;
    li.delay_ms = syn ? syn->delay_ms : nullptr;
    li.points = opt->detect == MM_DETECT_SYNAPSE_POINTS;
    li.scomp = syn ? syn->src_comp : nullptr;
    li.stim = stim_nA;
    li.cost = opt->schedule == MM_SCHED_COST ? opt->cost : nullptr;
    li.dt = opt->dt_ms;
    li.n_ext = opt->n_ext_sources;
    li.group_comps = opt->group_comps > 0 ? opt->group_comps
                   : (opt->precision == MM_FP64 ? kDefaultGroupComps : kDefaultGroupComps32);
    li.max_group_comps = opt->precision == MM_FP64 ? kMaxGroupComps : kMaxGroupComps32;
    // shared memory per item: FP64 d and rhs per compartment (16 B); FP32c
    // d, rhs and |g| per compartment (12 B) and per path its contribution
    // to the parent (d, rhs) and the potential across its head link (12 B)
    // FP32c (active conductance, rhs) pair, the implicit coupling and the
    // passive diagonal as pairs (the diagonal's place holds the rhs's low
    // words until the rhs is final; 24 B per compartment) and per path two
    // words (the head link's current, then the contribution to the parent)
    li.smem_per_comp = opt->precision == MM_FP64 ? 16 : 24;
    li.smem_per_seg = 0;
    li.path_items = opt->precision != MM_FP64;
    li.smem_per_path = opt->precision == MM_FP64 ? 0 : 8;
    li.giant_smem_limit = opt->precision == MM_FP64 ? 0 : kGiantSmemLimit;
    li.big_smem_limit = opt->precision == MM_FP64 ? 0 : kBigSmemLimit;
    mmh::Layout L;
    bool invalid = false;
    std::string m;
    try {
        m = mmh::build_layout(li, L, &invalid);
    } catch (const std::bad_alloc &) {
        return fail(net, MM_ENOMEM, "host allocation failed while building the layout");
    }
    if (!m.empty()) return fail(net, invalid ? MM_EINVAL : MM_ENOTSUP, m);
    if (L.dclass.size() > 1024) return fail(net, MM_ENOTSUP, "more than 1024 distinct delays");

    net->N = L.N;
    net->C = L.C;
    for (const auto &gr : L.groups) {
        net->item_neuron0.push_back(gr.neuron0);
        net->item_nneuron.push_back(gr.nneuron);
    }
    net->nsite = (int64_t)L.site_comp.size();
    net->S = li.S;
    net->R = L.R;
    net->n_src = L.n_src;
    net->n_ext = opt->n_ext_sources;
    net->min_dsteps = L.dclass.empty() ? 0 : L.dclass.front();
    net->detect = opt->detect;
    net->order = L.order;
    net->internal_of = L.internal_of;
    net->f_syn = L.f_syn;
    net->spk_cap = opt->spike_capacity > 0 ? opt->spike_capacity
                 : std::max<int64_t>(1 << 16, (int64_t)L.n_src * (li.points ? 16 : 64));

    const size_t C = (size_t)L.C, N = (size_t)L.N;
    mm_status st;
#define UP(dst, src, cnt) if ((st = upload(net, &(dst), (src), (cnt))) != MM_OK) return st
#define ZR(dst, cnt) if ((st = zeros(net, &(dst), (cnt))) != MM_OK) return st
    const bool f64 = opt->precision == MM_FP64;
    double *dL = nullptr, *dD = nullptr;
    int32_t *dpd = nullptr;
    UP(dL, L.L.data(), C);
    UP(dD, L.D.data(), C);
    UP(dpd, L.pdist.data(), C);
    if (f64) {
        ZR(net->V, C);
        ZR(net->m, C);
        ZR(net->h, C);
        ZR(net->n, C);
        ZR(net->area, C);
        ZR(net->gax, C);
        ZR(net->gsyn, (size_t)std::max<int64_t>(net->nsite, 1));
    } else {
        ZR(net->Vq, C);
        ZR(net->mq, C);
        ZR(net->hq, C);
        ZR(net->nq, C);
        {
            // constants of the FP32c path as float pairs, computed here in
            // FP64 in internal order: membrane area, axial conductance to the
            // parent (sign bit of the high word at path heads and somata) and
            // the passive diagonal after the elimination of Algorithm 1
            std::vector<float2> area2, gax2, dp2;
            passive_constants(L, *chan, opt->dt_ms, opt->scheme == MM_SCHEME_CN, area2, gax2, dp2);
            UP(net->area2, area2.data(), C);
            UP(net->gax2, gax2.data(), C);
            UP(net->dp2, dp2.data(), C);
        }
        {
            // X(V) and E(V) of the three gates for this dt, per 0.5 mV
            static_assert(sizeof(mmf::Tab4) == sizeof(float4), "table quads are float4");
            std::vector<mmf::Tab4> tab((size_t)mmf::kTabQuads * mmf::kTabIntervals);
            mmf::build_gate_table(opt->dt_ms, tab.data());
            UP(net->gtab, reinterpret_cast<const float4 *>(tab.data()), tab.size());
        }
        ZR(net->Vsoma, N);
        ZR(net->gsyn2, (size_t)std::max<int64_t>(net->nsite, 1));
        ZR(net->dr, (size_t)std::max<int64_t>(L.giant_comps, 1));
        ZR(net->drl, (size_t)std::max<int64_t>(L.giant_comps, 1));
        ZR(net->pq, (size_t)std::max<int64_t>(L.giant_paths, 1));
        std::vector<int64_t> soma_int(N), int_of(N);
        for (size_t k = 0; k < N; ++k) soma_int[k] = L.noff[k];
        for (size_t u = 0; u < N; ++u) int_of[u] = L.internal_of[u];
        UP(net->soma_internal, soma_int.data(), N);
        UP(net->internal_of64, int_of.data(), N);
    }
    ZR(net->scratch, 2 * std::max(C, N));
    UP(net->stim, L.stim.data(), N);
    UP(net->user_id, L.order.data(), N);
    UP(net->user2int, L.user2int.data(), C);
    UP(net->soma_of_user, L.soma_of_user.data(), N);
    UP(net->site_internal, L.site_internal.data(), (size_t)net->nsite);
    ZR(net->ring_nrn, (size_t)net->R * (size_t)std::max(net->n_src, 1));
    ZR(net->ring_cnt, (size_t)net->R);
    ZR(net->spk_nrn, (size_t)net->spk_cap);
    ZR(net->spk_comp, (size_t)net->spk_cap);
    int64_t *din_off = nullptr;
    int32_t *din_src = nullptr, *din_ds = nullptr;
    double *din_w = nullptr;
    float2 *din_w2 = nullptr;
    if (opt->deterministic_delivery) {
        net->ordered = true;
        net->fired_words = std::max(1, (net->n_src + 31) / 32);
        ZR(net->fired, (size_t)net->R * (size_t)net->fired_words);
        UP(din_off, L.in_off.data(), L.in_off.size());
        UP(din_src, L.in_src.data(), std::max<size_t>(L.in_src.size(), 1));
        UP(din_ds, L.in_dsteps.data(), std::max<size_t>(L.in_dsteps.size(), 1));
        if (f64) {
            UP(din_w, L.in_w.data(), std::max<size_t>(L.in_w.size(), 1));
        } else {
            const std::vector<float2> w2 = split_pairs(L.in_w);
            UP(din_w2, w2.data(), std::max<size_t>(w2.size(), 1));
        }
    }
    if (li.points) {
        UP(net->pt_of, L.pt_of.data(), L.pt_of.size());
        UP(net->soma_src, L.soma_src.data(), N);
        if (L.n_src > 0) {
            UP(net->pt_user_nrn, L.pt_user_nrn.data(), L.pt_user_nrn.size());
            UP(net->pt_user_comp, L.pt_user_comp.data(), L.pt_user_comp.size());
        }
    }
    ZR(net->spk_t, (size_t)net->spk_cap);
    ZR(net->ctl, 1);
    mmk::GroupRec *dgroups = nullptr;
    unsigned char *dmeta = nullptr;
    int32_t *dsite = nullptr;
    UP(dgroups, L.groups.data(), L.groups.size());
    UP(dmeta, L.meta.data(), L.meta.size());
    UP(dsite, L.site_comp.data(), std::max<size_t>(L.site_comp.size(), 1));
    int64_t *dout_off = nullptr;
    int32_t *dout_site = nullptr, *dout_ds = nullptr, *ddclass = nullptr;
    double *dout_w = nullptr;
    float2 *dout_w2 = nullptr;
    UP(dout_off, L.out_off.data(), L.out_off.size());
    UP(dout_site, L.out_site.data(), std::max<size_t>(L.out_site.size(), 1));
    UP(dout_ds, L.out_dsteps.data(), std::max<size_t>(L.out_dsteps.size(), 1));
    if (f64) {
        UP(dout_w, L.out_w.data(), std::max<size_t>(L.out_w.size(), 1));
    } else {
        const std::vector<float2> w2 = split_pairs(L.out_w);
        UP(dout_w2, w2.data(), std::max<size_t>(w2.size(), 1));
    }
    UP(ddclass, L.dclass.data(), std::max<size_t>(L.dclass.size(), 1));
#undef UP
#undef ZR

    // geometry and the resting state on the device
    mmk::InitArgs ia{};
    ia.L = dL;
    ia.diam = dD;
    ia.parent_dist = dpd;
    ia.C = L.C;
    ia.Ra = chan->Ra;
    ia.v_init = chan->v_init;
    if (f64) {
        ia.area = net->area;
        ia.gax = net->gax;
        ia.V = net->V;
        ia.m = net->m;
        ia.h = net->h;
        ia.n = net->n;
        MM_CKI(net, mmk_launch_init(ia, net->stream));
    } else {
        ia.Vq = net->Vq;
        ia.mq = net->mq;
        ia.hq = net->hq;
        ia.nq = net->nq;
        MM_CKI(net, mmk_launch_init_fp32c(ia, net->stream));
        MM_CKI(net, mmk_launch_fill_f64(net->Vsoma, chan->v_init, (int64_t)N, net->stream));
    }

    const int32_t smem_comps = std::max(L.max_comps, 1), smem_segs = std::max(L.max_segs, 1);
    const double decay = syn ? std::exp(-opt->dt_ms / syn->tau_ms) : 1.0;
    if (f64) {
        mmk::StepArgs &a = net->sa;
        a.V = net->V;
        a.m = net->m;
        a.h = net->h;
        a.n = net->n;
        a.area = net->area;
        a.gax = net->gax;
        a.stim = net->stim;
        a.user_id = net->user_id;
        a.groups = dgroups;
        a.n_groups = (int32_t)L.groups.size();
        a.meta = dmeta;
        a.smem_meta = L.max_meta;
        a.site_comp = dsite;
        a.gsyn = net->gsyn;
        a.ring_nrn = net->ring_nrn;
        a.ring_cnt = net->ring_cnt;
        a.R = net->R;
        a.N = std::max(net->n_src, 1);
        a.spk_nrn = net->spk_nrn;
        a.spk_comp = net->spk_comp;
        a.spk_t = net->spk_t;
        a.spk_cap = net->spk_cap;
        a.pt_of = net->pt_of;
        a.pt_user_nrn = net->pt_user_nrn;
        a.pt_user_comp = net->pt_user_comp;
        a.soma_src = net->soma_src;
        a.n_pt = li.points ? net->n_src : 0;
        a.fired = net->fired;
        a.fired_words = net->fired_words;
        a.ctl = net->ctl;
        a.smem_comps = smem_comps;
        a.smem_segs = smem_segs;
        a.gNa = chan->gNa;
        a.gK = chan->gK;
        a.gL = chan->gL;
        a.ENa = chan->ENa;
        a.EK = chan->EK;
        a.EL = chan->EL;
        a.cm_dt = chan->Cm * 1e3 / opt->dt_ms;
        a.gimp = opt->scheme == MM_SCHEME_CN ? 0.5 : 1.0;
        a.g_implicit = opt->scheme == MM_SCHEME_CN ? 0 : 1;
        a.e_syn = syn ? syn->e_rev_mV : 0.0;
        a.threshold = chan->threshold_mV;
        a.dt = opt->dt_ms;
        a.decay = decay;
    } else {
        auto pot = [](double E) {
            mmk::FxPot p;
            const double q = std::nearbyint(E * mmk::kVScaleD);
            p.q = (int32_t)q;
            p.res = (float)(E - q / mmk::kVScaleD);
            return p;
        };
        for (double E : {chan->ENa, chan->EK, chan->EL, chan->v_init, syn ? syn->e_rev_mV : 0.0})
            if (!(std::fabs(E) < 120.0)) return fail(net, MM_EINVAL, "potentials must lie within +-120 mV for MM_FP32C");
        mmk::StepArgs32 &a = net->sa32;
        a.Vq = net->Vq;
        a.mq = net->mq;
        a.hq = net->hq;
        a.nq = net->nq;
        a.Vsoma = net->Vsoma;
        a.area = net->area2;
        a.gax = net->gax2;
        a.dp = net->dp2;
        a.dr = net->dr;
        a.drl = net->drl;
        a.pq = net->pq;
        if (opt->time_items) {
            if ((st = zeros(net, &net->item_ns, L.groups.size())) != MM_OK) return st;
            a.item_ns = net->item_ns;
        }
        a.stim = net->stim;
        a.user_id = net->user_id;
        a.groups = dgroups;
        a.n_groups = (int32_t)L.groups.size();
        a.item0 = 0;
        a.item1 = L.n_small;
        a.queue = &net->ctl->queue_head;
        a.meta = dmeta;
        a.smem_meta = L.max_meta;
        a.site_comp = dsite;
        a.gsyn = net->gsyn2;
        a.ring_nrn = net->ring_nrn;
        a.ring_cnt = net->ring_cnt;
        a.R = net->R;
        a.N = std::max(net->n_src, 1);
        a.spk_nrn = net->spk_nrn;
        a.spk_comp = net->spk_comp;
        a.spk_t = net->spk_t;
        a.spk_cap = net->spk_cap;
        a.pt_of = net->pt_of;
        a.pt_user_nrn = net->pt_user_nrn;
        a.pt_user_comp = net->pt_user_comp;
        a.soma_src = net->soma_src;
        a.n_pt = li.points ? net->n_src : 0;
        a.fired = net->fired;
        a.fired_words = net->fired_words;
        a.ctl = net->ctl;
        a.smem_comps = smem_comps;
        a.smem_segs = smem_segs;
        // channel densities (mS/cm^2) times 1e3: conductance in uS per cm^2 of membrane
        a.gNa = split_pair(chan->gNa * 1e3);
        a.gK = split_pair(chan->gK * 1e3);
        a.gL = split_pair(chan->gL * 1e3);
        a.ENa = pot(chan->ENa);
        a.EK = pot(chan->EK);
        a.EL = pot(chan->EL);
        a.Esyn = pot(syn ? syn->e_rev_mV : 0.0);
        a.gimp = opt->scheme == MM_SCHEME_CN ? 0.5f : 1.0f;
        a.g_implicit = opt->scheme == MM_SCHEME_CN ? 0 : 1;
        a.gtab = net->gtab;
        a.decay = split_pair(decay);
        a.threshold = chan->threshold_mV;
        {
            const double q = std::ceil(chan->threshold_mV * mmk::kVScaleD);
            a.thr_q = (int32_t)std::max(-2147483647.0, std::min(2147483647.0, q));
        }
        a.dt64 = opt->dt_ms;
        a.C = L.C;
    }

    mmk::DeliverArgs &d = net->da;
    d.ring_nrn = net->ring_nrn;
    d.ring_cnt = net->ring_cnt;
    d.R = net->R;
    d.N = std::max(net->n_src, 1);
    d.out_off = dout_off;
    d.out_site = dout_site;
    d.out_w = dout_w;
    d.out_dsteps = dout_ds;
    d.dclass = ddclass;
    d.n_dclass = (int32_t)L.dclass.size();
    {
        // lanes per spike in the delivery kernel: the mean number of synapses
        // of a (source, delay) pair, rounded up to a power of two, <= 32
        int64_t pairs = 0;
        for (int32_t k = 0; k < L.n_src; ++k)
            for (int64_t q = L.out_off[(size_t)k]; q < L.out_off[(size_t)k + 1]; ++q)
                if (q == L.out_off[(size_t)k] || L.out_dsteps[(size_t)q] != L.out_dsteps[(size_t)q - 1]) ++pairs;
        const double fan = pairs > 0 ? (double)li.S / (double)pairs : 32.0;
        int gl = 1;
        while (gl < 32 && gl < fan) gl *= 2;
        d.lanes_per_src = gl;
    }
    d.gsyn = net->gsyn;
    d.ctl = net->ctl;
    d.gsyn2 = net->gsyn2;
    d.out_w2 = dout_w2;
    d.in_off = din_off;
    d.in_src = din_src;
    d.in_dsteps = din_ds;
    d.in_w = din_w;
    d.in_w2 = din_w2;
    d.fired = net->fired;
    d.fired_words = net->fired_words;
    d.nsite = net->nsite;

    // FP32c carves each item's shared memory from its own sizes (the largest
    // per-item need of the class); FP64 uses one carve for all items
    const size_t smem = f64 ? mmk_step_fp64_smem(smem_comps, smem_segs, L.max_meta) : (size_t)std::max<int64_t>(L.max_smem, 16);
    if (smem > kMaxSmem) return fail(net, MM_ENOTSUP, "a work item needs more shared memory than a block has");
    int threads = opt->block_threads > 0 ? opt->block_threads : (f64 ? kStepThreads : 512);
    if (threads != 128 && threads != 256 && threads != 512 && (f64 || threads != 1024))
        return fail(net, MM_EINVAL, "block_threads must be 128, 256 or 512 (or 1024 for MM_FP32C)");
    net->step_threads = threads;
    net->sa32.smem_bytes = (int32_t)smem;
    int per_sm = 0;
    if (f64) MM_CKI(net, mmk_step_fp64_blocks_per_sm(threads, (int)smem, &per_sm));
    else MM_CKI(net, mmk_step_fp32c_blocks_per_sm(threads, (int)smem, &per_sm));
    if (per_sm < 1) return fail(net, MM_ENOTSUP, "the step kernel does not fit on an SM");
    int sms = 0;
    MM_CK(net, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device));
    net->step_blocks = std::max(1, std::min(std::max(L.n_small, 1), per_sm * sms));
    net->n_small = L.n_small;
    net->n_big = L.n_big;
    net->n_giant = (int32_t)L.groups.size() - L.n_small - L.n_big;
    net->giant_blocks = std::max(1, std::min(net->n_giant, 4 * sms));
    if (!f64) {
        // large class: same kernel, its own queue and shared-memory size
        mmk::StepArgs32 &b = net->sa32b;
        b = net->sa32;
        b.item0 = L.n_small;
        b.item1 = L.n_small + L.n_big;
        b.queue = &net->ctl->big_head;
        b.smem_comps = std::max(L.big_max_comps, 1);
        b.smem_segs = std::max(L.big_max_segs, 1);
        b.smem_meta = L.big_max_meta;
        if (L.n_big > 0) {
            const size_t bsmem = (size_t)L.big_max_smem;
            b.smem_bytes = (int32_t)bsmem;
            if (bsmem > kMaxSmem) return fail(net, MM_ENOTSUP, "a large work item needs more shared memory than a block has");
            int bper = 0;
            MM_CKI(net, mmk_step_fp32c_blocks_per_sm(kBigThreads, (int)bsmem, &bper));
            if (bper < 1) return fail(net, MM_ENOTSUP, "the large-class step kernel does not fit on an SM");
            net->big_blocks = std::max(1, std::min(L.n_big, bper * sms));
            net->info.big_items = L.n_big;
            net->info.big_blocks = net->big_blocks;
            net->info.big_threads = kBigThreads;
            net->info.big_smem_bytes = (int32_t)bsmem;
            net->info.max_big_item_comps = L.big_max_comps;
            if (threads == kBigThreads) {  // one kernel instance: its limit must cover both classes
                int tmp = 0;
                MM_CKI(net, mmk_step_fp32c_blocks_per_sm(threads, (int)std::max(smem, bsmem), &tmp));
            }
        }
        mmk::StepArgs32 &g = net->sa32g;
        g = net->sa32;
        g.item0 = L.n_small + L.n_big;
        g.item1 = (int32_t)L.groups.size();
        g.queue = &net->ctl->giant_head;
        // the giant items' compartments in chunks for the assembly and
        // update kernels: first chunk of each giant item, then the total
        std::vector<int64_t> gch(1, 0);
        for (int32_t gi = g.item0; gi < g.item1; ++gi) {
            const int64_t nc = L.groups[(size_t)gi].ncomp;
            gch.push_back(gch.back() + (nc + mmk_giant_chunk() - 1) / mmk_giant_chunk());
        }
        int64_t *dgch = nullptr;
        if ((st = upload(net, &dgch, gch.data(), gch.size())) != MM_OK) return st;
        g.gchunk0 = dgch;
        net->giant_chunk_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(gch.back(), 4 * (int64_t)sms));
    }
    net->info.work_items = (int32_t)L.groups.size();
    net->info.blocks = net->step_blocks;
    net->info.threads = threads;
    net->info.blocks_per_sm = per_sm;
    net->info.smem_bytes = (int32_t)smem;
    net->info.max_item_comps = L.max_comps;
    net->info.max_item_segments = L.max_segs;
    net->info.max_item_waves = L.max_waves;
    net->info.giant_items = net->n_giant;
    for (size_t gi = 0; gi < L.groups.size(); ++gi) {
        const int cls = (int32_t)gi < L.n_small ? 0 : ((int32_t)gi < L.n_small + L.n_big ? 1 : 2);
        net->info.comps[cls] += L.groups[gi].ncomp;
        net->info.sites[cls] += L.groups[gi].nsite;
    }
    net->deliver_blocks = std::max(1, 2 * sms);
    net->ordered_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((net->nsite + 255) / 256, 16 * (int64_t)sms));
    MM_CK(net, cudaStreamSynchronize(net->stream));
    return MM_OK;
}

}  // namespace

extern "C" {

void mm_default_options(mm_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = MM_FP64;
    opt->schedule = MM_SCHED_SIZE_SORTED;
    opt->graph_steps = 40;
    opt->dt_ms = 0.025;
}

// the message of this thread's last failed mm_create_network (mm_last_error(NULL))
static thread_local std::string g_create_error;

mm_status mm_create_network(const mm_morphologies *morph, const mm_channel_params *chan, const mm_synapses *syn,
                            const double *stim_nA, const mm_options *opt, mm_net **out)
{
    if (!out) return MM_EINVAL;
    *out = nullptr;
    if (!morph || !chan) return MM_EINVAL;
    mm_options defaults;
    mm_default_options(&defaults);
    if (!opt) opt = &defaults;
    mm_net *net = new (std::nothrow) mm_net();
    if (!net) return MM_ENOMEM;
    mm_status st = build(net, morph, chan, syn, stim_nA, opt);
    if (st != MM_OK) {
        g_create_error = net->err;
        release_all(net);
        delete net;
        return st;
    }
    *out = net;
    return MM_OK;
}

mm_status mm_step(mm_net *net, int64_t n_steps, double dt_ms)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (n_steps < 0) return fail(net, MM_EINVAL, "n_steps must be >= 0");
    if (!(dt_ms == net->dt)) return fail(net, MM_EINVAL, "dt differs from the network's dt");
    while (!net->timing && net->graph_steps > 0 && n_steps >= net->graph_steps) {
        if ((st = ensure_graph(net, net->graph_steps, &net->gexec)) != MM_OK) return st;
        MM_CK(net, cudaGraphLaunch(net->gexec, net->stream));
        n_steps -= net->graph_steps;
        net->steps_done += net->graph_steps;
    }
    // the remainder (fewer steps than one graph) replays the one-step graph
    while (!net->timing && net->graph_steps > 0 && n_steps > 0) {
        if ((st = ensure_graph(net, 1, &net->gexec1)) != MM_OK) return st;
        MM_CK(net, cudaGraphLaunch(net->gexec1, net->stream));
        n_steps -= 1;
        net->steps_done += 1;
    }
    while (n_steps > 0) {
        const int k = (int)std::min<int64_t>(n_steps, 1 << 20);
        if ((st = launch_steps(net, net->stream, k)) != MM_OK) return st;
        n_steps -= k;
        net->steps_done += k;
    }
    return MM_OK;
}

mm_status mm_synchronize(mm_net *net)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    return check_device(net);
}

mm_status mm_read_state(mm_net *net, int32_t which, double *out, int64_t cap)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!out || cap < net->C) return fail(net, MM_EINVAL, "output buffer too small");
    if (which < MM_STATE_V || which > MM_STATE_GSYN) return fail(net, MM_EINVAL, "unknown state quantity");
    // dense internal-order values in the second half of the scratch, then a
    // gather into user order in its first half
    double *dense = net->scratch + std::max<int64_t>(net->C, net->N);
    const double *src = nullptr;
    if (net->precision == MM_FP64) {
        switch (which) {
        case MM_STATE_V: src = net->V; break;
        case MM_STATE_M: src = net->m; break;
        case MM_STATE_H: src = net->h; break;
        case MM_STATE_N: src = net->n; break;
        default:
            MM_CKI(net, mmk_launch_fill_f64(dense, 0.0, net->C, net->stream));
            MM_CKI(net, mmk_launch_scatter_f64(net->gsyn, net->site_internal, dense, net->nsite, net->stream));
            src = dense;
        }
    } else {
        switch (which) {
        case MM_STATE_V:
            MM_CKI(net, mmk_launch_vq_to_f64(net->Vq, dense, net->C, net->stream));
            // somata carry their FP64 accumulator
            MM_CKI(net, mmk_launch_scatter_f64(net->Vsoma, net->soma_internal, dense, net->N, net->stream));
            break;
        case MM_STATE_M: MM_CKI(net, mmk_launch_gq_to_f64(net->mq, dense, net->C, net->stream)); break;
        case MM_STATE_H: MM_CKI(net, mmk_launch_gq_to_f64(net->hq, dense, net->C, net->stream)); break;
        case MM_STATE_N: MM_CKI(net, mmk_launch_gq_to_f64(net->nq, dense, net->C, net->stream)); break;
        default:
            MM_CKI(net, mmk_launch_fill_f64(dense, 0.0, net->C, net->stream));
            MM_CKI(net, mmk_launch_scatter_f2_to_f64(net->gsyn2, net->site_internal, dense, net->nsite, net->stream));
        }
        src = dense;
    }
    MM_CKI(net, mmk_launch_gather_f64(src, net->user2int, net->scratch, net->C, net->stream));
    MM_CK(net, cudaMemcpyAsync(out, net->scratch, (size_t)net->C * sizeof(double), cudaMemcpyDeviceToHost, net->stream));
    return check_device(net);
}

mm_status mm_read_voltages(mm_net *net, double *out, int64_t cap) { return mm_read_state(net, MM_STATE_V, out, cap); }

mm_status mm_read_soma_voltages(mm_net *net, double *out, int64_t cap)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!out || cap < net->N) return fail(net, MM_EINVAL, "output buffer too small");
    const size_t bytes = (size_t)net->N * sizeof(double);
    if ((st = pinned(net, bytes)) != MM_OK) return st;
    if (net->precision == MM_FP64)
        MM_CKI(net, mmk_launch_gather_f64(net->V, net->soma_of_user, net->scratch, net->N, net->stream));
    else
        MM_CKI(net, mmk_launch_gather_f64(net->Vsoma, net->internal_of64, net->scratch, net->N, net->stream));
    MM_CK(net, cudaMemcpyAsync(net->pin, net->scratch, bytes, cudaMemcpyDeviceToHost, net->stream));
    if ((st = check_device(net)) != MM_OK) return st;
    std::memcpy(out, net->pin, bytes);
    return MM_OK;
}

namespace {
constexpr int64_t kSpikePrefetch = 4096;  // spike records copied with the soma voltages

// Drains the spike buffer given the control block snapshot c (taken after
// the stream synchronised); `pre` records (pre <= c.spk_count) already sit
// in the pinned buffer at pin_off as times, neurons, compartments.
mm_status drain_spikes(mm_net *net, mmk::DevCtl c, size_t pin_off, int64_t pre, int32_t *neuron, int32_t *comp,
                       double *t_ms, int64_t cap, int64_t *n_out)
{
    mm_status st;
    const int64_t held = std::min<int64_t>((int64_t)c.spk_count, net->spk_cap);
    const int32_t *nr = nullptr, *cp = nullptr;
    const double *tt = nullptr;
    if (held) {
        // times, neurons, compartments; the records not prefetched are copied now
        const size_t bt = (size_t)held * sizeof(double), bi = (size_t)held * sizeof(int32_t);
        if (held > pre) {
            if ((st = pinned(net, bt + 2 * bi)) != MM_OK) return st;
            pin_off = 0;
            MM_CK(net, cudaMemcpyAsync(net->pin, net->spk_t, bt, cudaMemcpyDeviceToHost, net->stream));
            MM_CK(net, cudaMemcpyAsync(net->pin + bt, net->spk_nrn, bi, cudaMemcpyDeviceToHost, net->stream));
            MM_CK(net, cudaMemcpyAsync(net->pin + bt + bi, net->spk_comp, bi, cudaMemcpyDeviceToHost, net->stream));
            MM_CK(net, cudaStreamSynchronize(net->stream));
            tt = (const double *)net->pin;
            nr = (const int32_t *)(net->pin + bt);
            cp = (const int32_t *)(net->pin + bt + bi);
        } else {
            const size_t pt = (size_t)pre * sizeof(double), pi = (size_t)pre * sizeof(int32_t);
            tt = (const double *)(net->pin + pin_off);
            nr = (const int32_t *)(net->pin + pin_off + pt);
            cp = (const int32_t *)(net->pin + pin_off + pt + pi);
        }
    }
    // order by (t, neuron, comp) as two unsigned keys: the bits of t mapped
    // to an order-preserving integer, then neuron and compartment
    struct Rec {
        uint64_t tk, nc;
        double t;
    };
    std::vector<Rec> rec((size_t)held);
    for (int64_t i = 0; i < held; ++i) {
        uint64_t b;
        std::memcpy(&b, &tt[i], sizeof(b));
        b = (b >> 63) ? ~b : (b | (1ull << 63));
        rec[(size_t)i] = {b, ((uint64_t)(uint32_t)nr[i] << 32) | (uint32_t)cp[i], tt[i]};
    }
    std::sort(rec.begin(), rec.end(), [](const Rec &a, const Rec &b) { return a.tk != b.tk ? a.tk < b.tk : a.nc < b.nc; });
    const int64_t w = std::min<int64_t>(held, cap);
    for (int64_t i = 0; i < w; ++i) {
        const Rec &r = rec[(size_t)i];
        neuron[i] = (int32_t)(r.nc >> 32);
        if (comp) comp[i] = (int32_t)(uint32_t)r.nc;
        t_ms[i] = r.t;
    }
    *n_out = held;
    const bool overflow = (c.err & mmk::MMK_ERR_OVERFLOW) != 0 || (int64_t)c.spk_count > net->spk_cap;
    // drain: reset the count and the overflow bit (the device is idle since
    // the synchronisation above; the write is ordered before later steps)
    c.spk_count = 0;
    c.err &= ~mmk::MMK_ERR_OVERFLOW;
    *net->pin_ctl_w = c;
    MM_CK(net, cudaMemcpyAsync(net->ctl, net->pin_ctl_w, sizeof(mmk::DevCtl), cudaMemcpyHostToDevice, net->stream));
    if (overflow) return fail(net, MM_EOVERFLOW, "spike buffer overflowed; raise mm_options.spike_capacity or read more often");
    if (w < held) return fail(net, MM_EOVERFLOW, "caller's spike arrays are smaller than the spike count");
    return MM_OK;
}
}  // namespace

mm_status mm_read_spike_points(mm_net *net, int32_t *neuron, int32_t *comp, double *t_ms, int64_t cap,
                               int64_t *n_out)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!n_out || cap < 0 || (cap > 0 && (!neuron || !t_ms))) return fail(net, MM_EINVAL, "bad spike output arguments");
    if ((st = check_device(net)) != MM_OK) return st;
    return drain_spikes(net, *net->pin_ctl, 0, 0, neuron, comp, t_ms, cap, n_out);
}

mm_status mm_read_outputs(mm_net *net, double *soma, int64_t soma_cap, int32_t *neuron, int32_t *comp,
                          double *t_ms, int64_t cap, int64_t *n_out)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!soma || soma_cap < net->N) return fail(net, MM_EINVAL, "output buffer too small");
    if (!n_out || cap < 0 || (cap > 0 && (!neuron || !t_ms))) return fail(net, MM_EINVAL, "bad spike output arguments");
    // one batch: soma voltages, the first records of the spike buffer, the
    // control block; one synchronisation
    const size_t bs = (size_t)net->N * sizeof(double);
    const int64_t pre = std::min<int64_t>(kSpikePrefetch, net->spk_cap);
    const size_t soff = (bs + 15) / 16 * 16;
    const size_t pt = (size_t)pre * sizeof(double), pi = (size_t)pre * sizeof(int32_t);
    if ((st = pinned(net, soff + pt + 2 * pi)) != MM_OK) return st;
    if (net->precision == MM_FP64)
        MM_CKI(net, mmk_launch_gather_f64(net->V, net->soma_of_user, net->scratch, net->N, net->stream));
    else
        MM_CKI(net, mmk_launch_gather_f64(net->Vsoma, net->internal_of64, net->scratch, net->N, net->stream));
    MM_CK(net, cudaMemcpyAsync(net->pin, net->scratch, bs, cudaMemcpyDeviceToHost, net->stream));
    MM_CK(net, cudaMemcpyAsync(net->pin + soff, net->spk_t, pt, cudaMemcpyDeviceToHost, net->stream));
    MM_CK(net, cudaMemcpyAsync(net->pin + soff + pt, net->spk_nrn, pi, cudaMemcpyDeviceToHost, net->stream));
    MM_CK(net, cudaMemcpyAsync(net->pin + soff + pt + pi, net->spk_comp, pi, cudaMemcpyDeviceToHost, net->stream));
    if ((st = check_device(net)) != MM_OK) return st;
    std::memcpy(soma, net->pin, bs);
    return drain_spikes(net, *net->pin_ctl, soff, pre, neuron, comp, t_ms, cap, n_out);
}

mm_status mm_read_spikes(mm_net *net, int32_t *neuron, double *t_ms, int64_t cap, int64_t *n_out)
{
    return mm_read_spike_points(net, neuron, nullptr, t_ms, cap, n_out);
}

mm_status mm_set_stimulus(mm_net *net, const double *stim_nA, int64_t n)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!stim_nA || n != net->N) return fail(net, MM_EINVAL, "stimulus must have n_neurons entries");
    for (int32_t k = 0; k < net->N; ++k)
        if (!std::isfinite(stim_nA[k])) return fail(net, MM_EINVAL, "stimulus must be finite");
    // the staging buffer is rewritten once its last upload has run; the
    // upload is ordered on the stream before every later step
    MM_CK(net, cudaEventSynchronize(net->ev_stim));
    for (int32_t k = 0; k < net->N; ++k) net->pin_stim[k] = stim_nA[net->order[(size_t)k]];
    MM_CK(net, cudaMemcpyAsync(net->stim, net->pin_stim, (size_t)net->N * sizeof(double), cudaMemcpyHostToDevice,
                               net->stream));
    MM_CK(net, cudaEventRecord(net->ev_stim, net->stream));
    return MM_OK;
}

mm_status mm_get_step(const mm_net *net, int64_t *step)
{
    if (!net || !step) return MM_EINVAL;
    *step = net->steps_done;
    return MM_OK;
}

mm_status mm_selftest_bounded_wait(int32_t device, uint32_t max_polls)
{
    if (max_polls < 1 || max_polls > (1u << 20)) return MM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return MM_ECUDA;
    }
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return MM_ENOMEM;
    }
    int h = 0;
    mm_status st = MM_OK;
    if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess || mmk_launch_wait_selftest(err, max_polls, nullptr) != 0 ||
        cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = MM_ECUDA;
    cudaFree(err);
    if (st != MM_OK) {
        cudaGetLastError();
        return st;
    }
    return (h & mmk::MMK_ERR_TIMEOUT) ? MM_ETIMEOUT : MM_OK;
}

mm_status mm_inject_spikes(mm_net *net, int64_t n, const int32_t *ext_src, const int64_t *step)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (n < 0 || (n > 0 && (!ext_src || !step))) return fail(net, MM_EINVAL, "bad spike arrays");
    if (n == 0) return MM_OK;
    if (net->n_ext <= 0) return fail(net, MM_EINVAL, "the network has no external spike sources");
    const int64_t now = net->steps_done;
    std::vector<std::pair<int64_t, int32_t>> seen((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        if (ext_src[k] < 0 || ext_src[k] >= net->n_ext) return fail(net, MM_EINVAL, "external source out of range");
        if (step[k] < 0 || step[k] >= now) return fail(net, MM_EINVAL, "a spike's step has not run yet");
        if (step[k] + 1 + net->min_dsteps < now)
            return fail(net, MM_EINVAL, "a spike handed in after its earliest delivery step");
        seen[(size_t)k] = {step[k], ext_src[k]};
    }
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
        return fail(net, MM_EINVAL, "a source spikes twice in one step");
    if (n > net->inj_cap) {
        MM_CK(net, cudaStreamSynchronize(net->stream));
        dev_free(net, net->inj_src);
        dev_free(net, net->inj_step);
        net->inj_src = nullptr;
        net->inj_step = nullptr;
        net->inj_cap = 0;
        const int64_t cap = std::max<int64_t>(n, 4096);
        net->inj_src = (int32_t *)dev_alloc(net, (size_t)cap * sizeof(int32_t));
        net->inj_step = (int64_t *)dev_alloc(net, (size_t)cap * sizeof(int64_t));
        if (!net->inj_src || !net->inj_step) return fail(net, MM_ENOMEM, "device allocation failed");
        net->inj_cap = cap;
    }
    // pinned staging (the copies are ordered on the stream; the staging is
    // reused only after a synchronisation)
    const size_t bs = (size_t)n * sizeof(int32_t), bt = (size_t)n * sizeof(int64_t);
    if ((st = pinned(net, bs + bt + 16)) != MM_OK) return st;
    MM_CK(net, cudaStreamSynchronize(net->stream));
    std::memcpy(net->pin, step, bt);
    std::memcpy(net->pin + bt, ext_src, bs);
    MM_CK(net, cudaMemcpyAsync(net->inj_step, net->pin, bt, cudaMemcpyHostToDevice, net->stream));
    MM_CK(net, cudaMemcpyAsync(net->inj_src, net->pin + bt, bs, cudaMemcpyHostToDevice, net->stream));
    MM_CKI(net, mmk_launch_inject(net->ring_nrn, net->ring_cnt, net->R, std::max(net->n_src, 1), net->N,
                                  net->fired, net->fired_words, net->inj_src, net->inj_step, n, net->ctl,
                                  net->stream));
    MM_CK(net, cudaStreamSynchronize(net->stream));
    return MM_OK;
}

mm_status mm_read_fired(mm_net *net, int64_t step0, int32_t n_steps, int32_t *neuron, int64_t *step, int64_t cap,
                        int64_t *n_out)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!n_out || n_steps < 0 || cap < 0 || (cap > 0 && (!neuron || !step))) return fail(net, MM_EINVAL, "bad arguments");
    if (net->detect != MM_DETECT_SOMA) return fail(net, MM_EINVAL, "mm_read_fired needs MM_DETECT_SOMA");
    *n_out = 0;
    const int64_t now = net->steps_done;
    if (step0 < 0 || step0 + n_steps > now || step0 < now - (net->R - 1))
        return fail(net, MM_EINVAL, "steps outside those run and still held in the spike ring");
    if (n_steps == 0) return MM_OK;
    const int32_t Ns = std::max(net->n_src, 1);
    std::vector<int32_t> cnt((size_t)net->R);
    MM_CK(net, cudaStreamSynchronize(net->stream));
    MM_CK(net, cudaMemcpy(cnt.data(), net->ring_cnt, (size_t)net->R * sizeof(int32_t), cudaMemcpyDeviceToHost));
    int64_t total = 0;
    std::vector<int32_t> ids;
    for (int64_t m = step0; m < step0 + n_steps; ++m) {
        const int slot = (int)(m % net->R);
        const int32_t c = std::min(cnt[(size_t)slot], Ns);
        ids.resize((size_t)c);
        if (c > 0)
            MM_CK(net, cudaMemcpy(ids.data(), net->ring_nrn + (int64_t)slot * Ns, (size_t)c * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost));
        std::vector<int32_t> own;
        for (int32_t id : ids)
            if (id >= 0 && id < net->N) own.push_back(net->order[(size_t)id]);
        std::sort(own.begin(), own.end());
        for (int32_t u : own) {
            if (total < cap) {
                neuron[total] = u;
                step[total] = m;
            }
            ++total;
        }
    }
    *n_out = total;
    if (total > cap) return fail(net, MM_EOVERFLOW, "caller's arrays are smaller than the spike count");
    return MM_OK;
}

// Checkpoint blob: a header, then every dynamic device array of the
// network's precision, the stimulus, the spike ring, the control block and
// the undrained spikes, in a fixed order.
namespace {
struct CkptHeader {
    char magic[8];
    int64_t C, nsite, N, R, spk_cap, steps_done;
    int32_t precision, n_src;
};

std::vector<std::pair<void *, size_t>> ckpt_regions(mm_net *net)
{
    std::vector<std::pair<void *, size_t>> r;
    const size_t C = (size_t)net->C, N = (size_t)net->N, ns = (size_t)net->nsite;
    if (net->precision == MM_FP64) {
        r.push_back({net->V, C * sizeof(double)});
        r.push_back({net->m, C * sizeof(double)});
        r.push_back({net->h, C * sizeof(double)});
        r.push_back({net->n, C * sizeof(double)});
        r.push_back({net->gsyn, ns * sizeof(double)});
    } else {
        r.push_back({net->Vq, C * sizeof(int32_t)});
        r.push_back({net->mq, C * sizeof(uint32_t)});
        r.push_back({net->hq, C * sizeof(uint32_t)});
        r.push_back({net->nq, C * sizeof(uint32_t)});
        r.push_back({net->Vsoma, N * sizeof(double)});
        r.push_back({net->gsyn2, ns * sizeof(float2)});
    }
    r.push_back({net->stim, N * sizeof(double)});
    r.push_back({net->ring_cnt, (size_t)net->R * sizeof(int32_t)});
    r.push_back({net->ring_nrn, (size_t)net->R * (size_t)std::max(net->n_src, 1) * sizeof(int32_t)});
    r.push_back({net->ctl, sizeof(mmk::DevCtl)});
    r.push_back({net->spk_nrn, (size_t)net->spk_cap * sizeof(int32_t)});
    r.push_back({net->spk_comp, (size_t)net->spk_cap * sizeof(int32_t)});
    if (net->fired) r.push_back({net->fired, (size_t)net->R * (size_t)net->fired_words * sizeof(uint32_t)});
    r.push_back({net->spk_t, (size_t)net->spk_cap * sizeof(double)});
    return r;
}

size_t ckpt_size(mm_net *net)
{
    size_t s = sizeof(CkptHeader);
    for (auto &r : ckpt_regions(net)) s += r.second;
    return s;
}
}  // namespace

mm_status mm_save_state(mm_net *net, void *buf, size_t cap, size_t *len)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!len) return fail(net, MM_EINVAL, "len must not be NULL");
    const size_t need = ckpt_size(net);
    *len = need;
    if (!buf) return MM_OK;
    if (cap < need) return fail(net, MM_EINVAL, "checkpoint buffer too small");
    if ((st = check_device(net)) != MM_OK) return st;
    char *p = (char *)buf;
    CkptHeader h{};
    std::memcpy(h.magic, "MMCKPT03", 8);
    h.C = net->C;
    h.nsite = net->nsite;
    h.N = net->N;
    h.R = net->R;
    h.spk_cap = net->spk_cap;
    h.steps_done = net->steps_done;
    h.precision = net->precision;
    h.n_src = net->n_src;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    for (auto &r : ckpt_regions(net)) {
        MM_CK(net, cudaMemcpy(p, r.first, r.second, cudaMemcpyDeviceToHost));
        p += r.second;
    }
    return MM_OK;
}

mm_status mm_load_state(mm_net *net, const void *buf, size_t len)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!buf || len != ckpt_size(net)) return fail(net, MM_EINVAL, "checkpoint size does not match this network");
    const char *p = (const char *)buf;
    CkptHeader h;
    std::memcpy(&h, p, sizeof(h));
    if (std::memcmp(h.magic, "MMCKPT03", 8) != 0 || h.C != net->C || h.nsite != net->nsite || h.N != net->N ||
        h.R != net->R || h.spk_cap != net->spk_cap || h.precision != net->precision || h.n_src != net->n_src)
        return fail(net, MM_EINVAL, "checkpoint was saved from a different network");
    p += sizeof(h);
    MM_CK(net, cudaStreamSynchronize(net->stream));
    for (auto &r : ckpt_regions(net)) {
        MM_CK(net, cudaMemcpy(r.first, p, r.second, cudaMemcpyHostToDevice));
        p += r.second;
    }
    net->steps_done = h.steps_done;
    return MM_OK;
}

mm_status mm_set_kernel_timing(mm_net *net, int32_t enable)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    net->timing = enable != 0;
    return MM_OK;
}

mm_status mm_read_kernel_timing(mm_net *net, mm_kernel_times *out, int32_t reset)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!out) return fail(net, MM_EINVAL, "out must not be NULL");
    if ((st = collect_timing(net)) != MM_OK) return st;
    *out = net->times;
    if (reset) net->times = mm_kernel_times{};
    return MM_OK;
}

mm_status mm_neuron_features(const mm_morphologies *morph, float *out, int64_t cap)
{
    if (!morph || !out || morph->n_neurons < 1 || !morph->comp_offset || !morph->parent || !morph->length_um ||
        !morph->diam_um)
        return MM_EINVAL;
    const int32_t N = morph->n_neurons;
    if (cap < (int64_t)N * MM_N_FEATURES) return MM_EINVAL;
    if (morph->comp_offset[0] != 0) return MM_EINVAL;
    for (int32_t k = 0; k < N; ++k) {
        const int64_t b = morph->comp_offset[k], n = morph->comp_offset[k + 1] - b;
        if (n < 1 || n > INT32_MAX / 2 || morph->parent[b] != -1) return MM_EINVAL;
        for (int64_t i = 1; i < n; ++i)
            if (morph->parent[b + i] < 0 || morph->parent[b + i] >= i) return MM_EINVAL;
        for (int64_t i = 0; i < n; ++i)
            if (!(morph->length_um[b + i] > 0.0) || !(morph->diam_um[b + i] > 0.0)) return MM_EINVAL;
    }
    try {
        for (int32_t k = 0; k < N; ++k) {
            const int64_t b = morph->comp_offset[k];
            mmh::neuron_features((int32_t)(morph->comp_offset[k + 1] - b), morph->parent + b, morph->length_um + b,
                                 morph->diam_um + b, out + (int64_t)k * MM_N_FEATURES);
        }
    } catch (const std::bad_alloc &) {
        return MM_ENOMEM;
    }
    return MM_OK;
}

mm_status mm_read_neuron_times(mm_net *net, double *out_us, int64_t cap)
{
    mm_status st = guard(net);
    if (st != MM_OK) return st;
    if (!out_us || cap < net->N) return fail(net, MM_EINVAL, "output buffer too small");
    if (!net->item_ns) return fail(net, MM_EINVAL, "the network was created without time_items");
    for (int32_t k : net->item_nneuron)
        if (k != 1) return fail(net, MM_EINVAL, "neuron times need one neuron per work item (group_comps = 1)");
    if ((st = check_device(net)) != MM_OK) return st;
    std::vector<unsigned long long> ns(net->item_neuron0.size());
    MM_CK(net, cudaMemcpy(ns.data(), net->item_ns, ns.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    const double steps = (double)std::max<int64_t>(1, net->steps_done);
    for (size_t i = 0; i < ns.size(); ++i)
        out_us[net->order[(size_t)net->item_neuron0[i]]] = (double)ns[i] * 1e-3 / steps;
    return MM_OK;
}

mm_status mm_get_launch_info(const mm_net *net, mm_launch_info *out)
{
    if (!net || !out) return MM_EINVAL;
    *out = net->info;
    return MM_OK;
}

const char *mm_last_error(const mm_net *net)
{
    if (!net) return g_create_error.c_str();
    return net->err.c_str();
}

const char *mm_status_string(mm_status s)
{
    switch (s) {
    case MM_OK: return "MM_OK";
    case MM_EINVAL: return "MM_EINVAL";
    case MM_ENOMEM: return "MM_ENOMEM";
    case MM_ECUDA: return "MM_ECUDA";
    case MM_ETIMEOUT: return "MM_ETIMEOUT";
    case MM_ENUMERIC: return "MM_ENUMERIC";
    case MM_EOVERFLOW: return "MM_EOVERFLOW";
    case MM_ESTATE: return "MM_ESTATE";
    case MM_ENOTSUP: return "MM_ENOTSUP";
    }
    return "MM_UNKNOWN";
}

void mm_destroy(mm_net *net)
{
    if (!net) return;
    cudaSetDevice(net->device);
    release_all(net);
    delete net;
}

}  // extern "C"

// mm_tune.cpp -- launch-configuration autotuner of the per-step kernel.
//
// The block shape (threads per block) and the work-item size (compartment
// budget of one item) of the persistent step kernel trade occupancy against
// the length of each item's serial elimination chain, and the best pair
// depends on the size distribution of the network.  The tuner measures
// instead of guessing: it builds a stratified sample of the network, runs
// every candidate pair on it through the public API and keeps the fastest.
// The paper balances its tasks by size only (Sec. 4); it has no tuner.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "mm.h"

namespace {

struct Sample {
    std::vector<int64_t> off;
    std::vector<int32_t> parent;
    std::vector<double> L, d, stim;
    std::vector<float> cost;
    std::vector<int32_t> src, dst, dcomp, scomp;
    std::vector<double> w, delay;
};

// Every k-th neuron in size order (k chosen so that the sample holds about
// `target` compartments), kept in their original relative order, with the
// synapses whose source and target are both in the sample.
void make_sample(const mm_morphologies *m, const mm_synapses *syn, const double *stim, const float *cost,
                 int64_t target, Sample &s)
{
    const int32_t N = m->n_neurons;
    const int64_t C = m->comp_offset[N];
    std::vector<int32_t> order((size_t)N);
    std::iota(order.begin(), order.end(), 0);
    auto size = [&](int32_t k) { return m->comp_offset[k + 1] - m->comp_offset[k]; };
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return size(a) > size(b); });
    const int64_t k = std::max<int64_t>(1, (C + target - 1) / std::max<int64_t>(target, 1));
    std::vector<int32_t> pick;
    for (int64_t r = 0; r < N; r += k) pick.push_back(order[(size_t)r]);
    std::sort(pick.begin(), pick.end());
    std::vector<int32_t> newid((size_t)N, -1);
    for (size_t i = 0; i < pick.size(); ++i) newid[(size_t)pick[i]] = (int32_t)i;
    s.off.assign(1, 0);
    for (int32_t u : pick) {
        const int64_t b = m->comp_offset[u], e = m->comp_offset[u + 1];
        for (int64_t i = b; i < e; ++i) {
            s.parent.push_back(m->parent[i]);
            s.L.push_back(m->length_um[i]);
            s.d.push_back(m->diam_um[i]);
        }
        s.off.push_back(s.off.back() + (e - b));
        s.stim.push_back(stim ? stim[u] : 0.0);
        if (cost) s.cost.push_back(cost[u]);
    }
    if (syn) {
        for (int64_t q = 0; q < syn->n; ++q) {
            const int32_t a = syn->src_neuron[q], b = syn->dst_neuron[q];
            if (a < 0 || a >= N || b < 0 || b >= N || newid[(size_t)a] < 0 || newid[(size_t)b] < 0) continue;
            s.src.push_back(newid[(size_t)a]);
            s.dst.push_back(newid[(size_t)b]);
            s.dcomp.push_back(syn->dst_comp[q]);
            if (syn->src_comp) s.scomp.push_back(syn->src_comp[q]);
            s.w.push_back(syn->weight_uS[q]);
            s.delay.push_back(syn->delay_ms[q]);
        }
    }
}

}  // namespace

extern "C" mm_status mm_autotune(const mm_morphologies *morph, const mm_channel_params *chan,
                                 const mm_synapses *syn, const double *stim_nA, const mm_options *opt,
                                 int64_t sample_comps, int32_t warmup, int32_t steps, mm_tune_point *points,
                                 int32_t cap, int32_t *n_points, mm_options *best)
{
    if (!morph || !chan || !opt || !best || !n_points || steps < 1 || warmup < 0 || sample_comps < 1 ||
        cap < 0 || (cap > 0 && !points))
        return MM_EINVAL;
    if (morph->n_neurons < 1 || !morph->comp_offset || !morph->parent || !morph->length_um || !morph->diam_um)
        return MM_EINVAL;
    if (opt->precision != MM_FP64 && opt->precision != MM_FP32C) return MM_EINVAL;
    if (opt->n_ext_sources != 0) return MM_ENOTSUP;  // its sample keeps synapses among sampled neurons only
    if (opt->schedule == MM_SCHED_COST && !opt->cost) return MM_EINVAL;
    if (syn && syn->n > 0 && (!syn->src_neuron || !syn->dst_neuron || !syn->dst_comp || !syn->weight_uS ||
                              !syn->delay_ms))
        return MM_EINVAL;
    *n_points = 0;

    Sample s;
    make_sample(morph, syn, stim_nA, opt->schedule == MM_SCHED_COST ? opt->cost : nullptr, sample_comps, s);
    mm_morphologies sm{};
    sm.n_neurons = (int32_t)(s.off.size() - 1);
    sm.comp_offset = s.off.data();
    sm.parent = s.parent.data();
    sm.length_um = s.L.data();
    sm.diam_um = s.d.data();
    mm_synapses ss{};
    if (syn) {
        ss = *syn;
        ss.n = (int64_t)s.src.size();
        ss.src_neuron = s.src.data();
        ss.dst_neuron = s.dst.data();
        ss.dst_comp = s.dcomp.data();
        ss.src_comp = syn->src_comp ? s.scomp.data() : nullptr;
        ss.weight_uS = s.w.data();
        ss.delay_ms = s.delay.data();
    }

    if (cudaSetDevice(opt->device) != cudaSuccess) return MM_ECUDA;
    cudaStream_t stream = (cudaStream_t)opt->cuda_stream;
    bool own = false;
    if (!stream) {
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) return MM_ECUDA;
        own = true;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (own) cudaStreamDestroy(stream);
        return MM_ECUDA;
    }

    const bool f32 = opt->precision == MM_FP32C;
    const int32_t threads32[] = {256, 512, 1024}, threads64[] = {128, 256, 512};
    const int32_t budgets[] = {1024, 2048, 4096, 8192};
    double best_ms = -1.0;
    mm_status first_err = MM_OK;
    int32_t n = 0;
    for (int ti = 0; ti < 3; ++ti) {
        for (int32_t gc : budgets) {
            mm_options o = *opt;
            o.block_threads = f32 ? threads32[ti] : threads64[ti];
            o.group_comps = gc;
            o.cuda_stream = stream;
            o.time_items = 0;
            o.cost = opt->schedule == MM_SCHED_COST ? s.cost.data() : nullptr;
            mm_tune_point p{o.block_threads, gc, MM_OK, -1.0};
            mm_net *net = nullptr;
            mm_status st = mm_create_network(&sm, chan, syn ? &ss : nullptr, s.stim.data(), &o, &net);
            if (st == MM_OK && warmup > 0) st = mm_step(net, warmup, o.dt_ms);
            if (st == MM_OK) st = mm_synchronize(net);
            if (st == MM_OK) {
                float ms = 0.f;
                if (cudaEventRecord(e0, stream) != cudaSuccess) st = MM_ECUDA;
                if (st == MM_OK) st = mm_step(net, steps, o.dt_ms);
                if (st == MM_OK && cudaEventRecord(e1, stream) != cudaSuccess) st = MM_ECUDA;
                if (st == MM_OK && cudaEventSynchronize(e1) != cudaSuccess) st = MM_ECUDA;
                if (st == MM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = MM_ECUDA;
                if (st == MM_OK) st = mm_synchronize(net);
                if (st == MM_OK) p.ms_per_step = (double)ms / steps;
            }
            if (net) mm_destroy(net);
            p.status = st;
            if (st != MM_OK && first_err == MM_OK) first_err = st;
            if (st == MM_OK && (best_ms < 0.0 || p.ms_per_step < best_ms)) {
                best_ms = p.ms_per_step;
                *best = *opt;
                best->block_threads = p.block_threads;
                best->group_comps = gc;
            }
            if (n < cap) points[n] = p;
            ++n;
            // invalid network inputs fail every candidate alike
            if (st == MM_EINVAL) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (own) cudaStreamDestroy(stream);
                *n_points = std::min(n, cap);
                return MM_EINVAL;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (own) cudaStreamDestroy(stream);
    *n_points = std::min(n, cap);
    if (best_ms < 0.0) return first_err == MM_OK ? MM_ENOTSUP : first_err;
    return MM_OK;
}

// mm_schedule.cpp -- the learned work-queue order end to end (mm_train_schedule).
//
// The paper orders its OpenMP tasks by neuron size (priority(size), and a
// global sort by size, Sec. 4).  Here the key is learned: a sample of neurons
// is timed by the solve kernel itself (each neuron its own work item,
// %globaltimer per item), an MLP learns log time from morphology features,
// and its prediction for every neuron becomes mm_options.cost.  Everything
// below is host orchestration of the library's own entry points; the timing
// and the model run in its kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "mm.h"

namespace {

// splitmix64: the sample and the hold-out split are drawn from the caller's seed
struct Rng {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    // uniform in [0, n)
    uint64_t below(uint64_t n) { return n ? next() % n : 0; }
};

}  // namespace

extern "C" mm_status mm_train_schedule(const mm_morphologies *morph, const mm_channel_params *chan,
                                       const double *stim_nA, const mm_options *opt, int32_t n_timed,
                                       int32_t steps, int32_t epochs, float lr, uint64_t seed, float *cost,
                                       int64_t cap, mm_schedule_report *report)
{
    if (!morph || !chan || !opt || !cost || n_timed < 10 || steps < 1 || epochs < 1 || !(lr > 0.0f))
        return MM_EINVAL;
    if (morph->n_neurons < 1 || !morph->comp_offset || !morph->parent || !morph->length_um || !morph->diam_um)
        return MM_EINVAL;
    const int32_t N = morph->n_neurons;
    if (cap < N) return MM_EINVAL;

    // features of every neuron (validates the morphology)
    std::vector<float> feats((size_t)N * MM_N_FEATURES);
    mm_status st = mm_neuron_features(morph, feats.data(), (int64_t)feats.size());
    if (st != MM_OK) return st;

    // the timed sample: k distinct neurons (partial Fisher-Yates), ascending
    Rng rng{seed};
    const int32_t k = n_timed < N ? n_timed : N;
    std::vector<int32_t> perm((size_t)N);
    std::iota(perm.begin(), perm.end(), 0);
    for (int32_t i = 0; i < k; ++i) {
        const int32_t j = i + (int32_t)rng.below((uint64_t)(N - i));
        std::swap(perm[(size_t)i], perm[(size_t)j]);
    }
    std::vector<int32_t> pick(perm.begin(), perm.begin() + k);
    std::sort(pick.begin(), pick.end());

    // their morphologies as a network of their own, without synapses
    std::vector<int64_t> off(1, 0);
    std::vector<int32_t> parent;
    std::vector<double> L, D, stim;
    for (int32_t u : pick) {
        const int64_t b = morph->comp_offset[u], e = morph->comp_offset[u + 1];
        parent.insert(parent.end(), morph->parent + b, morph->parent + e);
        L.insert(L.end(), morph->length_um + b, morph->length_um + e);
        D.insert(D.end(), morph->diam_um + b, morph->diam_um + e);
        off.push_back(off.back() + (e - b));
        stim.push_back(stim_nA ? stim_nA[u] : 0.0);
    }
    mm_morphologies sm{};
    sm.n_neurons = k;
    sm.comp_offset = off.data();
    sm.parent = parent.data();
    sm.length_um = L.data();
    sm.diam_um = D.data();
    mm_options o;
    mm_default_options(&o);
    o.precision = MM_FP32C;
    o.group_comps = 1;      // every neuron its own work item
    o.time_items = 1;
    o.graph_steps = 0;
    o.device = opt->device;
    o.dt_ms = opt->dt_ms;
    o.cuda_stream = opt->cuda_stream;
    o.allocator = opt->allocator;
    mm_net *net = nullptr;
    if ((st = mm_create_network(&sm, chan, nullptr, stim.data(), &o, &net)) != MM_OK) return st;
    std::vector<double> t_us((size_t)k);
    st = mm_step(net, steps, o.dt_ms);
    if (st == MM_OK) st = mm_read_neuron_times(net, t_us.data(), k);
    mm_destroy(net);
    if (st != MM_OK) return st;

    // labels log(time); 20 % held out
    std::vector<float> y((size_t)k);
    double mean_t = 0.0;
    for (int32_t i = 0; i < k; ++i) {
        y[(size_t)i] = (float)std::log(std::max(t_us[(size_t)i], 1e-3));
        mean_t += t_us[(size_t)i];
    }
    std::vector<int32_t> order((size_t)k);
    std::iota(order.begin(), order.end(), 0);
    for (int32_t i = k - 1; i > 0; --i) std::swap(order[(size_t)i], order[(size_t)rng.below((uint64_t)i + 1)]);
    const int32_t n_test = (int32_t)std::lround(0.2 * k);
    std::vector<float> Xtr, ytr, Xte, yte;
    for (int32_t r = 0; r < k; ++r) {
        const int32_t i = order[(size_t)r];
        const float *f = feats.data() + (size_t)pick[(size_t)i] * MM_N_FEATURES;
        auto &X = r < n_test ? Xte : Xtr;
        X.insert(X.end(), f, f + MM_N_FEATURES);
        (r < n_test ? yte : ytr).push_back(y[(size_t)i]);
    }

    mm_mlp *mlp = nullptr;
    if ((st = mm_mlp_create(seed, &mlp)) != MM_OK) return st;
    std::vector<float> losses((size_t)epochs);
    std::vector<float> pred((size_t)N), pte(yte.size());
    st = mm_mlp_train(mlp, Xtr.data(), ytr.data(), (int64_t)ytr.size(), epochs, lr, losses.data());
    if (st == MM_OK) st = mm_mlp_predict(mlp, feats.data(), N, pred.data());
    if (st == MM_OK && n_test > 0) st = mm_mlp_predict(mlp, Xte.data(), n_test, pte.data());
    mm_mlp_destroy(mlp);
    if (st != MM_OK) return st;

    for (int32_t u = 0; u < N; ++u) cost[u] = std::exp(pred[(size_t)u]);
    if (report) {
        double r2 = 0.0;
        if (n_test > 1) {
            double mu = 0.0, ss = 0.0, se = 0.0;
            for (float v : yte) mu += v;
            mu /= n_test;
            for (int32_t i = 0; i < n_test; ++i) {
                ss += (yte[(size_t)i] - mu) * (yte[(size_t)i] - mu);
                se += (yte[(size_t)i] - pte[(size_t)i]) * (yte[(size_t)i] - pte[(size_t)i]);
            }
            r2 = ss > 0.0 ? 1.0 - se / ss : 0.0;
        }
        // the size-only baseline: log time = a log(size) + b fitted by least
        // squares on the training neurons, scored on the same hold-out
        double r2s = 0.0;
        if (n_test > 1) {
            auto lsz = [&](int32_t r) {
                const int32_t u = pick[(size_t)order[(size_t)r]];
                return std::log((double)(morph->comp_offset[u + 1] - morph->comp_offset[u]));
            };
            double sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
            const int32_t ntr = k - n_test;
            for (int32_t r = n_test; r < k; ++r) {
                const double x = lsz(r), yv = y[(size_t)order[(size_t)r]];
                sx += x;
                sy += yv;
                sxx += x * x;
                sxy += x * yv;
            }
            const double den = ntr * sxx - sx * sx;
            const double a = den != 0.0 ? (ntr * sxy - sx * sy) / den : 0.0, b = (sy - a * sx) / ntr;
            double mu = 0.0, ss = 0.0, se = 0.0;
            for (float v : yte) mu += v;
            mu /= n_test;
            for (int32_t r = 0; r < n_test; ++r) {
                const double yv = yte[(size_t)r], e = yv - (a * lsz(r) + b);
                ss += (yv - mu) * (yv - mu);
                se += e * e;
            }
            r2s = ss > 0.0 ? 1.0 - se / ss : 0.0;
        }
        report->n_timed = k;
        report->n_holdout = n_test;
        report->r2_holdout = r2;
        report->r2_holdout_size_only = r2s;
        report->final_loss = losses.back();
        report->mean_time_us = mean_t / k;
    }
    return MM_OK;
}

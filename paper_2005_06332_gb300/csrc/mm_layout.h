// mm_layout.h -- host-side construction of the device layout of a network.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "mm_internal.h"

namespace mmh {

struct LayoutInput {
    int32_t N;
    const int64_t *comp_offset;
    const int32_t *parent;
    const double *length_um, *diam_um;
    int64_t S;
    const int32_t *src, *dst, *dcomp;
    // sources outside the network: src values N .. N + n_ext - 1 (soma
    // detection only); their spike source ids are the same values
    int32_t n_ext;
    const double *w, *delay_ms;
    // threshold tests at the synapse points (distinct (src, scomp) pairs;
    // scomp NULL: every synapse leaves from the soma) instead of the somata
    bool points;
    const int32_t *scomp;
    const double *stim;           // may be NULL
    const float *cost;            // may be NULL (size order)
    double dt;
    int32_t group_comps;          // compartment budget of a work item
    int32_t max_group_comps;      // largest neuron accepted
    // shared-memory model of a work item, bytes = meta + smem_per_comp * comps
    // + smem_per_seg * segments (+ smem_per_path * paths for path items);
    // items above giant_smem_limit go to the large shared-memory class if
    // they fit big_smem_limit (0: no such class), else they become giant
    // items (giant_smem_limit 0: no classes at all)
    int32_t smem_per_comp, smem_per_seg, giant_smem_limit, big_smem_limit;
    // FP32c: items are solved path by path (mmk::NrnQ tables with 16-bit
    // records, mmk::NrnG with 32-bit records for giant items), with
    // smem_per_path bytes per path
    bool path_items;
    int32_t smem_per_path;
};

struct Layout {
    int32_t N = 0;
    int64_t C = 0;
    std::vector<int32_t> order;         // internal neuron -> user neuron
    std::vector<int32_t> internal_of;   // user neuron -> internal neuron
    std::vector<int64_t> noff;          // internal compartment offset of each internal neuron [N+1]
    std::vector<int64_t> user2int;      // user compartment -> internal compartment [C]
    std::vector<int64_t> soma_of_user;  // internal soma compartment of each user neuron [N]
    std::vector<double> L, D;           // cylinders, internal order
    std::vector<int32_t> pdist;         // i - parent(i) in internal order, negated at segment tops (FP64)
                                        // or path heads (FP32c), 0 at somata
    std::vector<double> stim;           // internal order
    std::vector<mmk::GroupRec> groups;
    std::vector<unsigned char> meta;    // tree blobs (16-byte aligned per work item)
    int32_t max_comps = 0, max_segs = 0;
    int32_t max_waves = 0, max_meta = 0;
    // items [0, n_small) fit the regular shared-memory budget, the next n_big
    // the large one; the rest are giants
    int32_t n_small = 0, n_big = 0;
    int32_t big_max_comps = 0, big_max_segs = 0, big_max_meta = 0;
    // largest shared-memory need (model above) of one item of each class
    int64_t max_smem = 0, big_max_smem = 0;
    int64_t giant_comps = 0;            // compartments in giant items (size of the Hines scratch)
    int64_t giant_paths = 0;            // paths in giant items (size of the per-path scratch)
    std::vector<int32_t> site_comp;     // group-local compartment of each site
    std::vector<int64_t> site_internal; // internal compartment of each site
    // spike sources: internal neurons (soma detection) or detection points
    int32_t n_src = 0;
    std::vector<int64_t> pt_comp;       // points: internal compartment of each, ascending
    std::vector<int32_t> pt_user_nrn;   // points: user neuron and LOCAL user compartment
    std::vector<int32_t> pt_user_comp;
    std::vector<int32_t> soma_src;      // points: source id of each internal neuron's soma point, -1 if none
    std::vector<int32_t> pt_of;         // points: point id of each compartment, -1 where none and at somata
    std::vector<int64_t> out_off;       // outgoing synapses per source [n_src+1]
    std::vector<int32_t> out_site, out_dsteps;
    std::vector<double> out_w;
    std::vector<int32_t> dclass;        // distinct delays in steps, ascending
    // incoming synapses of each site in ascending synapse id (deterministic
    // delivery): source id, delay in steps, weight
    std::vector<int64_t> in_off;        // [nsite+1]
    std::vector<int32_t> in_src, in_dsteps;
    std::vector<double> in_w;
    int32_t R = 2;                      // spike ring depth (steps)
    double f_syn = 0.0;                 // fraction of compartments with a synapse
};

// The MM_N_FEATURES morphology features of one neuron (see mm.h), from its
// local parent array and cylinders.
void neuron_features(int32_t n, const int32_t *parent, const double *L_um, const double *d_um, float *out);

// Validates the inputs and builds the layout.  Returns "" on success, else
// a message; *invalid tells whether the inputs were invalid (vs. unsupported).
std::string build_layout(const LayoutInput &in, Layout &out, bool *invalid);

}  // namespace mmh

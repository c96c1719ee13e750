// mm_internal.h -- records and kernel arguments shared by the host runtime
// and the CUDA kernels of the multi-morphology stepper.
//
// Device layout (all per-compartment arrays in INTERNAL order):
//   * neurons are re-ordered by the schedule (largest cost first);
//   * inside a neuron, compartments are renumbered in depth-first preorder
//     (parent < child), visiting the deepest child first (deepest: the
//     longest path to a leaf, in compartments), so that every "path" -- a
//     compartment that does not continue its parent's path, its deepest
//     child, that one's deepest child, and so on down to a leaf -- is one
//     contiguous index range in which each compartment's parent is the one
//     before it; an unbranched run of the tree (a "segment") is contiguous
//     as well;
//   * consecutive neurons are packed into work items ("groups") whose
//     compartments are contiguous; one thread block solves one group at a
//     time, with the group's Hines diagonal and right-hand side in shared
//     memory (giant FP32c items: in a global scratch);
//   * FP32c: the paths of a neuron are sorted by level (0: the path from its
//     soma; level l + 1: paths that hang off a path of level l), so that the
//     leaves-to-root sweep of Algorithm 1 can run path by path from the
//     deepest level up and the root-to-leaves sweep from level 0 down;
//   * FP64: the segments of a group are sorted by height (0 = no child
//     segment), so that all segments of one height ("wave") can be
//     eliminated in parallel once the lower waves are done, and substituted
//     in the reverse order.
#pragma once
#include <stdint.h>
#include <vector_types.h>

namespace mmk {

// One segment of a group: compartments top .. top+len-1 (group-local), a
// path from top down to the bottom compartment top+len-1.
struct SegRec {
    int32_t top;      // group-local index of the first compartment
    int32_t len;      // >= 1
    int32_t parent;   // group-local index of top's parent; -1 for a soma segment
    int32_t child0;   // first entry of this segment's children in seg_child[]
    int32_t nchild;   // number of child segments (all hang off the bottom)
    int32_t neuron;   // soma segment: group-local neuron index; else -1
};

// Packed form of a segment inside a work item's tree blob (16 bytes;
// group-local indices fit 15 bits because a work item holds at most 32767
// compartments and segments).
struct SegP {
    int16_t top;      // group-local index of the first compartment
    int16_t len;      // >= 1
    int16_t parent;   // group-local index of top's parent; -1 for a soma segment
    int16_t nchild;   // number of child segments
    int16_t child0;   // first entry of this segment's children in the blob's child list
    int16_t neuron;   // soma segment: group-local neuron index; else -1
    int16_t pseg;     // index of the parent segment in the blob; -1 for a soma segment
    int16_t pad;
};

// FP32c work items are solved path by path, by a team of warps per sweep
// bundle (one neuron, or several consecutive small neurons swept together).
// Per bundle of an item (8 bytes): its paths are path0 .. path0 + npath - 1
// of the item, sorted by level (0: the paths from the somata) and, within a
// level, longest first; level l holds paths loffs[loff0 + l] ..
// loffs[loff0 + l + 1] - 1, and the first mcnt[loff0 + l] entries of that
// level's fold list belong to parent compartments shared by several paths.
struct NrnQ {
    int16_t path0;
    int16_t npath;
    int16_t nlevel;
    int16_t loff0;
};

// A path of an FP32c work item (8 bytes).
struct PathQ {
    int16_t head;     // group-local index of the first compartment
    int16_t end;      // one past the last compartment (a leaf)
    int16_t parent;   // group-local parent of head; -1 when head is a soma
    int16_t nflag;    // group-local neuron index | kPathAlone
};
// set in PathQ::nflag when no other path hangs off the same parent
// compartment: the path adds its contribution to the parent directly
constexpr int16_t kPathAlone = 0x4000;
constexpr int16_t kPathNeuron = 0x3FFF;

// One fold-list entry (4 bytes): low half a path's index in the item, high
// half the compartment its head hangs off.  The fold list holds the same
// paths as the path table, level by level (same level offsets); within a
// level the paths that share a parent compartment come first, sorted by that
// compartment (deepest first, then head), so that their contributions are
// summed in a fixed order; the paths alone on their parent follow.
typedef uint32_t KidQ;

// The same three tables with 32-bit indices, for FP32c giant items (beyond
// shared memory, solved from a global scratch): NrnG per bundle, PathG per
// path, KidG per fold entry {path, parent compartment}.
struct NrnG {
    int32_t path0, npath, nlevel, loff0;
};
struct PathG {
    int32_t head, end, parent, nflag;  // nflag: neuron index | kPathAloneG
};
constexpr int32_t kPathAloneG = 0x40000000;
constexpr int32_t kPathNeuronG = 0x3FFFFFFF;
typedef int2 KidG;

// One work item: a run of whole neurons.  Its tree is one contiguous,
// 16-byte aligned blob in global memory, staged into shared memory with a
// single bulk copy.  FP64 items: SegP[nseg] | int16 child[nchild] |
// int16 wave_off[nwave+1] (wave w holds segments wave_off[w] ..
// wave_off[w+1]-1; wave 0 holds the leaf segments), padded to 16 bytes.
// FP32c items: NrnQ[nbundle] | PathQ[npath] (at byte path_off) |
// KidQ[npath] (fold list, at fold_off) | int16 loffs[] (at loffs_off) |
// int16 mcnt[] (as many as loffs, at mcnt_off), padded to 16 bytes.
// Giant FP32c items (beyond shared memory) use the same layout with the
// 32-bit records NrnG, PathG, KidG and int32 loffs / mcnt.
struct GroupRec {
    int64_t comp0;    // internal index of the first compartment
    int64_t scratch0; // giant items: first entry in the global Hines scratch
    int64_t meta_off; // byte offset of the tree blob
    int32_t meta_bytes;
    int32_t ncomp;
    int32_t nseg;
    int32_t nchild;
    int32_t nwave;
    int32_t site0;    // first synaptic site (index into site_comp[] / gsyn[])
    int32_t nsite;
    int32_t neuron0;  // internal id of the first neuron
    int32_t nneuron;
    int32_t npath;
    int32_t nlevel;   // FP32c: the largest number of path levels of a neuron of the item
    int32_t path_off; // FP32c: byte offset of PathQ[0] inside the blob
    int32_t fold_off; // FP32c: byte offset of the fold list
    int32_t loffs_off;// FP32c: byte offset of the level offsets
    int32_t mcnt_off; // FP32c: byte offset of the per-level shared-parent counts
    int32_t pscratch0;// FP32c giant items: first entry in the global per-path scratch
    int32_t nbundle;  // FP32c: sweep bundles (NrnQ / NrnG records) of the item
    int32_t pad;
};

// Small device-side control block.
struct DevCtl {
    unsigned long long step_base;   // steps completed before the current launch batch
    unsigned long long spk_count;   // spikes appended to the output buffer
    unsigned int queue_head;        // next work item of the current step
    int err;                        // MMK_ERR_* bits
    unsigned int giant_head;        // next giant work item of the current step
    unsigned int big_head;          // next work item of the large shared-memory class
};

enum { MMK_ERR_OVERFLOW = 1, MMK_ERR_NUMERIC = 2, MMK_ERR_TIMEOUT = 4 };

// Arguments of the FP64 step kernel.
struct StepArgs {
    double *V, *m, *h, *n;            // state [C]
    const double *area;               // membrane area, cm^2 [C]
    const double *gax;                // axial conductance to the parent, uS [C] (0 at a soma)
    const double *stim;               // soma current per internal neuron, nA [N]
    const int32_t *user_id;           // internal neuron -> user id [N]
    const GroupRec *groups;
    int32_t n_groups;
    int32_t step_offset;              // step index = ctl->step_base + step_offset
    const unsigned char *meta;        // tree blobs of all work items
    int32_t smem_meta;                // bytes reserved for the largest blob
    const int32_t *site_comp;         // group-local compartment of each synaptic site
    double *gsyn;                     // merged synaptic conductance per site, uS
    int32_t *ring_nrn;                // [R * N] spike sources that fired, per step slot
    int32_t *ring_cnt;                // [R]
    int32_t R, N;                     // ring depth (steps) and slot capacity (spike sources)
    int32_t *spk_nrn;                 // output spikes (user ids) [spk_cap]
    int32_t *spk_comp;                // output spikes: LOCAL compartment of the crossing
    double *spk_t;
    long long spk_cap;
    // detection at synapse points (MM_DETECT_SYNAPSE_POINTS; all null under
    // soma detection, where a neuron's source id is its internal id)
    const int32_t *pt_of;             // point id of each compartment [C]; -1 where none and at somata
                                      // (a soma point is tested by the soma path)
    const int32_t *pt_user_nrn;       // user neuron and LOCAL compartment of each point
    const int32_t *pt_user_comp;
    const int32_t *soma_src;          // source id of each internal neuron's soma point, -1: none
    int32_t n_pt;
    int32_t fired_words;              // deterministic delivery: 32-bit words per step slot of `fired`
    uint32_t *fired;                  // deterministic delivery: [R * fired_words] bit per source that
                                      // fired in each step slot (nullptr otherwise)
    DevCtl *ctl;
    int32_t smem_comps, smem_segs;    // shared-memory capacity of one block (FP64)
    double gNa, gK, gL, ENa, EK, EL;
    double cm_dt;                     // Cm * 1e3 / dt: C_i/dt = area_i * cm_dt (nF/ms = uS)
    double e_syn, threshold, dt, decay;
    // time discretisation (MM_SCHEME_*): the implicit share of each axial
    // coupling (1, or 1/2 for Eq. 2 as printed) and whether the membrane
    // conductance enters the diagonal (backward Euler) or stays explicit
    double gimp;
    int32_t g_implicit;
    int32_t pad_scheme;
};

// Fixed-point state of the FP32c path: V = Vq * 2^-23 mV (int32, +-256 mV),
// gates x = q * 2^-32 (uint32).  FP32 increments are rounded once and added
// exactly, so the state itself never accumulates rounding.
constexpr float kVScale = 8388608.0f;          // 2^23 per mV
constexpr float kVInv = 1.0f / 8388608.0f;
constexpr double kVScaleD = 8388608.0;
constexpr double kVInvD = 1.0 / 8388608.0;
constexpr float kGScale = 4294967296.0f;       // 2^32
constexpr float kGInv = 1.0f / 4294967296.0f;
constexpr double kGScaleD = 4294967296.0;

// A reversal (or any fixed) potential split into its nearest fixed-point
// value and an FP32 residual: E = q * 2^-23 + res.
struct FxPot {
    int32_t q;
    float res;
};

// Arguments of the FP32c step kernel.  Float pairs (float2: .x the nearest
// float, .y the rest) carry every model constant and the synaptic
// conductances to about 44 bits.
struct StepArgs32 {
    int32_t *Vq;                      // [C]
    uint32_t *mq, *hq, *nq;           // [C]
    double *Vsoma;                    // [N] FP64 soma voltage accumulator
    const float2 *area;               // cm^2 [C]
    const float2 *gax;                // axial conductance to the parent, uS [C]; the sign bit of .x is set
                                      // at path heads (somata included): their link to the parent is
                                      // assembled per path
    const float2 *dp;                 // passive diagonal after the elimination of Algorithm 1 with the
                                      // membrane conductance left out (C/dt, leak, implicit axial
                                      // couplings), uS [C]: .x its nearest float, .y the constant
                                      // share of the active part that stands for the rest
    float2 *dr;                       // scratch for giant items per compartment: (active conductance, rhs),
                                      // then the substitution coefficients (f, c), then (f, dV)
    float *drl;                       // scratch for giant items: low word of the rhs per compartment
    float4 *pq;                       // scratch for giant items per path: its contribution to the parent
                                      // (active conductance, rhs) and the current across its head link (pair)
    const int64_t *gchunk0;           // giant items: first compartment chunk of each [item1 - item0 + 1]
    unsigned long long *item_ns;      // per work item solve time (ns, summed over steps) or nullptr
    const double *stim;               // nA [N]
    const int32_t *user_id;
    const GroupRec *groups;
    int32_t n_groups;
    int32_t step_offset;
    const unsigned char *meta;
    int32_t smem_meta;
    int32_t item0, item1;             // this launch's work items: [item0, item1)
    int32_t smem_bytes;               // dynamic shared memory of the launch (largest item need)
    unsigned int *queue;              // its work-queue counter (in ctl, reset by the delivery kernel)
    const int32_t *site_comp;
    float2 *gsyn;                     // per site, uS (pair)
    int32_t *ring_nrn;
    int32_t *ring_cnt;
    int32_t R, N;
    int32_t *spk_nrn;
    int32_t *spk_comp;
    double *spk_t;
    long long spk_cap;
    const int32_t *pt_of;             // detection points, as in StepArgs
    const int32_t *pt_user_nrn;
    const int32_t *pt_user_comp;
    const int32_t *soma_src;
    int32_t n_pt;
    int32_t fired_words;              // deterministic delivery, as in StepArgs
    uint32_t *fired;
    DevCtl *ctl;
    int32_t smem_comps, smem_segs;
    float2 gNa, gK, gL;               // channel densities times 1e3 (uS per cm^2 of membrane), pairs
    FxPot ENa, EK, EL, Esyn;
    float2 decay;                     // exp(-dt / tau_syn), pair
    const float4 *gtab;               // gate table for dt (mm_gate_table.h): 12 arrays of 481 float4
    int64_t C;                        // compartments (gate kernel)
    double threshold, dt64;
    float gimp;                       // implicit share of each axial coupling: 1 or 1/2 (as in StepArgs)
    int32_t g_implicit;               // membrane conductance in the diagonal (backward Euler)
    int32_t thr_q;                    // ceil(threshold * 2^23): V^n < threshold <= V^{n+1} is exactly
                                      // Vq^n < thr_q <= Vq^{n+1}
};


#ifdef __CUDACC__
// One threshold crossing of spike source src (user neuron, LOCAL compartment)
// at time ts within step n: the output record, and the source's entry in the
// ring slot of step n (delivered by the delivery kernel of the next step).
// The lanes of a warp that record together reserve their entries with one
// atomic per counter (a volley of point spikes would otherwise serialise on
// the two counters).
template <class A>
__device__ __forceinline__ void record_spike(const A &a, int src, int user_nrn, int user_comp, double ts,
                                             long long n)
{
    const unsigned mask = __activemask();
    const int lane = (int)(threadIdx.x & 31u);
    const int leader = __ffs(mask) - 1;
    const int cnt = __popc(mask);
    const int rank = __popc(mask & ((1u << lane) - 1u));
    const int slot = (int)(n % a.R);
    unsigned long long k0 = 0;
    int p0 = 0;
    if (lane == leader) {
        k0 = atomicAdd(&a.ctl->spk_count, (unsigned long long)cnt);
        p0 = atomicAdd(&a.ring_cnt[slot], cnt);
    }
    k0 = __shfl_sync(mask, k0, leader);
    p0 = __shfl_sync(mask, p0, leader);
    const unsigned long long k = k0 + (unsigned long long)rank;
    if ((long long)k < a.spk_cap) {
        a.spk_nrn[k] = user_nrn;
        a.spk_comp[k] = user_comp;
        a.spk_t[k] = ts;
    } else {
        atomicOr(&a.ctl->err, MMK_ERR_OVERFLOW);
    }
    a.ring_nrn[(long long)slot * a.N + p0 + rank] = src;
    if (a.fired) atomicOr(&a.fired[(long long)slot * a.fired_words + (src >> 5)], 1u << (src & 31));
}

// An upward crossing of the threshold between V^n = v0 and V^{n+1} = v1 at
// detection point p (linearly interpolated time).  The kernels test the
// crossing first and read the compartment's point id only where it crossed.
template <class A>
__device__ __forceinline__ void point_spike(const A &a, int p, double v0, double v1, long long n, double dt)
{
    const double ts = (double)n * dt + dt * (a.threshold - v0) / (v1 - v0);
    record_spike(a, p, a.pt_user_nrn[p], a.pt_user_comp[p], ts, n);
}

// Spike source of the soma of internal neuron nrn (-1: not tested).
template <class A>
__device__ __forceinline__ int soma_source(const A &a, int nrn)
{
    return a.soma_src ? a.soma_src[nrn] : nrn;
}
#endif

struct DeliverArgs {
    const int32_t *ring_nrn;
    int32_t *ring_cnt;
    int32_t R, N;
    const int64_t *out_off;           // [N+1] outgoing synapses of each internal source
    const int32_t *out_site;          // target synaptic site
    const double *out_w;              // weight, uS
    const int32_t *out_dsteps;        // round(delay/dt), ascending within a source
    const int32_t *dclass;            // distinct delays (steps), ascending
    int32_t n_dclass;
    int32_t lanes_per_src;            // lanes that scatter one spike's synapses (1, 2, 4, ..., 32)
    // deterministic delivery: the incoming synapses of each site in
    // ascending synapse id (source id, delay in steps, weight) and the ring
    // of per-step bitmasks of the sources that fired
    const int64_t *in_off;            // [nsite + 1]
    const int32_t *in_src;
    const int32_t *in_dsteps;
    const double *in_w;               // FP64 weights
    const float2 *in_w2;              // FP32c weights (float pairs)
    uint32_t *fired;                  // [R * fired_words]
    int32_t fired_words;
    int64_t nsite;
    int32_t step_offset;
    double *gsyn;
    DevCtl *ctl;
    float2 *gsyn2;                    // FP32c: per-site conductance as a float pair (gsyn unused)
    const float2 *out_w2;             // FP32c: weights as float pairs
};

struct InitArgs {
    const double *L, *diam;           // internal order
    const int32_t *parent_dist;       // i - parent(i), negated at segment tops (FP64) or path heads (FP32c), 0 at a soma
    int64_t C;
    double *area, *gax;
    double *V, *m, *h, *n;
    double Ra, v_init;
    // FP32c outputs (used when Vq != nullptr; the FP64 pointers are then
    // unused; the FP32c constants are computed on the host)
    int32_t *Vq;
    uint32_t *mq, *hq, *nq;
};

}  // namespace mmk

// Launch wrappers (defined in the .cu files; return a cudaError_t as int).
extern "C++" {
int mmk_launch_init(const mmk::InitArgs &a, void *stream);
int mmk_launch_deliver(const mmk::DeliverArgs &a, int blocks, void *stream);
int mmk_launch_step_fp64(const mmk::StepArgs &a, int blocks, int threads, void *stream);
int mmk_step_fp64_blocks_per_sm(int threads, int smem_bytes, int *blocks);
int mmk_launch_step_fp32c(const mmk::StepArgs32 &a, int blocks, int threads, void *stream);
int mmk_step_fp32c_blocks_per_sm(int threads, int smem_bytes, int *blocks);
size_t mmk_step_fp64_smem(int comps, int segs, int meta_bytes);
int mmk_launch_init_fp32c(const mmk::InitArgs &a, void *stream);
int mmk_launch_giant_fp32c(const mmk::StepArgs32 &a, int blocks, void *stream);
int mmk_launch_giant_assemble(const mmk::StepArgs32 &a, int chunk_blocks, void *stream);
int mmk_launch_giant_update(const mmk::StepArgs32 &a, int chunk_blocks, void *stream);
int mmk_giant_chunk();
int mmk_launch_deliver_fp32c(const mmk::DeliverArgs &a, int blocks, void *stream);
int mmk_launch_deliver_ordered(const mmk::DeliverArgs &a, int blocks, void *stream);
int mmk_launch_deliver_ordered_fp32c(const mmk::DeliverArgs &a, int blocks, void *stream);
int mmk_launch_vq_to_f64(const int32_t *vq, double *dst, int64_t n, void *stream);
int mmk_launch_gq_to_f64(const uint32_t *q, double *dst, int64_t n, void *stream);
int mmk_launch_scatter_f2_to_f64(const float2 *src, const int64_t *idx, double *dst, int64_t n, void *stream);
int mmk_launch_advance(mmk::DevCtl *ctl, int steps, void *stream);
int mmk_launch_wait_selftest(int *err, unsigned int max_polls, void *stream);
int mmk_launch_inject(int32_t *ring_nrn, int32_t *ring_cnt, int32_t R, int32_t Nsrc, int32_t N, uint32_t *fired,
                      int32_t fired_words, const int32_t *src, const int64_t *step, int64_t n, mmk::DevCtl *ctl,
                      void *stream);
int mmk_launch_gather_f64(const double *src, const int64_t *idx, double *dst, int64_t n, void *stream);
int mmk_launch_scatter_f64(const double *src, const int64_t *idx, double *dst, int64_t n, void *stream);
int mmk_launch_fill_f64(double *dst, double v, int64_t n, void *stream);
}

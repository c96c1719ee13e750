/*
 * mm.h -- C-ABI of the GB300 multi-morphology neuron stepper.
 *
 * The library advances many neurons of different shapes and sizes at once.
 * Each neuron is a tree of cylinder compartments; every time step it
 * updates the membrane voltage of every compartment: Hodgkin-Huxley gating
 * and currents, assembly of the neuron's Hines matrix, the Hines tree solve,
 * synaptic currents, spike detection (at the somata, or at the points where
 * synapses leave) and delayed spike delivery.  The
 * calls follow the paper's statement of the problem (Sec. 2): a network is
 * created from morphologies (compartment trees given by parent arrays),
 * channel parameters and synapses, stepped in time, and its voltages and
 * spikes are read back.
 *
 * Units: um, mV, ms, nA, uS, nF; channel densities in mS/cm^2, membrane
 * capacitance in uF/cm^2, axial resistivity in ohm*cm.
 *
 * Conventions shared by every call:
 *   - Pointers to inputs are HOST pointers, owned by the caller and only
 *     read during the call (the library copies what it keeps).
 *   - Device memory is owned by the library: allocated at create through
 *     the allocator in mm_options (or cudaMalloc when none is given) and
 *     released by mm_destroy.
 *   - Every call returns an mm_status and never throws.  After a CUDA error
 *     or a failed kernel check the network is poisoned: every later call
 *     except mm_last_error / mm_destroy returns MM_ESTATE.
 *   - mm_step is asynchronous on the network's stream; errors raised by its
 *     kernels surface at the next synchronising call (the mm_read_* calls,
 *     mm_save_state, mm_synchronize).
 *   - A network is used from one host thread at a time.
 */
#ifndef MM_H_
#define MM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mm_net mm_net; /* opaque, library-owned */

typedef enum {
    MM_OK = 0,
    MM_EINVAL = 1,     /* an argument or an input array is invalid */
    MM_ENOMEM = 2,     /* a device or host allocation failed */
    MM_ECUDA = 3,      /* a CUDA call failed */
    MM_ETIMEOUT = 4,   /* a bounded device wait gave up */
    MM_ENUMERIC = 5,   /* a soma voltage became NaN or infinite */
    MM_EOVERFLOW = 6,  /* more spikes than the spike buffer holds were detected */
    MM_ESTATE = 7,     /* the network is poisoned by an earlier error */
    MM_ENOTSUP = 8     /* valid request this build does not support */
} mm_status;

/* Arithmetic of the time step. */
enum {
    MM_FP64 = 0,   /* everything in FP64 */
    MM_FP32C = 1   /* FP32 increments on a fixed-point state (V in 2^-23 mV, gates
                      in 2^-32); model constants, currents and synaptic
                      conductances as float pairs, the Hines solve in FP32 on
                      the FP64-eliminated passive diagonal; FP64 soma voltage
                      and spike-crossing time.  Voltages must stay within
                      +-120 mV (the fixed-point range): a compartment driven
                      beyond it stops the network with MM_ENUMERIC */
};

/* Time discretisation of the voltage equation (Eq. 1) -- the reading of
 * Eq. 2 the Hines system follows. */
enum {
    MM_SCHEME_BE = 0,  /* backward Euler for dV with the membrane conductance
                          implicit: d_i = C_i/dt + G_i + sum_j g_ij, off-diagonal
                          -g_ij, rhs_i = -I_i + sum_j g_ij (V_j - V_i) (default) */
    MM_SCHEME_CN = 1   /* Eq. 2 as printed: half of each axial coupling implicit,
                          half and the membrane current explicit (Crank-Nicolson
                          in the diffusion): d_i = C_i/dt + sum_j g_ij / 2,
                          off-diagonal -g_ij / 2, same rhs.  Stable only while
                          dt G_i / C_i < 2 in every compartment */
};

/* Where the threshold test runs (Sec. 2, spike computation). */
enum {
    MM_DETECT_SOMA = 0,            /* at every soma; a spike of neuron k reaches every
                                      synapse with src_neuron k (default) */
    MM_DETECT_SYNAPSE_POINTS = 1   /* at every point of a morphology that a synapse leaves
                                      from: the distinct (src_neuron, src_comp) pairs.  A
                                      crossing at a point reaches the synapses leaving that
                                      point only; somata without such a synapse are not
                                      tested */
};

/* Order in which the per-step kernel takes its work items. */
enum {
    MM_SCHED_SIZE_SORTED = 0,  /* neurons sorted by compartment count, largest first */
    MM_SCHED_COST = 1          /* neurons sorted by mm_options.cost, largest first */
};

/* What mm_read_state reads. */
enum {
    MM_STATE_V = 0,      /* membrane voltage, mV */
    MM_STATE_M = 1,      /* Na activation gate */
    MM_STATE_H = 2,      /* Na inactivation gate */
    MM_STATE_N = 3,      /* K activation gate */
    MM_STATE_GSYN = 4    /* merged synaptic conductance, uS (0 where no synapse) */
};

/* Neuron morphologies (Sec. 2: compartments joined into an acyclic tree,
 * numbered so that every parent precedes its children).
 *   comp_offset [n_neurons+1]: neuron k owns compartments
 *                comp_offset[k] .. comp_offset[k+1]-1 (user numbering);
 *                comp_offset[0] = 0, strictly increasing.
 *   parent      [comp_offset[n]]: LOCAL parent index within the neuron;
 *                -1 at local index 0 (the soma) and 0 <= parent[i] < i elsewhere.
 *   length_um, diam_um [comp_offset[n]]: cylinder of each compartment, > 0. */
typedef struct {
    int32_t n_neurons;
    const int64_t *comp_offset;
    const int32_t *parent;
    const double *length_um;
    const double *diam_um;
} mm_morphologies;

/* Hodgkin-Huxley channels (the current I of Eq. 1) and cable constants. */
typedef struct {
    double gNa, gK, gL;     /* mS/cm^2 */
    double ENa, EK, EL;     /* mV */
    double Cm;              /* uF/cm^2 */
    double Ra;              /* ohm*cm */
    double v_init;          /* initial voltage, mV; gates start at steady state */
    double threshold_mV;    /* soma spike threshold (upward crossing) */
} mm_channel_params;

/* Exponential synapses.  Synapse s makes a spike of neuron src_neuron[s]
 * raise the conductance of compartment dst_comp[s] (LOCAL index) of neuron
 * dst_neuron[s] by weight_uS[s], round(delay_ms[s]/dt) + 1 steps after the
 * step in which the spike was detected; conductances decay with tau_ms and
 * drive the current g (V - e_rev_mV).  Arrays have n entries (n may be 0).
 * src_comp (may be NULL = every synapse leaves from the soma) is the LOCAL
 * compartment of src_neuron[s] the synapse leaves from; it is used under
 * MM_DETECT_SYNAPSE_POINTS only. */
typedef struct {
    int64_t n;
    const int32_t *src_neuron;
    const int32_t *dst_neuron;
    const int32_t *dst_comp;
    const double *weight_uS;   /* >= 0 */
    const double *delay_ms;    /* round(delay/dt) >= 1 */
    double tau_ms;             /* > 0 */
    double e_rev_mV;
    const int32_t *src_comp;   /* may be NULL */
} mm_synapses;

/* Device-memory allocator: alloc returns a device pointer (256-byte aligned)
 * or NULL; release frees it.  Used for every device buffer of a network. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*release)(void *ptr, void *ctx);
    void *ctx;
} mm_allocator;

typedef struct {
    int32_t precision;          /* MM_FP64 | MM_FP32C */
    int32_t schedule;           /* MM_SCHED_SIZE_SORTED | MM_SCHED_COST */
    int32_t graph_steps;        /* steps per captured CUDA graph; 0 = no graphs */
    int32_t block_threads;      /* threads per work item's block; 0 = automatic */
    int32_t group_comps;        /* compartment budget of one work item; 0 = automatic */
    int32_t device;             /* CUDA device ordinal */
    int32_t time_items;         /* MM_FP32C: record each work item's solve time (mm_read_neuron_times) */
    int32_t scheme;             /* MM_SCHEME_BE | MM_SCHEME_CN */
    int32_t detect;             /* MM_DETECT_SOMA | MM_DETECT_SYNAPSE_POINTS */
    int32_t deterministic_delivery; /* 0: spike events added to the synaptic conductances with
                                       atomics (order unspecified); 1: each site adds its events
                                       in ascending synapse id, as the oracle does (Sec. 2's
                                       event delivery made reproducible: runs repeat bit for bit,
                                       and under MM_FP64 the conductances equal the oracle's) */
    double dt_ms;               /* time step of the network, > 0 */
    int64_t spike_capacity;     /* spikes held between two mm_read_spikes; 0 = automatic */
    void *cuda_stream;          /* cudaStream_t to run on; NULL = a library-owned stream */
    const float *cost;          /* [n_neurons] per-neuron cost for MM_SCHED_COST, or NULL */
    mm_allocator allocator;     /* alloc == NULL: cudaMalloc / cudaFree */
    int32_t n_ext_sources;      /* spike sources outside this network (neurons simulated elsewhere,
                                   e.g. on other GPUs): synapse src_neuron values n_neurons ..
                                   n_neurons + n_ext_sources - 1 name them, and their spikes are
                                   handed in with mm_inject_spikes.  MM_DETECT_SOMA only; 0 = none */
} mm_options;

/* The largest neuron (compartments) the MM_FP64 path holds. */
#define MM_FP64_MAX_NEURON_COMPS 8192

/* Fill *opt with defaults: FP64, size-sorted, graphs of 40 steps, dt 0.025 ms. */
void mm_default_options(mm_options *opt);

/* Build a network (Sec. 2: morphologies, parent arrays, channel parameters,
 * synapses) and its device state at rest.  stim_nA [n_neurons]: constant
 * current injected into each soma from t = 0 (may be NULL: no stimulus).
 * On success *out owns the network; on failure *out is NULL.
 * Errors: MM_EINVAL (bad sizes, parent[i] >= i, non-positive geometry,
 * dst_comp or src_comp out of range, delay < dt, dt <= 0, unknown scheme or
 * detection mode, deterministic_delivery not 0 or 1), MM_ENOMEM, MM_ECUDA,
 * MM_ENOTSUP (e.g. MM_FP64 with a neuron of more than MM_FP64_MAX_NEURON_COMPS
 * compartments: the FP64 kernel holds a whole neuron in one block's shared
 * memory; MM_FP32C has no such limit). */
mm_status mm_create_network(const mm_morphologies *morph, const mm_channel_params *chan,
                            const mm_synapses *syn, const double *stim_nA,
                            const mm_options *opt, mm_net **out);

/* Advance n_steps >= 0 time steps of dt_ms, which must equal the network's
 * dt.  Asynchronous on the network's stream.  With graph_steps > 0 (and
 * kernel timing off) every step runs inside a CUDA graph: whole batches of
 * graph_steps steps replay the batch graph, the rest the one-step graph. */
mm_status mm_step(mm_net *net, int64_t n_steps, double dt_ms);

/* Wait for the network's stream and report any error its kernels raised. */
mm_status mm_synchronize(mm_net *net);

/* Copy the voltage of every compartment, in user numbering, into the host
 * array out [cap >= total compartments].  Synchronises. */
mm_status mm_read_voltages(mm_net *net, double *out, int64_t cap);

/* Like mm_read_voltages for any MM_STATE_* quantity. */
mm_status mm_read_state(mm_net *net, int32_t which, double *out, int64_t cap);

/* Soma voltage of every neuron, in user neuron order, into out [cap >= n_neurons]. */
mm_status mm_read_soma_voltages(mm_net *net, double *out, int64_t cap);

/* Drain the spikes detected since the last call: neuron (user id) and
 * crossing time t_ms, ordered by (t, neuron).  Writes min(cap, count)
 * records and the count to *n_out.  MM_EOVERFLOW if the device buffer
 * overflowed (the records it held are still returned).  Synchronises. */
mm_status mm_read_spikes(mm_net *net, int32_t *neuron, double *t_ms, int64_t cap, int64_t *n_out);

/* mm_read_spikes with the point of each spike: comp [cap] receives the
 * LOCAL compartment where the crossing was detected (0 under
 * MM_DETECT_SOMA); records ordered by (t, neuron, comp).  Drains the same
 * buffer as mm_read_spikes. */
mm_status mm_read_spike_points(mm_net *net, int32_t *neuron, int32_t *comp, double *t_ms, int64_t cap,
                               int64_t *n_out);

/* The per-step outputs of a host loop in one round trip: the soma voltage
 * of every neuron into soma [soma_cap >= n_neurons] (as
 * mm_read_soma_voltages) and the spikes detected since the last drain into
 * neuron, comp (may be NULL), t_ms [cap] with their count in *n_out (as
 * mm_read_spike_points, same order, same errors).  Synchronises once when
 * at most 4096 spikes are pending, twice otherwise. */
mm_status mm_read_outputs(mm_net *net, double *soma, int64_t soma_cap, int32_t *neuron, int32_t *comp,
                          double *t_ms, int64_t cap, int64_t *n_out);

/* Replace the soma stimulus of every neuron (host array [n], n = n_neurons). */
mm_status mm_set_stimulus(mm_net *net, const double *stim_nA, int64_t n);

/* Steps taken so far. */
mm_status mm_get_step(const mm_net *net, int64_t *step);

/* Checkpoint: the whole dynamic state (voltages, gates, synaptic
 * conductances, in-flight spikes, step counter).  mm_save_state with
 * buf == NULL stores the needed size in *len.  mm_load_state restores a
 * state saved from a network created with identical inputs and options;
 * the continued run is bitwise identical to an uninterrupted one. */
mm_status mm_save_state(mm_net *net, void *buf, size_t cap, size_t *len);
mm_status mm_load_state(mm_net *net, const void *buf, size_t len);

/* Per-kernel device time, measured with CUDA events recorded on the
 * network's stream around each launch while timing is enabled. */
typedef struct {
    double step_kernel_ms;          /* per-step kernel of the regular item class (currents, tree solve, V, gates), summed */
    int64_t step_kernel_launches;
    double deliver_kernel_ms;       /* spike-delivery kernel, summed */
    int64_t deliver_kernel_launches;
    double giant_kernel_ms;         /* FP32c giant items: phase A, solve and phase C + gate kernels, summed
                                       (the solve runs on a side stream beside the other classes) */
    int64_t giant_kernel_launches;  /* steps (solve-kernel launches) */
    double big_kernel_ms;           /* FP32c per-step kernel on the large shared-memory class, summed */
    int64_t big_kernel_launches;
} mm_kernel_times;

/* While enabled (enable != 0), mm_step launches every kernel directly (no
 * CUDA graph) with a start/stop event pair around it. */
mm_status mm_set_kernel_timing(mm_net *net, int32_t enable);

/* Synchronise and report the time accumulated since the last reset;
 * reset != 0 clears the totals afterwards. */
mm_status mm_read_kernel_timing(mm_net *net, mm_kernel_times *out, int32_t reset);

/* Algorithm 1 (Sec. 2) on a batch of independent trees, on the device.
 * Tree k holds entries tree_offset[k] .. tree_offset[k+1]-1 (n_comp in
 * total); per entry i (local index j within its tree): parent (LOCAL,
 * parent[0] = -1, 0 <= parent[j] < j), a = upper (row p(j), column j),
 * b = diagonal, c = lower (row j, column p(j)), rhs.  Writes the solution
 * of every system to x.  ALL pointers are DEVICE pointers; inputs are not
 * modified.  Runs on cuda_stream (NULL: the legacy default stream) and
 * returns after the solve has finished.  Allocates a device scratch of
 * n_comp doubles for the duration of the call.
 * Errors: MM_EINVAL (negative sizes, NULL arrays, a tree whose offsets do
 * not lie within [0, n_comp] in ascending order, or a tree that violates the
 * parent rule: such a tree is skipped and its entries of x are undefined,
 * the other trees are solved), MM_ENOMEM, MM_ECUDA. */
mm_status mm_hines_solve(int32_t n_trees, int64_t n_comp, const int64_t *tree_offset, const int32_t *parent,
                         const double *a, const double *b, const double *c, const double *rhs, double *x,
                         void *cuda_stream);

/* mm_hines_solve without any allocation (the paper has no counterpart):
 * for callers that may not allocate device memory at all, such as a
 * component inside a host application whose memory manager owns every
 * device byte (a cudaMalloc there fails or breaks its accounting), or a
 * latency-critical loop where an allocation could block or fail mid-run.
 * Same arguments, results and errors as mm_hines_solve; the caller still
 * passes every input and the output x.  The scratch is a fixed 8 MiB
 * device array inside this library (loaded on every GPU that loads the
 * library, until the process ends), so n_comp must not exceed 1,048,576
 * (MM_EINVAL otherwise).  Every call looks up that array's device address
 * (cudaGetSymbolAddress, with the caller's device current; the first call on
 * a device also loads the module there and should come before any stream
 * capture).  A failed call leaves no error behind: the status word is
 * cleared at the start of every call.  Every call on a device shares
 * the same scratch: calls whose work overlaps on the GPU race, so callers
 * order them (one stream, or wait for the previous call to return).
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
mm_status mm_hines_solve_noalloc(int32_t n_trees, int64_t n_comp, const int64_t *tree_offset,
                                 const int32_t *parent, const double *a, const double *b, const double *c,
                                 const double *rhs, double *x, void *cuda_stream);

/* Spikes of the external sources (mm_options.n_ext_sources), for a network
 * that is one part of a larger one split across devices or processes (the
 * paper's local and global spike buffers, Sec. 2: each part runs a global
 * step of local steps, then the spikes of that global step are exchanged).
 * Spike k: external source ext_src[k] (0 .. n_ext_sources - 1) crossed its
 * threshold in step step[k]; each of its synapses then delivers as a local
 * neuron's would, round(delay/dt) + 1 steps later.  Host arrays of n
 * entries.  A spike must be handed in before its earliest delivery:
 * step[k] < mm_get_step() <= step[k] + 1 + round(min delay / dt); a source
 * spikes at most once per step.  Stream-ordered before the next mm_step.
 * Errors: MM_EINVAL (bad arguments, a spike handed in too late, a source
 * out of range), MM_EOVERFLOW (more spikes in one step than sources),
 * MM_ENOMEM, MM_ECUDA. */
mm_status mm_inject_spikes(mm_net *net, int64_t n, const int32_t *ext_src, const int64_t *step);

/* The spikes this network's own neurons fired in steps step0 .. step0 +
 * n_steps - 1 (all already run, and no more than R - 1 = the largest delay
 * in steps + 1 steps back), in step order: user neuron ids in neuron[],
 * their steps in step[] (host arrays of cap entries); *n_out = how many
 * (MM_EOVERFLOW if more than cap).  These are what a part of a split
 * network sends to the others after each global step.  MM_DETECT_SOMA
 * only.  Synchronises.  Errors: MM_EINVAL, MM_EOVERFLOW, MM_ECUDA. */
mm_status mm_read_fired(mm_net *net, int64_t step0, int32_t n_steps, int32_t *neuron, int64_t *step, int64_t cap,
                        int64_t *n_out);

/* Exercises the step kernels' bounded wait (the paper has no counterpart):
 * a one-block kernel on `device` waits on an mbarrier that nothing arrives
 * at, giving up after max_polls polls (1 .. 2^20) as the step kernels give
 * up on a lost copy completion, and records the timeout in a device error
 * word that the host reads back.  Returns MM_ETIMEOUT when the wait ran out
 * and the error reached the host; the device stays usable.  Synchronises
 * the device.  Errors: MM_EINVAL, MM_ENOMEM, MM_ECUDA. */
mm_status mm_selftest_bounded_wait(int32_t device, uint32_t max_polls);

/* Per-neuron solve time, in microseconds per step, for a network created
 * with MM_FP32C, time_items = 1 and group_comps = 1 (every neuron its own
 * work item): the wall time from the moment a block takes the neuron's work
 * item to the end of its V update (%globaltimer), averaged over the steps
 * run since creation.  These are the labels of the learned cost model.
 * out [cap >= n_neurons], user neuron order.  Synchronises. */
mm_status mm_read_neuron_times(mm_net *net, double *out_us, int64_t cap);

/* Morphology features of every neuron (host computation, no GPU needed):
 * out [16 * n_neurons], row-major, one row of MM_N_FEATURES per neuron:
 *  0 log n            1 log(1 + depth)        2 log(1 + branch points)
 *  3 log(1 + leaves)  4 log(1 + segments)     5 log(1 + segment height)
 *  6 log(1 + critical path: sum over height waves of the longest segment)
 *  7 log(1 + longest segment)  8 mean segment length / 100
 *  9 log(1 + mean depth)       10 log(membrane area / um^2)
 * 11 mean diameter / um       12 branch points / n
 * 13 log(1 + widest wave)     14 critical path / n
 * 15 log(1 + children of the soma)
 * Errors: MM_EINVAL as for mm_create_network's morphology checks. */
#define MM_N_FEATURES 16
mm_status mm_neuron_features(const mm_morphologies *morph, float *out, int64_t cap);

/* ---------------------------------------------------------------------
 * Learned cost model: an MLP 16 -> 64 -> 64 -> 1 (ReLU) with BF16 weights
 * and FP32 accumulation, trained with Adam on FP32 master weights by the
 * library's own kernels.  It maps a neuron's MM_N_FEATURES morphology
 * features to its per-step solve time, the key by which MM_SCHED_COST
 * orders the work queue (the paper's priority(size) and sorting by size,
 * Sec. 4, with a learned key).  Parameters, flat (MM_MLP_PARAMS values):
 * W1 [64 x 16] row-major, b1 [64], W2 [64 x 64], b2 [64], W3 [1 x 64], b3 [1].
 * Inputs are standardised per feature and targets by mean / std (taken from
 * the training set by mm_mlp_train, or set by mm_mlp_set_normalisation).
 * All arrays are HOST arrays; the device holds the model.  Calls run on the
 * current device's default stream and return when done. */
#define MM_MLP_PARAMS 5313
typedef struct mm_mlp mm_mlp;

/* New model, He-uniform weights drawn from seed, zero biases, identity
 * standardisation. */
mm_status mm_mlp_create(uint64_t seed, mm_mlp **out);

/* Replace / read the FP32 master parameters (n = MM_MLP_PARAMS); setting
 * them resets the Adam moments and rounds the compute copy to BF16. */
mm_status mm_mlp_set_params(mm_mlp *mlp, const float *params, int64_t n);
mm_status mm_mlp_get_params(mm_mlp *mlp, float *params, int64_t n);

/* Standardisation: x' = (x - mu) / sd per feature (mu, sd [16], sd > 0),
 * y' = (y - y_mu) / y_sd. */
mm_status mm_mlp_set_normalisation(mm_mlp *mlp, const float *mu, const float *sd, float y_mu, float y_sd);

/* Mean squared error of the standardised prediction against the
 * standardised targets y [n] for inputs X [n x 16], and its gradient with
 * respect to the (BF16) parameters into grad [MM_MLP_PARAMS] (may be NULL). */
mm_status mm_mlp_loss_grad(mm_mlp *mlp, const float *X, const float *y, int64_t n, float *loss, float *grad,
                           int64_t grad_cap);

/* Full-batch Adam (beta 0.9 / 0.999, eps 1e-8) for `epochs` steps at
 * learning rate lr on X [n x 16], y [n]; sets the standardisation from the
 * data first.  loss_per_epoch [epochs] (may be NULL) receives the loss
 * before each step. */
mm_status mm_mlp_train(mm_mlp *mlp, const float *X, const float *y, int64_t n, int32_t epochs, float lr,
                       float *loss_per_epoch);

/* Predictions in target units for X [n x 16] into out [n]. */
mm_status mm_mlp_predict(mm_mlp *mlp, const float *X, int64_t n, float *out);

void mm_mlp_destroy(mm_mlp *mlp);

/* The learned work-queue order, end to end (Sec. 4's priority(size)
 * ordering with a learned key): from the network's inputs, time n_timed
 * neurons drawn from seed (each its own work item, MM_FP32C, `steps` steps,
 * no synapses, mm_read_neuron_times), train a fresh MLP (mm_mlp_train,
 * `epochs` Adam steps at lr) on 80 % of them to predict log time from the
 * morphology features, and write exp(prediction) for every neuron into
 * cost [cap >= n_neurons] (user neuron order): the key for
 * mm_options.cost with MM_SCHED_COST.  A network's layout is fixed when it
 * is created, so the costs serve the next mm_create_network.
 * opt: device, stream, allocator and dt_ms are used (the rest is ignored);
 * report (may be NULL) receives the held-out R^2 of log time and the last
 * training loss.  Synchronises.
 * Errors: MM_EINVAL (bad arguments or morphology, n_timed < 10, steps < 1,
 * epochs < 1, lr <= 0), MM_ENOMEM, MM_ECUDA. */
typedef struct {
    int32_t n_timed;        /* neurons timed (min(n_timed, n_neurons)) */
    int32_t n_holdout;      /* of which held out of the training */
    double r2_holdout;      /* R^2 of the predicted log time on the held-out neurons */
    double final_loss;      /* standardised MSE before the last Adam step */
    double mean_time_us;    /* mean measured solve time per step of the timed neurons */
    double r2_holdout_size_only; /* the same R^2 of a least-squares fit of log time on log size alone */
} mm_schedule_report;

mm_status mm_train_schedule(const mm_morphologies *morph, const mm_channel_params *chan, const double *stim_nA,
                            const mm_options *opt, int32_t n_timed, int32_t steps, int32_t epochs, float lr,
                            uint64_t seed, float *cost, int64_t cap, mm_schedule_report *report);

/* Launch configuration chosen for the per-step kernel. */
typedef struct {
    int32_t work_items;        /* neuron groups handed out by the device queue */
    int32_t blocks;            /* persistent blocks launched */
    int32_t threads;           /* threads per block */
    int32_t blocks_per_sm;     /* resident blocks per SM at this shared-memory size */
    int32_t smem_bytes;        /* dynamic shared memory per block */
    int32_t max_item_comps;    /* compartments of the largest work item */
    int32_t max_item_segments; /* unbranched segments of the largest work item */
    int32_t max_item_waves;    /* height waves of the deepest work item */
    int32_t giant_items;       /* FP32c work items solved from global memory (too big for shared memory) */
    /* FP32c work items above the regular shared-memory budget that still fit
     * one block's shared memory: solved by a second launch of the per-step
     * kernel, one block per SM (0 items: no such launch) */
    int32_t big_items;
    int32_t big_blocks;
    int32_t big_threads;
    int32_t big_smem_bytes;
    int32_t max_big_item_comps;
    /* compartments and synaptic sites in each class: regular, large, giant */
    int64_t comps[3];
    int64_t sites[3];
} mm_launch_info;

mm_status mm_get_launch_info(const mm_net *net, mm_launch_info *out);

/* One candidate launch configuration measured by mm_autotune. */
typedef struct {
    int32_t block_threads;  /* threads per block of the regular-class step kernel */
    int32_t group_comps;    /* compartment budget of one work item */
    mm_status status;       /* MM_OK, or why this candidate could not run */
    double ms_per_step;     /* mean over the timed steps; < 0 when status != MM_OK */
} mm_tune_point;

/* Launch-configuration autotuner of the per-step kernel.  The paper balances
 * its per-neuron tasks by size only (Sec. 4) and has no counterpart; here the
 * block shape and the work-item size are chosen by measurement.
 *
 * Builds a stratified sample of the network (every k-th neuron in size order,
 * about sample_comps compartments, with the synapses whose two ends are both
 * in the sample), then for each candidate -- block_threads 256/512/1024
 * (MM_FP32C) or 128/256/512 (MM_FP64), times group_comps 1024/2048/4096/8192
 * -- creates the sample network with *opt otherwise unchanged, runs `warmup`
 * steps and times `steps` steps with CUDA events on opt->cuda_stream (a
 * library-owned stream when NULL).  *best receives *opt with the fastest
 * candidate's block_threads and group_comps.  points (cap entries; NULL
 * allowed when cap == 0) receives the candidates in order, *n_points how many
 * were written.
 *
 * Inputs are as for mm_create_network (host pointers, caller-owned, read
 * during the call only).  Each candidate's network is created and destroyed
 * in turn, through opt->allocator.  Synchronous.
 * Errors: MM_EINVAL for bad arguments or invalid network inputs; MM_ENOTSUP
 * (or the first candidate's error) when no candidate runs. */
mm_status mm_autotune(const mm_morphologies *morph, const mm_channel_params *chan, const mm_synapses *syn,
                      const double *stim_nA, const mm_options *opt, int64_t sample_comps, int32_t warmup,
                      int32_t steps, mm_tune_point *points, int32_t cap, int32_t *n_points, mm_options *best);

/* Message of the last error on this network ("" if none); never NULL.
 * With net == NULL: the message of the calling thread's last failed
 * mm_create_network. */
const char *mm_last_error(const mm_net *net);

/* Static name of a status code. */
const char *mm_status_string(mm_status s);

/* Release the network and all its device memory (NULL is ignored). */
void mm_destroy(mm_net *net);

#ifdef __cplusplus
}
#endif
#endif /* MM_H_ */

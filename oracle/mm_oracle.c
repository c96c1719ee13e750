/*
 * mm_oracle.c -- plain, slow FP64 CPU oracle of the multi-morphology
 * Hodgkin-Huxley + Hines time stepper.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU
 * baseline leg of bench.py may load this.  It shares no code, header or
 * constant table with the CUDA library; both read the same seeded inputs.
 *
 * Units: um (lengths), cm^2 (areas), mV, ms, nA, uS, nF.
 *
 * What it computes, per time step n -> n+1 (t_n = n*dt), in this order:
 *   1. event delivery: every event whose arrival step is n adds its weight
 *      to the merged synaptic conductance of its target compartment,
 *      ascending by synapse id (local/global buffers, Sec. 2);
 *   2. currents at (V^n, gates^n, g_syn^n): Hodgkin-Huxley Na, K, leak,
 *      synaptic, and the soma stimulus (the current I of Eq. 1);
 *   3. assembly of the Hines system for dV = V^{n+1} - V^n, backward Euler
 *      with the membrane conductance implicit (Eq. 2, in the symmetric
 *      finite-volume reading, see below);
 *   4. the Hines solve (Algorithm 1, backward sweep from the leaves to the
 *      root over parent[], then forward substitution), V += dV;
 *   5. exponential-Euler gate update at V^{n+1};
 *   6. synaptic decay g_syn *= exp(-dt/tau);
 *   7. threshold test at every detection point: an upward crossing of
 *      theta between V^n and V^{n+1} is a spike at the linearly
 *      interpolated time; each synapse s leaving that point then arrives
 *      at step n + 1 + round(delay_s/dt).  The detection points are the
 *      somata (default), or, when synapses carry source compartments, the
 *      distinct (neuron, compartment) points where synapses leave
 *      (Sec. 2's spike computation over the points of a morphology that
 *      hold a synapse).
 *
 * Readings of the paper (Sec. 2) taken here:
 *   - Eq. 2 prints the same g_{i+1/2} for both off-diagonals and a
 *     half-explicit rhs; on a tree the link between i and p(i) carries one
 *     conductance g_{i,p(i)}, so the matrix is symmetric (the Hines
 *     property stated in Sec. 2): a_i = c_i = -g_{i,p(i)}, and
 *     d_i = C_i/dt + G_i + sum_j g_ij,  rhs_i = -I_i + sum_j g_ij (V_j - V_i).
 *   - Algorithm 1's backward loop is printed from n-1 down to 0; the root has
 *     no parent, so it runs down to 1 and the root is finished by
 *     rhs[0] /= b[0].
 *   - Compartment indices are 0-based with parent[0] = -1, parent[i] < i.
 *   - Capacitance is constant (Cm * area).
 *   - The spike test is at the soma (or at the synapse points, as above),
 *     threshold theta, upward crossing only.
 *
 * Scheme 1 (scheme argument of orc_assemble / orc_simulate) is Eq. 2 taken
 * as printed instead: off-diagonals a_i = b_i = -g/2 (half of each link's
 * coupling implicit), d_i = C_i/dt - (a_i + b_i), and a rhs with the other
 * half of the coupling and the current I explicit -- Crank-Nicolson in the
 * diffusion, forward Euler in the membrane current.  In the dV form used
 * here: b_i = C_i/dt + sum_j g_ij / 2, a_i = c_i = -g_{i,p(i)} / 2,
 * rhs_i = -I_i + sum_j g_ij (V_j - V_i).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    double gNa, gK, gL;      /* mS/cm^2 */
    double ENa, EK, EL;      /* mV */
    double Cm;               /* uF/cm^2 */
    double Ra;               /* ohm*cm */
    double v_init;           /* mV */
    double threshold;        /* mV */
    double tau_syn;          /* ms */
    double e_syn;            /* mV */
} orc_params;

/* ---------------------------------------------------------------- geometry */

/* Lateral area of a cylinder, cm^2 (1 um^2 = 1e-8 cm^2). */
double orc_area_cm2(double L_um, double d_um) { return ORC_PI * d_um * L_um * 1e-8; }

/* Axial resistance of half a cylinder, MOhm. */
double orc_rhalf_Mohm(double Ra, double L_um, double d_um)
{
    double len_cm = 0.5 * L_um * 1e-4;
    double rad_cm = 0.5 * d_um * 1e-4;
    double xsec_cm2 = ORC_PI * rad_cm * rad_cm;
    return Ra * len_cm / xsec_cm2 * 1e-6;
}

/* Per-compartment constants of all neurons:
 *   area_cm2[i], C_nF[i] = Cm * area * 1e3 (uF -> nF),
 *   gax_uS[i] = 1 / (Rhalf_i + Rhalf_{p(i)}) for i != soma, 0 at the soma.
 */
void orc_geometry(int32_t n_neurons, const int64_t *off, const int32_t *parent,
                  const double *L, const double *d, const orc_params *p,
                  double *area_cm2, double *C_nF, double *gax_uS)
{
    for (int32_t k = 0; k < n_neurons; ++k) {
        int64_t base = off[k];
        int64_t n = off[k + 1] - off[k];
        for (int64_t i = 0; i < n; ++i) {
            int64_t g = base + i;
            area_cm2[g] = orc_area_cm2(L[g], d[g]);
            C_nF[g] = p->Cm * area_cm2[g] * 1e3;
            if (i == 0) {
                gax_uS[g] = 0.0;
            } else {
                int64_t q = base + parent[g];
                gax_uS[g] = 1.0 / (orc_rhalf_Mohm(p->Ra, L[g], d[g]) + orc_rhalf_Mohm(p->Ra, L[q], d[q]));
            }
        }
    }
}

/* ------------------------------------------------------------- HH kinetics */

/* x / (exp(x) - 1), with its limit 1 - x/2 near x = 0 (expm1 keeps the
 * quotient accurate close to the removable singularity). */
double orc_exprelr(double x)
{
    if (fabs(x) < 1e-6) return 1.0 - 0.5 * x;
    return x / expm1(x);
}

/* Hodgkin-Huxley rate functions (1/ms) at V (mV), rest at -65 mV, q10 = 1:
 * r = {alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n}. */
void orc_rates(double V, double *r)
{
    r[0] = orc_exprelr(-(V + 40.0) / 10.0);
    r[1] = 4.0 * exp(-(V + 65.0) / 18.0);
    r[2] = 0.07 * exp(-(V + 65.0) / 20.0);
    r[3] = 1.0 / (1.0 + exp(-(V + 35.0) / 10.0));
    r[4] = 0.1 * orc_exprelr(-(V + 55.0) / 10.0);
    r[5] = 0.125 * exp(-(V + 65.0) / 80.0);
}

/* Steady-state gates alpha / (alpha + beta) at V. */
void orc_gates_inf(double V, double *m, double *h, double *n)
{
    double r[6];
    orc_rates(V, r);
    *m = r[0] / (r[0] + r[1]);
    *h = r[2] / (r[2] + r[3]);
    *n = r[4] / (r[4] + r[5]);
}

/* Exponential Euler for one gate with frozen V: exact solution of
 * dx/dt = alpha (1 - x) - beta x over dt. */
static double gate_exp_euler(double x, double alpha, double beta, double dt)
{
    double xinf = alpha / (alpha + beta);
    return xinf + (x - xinf) * exp(-dt * (alpha + beta));
}

void orc_gate_step(double V, double dt, double *m, double *h, double *n)
{
    double r[6];
    orc_rates(V, r);
    *m = gate_exp_euler(*m, r[0], r[1], dt);
    *h = gate_exp_euler(*h, r[2], r[3], dt);
    *n = gate_exp_euler(*n, r[4], r[5], dt);
}

/* ------------------------------------------------------------- Hines solve */

/* Algorithm 1 (Sec. 2): a = upper, b = diagonal, c = lower, p = parent.
 * Row i holds b[i] on the diagonal and c[i] at column p[i]; row p[i] holds
 * a[i] at column i.  On return rhs holds the solution; b is overwritten.
 * If ops != NULL it is incremented by the floating-point operations done
 * (the paper counts 8 per compartment). */
void orc_hines_solve(double *a, double *b, double *c, double *rhs,
                     const int32_t *p, int32_t n, int64_t *ops)
{
    int64_t cnt = 0;
    /* backward sweep, leaves to root */
    for (int32_t i = n - 1; i >= 1; --i) {
        double factor = a[i] / b[i];
        b[p[i]] -= factor * c[i];
        rhs[p[i]] -= factor * rhs[i];
        cnt += 5;
    }
    rhs[0] /= b[0];
    cnt += 1;
    /* forward sweep, root to leaves */
    for (int32_t i = 1; i <= n - 1; ++i) {
        rhs[i] -= c[i] * rhs[p[i]];
        rhs[i] /= b[i];
        cnt += 3;
    }
    if (ops) *ops += cnt;
}

/* ---------------------------------------------------------------- assembly */

/* Membrane conductance G (uS) and current I (nA, outward positive) of one
 * compartment at V with the given gates and merged synaptic conductance. */
static void membrane(const orc_params *p, double area, double V, double m, double h,
                     double n, double gsyn, double *G, double *I)
{
    double s = area * 1e3;                     /* mS/cm^2 * cm^2 -> uS */
    double gna = p->gNa * s * m * m * m * h;
    double gk = p->gK * s * n * n * n * n;
    double gl = p->gL * s;
#ifndef ORC_SUM_REVERSED
    *G = gna + gk + gl + gsyn;
    *I = gna * (V - p->ENa) + gk * (V - p->EK) + gl * (V - p->EL) + gsyn * (V - p->e_syn);
#else
    /* the same sums in the opposite order: an equally valid FP64 evaluation
     * whose rounding differs, built as a second library to measure how much
     * a neuron's trajectory depends on the last bits of the arithmetic */
    *G = gsyn + gl + gk + gna;
    *I = gsyn * (V - p->e_syn) + gl * (V - p->EL) + gk * (V - p->EK) + gna * (V - p->ENa);
#endif
}

/* Hines system of one neuron for dV (Eq. 2, symmetric reading), scheme 0:
 *   b_i   = C_i/dt + G_i + sum_{j~i} g_ij
 *   a_i = c_i = -g_{i,p(i)}                       (i >= 1)
 *   rhs_i = -I_i + sum_{j~i} g_ij (V_j - V_i)  (+ stim at the soma)
 * scheme 1 (Eq. 2 as printed: half of each coupling implicit, I explicit):
 *   b_i   = C_i/dt + sum_{j~i} g_ij / 2,  a_i = c_i = -g_{i,p(i)} / 2,
 *   rhs_i as in scheme 0.
 * All arrays are local to the neuron (length n). */
void orc_assemble(int32_t n, const int32_t *parent, const double *V, const double *m,
                  const double *h, const double *nn, const double *gsyn,
                  const double *area, const double *C, const double *gax,
                  double stim_nA, const orc_params *p, double dt, int scheme,
                  double *a, double *b, double *c, double *rhs)
{
    const double w = scheme == 1 ? 0.5 : 1.0;  /* implicit share of each coupling */
    for (int32_t i = 0; i < n; ++i) {
        double G, I;
        membrane(p, area[i], V[i], m[i], h[i], nn[i], gsyn[i], &G, &I);
        b[i] = scheme == 1 ? C[i] / dt : C[i] / dt + G;
        rhs[i] = -I;
        a[i] = 0.0;
        c[i] = 0.0;
    }
    rhs[0] += stim_nA;
    for (int32_t i = 1; i < n; ++i) {
        int32_t q = parent[i];
        double g = gax[i];
        a[i] = -w * g;
        c[i] = -w * g;
        b[i] += w * g;
        b[q] += w * g;
        rhs[i] += g * (V[q] - V[i]);
        rhs[q] += g * (V[i] - V[q]);
    }
}

/* ----------------------------------------------------------- the network */

typedef struct {
    int64_t *ids;
    int64_t len, cap;
} idlist;

static int idlist_push(idlist *l, int64_t v)
{
    if (l->len == l->cap) {
        int64_t nc = l->cap ? 2 * l->cap : 64;
        int64_t *ni = (int64_t *)realloc(l->ids, (size_t)nc * sizeof(int64_t));
        if (!ni) return -1;
        l->ids = ni;
        l->cap = nc;
    }
    l->ids[l->len++] = v;
    return 0;
}

static int cmp_i64(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return (a > b) - (a < b);
}

/* Simulate n_steps steps of the whole network from rest (or from the given
 * initial V; gates start at their steady state for that V, g_syn at 0),
 * with the assembly of the given scheme (0 or 1, see orc_assemble).
 *
 * Outputs (any may be NULL):
 *   V_out, m_out, h_out, n_out, g_out [n_comp] state after the last step
 *                                             (g_out: merged synaptic conductance)
 *   soma_trace [n_neurons * (n_steps + 1)]    soma V at t_0 .. t_nsteps
 *   spk_neuron, spk_comp, spk_t [spk_cap]     spikes in detection order: each step
 *                                             by (neuron, compartment); spk_comp is
 *                                             the local compartment (0: soma)
 * syn_src_comp [n_syn] (may be NULL) is the local compartment of the source
 * neuron each synapse leaves from; with it the threshold test runs at every
 * distinct (src, src_comp) point instead of at every soma.
 * Returns 0, -1 on bad input, -2 on allocation failure, -3 if more than
 * spk_cap spikes were detected (n_spk still counts all of them). */
int orc_simulate(int32_t n_neurons, const int64_t *off, const int32_t *parent,
                 const double *L, const double *diam, const double *stim_nA,
                 int64_t n_syn, const int32_t *syn_src, const int32_t *syn_dst,
                 const int32_t *syn_comp, const double *syn_w, const double *syn_delay_ms,
                 const int32_t *syn_src_comp,
                 const orc_params *p, double dt, int scheme, int64_t n_steps, const double *V_init,
                 double *V_out, double *m_out, double *h_out, double *n_out,
                 double *g_out, double *soma_trace, int32_t *spk_neuron, int32_t *spk_comp, double *spk_t,
                 int64_t spk_cap, int64_t *n_spk, int n_threads)
{
    int64_t C = off[n_neurons];
    int rc = 0;
    if (dt <= 0.0 || n_neurons < 0 || scheme < 0 || scheme > 1) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    double *area = malloc((size_t)C * sizeof(double));
    double *Cn = malloc((size_t)C * sizeof(double));
    double *gax = malloc((size_t)C * sizeof(double));
    double *V = malloc((size_t)C * sizeof(double));
    double *m = malloc((size_t)C * sizeof(double));
    double *h = malloc((size_t)C * sizeof(double));
    double *nn = malloc((size_t)C * sizeof(double));
    double *gs = calloc((size_t)C, sizeof(double));
    double *wa = malloc((size_t)C * sizeof(double));
    double *wb = malloc((size_t)C * sizeof(double));
    double *wc = malloc((size_t)C * sizeof(double));
    double *wr = malloc((size_t)C * sizeof(double));
    /* detection points: pt_start[k] .. pt_start[k+1]-1 are neuron k's,
     * ascending compartment pt_comp; out_start / out_syn list the synapses
     * leaving each point, ascending synapse id */
    int64_t n_pt_max = syn_src_comp ? (n_syn > 0 ? n_syn : 1) : (n_neurons > 0 ? n_neurons : 1);
    int64_t *pt_start = calloc((size_t)n_neurons + 1, sizeof(int64_t));
    int32_t *pt_comp = malloc((size_t)n_pt_max * sizeof(int32_t));
    int64_t *syn_pt = malloc((size_t)(n_syn > 0 ? n_syn : 1) * sizeof(int64_t));
    unsigned char *fired = calloc((size_t)n_pt_max, 1);
    double *tfire = malloc((size_t)n_pt_max * sizeof(double));
    double *vpre = malloc((size_t)n_pt_max * sizeof(double));
    int64_t *out_start = calloc((size_t)n_pt_max + 1, sizeof(int64_t));
    int64_t *out_syn = malloc((size_t)(n_syn > 0 ? n_syn : 1) * sizeof(int64_t));
    int64_t *dsteps = malloc((size_t)(n_syn > 0 ? n_syn : 1) * sizeof(int64_t));
    idlist *ring = NULL;
    int64_t R = 2;
    if (!area || !Cn || !gax || !V || !m || !h || !nn || !gs || !wa || !wb || !wc || !wr ||
        !fired || !tfire || !vpre || !pt_start || !pt_comp || !syn_pt || !out_start || !out_syn || !dsteps) {
        rc = -2;
        goto done;
    }

    /* validate */
    for (int32_t k = 0; k < n_neurons; ++k) {
        int64_t n = off[k + 1] - off[k];
        if (n < 1 || parent[off[k]] != -1) { rc = -1; goto done; }
        for (int64_t i = 1; i < n; ++i)
            if (parent[off[k] + i] < 0 || parent[off[k] + i] >= i) { rc = -1; goto done; }
    }
    for (int64_t s = 0; s < n_syn; ++s) {
        if (syn_src[s] < 0 || syn_src[s] >= n_neurons || syn_dst[s] < 0 || syn_dst[s] >= n_neurons ||
            syn_comp[s] < 0 || syn_comp[s] >= off[syn_dst[s] + 1] - off[syn_dst[s]]) { rc = -1; goto done; }
        if (syn_src_comp && (syn_src_comp[s] < 0 || syn_src_comp[s] >= off[syn_src[s] + 1] - off[syn_src[s]])) {
            rc = -1;
            goto done;
        }
        dsteps[s] = (int64_t)llround(syn_delay_ms[s] / dt);
        if (dsteps[s] < 1) { rc = -1; goto done; }
        if (dsteps[s] + 2 > R) R = dsteps[s] + 2;
    }

    orc_geometry(n_neurons, off, parent, L, diam, p, area, Cn, gax);

    /* detection points and the point each synapse leaves from */
    int64_t n_pt = 0;
    if (!syn_src_comp) {
        for (int32_t k = 0; k < n_neurons; ++k) {
            pt_start[k] = k;
            pt_comp[k] = 0;
        }
        pt_start[n_neurons] = n_neurons;
        n_pt = n_neurons;
        for (int64_t s = 0; s < n_syn; ++s) syn_pt[s] = syn_src[s];
    } else {
        /* the distinct compartments each neuron's synapses leave from, by a
         * mark per compartment (one neuron at a time) */
        int64_t *by_src = malloc((size_t)(n_syn > 0 ? n_syn : 1) * sizeof(int64_t));
        int64_t *bstart = calloc((size_t)n_neurons + 1, sizeof(int64_t));
        int64_t *mark = malloc((size_t)(C > 0 ? C : 1) * sizeof(int64_t));
        if (!by_src || !bstart || !mark) { free(by_src); free(bstart); free(mark); rc = -2; goto done; }
        for (int64_t i = 0; i < C; ++i) mark[i] = -1;
        for (int64_t s = 0; s < n_syn; ++s) bstart[syn_src[s] + 1]++;
        for (int32_t k = 0; k < n_neurons; ++k) bstart[k + 1] += bstart[k];
        {
            int64_t *fill = calloc((size_t)n_neurons + 1, sizeof(int64_t));
            if (!fill) { free(by_src); free(bstart); free(mark); rc = -2; goto done; }
            for (int64_t s = 0; s < n_syn; ++s) by_src[bstart[syn_src[s]] + fill[syn_src[s]]++] = s;
            free(fill);
        }
        for (int32_t k = 0; k < n_neurons; ++k) {
            pt_start[k] = n_pt;
            int32_t nk = (int32_t)(off[k + 1] - off[k]);
            for (int64_t e = bstart[k]; e < bstart[k + 1]; ++e) mark[off[k] + syn_src_comp[by_src[e]]] = 0;
            for (int32_t i = 0; i < nk; ++i)
                if (mark[off[k] + i] == 0) {
                    mark[off[k] + i] = n_pt;
                    pt_comp[n_pt++] = i;
                }
            for (int64_t e = bstart[k]; e < bstart[k + 1]; ++e) {
                int64_t s = by_src[e];
                syn_pt[s] = mark[off[k] + syn_src_comp[s]];
            }
        }
        pt_start[n_neurons] = n_pt;
        free(by_src); free(bstart); free(mark);
    }

    /* synapses leaving each point, ascending synapse id */
    for (int64_t s = 0; s < n_syn; ++s) out_start[syn_pt[s] + 1]++;
    for (int64_t q = 0; q < n_pt; ++q) out_start[q + 1] += out_start[q];
    {
        int64_t *fill = calloc((size_t)n_pt + 1, sizeof(int64_t));
        if (!fill) { rc = -2; goto done; }
        for (int64_t s = 0; s < n_syn; ++s) out_syn[out_start[syn_pt[s]] + fill[syn_pt[s]]++] = s;
        free(fill);
    }
    ring = calloc((size_t)R, sizeof(idlist));
    if (!ring) { rc = -2; goto done; }

    /* initial state */
    for (int64_t i = 0; i < C; ++i) {
        V[i] = V_init ? V_init[i] : p->v_init;
        orc_gates_inf(V[i], &m[i], &h[i], &nn[i]);
    }
    if (soma_trace)
        for (int32_t k = 0; k < n_neurons; ++k) soma_trace[(int64_t)k * (n_steps + 1)] = V[off[k]];

    const double decay = exp(-dt / p->tau_syn);
    int64_t nsp = 0;
    for (int64_t step = 0; step < n_steps; ++step) {
        /* 1. deliver events due at this step, ascending synapse id */
        idlist *due = &ring[step % R];
        if (due->len > 1) qsort(due->ids, (size_t)due->len, sizeof(int64_t), cmp_i64);
        for (int64_t e = 0; e < due->len; ++e) {
            int64_t s = due->ids[e];
            gs[off[syn_dst[s]] + syn_comp[s]] += syn_w[s];
        }
        due->len = 0;

        /* 2-7. every neuron independently */
#pragma omp parallel for schedule(dynamic, 4)
        for (int32_t k = 0; k < n_neurons; ++k) {
            int64_t b0 = off[k];
            int32_t n = (int32_t)(off[k + 1] - off[k]);
            for (int64_t q = pt_start[k]; q < pt_start[k + 1]; ++q) vpre[q] = V[b0 + pt_comp[q]];
            orc_assemble(n, parent + b0, V + b0, m + b0, h + b0, nn + b0, gs + b0,
                         area + b0, Cn + b0, gax + b0, stim_nA[k], p, dt, scheme,
                         wa + b0, wb + b0, wc + b0, wr + b0);
            orc_hines_solve(wa + b0, wb + b0, wc + b0, wr + b0, parent + b0, n, NULL);
            for (int32_t i = 0; i < n; ++i) {
                V[b0 + i] += wr[b0 + i];
                orc_gate_step(V[b0 + i], dt, &m[b0 + i], &h[b0 + i], &nn[b0 + i]);
                gs[b0 + i] *= decay;
            }
            for (int64_t q = pt_start[k]; q < pt_start[k + 1]; ++q) {
                double v0 = vpre[q], v1 = V[b0 + pt_comp[q]];
                fired[q] = 0;
                if (v0 < p->threshold && v1 >= p->threshold) {
                    fired[q] = 1;
                    tfire[q] = (double)step * dt + dt * (p->threshold - v0) / (v1 - v0);
                }
            }
        }
        /* spikes in point order (neuron, compartment); schedule their events */
        for (int32_t k = 0; k < n_neurons; ++k) {
            for (int64_t q = pt_start[k]; q < pt_start[k + 1]; ++q) {
                if (!fired[q]) continue;
                if (nsp < spk_cap) {
                    if (spk_neuron) spk_neuron[nsp] = k;
                    if (spk_comp) spk_comp[nsp] = pt_comp[q];
                    if (spk_t) spk_t[nsp] = tfire[q];
                } else {
                    rc = -3;
                }
                nsp++;
                for (int64_t o = out_start[q]; o < out_start[q + 1]; ++o) {
                    int64_t s = out_syn[o];
                    int64_t arrival = step + 1 + dsteps[s];
                    if (idlist_push(&ring[arrival % R], s)) { rc = -2; goto done; }
                }
            }
        }
        if (soma_trace)
            for (int32_t k = 0; k < n_neurons; ++k)
                soma_trace[(int64_t)k * (n_steps + 1) + step + 1] = V[off[k]];
    }
    if (n_spk) *n_spk = nsp;
    if (V_out) memcpy(V_out, V, (size_t)C * sizeof(double));
    if (m_out) memcpy(m_out, m, (size_t)C * sizeof(double));
    if (h_out) memcpy(h_out, h, (size_t)C * sizeof(double));
    if (n_out) memcpy(n_out, nn, (size_t)C * sizeof(double));
    if (g_out) memcpy(g_out, gs, (size_t)C * sizeof(double));

done:
    if (ring) {
        for (int64_t r = 0; r < R; ++r) free(ring[r].ids);
        free(ring);
    }
    free(area); free(Cn); free(gax); free(V); free(m); free(h); free(nn); free(gs);
    free(wa); free(wb); free(wc); free(wr); free(fired); free(tfire); free(vpre);
    free(pt_start); free(pt_comp); free(syn_pt);
    free(out_start); free(out_syn); free(dsteps);
    return rc;
}

/* ------------------------------------------------ a steppable network part */

/* The same step as orc_simulate (soma detection, scheme 0 or 1), kept as a
 * state that advances a few steps at a time and takes spikes of neurons
 * simulated elsewhere: the part of a network that one node of the paper's
 * cluster holds (Sec. 2: local steps, then the spikes of the global step
 * exchanged with MPI_AllGather and stored in the global buffer).  Synapse
 * sources n_neurons .. n_neurons + n_ext - 1 are external; orc_part_inject
 * schedules their synapses' events exactly as a local spike's are
 * scheduled (arrival n + 1 + round(delay/dt), ascending synapse id within a
 * step). */
typedef struct {
    int32_t N, n_ext, scheme;
    int64_t C, S, step, R;
    double dt, decay;
    orc_params p;
    int64_t *off;
    int32_t *parent;
    double *stim, *area, *Cn, *gax, *V, *m, *h, *n, *gs, *wa, *wb, *wc, *wr, *w, *vpre;
    int32_t *dst, *comp;
    int64_t *dsteps, *out_start, *out_syn;
    unsigned char *fired;
    idlist *ring;
    idlist hist;            /* spikes so far: neuron * 2^32 + step... as (step << 31 | neuron) */
} orc_part;

void orc_part_destroy(orc_part *q)
{
    if (!q) return;
    if (q->ring) {
        for (int64_t r = 0; r < q->R; ++r) free(q->ring[r].ids);
        free(q->ring);
    }
    free(q->hist.ids);
    free(q->off); free(q->parent); free(q->stim); free(q->area); free(q->Cn); free(q->gax);
    free(q->V); free(q->m); free(q->h); free(q->n); free(q->gs); free(q->wa); free(q->wb); free(q->wc);
    free(q->wr); free(q->w); free(q->vpre); free(q->dst); free(q->comp); free(q->dsteps);
    free(q->out_start); free(q->out_syn); free(q->fired);
    free(q);
}

orc_part *orc_part_create(int32_t n_neurons, const int64_t *off, const int32_t *parent, const double *L,
                          const double *diam, const double *stim_nA, int64_t n_syn, const int32_t *syn_src,
                          const int32_t *syn_dst, const int32_t *syn_comp, const double *syn_w,
                          const double *syn_delay_ms, int32_t n_ext, const orc_params *p, double dt, int scheme)
{
    if (n_neurons < 0 || n_ext < 0 || dt <= 0.0 || scheme < 0 || scheme > 1) return NULL;
    orc_part *q = calloc(1, sizeof(orc_part));
    if (!q) return NULL;
    const int64_t C = off[n_neurons], S = n_syn, NS = (int64_t)n_neurons + n_ext;
    q->N = n_neurons; q->n_ext = n_ext; q->scheme = scheme; q->C = C; q->S = S; q->dt = dt; q->p = *p; q->R = 2;
    q->off = malloc(((size_t)n_neurons + 1) * sizeof(int64_t));
    q->parent = malloc((size_t)(C > 0 ? C : 1) * sizeof(int32_t));
    q->stim = malloc((size_t)(n_neurons > 0 ? n_neurons : 1) * sizeof(double));
    double **arr[] = {&q->area, &q->Cn, &q->gax, &q->V, &q->m, &q->h, &q->n, &q->gs, &q->wa, &q->wb, &q->wc, &q->wr};
    for (size_t k = 0; k < sizeof(arr) / sizeof(arr[0]); ++k) *arr[k] = calloc((size_t)(C > 0 ? C : 1), sizeof(double));
    q->w = malloc((size_t)(S > 0 ? S : 1) * sizeof(double));
    q->dst = malloc((size_t)(S > 0 ? S : 1) * sizeof(int32_t));
    q->comp = malloc((size_t)(S > 0 ? S : 1) * sizeof(int32_t));
    q->dsteps = malloc((size_t)(S > 0 ? S : 1) * sizeof(int64_t));
    q->out_start = calloc((size_t)NS + 1, sizeof(int64_t));
    q->out_syn = malloc((size_t)(S > 0 ? S : 1) * sizeof(int64_t));
    q->fired = calloc((size_t)(n_neurons > 0 ? n_neurons : 1), 1);
    q->vpre = malloc((size_t)(n_neurons > 0 ? n_neurons : 1) * sizeof(double));
    if (!q->off || !q->parent || !q->stim || !q->w || !q->dst || !q->comp || !q->dsteps || !q->out_start ||
        !q->out_syn || !q->fired || !q->vpre) { orc_part_destroy(q); return NULL; }
    for (size_t k = 0; k < sizeof(arr) / sizeof(arr[0]); ++k) if (!*arr[k]) { orc_part_destroy(q); return NULL; }
    memcpy(q->off, off, ((size_t)n_neurons + 1) * sizeof(int64_t));
    memcpy(q->parent, parent, (size_t)C * sizeof(int32_t));
    for (int32_t k = 0; k < n_neurons; ++k) q->stim[k] = stim_nA ? stim_nA[k] : 0.0;
    for (int32_t k = 0; k < n_neurons; ++k) {
        int64_t nk = off[k + 1] - off[k];
        if (nk < 1 || parent[off[k]] != -1) { orc_part_destroy(q); return NULL; }
        for (int64_t i = 1; i < nk; ++i)
            if (parent[off[k] + i] < 0 || parent[off[k] + i] >= i) { orc_part_destroy(q); return NULL; }
    }
    for (int64_t s = 0; s < S; ++s) {
        if (syn_src[s] < 0 || syn_src[s] >= NS || syn_dst[s] < 0 || syn_dst[s] >= n_neurons ||
            syn_comp[s] < 0 || syn_comp[s] >= off[syn_dst[s] + 1] - off[syn_dst[s]]) { orc_part_destroy(q); return NULL; }
        q->dsteps[s] = (int64_t)llround(syn_delay_ms[s] / dt);
        if (q->dsteps[s] < 1) { orc_part_destroy(q); return NULL; }
        if (q->dsteps[s] + 2 > q->R) q->R = q->dsteps[s] + 2;
        q->w[s] = syn_w[s];
        q->dst[s] = syn_dst[s];
        q->comp[s] = syn_comp[s];
        q->out_start[syn_src[s] + 1]++;
    }
    for (int64_t k = 0; k < NS; ++k) q->out_start[k + 1] += q->out_start[k];
    {
        int64_t *fill = calloc((size_t)NS + 1, sizeof(int64_t));
        if (!fill) { orc_part_destroy(q); return NULL; }
        for (int64_t s = 0; s < S; ++s) q->out_syn[q->out_start[syn_src[s]] + fill[syn_src[s]]++] = s;
        free(fill);
    }
    q->ring = calloc((size_t)q->R, sizeof(idlist));
    if (!q->ring) { orc_part_destroy(q); return NULL; }
    orc_geometry(n_neurons, off, parent, L, diam, p, q->area, q->Cn, q->gax);
    for (int64_t i = 0; i < C; ++i) {
        q->V[i] = p->v_init;
        orc_gates_inf(q->V[i], &q->m[i], &q->h[i], &q->n[i]);
    }
    q->decay = exp(-dt / p->tau_syn);
    return q;
}

/* Schedules the events of source src (local neuron or external source) for
 * its spike in step st; -1 if an arrival would already be past. */
static int part_schedule(orc_part *q, int64_t src, int64_t st)
{
    for (int64_t o = q->out_start[src]; o < q->out_start[src + 1]; ++o) {
        int64_t s = q->out_syn[o];
        int64_t arrival = st + 1 + q->dsteps[s];
        if (arrival < q->step) return -1;
        if (idlist_push(&q->ring[arrival % q->R], s)) return -2;
    }
    return 0;
}

int orc_part_step(orc_part *q, int64_t n_steps)
{
    for (int64_t k = 0; k < n_steps; ++k) {
        const int64_t step = q->step;
        idlist *due = &q->ring[step % q->R];
        if (due->len > 1) qsort(due->ids, (size_t)due->len, sizeof(int64_t), cmp_i64);
        for (int64_t e = 0; e < due->len; ++e) {
            int64_t s = due->ids[e];
            q->gs[q->off[q->dst[s]] + q->comp[s]] += q->w[s];
        }
        due->len = 0;
        for (int32_t j = 0; j < q->N; ++j) {
            int64_t b0 = q->off[j];
            int32_t nj = (int32_t)(q->off[j + 1] - b0);
            q->vpre[j] = q->V[b0];
            orc_assemble(nj, q->parent + b0, q->V + b0, q->m + b0, q->h + b0, q->n + b0, q->gs + b0, q->area + b0,
                         q->Cn + b0, q->gax + b0, q->stim[j], &q->p, q->dt, q->scheme, q->wa + b0, q->wb + b0,
                         q->wc + b0, q->wr + b0);
            orc_hines_solve(q->wa + b0, q->wb + b0, q->wc + b0, q->wr + b0, q->parent + b0, nj, NULL);
            for (int32_t i = 0; i < nj; ++i) {
                q->V[b0 + i] += q->wr[b0 + i];
                orc_gate_step(q->V[b0 + i], q->dt, &q->m[b0 + i], &q->h[b0 + i], &q->n[b0 + i]);
                q->gs[b0 + i] *= q->decay;
            }
            q->fired[j] = q->vpre[j] < q->p.threshold && q->V[b0] >= q->p.threshold;
        }
        for (int32_t j = 0; j < q->N; ++j) {
            if (!q->fired[j]) continue;
            if (idlist_push(&q->hist, (step << 31) | (int64_t)j)) return -2;
            if (part_schedule(q, j, step)) return -2;
        }
        q->step = step + 1;
    }
    return 0;
}

/* The local spikes of steps step0 .. step0 + n_steps - 1, in step order
 * (neurons ascending within a step); returns how many (all of them, even
 * beyond cap). */
int64_t orc_part_fired(const orc_part *q, int64_t step0, int32_t n_steps, int32_t *neuron, int64_t *step, int64_t cap)
{
    int64_t k = 0;
    for (int64_t e = 0; e < q->hist.len; ++e) {
        int64_t st = q->hist.ids[e] >> 31, j = q->hist.ids[e] & 0x7FFFFFFF;
        if (st < step0 || st >= step0 + n_steps) continue;
        if (k < cap) { neuron[k] = (int32_t)j; step[k] = st; }
        ++k;
    }
    return k;
}

/* Spikes of external sources (0 .. n_ext - 1) in the given steps; 0, -1 if a
 * source is out of range or an event would arrive in a step already run. */
int orc_part_inject(orc_part *q, int64_t n, const int32_t *ext_src, const int64_t *step)
{
    for (int64_t k = 0; k < n; ++k) {
        if (ext_src[k] < 0 || ext_src[k] >= q->n_ext || step[k] >= q->step) return -1;
        int rc = part_schedule(q, (int64_t)q->N + ext_src[k], step[k]);
        if (rc) return rc;
    }
    return 0;
}

/* V, m, h, n and the merged synaptic conductance (any may be NULL), and the
 * number of steps run. */
int64_t orc_part_read(const orc_part *q, double *V, double *m, double *h, double *n, double *g)
{
    size_t b = (size_t)q->C * sizeof(double);
    if (V) memcpy(V, q->V, b);
    if (m) memcpy(m, q->m, b);
    if (h) memcpy(h, q->h, b);
    if (n) memcpy(n, q->n, b);
    if (g) memcpy(g, q->gs, b);
    return q->step;
}

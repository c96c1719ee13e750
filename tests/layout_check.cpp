// Host-side check of the FP32c work-item layout (paper_2005_06332_gb300/csrc/
// mm_layout.cpp), built and run by tests/test_layout_paths.py.
//
// For every work item it checks the invariants the kernels rely on for
// their shared-memory (16-bit) and giant (32-bit) path tables -- every index
// inside the item, the paths partitioning its compartments, each
// compartment after a path head having the previous one as its parent, path
// levels, sweep bundles holding whole neurons, the fold lists and the
// "alone" flags -- and then replays the FP32c kernels' path-by-path
// elimination and substitution in float on random coefficients, comparing
// with the elimination of Algorithm 1 in double over the same parent array:
// the diagonal split into a passive part (eliminated in double, kept as a
// float pair) and an active part that the float sweep carries up the tree
// as its perturbation, the couplings as float pairs, reciprocals refined by
// one Newton step.
//
// Paths of at least <warp path> compartments (optional 5th argument, 0 =
// none) are swept as the step kernel's whole warps sweep them: the path cut
// into 32 chunks, chunk products of the 2x2 matrices of the active part's
// recurrence and of the affine rhs and substitution maps combined by
// inclusive scans round by round, then the serial recurrences through each
// chunk from the scanned values (the lanes emulated one after another).
//
// Usage: layout_check <network file> <group_comps> <regular smem limit> <large smem limit> [warp path]
// Network file: int32 N | int64 C | int64 comp_offset[N+1] | int32 parent[C].
// Prints "bad=<violations> maxrel=<largest relative error>"; exit 0 iff bad == 0.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "mm_layout.h"

using namespace mmk;

namespace {

// Inclusive scan over 32 lanes, round by round as with shuffles (lane k
// combines with lane k - off); combine(own, earlier) returns the composition.
template <class V, class F>
void lane_scan(V *v, F combine)
{
    for (int off = 1; off < 32; off <<= 1) {
        V nv[32];
        for (int k = 0; k < 32; ++k) nv[k] = k >= off ? combine(v[k], v[k - off]) : v[k];
        for (int k = 0; k < 32; ++k) v[k] = nv[k];
    }
}

struct Mat {
    float m00, m01, m10, m11;
};
struct Aff {
    float a, b;
};

float rcp_nr(float x)
{
    const float r = 1.f / x;
    return std::fma(r, std::fma(-x, r, 1.f), r);
}

// Coefficients of one compartment for the sweeps: the implicit coupling to
// its parent (gh + gl), the passive eliminated diagonal's nearest float dh,
// f0 = gh / dh, and the factor fg = f0 gh of the active part's recurrence.
struct Co {
    std::vector<float> gh, gl, dh, f0, fg;
};

// One step of the serial elimination at compartment j of a path: its
// active part eb and rhs rb in, the next compartment's (ep, rp) out.
inline void elim_step(const Co &k, int j, float &eb, float &rb, float ep, float rp, float *f_out, float *c_out)
{
    const float dd = k.dh[j] + eb;
    const float r0 = 1.f / dd;
    const float inv = std::fma(r0, std::fma(-dd, r0, 1.f), r0);
    const float f = std::fma(k.gh[j], inv, k.gl[j] * inv);
    *f_out = f;
    *c_out = rb * inv;
    rb = std::fma(f, rb, rp);
    eb = std::fma(k.fg[j] * r0, eb, ep);
}

// The warp-swept elimination of the interior of the path [h, e): leaves
// (f_j, c_j) in (se, sr) for h < j < e and returns the head's (eh, rh).
void warp_eliminate(int h, int e, std::vector<float> &se, std::vector<float> &sr, const Co &k, float *eh, float *rh)
{
    const int m = e - 1 - h, cs = (m + 31) / 32;
    const float leafe = se[e - 1], leafr = sr[e - 1];
    Mat M[32];
    for (int ln = 0; ln < 32; ++ln) {
        const int t0 = std::min(ln * cs, m), t1 = std::min(t0 + cs, m);
        Mat q{1.f, 0.f, 0.f, 1.f};
        for (int tt = t0; tt < t1; ++tt) {
            const int j = e - 1 - tt;
            const float D = k.dh[j], En = se[j - 1];
            const float A = k.fg[j] + En, B = En * D;
            const float n00 = std::fma(A, q.m00, B * q.m10), n01 = std::fma(A, q.m01, B * q.m11);
            const float n10 = std::fma(D, q.m10, q.m00), n11 = std::fma(D, q.m11, q.m01);
            const float s = 1.f / (n00 + n01 + n10 + n11);
            q = {n00 * s, n01 * s, n10 * s, n11 * s};
        }
        M[ln] = q;
    }
    lane_scan(M, [](const Mat &o, const Mat &a) {
        const float n00 = std::fma(o.m00, a.m00, o.m01 * a.m10), n01 = std::fma(o.m00, a.m01, o.m01 * a.m11);
        const float n10 = std::fma(o.m10, a.m00, o.m11 * a.m10), n11 = std::fma(o.m10, a.m01, o.m11 * a.m11);
        const float s = 1.f / (std::fabs(n00) + std::fabs(n01) + std::fabs(n10) + std::fabs(n11));
        return Mat{n00 * s, n01 * s, n10 * s, n11 * s};
    });
    float eb0[32];
    Aff F[32];
    float nbe[32], nbr[32];
    for (int ln = 0; ln < 32; ++ln) {
        const Mat x = ln ? M[ln - 1] : Mat{1.f, 0.f, 0.f, 1.f};
        eb0[ln] = std::fma(x.m00, leafe, x.m01) / std::fma(x.m10, leafe, x.m11);
        const int t0 = std::min(ln * cs, m), t1 = std::min(t0 + cs, m);
        float eb = eb0[ln], A = 1.f, B = 0.f, rb = 0.f, fj, cj;
        nbe[ln] = nbr[ln] = 0.f;
        for (int tt = t0; tt < t1; ++tt) {
            const int j = e - 1 - tt;
            rb = B;
            elim_step(k, j, eb, rb, se[j - 1], sr[j - 1], &fj, &cj);
            A *= fj;
            B = rb;
            nbe[ln] = se[j - 1];
            nbr[ln] = sr[j - 1];
        }
        F[ln] = {A, B};
    }
    lane_scan(F, [](const Aff &o, const Aff &a) { return Aff{o.a * a.a, std::fma(o.a, a.b, o.b)}; });
    const int lastl = (m - 1) / cs;
    for (int ln = 0; ln < 32; ++ln) {
        const Aff x = ln ? F[ln - 1] : Aff{1.f, 0.f};
        const int t0 = std::min(ln * cs, m), t1 = std::min(t0 + cs, m);
        float eb = eb0[ln], rb = std::fma(x.a, leafr, x.b);
        for (int tt = t0; tt < t1; ++tt) {
            const int j = e - 1 - tt;
            const float we = tt + 1 < t1 ? se[j - 1] : nbe[ln], wr = tt + 1 < t1 ? sr[j - 1] : nbr[ln];
            float fj, cj;
            elim_step(k, j, eb, rb, we, wr, &fj, &cj);
            se[j] = fj;
            sr[j] = cj;
        }
        if (ln == lastl) {
            *eh = eb;
            *rh = rb;
        }
    }
}

// The warp-swept substitution x_j = f_j x_{j-1} + c_j for h < j < e from the
// head's x.
void warp_substitute(int h, int e, float xh, const std::vector<float> &sd, std::vector<float> &sr)
{
    const int m = e - 1 - h, cs = (m + 31) / 32;
    Aff F[32];
    for (int ln = 0; ln < 32; ++ln) {
        const int t0 = std::min(ln * cs, m), t1 = std::min(t0 + cs, m);
        float A = 1.f, B = 0.f;
        for (int tt = t0; tt < t1; ++tt) {
            const int j = h + 1 + tt;
            A *= sd[j];
            B = std::fma(sd[j], B, sr[j]);
        }
        F[ln] = {A, B};
    }
    lane_scan(F, [](const Aff &o, const Aff &a) { return Aff{o.a * a.a, std::fma(o.a, a.b, o.b)}; });
    for (int ln = 0; ln < 32; ++ln) {
        const Aff x = ln ? F[ln - 1] : Aff{1.f, 0.f};
        const int t0 = std::min(ln * cs, m), t1 = std::min(t0 + cs, m);
        float xs = std::fma(x.a, xh, x.b);
        for (int tt = t0; tt < t1; ++tt) {
            const int j = h + 1 + tt;
            xs = std::fma(sd[j], xs, sr[j]);
            sr[j] = xs;
        }
    }
}

struct Tables {  // an item's tables widened to int
    std::vector<int> nrn;    // 4 per sweep bundle: path0, npath, nlevel, loff0
    std::vector<int> path;   // 4 per path: head, end, parent, neuron
    std::vector<int> alone;  // per path
    std::vector<int> fold;   // 2 per entry: path, parent compartment
    std::vector<int> loffs, mcnt;
};

Tables read_tables(const GroupRec &G, const unsigned char *b, bool wide, long long *bad)
{
    Tables T;
    int nlo = 0;
    if (wide) {
        const NrnG *nr = (const NrnG *)b;
        const PathG *P = (const PathG *)(b + G.path_off);
        const KidG *F = (const KidG *)(b + G.fold_off);
        for (int k = 0; k < G.nbundle; ++k) {
            T.nrn.insert(T.nrn.end(), {nr[k].path0, nr[k].npath, nr[k].nlevel, nr[k].loff0});
            nlo += nr[k].nlevel + 1;
        }
        for (int p = 0; p < G.npath; ++p) {
            T.path.insert(T.path.end(), {P[p].head, P[p].end, P[p].parent, P[p].nflag & kPathNeuronG});
            T.alone.push_back((P[p].nflag & kPathAloneG) != 0);
            T.fold.insert(T.fold.end(), {F[p].x, F[p].y});
        }
        const int32_t *lo = (const int32_t *)(b + G.loffs_off), *mc = (const int32_t *)(b + G.mcnt_off);
        T.loffs.assign(lo, lo + nlo);
        T.mcnt.assign(mc, mc + nlo);
        if (G.mcnt_off + 4LL * nlo > G.meta_bytes) ++*bad;
    } else {
        const NrnQ *nr = (const NrnQ *)b;
        const PathQ *P = (const PathQ *)(b + G.path_off);
        const KidQ *F = (const KidQ *)(b + G.fold_off);
        for (int k = 0; k < G.nbundle; ++k) {
            T.nrn.insert(T.nrn.end(), {nr[k].path0, nr[k].npath, nr[k].nlevel, nr[k].loff0});
            nlo += nr[k].nlevel + 1;
        }
        for (int p = 0; p < G.npath; ++p) {
            T.path.insert(T.path.end(), {P[p].head, P[p].end, P[p].parent, P[p].nflag & kPathNeuron});
            T.alone.push_back((P[p].nflag & kPathAlone) != 0);
            T.fold.insert(T.fold.end(), {(int)(F[p] & 0xFFFFu), (int)(F[p] >> 16)});
        }
        const int16_t *lo = (const int16_t *)(b + G.loffs_off), *mc = (const int16_t *)(b + G.mcnt_off);
        T.loffs.assign(lo, lo + nlo);
        T.mcnt.assign(mc, mc + nlo);
        if (G.mcnt_off + 2LL * nlo > G.meta_bytes) ++*bad;
    }
    if (G.path_off % 16 || G.fold_off % 4 || G.meta_bytes % 16) ++*bad;
    return T;
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc < 5) return 2;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t N;
    int64_t C;
    if (std::fread(&N, 4, 1, f) != 1 || std::fread(&C, 8, 1, f) != 1) return 2;
    std::vector<int64_t> off((size_t)N + 1);
    std::vector<int32_t> par((size_t)C);
    if (std::fread(off.data(), 8, off.size(), f) != off.size() || std::fread(par.data(), 4, par.size(), f) != par.size())
        return 2;
    std::fclose(f);
    std::vector<double> L((size_t)C, 10.0), D((size_t)C, 1.0);
    mmh::LayoutInput in{};
    in.N = N;
    in.comp_offset = off.data();
    in.parent = par.data();
    in.length_um = L.data();
    in.diam_um = D.data();
    in.dt = 0.025;
    in.group_comps = std::atoi(argv[2]);
    in.max_group_comps = 1 << 30;
    in.smem_per_comp = 24;
    in.smem_per_seg = 0;
    in.giant_smem_limit = std::atoi(argv[3]);
    in.big_smem_limit = std::atoi(argv[4]);
    in.path_items = true;
    in.smem_per_path = 8;
    const int warp_min = argc > 5 ? std::atoi(argv[5]) : 0;
    long long nwarp_paths = 0;
    mmh::Layout lay;
    bool invalid = false;
    const std::string err = mmh::build_layout(in, lay, &invalid);
    if (!err.empty()) {
        std::printf("layout error: %s\n", err.c_str());
        return 1;
    }
    long long bad = 0;
    double maxrel = 0.0;
    std::mt19937 rng(1);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    int64_t gcomps = 0, gpaths = 0, covered = 0;
    const int nitems = (int)lay.groups.size();
    for (int gi = 0; gi < nitems; ++gi) {
        const GroupRec &G = lay.groups[(size_t)gi];
        const bool wide = gi >= lay.n_small + lay.n_big;
        const Tables T = read_tables(G, lay.meta.data() + G.meta_off, wide, &bad);
        if (wide) {
            if (G.scratch0 != gcomps || G.pscratch0 != gpaths) ++bad;
            gcomps += G.ncomp;
            gpaths += G.npath;
        } else {
            const int64_t need = G.meta_bytes + 24LL * G.ncomp + 8LL * G.npath;
            if (need > (gi < lay.n_small ? lay.max_smem : lay.big_max_smem) || G.ncomp > 32767 || G.npath > 32767) ++bad;
        }
        covered += G.ncomp;
        const int64_t c0 = G.comp0;
        auto H = [&](int p) { return T.path[4 * p]; };
        auto E = [&](int p) { return T.path[4 * p + 1]; };
        auto Pa = [&](int p) { return T.path[4 * p + 2]; };
        // nrnof: the sweep bundle of each path
        std::vector<int> cover(G.ncomp, 0), pathof(G.ncomp, -1), levelof(G.npath, -1), nrnof(G.npath, -1);
        int pcount = 0;
        if (G.nbundle < 1 || G.nbundle > G.nneuron) ++bad;
        for (int k = 0; k < G.nbundle; ++k) {
            const int p0 = T.nrn[4 * k], np = T.nrn[4 * k + 1], nl = T.nrn[4 * k + 2], l0 = T.nrn[4 * k + 3];
            if (p0 != pcount || l0 < 0 || l0 + nl >= (int)T.loffs.size() + 1) { ++bad; continue; }
            const int *lo = T.loffs.data() + l0;
            if (lo[0] != p0 || lo[nl] != p0 + np) ++bad;
            for (int l = 0; l < nl; ++l) {
                if (lo[l + 1] <= lo[l]) ++bad;
                int prev = 1 << 30;
                for (int p = lo[l]; p < lo[l + 1]; ++p) {
                    levelof[p] = l;
                    nrnof[p] = k;
                    if (E(p) - H(p) > prev) ++bad;  // longest first
                    prev = E(p) - H(p);
                }
            }
            pcount += np;
        }
        if (pcount != G.npath) ++bad;
        // every neuron has one soma path and all its paths in one bundle
        std::vector<int> somas(G.nneuron, 0), bundle_of(G.nneuron, -1);
        for (int p = 0; p < G.npath; ++p) {
            const int nrn = T.path[4 * p + 3];
            if (nrn < 0 || nrn >= G.nneuron) { ++bad; continue; }
            if (Pa(p) < 0) somas[nrn]++;
            if (bundle_of[nrn] < 0) bundle_of[nrn] = nrnof[p];
            else if (bundle_of[nrn] != nrnof[p]) ++bad;
        }
        for (int k = 0; k < G.nneuron; ++k) if (somas[k] != 1) ++bad;
        for (int p = 0; p < G.npath; ++p) {
            if (H(p) < 0 || E(p) > G.ncomp || E(p) <= H(p)) { ++bad; continue; }
            for (int j = H(p); j < E(p); ++j) { cover[j]++; pathof[j] = p; }
            for (int j = H(p) + 1; j < E(p); ++j)
                if (lay.pdist[(size_t)(c0 + j)] != 1) ++bad;  // parent is the compartment before
            if (Pa(p) < 0) {
                if (lay.pdist[(size_t)(c0 + H(p))] != 0 || levelof[p] != 0) ++bad;  // somata on level 0
            } else if (lay.pdist[(size_t)(c0 + H(p))] >= 0 || H(p) + lay.pdist[(size_t)(c0 + H(p))] != Pa(p)) {
                ++bad;  // heads carry the negated parent distance
            }
            if (E(p) < G.ncomp && lay.pdist[(size_t)(c0 + E(p))] == 1) ++bad;  // ends at a leaf
        }
        for (int j = 0; j < G.ncomp; ++j)
            if (cover[j] != 1) { ++bad; break; }
        std::vector<int> share(G.ncomp, 0);
        for (int p = 0; p < G.npath; ++p) if (Pa(p) >= 0) share[Pa(p)]++;
        for (int p = 0; p < G.npath; ++p) if ((Pa(p) >= 0 && share[Pa(p)] == 1) != (T.alone[p] != 0)) ++bad;
        for (int k = 0; k < G.nbundle; ++k) {
            const int nl = T.nrn[4 * k + 2], l0 = T.nrn[4 * k + 3];
            const int *lo = T.loffs.data() + l0, *mc = T.mcnt.data() + l0;
            for (int l = 0; l < nl; ++l) {
                std::vector<int> seen(G.npath, 0);
                int prev = 1 << 30;
                if (mc[l] < 0 || mc[l] > lo[l + 1] - lo[l] || (l == 0 && mc[l] != 0)) ++bad;
                for (int z = lo[l]; z < lo[l + 1]; ++z) {
                    const int c = T.fold[2 * z], att = T.fold[2 * z + 1];
                    if (c < lo[l] || c >= lo[l + 1]) { ++bad; continue; }
                    seen[c]++;
                    const bool shared = z < lo[l] + mc[l];
                    if (Pa(c) >= 0 && shared == (T.alone[c] != 0)) ++bad;
                    if (l > 0) {
                        if (Pa(c) != att || att < 0 || att >= G.ncomp || levelof[pathof[att]] != l - 1 ||
                            nrnof[pathof[att]] != k || att >= E(pathof[att]) - 1)
                            ++bad;
                        if (shared) {
                            if (att > prev) ++bad;
                            prev = att;
                        }
                    }
                }
                for (int c = lo[l]; c < lo[l + 1]; ++c)
                    if (seen[c] != 1) { ++bad; break; }
            }
        }
        // the kernels' sweeps in float against Algorithm 1 in double
        std::vector<int> pp(G.ncomp);
        for (int j = 0; j < G.ncomp; ++j) {
            const int pd = lay.pdist[(size_t)(c0 + j)];
            pp[j] = pd == 0 ? -1 : j - std::abs(pd);
        }
        // coupling g, passive diagonal d0 = d + sum of couplings, active part a
        std::vector<double> d(G.ncomp), a(G.ncomp), r(G.ncomp), g(G.ncomp), x(G.ncomp);
        for (int j = 0; j < G.ncomp; ++j) {
            g[j] = pp[j] >= 0 ? 0.05 + U(rng) : 0.0;
            d[j] = 1.0 + 0.1 * U(rng);
            a[j] = 0.3 * U(rng);
            r[j] = U(rng) - 0.5;
        }
        std::vector<double> d0(d);
        for (int j = 0; j < G.ncomp; ++j) if (pp[j] >= 0) { d0[j] += g[j]; d0[pp[j]] += g[j]; }
        {
            std::vector<double> b(d0), rr(r);
            for (int j = 0; j < G.ncomp; ++j) b[j] += a[j];
            for (int j = G.ncomp - 1; j >= 1; --j) {
                if (pp[j] < 0) continue;
                const double fct = g[j] / b[j];
                b[pp[j]] -= fct * g[j];
                rr[pp[j]] += fct * rr[j];
            }
            for (int j = 0; j < G.ncomp; ++j) x[j] = (rr[j] + (pp[j] >= 0 ? g[j] * x[pp[j]] : 0.0)) / b[j];
        }
        std::vector<double> dp(d0);  // the passive part eliminated in double
        for (int j = G.ncomp - 1; j >= 1; --j)
            if (pp[j] >= 0) dp[pp[j]] -= g[j] * g[j] / dp[j];
        // the low word of d0' enters the active part: eps_j = dl_j minus the
        // children's dl at the passive coupling factor
        std::vector<double> eps(G.ncomp);
        for (int j = 0; j < G.ncomp; ++j) eps[j] = dp[j] - (double)(float)dp[j];
        for (int j = G.ncomp - 1; j >= 1; --j)
            if (pp[j] >= 0) eps[pp[j]] -= (g[j] / dp[j]) * (g[j] / dp[j]) * (dp[j] - (double)(float)dp[j]);
        Co k;
        k.gh.resize(G.ncomp); k.gl.resize(G.ncomp); k.dh.resize(G.ncomp); k.f0.resize(G.ncomp); k.fg.resize(G.ncomp);
        for (int j = 0; j < G.ncomp; ++j) {
            k.gh[j] = (float)g[j];
            k.gl[j] = (float)(g[j] - (double)k.gh[j]);
            k.dh[j] = (float)dp[j];
            k.f0[j] = k.gh[j] * rcp_nr(k.dh[j]);
            k.fg[j] = k.f0[j] * k.gh[j];
        }
        std::vector<float> se(G.ncomp), sr(G.ncomp), scd(G.npath), scr(G.npath);
        for (int j = 0; j < G.ncomp; ++j) {
            se[j] = (float)a[j] + (float)eps[j];
            sr[j] = (float)r[j];
        }
        for (int kk = 0; kk < G.nbundle; ++kk) {
            const int nl = T.nrn[4 * kk + 2], l0 = T.nrn[4 * kk + 3];
            const int *lo = T.loffs.data() + l0, *mc = T.mcnt.data() + l0;
            for (int l = nl - 1; l >= 0; --l) {
                for (int p = lo[l]; p < lo[l + 1]; ++p) {
                    const int h = H(p);
                    int j = E(p) - 1;
                    float eb = se[j], rb = sr[j];
                    if (warp_min > 0 && E(p) - h >= warp_min) {
                        warp_eliminate(h, E(p), se, sr, k, &eb, &rb);
                        ++nwarp_paths;
                    } else {
                        for (; j > h; --j) {
                            float fj, cj;
                            elim_step(k, j, eb, rb, se[j - 1], sr[j - 1], &fj, &cj);
                            se[j] = fj;
                            sr[j] = cj;
                        }
                    }
                    const float inv = rcp_nr(k.dh[h] + eb);
                    if (Pa(p) < 0) { sr[h] = rb * inv; continue; }
                    const float fh = std::fma(k.gh[h], inv, k.gl[h] * inv);
                    se[h] = fh;
                    sr[h] = rb * inv;
                    const float ce = k.f0[h] * fh * eb, cr = fh * rb;
                    if (T.alone[p]) { se[Pa(p)] += ce; sr[Pa(p)] += cr; } else { scd[p] = ce; scr[p] = cr; }
                }
                const int zend = lo[l] + mc[l];
                for (int z = lo[l]; z < zend; ++z) {
                    const int att = T.fold[2 * z + 1];
                    if (z > lo[l] && T.fold[2 * z - 1] == att) continue;
                    float ad = 0.f, ar = 0.f;
                    for (int y = z; y < zend && T.fold[2 * y + 1] == att; ++y) { ad += scd[T.fold[2 * y]]; ar += scr[T.fold[2 * y]]; }
                    se[att] += ad;
                    sr[att] += ar;
                }
            }
            for (int l = 0; l < nl; ++l)
                for (int p = lo[l]; p < lo[l + 1]; ++p) {
                    const int h = H(p);
                    float xx = Pa(p) >= 0 ? std::fma(se[h], sr[Pa(p)], sr[h]) : sr[h];
                    sr[h] = xx;
                    if (warp_min > 0 && E(p) - h >= warp_min)
                        warp_substitute(h, E(p), xx, se, sr);
                    else
                        for (int j = h + 1; j < E(p); ++j) { xx = std::fma(se[j], xx, sr[j]); sr[j] = xx; }
                }
        }
        for (int j = 0; j < G.ncomp; ++j) maxrel = std::max(maxrel, std::fabs(sr[j] - x[j]) / (std::fabs(x[j]) + 1e-3));
    }
    if (gcomps != lay.giant_comps || gpaths != lay.giant_paths || covered != C) ++bad;
    std::printf("items=%d small=%d large=%d giant=%d warp_paths=%lld bad=%lld maxrel=%.3e\n", nitems, lay.n_small,
                lay.n_big, nitems - lay.n_small - lay.n_big, nwarp_paths, bad, maxrel);
    return bad ? 1 : 0;
}

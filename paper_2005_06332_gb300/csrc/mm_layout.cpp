// mm_layout.cpp -- validation and device layout of a network (host side).
//
// The paper stores each neuron as parent-indexed arrays and solves it with
// Algorithm 1, neuron after neuron, one OpenMP task per neuron; it balances
// multi-morphology runs by sorting neurons by size before the simulation
// (Sec. 4).  Here the same pre-processing feeds a GPU layout instead:
//   1. neurons are ordered by cost (compartment count or a supplied
//      prediction), largest first, so that the work queue hands the longest
//      items out first;
//   2. each tree is renumbered in depth-first preorder, which keeps
//      parent < child (the numbering Algorithm 1 needs); the deepest child
//      is visited first, so that each path (a compartment that does not
//      continue its parent's path, then its deepest child, and so on down to
//      a leaf) is a contiguous range whose compartments each have the
//      previous one as their parent, and every unbranched segment is
//      contiguous too;
//   3. consecutive neurons are packed into work items of about
//      `group_comps` compartments; FP32c items get path tables (paths by
//      level, per-level fold lists of paths sharing a parent compartment),
//      the schedule of the path-by-path leaves-to-root / root-to-leaves
//      sweeps; FP64 items get their segments sorted into height waves;
//   4. synapse targets are merged into synaptic sites (one conductance per
//      compartment that receives synapses) and outgoing synapses are stored
//      per source neuron, sorted by delay, for delivery.
#include "mm_layout.h"

#include <algorithm>
#include <climits>
#include <cstring>
#include <cmath>
#include <map>
#include <numeric>
#include <sstream>

namespace mmh {

namespace {

std::string msg(const std::ostringstream &o) { return o.str(); }

struct NeuronScratch {
    std::vector<int32_t> ccount, cstart, clist, newl, oldof, pnew, nch, stack, depth;
    std::vector<int32_t> seg_top, seg_len, seg_par, seg_height, seg_of_bottom, seg_of_top;
};

// One path of a work item before packing.
struct PathTmp {
    int32_t head, end, parent, neuron, level;
};

// The tables of an FP32c work item solved path by path (see mmk::NrnQ):
// per neuron its paths by (level, longest first, head); per level a fold
// list of the same paths, those sharing a parent compartment first (sorted
// by that compartment, deepest first, then head), then the paths alone on
// their parent compartment.  Emitted with 16-bit (shared-memory items) or
// 32-bit (giant items) records.
struct PathBlob {
    std::vector<int32_t> nrn;    // 4 per bundle: path0, npath, nlevel, loff0
    std::vector<int32_t> path;   // 4 per path: head, end, parent, neuron | alone
    std::vector<int32_t> fold;   // 2 per entry: path, parent compartment
    std::vector<int32_t> loffs, mcnt;
    int32_t nlevel = 0, npath = 0, nbundle = 0;
};

// Neurons of an item are swept in bundles: consecutive neurons are merged
// until a bundle holds at least this many compartments, so that a warp team
// sweeps the paths of many small neurons level by level together instead of
// one small neuron after the other (the paths of different neurons never
// interact).  A neuron at least this large is a bundle of its own.
constexpr int32_t kBundleComps = 256;

// paths: every path of the item (group-local compartments), neurons in
// order, each neuron's paths contiguous; nsize: compartments per neuron.
void build_path_blob(std::vector<PathTmp> &paths, int32_t nneuron, const std::vector<int32_t> &nsize, PathBlob &b)
{
    std::vector<int32_t> bundle((size_t)nneuron, 0);
    {
        int32_t cur = 0, acc = 0;
        for (int32_t k = 0; k < nneuron; ++k) {
            if (acc >= kBundleComps) {
                ++cur;
                acc = 0;
            }
            bundle[(size_t)k] = cur;
            acc += nsize[(size_t)k];
        }
        b.nbundle = cur + 1;
    }
    std::stable_sort(paths.begin(), paths.end(), [&](const PathTmp &a, const PathTmp &c) {
        if (bundle[(size_t)a.neuron] != bundle[(size_t)c.neuron]) return bundle[(size_t)a.neuron] < bundle[(size_t)c.neuron];
        if (a.level != c.level) return a.level < c.level;
        if (a.end - a.head != c.end - c.head) return a.end - a.head > c.end - c.head;
        return a.head < c.head;
    });
    const int32_t np = (int32_t)paths.size();
    b.npath = np;
    std::map<int32_t, int32_t> share;  // parent compartment -> paths hanging off it
    for (int32_t q = 0; q < np; ++q)
        if (paths[(size_t)q].parent >= 0) share[paths[(size_t)q].parent]++;
    auto shared = [&](int32_t x) { return paths[(size_t)x].parent >= 0 && share[paths[(size_t)x].parent] > 1; };
    b.nrn.assign(4 * (size_t)b.nbundle, 0);
    b.path.resize(4 * (size_t)np);
    b.fold.resize(2 * (size_t)np);
    b.loffs.clear();
    b.mcnt.clear();
    b.nlevel = 0;
    for (int32_t q = 0; q < np; ++q) {
        const PathTmp &P = paths[(size_t)q];
        const bool alone = P.parent >= 0 && share[P.parent] == 1;
        b.path[4 * (size_t)q] = P.head;
        b.path[4 * (size_t)q + 1] = P.end;
        b.path[4 * (size_t)q + 2] = P.parent;
        b.path[4 * (size_t)q + 3] = P.neuron | (alone ? (1 << 30) : 0);
    }
    int32_t i = 0;
    std::vector<int32_t> lv;
    for (int32_t k = 0; k < b.nbundle; ++k) {
        const int32_t p0 = i;
        while (i < np && bundle[(size_t)paths[(size_t)i].neuron] == k) ++i;
        const int32_t nl = i > p0 ? paths[(size_t)i - 1].level + 1 : 0;
        const size_t lbase = b.loffs.size();
        b.nrn[4 * (size_t)k] = p0;
        b.nrn[4 * (size_t)k + 1] = i - p0;
        b.nrn[4 * (size_t)k + 2] = nl;
        b.nrn[4 * (size_t)k + 3] = (int32_t)lbase;
        for (int32_t l = 0, q = p0; l <= nl; ++l) {
            while (q < i && paths[(size_t)q].level < l) ++q;
            b.loffs.push_back(q);
            b.mcnt.push_back(0);
        }
        for (int32_t l = 0; l < nl; ++l) {
            const int32_t s = b.loffs[lbase + (size_t)l], e = b.loffs[lbase + (size_t)l + 1];
            lv.resize((size_t)(e - s));
            std::iota(lv.begin(), lv.end(), s);
            std::sort(lv.begin(), lv.end(), [&](int32_t x, int32_t y) {
                if (shared(x) != shared(y)) return shared(x);
                if (paths[(size_t)x].parent != paths[(size_t)y].parent) return paths[(size_t)x].parent > paths[(size_t)y].parent;
                return paths[(size_t)x].head < paths[(size_t)y].head;
            });
            int32_t m = 0;
            for (int32_t z = s; z < e; ++z) {
                const int32_t c = lv[(size_t)(z - s)];
                m += shared(c) ? 1 : 0;
                b.fold[2 * (size_t)z] = c;
                b.fold[2 * (size_t)z + 1] = paths[(size_t)c].parent;
            }
            b.mcnt[lbase + (size_t)l] = m;
        }
        b.nlevel = std::max(b.nlevel, nl);
    }
}

// Byte offsets of the tables in the blob and its size, for 16-bit (wide =
// false) or 32-bit records.
struct BlobOffsets {
    int64_t path_off, fold_off, loffs_off, mcnt_off, bytes;
};

BlobOffsets blob_offsets(const PathBlob &b, bool wide)
{
    BlobOffsets o;
    const int64_t w = wide ? 4 : 2;  // bytes per index
    o.path_off = (4 * w * b.nbundle + 15) & ~15LL;
    o.fold_off = o.path_off + 4 * w * b.npath;
    o.loffs_off = o.fold_off + 2 * w * b.npath;
    o.mcnt_off = o.loffs_off + w * (int64_t)b.loffs.size();
    o.bytes = (o.mcnt_off + w * (int64_t)b.mcnt.size() + 15) & ~15LL;
    return o;
}

// The blob itself (offsets as blob_offsets; 16-bit records pack the alone
// flag as mmk::kPathAlone and the fold entries as mmk::KidQ).
std::vector<unsigned char> emit_path_blob(const PathBlob &b, bool wide)
{
    const BlobOffsets o = blob_offsets(b, wide);
    std::vector<unsigned char> blob((size_t)o.bytes, 0);
    auto put32 = [&](int64_t off, const std::vector<int32_t> &v) { std::memcpy(blob.data() + off, v.data(), 4 * v.size()); };
    auto put16 = [&](int64_t off, const std::vector<int32_t> &v) {
        for (size_t i = 0; i < v.size(); ++i) {
            const int16_t x = (int16_t)v[i];
            std::memcpy(blob.data() + off + 2 * (int64_t)i, &x, 2);
        }
    };
    if (wide) {
        std::vector<int32_t> pathg(b.path);
        for (size_t q = 0; q < (size_t)b.npath; ++q)
            pathg[4 * q + 3] = (b.path[4 * q + 3] & ((1 << 30) - 1)) | ((b.path[4 * q + 3] >> 30) ? mmk::kPathAloneG : 0);
        put32(0, b.nrn);
        put32(o.path_off, pathg);
        put32(o.fold_off, b.fold);
        put32(o.loffs_off, b.loffs);
        put32(o.mcnt_off, b.mcnt);
    } else {
        std::vector<int32_t> path16(b.path), fold16((size_t)b.npath);
        for (size_t q = 0; q < (size_t)b.npath; ++q) {
            path16[4 * q + 3] = (b.path[4 * q + 3] & ((1 << 30) - 1)) | ((b.path[4 * q + 3] >> 30) ? mmk::kPathAlone : 0);
            fold16[q] = (int32_t)((uint32_t)b.fold[2 * q] | ((uint32_t)(uint16_t)b.fold[2 * q + 1] << 16));
        }
        put16(0, b.nrn);
        put16(o.path_off, path16);
        put32(o.fold_off, fold16);
        put16(o.loffs_off, b.loffs);
        put16(o.mcnt_off, b.mcnt);
    }
    return blob;
}

}  // namespace

void neuron_features(int32_t n, const int32_t *parent, const double *L_um, const double *d_um, float *out)
{
    // children and depth in the given numbering (parent < child)
    std::vector<int32_t> nch((size_t)n, 0), depth((size_t)n, 0);
    for (int32_t i = 1; i < n; ++i) {
        nch[(size_t)parent[i]]++;
        depth[(size_t)i] = depth[(size_t)parent[i]] + 1;
    }
    int64_t leaves = 0, branch = 0, depth_sum = 0;
    int32_t depth_max = 0;
    double area = 0.0, dsum = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        if (nch[(size_t)i] == 0) ++leaves;
        if (nch[(size_t)i] >= 2) ++branch;
        depth_sum += depth[(size_t)i];
        depth_max = std::max(depth_max, depth[(size_t)i]);
        area += 3.14159265358979323846 * d_um[i] * L_um[i];
        dsum += d_um[i];
    }
    // segments of the depth-first preorder renumbering, their heights and the
    // critical path of the wave-ordered sweep (as in build_layout)
    std::vector<int32_t> cstart((size_t)n + 1, 0), clist((size_t)std::max(n - 1, 1)), fill((size_t)n, 0);
    for (int32_t i = 0; i < n; ++i) cstart[(size_t)i + 1] = cstart[(size_t)i] + nch[(size_t)i];
    for (int32_t i = 1; i < n; ++i) clist[(size_t)(cstart[(size_t)parent[i]] + fill[(size_t)parent[i]]++)] = i;
    std::vector<int32_t> newl((size_t)n), oldof((size_t)n), st;
    st.push_back(0);
    int32_t next = 0;
    while (!st.empty()) {
        const int32_t x = st.back();
        st.pop_back();
        newl[(size_t)x] = next;
        oldof[(size_t)next++] = x;
        for (int32_t c = cstart[(size_t)x + 1] - 1; c >= cstart[(size_t)x]; --c) st.push_back(clist[(size_t)c]);
    }
    std::vector<int32_t> seg_top, seg_len, seg_par, seg_h;
    std::vector<int32_t> seg_of_bottom((size_t)n, -1);
    for (int32_t j = 0; j < n; ++j) {
        const int32_t x = oldof[(size_t)j];
        const int32_t pj = j == 0 ? -1 : newl[(size_t)parent[x]];
        const bool cont = j > 0 && pj == j - 1 && nch[(size_t)oldof[(size_t)(j - 1)]] == 1;
        if (!cont) {
            seg_top.push_back(j);
            seg_len.push_back(1);
            seg_par.push_back(pj);
            seg_h.push_back(0);
        } else {
            seg_len.back()++;
        }
    }
    const int32_t ns = (int32_t)seg_top.size();
    for (int32_t s = 0; s < ns; ++s) seg_of_bottom[(size_t)(seg_top[(size_t)s] + seg_len[(size_t)s] - 1)] = s;
    for (int32_t s = ns - 1; s >= 1; --s) {
        const int32_t ps = seg_of_bottom[(size_t)seg_par[(size_t)s]];
        if (ps >= 0) seg_h[(size_t)ps] = std::max(seg_h[(size_t)ps], seg_h[(size_t)s] + 1);
    }
    int32_t H = 0, maxlen = 0;
    for (int32_t s = 0; s < ns; ++s) {
        H = std::max(H, seg_h[(size_t)s]);
        maxlen = std::max(maxlen, seg_len[(size_t)s]);
    }
    std::vector<int32_t> wmax((size_t)H + 1, 0), wcount((size_t)H + 1, 0);
    for (int32_t s = 0; s < ns; ++s) {
        wmax[(size_t)seg_h[(size_t)s]] = std::max(wmax[(size_t)seg_h[(size_t)s]], seg_len[(size_t)s]);
        wcount[(size_t)seg_h[(size_t)s]]++;
    }
    int64_t crit = 0;
    int32_t wwide = 0;
    for (int32_t w = 0; w <= H; ++w) {
        crit += wmax[(size_t)w];
        wwide = std::max(wwide, wcount[(size_t)w]);
    }
    out[0] = (float)std::log((double)n);
    out[1] = (float)std::log1p((double)depth_max);
    out[2] = (float)std::log1p((double)branch);
    out[3] = (float)std::log1p((double)leaves);
    out[4] = (float)std::log1p((double)ns);
    out[5] = (float)std::log1p((double)(H + 1));
    out[6] = (float)std::log1p((double)crit);
    out[7] = (float)std::log1p((double)maxlen);
    out[8] = (float)((double)n / (double)ns / 100.0);
    out[9] = (float)std::log1p((double)depth_sum / (double)n);
    out[10] = (float)std::log(area);
    out[11] = (float)(dsum / (double)n);
    out[12] = (float)((double)branch / (double)n);
    out[13] = (float)std::log1p((double)wwide);
    out[14] = (float)((double)crit / (double)n);
    out[15] = (float)std::log1p((double)nch[0]);
}

std::string build_layout(const LayoutInput &in, Layout &out, bool *invalid)
{
    *invalid = true;
    std::ostringstream e;
    const int32_t N = in.N;
    if (N < 1) { e << "n_neurons must be >= 1"; return msg(e); }
    if (!in.comp_offset || !in.parent || !in.length_um || !in.diam_um) { e << "morphology arrays must not be NULL"; return msg(e); }
    if (!(in.dt > 0.0) || !std::isfinite(in.dt)) { e << "dt must be > 0"; return msg(e); }
    if (in.comp_offset[0] != 0) { e << "comp_offset[0] must be 0"; return msg(e); }
    for (int32_t k = 0; k < N; ++k) {
        int64_t n = in.comp_offset[k + 1] - in.comp_offset[k];
        if (n < 1) { e << "neuron " << k << " has no compartments"; return msg(e); }
        if (n > (int64_t)INT32_MAX / 2) { e << "neuron " << k << " is too large"; return msg(e); }
    }
    const int64_t C = in.comp_offset[N];
    for (int32_t k = 0; k < N; ++k) {
        const int64_t b = in.comp_offset[k], n = in.comp_offset[k + 1] - b;
        if (in.parent[b] != -1) { e << "neuron " << k << ": parent[0] must be -1"; return msg(e); }
        for (int64_t i = 1; i < n; ++i) {
            const int32_t p = in.parent[b + i];
            if (p < 0 || p >= i) { e << "neuron " << k << ": parent[" << i << "] = " << p << " is not in [0, " << i << ")"; return msg(e); }
        }
    }
    for (int64_t i = 0; i < C; ++i) {
        if (!(in.length_um[i] > 0.0) || !(in.diam_um[i] > 0.0) || !std::isfinite(in.length_um[i]) ||
            !std::isfinite(in.diam_um[i])) { e << "compartment " << i << ": length and diameter must be positive and finite"; return msg(e); }
    }
    if (in.S < 0) { e << "negative synapse count"; return msg(e); }
    if (in.n_ext < 0 || (in.n_ext > 0 && in.points)) { e << "external sources need soma detection"; return msg(e); }
    if (in.S > 0 && (!in.src || !in.dst || !in.dcomp || !in.w || !in.delay_ms)) { e << "synapse arrays must not be NULL"; return msg(e); }
    int64_t max_ds = 0;
    std::vector<int32_t> dsteps((size_t)in.S);
    for (int64_t s = 0; s < in.S; ++s) {
        const int32_t a = in.src[s], b = in.dst[s];
        if (a < 0 || a >= N + in.n_ext || b < 0 || b >= N) { e << "synapse " << s << ": neuron id out of range"; return msg(e); }
        const int64_t nb = in.comp_offset[b + 1] - in.comp_offset[b];
        if (in.dcomp[s] < 0 || in.dcomp[s] >= nb) { e << "synapse " << s << ": dst_comp out of range"; return msg(e); }
        if (in.points && in.scomp &&
            (in.scomp[s] < 0 || in.scomp[s] >= in.comp_offset[a + 1] - in.comp_offset[a])) {
            e << "synapse " << s << ": src_comp out of range";
            return msg(e);
        }
        if (!(in.w[s] >= 0.0) || !std::isfinite(in.w[s])) { e << "synapse " << s << ": weight must be finite and >= 0"; return msg(e); }
        const double q = in.delay_ms[s] / in.dt;
        if (!std::isfinite(q)) { e << "synapse " << s << ": delay must be finite"; return msg(e); }
        const long long d = std::llround(q);
        if (d < 1) { e << "synapse " << s << ": delay is shorter than dt"; return msg(e); }
        if (d > 1000000) { *invalid = false; e << "synapse " << s << ": delay of more than 1e6 steps"; return msg(e); }
        dsteps[(size_t)s] = (int32_t)d;
        max_ds = std::max<int64_t>(max_ds, d);
    }
    if (in.stim) {
        for (int32_t k = 0; k < N; ++k)
            if (!std::isfinite(in.stim[k])) { e << "stim of neuron " << k << " is not finite"; return msg(e); }
    }
    if (in.cost) {
        for (int32_t k = 0; k < N; ++k)
            if (!std::isfinite(in.cost[k])) { e << "cost of neuron " << k << " is not finite"; return msg(e); }
    }
    *invalid = false;
    for (int32_t k = 0; k < N; ++k) {
        const int64_t n = in.comp_offset[k + 1] - in.comp_offset[k];
        if (n > in.max_group_comps) {
            e << "neuron " << k << " has " << n << " compartments; this build holds at most " << in.max_group_comps
              << " per neuron";
            return msg(e);
        }
    }

    Layout &L = out;
    L.N = N;
    L.C = C;

    // 1. order: largest cost first, ties by user id
    L.order.resize((size_t)N);
    std::iota(L.order.begin(), L.order.end(), 0);
    auto size_of = [&](int32_t u) { return in.comp_offset[u + 1] - in.comp_offset[u]; };
    if (in.cost) {
        std::stable_sort(L.order.begin(), L.order.end(), [&](int32_t a, int32_t b) { return in.cost[a] > in.cost[b]; });
    } else {
        std::stable_sort(L.order.begin(), L.order.end(), [&](int32_t a, int32_t b) { return size_of(a) > size_of(b); });
    }
    L.internal_of.assign((size_t)N, 0);
    for (int32_t k = 0; k < N; ++k) L.internal_of[(size_t)L.order[(size_t)k]] = k;
    L.noff.assign((size_t)N + 1, 0);
    for (int32_t k = 0; k < N; ++k) L.noff[(size_t)k + 1] = L.noff[(size_t)k] + size_of(L.order[(size_t)k]);

    L.L.resize((size_t)C);
    L.D.resize((size_t)C);
    L.pdist.resize((size_t)C);
    L.user2int.resize((size_t)C);
    L.soma_of_user.resize((size_t)N);
    L.stim.assign((size_t)N, 0.0);
    for (int32_t k = 0; k < N; ++k) {
        const int32_t u = L.order[(size_t)k];
        L.soma_of_user[(size_t)u] = L.noff[(size_t)k];
        if (in.stim) L.stim[(size_t)k] = in.stim[u];
    }

    // 3a. group boundaries (at most kPathNeuron + 1 neurons per item, the
    // range of a path's neuron index)
    std::vector<int32_t> gstart;
    {
        int64_t cur = 0;
        int32_t cnt = 0;
        for (int32_t k = 0; k < N; ++k) {
            const int64_t n = L.noff[(size_t)k + 1] - L.noff[(size_t)k];
            if (k == 0 || cur + n > in.group_comps || cnt > mmk::kPathNeuron) {
                gstart.push_back(k);
                cur = 0;
                cnt = 0;
            }
            cur += n;
            ++cnt;
        }
        gstart.push_back(N);
    }
    const int32_t G = (int32_t)gstart.size() - 1;
    L.groups.clear();
    L.groups.reserve((size_t)G);
    std::vector<mmk::GroupRec> bigs, giants;

    // 2 + 3b. per group: renumber its neurons, cut segments, sort into waves
    NeuronScratch ws;
    std::vector<mmk::SegRec> gsegs;
    std::vector<std::vector<int32_t>> gkids;
    std::vector<int32_t> gheight, gpseg, glevel, perm, newidx;
    std::vector<PathTmp> gpaths;
    std::vector<int32_t> gsize;  // compartments of each neuron of the item
    L.max_comps = 0;
    L.max_segs = 0;
    L.max_waves = 0;
    for (int32_t g = 0; g < G; ++g) {
        const int32_t k0 = gstart[(size_t)g], k1 = gstart[(size_t)g + 1];
        const int64_t comp0 = L.noff[(size_t)k0];
        gsegs.clear();
        gkids.clear();
        gheight.clear();
        gpseg.clear();
        glevel.clear();
        gpaths.clear();
        gsize.clear();
        for (int32_t k = k0; k < k1; ++k) {
            const int32_t u = L.order[(size_t)k];
            const int64_t ub = in.comp_offset[u];
            const int32_t n = (int32_t)size_of(u);
            gsize.push_back(n);
            const int64_t ib = L.noff[(size_t)k];
            const int32_t lb = (int32_t)(ib - comp0);
            const int32_t *par = in.parent + ub;
            // children lists (ascending old index)
            ws.ccount.assign((size_t)n, 0);
            for (int32_t i = 1; i < n; ++i) ws.ccount[(size_t)par[i]]++;
            ws.cstart.assign((size_t)n + 1, 0);
            for (int32_t i = 0; i < n; ++i) ws.cstart[(size_t)i + 1] = ws.cstart[(size_t)i] + ws.ccount[(size_t)i];
            ws.clist.resize((size_t)std::max(n - 1, 1));
            {
                std::vector<int32_t> &fill = ws.nch;
                fill.assign((size_t)n, 0);
                for (int32_t i = 1; i < n; ++i) {
                    const int32_t p = par[i];
                    ws.clist[(size_t)(ws.cstart[(size_t)p] + fill[(size_t)p]++)] = i;
                }
            }
            // depth-first preorder; the deepest child (longest path to a leaf,
            // in compartments) is visited first, ties by smallest index
            ws.depth.assign((size_t)n, 1);
            for (int32_t i = n - 1; i >= 1; --i)
                ws.depth[(size_t)par[i]] = std::max(ws.depth[(size_t)par[i]], ws.depth[(size_t)i] + 1);
            for (int32_t x = 0; x < n; ++x) {
                std::sort(ws.clist.begin() + ws.cstart[(size_t)x], ws.clist.begin() + ws.cstart[(size_t)x + 1],
                          [&](int32_t a, int32_t b) {
                              if (ws.depth[(size_t)a] != ws.depth[(size_t)b]) return ws.depth[(size_t)a] > ws.depth[(size_t)b];
                              return a < b;
                          });
            }
            ws.newl.resize((size_t)n);
            ws.oldof.resize((size_t)n);
            ws.stack.clear();
            ws.stack.push_back(0);
            int32_t next = 0;
            while (!ws.stack.empty()) {
                const int32_t x = ws.stack.back();
                ws.stack.pop_back();
                ws.newl[(size_t)x] = next;
                ws.oldof[(size_t)next] = x;
                ++next;
                for (int32_t c = ws.cstart[(size_t)x + 1] - 1; c >= ws.cstart[(size_t)x]; --c)
                    ws.stack.push_back(ws.clist[(size_t)c]);
            }
            ws.pnew.resize((size_t)n);
            ws.nch.assign((size_t)n, 0);
            for (int32_t j = 0; j < n; ++j) {
                const int32_t x = ws.oldof[(size_t)j];
                const int32_t pj = (j == 0) ? -1 : ws.newl[(size_t)par[x]];
                ws.pnew[(size_t)j] = pj;
                if (pj >= 0) ws.nch[(size_t)pj]++;
                L.L[(size_t)(ib + j)] = in.length_um[ub + x];
                L.D[(size_t)(ib + j)] = in.diam_um[ub + x];
                L.pdist[(size_t)(ib + j)] = (j == 0) ? 0 : (j - pj);
                L.user2int[(size_t)(ub + x)] = ib + j;
            }
            // segments: j starts one unless it is the only child of j-1
            const size_t s_first = gsegs.size();
            ws.seg_of_bottom.assign((size_t)n, -1);
            for (int32_t j = 0; j < n; ++j) {
                const bool cont = (j > 0 && ws.pnew[(size_t)j] == j - 1 && ws.nch[(size_t)(j - 1)] == 1);
                if (!cont) {
                    // segment tops carry a negative parent distance (FP32c items
                    // re-mark path heads instead, below)
                    if (j > 0) L.pdist[(size_t)(ib + j)] = -L.pdist[(size_t)(ib + j)];
                    mmk::SegRec s;
                    s.top = lb + j;
                    s.len = 1;
                    s.parent = (j == 0) ? -1 : lb + ws.pnew[(size_t)j];
                    s.child0 = 0;
                    s.nchild = 0;
                    s.neuron = (j == 0) ? (k - k0) : -1;
                    gsegs.push_back(s);
                    gkids.emplace_back();
                    gheight.push_back(0);
                } else {
                    gsegs.back().len++;
                }
            }
            ws.seg_of_top.assign((size_t)n, -1);
            for (size_t s = s_first; s < gsegs.size(); ++s) {
                const int32_t bottom = gsegs[s].top + gsegs[s].len - 1 - lb;
                ws.seg_of_bottom[(size_t)bottom] = (int32_t)s;
                ws.seg_of_top[(size_t)(gsegs[s].top - lb)] = (int32_t)s;
                gpseg.push_back(-1);
                glevel.push_back(0);
            }
            // children and heights (child segments have larger tops than their parents)
            for (size_t s = gsegs.size(); s-- > s_first + 1;) {
                const int32_t pb = gsegs[s].parent - lb;
                const int32_t ps = ws.seg_of_bottom[(size_t)pb];
                if (ps < 0) { e << "internal: segment parent is not a segment bottom"; return msg(e); }
                gkids[(size_t)ps].insert(gkids[(size_t)ps].begin(), (int32_t)s);
                gheight[(size_t)ps] = std::max(gheight[(size_t)ps], gheight[s] + 1);
                gpseg[s] = ps;
            }
            // paths: a segment heads one unless it is its parent's first
            // (deepest) child, whose top directly follows the parent's bottom;
            // a path runs down the first children to a leaf
            for (size_t s = s_first; s < gsegs.size(); ++s) {
                const bool head = gsegs[s].parent < 0 || gsegs[s].top != gsegs[s].parent + 1;
                if (!head) {
                    glevel[s] = glevel[(size_t)gpseg[s]];
                    continue;
                }
                glevel[s] = gsegs[s].parent < 0 ? 0 : glevel[(size_t)gpseg[s]] + 1;
                size_t c = s;
                for (;;) {
                    const int32_t nb = gsegs[c].top + gsegs[c].len - lb;  // one past the bottom
                    const int32_t nx = nb < n ? ws.seg_of_top[(size_t)nb] : -1;
                    if (nx < 0 || gsegs[(size_t)nx].parent != gsegs[c].top + gsegs[c].len - 1) break;
                    c = (size_t)nx;
                }
                gpaths.push_back(PathTmp{gsegs[s].top, gsegs[c].top + gsegs[c].len, gsegs[s].parent, k - k0,
                                         glevel[s]});
            }
        }
        // sort by (height, longest first, top)
        const int32_t ns = (int32_t)gsegs.size();
        perm.resize((size_t)ns);
        std::iota(perm.begin(), perm.end(), 0);
        std::sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
            if (gheight[(size_t)a] != gheight[(size_t)b]) return gheight[(size_t)a] < gheight[(size_t)b];
            if (gsegs[(size_t)a].len != gsegs[(size_t)b].len) return gsegs[(size_t)a].len > gsegs[(size_t)b].len;
            return gsegs[(size_t)a].top < gsegs[(size_t)b].top;
        });
        newidx.resize((size_t)ns);
        for (int32_t i = 0; i < ns; ++i) newidx[(size_t)perm[(size_t)i]] = i;
        mmk::GroupRec gr{};
        gr.comp0 = comp0;
        gr.scratch0 = 0;
        gr.ncomp = (int32_t)(L.noff[(size_t)k1] - comp0);
        gr.nseg = ns;
        gr.neuron0 = k0;
        gr.nneuron = k1 - k0;
        int32_t maxh = 0;
        int64_t nkids = 0;
        for (int32_t i = 0; i < ns; ++i) {
            maxh = std::max(maxh, gheight[(size_t)perm[(size_t)i]]);
            nkids += (int64_t)gkids[(size_t)perm[(size_t)i]].size();
        }
        // shared-memory need: FP64 items hold the segment blob, FP32c items
        // the path tables (16-bit records) plus per-path slots
        PathBlob pb;
        int64_t smem_need;
        if (in.path_items) {
            build_path_blob(gpaths, gr.nneuron, gsize, pb);
            if (gr.ncomp <= 32767 && pb.npath <= 32767) {
                smem_need = blob_offsets(pb, false).bytes + (int64_t)in.smem_per_comp * gr.ncomp +
                            (int64_t)in.smem_per_path * pb.npath;
            } else {
                smem_need = INT64_MAX;
            }
        } else {
            const int64_t small_meta = ((int64_t)ns * (int64_t)sizeof(mmk::SegP) + 2 * nkids + 2 * (maxh + 2) + 15) & ~15LL;
            smem_need = small_meta + (int64_t)in.smem_per_comp * gr.ncomp + (int64_t)in.smem_per_seg * ns;
        }
        const bool over = in.giant_smem_limit > 0 && smem_need > in.giant_smem_limit;
        const bool big = over && in.big_smem_limit > 0 && smem_need <= in.big_smem_limit;
        const bool giant = (in.path_items ? (gr.ncomp > 32767 || pb.npath > 32767) : (gr.ncomp > 32767 || ns > 32767)) ||
                           (over && !big);
        if (giant && in.giant_smem_limit <= 0) {
            *invalid = false;
            e << "a work item of " << gr.ncomp << " compartments exceeds what this precision holds";
            return msg(e);
        }
        std::vector<unsigned char> blob;
        if (in.path_items) {
            // links inside paths are assembled per compartment; path heads
            // (negative parent distance) link to their parent in the sweep
            for (int64_t c = comp0; c < comp0 + gr.ncomp; ++c) {
                const int32_t pd = std::abs(L.pdist[(size_t)c]);
                L.pdist[(size_t)c] = pd == 1 ? 1 : -pd;
            }
            // 16-bit records for items staged in shared memory, 32-bit for giants
            const BlobOffsets o = blob_offsets(pb, giant);
            blob = emit_path_blob(pb, giant);
            gr.nbundle = pb.nbundle;
            gr.path_off = (int32_t)o.path_off;
            gr.fold_off = (int32_t)o.fold_off;
            gr.loffs_off = (int32_t)o.loffs_off;
            gr.mcnt_off = (int32_t)o.mcnt_off;
            gr.npath = pb.npath;
            gr.nlevel = pb.nlevel;
            if (giant) {
                gr.scratch0 = L.giant_comps;
                L.giant_comps += gr.ncomp;
                if (L.giant_paths + pb.npath > INT32_MAX) {
                    e << "giant work items hold more than 2^31 paths";
                    return msg(e);
                }
                gr.pscratch0 = (int32_t)L.giant_paths;
                L.giant_paths += pb.npath;
            }
        } else {
            // the segment blob: records in wave order, child lists, wave offsets
            std::vector<int32_t> woff;
            {
                int32_t i = 0;
                for (int32_t h = 0; h <= maxh; ++h) {
                    while (i < ns && gheight[(size_t)perm[(size_t)i]] < h) ++i;
                    woff.push_back(i);
                }
                woff.push_back(ns);
            }
            gr.nchild = (int32_t)nkids;
            gr.nwave = maxh + 1;
            auto put = [&blob](const void *p, size_t n) {
                const unsigned char *c = (const unsigned char *)p;
                blob.insert(blob.end(), c, c + n);
            };
            std::vector<int16_t> kids;
            std::vector<mmk::SegP> recs((size_t)ns);
            for (int32_t i = 0; i < ns; ++i) {
                const int32_t sidx = perm[(size_t)i];
                const mmk::SegRec &r = gsegs[(size_t)sidx];
                mmk::SegP q;
                q.top = (int16_t)r.top;
                q.len = (int16_t)r.len;
                q.parent = (int16_t)r.parent;
                q.nchild = (int16_t)gkids[(size_t)sidx].size();
                q.child0 = (int16_t)kids.size();
                q.neuron = (int16_t)r.neuron;
                q.pseg = (int16_t)(gpseg[(size_t)sidx] < 0 ? -1 : newidx[(size_t)gpseg[(size_t)sidx]]);
                q.pad = 0;
                for (int32_t c : gkids[(size_t)sidx]) kids.push_back((int16_t)newidx[(size_t)c]);
                recs[(size_t)i] = q;
            }
            std::vector<int16_t> w16(woff.begin(), woff.end());
            put(recs.data(), recs.size() * sizeof(mmk::SegP));
            put(kids.data(), kids.size() * 2);
            put(w16.data(), w16.size() * 2);
        }
        blob.resize((blob.size() + 15) & ~(size_t)15, 0);
        gr.meta_off = (int64_t)L.meta.size();
        gr.meta_bytes = (int32_t)blob.size();
        L.meta.insert(L.meta.end(), blob.begin(), blob.end());
        if (giant) {
            giants.push_back(gr);
        } else if (big) {
            bigs.push_back(gr);
            L.big_max_comps = std::max(L.big_max_comps, gr.ncomp);
            L.big_max_segs = std::max(L.big_max_segs, in.path_items ? gr.npath : ns);
            L.big_max_meta = std::max(L.big_max_meta, gr.meta_bytes);
            L.big_max_smem = std::max<int64_t>(L.big_max_smem, smem_need);
        } else {
            L.groups.push_back(gr);
            L.max_smem = std::max<int64_t>(L.max_smem, smem_need);
            L.max_comps = std::max(L.max_comps, gr.ncomp);
            L.max_segs = std::max(L.max_segs, in.path_items ? gr.npath : ns);
            L.max_waves = std::max(L.max_waves, in.path_items ? gr.nlevel : gr.nwave);
            L.max_meta = std::max(L.max_meta, gr.meta_bytes);
        }
    }
    L.n_small = (int32_t)L.groups.size();
    L.n_big = (int32_t)bigs.size();
    L.groups.insert(L.groups.end(), bigs.begin(), bigs.end());
    L.groups.insert(L.groups.end(), giants.begin(), giants.end());

    // 4a. synaptic sites: one per compartment that receives a synapse
    std::vector<int32_t> site_of((size_t)C, -1);
    for (int64_t s = 0; s < in.S; ++s) {
        const int64_t ic = L.user2int[(size_t)(in.comp_offset[in.dst[s]] + in.dcomp[s])];
        site_of[(size_t)ic] = 0;
    }
    {
        // items in compartment order (giant items sit at the end of groups[])
        std::vector<int32_t> by_comp(L.groups.size());
        std::iota(by_comp.begin(), by_comp.end(), 0);
        std::sort(by_comp.begin(), by_comp.end(),
                  [&](int32_t x, int32_t y) { return L.groups[(size_t)x].comp0 < L.groups[(size_t)y].comp0; });
        int32_t ns = 0;
        size_t gpos = 0;
        for (auto &gr : L.groups) { gr.site0 = 0; gr.nsite = 0; }
        for (int64_t i = 0; i < C; ++i) {
            if (site_of[(size_t)i] < 0) continue;
            while (i >= L.groups[(size_t)by_comp[gpos]].comp0 + L.groups[(size_t)by_comp[gpos]].ncomp) ++gpos;
            mmk::GroupRec &gr = L.groups[(size_t)by_comp[gpos]];
            if (gr.nsite == 0) gr.site0 = ns;
            gr.nsite++;
            site_of[(size_t)i] = ns++;
            L.site_comp.push_back((int32_t)(i - gr.comp0));
            L.site_internal.push_back(i);
        }
        for (auto &gr : L.groups) if (gr.nsite == 0) gr.site0 = ns;
        L.f_syn = C > 0 ? (double)ns / (double)C : 0.0;
    }

    // 4b. delays and the outgoing synapses of each source, sorted by delay
    {
        std::vector<char> seen((size_t)max_ds + 1, 0);
        for (int64_t s = 0; s < in.S; ++s) seen[(size_t)dsteps[(size_t)s]] = 1;
        L.dclass.clear();
        for (int64_t d = 1; d <= max_ds; ++d) if (seen[(size_t)d]) L.dclass.push_back((int32_t)d);
        L.R = (int32_t)(max_ds + 2);
    }
    // 4c. spike sources: the internal neurons, or the detection points in
    //     internal compartment order
    std::vector<int32_t> src_id((size_t)in.S);
    if (!in.points) {
        // internal neurons 0 .. N-1, then the external sources N .. N + n_ext - 1
        L.n_src = N + in.n_ext;
        for (int64_t s = 0; s < in.S; ++s)
            src_id[(size_t)s] = in.src[s] < N ? L.internal_of[(size_t)in.src[s]] : in.src[s];
    } else {
        std::vector<int64_t> ic((size_t)in.S);
        for (int64_t s = 0; s < in.S; ++s)
            ic[(size_t)s] = L.user2int[(size_t)(in.comp_offset[in.src[s]] + (in.scomp ? in.scomp[s] : 0))];
        L.pt_comp = ic;
        std::sort(L.pt_comp.begin(), L.pt_comp.end());
        L.pt_comp.erase(std::unique(L.pt_comp.begin(), L.pt_comp.end()), L.pt_comp.end());
        if (L.pt_comp.size() > (size_t)INT32_MAX / 2) { *invalid = false; e << "too many detection points"; return msg(e); }
        L.n_src = (int32_t)L.pt_comp.size();
        L.pt_user_nrn.assign(L.pt_comp.size(), 0);
        L.pt_user_comp.assign(L.pt_comp.size(), 0);
        L.soma_src.assign((size_t)N, -1);
        L.pt_of.assign((size_t)C, -1);
        for (int64_t s = 0; s < in.S; ++s) {
            const int64_t c = ic[(size_t)s];
            const int32_t id = (int32_t)(std::lower_bound(L.pt_comp.begin(), L.pt_comp.end(), c) - L.pt_comp.begin());
            src_id[(size_t)s] = id;
            const int32_t uc = in.scomp ? in.scomp[s] : 0;
            L.pt_user_nrn[(size_t)id] = in.src[s];
            L.pt_user_comp[(size_t)id] = uc;
            if (uc == 0)
                L.soma_src[(size_t)L.internal_of[(size_t)in.src[s]]] = id;
            else
                L.pt_of[(size_t)c] = id;
        }
    }
    L.out_off.assign((size_t)L.n_src + 1, 0);
    for (int64_t s = 0; s < in.S; ++s) L.out_off[(size_t)src_id[(size_t)s] + 1]++;
    for (int32_t k = 0; k < L.n_src; ++k) L.out_off[(size_t)k + 1] += L.out_off[(size_t)k];
    std::vector<int64_t> order_s((size_t)in.S);
    {
        std::vector<int64_t> fill(L.out_off.begin(), L.out_off.end() - 1);
        for (int64_t s = 0; s < in.S; ++s) order_s[(size_t)fill[(size_t)src_id[(size_t)s]]++] = s;
    }
    if (L.dclass.size() > 1) {
        for (int32_t k = 0; k < L.n_src; ++k)
            std::stable_sort(order_s.begin() + L.out_off[(size_t)k], order_s.begin() + L.out_off[(size_t)k + 1],
                             [&](int64_t a, int64_t b) { return dsteps[(size_t)a] < dsteps[(size_t)b]; });
    }
    L.out_site.resize((size_t)in.S);
    L.out_dsteps.resize((size_t)in.S);
    L.out_w.resize((size_t)in.S);
    for (int64_t q = 0; q < in.S; ++q) {
        const int64_t s = order_s[(size_t)q];
        const int64_t ic = L.user2int[(size_t)(in.comp_offset[in.dst[s]] + in.dcomp[s])];
        L.out_site[(size_t)q] = site_of[(size_t)ic];
        L.out_dsteps[(size_t)q] = dsteps[(size_t)s];
        L.out_w[(size_t)q] = in.w[s];
    }
    // 4d. incoming synapses of each site, ascending synapse id
    {
        const size_t nsite = L.site_comp.size();
        std::vector<int32_t> tsite((size_t)in.S);
        L.in_off.assign(nsite + 1, 0);
        for (int64_t s = 0; s < in.S; ++s) {
            const int64_t ic = L.user2int[(size_t)(in.comp_offset[in.dst[s]] + in.dcomp[s])];
            tsite[(size_t)s] = site_of[(size_t)ic];
            L.in_off[(size_t)tsite[(size_t)s] + 1]++;
        }
        for (size_t k = 0; k < nsite; ++k) L.in_off[k + 1] += L.in_off[k];
        L.in_src.resize((size_t)in.S);
        L.in_dsteps.resize((size_t)in.S);
        L.in_w.resize((size_t)in.S);
        std::vector<int64_t> fill(L.in_off.begin(), L.in_off.end() - 1);
        for (int64_t s = 0; s < in.S; ++s) {
            const int64_t q = fill[(size_t)tsite[(size_t)s]]++;
            L.in_src[(size_t)q] = src_id[(size_t)s];
            L.in_dsteps[(size_t)q] = dsteps[(size_t)s];
            L.in_w[(size_t)q] = in.w[s];
        }
    }
    return "";
}

}  // namespace mmh

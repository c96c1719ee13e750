// Host-side dump of the spike-source tables of the layout (paper_2005_06332_gb300/
// csrc/mm_layout.cpp), built and run by tests/test_layout_sources.py, which
// recomputes every table from the synapse arrays and compares.
//
// Usage: sources_check <network file> <points 0|1> <out file>
// Network file: int32 N | int64 C | int64 S | int64 comp_offset[N+1] |
//               int32 parent[C] | int32 src[S] | int32 dst[S] | int32 dcomp[S] |
//               int32 scomp[S] | float64 w[S] | float64 delay_ms[S]
// Out file (little-endian): int32 n_src | int64 nsite |
//   int64 user2int[C] | int32 internal_of[N] | int64 site_internal[nsite] |
//   int64 out_off[n_src+1] | int32 out_site, out_dsteps[S] | float64 out_w[S] |
//   int64 in_off[nsite+1] | int32 in_src, in_dsteps[S] | float64 in_w[S] |
//   (points only) int32 pt_of[C] | int32 soma_src[N] | int32 pt_user_nrn, pt_user_comp[n_src]
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "mm_layout.h"

namespace {

template <class T>
bool rd(FILE *f, std::vector<T> &v, size_t n)
{
    v.resize(n);
    return n == 0 || std::fread(v.data(), sizeof(T), n, f) == n;
}

template <class T>
void wr(FILE *f, const std::vector<T> &v)
{
    if (!v.empty()) std::fwrite(v.data(), sizeof(T), v.size(), f);
}

}  // namespace

int main(int argc, char **argv)
{
    if (argc < 4) return 2;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t N;
    int64_t C, S;
    if (std::fread(&N, 4, 1, f) != 1 || std::fread(&C, 8, 1, f) != 1 || std::fread(&S, 8, 1, f) != 1) return 2;
    std::vector<int64_t> off;
    std::vector<int32_t> par, src, dst, dcomp, scomp;
    std::vector<double> w, delay;
    if (!rd(f, off, (size_t)N + 1) || !rd(f, par, (size_t)C) || !rd(f, src, (size_t)S) || !rd(f, dst, (size_t)S) ||
        !rd(f, dcomp, (size_t)S) || !rd(f, scomp, (size_t)S) || !rd(f, w, (size_t)S) || !rd(f, delay, (size_t)S))
        return 2;
    std::fclose(f);
    const bool points = std::atoi(argv[2]) != 0;
    std::vector<double> L((size_t)C, 10.0), D((size_t)C, 1.0);
    mmh::LayoutInput in{};
    in.N = N;
    in.comp_offset = off.data();
    in.parent = par.data();
    in.length_um = L.data();
    in.diam_um = D.data();
    in.S = S;
    in.src = src.data();
    in.dst = dst.data();
    in.dcomp = dcomp.data();
    in.w = w.data();
    in.delay_ms = delay.data();
    in.points = points;
    in.scomp = scomp.data();
    in.dt = 0.025;
    in.group_comps = 2048;
    in.max_group_comps = 1 << 30;
    in.smem_per_comp = 12;
    in.giant_smem_limit = 110 * 1024;
    in.big_smem_limit = 224 * 1024;
    in.path_items = true;
    in.smem_per_path = 12;
    mmh::Layout lay;
    bool invalid = false;
    const std::string err = mmh::build_layout(in, lay, &invalid);
    if (!err.empty()) {
        std::printf("layout error: %s\n", err.c_str());
        return 1;
    }
    FILE *o = std::fopen(argv[3], "wb");
    if (!o) return 2;
    const int64_t nsite = (int64_t)lay.site_internal.size();
    std::fwrite(&lay.n_src, 4, 1, o);
    std::fwrite(&nsite, 8, 1, o);
    wr(o, lay.user2int);
    wr(o, lay.internal_of);
    wr(o, lay.site_internal);
    wr(o, lay.out_off);
    wr(o, lay.out_site);
    wr(o, lay.out_dsteps);
    wr(o, lay.out_w);
    wr(o, lay.in_off);
    wr(o, lay.in_src);
    wr(o, lay.in_dsteps);
    wr(o, lay.in_w);
    if (points) {
        wr(o, lay.pt_of);
        wr(o, lay.soma_src);
        wr(o, lay.pt_user_nrn);
        wr(o, lay.pt_user_comp);
    }
    std::fclose(o);
    std::printf("ok n_src=%d nsite=%lld\n", lay.n_src, (long long)nsite);
    return 0;
}

// Host check of the FP32c gate table (csrc/mm_gate_table.h): builds the table
// for the given dt and, for every line "vq qm qh qn" on stdin, prints the six
// table functions at V = vq 2^-23 mV (X_m E_m X_h E_h X_n E_n, each its float
// pair summed in double) and the three stepped gates.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "mm_gate_table.h"

int main(int argc, char **argv)
{
    if (argc != 2) return 2;
    const double dt = std::atof(argv[1]);
    std::vector<mmf::Tab4> tab((size_t)mmf::kTabQuads * mmf::kTabIntervals);
    mmf::build_gate_table(dt, tab.data());
    long long vq, q[3];
    while (std::scanf("%lld %lld %lld %lld", &vq, &q[0], &q[1], &q[2]) == 4) {
        const mmf::TabIndex t = mmf::tab_index((int32_t)vq);
        mmf::Tab4 f[mmf::kTabQuads];  // the interval's quads
        for (int k = 0; k < mmf::kTabQuads; ++k) f[k] = tab[(size_t)k * mmf::kTabIntervals + t.i];
        for (int fn = 0; fn < mmf::kTabFuncs; ++fn) {
            const mmf::F2 v = mmf::tab_eval(f[2 * fn], f[2 * fn + 1], t.u);
            std::printf("%.17g ", (double)v.hi + (double)v.lo);
        }
        for (int g = 0; g < 3; ++g) std::printf("%u ", mmf::tab_gate_step((uint32_t)q[g], f + 4 * g, t.u));
        std::printf("\n");
    }
    return 0;
}

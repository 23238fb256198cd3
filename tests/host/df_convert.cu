// Host-side check of the double-float -> FP64 assembly used by the tensor-core epilogues: the branch-free
// df_to_double_nb must equal df_to_double bit for bit whenever it does not flag a special case, and both must be
// within 2^-51 relative of (double)hi + (double)lo scaled by 2^E (FP64 arithmetic as the independent reference;
// the assembly truncates the low word beyond 53 bits, so a result just below a power of two may land on it).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../../paper_2106_06149_gb300/csrc/common.cuh"

static bool close(double a, double ref) { return std::fabs(a - ref) <= std::ldexp(std::fabs(ref), -51); }

int main() {
    std::mt19937_64 g(7);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    std::uniform_int_distribution<int> ue(-60, 60), uE(-400, 400);
    long n = 0, special = 0, mismatch = 0, far = 0;
    for (int it = 0; it < 2000000; ++it) {
        const double x = std::ldexp(u(g), ue(g));
        float hi = (float)x, lo = (float)(x - (double)hi);
        if (it % 7 == 0) lo = std::ldexp((float)u(g), ue(g));                 // unnormalised pairs
        if (it % 11 == 0) hi = 0.f;
        if (it % 13 == 0) lo = 0.f;
        if (it % 17 == 0) {                                                   // hi a power of two, lo opposite
            hi = std::ldexp(1.0f, ue(g));
            lo = -std::ldexp(std::fabs((float)u(g)), ue(g) - 30);
        }
        const int E = uE(g);
        bool sp = false;
        const double a = osv::df_to_double_nb(hi, lo, E, sp);
        const double b = osv::df_to_double(hi, lo, E);
        const double ref = std::ldexp((double)hi + (double)lo, E);
        ++n;
        if (!close(b, ref)) ++far;
        if (sp) { ++special; continue; }
        if (std::memcmp(&a, &b, 8) != 0) ++mismatch;
    }
    // special cases must be flagged: infinities, NaN, exponents outside the normal range
    bool sp1 = false, sp2 = false, sp3 = false;
    osv::df_to_double_nb(INFINITY, 0.f, 0, sp1);
    osv::df_to_double_nb(1.0f, 0.f, 1100, sp2);
    osv::df_to_double_nb(1.0f, 0.f, -1100, sp3);
    printf("n=%ld special=%ld mismatch=%ld beyond_2^-51=%ld flags=%d%d%d\n", n, special, mismatch, far, sp1, sp2, sp3);
    return (mismatch == 0 && far == 0 && sp1 && sp2 && sp3) ? 0 : 1;
}

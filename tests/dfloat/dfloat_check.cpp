// Host check of the double-float helpers of csrc/dfloat.cuh (built by tests/test_dfloat.py with
// g++ -ffp-contract=off).  Prints the largest errors found over seeded random operands; the
// references are computed in long double.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "dfloat.cuh"

using rbki::dfl;

static uint64_t state = 0x9E3779B97F4A7C15ull;
static double uniform() {   // splitmix64 -> [0, 1)
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1p-53;
}
static double value() {     // sign, 2^[-20, 20) magnitude, random mantissa
    const double m = 1.0 + uniform();
    const int e = (int)(uniform() * 40.0) - 20;
    return (uniform() < 0.5 ? -1.0 : 1.0) * std::ldexp(m, e);
}
static long double ld(dfl x) { return (long double)x.hi + (long double)x.lo; }
static dfl make(double v) { return rbki::df_from_double(v); }

int main() {
    int sum_inexact = 0, prod_inexact = 0;
    long double e_mul = 0, e_fms = 0, e_rcp = 0, e_rsqrt = 0, e_round = 0, e_norm = 0;
    for (int it = 0; it < 200000; ++it) {
        const float a = (float)value(), b = (float)value();
        const dfl s = rbki::df_two_sum(a, b);
        if ((long double)s.hi + (long double)s.lo != (long double)a + (long double)b) ++sum_inexact;
        // TwoProd inside df_mul with zero low parts: p + e must equal a b exactly
        const dfl p = rbki::df_mul(dfl{a, 0.f}, dfl{b, 0.f});
        if ((long double)p.hi + (long double)p.lo != (long double)a * (long double)b) ++prod_inexact;
        const double xv = value(), yv = value(), wv = value();
        const dfl x = make(xv), y = make(yv), w = make(wv);
        const long double X = ld(x), Y = ld(y), W = ld(w);
        // |lo| <= ulp(hi)/2: the pair is normalised
        const dfl m = rbki::df_mul(x, y);
        if (std::fabs((long double)m.lo) > std::ldexp(std::fabs((long double)m.hi), -24)) e_norm = 1;
        e_mul = std::fmax(e_mul, std::fabs((ld(m) - X * Y) / (X * Y)));
        const dfl f = rbki::df_fms(w, x, y);
        e_fms = std::fmax(e_fms, std::fabs(ld(f) - (W - X * Y)) / (std::fabs(W) + std::fabs(X * Y)));
        const dfl d = make(std::fabs(xv));
        const long double D = ld(d);
        e_rcp = std::fmax(e_rcp, std::fabs(ld(rbki::df_rcp(d)) * D - 1.0L));
        const long double r = ld(rbki::df_rsqrt(d));
        e_rsqrt = std::fmax(e_rsqrt, std::fabs(r * r * D - 1.0L));
        e_round = std::fmax(e_round, std::fabs(((long double)rbki::df_to_double(x) - (long double)xv) / (long double)xv));
    }
    std::printf("sum_inexact %d prod_inexact %d denormalised %d\n", sum_inexact, prod_inexact, (int)e_norm);
    std::printf("mul %.3Le fms %.3Le rcp %.3Le rsqrt %.3Le round %.3Le\n", e_mul, e_fms, e_rcp, e_rsqrt, e_round);
    return 0;
}

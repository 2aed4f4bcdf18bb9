// Host check of the double-float helpers of the CUDA kernels
// (paper_2405_10505_gb300/csrc/kernel_bodies.cuh, compiled here for the host):
//   df_round    - must equal the IEEE double-to-float conversion (round to
//                 nearest, ties to even) bit for bit;
//   df_add_prod - a sum of eight exact float products in double-float must
//                 stay within 2^-44 of the largest term of the exact sum.
//   the FP64 path's double-float helpers (split, ten-term sums of products,
//                 product, sum, square root, reciprocal) and the Newton
//                 reciprocal in double, against long double.
// Prints "round <checked> <mismatches>", "sum <checked> <worst error / 2^-46>"
// and "fp64 <split> <sum10> <mul> <add> <sqrt> <rcp> <newton>" (relative errors).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "kernel_bodies.cuh"

using namespace fblts;

int main() {
    std::mt19937_64 g(2405);
    long n = 0, bad = 0;
    auto chk = [&](double x) {
        const float a = df_round(x), b = (float)x;
        unsigned ua, ub;
        std::memcpy(&ua, &a, 4);
        std::memcpy(&ub, &b, 4);
        ++n;
        if (ua != ub && !(std::isnan(a) && std::isnan(b))) ++bad;
    };
    for (int i = 0; i < 4000000; ++i) {   // random bit patterns: every exponent, NaN and infinity
        const unsigned long long u = g();
        double x;
        std::memcpy(&x, &u, 8);
        chk(x);
    }
    std::uniform_real_distribution<double> U(-1e4, 1e4);
    for (int i = 0; i < 1000000; ++i) chk(U(g));
    for (int i = 0; i < 500000; ++i) {    // exact ties and their neighbours (the 29 dropped bits = 2^28 +- 1)
        const double d = (float)U(g);
        unsigned long long u;
        std::memcpy(&u, &d, 8);
        for (long long k = -1; k <= 1; ++k) {
            const unsigned long long v = u + (1ull << 28) + (unsigned long long)k;
            double y;
            std::memcpy(&y, &v, 8);
            chk(y);
            chk(-y);
        }
    }
    const double special[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                              3.402823567797337e38, 1e39, -1e39, 1.1754943508222875e-38, 1e-40, INFINITY, -INFINITY, NAN};
    for (double x : special) chk(x);
    std::printf("round %ld %ld\n", n, bad);

    // sums of 8 products of floats spanning a few decades, as in the cell pass
    std::uniform_real_distribution<float> F(-1.f, 1.f);
    std::uniform_int_distribution<int> E(-6, 6);
    long m = 0;
    double worst = 0.0;
    for (int t = 0; t < 200000; ++t) {
        float2 s = make_float2(0.f, 0.f);
        long double exact = 0.0L, big = 0.0L;
        for (int j = 0; j < 8; ++j) {
            const float a = std::ldexp(F(g), E(g)), b = std::ldexp(F(g), E(g));
            df_add_prod(s, a, b);
            const long double p = (long double)a * (long double)b;   // exact: 48 bits
            exact += p;
            big = std::fmax(big, std::fabs(p));
        }
        const long double got = (long double)s.x + (long double)s.y;
        if (big > 0) worst = std::fmax(worst, (double)(std::fabs(got - exact) / big) / std::ldexp(1.0, -46));
        ++m;
    }
    std::printf("sum %ld %.6f\n", m, worst);

    // the FP64 path's helpers against long double (relative errors)
    std::uniform_real_distribution<double> D(0.5, 2.0);
    std::uniform_int_distribution<int> X(-20, 20);
    double e_split = 0, e_sum10 = 0, e_mul = 0, e_add = 0, e_sqrt = 0, e_rcp = 0, e_nr = 0;
    for (int t = 0; t < 200000; ++t) {
        const double a = std::ldexp(D(g), X(g)) * (t & 1 ? -1.0 : 1.0), b = std::ldexp(D(g), X(g));
        const float2 sa = df_split(a), sb = df_split(b);
        e_split = std::fmax(e_split, std::fabs(df_value(sa) - a) / std::fabs(a));
        const long double pa = (long double)df_value(sa), pb = (long double)df_value(sb);
        const float2 pm = ff_mul(sa, sb), ps = ff_add(sa, sb);
        e_mul = std::fmax(e_mul, (double)(std::fabs((long double)df_value(pm) - pa * pb) / std::fabs(pa * pb)));
        const long double exact_sum = pa + pb;
        if (exact_sum != 0)   // relative to the larger operand (cancellation is exact in the leading parts)
            e_add = std::fmax(e_add, (double)(std::fabs((long double)df_value(ps) - exact_sum) /
                                              std::fmax(std::fabs(pa), std::fabs(pb))));
        const float2 rt = ff_sqrt(sb), rc = ff_rcp(sb);
        e_sqrt = std::fmax(e_sqrt, (double)(std::fabs((long double)df_value(rt) - std::sqrt(pb)) / std::sqrt(pb)));
        e_rcp = std::fmax(e_rcp, (double)(std::fabs((long double)df_value(rc) - 1.0L / pb) * pb));
        e_nr = std::fmax(e_nr, (double)(std::fabs((long double)rcp_nr(b) - 1.0L / (long double)b) * (long double)b));
        // a ten-term sum of products, as in the edgesOnEdge sums
        float2 s10 = make_float2(0.f, 0.f);
        long double ex = 0.0L, big = 0.0L;
        for (int j = 0; j < 10; ++j) {
            const double w = std::ldexp(D(g), X(g) / 4) * (j & 1 ? -1.0 : 1.0), f = std::ldexp(D(g), X(g) / 4);
            const float2 sw = df_split(w), sf = df_split(f);
            df_fma(s10, sw, sf);
            const long double p = (long double)df_value(sw) * (long double)df_value(sf);
            ex += p;
            big = std::fmax(big, std::fabs(p));
        }
        e_sum10 = std::fmax(e_sum10, (double)(std::fabs((long double)df_value(s10) - ex) / big));
    }
    std::printf("fp64 %.3e %.3e %.3e %.3e %.3e %.3e %.3e\n", e_split, e_sum10, e_mul, e_add, e_sqrt, e_rcp, e_nr);
    return 0;
}

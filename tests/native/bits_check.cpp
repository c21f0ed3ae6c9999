// Host-side check of the integer-pipe geometry and FP32-pair helpers of the
// cell walk against their plain FP64 definitions.  Prints "ok <cases>" or the
// first failing case; exit status 0 on success.
#include <cmath>
#include <cstdio>
#include <random>
#include "bits.cuh"

using namespace rg;

static int fails = 0;
static long long cases = 0;
#define CHECK(c, ...) do { ++cases; if (!(c)) { if (fails++ < 10) { std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

static int coord_ref(double p, bool neg, int L) {
    double y = std::ldexp(p, L);
    double r = neg ? std::ceil(y) - 1.0 : std::floor(y);
    return (int)r;
}

static void check_coord(double p, int L) {
    for (int neg = 0; neg < 2; ++neg) {
        int r = coord_ref(p, neg, L), c = cell_coord(p, neg, L);
        int n = 1 << L;
        bool rin = r >= 0 && r < n, cin = c >= 0 && c < n;
        CHECK(rin == cin && (!rin || r == c), "cell_coord p=%.17g neg=%d L=%d ref=%d got=%d", p, neg, L, r, c);
    }
}

int main() {
    std::mt19937_64 g(2001011252ull);
    std::uniform_real_distribution<double> U(-0.5, 1.5);
    // dyadic: every m < 2^15 at several levels, plus large m
    for (int l = 0; l <= 30; l += 3)
        for (uint32_t m = 0; m < (1u << 15); m += (l < 10 ? 1 : 7))
            CHECK(dyadic(m, l) == std::ldexp((double)m, -l), "dyadic m=%u l=%d", m, l);
    for (int i = 0; i < 100000; ++i) {
        uint32_t m = (uint32_t)(g() >> 33);
        int l = (int)(g() % 40);
        CHECK(dyadic(m, l) == std::ldexp((double)m, -l), "dyadic m=%u l=%d", m, l);
    }
    // cell coordinates: random points, cell faces and their neighbours
    for (int L = 0; L <= 20; ++L) {
        for (int i = 0; i < 20000; ++i) check_coord(U(g), L);
        for (int i = 0; i < 4000; ++i) {
            double f = std::ldexp((double)(g() % ((1ull << L) + 1)), -L);
            check_coord(f, L);
            check_coord(std::nextafter(f, 2.0), L);
            check_coord(std::nextafter(f, -1.0), L);
        }
        const double sp[] = {0.0, -0.0, 1.0, -1e-300, 1e-300, 5e-324, -5e-324, 0.9999999999999999, 1.0000000000000002,
                             1.9999999999999998, 2.0, 7.0, -0.75, 0.5, 0.25};
        for (double p : sp) check_coord(p, L);
    }
    // order keys: same order as <, -0 == +0
    for (int i = 0; i < 200000; ++i) {
        double a = (g() & 1) ? U(g) * 1e-3 : U(g), b = (i % 3 == 0) ? a : ((g() & 1) ? -a : U(g));
        if (i % 11 == 0) b = std::nextafter(a, 5.0);
        CHECK((a < b) == (order_key(a) < order_key(b)) && (a == b) == (order_key(a) == order_key(b)),
              "order a=%.17g b=%.17g", a, b);
        CHECK(from_key(order_key(a)) == a, "from_key a=%.17g", a);
    }
    CHECK(order_key(-0.0) == order_key(0.0), "order -0");
    // sign tests
    const double ks[] = {0.0, -0.0, 1e-300, -1e-300, 0.5, -0.5};
    for (double k : ks) {
        CHECK(is_neg(k) == (k < 0.0), "is_neg %g", k);
        CHECK(is_pos(k) == (k > 0.0), "is_pos %g", k);
        CHECK(is_zero(k) == (k == 0.0), "is_zero %g", k);
    }
    // FP32 pairs: ~44-bit sums and products
    std::uniform_real_distribution<double> V(1e12, 3e15);
    for (int i = 0; i < 200000; ++i) {
        double x = V(g) * ((g() & 1) ? 1 : -1), y = V(g) * 1e-3 * ((g() & 1) ? 1 : -1);
        f2 a = f2_of(x), b = f2_of(y);
        double s = f2_val(f2_add(a, b)), ref = f2_val(a) + f2_val(b);
        CHECK(std::fabs(s - ref) <= 1e-13 * std::fabs(ref) + 1e-13 * std::fabs(f2_val(a)), "f2_add %.17g %.17g", x, y);
        double z = 1e-11 * (1 + (double)(g() % 1000) / 997.0);
        f2 c = f2_of(z);
        double pr = f2_val(f2_mul(a, c)), pref = f2_val(a) * f2_val(c);
        CHECK(std::fabs(pr - pref) <= 4e-13 * std::fabs(pref), "f2_mul %.17g %.17g", x, z);
        float w = (float)(z * 1e11);
        double pf = f2_val(f2_mul_f(a, w)), pfref = f2_val(a) * (double)w;
        CHECK(std::fabs(pf - pfref) <= 4e-13 * std::fabs(pfref), "f2_mul_f %.17g %g", x, w);
    }
    if (fails) {
        std::printf("FAIL %d of %lld\n", fails, cases);
        return 1;
    }
    std::printf("ok %lld\n", cases);
    return 0;
}

// Host check of sta::int_add against the CPU's IEEE binary64 addition (round to nearest
// even).  Prints "<cases> <mismatches>" and the first mismatches.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>

#include "softfloat.cuh"

static uint64_t s = 0x9e3779b97f4a7c15ull;
static uint64_t rnd() {  // xorshift64*
    s ^= s >> 12; s ^= s << 25; s ^= s >> 27;
    return s * 0x2545f4914f6cdd1dull;
}
static double from(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }
static uint64_t bits(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }

static long long cases = 0, bad = 0;
static void check(double a, double b) {
    volatile double ref = a + b;
    double got = sta::int_add(a, b);
    ++cases;
    if (bits(got) != bits(ref) && !(std::isnan(got) && std::isnan(ref))) {
        if (++bad <= 10)
            printf("MISMATCH a=%a b=%a got=%a ref=%a\n", a, b, got, (double)ref);
    }
}

static double rnd_normal(int emin, int emax) {
    uint64_t e = (uint64_t)(emin + (int)(rnd() % (uint64_t)(emax - emin + 1)));
    return from((rnd() & 0x800fffffffffffffull) | (e << 52));
}

int main() {
    const double special[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN,
                              from(1), from(0x000fffffffffffffull), from(0x0010000000000000ull),
                              from(0x7fefffffffffffffull), from(0xffefffffffffffffull),
                              from(0x8000000000000001ull), 0x1p-1022, -0x1p-1022, 0x1p1023};
    for (double a : special)
        for (double b : special) check(a, b);
    for (int i = 0; i < 2000000; ++i) check(from(rnd()), from(rnd()));  // any bit pattern
    for (int i = 0; i < 4000000; ++i) {  // normal operands, exponent gaps 0..70
        double a = rnd_normal(900, 1100);
        int gap = (int)(rnd() % 71);
        uint64_t ea = (bits(a) >> 52) & 0x7ff;
        uint64_t eb = ea > (uint64_t)gap ? ea - gap : 1;
        double b = from((rnd() & 0x800fffffffffffffull) | (eb << 52));
        check(a, b);
        check(b, a);
    }
    for (int i = 0; i < 2000000; ++i) {  // near cancellation
        double a = rnd_normal(1000, 1050);
        double b = -a * (1.0 + ldexp((double)(int64_t)(rnd() % 2000) - 1000.0, -52));
        check(a, b);
        check(a, -nextafter(a, 0.0));
    }
    for (int i = 0; i < 2000000; ++i) {  // exact ties and near ties
        double a = rnd_normal(1000, 1050);
        int ea = (int)((bits(a) >> 52) & 0x7ff) - 1075;  // exponent of a's ulp
        double odd = (double)(2 * (int64_t)(rnd() % 64) + 1);
        double b = ldexp(odd, ea - 1) * ((rnd() & 1) ? 1.0 : -1.0);  // odd half-ulps
        check(a, b);
        check(a, nextafter(b, 0.0));
        check(a, nextafter(b, 2 * b));
    }
    for (int i = 0; i < 1000000; ++i) {  // results near the subnormal and overflow edges
        check(rnd_normal(1, 60), rnd_normal(1, 60) * ((rnd() & 1) ? 1.0 : -1.0));
        check(rnd_normal(2000, 2046), rnd_normal(2000, 2046));
    }
    printf("%lld %lld\n", cases, bad);
    return bad != 0;
}

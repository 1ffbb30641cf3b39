// Host check of the integer helpers of the uniform-grid location
// (dlm_device.cuh): first_cell_xi against the FP64 arithmetic it replaces
// (2 t - 1 rounded to nearest, ties to even, for t = d 2^s in [0, 1)),
// exact_scaled against ldexp, and division_magic against integer division.
// Prints the number of mismatches; exits non-zero on any.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "dlm_device.cuh"

using namespace fsi::dlmd;

static long long bits_of(double d)
{
    long long b;
    std::memcpy(&b, &d, sizeof b);
    return b;
}

int main()
{
    std::mt19937_64 rng(20260);
    long long bad = 0, n = 0;
    auto check_xi = [&](double d, int s) {
        const double t = std::ldexp(d, s);
        if (!(t >= 0.0 && t < 1.0)) return;
        volatile double two_t = 2.0 * t;  // exact; the subtraction rounds once
        const double ref = two_t - 1.0;
        ++n;
        if (bits_of(ref) != bits_of(first_cell_xi(bits_of(d), s))) {
            if (bad < 5) std::printf("first_cell_xi d=%a s=%d\n", d, s);
            ++bad;
        }
    };
    for (int s : {0, 1, 4, 7, 31, 52, 53, 200, 1000}) {
        for (int i = 0; i < 60000; ++i) {
            const int e = -(int)(rng() % 80) - 1;
            const uint64_t m = rng() & 0xfffffffffffffULL;
            check_xi(std::ldexp(std::ldexp(1.0 + std::ldexp((double)m, -52), e), -s), s);
            // few significant bits: rounding ties
            const uint64_t m2 = (rng() & 0xff) << (rng() % 45);
            check_xi(std::ldexp(std::ldexp(1.0 + std::ldexp((double)(m2 & 0xfffffffffffffULL), -52), e), -s), s);
            // subnormal d
            const uint64_t sub = rng() & 0xfffffffffffffULL;
            double ds;
            std::memcpy(&ds, &sub, sizeof ds);
            check_xi(ds, s);
        }
        check_xi(0.0, s);
        check_xi(-0.0, s);
        check_xi(std::ldexp(0.5, -s), s);
        check_xi(std::nextafter(std::ldexp(1.0, -s), 0.0), s);
    }
    for (int i = 0; i < 200000; ++i) {
        long long Z = (long long)(rng() >> 11) - (1LL << 52);
        if (Z == 0) continue;
        const int p = (int)(rng() % 80) - 60;
        ++n;
        if (bits_of(exact_scaled(Z, p)) != bits_of(std::ldexp((double)Z, p))) {
            if (bad < 10) std::printf("exact_scaled Z=%lld p=%d\n", Z, p);
            ++bad;
        }
    }
    for (int d : {1, 2, 3, 7, 100, 127, 128, 129, 1000, 65537, (1 << 30) + 1, 2147483647}) {
        unsigned long long M;
        int k;
        division_magic(d, M, k);
        for (int i = 0; i < 100000; ++i) {
            const unsigned v = i < 2000 ? (unsigned)i : (i < 4000 ? 2147483647u - (unsigned)(i - 2000)
                                                               : (unsigned)(rng() % 2147483648ULL));
            ++n;
            if ((unsigned)(((unsigned long long)v * M) >> k) != v / (unsigned)d) {
                if (bad < 15) std::printf("division_magic d=%d v=%u\n", d, v);
                ++bad;
            }
        }
    }
    std::printf("checked %lld, mismatches %lld\n", n, bad);
    return bad != 0;
}

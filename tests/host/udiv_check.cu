// Host-side check of the multiply-shift unsigned divider (compiled by nvcc as
// host code): quotients equal the hardware division for every divisor the
// kernels use (sub-ray counts, image sides, grid sides) and for random 32-bit
// divisors, over edge numerators (0, multiples of d and their neighbours,
// 2^32 - 1) and random numerators.  Prints the number of mismatches.
#include <cstdio>
#include <cstdint>
#include "rtu_math.cuh"

using namespace rtu;

static uint32_t xs(uint64_t& s) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    return (uint32_t)(s >> 11);
}

int main() {
    uint64_t seed = 0x9e3779b97f4a7c15ull;
    long bad = 0, checked = 0;
    auto check = [&](uint32_t n, uint32_t d, const UDiv& u) {
        ++checked;
        if (udiv(n, u) != n / d) {
            if (bad < 5) printf("mismatch n=%u d=%u got=%u want=%u\n", n, d, udiv(n, u), n / d);
            ++bad;
        }
    };
    for (uint32_t d = 1; d <= 70000; ++d) {
        const UDiv u = udiv_make(d);
        const uint32_t edge[] = {0u, 1u, d - 1, d, d + 1, 2 * d - 1, 2 * d, 0xffffffffu, 0xfffffffeu,
                                 (0xffffffffu / d) * d, (0xffffffffu / d) * d - 1, 1u << 24, (1u << 24) - 1};
        for (uint32_t n : edge) check(n, d, u);
        for (int k = 0; k < 64; ++k) check(xs(seed), d, u);
    }
    for (int k = 0; k < 200000; ++k) {
        uint32_t d = xs(seed);
        if (d == 0) d = 1;
        const UDiv u = udiv_make(d);
        check(xs(seed), d, u);
        check(0xffffffffu, d, u);
        check(d, u.m ? d : d, u);
        check(d - 1, d, u);
    }
    printf("checked %ld mismatches %ld\n", checked, bad);
    return 0;
}

// Prints, for each divisor on stdin, the number of dividends (from a fixed
// list and a seeded sweep) where FastDiv::div differs from n / d.
#include <cstdio>
#include <cstdint>
#include "fastdiv.h"

int main()
{
    unsigned long long d_in;
    while (std::scanf("%llu", &d_in) == 1) {
        const uint32_t d = (uint32_t)d_in;
        const FastDiv f = FastDiv::make(d);
        uint64_t bad = 0, checked = 0;
        auto check = [&](uint32_t n) {
            checked++;
            if (f.div(n) != n / d) bad++;
        };
        const uint32_t edges[] = {0u, 1u, 2u, d - 1, d, d + 1, 2 * d - 1, 2 * d, 0x7fffffffu, 0x80000000u,
                                  0xfffffffeu, 0xffffffffu};
        for (uint32_t n : edges) check(n);
        for (uint64_t q = 1; q * d <= 0xffffffffull && q < (1u << 20); q = q * 3 + 1) {
            check((uint32_t)(q * d - 1));
            check((uint32_t)(q * d));
        }
        uint64_t x = 0x9E3779B97F4A7C15ull ^ d;   // splitmix64 sweep
        for (int i = 0; i < 200000; i++) {
            x += 0x9E3779B97F4A7C15ull;
            uint64_t z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            check((uint32_t)(z ^ (z >> 31)));
        }
        std::printf("%u %llu %llu\n", d, (unsigned long long)bad, (unsigned long long)checked);
    }
    return 0;
}

// fastdiv.h -- unsigned 32-bit division by a divisor fixed at run time.
//
// Follows Granlund & Montgomery, "Division by Invariant Integers using
// Multiplication" (PLDI 1994), Section 4 (unsigned division, N = 32): with
// l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1, the quotient of
// every 32-bit n is
//     t = mulhi(m, n),  q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
// One multiply-high, a subtract, an add and two shifts instead of the
// integer division sequence.  Host and device share this header; plain C++
// compilers see ordinary functions.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define GTX_HD __host__ __device__ __forceinline__
#else
#define GTX_HD inline
#endif

struct FastDiv {
    uint32_t d, m, s1, s2;

    static FastDiv make(uint32_t d)
    {
        FastDiv f;
        f.d = d < 1 ? 1 : d;
        uint32_t l = 0;
        while (l < 32 && (1ull << l) < f.d) l++;
        // 2^l - d < 2^(l-1) <= 2^31, so the product stays below 2^63
        f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - f.d)) / f.d + 1);
        f.s1 = l < 1 ? l : 1;
        f.s2 = l > 1 ? l - 1 : 0;
        return f;
    }

    GTX_HD uint32_t div(uint32_t n) const
    {
#ifdef __CUDA_ARCH__
        const uint32_t t = __umulhi(m, n);
#else
        const uint32_t t = (uint32_t)(((uint64_t)m * n) >> 32);
#endif
        return (t + ((n - t) >> s1)) >> s2;
    }
};

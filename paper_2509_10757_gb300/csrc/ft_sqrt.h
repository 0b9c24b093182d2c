// ft_sqrt.h -- the FP32 magnitude of a keypoint's intensity moments
// (next row f3, orientation) without double precision.
//
// The orientation reading takes |m| = sqrt(m10^2 + m01^2) in double,
// rounded to float.  For an integer n below 2^48 that value is the
// correctly rounded float square root of n: a float midpoint m' near
// sqrt(n) in [2^e, 2^(e+1)) (e <= 23) is an odd multiple of 2^(e-24), so
// n - m'^2 is a nonzero multiple of 2^(2e-48) (a float midpoint squared is
// never an integer there), |sqrt(n) - m'| >= 2^(2e-48) / 2^(e+2) = 2^(e-50),
// more than the double rounding's 2^(e-53): the double result and sqrt(n)
// round to the same float.  The moments of the radius-15 disk stay below
// 2^20 in magnitude, so n < 2^41.
//
// float_sqrt_rn takes the FP32 square root of n rounded to float (within
// one unit in the last place of the result) and settles it with exact
// 64-bit integer comparisons of n against the squares of the candidate's
// rounding interval ends.  Host and device code (the host form is tested
// against the double definition on the CPU).
#pragma once

#include <cstdint>
#include <cstring>
#ifndef __CUDACC__
#include <cmath>
#define FT_HD inline
#else
#define FT_HD __host__ __device__ __forceinline__
#endif

namespace ft {

FT_HD uint32_t ft_float_bits(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
#endif
}

FT_HD float ft_bits_float(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}

// Where n lies against the rounding interval of the positive normal float
// with bits b: -1 below its lower end, +1 above its upper end, 0 inside
// (ends included: the ends are never hit for n < 2^48).  With
// f = F 2^G (2^23 <= F < 2^24) the upper end is (4F + 2) 2^(G-2) and the
// lower end (4F - 2) 2^(G-2), or (4F - 1) 2^(G-2) when F = 2^23 (the float
// below has half the spacing); both sides are scaled by 2^(4 - 2G).
FT_HD int ft_sqrt_side(uint64_t n, uint32_t b)
{
    const int G = (int)(b >> 23) - 127 - 23;
    const uint64_t F = (uint64_t)((b & 0x7fffffu) | 0x800000u);
    const uint64_t N = n << (4 - 2 * G);
    const uint64_t lo = F == 0x800000u ? 4 * F - 1 : 4 * F - 2, hi = 4 * F + 2;
    if (N > hi * hi) return 1;
    if (N < lo * lo) return -1;
    return 0;
}

// float(sqrt((double)n)) for 1 <= n < 2^41, in FP32 and integer arithmetic
FT_HD float float_sqrt_rn(uint64_t n)
{
#ifdef __CUDA_ARCH__
    uint32_t b = __float_as_uint(__fsqrt_rn(__ull2float_rn(n)));
#else
    uint32_t b = ft_float_bits(std::sqrt((float)n));
#endif
    const int side = ft_sqrt_side(n, b);
    b += side;      // the neighbour on that side (adjacent floats differ by one in their bits)
    return ft_bits_float(b);
}

}  // namespace ft

// The numerator of the 5-point (2D) or 7-point (3D) Laplacian at a node,
//     S = sum_k u_k - N u_p   (N = 2d neighbours u_k, centre u_p),
// summed exactly in 64-bit integers and rounded once to double.
//
// Why: the FP64 defect f + S / h^2 (TGCS step 3, Eq. discr) of the mixed
// form's refinement and of the plain FP64 cycle costs 12 FP64 operations a node in
// the sum-of-differences form, and GB300's FP64 pipe is slow enough that the
// defect pass is bound by it rather than by HBM.  Here the FP64 pipe does only
// the conversion of S and the scaling by 2^k; the rest is integer work.
//
// How: every value x = m 2^(e - 1075) (m the 53-bit significand, implicit
// bit included; denormals with e = 1) is put on the largest exponent E of the
// N + 1 values as (m << 5) >> (E - e).  With |m << 5| < 2^58 and N <= 6 the
// sum stays below 2^62.  Values within 5 binades of the largest are exact;
// a smaller one loses at most one unit of 2^(E - 1080), 1/32 of an ulp of the
// largest value.  The result is S 2^(E - 1080), S rounded once (to nearest)
// by the int64 -> double conversion; the scaling by a power of two is exact.
// A sum of 0 is returned as +0.0 whatever E.  Not finite values, or a
// nonzero sum whose largest value lies below 2^-1015 (E < 60), return false
// and the caller uses the plain FP64 sum.
//
// Compiled both by nvcc (device) and by a host C++ compiler (the CPU test of
// this arithmetic against exact rationals).
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define EXL_HD __host__ __device__ __forceinline__
#else
#include <string.h>
#define EXL_HD inline
#endif

namespace exl {

EXL_HD uint64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

EXL_HD double double_of(uint64_t b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
#endif
}

// biased exponent, denormals (and zero) counted as 1
EXL_HD int binade(uint64_t b) {
    const int e = (int)((b >> 52) & 0x7ff);
    return e ? e : 1;
}

// the signed significand << 5, shifted right by sh >= 0 (truncating its magnitude)
EXL_HD int64_t aligned(uint64_t b, int sh) {
    uint64_t m = (b & 0xfffffffffffffull) | (((b >> 52) & 0x7ff) ? (1ull << 52) : 0ull);
    m <<= 5;
    m = sh < 64 ? (m >> sh) : 0ull;
    return (b >> 63) ? -(int64_t)m : (int64_t)m;
}

// S = sum_k nb[k] - N up into *out; false when the caller must use FP64 instead
template <int N>
EXL_HD bool lap_sum_exact(double up, const double (&nb)[N], double *out) {
    const uint64_t bp = bits_of(up);
    uint64_t b[N];
    int E = binade(bp);
#pragma unroll
    for (int k = 0; k < N; k++) {
        b[k] = bits_of(nb[k]);
        const int e = binade(b[k]);
        E = e > E ? e : E;
    }
    if (E == 0x7ff) return false;
    int64_t s = -(int64_t)N * aligned(bp, E - binade(bp));
#pragma unroll
    for (int k = 0; k < N; k++) s += aligned(b[k], E - binade(b[k]));
    if (s == 0) {   // includes a neighbourhood of zeros (a solve's start from u = 0)
        *out = 0.0;
        return true;
    }
    if (E < 60) return false;
    // 2^(E - 1080): biased exponent E - 57 >= 3
    *out = (double)s * double_of((uint64_t)(E - 57) << 52);
    return true;
}

}  // namespace exl

// Exact octree geometry on the integer pipes, and FP32 pair ("double-float")
// arithmetic, for the cell walk of Sect. 4.3.
//
// GB300 issues FP64 instructions -- conversions and comparisons included -- at
// 2 lanes per clock per SM, against 128 for FP32 and 64 for integer ops.  The
// walk therefore keeps only the two FP64 operations whose rounding defines the
// path (face - p and its product with 1/k, plus the position update) and does
// everything else on the other pipes, with results bit-identical to the plain
// FP64 expressions they replace:
//   dyadic(m, l)       == (double)m * 2^-l                  (face coordinates)
//   cell_coord(p,n,L)  == floor(p 2^L), or ceil(p 2^L) - 1   (cell of p + eps k)
//   order_key(t)       orders doubles as < does (-0 == +0)
// The header also compiles as host C++ so that these identities are checked
// on the CPU against the FP64 definitions.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define RG_HD __host__ __device__ __forceinline__
#else
#define RG_HD inline
#endif

namespace rg {

RG_HD int64_t dbits(double x) {
#if defined(__CUDA_ARCH__)
    return __double_as_longlong(x);
#else
    int64_t b;
    std::memcpy(&b, &x, 8);
    return b;
#endif
}

RG_HD double bitsd(int64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double(b);
#else
    double x;
    std::memcpy(&x, &b, 8);
    return x;
#endif
}

RG_HD int clz32(uint32_t m) {
#if defined(__CUDA_ARCH__)
    return __clz((int)m);
#else
    return m ? __builtin_clz(m) : 32;
#endif
}

// exactly m 2^-l, for 0 <= m < 2^31 and 0 <= l <= 1000
RG_HD double dyadic(uint32_t m, int l) {
    if (m == 0u) return 0.0;
    const int e = 31 - clz32(m);   // 2^e <= m < 2^(e+1)
    const uint64_t mant = ((uint64_t)m << (52 - e)) & ((1ull << 52) - 1ull);
    return bitsd((int64_t)(((uint64_t)(1023 + e - l) << 52) | mant));
}

// k < 0.0 as an FP64 comparison gives it (-0.0 is not negative)
RG_HD bool is_neg(double k) {
    const int64_t b = dbits(k);
    return b < 0 && b != INT64_MIN;
}
RG_HD bool is_pos(double k) { return dbits(k) > 0; }   // k > 0.0 for non-NaN k
RG_HD bool is_zero(double k) { return (dbits(k) & INT64_MAX) == 0; }

// Integer coordinate at level L of the cell holding p + eps k: floor(p 2^L)
// for k >= 0, ceil(p 2^L) - 1 for k < 0 (neg).  Exact for p in (-1, 2);
// beyond, any value outside [0, 2^L) (the callers only test that range).
RG_HD int cell_coord(double p, bool neg, int L) {
    const int64_t b = dbits(p);
    if (b <= 0) {
        if (b == 0 || b == INT64_MIN) return neg ? -1 : 0;   // p = +-0
        return -1;                                            // p < 0
    }
    const int e = (int)(b >> 52) - 1023;   // p > 0: 2^e <= p < 2^(e+1)
    if (e + L < 0) return 0;               // 0 < p 2^L < 1
    if (e >= 1) return (1 << L) + 1;       // p >= 2
    const int sh = 52 - (e + L);           // p 2^L = M 2^-sh, sh >= 52 - L
    const uint64_t M = ((uint64_t)b & ((1ull << 52) - 1ull)) | (1ull << 52);
    const int fl = (int)(M >> sh);
    const bool whole = (M & ((1ull << sh) - 1ull)) == 0ull;
    return (neg && whole) ? fl - 1 : fl;
}

// Signed integer whose order is that of the doubles (NaN excluded), with
// -0.0 and +0.0 equal
RG_HD int64_t order_key(double t) {
    const int64_t b = dbits(t);
    return b >= 0 ? b : -(b & INT64_MAX);
}
RG_HD double from_key(int64_t k) { return k >= 0 ? bitsd(k) : bitsd((-k) | INT64_MIN); }

// ---------------------------------------------------------------------------
// FP32 pairs: value = h + l with |l| <= ulp(h) / 2 (Dekker 1971; Knuth's
// two-sum).  About 44 significant bits.
// ---------------------------------------------------------------------------
struct f2 {
    float h, l;
};

RG_HD f2 two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
RG_HD f2 fast_two_sum(float a, float b) {   // |a| >= |b|
    float s = a + b;
    return {s, b - (s - a)};
}
RG_HD f2 two_prod(float a, float b) {
    float p = a * b;
#if defined(__CUDA_ARCH__)
    return {p, __fmaf_rn(a, b, -p)};
#else
    return {p, std::fma(a, b, -p)};
#endif
}
RG_HD float fma_(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}
RG_HD f2 f2_add(f2 x, f2 y) {
    f2 s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, s.l + (x.l + y.l));
}
RG_HD f2 f2_add_f(f2 x, float y) {
    f2 s = two_sum(x.h, y);
    return fast_two_sum(s.h, s.l + x.l);
}
RG_HD f2 f2_mul(f2 x, f2 y) {
    f2 p = two_prod(x.h, y.h);
    return fast_two_sum(p.h, fma_(x.h, y.l, fma_(x.l, y.h, p.l)));
}
RG_HD f2 f2_mul_f(f2 x, float y) {
    f2 p = two_prod(x.h, y);
    return fast_two_sum(p.h, fma_(x.l, y, p.l));
}
RG_HD f2 f2_neg(f2 x) { return {-x.h, -x.l}; }
// split of a double (host or once per ray)
RG_HD f2 f2_of(double d) {
    float h = (float)d;
    return {h, (float)(d - (double)h)};
}
RG_HD double f2_val(f2 x) { return (double)x.h + (double)x.l; }

}  // namespace rg

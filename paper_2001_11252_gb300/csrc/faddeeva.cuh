// Accurate Hjerting-Voigt option: H(a,x) and Im w of the Faddeeva function in
// FP32 (Sect. 3.3.2 weighs fast approximations of H against an accurate
// evaluation).  Host/device code: on the GPU the four helpers below are the
// CUDA intrinsics; the header also compiles as host C++ so that its arithmetic
// is checked on the CPU against scipy's wofz (tests/native/faddeeva_check.cpp).
#pragma once
#include <cmath>
#include <utility>
#include "bits.cuh"

namespace rg {

constexpr float kFadPiF = 3.14159265358979f;
constexpr float kFadSqrtPiF = 1.7724538509055159f;

RG_HD float fdiv_fast(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
RG_HD int round_int(float x) {
#if defined(__CUDA_ARCH__)
    return __float2int_rn(x);
#else
    return (int)std::nearbyint(x);
#endif
}
RG_HD void sincospi_f(float x, float* s, float* c) {
#if defined(__CUDA_ARCH__)
    sincospif(x, s, c);
#else
    const double t = 3.14159265358979323846 * (double)x;
    *s = (float)std::sin(t);
    *c = (float)std::cos(t);
#endif
}
RG_HD float sinpi_f(float x) {
#if defined(__CUDA_ARCH__)
    return sinpif(x);
#else
    return (float)std::sin(3.14159265358979323846 * (double)x);
#endif
}

// ---------------------------------------------------------------------------
// Accurate H(a,x) option: H + iK = w(x + ia), the Faddeeva function
//   w(z) = (i/pi) int exp(-t^2) / (z - t) dt,   Im z > 0.
// The trapezoidal rule of step h on the nodes n h misses only the residue of
// the pole t = z, known in closed form (Matta & Reichel 1971; Hunter & Regan
// 1972):  w = (i h/pi) sum_n e^{-n^2 h^2} / (z - n h)
//             + 2 e^{-z^2} / (1 - e^{-2 pi i z / h}),
// with a remainder of order e^{-pi^2/h^2} (h = 1/2: e^-39.5).  Every node
// adds a positive Lorentzian (h/pi) e^{-n^2 h^2} a / ((x - n h)^2 + a^2) to
// H, except that for small a the term of the node m nearest to x and the
// residue term are both large and nearly cancel.  They are combined exactly:
// with zeta = z - m h, u = -zeta (zeta + 2 m h), v = 2 pi i zeta / h,
//   node m + residue = (i h/pi) e^{-m^2 h^2} E(u) (zeta + 2 m h) + 2 e^{-z^2} B(v),
// E(u) = (e^u - 1)/u and B(v) = 1/(1 - e^{-v}) - 1/v, both regular at 0 (Taylor
// and Bernoulli-number series there), so FP32 keeps ~5e-7 relative accuracy
// in H and K for 0 <= a <= 1 for |x| <= 8 (nodes |n| <= 11; weights below
// e^-30 are left out).  The remainder grows like e^{2 pi a/h - pi^2/h^2}: 4e-6
// at a = 2, and the rule is not valid beyond (a line of Table 1 reaches a = 2
// only below ~0.01 K).  Beyond |x| = 8 the asymptotic series of w is cheaper
// and as accurate (fad_far).
// ---------------------------------------------------------------------------
// (h/pi) e^{-n^2 h^2} for h = 1/2, at compile time: e^{-1/4} by its Taylor
// series, raised to the power n^2
RG_HD constexpr double fad_weight(int n) {
    double q = 1.0, t = 1.0;
    for (int k = 1; k < 24; ++k) {
        t *= -0.25 / k;
        q += t;
    }
    double r = 1.0;
    for (int i = 0; i < n * n; ++i) r *= q;
    return 0.5 / 3.14159265358979323846 * r;
}

// the Lorentzian of node N (skipped when N is the node m handled apart)
template <int N>
RG_HD void fad_node(float a, float a2, float xh, float xl, int m, float& H, float& K) {
    constexpr float w = (float)fad_weight(N < 0 ? -N : N);
    const float d = (xh - 0.5f * (float)N) + xl;
    const float r = fdiv_fast(1.0f, fmaf(d, d, a2));
    if (N != m) {
        H = fmaf(w * a, r, H);
        K = fmaf(w * d, r, K);
    }
}

template <int... I>
RG_HD void fad_nodes(float a, float xh, float xl, int m, float& H, float& K, std::integer_sequence<int, I...>) {
    const float a2 = a * a;
    (fad_node<I - 11>(a, a2, xh, xl, m, H, K), ...);
}

// Far wing, |x| > 8: w(z) = (i/sqrt(pi)) sum_k c_k z^-(2k+1), c_k = (2k-1)!!/2^k
// (Laplace's asymptotic series; the e^{-z^2} part is below e^-64 there).  With
// u = 1/z and v = u^2 the imaginary parts of every product add with one sign
// for a <= 1, so H and K keep FP32 accuracy; six terms leave < 3e-8.
RG_HD void fad_far(float a, float x, float& H, float& K) {
    const float q = fdiv_fast(1.0f, fmaf(x, x, a * a));
    const float ur = x * q, ui = -a * q;
    const float vr = ur * ur - ui * ui, vi = 2.0f * ur * ui;
    float pr = 945.0f / 32.0f, pi = 0.0f;
    const float c[5] = {105.0f / 16.0f, 15.0f / 8.0f, 0.75f, 0.5f, 1.0f};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float tr = pr * vr - pi * vi;
        pi = pr * vi + pi * vr;
        pr = tr + c[k];
    }
    H = -(ur * pi + ui * pr) * (1.0f / kFadSqrtPiF);
    K = (ur * pr - ui * pi) * (1.0f / kFadSqrtPiF);
}

// H and K = Im w at z = (xh + xl) + i a, x carried as an FP32 pair
RG_HD void faddeeva_hk(float a, float xh, float xl, float& H, float& K) {
    if (!(fabsf(xh) <= 8.0f)) {
        fad_far(a, xh + xl, H, K);
        return;
    }
    const int m = round_int(2.0f * xh);
    H = 0.0f;
    K = 0.0f;
    fad_nodes(a, xh, xl, m, H, K, std::make_integer_sequence<int, 23>{});
    const float mf = (float)m;
    const float d = (xh - 0.5f * mf) + xl;   // zeta = d + i a, |d| <= 1/4
    // node m: (i h/pi) e^{-m^2/4} E(u) (zeta + m), u = -zeta (zeta + m)
    const float pr = d + mf;
    const float ur = fmaf(a, a, -d * pr), ui = -a * (2.0f * d + mf);
    float er, ei;
    if (ur * ur + ui * ui < 0.25f) {
        // E(u) = sum_k u^k / (k + 1)!
        er = 1.0f / 362880.0f;
        ei = 0.0f;
        const float c[8] = {1.0f / 40320.0f, 1.0f / 5040.0f, 1.0f / 720.0f, 1.0f / 120.0f,
                            1.0f / 24.0f, 1.0f / 6.0f, 0.5f, 1.0f};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float tr = er * ur - ei * ui;
            ei = er * ui + ei * ur;
            er = tr + c[k];
        }
    } else {
        // e^u - 1 = (expm1(ur) cos ui - 2 sin^2(ui/2)) + i e^ur sin ui
        float su, cu;
        sincosf(ui, &su, &cu);
        const float sh = sinf(0.5f * ui);
        const float nr = expm1f(ur) * cu - 2.0f * sh * sh, ni = expf(ur) * su;
        const float q = fdiv_fast(1.0f, ur * ur + ui * ui);
        er = (nr * ur + ni * ui) * q;
        ei = (ni * ur - nr * ui) * q;
    }
    const float cm = (0.5f / kFadPiF) * expf(-0.25f * mf * mf);
    H = fmaf(-cm, er * a + ei * pr, H);
    K = fmaf(cm, er * pr - ei * a, K);
    // residue part: 2 e^{-z^2} B(v), e^{-z^2} = e^{a^2 - x^2} (cos 2ax - i sin 2ax)
    const float x2 = xh * xh;
    const float lo = fmaf(xh, xh, -x2) + 2.0f * xh * xl;
    const float g = expf(fmaf(a, a, -x2)) * (1.0f - lo);
    float s2, c2;
    sincosf(2.0f * a * xh, &s2, &c2);
    const float gr = g * c2, gi = -g * s2;
    const float vr = -4.0f * kFadPiF * a, vi = 4.0f * kFadPiF * d;
    float br, bi;
    if (vr * vr + vi * vi < 1.0f) {
        // B(v) = 1/2 + v/12 - v^3/720 + v^5/30240 - v^7/1209600 + v^9/47900160
        const float wr = vr * vr - vi * vi, wi = 2.0f * vr * vi;
        br = 1.0f / 47900160.0f;
        bi = 0.0f;
        const float c[4] = {-1.0f / 1209600.0f, 1.0f / 30240.0f, -1.0f / 720.0f, 1.0f / 12.0f};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float tr = br * wr - bi * wi;
            bi = br * wi + bi * wr;
            br = tr + c[k];
        }
        const float tr = br * vr - bi * vi;
        bi = br * vi + bi * vr;
        br = tr + 0.5f;
    } else {
        // 1 - e^{-v} = (2 sin^2(2 pi d) - expm1(4 pi a) cos(4 pi d)) + i e^{4 pi a} sin(4 pi d)
        float s4, c4;
        sincospi_f(4.0f * d, &s4, &c4);
        const float sd = sinpi_f(2.0f * d);
        const float ea = 4.0f * kFadPiF * a;
        const float Dr = 2.0f * sd * sd - expm1f(ea) * c4, Di = expf(ea) * s4;
        const float qd = fdiv_fast(1.0f, Dr * Dr + Di * Di), qv = fdiv_fast(1.0f, vr * vr + vi * vi);
        br = Dr * qd - vr * qv;
        bi = vi * qv - Di * qd;
    }
    H = fmaf(2.0f, gr * br - gi * bi, H);
    K = fmaf(2.0f, gr * bi + gi * br, K);
}

RG_HD float faddeeva_h(float a, float xh, float xl) {
    float H, K;
    faddeeva_hk(a, xh, xl, H, K);
    return H;
}

// H with its partial derivatives from w' = -2 z w + 2i/sqrt(pi):
// dH/dx = Re w' = 2 (a K - x H), dH/da = -Im w' = 2 (x K + a H) - 2/sqrt(pi).
// Beyond |x| = 8 the identity for dH/da cancels, so w' is taken from the
// derivative of the asymptotic series, w' = -(i/sqrt(pi)) v sum_k (2k+1) c_k v^k.
RG_HD void faddeeva_derivs(float a, float x, float& H, float& Ha, float& Hx) {
    float K;
    faddeeva_hk(a, x, 0.0f, H, K);
    if (fabsf(x) <= 8.0f) {
        Hx = 2.0f * (a * K - x * H);
        Ha = 2.0f * (x * K + a * H) - 2.0f / kFadSqrtPiF;
        return;
    }
    const float q = fdiv_fast(1.0f, fmaf(x, x, a * a));
    const float ur = x * q, ui = -a * q;
    const float vr = ur * ur - ui * ui, vi = 2.0f * ur * ui;
    float pr = 10395.0f / 32.0f, pi = 0.0f;
    const float c[5] = {945.0f / 16.0f, 105.0f / 8.0f, 15.0f / 4.0f, 1.5f, 1.0f};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float tr = pr * vr - pi * vi;
        pi = pr * vi + pi * vr;
        pr = tr + c[k];
    }
    const float tr = vr * pr - vi * pi, ti = vr * pi + vi * pr;
    Hx = ti * (1.0f / kFadSqrtPiF);
    Ha = tr * (1.0f / kFadSqrtPiF);
}

}  // namespace rg

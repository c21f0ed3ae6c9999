// Device building blocks of the resonant-line Monte Carlo path on GB300
// (sm_103a): counter-based random streams, the Hjerting-Voigt function, u_par
// sampling, phase functions, and the FP64 octree walk.  Each function cites
// the passage of Michel-Dansac et al. (2020) it implements.
//
// Precision policy (GB300 runs FP64 at ~1/70 of the FP32 rate): packet
// position, distances to faces and borders, frequency and tau accumulation are
// FP64; Voigt, velocity sampling, phase functions and peeling weights are FP32.
// FP64 division, square root and logarithm stay off the per-scattering path.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>
#include "internal.h"
#include "bits.cuh"
#include "faddeeva.cuh"

namespace rg {

// CODATA 2018, cgs (kernel-side copy)
constexpr double kC = 2.99792458e10;
// H(a,x) evaluation the kernels of this translation unit are built for:
// Tasitsiomi's form (default) or the Faddeeva function (RG_FADDEEVA=1)
#ifndef RG_FADDEEVA
#define RG_FADDEEVA 0
#endif
constexpr bool kFaddeeva = RG_FADDEEVA != 0;

constexpr float kPiF = 3.14159265358979f;
constexpr float kSqrtPiF = 1.7724538509055159f;
constexpr float kTwoPiF = 6.2831853071795865f;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. 2011).  Key = run seed; counter = (draw block
// lo, hi, packet id lo, hi).  Draw word n of a packet is word n%4 of block n/4.
// ---------------------------------------------------------------------------
// one Philox4x32-10 round of counter (c0, c1, c2, c3) under key (k0, k1)
__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                             uint32_t k0, uint32_t k1) {
    // each 32x32 -> 64-bit product as one wide multiply
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
}

// one Philox4x32-10 block; kept out of line so that the draw sites of the
// transport loop share one copy of the ten rounds
static __device__ __noinline__ uint4 philox_block(uint32_t blk, uint32_t id0, uint32_t id1, uint32_t k0, uint32_t k1) {
    uint32_t c0 = blk, c1 = 0, c2 = id0, c3 = id1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        philox_round(c0, c1, c2, c3, k0, k1);
    }
    return make_uint4(c0, c1, c2, c3);
}

// Draw words of a packet's stream.  Each thread owns a ring of kRing words in
// dynamic shared memory (word i in row i % kRing of the thread's column, so
// the lanes of a warp always hit distinct banks).  top_up(), called where the
// warp is converged, computes the next blocks of every lane together (two
// blocks interleaved for instruction-level parallelism); word() computes a
// block by itself only when the ring runs dry (extra rejection trials).
// Dynamic shared memory of a kernel using Rng starts with kRing * blockDim.x
// words for the rings.
constexpr uint32_t kRing = 16;

struct Rng {
    uint32_t k0, k1, id0, id1;
    uint32_t n;       // next draw index
    uint32_t avail;   // words n .. avail - 1 are in the ring; avail % 4 == 0

    static __device__ __forceinline__ uint32_t& slot(uint32_t i) {
        extern __shared__ uint32_t s_dyn[];
        return s_dyn[(i & (kRing - 1u)) * blockDim.x + threadIdx.x];
    }
    __device__ __forceinline__ void put(uint32_t first, uint4 w) {
        slot(first) = w.x; slot(first + 1u) = w.y; slot(first + 2u) = w.z; slot(first + 3u) = w.w;
    }
    __device__ __forceinline__ uint32_t word() {
        if (n == avail) {
            put(avail, philox_block(avail >> 2, id0, id1, k0, k1));
            avail += 4u;
        }
        return slot(n++);
    }
    // fill the ring to kRing - 3 .. kRing words ahead; the round keys come
    // from the kernel parameters (the same for every lane), so each round's
    // key XOR reads them directly instead of stepping the key per lane
    __device__ __forceinline__ void top_up(const Params& P) {
        if (avail - n <= kRing - 8u) {
            const uint32_t blk = avail >> 2;
            uint32_t a0 = blk, a1 = 0u, a2 = id0, a3 = id1;
            uint32_t b0 = blk + 1u, b1 = 0u, b2 = id0, b3 = id1;
#pragma unroll
            for (int r = 0; r < 10; ++r) {
                philox_round(a0, a1, a2, a3, P.round_key[r][0], P.round_key[r][1]);
                philox_round(b0, b1, b2, b3, P.round_key[r][0], P.round_key[r][1]);
            }
            put(avail, make_uint4(a0, a1, a2, a3));
            put(avail + 4u, make_uint4(b0, b1, b2, b3));
            avail += 8u;
        }
        if (avail - n <= kRing - 4u) {
            put(avail, philox_block(avail >> 2, id0, id1, k0, k1));
            avail += 4u;
        }
    }
    // ((w >> 9) + 1/2) 2^-23: in (0, 1), exactly representable in FP32, and
    // so is 1 - u
    __device__ __forceinline__ float u23() {
        return __uint2float_rn(word() >> 9) * 0x1p-23f + 0x1p-24f;
    }
    // ((wa >> 6) 2^26 + (wb >> 6) + 1/2) 2^-52 from two consecutive words
    __device__ __forceinline__ double u52() {
        uint32_t wa = word(), wb = word();
        double m = __fma_rn((double)(wa >> 6), 67108864.0, (double)(wb >> 6));
        return __fma_rn(m, 0x1p-52, 0x1p-53);
    }
    // tau_event = -ln r (Sect. 3) for r = u52 of the next two words, in FP32:
    // r = (ma 2^26 + mb + 1/2) 2^-52; below 1/2 -log(r), above it
    // -log1p(-(1 - r)) with 1 - r formed exactly from the complemented
    // integers, so the relative error stays ~1e-7 over the whole range
    __device__ __forceinline__ float tau_event() {
        uint32_t ma = word() >> 6, mb = word() >> 6;
        const bool hi = ma >= (1u << 25);
        if (hi) { ma = (1u << 26) - 1u - ma; mb = (1u << 26) - 1u - mb; }
        float v = fmaf(__uint2float_rn(ma), 0x1p-26f, (__uint2float_rn(mb) + 0.5f) * 0x1p-52f);
        return hi ? -log1pf(-v) : -logf(v);
    }
    // refill the ring after the packet state was restored from memory
    __device__ __forceinline__ void resume() {
        avail = n & ~3u;
        if (n & 3u) {
            put(avail, philox_block(avail >> 2, id0, id1, k0, k1));
            avail += 4u;
        }
    }
    // stream of packet pid, next draw `start`
    __device__ void init(const Params& P, uint64_t pid, uint32_t start = 0) {
        k0 = P.key0; k1 = P.key1;
        id0 = (uint32_t)pid; id1 = (uint32_t)(pid >> 32);
        n = start;
        avail = start & ~3u;
        if (n & 3u) {
            put(avail, philox_block(avail >> 2, id0, id1, k0, k1));
            avail += 4u;
        }
    }
};

// ---------------------------------------------------------------------------
// Hjerting-Voigt function, Tasitsiomi (2006) eqs. 7-8 (Sect. 3.3.2).  x^2 is
// formed in FP64 and its rounding to FP32 is fed back into exp(-x^2) to first
// order, so H keeps ~1e-7 relative accuracy where exp(-x^2) dominates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float voigt_h(float a, double x) {
    double x2d = x * x;
    float x2 = (float)x2d;
    float lo = (float)(x2d - (double)x2);
    float e = expf(-x2) * (1.0f - lo);
    float z = __fdividef(x2 - 0.855f, x2 + 3.42f);
    float q = 0.0f;
    if (z > 0.0f) {
        q = z * (1.0f + __fdividef(21.0f, x2)) * __fdividef(a, kPiF * (x2 + 1.0f)) *
            (0.1117f + z * (4.421f + z * (-9.207f + 5.674f * z)));
    }
    return kSqrtPiF * q + e;
}

// Same function for x carried as an unevaluated FP32 pair x = xh + xl: x^2 is
// xh^2 plus its exact rounding error plus 2 xh xl, all in FP32.
__device__ __forceinline__ float voigt_h2(float a, float xh, float xl) {
    float x2 = xh * xh;
    float lo = fmaf(xh, xh, -x2) + 2.0f * xh * xl;
    float e = expf(-x2) * (1.0f - lo);
    float z = __fdividef(x2 - 0.855f, x2 + 3.42f);
    float q = 0.0f;
    if (z > 0.0f) {
        q = z * (1.0f + __fdividef(21.0f, x2)) * __fdividef(a, kPiF * (x2 + 1.0f)) *
            (0.1117f + z * (4.421f + z * (-9.207f + 5.674f * z)));
    }
    return kSqrtPiF * q + e;
}

// H with its partial derivatives in a and x (the derivative of this
// approximation, which is what the adjoint differentiates)
__device__ __forceinline__ void voigt_derivs(float a, float x, float& H, float& Ha, float& Hx) {
    float s = x * x;
    float e = expf(-s);
    float Q = 0.0f, dQ = 0.0f;
    float z = (s - 0.855f) / (s + 3.42f);
    if (z > 0.0f) {
        float w = s + 3.42f;
        float zp = 4.275f / (w * w);
        float Pz = 0.1117f + z * (4.421f + z * (-9.207f + 5.674f * z));
        float Pp = 4.421f + z * (-18.414f + 17.022f * z);
        float A1 = 1.0f + 21.0f / s;
        float inv = 1.0f / (kPiF * (s + 1.0f));
        Q = z * A1 * Pz * inv;
        dQ = (zp * A1 * Pz - z * (21.0f / (s * s)) * Pz + z * A1 * Pp * zp) * inv - Q / (s + 1.0f);
    }
    H = kSqrtPiF * a * Q + e;
    Ha = kSqrtPiF * Q;
    Hx = 2.0f * x * (kSqrtPiF * a * dQ - e);
}

// H by the option the kernels are built for (kFaddeeva), x as an FP32 pair
__device__ __forceinline__ float voigt_sel(float a, float xh, float xl) {
    if constexpr (kFaddeeva) return faddeeva_h(a, xh, xl);
    else return voigt_h2(a, xh, xl);
}
__device__ __forceinline__ float voigt_sel(float a, double x) {
    if constexpr (kFaddeeva) {
        const float xh = (float)x;
        return faddeeva_h(a, xh, (float)(x - (double)xh));
    } else {
        return voigt_h(a, x);
    }
}

// ---------------------------------------------------------------------------
// u_par (Sect. 3.3.3): rejection method of Zheng & Miralda-Escude (2002) with
// the fitted separation u0(x, log10 a), clamped at 0; |x| >= x_gauss: Gaussian
// N(1/|x|, 1/2).  Returns u_par for frequency x (scatterer's Doppler units).
// ---------------------------------------------------------------------------
// u0(x, zeta) of Sect. 3.3.3 is a degree-5 polynomial in x whose monomial
// form cancels heavily for x ~ 5-8 (terms of a few hundred summing to O(1)),
// while u_par moves one-for-one with u0.  Once per leaf and line the kernel
// forms the monomial coefficients in FP64 (zeta = log10 a) and re-expresses
// the same polynomial in Chebyshev polynomials of t = x/4 - 1 on [0, 8]; the
// per-draw evaluation is then an FP32 Clenshaw sum, accurate to ~6e-7.
struct U0Coef {
    float b[6];
};

__device__ __forceinline__ void u0_coeffs(double a, U0Coef& k) {
    double z = log10(a);
    double c0 = __fma_rn(z, __fma_rn(z, 0.351479, 2.014446), 2.648963);
    double c1 = __fma_rn(z, __fma_rn(z, -0.640003, -3.675859), -4.058673);
    double c2 = __fma_rn(z, __fma_rn(z, 0.370294, 2.117133), 3.017395);
    double c3 = __fma_rn(z, __fma_rn(z, -0.096312, -0.565886), -0.869789);
    double c4 = __fma_rn(z, __fma_rn(z, 0.011557, 0.070103), 0.110987);
    double c5 = __fma_rn(z, __fma_rn(z, -0.000519, -0.003240), -0.005200);
    // x^k = (4 (t + 1))^k in Chebyshev polynomials T_j(t): exact integer weights
    k.b[0] = (float)(c0 + 4.0 * c1 + 24.0 * c2 + 160.0 * c3 + 1120.0 * c4 + 8064.0 * c5);
    k.b[1] = (float)(4.0 * c1 + 32.0 * c2 + 240.0 * c3 + 1792.0 * c4 + 13440.0 * c5);
    k.b[2] = (float)(8.0 * c2 + 96.0 * c3 + 896.0 * c4 + 7680.0 * c5);
    k.b[3] = (float)(16.0 * c3 + 256.0 * c4 + 2880.0 * c5);
    k.b[4] = (float)(32.0 * c4 + 640.0 * c5);
    k.b[5] = (float)(64.0 * c5);
}

__device__ __forceinline__ float u0_eval(const U0Coef& k, float x) {
    float t = fmaf(x, 0.25f, -1.0f);
    float t2 = 2.0f * t;
    float b1 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int j = 5; j >= 1; --j) {
        float b0 = fmaf(t2, b1, k.b[j] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fmaxf(fmaf(t, b1, k.b[0] - b2), 0.0f);
}

// The two branches of the comparison function are sampled through their
// angular variable theta = atan((u - x)/a): branch 1 covers theta in
// (-pi/2, theta0], branch 2 (theta0, pi/2).  In FP32 theta itself cannot
// resolve the poles, so the code works with the distances to the poles,
// A = theta0 + pi/2 and B = pi/2 - theta0 (formed without cancellation), and
// u = x - a / tan(A r) or u = x + a / tan(B (1 - r)).
__device__ __forceinline__ float sample_upar(Rng& rng, float x, float a, const U0Coef& u0c, float x_gauss,
                                             uint32_t& trials, bool& err) {
    float sg = x < 0.0f ? -1.0f : 1.0f;
    float xa = fabsf(x);
    if (xa >= x_gauss) {
        float r1 = rng.u23(), r2 = rng.u23();
        trials += 1;
        return sg * (1.0f / xa + sqrtf(-logf(r1)) * cospif(2.0f * r2));
    }
    float u0 = u0_eval(u0c, xa);
    float t = __fdividef(u0 - xa, a);
    // the pole nearer to theta0 gets atan(1/|t|) (no cancellation), the other
    // pi minus it; one arctangent for both signs of t
    const float at = atanf(__fdividef(1.0f, fabsf(t)));
    const bool lo = t < 0.0f;
    const float A = lo ? at : kPiF - at;
    const float B = lo ? kPiF - at : at;
    float e0 = expf(-u0 * u0);
    float p = __fdividef(A, A + e0 * B);
    float u0sq = u0 * u0;
    for (uint32_t n = 0; n < (1u << 22); ++n) {
        float r1 = rng.u23(), r2 = rng.u23(), r3 = rng.u23();
        ++trials;
        const bool b1 = r1 <= p;
        float tn = tanf(b1 ? A * r2 : B * (1.0f - r2));
        const float q = __fdividef(a, tn);
        float u = b1 ? xa - q : xa + q;
        float lim = b1 ? 0.0f : u0sq;
        if (r3 <= expf(lim - u * u)) return sg * u;
    }
    err = true;
    return 0.0f;
}

// ---------------------------------------------------------------------------
// Phase functions (Sect. 3.3.1, Eqs. Pcore, Pwing, Pdust) and their inversion.
// HG inversion carries the square the printed formula omits.
// ---------------------------------------------------------------------------
enum { PH_ISO = 0, PH_CORE = 1, PH_WING = 2, PH_HG = 3 };

// mu and sin(theta) = sqrt(1 - mu^2), the latter formed from (1 - mu)(1 + mu)
// so that it stays accurate near forward / backward scattering
__device__ __forceinline__ float mu_sample(int kind, float r, float g, float& st) {
    if (kind == PH_CORE || kind == PH_WING) {
        // Inversion of the CDF r = C(mu) of Eqs. Pcore / Pwing.  With y the
        // distance of mu from the nearer end, y = 1 + mu for r < 1/2 and
        // y = 1 - mu otherwise, the CDF reads y (y^2 - 3y + c1) = c2 q with
        // q = min(r, 1 - r) (core: c1 = 14, c2 = 24; wing: c1 = 6, c2 = 8).
        // The left side h(y) rises monotonically on [0, 1] (h' >= c1 - 3) and
        // is concave there, so Newton's method from y = c2 q / c1 (below the
        // root) converges monotonically; three steps reach FP32 rounding for
        // both laws, and y carries relative accuracy near mu = -1 and +1.
        const bool core = kind == PH_CORE;
        const float c1 = core ? 14.0f : 6.0f, c2 = core ? 24.0f : 8.0f;
        const bool lo = r < 0.5f;
        const float q = lo ? r : 1.0f - r;   // exact: r has 23 significant bits
        const float cq = c2 * q;
        float y = q * (core ? 24.0f / 14.0f : 8.0f / 6.0f);   // c2 q / c1
#pragma unroll
        for (int it = 0; it < 3; ++it) {
            const float h = y * fmaf(y, y - 3.0f, c1) - cq;
            const float hp = fmaf(3.0f * y, y - 2.0f, c1);
            y = y - __fdividef(h, hp);
        }
        y = fminf(fmaxf(y, 0.0f), 1.0f);
        st = sqrtf(y * (2.0f - y));
        return lo ? y - 1.0f : 1.0f - y;
    }
    if (kind == PH_HG && g != 0.0f) {
        float t = (1.0f - g * g) / (1.0f - g + 2.0f * g * r);
        float inv2g = 0.5f / g;
        float omu = (t - (1.0f - g)) * (t + (1.0f - g)) * inv2g;   // 1 - mu
        float opu = ((1.0f + g) - t) * ((1.0f + g) + t) * inv2g;   // 1 + mu
        omu = fminf(2.0f, fmaxf(0.0f, omu));
        opu = fminf(2.0f, fmaxf(0.0f, opu));
        st = sqrtf(omu * opu);
        return fminf(1.0f, fmaxf(-1.0f, 1.0f - omu));
    }
    st = 2.0f * sqrtf(r * (1.0f - r));
    return 2.0f * r - 1.0f;
}

// phase function per unit mu (integrates to one over [-1, 1])
__device__ __forceinline__ float phase_p(int kind, float mu, float g) {
    if (kind == PH_CORE) return 0.4583333333f + 0.125f * mu * mu;
    if (kind == PH_WING) return 0.375f * (1.0f + mu * mu);
    if (kind == PH_HG) {
        float d = 1.0f + g * g - 2.0f * g * mu;
        return 0.5f * (1.0f - g * g) * rsqrtf(d * d * d);
    }
    return 0.5f;
}

// orthonormal basis (b1, b2) perpendicular to unit n: Duff et al. (2017)
__device__ __forceinline__ void onb(float nx, float ny, float nz, float3& b1, float3& b2) {
    float sg = copysignf(1.0f, nz);
    float a = __fdividef(-1.0f, sg + nz);
    float b = nx * ny * a;
    b1 = make_float3(1.0f + sg * nx * nx * a, sg * b, -sg * nx);
    b2 = make_float3(b, sg + ny * ny * a, -ny);
}

// ---------------------------------------------------------------------------
// Octree walk (Sect. 4.3).  Cells entered by a packet at p moving along k are
// the ones containing p + eps k.  Integer coordinates are kept at the finest
// level L of the tree: I = floor(p 2^L) for k >= 0, ceil(p 2^L) - 1 for k < 0.
// ---------------------------------------------------------------------------
struct Where {
    int leaf, oct, level;
    int i, j, k;   // integer coordinates of the leaf at its level
};

// integer coordinate at level L of the cell holding p + eps k (bits.cuh)
__device__ __forceinline__ int dir_coord(double p, double k, int L) { return cell_coord(p, is_neg(k), L); }

// slab domains are periodic in x and y (Sect. 4): bring p + eps k into the box
__device__ __forceinline__ void wrap_periodic(const Geo& G, double p[3], const double k[3]) {
    if (G.dom_kind != 1) return;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        int c = dir_coord(p[ax], k[ax], 1);
        if (c >= 2) p[ax] = p[ax] - 1.0;
        else if (c < 0) p[ax] = p[ax] + 1.0;
    }
}

// descend from the son value `code` of a cell at level m in oct `oct`
__device__ __forceinline__ void descend(const Geo& G, int code, int m, int oct,
                                        int tx, int ty, int tz, Where& w, uint32_t& loads) {
    const int L = G.max_level;
    while (code > 0) {
        oct = code;
        ++m;
        int s = L - m;
        int child = ((tx >> s) & 1) | (((ty >> s) & 1) << 1) | (((tz >> s) & 1) << 2);
        code = __ldg(G.son + 8 * oct + child);
        ++loads;
    }
    int s = L - m;
    w.leaf = -code - 1;
    w.oct = oct;
    w.level = m;
    w.i = tx >> s;
    w.j = ty >> s;
    w.k = tz >> s;
}

// where-is-point: the dense top grid at level S gives the deepest cell at level
// <= S holding the target; descend from there.  False if outside the box.
__device__ __forceinline__ bool locate(const Geo& G, int tx, int ty, int tz, Where& w,
                                       uint32_t& loads) {
    const int L = G.max_level;
    const int n = 1 << L;
    if ((unsigned)tx >= (unsigned)n || (unsigned)ty >= (unsigned)n || (unsigned)tz >= (unsigned)n)
        return false;
    const int S = G.top_level;
    const int s = L - S;
    long long idx = (((long long)(tz >> s) << S) + (ty >> s)) << S;
    idx += (tx >> s);
    int4 e = __ldg(G.top + idx);
    ++loads;
    descend(G, e.x, e.y, e.z, tx, ty, tz, w, loads);
    return true;
}

__device__ __forceinline__ bool locate_point(const Geo& G, const double p[3], const double k[3],
                                             Where& w, uint32_t& loads) {
    const int L = G.max_level;
    return locate(G, dir_coord(p[0], k[0], L), dir_coord(p[1], k[1], L), dir_coord(p[2], k[2], L), w, loads);
}

// Neighbour search after crossing a face (Sect. 4.3): the target is first
// looked for inside the father cell of the current leaf (its own oct), then in
// the father's neighbour across the face, then from the top grid.
__device__ __forceinline__ bool next_leaf(const Geo& G, const double p[3], const double k[3],
                                          int axis, Where& w, uint32_t& son_loads,
                                          uint32_t& nbor_loads) {
    const int L = G.max_level;
    int t[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) t[ax] = dir_coord(p[ax], k[ax], L);
    const int n = 1 << L;
    if ((unsigned)t[0] >= (unsigned)n || (unsigned)t[1] >= (unsigned)n || (unsigned)t[2] >= (unsigned)n)
        return false;
    const int l = w.level;
    const int sh = L - l;
    int fi = w.i >> 1, fj = w.j >> 1, fk = w.k >> 1;
    // the cell to descend from: the father's child, else the father's
    // neighbour across the face, else the top-grid cell; one descent for all
    int code = 0, m = 0, oct = 0;
    bool got = false;
    if ((t[0] >> (sh + 1)) == fi && (t[1] >> (sh + 1)) == fj && (t[2] >> (sh + 1)) == fk) {
        int child = ((t[0] >> sh) & 1) | (((t[1] >> sh) & 1) << 1) | (((t[2] >> sh) & 1) << 2);
        code = __ldg(G.son + 8 * w.oct + child);
        m = l;
        oct = w.oct;
        got = true;
    } else if (l >= 2) {
        const bool up = is_pos(axis == 0 ? k[0] : (axis == 1 ? k[1] : k[2]));
        int face = 2 * axis + (up ? 1 : 0);
        int4 a = __ldg(G.nbr + 2 * w.oct);
        int4 b = __ldg(G.nbr + 2 * w.oct + 1);
        ++nbor_loads;
        int nc = face == 0 ? a.x : face == 1 ? a.y : face == 2 ? a.z : face == 3 ? a.w : face == 4 ? b.x : b.y;
        int nl = (b.w >> (5 * face)) & 31;
        if (nc >= 0 && nl >= 1) {
            // coordinates of the neighbour cell at its level nl (<= l - 1)
            int f[3] = {fi, fj, fk};
            int nf = 1 << (l - 1);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax)
                if (ax == axis) f[ax] = (f[ax] + (up ? 1 : -1) + nf) & (nf - 1);
            int d = (l - 1) - nl;
            int s2 = L - nl;
            if ((t[0] >> s2) == (f[0] >> d) && (t[1] >> s2) == (f[1] >> d) && (t[2] >> s2) == (f[2] >> d)) {
                code = __ldg(G.son + nc);
                m = nl;
                oct = nc >> 3;
                got = true;
            }
        }
    }
    if (!got) {
        const int S = G.top_level;
        const int s = L - S;
        long long idx = (((long long)(t[2] >> s) << S) + (t[1] >> s)) << S;
        idx += (t[0] >> s);
        int4 e = __ldg(G.top + idx);
        code = e.x;
        m = e.y;
        oct = e.z;
    }
    ++son_loads;
    descend(G, code, m, oct, t[0], t[1], t[2], w, son_loads);
    return true;
}

// distance along k from p to the exit face of leaf w (FP64, exactly the
// oracle's (face - p) * (1/k)); axis = crossed axis, ties to the lowest axis.
// Face coordinates, the choice of the minimum and the clamp at zero run on
// the integer pipes (bits.cuh).
__device__ __forceinline__ double face_distance(const double p[3], const double k[3],
                                                const double inv[3], const Where& w, int& axis) {
    const int c[3] = {w.i, w.j, w.k};
    int64_t best = INT64_MAX;
    int ba = -1;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (is_zero(k[ax])) continue;
        double face = dyadic((uint32_t)(is_pos(k[ax]) ? c[ax] + 1 : c[ax]), w.level);
        int64_t t = order_key(__dmul_rn(__dsub_rn(face, p[ax]), inv[ax]));
        if (t < best) { best = t; ba = ax; }
    }
    axis = ba;
    if (ba < 0) return __longlong_as_double(0x7ff0000000000000LL);   // +inf (k = 0)
    return best < 0 ? 0.0 : bitsd(best);
}

// distance along k from p to the domain border (FP64, same operation order as
// the oracle)
__device__ __forceinline__ double border_distance(const Geo& G, const double p[3],
                                                  const double k[3], const double inv[3]) {
    if (G.dom_kind == 0 || G.dom_kind == 3) {
        double d0 = __dsub_rn(p[0], G.dom_c[0]);
        double d1 = __dsub_rn(p[1], G.dom_c[1]);
        double d2 = __dsub_rn(p[2], G.dom_c[2]);
        double b = __dadd_rn(__dadd_rn(__dmul_rn(d0, k[0]), __dmul_rn(d1, k[1])), __dmul_rn(d2, k[2]));
        double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
        double cc = __dsub_rn(r2, __dmul_rn(G.dom_R, G.dom_R));
        double disc = __dsub_rn(__dmul_rn(b, b), cc);
        if (disc < 0.0) disc = 0.0;
        double sq = __dsqrt_rn(disc);
        double t = b > 0.0 ? __ddiv_rn(-cc, __dadd_rn(b, sq)) : __dsub_rn(sq, b);
        if (G.dom_kind == 3) {
            // shell: also the entry into the inner sphere, when the ray meets it
            double ci = __dsub_rn(r2, __dmul_rn(G.dom_Rin, G.dom_Rin));
            if (ci <= 0.0) return 0.0;   // inside the hole: outside the domain
            double di = __dsub_rn(__dmul_rn(b, b), ci);
            if (b < 0.0 && di >= 0.0) {
                double ti = __ddiv_rn(ci, __dadd_rn(-b, __dsqrt_rn(di)));
                if (ti < t) t = ti;
            }
        }
        return t < 0.0 ? 0.0 : t;
    }
    double best = __longlong_as_double(0x7ff0000000000000ULL);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (G.dom_kind == 1 && ax != 2) continue;
        if (k[ax] == 0.0) continue;
        double edge = k[ax] > 0.0 ? __dadd_rn(G.dom_c[ax], G.dom_R) : __dsub_rn(G.dom_c[ax], G.dom_R);
        double t = __dmul_rn(__dsub_rn(edge, p[ax]), inv[ax]);
        if (t < best) best = t;
    }
    return best < 0.0 ? 0.0 : best;
}

// smallest distance from p to any face of leaf w (box units, FP64), for the
// guaranteed-inside budget of the scattering loop
__device__ __forceinline__ double inner_distance(const double p[3], const Where& w) {
    const int c[3] = {w.i, w.j, w.k};
    int64_t best = order_key(dyadic(1u, w.level));
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        double lo = dyadic((uint32_t)c[ax], w.level), hi = dyadic((uint32_t)c[ax] + 1u, w.level);
        int64_t d1 = order_key(__dsub_rn(p[ax], lo)), d2 = order_key(__dsub_rn(hi, p[ax]));
        best = min(best, min(d1, d2));
    }
    return from_key(best);
}

// move to the exit face along `axis` and snap the crossing coordinate
__device__ __forceinline__ void move_to_face(double p[3], const double k[3], int axis, double t,
                                             const Where& w) {
    const int c[3] = {w.i, w.j, w.k};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (ax == axis) p[ax] = dyadic((uint32_t)(is_pos(k[ax]) ? c[ax] + 1 : c[ax]), w.level);
        else p[ax] = __fma_rn(t, k[ax], p[ax]);
    }
}

// ---------------------------------------------------------------------------
// Cell state cached while a packet stays in one leaf
// ---------------------------------------------------------------------------
template <int NL>
struct CellCache {
    float vx, vy, vz;
    float kap_d;                 // dust opacity (cm^-1)
    int flags;
    double invdnu[NL];           // 1 / Delta nu_D (1/Hz)
    double dnu0;                 // Delta nu_D of line 0 (Hz)
    float dnu0_f;
    double xa[NL], xb[NL];       // x_i = xa_i + xb_i x_0 (line i's Doppler units from line 0's)
    float a[NL], kap0[NL];       // Voigt a, n_X sigma_0 (cm^-1)
    float vth_c[NL];             // v_th / c
    float q0;                    // nu0_0 / Delta nu_D,0 = c / v_th,0
    float T;
    unsigned u0mask;             // lines whose u0 coefficients are cached for this leaf
};

template <int NL>
__device__ __forceinline__ void load_cell(const Params& P, const Geo& G, int leaf, CellCache<NL>& cc) {
    float4 r0 = __ldg(G.rec + 2 * leaf);
    float4 r1 = __ldg(G.rec + 2 * leaf + 1);
    cc.vx = r0.y; cc.vy = r0.z; cc.vz = r0.w;
    cc.T = r1.x;
    cc.kap_d = r1.y * P.dust_sigma;
    cc.flags = __float_as_int(r1.w);
    cc.u0mask = 0u;
    float T = fmaxf(r1.x, 1e-30f);
    float rs = rsqrtf(T);
    // one Newton step in FP64 on 1/sqrt(T): x enters exp(-x^2) and must carry
    // ~1e-10 relative accuracy
    double rd = (double)rs;
    double Td = (double)T;
    rd = rd * __fma_rn(-0.5 * Td, rd * rd, 1.5);
#pragma unroll
    for (int i = 0; i < NL; ++i) {
        const LineDev& L = P.line[i];
        float n = (L.dens == 1 ? r1.z : r0.x) * L.abund;
        cc.invdnu[i] = L.invdnu_pref * rd;
        cc.a[i] = L.a_pref * rs;
        cc.kap0[i] = n * L.sig_pref * rs;
        cc.vth_c[i] = L.vth_over_c_pref * T * rs;
    }
    cc.dnu0 = P.line[0].dnu_pref * (Td * rd);
    cc.dnu0_f = (float)cc.dnu0;
    cc.q0 = 1.0f / cc.vth_c[0];
#pragma unroll
    for (int i = 1; i < NL; ++i) {
        cc.xa[i] = P.line[i].nu0_gap * cc.invdnu[i];
        cc.xb[i] = cc.dnu0 * cc.invdnu[i];
    }
}

// gas-frame frequency from the line-0 Doppler offset x = xh + xl, and back
template <int NL>
__device__ __forceinline__ double nu_of_x(const Params& P, const CellCache<NL>& cc, float xh, float xl) {
    return __fma_rn((double)xh + (double)xl, cc.dnu0, P.line[0].nu0);
}
template <int NL>
__device__ __forceinline__ void x_of_nu(const Params& P, const CellCache<NL>& cc, double nu, float& xh, float& xl) {
    double x = (nu - P.line[0].nu0) * cc.invdnu[0];
    xh = (float)x;
    xl = (float)(x - (double)xh);
}

// total opacity (cm^-1) at the line-0 Doppler offset x = xh + xl; per-line
// opacities in kl[], each line's own Doppler offset (FP32) in xin[]
template <int NL>
__device__ __forceinline__ float opacity_x(const Params& P, const CellCache<NL>& cc, float xh, float xl,
                                           float kl[NL], float xin[NL]) {
    kl[0] = cc.kap0[0] * voigt_sel(cc.a[0], xh, xl);
    xin[0] = xh;
    float tot = cc.kap_d + kl[0];
#pragma unroll
    for (int i = 1; i < NL; ++i) {
        double x = __fma_rn((double)xh + (double)xl, cc.xb[i], cc.xa[i]);
        xin[i] = (float)x;
        kl[i] = cc.kap0[i] * voigt_sel(cc.a[i], x);
        tot += kl[i];
    }
    return tot;
}

// beta = k . v / c in FP64
template <int NL>
__device__ __forceinline__ double beta_of(const CellCache<NL>& cc, const double k[3]) {
    return __fma_rn(k[0], (double)cc.vx, __fma_rn(k[1], (double)cc.vy, k[2] * (double)cc.vz)) * (1.0 / kC);
}

// nu_ext = nu_gas (1 + beta) and its inverse nu_gas = nu_ext / (1 + beta)
// evaluated as a series in beta (|beta| < 1e-2; error < beta^5)
__device__ __forceinline__ double to_gas(double nu_ext, double b) {
    double s = __fma_rn(b, __fma_rn(b, __fma_rn(b, __fma_rn(-b, b, b), -b), b), -b);
    // s = -b + b^2 - b^3 + b^4 - b^5
    return __fma_rn(nu_ext, s, nu_ext);
}
__device__ __forceinline__ double to_ext(double nu_gas, double b) { return __fma_rn(nu_gas, b, nu_gas); }

// ---------------------------------------------------------------------------
// Opacity along a ray at fixed external frequency and direction (the peeling
// integral and its adjoint, Sect. 3.1 opacities in each leaf's frame), with no
// FP64 instruction per leaf: the gas-frame offset nu_gas - nu0_i and the
// Doppler offset x_i are formed in FP32 pairs (~1e-13 relative), so x keeps
// the accuracy of the FP64 expression to_gas(nu_ext, beta) - nu0 over 1/Delta nu.
// ---------------------------------------------------------------------------
template <int NL>
struct RayNu {
    f2 nu;         // nu_ext
    f2 d[NL];      // nu_ext - nu0_i
    f2 k[3];       // direction
};

template <int NL>
__device__ __forceinline__ void ray_nu(const Params& P, double nu_ext, const double k[3], RayNu<NL>& r) {
    r.nu = f2_of(nu_ext);
#pragma unroll
    for (int i = 0; i < NL; ++i) r.d[i] = f2_of(nu_ext - P.line[i].nu0);
#pragma unroll
    for (int j = 0; j < 3; ++j) r.k[j] = f2_of(k[j]);
}

// 1/sqrt(T) as a pair: r + r (1 - T r^2) / 2 with T r^2 formed exactly
__device__ __forceinline__ f2 rsqrt_pair(float T, float& rs) {
    rs = rsqrtf(T);
    float t = T * rs;
    float te = __fmaf_rn(T, rs, -t);   // T rs = t + te
    float e = __fmaf_rn(-t, rs, 1.0f) - te * rs;
    return fast_two_sum(rs, 0.5f * rs * e);
}

// kappa (cm^-1) of the leaf record (r0, r1) at the ray's frequency, per line
// in kl[] and each line's Doppler offset in xh[], xl[]; beta = k . v / c
// returned as a pair
template <int NL>
__device__ __forceinline__ float ray_opacity(const Params& P, const RayNu<NL>& R, float4 r0, float4 r1,
                                             float kl[NL], float xh[NL], float xl[NL], f2& beta) {
    constexpr double kInvC = 1.0 / kC;
    const f2 invc = {(float)kInvC, (float)(kInvC - (double)(float)kInvC)};
    f2 kv = f2_mul_f(R.k[0], r0.y);
    kv = f2_add(kv, f2_mul_f(R.k[1], r0.z));
    kv = f2_add(kv, f2_mul_f(R.k[2], r0.w));
    beta = f2_mul(kv, invc);
    // nu_gas = nu_ext (1 + s), s = -b + b^2 - b^3 + b^4 - b^5 (to_gas)
    const float bh = beta.h;
    const float tail = bh * bh * (1.0f - bh * (1.0f - bh * (1.0f - bh)));
    const f2 dn = f2_mul(R.nu, f2_add_f(f2_neg(beta), tail));
    float rs;
    const f2 rr = rsqrt_pair(fmaxf(r1.x, 1e-30f), rs);
    float tot = r1.y * P.dust_sigma;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
        const LineDev& L = P.line[i];
        const f2 x = f2_mul(f2_mul(f2_add(R.d[i], dn), f2{L.invdnu_h, L.invdnu_l}), rr);
        const float n = (L.dens == 1 ? r1.z : r0.x) * L.abund;
        xh[i] = x.h;
        xl[i] = x.l;
        kl[i] = n * L.sig_pref * rs * voigt_sel(L.a_pref * rs, x.h, x.l);
        tot += kl[i];
    }
    return tot;
}

}  // namespace rg

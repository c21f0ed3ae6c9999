// Kernels of the resonant-line Monte Carlo path (Michel-Dansac et al. 2020)
// for GB300 (sm_103a).
//
// k_propagate is a persistent kernel: every lane owns one photon packet and
// advances it one walk step (a cell crossing or an interaction, Sect. 3) per
// loop iteration; a lane whose packet has escaped, was absorbed or capped
// refills itself from a global work queue with one warp-aggregated atomic, so
// packets with 1 or 1e6 scatterings share the machine without tail effects
// (the role of the master-worker bundles of Sect. 4.4).
//
// The packet state lives in registers: every function on the per-step path is
// inlined and indexes its arrays with compile-time constants (the loops over
// lines and peeling directions are unrolled).  The peeling ray walk, which is
// long and called from several places, is a separate function that reads the
// problem description through a device-side copy of the parameters.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include "device.cuh"
#include "internal.h"

// This file is compiled twice: the kernels of each build evaluate H(a,x) by
// one method (device.cuh, kFaddeeva), live in their own inline namespace (so
// the two builds' kernels never share a symbol) and are launched through
// launchers whose names carry the method (internal.h).
#if RG_FADDEEVA
#define RG_KVAR voigt_faddeeva
#define RG_SFX(name) name##_fad
#else
#define RG_KVAR voigt_tasitsiomi
#define RG_SFX(name) name
#endif

namespace rg {
inline namespace RG_KVAR {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kInf = __builtin_huge_val();

// per-thread event counters of the transport kernel, kept in shared memory
// (they are touched rarely; registers are the scarce resource there): 15
// words per thread so that the lanes of a warp fall in distinct banks
struct Tallies {
    uint32_t cross, peel_rays, peel_cells, trials, leaf_loads, son_loads, nbor_loads;
    uint32_t scatt_line, scatt_dust;
    uint32_t pk, esc, abs, cap, err;
    uint32_t pad;
};
static_assert(sizeof(Tallies) == 15 * 4, "odd word stride");

template <int NL>
struct Packet {
    double p0, p1, p2;     // position (box units)
    double kd0, kd1, kd2;  // direction used by the FP64 geometry (the sampled FP32 one, or the exact input)
    double tau;            // optical depth left to the next interaction (formed from tauf when tau_fresh)
    double path;           // distance travelled (box units)
    double nu_enter;       // external-frame frequency when the packet entered its leaf
    long long idx, nscatt, nsteps;
    Where w;
    Rng rng;
    int mi;                // model of a batch run (0 otherwise)
    float kx, ky, kz;      // direction (unit vector, as sampled in FP32)
    float xh, xl;          // gas-frame Doppler offset of line 0 in this leaf, x = xh + xl
    float tauf;            // FP32 copy of tau
    float budget;          // path length guaranteed to stay inside the leaf
    int status, zero_run;
    bool tau_fresh, enter, fresh;
    bool halt;             // the peel record buffer passed its high-water mark: suspend
    CellCache<NL> cc;
};

// k_out = mu k + sin(theta) (cos(phi) e1 + sin(phi) e2), phi = 2 pi r_phi, for an
// orthonormal basis (e1, e2) of the plane perpendicular to k
__device__ __forceinline__ void dir_from_basis(float kx, float ky, float kz, const float3& e1, const float3& e2,
                                               float mu, float st, float r_phi, float& ox, float& oy, float& oz) {
    float sn, cs;
    sincospif(2.0f * r_phi, &sn, &cs);
    float x = mu * kx + st * (cs * e1.x + sn * e2.x);
    float y = mu * ky + st * (cs * e1.y + sn * e2.y);
    float z = mu * kz + st * (cs * e1.z + sn * e2.z);
    float nn = rsqrtf(x * x + y * y + z * z);
    ox = x * nn;
    oy = y * nn;
    oz = z * nn;
}

__device__ __forceinline__ void dir_from(float kx, float ky, float kz, float mu, float st, float r_phi,
                                         float& ox, float& oy, float& oz) {
    float3 e1, e2;
    onb(kx, ky, kz, e1, e2);
    dir_from_basis(kx, ky, kz, e1, e2, mu, st, r_phi, ox, oy, oz);
}

// ---------------------------------------------------------------------------
// Optical depth along a ray (the peeling integral, Sect. 3.1 opacities summed
// over the leaves of the walk of Sect. 4.3) from p in leaf w along k to the
// domain border at external frequency nu_ext.  Per leaf: the record (32 B),
// the FP32-pair opacity, the FP64 face distance, the integer neighbour
// search; tau is summed as an FP32 pair.
// ---------------------------------------------------------------------------
template <int NL>
struct Ray {
    double p[3], k[3], inv[3];
    Where w;
    RayNu<NL> R;
    f2 tau;
    int n, zero_run;
};

template <int NL>
__device__ __forceinline__ void ray_start(const Params& P, Ray<NL>& r, double p0, double p1, double p2, Where w,
                                          double k0, double k1, double k2, double nu_ext) {
    r.p[0] = p0; r.p[1] = p1; r.p[2] = p2;
    r.k[0] = k0; r.k[1] = k1; r.k[2] = k2;
#pragma unroll
    for (int j = 0; j < 3; ++j) r.inv[j] = is_zero(r.k[j]) ? 0.0 : __drcp_rn(r.k[j]);
    r.w = w;
    ray_nu<NL>(P, nu_ext, r.k, r.R);
    r.tau = f2{0.0f, 0.0f};
    r.n = 0;
    r.zero_run = 0;
}

// one leaf of the walk; true when the ray is done (border, box edge, tau
// beyond tstop, or a stuck walk)
template <int NL>
__device__ __forceinline__ bool ray_step(const Params& P, Ray<NL>& r, float tstop, int32_t* cells, double* lens,
                                         int cap, uint32_t& sl, uint32_t& nl) {
    const float4 r0 = __ldg(P.g.rec + 2 * r.w.leaf);
    const float4 r1 = __ldg(P.g.rec + 2 * r.w.leaf + 1);
    float kl[NL], xh[NL], xl[NL];
    f2 beta;
    const float kap = ray_opacity<NL>(P, r.R, r0, r1, kl, xh, xl, beta);
    int axis;
    const double tf = face_distance(r.p, r.k, r.inv, r.w, axis);
    bool border = false;
    double l = tf;
    if (__float_as_int(r1.w) & kFlagBorder) {
        const double tb = border_distance(P.g, r.p, r.k, r.inv);
        border = order_key(tb) <= order_key(tf);
        if (border) l = tb;
    }
    r.tau = f2_add_f(r.tau, kap * (float)l * P.g.box_cm_f);
    if (cells != nullptr && r.n < cap) {
        cells[r.n] = r.w.leaf;
        lens[r.n] = l;
    }
    ++r.n;
    if (border || r.tau.h > tstop) return true;
    r.zero_run = order_key(tf) > 0 ? 0 : r.zero_run + 1;
    if (r.zero_run > 64) return true;
    move_to_face(r.p, r.k, axis, tf, r.w);
    wrap_periodic(P.g, r.p, r.k);
    return !next_leaf(P.g, r.p, r.k, axis, r.w, sl, nl);
}

__device__ __forceinline__ float tau_stop_f(double tau_stop) {
    return tau_stop >= 3.0e38 ? __int_as_float(0x7f800000) : (float)tau_stop;
}

// adjoint contribution of one leaf crossed over length l: grad[leaf][j] +=
// scale L l d kappa / d theta_j (Sect. 3.1 opacities differentiated in n_HI,
// v, T and n_dust)
template <int NL>
__device__ __forceinline__ void grad_add(const Params& P, const Ray<NL>& r, const float4& r0, const float4& r1,
                                         const float xh[NL], const f2& beta, double l, float scale) {
    float dk[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, P.dust_sigma};
    const float Tm = fmaxf(r1.x, 1e-30f);
    const float rs = rsqrtf(Tm);
    // nu_gas = nu_ext / (1 + beta)
    const float opb = 1.0f + beta.h;
    const float nug = r.R.nu.h / opb;
    const float kf[3] = {r.R.k[0].h, r.R.k[1].h, r.R.k[2].h};
#pragma unroll
    for (int i = 0; i < NL; ++i) {
        const LineDev& L = P.line[i];
        const float a = L.a_pref * rs;
        const float x = xh[i];
        float H, Ha, Hx;
        if constexpr (kFaddeeva) faddeeva_derivs(a, x, H, Ha, Hx);
        else voigt_derivs(a, x, H, Ha, Hx);
        const float s0 = L.sig_pref * rs;
        const float nX = (L.dens == 1 ? r1.z : r0.x) * L.abund;
        if (L.dens != 1) dk[0] += L.abund * s0 * H;
        // x = (nu_ext / (1 + beta) - nu0) / dnu:  dx/dv_j = -(nu_gas / dnu) k_j / (c (1 + beta))
        const float dxdv = -(nug * L.invdnu_h * rs) / ((float)kC * opb);
        const float t = nX * s0 * Hx * dxdv;
        dk[1] += t * kf[0];
        dk[2] += t * kf[1];
        dk[3] += t * kf[2];
        // sigma0, a and x all scale as T^(-1/2)
        dk[4] += nX * s0 * (-0.5f / Tm) * (H + a * Ha + x * Hx);
    }
    const float f = scale * P.g.box_cm_f * (float)l;
    if (f != 0.0f) {
        // the leaf's six derivatives sit in one 32-byte sector: two vector atomics
        float4* g = reinterpret_cast<float4*>(P.adj_grad) + 2 * (long long)r.w.leaf;
        atomicAdd(g, make_float4(f * dk[0], f * dk[1], f * dk[2], f * dk[3]));
        atomicAdd(reinterpret_cast<float2*>(g + 1), make_float2(f * dk[4], f * dk[5]));
    }
}

// one leaf of a peeling ray's walk: its optical depth (grad false) or, on the
// adjoint's second walk, its gradient contribution (grad true).  Both walks
// share the leaf load, the opacity and the geometry, so the lanes of a warp
// in different walks stay together; true when the ray is done (border, box
// edge, tau beyond tstop on the first walk, or a stuck walk)
template <int NL>
__device__ __forceinline__ bool peel_step(const Params& P, Ray<NL>& r, bool grad, float scale, float tstop,
                                          uint32_t& sl, uint32_t& nl) {
    const float4 r0 = __ldg(P.g.rec + 2 * r.w.leaf);
    const float4 r1 = __ldg(P.g.rec + 2 * r.w.leaf + 1);
    float kl[NL], xh[NL], xl[NL];
    f2 beta;
    const float kap = ray_opacity<NL>(P, r.R, r0, r1, kl, xh, xl, beta);
    int axis;
    const double tf = face_distance(r.p, r.k, r.inv, r.w, axis);
    bool border = false;
    double l = tf;
    if (__float_as_int(r1.w) & kFlagBorder) {
        const double tb = border_distance(P.g, r.p, r.k, r.inv);
        border = order_key(tb) <= order_key(tf);
        if (border) l = tb;
    }
    if (grad) {
        grad_add<NL>(P, r, r0, r1, xh, beta, l, scale);
        if (border) return true;
    } else {
        r.tau = f2_add_f(r.tau, kap * (float)l * P.g.box_cm_f);
        ++r.n;
        if (border || r.tau.h > tstop) return true;
    }
    r.zero_run = order_key(tf) > 0 ? 0 : r.zero_run + 1;
    if (r.zero_run > 64) return true;
    move_to_face(r.p, r.k, axis, tf, r.w);
    wrap_periodic(P.g, r.p, r.k);
    return !next_leaf(P.g, r.p, r.k, axis, r.w, sl, nl);
}

// one peeling ray towards direction d (weight wt per sr, gas-frame frequency
// nu_o_gas in the event's leaf), appended to the record buffer for the peel
// kernel; one atomic per converged group of lanes.  A reservation at or past
// the high-water mark asks the packet's warp to suspend.
template <int NL>
__device__ __forceinline__ void peel_emit(const Params& P, Packet<NL>& s, int d, float wt, double nu_o_gas,
                                          Tallies& tl) {
    const double b = __fma_rn(P.dirs[d][0], (double)s.cc.vx,
                              __fma_rn(P.dirs[d][1], (double)s.cc.vy, P.dirs[d][2] * (double)s.cc.vz)) * (1.0 / kC);
    const double nu_ext = to_ext(nu_o_gas, b);
    const unsigned m = __activemask();
    const int lane = (int)(threadIdx.x & 31u), leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(P.peel_count, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    const unsigned long long slot = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
    if (base >= P.peel_hw) s.halt = true;
    ++tl.peel_rays;
    if (slot >= P.peel_cap) return;   // cannot happen: peel_hw leaves room for every resident thread
    PeelRec& r = P.peel_rec[slot];
    r.p[0] = s.p0; r.p[1] = s.p1; r.p[2] = s.p2;
    r.nu_ext = nu_ext;
    r.w[0] = s.w.leaf; r.w[1] = s.w.oct; r.w[2] = s.w.level; r.w[3] = s.w.i; r.w[4] = s.w.j; r.w[5] = s.w.k;
    r.wt = wt;
    r.d = d;
}

// ---------------------------------------------------------------------------
// interactions (Sect. 3.2)
// ---------------------------------------------------------------------------
template <int NL, bool PEEL>
__device__ __forceinline__ void scatter_dust(const Params& P, Packet<NL>& s, Tallies& tl) {
    float r_alb = s.rng.u23();
    if (r_alb > P.dust_albedo) {
        s.status = RASCAS_PK_ABSORBED_;
        return;
    }
    float r_mu = s.rng.u23(), r_phi = s.rng.u23();
    float st;
    float mu = mu_sample(PH_HG, r_mu, P.dust_g, st);
    if (PEEL) {
        double nu_gas = nu_of_x(P, s.cc, s.xh, s.xl);   // coherent in the gas frame
#pragma unroll
        for (int d = 0; d < kMaxDirs; ++d) {
            if (d < P.ndir) {
                float muo = s.kx * (float)P.dirs[d][0] + s.ky * (float)P.dirs[d][1] + s.kz * (float)P.dirs[d][2];
                float wt = phase_p(PH_HG, muo, P.dust_g) * (1.0f / kTwoPiF);
                peel_emit<NL>(P, s, d, wt, nu_gas, tl);
            }
        }
    }
    if (!P.keep_dir) {
        dir_from(s.kx, s.ky, s.kz, mu, st, r_phi, s.kx, s.ky, s.kz);
        s.kd0 = (double)s.kx; s.kd1 = (double)s.ky; s.kd2 = (double)s.kz;
    }
    ++tl.scatt_dust;
}

// x = xh + xl advanced by d, kept as a normalised FP32 pair (two-sum)
__device__ __forceinline__ void pair_add(float& xh, float& xl, float d) {
    float sum = xh + d;
    float bb = sum - xh;
    float err = (xh - (sum - bb)) + (d - bb);
    float lo = xl + err;
    float hi = sum + lo;
    xl = lo - (hi - sum);
    xh = hi;
}

// resonant or fluorescent scattering on line IL (Sects. 3.2.1, 3.2.3, 3.3)
template <int NL, bool PEEL, int IL>
__device__ __forceinline__ void scatter_line(const Params& P, const Geo& G, Packet<NL>& s, float x_in, Tallies& tl) {
    const LineDev& L = P.line[IL];
    int ch = 0;
    double chnu = L.nu0;
    if (L.nchan > 1) {
        float r = s.rng.u23();
        ch = L.nchan - 1;
#pragma unroll
        for (int c = kMaxChan - 2; c >= 0; --c)
            if (c < L.nchan - 1 && r < L.chan_cum[c]) ch = c;
#pragma unroll
        for (int c = 1; c < kMaxChan; ++c)
            if (c == ch) chnu = L.chan_nu[c];
    }
    // u0 coefficients of this line for this leaf: computed at the first
    // scattering in the leaf, then read from shared memory
    U0Coef u0c;
    {
        // after the draw rings of Rng
        extern __shared__ float s_u0[];
        float* col = s_u0 + (size_t)(kRing + IL * 6) * blockDim.x + threadIdx.x;
        if (!(s.cc.u0mask & (1u << IL))) {
            u0_coeffs(L.a_over_invdnu * s.cc.invdnu[IL], u0c);
#pragma unroll
            for (int c = 0; c < 6; ++c) col[c * blockDim.x] = u0c.b[c];
            s.cc.u0mask |= 1u << IL;
        } else {
#pragma unroll
            for (int c = 0; c < 6; ++c) u0c.b[c] = col[c * blockDim.x];
        }
    }
    bool err = false;
    uint32_t trials = 0;
    float upar = sample_upar(s.rng, x_in, s.cc.a[IL], u0c, P.x_gauss, trials, err);
    tl.trials += trials;
    if (err) {
        s.status = RASCAS_PK_ERROR_;
        return;
    }
    // u_perp pair (Sect. 3.2.1), polar form; core-skipping restricts the
    // Gaussian to |u_perp| >= x_crit for core photons (|x_in| < x_crit)
    float r1 = s.rng.u23(), r2 = s.rng.u23();
    float xc2 = 0.0f;
    if (P.core_skip_on) {
        float xc = P.core_skip;
        if (P.core_skip_f > 0.0f)   // tau_cell: line-centre optical depth across the leaf
            xc = P.core_skip_f * cbrtf(s.cc.a[IL] * (s.cc.kap0[IL] * ldexpf(G.box_cm_f, -s.w.level)));
        if (fabsf(x_in) < xc) xc2 = xc * xc;
    }
    float rho = sqrtf(xc2 - logf(r1));
    float sn, cs;
    sincospif(2.0f * r2, &sn, &cs);
    float up1 = rho * cs, up2 = rho * sn;
    const float kx = s.kx, ky = s.ky, kz = s.kz;
    float3 e1, e2;
    onb(kx, ky, kz, e1, e2);
    float vx = upar * kx + up1 * e1.x + up2 * e2.x;   // scatterer velocity / v_th
    float vy = upar * ky + up1 * e1.y + up2 * e2.y;
    float vz = upar * kz + up1 * e1.z + up2 * e2.z;
    int kind;
    if (ch > 0 || P.isotropic || L.phase != 0) kind = PH_ISO;
    else kind = fabsf(x_in - upar) < 0.2f ? PH_CORE : PH_WING;
    float r_mu = s.rng.u23(), r_phi = s.rng.u23();
    float st;
    float mu = mu_sample(kind, r_mu, 0.0f, st);
    float ox = kx, oy = ky, oz = kz;
    if (P.keep_dir) mu = 1.0f;
    else dir_from_basis(kx, ky, kz, e1, e2, mu, st, r_phi, ox, oy, oz);
    const float vthc = s.cc.vth_c[IL];
    // recoil term (1 - mu) h nu / (m c^2) of Eq. (nuout_nuin)
    const float recp = P.recoil ? L.recoil_pref * (P.line[0].nu0_f + s.xh * s.cc.dnu0_f) : 0.0f;
    if (PEEL) {
        double nu_in = nu_of_x(P, s.cc, s.xh, s.xl);
#pragma unroll
        for (int d = 0; d < kMaxDirs; ++d) {
            if (d < P.ndir) {
                float dx = (float)P.dirs[d][0], dy = (float)P.dirs[d][1], dz = (float)P.dirs[d][2];
                float muo = kx * dx + ky * dy + kz * dz;
                float uo = dx * vx + dy * vy + dz * vz;
                double nu_o;
                if (ch > 0) {
                    nu_o = __fma_rn(chnu, (double)(uo * vthc), chnu);
                } else {
                    float rec = (1.0f - muo) * recp;
                    float f = ((uo - upar) * vthc - rec) / (1.0f + rec);
                    nu_o = __fma_rn(nu_in, (double)f, nu_in);
                }
                float wt = phase_p(kind, muo, 0.0f) * (1.0f / kTwoPiF);
                peel_emit<NL>(P, s, d, wt, nu_o, tl);
            }
        }
    }
    float uout = ox * vx + oy * vy + oz * vz;
    if (ch > 0) {
        double nu = __fma_rn(chnu, (double)(uout * vthc), chnu);
        x_of_nu(P, s.cc, nu, s.xh, s.xl);
    } else {
        // nu_out = nu_in (1 + f)  <=>  x_out = x_in + (nu0/Delta nu + x_in) f
        float rec = (1.0f - mu) * recp;
        float f = __fdividef((uout - upar) * vthc - rec, 1.0f + rec);
        pair_add(s.xh, s.xl, (s.cc.q0 + s.xh) * f);
    }
    if (!P.keep_dir) {
        s.kx = ox; s.ky = oy; s.kz = oz;
        s.kd0 = (double)ox; s.kd1 = (double)oy; s.kd2 = (double)oz;
    }
    ++tl.scatt_line;
}

template <int NL>
__device__ __forceinline__ void trace_record(const Packet<NL>& s, const TraceOut& tr, double nu_ext) {
    int32_t c = tr.nev[s.idx];
    if (c >= tr.max_events) return;
    TraceEvent& e = tr.ev[(long long)s.idx * tr.max_events + c];
    e.p[0] = s.p0; e.p[1] = s.p1; e.p[2] = s.p2;
    e.k[0] = s.kd0; e.k[1] = s.kd1; e.k[2] = s.kd2;
    e.nu = nu_ext;
    e.leaf = s.w.leaf; e.level = s.w.level; e.ijk[0] = s.w.i; e.ijk[1] = s.w.j; e.ijk[2] = s.w.k;
    e.status = s.status;
    e.ndraw = s.rng.n;
    e.nscatt = s.nscatt;
    e.nsteps = s.nsteps;
    tr.nev[s.idx] = c + 1;
}

// external-frame frequency of the packet now
template <int NL>
__device__ __forceinline__ double nu_ext_now(const Params& P, const Packet<NL>& s) {
    if (s.w.leaf < 0 || s.enter) return s.nu_enter;
    const double k[3] = {s.kd0, s.kd1, s.kd2};
    return to_ext(nu_of_x(P, s.cc, s.xh, s.xl), beta_of(s.cc, k));
}

// packet start: read the initial condition, key its random stream, find its
// leaf, draw its first tau_event (Sect. 2: PPIC lists; Sect. 3)
template <int NL, bool TRACE>
__device__ __forceinline__ void begin_packet(const Params& P, const Geo& G, const PacketsIn& in, long long idx,
                                             Packet<NL>& s, Tallies& tl, const TraceOut& tr) {
    s.idx = idx;
    double p[3] = {in.pos[3 * idx], in.pos[3 * idx + 1], in.pos[3 * idx + 2]};
    const double k[3] = {in.dir[3 * idx], in.dir[3 * idx + 1], in.dir[3 * idx + 2]};
    s.kx = (float)k[0]; s.ky = (float)k[1]; s.kz = (float)k[2];
    s.kd0 = k[0]; s.kd1 = k[1]; s.kd2 = k[2];
    s.nu_enter = in.nu[idx];
    s.rng.init(P, in.id[idx]);
    s.nscatt = 0;
    s.nsteps = 0;
    s.path = 0.0;
    s.budget = 0.0f;
    s.zero_run = 0;
    s.status = RASCAS_PK_ACTIVE_;
    s.enter = true;
    s.fresh = true;
    s.halt = false;
    wrap_periodic(G, p, k);
    s.p0 = p[0]; s.p1 = p[1]; s.p2 = p[2];
    if (!locate_point(G, p, k, s.w, tl.son_loads)) {
        s.status = RASCAS_PK_ERROR_;
        s.enter = false;
        s.w.leaf = -1; s.w.oct = 0; s.w.level = 0; s.w.i = s.w.j = s.w.k = 0;
    }
    if (TRACE && tr.nev) trace_record<NL>(s, tr, s.nu_enter);
    if (s.status == RASCAS_PK_ACTIVE_) {
        s.tauf = s.rng.tau_event();
        s.tau_fresh = true;
    }
}

template <int NL>
__device__ __forceinline__ void finish_packet(const Params& P, const Geo& G, const Packet<NL>& s, const PacketsOut& out,
                                              Tallies& tl) {
    double nu_ext = nu_ext_now<NL>(P, s);
    long long i = s.idx;
    if (out.status) out.status[i] = s.status;
    if (out.nscatt) out.nscatt[i] = s.nscatt;
    if (out.nu) out.nu[i] = nu_ext;
    if (out.path) out.path[i] = s.path;
    if (out.pos) { out.pos[3 * i] = s.p0; out.pos[3 * i + 1] = s.p1; out.pos[3 * i + 2] = s.p2; }
    if (out.dir) { out.dir[3 * i] = s.kd0; out.dir[3 * i + 1] = s.kd1; out.dir[3 * i + 2] = s.kd2; }
    ++tl.pk;
    tl.esc += s.status == RASCAS_PK_ESCAPED_;
    tl.abs += s.status == RASCAS_PK_ABSORBED_;
    tl.cap += s.status == RASCAS_PK_CAPPED_;
    tl.err += s.status == RASCAS_PK_ERROR_;
    if (s.status == RASCAS_PK_ESCAPED_ && G.spec != nullptr) {
        double t = __ddiv_rn(__dsub_rn(nu_ext, G.nu_lo), G.nu_range);
        double fb = floor(__dmul_rn(t, (double)G.nbin));
        if (fb >= 0.0 && fb < (double)G.nbin) atomicAdd(G.spec + (int)fb, 1.0f);
    }
}

// one loop iteration for an active packet: enter a leaf if needed, then one
// walk step -- an interaction inside the leaf, a face crossing, or the
// escape through the domain border (Sect. 3, Sect. 4.3).  Each phase appears
// once, so the loop body stays small for the instruction cache.
template <int NL, bool PEEL, bool TRACE>
__device__ __forceinline__ void advance(const Params& P, const Geo& G, Packet<NL>& s, Tallies& tl,
                                        const TraceOut& tr) {
    bool evt = false;
    s.rng.top_up(P);   // the warp is converged here: draw blocks for all lanes at once
    if (s.enter) {
        load_cell<NL>(P, G, s.w.leaf, s.cc);
        ++tl.leaf_loads;
        const double k[3] = {s.kd0, s.kd1, s.kd2};
        double nu_gas = to_gas(s.nu_enter, beta_of(s.cc, k));
        x_of_nu(P, s.cc, nu_gas, s.xh, s.xl);
        s.budget = 0.0f;
        s.enter = false;
        if (PEEL && s.fresh) {
            // peeling of the isotropic emission (weight 1/4pi per sr)
#pragma unroll
            for (int d = 0; d < kMaxDirs; ++d)
                if (d < P.ndir)
                    peel_emit<NL>(P, s, d, 1.0f / (2.0f * kTwoPiF), nu_gas, tl);
        }
        s.fresh = false;
    }
    if (P.max_steps > 0 && s.nsteps >= P.max_steps) {
        s.status = RASCAS_PK_CAPPED_;
        evt = true;
    } else {
        ++s.nsteps;
        float kl[NL], xin[NL];
        const float kap = opacity_x<NL>(P, s.cc, s.xh, s.xl, kl, xin);
        const bool border_leaf = (s.cc.flags & kFlagBorder) != 0;
        bool inter = false, exact = false;
        float li_f = 0.0f;
        double li_d = 0.0;
        if (!border_leaf) {
            li_f = __fdividef(s.tauf, kap * G.box_cm_f);
            float dec = __fmaf_ru(li_f, 1.0f + 0x1p-20f, 4e-16f);
            if (dec < s.budget) {
                s.budget = __fsub_rd(s.budget, dec);
                inter = true;
            }
        }
        if (!inter) {
            // exact FP64 step: distances to the faces and the border
            if (s.tau_fresh) {
                s.tau = (double)s.tauf;
                s.tau_fresh = false;
            }
            const double k[3] = {s.kd0, s.kd1, s.kd2};
            // 1/k (the direction changes at almost every scattering, so it
            // is formed here rather than kept)
            const double inv[3] = {is_zero(k[0]) ? 0.0 : __drcp_rn(k[0]), is_zero(k[1]) ? 0.0 : __drcp_rn(k[1]),
                                   is_zero(k[2]) ? 0.0 : __drcp_rn(k[2])};
            double p[3] = {s.p0, s.p1, s.p2};
            int axis;
            double tf = face_distance(p, k, inv, s.w, axis);
            double tb = border_leaf ? border_distance(G, p, k, inv) : kInf;
            bool border = tb <= tf;
            double l = border ? tb : tf;
            double tau_cell = __dmul_rn(__dmul_rn((double)kap, l), G.box_cm);
            if (tau_cell >= s.tau) {
                li_d = s.tau / __dmul_rn((double)kap, G.box_cm);
                inter = true;
                exact = true;
            } else {
                s.tau = __dsub_rn(s.tau, tau_cell);
                s.tauf = (float)s.tau;
                s.path += l;
                if (border) {
                    s.p0 = __fma_rn(l, k[0], s.p0);
                    s.p1 = __fma_rn(l, k[1], s.p1);
                    s.p2 = __fma_rn(l, k[2], s.p2);
                    s.status = RASCAS_PK_ESCAPED_;
                    evt = true;
                } else {
                    ++tl.cross;
                    s.zero_run = tf > 0.0 ? 0 : s.zero_run + 1;
                    double nu_ext = to_ext(nu_of_x(P, s.cc, s.xh, s.xl), beta_of(s.cc, k));
                    move_to_face(p, k, axis, tf, s.w);
                    wrap_periodic(G, p, k);
                    s.p0 = p[0]; s.p1 = p[1]; s.p2 = p[2];
                    Where nw = s.w;
                    if (s.zero_run > 64) {
                        s.status = RASCAS_PK_ERROR_;   // stuck walk
                        evt = true;
                    } else if (!next_leaf(G, p, k, axis, nw, tl.son_loads, tl.nbor_loads)) {
                        s.status = RASCAS_PK_ESCAPED_;   // left the box
                        evt = true;
                    } else {
                        s.w = nw;
                        s.nu_enter = nu_ext;
                        s.enter = true;
                    }
                }
            }
        }
        if (inter) {
            if (exact) {
                s.p0 = __fma_rn(li_d, s.kd0, s.p0);
                s.p1 = __fma_rn(li_d, s.kd1, s.p1);
                s.p2 = __fma_rn(li_d, s.kd2, s.p2);
                s.path += li_d;
                const double p[3] = {s.p0, s.p1, s.p2};
                double D = inner_distance(p, s.w);
                s.budget = __fsub_rd(__double2float_rd(D * (1.0 - 0x1p-20)), 4e-16f);
            } else {
                const double l = (double)li_f;
                s.p0 = __fma_rn(l, s.kd0, s.p0);
                s.p1 = __fma_rn(l, s.kd1, s.p1);
                s.p2 = __fma_rn(l, s.kd2, s.p2);
                s.path += l;
            }
            // Sect. 3.2: dust with P = tau_d / tau, else line X with P = tau_X / tau
            float rk = s.rng.u23() * kap;
            if (rk < s.cc.kap_d) {
                scatter_dust<NL, PEEL>(P, s, tl);
            } else {
                int il = NL - 1;
#pragma unroll
                for (int i = NL - 2; i >= 0; --i) {
                    float ai = s.cc.kap_d;
#pragma unroll
                    for (int j = 0; j <= i; ++j) ai += kl[j];
                    if (rk < ai) il = i;
                }
                if (il == 0) scatter_line<NL, PEEL, 0>(P, G, s, xin[0], tl);
                if (NL > 1 && il == 1) scatter_line<NL, PEEL, (NL > 1 ? 1 : 0)>(P, G, s, xin[NL > 1 ? 1 : 0], tl);
                if (NL > 2 && il == 2) scatter_line<NL, PEEL, (NL > 2 ? 2 : 0)>(P, G, s, xin[NL > 2 ? 2 : 0], tl);
                if (NL > 3 && il == 3) scatter_line<NL, PEEL, (NL > 3 ? 3 : 0)>(P, G, s, xin[NL > 3 ? 3 : 0], tl);
            }
            if (s.status == RASCAS_PK_ACTIVE_) {
                ++s.nscatt;
                if (P.max_scatt > 0 && s.nscatt >= P.max_scatt) s.status = RASCAS_PK_CAPPED_;
            }
            evt = true;
            if (s.status == RASCAS_PK_ACTIVE_) {
                if (TRACE && tr.nev) trace_record<NL>(s, tr, nu_ext_now<NL>(P, s));
                evt = false;
                s.tauf = s.rng.tau_event();
                s.tau_fresh = true;
            }
        }
    }
    if (TRACE && evt && tr.nev) trace_record<NL>(s, tr, nu_ext_now<NL>(P, s));
}

// nanoseconds of the GPU's global timer
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded device work: true (for the whole warp) once this thread has run
// max_iter loop iterations, the launch has run time_limit_ns, or another warp
// has raised the abort flag; the first warp to stop raises it.  `iters` is
// the same in every lane of the warp (the loops are warp-synchronous).
__device__ __forceinline__ bool out_of_bounds(const Params& P, uint32_t& iters, unsigned long long t0) {
    ++iters;
    bool stop = P.max_iter != 0u && iters > P.max_iter;
    if ((iters & 255u) == 0u) {
        if (*(volatile unsigned int*)P.abort_flag != 0u) stop = true;
        if (P.time_limit_ns != 0ull && global_ns() - t0 > P.time_limit_ns) stop = true;
    }
    if (!__any_sync(kFull, stop)) return false;
    if ((threadIdx.x & 31u) == 0u) atomicExch(P.abort_flag, 1u);
    return true;
}

__device__ __forceinline__ void flush(const Params& P, unsigned long long v, int which) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(P.counters + which, v);
}

// model of packet idx in a batch: the last m with model_first[m] <= idx
__device__ __forceinline__ int model_of(const Params& P, long long idx) {
    int lo = 0, hi = P.nmodels;   // model_first[lo] <= idx < model_first[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(P.model_first + mid) <= idx) lo = mid;
        else hi = mid;
    }
    return lo;
}

// resident blocks of 128 threads per SM the transport kernel is compiled for
// (registers per thread <= 65536 / (128 x this)); 4 measured fastest (5 and 6
// need 96 and 80 registers and lose 2-12 %)
#ifndef RG_PROP_MINB
#define RG_PROP_MINB 4
#endif

template <int NL, bool PEEL, bool BATCH, bool TRACE>
__global__ void __launch_bounds__(128, RG_PROP_MINB)
k_propagate(const __grid_constant__ Params P, PacketsIn in, PacketsOut out, TraceOut tr) {
    Packet<NL> s;
    extern __shared__ uint32_t s_dyn[];
    Tallies& tl = reinterpret_cast<Tallies*>(s_dyn + (kRing + 6 * NL) * blockDim.x)[threadIdx.x];
    tl = Tallies{};
    const unsigned lane = threadIdx.x & 31u;
    bool have = false, drained = false;
    s.mi = 0;
    uint32_t iters = 0;
    const unsigned long long t0 = P.limits ? global_ns() : 0ull;
    // batch runs: a lane reserves P.refill consecutive packets per queue grab
    long long next = 0, end = 0;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (PEEL && P.save_flag[gt]) {
        // a packet suspended by the previous round of this launch shape
        s = static_cast<const Packet<NL>*>(P.save)[gt];
        s.rng.resume();
        s.cc.u0mask = 0u;
        s.halt = false;
        P.save_flag[gt] = 0;
        have = true;
    }
    for (;;) {
        if (P.limits && out_of_bounds(P, iters, t0)) {
            // a limit was reached: the packet in flight stays unfinished
            if (have && out.status) out.status[s.idx] = RASCAS_PK_ACTIVE_;
            break;
        }
        if (PEEL && __any_sync(kFull, have && s.halt)) {
            // the record buffer is nearly full: park this warp's packets for
            // the next round, after the peel kernel has drained the records
            if (have) {
                s.halt = false;
                static_cast<Packet<NL>*>(P.save)[gt] = s;
                P.save_flag[gt] = 1;
            }
            if (lane == 0) atomicAdd(P.suspended, 1u);
            break;
        }
        bool want = !have && !drained;
        if constexpr (BATCH) {
            if (want && next < end) {
                // the next packet of this lane's reservation
                const long long idx = next++;
                s.mi = model_of(P, idx);
                begin_packet<NL, TRACE>(P, P.models[s.mi], in, idx, s, tl, tr);
                have = true;
                want = false;
            }
        }
        unsigned m = __ballot_sync(kFull, want);
        if (m) {
            int leader = __ffs(m) - 1;
            const int grab = BATCH ? P.refill : 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(P.head, (unsigned long long)__popc(m) * grab);
            base = __shfl_sync(kFull, base, leader);
            if (want) {
                long long idx = in.first + (long long)base + (long long)__popc(m & ((1u << lane) - 1u)) * grab;
                if constexpr (BATCH) {
                    next = idx + 1;
                    end = min(idx + grab, in.n);
                }
                if (idx < in.n) {
                    if constexpr (BATCH) {
                        s.mi = model_of(P, idx);
                        begin_packet<NL, TRACE>(P, P.models[s.mi], in, idx, s, tl, tr);
                    } else {
                        begin_packet<NL, TRACE>(P, P.g, in, idx, s, tl, tr);
                    }
                    have = true;
                } else {
                    drained = true;
                }
            }
        }
        if (!__any_sync(kFull, have)) {
            if (__all_sync(kFull, drained)) break;
            continue;
        }
        if (have) {
            const Geo& G = BATCH ? P.models[s.mi] : P.g;
            if (s.status == RASCAS_PK_ACTIVE_) advance<NL, PEEL, TRACE>(P, G, s, tl, tr);
            if (s.status != RASCAS_PK_ACTIVE_) {
                finish_packet<NL>(P, G, s, out, tl);
                have = false;
            }
        }
    }
    flush(P, tl.pk, CNT_PACKETS);
    flush(P, tl.esc, CNT_ESCAPED);
    flush(P, tl.abs, CNT_ABSORBED);
    flush(P, tl.cap, CNT_CAPPED);
    flush(P, tl.err, CNT_ERRORS);
    flush(P, tl.scatt_line, CNT_SCATT_LINE);
    flush(P, tl.scatt_dust, CNT_SCATT_DUST);
    flush(P, tl.cross, CNT_CROSS);
    flush(P, tl.peel_rays, CNT_PEEL_RAYS);
    flush(P, tl.peel_cells, CNT_PEEL_CELLS);
    flush(P, tl.trials, CNT_UPAR_TRIALS);
    flush(P, tl.leaf_loads, CNT_LEAF_LOADS);
    flush(P, tl.son_loads, CNT_SON_LOADS);
    flush(P, tl.nbor_loads, CNT_NBOR_LOADS);
}

// ---------------------------------------------------------------------------
// ray optical depths (peeling integral without cut-off) and probes
// ---------------------------------------------------------------------------
// Set-up of each ray: periodic wrap, the leaf holding the start point, 1/k
// and the FP32-pair frequency constants (the FP64 work of a ray, done here
// with every lane busy rather than by single lanes inside the walk)
template <int NL>
__global__ void k_ray_prep(const Params* __restrict__ G, long long n, const double* pos, const double* dir,
                           const double* nu, RayInit* init) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Params& P = *G;
    double p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    const double k[3] = {dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]};
    uint32_t loads = 0;
    wrap_periodic(P.g, p, k);
    Where w;
    RayInit r;
    if (!locate_point(P.g, p, k, w, loads)) w.leaf = -1, w.oct = w.level = w.i = w.j = w.k = 0;
    RayNu<NL> R;
    ray_nu<NL>(P, nu ? nu[i] : 0.0, k, R);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        r.p[j] = p[j];
        r.k[j] = k[j];
        r.inv[j] = is_zero(k[j]) ? 0.0 : __drcp_rn(k[j]);
        r.kp[j][0] = R.k[j].h;
        r.kp[j][1] = R.k[j].l;
    }
    r.w[0] = w.leaf; r.w[1] = w.oct; r.w[2] = w.level; r.w[3] = w.i; r.w[4] = w.j; r.w[5] = w.k;
    r.nu[0] = R.nu.h;
    r.nu[1] = R.nu.l;
#pragma unroll
    for (int j = 0; j < kMaxLines; ++j) {
        r.d[j][0] = j < NL ? R.d[j < NL ? j : 0].h : 0.0f;
        r.d[j][1] = j < NL ? R.d[j < NL ? j : 0].l : 0.0f;
    }
    init[i] = r;
}

template <int NL>
__device__ __forceinline__ void ray_load(const RayInit* __restrict__ in, long long i, Ray<NL>& r) {
    const RayInit& q = in[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        r.p[j] = q.p[j];
        r.k[j] = q.k[j];
        r.inv[j] = q.inv[j];
        r.R.k[j] = f2{q.kp[j][0], q.kp[j][1]};
    }
    r.w.leaf = q.w[0]; r.w.oct = q.w[1]; r.w.level = q.w[2]; r.w.i = q.w[3]; r.w.j = q.w[4]; r.w.k = q.w[5];
    r.R.nu = f2{q.nu[0], q.nu[1]};
#pragma unroll
    for (int j = 0; j < NL; ++j) r.R.d[j] = f2{q.d[j][0], q.d[j][1]};
    r.tau = f2{0.0f, 0.0f};
    r.n = 0;
    r.zero_run = 0;
}

// Persistent walk: each lane walks one ray leaf by leaf and takes the next ray
// from the queue head as soon as its ray is done, so the lanes of a warp stay
// busy whatever the spread of ray lengths. Eight blocks per SM (64 registers,
// a few spilled values) hide more of the dependent leaf-record loads than the
// five that the unconstrained register count allows.
template <int NL>
__global__ void __launch_bounds__(128, 8) k_ray_tau(const Params* __restrict__ G, long long n,
                                                 const RayInit* __restrict__ init, double* tau, int32_t* cells,
                                                 double* lens, int cap, int32_t* ncell) {
    const Params& P = *G;
    const unsigned lane = threadIdx.x & 31u;
    Ray<NL> r;
    long long i = -1;
    bool active = false, drained = false;
    uint32_t sl = 0, nl = 0, steps = 0;
    const float tstop = __int_as_float(0x7f800000);
    for (;;) {
        const bool want = !active && !drained;
        const unsigned m = __ballot_sync(kFull, want);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(P.head, (unsigned long long)__popc(m));
            base = __shfl_sync(kFull, base, leader);
            if (want) {
                i = (long long)base + __popc(m & ((1u << lane) - 1u));
                if (i < n) {
                    ray_load<NL>(init, i, r);
                    if (r.w.leaf >= 0) {
                        steps = 0;
                        active = true;
                    } else {
                        tau[i] = 0.0;
                        if (ncell) ncell[i] = 0;
                    }
                } else {
                    drained = true;
                }
            }
        }
        if (!__any_sync(kFull, active)) {
            if (__all_sync(kFull, drained)) break;
            continue;
        }
        if (active) {
            bool done = ray_step<NL>(P, r, tstop, cells ? cells + i * cap : nullptr, lens ? lens + i * cap : nullptr,
                                     cap, sl, nl);
            if (++steps >= (1u << 26)) done = true;
            if (done) {
                tau[i] = f2_val(r.tau);
                if (ncell) ncell[i] = r.n;
                active = false;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Deferred peeling (Sect. 3.1 peeling; adjoint of the peeled optical depths):
// each lane walks one record's ray leaf by leaf and takes the next record as
// soon as its ray is done.  Forward: w exp(-tau) into the spectrum, image and
// cube bins of the record.  Adjoint (P.adj_grad set): the ray is walked a
// second time with the scale -G w exp(-tau), G the loss gradient at those bins.
// ---------------------------------------------------------------------------
// a peeling ray from its record i: start point and leaf from the PeelRec,
// frequency pairs from the PeelPrep of the prep pass, direction terms from
// the parameters
template <int NL>
__device__ __forceinline__ void ray_from_prep(const Params& P, unsigned long long i, Ray<NL>& r) {
    const PeelRec& q = P.peel_rec[i];
    const PeelPrep& pp = P.peel_prep[i];
    const int d = q.d;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        r.p[j] = q.p[j];
        r.k[j] = P.dirs[d][j];
        r.inv[j] = P.dir_inv[d][j];
        r.R.k[j] = f2{P.dir_kp[d][j][0], P.dir_kp[d][j][1]};
    }
    r.w.leaf = q.w[0]; r.w.oct = q.w[1]; r.w.level = q.w[2]; r.w.i = q.w[3]; r.w.j = q.w[4]; r.w.k = q.w[5];
    r.R.nu = f2{pp.nu[0], pp.nu[1]};
#pragma unroll
    for (int l = 0; l < NL; ++l) r.R.d[l] = f2{pp.d[l][0], pp.d[l][1]};
    r.tau = f2{0.0f, 0.0f};
    r.n = 0;
    r.zero_run = 0;
}

// spectrum channel (or -1) and image pixel (or -1) of a peeled contribution
__device__ __forceinline__ void peel_bins(const Params& P, const PeelRec& q, int& ch, long long& px) {
    const int nbin = P.g.nbin;
    // the plain definitions' operations, unfused (exact ties bin as in the oracle)
    const double t = __ddiv_rn(__dsub_rn(q.nu_ext, P.g.nu_lo), P.g.nu_range);
    const double fb = floor(__dmul_rn(t, (double)nbin));
    ch = (fb >= 0.0 && fb < (double)nbin) ? (int)fb : -1;
    px = -1;
    if (P.npix > 0) {
        const int d = q.d;
        const double r0 = __dsub_rn(q.p[0], P.img_c[0]), r1 = __dsub_rn(q.p[1], P.img_c[1]);
        const double r2 = __dsub_rn(q.p[2], P.img_c[2]);
        const double u = __dadd_rn(__dadd_rn(__dmul_rn(r0, P.eu[d][0]), __dmul_rn(r1, P.eu[d][1])),
                                   __dmul_rn(r2, P.eu[d][2]));
        const double v = __dadd_rn(__dadd_rn(__dmul_rn(r0, P.ev[d][0]), __dmul_rn(r1, P.ev[d][1])),
                                   __dmul_rn(r2, P.ev[d][2]));
        const double fu = floor(__dmul_rn(__dadd_rn(__ddiv_rn(u, P.fov), 0.5), (double)P.npix));
        const double fv = floor(__dmul_rn(__dadd_rn(__ddiv_rn(v, P.fov), 0.5), (double)P.npix));
        if (fu >= 0.0 && fu < (double)P.npix && fv >= 0.0 && fv < (double)P.npix)
            px = (long long)fv * P.npix + (long long)fu;
    }
}

// true when a ray's walk ends in its first leaf without a contribution: the
// first step of ray_step (same arithmetic) stops it with tau beyond tau_stop
template <int NL>
__device__ __forceinline__ bool first_leaf_dark(const Params& P, const Ray<NL>& r, float tstop) {
    const float4 r0 = __ldg(P.g.rec + 2 * r.w.leaf);
    const float4 r1 = __ldg(P.g.rec + 2 * r.w.leaf + 1);
    float kl[NL], xh[NL], xl[NL];
    f2 beta;
    const float kap = ray_opacity<NL>(P, r.R, r0, r1, kl, xh, xl, beta);
    int axis;
    const double tf = face_distance(r.p, r.k, r.inv, r.w, axis);
    bool border = false;
    double l = tf;
    if (__float_as_int(r1.w) & kFlagBorder) {
        const double tb = border_distance(P.g, r.p, r.k, r.inv);
        border = order_key(tb) <= order_key(tf);
        if (border) l = tb;
    }
    const f2 tau = f2_add_f(r.tau, kap * (float)l * P.g.box_cm_f);
    return (border || tau.h > tstop) && !(f2_val(tau) <= P.tau_stop);
}

// prep pass of a round: the per-ray FP64 work of the peeling records (the
// frequency pairs of the walk; the first leaf, and the detector bins of the
// rays that get past it), one record per thread with every lane busy, so
// that the walk kernel, where a lane starts or ends a ray alone, does none of
// it.  The rays that get past their first leaf are listed (one atomic per
// warp) for the walk kernel; the others, dark after one leaf, are counted
// here
template <int NL>
__global__ void __launch_bounds__(256) k_peel_prep(const Params* __restrict__ G) {
    const Params& P = *G;
    const unsigned long long cnt = *P.peel_count;
    const unsigned long long n = cnt < P.peel_cap ? cnt : P.peel_cap;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const float tstop = tau_stop_f(P.tau_stop);
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long dark_cells = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned am = __activemask();
        const PeelRec q = P.peel_rec[i];
        PeelPrep o;
        Ray<NL> r;
        r.R.nu = f2_of(q.nu_ext);
        o.nu[0] = r.R.nu.h;
        o.nu[1] = r.R.nu.l;
#pragma unroll
        for (int l = 0; l < kMaxLines; ++l) {
            const f2 dl = l < NL ? f2_of(q.nu_ext - P.line[l].nu0) : f2{0.0f, 0.0f};
            if (l < NL) r.R.d[l] = dl;
            o.d[l][0] = dl.h;
            o.d[l][1] = dl.l;
        }
        const int d = q.d;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            r.p[j] = q.p[j];
            r.k[j] = P.dirs[d][j];
            r.inv[j] = P.dir_inv[d][j];
            r.R.k[j] = f2{P.dir_kp[d][j][0], P.dir_kp[d][j][1]};
        }
        r.w.leaf = q.w[0]; r.w.oct = q.w[1]; r.w.level = q.w[2]; r.w.i = q.w[3]; r.w.j = q.w[4]; r.w.k = q.w[5];
        r.tau = f2{0.0f, 0.0f};
        const bool dark = first_leaf_dark<NL>(P, r, tstop);
        if (dark) {
            ++dark_cells;
        } else {
            int ch = -1;
            long long px = -1;
            peel_bins(P, q, ch, px);
            o.ch = ch;
            o.dir = d;
            o.wt = q.wt;
            o.dark = 0;
            o.px = px;
            P.peel_prep[i] = o;
        }
        const unsigned m = __ballot_sync(am, !dark);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(P.peel_nlive, (unsigned long long)__popc(m));
            base = __shfl_sync(am, base, leader);
            if (!dark) P.peel_live[base + __popc(m & ((1u << lane) - 1u))] = i;
        }
    }
    flush(P, dark_cells, CNT_PEEL_CELLS);
    flush(P, dark_cells, CNT_LEAF_LOADS);
}

template <int NL, bool ADJ>
__global__ void __launch_bounds__(128, ADJ ? 3 : 4) k_peel(const Params* __restrict__ G) {
    const Params& P = *G;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long n = *P.peel_nlive;   // the rays the prep pass listed
    const float tstop = tau_stop_f(P.tau_stop);
    // ADJ: the adjoint's launch (P.adj_grad set): each contributing ray is
    // walked a second time for its gradient
    const bool adj = ADJ;
    const long long npix2 = (long long)P.npix * P.npix;
    Ray<NL> r;
    unsigned long long i = 0;
    bool active = false, drained = false;
    int phase = 0;           // 0: optical depth, 1: adjoint walk
    float scale = 0.0f;
    uint32_t sl = 0, nl = 0, steps = 0, cells = 0;
    uint32_t iters = 0;
    const unsigned long long t0 = P.limits ? global_ns() : 0ull;
    for (;;) {
        if (P.limits && out_of_bounds(P, iters, t0)) break;
        const bool want = !active && !drained;
        const unsigned m = __ballot_sync(kFull, want);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(P.peel_head, (unsigned long long)__popc(m));
            base = __shfl_sync(kFull, base, leader);
            if (want) {
                const unsigned long long j = base + __popc(m & ((1u << lane) - 1u));
                if (j < n) {
                    i = P.peel_live[j];
                    ray_from_prep<NL>(P, i, r);
                    phase = 0;
                    steps = 0;
                    active = true;
                } else {
                    drained = true;
                }
            }
        }
        if (!__any_sync(kFull, active)) {
            if (__all_sync(kFull, drained)) break;
            continue;
        }
        if (active) {
            bool done;
            if constexpr (ADJ) done = peel_step<NL>(P, r, phase != 0, scale, tstop, sl, nl);
            else done = ray_step<NL>(P, r, tstop, nullptr, nullptr, 0, sl, nl);
            if (++steps >= (1u << 26)) done = true;
            if (done && phase == 0) {
                cells += r.n;
                active = false;
                const double tau = f2_val(r.tau);
                if (tau <= P.tau_stop) {
                    const PeelPrep& pp = P.peel_prep[i];
                    const float f = pp.wt * expf(-(float)tau);
                    const int ch = pp.ch;
                    const long long px = pp.px;
                    const int nbin = P.g.nbin, d = pp.dir;
                    if (adj) {
                        float Gs = 0.0f;
                        if (ch >= 0 && P.adj_g_spec) Gs += __ldg(P.adj_g_spec + d * nbin + ch);
                        if (px >= 0 && P.adj_g_img) Gs += __ldg(P.adj_g_img + d * npix2 + px);
                        if (px >= 0 && ch >= 0 && P.cube && P.adj_g_cube)
                            Gs += __ldg(P.adj_g_cube + (d * npix2 + px) * nbin + ch);
                        if (Gs != 0.0f && f != 0.0f) {
                            ray_from_prep<NL>(P, i, r);
                            scale = -Gs * f;
                            phase = 1;
                            steps = 0;
                            active = true;
                        }
                    } else {
                        if (ch >= 0) atomicAdd(P.pspec + d * nbin + ch, f);
                        if (px >= 0) {
                            atomicAdd(P.pimg + d * npix2 + px, f);
                            if (ch >= 0 && P.cube) atomicAdd(P.pcube + (d * npix2 + px) * nbin + ch, f);
                        }
                    }
                }
            } else if (done) {
                active = false;
            }
        }
    }
    flush(P, cells, CNT_PEEL_CELLS);
    flush(P, cells, CNT_LEAF_LOADS);
    flush(P, sl, CNT_SON_LOADS);
    flush(P, nl, CNT_NBOR_LOADS);
}

#if !RG_FADDEEVA
// ---------------------------------------------------------------------------
// Column densities along rays (the ray-tracing use of Sects. 5 and 6: optical
// depths of ionising photons and sight-line columns): the walk of ray_step
// with n_HI, n_dust and n_metal times the path length summed per leaf as FP32
// pairs; no line profile, so the walk touches 12 of the record's 32 bytes.
// ---------------------------------------------------------------------------
struct ColRay {
    double p[3], k[3], inv[3];
    Where w;
    f2 nh, nd, nm;
    int n, zero_run;
};

__device__ __forceinline__ bool col_step(const Params& P, ColRay& r, uint32_t& sl, uint32_t& nl) {
    const float4 r0 = __ldg(P.g.rec + 2 * r.w.leaf);
    const float4 r1 = __ldg(P.g.rec + 2 * r.w.leaf + 1);
    int axis;
    const double tf = face_distance(r.p, r.k, r.inv, r.w, axis);
    bool border = false;
    double l = tf;
    if (__float_as_int(r1.w) & kFlagBorder) {
        const double tb = border_distance(P.g, r.p, r.k, r.inv);
        border = order_key(tb) <= order_key(tf);
        if (border) l = tb;
    }
    const float lc = (float)l * P.g.box_cm_f;
    r.nh = f2_add_f(r.nh, r0.x * lc);
    r.nd = f2_add_f(r.nd, r1.y * lc);
    r.nm = f2_add_f(r.nm, r1.z * lc);
    ++r.n;
    if (border) return true;
    r.zero_run = order_key(tf) > 0 ? 0 : r.zero_run + 1;
    if (r.zero_run > 64) return true;
    move_to_face(r.p, r.k, axis, tf, r.w);
    wrap_periodic(P.g, r.p, r.k);
    return !next_leaf(P.g, r.p, r.k, axis, r.w, sl, nl);
}

// persistent walk over the rays set up by k_ray_prep; the queue head P.head
// must be zero on entry
__global__ void __launch_bounds__(128, 8) k_ray_columns(const Params* __restrict__ G, long long n,
                                                     const RayInit* __restrict__ init, double* cols, double* tau,
                                                     double sig_hi, double sig_d, int32_t* ncell) {
    const Params& P = *G;
    const unsigned lane = threadIdx.x & 31u;
    ColRay r;
    long long i = -1;
    bool active = false, drained = false;
    uint32_t sl = 0, nl = 0, steps = 0;
    for (;;) {
        const bool want = !active && !drained;
        const unsigned m = __ballot_sync(kFull, want);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(P.head, (unsigned long long)__popc(m));
            base = __shfl_sync(kFull, base, leader);
            if (want) {
                i = (long long)base + __popc(m & ((1u << lane) - 1u));
                if (i < n) {
                    const RayInit& q = init[i];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        r.p[j] = q.p[j];
                        r.k[j] = q.k[j];
                        r.inv[j] = q.inv[j];
                    }
                    r.w.leaf = q.w[0]; r.w.oct = q.w[1]; r.w.level = q.w[2];
                    r.w.i = q.w[3]; r.w.j = q.w[4]; r.w.k = q.w[5];
                    r.nh = r.nd = r.nm = f2{0.0f, 0.0f};
                    r.n = 0;
                    r.zero_run = 0;
                    if (r.w.leaf >= 0) {
                        steps = 0;
                        active = true;
                    } else {
                        cols[3 * i] = cols[3 * i + 1] = cols[3 * i + 2] = 0.0;
                        if (tau) tau[i] = 0.0;
                        if (ncell) ncell[i] = 0;
                    }
                } else {
                    drained = true;
                }
            }
        }
        if (!__any_sync(kFull, active)) {
            if (__all_sync(kFull, drained)) break;
            continue;
        }
        if (active) {
            bool done = col_step(P, r, sl, nl);
            if (++steps >= (1u << 26)) done = true;
            if (done) {
                const double nh = f2_val(r.nh), nd = f2_val(r.nd);
                cols[3 * i] = nh;
                cols[3 * i + 1] = nd;
                cols[3 * i + 2] = f2_val(r.nm);
                if (tau) tau[i] = __fma_rn(sig_hi, nh, sig_d * nd);
                if (ncell) ncell[i] = r.n;
                active = false;
            }
        }
    }
}

__global__ void k_grad_unpack(long long n, const float4* __restrict__ src, float* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = src[2 * i], b = src[2 * i + 1];
    dst[i] = a.x;
    dst[n + i] = a.y;
    dst[2 * n + i] = a.z;
    dst[3 * n + i] = a.w;
    dst[4 * n + i] = b.x;
    dst[5 * n + i] = b.y;
}

__global__ void k_pack_fields(long long n, const float* nh, const float* vx, const float* vy, const float* vz,
                              const float* T, const float* nd, const float* nm, float4* rec) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float flags = rec[2 * i + 1].w;   // the domain flags stay
    rec[2 * i] = make_float4(nh[i], vx[i], vy[i], vz[i]);
    rec[2 * i + 1] = make_float4(T[i], nd[i], nm ? nm[i] : 0.0f, flags);
}

// H(a, x) by either method (method 1: the Faddeeva function)
__global__ void k_eval_voigt(long long n, const float* a, const double* x, float* H, int method) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (method == 1) {
        const float xh = (float)x[i];
        H[i] = faddeeva_h(a[i], xh, (float)(x[i] - (double)xh));
    } else {
        H[i] = voigt_h(a[i], x[i]);
    }
}

__global__ void k_sample_upar(Params P, long long n, const double* x, const float* a, const uint64_t* id,
                              float* u, int32_t* nd) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Rng rng;
    rng.init(P, id[i]);
    uint32_t trials = 0;
    bool err = false;
    U0Coef c;
    u0_coeffs((double)a[i], c);
    u[i] = sample_upar(rng, (float)x[i], a[i], c, P.x_gauss, trials, err);
    nd[i] = err ? -1 : (int32_t)rng.n;
}

#endif  // !RG_FADDEEVA

}  // inline namespace RG_KVAR

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// draw rings, the u0 coefficient cache of each line, the event counters
static size_t smem_bytes(int nline, int block) {
    return (size_t)(kRing + nline * 6) * block * sizeof(float) + (size_t)block * sizeof(Tallies);
}

template <int NL>
static cudaError_t launch_nl(const Params& P, const PacketsIn& in, const PacketsOut& out, const TraceOut& tr,
                             int grid, int block, cudaStream_t st) {
    size_t smem = smem_bytes(NL, block);
    // per-event traces are recorded by single-model runs without peeling only
    if (tr.nev && (P.nmodels > 0 || P.ndir > 0)) return cudaErrorInvalidValue;
    if (P.nmodels > 0) k_propagate<NL, false, true, false><<<grid, block, smem, st>>>(P, in, out, tr);
    else if (P.ndir > 0) k_propagate<NL, true, false, false><<<grid, block, smem, st>>>(P, in, out, tr);
    else if (tr.nev) k_propagate<NL, false, false, true><<<grid, block, smem, st>>>(P, in, out, tr);
    else k_propagate<NL, false, false, false><<<grid, block, smem, st>>>(P, in, out, tr);
    return cudaGetLastError();
}

cudaError_t RG_SFX(launch_propagate)(const Params& P, const PacketsIn& in, const PacketsOut& out, const TraceOut& tr,
                             int grid, int block, cudaStream_t st) {
    switch (P.nline) {
        case 1: return launch_nl<1>(P, in, out, tr, grid, block, st);
        case 2: return launch_nl<2>(P, in, out, tr, grid, block, st);
        case 3: return launch_nl<3>(P, in, out, tr, grid, block, st);
        case 4: return launch_nl<4>(P, in, out, tr, grid, block, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int NL>
static int ray_occ() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ray_tau<NL>, 128, 0);
    return nb > 0 ? nb : 1;
}

template <int NL, bool ADJ>
static int peel_occ() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_peel<NL, ADJ>, 128, 0);
    return nb > 0 ? nb : 1;
}

cudaError_t RG_SFX(launch_peel)(const Params& P, int sms, cudaStream_t st) {
    const Params* G = P.self;
    const bool adj = P.adj_grad != nullptr;
    switch (P.nline) {
        case 1: k_peel_prep<1><<<sms * 8, 256, 0, st>>>(G); break;
        case 2: k_peel_prep<2><<<sms * 8, 256, 0, st>>>(G); break;
        case 3: k_peel_prep<3><<<sms * 8, 256, 0, st>>>(G); break;
        case 4: k_peel_prep<4><<<sms * 8, 256, 0, st>>>(G); break;
        default: return cudaErrorInvalidValue;
    }
    switch (P.nline * 2 + (adj ? 1 : 0)) {
        case 2: k_peel<1, false><<<sms * peel_occ<1, false>(), 128, 0, st>>>(G); break;
        case 3: k_peel<1, true><<<sms * peel_occ<1, true>(), 128, 0, st>>>(G); break;
        case 4: k_peel<2, false><<<sms * peel_occ<2, false>(), 128, 0, st>>>(G); break;
        case 5: k_peel<2, true><<<sms * peel_occ<2, true>(), 128, 0, st>>>(G); break;
        case 6: k_peel<3, false><<<sms * peel_occ<3, false>(), 128, 0, st>>>(G); break;
        case 7: k_peel<3, true><<<sms * peel_occ<3, true>(), 128, 0, st>>>(G); break;
        case 8: k_peel<4, false><<<sms * peel_occ<4, false>(), 128, 0, st>>>(G); break;
        case 9: k_peel<4, true><<<sms * peel_occ<4, true>(), 128, 0, st>>>(G); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// the queue head P.head must be zero on entry
cudaError_t RG_SFX(launch_ray_tau)(const Params& P, long long n, const double* pos, const double* dir, const double* nu,
                           double* tau, int32_t* cells, double* lens, int cap, int32_t* ncell, RayInit* init,
                           int sms, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int block = 128;
    const int per_sm = P.nline == 1 ? ray_occ<1>() : P.nline == 2 ? ray_occ<2>() : P.nline == 3 ? ray_occ<3>()
                                                                                               : ray_occ<4>();
    const long long need = (n + block - 1) / block;
    const unsigned grid = (unsigned)std::min<long long>(need, (long long)sms * per_sm);
    const unsigned gp = (unsigned)need;
    const Params* G = P.self;
    switch (P.nline) {
#define RG_RAY(NLV)                                                                          \
    case NLV:                                                                                \
        k_ray_prep<NLV><<<gp, block, 0, st>>>(G, n, pos, dir, nu, init);                     \
        k_ray_tau<NLV><<<grid, block, 0, st>>>(G, n, init, tau, cells, lens, cap, ncell);    \
        break;
        RG_RAY(1)
        RG_RAY(2)
        RG_RAY(3)
        RG_RAY(4)
#undef RG_RAY
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

#if !RG_FADDEEVA
int propagate_block_size() { return 128; }

size_t propagate_smem(int nline, int block) { return smem_bytes(nline, block); }

template <int NL, bool PEEL, bool BATCH>
static int occ(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_propagate<NL, PEEL, BATCH, false>, block,
                                                  smem_bytes(NL, block));
    return nb;
}

int propagate_blocks_per_sm(int block, bool peel) {
    return peel ? occ<1, true, false>(block) : occ<1, false, false>(block);
}

int propagate_batch_blocks_per_sm(int nline, int block) {
    switch (nline) {
        case 1: return occ<1, false, true>(block);
        case 2: return occ<2, false, true>(block);
        case 3: return occ<3, false, true>(block);
        default: return occ<4, false, true>(block);
    }
}

size_t packet_save_bytes(int nline) {
    switch (nline) {
        case 1: return sizeof(Packet<1>);
        case 2: return sizeof(Packet<2>);
        case 3: return sizeof(Packet<3>);
        default: return sizeof(Packet<4>);
    }
}

cudaError_t launch_ray_columns(const Params& P, long long n, const double* pos, const double* dir, double* cols,
                               double* tau, double sig_hi, double sig_d, int32_t* ncell, RayInit* init, int sms,
                               cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int block = 128;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ray_columns, block, 0);
    if (per_sm < 1) per_sm = 1;
    const long long need = (n + block - 1) / block;
    const unsigned grid = (unsigned)std::min<long long>(need, (long long)sms * per_sm);
    k_ray_prep<1><<<(unsigned)need, block, 0, st>>>(P.self, n, pos, dir, nullptr, init);
    k_ray_columns<<<grid, block, 0, st>>>(P.self, n, init, cols, tau, sig_hi, sig_d, ncell);
    return cudaGetLastError();
}

cudaError_t launch_grad_unpack(long long nleaf, const float4* src, float* dst, cudaStream_t st) {
    if (nleaf <= 0) return cudaSuccess;
    k_grad_unpack<<<(unsigned)((nleaf + 255) / 256), 256, 0, st>>>(nleaf, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_pack_fields(long long n, const float* nh, const float* vx, const float* vy, const float* vz,
                               const float* T, const float* nd, const float* nm, float4* rec, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_pack_fields<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, nh, vx, vy, vz, T, nd, nm, rec);
    return cudaGetLastError();
}

cudaError_t launch_eval_voigt(long long n, const float* a, const double* x, float* H, int method, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_eval_voigt<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, x, H, method);
    return cudaGetLastError();
}

cudaError_t launch_sample_upar(const Params& P, long long n, const double* x, const float* a, const uint64_t* id,
                               float* u, int32_t* nd, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_sample_upar<<<(unsigned)((n + 127) / 128), 128, kRing * 128 * sizeof(uint32_t), st>>>(P, n, x, a, id, u, nd);
    return cudaGetLastError();
}

#endif  // !RG_FADDEEVA

}  // namespace rg

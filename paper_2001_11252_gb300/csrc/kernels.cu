// Kernels of the resonant-line Monte Carlo path (Michel-Dansac et al. 2020)
// for GB300 (sm_103a).
//
// k_propagate is a persistent kernel: every lane owns one photon packet and
// advances it one walk step (a cell crossing or an interaction, Sect. 3) per
// loop iteration; a lane whose packet has escaped, was absorbed or capped
// refills itself from a global work queue with one warp-aggregated atomic, so
// packets with 1 or 1e6 scatterings share the machine without tail effects
// (the role of the master-worker bundles of Sect. 4.4).
#include <cstdint>
#include <cuda_runtime.h>
#include "device.cuh"
#include "internal.h"

namespace rg {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kInf = __builtin_huge_val();

struct Tallies {
    uint32_t cross, peel_rays, peel_cells, trials, leaf_loads, son_loads, nbor_loads;
    uint32_t scatt_line, scatt_dust;
};

template <int NL>
struct Packet {
    double p[3], k[3], inv[3];
    double nu;     // gas-frame frequency in the current leaf
    double tau;    // optical depth left to the next interaction
    double path;
    long long idx;
    long long nscatt, nsteps;
    Where w;
    Rng rng;
    float budget;  // path length guaranteed to stay inside the leaf
    int status;
    int zero_run;  // consecutive zero-length crossings (guards against a stuck walk)
    bool inv_ok;
    CellCache<NL> cc;
};

__device__ __forceinline__ void dir_from(float kx, float ky, float kz, float mu, float r_phi, double out[3]) {
    float3 e1, e2;
    onb(kx, ky, kz, e1, e2);
    float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    float s, c;
    sincospif(2.0f * r_phi, &s, &c);
    float ox = mu * kx + st * (c * e1.x + s * e2.x);
    float oy = mu * ky + st * (c * e1.y + s * e2.y);
    float oz = mu * kz + st * (c * e1.z + s * e2.z);
    float nn = 1.0f / sqrtf(ox * ox + oy * oy + oz * oz);
    out[0] = (double)(ox * nn);
    out[1] = (double)(oy * nn);
    out[2] = (double)(oz * nn);
}

// ---------------------------------------------------------------------------
// peeling ray: optical depth from p (in leaf w) along direction d to the
// domain border at external frequency nu_ext; stops once tau > tau_stop
// ---------------------------------------------------------------------------
template <int NL>
__device__ double ray_walk(const Params& P, const double p0[3], Where w, const double k[3],
                           const double inv[3], double nu_ext, double tau_stop, Tallies& tl,
                           int32_t* cells, double* lens, int cap, int32_t* ncell) {
    double p[3] = {p0[0], p0[1], p0[2]};
    double tau = 0.0;
    int n = 0, zero_run = 0;
    for (int guard = 0; guard < (1 << 26); ++guard) {
        CellCache<NL> cc;
        load_cell<NL>(P, w.leaf, cc);
        ++tl.leaf_loads;
        double nu = to_gas(nu_ext, beta_of(cc, k));
        float kl[NL];
        float kap = opacity<NL>(P, cc, nu, kl);
        int axis;
        double tf = face_distance(p, k, inv, w, axis);
        double tb = (cc.flags & kFlagBorder) ? border_distance(P, p, k, inv) : kInf;
        bool border = tb <= tf;
        double l = border ? tb : tf;
        tau = __dadd_rn(tau, __dmul_rn(__dmul_rn((double)kap, l), P.box_cm));
        if (cells != nullptr && n < cap) {
            cells[n] = w.leaf;
            lens[n] = l;
        }
        ++n;
        if (border || tau > tau_stop) break;
        zero_run = tf > 0.0 ? 0 : zero_run + 1;
        if (zero_run > 64) break;
        move_to_face(p, k, axis, tf, w);
        wrap_periodic(P, p, k);
        if (!next_leaf(P, p, k, axis, w, tl.son_loads, tl.nbor_loads)) break;
    }
    tl.peel_cells += n;
    if (ncell) *ncell = n;
    return tau;
}

template <int NL>
__device__ void peel(const Params& P, const Packet<NL>& s, int d, float w, double nu_o_gas, Tallies& tl) {
    double ko[3] = {P.dirs[d][0], P.dirs[d][1], P.dirs[d][2]};
    double inv[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) inv[ax] = ko[ax] != 0.0 ? 1.0 / ko[ax] : 0.0;
    double nu_ext = to_ext(nu_o_gas, beta_of(s.cc, ko));
    ++tl.peel_rays;
    double tau = ray_walk<NL>(P, s.p, s.w, ko, inv, nu_ext, P.tau_stop, tl, nullptr, nullptr, 0, nullptr);
    if (tau > P.tau_stop) return;
    float f = w * expf(-(float)tau);
    double t = __dmul_rn(__dsub_rn(nu_ext, P.nu_lo), P.nu_inv_range);
    int ch = (int)floor(t * (double)P.nbin);
    bool chok = t >= 0.0 && ch >= 0 && ch < P.nbin;
    if (chok) atomicAdd(P.pspec + d * P.nbin + ch, f);
    if (P.npix > 0) {
        double r0 = s.p[0] - P.img_c[0], r1 = s.p[1] - P.img_c[1], r2 = s.p[2] - P.img_c[2];
        double u = r0 * P.eu[d][0] + r1 * P.eu[d][1] + r2 * P.eu[d][2];
        double v = r0 * P.ev[d][0] + r1 * P.ev[d][1] + r2 * P.ev[d][2];
        double fu = floor((u * P.inv_fov + 0.5) * (double)P.npix);
        double fv = floor((v * P.inv_fov + 0.5) * (double)P.npix);
        if (fu >= 0.0 && fu < (double)P.npix && fv >= 0.0 && fv < (double)P.npix) {
            long long px = (long long)fv * P.npix + (long long)fu;
            long long npix2 = (long long)P.npix * P.npix;
            atomicAdd(P.pimg + d * npix2 + px, f);
            if (chok && P.cube) atomicAdd(P.pcube + (d * npix2 + px) * P.nbin + ch, f);
        }
    }
}

// ---------------------------------------------------------------------------
// interactions (Sect. 3.2)
// ---------------------------------------------------------------------------
template <int NL, bool PEEL>
__device__ void scatter_dust(const Params& P, Packet<NL>& s, Tallies& tl) {
    float r_alb = s.rng.u24();
    if (r_alb > P.dust_albedo) {
        s.status = RASCAS_PK_ABSORBED_;
        return;
    }
    float r_mu = s.rng.u24(), r_phi = s.rng.u24();
    float mu = mu_sample(PH_HG, r_mu, P.dust_g);
    float kx = (float)s.k[0], ky = (float)s.k[1], kz = (float)s.k[2];
    if (PEEL) {
        for (int d = 0; d < P.ndir; ++d) {
            float muo = kx * (float)P.dirs[d][0] + ky * (float)P.dirs[d][1] + kz * (float)P.dirs[d][2];
            float w = phase_p(PH_HG, muo, P.dust_g) * (1.0f / kTwoPiF);
            peel<NL>(P, s, d, w, s.nu, tl);
        }
    }
    if (!P.keep_dir) {
        dir_from(kx, ky, kz, mu, r_phi, s.k);
        s.inv_ok = false;
    }
    ++tl.scatt_dust;
}

template <int NL, bool PEEL>
__device__ void scatter_line(const Params& P, Packet<NL>& s, int il, Tallies& tl) {
    const LineDev& L = P.line[il];
    float x_in = (float)((s.nu - L.nu0) * s.cc.invdnu[il]);
    int ch = 0;
    if (L.nchan > 1) {
        float r = s.rng.u24();
        ch = L.nchan - 1;
        for (int c = 0; c < L.nchan - 1; ++c)
            if (r < L.chan_cum[c]) { ch = c; break; }
    }
    bool err = false;
    uint32_t trials = 0;
    float upar = sample_upar(s.rng, x_in, s.cc.a[il], P.x_gauss, trials, err);
    tl.trials += trials;
    if (err) {
        s.status = RASCAS_PK_ERROR_;
        return;
    }
    float r1 = s.rng.u24(), r2 = s.rng.u24();
    float rho = sqrtf(-logf(r1));
    float sn, cs;
    sincospif(2.0f * r2, &sn, &cs);
    float up1 = rho * cs, up2 = rho * sn;
    float kx = (float)s.k[0], ky = (float)s.k[1], kz = (float)s.k[2];
    float3 e1, e2;
    onb(kx, ky, kz, e1, e2);
    float vx = upar * kx + up1 * e1.x + up2 * e2.x;   // scatterer velocity / v_th
    float vy = upar * ky + up1 * e1.y + up2 * e2.y;
    float vz = upar * kz + up1 * e1.z + up2 * e2.z;
    int kind;
    if (ch > 0 || P.isotropic || L.phase != 0) kind = PH_ISO;
    else kind = fabsf(x_in - upar) < 0.2f ? PH_CORE : PH_WING;
    float r_mu = s.rng.u24(), r_phi = s.rng.u24();
    float mu = mu_sample(kind, r_mu, 0.0f);
    double kout[3];
    if (P.keep_dir) {
        kout[0] = s.k[0]; kout[1] = s.k[1]; kout[2] = s.k[2];
        mu = 1.0f;
    } else {
        dir_from(kx, ky, kz, mu, r_phi, kout);
    }
    const float vthc = s.cc.vth_c[il];
    const float recp = P.recoil ? L.recoil_pref * (float)s.nu : 0.0f;
    if (PEEL) {
        for (int d = 0; d < P.ndir; ++d) {
            float ox = (float)P.dirs[d][0], oy = (float)P.dirs[d][1], oz = (float)P.dirs[d][2];
            float muo = kx * ox + ky * oy + kz * oz;
            float uo = ox * vx + oy * vy + oz * vz;
            double nu_o;
            if (ch > 0) {
                nu_o = __fma_rn(L.chan_nu[ch], (double)(uo * vthc), L.chan_nu[ch]);
            } else {
                float rec = (1.0f - muo) * recp;
                float f = ((uo - upar) * vthc - rec) / (1.0f + rec);
                nu_o = __fma_rn(s.nu, (double)f, s.nu);
            }
            float w = phase_p(kind, muo, 0.0f) * (1.0f / kTwoPiF);
            peel<NL>(P, s, d, w, nu_o, tl);
        }
    }
    float uout = (float)kout[0] * vx + (float)kout[1] * vy + (float)kout[2] * vz;
    if (ch > 0) {
        s.nu = __fma_rn(L.chan_nu[ch], (double)(uout * vthc), L.chan_nu[ch]);
    } else {
        float rec = (1.0f - mu) * recp;
        float f = ((uout - upar) * vthc - rec) / (1.0f + rec);
        s.nu = __fma_rn(s.nu, (double)f, s.nu);
    }
    if (!P.keep_dir) {
        s.k[0] = kout[0]; s.k[1] = kout[1]; s.k[2] = kout[2];
        s.inv_ok = false;
    }
    ++tl.scatt_line;
}

template <int NL>
__device__ __forceinline__ void trace_record(const Params& P, const Packet<NL>& s, const TraceOut& tr) {
    if (tr.nev == nullptr) return;
    int32_t c = tr.nev[s.idx];
    if (c >= tr.max_events) return;
    TraceEvent& e = tr.ev[(long long)s.idx * tr.max_events + c];
    double b = beta_of(s.cc, s.k);
    for (int ax = 0; ax < 3; ++ax) { e.p[ax] = s.p[ax]; e.k[ax] = s.k[ax]; }
    e.nu = s.status == RASCAS_PK_ERROR_ ? s.nu : to_ext(s.nu, b);
    e.leaf = s.w.leaf; e.level = s.w.level; e.ijk[0] = s.w.i; e.ijk[1] = s.w.j; e.ijk[2] = s.w.k;
    e.status = s.status;
    e.ndraw = s.rng.n;
    e.nscatt = s.nscatt;
    e.nsteps = s.nsteps;
    tr.nev[s.idx] = c + 1;
}

template <int NL, bool PEEL>
__device__ void interact(const Params& P, Packet<NL>& s, double li, bool exact, float kap,
                         const float kl[NL], Tallies& tl, const TraceOut& tr) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) s.p[ax] = __fma_rn(li, s.k[ax], s.p[ax]);
    s.path += li;
    if (exact) {
        double D = inner_distance(s.p, s.w);
        s.budget = __fsub_rd(__double2float_rd(D * (1.0 - 0x1p-20)), 4e-16f);
    }
    // Sect. 3.2: dust with P = tau_d / tau, else line X with P = tau_X / tau
    float r = s.rng.u24();
    float rk = r * kap;
    if (rk < s.cc.kap_d) {
        scatter_dust<NL, PEEL>(P, s, tl);
    } else {
        float acc = s.cc.kap_d;
        int il = NL - 1;
#pragma unroll
        for (int i = 0; i < NL - 1; ++i) {
            acc += kl[i];
            if (rk < acc) { il = i; break; }
        }
        scatter_line<NL, PEEL>(P, s, il, tl);
    }
    if (s.status == RASCAS_PK_ACTIVE_) {
        ++s.nscatt;
        if (P.max_scatt > 0 && s.nscatt >= P.max_scatt) s.status = RASCAS_PK_CAPPED_;
    }
    trace_record<NL>(P, s, tr);
    if (s.status == RASCAS_PK_ACTIVE_) s.tau = tau_event(s.rng.u52());
}

// one walk step: an interaction inside the current leaf, a face crossing, or
// the escape through the domain border (Sect. 3, Sect. 4.3)
template <int NL, bool PEEL>
__device__ void step(const Params& P, Packet<NL>& s, Tallies& tl, const TraceOut& tr) {
    if (P.max_steps > 0 && s.nsteps >= P.max_steps) {
        s.status = RASCAS_PK_CAPPED_;
        trace_record<NL>(P, s, tr);
        return;
    }
    ++s.nsteps;
    float kl[NL];
    float kap = opacity<NL>(P, s.cc, s.nu, kl);
    const bool border_leaf = (s.cc.flags & kFlagBorder) != 0;
    if (!border_leaf) {
        float li = (float)s.tau / (kap * (float)P.box_cm);
        float dec = __fmaf_ru(li, 1.0f + 0x1p-20f, 4e-16f);
        if (dec < s.budget) {
            s.budget = __fsub_rd(s.budget, dec);
            interact<NL, PEEL>(P, s, (double)li, false, kap, kl, tl, tr);
            return;
        }
    }
    if (!s.inv_ok) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) s.inv[ax] = s.k[ax] != 0.0 ? 1.0 / s.k[ax] : 0.0;
        s.inv_ok = true;
    }
    int axis;
    double tf = face_distance(s.p, s.k, s.inv, s.w, axis);
    double tb = border_leaf ? border_distance(P, s.p, s.k, s.inv) : kInf;
    bool border = tb <= tf;
    double l = border ? tb : tf;
    double tau_cell = __dmul_rn(__dmul_rn((double)kap, l), P.box_cm);
    if (tau_cell >= s.tau) {
        double li = s.tau / __dmul_rn((double)kap, P.box_cm);
        interact<NL, PEEL>(P, s, li, true, kap, kl, tl, tr);
        return;
    }
    s.tau = __dsub_rn(s.tau, tau_cell);
    s.path += l;
    if (border) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) s.p[ax] = __fma_rn(l, s.k[ax], s.p[ax]);
        s.status = RASCAS_PK_ESCAPED_;
        trace_record<NL>(P, s, tr);
        return;
    }
    ++tl.cross;
    s.zero_run = tf > 0.0 ? 0 : s.zero_run + 1;
    if (s.zero_run > 64) {
        s.status = RASCAS_PK_ERROR_;
        trace_record<NL>(P, s, tr);
        return;
    }
    double nu_ext = to_ext(s.nu, beta_of(s.cc, s.k));
    move_to_face(s.p, s.k, axis, tf, s.w);
    wrap_periodic(P, s.p, s.k);
    Where nw = s.w;
    if (!next_leaf(P, s.p, s.k, axis, nw, tl.son_loads, tl.nbor_loads)) {
        s.status = RASCAS_PK_ESCAPED_;   // left the box
        trace_record<NL>(P, s, tr);
        return;
    }
    s.w = nw;
    load_cell<NL>(P, s.w.leaf, s.cc);
    ++tl.leaf_loads;
    s.nu = to_gas(nu_ext, beta_of(s.cc, s.k));
    s.budget = 0.0f;
}

template <int NL, bool PEEL>
__device__ void start_packet(const Params& P, const PacketsIn& in, long long idx, Packet<NL>& s,
                             Tallies& tl, const TraceOut& tr) {
    s.idx = idx;
    for (int ax = 0; ax < 3; ++ax) {
        s.p[ax] = in.pos[3 * idx + ax];
        s.k[ax] = in.dir[3 * idx + ax];
    }
    double nu_ext = in.nu[idx];
    s.rng.init(P, in.id[idx]);
    s.nscatt = 0;
    s.nsteps = 0;
    s.path = 0.0;
    s.budget = 0.0f;
    s.inv_ok = false;
    s.zero_run = 0;
    s.status = RASCAS_PK_ACTIVE_;
    wrap_periodic(P, s.p, s.k);
    if (!locate_point(P, s.p, s.k, s.w, tl.son_loads)) {
        s.status = RASCAS_PK_ERROR_;
        s.nu = nu_ext;
        s.w.leaf = -1; s.w.level = 0; s.w.i = s.w.j = s.w.k = 0;
        s.cc.vx = s.cc.vy = s.cc.vz = 0.0f;
        trace_record<NL>(P, s, tr);
        return;
    }
    load_cell<NL>(P, s.w.leaf, s.cc);
    ++tl.leaf_loads;
    s.nu = to_gas(nu_ext, beta_of(s.cc, s.k));
    if (PEEL) {
        for (int d = 0; d < P.ndir; ++d) peel<NL>(P, s, d, 1.0f / (2.0f * kTwoPiF), s.nu, tl);
    }
    trace_record<NL>(P, s, tr);
    s.tau = tau_event(s.rng.u52());
}

template <int NL>
__device__ void finish_packet(const Params& P, const Packet<NL>& s, const PacketsOut& out,
                              uint32_t cnt[5]) {
    double nu_ext = s.status == RASCAS_PK_ERROR_ && s.w.leaf < 0 ? s.nu : to_ext(s.nu, beta_of(s.cc, s.k));
    long long i = s.idx;
    if (out.status) out.status[i] = s.status;
    if (out.nscatt) out.nscatt[i] = s.nscatt;
    if (out.nu) out.nu[i] = nu_ext;
    if (out.path) out.path[i] = s.path;
    for (int ax = 0; ax < 3; ++ax) {
        if (out.pos) out.pos[3 * i + ax] = s.p[ax];
        if (out.dir) out.dir[3 * i + ax] = s.k[ax];
    }
    ++cnt[0];
    if (s.status >= 1 && s.status <= 4) ++cnt[s.status];
    if (s.status == RASCAS_PK_ESCAPED_ && P.spec != nullptr) {
        double t = __dmul_rn(__dsub_rn(nu_ext, P.nu_lo), P.nu_inv_range);
        double fb = floor(t * (double)P.nbin);
        if (fb >= 0.0 && fb < (double)P.nbin) atomicAdd(P.spec + (int)fb, 1.0f);
    }
}

__device__ __forceinline__ void flush(const Params& P, unsigned long long v, int which) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(P.counters + which, v);
}

template <int NL, bool PEEL>
__global__ void __launch_bounds__(128) k_propagate(Params P, PacketsIn in, PacketsOut out, TraceOut tr) {
    Packet<NL> s;
    Tallies tl = {};
    uint32_t cnt[5] = {0, 0, 0, 0, 0};
    const unsigned lane = threadIdx.x & 31u;
    bool have = false, drained = false;
    for (;;) {
        bool want = !have && !drained;
        unsigned m = __ballot_sync(kFull, want);
        if (m) {
            int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(P.head, (unsigned long long)__popc(m));
            base = __shfl_sync(kFull, base, leader);
            if (want) {
                long long idx = (long long)base + __popc(m & ((1u << lane) - 1u));
                if (idx < in.n) {
                    start_packet<NL, PEEL>(P, in, idx, s, tl, tr);
                    if (s.status == RASCAS_PK_ACTIVE_) have = true;
                    else finish_packet<NL>(P, s, out, cnt);
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
            step<NL, PEEL>(P, s, tl, tr);
            if (s.status != RASCAS_PK_ACTIVE_) {
                finish_packet<NL>(P, s, out, cnt);
                have = false;
            }
        }
    }
    flush(P, cnt[0], CNT_PACKETS);
    flush(P, cnt[1], CNT_ESCAPED);
    flush(P, cnt[2], CNT_ABSORBED);
    flush(P, cnt[3], CNT_CAPPED);
    flush(P, cnt[4], CNT_ERRORS);
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
template <int NL>
__global__ void k_ray_tau(Params P, long long n, const double* pos, const double* dir, const double* nu,
                          double* tau, int32_t* cells, double* lens, int cap, int32_t* ncell) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    double k[3] = {dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]};
    double inv[3];
    for (int ax = 0; ax < 3; ++ax) inv[ax] = k[ax] != 0.0 ? 1.0 / k[ax] : 0.0;
    Tallies tl = {};
    wrap_periodic(P, p, k);
    Where w;
    if (!locate_point(P, p, k, w, tl.son_loads)) {
        tau[i] = 0.0;
        if (ncell) ncell[i] = 0;
        return;
    }
    tau[i] = ray_walk<NL>(P, p, w, k, inv, nu[i], kInf, tl, cells ? cells + i * cap : nullptr,
                          lens ? lens + i * cap : nullptr, cap, ncell ? ncell + i : nullptr);
}

__global__ void k_eval_voigt(long long n, const float* a, const double* x, float* H) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) H[i] = voigt_h(a[i], x[i]);
}

__global__ void k_sample_upar(Params P, long long n, const double* x, const float* a, const uint64_t* id,
                              float* u, int32_t* nd) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Rng rng;
    rng.init(P, id[i]);
    uint32_t trials = 0;
    bool err = false;
    u[i] = sample_upar(rng, (float)x[i], a[i], P.x_gauss, trials, err);
    nd[i] = err ? -1 : (int32_t)rng.n;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int propagate_block_size() { return 128; }

template <int NL, bool PEEL>
static int occ(int block) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_propagate<NL, PEEL>, block, 0);
    return nb;
}

int propagate_blocks_per_sm(int block, bool peel) {
    return peel ? occ<1, true>(block) : occ<1, false>(block);
}

template <int NL>
static cudaError_t launch_nl(const Params& P, const PacketsIn& in, const PacketsOut& out, const TraceOut& tr,
                             int grid, int block, cudaStream_t st) {
    if (P.ndir > 0) k_propagate<NL, true><<<grid, block, 0, st>>>(P, in, out, tr);
    else k_propagate<NL, false><<<grid, block, 0, st>>>(P, in, out, tr);
    return cudaGetLastError();
}

cudaError_t launch_propagate(const Params& P, const PacketsIn& in, const PacketsOut& out, const TraceOut& tr,
                             int grid, int block, cudaStream_t st) {
    switch (P.nline) {
        case 1: return launch_nl<1>(P, in, out, tr, grid, block, st);
        case 2: return launch_nl<2>(P, in, out, tr, grid, block, st);
        case 3: return launch_nl<3>(P, in, out, tr, grid, block, st);
        case 4: return launch_nl<4>(P, in, out, tr, grid, block, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ray_tau(const Params& P, long long n, const double* pos, const double* dir, const double* nu,
                           double* tau, int32_t* cells, double* lens, int cap, int32_t* ncell, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int block = 128;
    long long grid = (n + block - 1) / block;
    switch (P.nline) {
        case 1: k_ray_tau<1><<<(unsigned)grid, block, 0, st>>>(P, n, pos, dir, nu, tau, cells, lens, cap, ncell); break;
        case 2: k_ray_tau<2><<<(unsigned)grid, block, 0, st>>>(P, n, pos, dir, nu, tau, cells, lens, cap, ncell); break;
        case 3: k_ray_tau<3><<<(unsigned)grid, block, 0, st>>>(P, n, pos, dir, nu, tau, cells, lens, cap, ncell); break;
        case 4: k_ray_tau<4><<<(unsigned)grid, block, 0, st>>>(P, n, pos, dir, nu, tau, cells, lens, cap, ncell); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_eval_voigt(long long n, const float* a, const double* x, float* H, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_eval_voigt<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, x, H);
    return cudaGetLastError();
}

cudaError_t launch_sample_upar(const Params& P, long long n, const double* x, const float* a, const uint64_t* id,
                               float* u, int32_t* nd, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_sample_upar<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(P, n, x, a, id, u, nd);
    return cudaGetLastError();
}

}  // namespace rg

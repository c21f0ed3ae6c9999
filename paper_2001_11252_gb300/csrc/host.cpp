// Host side of the C ABI (include/rascas_gb300.h): context, octree loader
// (validation, father/neighbour links of Sect. 4.3, top-level lookup grid,
// packed leaf records), problem set-up and kernel launches.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rascas_gb300.h"
#include "internal.h"

using rg::Params;

namespace {

// CODATA 2018, cgs (host-side copy for the line constants)
constexpr double kC = 2.99792458e10;
constexpr double kKB = 1.380649e-16;
constexpr double kH = 6.62607015e-27;
constexpr double kME = 9.1093837015e-28;
constexpr double kE = 4.803204712570263e-10;
constexpr double kPi = 3.14159265358979323846;
// peeling records per round of deferred peeling (64 B each)
constexpr unsigned long long kPeelCap = 1ull << 23;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t b) {
        if (b <= bytes) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, b);
        if (e == cudaSuccess) bytes = b;
        else p = nullptr;
        return e;
    }
};

// an octree and its leaf records as prepared on the host (Sect. 4.3 indices)
struct HostMesh {
    int noct = 0, nleaf = 0, max_level = 0, top_level = 0;
    double box_cm = 0.0;
    bool has_metal = false;
    std::vector<int> son, nbr, top;   // 8 per oct, 8 per oct, 4 per top-grid region
    std::vector<float> rec;           // 8 per leaf
    std::vector<int> leaf_level, leaf_ijk;
};

}  // namespace

struct rascas_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err = "no error";
    int sms = 0;
    // mesh
    bool has_mesh = false;
    HostMesh mesh;
    DevBuf d_rec, d_son, d_nbr, d_top;
    // problem
    bool has_domain = false, has_lines = false, has_phys = false, has_det = false;
    rascas_domain dom{};
    rascas_physics phys{};
    rascas_detector det{};
    Params P{};
    DevBuf d_spec, d_pspec, d_pimg, d_pcube, d_counters, d_params;
    DevBuf stage_in, stage_out, stage_aux, stage_adj, ray_init;
    DevBuf peel_rec, peel_prep, peel_live, peel_save, peel_flag, peel_ctl;   // deferred peeling
    DevBuf grad_vec;                                    // adjoint: per-leaf gradient vectors
    unsigned long long peel_cap = kPeelCap;
    // batch of independent models
    struct Batch {
        int nmodels = 0, nbin = 0, nline_at_load = 0;
        long long npackets = 0;
        std::vector<int> order;          // scheduled position -> model index
        std::vector<long long> first;    // packet prefix sums in scheduled order
        DevBuf d_rec, d_son, d_nbr, d_top, d_geo, d_first, d_pos, d_dir, d_nu, d_id, d_spec;
        int block = 128, blocks_per_sm = 0;   // launch shape (autotuned)
        int refill = 1;                       // packets a lane reserves per queue grab (autotuned)
        cudaGraphExec_t graph = nullptr;
        cudaStream_t graph_stream = nullptr;
        unsigned long long graph_key = 0;
    } batch;
    cudaStream_t own_stream = nullptr;    // for graph capture when the context's stream is the legacy one
    unsigned long long version = 1;       // bumped by every set-up call
    // device address of the allocation-free entry point's static scratch,
    // resolved when the context is created (the module load that backs it
    // happens then, not inside rascas_propagate_noalloc)
    void* noalloc_base = nullptr;
    size_t noalloc_bytes = 0;
};

namespace {

int fail(rascas_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(rascas_ctx* c, cudaError_t e, const char* what) {
    return fail(c, e == cudaErrorMemoryAllocation ? RASCAS_E_OOM : RASCAS_E_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

cudaError_t to_host(void* dst, const void* src, size_t bytes, int mem) {
    if (mem == RASCAS_DEVICE) return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    std::memcpy(dst, src, bytes);
    return cudaSuccess;
}

// leaf flags for a domain: a leaf is interior when it lies strictly inside the
// domain with a relative margin; then no ray from inside it reaches the border
// before one of its faces, and the walk skips the border distance there
void mesh_flags(HostMesh& M, const rascas_domain* dom) {
    for (int i = 0; i < M.nleaf; ++i) {
        int l = M.leaf_level[i];
        double h = std::ldexp(1.0, -l);
        double lo[3], hi[3];
        for (int ax = 0; ax < 3; ++ax) {
            lo[ax] = M.leaf_ijk[3 * (size_t)i + ax] * h;
            hi[ax] = lo[ax] + h;
        }
        bool interior = false;
        if (dom) {
            const double* c = dom->centre;
            double R = dom->size;
            const double m = 1e-9 * (R > 0 ? R : 1.0);
            if (dom->kind == RASCAS_DOMAIN_SPHERE || dom->kind == RASCAS_DOMAIN_SHELL) {
                double d2 = 0.0, n2 = 0.0;
                for (int ax = 0; ax < 3; ++ax) {
                    double far = std::fmax(std::fabs(lo[ax] - c[ax]), std::fabs(hi[ax] - c[ax]));
                    double near = c[ax] < lo[ax] ? lo[ax] - c[ax] : (c[ax] > hi[ax] ? c[ax] - hi[ax] : 0.0);
                    d2 += far * far;
                    n2 += near * near;
                }
                interior = std::sqrt(d2) < R - m;
                if (dom->kind == RASCAS_DOMAIN_SHELL) interior = interior && std::sqrt(n2) > dom->inner + m;
            } else {
                interior = true;
                for (int ax = 0; ax < 3; ++ax) {
                    if (dom->kind == RASCAS_DOMAIN_SLAB && ax != 2) continue;
                    if (!(lo[ax] > c[ax] - R + m && hi[ax] < c[ax] + R - m)) interior = false;
                }
            }
        }
        int flags = interior ? 0 : rg::kFlagBorder;
        std::memcpy(&M.rec[8 * (size_t)i + 7], &flags, 4);
    }
}

// validate an octree and build its host-side indices: BFS levels and
// coordinates, father and neighbour cells per oct (Sect. 4.3), the dense top
// grid, packed leaf records.  Returns 0 or an error message.
const char* build_mesh(const rascas_octree* t, int mem, HostMesh& M, cudaError_t& cerr) {
    cerr = cudaSuccess;
    if (t->noct < 1 || t->nleaf < 1 || !t->son || !t->n_HI || !t->vx || !t->vy || !t->vz || !t->T || !t->n_dust)
        return "octree: missing array or empty tree";
    if (!(t->box_cm > 0.0)) return "octree: box_cm must be > 0";
    const int noct = t->noct, nleaf = t->nleaf;
    std::vector<int> son((size_t)8 * noct);
    if ((cerr = to_host(son.data(), t->son, son.size() * 4, mem)) != cudaSuccess) return "octree: copy failed";
    std::vector<float> f[7];
    const float* src[7] = {t->n_HI, t->vx, t->vy, t->vz, t->T, t->n_dust, t->n_metal};
    for (int i = 0; i < 7; ++i) {
        f[i].assign(nleaf, 0.0f);
        if (src[i] && (cerr = to_host(f[i].data(), src[i], (size_t)nleaf * 4, mem)) != cudaSuccess)
            return "octree: copy failed";
    }
    std::vector<int> oct_level(noct, 0), oct_org((size_t)3 * noct, 0), oct_father(noct, -1);
    std::vector<int> lvl(nleaf, 0), ijk((size_t)3 * nleaf, 0);
    std::vector<int> queue;
    queue.reserve(noct);
    queue.push_back(0);
    oct_level[0] = 1;
    int max_level = 1;
    size_t seen_leaf = 0;
    for (size_t qi = 0; qi < queue.size(); ++qi) {
        int o = queue[qi];
        int l = oct_level[o];
        if (l > 21) return "octree: deeper than 21 levels";
        max_level = l > max_level ? l : max_level;
        for (int c = 0; c < 8; ++c) {
            int ci[3] = {oct_org[3 * (size_t)o] + (c & 1), oct_org[3 * (size_t)o + 1] + ((c >> 1) & 1),
                         oct_org[3 * (size_t)o + 2] + ((c >> 2) & 1)};
            int v = son[(size_t)8 * o + c];
            if (v > 0) {
                if (v >= noct || oct_level[v] != 0) return "octree: bad or repeated oct link";
                oct_level[v] = l + 1;
                oct_father[v] = 8 * o + c;
                for (int ax = 0; ax < 3; ++ax) oct_org[3 * (size_t)v + ax] = 2 * ci[ax];
                queue.push_back(v);
            } else if (v < 0) {
                long long leaf = -(long long)v - 1;
                if (leaf >= nleaf || lvl[leaf] != 0) return "octree: bad or repeated leaf link";
                lvl[leaf] = l;
                for (int ax = 0; ax < 3; ++ax) ijk[3 * leaf + ax] = ci[ax];
                ++seen_leaf;
            } else {
                return "octree: son value 0";
            }
        }
    }
    if ((int)queue.size() != noct || (int)seen_leaf != nleaf) return "octree: unreachable octs or leaves";
    // neighbour links: per oct the 6 cells (level l-1, or the deepest coarser
    // cell when the tree is not graded) across the faces of its father cell,
    // wrapped periodically; -1 for the root oct
    auto find_cell = [&](int cx, int cy, int cz, int target, int& level_out) {
        int o = 0;
        for (int m = 1;; ++m) {
            int s = target - m;
            int child = ((cx >> s) & 1) | (((cy >> s) & 1) << 1) | (((cz >> s) & 1) << 2);
            int cell = 8 * o + child;
            int v = son[cell];
            if (m == target || v < 0) {
                level_out = m;
                return cell;
            }
            o = v;
        }
    };
    std::vector<int> nbr((size_t)8 * noct, -1);
    for (int o = 0; o < noct; ++o) {
        int l = oct_level[o];
        int packed = 0;
        nbr[8 * (size_t)o + 6] = oct_father[o];
        if (l >= 2) {
            int fl = l - 1;
            int nf = 1 << fl;
            int F[3] = {oct_org[3 * (size_t)o] >> 1, oct_org[3 * (size_t)o + 1] >> 1, oct_org[3 * (size_t)o + 2] >> 1};
            for (int face = 0; face < 6; ++face) {
                int ax = face >> 1;
                int G[3] = {F[0], F[1], F[2]};
                G[ax] = (G[ax] + ((face & 1) ? 1 : -1) + nf) & (nf - 1);
                int nl = 0;
                int cell = find_cell(G[0], G[1], G[2], fl, nl);
                nbr[8 * (size_t)o + face] = cell;
                packed |= (nl & 31) << (5 * face);
            }
        }
        nbr[8 * (size_t)o + 7] = packed;
    }
    // dense top grid at level S: deepest cell at level <= S over each region
    int S = max_level < 6 ? max_level : 6;
    size_t ntop = (size_t)1 << (3 * S);
    std::vector<int> top(4 * ntop, 0);
    for (size_t r = 0; r < ntop; ++r) {
        int cx = (int)(r & ((1u << S) - 1)), cy = (int)((r >> S) & ((1u << S) - 1)), cz = (int)(r >> (2 * S));
        int o = 0;
        for (int m = 1;; ++m) {
            int s = S - m;
            int child = ((cx >> s) & 1) | (((cy >> s) & 1) << 1) | (((cz >> s) & 1) << 2);
            int v = son[8 * (size_t)o + child];
            if (v < 0 || m == S) {
                top[4 * r] = v;
                top[4 * r + 1] = m;
                top[4 * r + 2] = o;
                break;
            }
            o = v;
        }
    }
    M.rec.assign((size_t)8 * nleaf, 0.0f);
    for (int i = 0; i < nleaf; ++i) {
        float* r = &M.rec[8 * (size_t)i];
        for (int j = 0; j < 7; ++j) r[j] = f[j][i];
    }
    M.noct = noct;
    M.nleaf = nleaf;
    M.max_level = max_level;
    M.top_level = S;
    M.box_cm = t->box_cm;
    M.has_metal = t->n_metal != nullptr;
    M.son.swap(son);
    M.nbr.swap(nbr);
    M.top.swap(top);
    M.leaf_level.swap(lvl);
    M.leaf_ijk.swap(ijk);
    return nullptr;
}

}  // namespace

extern "C" {

int rascas_create(rascas_ctx** out, int device) {
    if (!out) return RASCAS_E_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return RASCAS_E_CUDA;
    rascas_ctx* ctx = new (std::nothrow) rascas_ctx();
    if (!ctx) return RASCAS_E_OOM;
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete ctx;
        return RASCAS_E_CUDA;
    }
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (rg::noalloc_scratch(&ctx->noalloc_base, &ctx->noalloc_bytes) != cudaSuccess) {
        delete ctx;
        return RASCAS_E_CUDA;
    }
    if (ctx->d_counters.ensure(sizeof(unsigned long long) * rg::kCounterWords) != cudaSuccess ||
        ctx->d_params.ensure(sizeof(Params)) != cudaSuccess) {
        ctx->d_counters.release();
        delete ctx;
        return RASCAS_E_OOM;
    }
    ctx->P.self = (const Params*)ctx->d_params.p;
    ctx->P.counters = (unsigned long long*)ctx->d_counters.p;
    ctx->P.head = ctx->P.counters + rg::CNT_N;
    ctx->P.abort_flag = (unsigned int*)(ctx->P.counters + rg::CNT_N + 1);
    ctx->P.tau_stop = 50.0;
    ctx->P.x_gauss = 8.0f;
    ctx->P.recoil = 1;
    ctx->P.refill = 1;
    *out = ctx;
    return RASCAS_OK;
}

int rascas_destroy(rascas_ctx* ctx) {
    if (!ctx) return RASCAS_E_ARG;
    cudaSetDevice(ctx->device);
    for (DevBuf* b : {&ctx->d_rec, &ctx->d_son, &ctx->d_nbr, &ctx->d_top, &ctx->d_spec, &ctx->d_pspec,
                      &ctx->d_pimg, &ctx->d_pcube, &ctx->d_counters, &ctx->d_params, &ctx->stage_in,
                      &ctx->stage_out, &ctx->stage_aux, &ctx->stage_adj, &ctx->ray_init, &ctx->peel_rec,
                      &ctx->peel_prep, &ctx->peel_live, &ctx->peel_save, &ctx->peel_flag, &ctx->peel_ctl,
                      &ctx->grad_vec})
        b->release();
    auto& B = ctx->batch;
    for (DevBuf* b : {&B.d_rec, &B.d_son, &B.d_nbr, &B.d_top, &B.d_geo, &B.d_first, &B.d_pos, &B.d_dir, &B.d_nu,
                      &B.d_id, &B.d_spec})
        b->release();
    if (B.graph) cudaGraphExecDestroy(B.graph);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return RASCAS_OK;
}

const char* rascas_last_error(const rascas_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int rascas_set_stream(rascas_ctx* ctx, void* stream) {
    if (!ctx) return RASCAS_E_ARG;
    ctx->stream = (cudaStream_t)stream;
    return RASCAS_OK;
}

int rascas_load_octree(rascas_ctx* ctx, const rascas_octree* t, int mem) {
    if (!ctx || !t) return RASCAS_E_ARG;
    CK(cudaSetDevice(ctx->device));
    HostMesh M;
    cudaError_t ce;
    const char* err = build_mesh(t, mem, M, ce);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "load_octree");
    if (err) return fail(ctx, RASCAS_E_ARG, err);
    mesh_flags(M, ctx->has_domain ? &ctx->dom : nullptr);
    CK(ctx->d_rec.ensure(M.rec.size() * 4));
    CK(ctx->d_son.ensure(M.son.size() * 4));
    CK(ctx->d_nbr.ensure(M.nbr.size() * 4));
    CK(ctx->d_top.ensure(M.top.size() * 4));
    CK(cudaMemcpy(ctx->d_rec.p, M.rec.data(), M.rec.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_son.p, M.son.data(), M.son.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_nbr.p, M.nbr.data(), M.nbr.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_top.p, M.top.data(), M.top.size() * 4, cudaMemcpyHostToDevice));
    Params& P = ctx->P;
    P.g.rec = (const float4*)ctx->d_rec.p;
    P.g.son = (const int*)ctx->d_son.p;
    P.g.nbr = (const int4*)ctx->d_nbr.p;
    P.g.top = (const int4*)ctx->d_top.p;
    P.g.top_level = M.top_level;
    P.g.max_level = M.max_level;
    P.g.nleaf = M.nleaf;
    P.g.noct = M.noct;
    P.g.box_cm = M.box_cm;
    P.g.box_cm_f = (float)M.box_cm;
    ctx->mesh = std::move(M);
    ctx->has_mesh = true;
    return RASCAS_OK;
}

int rascas_set_domain(rascas_ctx* ctx, const rascas_domain* d) {
    if (!ctx || !d) return RASCAS_E_ARG;
    if (d->kind < 0 || d->kind > 3 || !(d->size > 0.0) ||
        (d->kind == RASCAS_DOMAIN_SHELL && !(d->inner >= 0.0 && d->inner < d->size)))
        return fail(ctx, RASCAS_E_ARG, "domain: bad kind or size");
    ctx->dom = *d;
    ctx->has_domain = true;
    Params& P = ctx->P;
    P.g.dom_kind = d->kind;
    for (int ax = 0; ax < 3; ++ax) P.g.dom_c[ax] = d->centre[ax];
    P.g.dom_R = d->size;
    P.g.dom_Rin = d->kind == RASCAS_DOMAIN_SHELL ? d->inner : 0.0;
    if (ctx->has_mesh) {
        CK(cudaSetDevice(ctx->device));
        mesh_flags(ctx->mesh, &ctx->dom);
        CK(cudaMemcpy(ctx->d_rec.p, ctx->mesh.rec.data(), ctx->mesh.rec.size() * 4, cudaMemcpyHostToDevice));
    }
    return RASCAS_OK;
}

int rascas_set_lines(rascas_ctx* ctx, const rascas_line* lines, int32_t nline, const rascas_dust* dust) {
    if (!ctx || nline < 1 || nline > RASCAS_MAX_LINES || !lines)
        return fail(ctx, RASCAS_E_ARG, "lines: need 1..4 lines");
    Params& P = ctx->P;
    for (int i = 0; i < nline; ++i) {
        const rascas_line& L = lines[i];
        if (!(L.nu0 > 0 && L.A_ul > 0 && L.f_lu > 0 && L.mass_g > 0) || L.nchan < 1 || L.nchan > RASCAS_MAX_CHANNELS ||
            (L.density != 0 && L.density != 1))
            return fail(ctx, RASCAS_E_ARG, "lines: bad line data");
        rg::LineDev& D = P.line[i];
        D.nu0 = L.nu0;
        D.nu0_f = (float)L.nu0;
        double vp = std::sqrt(2.0 * kKB / L.mass_g);
        D.vth_pref = vp;
        D.invdnu_pref = kC / (L.nu0 * vp);
        D.invdnu_h = (float)D.invdnu_pref;
        D.invdnu_l = (float)(D.invdnu_pref - (double)D.invdnu_h);
        D.dnu_pref = L.nu0 * vp / kC;
        D.nu0_gap = lines[0].nu0 - L.nu0;
        D.a_pref = (float)(L.A_ul * kC / (4.0 * kPi * L.nu0 * vp));
        D.a_over_invdnu = L.A_ul / (4.0 * kPi);
        D.sig_pref = (float)(std::sqrt(kPi) * kE * kE * L.f_lu / (kME * L.nu0 * vp));
        D.abund = (float)L.abundance;
        D.recoil_pref = (float)(kH / (L.mass_g * kC * kC));
        D.vth_over_c_pref = (float)(vp / kC);
        D.dens = L.density;
        D.phase = L.phase;
        D.nchan = L.nchan;
        double tot = 0.0;
        for (int c = 0; c < L.nchan; ++c) tot += L.chan_A[c];
        double acc = 0.0;
        for (int c = 0; c < rg::kMaxChan; ++c) {
            if (c < L.nchan) {
                acc += L.chan_A[c];
                D.chan_cum[c] = (float)(acc / tot);
                D.chan_nu[c] = L.chan_nu[c];
            } else {
                D.chan_cum[c] = 1.0f;
                D.chan_nu[c] = L.nu0;
            }
        }
    }
    P.nline = nline;
    ++ctx->version;
    P.dust_sigma = dust ? (float)dust->sigma : 0.0f;
    P.dust_albedo = dust ? (float)dust->albedo : 0.0f;
    P.dust_g = dust ? (float)dust->g : 0.0f;
    ctx->has_lines = true;
    return RASCAS_OK;
}

// the walk kernels built for the H(a,x) method of the parameters
static cudaError_t walk_propagate(const rg::Params& P, const rg::PacketsIn& in, const rg::PacketsOut& out,
                                  const rg::TraceOut& tr, int grid, int block, cudaStream_t st) {
    return P.voigt == RASCAS_VOIGT_FADDEEVA ? rg::launch_propagate_fad(P, in, out, tr, grid, block, st)
                                            : rg::launch_propagate(P, in, out, tr, grid, block, st);
}
static cudaError_t walk_peel(const rg::Params& P, int sms, cudaStream_t st) {
    return P.voigt == RASCAS_VOIGT_FADDEEVA ? rg::launch_peel_fad(P, sms, st) : rg::launch_peel(P, sms, st);
}
static cudaError_t walk_ray_tau(const rg::Params& P, long long n, const double* pos, const double* dir,
                                const double* nu, double* tau, int32_t* cells, double* lens, int cap,
                                int32_t* ncell, rg::RayInit* init, int sms, cudaStream_t st) {
    return P.voigt == RASCAS_VOIGT_FADDEEVA
               ? rg::launch_ray_tau_fad(P, n, pos, dir, nu, tau, cells, lens, cap, ncell, init, sms, st)
               : rg::launch_ray_tau(P, n, pos, dir, nu, tau, cells, lens, cap, ncell, init, sms, st);
}

int rascas_set_voigt(rascas_ctx* ctx, int method) {
    if (!ctx) return RASCAS_E_ARG;
    if (method != RASCAS_VOIGT_TASITSIOMI && method != RASCAS_VOIGT_FADDEEVA)
        return fail(ctx, RASCAS_E_ARG, "voigt: unknown method");
    ctx->P.voigt = method;
    ++ctx->version;
    return RASCAS_OK;
}

int rascas_set_physics(rascas_ctx* ctx, const rascas_physics* ph) {
    if (!ctx || !ph) return RASCAS_E_ARG;
    if (!(ph->x_gauss > 0.0) || ph->max_scatt < 0 || ph->max_steps < 0 || !(ph->tau_stop > 0.0) ||
        !(ph->core_skip >= 0.0) || !(ph->core_skip_f >= 0.0))
        return fail(ctx, RASCAS_E_ARG, "physics: bad values");
    ctx->phys = *ph;
    Params& P = ctx->P;
    P.recoil = ph->recoil;
    P.isotropic = ph->isotropic;
    P.keep_dir = ph->keep_dir;
    P.x_gauss = (float)ph->x_gauss;
    P.max_scatt = ph->max_scatt;
    P.max_steps = ph->max_steps;
    P.tau_stop = ph->tau_stop;
    P.key0 = (uint32_t)ph->seed;
    P.key1 = (uint32_t)(ph->seed >> 32);
    for (int r = 0; r < 10; ++r) {   // the Philox4x32-10 key schedule (Salmon et al. 2011)
        P.round_key[r][0] = P.key0 + (uint32_t)r * 0x9E3779B9u;
        P.round_key[r][1] = P.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    P.core_skip = (float)ph->core_skip;
    P.core_skip_f = (float)ph->core_skip_f;
    P.core_skip_on = ph->core_skip > 0.0 || ph->core_skip_f > 0.0;
    ++ctx->version;
    ctx->has_phys = true;
    return RASCAS_OK;
}

int rascas_set_limits(rascas_ctx* ctx, int64_t max_iterations, double time_limit_s) {
    if (!ctx || max_iterations < 0 || max_iterations > 0xffffffffLL || !(time_limit_s >= 0.0) ||
        !(time_limit_s < 1.8e10))
        return fail(ctx, RASCAS_E_ARG, "set_limits: bad values");
    Params& P = ctx->P;
    P.max_iter = (unsigned int)max_iterations;
    P.time_limit_ns = (unsigned long long)(time_limit_s * 1e9);
    if (time_limit_s > 0.0 && P.time_limit_ns == 0ull) P.time_limit_ns = 1ull;
    P.limits = P.max_iter != 0u || P.time_limit_ns != 0ull;
    ++ctx->version;
    return RASCAS_OK;
}

int rascas_set_detector(rascas_ctx* ctx, const rascas_detector* d) {
    if (!ctx || !d) return RASCAS_E_ARG;
    if (d->nbin < 1 || !(d->nu_hi > d->nu_lo) || d->ndir < 0 || d->ndir > RASCAS_MAX_DIRS || d->npix < 0 ||
        (d->npix > 0 && !(d->fov > 0)))
        return fail(ctx, RASCAS_E_ARG, "detector: bad values");
    CK(cudaSetDevice(ctx->device));
    ctx->det = *d;
    Params& P = ctx->P;
    P.g.nu_lo = d->nu_lo;
    P.g.nu_range = d->nu_hi - d->nu_lo;
    P.g.nbin = d->nbin;
    P.ndir = d->ndir;
    P.npix = d->npix;
    P.cube = d->cube && d->npix > 0 && d->ndir > 0;
    P.fov = d->npix > 0 ? d->fov : 1.0;
    for (int ax = 0; ax < 3; ++ax) P.img_c[ax] = d->centre[ax];
    for (int i = 0; i < d->ndir; ++i) {
        double n2 = d->dirs[i][0] * d->dirs[i][0] + d->dirs[i][1] * d->dirs[i][1] + d->dirs[i][2] * d->dirs[i][2];
        if (!(n2 > 0)) return fail(ctx, RASCAS_E_ARG, "detector: zero direction");
        double nn = std::sqrt(n2);
        double n[3] = {d->dirs[i][0] / nn, d->dirs[i][1] / nn, d->dirs[i][2] / nn};
        for (int ax = 0; ax < 3; ++ax) {
            P.dirs[i][ax] = n[ax];
            // 1/k correctly rounded, as the walk's face distances need it
            P.dir_inv[i][ax] = n[ax] != 0.0 ? 1.0 / n[ax] : 0.0;
            P.dir_kp[i][ax][0] = (float)n[ax];
            P.dir_kp[i][ax][1] = (float)(n[ax] - (double)(float)n[ax]);
        }
        // image plane basis: Duff et al. (2017)
        double sg = std::copysign(1.0, n[2]);
        double a = -1.0 / (sg + n[2]);
        double b = n[0] * n[1] * a;
        P.eu[i][0] = 1.0 + sg * n[0] * n[0] * a;
        P.eu[i][1] = sg * b;
        P.eu[i][2] = -sg * n[0];
        P.ev[i][0] = b;
        P.ev[i][1] = sg + n[1] * n[1] * a;
        P.ev[i][2] = -n[1];
    }
    size_t npix2 = (size_t)d->npix * d->npix;
    CK(ctx->d_spec.ensure((size_t)d->nbin * 4));
    CK(ctx->d_pspec.ensure((size_t)(d->ndir > 0 ? d->ndir : 1) * d->nbin * 4));
    CK(ctx->d_pimg.ensure((size_t)(d->ndir > 0 ? d->ndir : 1) * (npix2 > 0 ? npix2 : 1) * 4));
    if (P.cube) CK(ctx->d_pcube.ensure((size_t)d->ndir * npix2 * d->nbin * 4));
    P.g.spec = (float*)ctx->d_spec.p;
    P.pspec = (float*)ctx->d_pspec.p;
    P.pimg = (float*)ctx->d_pimg.p;
    P.pcube = P.cube ? (float*)ctx->d_pcube.p : nullptr;
    ctx->has_det = true;
    return rascas_zero_tallies(ctx);
}

int rascas_set_peel_capacity(rascas_ctx* ctx, int64_t records) {
    if (!ctx || records < 1) return fail(ctx, RASCAS_E_ARG, "set_peel_capacity: records must be >= 1");
    ctx->peel_cap = (unsigned long long)records;
    return RASCAS_OK;
}

int rascas_zero_tallies(rascas_ctx* ctx) {
    if (!ctx) return RASCAS_E_ARG;
    if (!ctx->has_det) return RASCAS_OK;
    CK(cudaSetDevice(ctx->device));
    const rascas_detector& d = ctx->det;
    size_t npix2 = (size_t)d.npix * d.npix;
    CK(cudaMemsetAsync(ctx->d_spec.p, 0, (size_t)d.nbin * 4, ctx->stream));
    if (d.ndir > 0) {
        CK(cudaMemsetAsync(ctx->d_pspec.p, 0, (size_t)d.ndir * d.nbin * 4, ctx->stream));
        if (npix2) CK(cudaMemsetAsync(ctx->d_pimg.p, 0, (size_t)d.ndir * npix2 * 4, ctx->stream));
        if (ctx->P.cube) CK(cudaMemsetAsync(ctx->d_pcube.p, 0, (size_t)d.ndir * npix2 * d.nbin * 4, ctx->stream));
    }
    return RASCAS_OK;
}

}  // extern "C"

namespace {

int check_ready(rascas_ctx* ctx) {
    if (!ctx->has_mesh) return fail(ctx, RASCAS_E_STATE, "no octree loaded");
    if (!ctx->has_domain) return fail(ctx, RASCAS_E_STATE, "no domain set");
    if (!ctx->has_lines) return fail(ctx, RASCAS_E_STATE, "no lines set");
    if (!ctx->has_phys) return fail(ctx, RASCAS_E_STATE, "no physics set");
    if (ctx->P.nline > 0) {
        for (int i = 0; i < ctx->P.nline; ++i)
            if (ctx->P.line[i].dens == 1 && !ctx->mesh.has_metal)
                return fail(ctx, RASCAS_E_STATE, "a line needs n_metal but the octree has none");
    }
    return RASCAS_OK;
}

// stage n packets from host into device buffers; returns device views
struct Staged {
    rg::PacketsIn in;
    rg::PacketsOut out;
};

int persistent_grid(rascas_ctx* ctx, bool peel) {
    int block = rg::propagate_block_size();
    int per_sm = rg::propagate_blocks_per_sm(block, peel);
    if (per_sm < 1) per_sm = 1;
    return ctx->sms * per_sm;
}

int run_propagate(rascas_ctx* ctx, const rascas_packets_in* in, int64_t n, const rascas_packets_out* out,
                  int mem, rascas_run_stats* stats, rascas_event* events, int32_t* nevents, int32_t max_events,
                  bool tallies, const Params* adj = nullptr) {
    if (!ctx || !in || n < 0 || (mem != RASCAS_HOST && mem != RASCAS_DEVICE)) return fail(ctx, RASCAS_E_ARG, "bad arguments");
    if (n > 0 && (!in->pos || !in->dir || !in->nu || !in->id)) return fail(ctx, RASCAS_E_ARG, "packets: null array");
    int r = check_ready(ctx);
    if (r) return r;
    CK(cudaSetDevice(ctx->device));
    Params P = adj ? *adj : ctx->P;
    if (!tallies || !ctx->has_det) {
        P.g.spec = nullptr;
        P.ndir = 0;
        if (!ctx->has_det) {
            P.g.nbin = 1;
            P.g.nu_lo = 0.0;
            P.g.nu_range = 1.0;
        }
    }
    rg::PacketsIn din{in->pos, in->dir, in->nu, in->id, (long long)n, 0};
    rg::PacketsOut dout{};
    if (out) dout = rg::PacketsOut{out->status, out->nscatt, out->nu, out->pos, out->dir, out->path};
    rg::TraceOut tr{nullptr, nullptr, max_events};
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n;
    if (mem == RASCAS_HOST && n > 0) {
        size_t bin = N * (3 + 3 + 1 + 1) * 8;
        CK(ctx->stage_in.ensure(bin));
        char* b = (char*)ctx->stage_in.p;
        double* pos = (double*)b;
        double* dir = pos + 3 * N;
        double* nu = dir + 3 * N;
        uint64_t* id = (uint64_t*)(nu + N);
        CK(cudaMemcpyAsync(pos, in->pos, 3 * N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dir, in->dir, 3 * N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(nu, in->nu, N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(id, in->id, N * 8, cudaMemcpyHostToDevice, st));
        din = rg::PacketsIn{pos, dir, nu, id, (long long)n, 0};
        if (out) {
            size_t bout = N * (4 + 8 + 8 + 24 + 24 + 8) + 64;
            CK(ctx->stage_out.ensure(bout));
            char* o = (char*)ctx->stage_out.p;
            double* onu = (double*)o;
            double* opos = onu + N;
            double* odir = opos + 3 * N;
            double* opath = odir + 3 * N;
            int64_t* ons = (int64_t*)(opath + N);
            int32_t* ost = (int32_t*)(ons + N);
            dout = rg::PacketsOut{out->status ? ost : nullptr, out->nscatt ? ons : nullptr, out->nu ? onu : nullptr,
                                  out->pos ? opos : nullptr, out->dir ? odir : nullptr, out->path ? opath : nullptr};
        }
        if (events) {
            size_t bev = N * (size_t)max_events * sizeof(rg::TraceEvent) + N * 4;
            CK(ctx->stage_aux.ensure(bev));
            tr.ev = (rg::TraceEvent*)ctx->stage_aux.p;
            tr.nev = (int32_t*)((char*)ctx->stage_aux.p + N * (size_t)max_events * sizeof(rg::TraceEvent));
        }
    } else if (events) {
        tr.ev = (rg::TraceEvent*)events;
        tr.nev = nevents;
    }
    if (tr.nev) CK(cudaMemsetAsync(tr.nev, 0, N * 4, st));
    CK(cudaMemsetAsync(ctx->d_counters.p, 0, sizeof(unsigned long long) * rg::kCounterWords, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, st));
    }
    if (n > 0 && P.ndir > 0) {
        // deferred peeling: rounds of (scattering kernel appending peeling
        // rays, peel kernel walking them) until no packet was parked
        const int grid = persistent_grid(ctx, true), block = rg::propagate_block_size();
        const size_t threads = (size_t)grid * block;
        const unsigned long long margin = (unsigned long long)threads * (2 * P.ndir + 1) + 4096;
        const unsigned long long cap = std::max<unsigned long long>(ctx->peel_cap, 4 * margin);
        CK(ctx->peel_rec.ensure(cap * sizeof(rg::PeelRec)));
        CK(ctx->peel_prep.ensure(cap * sizeof(rg::PeelPrep)));
        CK(ctx->peel_live.ensure(cap * sizeof(unsigned long long)));
        CK(ctx->peel_save.ensure(threads * rg::packet_save_bytes(P.nline)));
        CK(ctx->peel_flag.ensure(threads * sizeof(int)));
        CK(ctx->peel_ctl.ensure(4 * sizeof(unsigned long long)));
        unsigned long long* ctl = (unsigned long long*)ctx->peel_ctl.p;
        P.peel_rec = (rg::PeelRec*)ctx->peel_rec.p;
        P.peel_prep = (rg::PeelPrep*)ctx->peel_prep.p;
        P.peel_live = (unsigned long long*)ctx->peel_live.p;
        P.peel_count = ctl;
        P.peel_head = ctl + 1;
        P.suspended = (unsigned int*)(ctl + 2);
        P.peel_nlive = ctl + 3;
        P.peel_cap = cap;
        P.peel_hw = cap - margin;
        P.save = ctx->peel_save.p;
        P.save_flag = (int*)ctx->peel_flag.p;
        CK(cudaMemsetAsync(P.save_flag, 0, threads * sizeof(int), st));
        CK(cudaMemcpyAsync(ctx->d_params.p, &P, sizeof(Params), cudaMemcpyHostToDevice, st));
        for (long long round = 0;; ++round) {
            CK(cudaMemsetAsync(ctl, 0, 4 * sizeof(unsigned long long), st));
            CK(walk_propagate(P, din, dout, tr, grid, block, st));
            CK(walk_peel(P, ctx->sms, st));
            unsigned int parked = 0, aborted = 0;
            CK(cudaMemcpyAsync(&parked, P.suspended, sizeof(parked), cudaMemcpyDeviceToHost, st));
            if (P.limits) CK(cudaMemcpyAsync(&aborted, P.abort_flag, sizeof(aborted), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (aborted) break;
            if (parked == 0) break;
            if (round > (1LL << 30)) return fail(ctx, RASCAS_E_STATE, "propagate: peeling rounds do not end");
        }
    } else {
        CK(cudaMemcpyAsync(ctx->d_params.p, &P, sizeof(Params), cudaMemcpyHostToDevice, st));
        if (n > 0) {
            int grid = persistent_grid(ctx, false);
            CK(walk_propagate(P, din, dout, tr, grid, rg::propagate_block_size(), st));
        }
    }
    if (stats) CK(cudaEventRecord(e1, st));
    if (mem == RASCAS_HOST && n > 0) {
        if (out) {
            if (out->status) CK(cudaMemcpyAsync(out->status, dout.status, N * 4, cudaMemcpyDeviceToHost, st));
            if (out->nscatt) CK(cudaMemcpyAsync(out->nscatt, dout.nscatt, N * 8, cudaMemcpyDeviceToHost, st));
            if (out->nu) CK(cudaMemcpyAsync(out->nu, dout.nu, N * 8, cudaMemcpyDeviceToHost, st));
            if (out->pos) CK(cudaMemcpyAsync(out->pos, dout.pos, 3 * N * 8, cudaMemcpyDeviceToHost, st));
            if (out->dir) CK(cudaMemcpyAsync(out->dir, dout.dir, 3 * N * 8, cudaMemcpyDeviceToHost, st));
            if (out->path) CK(cudaMemcpyAsync(out->path, dout.path, N * 8, cudaMemcpyDeviceToHost, st));
        }
        if (events) {
            CK(cudaMemcpyAsync(events, tr.ev, N * (size_t)max_events * sizeof(rg::TraceEvent), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(nevents, tr.nev, N * 4, cudaMemcpyDeviceToHost, st));
        }
    }
    unsigned long long cnt[rg::kCounterWords] = {};
    if (stats || mem == RASCAS_HOST || ctx->phys.fail_on_cap || P.limits) {
        CK(cudaMemcpyAsync(cnt, ctx->d_counters.p, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (stats) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        stats->packets = (int64_t)cnt[rg::CNT_PACKETS];
        stats->escaped = (int64_t)cnt[rg::CNT_ESCAPED];
        stats->absorbed = (int64_t)cnt[rg::CNT_ABSORBED];
        stats->capped = (int64_t)cnt[rg::CNT_CAPPED];
        stats->errors = (int64_t)cnt[rg::CNT_ERRORS];
        stats->nscatt_line = (int64_t)cnt[rg::CNT_SCATT_LINE];
        stats->nscatt_dust = (int64_t)cnt[rg::CNT_SCATT_DUST];
        stats->ncross = (int64_t)cnt[rg::CNT_CROSS];
        stats->npeel_rays = (int64_t)cnt[rg::CNT_PEEL_RAYS];
        stats->npeel_cells = (int64_t)cnt[rg::CNT_PEEL_CELLS];
        stats->upar_trials = (int64_t)cnt[rg::CNT_UPAR_TRIALS];
        stats->leaf_loads = (int64_t)cnt[rg::CNT_LEAF_LOADS];
        stats->son_loads = (int64_t)cnt[rg::CNT_SON_LOADS];
        stats->nbor_loads = (int64_t)cnt[rg::CNT_NBOR_LOADS];
        stats->kernel_ms = ms;
    }
    if (P.limits && cnt[rg::CNT_N + 1] != 0)
        return fail(ctx, RASCAS_E_TIMEOUT, "propagate: a device iteration or time limit was reached (rascas_set_limits)");
    if (ctx->phys.fail_on_cap && cnt[rg::CNT_CAPPED] > 0)
        return fail(ctx, RASCAS_E_CAPPED, "some packets reached a cap");
    return RASCAS_OK;
}

}  // namespace

extern "C" {

int rascas_propagate(rascas_ctx* ctx, const rascas_packets_in* in, int64_t n, const rascas_packets_out* out, int mem,
                     rascas_run_stats* stats) {
    return run_propagate(ctx, in, n, out, mem, stats, nullptr, nullptr, 0, true);
}

int rascas_trace(rascas_ctx* ctx, const rascas_packets_in* in, int64_t n, int32_t max_events, rascas_event* events,
                 int32_t* nevents, int mem) {
    if (!ctx || max_events < 1 || !events || !nevents) return fail(ctx, RASCAS_E_ARG, "trace: bad arguments");
    static_assert(sizeof(rascas_event) == sizeof(rg::TraceEvent), "event layout");
    return run_propagate(ctx, in, n, nullptr, mem, nullptr, events, nevents, max_events, false);
}

int rascas_get_tally(rascas_ctx* ctx, int kind, float* dst, size_t count, int mem) {
    if (!ctx || !dst) return RASCAS_E_ARG;
    if (!ctx->has_det) return fail(ctx, RASCAS_E_STATE, "no detector set");
    const rascas_detector& d = ctx->det;
    size_t npix2 = (size_t)d.npix * d.npix;
    const void* src = nullptr;
    size_t need = 0;
    switch (kind) {
        case RASCAS_TALLY_SPECTRUM: src = ctx->d_spec.p; need = d.nbin; break;
        case RASCAS_TALLY_PEEL_SPECTRA: src = ctx->d_pspec.p; need = (size_t)d.ndir * d.nbin; break;
        case RASCAS_TALLY_PEEL_IMAGES: src = ctx->d_pimg.p; need = (size_t)d.ndir * npix2; break;
        case RASCAS_TALLY_PEEL_CUBES: src = ctx->P.cube ? ctx->d_pcube.p : nullptr; need = (size_t)d.ndir * npix2 * d.nbin; break;
        default: return fail(ctx, RASCAS_E_ARG, "tally: unknown kind");
    }
    if (!src || need == 0) return fail(ctx, RASCAS_E_STATE, "tally: not accumulated by this detector");
    if (count != need) return fail(ctx, RASCAS_E_ARG, "tally: count does not match the detector shape");
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpyAsync(dst, src, need * 4, mem == RASCAS_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    if (mem != RASCAS_DEVICE) CK(cudaStreamSynchronize(ctx->stream));
    return RASCAS_OK;
}

int rascas_ray_tau(rascas_ctx* ctx, int64_t n, const double* pos, const double* dir, const double* nu, double* tau,
                   int32_t* cells, double* lens, int32_t cap, int32_t* ncell, int mem) {
    if (!ctx || n < 0 || !pos || !dir || !nu || !tau || cap < 0 || ((cells || lens) && (!cells || !lens || cap == 0)))
        return fail(ctx, RASCAS_E_ARG, "ray_tau: bad arguments");
    int r = check_ready(ctx);
    if (r) return r;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n;
    if (n == 0) return RASCAS_OK;
    const double *dpos = pos, *ddir = dir, *dnu = nu;
    double *dtau = tau, *dlens = lens;
    int32_t *dcells = cells, *dncell = ncell;
    if (mem == RASCAS_HOST) {
        size_t b = N * 8 * 8 + N * 4 + (cells ? N * (size_t)cap * 12 : 0) + 64;
        CK(ctx->stage_aux.ensure(b));
        char* p = (char*)ctx->stage_aux.p;
        double* a = (double*)p;
        dpos = a; ddir = a + 3 * N; dnu = a + 6 * N; dtau = a + 7 * N;
        dncell = (int32_t*)(a + 8 * N);
        char* q = (char*)(dncell + N);
        q = (char*)(((uintptr_t)q + 15) & ~(uintptr_t)15);
        dlens = cells ? (double*)q : nullptr;
        dcells = cells ? (int32_t*)(q + N * (size_t)cap * 8) : nullptr;
        CK(cudaMemcpyAsync((void*)dpos, pos, 3 * N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)ddir, dir, 3 * N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)dnu, nu, N * 8, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(ctx->d_params.p, &ctx->P, sizeof(Params), cudaMemcpyHostToDevice, st));
    CK(ctx->ray_init.ensure(N * sizeof(rg::RayInit)));
    CK(cudaMemsetAsync(ctx->P.head, 0, sizeof(unsigned long long), st));
    CK(walk_ray_tau(ctx->P, (long long)n, dpos, ddir, dnu, dtau, dcells, dlens, cap,
                          (mem == RASCAS_HOST || ncell) ? dncell : nullptr, (rg::RayInit*)ctx->ray_init.p, ctx->sms,
                          st));
    if (mem == RASCAS_HOST) {
        CK(cudaMemcpyAsync(tau, dtau, N * 8, cudaMemcpyDeviceToHost, st));
        if (ncell) CK(cudaMemcpyAsync(ncell, dncell, N * 4, cudaMemcpyDeviceToHost, st));
        if (cells) {
            CK(cudaMemcpyAsync(cells, dcells, N * (size_t)cap * 4, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(lens, dlens, N * (size_t)cap * 8, cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
    }
    return RASCAS_OK;
}

int rascas_ray_columns(rascas_ctx* ctx, int64_t n, const double* pos, const double* dir, double sigma_HI,
                       double sigma_dust, double* cols, double* tau, int32_t* ncell, int mem) {
    if (!ctx || n < 0 || !pos || !dir || !cols || !(sigma_HI >= 0.0) || !(sigma_dust >= 0.0) ||
        (mem != RASCAS_HOST && mem != RASCAS_DEVICE))
        return fail(ctx, RASCAS_E_ARG, "ray_columns: bad arguments");
    if (!ctx->has_mesh) return fail(ctx, RASCAS_E_STATE, "no octree loaded");
    if (!ctx->has_domain) return fail(ctx, RASCAS_E_STATE, "no domain set");
    CK(cudaSetDevice(ctx->device));
    if (n == 0) return RASCAS_OK;
    cudaStream_t st = ctx->stream;
    const size_t N = (size_t)n;
    const double *dpos = pos, *ddir = dir;
    double *dcols = cols, *dtau = tau;
    int32_t* dncell = ncell;
    if (mem == RASCAS_HOST) {
        CK(ctx->stage_aux.ensure(N * (3 + 3 + 3 + 1) * 8 + N * 4 + 64));
        double* a = (double*)ctx->stage_aux.p;
        dpos = a; ddir = a + 3 * N; dcols = a + 6 * N; dtau = tau ? a + 9 * N : nullptr;
        dncell = ncell ? (int32_t*)(a + 10 * N) : nullptr;
        CK(cudaMemcpyAsync((void*)dpos, pos, 3 * N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync((void*)ddir, dir, 3 * N * 8, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(ctx->d_params.p, &ctx->P, sizeof(Params), cudaMemcpyHostToDevice, st));
    CK(ctx->ray_init.ensure(N * sizeof(rg::RayInit)));
    CK(cudaMemsetAsync(ctx->P.head, 0, sizeof(unsigned long long), st));
    CK(rg::launch_ray_columns(ctx->P, (long long)n, dpos, ddir, dcols, dtau, sigma_HI, sigma_dust, dncell,
                              (rg::RayInit*)ctx->ray_init.p, ctx->sms, st));
    if (mem == RASCAS_HOST) {
        CK(cudaMemcpyAsync(cols, dcols, 3 * N * 8, cudaMemcpyDeviceToHost, st));
        if (tau) CK(cudaMemcpyAsync(tau, dtau, N * 8, cudaMemcpyDeviceToHost, st));
        if (ncell) CK(cudaMemcpyAsync(ncell, dncell, N * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return RASCAS_OK;
}

int rascas_probe_issue_rates(rascas_ctx* ctx, double* rates) {
    if (!ctx || !rates) return fail(ctx, RASCAS_E_ARG, "probe_issue_rates: bad arguments");
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    DevBuf scratch;
    CK(scratch.ensure(4096));
    cudaError_t e = rg::probe_issue_rates(ctx->sms, scratch.p, rates);
    scratch.release();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "probe_issue_rates");
    return RASCAS_OK;
}

int rascas_eval_voigt(rascas_ctx* ctx, int64_t n, const float* a, const double* x, float* H, int mem) {
    if (!ctx || n < 0 || !a || !x || !H) return fail(ctx, RASCAS_E_ARG, "eval_voigt: bad arguments");
    CK(cudaSetDevice(ctx->device));
    const size_t N = (size_t)n;
    if (n == 0) return RASCAS_OK;
    cudaStream_t st = ctx->stream;
    if (mem == RASCAS_HOST) {
        CK(ctx->stage_aux.ensure(N * 16 + 64));
        double* dx = (double*)ctx->stage_aux.p;
        float* da = (float*)(dx + N);
        float* dH = da + N;
        CK(cudaMemcpyAsync(dx, x, N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(da, a, N * 4, cudaMemcpyHostToDevice, st));
        CK(rg::launch_eval_voigt((long long)n, da, dx, dH, ctx->P.voigt, st));
        CK(cudaMemcpyAsync(H, dH, N * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return RASCAS_OK;
    }
    CK(rg::launch_eval_voigt((long long)n, a, x, H, ctx->P.voigt, st));
    return RASCAS_OK;
}

int rascas_sample_upar(rascas_ctx* ctx, int64_t n, const double* x, const float* a, const uint64_t* id, float* u,
                       int32_t* ndraw, int mem) {
    if (!ctx || n < 0 || !x || !a || !id || !u || !ndraw) return fail(ctx, RASCAS_E_ARG, "sample_upar: bad arguments");
    if (!ctx->has_phys) return fail(ctx, RASCAS_E_STATE, "no physics set");
    CK(cudaSetDevice(ctx->device));
    const size_t N = (size_t)n;
    if (n == 0) return RASCAS_OK;
    cudaStream_t st = ctx->stream;
    if (mem == RASCAS_HOST) {
        CK(ctx->stage_aux.ensure(N * 28 + 64));
        double* dx = (double*)ctx->stage_aux.p;
        uint64_t* did = (uint64_t*)(dx + N);
        float* da = (float*)(did + N);
        float* du = da + N;
        int32_t* dn = (int32_t*)(du + N);
        CK(cudaMemcpyAsync(dx, x, N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(did, id, N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(da, a, N * 4, cudaMemcpyHostToDevice, st));
        CK(rg::launch_sample_upar(ctx->P, (long long)n, dx, da, did, du, dn, st));
        CK(cudaMemcpyAsync(u, du, N * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ndraw, dn, N * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return RASCAS_OK;
    }
    CK(rg::launch_sample_upar(ctx->P, (long long)n, x, a, id, u, ndraw, st));
    return RASCAS_OK;
}

int rascas_propagate_noalloc(rascas_ctx* ctx, const rascas_packets_in* in, int64_t n,
                             const rascas_packets_out* out, rascas_run_stats* stats) {
    if (!ctx || !in || n < 0) return fail(ctx, RASCAS_E_ARG, "propagate_noalloc: bad arguments");
    if (n > RASCAS_NOALLOC_MAX_PACKETS)
        return fail(ctx, RASCAS_E_ARG,
                    "propagate_noalloc: n exceeds RASCAS_NOALLOC_MAX_PACKETS (" +
                        std::to_string(RASCAS_NOALLOC_MAX_PACKETS) + "); split the packet list");
    if (n > 0 && (!in->pos || !in->dir || !in->nu || !in->id)) return fail(ctx, RASCAS_E_ARG, "packets: null array");
    int r = check_ready(ctx);
    if (r) return r;
    CK(cudaSetDevice(ctx->device));
    char* base = (char*)ctx->noalloc_base;
    const size_t bytes = ctx->noalloc_bytes;
    // layout: counters, queue head, abort flag | parameter copy | packet staging
    const size_t N = (size_t)n;
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    size_t off = 0;
    unsigned long long* cnt_d = (unsigned long long*)(base + off);
    off += al(sizeof(unsigned long long) * rg::kCounterWords);
    Params* par_d = (Params*)(base + off);
    off += al(sizeof(Params));
    double* pos = (double*)(base + off); off += al(3 * N * 8);
    double* dir = (double*)(base + off); off += al(3 * N * 8);
    double* nu = (double*)(base + off); off += al(N * 8);
    uint64_t* id = (uint64_t*)(base + off); off += al(N * 8);
    int32_t* ost = (int32_t*)(base + off); off += al(N * 4);
    int64_t* ons = (int64_t*)(base + off); off += al(N * 8);
    double* onu = (double*)(base + off); off += al(N * 8);
    double* opos = (double*)(base + off); off += al(3 * N * 8);
    double* odir = (double*)(base + off); off += al(3 * N * 8);
    double* opath = (double*)(base + off); off += al(N * 8);
    if (off > bytes) return fail(ctx, RASCAS_E_ARG, "propagate_noalloc: scratch layout exceeds the static array");
    Params P = ctx->P;
    P.g.spec = nullptr;   // per-packet outputs only: no tallies, no peeling
    P.ndir = 0;
    P.counters = cnt_d;
    P.head = cnt_d + rg::CNT_N;
    P.abort_flag = (unsigned int*)(cnt_d + rg::CNT_N + 1);
    P.self = par_d;
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(cnt_d, 0, sizeof(unsigned long long) * rg::kCounterWords, st));
    CK(cudaMemcpyAsync(par_d, &P, sizeof(Params), cudaMemcpyHostToDevice, st));
    rg::PacketsIn din{pos, dir, nu, id, (long long)n, 0};
    rg::PacketsOut dout{};
    if (out) dout = rg::PacketsOut{out->status ? ost : nullptr, out->nscatt ? ons : nullptr, out->nu ? onu : nullptr,
                                   out->pos ? opos : nullptr, out->dir ? odir : nullptr, out->path ? opath : nullptr};
    rg::TraceOut tr{nullptr, nullptr, 0};
    if (n > 0) {
        CK(cudaMemcpyAsync(pos, in->pos, 3 * N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dir, in->dir, 3 * N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(nu, in->nu, N * 8, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(id, in->id, N * 8, cudaMemcpyHostToDevice, st));
        CK(walk_propagate(P, din, dout, tr, persistent_grid(ctx, false), rg::propagate_block_size(), st));
        if (out) {
            if (out->status) CK(cudaMemcpyAsync(out->status, ost, N * 4, cudaMemcpyDeviceToHost, st));
            if (out->nscatt) CK(cudaMemcpyAsync(out->nscatt, ons, N * 8, cudaMemcpyDeviceToHost, st));
            if (out->nu) CK(cudaMemcpyAsync(out->nu, onu, N * 8, cudaMemcpyDeviceToHost, st));
            if (out->pos) CK(cudaMemcpyAsync(out->pos, opos, 3 * N * 8, cudaMemcpyDeviceToHost, st));
            if (out->dir) CK(cudaMemcpyAsync(out->dir, odir, 3 * N * 8, cudaMemcpyDeviceToHost, st));
            if (out->path) CK(cudaMemcpyAsync(out->path, opath, N * 8, cudaMemcpyDeviceToHost, st));
        }
    }
    unsigned long long cnt[rg::kCounterWords] = {};
    CK(cudaMemcpyAsync(cnt, cnt_d, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->packets = (int64_t)cnt[rg::CNT_PACKETS];
        stats->escaped = (int64_t)cnt[rg::CNT_ESCAPED];
        stats->absorbed = (int64_t)cnt[rg::CNT_ABSORBED];
        stats->capped = (int64_t)cnt[rg::CNT_CAPPED];
        stats->errors = (int64_t)cnt[rg::CNT_ERRORS];
        stats->nscatt_line = (int64_t)cnt[rg::CNT_SCATT_LINE];
        stats->nscatt_dust = (int64_t)cnt[rg::CNT_SCATT_DUST];
        stats->ncross = (int64_t)cnt[rg::CNT_CROSS];
        stats->upar_trials = (int64_t)cnt[rg::CNT_UPAR_TRIALS];
        stats->leaf_loads = (int64_t)cnt[rg::CNT_LEAF_LOADS];
        stats->son_loads = (int64_t)cnt[rg::CNT_SON_LOADS];
        stats->nbor_loads = (int64_t)cnt[rg::CNT_NBOR_LOADS];
    }
    if (P.limits && cnt[rg::CNT_N + 1] != 0)
        return fail(ctx, RASCAS_E_TIMEOUT, "propagate_noalloc: a device iteration or time limit was reached");
    if (ctx->phys.fail_on_cap && cnt[rg::CNT_CAPPED] > 0)
        return fail(ctx, RASCAS_E_CAPPED, "some packets reached a cap");
    return RASCAS_OK;
}

int rascas_load_batch(rascas_ctx* ctx, const rascas_model* models, int32_t nmodels, int32_t nbin, int mem) {
    if (!ctx || !models || nmodels < 1 || nbin < 1 || (mem != RASCAS_HOST && mem != RASCAS_DEVICE))
        return fail(ctx, RASCAS_E_ARG, "load_batch: bad arguments");
    if (!ctx->has_lines) return fail(ctx, RASCAS_E_STATE, "load_batch: set the lines first");
    CK(cudaSetDevice(ctx->device));
    auto& B = ctx->batch;
    const Params& P = ctx->P;
    std::vector<HostMesh> meshes(nmodels);
    std::vector<double> cost(nmodels, 0.0);
    for (int m = 0; m < nmodels; ++m) {
        const rascas_model& md = models[m];
        if (md.domain.kind < 0 || md.domain.kind > 3 || !(md.domain.size > 0.0) || !(md.nu_hi > md.nu_lo) ||
            (md.domain.kind == RASCAS_DOMAIN_SHELL && !(md.domain.inner >= 0.0 && md.domain.inner < md.domain.size)) ||
            md.npackets < 0 || (md.npackets > 0 && (!md.packets.pos || !md.packets.dir || !md.packets.nu ||
                                                   !md.packets.id)))
            return fail(ctx, RASCAS_E_ARG, "load_batch: model " + std::to_string(m) + ": bad domain, axis or packets");
        cudaError_t ce;
        const char* err = build_mesh(&md.tree, mem, meshes[m], ce);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "load_batch");
        if (err) return fail(ctx, RASCAS_E_ARG, "load_batch: model " + std::to_string(m) + ": " + err);
        for (int i = 0; i < P.nline; ++i)
            if (P.line[i].dens == 1 && !meshes[m].has_metal)
                return fail(ctx, RASCAS_E_STATE, "load_batch: a line needs n_metal but a model has none");
        mesh_flags(meshes[m], &md.domain);
        // expected scatterings per packet grow with the line-centre optical
        // depth across the domain: schedule the costliest models first
        double t = 0.0;
        const HostMesh& M = meshes[m];
        for (int i = 0; i < M.nleaf; ++i) {
            double n = M.rec[8 * (size_t)i], T = std::fmax((double)M.rec[8 * (size_t)i + 4], 1e-30);
            t = std::fmax(t, n * P.line[0].abund * P.line[0].sig_pref / std::sqrt(T));
        }
        cost[m] = t * md.domain.size * M.box_cm;
    }
    B.order.resize(nmodels);
    for (int m = 0; m < nmodels; ++m) B.order[m] = m;
    std::stable_sort(B.order.begin(), B.order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    // concatenate meshes and packets in scheduled order
    size_t nrec = 0, nson = 0, nnbr = 0, ntop = 0;
    long long npk = 0;
    B.first.assign(nmodels + 1, 0);
    for (int k = 0; k < nmodels; ++k) {
        const HostMesh& M = meshes[B.order[k]];
        nrec += M.rec.size(); nson += M.son.size(); nnbr += M.nbr.size(); ntop += M.top.size();
        npk += models[B.order[k]].npackets;
        B.first[k + 1] = npk;
    }
    CK(B.d_rec.ensure(nrec * 4)); CK(B.d_son.ensure(nson * 4)); CK(B.d_nbr.ensure(nnbr * 4));
    CK(B.d_top.ensure(ntop * 4)); CK(B.d_geo.ensure(sizeof(rg::Geo) * nmodels));
    CK(B.d_first.ensure(sizeof(long long) * (nmodels + 1)));
    CK(B.d_spec.ensure(sizeof(float) * (size_t)nmodels * nbin));
    size_t pk_bytes = (size_t)(npk > 0 ? npk : 1) * 8;
    CK(B.d_pos.ensure(3 * pk_bytes)); CK(B.d_dir.ensure(3 * pk_bytes));
    CK(B.d_nu.ensure(pk_bytes)); CK(B.d_id.ensure(pk_bytes));
    std::vector<rg::Geo> geo(nmodels);
    size_t orec = 0, oson = 0, onbr = 0, otop = 0;
    for (int k = 0; k < nmodels; ++k) {
        int m = B.order[k];
        const HostMesh& M = meshes[m];
        const rascas_model& md = models[m];
        char* drec = (char*)B.d_rec.p + orec * 4;
        char* dson = (char*)B.d_son.p + oson * 4;
        char* dnbr = (char*)B.d_nbr.p + onbr * 4;
        char* dtop = (char*)B.d_top.p + otop * 4;
        CK(cudaMemcpy(drec, M.rec.data(), M.rec.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dson, M.son.data(), M.son.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dnbr, M.nbr.data(), M.nbr.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dtop, M.top.data(), M.top.size() * 4, cudaMemcpyHostToDevice));
        rg::Geo& G = geo[k];
        G.rec = (const float4*)drec; G.son = (const int*)dson; G.nbr = (const int4*)dnbr; G.top = (const int4*)dtop;
        G.top_level = M.top_level; G.max_level = M.max_level; G.nleaf = M.nleaf; G.noct = M.noct;
        G.box_cm = M.box_cm; G.box_cm_f = (float)M.box_cm;
        G.dom_kind = md.domain.kind;
        for (int ax = 0; ax < 3; ++ax) G.dom_c[ax] = md.domain.centre[ax];
        G.dom_R = md.domain.size;
        G.dom_Rin = md.domain.kind == RASCAS_DOMAIN_SHELL ? md.domain.inner : 0.0;
        G.nu_lo = md.nu_lo; G.nu_range = md.nu_hi - md.nu_lo; G.nbin = nbin;
        G.spec = (float*)B.d_spec.p + (size_t)m * nbin;
        orec += M.rec.size(); oson += M.son.size(); onbr += M.nbr.size(); otop += M.top.size();
        const size_t n = (size_t)md.npackets, o = (size_t)B.first[k];
        if (n > 0) {
            cudaMemcpyKind kind = mem == RASCAS_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            CK(cudaMemcpy((double*)B.d_pos.p + 3 * o, md.packets.pos, 3 * n * 8, kind));
            CK(cudaMemcpy((double*)B.d_dir.p + 3 * o, md.packets.dir, 3 * n * 8, kind));
            CK(cudaMemcpy((double*)B.d_nu.p + o, md.packets.nu, n * 8, kind));
            CK(cudaMemcpy((uint64_t*)B.d_id.p + o, md.packets.id, n * 8, kind));
        }
    }
    CK(cudaMemcpy(B.d_geo.p, geo.data(), sizeof(rg::Geo) * nmodels, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(B.d_first.p, B.first.data(), sizeof(long long) * (nmodels + 1), cudaMemcpyHostToDevice));
    B.nmodels = nmodels;
    B.nbin = nbin;
    B.npackets = npk;
    B.nline_at_load = P.nline;
    ++ctx->version;
    return RASCAS_OK;
}

}  // extern "C"

namespace {

void fill_stats(rascas_run_stats* stats, const unsigned long long* cnt, double ms) {
    std::memset(stats, 0, sizeof(*stats));
    stats->packets = (int64_t)cnt[rg::CNT_PACKETS];
    stats->escaped = (int64_t)cnt[rg::CNT_ESCAPED];
    stats->absorbed = (int64_t)cnt[rg::CNT_ABSORBED];
    stats->capped = (int64_t)cnt[rg::CNT_CAPPED];
    stats->errors = (int64_t)cnt[rg::CNT_ERRORS];
    stats->nscatt_line = (int64_t)cnt[rg::CNT_SCATT_LINE];
    stats->nscatt_dust = (int64_t)cnt[rg::CNT_SCATT_DUST];
    stats->ncross = (int64_t)cnt[rg::CNT_CROSS];
    stats->upar_trials = (int64_t)cnt[rg::CNT_UPAR_TRIALS];
    stats->leaf_loads = (int64_t)cnt[rg::CNT_LEAF_LOADS];
    stats->son_loads = (int64_t)cnt[rg::CNT_SON_LOADS];
    stats->nbor_loads = (int64_t)cnt[rg::CNT_NBOR_LOADS];
    stats->kernel_ms = ms;
}

// the batch run; `out` (device buffers in scheduled order, or all null) gets
// per-packet results, in which case the persistent launch is made directly
// rather than from the captured graph
int run_batch(rascas_ctx* ctx, int32_t mode, const rg::PacketsOut& out, rascas_run_stats* stats) {
    if (!ctx || (mode != RASCAS_BATCH_PERSISTENT && mode != RASCAS_BATCH_PER_MODEL))
        return fail(ctx, RASCAS_E_ARG, "propagate_batch: bad arguments");
    auto& B = ctx->batch;
    if (B.nmodels < 1) return fail(ctx, RASCAS_E_STATE, "propagate_batch: no batch loaded");
    if (!ctx->has_lines || !ctx->has_phys) return fail(ctx, RASCAS_E_STATE, "propagate_batch: lines or physics unset");
    if (B.nline_at_load != ctx->P.nline) return fail(ctx, RASCAS_E_STATE, "propagate_batch: lines changed since load_batch");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    if (!st) {
        if (!ctx->own_stream) CK(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking));
        st = ctx->own_stream;
    }
    Params P = ctx->P;
    P.ndir = 0;
    P.g.spec = nullptr;
    P.models = (const rg::Geo*)B.d_geo.p;
    P.model_first = (const long long*)B.d_first.p;
    P.nmodels = B.nmodels;
    P.refill = B.refill;
    rg::PacketsIn in{(const double*)B.d_pos.p, (const double*)B.d_dir.p, (const double*)B.d_nu.p,
                     (const uint64_t*)B.d_id.p, B.npackets, 0};
    rg::TraceOut tr{nullptr, nullptr, 0};
    const bool direct = out.status || out.nscatt || out.nu || out.pos || out.dir || out.path;
    const int block = B.block;
    int per_sm = B.blocks_per_sm > 0 ? B.blocks_per_sm : rg::propagate_batch_blocks_per_sm(P.nline, block);
    if (per_sm < 1) per_sm = 1;
    const int grid = ctx->sms * per_sm;
    const size_t cnt_bytes = sizeof(unsigned long long) * rg::kCounterWords;
    const size_t spec_bytes = sizeof(float) * (size_t)B.nmodels * B.nbin;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, st));
    if (mode == RASCAS_BATCH_PERSISTENT && !direct) {
        // one persistent launch over every model's packets, replayed from a
        // captured CUDA graph (re-captured when the set-up or shape changed)
        unsigned long long key = ctx->version * 1000003ULL +
                                 (unsigned long long)((block * 64 + per_sm) * 4096 + B.refill);
        if (!B.graph || B.graph_key != key || B.graph_stream != st) {
            if (B.graph) {
                cudaGraphExecDestroy(B.graph);
                B.graph = nullptr;
            }
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            cudaError_t e1c = cudaMemsetAsync(ctx->d_counters.p, 0, cnt_bytes, st);
            cudaError_t e2c = cudaMemsetAsync(B.d_spec.p, 0, spec_bytes, st);
            cudaError_t e3c = walk_propagate(P, in, out, tr, grid, block, st);
            cudaError_t ec = cudaStreamEndCapture(st, &g);
            if (e1c != cudaSuccess || e2c != cudaSuccess || e3c != cudaSuccess || ec != cudaSuccess)
                return cuda_fail(ctx, ec != cudaSuccess ? ec : (e3c != cudaSuccess ? e3c : e1c), "batch graph capture");
            cudaError_t ei = cudaGraphInstantiate(&B.graph, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) return cuda_fail(ctx, ei, "cudaGraphInstantiate");
            B.graph_key = key;
            B.graph_stream = st;
        }
        CK(cudaGraphLaunch(B.graph, st));
    } else if (mode == RASCAS_BATCH_PERSISTENT) {
        CK(cudaMemsetAsync(ctx->d_counters.p, 0, cnt_bytes, st));
        CK(cudaMemsetAsync(B.d_spec.p, 0, spec_bytes, st));
        CK(walk_propagate(P, in, out, tr, grid, block, st));
    } else {
        // the plain alternative: one launch per model, in sequence
        CK(cudaMemsetAsync(ctx->d_counters.p, 0, cnt_bytes, st));
        CK(cudaMemsetAsync(B.d_spec.p, 0, spec_bytes, st));
        for (int k = 0; k < B.nmodels; ++k) {
            long long n = B.first[k + 1] - B.first[k];
            if (n <= 0) continue;
            Params Pk = P;
            Pk.models = (const rg::Geo*)B.d_geo.p + k;
            Pk.model_first = (const long long*)B.d_first.p + k;
            Pk.nmodels = 1;
            rg::PacketsIn ink = in;
            ink.first = B.first[k];
            ink.n = B.first[k + 1];
            long long blocks = (n + (long long)block * Pk.refill - 1) / ((long long)block * Pk.refill);
            int gk = (int)(blocks < grid ? blocks : grid);
            CK(cudaMemsetAsync(P.head, 0, sizeof(unsigned long long), st));
            CK(walk_propagate(Pk, ink, out, tr, gk, block, st));
        }
    }
    CK(cudaEventRecord(e1, st));
    unsigned long long cnt[rg::kCounterWords] = {};
    CK(cudaMemcpyAsync(cnt, ctx->d_counters.p, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (stats) fill_stats(stats, cnt, ms);
    if (P.limits && cnt[rg::CNT_N + 1] != 0)
        return fail(ctx, RASCAS_E_TIMEOUT, "propagate_batch: a device iteration or time limit was reached");
    return RASCAS_OK;
}

}  // namespace

extern "C" {

int rascas_propagate_batch(rascas_ctx* ctx, int32_t mode, rascas_run_stats* stats) {
    return run_batch(ctx, mode, rg::PacketsOut{}, stats);
}

int rascas_propagate_batch_packets(rascas_ctx* ctx, int32_t mode, const rascas_packets_out* out, int mem,
                                   rascas_run_stats* stats) {
    if (!ctx || !out || (mem != RASCAS_HOST && mem != RASCAS_DEVICE))
        return fail(ctx, RASCAS_E_ARG, "propagate_batch_packets: bad arguments");
    auto& B = ctx->batch;
    if (B.nmodels < 1) return fail(ctx, RASCAS_E_STATE, "propagate_batch_packets: no batch loaded");
    CK(cudaSetDevice(ctx->device));
    // results land in scheduled order on the device, then move per model to
    // the caller's order (models as given to rascas_load_batch)
    const size_t N = (size_t)(B.npackets > 0 ? B.npackets : 1);
    CK(ctx->stage_out.ensure(N * (4 + 8 + 8 + 24 + 24 + 8) + 64));
    char* o = (char*)ctx->stage_out.p;
    double* onu = (double*)o;
    double* opos = onu + N;
    double* odir = opos + 3 * N;
    double* opath = odir + 3 * N;
    int64_t* ons = (int64_t*)(opath + N);
    int32_t* ost = (int32_t*)(ons + N);
    rg::PacketsOut dout{out->status ? ost : nullptr, out->nscatt ? ons : nullptr, out->nu ? onu : nullptr,
                        out->pos ? opos : nullptr, out->dir ? odir : nullptr, out->path ? opath : nullptr};
    if (!(dout.status || dout.nscatt || dout.nu || dout.pos || dout.dir || dout.path))
        return fail(ctx, RASCAS_E_ARG, "propagate_batch_packets: no output array");
    int r = run_batch(ctx, mode, dout, stats);
    if (r != RASCAS_OK && r != RASCAS_E_TIMEOUT) return r;
    cudaStream_t st = ctx->stream ? ctx->stream : ctx->own_stream;
    const cudaMemcpyKind kind = mem == RASCAS_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    // caller offset of each model: prefix sums over the models in given order
    std::vector<long long> off_given(B.nmodels + 1, 0);
    std::vector<long long> count(B.nmodels, 0);
    for (int k = 0; k < B.nmodels; ++k) count[B.order[k]] = B.first[k + 1] - B.first[k];
    for (int m = 0; m < B.nmodels; ++m) off_given[m + 1] = off_given[m] + count[m];
    for (int k = 0; k < B.nmodels; ++k) {
        const size_t src = (size_t)B.first[k], n = (size_t)(B.first[k + 1] - B.first[k]);
        const size_t dst = (size_t)off_given[B.order[k]];
        if (n == 0) continue;
        if (out->status) CK(cudaMemcpyAsync(out->status + dst, ost + src, n * 4, kind, st));
        if (out->nscatt) CK(cudaMemcpyAsync(out->nscatt + dst, ons + src, n * 8, kind, st));
        if (out->nu) CK(cudaMemcpyAsync(out->nu + dst, onu + src, n * 8, kind, st));
        if (out->pos) CK(cudaMemcpyAsync(out->pos + 3 * dst, opos + 3 * src, 3 * n * 8, kind, st));
        if (out->dir) CK(cudaMemcpyAsync(out->dir + 3 * dst, odir + 3 * src, 3 * n * 8, kind, st));
        if (out->path) CK(cudaMemcpyAsync(out->path + dst, opath + src, n * 8, kind, st));
    }
    CK(cudaStreamSynchronize(st));
    return r;
}

int rascas_get_batch_spectra(rascas_ctx* ctx, float* dst, size_t count, int mem) {
    if (!ctx || !dst) return RASCAS_E_ARG;
    auto& B = ctx->batch;
    if (B.nmodels < 1) return fail(ctx, RASCAS_E_STATE, "get_batch_spectra: no batch loaded");
    if (count != (size_t)B.nmodels * B.nbin) return fail(ctx, RASCAS_E_ARG, "get_batch_spectra: count != nmodels*nbin");
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpy(dst, B.d_spec.p, count * 4, mem == RASCAS_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return RASCAS_OK;
}

int rascas_autotune_batch(rascas_ctx* ctx, int64_t max_scatt, rascas_tune* best, rascas_tune* tried, int32_t max_tried,
                          int32_t* ntried) {
    if (!ctx || max_scatt < 1) return fail(ctx, RASCAS_E_ARG, "autotune_batch: bad arguments");
    auto& B = ctx->batch;
    if (B.nmodels < 1) return fail(ctx, RASCAS_E_STATE, "autotune_batch: no batch loaded");
    const long long saved_scatt = ctx->P.max_scatt;
    const int saved_block = B.block, saved_per_sm = B.blocks_per_sm, saved_refill = B.refill;
    ctx->P.max_scatt = max_scatt;   // short runs of the same batch, each packet capped
    ++ctx->version;
    rascas_tune bt{0, 0, 0, 0.0};
    int nt = 0;
    int rc = RASCAS_OK;
    auto trial = [&](int block, int per_sm, int refill) {
        B.block = block;
        B.blocks_per_sm = per_sm;
        B.refill = refill;
        rascas_run_stats st;
        rc = rascas_propagate_batch(ctx, RASCAS_BATCH_PERSISTENT, &st);
        if (rc != RASCAS_OK) return;
        rascas_tune t{block, per_sm, refill, st.kernel_ms};
        if (tried && nt < max_tried) tried[nt] = t;
        ++nt;
        if (bt.ms == 0.0 || t.ms < bt.ms) bt = t;
    };
    // launch shape first (one packet per grab), then the refill granularity
    // at the best shape
    for (int block : {64, 128}) {
        int occ = rg::propagate_batch_blocks_per_sm(ctx->P.nline, block);
        for (int per_sm = 1; per_sm <= occ && rc == RASCAS_OK; ++per_sm) trial(block, per_sm, 1);
    }
    const int sb = bt.block, sp = bt.blocks_per_sm;
    for (int refill : {2, 4, 8, 16}) {
        if (rc != RASCAS_OK) break;
        trial(sb, sp, refill);
    }
    ctx->P.max_scatt = saved_scatt;
    ++ctx->version;
    if (rc != RASCAS_OK) {
        B.block = saved_block;
        B.blocks_per_sm = saved_per_sm;
        B.refill = saved_refill;
        return rc;
    }
    B.block = bt.block;
    B.blocks_per_sm = bt.blocks_per_sm;
    B.refill = bt.refill;
    if (best) *best = bt;
    if (ntried) *ntried = nt;
    return RASCAS_OK;
}

int rascas_set_batch_launch(rascas_ctx* ctx, const rascas_tune* shape) {
    if (!ctx || !shape || shape->block < 32 || shape->block > rg::propagate_block_size() || shape->block % 32 != 0 ||
        shape->blocks_per_sm < 0 || shape->refill < 1 || shape->refill > 4096)
        return fail(ctx, RASCAS_E_ARG, "set_batch_launch: block 32..128 in steps of 32, blocks_per_sm >= 0, refill 1..4096");
    auto& B = ctx->batch;
    B.block = shape->block;
    B.blocks_per_sm = shape->blocks_per_sm;
    B.refill = shape->refill;
    return RASCAS_OK;
}

int rascas_update_fields(rascas_ctx* ctx, const float* n_HI, const float* vx, const float* vy, const float* vz,
                         const float* T, const float* n_dust, const float* n_metal, int mem) {
    if (!ctx || !n_HI || !vx || !vy || !vz || !T || !n_dust) return fail(ctx, RASCAS_E_ARG, "update_fields: null array");
    if (!ctx->has_mesh) return fail(ctx, RASCAS_E_STATE, "update_fields: no octree loaded");
    CK(cudaSetDevice(ctx->device));
    const size_t N = (size_t)ctx->mesh.nleaf;
    if (mem == RASCAS_DEVICE) {
        CK(rg::launch_pack_fields((long long)N, n_HI, vx, vy, vz, T, n_dust, n_metal, (float4*)ctx->d_rec.p,
                                  ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        // keep the host copy of the records in step (used when the domain changes)
        CK(cudaMemcpy(ctx->mesh.rec.data(), ctx->d_rec.p, N * 32, cudaMemcpyDeviceToHost));
    } else {
        const float* src[7] = {n_HI, vx, vy, vz, T, n_dust, n_metal};
        for (size_t i = 0; i < N; ++i)
            for (int j = 0; j < 7; ++j) ctx->mesh.rec[8 * i + j] = src[j] ? src[j][i] : 0.0f;
        CK(cudaMemcpy(ctx->d_rec.p, ctx->mesh.rec.data(), N * 32, cudaMemcpyHostToDevice));
    }
    if (n_metal) ctx->mesh.has_metal = true;
    return RASCAS_OK;
}

int rascas_peel_adjoint(rascas_ctx* ctx, const rascas_packets_in* in, int64_t n, const float* g_cube,
                        const float* g_img, const float* g_spec, float* grad, int mem) {
    if (!ctx || !in || n < 0 || !grad || (!g_cube && !g_img && !g_spec))
        return fail(ctx, RASCAS_E_ARG, "peel_adjoint: bad arguments");
    if (!ctx->has_det || ctx->det.ndir < 1) return fail(ctx, RASCAS_E_STATE, "peel_adjoint: no peeling directions");
    if (g_cube && !ctx->P.cube) return fail(ctx, RASCAS_E_STATE, "peel_adjoint: the detector accumulates no cubes");
    int r = check_ready(ctx);
    if (r) return r;
    CK(cudaSetDevice(ctx->device));
    const rascas_detector& d = ctx->det;
    const size_t npix2 = (size_t)d.npix * d.npix;
    const size_t n_cube = g_cube ? (size_t)d.ndir * npix2 * d.nbin : 0;
    const size_t n_img = g_img ? (size_t)d.ndir * npix2 : 0;
    const size_t n_spec = g_spec ? (size_t)d.ndir * d.nbin : 0;
    const size_t n_grad = 6 * (size_t)ctx->mesh.nleaf;
    cudaStream_t st = ctx->stream;
    Params P = ctx->P;
    float* dgrad = grad;
    if (mem == RASCAS_HOST) {
        CK(ctx->stage_adj.ensure((n_cube + n_img + n_spec + n_grad) * 4 + 256));
        float* b = (float*)ctx->stage_adj.p;
        float* dc = g_cube ? b : nullptr; b += n_cube;
        float* di = g_img ? b : nullptr; b += n_img;
        float* ds = g_spec ? b : nullptr; b += n_spec;
        dgrad = b;
        if (dc) CK(cudaMemcpyAsync(dc, g_cube, n_cube * 4, cudaMemcpyHostToDevice, st));
        if (di) CK(cudaMemcpyAsync(di, g_img, n_img * 4, cudaMemcpyHostToDevice, st));
        if (ds) CK(cudaMemcpyAsync(ds, g_spec, n_spec * 4, cudaMemcpyHostToDevice, st));
        P.adj_g_cube = dc; P.adj_g_img = di; P.adj_g_spec = ds;
    } else {
        P.adj_g_cube = g_cube; P.adj_g_img = g_img; P.adj_g_spec = g_spec;
    }
    // the walks accumulate each leaf's six derivatives as two vectors in one
    // 32-byte sector ([nleaf][8]); unpacked into the caller's [6][nleaf] after
    const size_t nleaf = (size_t)ctx->mesh.nleaf;
    CK(ctx->grad_vec.ensure(nleaf * 8 * sizeof(float)));
    P.adj_grad = (float*)ctx->grad_vec.p;
    P.g.spec = nullptr;   // the replay leaves the escape spectrum alone
    CK(cudaMemsetAsync(ctx->grad_vec.p, 0, nleaf * 8 * sizeof(float), st));
    // replay of the propagation (same packets, same streams, hence the same
    // scattering and peeling record) with peeling accumulating gradients
    r = run_propagate(ctx, in, n, nullptr, mem, nullptr, nullptr, nullptr, 0, true, &P);
    if (r) return r;
    CK(rg::launch_grad_unpack((long long)nleaf, (const float4*)ctx->grad_vec.p, dgrad, st));
    if (mem == RASCAS_HOST) {
        CK(cudaMemcpyAsync(grad, dgrad, n_grad * 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return RASCAS_OK;
}

}  // extern "C"

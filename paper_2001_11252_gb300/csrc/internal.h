// Internal types shared by the host side (host.cpp) and the kernels (kernels.cu)
// of the GB300 resonant-line Monte Carlo library.  Not part of the C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rg {

constexpr int kMaxLines = 4;
constexpr int kMaxChan = 4;
constexpr int kMaxDirs = 8;

// per-packet status values (same numbers as RASCAS_PK_* of the C ABI)
constexpr int RASCAS_PK_ACTIVE_ = 0;
constexpr int RASCAS_PK_ESCAPED_ = 1;
constexpr int RASCAS_PK_ABSORBED_ = 2;
constexpr int RASCAS_PK_CAPPED_ = 3;
constexpr int RASCAS_PK_ERROR_ = 4;

// leaf flags (bits of the 8th word of the leaf record)
constexpr int kFlagBorder = 1;   // the leaf touches or crosses the domain border

// counters accumulated by the kernels (u64 each)
enum Counter {
    CNT_PACKETS = 0, CNT_ESCAPED, CNT_ABSORBED, CNT_CAPPED, CNT_ERRORS,
    CNT_SCATT_LINE, CNT_SCATT_DUST, CNT_CROSS, CNT_PEEL_RAYS, CNT_PEEL_CELLS,
    CNT_UPAR_TRIALS, CNT_LEAF_LOADS, CNT_SON_LOADS, CNT_NBOR_LOADS,
    CNT_N
};

struct LineDev {
    double nu0;          // rest frequency (Hz)
    float nu0_f;
    double vth_pref;     // sqrt(2 k_B / m): v_th = vth_pref * sqrt(T)
    double invdnu_pref;  // c / nu0 / vth_pref: 1/Delta nu_D = invdnu_pref / sqrt(T)
    float invdnu_h, invdnu_l;  // invdnu_pref as an FP32 pair (hi + lo)
    double dnu_pref;     // nu0 vth_pref / c: Delta nu_D = dnu_pref sqrt(T)
    double nu0_gap;      // nu0 of line 0 minus nu0 of this line
    float a_pref;        // A_ul / (4 pi nu0 / c * vth_pref): a = a_pref / sqrt(T)
    double a_over_invdnu; // A_ul / (4 pi): a = a_over_invdnu * (1 / Delta nu_D)
    float sig_pref;      // sqrt(pi) e^2 f / (m_e c) * c / (nu0 vth_pref): sigma0 = sig_pref / sqrt(T)
    float abund;         // density multiplier
    float recoil_pref;   // h / (m c^2): recoil term = (1 - mu) * h nu / (m c^2)
    float vth_over_c_pref; // vth_pref / c
    int dens;            // 0: n_HI, 1: n_metal
    int phase;           // 0: Lya core/wing, 1: isotropic
    int nchan;
    float chan_cum[kMaxChan];  // cumulative A_i / sum A
    double chan_nu[kMaxChan];
};

// One medium: its octree, leaf records, domain and escape-spectrum axis.  A
// single-model run keeps it inside Params; a batch keeps one per model in a
// device table.
struct Geo {
    const float4* rec;     // [2*nleaf]: {n_HI, vx, vy, vz}, {T, n_dust, n_metal, flags}
    const int* son;        // [8*noct]
    const int4* nbr;       // [2*noct]: {nb0, nb1, nb2, nb3}, {nb4, nb5, father, packed levels}
    const int4* top;       // [(2^S)^3]: {code, level, oct, 0}
    int top_level, max_level, nleaf, noct;
    double box_cm;
    float box_cm_f;
    int dom_kind;          // 0 sphere, 1 slab (periodic x, y), 2 cube, 3 shell
    double dom_c[3];
    double dom_R;          // sphere / shell outer radius, slab half-thickness, cube half side
    double dom_Rin;        // shell inner radius
    // escape spectrum: bin = floor((nu - nu_lo) / nu_range * nbin), the
    // plain definition's operations in FP64 (exact ties bin as in the oracle)
    double nu_lo, nu_range;
    int nbin;
    float* spec;
};

// one peeling ray (Sect. 3.1 peeling): written by the scattering kernel at an
// emission or a scattering, walked and tallied by the peel kernel
struct PeelRec {
    double p[3];       // event position (box units)
    double nu_ext;     // external-frame frequency towards the observer (Hz)
    int w[6];          // leaf, oct, level, i, j, k of the event's leaf
    float wt;          // weight per sr
    int d;             // observer direction
};
static_assert(sizeof(PeelRec) == 64, "PeelRec is one 64-byte record");

// set-up of a peeling ray formed from its PeelRec by a prep pass before the
// walk (every lane busy): the frequency as FP32 pairs (hi, lo), the ray's
// first leaf, and the detector bins of the rays that get past it, so that
// the walk kernel does no per-ray FP64 work of its own
struct alignas(16) PeelPrep {
    float nu[2];             // nu_ext
    float d[kMaxLines][2];   // nu_ext - nu0 of each line
    int ch;                  // spectrum channel, -1 outside the frequency range (or dark)
    int dir;                 // observer direction
    float wt;                // weight per sr
    int dark;                // 0 in every record written: a ray that ends dark in its first leaf gets none (and is not listed)
    long long px;            // image pixel, -1 outside the image (or dark)
};
static_assert(sizeof(PeelPrep) == 64, "PeelPrep is one 64-byte record");

struct Params {
    const Params* self;    // device-side copy of these parameters (read by the peeling walk)
    Geo g;                 // the medium of a single-model run
    // batch of independent models (Geo per model, packet index ranges)
    const Geo* models;
    const long long* model_first;   // [nmodels + 1] prefix sums of packet counts
    int nmodels;
    // opacity sources
    int nline;
    LineDev line[kMaxLines];
    float dust_sigma, dust_albedo, dust_g;
    // physics
    int recoil, isotropic, keep_dir;
    float x_gauss;
    long long max_scatt, max_steps;
    double tau_stop;
    uint32_t key0, key1;
    uint32_t round_key[10][2];   // Philox4x32-10 key of each round (key0, key1 bumped by the Weyl constants)
    // peeling detector (single-model runs)
    int ndir, npix, cube;
    double dirs[kMaxDirs][3];
    double eu[kMaxDirs][3], ev[kMaxDirs][3];
    double img_c[3];
    double fov;
    float* pspec;
    float* pimg;
    float* pcube;
    // adjoint of the peeled optical depths (peeling accumulates gradients
    // instead of tallies when adj_grad is set)
    const float* adj_g_cube;   // dL/dcube [ndir][npix][npix][nbin] (or null)
    const float* adj_g_img;    // dL/dimage [ndir][npix][npix] (or null)
    const float* adj_g_spec;   // dL/dspectrum [ndir][nbin] (or null)
    float* adj_grad;           // [nleaf][8]: n_HI, vx, vy, vz, T, n_dust, 0, 0 (two 16-byte vectors per leaf)
    // deferred peeling: the scattering kernel appends PeelRec records; a warp
    // whose reservation starts at or past peel_hw suspends its packets (state
    // to save[], flag in save_flag[], one slot per thread of the launch) so
    // that the peel kernel can drain the records before the next round
    PeelRec* peel_rec;
    PeelPrep* peel_prep;       // [peel_cap], written by the prep pass of each round
    unsigned long long* peel_live;    // [peel_cap]: records past their first leaf, listed by the prep pass
    unsigned long long* peel_nlive;   // their number
    unsigned long long* peel_count;   // records appended this round
    unsigned long long* peel_head;    // queue head of the peel kernel
    unsigned long long peel_cap, peel_hw;
    void* save;
    int* save_flag;
    unsigned int* suspended;          // warps suspended this round
    double dir_inv[kMaxDirs][3];      // 1 / dirs (0 where a component is 0)
    float dir_kp[kMaxDirs][3][2];     // dirs as FP32 pairs
    int voigt;                        // H(a,x) method of the walk kernels (host side: picks the build)
    // core-skipping (Sect. 3.2.1): scatterings with |x_in| < x_crit draw the
    // perpendicular velocity from the Gaussian restricted to |u_perp| >= x_crit;
    // x_crit = core_skip, or core_skip_f (a tau_cell)^(1/3) when core_skip_f > 0
    int core_skip_on;
    float core_skip, core_skip_f;
    // bounded device work of the persistent kernels: per-thread loop
    // iterations and nanoseconds of %globaltimer per launch (0 = no limit);
    // a kernel that reaches one raises *abort_flag, every warp then stops
    int limits;
    unsigned int max_iter;
    unsigned long long time_limit_ns;
    unsigned int* abort_flag;
    // batch queue: consecutive packets a lane reserves per queue grab
    int refill;
    // run scratch
    unsigned long long* counters;  // [CNT_N]
    unsigned long long* head;      // work-queue head
};

// words of the counter block: CNT_N counters, the work-queue head, the abort flag
constexpr int kCounterWords = CNT_N + 2;

struct PacketsIn {
    const double* pos;
    const double* dir;
    const double* nu;
    const uint64_t* id;
    long long n;       // packets [first, n) of the arrays are propagated
    long long first;
};

struct PacketsOut {
    int32_t* status;
    int64_t* nscatt;
    double* nu;
    double* pos;
    double* dir;
    double* path;
};

struct TraceEvent {  // mirrors rascas_event
    double p[3], k[3], nu;
    int32_t leaf, level, ijk[3], status;
    int64_t ndraw, nscatt, nsteps;
};

struct TraceOut {
    TraceEvent* ev;     // [n][max_events] or null
    int32_t* nev;       // [n]
    int max_events;
};

// launchers (kernels.cu).  The three that run the walk exist twice: the plain
// names launch kernels that evaluate H(a,x) by Tasitsiomi's form, the _fad
// names kernels that evaluate the Faddeeva function (Params::voigt selects).
cudaError_t launch_propagate(const Params& P, const PacketsIn& in, const PacketsOut& out,
                             const TraceOut& tr, int grid, int block, cudaStream_t st);
cudaError_t launch_propagate_fad(const Params& P, const PacketsIn& in, const PacketsOut& out,
                                 const TraceOut& tr, int grid, int block, cudaStream_t st);
// start state of one ray of rascas_ray_tau, written by a set-up pass
struct RayInit {
    double p[3], k[3], inv[3];
    int w[6];              // leaf, oct, level, i, j, k; w[0] < 0: outside the box
    float nu[2];           // nu_ext as an FP32 pair
    float kp[3][2];        // direction as FP32 pairs
    float d[kMaxLines][2]; // nu_ext - nu0_i as FP32 pairs
};
static_assert(sizeof(RayInit) % 16 == 0, "RayInit keeps 16-byte alignment");

// init: scratch of n RayInit on the device
// deferred peeling: walk and tally the records of one round (reads the
// record count from P.peel_count; P.peel_head must be zero on entry)
cudaError_t launch_peel(const Params& P, int sms, cudaStream_t st);
cudaError_t launch_peel_fad(const Params& P, int sms, cudaStream_t st);
// bytes of one suspended packet state for nline lines
size_t packet_save_bytes(int nline);

cudaError_t launch_ray_tau(const Params& P, long long n, const double* pos, const double* dir,
                           const double* nu, double* tau, int32_t* cells, double* lens, int cap, int32_t* ncell,
                           RayInit* init, int sms, cudaStream_t st);
cudaError_t launch_ray_tau_fad(const Params& P, long long n, const double* pos, const double* dir,
                               const double* nu, double* tau, int32_t* cells, double* lens, int cap, int32_t* ncell,
                               RayInit* init, int sms, cudaStream_t st);
// column densities along rays (default build only): cols[3i..3i+2] = N_HI,
// N_dust, N_metal; tau[i] = sig_hi N_HI + sig_d N_dust (either may be null)
cudaError_t launch_ray_columns(const Params& P, long long n, const double* pos, const double* dir, double* cols,
                               double* tau, double sig_hi, double sig_d, int32_t* ncell, RayInit* init, int sms,
                               cudaStream_t st);
// the adjoint's per-leaf gradient vectors [nleaf][8] into the caller's layout [6][nleaf]
cudaError_t launch_grad_unpack(long long nleaf, const float4* src, float* dst, cudaStream_t st);
cudaError_t launch_pack_fields(long long n, const float* nh, const float* vx, const float* vy, const float* vz,
                               const float* T, const float* nd, const float* nm, float4* rec, cudaStream_t st);
cudaError_t launch_eval_voigt(long long n, const float* a, const double* x, float* H, int method, cudaStream_t st);
cudaError_t launch_sample_upar(const Params& P, long long n, const double* x, const float* a,
                               const uint64_t* id, float* u, int32_t* ndraw, cudaStream_t st);
cudaError_t noalloc_scratch(void** ptr, size_t* bytes);
// issue rates of the FP32 FMA, FP64 FMA, MUFU and IMAD pipes (probe_rates.cu)
cudaError_t probe_issue_rates(int sms, void* scratch, double rates[4]);
int propagate_block_size();
size_t propagate_smem(int nline, int block);
int propagate_blocks_per_sm(int block, bool peel);
int propagate_batch_blocks_per_sm(int nline, int block);

}  // namespace rg

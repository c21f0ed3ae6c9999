/*
 * rascas_gb300.h -- C ABI of the GB300 resonant-line Monte Carlo library.
 *
 * The library propagates photon packets of resonant lines (H I Lyman-alpha,
 * metal lines with fluorescent channels) and dust through a graded octree of
 * gas cells on one NVIDIA GB300 GPU (sm_103a), following Michel-Dansac et al.
 * (2020), "RASCAS: RAdiation SCattering in Astrophysical Simulations":
 *   - packets are independent and the transfer is passive (Sect. 2);
 *   - optical depth tau_event = -ln r, walked cell to cell (Sect. 3);
 *   - line opacity with the Hjerting-Voigt function, dust opacity (Sect. 3.1);
 *   - resonant scattering with u_par rejection sampling, core/wing phase
 *     functions and recoil, dust absorption / Henyey-Greenstein scattering,
 *     fluorescent decay channels (Sects. 3.2, 3.3);
 *   - graded octree with son/father/neighbour links (Sect. 4.3);
 *   - peeling towards fixed observer directions into spectra, images and
 *     spectral cubes (Sect. 5.1).
 *
 * Conventions for every call:
 *   - Every function returns a rascas_status (0 = success, < 0 = error); no
 *     C++ exception crosses the ABI.  rascas_last_error() gives the text of
 *     the last error of a context.
 *   - Pointers marked "mem" are host pointers when mem == RASCAS_HOST and
 *     device pointers (on the context's device) when mem == RASCAS_DEVICE.
 *     Inputs are copied or only read during the call; the caller keeps
 *     ownership of every buffer it passes.  Outputs are written into caller
 *     buffers.
 *   - Work runs on the context's stream (rascas_set_stream; default: the
 *     legacy default stream).  Calls that take host buffers, return stats or
 *     copy tallies to the host synchronise that stream before returning; the
 *     others are asynchronous with respect to the host.
 *   - A context is not thread-safe: use one context per host thread.
 *   - Units: cgs; positions in box units, the box being [0,1)^3 of physical
 *     size box_cm; frequencies in Hz in the external (observer) frame.
 */
#ifndef RASCAS_GB300_H
#define RASCAS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rascas_ctx rascas_ctx;

typedef enum {
    RASCAS_OK = 0,
    RASCAS_E_ARG = -1,      /* invalid argument (null pointer, bad size, malformed octree) */
    RASCAS_E_OOM = -2,      /* device or host allocation failed */
    RASCAS_E_CUDA = -3,     /* a CUDA runtime call failed */
    RASCAS_E_STATE = -4,    /* call made before the state it needs was set */
    RASCAS_E_TIMEOUT = -5,  /* a bounded device wait gave up */
    RASCAS_E_CAPPED = -6    /* some packets hit a cap and fail_on_cap was set */
} rascas_status;

enum { RASCAS_HOST = 0, RASCAS_DEVICE = 1 };

/* per-packet status (Sect. 4.4: escaped / absorbed; "capped" when a packet
 * reached the step or scattering cap; "error" for an internal failure) */
enum { RASCAS_PK_ACTIVE = 0, RASCAS_PK_ESCAPED = 1, RASCAS_PK_ABSORBED = 2,
       RASCAS_PK_CAPPED = 3, RASCAS_PK_ERROR = 4 };

enum { RASCAS_DOMAIN_SPHERE = 0, RASCAS_DOMAIN_SLAB = 1, RASCAS_DOMAIN_CUBE = 2, RASCAS_DOMAIN_SHELL = 3 };
enum { RASCAS_VOIGT_TASITSIOMI = 0, RASCAS_VOIGT_FADDEEVA = 1 };

enum { RASCAS_TALLY_SPECTRUM = 0,   /* [nbin] escape spectrum, 1 per escaped packet */
       RASCAS_TALLY_PEEL_SPECTRA = 1, /* [ndir][nbin] peeled flux per sr */
       RASCAS_TALLY_PEEL_IMAGES = 2,  /* [ndir][npix][npix] (row = v, column = u) */
       RASCAS_TALLY_PEEL_CUBES = 3 }; /* [ndir][npix][npix][nbin] */

#define RASCAS_MAX_LINES 4
#define RASCAS_MAX_CHANNELS 4
#define RASCAS_MAX_DIRS 8

/* Graded octree and leaf fields (Sect. 4.3, Fig. amr_struct).
 * Oct 0 is the root oct: level 1, its 8 cells of size 1/2 cover the box.
 * son[8*oct + child], child = (ix&1) | (iy&1)<<1 | (iz&1)<<2 with (ix,iy,iz)
 * the integer coordinates of the cell at its level: > 0 = the oct that
 * refines the cell, < 0 = -(leaf + 1), the leaf's index in the field arrays.
 * Neighbouring leaves should differ by at most one level (graded tree, as the
 * paper requires); other trees are accepted but walk more slowly.
 * Fields per leaf: n_HI and n_metal (cm^-3, n_metal may be NULL = 0), bulk
 * velocity vx,vy,vz (cm/s), temperature T (K), n_dust (pseudo density per H
 * atom of Sect. 3.1.2, multiplies the dust cross section). */
typedef struct {
    int32_t noct;
    int32_t nleaf;
    const int32_t *son;
    const float *n_HI, *vx, *vy, *vz, *T, *n_dust, *n_metal;
    double box_cm;
} rascas_octree;

/* Domain of the computational volume (Sect. 4 names spheres, shells, cubes
 * and slabs): a sphere (centre, radius = size), a shell (centre, outer radius
 * = size, inner radius = inner: the volume between the two spheres), a slab
 * |z - centre_z| <= size, periodic in x and y (Sect. 4, footnote on slabs),
 * or a cube (centre, half side = size).  Packets escape at its border; a
 * point outside the domain is at distance 0 from it.  `inner` is read for
 * shells only (0 <= inner < size). */
typedef struct {
    int32_t kind;
    double centre[3];
    double size;
    double inner;
} rascas_domain;

/* One absorption line (Sect. 3.1.1, Table 1): rest frequency nu0 (Hz),
 * Einstein A of the resonant channel, oscillator strength f_lu, scatterer
 * mass (g); density: 0 = n_HI, 1 = n_metal, times `abundance`; phase: 0 =
 * Lya core/wing (Eqs. Pcore, Pwing), 1 = isotropic.  Decay channels
 * (Sect. 3.2.3): chan_A/chan_nu[0] is the resonant channel (= A_ul, nu0),
 * the others fluorescent; nchan in [1, RASCAS_MAX_CHANNELS]. */
typedef struct {
    double nu0, A_ul, f_lu, mass_g, abundance;
    int32_t density, phase, nchan;
    double chan_A[RASCAS_MAX_CHANNELS];
    double chan_nu[RASCAS_MAX_CHANNELS];
} rascas_line;

/* Dust (Sects. 3.1.2, 3.2.2): cross section per unit n_dust (cm^2, constant
 * across the line), albedo, Henyey-Greenstein asymmetry g. */
typedef struct {
    double sigma, albedo, g;
} rascas_dust;

/* Switches: recoil (Eq. nuout_nuin denominator), isotropic phase function for
 * every line, keep_dir (scatterings keep the direction: the error-budget
 * experiment of Sect. 4.5), Gaussian u_par branch threshold (Sect. 3.3.3,
 * default 8), per-packet caps on scatterings and walk steps (0 = none),
 * tau_stop: peeling rays stop once tau > tau_stop (their contribution is
 * below exp(-tau_stop)), run seed of the Philox4x32-10 streams, fail_on_cap:
 * make rascas_propagate return RASCAS_E_CAPPED when a packet was capped.
 * Core-skipping (Sect. 3.2.1, the acceleration the paper uses for its galaxy
 * image, Sect. 5.1): a scattering whose frequency lies in the core,
 * |x_in| < x_crit in the scatterer's Doppler units, draws the scatterer's
 * perpendicular velocity from the Maxwellian restricted to |u_perp| >= x_crit
 * (Ahn et al. 2002; Dijkstra et al. 2006), which moves the photon to the wing
 * at once.  x_crit = core_skip (>= 0; 0 = off), or, when core_skip_f > 0,
 * x_crit = core_skip_f (a tau_cell)^(1/3) per scattering, tau_cell being the
 * line-centre optical depth of the scattering line across the packet's leaf
 * (the paper follows Smith et al. 2015, whose rule it does not print; this
 * form follows the (a tau)^(1/3) frequency scale at which thick media let
 * photons out).  It biases the redistribution: spectra of dust-free media
 * stay the same for x_crit well inside their peaks; with dust it
 * underestimates the extinction (Sect. 3.2.1).  RASCAS_E_ARG for negative
 * values. */
typedef struct {
    int32_t recoil, isotropic, keep_dir, fail_on_cap;
    double x_gauss;
    int64_t max_scatt, max_steps;
    double tau_stop;
    uint64_t seed;
    double core_skip, core_skip_f;
} rascas_physics;

/* Detector: frequency axis [nu_lo, nu_hi) in nbin bins (external frame),
 * shared by the escape spectrum and the peeled spectra/cubes; ndir peeling
 * directions (unit vectors, normalised by the library); npix x npix images of
 * side fov (box units) centred on `centre`, in the plane spanned by the
 * orthonormal basis of Duff et al. (2017) built on each direction; cube = 1
 * also accumulates spectral cubes. */
typedef struct {
    double nu_lo, nu_hi;
    int32_t nbin, ndir, npix, cube;
    double dirs[RASCAS_MAX_DIRS][3];
    double fov;
    double centre[3];
} rascas_detector;

/* Packet initial conditions (the paper's PPIC list, Sect. 2): pos[3n], dir[3n]
 * (xyz interleaved, unit vectors), nu[n] (external frame, Hz, along dir),
 * id[n] (keys the packet's random stream). */
typedef struct {
    const double *pos, *dir, *nu;
    const uint64_t *id;
} rascas_packets_in;

/* Per-packet results; any member may be NULL.  pos/dir [3n], path = total
 * distance travelled (box units). */
typedef struct {
    int32_t *status;
    int64_t *nscatt;
    double *nu, *pos, *dir, *path;
} rascas_packets_out;

typedef struct {
    int64_t packets, escaped, absorbed, capped, errors;
    int64_t nscatt_line, nscatt_dust, ncross, npeel_rays, npeel_cells;
    int64_t upar_trials, leaf_loads, son_loads, nbor_loads;
    double kernel_ms;
} rascas_run_stats;

/* One traced event (state after an interaction, an escape, or at emission). */
typedef struct {
    double p[3], k[3], nu;
    int32_t leaf, level, ijk[3], status;
    int64_t ndraw, nscatt, nsteps;
} rascas_event;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device`.  Allocates nothing large. */
int rascas_create(rascas_ctx **out, int device);
/* Free every device buffer of the context and the context itself. */
int rascas_destroy(rascas_ctx *ctx);
/* Text of the last error on this context (never NULL). */
const char *rascas_last_error(const rascas_ctx *ctx);
/* Stream for all later work (a cudaStream_t passed as void*, NULL = legacy). */
int rascas_set_stream(rascas_ctx *ctx, void *stream);

/* ---- problem set-up (the paper's problem statement: mesh + fields,
 *      lines, domain, sources, peeling directions) -----------------------
 * Set-up calls copy their arguments into the context (the caller keeps its
 * structs) and return RASCAS_E_ARG for out-of-range values without changing
 * the context.  They may be called in any order before the first run and
 * again between runs; rascas_propagate and the calls after it need the
 * octree, domain, lines and physics (RASCAS_E_STATE otherwise). */

/* Copy an octree and its leaf fields to the device (mem: where the arrays
 * live).  Validates the tree (RASCAS_E_ARG on malformed input), derives the
 * father and neighbour links of Sect. 4.3 and the leaf levels, and packs the
 * fields into 32-byte leaf records. */
int rascas_load_octree(rascas_ctx *ctx, const rascas_octree *tree, int mem);
/* The computational domain of Sect. 4 (sphere, shell, slab periodic in x and
 * y, cube) inside the unit box.  Leaves that cannot reach its border are
 * flagged so that the walk skips the border distance there (re-derived when
 * the octree or the domain changes). */
int rascas_set_domain(rascas_ctx *ctx, const rascas_domain *dom);
/* The absorbers of Sect. 3.1: nline (1..RASCAS_MAX_LINES) lines of Table 1
 * with their decay channels (Sect. 3.2.3), and dust (Sects. 3.1.2, 3.2.2;
 * dust may be NULL = none).  Line i's opacity is its density times
 * sigma0 H(a, x) with sigma0 = sqrt(pi) e^2 f_lu / (m_e c Delta nu_D) and
 * a = A_ul / (4 pi Delta nu_D), Delta nu_D = nu0 v_th / c,
 * v_th = sqrt(2 k_B T / mass_g) (Sect. 3.1.1). */
int rascas_set_lines(rascas_ctx *ctx, const rascas_line *lines, int32_t nline, const rascas_dust *dust);
/* The switches, caps and random-stream seed of rascas_physics above
 * (Sects. 3.2, 3.3, 4.5). */
int rascas_set_physics(rascas_ctx *ctx, const rascas_physics *phys);
/* Bounded device work.  The persistent kernels of rascas_propagate, _trace,
 * _propagate_noalloc and _propagate_batch, and the peeling kernel, give up
 * once a thread has run max_iterations loop iterations (one walk step per
 * iteration; 0 = no limit, at most 2^32 - 1) or a launch has run
 * time_limit_s seconds of the GPU's global timer (0 = no limit; checked
 * every 256 iterations).  The call then returns RASCAS_E_TIMEOUT; packets in
 * flight are left unfinished (status RASCAS_PK_ACTIVE where statuses are
 * returned), packets never started keep their output slots untouched, and
 * tallies hold what was accumulated.  The context stays usable.  Default:
 * no limits.  Not in the paper: a guard of this implementation. */
int rascas_set_limits(rascas_ctx *ctx, int64_t max_iterations, double time_limit_s);
/* How every later call evaluates the Hjerting-Voigt function H(a, x) of the
 * line opacities (Sect. 3.3.2 weighs several approximations against an
 * accurate evaluation):
 *   RASCAS_VOIGT_TASITSIOMI (default): Tasitsiomi (2006) eqs. 7-8, the
 *     paper's fast form, ~1 % from H for Lya at 1e4 K and worse at larger a;
 *   RASCAS_VOIGT_FADDEEVA: H = Re w(x + ia) of the Faddeeva function, by the
 *     trapezoidal rule on w's integral with its pole residue in closed form,
 *     within ~5e-7 relative in FP32 for 0 <= a <= 1 at every x (4e-6 at
 *     a = 2).  The rule's remainder grows like exp(4 pi a - pi^2 / h^2) with
 *     its step h = 1/2, so the evaluation is not valid for a > 2; a line of
 *     Table 1 reaches a = 2 only below ~0.01 K.
 * Applies to rascas_propagate, _ray_tau, _trace, _propagate_batch, the
 * peeling tallies, rascas_peel_adjoint and rascas_eval_voigt.  The context
 * keeps the method; RASCAS_E_ARG for any other value. */
int rascas_set_voigt(rascas_ctx *ctx, int method);
/* The mock observations of Sect. 5.1 (peeling-off towards fixed observer
 * directions into spectra, images and spectral cubes) and the frequency axis
 * of the angle-integrated escape spectrum (Sect. 4.4 outputs).  Allocates the
 * tallies and zeroes them (their shapes follow the detector). */
int rascas_set_detector(rascas_ctx *ctx, const rascas_detector *det);
/* Zero every tally of the detector (asynchronous, on the context's stream). */
int rascas_zero_tallies(rascas_ctx *ctx);
/* Capacity, in records, of the device buffers of peeling rays (one per
 * emission or scattering and observer direction, Sect. 3.1 peeling) that the
 * scattering kernel appends and the peel kernel then walks and tallies; each
 * record takes 136 bytes (the ray; its frequency pairs and bins formed before
 * the walk; its place in the list of rays to walk).  When the buffer fills, the packets in flight are parked
 * in device memory and resumed once the records are walked: results do not
 * depend on the capacity, only the number of rounds does.  Default 2^23
 * records (1.06 GiB); a value below the floor set by the launch shape (a few
 * resident-thread multiples) is raised to it.  RASCAS_E_ARG if records < 1. */
int rascas_set_peel_capacity(rascas_ctx *ctx, int64_t records);

/* ---- the hot path -------------------------------------------------------- */

/* Propagate n packets until each escapes, is absorbed or is capped, peeling
 * at emission and at every scattering when the detector has directions.
 * Tallies accumulate across calls.  in/out pointers follow `mem`; out may be
 * NULL; stats may be NULL (then, without peeling, the call does not
 * synchronise when mem == RASCAS_DEVICE; with peeling it synchronises once per
 * round of the peeling-ray buffer, see rascas_set_peel_capacity). */
int rascas_propagate(rascas_ctx *ctx, const rascas_packets_in *in, int64_t n,
                     const rascas_packets_out *out, int mem, rascas_run_stats *stats);

/* Copy a tally (kind = RASCAS_TALLY_*) into dst (count floats, mem): the
 * escape spectrum (one per escaped packet, Sect. 4.4) or the peeled spectra,
 * images and cubes (sums of w exp(-tau) per bin, Sect. 5.1).  count must be
 * the tally's size (RASCAS_E_ARG otherwise); RASCAS_E_STATE when the
 * detector does not accumulate that kind.  Host copies synchronise. */
int rascas_get_tally(rascas_ctx *ctx, int kind, float *dst, size_t count, int mem);

/* Optical depth from pos[3i] along dir[3i] to the domain border at external
 * frequency nu[i] (the peeling ray integral, no tau_stop).  Optionally the
 * leaves crossed and the path length in each (cells/lens [n][cap], ncell[n]
 * = number of cells crossed, which may exceed cap).  All pointers follow mem;
 * cells/lens/ncell may be NULL. */
int rascas_ray_tau(rascas_ctx *ctx, int64_t n, const double *pos, const double *dir,
                   const double *nu, double *tau, int32_t *cells, double *lens,
                   int32_t cap, int32_t *ncell, int mem);

/* Column densities along rays, the ray-tracing use of the walk (the paper's
 * escape fractions of ionising photons from optical depths integrated along
 * many rays, and column densities along arbitrary sight lines: Sect. 5
 * introduction, Sect. 6).  For ray i from pos[3i] along dir[3i] to the domain
 * border (the leaves of the walk of Sect. 4.3, the same as rascas_ray_tau's):
 *   cols[3i] = sum n_HI l L, cols[3i+1] = sum n_dust l L,
 *   cols[3i+2] = sum n_metal l L        (cm^-2; n_dust in its own units x cm)
 *   tau[i] = sigma_HI cols[3i] + sigma_dust cols[3i+1]
 * (a continuum optical depth, e.g. sigma_HI = 6.3e-18 cm^2 at 13.6 eV) and
 * ncell[i] = leaves crossed.  tau and ncell may be NULL; pointers follow mem.
 * Rays starting outside the box get zeros.  Needs the octree and domain. */
int rascas_ray_columns(rascas_ctx *ctx, int64_t n, const double *pos, const double *dir, double sigma_HI,
                       double sigma_dust, double *cols, double *tau, int32_t *ncell, int mem);

/* Run packets like rascas_propagate (same streams, no tallies) and record up
 * to max_events events per packet into events[n][max_events]; nevents[n]
 * gets how many were recorded.  Event 0 is the state at emission. */
int rascas_trace(rascas_ctx *ctx, const rascas_packets_in *in, int64_t n, int32_t max_events,
                 rascas_event *events, int32_t *nevents, int mem);

/* ---- device-function probes (parity of the building blocks) ------------ */

/* H(a, x) at a[i], x[i] by the context's method (rascas_set_voigt; default
 * the Tasitsiomi 2006 form of the hot path, Sect. 3.3.2). */
int rascas_eval_voigt(rascas_ctx *ctx, int64_t n, const float *a, const double *x, float *H, int mem);
/* One u_par draw (Sect. 3.3.3) per i for frequency x[i], Voigt parameter a[i],
 * on the stream of packet id[i] starting at draw 0; ndraw[i] = words used. */
int rascas_sample_upar(rascas_ctx *ctx, int64_t n, const double *x, const float *a,
                       const uint64_t *id, float *u, int32_t *ndraw, int mem);

/* Issue rates of the device's arithmetic pipes, measured by timing long
 * chains of one instruction kind over a full grid (the denominators of the
 * instruction-issue roofline of the scattering loop, which is bound by
 * arithmetic, not by HBM): rates[0] FP32 FMA, rates[1] FP64 FMA, rates[2]
 * special-function (MUFU EX2), rates[3] 32-bit integer multiply-add, each in
 * warp-instructions per second for the whole device.  Runs on the legacy
 * default stream for about a tenth of a second; synchronises.  Not in the
 * paper: a measurement aid. */
int rascas_probe_issue_rates(rascas_ctx *ctx, double *rates);

/* ---- adjoint (gradients of the peeled tallies) --------------------------- */

/* Replace the leaf fields of the loaded octree (same tree, same leaf order;
 * arrays of nleaf floats per `mem`, n_metal may be NULL).  The domain flags
 * are kept. */
int rascas_update_fields(rascas_ctx *ctx, const float *n_HI, const float *vx, const float *vy, const float *vz,
                         const float *T, const float *n_dust, const float *n_metal, int mem);

/* Gradient of L = sum(g_cube * cube) + sum(g_img * image) + sum(g_spec *
 * spectrum) with respect to each leaf's n_HI, vx, vy, vz, T and n_dust, with
 * the scattering record held fixed: the positions, directions, external
 * frequencies and weights of every peeling event of the given packets are
 * those of rascas_propagate on the same packets (the run is replayed: same
 * streams, same fields), and only the optical depths of the peeling rays
 * (Sect. 3.1 opacities along each ray, Sect. 5.1 peeling) are differentiated:
 *     dL/dtheta_c = - sum_events G_e w_e exp(-tau_e) L l_(e,c) dkappa_c/dtheta_c.
 * Each ray is walked twice (tau first, then the gradients), so nothing per ray
 * is stored; the context keeps a device buffer of 32 bytes per leaf in which
 * each leaf's six derivatives accumulate together (RASCAS_E_OOM if it cannot
 * be allocated).  g_* follow the detector shapes of rascas_get_tally (any may
 * be NULL, not all); grad receives [6][nleaf] floats (n_HI, vx, vy, vz, T,
 * n_dust), zeroed first.  Not in the paper: the adjoint is an addition.
 * All pointers follow `mem`; tallies are left untouched. */
int rascas_peel_adjoint(rascas_ctx *ctx, const rascas_packets_in *in, int64_t n, const float *g_cube,
                        const float *g_img, const float *g_spec, float *grad, int mem);

/* ---- batches of independent models --------------------------------------- */

/* One independent model of a batch: its own octree and leaf fields, domain,
 * escape-spectrum axis [nu_lo, nu_hi) and packet list (npackets entries).
 * Lines, dust and physics switches are the context's.  The paper's master
 * distributes bundles of packets of many domains to workers (Sect. 4.4); here
 * every model's packets feed one device work queue. */
typedef struct {
    rascas_octree tree;
    rascas_domain domain;
    double nu_lo, nu_hi;
    rascas_packets_in packets;
    int64_t npackets;
} rascas_model;

enum { RASCAS_BATCH_PERSISTENT = 0,   /* one persistent launch over all models (CUDA graph) */
       RASCAS_BATCH_PER_MODEL = 1 };  /* one launch per model, in sequence (the plain way) */

/* Launch shape tried by the autotuner and its time for the capped batch:
 * threads per block, resident blocks per SM, and the refill granularity
 * (consecutive packets a lane reserves per grab from the work queue, the
 * analogue of the paper's bundles of N_bundle packets, Sects. 4.4, 4.6). */
typedef struct {
    int32_t block, blocks_per_sm, refill;
    double ms;
} rascas_tune;

/* Copy nmodels models to the device (arrays per `mem`), validating each octree
 * like rascas_load_octree.  Needs the lines set (the queue is ordered by each
 * model's estimated line-centre optical depth, costliest first).  Escape
 * spectra: nbin bins per model. */
int rascas_load_batch(rascas_ctx *ctx, const rascas_model *models, int32_t nmodels, int32_t nbin, int mem);
/* Propagate every packet of the loaded batch (spectra are zeroed first);
 * mode = RASCAS_BATCH_*.  Synchronises; stats (may be NULL) cover the batch,
 * kernel_ms the device time of the whole call. */
int rascas_propagate_batch(rascas_ctx *ctx, int32_t mode, rascas_run_stats *stats);
/* rascas_propagate_batch that also returns per-packet results: out's arrays
 * (any may be NULL, not all) hold every packet of the batch, models in the
 * order given to rascas_load_batch, each model's packets in its own order
 * ([sum of npackets] entries; pos and dir x3).  The persistent launch is made
 * directly (not from the captured graph).  Synchronises. */
int rascas_propagate_batch_packets(rascas_ctx *ctx, int32_t mode, const rascas_packets_out *out, int mem,
                                   rascas_run_stats *stats);
/* Escape spectra [nmodels][nbin] in the order the models were given. */
int rascas_get_batch_spectra(rascas_ctx *ctx, float *dst, size_t count, int mem);
/* Time the persistent batch launch, each packet capped at max_scatt
 * scatterings: block sizes {64, 128} x every resident-block count per SM with
 * one packet per queue grab, then refill granularities {2, 4, 8, 16} at the
 * fastest shape; keep the fastest for later rascas_propagate_batch calls.
 * tried (may be NULL) receives up to max_tried timings. */
/* Set the batch launch shape by hand (shape->ms is ignored): block = 32, 64,
 * 96 or 128 threads, blocks_per_sm >= 0 (0 = as many as fit), refill >= 1
 * (at most 4096).  Results do not depend on the shape. */
int rascas_set_batch_launch(rascas_ctx *ctx, const rascas_tune *shape);
int rascas_autotune_batch(rascas_ctx *ctx, int64_t max_scatt, rascas_tune *best, rascas_tune *tried,
                          int32_t max_tried, int32_t *ntried);

/* ---- allocation-free variant ------------------------------------------- */

/* Largest n accepted by rascas_propagate_noalloc. */
#define RASCAS_NOALLOC_MAX_PACKETS 57344

/* rascas_propagate for callers that must not allocate device memory while
 * they run -- for example an application that hands all free HBM to another
 * framework's memory pool at start-up, or a latency-critical loop where a
 * cudaMalloc (which can synchronise the device) is not acceptable.  This call
 * itself performs no cudaMalloc, cudaFree or allocating library call: its
 * device scratch (work-queue head, counters, a parameter copy and the staging
 * of up to RASCAS_NOALLOC_MAX_PACKETS packets, 8 MiB in all) is a static
 * device array that every GPU loading the library holds until the process
 * exits.  rascas_create looks up the array's device address, which loads the
 * module holding it: the 8 MiB are taken then, so create the context before
 * handing the free memory to another pool.  The context must already be set
 * up (octree, domain, lines, physics).  No counterpart in the paper: this is
 * an interface variant only.
 *
 * in/out are HOST arrays (as rascas_packets_in / rascas_packets_out); out and
 * stats may be NULL.  Results per packet are identical to rascas_propagate on
 * the same packets; tallies and peeling are not accumulated (per-packet
 * outputs only).  n > RASCAS_NOALLOC_MAX_PACKETS returns RASCAS_E_ARG.
 * Every call reuses the same array and clears the parts that must start at
 * zero; calls that overlap on the GPU (several host threads, streams or
 * contexts on one device at once) race on it and must be serialised by the
 * caller.  The call synchronises the context's stream before returning. */
int rascas_propagate_noalloc(rascas_ctx *ctx, const rascas_packets_in *in, int64_t n,
                             const rascas_packets_out *out, rascas_run_stats *stats);

#ifdef __cplusplus
}
#endif
#endif

/*
 * Plain FP64 CPU oracle for resonant-line Monte Carlo transfer through a
 * graded octree (Michel-Dansac et al. 2020, "RASCAS", Sects. 3 and 4).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The product path
 * (the CUDA library) never calls it, and it shares no code with it.
 *
 * Everything is double precision, written for clarity rather than speed:
 * every random word is recomputed from the Philox counter, every cell visit
 * recomputes its opacities from the raw fields, every neighbour is found by a
 * descent from the root.  Build with -ffp-contract=off so that the geometry is
 * evaluated exactly as written (explicit fma() where a fused multiply-add is
 * meant).
 *
 * Readings where the paper is silent (they are listed with the rest in the
 * design notes):
 *  - RNG: Philox4x32-10; key = 64-bit run seed, counter = (draw block lo,
 *    draw block hi, packet id lo, packet id hi); draw word n of a packet is
 *    word (n mod 4) of block n/4.  u23 = ((w>>9)+1/2) 2^-23 for every
 *    single-precision draw (exactly representable in FP32 together with
 *    1 - u23), u52 from two words for tau_event.
 *  - Fixed draw order per event: tau_event (2 words); interaction choice (1);
 *    dust: albedo (1), mu (1), phi (1); line: channel (1, only when the line
 *    has several decay channels), u_par trials (3 words per trial, 2 for the
 *    Gaussian branch), u_perp pair (2), mu (1), phi (1).  Peeling draws none.
 *  - Frame change: nu_ext = nu_gas (1 + k.v/c) (Sect. 3, first order) and its
 *    exact inverse nu_gas = nu_ext / (1 + k.v/c).
 *  - Distances to faces: t = (face - p) * (1/k), with 1/k taken once per
 *    direction; crossing coordinate snapped to the face; ties between axes go
 *    to the lowest axis index; the cell a packet is in is the one containing
 *    p + eps k (a point on a face belongs to the cell the packet moves into).
 *  - HG inversion with the square that the printed formula lacks (Sect. 3.3.1).
 *  - u0 polynomial (Sect. 3.3.3) clamped to u0 >= 0, applied to |x|.
 *  - Gaussian branch for |x| >= x_gauss: N(1/|x|, 1/2).
 *  - Core/wing test |x_in - u_par| < 0.2 (Sect. 3.2.1, scatterer frame).
 *  - Dust scattering is coherent in the gas frame.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_API __attribute__((visibility("default")))

/* CODATA 2018, cgs */
static const double OC = 2.99792458e10;
static const double OKB = 1.380649e-16;
static const double OH = 6.62607015e-27;
static const double OME = 9.1093837015e-28;
static const double OE = 4.803204712570263e-10;
static const double OPI = 3.14159265358979323846;

#define ORA_MAXLINE 4
#define ORA_MAXCHAN 4
#define ORA_MAXDIR 8

enum { ORA_ACTIVE = 0, ORA_ESCAPED = 1, ORA_ABSORBED = 2, ORA_CAPPED = 3, ORA_ERROR = 4 };
enum { ORA_DOM_SPHERE = 0, ORA_DOM_SLAB = 1, ORA_DOM_CUBE = 2, ORA_DOM_SHELL = 3 };

typedef struct {
    /* mesh (Sect. 4.3): son per cell, physical fields per leaf */
    const int32_t *son;
    const float *n_HI, *vx, *vy, *vz, *T, *n_dust, *n_metal;
    int64_t noct, nleaf;
    double box_cm;
    /* domain (Sect. 4) */
    int64_t dom_kind;
    double dom_c[3];
    double dom_size;
    double dom_inner;   /* shell inner radius */
    /* lines (Sect. 3.1.1, Table 1) */
    int64_t nline;
    double line_nu[ORA_MAXLINE], line_A[ORA_MAXLINE], line_f[ORA_MAXLINE], line_m[ORA_MAXLINE];
    double line_abund[ORA_MAXLINE];
    int64_t line_dens[ORA_MAXLINE], line_phase[ORA_MAXLINE], line_nchan[ORA_MAXLINE];
    double chan_A[ORA_MAXLINE][ORA_MAXCHAN], chan_nu[ORA_MAXLINE][ORA_MAXCHAN];
    /* dust (Sects. 3.1.2, 3.2.2) */
    double dust_sigma, dust_albedo, dust_g;
    /* physics switches */
    int64_t recoil, isotropic, keep_dir, max_scatt, max_steps;
    double x_gauss;
    uint64_t seed;
    /* detector: frequency axis (external frame), peeling directions, image */
    double nu_lo, nu_hi;
    int64_t nbin, ndir, npix, cube;
    double dirs[ORA_MAXDIR][3];
    double fov, img_c[3];
    /* H(a,x) evaluation: 0 Tasitsiomi (2006), 1 the Faddeeva function */
    int64_t voigt;
    /* core-skipping (Sect. 3.2.1): critical frequency x_crit of the
     * truncated perpendicular-velocity draw; core_skip_f > 0 sets
     * x_crit = core_skip_f (a tau_cell)^(1/3) per scattering, else
     * x_crit = core_skip (0 = off) */
    double core_skip, core_skip_f;
} ora_cfg;

typedef struct {
    double p[3], k[3], nu;      /* position (box units), direction, external-frame frequency */
    int64_t leaf, level, ijk[3];
    uint64_t pid, ndraw;
    int64_t nscatt, nsteps, status;
    double path;                /* total path length (box units) */
} ora_state;

/* one peeling event: the fixed scattering record used by the adjoint */
typedef struct {
    double p[3];
    int64_t leaf, level, ijk[3];
    int64_t dir;      /* peeling direction index */
    double w;         /* weight per steradian */
    double nu;        /* external-frame frequency along the direction */
} ora_peel_event;

typedef struct {
    double *spec;   /* [nbin] escape spectrum, weight 1 per escaped packet */
    double *pspec;  /* [ndir*nbin] peeled spectra */
    double *pimg;   /* [ndir*npix*npix] peeled images */
    double *pcube;  /* [ndir*npix*npix*nbin] peeled cubes (optional) */
    int64_t ncross, nscatt_line, nscatt_dust, npeel;
    ora_peel_event *events;   /* optional record of every peeling event */
    int64_t nev, cap;
} ora_tally;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011)                     */
/* ------------------------------------------------------------------ */
ORA_API void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    memcpy(out, c, sizeof c);
}

/* draw word n of packet pid */
ORA_API uint32_t ora_word(uint64_t seed, uint64_t pid, uint64_t n)
{
    uint64_t blk = n >> 2;
    uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), (uint32_t)pid, (uint32_t)(pid >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    ora_philox4x32_10(ctr, key, out);
    return out[n & 3];
}

static double u23(const ora_cfg *cf, ora_state *s)
{
    uint32_t w = ora_word(cf->seed, s->pid, s->ndraw++);
    return ((double)(w >> 9) + 0.5) * 0x1p-23;
}

static double u52(const ora_cfg *cf, ora_state *s)
{
    uint32_t wa = ora_word(cf->seed, s->pid, s->ndraw++);
    uint32_t wb = ora_word(cf->seed, s->pid, s->ndraw++);
    double m = (double)(wa >> 6) * 67108864.0 + (double)(wb >> 6);
    return (m + 0.5) * 0x1p-52;
}

/* ------------------------------------------------------------------ */
/* Hjerting-Voigt H(a,x): Tasitsiomi (2006) eqs. 7-8 (Sect. 3.3.2)      */
/* ------------------------------------------------------------------ */
ORA_API double ora_voigt(double a, double x)
{
    double x2 = x * x;
    double z = (x2 - 0.855) / (x2 + 3.42);
    double q = 0.0;
    if (z > 0.0) {
        q = z * (1.0 + 21.0 / x2) * a / (OPI * (x2 + 1.0))
            * (0.1117 + z * (4.421 + z * (-9.207 + 5.674 * z)));
    }
    return sqrt(OPI) * q + exp(-x2);
}

/* ------------------------------------------------------------------ */
/* Accurate H(a,x) (Sect. 3.3.2 offers more accurate Voigt evaluations  */
/* beside Tasitsiomi's).  H = Re w(x + ia) with w the Faddeeva function  */
/*   w(z) = (i/pi) int exp(-t^2) / (z - t) dt,   Im z > 0.               */
/* The trapezoidal rule on the nodes t_n = delta + n h misses only the   */
/* residue of the pole t = z, which is known in closed form (Matta &      */
/* Reichel 1971; Hunter & Regan 1972):                                   */
/*   w(z) = (i h/pi) sum_n exp(-t_n^2) / (z - t_n)                       */
/*          + 2 exp(-z^2) / (1 - exp(-2 pi i (z - delta) / h))            */
/* up to O(exp(-pi^2/h^2)), for 0 < Im z < pi/h.  The nodes are put half  */
/* a step either side of x (delta = x + h/2), so no node comes closer     */
/* than h/2 to the pole and the residue term becomes                      */
/* 2 exp(-z^2) / (1 + exp(2 pi a / h)): every term stays bounded and the  */
/* Lorentz terms of Re w are all positive.  h = 1/4 puts the remainder    */
/* near e^-158; nodes with |t_n| > 9 (weights below e^-81) are left out.  */
/* Defined for 0 < a <= 5; H(0, x) is the limit exp(-x^2) (Im w is then   */
/* not formed).                                                           */
/* ------------------------------------------------------------------ */
ORA_API void ora_faddeeva(double a, double x, double *re, double *im)
{
    if (a <= 0.0) {
        *re = exp(-x * x);
        *im = NAN;
        return;
    }
    if (!(a <= 5.0)) {
        *re = *im = NAN;
        return;
    }
    const double h = 0.25, tmax = 9.0;
    const double complex z = x + I * a;
    const long nlo = (long)ceil((-tmax - x) / h - 0.5), nhi = (long)floor((tmax - x) / h - 0.5);
    double complex s = 0.0;
    for (long n = nlo; n <= nhi; ++n) {
        const double t = x + ((double)n + 0.5) * h;
        s += exp(-t * t) / (z - t);
    }
    double complex w = (I * h / OPI) * s + 2.0 * cexp(-z * z) / (1.0 + exp(2.0 * OPI * a / h));
    *re = creal(w);
    *im = cimag(w);
}

/* H(a,x) by the method the configuration names */
static double voigt_of(const ora_cfg *cf, double a, double x)
{
    if (cf->voigt == 1) {
        double re, im;
        ora_faddeeva(a, x, &re, &im);
        return re;
    }
    return ora_voigt(a, x);
}

/* ------------------------------------------------------------------ */
/* line and dust opacity in one cell (Sect. 3.1)                        */
/* ------------------------------------------------------------------ */
typedef struct {
    double vth, dnu, a, x, sigma;   /* per line */
} ora_lineprop;

static double line_density(const ora_cfg *cf, int il, int64_t leaf)
{
    double n;
    if (cf->line_dens[il] == 1) n = (double)cf->n_metal[leaf];
    else n = (double)cf->n_HI[leaf];
    return n * cf->line_abund[il];
}

static void line_props(const ora_cfg *cf, int il, int64_t leaf, double nu_gas, ora_lineprop *lp)
{
    double T = (double)cf->T[leaf];
    lp->vth = sqrt(2.0 * OKB * T / cf->line_m[il]);
    lp->dnu = cf->line_nu[il] * lp->vth / OC;
    lp->a = cf->line_A[il] / (4.0 * OPI * lp->dnu);
    lp->x = (nu_gas - cf->line_nu[il]) / lp->dnu;
    lp->sigma = sqrt(OPI) * OE * OE * cf->line_f[il] / (OME * OC * lp->dnu) * voigt_of(cf, lp->a, lp->x);
}

/* exported for the pins: v_th, Delta nu_D, a, x, sigma of line il in a leaf */
ORA_API void ora_line_props(const ora_cfg *cf, int64_t il, int64_t leaf, double nu_gas, double out[5])
{
    ora_lineprop lp;
    line_props(cf, (int)il, leaf, nu_gas, &lp);
    out[0] = lp.vth;
    out[1] = lp.dnu;
    out[2] = lp.a;
    out[3] = lp.x;
    out[4] = lp.sigma;
}

static double beta_of(const ora_cfg *cf, int64_t leaf, const double k[3])
{
    return (k[0] * (double)cf->vx[leaf] + k[1] * (double)cf->vy[leaf] + k[2] * (double)cf->vz[leaf]) / OC;
}

/* total and per-channel opacities (cm^-1) at external frequency nu along k */
static double opacity(const ora_cfg *cf, int64_t leaf, double nu_ext, const double k[3],
                      double kap_line[ORA_MAXLINE], double *kap_dust)
{
    double nu_gas = nu_ext / (1.0 + beta_of(cf, leaf, k));
    double tot = 0.0;
    for (int il = 0; il < cf->nline; ++il) {
        ora_lineprop lp;
        line_props(cf, il, leaf, nu_gas, &lp);
        kap_line[il] = line_density(cf, il, leaf) * lp.sigma;
        tot += kap_line[il];
    }
    *kap_dust = (double)cf->n_dust[leaf] * cf->dust_sigma;
    tot += *kap_dust;
    return tot;
}

ORA_API double ora_opacity(const ora_cfg *cf, int64_t leaf, double nu_ext, const double k[3])
{
    double kl[ORA_MAXLINE], kd;
    return opacity(cf, leaf, nu_ext, k, kl, &kd);
}

/* ------------------------------------------------------------------ */
/* u_par: rejection method of Zheng & Miralda-Escude (2002) with the    */
/* u0(x, log10 a) polynomial of Sect. 3.3.3                             */
/* ------------------------------------------------------------------ */
ORA_API double ora_u0(double x, double a)
{
    double z = log10(a);
    double u0 = 2.648963 + 2.014446 * z + 0.351479 * z * z
        + x * (-4.058673 - 3.675859 * z - 0.640003 * z * z
        + x * (3.017395 + 2.117133 * z + 0.370294 * z * z
        + x * (-0.869789 - 0.565886 * z - 0.096312 * z * z
        + x * (0.110987 + 0.070103 * z + 0.011557 * z * z
        + x * (-0.005200 - 0.003240 * z - 0.000519 * z * z)))));
    return u0 < 0.0 ? 0.0 : u0;
}

static double sample_upar(const ora_cfg *cf, ora_state *s, double x, double a, int *err)
{
    double sgn = x < 0.0 ? -1.0 : 1.0;
    double xa = fabs(x);
    if (xa >= cf->x_gauss) {
        double r1 = u23(cf, s), r2 = u23(cf, s);
        return sgn * (1.0 / xa + sqrt(-log(r1)) * cos(2.0 * OPI * r2));
    }
    double u0 = ora_u0(xa, a);
    double th0 = atan((u0 - xa) / a);
    double e0 = exp(-u0 * u0);
    double p = (th0 + OPI / 2) / ((1.0 - e0) * th0 + (1.0 + e0) * OPI / 2);
    for (long trial = 0; trial < 100000000L; ++trial) {
        double r1 = u23(cf, s), r2 = u23(cf, s), r3 = u23(cf, s);
        double u;
        if (r1 <= p) {
            double th = -OPI / 2 + (th0 + OPI / 2) * r2;
            u = a * tan(th) + xa;
            if (r3 <= exp(-u * u)) return sgn * u;
        } else {
            double th = th0 + (OPI / 2 - th0) * r2;
            u = a * tan(th) + xa;
            if (r3 <= exp(u0 * u0 - u * u)) return sgn * u;
        }
    }
    *err = 1;
    return 0.0;
}

/* exported for distribution tests: n samples for one packet stream */
ORA_API void ora_sample_upar_n(const ora_cfg *cf, uint64_t pid, double x, double a, int64_t n, double *out)
{
    ora_state s;
    memset(&s, 0, sizeof s);
    s.pid = pid;
    int err = 0;
    for (int64_t i = 0; i < n; ++i) out[i] = sample_upar(cf, &s, x, a, &err);
}

/* ------------------------------------------------------------------ */
/* phase functions (Sect. 3.3.1) and their inverse-CDF samplers         */
/* ------------------------------------------------------------------ */
enum { PH_ISO = 0, PH_CORE = 1, PH_WING = 2, PH_HG = 3 };

ORA_API double ora_mu_sample(int kind, double r, double g)
{
    if (kind == PH_CORE) {
        double B = 6.0 * (2.0 * r - 1.0);
        double A = sqrt(B * B + 11.0 * 11.0 * 11.0 / 27.0);
        return cbrt(A + B) - cbrt(A - B);
    }
    if (kind == PH_WING) {
        double B = 4.0 * r - 2.0;
        double A = sqrt(B * B + 1.0);
        return cbrt(A + B) - cbrt(A - B);
    }
    if (kind == PH_HG && g != 0.0) {
        double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * r);
        return (1.0 + g * g - t * t) / (2.0 * g);
    }
    return 2.0 * r - 1.0;
}

/* phase function per unit mu (integrates to 1 over [-1,1]) */
ORA_API double ora_phase(int kind, double mu, double g)
{
    if (kind == PH_CORE) return 11.0 / 24.0 + 3.0 * mu * mu / 24.0;
    if (kind == PH_WING) return 3.0 * (1.0 + mu * mu) / 8.0;
    if (kind == PH_HG) return 0.5 * (1.0 - g * g) / pow(1.0 + g * g - 2.0 * g * mu, 1.5);
    return 0.5;
}

/* orthonormal basis (b1, b2) perpendicular to unit n: Duff et al. (2017) */
static void onb(const double n[3], double b1[3], double b2[3])
{
    double sg = copysign(1.0, n[2]);
    double a = -1.0 / (sg + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sg * n[0] * n[0] * a;
    b1[1] = sg * b;
    b1[2] = -sg * n[0];
    b2[0] = b;
    b2[1] = sg + n[1] * n[1] * a;
    b2[2] = -n[1];
}

ORA_API void ora_onb(const double n[3], double b1[3], double b2[3]) { onb(n, b1, b2); }

static void dir_from(const double k[3], double mu, double phi, double out[3])
{
    double e1[3], e2[3];
    onb(k, e1, e2);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double c = cos(phi), s = sin(phi);
    for (int i = 0; i < 3; ++i) out[i] = mu * k[i] + st * (c * e1[i] + s * e2[i]);
    double nn = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
    for (int i = 0; i < 3; ++i) out[i] /= nn;
}

/* ------------------------------------------------------------------ */
/* octree: root descent (Sect. 4.3)                                     */
/* ------------------------------------------------------------------ */

/* Integer coordinate, at level l, of the cell entered by a packet at p moving
 * along k: the cell containing p + eps k for an infinitesimal eps.  Along an
 * axis with k >= 0 this is floor(p 2^l); with k < 0 it is ceil(p 2^l) - 1, so
 * that a point lying exactly on a face belongs to the cell on the side the
 * packet moves into. */
static int64_t coord_at(const double p[3], const double k[3], int ax, int64_t l)
{
    double y = ldexp(p[ax], (int)l);
    if (k[ax] < 0.0) return (int64_t)ceil(y) - 1;
    return (int64_t)floor(y);
}

/* leaf entered at p along k by descent from the root oct; -1 outside the box */
static int64_t descend(const ora_cfg *cf, const double p[3], const double k[3],
                       int64_t *level, int64_t ijk[3])
{
    int64_t oct = 0;
    for (int64_t l = 1; l < 64; ++l) {
        int64_t c[3];
        for (int ax = 0; ax < 3; ++ax) {
            c[ax] = coord_at(p, k, ax, l);
            if (c[ax] < 0 || c[ax] >= ((int64_t)1 << l)) return -1;
        }
        int child = (int)((c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2));
        int32_t sv = cf->son[8 * oct + child];
        if (sv < 0) {
            *level = l;
            for (int ax = 0; ax < 3; ++ax) ijk[ax] = c[ax];
            return -(int64_t)sv - 1;
        }
        oct = sv;
    }
    return -1;
}

static int periodic_axis(const ora_cfg *cf, int ax)
{
    return cf->dom_kind == ORA_DOM_SLAB && ax < 2;
}

/* slab domain: x and y are periodic; bring p + eps k back into the box */
static void wrap_periodic(const ora_cfg *cf, double p[3], const double k[3])
{
    for (int ax = 0; ax < 3; ++ax) {
        if (!periodic_axis(cf, ax)) continue;
        int64_t c = coord_at(p, k, ax, 1);
        if (c >= 2) p[ax] = p[ax] - 1.0;
        else if (c < 0) p[ax] = p[ax] + 1.0;
    }
}

ORA_API int64_t ora_locate(const ora_cfg *cf, const double p_in[3], const double k[3],
                           int64_t *level, int64_t ijk[3])
{
    double p[3] = {p_in[0], p_in[1], p_in[2]};
    wrap_periodic(cf, p, k);
    return descend(cf, p, k, level, ijk);
}

/* ------------------------------------------------------------------ */
/* geometry of one step                                                 */
/* ------------------------------------------------------------------ */

/* distance (box units) to the exit face of the leaf along k; *axis gets the
 * crossed axis.  inv[] = 1/k per axis (0 where k = 0, never used). */
static double face_distance(const ora_state *s, const double inv[3], int *axis)
{
    double h = ldexp(1.0, -(int)s->level);
    double best = INFINITY;
    int ba = -1;
    for (int ax = 0; ax < 3; ++ax) {
        if (s->k[ax] == 0.0) continue;
        double face = s->k[ax] > 0.0 ? (double)(s->ijk[ax] + 1) * h : (double)s->ijk[ax] * h;
        double t = (face - s->p[ax]) * inv[ax];
        if (t < best) {
            best = t;
            ba = ax;
        }
    }
    *axis = ba;
    return best < 0.0 ? 0.0 : best;
}

/* distance (box units) from p along k to the border of the domain */
static double border_distance(const ora_cfg *cf, const double p[3], const double k[3], const double inv[3])
{
    const double *c = cf->dom_c;
    double R = cf->dom_size;
    if (cf->dom_kind == ORA_DOM_SPHERE || cf->dom_kind == ORA_DOM_SHELL) {
        double d0 = p[0] - c[0], d1 = p[1] - c[1], d2 = p[2] - c[2];
        double b = d0 * k[0] + d1 * k[1] + d2 * k[2];
        double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        double cc = r2 - R * R;
        double disc = b * b - cc;
        if (disc < 0.0) disc = 0.0;
        double sq = sqrt(disc);
        double t = b > 0.0 ? -cc / (b + sq) : sq - b;
        if (cf->dom_kind == ORA_DOM_SHELL) {
            /* a shell ends at the outer sphere and at the inner one: the first
             * root of |p + t k - c| = inner when the ray moves inwards and
             * meets it; a point inside the inner sphere is outside the domain */
            double ci = r2 - cf->dom_inner * cf->dom_inner;
            if (ci <= 0.0) return 0.0;
            double di = b * b - ci;
            if (b < 0.0 && di >= 0.0) {
                double ti = ci / (-b + sqrt(di));
                if (ti < t) t = ti;
            }
        }
        return t < 0.0 ? 0.0 : t;
    }
    double best = INFINITY;
    for (int ax = 0; ax < 3; ++ax) {
        if (cf->dom_kind == ORA_DOM_SLAB && ax != 2) continue;
        if (k[ax] == 0.0) continue;
        double edge = k[ax] > 0.0 ? c[ax] + R : c[ax] - R;
        double t = (edge - p[ax]) * inv[ax];
        if (t < best) best = t;
    }
    return best < 0.0 ? 0.0 : best;
}

static void inverse_dir(const double k[3], double inv[3])
{
    for (int ax = 0; ax < 3; ++ax) inv[ax] = k[ax] != 0.0 ? 1.0 / k[ax] : 0.0;
}

/* move p to the exit face along `axis` (distance t) and find the next leaf.
 * Returns 0 on success, 1 if the packet left the box. */
static int cross_face(const ora_cfg *cf, double p[3], const double k[3], int axis, double t,
                      int64_t *leaf, int64_t *level, int64_t ijk[3])
{
    double h = ldexp(1.0, -(int)*level);
    double face = k[axis] > 0.0 ? (double)(ijk[axis] + 1) * h : (double)ijk[axis] * h;
    for (int ax = 0; ax < 3; ++ax)
        if (ax != axis) p[ax] = fma(t, k[ax], p[ax]);
    p[axis] = face;
    wrap_periodic(cf, p, k);
    int64_t nlv, nijk[3];
    int64_t nleaf = descend(cf, p, k, &nlv, nijk);
    if (nleaf < 0) return 1;
    *leaf = nleaf;
    *level = nlv;
    for (int ax = 0; ax < 3; ++ax) ijk[ax] = nijk[ax];
    return 0;
}

/* ------------------------------------------------------------------ */
/* peeling (Sect. 5.1: peeling-off towards fixed observer directions)   */
/* ------------------------------------------------------------------ */

/* optical depth from p (inside `leaf`) along k to the domain border at
 * external frequency nu; stops once tau > tau_stop.  Optionally records the
 * leaves crossed and the path length in each. */
static double ray_tau(const ora_cfg *cf, const double p0[3], const double k[3], double nu_ext,
                      int64_t leaf, int64_t level, const int64_t ijk0[3], double tau_stop,
                      int64_t *cells, double *lens, int64_t cap, int64_t *ncell)
{
    double p[3] = {p0[0], p0[1], p0[2]};
    int64_t ijk[3] = {ijk0[0], ijk0[1], ijk0[2]};
    double inv[3];
    inverse_dir(k, inv);
    double tau = 0.0;
    int64_t n = 0;
    for (long guard = 0; guard < 100000000L; ++guard) {
        ora_state tmp;
        memcpy(tmp.p, p, sizeof p);
        memcpy(tmp.k, k, sizeof tmp.k);
        tmp.level = level;
        memcpy(tmp.ijk, ijk, sizeof ijk);
        int axis;
        double tf = face_distance(&tmp, inv, &axis);
        double tb = border_distance(cf, p, k, inv);
        double l = tb <= tf ? tb : tf;
        double kl[ORA_MAXLINE], kd;
        double kap = opacity(cf, leaf, nu_ext, k, kl, &kd);
        tau += kap * l * cf->box_cm;
        if (cells && n < cap) {
            cells[n] = leaf;
            lens[n] = l;
        }
        ++n;
        if (tb <= tf || tau > tau_stop) break;
        if (cross_face(cf, p, k, axis, tf, &leaf, &level, ijk)) break;
    }
    if (ncell) *ncell = n;
    return tau;
}

ORA_API double ora_ray_tau(const ora_cfg *cf, const double p[3], const double k[3], double nu_ext,
                           double tau_stop, int64_t *cells, double *lens, int64_t cap, int64_t *ncell)
{
    int64_t level, ijk[3];
    double pp[3] = {p[0], p[1], p[2]};
    wrap_periodic(cf, pp, k);
    int64_t leaf = descend(cf, pp, k, &level, ijk);
    p = pp;
    if (leaf < 0) {
        if (ncell) *ncell = 0;
        return 0.0;
    }
    return ray_tau(cf, p, k, nu_ext, leaf, level, ijk, tau_stop, cells, lens, cap, ncell);
}

/* Column densities from p along k to the domain border (the ray integral of
 * Sect. 3.1 without the line profile: the quantity behind escape fractions of
 * ionising photons and sight-line columns, Sects. 5 and 6):
 *   cols[0] = sum n_HI l L, cols[1] = sum n_dust l L, cols[2] = sum n_metal l L
 * over the leaves of the walk of Sect. 4.3 (cm^-2; n_dust in its own units
 * times cm).  Returns the number of leaves crossed; 0 outside the box. */
ORA_API int64_t ora_ray_columns(const ora_cfg *cf, const double p_in[3], const double k[3], double cols[3])
{
    double p[3] = {p_in[0], p_in[1], p_in[2]};
    wrap_periodic(cf, p, k);
    int64_t level, ijk[3];
    int64_t leaf = descend(cf, p, k, &level, ijk);
    cols[0] = cols[1] = cols[2] = 0.0;
    if (leaf < 0) return 0;
    double inv[3];
    inverse_dir(k, inv);
    int64_t n = 0;
    for (long guard = 0; guard < 100000000L; ++guard) {
        ora_state tmp;
        memcpy(tmp.p, p, sizeof p);
        memcpy(tmp.k, k, sizeof tmp.k);
        tmp.level = level;
        memcpy(tmp.ijk, ijk, sizeof ijk);
        int axis;
        double tf = face_distance(&tmp, inv, &axis);
        double tb = border_distance(cf, p, k, inv);
        double l = tb <= tf ? tb : tf;
        double lc = l * cf->box_cm;
        cols[0] += (double)cf->n_HI[leaf] * lc;
        cols[1] += (double)cf->n_dust[leaf] * lc;
        cols[2] += (cf->n_metal ? (double)cf->n_metal[leaf] : 0.0) * lc;
        ++n;
        if (tb <= tf) break;
        if (cross_face(cf, p, k, axis, tf, &leaf, &level, ijk)) break;
    }
    return n;
}

/* detector bins of a peeling event: channel (or -1) and pixel (or -1) */
static void peel_bins(const ora_cfg *cf, const double p[3], int d, double nu_o_ext, int64_t *ch, int64_t *px)
{
    const double *ko = cf->dirs[d];
    double t = (nu_o_ext - cf->nu_lo) / (cf->nu_hi - cf->nu_lo);
    int64_t c = (int64_t)floor(t * (double)cf->nbin);
    *ch = (c >= 0 && c < cf->nbin) ? c : -1;
    *px = -1;
    if (cf->npix > 0) {
        double eu[3], ev[3];
        onb(ko, eu, ev);
        double r[3] = {p[0] - cf->img_c[0], p[1] - cf->img_c[1], p[2] - cf->img_c[2]};
        double u = r[0] * eu[0] + r[1] * eu[1] + r[2] * eu[2];
        double v = r[0] * ev[0] + r[1] * ev[1] + r[2] * ev[2];
        int64_t iu = (int64_t)floor((u / cf->fov + 0.5) * (double)cf->npix);
        int64_t iv = (int64_t)floor((v / cf->fov + 0.5) * (double)cf->npix);
        if (iu >= 0 && iu < cf->npix && iv >= 0 && iv < cf->npix) *px = iv * cf->npix + iu;
    }
}

/* The oracle applies no peeling cut-off of its own (Sect. 5.1 peeling sums
 * w exp(-tau) over every event): a ray is walked until exp(-tau) underflows
 * to zero in double precision.  Beyond tau = 746, exp(-tau) is 0 in IEEE
 * binary64 (the smallest subnormal is exp(-744.4)), so stopping there leaves
 * every tally and every gradient bit-identical to walking on to the border. */
#define ORA_TAU_UNDERFLOW 746.0

/* add the contribution w exp(-tau) of one event to spectra, images, cubes */
static void peel_deposit(const ora_cfg *cf, ora_tally *ty, const ora_peel_event *e)
{
    int d = (int)e->dir;
    double tau = ray_tau(cf, e->p, cf->dirs[d], e->nu, e->leaf, e->level, e->ijk, ORA_TAU_UNDERFLOW, 0, 0, 0, 0);
    if (tau > ORA_TAU_UNDERFLOW) return;
    double f = e->w * exp(-tau);
    int64_t ch, px;
    peel_bins(cf, e->p, d, e->nu, &ch, &px);
    if (ch >= 0 && ty->pspec) ty->pspec[d * cf->nbin + ch] += f;
    if (px >= 0) {
        if (ty->pimg) ty->pimg[d * cf->npix * cf->npix + px] += f;
        if (ch >= 0 && cf->cube && ty->pcube) ty->pcube[(d * cf->npix * cf->npix + px) * cf->nbin + ch] += f;
    }
}

static void peel_add(const ora_cfg *cf, ora_tally *ty, const ora_state *s, int d,
                     double w, double nu_o_ext)
{
    ora_peel_event e;
    memcpy(e.p, s->p, sizeof e.p);
    e.leaf = s->leaf;
    e.level = s->level;
    memcpy(e.ijk, s->ijk, sizeof e.ijk);
    e.dir = d;
    e.w = w;
    e.nu = nu_o_ext;
    if (ty->events && ty->nev < ty->cap) ty->events[ty->nev] = e;
    if (ty->events) ty->nev++;
    ty->npeel++;
    peel_deposit(cf, ty, &e);
}

ORA_API void ora_peel_from_events(const ora_cfg *cf, const ora_peel_event *ev, int64_t n, ora_tally *ty)
{
    for (int64_t i = 0; i < n; ++i) peel_deposit(cf, ty, ev + i);
}

/* ------------------------------------------------------------------ */
/* adjoint of the peeled optical depths with the event record fixed     */
/* ------------------------------------------------------------------ */

/* Tasitsiomi H(a,x) with its partial derivatives in a and x */
ORA_API void ora_voigt_derivs(double a, double x, double *H, double *dHda, double *dHdx)
{
    double s = x * x;
    double e = exp(-s);
    double Q = 0.0, dQds = 0.0;
    double z = (s - 0.855) / (s + 3.42);
    if (z > 0.0) {
        double zp = 4.275 / ((s + 3.42) * (s + 3.42));
        double P = 0.1117 + z * (4.421 + z * (-9.207 + 5.674 * z));
        double Pp = 4.421 + z * (-18.414 + 17.022 * z);
        double A1 = 1.0 + 21.0 / s;
        double den = OPI * (s + 1.0);
        Q = z * A1 * P / den;
        dQds = (zp * A1 * P - z * (21.0 / (s * s)) * P + z * A1 * Pp * zp) / den - Q / (s + 1.0);
    }
    *H = sqrt(OPI) * a * Q + e;
    *dHda = sqrt(OPI) * Q;
    *dHdx = sqrt(OPI) * a * dQds * 2.0 * x - 2.0 * x * e;
}

/* The Faddeeva H(a,x) with its partial derivatives: with w' = -2 z w +
 * 2i/sqrt(pi), dH/dx = Re w' = 2 (a Im w - x H) and dH/da = Re(i w') =
 * 2 (x Im w + a H) - 2/sqrt(pi). */
ORA_API void ora_faddeeva_derivs(double a, double x, double *H, double *dHda, double *dHdx)
{
    double re, im;
    ora_faddeeva(a, x, &re, &im);
    *H = re;
    *dHda = 2.0 * (x * im + a * re) - 2.0 / sqrt(OPI);
    *dHdx = 2.0 * (a * im - x * re);
}

/* d kappa / d theta of one leaf at external frequency nu along k, for theta =
 * (n_HI, vx, vy, vz, T, n_dust) */
static void opacity_grad(const ora_cfg *cf, int64_t leaf, double nu_ext, const double k[3], double dk[6])
{
    double b = beta_of(cf, leaf, k);
    double nu_gas = nu_ext / (1.0 + b);
    double T = (double)cf->T[leaf];
    for (int j = 0; j < 6; ++j) dk[j] = 0.0;
    for (int il = 0; il < cf->nline; ++il) {
        ora_lineprop lp;
        line_props(cf, il, leaf, nu_gas, &lp);
        double H, dHa, dHx;
        if (cf->voigt == 1) ora_faddeeva_derivs(lp.a, lp.x, &H, &dHa, &dHx);
        else ora_voigt_derivs(lp.a, lp.x, &H, &dHa, &dHx);
        double s0 = sqrt(OPI) * OE * OE * cf->line_f[il] / (OME * OC * lp.dnu);
        double nX = line_density(cf, il, leaf);
        if (cf->line_dens[il] != 1) dk[0] += cf->line_abund[il] * s0 * H;
        /* x = (nu_ext/(1+beta) - nu0)/dnu:  dx/dv_j = -nu_gas k_j / (c (1+beta) dnu) */
        double dxdv = -nu_gas / (OC * (1.0 + b) * lp.dnu);
        for (int j = 0; j < 3; ++j) dk[1 + j] += nX * s0 * dHx * dxdv * k[j];
        /* sigma0, a and x all scale as T^-1/2 */
        dk[4] += nX * s0 * (-0.5 / T) * (H + lp.a * dHa + lp.x * dHx);
    }
    dk[5] = cf->dust_sigma;
}

/* second walk of a ray: grad[j][leaf] += scale * L * l * dkappa_j/dtheta */
static void ray_grad(const ora_cfg *cf, const ora_peel_event *e, double scale, double *grad)
{
    const double *k = cf->dirs[e->dir];
    double p[3] = {e->p[0], e->p[1], e->p[2]};
    int64_t leaf = e->leaf, level = e->level, ijk[3] = {e->ijk[0], e->ijk[1], e->ijk[2]};
    double inv[3];
    inverse_dir(k, inv);
    int64_t n = cf->nleaf;
    for (long guard = 0; guard < 100000000L; ++guard) {
        ora_state tmp;
        memcpy(tmp.p, p, sizeof p);
        memcpy(tmp.k, k, sizeof tmp.k);
        tmp.level = level;
        memcpy(tmp.ijk, ijk, sizeof ijk);
        int axis;
        double tf = face_distance(&tmp, inv, &axis);
        double tb = border_distance(cf, p, k, inv);
        double l = tb <= tf ? tb : tf;
        double dk[6];
        opacity_grad(cf, leaf, e->nu, k, dk);
        for (int j = 0; j < 6; ++j) grad[j * n + leaf] += scale * cf->box_cm * l * dk[j];
        if (tb <= tf) break;
        if (cross_face(cf, p, k, axis, tf, &leaf, &level, ijk)) break;
    }
}

/* gradient of L = sum g_cube*cube + g_img*img + g_spec*spec over the events:
 * dL/dtheta_c = -sum_e G_e w_e exp(-tau_e) d tau_e / d theta_c */
ORA_API void ora_adjoint_events(const ora_cfg *cf, const ora_peel_event *ev, int64_t n, const double *g_cube,
                                const double *g_img, const double *g_spec, double *grad)
{
    for (int64_t i = 0; i < n; ++i) {
        const ora_peel_event *e = ev + i;
        int d = (int)e->dir;
        double tau = ray_tau(cf, e->p, cf->dirs[d], e->nu, e->leaf, e->level, e->ijk, ORA_TAU_UNDERFLOW, 0, 0, 0, 0);
        if (tau > ORA_TAU_UNDERFLOW) continue;
        int64_t ch, px;
        peel_bins(cf, e->p, d, e->nu, &ch, &px);
        double G = 0.0;
        if (ch >= 0 && g_spec) G += g_spec[d * cf->nbin + ch];
        if (px >= 0 && g_img) G += g_img[d * cf->npix * cf->npix + px];
        if (px >= 0 && ch >= 0 && g_cube && cf->cube) G += g_cube[(d * cf->npix * cf->npix + px) * cf->nbin + ch];
        if (G == 0.0) continue;
        ray_grad(cf, e, -G * e->w * exp(-tau), grad);
    }
}

/* ------------------------------------------------------------------ */
/* interactions (Sect. 3.2)                                             */
/* ------------------------------------------------------------------ */

/* peel towards every direction for an isotropic emission at the current
 * position, gas-frame frequency nu_gas of the current cell */
static void peel_emission(const ora_cfg *cf, ora_tally *ty, const ora_state *s, double nu_gas)
{
    for (int d = 0; d < cf->ndir; ++d) {
        double nu_o = nu_gas * (1.0 + beta_of(cf, s->leaf, cf->dirs[d]));
        peel_add(cf, ty, s, d, 1.0 / (4.0 * OPI), nu_o);
    }
}

/* peeling of the emission of a packet in state s (its first event) */
ORA_API void ora_emission(const ora_cfg *cf, const ora_state *s, ora_tally *ty)
{
    if (s->status != ORA_ACTIVE || cf->ndir < 1) return;
    peel_emission(cf, ty, s, s->nu / (1.0 + beta_of(cf, s->leaf, s->k)));
}

static void scatter_dust(const ora_cfg *cf, ora_state *s, ora_tally *ty, double nu_gas)
{
    double r_alb = u23(cf, s);
    if (r_alb > cf->dust_albedo) {
        s->status = ORA_ABSORBED;
        return;
    }
    double r_mu = u23(cf, s), r_phi = u23(cf, s);
    double mu = ora_mu_sample(PH_HG, r_mu, cf->dust_g);
    double kin[3] = {s->k[0], s->k[1], s->k[2]};
    double kout[3];
    if (cf->keep_dir) memcpy(kout, kin, sizeof kout);
    else dir_from(kin, mu, 2.0 * OPI * r_phi, kout);
    for (int d = 0; d < cf->ndir; ++d) {
        const double *ko = cf->dirs[d];
        double muo = kin[0] * ko[0] + kin[1] * ko[1] + kin[2] * ko[2];
        double w = ora_phase(PH_HG, muo, cf->dust_g) / (2.0 * OPI);
        double nu_o = nu_gas * (1.0 + beta_of(cf, s->leaf, ko));
        peel_add(cf, ty, s, d, w, nu_o);
    }
    memcpy(s->k, kout, sizeof kout);
    s->nu = nu_gas * (1.0 + beta_of(cf, s->leaf, s->k));
    ty->nscatt_dust++;
}

/* Perpendicular velocity components (u_perp1, u_perp2) of the scatterer
 * (Sect. 3.2.1: each from the unbiased Gaussian exp(-u^2)/sqrt(pi)), drawn
 * as a pair in polar form from two words.  Core-skipping (Sect. 3.2.1, after
 * Ahn et al. 2002; the truncated draw of Dijkstra et al. 2006): when
 * |x_in| < x_crit the pair comes from the same 2-D Gaussian restricted to
 * |u_perp| >= x_crit, whose radius has P(|u_perp| > r) = exp(x_crit^2 - r^2),
 * so r = sqrt(x_crit^2 - ln r1).  x_crit = 0 is the plain draw. */
static void sample_uperp(const ora_cfg *cf, ora_state *s, double x_in, double x_crit, double *u1, double *u2)
{
    double r1 = u23(cf, s), r2 = u23(cf, s);
    double xc2 = fabs(x_in) < x_crit ? x_crit * x_crit : 0.0;
    double rho = sqrt(xc2 - log(r1));
    *u1 = rho * cos(2.0 * OPI * r2);
    *u2 = rho * sin(2.0 * OPI * r2);
}

/* exported for the pins: n pairs from one packet stream, starting at draw 0 */
ORA_API void ora_sample_uperp_n(const ora_cfg *cf, uint64_t pid, double x_in, double x_crit, int64_t n, double *out)
{
    ora_state s;
    memset(&s, 0, sizeof s);
    s.pid = pid;
    for (int64_t i = 0; i < n; ++i) sample_uperp(cf, &s, x_in, x_crit, out + 2 * i, out + 2 * i + 1);
}

/* Critical frequency of core-skipping for a scattering on line il in the
 * packet's leaf.  The paper uses the scheme of Smith et al. (2015) without
 * printing it; the reading taken here scales x_crit with (a tau_cell)^(1/3),
 * the frequency scale at which a thick medium lets photons out (the slab
 * spectrum of Sect. 3.4.2 peaks near 1.07 (a tau0)^(1/3)), with tau_cell the
 * line-centre optical depth across the leaf (H -> 1) and a user factor. */
static double core_skip_xcrit(const ora_cfg *cf, int il, const ora_state *s, const ora_lineprop *lp)
{
    if (cf->core_skip_f > 0.0) {
        double sigma0 = sqrt(OPI) * OE * OE * cf->line_f[il] / (OME * OC * lp->dnu);
        double tau_cell = line_density(cf, il, s->leaf) * sigma0 * ldexp(1.0, -(int)s->level) * cf->box_cm;
        return cf->core_skip_f * cbrt(lp->a * tau_cell);
    }
    return cf->core_skip;
}

/* exported for the pins: x_crit of line il in leaf `leaf` at level `level` */
ORA_API double ora_core_skip_xcrit(const ora_cfg *cf, int64_t il, int64_t leaf, int64_t level)
{
    ora_state s;
    memset(&s, 0, sizeof s);
    s.leaf = leaf;
    s.level = level;
    ora_lineprop lp;
    line_props(cf, (int)il, leaf, cf->line_nu[il], &lp);
    return core_skip_xcrit(cf, (int)il, &s, &lp);
}

static int scatter_line(const ora_cfg *cf, ora_state *s, ora_tally *ty, int il, double nu_gas)
{
    int64_t leaf = s->leaf;
    ora_lineprop lp;
    line_props(cf, il, leaf, nu_gas, &lp);
    /* decay channel (Sect. 3.2.3): P_i = A_i / sum A */
    int ch = 0;
    if (cf->line_nchan[il] > 1) {
        double r = u23(cf, s);
        double Atot = 0.0;
        for (int c = 0; c < cf->line_nchan[il]; ++c) Atot += cf->chan_A[il][c];
        double acc = 0.0;
        ch = (int)cf->line_nchan[il] - 1;
        for (int c = 0; c < cf->line_nchan[il]; ++c) {
            acc += cf->chan_A[il][c];
            if (r * Atot < acc) {
                ch = c;
                break;
            }
        }
    }
    int err = 0;
    double upar = sample_upar(cf, s, lp.x, lp.a, &err);
    if (err) return 1;
    double up1, up2;
    sample_uperp(cf, s, lp.x, core_skip_xcrit(cf, il, s, &lp), &up1, &up2);
    double kin[3] = {s->k[0], s->k[1], s->k[2]};
    double e1[3], e2[3];
    onb(kin, e1, e2);
    double vX[3];   /* scatterer velocity in units of vth */
    for (int i = 0; i < 3; ++i) vX[i] = upar * kin[i] + up1 * e1[i] + up2 * e2[i];
    int kind;
    if (ch > 0 || cf->isotropic || cf->line_phase[il] != 0) kind = PH_ISO;
    else kind = fabs(lp.x - upar) < 0.2 ? PH_CORE : PH_WING;
    double r_mu = u23(cf, s), r_phi = u23(cf, s);
    double mu = ora_mu_sample(kind, r_mu, 0.0);
    double kout[3];
    if (cf->keep_dir) {
        memcpy(kout, kin, sizeof kout);
        mu = 1.0;
    } else {
        dir_from(kin, mu, 2.0 * OPI * r_phi, kout);
    }
    double m = cf->line_m[il];
    /* peeling: same atom, outgoing direction k_o */
    for (int d = 0; d < cf->ndir; ++d) {
        const double *ko = cf->dirs[d];
        double muo = kin[0] * ko[0] + kin[1] * ko[1] + kin[2] * ko[2];
        double uo = ko[0] * vX[0] + ko[1] * vX[1] + ko[2] * vX[2];
        double nu_o;
        if (ch > 0) {
            nu_o = cf->chan_nu[il][ch] * (1.0 + uo * lp.vth / OC);
        } else {
            double rec = cf->recoil ? (1.0 - muo) * OH * nu_gas / (m * OC * OC) : 0.0;
            nu_o = nu_gas * (1.0 + (uo - upar) * lp.vth / OC) / (1.0 + rec);
        }
        double w = ora_phase(kind, muo, 0.0) / (2.0 * OPI);
        peel_add(cf, ty, s, d, w, nu_o * (1.0 + beta_of(cf, leaf, ko)));
    }
    double uout = kout[0] * vX[0] + kout[1] * vX[1] + kout[2] * vX[2];
    double nu_out;
    if (ch > 0) {
        nu_out = cf->chan_nu[il][ch] * (1.0 + uout * lp.vth / OC);
    } else {
        /* Eq. (nuout_nuin) */
        double rec = cf->recoil ? (1.0 - mu) * OH * nu_gas / (m * OC * OC) : 0.0;
        nu_out = nu_gas * (1.0 + (uout - upar) * lp.vth / OC) / (1.0 + rec);
    }
    memcpy(s->k, kout, sizeof kout);
    s->nu = nu_out * (1.0 + beta_of(cf, leaf, s->k));
    ty->nscatt_line++;
    return 0;
}

/* ------------------------------------------------------------------ */
/* one event: draw tau_event, walk, interact (Sect. 3, Eq. tau_event)   */
/* ------------------------------------------------------------------ */
ORA_API int ora_init_state(const ora_cfg *cf, ora_state *s, const double p[3], const double k[3],
                           double nu, uint64_t pid)
{
    memset(s, 0, sizeof *s);
    memcpy(s->p, p, sizeof s->p);
    memcpy(s->k, k, sizeof s->k);
    s->nu = nu;
    s->pid = pid;
    wrap_periodic(cf, s->p, s->k);
    s->leaf = descend(cf, s->p, s->k, &s->level, s->ijk);
    s->status = s->leaf < 0 ? ORA_ERROR : ORA_ACTIVE;
    return (int)s->status;
}

ORA_API int ora_event(const ora_cfg *cf, ora_state *s, ora_tally *ty)
{
    if (s->status != ORA_ACTIVE) return (int)s->status;
    double tau_rem = -log(u52(cf, s));
    double inv[3];
    inverse_dir(s->k, inv);
    for (;;) {
        if (cf->max_steps > 0 && s->nsteps >= cf->max_steps) {
            s->status = ORA_CAPPED;
            return (int)s->status;
        }
        s->nsteps++;
        int axis;
        double tf = face_distance(s, inv, &axis);
        double tb = border_distance(cf, s->p, s->k, inv);
        int border = tb <= tf;
        double l = border ? tb : tf;
        double kl[ORA_MAXLINE], kd;
        double kap = opacity(cf, s->leaf, s->nu, s->k, kl, &kd);
        double tau_cell = kap * l * cf->box_cm;
        if (tau_cell >= tau_rem) {
            /* interaction inside this cell */
            double li = tau_rem / (kap * cf->box_cm);
            for (int ax = 0; ax < 3; ++ax) s->p[ax] = fma(li, s->k[ax], s->p[ax]);
            s->path += li;
            double r = u23(cf, s);
            double nu_gas = s->nu / (1.0 + beta_of(cf, s->leaf, s->k));
            /* Sect. 3.2: dust with P = tau_d/tau, else line X with P = tau_X/tau */
            double acc = kd;
            if (r * kap < acc) {
                scatter_dust(cf, s, ty, nu_gas);
            } else {
                int il = (int)cf->nline - 1;
                for (int i = 0; i < cf->nline; ++i) {
                    acc += kl[i];
                    if (r * kap < acc) {
                        il = i;
                        break;
                    }
                }
                if (scatter_line(cf, s, ty, il, nu_gas)) {
                    s->status = ORA_ERROR;
                    return (int)s->status;
                }
            }
            if (s->status == ORA_ACTIVE) {
                s->nscatt++;
                if (cf->max_scatt > 0 && s->nscatt >= cf->max_scatt) s->status = ORA_CAPPED;
            }
            return (int)s->status;
        }
        tau_rem -= tau_cell;
        s->path += l;
        if (border) {
            for (int ax = 0; ax < 3; ++ax) s->p[ax] = fma(l, s->k[ax], s->p[ax]);
            s->status = ORA_ESCAPED;
            return (int)s->status;
        }
        ty->ncross++;
        if (cross_face(cf, s->p, s->k, axis, tf, &s->leaf, &s->level, s->ijk)) {
            s->status = ORA_ESCAPED;
            return (int)s->status;
        }
    }
}

static void escape_tally(const ora_cfg *cf, ora_tally *ty, const ora_state *s)
{
    if (s->status != ORA_ESCAPED || !ty->spec) return;
    double t = (s->nu - cf->nu_lo) / (cf->nu_hi - cf->nu_lo);
    int64_t b = (int64_t)floor(t * (double)cf->nbin);
    if (b >= 0 && b < cf->nbin) ty->spec[b] += 1.0;
}

/* propagate packets [0, n): outputs per packet (nullable) and tallies */
ORA_API int ora_run(const ora_cfg *cf, int64_t n, const double *pos, const double *dir,
                    const double *nu, const uint64_t *ids,
                    int32_t *status, int64_t *nscatt, double *nu_out, double *pos_out,
                    double *dir_out, double *path_out, ora_tally *ty)
{
    for (int64_t i = 0; i < n; ++i) {
        ora_state s;
        ora_init_state(cf, &s, pos + 3 * i, dir + 3 * i, nu[i], ids[i]);
        if (s.status == ORA_ACTIVE && cf->ndir > 0) {
            double nu_gas = s.nu / (1.0 + beta_of(cf, s.leaf, s.k));
            peel_emission(cf, ty, &s, nu_gas);
        }
        while (s.status == ORA_ACTIVE) ora_event(cf, &s, ty);
        escape_tally(cf, ty, &s);
        if (status) status[i] = (int32_t)s.status;
        if (nscatt) nscatt[i] = s.nscatt;
        if (nu_out) nu_out[i] = s.nu;
        if (pos_out) memcpy(pos_out + 3 * i, s.p, sizeof s.p);
        if (dir_out) memcpy(dir_out + 3 * i, s.k, sizeof s.k);
        if (path_out) path_out[i] = s.path;
    }
    return 0;
}

ORA_API int64_t ora_sizeof_cfg(void) { return (int64_t)sizeof(ora_cfg); }
ORA_API int64_t ora_sizeof_state(void) { return (int64_t)sizeof(ora_state); }
ORA_API int64_t ora_sizeof_tally(void) { return (int64_t)sizeof(ora_tally); }
ORA_API int64_t ora_sizeof_event(void) { return (int64_t)sizeof(ora_peel_event); }

"""Seeded synthetic inputs for the resonant-line Monte Carlo transfer path.

This package only *generates inputs*: graded octrees, per-leaf gas fields,
photon-packet initial conditions (the "PPIC" lists of the paper, Sect. 2:
ID, position, direction, frequency) and the atomic data of Table 1.  It holds
none of the transfer method's arithmetic (no opacities, no Voigt function,
no scattering, no walk).  Both the CUDA path and the FP64 oracle consume what
it returns, so neither depends on the other.

The one place where a physical formula appears is the *recipe* that turns a
stated line-centre optical depth into a density (``density_for_tau0``): a
workload is specified by its optical depth, and converting that number into
the n_HI value written into the leaf arrays is part of defining the input.
It uses its own copy of the CODATA constants.

Geometry conventions (shared by every consumer):
  * the simulation box is the unit cube [0,1)^3 in box units, of physical
    size ``box_cm``;
  * oct 0 is the root oct at level 1 (its 8 cells have size 1/2);
  * ``son[8*oct + child]`` with ``child = (ix&1) | (iy&1)<<1 | (iz&1)<<2``
    (ix,iy,iz the integer coordinates of the cell at its level) holds either
    the index (>0) of the oct that refines the cell, or ``-(leaf+1)`` for a
    leaf cell (Sect. 4.3, Fig. "amr_struct": positive son = oct, negative
    son = leaf index into the physical-property arrays);
  * octs and leaves are numbered depth-first (Sect. 4.3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# CODATA 2018 constants, cgs (the paper prints none).  Used only by the input
# recipe below (density from a stated optical depth, line frequencies).
# --------------------------------------------------------------------------
C_CGS = 2.99792458e10
KB_CGS = 1.380649e-16
H_CGS = 6.62607015e-27
ME_CGS = 9.1093837015e-28
E_ESU = 4.803204712570263e-10
MP_CGS = 1.67262192369e-24
AMU_CGS = 1.66053906660e-24
KPC_CM = 3.0856775814913673e21

# --------------------------------------------------------------------------
# Table 1 (Appendix A): atomic data.  Wavelengths are vacuum, in Angstrom.
# Each absorption line lists its decay channels; channel 0 is the resonant
# one (same lower level), the others are fluorescent (Sect. 3.2.3).
# --------------------------------------------------------------------------


@dataclass
class Line:
    name: str
    lambda_A: float        # absorption line wavelength (Angstrom)
    A_ul: float            # Einstein A of the resonant channel (s^-1)
    f_lu: float            # oscillator strength
    mass_g: float          # scatterer mass (g)
    density: int = 0       # 0: n_HI field, 1: n_metal field, 2: n_HI * abundance
    abundance: float = 1.0  # multiplies the density field (deuterium: D/H)
    phase: int = 0         # 0: Lya core/wing (Eqs. Pcore/Pwing), 1: isotropic
    channels: list = field(default_factory=list)  # [(A_ul_i, lambda_i_A)], [0] resonant

    def all_channels(self):
        return [(self.A_ul, self.lambda_A)] + list(self.channels)


def lya():
    """H I Lyman-alpha, Table 1 row 1 (1215.67 A, A=6.265e8, f=0.416)."""
    return Line("HI_1216", 1215.67, 6.265e8, 0.416, MP_CGS, density=0, phase=0)


def d_lya(d_over_h=3.0e-5):
    """D Lyman-alpha, Table 1 row 2 (1215.34 A), density n_HI * D/H."""
    return Line("DI_1215", 1215.34, 6.265e8, 0.416, 2.01410177812 * AMU_CGS,
                density=2, abundance=d_over_h, phase=0)


def siII_1190():
    """Si II 1190.42 A (A=6.53e8, f=0.277) with fluorescent 1194.50* (A=3.45e9)."""
    return Line("SiII_1190", 1190.42, 6.53e8, 0.277, 28.0855 * AMU_CGS,
                density=1, phase=1, channels=[(3.45e9, 1194.50)])


def siII_1193():
    """Si II 1193.28 A (A=2.69e9, f=0.575) with fluorescent 1197.39* (A=1.40e9)."""
    return Line("SiII_1193", 1193.28, 2.69e9, 0.575, 28.0855 * AMU_CGS,
                density=1, phase=1, channels=[(1.40e9, 1197.39)])


def feII_2344():
    """Fe II 2344.21 A (A=1.73e8, f=0.114) with fluorescent 2365.55* (A=5.90e7)
    and 2381.49* (A=3.10e7): the UV1 multiplet line with three channels."""
    return Line("FeII_2344", 2344.21, 1.73e8, 0.114, 55.845 * AMU_CGS,
                density=1, phase=1, channels=[(5.90e7, 2365.55), (3.10e7, 2381.49)])


def feII_2374():
    """Fe II 2374.46 A (A=4.25e7, f=0.0359) with fluorescent 2396.35* (A=2.59e8)."""
    return Line("FeII_2374", 2374.46, 4.25e7, 0.0359, 55.845 * AMU_CGS,
                density=1, phase=1, channels=[(2.59e8, 2396.35)])


def mgII_2796():
    """Mg II 2796.35 A (A=2.60e8, f=0.608), resonant only."""
    return Line("MgII_2796", 2796.35, 2.60e8, 0.608, 24.305 * AMU_CGS, density=1, phase=1)


def mgII_2803():
    """Mg II 2803.53 A (A=2.57e8, f=0.303), resonant only."""
    return Line("MgII_2803", 2803.53, 2.57e8, 0.303, 24.305 * AMU_CGS, density=1, phase=1)


def nu_of(lambda_A):
    return C_CGS / (lambda_A * 1e-8)


def doppler_width(line: Line, T):
    return nu_of(line.lambda_A) * math.sqrt(2.0 * KB_CGS * T / line.mass_g) / C_CGS


def density_for_tau0(line: Line, T, tau0, length_cm):
    """Recipe: n such that n * sigma0 * length = tau0, with sigma0 the
    line-centre cross section of Eq. (sigma) taken with H -> 1."""
    dnu = doppler_width(line, T)
    sigma0 = math.sqrt(math.pi) * E_ESU ** 2 * line.f_lu / (ME_CGS * C_CGS * dnu)
    return tau0 / (sigma0 * length_cm)


# --------------------------------------------------------------------------
# Graded octree builder
# --------------------------------------------------------------------------


def _part1by2(v):
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton(ix, iy, iz):
    return _part1by2(ix) | (_part1by2(iy) << np.uint64(1)) | (_part1by2(iz) << np.uint64(2))


_CHILD = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], dtype=np.int64)


@dataclass
class Octree:
    son: np.ndarray          # int32 [8*noct]
    oct_level: np.ndarray    # int32 [noct]
    oct_origin: np.ndarray   # int64 [noct,3] integer coords of child 0 at the oct's level
    leaf_level: np.ndarray   # int32 [nleaf]
    leaf_ijk: np.ndarray     # int64 [nleaf,3] integer coords at the leaf's level
    max_level: int

    @property
    def noct(self):
        return int(self.oct_level.size)

    @property
    def nleaf(self):
        return int(self.leaf_level.size)

    def leaf_centres(self):
        h = np.ldexp(1.0, -self.leaf_level.astype(np.int64))
        return (self.leaf_ijk.astype(np.float64) + 0.5) * h[:, None]

    def leaf_size(self):
        return np.ldexp(1.0, -self.leaf_level.astype(np.int64))


def build_octree(refine, max_level):
    """Build a depth-first-numbered octree.

    ``refine(level, i, j, k)`` gets int64 arrays of integer cell coordinates at
    ``level`` and returns a bool array: which of those cells are split.  Cells
    at ``max_level`` are never split.
    """
    levels, origins = [], []
    cur = np.zeros((1, 3), dtype=np.int64)  # octs at level 1
    lvl = 1
    cell_ref = []  # per level: bool [noct_l*8]
    while True:
        levels.append(np.full(cur.shape[0], lvl, dtype=np.int32))
        origins.append(cur)
        cells = (cur[:, None, :] + _CHILD[None, :, :]).reshape(-1, 3)
        if lvl < max_level:
            r = np.asarray(refine(lvl, cells[:, 0], cells[:, 1], cells[:, 2]), dtype=bool)
        else:
            r = np.zeros(cells.shape[0], dtype=bool)
        cell_ref.append(r)
        if not r.any():
            break
        cur = 2 * cells[r]
        lvl += 1
    oct_level = np.concatenate(levels)
    oct_origin = np.concatenate(origins)
    refined = np.concatenate(cell_ref)
    noct = oct_level.size
    # BFS numbering: octs of level l+1 are created in the order of refined cells.
    son_bfs = np.empty(8 * noct, dtype=np.int64)
    child_oct_bfs = np.arange(1, noct, dtype=np.int64)
    son_bfs[refined] = child_oct_bfs
    cell_level = np.repeat(oct_level, 8)
    cell_ijk = (oct_origin[:, None, :] + _CHILD[None, :, :]).reshape(-1, 3)
    leaf_mask = ~refined
    leaf_lvl = cell_level[leaf_mask]
    leaf_ijk = cell_ijk[leaf_mask]
    # depth-first order == Morton order at the finest level (ties: coarser first)
    Lm = int(oct_level.max())
    okey = morton(*(oct_origin << (Lm - oct_level.astype(np.int64))[:, None]).T)
    oorder = np.lexsort((oct_level, okey))
    onew = np.empty(noct, dtype=np.int64)
    onew[oorder] = np.arange(noct)
    lkey = morton(*(leaf_ijk << (Lm - leaf_lvl.astype(np.int64))[:, None]).T)
    lorder = np.argsort(lkey, kind="stable")
    lnew = np.empty(leaf_lvl.size, dtype=np.int64)
    lnew[lorder] = np.arange(leaf_lvl.size)
    leaf_bfs_index = np.full(8 * noct, -1, dtype=np.int64)
    leaf_bfs_index[leaf_mask] = np.arange(leaf_lvl.size)
    son_new_val = np.where(refined, onew[np.where(refined, son_bfs, 0)],
                           -(lnew[np.maximum(leaf_bfs_index, 0)] + 1))
    son = np.empty(8 * noct, dtype=np.int32)
    cell_oct_new = np.repeat(onew, 8) * 8 + np.tile(np.arange(8), noct)
    son[cell_oct_new] = son_new_val
    assert np.all(son[1:8 * noct] != 0)
    return Octree(son=son,
                  oct_level=oct_level[oorder].astype(np.int32),
                  oct_origin=oct_origin[oorder],
                  leaf_level=leaf_lvl[lorder].astype(np.int32),
                  leaf_ijk=leaf_ijk[lorder],
                  max_level=Lm)


def uniform_octree(level):
    """Regular (2^level)^3 grid of leaves."""
    return build_octree(lambda l, i, j, k: np.full(i.shape, l < level), level)


def sphere_octree(base_level, max_level, centre=(0.5, 0.5, 0.5), radius=0.45, grade=2.0):
    """All cells up to ``base_level``; beyond it, a cell at level l is split
    while it lies within ``grade`` cell sizes of the ball.  With grade >=
    sqrt(3)+... >= 2 neighbouring leaves differ by at most one level."""
    c = np.asarray(centre, dtype=np.float64)

    def refine(l, i, j, k):
        h = math.ldexp(1.0, -l)
        lo = np.stack([i, j, k], 1) * h
        d = np.clip(c[None, :], lo, lo + h) - c[None, :]
        dist = np.sqrt((d * d).sum(1)) - radius
        return (l < base_level) | (dist < grade * h)

    return build_octree(refine, max_level)


def check_graded(tree: Octree):
    """True if face-neighbouring leaves differ by at most one level."""
    Lm = tree.max_level
    lut = {}
    for lv, (i, j, k), idx in zip(tree.leaf_level, tree.leaf_ijk, range(tree.nleaf)):
        lut[(int(lv), int(i), int(j), int(k))] = idx
    n = 1 << Lm
    for lv, (i, j, k) in zip(tree.leaf_level, tree.leaf_ijk):
        s = 1 << (Lm - lv)
        for ax in range(3):
            for sgn in (-1, 1):
                p = [i * s, j * s, k * s]
                p[ax] = p[ax] + (s if sgn > 0 else -1)
                if p[ax] < 0 or p[ax] >= n:
                    continue
                # leaf containing the fine point p
                found = None
                for l2 in range(1, Lm + 1):
                    key = (l2, p[0] >> (Lm - l2), p[1] >> (Lm - l2), p[2] >> (Lm - l2))
                    if key in lut:
                        found = l2
                        break
                if found is None or abs(found - int(lv)) > 1:
                    return False
    return True


# --------------------------------------------------------------------------
# Gas fields and workloads
# --------------------------------------------------------------------------


@dataclass
class Medium:
    tree: Octree
    box_cm: float
    n_HI: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    T: np.ndarray
    n_dust: np.ndarray
    n_metal: np.ndarray


def uniform_medium(tree, box_cm, n_HI, T, n_dust=0.0, n_metal=0.0):
    n = tree.nleaf
    f = lambda v: np.full(n, v, dtype=np.float32)
    return Medium(tree, float(box_cm), f(n_HI), f(0.0), f(0.0), f(0.0), f(T), f(n_dust), f(n_metal))


@dataclass
class Domain:
    kind: int            # 0 sphere, 1 slab (periodic x,y), 2 cube, 3 shell
    centre: tuple = (0.5, 0.5, 0.5)
    size: float = 0.45   # sphere / shell outer radius, slab half-thickness, cube half-size (box units)
    inner: float = 0.0   # shell inner radius


@dataclass
class Dust:
    sigma: float = 0.0   # cross section per unit n_dust (cm^2), constant across the line
    albedo: float = 0.32  # Sect. 3.2.2 default
    g: float = 0.73       # Henyey-Greenstein asymmetry, Sect. 3.2.2 default


@dataclass
class Physics:
    recoil: int = 1
    isotropic: int = 0         # 1: isotropic phase function for every line (test mode)
    keep_direction: int = 0    # 1: scatterings keep k (error-budget test, Sect. 4.5)
    x_gauss: float = 8.0       # u_par Gaussian branch threshold (Sect. 3.3.3 default)
    max_scatt: int = 0         # 0: no cap
    max_steps: int = 0         # 0: no cap
    tau_stop: float = 50.0     # peeling rays stop once tau exceeds this (contribution < e^-tau_stop)
    seed: int = 0
    voigt: int = 0             # H(a,x): 0 Tasitsiomi (2006), 1 the Faddeeva function (accurate option)
    core_skip: float = 0.0     # core-skipping critical frequency x_crit (0 = off)
    core_skip_f: float = 0.0   # > 0: x_crit = core_skip_f * (a tau_cell)^(1/3) per scattering instead


@dataclass
class Detector:
    """Frequency axis (external frame, Hz) shared by the escape spectrum and
    the peeled spectra/cubes, plus peeling directions and the image plane."""
    nu_lo: float
    nu_hi: float
    nbin: int
    dirs: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    npix: int = 0
    fov: float = 1.0                   # image side (box units)
    centre: tuple = (0.5, 0.5, 0.5)     # image centre (box units)
    cube: int = 0                      # 1: accumulate spectral cubes


@dataclass
class Packets:
    pos: np.ndarray   # float64 [n,3] box units
    dir: np.ndarray   # float64 [n,3] unit vectors
    nu: np.ndarray    # float64 [n] external-frame frequency (Hz) along dir
    ids: np.ndarray   # uint64 [n]

    @property
    def n(self):
        return int(self.nu.size)


def point_source(n, pos, nu, seed, first_id=0):
    """n packets at ``pos`` with isotropic directions (Sect. 2: isotropic
    sources) and frequency ``nu``; directions from numpy's PCG64 stream."""
    rng = np.random.default_rng(seed)
    mu = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    d = np.stack([s * np.cos(phi), s * np.sin(phi), mu], 1)
    d /= np.linalg.norm(d, axis=1)[:, None]
    p = np.tile(np.asarray(pos, dtype=np.float64), (n, 1))
    return Packets(p, d, np.full(n, float(nu)), np.arange(first_id, first_id + n, dtype=np.uint64))


@dataclass
class Workload:
    name: str
    medium: Medium
    domain: Domain
    lines: list
    dust: Dust
    physics: Physics
    detector: Detector
    packets: Packets


RUN_SEED = 2001_11252


def x_axis(line: Line, T, xlo, xhi, nbin):
    """Detector frequency axis from a range in Doppler units x of ``line`` at T
    (x = (nu - nu0)/Delta nu_D, Sect. 3.1.1)."""
    nu0, dnu = nu_of(line.lambda_A), doppler_width(line, T)
    return nu0 + xlo * dnu, nu0 + xhi * dnu, nbin


def slab(tau0=1e4, T=1e4, n_packets=2000, level=4, recoil=0, isotropic=1, seed_offset=0, tau_dust=0.0,
         albedo=0.32):
    """Static homogeneous H I slab (Sect. 3.4.2): (2^level)^3 grid, slab
    domain |z-1/2| <= 1/2 with periodic x,y, half-thickness line-centre
    optical depth tau0, T, zero velocity, half-thickness dust optical depth
    tau_dust (albedo, g = 0.73); packets at the mid-plane at x_in = 0,
    isotropic."""
    tree = uniform_octree(level)
    L = 1.0 * KPC_CM
    line = lya()
    n = density_for_tau0(line, T, tau0, 0.5 * L) if tau0 > 0 else 0.0
    dust = Dust(sigma=4.0e-22, albedo=albedo)
    med = uniform_medium(tree, L, n, T, n_dust=tau_dust / (dust.sigma * 0.5 * L))
    seed = RUN_SEED + 0 + seed_offset
    pk = point_source(n_packets, (0.5, 0.5, 0.5), nu_of(line.lambda_A), seed ^ 0xA5A5)
    lo, hi, nb = x_axis(line, T, -60.0, 60.0, 200)
    return Workload("slab", med, Domain(1, (0.5, 0.5, 0.5), 0.5), [line], dust,
                    Physics(recoil=recoil, isotropic=isotropic, seed=seed), Detector(lo, hi, nb), pk)


def sphere(tau0=1e6, T=1e4, tau_dust=0.0, n_packets=1_000_000, base=3, max_level=6,
           recoil=0, isotropic=0, seed_offset=0, xrange=60.0):
    """Static homogeneous sphere, H I + dust (Sect. 3.4.2): 8^3 root refined to
    64^3 equivalent inside the sphere (centre 1/2, R=0.45 box), centre-to-edge
    line-centre optical depth tau0, dust albedo 0.32, centre-to-edge dust
    optical depth tau_dust; packets at the centre at x_in = 0."""
    tree = sphere_octree(base, max_level)
    L = 1.0 * KPC_CM
    R = 0.45
    line = lya()
    n = density_for_tau0(line, T, tau0, R * L)
    dust = Dust(sigma=4.0e-22)
    nd = tau_dust / (dust.sigma * R * L)
    med = uniform_medium(tree, L, n, T, n_dust=nd)
    seed = RUN_SEED + 1 + seed_offset
    pk = point_source(n_packets, (0.5, 0.5, 0.5), nu_of(line.lambda_A), seed ^ 0xA5A5)
    lo, hi, nb = x_axis(line, T, -xrange, xrange, 200)
    return Workload("sphere", med, Domain(0, (0.5, 0.5, 0.5), R), [line], dust,
                    Physics(recoil=recoil, isotropic=isotropic, seed=seed), Detector(lo, hi, nb), pk)


def deuterium_sphere(N_HI=2e19, T=1e4, d_over_h=3.0e-5, n_packets=10000, base=3, max_level=6, xrange=20.0,
                     with_d=True, seed_offset=0):
    """Static sphere of H I mixed with deuterium (Appendix A, Fig.
    sphere_deuterium_effect): centre-to-edge column N_HI, T, D/H, no dust,
    Lya packets at the centre at the H line centre (x_in = 0), core/wing
    phase functions, no recoil; spectrum in the H line's Doppler units over
    +-xrange.  with_d=False gives the pure H I sphere on the same packets."""
    tree = sphere_octree(base, max_level)
    L = 1.0 * KPC_CM
    R = 0.45
    h = lya()
    lines = [h, d_lya(d_over_h)] if with_d else [h]
    med = uniform_medium(tree, L, N_HI / (R * L), T)
    seed = RUN_SEED + 6 + seed_offset
    pk = point_source(n_packets, (0.5, 0.5, 0.5), nu_of(h.lambda_A), seed ^ 0xA5A5)
    lo, hi, nb = x_axis(h, T, -xrange, xrange, 200)
    return Workload("deuterium_sphere", med, Domain(0, (0.5, 0.5, 0.5), R), lines, Dust(sigma=4.0e-22),
                    Physics(recoil=0, isotropic=0, seed=seed), Detector(lo, hi, nb), pk)


def shell(tau0=1e4, T=1e4, inner=0.25, outer=0.45, n_packets=2000, v_max_kms=0.0, base=3, max_level=5,
          seed_offset=0):
    """Shell domain (Sect. 4: spheres, shells, cubes and slabs): uniform H I
    between radii `inner` and `outer` (box units) about the box centre, line
    centre optical depth tau0 across the shell (outer - inner), radial velocity
    v_max r / outer, no dust; packets uniform in the shell volume, isotropic,
    at line centre in the gas frame; packets escape through either sphere."""
    tree = sphere_octree(base, max_level, radius=outer)
    L = 1.0 * KPC_CM
    line = lya()
    n = density_for_tau0(line, T, tau0, (outer - inner) * L)
    med = uniform_medium(tree, L, n, T)
    if v_max_kms:
        ctr = tree.leaf_centres() - 0.5
        v = (v_max_kms * 1e5 / outer) * ctr
        med.vx, med.vy, med.vz = (v[:, i].astype(np.float32) for i in range(3))
    seed = RUN_SEED + 8 + seed_offset
    rng = np.random.default_rng(seed ^ 0xA5A5)
    r = (inner ** 3 + (outer ** 3 - inner ** 3) * rng.random(n_packets)) ** (1.0 / 3.0)
    u = rng.normal(size=(n_packets, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    pos = 0.5 + r[:, None] * u
    mu = 2.0 * rng.random(n_packets) - 1.0
    phi = 2.0 * math.pi * rng.random(n_packets)
    st = np.sqrt(1.0 - mu * mu)
    d = np.stack([st * np.cos(phi), st * np.sin(phi), mu], 1)
    vel = np.zeros((n_packets, 3))
    if v_max_kms:
        vel = (v_max_kms * 1e5 / outer) * (pos - 0.5)
    beta = (d * vel).sum(1) / C_CGS
    nu = nu_of(line.lambda_A) * (1.0 + beta)
    pk = Packets(pos, d, nu, np.arange(n_packets, dtype=np.uint64))
    lo, hi, nb = x_axis(line, T, -40.0, 40.0, 200)
    return Workload("shell", med, Domain(3, (0.5, 0.5, 0.5), outer, inner), [line], Dust(sigma=4.0e-22),
                    Physics(recoil=0, isotropic=0, seed=seed), Detector(lo, hi, nb), pk)


def mgII_wind(N_MgII=1e15, T=1e4, v_max_kms=200.0, n_packets=4000, base=3, max_level=5, seed_offset=0):
    """Mg II doublet in a wind (Table 1; the doublet of Sect. 1): centre-to-edge
    Mg II column N_MgII, a static core of radius R/10 and beyond it a radial
    velocity rising linearly to v_max at R, no dust; packets at the centre, 2/3
    at the 2796 and 1/3 at the 2803 line centre (the ratio of their oscillator
    strengths), isotropic; escape spectrum over 2785-2815 A."""
    tree = sphere_octree(base, max_level)
    L = 1.0 * KPC_CM
    R = 0.45
    med = uniform_medium(tree, L, 0.0, T, n_metal=N_MgII / (R * L))
    ctr = tree.leaf_centres() - 0.5
    r = np.linalg.norm(ctr, axis=1)
    rc = 0.1 * R
    scale = np.where(r > rc, (r - rc) / (R - rc) / np.maximum(r, 1e-30), 0.0)
    v = (v_max_kms * 1e5) * ctr * scale[:, None]
    med.vx, med.vy, med.vz = (v[:, i].astype(np.float32) for i in range(3))
    seed = RUN_SEED + 9 + seed_offset
    l96, l03 = mgII_2796(), mgII_2803()
    pk = point_source(n_packets, (0.5, 0.5, 0.5), nu_of(l96.lambda_A), seed ^ 0xA5A5)
    rng = np.random.default_rng(seed)
    red = rng.random(n_packets) < 1.0 / 3.0
    pk.nu = np.where(red, nu_of(l03.lambda_A), nu_of(l96.lambda_A))
    return Workload("mgII", med, Domain(0, (0.5, 0.5, 0.5), R), [l96, l03], Dust(sigma=4.0e-22),
                    Physics(recoil=0, isotropic=0, seed=seed), Detector(nu_of(2815.0), nu_of(2785.0), 600), pk)


PEEL_DIRS_3 = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0],
                        [1.0 / math.sqrt(3.0)] * 3])


def expanding_sphere(N_HI=1e20, T=1e4, v_max_kms=200.0, tau_dust=0.5, n_packets=1_000_000,
                     base=3, max_level=6, npix=100, nchan=200, seed_offset=0):
    """Expanding sphere with peeling: the sphere octree, centre-to-edge column
    N_HI, radial velocity v_max * r/R at leaf centres, dust, core/wing phase
    functions and recoil; 3 peeling directions into npix^2 x nchan cubes over
    +-1000 km/s."""
    tree = sphere_octree(base, max_level)
    L = 1.0 * KPC_CM
    R = 0.45
    line = lya()
    n = N_HI / (R * L)
    dust = Dust(sigma=4.0e-22)
    nd = tau_dust / (dust.sigma * R * L)
    med = uniform_medium(tree, L, n, T, n_dust=nd)
    ctr = tree.leaf_centres() - 0.5
    v = (v_max_kms * 1e5 / R) * ctr
    med.vx, med.vy, med.vz = (v[:, i].astype(np.float32) for i in range(3))
    seed = RUN_SEED + 2 + seed_offset
    nu0 = nu_of(line.lambda_A)
    pk = point_source(n_packets, (0.5, 0.5, 0.5), nu0, seed ^ 0xA5A5)
    vmax = 1000e5
    det = Detector(nu0 * (1 - vmax / C_CGS), nu0 * (1 + vmax / C_CGS), nchan,
                   dirs=PEEL_DIRS_3.copy(), npix=npix, fov=2 * R, centre=(0.5, 0.5, 0.5), cube=1)
    return Workload("expanding", med, Domain(0, (0.5, 0.5, 0.5), R), [line], dust,
                    Physics(recoil=1, isotropic=0, seed=seed), det, pk)


def batch_models(n_models=512, packet_scale=1.0, seed_offset=0, max_scatt=0):
    """Many independent homogeneous models (the batching workload): geometry
    slab or sphere with equal probability; line-centre optical depth tau0
    log-uniform in [1e2, 1e7] (centre-to-edge / half-thickness); T log-uniform
    in [1e2, 1e5] K; v_max uniform in [0, 300] km/s (sphere: radial v_max r/R;
    slab: v_z = v_max (z - 1/2)/(1/2)); uniform grid of depth d in {2..5}
    ((2^d)^3 leaves); packets log-uniform in [1e3, 1e5] times packet_scale
    (at least 1); Lya only, no dust; escape spectrum over
    x in +-(4 (a tau0)^(1/3) + 10) of each model.  Returns Workloads that share
    one line list and physics."""
    seed = RUN_SEED + 3 + seed_offset
    rng = np.random.default_rng(seed ^ 0xA5A5)
    line = lya()
    L = 1.0 * KPC_CM
    out = []
    first_id = 0
    for m in range(n_models):
        slab_geom = rng.random() < 0.5
        tau0 = 10 ** rng.uniform(2, 7)
        T = 10 ** rng.uniform(2, 5)
        vmax = rng.uniform(0, 300) * 1e5
        depth = int(rng.integers(2, 6))
        npk = max(1, int(round(10 ** rng.uniform(3, 5) * packet_scale)))
        tree = uniform_octree(depth)
        ctr = tree.leaf_centres()
        if slab_geom:
            dom = Domain(1, (0.5, 0.5, 0.5), 0.5)
            n = density_for_tau0(line, T, tau0, 0.5 * L)
            med = uniform_medium(tree, L, n, T)
            med.vz = (vmax * (ctr[:, 2] - 0.5) / 0.5).astype(np.float32)
        else:
            R = 0.45
            dom = Domain(0, (0.5, 0.5, 0.5), R)
            n = density_for_tau0(line, T, tau0, R * L)
            med = uniform_medium(tree, L, n, T)
            v = (vmax / R) * (ctr - 0.5)
            med.vx, med.vy, med.vz = (v[:, i].astype(np.float32) for i in range(3))
        dnu = doppler_width(line, T)
        a = line.A_ul / (4 * math.pi * dnu)
        xr = 4.0 * (a * tau0) ** (1.0 / 3.0) + 10.0 + vmax / (math.sqrt(2 * KB_CGS * T / line.mass_g))
        lo, hi, nb = x_axis(line, T, -xr, xr, 200)
        pk = point_source(npk, (0.5, 0.5, 0.5), nu_of(line.lambda_A), int(rng.integers(0, 2**31)),
                          first_id=first_id)
        first_id += npk
        out.append(Workload("batch%03d" % m, med, dom, [line], Dust(),
                            Physics(recoil=1, isotropic=0, seed=seed, max_scatt=max_scatt), Detector(lo, hi, nb), pk))
    return out


def siII_sphere(tau0=1e3, T=1e4, n_packets=400, base=3, max_level=4, tau_dust=0.2, v_max_kms=50.0):
    """Sphere of Si II (with a little H I and dust) lit at the Si II 1193.28 A
    line centre: exercises several lines at once and the fluorescent decay
    channels of Sect. 3.2.3 (1193 -> 1197*, 1190 -> 1194*)."""
    tree = sphere_octree(base, max_level)
    L = 1.0 * KPC_CM
    R = 0.45
    l1193, l1190 = siII_1193(), siII_1190()
    n_si = density_for_tau0(l1193, T, tau0, R * L)
    dust = Dust(sigma=4.0e-22)
    nd = tau_dust / (dust.sigma * R * L)
    med = uniform_medium(tree, L, 1e-3 * n_si, T, n_dust=nd, n_metal=n_si)
    ctr = tree.leaf_centres() - 0.5
    v = (v_max_kms * 1e5 / R) * ctr
    med.vx, med.vy, med.vz = (v[:, i].astype(np.float32) for i in range(3))
    seed = RUN_SEED + 5
    nu0 = nu_of(l1193.lambda_A)
    pk = point_source(n_packets, (0.5, 0.5, 0.5), nu0, seed ^ 0xA5A5)
    lo, hi = nu_of(1199.0), nu_of(1188.0)
    det = Detector(lo, hi, 400, dirs=PEEL_DIRS_3[:2].copy(), npix=4, fov=2 * R, cube=1)
    return Workload("siII", med, Domain(0, (0.5, 0.5, 0.5), R), [lya(), l1190, l1193], dust,
                    Physics(recoil=1, isotropic=0, seed=seed), det, pk)


def feII_sphere(tau0=1e4, T=1e4, n_packets=4000, base=3, max_level=4, seed_offset=0):
    """Static sphere of Fe II (UV1 lines 2344 and 2374, Table 1) lit at the
    2344.21 A line centre at its centre, no dust: a photon scatters in 2344
    until it decays through a fluorescent channel (2365.55* or 2381.49*, where
    the gas is transparent) or escapes in the resonant line.  Escape spectrum
    over 2335-2405 A."""
    tree = sphere_octree(base, max_level)
    L = 1.0 * KPC_CM
    R = 0.45
    l2344, l2374 = feII_2344(), feII_2374()
    n_fe = density_for_tau0(l2344, T, tau0, R * L)
    med = uniform_medium(tree, L, 0.0, T, n_metal=n_fe)
    seed = RUN_SEED + 7 + seed_offset
    pk = point_source(n_packets, (0.5, 0.5, 0.5), nu_of(l2344.lambda_A), seed ^ 0xA5A5)
    return Workload("feII", med, Domain(0, (0.5, 0.5, 0.5), R), [l2344, l2374], Dust(sigma=4.0e-22),
                    Physics(recoil=0, isotropic=0, seed=seed), Detector(nu_of(2405.0), nu_of(2335.0), 700), pk)


# --------------------------------------------------------------------------
# Synthetic galaxy octree (levels base..max, lognormal fields)
# --------------------------------------------------------------------------
ZSUN = 0.0134


def grf(n, slope, rng):
    """Gaussian random field on an n^3 periodic grid with power spectrum
    P(k) ~ k^slope, zero mean, unit variance."""
    kx = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kz = np.fft.rfftfreq(n)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    white = rng.normal(size=(n, n, n)).astype(np.float32)
    f = np.fft.rfftn(white) * amp
    del white
    out = np.fft.irfftn(f, s=(n, n, n), axes=(0, 1, 2)).astype(np.float32)
    out -= out.mean()
    out /= out.std()
    return out


def _block_max(a, f):
    n = a.shape[0] // f
    return a.reshape(n, f, n, f, n, f).max(axis=(1, 3, 5))


def galaxy(n_leaf=10_000_000, grid_level=8, base_level=6, max_level=14, n_packets=10_000_000,
           box_kpc=20.0, Z=0.3, seed_offset=0, npix=256, nchan=400, ndir=4, si_fraction=0.2):
    """Synthetic galaxy medium: log10 n_HI a Gaussian random field with
    P(k) ~ k^-11/3, median 1e-2 cm^-3 and 2 dex scatter; log T a second field,
    median 1e4 K, 0.7 dex, clipped to [1e2, 1e6]; a Kolmogorov velocity field
    (each component P(k) ~ k^-11/3), 3D rms 50 km/s; dust n_HI Z/Z0 (Z0 = 0.005,
    Sect. 3.1.2); Si II n_HI 3.2e-5 Z/Zsun.  Fields are piecewise constant on a
    (2^grid_level)^3 grid.  Octree: all cells to base_level, then a cell of
    size h is split while max n_HI over the cell widened by 2h on each side,
    times (h box)^3, exceeds a column-mass threshold tuned to ~n_leaf leaves
    (widening by 2h keeps neighbouring leaves within one level).  Packets
    (80% Lya, 10% each Si II 1190/1193) are emitted from leaves with
    probability ~ n_HI^2 V, uniformly inside the leaf, isotropically, at line
    centre in the gas frame broadened by a Gaussian of the leaf's Doppler
    width; 4 peeling directions into npix^2 x nchan cubes over +-2000 km/s of
    Lya."""
    import scipy.ndimage as ndi
    seed = RUN_SEED + 4 + seed_offset
    rng = np.random.default_rng(seed ^ 0xA5A5)
    G = grid_level
    ng = 1 << G
    L = box_kpc * KPC_CM
    logn = (-2.0 + 2.0 * grf(ng, -11.0 / 3.0, rng)).astype(np.float32)
    nH = np.power(10.0, logn, dtype=np.float32)
    logT = np.clip(4.0 + 0.7 * grf(ng, -11.0 / 3.0, rng), 2.0, 6.0)
    Tg = np.power(10.0, logT).astype(np.float32)
    vel = [grf(ng, -11.0 / 3.0, rng) for _ in range(3)]
    vs = 50e5 / math.sqrt(3.0)
    # refinement criterion: dilated maxima per level
    mx = {}
    for l in range(1, G + 1):
        pooled = _block_max(nH, 1 << (G - l)) if l < G else nH
        mx[l] = ndi.maximum_filter(pooled, size=5, mode="wrap")
    fine = ndi.maximum_filter(nH, size=3, mode="wrap")

    def n_leaves(thr):
        # exact leaf count of the tree the criterion below builds
        total = 0.0
        exists = np.ones((1 << base_level,) * 3, bool)
        refined = None
        for l in range(base_level, G + 1):
            if l > base_level:
                exists = refined.repeat(2, 0).repeat(2, 1).repeat(2, 2)
            crit = mx[l].astype(np.float64) * (L / (1 << l)) ** 3 >= thr
            refined = exists & crit if l < max_level else np.zeros_like(exists)
            total += float(np.count_nonzero(exists & ~refined))
        if G < max_level:
            f = fine[refined].astype(np.float64)
            per = np.ones(f.size)
            for l in range(G + 1, max_level + 1):
                more = f * (L / (1 << l)) ** 3 >= thr if l < max_level else np.zeros(f.size, bool)
                per = np.where(more, per * 8.0, per)
                f = np.where(more, f, 0.0)
            total += float(np.sum(8.0 * per))
        return total

    lo, hi = 1e20, 1e90
    target = 1.5 * n_leaf   # the count above splits whole grid cells; the built tree splits ~2/3 as many
    for _ in range(24):
        mid = math.sqrt(lo * hi)
        if n_leaves(mid) > target:
            lo = mid
        else:
            hi = mid
    thr = math.sqrt(lo * hi)

    def region_max(l, i, j, k):
        # max density over the grid cells met by the cell widened by 2 cells
        # of its own size (a cell below the grid level meets at most 3 per axis)
        s = l - G
        lo = [((c - 2) >> s) for c in (i, j, k)]
        hi = [((c + 3 + (1 << s) - 1) >> s) - 1 for c in (i, j, k)]
        m = np.zeros(i.shape, np.float32)
        for a in range(3):
            for b in range(3):
                for c in range(3):
                    gx, gy, gz = lo[0] + a, lo[1] + b, lo[2] + c
                    ok = (gx <= hi[0]) & (gy <= hi[1]) & (gz <= hi[2])
                    v = nH[gx % ng, gy % ng, gz % ng]
                    m = np.where(ok, np.maximum(m, v), m)
        return m

    def refine(l, i, j, k):
        h3 = (L / (1 << l)) ** 3
        if l < base_level:
            return np.ones(i.shape, bool)
        m = mx[l][i, j, k] if l <= G else region_max(l, i, j, k)
        return m.astype(np.float64) * h3 >= thr

    tree = build_octree(refine, max_level)
    ctr = tree.leaf_centres()
    gi = np.minimum((ctr * ng).astype(np.int64), ng - 1)
    idx = (gi[:, 0], gi[:, 1], gi[:, 2])
    n_leafHI = nH[idx]
    Tl = Tg[idx]
    med = Medium(tree, L, n_leafHI.astype(np.float32), (vs * vel[0][idx]).astype(np.float32),
                 (vs * vel[1][idx]).astype(np.float32), (vs * vel[2][idx]).astype(np.float32),
                 Tl.astype(np.float32), (n_leafHI * (Z * ZSUN / 0.005)).astype(np.float32),
                 (n_leafHI * 3.2e-5 * Z).astype(np.float32))
    del vel, mx, fine
    lines = [lya(), siII_1190(), siII_1193()]
    # sources: leaf chosen with probability ~ n^2 V (cumulative sum + bisection)
    w = (n_leafHI.astype(np.float64) ** 2) * tree.leaf_size() ** 3
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    srng = np.random.default_rng(seed ^ 0x5A5A)
    leaf = np.searchsorted(cdf, srng.random(n_packets), side="right")
    leaf = np.minimum(leaf, tree.nleaf - 1)
    h = tree.leaf_size()[leaf]
    pos = tree.leaf_ijk[leaf] * h[:, None] + srng.random((n_packets, 3)) * h[:, None]
    pos = np.minimum(pos, np.nextafter(1.0, 0.0))
    mu = 2.0 * srng.random(n_packets) - 1.0
    phi = 2.0 * math.pi * srng.random(n_packets)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    d = np.stack([st * np.cos(phi), st * np.sin(phi), mu], 1)
    d /= np.linalg.norm(d, axis=1)[:, None]
    which = srng.random(n_packets)
    lam = np.where(which < 1 - si_fraction, lines[0].lambda_A,
                   np.where(which < 1 - si_fraction / 2, lines[1].lambda_A, lines[2].lambda_A))
    mass = np.where(which < 1 - si_fraction, lines[0].mass_g, lines[1].mass_g)
    nu0 = C_CGS / (lam * 1e-8)
    vth = np.sqrt(2.0 * KB_CGS * Tl[leaf].astype(np.float64) / mass)
    nu_gas = nu0 * (1.0 + vth / C_CGS * srng.normal(size=n_packets) / math.sqrt(2.0))
    v = np.stack([med.vx[leaf], med.vy[leaf], med.vz[leaf]], 1).astype(np.float64)
    nu_ext = nu_gas * (1.0 + (d * v).sum(1) / C_CGS)
    pk = Packets(pos, d, nu_ext, np.arange(n_packets, dtype=np.uint64))
    nuL = nu_of(lines[0].lambda_A)
    vmax = 2000e5
    dirs = np.array([[0, 0, 1.0], [1.0, 0, 0], [0, 1.0, 0], [1.0, 1.0, 1.0]])[:ndir]
    det = Detector(nuL * (1 - vmax / C_CGS), nuL * (1 + vmax / C_CGS), nchan, dirs=dirs, npix=npix, fov=1.0,
                   centre=(0.5, 0.5, 0.5), cube=1)
    dust = Dust(sigma=4.0e-22)
    return Workload("galaxy", med, Domain(2, (0.5, 0.5, 0.5), 0.5), lines, dust,
                    Physics(recoil=1, isotropic=0, seed=seed, max_scatt=100000), det, pk)

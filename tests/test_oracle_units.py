"""Pins of the FP64 oracle's building blocks against what the paper and the
mathematics fix (no GPU).  Each test names the passage it checks."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- RNG
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors."""
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt")) if l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_word_stream_layout():
    """Draw n of a packet = word n%4 of block n/4 with counter (blk, pid)."""
    seed, pid = 0x123456789ABCDEF0, 0x0000000A00000007
    for n in [0, 1, 2, 3, 4, 7, 1 << 34 | 5]:
        blk = n >> 2
        out = oracle.philox4x32_10([blk & 0xFFFFFFFF, blk >> 32, pid & 0xFFFFFFFF, pid >> 32],
                                   [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.word(seed, pid, n) == out[n & 3]


# ---------------------------------------------------------------- Voigt
def _H_quad(a, x):
    """H(a,x) by direct quadrature of its defining integral (Sect. 3.1.1)."""
    from scipy.integrate import quad
    f = lambda y: math.exp(-y * y) / ((y - x) ** 2 + a * a)
    lo, hi = min(-12.0, x - 50 * a), max(12.0, x + 50 * a)
    pts = sorted({x - 10 * a, x, x + 10 * a})
    pts = [p for p in pts if lo < p < hi]
    v, _ = quad(f, lo, hi, points=pts, limit=400, epsabs=0, epsrel=1e-11)
    tail = 0.0  # e^{-y^2} beyond |y| > 12 is < 1e-62
    return a / math.pi * (v + tail)


def test_voigt_reference_quadrature_vs_faddeeva():
    """The truth used below (scipy wofz) agrees with quadrature of H's integral."""
    from scipy.special import wofz
    for a in [1e-3, 1e-2]:
        for x in [0.0, 0.7, 2.0, 3.5, 6.0]:
            assert abs(_H_quad(a, x) / wofz(x + 1j * a).real - 1) < 1e-8


@pytest.mark.parametrize("a,tol", [(1e-4, 0.013), (4.717e-4, 0.013), (1e-3, 0.013), (1e-2, 0.025)])
def test_voigt_tasitsiomi_accuracy(a, tol):
    """Tasitsiomi (2006) H(a,x): ~1% for Lya at 1e4 K (a~4.7e-4), degrading
    at larger a (Sect. 3.3.2)."""
    from scipy.special import wofz
    xs = np.concatenate([np.linspace(0, 10, 2001), np.linspace(10, 200, 381)])
    H = np.array([oracle.voigt(a, x) for x in xs])
    Ht = wofz(xs + 1j * a).real
    err = np.abs(H / Ht - 1)
    assert err.max() < tol
    assert err.max() > 1e-3  # it is an approximation, not the exact function


def test_voigt_limits():
    """H(0,x) = exp(-x^2); far wing H -> a/(sqrt(pi) x^2); even in x."""
    for x in [0.0, 0.3, 1.0, 2.5, 4.0]:
        assert oracle.voigt(0.0, x) == math.exp(-x * x)
    a = 4.7e-4
    for x in [300.0, 1e3, 1e4]:
        assert abs(oracle.voigt(a, x) / (a / (math.sqrt(math.pi) * x * x)) - 1) < 2e-3
    for x in [0.5, 3.3, 7.0]:
        assert oracle.voigt(a, x) == oracle.voigt(a, -x)


# ---------------------------------------------------------------- u_par
def _upar_density(x, a):
    """Normalised target density of u_par, Eq. (uparallel_distribution)."""
    from scipy.special import wofz
    H = wofz(x + 1j * a).real
    return lambda u: a / (math.pi * H) * np.exp(-u * u) / (a * a + (x - u) ** 2)


@pytest.mark.parametrize("a", [4.717e-4, 1e-2])
@pytest.mark.parametrize("x", [0.0, 0.5, 1.0, 2.0, 3.0, 5.0, -2.0, 7.9])
def test_upar_matches_density(x, a):
    """Rejection sampling of Zheng & Miralda-Escude (2002) with the u0
    polynomial (Sect. 3.3.3) reproduces f(u_par) (chi-square over bins of
    equal probability mass)."""
    from scipy.integrate import quad
    from scipy.stats import chisquare
    n = 200_000
    wl = synth.slab(n_packets=1)
    o = oracle.Oracle(wl)
    pid = int(1000 * abs(x)) + (7 if x < 0 else 0)
    u = o.upar_samples(x, a, n, pid=pid)
    f = _upar_density(x, a)
    # bin edges from an independent stream; expected mass per bin by quadrature
    ref = o.upar_samples(x, a, 20_000, pid=pid + 500_000)
    edges = np.unique(np.quantile(ref, np.linspace(0, 1, 41)[1:-1]))
    edges = np.concatenate([[-np.inf], edges, [np.inf]])
    mass = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        l2, h2 = max(lo, x - 12.0), min(hi, x + 12.0)
        l2, h2 = max(l2, -12.0 + min(0.0, x)), min(h2, 12.0 + max(0.0, x))
        pts = [q for q in (x, 0.0) if l2 < q < h2]
        mass.append(quad(f, l2, h2, points=pts or None, limit=500, epsabs=1e-13)[0] if h2 > l2 else 0.0)
    mass = np.array(mass)
    obs, _ = np.histogram(u, edges)
    exp_ = mass / mass.sum() * n
    assert chisquare(obs, exp_).pvalue > 1e-4


def test_upar_gaussian_branch():
    """|x| >= 8: u_par ~ N(1/|x|, 1/2) with the sign of x (Sect. 3.3.3)."""
    o = oracle.Oracle(synth.slab(n_packets=1))
    for x in [8.0, 12.0, -20.0]:
        u = o.upar_samples(x, 4.7e-4, 100_000, pid=3)
        assert abs(u.mean() - math.copysign(1 / abs(x), x)) < 5 * math.sqrt(0.5 / u.size)
        assert abs(u.var() - 0.5) < 0.02


def test_u0_clamped_non_negative():
    """The u0(x, log10 a) polynomial is negative near x=0 at small a; the
    oracle clamps it at 0 so that the g2 acceptance stays <= 1."""
    assert oracle.u0(0.0, 4.7e-4) == 0.0
    assert oracle.u0(3.0, 4.7e-4) > 0.0


# ---------------------------------------------------------------- phase functions
def _cdf(kind, mu, g=0.0):
    if kind == oracle.PH_CORE:
        return (mu ** 3 + 11 * mu + 12) / 24.0
    if kind == oracle.PH_WING:
        return (mu ** 3 + 3 * mu + 4) / 8.0
    if kind == oracle.PH_HG:
        return (1 - g * g) / (2 * g) * ((1 + g * g - 2 * g * mu) ** -0.5 - 1 / (1 + g))
    return (mu + 1) / 2


@pytest.mark.parametrize("kind,g", [(oracle.PH_CORE, 0), (oracle.PH_WING, 0), (oracle.PH_HG, 0.73),
                                    (oracle.PH_HG, -0.4), (oracle.PH_ISO, 0)])
def test_phase_inversion(kind, g):
    """mu(r) inverts the CDF of P_core, P_wing (Eqs. Pcore/Pwing) and P_HG
    (Eq. Pdust): CDF(mu(r)) = r, mu in [-1,1], density integrates to 1."""
    from scipy.integrate import quad
    for r in np.linspace(1e-6, 1 - 1e-6, 101):
        mu = oracle.mu_sample(kind, r, g)
        assert -1 - 1e-12 <= mu <= 1 + 1e-12
        assert abs(_cdf(kind, mu, g) - r) < 1e-10
    assert abs(quad(lambda m: oracle.phase(kind, m, g), -1, 1)[0] - 1) < 1e-10


def test_hg_mean_is_g():
    from scipy.integrate import quad
    for g in [0.73, 0.2, -0.5]:
        m = quad(lambda mu: mu * oracle.phase(oracle.PH_HG, mu, g), -1, 1)[0]
        assert abs(m - g) < 1e-10
        r = (np.arange(200000) + 0.5) / 200000
        mus = np.array([oracle.mu_sample(oracle.PH_HG, x, g) for x in r[::50]])
        assert abs(mus.mean() - g) < 2e-3


def test_onb_orthonormal():
    rng = np.random.default_rng(1)
    vs = list(rng.normal(size=(200, 3))) + [np.array([0, 0, 1.0]), np.array([0, 0, -1.0]),
                                            np.array([1.0, 0, 0]), np.array([0, -1.0, 0])]
    for v in vs:
        n = v / np.linalg.norm(v)
        b1, b2 = oracle.onb(n)
        M = np.stack([b1, b2, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-14)


def test_opacity_frame_change():
    """Sect. 3 frame change: a leaf moving with velocity v presents to a photon
    of external frequency nu_ext along k the opacity of the gas at rest at
    nu_gas = nu_ext / (1 + k.v/c); a velocity perpendicular to k changes
    nothing; the Doppler offset moves by k.v / v_th widths."""
    wl = synth.slab(tau0=1e3, T=1e4, n_packets=1)
    o = oracle.Oracle(wl)
    ln = wl.lines[0]
    nu0, dnu = synth.nu_of(ln.lambda_A), synth.doppler_width(ln, 1e4)
    nleaf = wl.medium.tree.nleaf
    leaf = 7
    v = np.float32(1.0e7)                     # 100 km/s
    rng = np.random.default_rng(4)
    for _ in range(40):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        x = rng.uniform(-8, 8)
        nu_gas = nu0 + x * dnu
        o.set_field("vx", np.zeros(nleaf))
        kap_rest = o.opacity(leaf, nu_gas, k)
        o.set_field("vx", np.full(nleaf, v))
        beta = k[0] * float(v) / synth.C_CGS
        kap_moving = o.opacity(leaf, nu_gas * (1.0 + beta), k)
        assert abs(kap_moving / kap_rest - 1) < 1e-9
        # perpendicular motion: no shift
        kp = np.array([0.0, k[1], k[2]])
        kp /= np.linalg.norm(kp)
        o.set_field("vx", np.zeros(nleaf))
        kap_p0 = o.opacity(leaf, nu_gas, kp)
        o.set_field("vx", np.full(nleaf, v))
        assert o.opacity(leaf, nu_gas, kp) == kap_p0
    # the line centre seen from a receding leaf sits k.v/c nu0 to the red
    o.set_field("vx", np.full(nleaf, v))
    k = np.array([-1.0, 0.0, 0.0])
    shift = nu0 * (1.0 - float(v) / synth.C_CGS)
    nus = shift + np.linspace(-0.05, 0.05, 201) * dnu
    kaps = [o.opacity(leaf, f, k) for f in nus]
    assert abs((nus[int(np.argmax(kaps))] - shift) / dnu) <= 0.0005 + 1e-12

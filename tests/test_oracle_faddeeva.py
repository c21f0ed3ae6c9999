"""Pins of the oracle's accurate H(a,x) option (the Faddeeva function, the
accurate alternative to Tasitsiomi's form discussed in Sect. 3.3.2) against
what the mathematics fixes: scipy's wofz (the reference the paper itself uses
for its Voigt accuracy map), quadrature of H's defining integral, Dawson's
function on the real axis, the a -> 0 and far-wing limits, the normalisation,
the derivatives, and a transfer run whose mean free path at line centre
follows H(a,0) = exp(a^2) erfc(a).  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth

SQPI = math.sqrt(math.pi)


def _H_quad(a, x):
    """H(a,x) = (1/pi) int_{-pi/2}^{pi/2} exp(-(x + a tan phi)^2) dphi, the
    defining integral after y = x + a tan(phi) (smooth integrand)."""
    from scipy.integrate import quad
    f = lambda p: math.exp(-(x + a * math.tan(p)) ** 2)
    # the integrand is large where |x + a tan phi| < 6
    lo = math.atan((-6.0 - x) / a)
    hi = math.atan((6.0 - x) / a)
    # the Gaussian core y ~ 0 can be a narrow spike in phi: split around it
    pts = sorted({math.atan((y - x) / a) for y in (-3.0, -1.5, -0.5, 0.0, 0.5, 1.5, 3.0)})
    edges = [lo] + [p for p in pts if lo < p < hi] + [hi]
    v = sum(quad(f, e0, e1, limit=400, epsabs=0, epsrel=1e-12)[0] for e0, e1 in zip(edges[:-1], edges[1:]))
    return v / math.pi


A_GRID = [1e-7, 1e-5, 1e-4, 4.717e-4, 1e-3, 1e-2, 0.1, 0.5, 1.0, 3.0]
X_GRID = np.concatenate([np.linspace(0.0, 10.0, 401), [10.13, 15.0, 40.0, 300.0, 1e3, 1e4, 1e5],
                         -np.linspace(0.05, 9.0, 37)])


@pytest.mark.parametrize("a", A_GRID)
def test_faddeeva_matches_wofz(a):
    """Re and Im of w(x + ia) agree with scipy.special.wofz to ~1e-13."""
    from scipy.special import wofz
    ref = wofz(X_GRID + 1j * a)
    got = np.array([oracle.faddeeva(a, x) for x in X_GRID])
    assert np.max(np.abs(got.real / ref.real - 1)) < 2e-13
    assert np.max(np.abs(got.imag - ref.imag) / np.abs(ref)) < 2e-13


@pytest.mark.parametrize("a,x", [(1e-3, 0.0), (1e-3, 1.7), (1e-3, 3.25), (4.7e-4, 4.0), (1e-2, 2.6),
                                 (0.2, 0.9), (0.2, 6.0), (1.0, 3.0)])
def test_faddeeva_matches_quadrature(a, x):
    """H agrees with direct quadrature of its defining integral."""
    assert abs(oracle.voigt(a, x, method=1) / _H_quad(a, x) - 1) < 1e-9


def test_faddeeva_real_axis_dawson():
    """As a -> 0, Re w -> exp(-x^2) and Im w -> (2/sqrt(pi)) F(x), F Dawson's
    integral."""
    from scipy.special import dawsn
    a = 1e-12
    for x in [0.0, 0.3, 1.0, 1.5, 2.5, 4.0, 7.0, 20.0]:
        w = oracle.faddeeva(a, x)
        assert abs(w.real - math.exp(-x * x)) <= 1e-10 * math.exp(-x * x) + 2 * a / SQPI
        # first order in a: d Im w / da = Re w'(x) = -2 x exp(-x^2)
        assert abs(w.imag - 2 / SQPI * dawsn(x) + 2 * a * x * math.exp(-x * x)) < 1e-14
    assert oracle.faddeeva(0.0, 1.3).real == math.exp(-1.3 * 1.3)


def test_faddeeva_far_wing_and_symmetry():
    """Far wing: H = a/(sqrt(pi) x^2) (1 + (3/2 - a^2)/x^2 + ...); H is even
    and Im w odd in x."""
    a = 4.7e-4
    for x in [1e3, 1e4, 1e5]:
        asym = a / (SQPI * x * x) * (1 + (1.5 - a * a) / (x * x))
        assert abs(oracle.voigt(a, x, method=1) / asym - 1) < 1e-10
    for a in [1e-4, 0.3]:
        for x in [0.4, 2.2, 6.1, 50.0]:
            wp, wm = oracle.faddeeva(a, x), oracle.faddeeva(a, -x)
            assert abs(wp.real - wm.real) <= 1e-15 * wp.real
            assert abs(wp.imag + wm.imag) <= 1e-15 * abs(wp.imag)


@pytest.mark.parametrize("a", [1e-3, 0.1])
def test_faddeeva_normalisation(a):
    """int H(a,x) dx = sqrt(pi) (the profile phi = H / (sqrt(pi) dnu) is
    normalised, Sect. 3.1.1)."""
    from scipy.integrate import quad
    X = 50.0
    f = lambda x: oracle.voigt(a, x, method=1)
    core, _ = quad(f, 0.0, 8.0, limit=400, epsrel=1e-12)
    wing, _ = quad(f, 8.0, X, limit=400, epsrel=1e-12)
    # beyond X: int a/(sqrt(pi) x^2) (1 + 3/(2x^2)) dx
    tail = a / SQPI * (1 / X + 0.5 / X ** 3)
    assert abs(2 * (core + wing + tail) / SQPI - 1) < 1e-7


def test_faddeeva_derivatives_match_differences():
    """dH/da and dH/dx from the derivative identity of w agree with central
    differences of H."""
    for a in [1e-4, 4.7e-4, 1e-2, 0.3]:
        for x in [0.0, 0.6, 1.9, 3.0, 4.4, 9.0, 60.0]:
            H, Ha, Hx = oracle.faddeeva_derivs(a, x)
            assert H == oracle.voigt(a, x, method=1)
            da = 1e-4 * a
            ha = (oracle.voigt(a + da, x, method=1) - oracle.voigt(a - da, x, method=1)) / (2 * da)
            dx = 1e-5 * max(1.0, x)
            hx = (oracle.voigt(a, x + dx, method=1) - oracle.voigt(a, x - dx, method=1)) / (2 * dx)
            assert abs(Ha - ha) <= 1e-6 * abs(ha) + 1e-12
            assert abs(Hx - hx) <= 1e-6 * max(abs(hx), H / max(1.0, x)) + 1e-13


def test_tasitsiomi_within_its_accuracy_of_faddeeva():
    """The two H evaluations differ by Tasitsiomi's ~1 % for Lya at 1e4 K."""
    a = 4.717e-4
    xs = np.linspace(0.0, 30.0, 601)
    r = np.array([oracle.voigt(a, x) / oracle.voigt(a, x, method=1) - 1 for x in xs])
    assert np.max(np.abs(r)) < 0.013
    assert np.max(np.abs(r)) > 1e-3


def test_mean_free_path_faddeeva():
    """Transfer with the Faddeeva H: the mean distance to the first scattering
    of packets emitted at line centre is R / (tau0 H(a,0)), with H(a,0) =
    exp(a^2) erfc(a); at T = 1 K (a ~ 0.047) this is 5 % longer than with
    Tasitsiomi's H(a,0) = 1 (App. B)."""
    from scipy.special import erfcx
    n, tau0, T = 20000, 10.0, 1.0
    wl = synth.sphere(tau0=tau0, T=T, n_packets=n, base=3, max_level=3)
    wl.physics.max_scatt = 1
    wl.physics.voigt = 1
    ln = wl.lines[0]
    a = ln.A_ul / (4 * math.pi * synth.doppler_width(ln, T))
    out, _ = oracle.Oracle(wl).run(threads=8)
    first = out["path"][out["status"] == oracle.CAPPED]
    lam = wl.domain.size / (tau0 * erfcx(a))
    assert first.size > 0.999 * n
    assert abs(first.mean() / lam - 1) < 4 / math.sqrt(first.size)
    # and rejects the H(a,0) = 1 prediction at the same 4 sigma
    assert abs(first.mean() / (wl.domain.size / tau0) - 1) > 4 / math.sqrt(first.size)

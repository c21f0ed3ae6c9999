"""Pins of the oracle's core-skipping option (Sect. 3.2.1; no GPU).

Core-skipping biases the frequency redistribution of scatterings in the line
core: the scatterer's perpendicular velocity is drawn from the 2-D Gaussian
restricted to |u_perp| >= x_crit (Ahn et al. 2002; Dijkstra et al. 2006), so
a core photon leaves the core in one scattering instead of thousands.  The
paper uses it with Smith et al.'s (2015) choice of x_crit, not printed; the
oracle takes x_crit as given, or x_crit = f (a tau_cell)^(1/3) per leaf.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import synth


def _o(**kw):
    wl = synth.slab(tau0=1e4, T=1e4, n_packets=1)
    for k, v in kw.items():
        setattr(wl.physics, k, v)
    return wl, oracle.Oracle(wl)


def test_plain_perpendicular_draw():
    """x_crit = 0: each component ~ N(0, 1/2) (the unbiased Maxwellian of
    Sect. 3.2.1), the two uncorrelated."""
    _, o = _o()
    u = o.uperp_samples(0.3, 0.0, 200_000, pid=5)
    for j in range(2):
        assert stats.kstest(u[:, j], stats.norm(0.0, math.sqrt(0.5)).cdf).pvalue > 1e-3
    assert abs(np.corrcoef(u[:, 0], u[:, 1])[0, 1]) < 0.01


@pytest.mark.parametrize("x_crit", [0.5, 2.0, 4.0])
def test_truncated_perpendicular_draw(x_crit):
    """|x_in| < x_crit: the radius follows P(rho > r) = exp(x_crit^2 - r^2)
    for r >= x_crit (the 2-D Gaussian restricted to rho >= x_crit), the angle
    is uniform; |x_in| >= x_crit: the plain Rayleigh law P(rho > r) = exp(-r^2)."""
    _, o = _o()
    u = o.uperp_samples(0.9 * x_crit, x_crit, 100_000, pid=11)
    rho = np.hypot(u[:, 0], u[:, 1])
    assert rho.min() >= x_crit * (1 - 1e-12)
    cdf = lambda r: 1.0 - np.exp(x_crit ** 2 - np.maximum(r, x_crit) ** 2)
    assert stats.kstest(rho, cdf).pvalue > 1e-3
    ang = (np.arctan2(u[:, 1], u[:, 0]) / (2 * math.pi)) % 1.0
    assert stats.kstest(ang, "uniform").pvalue > 1e-3
    # outside the core the draw is the plain one, word for word
    v = o.uperp_samples(1.1 * x_crit, x_crit, 1000, pid=11)
    w = o.uperp_samples(1.1 * x_crit, 0.0, 1000, pid=11)
    assert np.array_equal(v, w)
    rho2 = np.hypot(*o.uperp_samples(1.1 * x_crit, x_crit, 50_000, pid=12).T)
    assert stats.kstest(rho2, lambda r: 1.0 - np.exp(-r * r)).pvalue > 1e-3


def test_auto_critical_frequency():
    """x_crit = f (a tau_cell)^(1/3) with tau_cell the line-centre optical
    depth across the leaf: slab of config 1 (16^3 grid, tau0 = 1e4 over the
    half-thickness 1/2, so tau_cell = tau0 / 8 across a level-4 leaf)."""
    wl, o = _o(core_skip_f=0.2)
    a = o.line_props(0, 0, synth.nu_of(wl.lines[0].lambda_A))[2]
    xc = o.core_skip_xcrit(0, 0, 4)
    assert abs(xc / (0.2 * (a * 1e4 / 8) ** (1 / 3)) - 1) < 1e-6, xc
    wl, o = _o(core_skip=1.5)
    assert o.core_skip_xcrit(0, 0, 4) == 1.5


def test_core_skip_zero_is_the_plain_run():
    """core_skip = 0 (the default) leaves every history unchanged."""
    wl = synth.slab(tau0=1e3, T=1e2, n_packets=200)
    r0, _ = oracle.Oracle(wl).run(threads=4)
    wl.physics.core_skip = 0.0
    wl.physics.core_skip_f = 0.0
    r1, _ = oracle.Oracle(wl).run(threads=4)
    for k in ("status", "nscatt", "nu", "pos"):
        assert np.array_equal(r0[k], r1[k]), k


def test_thick_slab_spectrum_unchanged_by_core_skipping():
    """A dust-free thick slab (T = 10 K, a tau0 ~ 300): skipping the core
    below x_crit = 1.5 (well inside the emergent peaks near 1.07 (a tau0)^(1/3)
    ~ 7) cuts the scatterings several-fold and leaves the escape spectrum as
    it was (the method's claim for media without dust, Sect. 3.2.1).  The bias
    grows as x_crit nears the peaks: at x_crit = 3 <|x|> moves out by ~3 %."""
    n = 3000
    wl = synth.slab(tau0=2e4, T=10.0, n_packets=n)
    ln = wl.lines[0]
    x_of = lambda nu: (nu - synth.nu_of(ln.lambda_A)) / synth.doppler_width(ln, 10.0)
    r0, _ = oracle.Oracle(wl).run(threads=8)
    wl.physics.core_skip = 1.5
    r1, _ = oracle.Oracle(wl).run(threads=8)
    assert (r0["status"] == oracle.ESCAPED).all() and (r1["status"] == oracle.ESCAPED).all()
    x0, x1 = np.abs(x_of(r0["nu"])), np.abs(x_of(r1["nu"]))
    speed = r0["nscatt"].mean() / r1["nscatt"].mean()
    print("core-skipping x_crit = 1.5: <N> %.0f -> %.0f (x%.1f), <|x|> %.3f vs %.3f, KS p %.3f"
          % (r0["nscatt"].mean(), r1["nscatt"].mean(), speed, x0.mean(), x1.mean(),
             stats.ks_2samp(x0, x1).pvalue))
    assert speed > 4.0
    # the two runs are independent samples (the streams part at the first
    # core scattering): the means agree within 4 standard errors and 2 %
    se = math.sqrt(x0.var() / n + x1.var() / n)
    assert abs(x1.mean() - x0.mean()) < 4 * se
    assert abs(x1.mean() / x0.mean() - 1) < 0.02
    assert stats.ks_2samp(x0, x1).pvalue > 1e-3

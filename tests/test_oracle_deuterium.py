"""Oracle pins for a medium of two resonant species (Appendix A: H I mixed
with deuterium, D/H = 3e-5): the opacity sums both lines, the D line sits at
its Table 1 wavelength with its own (heavier) Doppler width and cross
section, and the D density is n_HI x D/H.  The Voigt profile here is taken
from the Faddeeva function (scipy), so these pins also bound the oracle's
Tasitsiomi approximation (within ~1.3 %)."""
import math

import numpy as np
import pytest

import oracle
import synth


def _voigt_exact(a, x):
    from scipy.special import wofz
    return float(np.real(wofz(x + 1j * a)))


def _sigma0(line, T):
    dnu = synth.doppler_width(line, T)
    return math.sqrt(math.pi) * synth.E_ESU ** 2 * line.f_lu / (synth.ME_CGS * synth.C_CGS * dnu), dnu


def test_deuterium_opacity():
    pytest.importorskip("scipy")
    T, dh = 1e4, 3.0e-5
    wl = synth.deuterium_sphere(T=T, d_over_h=dh, n_packets=1, base=2, max_level=3)
    o = oracle.Oracle(wl)
    h, d = wl.lines
    leaf = 0
    n = float(wl.medium.n_HI[leaf])
    k = np.array([1.0, 0.0, 0.0])
    nuH, nuD = synth.nu_of(h.lambda_A), synth.nu_of(d.lambda_A)
    sH, dnuH = _sigma0(h, T)
    sD, dnuD = _sigma0(d, T)
    aH = h.A_ul / (4 * math.pi * dnuH)
    aD = d.A_ul / (4 * math.pi * dnuD)
    xD = (nuD - nuH) / dnuH
    assert abs(xD - 6.33) < 0.01                          # Sect. A: the dip at x ~ 6.3
    assert abs(dnuD / dnuH - math.sqrt(synth.MP_CGS / d.mass_g) * nuD / nuH) < 1e-12
    # the opacity peaks at the D line centre, pulled slightly towards the H
    # line by the slope of its wing: same peak as the exact profiles give
    nus = nuD + np.linspace(-3, 3, 601) * dnuD
    kap = np.array([o.opacity(leaf, float(v), k) for v in nus])
    ref = np.array([sH * _voigt_exact(aH, (v - nuH) / dnuH) + dh * sD * _voigt_exact(aD, (v - nuD) / dnuD)
                    for v in nus])
    assert abs(kap.argmax() - ref.argmax()) <= 1
    assert abs((nus[kap.argmax()] - nuD) / dnuD) <= 0.05
    # value at the D line centre and at the mirror point of the H line
    exp_D = n * (sH * _voigt_exact(aH, xD) + dh * sD * _voigt_exact(aD, 0.0))
    exp_M = n * (sH * _voigt_exact(aH, -xD) + dh * sD * _voigt_exact(aD, (2 * nuH - nuD - nuD) / dnuD))
    got_D = o.opacity(leaf, nuD, k)
    got_M = o.opacity(leaf, 2 * nuH - nuD, k)
    assert abs(got_D / exp_D - 1) < 0.02, (got_D, exp_D)
    assert abs(got_M / exp_M - 1) < 0.02, (got_M, exp_M)
    assert got_D / got_M > 5      # the D line dominates its neighbourhood
    # without deuterium the two points are mirror images
    o2 = oracle.Oracle(synth.deuterium_sphere(T=T, with_d=False, n_packets=1, base=2, max_level=3))
    assert abs(o2.opacity(leaf, nuD, k) / o2.opacity(leaf, 2 * nuH - nuD, k) - 1) < 1e-9

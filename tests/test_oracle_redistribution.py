"""Frequency redistribution in one scattering (Sects. 3.2.1, 3.3), pinned by
an independent Monte Carlo of its definition: the atom's velocity along the
photon, u_par, has density proportional to exp(-u^2) / ((x_in - u)^2 + a^2)
(drawn here by inverting its CDF on a fine grid, not by the rejection method
of the oracle), the perpendicular components are Gaussian with variance 1/2,
the photon is re-emitted coherently in the atom frame with mu from the phase
function, so that x_out = x_in - u_par (1 - mu) + sqrt(1 - mu^2) g with g a
Gaussian of variance 1/2 (no recoil; the (1 + x/q0) factor of the exact
frequency change is below 1e-3 here).  The oracle's single scatterings must
follow the same law (two-sample KS)."""
import math

import numpy as np
import pytest

import oracle
import synth


def _reference(x_in, a, kind, n, rng, perp=True):
    u = np.linspace(x_in - 60.0, x_in + 60.0, 2_000_001)
    w = np.exp(-u * u) / ((x_in - u) ** 2 + a * a)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    upar = np.interp(rng.random(n), cdf, u)
    r = rng.random(n)
    if kind == "iso":
        mu = 2 * r - 1
    else:
        mus = np.linspace(-1, 1, 20001)
        core = np.abs(x_in - upar) < 0.2
        pc = np.cumsum(11.0 / 24 + 3.0 / 24 * mus ** 2)
        pw = np.cumsum(3.0 / 8 * (1 + mus ** 2))
        pc /= pc[-1]
        pw /= pw[-1]
        mu = np.where(core, np.interp(r, pc, mus), np.interp(r, pw, mus))
    g = rng.normal(0.0, math.sqrt(0.5), n) if perp else 0.0
    return x_in - upar * (1 - mu) + np.sqrt(1 - mu * mu) * g


def _oracle(x_in, kind, n):
    wl = synth.slab(tau0=1e9, T=1e4, n_packets=1, isotropic=1 if kind == "iso" else 0)
    o = oracle.Oracle(wl)
    h = wl.lines[0]
    nu0, dnu = synth.nu_of(h.lambda_A), synth.doppler_width(h, 1e4)
    p = np.array([0.5, 0.5, 0.5])
    k = np.array([0.6, 0.0, 0.8])
    out = []
    for pid in range(n):
        s = o.new_state(p, k, nu0 + x_in * dnu, pid + 1000)
        o.event(s)
        if s.nscatt == 1:
            out.append((s.nu - nu0) / dnu)
    return np.array(out)


@pytest.mark.parametrize("x_in,kind", [(0.0, "iso"), (2.0, "iso"), (5.0, "iso"), (0.0, "lya"), (3.0, "lya")])
def test_single_scattering_redistribution(x_in, kind):
    from scipy.stats import ks_2samp
    a = synth.lya().A_ul / (4 * math.pi * synth.doppler_width(synth.lya(), 1e4))
    n = 20000
    got = _oracle(x_in, kind, n)
    assert len(got) > 0.99 * n
    ref = _reference(x_in, a, kind, 200000, np.random.default_rng(3))
    p = ks_2samp(got, ref).pvalue
    print(x_in, kind, "mean %.4f vs %.4f, sd %.4f vs %.4f, KS p %.3g" % (got.mean(), ref.mean(), got.std(), ref.std(), p))
    assert p > 1e-3
    # the test has teeth: leaving out the perpendicular velocity is rejected
    wrong = _reference(x_in, a, kind, 200000, np.random.default_rng(4), perp=False)
    assert ks_2samp(got, wrong).pvalue < 1e-6


def test_recoil_denominator():
    """Eq. nuout_nuin: with the same draws (same packet stream) a scattering
    with recoil differs from one without only by the denominator
    1 + (1 - mu) h nu_in / (m c^2), mu = k_out . k_in."""
    res = {}
    for rec in (0, 1):
        wl = synth.slab(tau0=1e9, T=1e4, n_packets=1, isotropic=0, recoil=rec)
        o = oracle.Oracle(wl)
        h = wl.lines[0]
        nu0, dnu = synth.nu_of(h.lambda_A), synth.doppler_width(h, 1e4)
        k_in = np.array([0.6, 0.0, 0.8])
        out = []
        for pid in range(400):
            nu_in = nu0 + (pid % 9 - 4) * 0.7 * dnu
            s = o.new_state(np.array([0.5, 0.5, 0.5]), k_in, nu_in, pid + 77)
            o.event(s)
            out.append((s.nscatt, s.nu, np.dot(np.array(s.k), k_in), nu_in))
        res[rec] = out
    m = synth.lya().mass_g
    checked = 0
    for (n0, nu_a, mu_a, nu_in), (n1, nu_b, mu_b, _) in zip(res[0], res[1]):
        assert n0 == n1 == 1
        assert mu_a == mu_b                      # same draws, same direction
        expect = nu_a / (1.0 + (1.0 - mu_a) * synth.H_CGS * nu_in / (m * synth.C_CGS ** 2))
        assert abs(nu_b / expect - 1) < 1e-14
        checked += 1
    assert checked == 400

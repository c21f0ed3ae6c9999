"""H I mixed with deuterium (Appendix A: D/H = 3e-5, T = 1e4 K): two resonant
species in one medium on the GPU.  Per-step replay and coupled whole runs
against the oracle on a thinner sphere; at the paper's column (N_HI = 2e19)
the escape spectrum loses its photons near the D line centre, x ~ 6.33 in the
H line's Doppler units, and only there."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, gpu_run, oracle_run
from gpu_util import replay_steps as _replay
from test_gpu_parity import _ks, _x

pytestmark = pytest.mark.gpu


def test_deuterium_replay_per_step():
    wl = synth.deuterium_sphere(N_HI=2e17, n_packets=64)
    st = _replay(wl, 64, 200)
    print("deuterium", st)
    assert st["steps"] > 1000
    assert st["mismatch"] <= 0.002 * st["steps"] + 2
    assert st["pos"] < 1e-6 and st["dir"] < 1e-6 and st["x"] < 3e-5


def test_deuterium_run_matches_oracle():
    n = 400
    wl = synth.deuterium_sphere(N_HI=2e17, n_packets=n)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets, device=True)
    r, tal = oracle_run(wl)
    same = (g["nscatt"] == r["nscatt"]).mean()
    print("deuterium: identical %.4f <N> %.1f vs %.1f" % (same, g["nscatt"].mean(), r["nscatt"].mean()))
    assert st["escaped"] == n
    assert abs(g["nscatt"].mean() / r["nscatt"].mean() - 1) < 0.01 or same > 0.9
    assert _ks(_x(wl, g["nu"]), _x(wl, r["nu"])) > 0.01


def test_deuterium_dip_at_paper_column():
    import torch
    n = 1 << 14
    spec = {}
    for with_d in (True, False):
        wl = synth.deuterium_sphere(N_HI=2e19, n_packets=n, with_d=with_d)
        ctx = context(wl)
        g, st = gpu_run(ctx, wl.packets, device=True)
        assert st["escaped"] == n and st["errors"] == 0
        spec[with_d] = ctx.get_tally(0).astype(np.float64)
        ctx.close()
    h, d = synth.lya(), synth.d_lya()
    xD = (synth.nu_of(d.lambda_A) - synth.nu_of(h.lambda_A)) / synth.doppler_width(h, 1e4)
    edges = np.linspace(-20, 20, 201)
    win = (edges[:-1] >= xD - 0.5) & (edges[1:] <= xD + 0.5)
    red = (edges[:-1] >= -12) & (edges[1:] <= -2)
    blue = (edges[:-1] >= 2) & (edges[1:] <= xD - 1.5)
    dip = spec[True][win].sum() / spec[False][win].sum()
    rr = spec[True][red].sum() / spec[False][red].sum()
    rb = spec[True][blue].sum() / spec[False][blue].sum()
    print("deuterium x_D %.3f: window ratio %.3f, red side %.3f, blue side below the dip %.3f" % (xD, dip, rr, rb))
    sig_r = math.sqrt(2.0 / spec[False][red].sum())
    assert dip < 0.7
    assert abs(rr - 1) < 4 * sig_r + 0.02

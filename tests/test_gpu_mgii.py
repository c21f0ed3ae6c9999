"""Mg II doublet in an outflow on the GPU (two metal lines of one ion,
isotropic phase function): coupled runs against the oracle, and on 2^16
packets the exact property that every photon leaves in the line it was
emitted in."""
import numpy as np
import pytest

import synth
from gpu_util import context, gpu_run, oracle_run
from test_gpu_parity import _ks

pytestmark = pytest.mark.gpu


def test_mgii_run_matches_oracle():
    n = 2000
    wl = synth.mgII_wind(n_packets=n)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    r, _ = oracle_run(wl)
    same = (g["nscatt"] == r["nscatt"]).mean()
    print("Mg II: identical %.4f <N> %.2f vs %.2f" % (same, g["nscatt"].mean(), r["nscatt"].mean()))
    assert st["escaped"] == n and same > 0.95
    lam_g, lam_r = synth.C_CGS / g["nu"] * 1e8, synth.C_CGS / r["nu"] * 1e8
    assert _ks(lam_g, lam_r) > 0.01


def test_mgii_lines_stay_apart_on_gpu():
    n = 1 << 16
    wl = synth.mgII_wind(n_packets=n)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets, device=True)
    lam = synth.C_CGS / g["nu"] * 1e8
    born_red = np.abs(synth.C_CGS / wl.packets.nu * 1e8 - 2803.53) < 0.01
    assert np.array_equal(np.abs(lam - 2803.53) < 4.0, born_red)
    assert np.array_equal(np.abs(lam - 2796.35) < 4.0, ~born_red)
    assert int(ctx.get_tally(0).sum()) == n

"""Fe II UV1 fluorescence (Sect. 3.2.3, Table 1) on the GPU: a line with two
fluorescent channels and a second line with one.  Coupled runs against the
oracle, and on 2^16 packets the two exact laws of the channel choice: the
2365.55 / 2381.49 split A_2366 / (A_2366 + A_2381) and the geometric number of
scatterings before the first fluorescent decay."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _lam(nu):
    return synth.C_CGS / nu * 1e8


def test_feii_run_matches_oracle():
    n = 4000
    wl = synth.feII_sphere(tau0=1e4, n_packets=n)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    r, _ = oracle_run(wl)
    same = (g["nscatt"] == r["nscatt"]).mean()
    print("Fe II: identical %.4f <N> %.3f vs %.3f" % (same, g["nscatt"].mean(), r["nscatt"].mean()))
    assert st["escaped"] == n and st["errors"] == 0
    assert same > 0.99
    both = g["nscatt"] == r["nscatt"]
    assert np.all(np.abs(_lam(g["nu"][both]) - _lam(r["nu"][both])) < 0.01)


def test_feii_channel_laws_on_gpu():
    n = 1 << 16
    wl = synth.feII_sphere(tau0=1e4, n_packets=n)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets, device=True)
    lam = _lam(g["nu"])
    f66 = int((np.abs(lam - 2365.55) < 0.5).sum())
    f81 = int((np.abs(lam - 2381.49) < 0.5).sum())
    res = int((np.abs(lam - 2344.21) < 0.5).sum())
    assert res + f66 + f81 == n and res < 0.01 * n
    p = 5.90e7 / (5.90e7 + 3.10e7)
    m = f66 + f81
    print("Fe II: 2366 share %.4f (exact %.4f), resonant escapes %d" % (f66 / m, p, res))
    assert abs(f66 / m - p) < 4 * math.sqrt(p * (1 - p) / m)
    q = (5.90e7 + 3.10e7) / (1.73e8 + 5.90e7 + 3.10e7)
    fl = g["nscatt"][np.abs(lam - 2344.21) > 5]
    assert abs(fl.mean() - 1 / q) < 4 * math.sqrt((1 - q) / q ** 2 / len(fl))
    # the escape spectrum holds the same photons
    assert int(ctx.get_tally(0).sum()) == n

"""Fluorescent decay channels (Sect. 3.2.3) pinned on a multi-channel line:
Fe II 2344 (Table 1) decays to 2344 (resonant), 2365.55* or 2381.49*.  In a
sphere thick in 2344 (tau0 = 1e4) almost every photon ends in a fluorescent
channel, where the gas is transparent, and the two channels share the photons
in the ratio of their Einstein coefficients, A_2366 / (A_2366 + A_2381) =
0.6556; the mean number of scatterings is the mean of a geometric law with
success probability (A_2366 + A_2381) / sum A = 0.342 -- both exact."""
import math

import numpy as np

import oracle
import synth


def _counts(wl, nu, status):
    lam = synth.C_CGS / nu * 1e8
    esc = status == oracle.ESCAPED
    win = lambda l0: int((esc & (np.abs(lam - l0) < 0.5)).sum())
    return win(2344.21), win(2365.55), win(2381.49), win(2396.35), int(esc.sum())


def test_feii_channel_ratio():
    n = 6000
    wl = synth.feII_sphere(tau0=1e4, n_packets=n)
    out, _ = oracle.Oracle(wl).run(threads=8)
    res, f66, f81, f96, esc = _counts(wl, out["nu"], out["status"])
    assert esc == n                             # no dust: everything escapes
    assert f96 == 0                             # 2374 is 30 A away: never excited
    assert res + f66 + f81 == n                 # every photon leaves in one of the three
    assert res < 0.01 * n                       # the resonant channel is trapped
    p = 5.90e7 / (5.90e7 + 3.10e7)
    m = f66 + f81
    assert abs(f66 / m - p) < 4 * math.sqrt(p * (1 - p) / m)
    # scatterings until the first fluorescent decay: geometric with success q
    q = (5.90e7 + 3.10e7) / (1.73e8 + 5.90e7 + 3.10e7)
    fl = out["nscatt"][np.abs(synth.C_CGS / out["nu"] * 1e8 - 2344.21) > 5]
    assert abs(fl.mean() - 1 / q) < 4 * math.sqrt((1 - q) / q ** 2 / len(fl))

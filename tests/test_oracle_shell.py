"""Shell domain (Sect. 4: the domain class implements spheres, shells, cubes
and slabs): the distance to the border along a ray ends at the outer sphere
or, for rays moving inwards that meet it, at the inner sphere -- closed forms
for radial and oblique rays; packets leave through one of the two spheres."""
import math

import numpy as np
import pytest

import oracle
import synth

RIN, ROUT = 0.25, 0.45


def _path(o, p, k):
    _, _, lens, n = o.ray_tau(p, k, synth.nu_of(1215.67) * 1.01, cap=100000)
    return lens.sum(), n


@pytest.mark.parametrize("r0", [0.3, 0.37, 0.44])
def test_shell_path_lengths(r0):
    wl = synth.shell(n_packets=1)
    o = oracle.Oracle(wl)
    c = np.array([0.5, 0.5, 0.5])
    rng = np.random.default_rng(int(r0 * 100))
    for _ in range(20):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        p = c + r0 * u
        # radially outwards and inwards
        L, _ = _path(o, p, u)
        assert abs(L - (ROUT - r0)) < 1e-12
        L, _ = _path(o, p, -u)
        assert abs(L - (r0 - RIN)) < 1e-12
        # oblique: impact parameter b about the centre
        w = rng.normal(size=3)
        w -= w.dot(u) * u
        w /= np.linalg.norm(w)
        for cosang in (-0.9, -0.5, -0.1, 0.3):
            k = cosang * u + math.sqrt(1 - cosang ** 2) * w
            b = r0 * math.sqrt(1 - cosang ** 2)
            s0 = r0 * cosang                       # distance along k to closest approach is -s0
            if cosang < 0 and b < RIN:
                exp = -s0 - math.sqrt(RIN ** 2 - b ** 2)   # meets the inner sphere
            else:
                exp = math.sqrt(ROUT ** 2 - b ** 2) - s0
            L, _ = _path(o, p, k)
            assert abs(L - exp) < 1e-12, (r0, cosang, L, exp)


def test_shell_packets_leave_through_a_sphere():
    wl = synth.shell(tau0=1e3, n_packets=300)
    out, _ = oracle.Oracle(wl).run(threads=8)
    assert (out["status"] == oracle.ESCAPED).all()
    r = np.linalg.norm(out["pos"] - 0.5, axis=1)
    on = (np.abs(r - RIN) < 1e-12) | (np.abs(r - ROUT) < 1e-12)
    assert on.all(), r[~on][:5]
    f_in = (np.abs(r - RIN) < 1e-12).mean()
    assert 0.05 < f_in < 0.6     # both exits are used

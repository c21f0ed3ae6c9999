"""Pins of the oracle's adjoint: with the peeling record fixed (positions,
directions, external frequencies, weights of every peeling event), the peeled
cube is a smooth function of the leaf fields through the optical depths of the
peeling rays, and the analytic gradient must match central finite differences
of that function.  The GPU adjoint is checked against this oracle."""
import numpy as np
import pytest

import oracle
import synth

FIELDS = ["n_HI", "vx", "vy", "vz", "T", "n_dust"]


def _setup():
    wl = synth.expanding_sphere(N_HI=3e17, tau_dust=0.3, n_packets=30, npix=8, nchan=24, base=3, max_level=3)
    wl.physics.tau_stop = float("inf")
    o = oracle.Oracle(wl)
    out, tal = o.run(record_events=200000)
    return wl, o, tal


def test_voigt_derivatives_match_differences():
    """dH/da and dH/dx of the implemented H (Tasitsiomi form)."""
    import ctypes as C
    for a in (4.7e-4, 1e-2):
        for x in (0.0, 0.5, 0.93, 1.7, 3.0, 7.5, -2.2, 40.0):
            H, Ha, Hx = C.c_double(), C.c_double(), C.c_double()
            oracle.lib().ora_voigt_derivs(a, x, C.byref(H), C.byref(Ha), C.byref(Hx))
            assert abs(H.value - oracle.voigt(a, x)) <= 1e-15 * abs(H.value)
            ha = (oracle.voigt(1.5 * a, x) - oracle.voigt(0.5 * a, x)) / a   # H is linear in a
            hx = (oracle.voigt(a, x + 1e-6) - oracle.voigt(a, x - 1e-6)) / 2e-6
            assert abs(Ha.value - ha) <= 1e-6 * (abs(ha) + 1e-12)
            assert abs(Hx.value - hx) <= 1e-6 * (abs(hx) + 1e-9)


@pytest.mark.parametrize("which", ["cube", "image", "spectrum"])
def test_adjoint_matches_finite_differences(which):
    wl, o, tal = _setup()
    ev = tal["events"]
    rng = np.random.default_rng(7)
    g = {"cube": None, "image": None, "spectrum": None}
    key = {"cube": "pcube", "image": "pimg", "spectrum": "pspec"}[which]
    g[which] = rng.normal(size=tal[key].shape)
    grad = o.adjoint(ev, g_cube=g["cube"], g_img=g["image"], g_spec=g["spectrum"])

    def loss():
        t = o.peel_from_events(ev)
        return float((g[which] * t[key]).sum())

    m = wl.medium
    for j, name in enumerate(FIELDS):
        base = np.array(getattr(m, name), dtype=np.float32)
        cells = list(np.argsort(-np.abs(grad[j]))[:4]) + list(rng.integers(0, base.size, 2))
        for c in cells:
            v0 = float(base[c])
            h = max(abs(v0) * 1e-3, 1e3 if name.startswith("v") else 1e-30)
            vals = []
            for sgn in (1, -1):
                f = base.copy()
                f[c] = np.float32(v0 + sgn * h)
                vals.append(float(f[c]))
                o.set_field(name, f)
                vals.append(loss())
            o.set_field(name, base)
            fd = (vals[1] - vals[3]) / (vals[0] - vals[2])
            scale = np.abs(grad[j]).max() + 1e-300
            assert abs(fd - grad[j, c]) <= 2e-4 * abs(grad[j, c]) + 1e-7 * scale, (name, c, fd, grad[j, c])

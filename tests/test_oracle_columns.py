"""Pins of the oracle's column densities along rays (no GPU).

The paper's ray-tracing by-product (Sect. 5 introduction and Sect. 6: escape
fractions of ionising photons from optical depths integrated along many rays,
column densities along arbitrary sight lines) is the walk of Sect. 4.3 with
the line profile left out: N_X = sum over the leaves crossed of n_X l L."""
import math

import numpy as np
import pytest

import oracle
import synth


def _chord(p, k, c, R):
    d = np.asarray(p) - np.asarray(c)
    b = d @ k
    return -b + math.sqrt(b * b - (d @ d - R * R))


@pytest.mark.parametrize("mesh", ["one_cell", "sphere"])
def test_uniform_sphere_chords(mesh):
    """Uniform sphere: N_HI = n t L and N_dust = n_dust t L with t the
    closed-form chord from p to the sphere along k (1e-12)."""
    if mesh == "one_cell":
        wl = synth.sphere(tau0=1e4, T=1e4, tau_dust=0.5, n_packets=1, base=1, max_level=1)
    else:
        wl = synth.sphere(tau0=1e4, T=1e4, tau_dust=0.5, n_packets=1, base=3, max_level=6)
    o = oracle.Oracle(wl)
    rng = np.random.default_rng(3)
    c, R, L = np.array(wl.domain.centre), wl.domain.size, wl.medium.box_cm
    n_hi, n_d = float(wl.medium.n_HI[0]), float(wl.medium.n_dust[0])
    for i in range(300):
        v = rng.normal(size=3)
        p = c + v / np.linalg.norm(v) * R * rng.random() ** (1 / 3) * 0.99
        if i < 20:
            p = c.copy()
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        cols, ncell = o.ray_columns(p, k)
        t = _chord(p, k, c, R)
        assert ncell >= 1
        assert abs(cols[0] / (n_hi * t * L) - 1) < 1e-12, (i, cols[0], n_hi * t * L)
        assert abs(cols[1] / (n_d * t * L) - 1) < 1e-12
        assert cols[2] == 0.0
    # from the centre: the centre-to-edge column that defines tau0
    cols, _ = o.ray_columns(c, np.array([0.0, 0.0, 1.0]))
    assert abs(cols[0] / (n_hi * R * L) - 1) < 1e-12


def test_columns_follow_the_walk_of_ray_tau():
    """On a graded galaxy octree the columns cross the same leaves with the
    same path lengths as the optical-depth walk: N_HI = sum n_HI[cell] l L
    over ray_tau's leaf list."""
    wl = synth.galaxy(n_leaf=60_000, grid_level=5, base_level=3, max_level=8, n_packets=4, npix=4, nchan=4)
    o = oracle.Oracle(wl)
    rng = np.random.default_rng(9)
    L = wl.medium.box_cm
    nh = wl.medium.n_HI.astype(np.float64)
    nd = wl.medium.n_dust.astype(np.float64)
    nm = wl.medium.n_metal.astype(np.float64)
    nu0 = synth.nu_of(wl.lines[0].lambda_A)
    for i in range(60):
        p = rng.random(3)
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        cols, ncell = o.ray_columns(p, k)
        _, cells, lens, n2 = o.ray_tau(p, k, nu0, cap=100_000)
        assert ncell == n2
        ref = [(x[cells] * lens).sum() * L for x in (nh, nd, nm)]
        for j in range(3):
            assert abs(cols[j] - ref[j]) <= 1e-12 * abs(ref[j]) + 1e-300, (i, j)


def test_ray_outside_the_box():
    wl = synth.sphere(tau0=1e3, T=1e4, n_packets=1, base=2, max_level=3)
    cols, n = oracle.Oracle(wl).ray_columns([1.5, 0.5, 0.5], [1.0, 0.0, 0.0])
    assert n == 0 and (cols == 0).all()

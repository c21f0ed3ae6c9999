"""Column densities along rays (rascas_ray_columns; the ray-tracing use of
Sects. 5 and 6) on the GPU against the FP64 oracle (needs a GB300)."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context

pytestmark = pytest.mark.gpu


def _rays(wl, n, rng, inside):
    if inside:
        c = np.array(wl.domain.centre)
        v = rng.normal(size=(n, 3))
        pos = c + v / np.linalg.norm(v, axis=1)[:, None] * (wl.domain.size * 0.99 * rng.random(n) ** (1 / 3))[:, None]
    else:
        pos = rng.random((n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pos[:16] = np.round(pos[:16] * 64) / 64    # start on faces, edges, corners
    d[:8, 0] = 0.0
    d[:8] /= np.linalg.norm(d[:8], axis=1)[:, None]
    return pos, d


@pytest.mark.parametrize("which", ["sphere", "galaxy", "slab"])
def test_columns_match_oracle(which):
    """Same number of leaves as the oracle's walk (bit-exact walk), columns
    within 1e-6 relative, tau = sigma_HI N_HI + sigma_d N_dust."""
    rng = np.random.default_rng(21)
    if which == "sphere":
        wl = synth.sphere(tau0=1e5, T=1e4, tau_dust=0.7, n_packets=1, base=3, max_level=6)
    elif which == "slab":
        wl = synth.slab(tau0=1e4, T=1e4, tau_dust=0.3, n_packets=1)
    else:
        wl = synth.galaxy(n_leaf=150_000, grid_level=6, base_level=4, max_level=10, n_packets=4, npix=4, nchan=4)
    ctx = context(wl)
    o = oracle.Oracle(wl)
    pos, d = _rays(wl, 2000, rng, which == "sphere")
    sig_hi, sig_d = 6.3e-18, 4e-22
    cols, tau, ncell = ctx.ray_columns(pos, d, sig_hi, sig_d)
    for i in range(pos.shape[0]):
        c_o, n_o = o.ray_columns(pos[i], d[i])
        assert ncell[i] == n_o, i
        for j in range(3):
            assert abs(cols[i, j] - c_o[j]) <= 1e-6 * abs(c_o[j]) + 1e-300, (i, j, cols[i, j], c_o[j])
        t_o = sig_hi * c_o[0] + sig_d * c_o[1]
        assert abs(tau[i] - t_o) <= 1e-6 * t_o + 1e-300


def test_columns_closed_form_and_device_buffers():
    """Uniform sphere from its centre: N_HI = n R L for every direction
    (1e-6), through torch device buffers on torch's stream; rays outside the
    box get zeros."""
    import torch
    wl = synth.sphere(tau0=1e6, T=1e4, tau_dust=1.0, n_packets=1, base=3, max_level=6)
    ctx = context(wl)
    rng = np.random.default_rng(4)
    n = 1 << 16
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pos = np.tile(np.array(wl.domain.centre), (n, 1))
    pos[-3:] = [[1.5, 0.5, 0.5], [-0.1, 0.5, 0.5], [0.5, 0.5, 2.0]]
    dev = torch.device("cuda:0")
    cols, tau, ncell = ctx.ray_columns(torch.tensor(pos, device=dev), torch.tensor(d, device=dev))
    cols, ncell = cols.cpu().numpy(), ncell.cpu().numpy()
    N = float(wl.medium.n_HI[0]) * wl.domain.size * wl.medium.box_cm
    assert np.abs(cols[:-3, 0] / N - 1).max() < 1e-6
    assert (cols[-3:] == 0).all() and (ncell[-3:] == 0).all() and ncell[:-3].min() >= 1

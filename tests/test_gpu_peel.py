"""Deferred peeling (Sect. 3.1 peeling): the scattering kernel appends one
record per emission or scattering and observer direction, the peel kernel
walks and tallies them; when the record buffer fills, packets are parked in
device memory and resumed after the records are walked.  Parking must not
change any packet's history, and the tallies only by the order of their
floating-point sums."""
import numpy as np
import pytest

import synth
from gpu_util import context, gpu_run

pytestmark = pytest.mark.gpu


def test_parked_rounds_give_the_same_run():
    wl = synth.expanding_sphere(N_HI=1e19, n_packets=400, npix=16, nchan=40)
    one = context(wl)
    g1, s1 = gpu_run(one, wl.packets)
    many = context(wl)
    many.set_peel_capacity(1)   # raised to the floor of the launch shape: many rounds
    g2, s2 = gpu_run(many, wl.packets)
    print("peeling rays", s1["npeel_rays"], "cells", s1["npeel_cells"])
    assert s1["npeel_rays"] > 4_000_000   # several rounds at the floor capacity
    for k in ("status", "nscatt", "nu", "pos", "dir", "path"):
        assert np.array_equal(g1[k], g2[k]), k
    for k in ("escaped", "absorbed", "capped", "nscatt_line", "nscatt_dust", "npeel_rays", "npeel_cells"):
        assert s1[k] == s2[k], k
    for kind in (1, 2, 3):
        a, b = one.get_tally(kind), many.get_tally(kind)
        assert np.allclose(a, b, rtol=2e-5, atol=1e-6 * float(np.abs(a).max())), kind
    one.close()
    many.close()


def test_peel_capacity_argument():
    import paper_2001_11252_gb300 as rg
    wl = synth.expanding_sphere(N_HI=1e17, n_packets=10, npix=4, nchan=8)
    ctx = context(wl)
    with pytest.raises(rg.RascasError):
        ctx.set_peel_capacity(0)
    ctx.close()

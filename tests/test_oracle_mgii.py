"""Mg II doublet (Table 1) in an outflow: two resonant lines of one ion,
770 km/s apart.  With v_max = 200 km/s the lines never overlap and neither
line has a fluorescent channel, so each photon leaves in the line it was
emitted in (exact), redshifted by the outflow; the 2796 line, twice as
thick, keeps its photons longer."""
import numpy as np

import oracle
import synth


def test_mgii_doublet_lines_stay_apart():
    n = 3000
    wl = synth.mgII_wind(N_MgII=1e15, n_packets=n)
    out, _ = oracle.Oracle(wl).run(threads=8)
    assert (out["status"] == oracle.ESCAPED).all()
    lam = synth.C_CGS / out["nu"] * 1e8
    born_red = np.abs(synth.C_CGS / wl.packets.nu * 1e8 - 2803.53) < 0.01
    near03 = np.abs(lam - 2803.53) < 4.0
    near96 = np.abs(lam - 2796.35) < 4.0
    assert np.array_equal(near03, born_red) and np.array_equal(near96, ~born_red)
    # outflow: both lines escape redshifted on average
    assert lam[near96].mean() > 2796.35 and lam[near03].mean() > 2803.53
    # the stronger line scatters more
    assert out["nscatt"][near96].mean() > 1.3 * out["nscatt"][near03].mean()

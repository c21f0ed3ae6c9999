"""Bounded device work and caps (needs a GB300): a persistent kernel that
reaches its iteration or time limit returns RASCAS_E_TIMEOUT and leaves the
context usable; fail_on_cap turns capped packets into RASCAS_E_CAPPED.  The
limits are made to run out on purpose with tiny values: no GPU fault, no
hang, only an error status read on the host."""
import numpy as np
import pytest

import synth
from gpu_util import context, gpu_run

pytestmark = pytest.mark.gpu


def _timeout(fn):
    import paper_2001_11252_gb300 as rg
    with pytest.raises(rg.RascasError) as e:
        fn()
    assert "E_TIMEOUT" in str(e.value), str(e.value)


@pytest.mark.parametrize("limit", ["iterations", "time"])
def test_propagate_limit_returns_timeout(limit):
    wl = synth.slab(tau0=1e5, T=1e4, n_packets=4096)
    ctx = context(wl)
    ref, st_ref = gpu_run(ctx, wl.packets)
    if limit == "iterations":
        ctx.set_limits(max_iterations=50)
    else:
        ctx.set_limits(time_limit_s=1e-6)
    # device buffers, so that slots of packets never started keep their -1
    import torch
    dev = torch.device("cuda:0")
    pk = wl.packets
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
    out = {"status": torch.full((pk.n,), -1, dtype=torch.int32, device=dev)}
    _timeout(lambda: ctx.propagate(t(pk.pos, torch.float64), t(pk.dir, torch.float64), t(pk.nu, torch.float64),
                                   t(pk.ids.view(np.int64), torch.int64), out=out))
    status = out["status"].cpu().numpy()
    # packets in flight were left unfinished, the rest untouched or finished
    print(limit, "statuses after the limit:", np.unique(status, return_counts=True))
    assert (status == 0).any()
    assert np.isin(status, [-1, 0, 1]).all()
    # the context is still usable and gives the same results without limits
    ctx.set_limits(0, 0.0)
    again, st = gpu_run(ctx, wl.packets)
    for k in ("status", "nscatt", "nu", "pos"):
        assert np.array_equal(again[k], ref[k]), k
    assert st["nscatt_line"] == st_ref["nscatt_line"]


def test_limits_far_away_change_nothing():
    wl = synth.sphere(tau0=1e4, T=1e4, tau_dust=1.0, n_packets=2048, base=3, max_level=5)
    ctx = context(wl)
    ref, _ = gpu_run(ctx, wl.packets)
    ctx.set_limits(max_iterations=1 << 30, time_limit_s=600.0)
    got, _ = gpu_run(ctx, wl.packets)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), k


def test_peeling_and_batch_limits_return_timeout():
    import paper_2001_11252_gb300 as rg
    wl = synth.expanding_sphere(N_HI=1e19, n_packets=2048, npix=8, nchan=24, base=3, max_level=5)
    ctx = context(wl)
    ctx.set_limits(max_iterations=20)
    _timeout(lambda: ctx.propagate(wl.packets.pos, wl.packets.dir, wl.packets.nu, wl.packets.ids, out={}))
    ctx.set_limits(0, 0.0)
    ctx.zero_tallies()
    st = ctx.propagate(wl.packets.pos, wl.packets.dir, wl.packets.nu, wl.packets.ids, out={})
    assert st["escaped"] + st["absorbed"] == wl.packets.n
    models = synth.batch_models(12, packet_scale=0.01, seed_offset=3)
    b = rg.Context(0)
    b.set_lines(models[0].lines, models[0].dust)
    ph = models[0].physics
    b.set_physics(ph.recoil, ph.isotropic, 0, ph.x_gauss, 20000, 0, ph.tau_stop, ph.seed)
    b.load_batch(models, nbin=50)
    ref = b.propagate_batch(rg.BATCH_PERSISTENT)
    b.set_limits(max_iterations=30)
    _timeout(lambda: b.propagate_batch(rg.BATCH_PERSISTENT))
    b.set_limits(0, 0.0)
    st = b.propagate_batch(rg.BATCH_PERSISTENT)
    assert st["nscatt_line"] == ref["nscatt_line"]


def test_fail_on_cap_returns_capped():
    import paper_2001_11252_gb300 as rg
    wl = synth.slab(tau0=1e4, T=1e4, n_packets=512)
    ctx = context(wl)
    ph = wl.physics
    ctx.set_physics(ph.recoil, ph.isotropic, 0, ph.x_gauss, 10, 0, ph.tau_stop, ph.seed, fail_on_cap=1)
    out = {"status": np.zeros(512, np.int32), "nscatt": np.zeros(512, np.int64)}
    with pytest.raises(rg.RascasError) as e:
        ctx.propagate(wl.packets.pos, wl.packets.dir, wl.packets.nu, wl.packets.ids, out=out)
    assert "E_CAPPED" in str(e.value)
    # the outputs were written before the error was returned
    assert (out["status"] == rg.PK_CAPPED).sum() > 0 and (out["nscatt"] <= 10).all()
    assert ((out["status"] == rg.PK_CAPPED) == (out["nscatt"] == 10)).all()
    # without the flag the same run succeeds
    ctx.set_physics(ph.recoil, ph.isotropic, 0, ph.x_gauss, 10, 0, ph.tau_stop, ph.seed, fail_on_cap=0)
    st = ctx.propagate(wl.packets.pos, wl.packets.dir, wl.packets.nu, wl.packets.ids, out=out)
    assert st["capped"] > 0

"""Parity at the full sizes the bench measures, in the launch shape it times
(the persistent grid over one batch of 2^18 packets; 2^20 rays through the
9.2-million-leaf galaxy), checked on sampled outputs that the oracle computes
one by one, plus properties that hold at any size."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context

pytestmark = pytest.mark.gpu

P_BENCH = 1 << 18


def _bench_sphere():
    import bench
    wl = bench.workload(8)
    return wl, bench.packets(wl, 0, P_BENCH)


def test_sphere_bench_batch_sampled_packets():
    """Static sphere, tau0 = 1e6, tau_dust = 1: the whole batch on the GPU;
    4096 sampled packets rerun by the oracle on the same random streams."""
    import torch
    wl, pk = _bench_sphere()
    ctx = context(wl)
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
    out = {"status": torch.zeros(P_BENCH, dtype=torch.int32, device=dev),
           "nscatt": torch.zeros(P_BENCH, dtype=torch.int64, device=dev),
           "nu": torch.zeros(P_BENCH, dtype=torch.float64, device=dev)}
    st = ctx.propagate(t(pk.pos, torch.float64), t(pk.dir, torch.float64), t(pk.nu, torch.float64),
                       t(pk.ids.view(np.int64), torch.int64), out=out)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    # properties of the whole batch
    assert st["packets"] == P_BENCH and st["errors"] == 0
    assert st["escaped"] + st["absorbed"] + st["capped"] == P_BENCH
    assert st["nscatt_line"] + st["nscatt_dust"] == int(g["nscatt"].sum())
    assert int(ctx.get_tally(0).sum()) <= st["escaped"]
    # sampled packets, one by one on the oracle
    sel = np.sort(np.random.default_rng(5).choice(P_BENCH, 4096, replace=False))
    sub = synth.Packets(pk.pos[sel], pk.dir[sel], pk.nu[sel], pk.ids[sel])
    r, _ = oracle.Oracle(wl).run(packets=sub, threads=16, chunk=1)
    same = (g["status"][sel] == r["status"]) & (g["nscatt"][sel] == r["nscatt"])
    print("full-size sphere: identical histories %d / %d, <N> %.4g vs %.4g"
          % (same.sum(), sel.size, g["nscatt"][sel].mean(), r["nscatt"].mean()))
    # the mean scattering count of the sampled packets within 1 %
    assert abs(g["nscatt"][sel].mean() / r["nscatt"].mean() - 1) < 0.01
    # Histories with the same decisions end at nearly the same frequency: the
    # FP32 velocity sampling differs from FP64 by ~1e-7 per scattering and the
    # difference random-walks over ~3e5 scatterings, except where a far-wing
    # draw (u_par = x - a / tan(A r) with small A r) magnifies it.
    dnu = synth.doppler_width(wl.lines[0], 1e4)
    dx = np.abs(g["nu"][sel][same] - r["nu"][same]) / dnu
    print("final |x_gpu - x_oracle| of identical-count histories:", np.sort(dx))
    assert same.mean() >= 0.75, same.mean()
    assert np.median(dx) < 1e-5 and (dx < 1e-2).mean() >= 0.8, np.sort(dx)


def test_sphere_bench_batch_replay_per_step():
    """The first events of every packet of the batch, traced on the GPU with
    the bench's launch shape; 256 sampled packets replayed step by step by the
    oracle from the GPU's states."""
    wl, pk = _bench_sphere()
    ctx = context(wl)
    ev, cnt = ctx.trace(pk.pos, pk.dir, pk.nu, pk.ids, 12)
    assert cnt.min() >= 1
    o = oracle.Oracle(wl)
    sel = np.random.default_rng(6).choice(P_BENCH, 256, replace=False)
    steps = mism = 0
    pos = dirn = xerr = 0.0
    dnu = synth.doppler_width(wl.lines[0], 1e4)
    for i in sel:
        for j in range(int(cnt[i]) - 1):
            a, b = ev[i, j], ev[i, j + 1]
            s = oracle.State()
            s.p[:] = list(a["p"]); s.k[:] = list(a["k"]); s.nu = float(a["nu"])
            s.leaf, s.level = int(a["leaf"]), int(a["level"])
            s.ijk[:] = [int(v) for v in a["ijk"]]
            s.pid = int(pk.ids[i]); s.ndraw = int(a["ndraw"])
            s.nscatt, s.nsteps, s.status = int(a["nscatt"]), int(a["nsteps"]), 0
            o.event(s)
            steps += 1
            if not (s.status == b["status"] and s.ndraw == b["ndraw"] and s.leaf == b["leaf"]
                    and s.nscatt == b["nscatt"]):
                mism += 1
                continue
            step = np.linalg.norm(np.array(b["p"]) - np.array(a["p"])) + 1e-300
            pos = max(pos, np.abs(np.array(s.p) - b["p"]).max() / step)
            dirn = max(dirn, np.abs(np.array(s.k) - b["k"]).max())
            xerr = max(xerr, abs(s.nu - b["nu"]) / dnu)
    print("full-size replay: steps %d mismatches %d pos %.2e dir %.2e x %.2e" % (steps, mism, pos, dirn, xerr))
    assert steps > 2000
    assert mism <= 0.002 * steps + 2
    assert pos < 1e-6 and dirn < 1e-6 and xerr < 3e-5


def test_galaxy_full_size_rays_sampled():
    """2^20 rays through the 9.2-million-leaf galaxy as the bench casts them;
    64 sampled rays walked by the oracle: same optical depth (1e-6), and the
    same leaves with the same FP64 path lengths."""
    import torch
    n = 1 << 20
    wl = synth.galaxy(n_packets=n)
    ctx = context(wl)
    rng = np.random.default_rng(7)
    mu = 2 * rng.random(n) - 1
    phi = 2 * math.pi * rng.random(n)
    stt = np.sqrt(1 - mu * mu)
    d = np.stack([stt * np.cos(phi), stt * np.sin(phi), mu], 1)
    nu0 = synth.nu_of(wl.lines[0].lambda_A)
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev, torch.float64)
    tau, _, _, ncell = ctx.ray_tau(t(wl.packets.pos[:n]), t(d), t(np.full(n, nu0)))
    tau, ncell = tau.cpu().numpy(), ncell.cpu().numpy()
    assert np.all(np.isfinite(tau)) and np.all(tau >= 0) and ncell.min() >= 1
    sel = np.random.default_rng(8).choice(n, 64, replace=False)
    cap = 8192
    _, cells, lens, nc2 = ctx.ray_tau(wl.packets.pos[sel], d[sel], np.full(64, nu0), cap=cap)
    o = oracle.Oracle(wl)
    for j, i in enumerate(sel):
        t_o, c_o, l_o, n_o = o.ray_tau(wl.packets.pos[i], d[i], nu0, cap=cap)
        assert ncell[i] == n_o == nc2[j]
        m = min(n_o, cap)
        assert np.array_equal(cells[j, :m], c_o[:m]) and np.array_equal(lens[j, :m], l_o[:m]), i
        assert abs(tau[i] - t_o) <= 1e-6 * abs(t_o), (i, tau[i], t_o)


def test_galaxy_full_size_core_skip_sampled_packets():
    """The bench's core-skipped galaxy run (9.2-million-leaf octree as
    generated, x_crit = 0.5 (a tau_cell)^(1/3), peeling into 4 x 256^2 x 400
    cubes) at 2^18 packets in the bench's launch shape; 256 sampled packets
    rerun by the oracle on the same streams: identical fates and scattering
    counts for almost all, every packet finished without a cap."""
    import torch
    n = 1 << 18
    wl = synth.galaxy(n_packets=n)
    wl.physics.core_skip_f = 0.5
    wl.physics.max_scatt = 1_000_000
    ctx = context(wl)
    dev = torch.device("cuda:0")
    pk = wl.packets
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
    out = {"status": torch.zeros(n, dtype=torch.int32, device=dev),
           "nscatt": torch.zeros(n, dtype=torch.int64, device=dev)}
    st = ctx.propagate(t(pk.pos, torch.float64), t(pk.dir, torch.float64), t(pk.nu, torch.float64),
                       t(pk.ids.view(np.int64), torch.int64), out=out)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    assert st["packets"] == n and st["errors"] == 0 and st["capped"] == 0
    assert st["escaped"] + st["absorbed"] == n
    assert st["npeel_rays"] == 4 * (st["nscatt_line"] + st["nscatt_dust"] + n)
    sel = np.sort(np.random.default_rng(9).choice(n, 256, replace=False))
    sub = synth.Packets(pk.pos[sel], pk.dir[sel], pk.nu[sel], pk.ids[sel])
    r, _ = oracle.Oracle(wl).run(packets=sub, threads=16, chunk=4)
    same = ((g["status"][sel] == r["status"]) & (g["nscatt"][sel] == r["nscatt"])).mean()
    print("galaxy core-skipped: identical %.4f, <N> %.3f vs %.3f, statuses %s"
          % (same, g["nscatt"][sel].mean(), r["nscatt"].mean(), np.bincount(r["status"], minlength=5)))
    assert same > 0.97

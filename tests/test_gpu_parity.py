"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances (the hot path's own statement): cell indices and octree walks
bit-exact; per-step tau, Voigt and distances within 1e-6 relative; escape
spectra, images and mean scattering counts statistically (KS / chi-square
p > 0.01, <N_scatt> within 1%).  Runs are coupled: both sides draw the same
Philox4x32-10 words for a packet id, so per-packet histories agree until an
FP32 decision (a rejection test, a branch) lands within rounding of its
threshold."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import context, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def _x(wl, nu):
    ln = wl.lines[0]
    return (nu - synth.nu_of(ln.lambda_A)) / synth.doppler_width(ln, float(wl.medium.T[0]))


# ---------------------------------------------------------------- building blocks
def test_voigt_matches_oracle():
    """H(a,x) (Tasitsiomi form, Sect. 3.3.2) within 1e-6 relative."""
    wl = synth.slab(n_packets=1)
    ctx = context(wl)
    rng = np.random.default_rng(3)
    a = np.concatenate([np.full(4000, 4.717e-4), 10 ** rng.uniform(-5, -1.5, 4000)]).astype(np.float32)
    x = np.concatenate([rng.uniform(-12, 12, 4000), np.concatenate([rng.uniform(-5, 5, 2000),
                                                                    10 ** rng.uniform(0, 4, 2000)])])
    x[:8] = [0.0, 0.9246, -0.9247, 3.0, 3.3, 8.0, 1e3, -2.5]
    H = ctx.eval_voigt(a, x).astype(np.float64)
    ref = np.array([oracle.voigt(float(ai), float(xi)) for ai, xi in zip(a, x)])
    rel = np.abs(H / ref - 1)
    assert rel.max() < 1e-6, (rel.max(), x[rel.argmax()], a[rel.argmax()])


def test_upar_matches_oracle_streams():
    """u_par draws on identical streams (Sect. 3.3.3): same number of words,
    same value to FP32 accuracy, apart from rare FP32-vs-FP64 accept ties."""
    wl = synth.slab(n_packets=1)
    ctx = context(wl)
    o = oracle.Oracle(wl)
    rng = np.random.default_rng(4)
    n = 3000
    x = np.concatenate([rng.uniform(-9, 9, n // 2), rng.uniform(-3, 3, n // 2)])
    a = np.where(rng.random(n) < 0.5, 4.717e-4, 10 ** rng.uniform(-4, -2, n)).astype(np.float32)
    ids = np.arange(n, dtype=np.uint64) + 777
    u, nd = ctx.sample_upar(x, a, ids)
    ref = np.array([o.upar_samples(float(np.float32(xi)), float(ai), 1, pid=int(i))[0]
                    for xi, ai, i in zip(x, a, ids)])
    same = np.abs(u - ref) <= 2e-5 * (1 + np.abs(ref))
    assert (nd > 0).all()
    assert same.mean() > 0.998, same.mean()


# ---------------------------------------------------------------- walk
@pytest.mark.parametrize("which", ["sphere", "slab", "expanding", "galaxy", "shell"])
def test_ray_walk_bit_exact(which):
    """Octree walk (Sect. 4.3): identical leaf sequence and identical FP64
    path lengths per leaf; tau within 1e-6 relative."""
    if which == "sphere":
        wl = synth.sphere(tau0=1e4, T=1e4, tau_dust=0.5, n_packets=1, base=3, max_level=6)
    elif which == "slab":
        wl = synth.slab(tau0=1e3, n_packets=1)
    elif which == "galaxy":
        wl = synth.galaxy(n_leaf=150_000, grid_level=6, base_level=4, max_level=10, n_packets=10, npix=8, nchan=8)
    elif which == "shell":
        wl = synth.shell(n_packets=1, v_max_kms=100.0)
    else:
        wl = synth.expanding_sphere(n_packets=1)
    ctx = context(wl)
    o = oracle.Oracle(wl)
    rng = np.random.default_rng(11)
    n = 400
    pos = rng.uniform(0.1, 0.9, (n, 3))
    if which == "slab":
        pos[:, 2] = rng.uniform(0.0, 1.0, n)
    elif which == "galaxy":
        pos = rng.uniform(0.0, 1.0, (n, 3))
    else:
        c = np.array(wl.domain.centre)
        r = wl.domain.size * rng.random(n) ** (1 / 3) * 0.999
        v = rng.normal(size=(n, 3))
        pos = c + v / np.linalg.norm(v, axis=1)[:, None] * r[:, None]
    pos[:20] = np.round(pos[:20] * 64) / 64      # start on faces/edges/corners
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    d[:10, 0] = 0.0
    d[:10] /= np.linalg.norm(d[:10], axis=1)[:, None]
    nu0 = synth.nu_of(wl.lines[0].lambda_A)
    dnu = synth.doppler_width(wl.lines[0], 1e4)
    nu = nu0 + rng.uniform(-10, 10, n) * dnu
    cap = 4096
    tau, cells, lens, ncell = ctx.ray_tau(pos, d, nu, cap=cap)
    for i in range(n):
        t_o, c_o, l_o, n_o = o.ray_tau(pos[i], d[i], nu[i], cap=cap)
        assert ncell[i] == n_o
        m = min(n_o, cap)
        assert np.array_equal(cells[i, :m], c_o[:m]), i
        assert np.array_equal(lens[i, :m], l_o[:m]), i
        assert abs(tau[i] - t_o) <= 1e-6 * abs(t_o) + 1e-300, (i, tau[i], t_o)


# ---------------------------------------------------------------- per-step replay
def _replay(wl, n_packets, max_events):
    ctx = context(wl)
    o = oracle.Oracle(wl)
    pk = wl.packets
    ev, cnt = ctx.trace(pk.pos[:n_packets], pk.dir[:n_packets], pk.nu[:n_packets], pk.ids[:n_packets], max_events)
    ln = wl.lines[0]
    stats = {"steps": 0, "mismatch": 0, "pos": 0.0, "dir": 0.0, "x": 0.0}
    for i in range(n_packets):
        for j in range(cnt[i] - 1):
            a, b = ev[i, j], ev[i, j + 1]
            s = oracle.State()
            s.p[:] = list(a["p"]); s.k[:] = list(a["k"]); s.nu = float(a["nu"])
            s.leaf, s.level = int(a["leaf"]), int(a["level"])
            s.ijk[:] = [int(v) for v in a["ijk"]]
            s.pid = int(pk.ids[i]); s.ndraw = int(a["ndraw"])
            s.nscatt, s.nsteps, s.status = int(a["nscatt"]), int(a["nsteps"]), 0
            o.event(s)
            stats["steps"] += 1
            ok = (s.status == b["status"] and s.ndraw == b["ndraw"] and s.leaf == b["leaf"]
                  and s.nscatt == b["nscatt"] and s.nsteps == b["nsteps"])
            if not ok:
                stats["mismatch"] += 1
                continue
            step = np.linalg.norm(np.array(b["p"]) - np.array(a["p"])) + 1e-300
            stats["pos"] = max(stats["pos"], np.abs(np.array(s.p) - b["p"]).max() / step)
            de = np.abs(np.array(s.k) - b["k"]).max()
            if de > stats["dir"]:
                stats["dir"] = de
                stats["dir_case"] = (list(a["k"]), list(b["k"]), list(s.k), int(a["ndraw"]), int(b["ndraw"]))
            dnu = synth.doppler_width(ln, float(wl.medium.T[b["leaf"]]))
            stats["x"] = max(stats["x"], abs(s.nu - b["nu"]) / dnu)
    return stats


@pytest.mark.parametrize("which", ["slab", "sphere_dust", "expanding"])
def test_trace_replay_per_step(which):
    """Each GPU event, replayed by the oracle from the GPU's state, lands on
    the same leaf with the same draw count and status; positions agree to
    1e-6 of the step; directions to 1e-6 and outgoing frequencies to 3e-5
    Doppler widths (both produced by FP32 velocity and angle sampling: a few
    FP32 ulps of |x| + |u_par| <= ~20)."""
    if which == "slab":
        wl = synth.slab(tau0=1e4, n_packets=64)
    elif which == "sphere_dust":
        wl = synth.sphere(tau0=1e4, T=1e4, tau_dust=1.0, n_packets=64)
    else:
        wl = synth.expanding_sphere(n_packets=64, N_HI=1e18)
    st = _replay(wl, 64, 200)
    print(which, st)
    assert st["steps"] > 1000
    assert st["mismatch"] <= 0.002 * st["steps"] + 2
    assert st["pos"] < 1e-6
    assert st["dir"] < 1e-6
    assert st["x"] < 3e-5


# ---------------------------------------------------------------- whole runs
def _ks(a, b):
    from scipy.stats import ks_2samp
    return ks_2samp(a, b).pvalue


def test_slab_run_matches_oracle():
    """Static slab, tau0 = 1e4, T = 1e4 K, 2000 packets (Sect. 3.4.2)."""
    wl = synth.slab(tau0=1e4, T=1e4, n_packets=2000)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    r, tal = oracle_run(wl)
    assert np.all(g["status"] == oracle.ESCAPED) and np.all(r["status"] == oracle.ESCAPED)
    assert st["packets"] == 2000 and st["escaped"] == 2000
    same = (g["nscatt"] == r["nscatt"]).mean()
    mg, mr = g["nscatt"].mean(), r["nscatt"].mean()
    print("slab: identical histories %.4f, <N> gpu %.1f oracle %.1f" % (same, mg, mr))
    assert abs(mg / mr - 1) < 0.01
    assert same > 0.5
    assert _ks(_x(wl, g["nu"]), _x(wl, r["nu"])) > 0.01
    spec = ctx.get_tally(0)
    assert spec.sum() == 2000
    assert st["nscatt_line"] == g["nscatt"].sum()


@pytest.mark.parametrize("tau_dust", [0.0, 1.0])
def test_sphere_run_matches_oracle(tau_dust):
    """Static sphere with dust (the 3-level 8^3 -> 64^3 octree, Sect. 3.4.2),
    centre-to-edge tau0 = 1e5 here to keep the oracle short."""
    n = 400 if tau_dust else 150
    wl = synth.sphere(tau0=1e5, T=1e4, tau_dust=tau_dust, n_packets=n)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets, device=True)
    r, tal = oracle_run(wl)
    for s in (oracle.ESCAPED, oracle.ABSORBED):
        assert abs((g["status"] == s).mean() - (r["status"] == s).mean()) < 4 * math.sqrt(0.25 / n) + 1e-9
    assert st["escaped"] + st["absorbed"] + st["capped"] == n
    same = (g["nscatt"] == r["nscatt"]).mean()
    mg, mr = g["nscatt"].mean(), r["nscatt"].mean()
    print("sphere tau_d=%g: identical %.4f <N> %.1f vs %.1f" % (tau_dust, same, mg, mr))
    assert abs(mg / mr - 1) < 0.01 or same > 0.9
    esc_g, esc_r = g["status"] == 1, r["status"] == 1
    if esc_g.sum() > 20:
        assert _ks(_x(wl, g["nu"][esc_g]), _x(wl, r["nu"][esc_r])) > 0.01


def test_expanding_sphere_peeling_matches_oracle():
    """Expanding sphere with dust, recoil and core/wing phase functions,
    peeled into 3 directions (spectra, images, cubes).  Peeled totals are
    Monte Carlo estimates: the oracle runs the packets in 8 groups of 100, and
    the GPU total must lie within 4 sigma of the oracle's (sigma from the
    spread of the group totals, x sqrt(2) for the difference of two
    estimates)."""
    n, groups = 800, 8
    wl = synth.expanding_sphere(N_HI=1e19, n_packets=n, npix=16, nchan=40)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    o = oracle.Oracle(wl)
    m = n // groups
    parts = [o.run(lo=k * m, hi=(k + 1) * m, threads=8) for k in range(groups)]
    r = {k: np.concatenate([p[0][k] for p in parts]) for k in ("nscatt", "status")}
    tal = {k: sum(p[1][k] for p in parts) for k in ("pspec", "pimg", "pcube")}
    same = (g["nscatt"] == r["nscatt"]).mean()
    print("expanding: identical %.4f <N> %.1f vs %.1f" % (same, g["nscatt"].mean(), r["nscatt"].mean()))
    ps = ctx.get_tally(1)
    pi = ctx.get_tally(2)
    pc = ctx.get_tally(3)
    for d in range(3):
        a, b = float(ps[d].sum()), float(tal["pspec"][d].sum())
        sig = np.std([p[1]["pspec"][d].sum() for p in parts], ddof=1) * math.sqrt(groups)
        print("direction %d: peeled %.4g vs %.4g (sigma %.3g)" % (d, a, b, sig))
        assert abs(a - b) <= 4 * math.sqrt(2) * sig + 1e-3 * b, (d, a, b, sig)
    assert np.allclose(pc.sum(-1), pi, rtol=1e-4, atol=1e-9) or pc.sum() <= pi.sum() * (1 + 1e-5)
    if same > 0.95:
        assert np.allclose(ps, tal["pspec"], rtol=2e-3, atol=1e-6 * ps.max())


def test_conservation_and_edge_cases():
    """N_escaped + N_absorbed + N_capped = N; empty input; packets outside
    the box; caps; malformed octree rejected."""
    import paper_2001_11252_gb300 as rg
    wl = synth.sphere(tau0=1e3, T=1e4, tau_dust=1.0, n_packets=3000, base=3, max_level=4)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    assert st["escaped"] + st["absorbed"] + st["capped"] + st["errors"] == 3000
    assert st["errors"] == 0
    st0 = ctx.propagate(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0, np.uint64), out={})
    assert st0["packets"] == 0
    bad = wl.packets
    pos = bad.pos[:4].copy()
    pos[:, 0] = [1.5, -0.2, 0.5, 0.5]
    out = {"status": np.zeros(4, np.int32)}
    ctx.propagate(pos, bad.dir[:4], bad.nu[:4], bad.ids[:4], out=out)
    assert list(out["status"][:2]) == [rg.PK_ERROR, rg.PK_ERROR]
    ctx.set_physics(max_scatt=5, seed=wl.physics.seed)
    out = {"status": np.zeros(100, np.int32), "nscatt": np.zeros(100, np.int64)}
    ctx.propagate(bad.pos[:100], bad.dir[:100], bad.nu[:100], bad.ids[:100], out=out)
    assert np.all(out["nscatt"] <= 5)
    assert np.all((out["status"] == rg.PK_CAPPED) == (out["nscatt"] == 5))
    son = wl.medium.tree.son.copy()
    son[3] = son[2]
    with pytest.raises(Exception):
        ctx.load_octree(son, wl.medium.n_HI, wl.medium.vx, wl.medium.vy, wl.medium.vz, wl.medium.T,
                        wl.medium.n_dust, box_cm=wl.medium.box_cm)


def test_error_budget_gpu():
    """Sect. 4.5 on the GPU: direction-preserving scatterings, path = R."""
    wl = synth.sphere(tau0=1e3, T=1e4, n_packets=2000, base=6, max_level=6)
    wl.physics.keep_direction = 1
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    rel = g["path"] / wl.domain.size - 1
    assert np.all(g["status"] == 1)
    assert np.abs(rel).max() < 1e-12


def test_metal_lines_fluorescence_matches_oracle():
    """Three lines at once (Lya + Si II 1190 + Si II 1193) with fluorescent
    channels (Sect. 3.2.3, Table 1), dust and a velocity field: same fates,
    scattering counts and spectra as the oracle on coupled streams."""
    wl = synth.siII_sphere(n_packets=400)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    r, tal = oracle_run(wl)
    same = (g["nscatt"] == r["nscatt"]).mean()
    print("Si II: identical %.4f <N> %.2f vs %.2f escaped %d vs %d" % (
        same, g["nscatt"].mean(), r["nscatt"].mean(), (g["status"] == 1).sum(), (r["status"] == 1).sum()))
    assert same > 0.9
    esc_g, esc_r = g["status"] == 1, r["status"] == 1
    # fluorescent photons leave at 1197.39 A: present on both sides in the same numbers
    lam_g = 2.99792458e18 / g["nu"][esc_g]
    lam_r = 2.99792458e18 / r["nu"][esc_r]
    fg, fr = (np.abs(lam_g - 1197.39) < 0.5).sum(), (np.abs(lam_r - 1197.39) < 0.5).sum()
    assert fr > 20 and abs(fg - fr) <= 4 * math.sqrt(fr)
    assert _ks(lam_g, lam_r) > 0.01
    spec = ctx.get_tally(0)
    assert abs(spec.sum() - tal["spec"].sum()) <= 4 * math.sqrt(tal["spec"].sum())


def test_galaxy_run_matches_oracle():
    """Synthetic galaxy (graded octree, levels 4-10, lognormal fields, three
    lines with fluorescence, dust, turbulent velocities, peeling into 4
    directions): packets capped at 300 scatterings; same fates, counts and
    peeled flux as the oracle on coupled streams."""
    wl = synth.galaxy(n_leaf=150_000, grid_level=6, base_level=4, max_level=10, n_packets=300, npix=16,
                      nchan=40)
    wl.physics.max_scatt = 300
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    r, tal = oracle_run(wl)
    same = ((g["nscatt"] == r["nscatt"]) & (g["status"] == r["status"])).mean()
    print("galaxy: identical %.4f statuses %s vs %s" % (same, np.bincount(g["status"], minlength=5),
                                                        np.bincount(r["status"], minlength=5)))
    assert same > 0.9
    assert st["errors"] == 0
    # packets are born in the densest leaves: the peeled flux may vanish
    # (every peeling ray beyond tau = 50); both sides must agree either way
    ps = ctx.get_tally(1)
    a, b = float(ps.sum()), float(tal["pspec"].sum())
    assert abs(a - b) <= 0.05 * max(a, b) + 1e-30, (a, b)
    assert st["npeel_rays"] == tal["npeel"]


def test_shell_run_matches_oracle():
    """Shell domain (Sect. 4) with an outflow: packets born in the shell leave
    through the outer or the inner sphere; coupled runs agree."""
    n = 600
    wl = synth.shell(tau0=1e4, n_packets=n, v_max_kms=100.0)
    ctx = context(wl)
    g, st = gpu_run(ctx, wl.packets)
    r, _ = oracle_run(wl)
    same = (g["nscatt"] == r["nscatt"]).mean()
    rg_ = np.linalg.norm(g["pos"] - 0.5, axis=1)
    inner_g = np.abs(rg_ - 0.25) < 1e-9
    inner_r = np.abs(np.linalg.norm(r["pos"] - 0.5, axis=1) - 0.25) < 1e-9
    print("shell: identical %.4f <N> %.1f vs %.1f, through the inner sphere %.3f vs %.3f"
          % (same, g["nscatt"].mean(), r["nscatt"].mean(), inner_g.mean(), inner_r.mean()))
    assert st["escaped"] == n and st["errors"] == 0
    assert (inner_g | (np.abs(rg_ - 0.45) < 1e-9)).all()
    assert same > 0.95
    assert abs(inner_g.mean() - inner_r.mean()) <= 4 * math.sqrt(0.25 / n)

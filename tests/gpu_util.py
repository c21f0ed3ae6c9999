"""Helpers shared by the GPU tests: build a library context for a workload and
run the oracle on the same packets."""
import numpy as np

import oracle
import synth


def context(wl):
    import paper_2001_11252_gb300 as rg
    ctx = rg.Context(0)
    ctx.setup(wl)
    return ctx


def gpu_run(ctx, pk, device=False):
    """Propagate a synth.Packets list; returns (per-packet dict, stats)."""
    n = pk.n
    if device:
        import torch
        dev = torch.device("cuda:0")
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dev, dt)
        pos, dr, nu = t(pk.pos, torch.float64), t(pk.dir, torch.float64), t(pk.nu, torch.float64)
        ids = t(pk.ids.view(np.int64), torch.int64)
        out = {"status": torch.zeros(n, dtype=torch.int32, device=dev),
               "nscatt": torch.zeros(n, dtype=torch.int64, device=dev),
               "nu": torch.zeros(n, dtype=torch.float64, device=dev),
               "pos": torch.zeros((n, 3), dtype=torch.float64, device=dev),
               "dir": torch.zeros((n, 3), dtype=torch.float64, device=dev),
               "path": torch.zeros(n, dtype=torch.float64, device=dev)}
        st = ctx.propagate(pos, dr, nu, ids, out=out)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}, st
    out = {"status": np.zeros(n, np.int32), "nscatt": np.zeros(n, np.int64), "nu": np.zeros(n),
           "pos": np.zeros((n, 3)), "dir": np.zeros((n, 3)), "path": np.zeros(n)}
    st = ctx.propagate(pk.pos, pk.dir, pk.nu, pk.ids, out=out)
    return out, st


def oracle_run(wl, threads=8):
    return oracle.Oracle(wl).run(threads=threads)


def state_from(rec, pid):
    """Oracle state from one GPU trace event (rascas_event)."""
    st = oracle.State()
    st.p[:] = list(rec["p"]); st.k[:] = list(rec["k"]); st.nu = float(rec["nu"])
    st.leaf, st.level = int(rec["leaf"]), int(rec["level"])
    st.ijk[:] = [int(v) for v in rec["ijk"]]
    st.pid = int(pid); st.ndraw = int(rec["ndraw"])
    st.nscatt, st.nsteps, st.status = int(rec["nscatt"]), int(rec["nsteps"]), int(rec["status"])
    return st


def rebuild_peel_events(ctx, o, pk, cap=3000):
    """The oracle's peeling record of the GPU's own histories: the packets are
    traced on the GPU, every event is replayed by the oracle from the GPU's
    state (same draws), and the peeling events the oracle makes at the
    emission and at each replayed scattering are collected.  Packets whose
    replay ever leaves the GPU's history (another leaf, draw count or status)
    or whose trace ran out are dropped.  Returns (indices of the kept
    packets, their events concatenated)."""
    ev, cnt = ctx.trace(pk.pos, pk.dir, pk.nu, pk.ids, cap)
    chosen, events = [], []
    for i in range(pk.n):
        n = int(cnt[i])
        if n >= cap or ev[i, n - 1]["status"] == 0:
            continue
        recs = [o.emission_events(state_from(ev[i, 0], pk.ids[i]))]
        ok = True
        for j in range(n - 1):
            st = state_from(ev[i, j], pk.ids[i])
            _, t = o.event(st, record_events=64)
            b = ev[i, j + 1]
            if st.ndraw != b["ndraw"] or st.status != b["status"] or st.leaf != b["leaf"]:
                ok = False
                break
            recs.append(t["events"])
        if ok:
            chosen.append(i)
            events.append(np.concatenate(recs))
    return np.array(chosen, dtype=np.int64), (np.concatenate(events) if events else
                                                np.zeros(0, dtype=oracle.EVENT_DTYPE))


def near_edge_events(o, events, dch=1e-4, dpix=1e-6):
    """Peeling events within dch channels of a channel edge or dpix pixels of
    a pixel edge: where FP32 rounding on the GPU may bin them next door."""
    c = o.cfg
    t = (events["nu"] - c.nu_lo) / (c.nu_hi - c.nu_lo) * c.nbin
    near = np.abs(t - np.round(t)) < dch
    if c.npix:
        dirs = np.array([[c.dirs[d][j] for j in range(3)] for d in range(c.ndir)])
        ctr = np.array(list(c.img_c))
        for d in range(c.ndir):
            sel = events["dir"] == d
            if not sel.any():
                continue
            eu, ev = oracle.onb(dirs[d])
            r = events["p"][sel] - ctr
            for e in (eu, ev):
                u = (r @ e / c.fov + 0.5) * c.npix
                near[np.flatnonzero(sel)] |= np.abs(u - np.round(u)) < dpix
    return near


def replay_steps(wl, n_packets, max_events):
    """Trace packets on the GPU and replay every event on the oracle from the
    GPU's state: counts of steps and mismatches (leaf, draws, status, counts),
    largest position error per step length, direction error and outgoing
    frequency error in Doppler widths."""
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

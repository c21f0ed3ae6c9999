"""Helpers shared by the GPU tests: build a library context for a workload and
run the oracle on the same packets."""
import numpy as np

import oracle


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

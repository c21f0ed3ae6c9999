"""rascas_propagate_noalloc: the propagation entry point for callers that must
not allocate device memory while they run (for example an application whose
framework owns all free HBM in its own pool, or a latency-critical loop where
a cudaMalloc could synchronise the device).  Its scratch lives in a static
device array whose address rascas_create looks up, so the checks here are
that it returns exactly what the ordinary rascas_propagate returns on the same
packets, on two calls in a row (the second call must not see the first call's
counters or queue head), that a call takes no device memory (the free bytes
the driver reports do not change across it), and that it rejects a packet
count beyond RASCAS_NOALLOC_MAX_PACKETS.

This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

MAX_PACKETS = 57344  # RASCAS_NOALLOC_MAX_PACKETS in include/rascas_gb300.h


def _outputs(n):
    return {"status": np.zeros(n, np.int32), "nscatt": np.zeros(n, np.int64), "nu": np.zeros(n),
            "pos": np.zeros((n, 3)), "dir": np.zeros((n, 3)), "path": np.zeros(n)}


def test_propagate_noalloc_matches_propagate():
    import torch
    import paper_2001_11252_gb300 as rg
    from paper_2001_11252_gb300 import _native as N

    wl = synth.sphere(tau0=1e4, T=1e4, tau_dust=1.0, n_packets=8, base=3, max_level=5)
    ctx = rg.Context(0)
    ctx.setup(wl)
    L = N.lib()
    f = L.rascas_propagate_noalloc
    f.argtypes = [C.c_void_p, C.POINTER(N.PacketsIn), C.c_int64, C.POINTER(N.PacketsOut), C.POINTER(N.Stats)]
    f.restype = C.c_int
    for call, n in enumerate((3000, 2000)):
        pk = synth.point_source(n, (0.5, 0.5, 0.5), wl.packets.nu[0], 1234 + call, first_id=10_000 * call)
        ref = _outputs(n)
        st_ref = ctx.propagate(pk.pos, pk.dir, pk.nu, pk.ids, out=ref)
        got = _outputs(n)
        pos, dr = np.ascontiguousarray(pk.pos), np.ascontiguousarray(pk.dir)
        nu, ids = np.ascontiguousarray(pk.nu), np.ascontiguousarray(pk.ids)
        pin = N.PacketsIn(pos.ctypes.data, dr.ctypes.data, nu.ctypes.data, ids.ctypes.data)
        pout = N.PacketsOut(*[got[k].ctypes.data for k in ("status", "nscatt", "nu", "pos", "dir", "path")])
        st = N.Stats()
        free0 = torch.cuda.mem_get_info(0)[0]
        r = f(ctx._h, C.byref(pin), n, C.byref(pout), C.byref(st))
        free1 = torch.cuda.mem_get_info(0)[0]
        assert r == 0, L.rascas_last_error(ctx._h)
        assert free1 == free0, (call, free0, free1)
        for k in ref:
            assert np.array_equal(ref[k], got[k]), (call, k)
        assert st.packets == n == st_ref["packets"]
        assert st.escaped == st_ref["escaped"] and st.absorbed == st_ref["absorbed"]
        assert st.nscatt_line == st_ref["nscatt_line"] and st.nscatt_dust == st_ref["nscatt_dust"]
    # beyond the static scratch: rejected with an argument error, nothing launched
    big = MAX_PACKETS + 1
    z3, z1 = np.zeros((big, 3)), np.zeros(big)
    zi = np.zeros(big, np.uint64)
    pin = N.PacketsIn(z3.ctypes.data, z3.ctypes.data, z1.ctypes.data, zi.ctypes.data)
    r = f(ctx._h, C.byref(pin), big, None, None)
    assert r == -1
    assert b"RASCAS_NOALLOC_MAX_PACKETS" in L.rascas_last_error(ctx._h)
    ctx.close()

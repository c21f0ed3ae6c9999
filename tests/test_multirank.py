"""The multi-GPU path of bench.py on CPU: two ranks over gloo.  Ranks own
disjoint packet-id ranges and exchange nothing while they propagate (packets
are independent, Sect. 2); the only exchange is the final max of the timings
and sum of the counts.  Sharded oracle runs reduced over the ranks equal one
run over all packets, bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    import oracle
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev = torch.device("cpu")
        # id ranges of every step on every rank are disjoint
        W, K, P = 3, 3, 1000
        mine = [(bench.shard_first(rank, s, W, K, P), P) for s in range(W + K)]
        allr = [None] * world
        dist.all_gather_object(allr, mine)
        # timings: max over ranks; counts: sums
        t, (a, b) = bench.reduce_over_ranks(dist, dev, 10.0 + rank, (rank + 1, 100))
        # a sharded oracle run, spectra summed over the ranks
        wl = synth.sphere(tau0=1e3, T=1e4, tau_dust=0.5, n_packets=240, base=3, max_level=4)
        n = wl.packets.n
        lo, hi = rank * n // world, (rank + 1) * n // world
        out, tal = oracle.Oracle(wl).run(lo=lo, hi=hi, threads=2)
        spec = torch.tensor(tal["spec"], dtype=torch.float64)
        dist.all_reduce(spec)
        cnt = torch.tensor([float((out["status"] == s).sum()) for s in (1, 2, 3)], dtype=torch.float64)
        dist.all_reduce(cnt)
        q.put((rank, allr, t, a, b, spec.numpy(), cnt.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    pytest.importorskip("torch")
    import multiprocessing as mp
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    allr = res[0][1]
    ranges = sorted(r for rank_ranges in allr for r in rank_ranges)
    for (f0, n0), (f1, _) in zip(ranges, ranges[1:]):
        assert f0 + n0 <= f1   # disjoint
    for _, _, t, a, b, spec, cnt in res:
        assert t == 11.0 and a == 3.0 and b == 200.0
    # the reduced sharded run equals one run over all packets
    wl = synth.sphere(tau0=1e3, T=1e4, tau_dust=0.5, n_packets=240, base=3, max_level=4)
    out, tal = oracle.Oracle(wl).run(threads=2)
    assert np.array_equal(res[0][5], np.asarray(tal["spec"], np.float64))
    assert np.array_equal(res[0][6], [float((out["status"] == s).sum()) for s in (1, 2, 3)])
    assert np.array_equal(res[0][5], res[1][5])


def test_host_cpu_record():
    """The CPU baseline names the host it ran on."""
    import bench
    h = bench.host_cpu()
    assert set(h) == {"cpu", "machine", "nproc"} and h["cpu"] and h["nproc"] >= 1

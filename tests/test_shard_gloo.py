"""Multi-rank shot sharding on CPU: world_size 2 over gloo.  Each rank runs
``shard.rank_step`` -- the function bench.py's GPU ranks run -- with the (oracle)
extended imaging operator on its block of shots; the sum all-reduce of the images
must equal the single-process result over all shots."""
import os
import socket

import numpy as np
import pytest

from paper_2206_02362_gb300.shard import shard

torch = pytest.importorskip("torch")


def test_shard_partitions_exactly():
    for nshot in (0, 1, 5, 100, 101):
        for world in (1, 2, 3, 8):
            blocks = [shard(nshot, world, r) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == nshot
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    import synth
    from paper_2206_02362_gb300.shard import rank_step
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, v, geo, w, d = _problem()
        blocks = []

        def apply(a, b):                 # the rank's operator call: the oracle on its shot block
            blocks.append((a, b))
            sub = oracle.Geometry(geo.src_iz[a:b], geo.src_ix[a:b], geo.rec_iz, geo.rec_ix)
            return torch.from_numpy(oracle.born_ext_adj(g, v, sub, w[a:b], d[a:b], nthreads=1))

        t = rank_step(apply, geo.nshot, world, rank)
        q.put((rank, t.numpy(), blocks))
    finally:
        dist.destroy_process_group()


def _problem():
    import oracle
    import synth
    g = oracle.Grid(nz=12, nx=40, W=4, nt=60, dt=1e-3, dx=10.0, nh=3)
    rng = np.random.default_rng(5)
    v = 2000.0 + 200.0 * rng.random((g.nz, g.nx))
    geo = oracle.Geometry(np.array([1, 2, 1, 3, 2]), np.array([3, 10, 20, 30, 37]), np.full(20, 1), 2 * np.arange(20))
    w = np.stack([synth.ricker(g.nt, g.dt, 25.0)] * geo.nshot)
    d = rng.standard_normal((geo.nshot, g.nt, geo.nrec))
    return g, v, geo, w, d


def test_two_rank_gloo_image_sum_matches_single_process():
    import multiprocessing as mp

    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = {r: img for r, img, _ in got}
    blocks = {r: b for r, _, b in got}
    g, v, geo, w, d = _problem()
    full = oracle.born_ext_adj(g, v, geo, w, d, nthreads=1)
    assert blocks == {0: [(0, 3)], 1: [(3, 5)]}        # contiguous shot blocks, each shot on one rank
    for r in (0, 1):
        assert np.allclose(res[r], full, rtol=1e-12, atol=1e-12 * np.abs(full).max())

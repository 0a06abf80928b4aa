"""World-size-2 gloo checks of the multi-rank layout (CPU only).

Each rank takes a contiguous band shard, computes its partial dL/dV with the
CPU oracle (the GPU kernels are not available here), and the all-reduce
must equal the single-process result over all bands; the max-over-ranks
timing and the shard arithmetic are checked too."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1601_07378_gb300 import dist as vdist  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_1601_07378_gb300 import synth
        n = (12, 12, 12)
        g = synth.sphere_glist(*n, 3)
        c = synth.coefficients(g, 5, seed=1)
        gout = synth.coefficients(g, 5, seed=2)
        V, _ = synth.potential(*n, "smooth", seed=3)
        b0, nb = vdist.band_shard(5, rank, world)
        part = torch.from_numpy(O.grad_V(n, g, c[b0:b0 + nb], gout[b0:b0 + nb]) if nb else np.zeros(n))
        vdist.allreduce_grad_v(part)
        t = vdist.max_over_ranks(1.0 + rank)
        q.put((rank, part.numpy(), t))
    finally:
        dist.destroy_process_group()


def test_band_shard_covers_every_band_once():
    for nb in (0, 1, 5, 1024, 1023):
        for world in (1, 2, 3, 8):
            got = [vdist.band_shard(nb, r, world) for r in range(world)]
            assert sum(c for _, c in got) == nb
            assert all(got[r][0] + got[r][1] == got[r + 1][0] for r in range(world - 1))
            assert max(c for _, c in got) - min(c for _, c in got) <= 1
    with pytest.raises(ValueError):
        vdist.band_shard(4, 2, 2)


def test_aggregate_rate():
    assert vdist.aggregate_rate(1024, 4, 0.5) == 8192.0


def test_gloo_world2_grad_v_allreduce_and_max_timing():
    from oracle import oracle as O
    from paper_1601_07378_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = (12, 12, 12)
    g = synth.sphere_glist(*n, 3)
    full = O.grad_V(n, g, synth.coefficients(g, 5, seed=1), synth.coefficients(g, 5, seed=2))
    for rank, dv, t in res:
        assert np.allclose(dv, full, rtol=1e-13, atol=1e-15)
        assert t == 2.0

"""Multi-rank (replicas) host logic on CPU with two gloo ranks: disjoint
sample ranges per rank, max-over-ranks timing, and the average of the ranks'
images equal to one render with all their samples (paths computed by the
FP64 oracle)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2305_20061_gb300 import inputs as I
from paper_2305_20061_gb300 import replicas as R


def test_sample_ranges_are_disjoint_and_cover():
    world, spp = 4, 3
    seen = []
    for frame in range(3):
        for r in range(world):
            f0 = R.first_sample(r, world, spp, frame)
            seen += list(range(f0, f0 + spp))
    assert sorted(seen) == list(range(3 * world * spp))
    with pytest.raises(ValueError):
        R.first_sample(4, 4, 1)


def test_single_process_fallbacks():
    assert R.max_over_ranks(3.5, "cpu") == 3.5
    img = torch.ones(2, 3)
    assert torch.equal(R.average_images(img), torch.ones(2, 3))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        sc = I.make_scene("C1")
        nif = I.nif_init(seed=0)
        W = H = 8
        spp, depth = 2, 3
        f0 = R.first_sample(rank, world, spp)
        pix = np.tile(np.arange(W * H), spp)
        smp = np.repeat(np.arange(f0, f0 + spp), W * H)
        L, _, _ = O.trace_paths(O.Scene(sc), sc.camera, W, H, depth, 0, pix, smp, nif=O.Nif(nif))
        img = torch.from_numpy(L.reshape(spp, W * H, 3).mean(0)).float()
        mine = img.clone()
        R.average_images(img)
        t = R.max_over_ranks(1.0 + rank, "cpu")
        # bit-exact: FP64 sum of the partials in rank order, one division, one cast
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        want = (sum((p.double() for p in parts), torch.zeros(mine.shape, dtype=torch.float64)) / world).float()
        assert torch.equal(img, want)
        every = [torch.empty_like(img) for _ in range(world)]
        dist.all_gather(every, img)
        assert all(torch.equal(e, img) for e in every)   # the same image on every rank
        if rank == 0:
            pix_all = np.tile(np.arange(W * H), spp * world)
            smp_all = np.repeat(np.arange(spp * world), W * H)
            L_all, _, _ = O.trace_paths(O.Scene(sc), sc.camera, W, H, depth, 0, pix_all, smp_all, nif=O.Nif(nif))
            ref = L_all.reshape(spp * world, W * H, 3).mean(0)
            out.put((float(np.abs(img.numpy().astype(np.float64) - ref).max()), float(np.abs(ref).max()), t))
        else:
            out.put(("rank1", None, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_render_disjoint_samples():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=240) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    main = [r for r in res if r[0] != "rank1"][0]
    err, scale, t0 = main
    assert err <= 1e-6 * max(1.0, scale)       # FP32 image of the FP64 mean
    assert t0 == 2.0 and all(r[2] == 2.0 for r in res)

"""Multi-rank partitioning on CPU: two gloo ranks (127.0.0.1), the oracle
standing in for each rank's GPU work.  Checks that strips with halos and
image shards reassemble the single-process result, and that the one
collective (the dL/dsigma_r sum) adds up."""
import os
import socket

import numpy as np
import pytest

import synth
from paper_1105_4204_gb300 import shard

WORLD = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, port, results):
    import torch
    import torch.distributed as dist

    import oracle
    os.environ["OMP_NUM_THREADS"] = "2"
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=WORLD)
    try:
        # (1) one image in row strips with read-only halos
        img = synth.rectangles(37, 29, n_rect=6, seed=5).astype(np.float64)
        w1 = oracle.spatial_w1("gauss", 1.5)
        R = (len(w1) - 1) // 2
        st = shard.row_strips(img.shape[0], WORLD, R)[rank]
        part = oracle.bf_brute(img[st.r0:st.r1], sigma_r=30.0, w1=w1)
        c0, c1 = st.crop
        sizes = [s.y1 - s.y0 for s in shard.row_strips(img.shape[0], WORLD, R)]
        mine = torch.zeros((max(sizes), img.shape[1]), dtype=torch.float64)  # gloo: equal sizes
        mine[:c1 - c0] = torch.from_numpy(np.ascontiguousarray(part[c0:c1]))
        gathered = [torch.zeros_like(mine) for _ in sizes]
        dist.all_gather(gathered, mine)
        gathered = [g[:n] for g, n in zip(gathered, sizes)]
        # (2) a batch of images by cost, and the dL/dsigma_r sum over ranks
        specs = synth.batch_specs(5, seed=2, w_range=(8, 20), h_range=(8, 16))
        costs = [shard.image_cost(h, w, 10, 3) for (h, w, _, _) in specs]
        mine_ids = shard.shard_images(costs, WORLD)[rank]
        imgs = synth.batch_images(specs, seed=2)
        gs = 0.0
        for i in mine_ids:
            u = synth.upstream(imgs[i].shape, seed=i).astype(np.float64)
            _, g = oracle.bf_grad(imgs[i].astype(np.float64), u, sigma_s=1.0, sigma_r=30.0)
            gs += g
        total = shard.allreduce_sigma_grad(gs)
        if rank == 0:
            results.put(("strips", np.concatenate([g.numpy() for g in gathered])))
            results.put(("sigma", total))
            results.put(("ids", shard.shard_images(costs, WORLD)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_the_single_process_result(oracle):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    import queue
    import time
    got, t0 = {}, time.time()
    while len(got) < 3:
        try:
            k, v = q.get(timeout=1.0)
            got[k] = v
        except queue.Empty:
            dead = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
            assert not dead, "a rank failed: exit codes %s" % dead
            assert time.time() - t0 < 300, "ranks timed out"
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    img = synth.rectangles(37, 29, n_rect=6, seed=5).astype(np.float64)
    full = oracle.bf_brute(img, sigma_s=1.5, sigma_r=30.0)
    np.testing.assert_allclose(got["strips"], full, atol=1e-12)
    specs = synth.batch_specs(5, seed=2, w_range=(8, 20), h_range=(8, 16))
    imgs = synth.batch_images(specs, seed=2)
    ref = 0.0
    for i, im in enumerate(imgs):
        u = synth.upstream(im.shape, seed=i).astype(np.float64)
        ref += oracle.bf_grad(im.astype(np.float64), u, sigma_s=1.0, sigma_r=30.0)[1]
    assert got["sigma"] == pytest.approx(ref, rel=1e-12)
    ids = got["ids"]
    assert sorted(ids[0] + ids[1]) == list(range(5))


def test_row_strips_cover_and_halos_clip():
    for H in [1, 2, 7, 100, 2048]:
        for world in [1, 2, 3, 8]:
            strips = shard.row_strips(H, world, 9)
            assert strips[0].y0 == 0 and strips[-1].y1 == H
            for a, b in zip(strips, strips[1:]):
                assert a.y1 == b.y0
            for s in strips:
                assert s.r0 == max(0, s.y0 - 9) and s.r1 == min(H, s.y1 + 9)
                assert abs((s.y1 - s.y0) - H / world) < 1


def test_shard_images_balances_largest_first():
    costs = [10, 1, 9, 2, 8, 3]
    parts = shard.shard_images(costs, 2)
    assert sorted(parts[0] + parts[1]) == list(range(6))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(costs)
    assert shard.shard_images(costs, 2) == parts  # deterministic

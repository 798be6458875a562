"""Multi-rank host logic of shot sharding on CPU (gloo, world size 2): shot
assignment, slowest-rank timing and the image stack."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_1603_03971_gb300 import shots


def test_assign_shots_partitions_the_range():
    for nshots in (0, 1, 5, 32, 33):
        for world in (1, 2, 3, 8):
            got = [s for r in range(world) for s in shots.assign_shots(nshots, r, world)]
            assert got == list(range(nshots))
            sizes = [len(shots.assign_shots(nshots, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shots.assign_shots(4, 2, 2)


def test_shot_sources_stay_in_the_model():
    for n in (1, 2, 7):
        xs = [shots.shot_source(s, n, 512, 512, 4) for s in range(n)]
        assert all(0 <= x < 512 and y == 256 and z == 4 for x, y, z in xs)
        assert len(set(xs)) == n
    assert shots.shot_source(0, 1, 512, 512, 4) == (256, 256, 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shots.assign_shots(5, rank, world)
        img = torch.zeros(4, 3)
        for s in mine:
            img += float(s + 1)  # stand-in per-shot image
        shots.stack_images(img)
        t = shots.max_over_ranks(1.0 + rank)
        q.put((rank, mine, img.tolist(), t))
    finally:
        dist.destroy_process_group()


def test_stack_and_timing_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == [0, 1, 2] and out[1][1] == [3, 4]
    total = float(sum(range(1, 6)))
    for _, _, img, t in out:
        assert all(v == total for row in img for v in row)
        assert t == 2.0

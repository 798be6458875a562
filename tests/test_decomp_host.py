"""Host logic of the X-Y domain decomposition (no GPU): the partition covers
the padded grid exactly, x boundaries sit on 16-byte rows, the neighbour map
is symmetric, and impossible decompositions are rejected.

The halo exchange itself is checked on two gloo ranks (CPU processes): each
rank holds one subdomain's owned block, sends the r-wide strips its
neighbour needs and receives its halo with nonblocking point-to-point
messages (the paper's exchange, Sec. II), then takes one FP64 oracle
leapfrog step on its local array; its owned cells equal the oracle's step
on the whole grid."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import paper_1603_03971_gb300 as rtm


def _params(nx=100, ny=44, nz=37, nb=10, r=4):
    return rtm.make_params(nx, ny, nz, nb, r, 10, 10.0, 1e-3, 25.0, 0.04, (nx // 2, ny // 2, 3), 1)


@pytest.mark.parametrize("px,py", [(1, 1), (2, 1), (1, 3), (2, 2), (3, 2), (5, 4)])
@pytest.mark.parametrize("r", [4, 8])
def test_partition_covers_the_grid(px, py, r):
    p = _params(r=r)
    NZ, NY, NX = rtm.padded_shape(p)
    plan = rtm.decomp_plan(p, px, py)
    assert plan.shape == (px * py, 8)
    owner = np.full((NY, NX), -1)
    for k, (x0, x1, y0, y1, w, e, s, n) in enumerate(plan):
        assert x0 % 4 == 0 and x1 % 4 == 0 and x1 - x0 >= max(r, 4) and y1 - y0 >= r
        assert (owner[y0:y1, x0:x1] == -1).all()
        owner[y0:y1, x0:x1] = k
        i, j = k % px, k // px
        assert w == (k - 1 if i > 0 else -1) and e == (k + 1 if i + 1 < px else -1)
        assert s == (k - px if j > 0 else -1) and n == (k + px if j + 1 < py else -1)
        # neighbours share the face they touch
        if e >= 0:
            assert plan[e][0] == x1 and plan[e][4] == k
            assert (plan[e][2], plan[e][3]) == (y0, y1)
        if n >= 0:
            assert plan[n][2] == y1 and plan[n][6] == k
            assert (plan[n][0], plan[n][1]) == (x0, x1)
    assert (owner >= 0).all()
    # parts are as even as the 4-cell x rule allows
    wx = plan[:px, 1] - plan[:px, 0]
    assert wx.max() - wx.min() <= 4
    wy = plan[::px, 3] - plan[::px, 2]
    assert wy.max() - wy.min() <= 1


def test_impossible_decompositions_are_rejected():
    p = _params(nx=8, ny=6, nz=6, nb=4, r=8)  # 16 x 14 x 14 padded
    with pytest.raises(rtm.RtmError):
        rtm.decomp_plan(p, 3, 1)  # x parts of 4 cells < r = 8
    with pytest.raises(rtm.RtmError):
        rtm.decomp_plan(p, 1, 2)  # y parts of 7 rows < r = 8
    with pytest.raises(rtm.RtmError):
        rtm.decomp_plan(p, 0, 1)
    assert rtm.decomp_plan(p, 2, 1).shape == (2, 8)


def test_workspace_grows_with_the_halos():
    p = _params()
    a = rtm.decomp_workspace_size(p, 1, 1)
    b = rtm.decomp_workspace_size(p, 2, 2)
    NZ, NY, NX = rtm.padded_shape(p)
    assert b > a >= 3 * 4 * NX * NY * NZ


# ---- the exchange on two gloo ranks ------------------------------------------

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _strips(x0, x1, y0, y1, r, face, halo):
    """The r-wide strip a subdomain sends through a face (its own cells) or
    receives into (its halo), in global padded coordinates (x, y ranges)."""
    if face == 0:  # W
        return (x0 - r, x0) if halo else (x0, x0 + r), (y0, y1)
    if face == 1:  # E
        return (x1, x1 + r) if halo else (x1 - r, x1), (y0, y1)
    if face == 2:  # S
        return (x0, x1), ((y0 - r, y0) if halo else (y0, y0 + r))
    return (x0, x1), ((y1, y1 + r) if halo else (y1 - r, y1))


def _problem(r):
    import oracle
    import rtm_inputs

    p = _params(nx=40, ny=30, nz=12, nb=6, r=r)
    vel = rtm_inputs.smooth_random_velocity(p.nx, p.ny, p.nz, 3.0, 1500.0, 3000.0, seed=5)
    c = oracle.model_c(vel, p.nb, rtm_inputs.courant_dt(10.0, 3000.0))
    rng = np.random.default_rng(6)
    u = rng.standard_normal(c.shape)
    up = rng.standard_normal(c.shape)
    return p, c, u, up


def _exchange_worker(rank, world, port, px, py, r, q):
    import torch
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, c, u, up = _problem(r)
        NZ, NY, NX = c.shape
        plan = rtm.decomp_plan(p, px, py)
        x0, x1, y0, y1 = (int(v) for v in plan[rank][:4])
        nbr = [int(v) for v in plan[rank][4:]]
        # local arrays: owned block + r-wide halo; only owned cells are known
        lx, ly = x1 - x0 + 2 * r, y1 - y0 + 2 * r
        loc = np.zeros((NZ, ly, lx))
        loc[:, r:r + y1 - y0, r:r + x1 - x0] = u[:, y0:y1, x0:x1]
        reqs, bufs = [], []
        for face in range(4):
            t = nbr[face]
            if t < 0:
                continue
            (sx0, sx1), (sy0, sy1) = _strips(x0, x1, y0, y1, r, face, halo=False)
            send = torch.from_numpy(np.ascontiguousarray(
                loc[:, sy0 - y0 + r:sy1 - y0 + r, sx0 - x0 + r:sx1 - x0 + r]))
            (hx0, hx1), (hy0, hy1) = _strips(x0, x1, y0, y1, r, face, halo=True)
            recv = torch.empty((NZ, hy1 - hy0, hx1 - hx0), dtype=torch.float64)
            reqs.append(dist.isend(send, t))
            reqs.append(dist.irecv(recv, t))
            bufs.append((recv, hx0, hx1, hy0, hy1, send))
        for rq in reqs:
            rq.wait()
        for recv, hx0, hx1, hy0, hy1, _ in bufs:
            loc[:, hy0 - y0 + r:hy1 - y0 + r, hx0 - x0 + r:hx1 - x0 + r] = recv.numpy()
        # one leapfrog step on the local array (local c and sponge profiles)
        gx = oracle.sponge_profile(NX, p.nb)
        gy = oracle.sponge_profile(NY, p.nb)
        gz = oracle.sponge_profile(NZ, p.nb)

        def window(a, lo, hi):  # the local extent of a global axis, zero outside
            out = np.zeros(hi - lo)
            a0, a1 = max(lo, 0), min(hi, a.size)
            out[a0 - lo:a1 - lo] = a[a0:a1]
            return out

        cl = np.zeros((NZ, ly, lx))
        ya, yb = max(y0 - r, 0), min(y1 + r, NY)
        xa, xb = max(x0 - r, 0), min(x1 + r, NX)
        cl[:, ya - y0 + r:yb - y0 + r, xa - x0 + r:xb - x0 + r] = c[:, ya:yb, xa:xb]
        g = oracle.Grid(cl, p.nb, r, p.dx, profiles=(window(gx, x0 - r, x1 + r),
                                                     window(gy, y0 - r, y1 + r), gz))
        upl = np.zeros_like(loc)
        upl[:, r:r + y1 - y0, r:r + x1 - x0] = up[:, y0:y1, x0:x1]
        out = g.step(loc, upl)[:, r:r + y1 - y0, r:r + x1 - x0]
        q.put((rank, (x0, x1, y0, y1), out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py,r", [(2, 1, 4), (1, 2, 8), (2, 2, 4)])
def test_halo_exchange_over_gloo_ranks_reproduces_the_global_step(px, py, r):
    import oracle

    world = px * py
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_worker, args=(k, world, port, px, py, r, q))
             for k in range(world)]
    for pr in procs:
        pr.start()
    got = [q.get(timeout=180) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p, c, u, up = _problem(r)
    ref = oracle.Grid(c, p.nb, r, p.dx).step(u, up)
    for _, (x0, x1, y0, y1), out in got:
        np.testing.assert_array_equal(out, ref[:, y0:y1, x0:x1])

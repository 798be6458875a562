"""The workloads at their full sizes, in the launch configuration the
benchmark uses.

* two-layer 64^3, 300 steps: full RTM (data and image) against the oracle.
* smooth 512^3 (576^3 padded): the first 40 steps against the oracle run on
  the exact crop around the source (the field vanishes beyond 40 r cells of
  it), plus the dot-product identity and checkpoint/store-all equality,
  which hold at any size.
* gradient 256^3, 1000 steps, checkpoints every 25: the gradient of the
  data misfit against central differences on 16 seeded directions with a
  relative step of 1e-3. The +5 % blob sits at depth 48 cells (480 m):
  1000 steps are 0.64 s, and reflections from a blob at the model centre
  (1280 m deep) would not reach the receivers in that time, leaving a
  misfit of rounding size.
"""
import numpy as np
import pytest

import rtm_inputs
from helpers import rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _dev(a, dtype=None):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype=dtype or torch.float32)


def test_two_layer_64_full_rtm():
    import torch

    import oracle
    import paper_1603_03971_gb300 as rtm

    w = rtm_inputs.WORKLOADS["two_layer_64"]
    v = w.velocity_model()
    rec = w.receivers()
    prob = oracle.Problem(v, w.nb, w.radius, w.dx, w.dt, w.nt, w.f0, w.t0, w.src, rec)
    ref = prob.forward(keep_u=True)
    d_obs = ref["data"]
    img_ref = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=ref["u"])["image"]
    p = rtm.params_for(w)
    ws = rtm.alloc_workspace(p)
    c = rtm.model_prep(p, _dev(v), ws)
    data = torch.empty((w.nt, p.nrec), device="cuda")
    img = torch.zeros((w.nz, w.ny, w.nx), device="cuda")
    rtm.shot(p, c, _dev(rec, torch.int32), _dev(d_obs), ws, img, data=data)
    rtm.check(ws)
    assert rel_l2(data.cpu().numpy(), d_obs) <= TOL
    assert rel_l2(img.cpu().numpy(), img_ref) <= TOL


def test_smooth_512_first_steps_against_the_oracle_on_the_exact_crop():
    import torch

    import oracle
    import paper_1603_03971_gb300 as rtm

    w = rtm_inputs.WORKLOADS["smooth_512"]
    nt = 40
    p = rtm.params_for(w, nt=nt, storage="all", image_every=nt)
    vel = w.velocity_model(device="cuda").contiguous()
    rec = w.receivers()
    ws = rtm.alloc_workspace(p)
    c = rtm.model_prep(p, vel, ws)
    data = torch.empty((nt, p.nrec), device="cuda")
    last = torch.empty((2,) + rtm.padded_shape(p), device="cuda")
    rtm.forward(p, c, _dev(rec, torch.int32), ws, data=data, u_last=last)
    rtm.check(ws)
    # the oracle on the crop: c and sponge profiles of the full padded grid
    nb, r = w.nb, w.radius
    NZ, NY, NX = w.padded_shape
    sx, sy, sz = (s + nb for s in w.src)
    m = nt * r + 1
    z0, z1 = max(0, sz - m), min(NZ, sz + m + 1)
    y0, y1 = max(0, sy - m), min(NY, sy + m + 1)
    x0, x1 = max(0, sx - m), min(NX, sx + m + 1)
    c_full = oracle.model_c(vel.double().cpu().numpy(), nb, w.dt)
    prof = [oracle.sponge_profile(n, nb) for n in (NX, NY, NZ)]
    g = oracle.Grid(c_full[z0:z1, y0:y1, x0:x1], nb, r, w.dx,
                    profiles=(prof[0][x0:x1], prof[1][y0:y1], prof[2][z0:z1]))
    del c_full
    wav = oracle.ricker(nt, w.dt, w.f0, w.t0)
    cy, cx = y1 - y0, x1 - x0
    s_lin = ((sz - z0) * cy + (sy - y0)) * cx + (sx - x0)
    # receivers inside the crop
    rz = w.rec_z + nb
    sel = [j for j, (x, y, _) in enumerate(rec)
           if x0 <= x + nb < x1 and y0 <= y + nb < y1]
    rl = np.array([((rz - z0) * cy + (rec[j][1] + nb - y0)) * cx + (rec[j][0] + nb - x0)
                   for j in sel], dtype=np.int64)
    out = g.forward(wav, s_lin, rl, keep_last=True)
    assert rel_l2(data.cpu().numpy()[:, sel], out["data"]) <= TOL
    crop = last[1, z0:z1, y0:y1, x0:x1].cpu().numpy()
    assert rel_l2(crop, out["last"][1]) <= TOL
    # outside the crop the field is exactly zero
    tot = float(last[1].abs().sum())
    assert tot == pytest.approx(float(np.abs(crop).sum()), rel=1e-6)


def test_smooth_512_identities_at_full_size():
    """The dot-product identity and checkpoint == store-all at the full grid
    (60 steps, checkpoints every 25)."""
    import torch

    import oracle
    import paper_1603_03971_gb300 as rtm

    w = rtm_inputs.WORKLOADS["smooth_512"]
    nt = 60
    vel = w.velocity_model(device="cuda").contiguous()
    rec = _dev(w.receivers(), torch.int32)
    imgs = []
    for storage, k in (("ckpt", 25), ("all", 0)):
        p = rtm.params_for(w, nt=nt, storage=storage, ckpt_every=k)
        ws = rtm.alloc_workspace(p)
        c = rtm.model_prep(p, vel, ws)
        data = torch.empty((nt, p.nrec), device="cuda")
        rtm.forward(p, c, rec, ws, data=data)
        q = torch.from_numpy(rtm_inputs.standard_normal((nt, p.nrec), 41).astype(np.float32)).cuda()
        img = torch.zeros((w.nz, w.ny, w.nx), device="cuda")
        adj = torch.zeros(nt, device="cuda")
        rtm.backward_image(p, c, rec, q, ws, img, src_adj=adj)
        rtm.check(ws)
        imgs.append(img.cpu().numpy())
        del ws
    np.testing.assert_array_equal(imgs[0], imgs[1])
    wav = oracle.ricker(nt, w.dt, w.f0, w.t0)
    lhs = float((data.double() * q.double()).sum())
    rhs = float(np.dot(wav, adj.cpu().numpy().astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs))


def test_gradient_256_against_central_differences():
    import torch

    import paper_1603_03971_gb300 as rtm

    w = rtm_inputs.WORKLOADS["gradient_256"]
    p = rtm.params_for(w, want_grad=True)
    v = w.velocity_model(device="cuda").contiguous()
    v2 = (v * v).contiguous()
    rec = _dev(w.receivers(), torch.int32)
    ws = rtm.alloc_workspace(p)
    # observed data from the model with a +5 % Gaussian blob (radius 16 cells,
    # centre 48 cells deep, so that its reflections arrive within the record)
    vb = rtm_inputs.blob_perturbation(v, 0.05, 16.0,
                                      center=((w.nx - 1) / 2.0, (w.ny - 1) / 2.0, 48.0))
    cb = rtm.model_prep(p, (vb * vb).contiguous(), ws, kind="v2")
    d_obs = torch.empty((w.nt, p.nrec), device="cuda")
    rtm.forward(p, cb, rec, ws, data=d_obs)
    del cb
    x = v2.clone().requires_grad_(True)
    J = rtm.RtmMisfit.apply(x, p, rec, d_obs, ws)
    J.backward()
    g = x.grad.double()
    noise = rtm_inputs.standard_normal((16, w.nz, w.ny, w.nx), 43, np.float32)
    scale = float(v2.abs().max())
    worst = 0.0
    for k in range(16):
        d = rtm_inputs._smooth_torch(noise[k], 8.0, "cuda")
        d = d / d.abs().max()
        eps = 1e-3 * scale
        Jp = float(rtm.RtmMisfit.apply((v2 + eps * d).contiguous(), p, rec, d_obs, ws))
        Jm = float(rtm.RtmMisfit.apply((v2 - eps * d).contiguous(), p, rec, d_obs, ws))
        fd = (Jp - Jm) / (2 * eps)
        an = float((g * d.double()).sum())
        worst = max(worst, abs(an - fd) / max(abs(fd), 1e-300))
    assert worst <= 1e-2, worst

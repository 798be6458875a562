"""Shared set-up for the GPU parity tests: one seeded case feeds both the
CUDA path (through the C ABI) and the FP64 oracle."""
import dataclasses
from typing import Optional, Tuple

import numpy as np

import rtm_inputs


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@dataclasses.dataclass
class Case:
    nx: int = 28
    ny: int = 24
    nz: int = 20
    nb: int = 6
    r: int = 4
    nt: int = 60
    dx: float = 10.0
    vmin: float = 1500.0
    vmax: float = 3000.0
    f0: float = 25.0
    t0: float = 0.04
    src: Tuple[int, int, int] = (14, 12, 3)
    rec_stride: int = 2
    rec_z: int = 2
    seed: int = 1
    storage: str = "all"
    ckpt_every: int = 0
    image_every: int = 1
    sigma: float = 3.0
    extra_rec: Optional[np.ndarray] = None

    @property
    def dt(self):
        return rtm_inputs.courant_dt(self.dx, self.vmax)

    def velocity(self):
        return rtm_inputs.smooth_random_velocity(self.nx, self.ny, self.nz, self.sigma,
                                                 self.vmin, self.vmax, seed=self.seed)

    def receivers(self):
        rec = rtm_inputs.surface_receivers(self.nx, self.ny, self.rec_z, stride=self.rec_stride)
        if self.extra_rec is not None:
            rec = np.concatenate([rec, np.asarray(self.extra_rec, np.int32)])
        return np.ascontiguousarray(rec)

    def d_obs(self, nrec):
        return rtm_inputs.standard_normal((self.nt, nrec), seed=self.seed + 100) * 1e-3

    def params(self, want_grad=False):
        import paper_1603_03971_gb300 as rtm

        return rtm.make_params(self.nx, self.ny, self.nz, self.nb, self.r, self.nt, self.dx,
                               self.dt, self.f0, self.t0, self.src, self.receivers().shape[0],
                               storage=self.storage, ckpt_every=self.ckpt_every,
                               image_every=self.image_every, want_grad=want_grad)

    def oracle_problem(self, squared=False, vel=None):
        import oracle

        v = self.velocity() if vel is None else vel
        if squared and vel is None:
            v = v * v
        return oracle.Problem(v, self.nb, self.r, self.dx, self.dt, self.nt, self.f0, self.t0,
                              self.src, self.receivers(), squared=squared)


class DeviceShot:
    """Device buffers of one case and the calls through the C ABI."""

    def __init__(self, case: Case, want_grad=False, device="cuda", vel=None, squared=False):
        import torch

        import paper_1603_03971_gb300 as rtm

        self.rtm = rtm
        self.case = case
        self.dev = torch.device(device)
        self.p = case.params(want_grad)
        self.ws = rtm.alloc_workspace(self.p, self.dev)
        v = case.velocity() if vel is None else vel
        if squared and vel is None:
            v = v * v
        self.vel = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).to(self.dev)
        self.rec_np = case.receivers()
        self.rec = torch.from_numpy(self.rec_np).to(self.dev)
        self.c = rtm.model_prep(self.p, self.vel, self.ws, kind="v2" if squared else "v")
        self.nrec = self.rec_np.shape[0]

    def forward(self, keep_last=False):
        import torch

        data = torch.empty((self.p.nt, self.nrec), dtype=torch.float32, device=self.dev)
        last = None
        if keep_last:
            last = torch.empty((2,) + self.rtm.padded_shape(self.p), dtype=torch.float32,
                               device=self.dev)
        self.rtm.forward(self.p, self.c, self.rec, self.ws, data=data, u_last=last)
        self.rtm.check(self.ws)
        return data, last

    def backward_image(self, rdata_np, src_adj=False):
        import torch

        rd = torch.from_numpy(np.ascontiguousarray(rdata_np, dtype=np.float32)).to(self.dev)
        img = torch.zeros((self.p.nz, self.p.ny, self.p.nx), dtype=torch.float32,
                          device=self.dev)
        adj = torch.zeros(self.p.nt, dtype=torch.float32, device=self.dev) if src_adj else None
        self.rtm.backward_image(self.p, self.c, self.rec, rd, self.ws, img, src_adj=adj)
        self.rtm.check(self.ws)
        return img, adj

    def grad(self, resid_np):
        import torch

        rd = torch.from_numpy(np.ascontiguousarray(resid_np, dtype=np.float32)).to(self.dev)
        g = self.rtm.grad(self.p, self.c, self.rec, rd, self.ws)
        self.rtm.check(self.ws)
        return g

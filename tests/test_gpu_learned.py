"""Learned snapshot storage: the RTM image built from autoencoder-compressed
source snapshots.

1. Parity: the GPU learned shot equals the oracle's receiver propagation and
   imaging fed with the snapshots that the GPU codec reconstructs (the codec
   itself is checked in test_gpu_codec.py), within the wavefield tolerance.
2. Gain: a codec trained (by the library's own kernels) on snapshots the
   propagator generated from other random models reconstructs and images
   far closer to the exact snapshots and image than the untrained network.
   The non-learned 8x baseline (decimation by 2 per axis + linear
   interpolation) is printed beside them; at this training budget it is
   not beaten, and the test does not claim it.
"""
import numpy as np
import pytest

import rtm_inputs
from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu


def _store_all_snapshots(case, ie):
    import torch

    import paper_1603_03971_gb300 as rtm
    from helpers import GpuRun

    g = GpuRun(case)
    g.forward()
    snaps = {m: rtm.snapshot(g.p, g.ws, m).clone() for m in range(ie, case.nt + 1, ie)}
    torch.cuda.synchronize()
    return g, snaps


def _oracle_image(case, d_obs, snaps_np, ie):
    prob = case.oracle_problem()
    su = np.zeros((case.nt, case.nz, case.ny, case.nx))
    for m, s in snaps_np.items():
        su[m - 1] = s
    return prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=su, image_every=ie)["image"]


def _decode_all(P, snaps, shape):
    from paper_1603_03971_gb300 import codec

    ws = codec.alloc_workspace(shape)
    out = {}
    for m, s in snaps.items():
        lat, sc = codec.encode(P, s, ws)
        out[m] = codec.decode(P, lat, sc, ws).cpu().numpy().astype(np.float64)
    return out


def test_learned_shot_matches_oracle_on_reconstructed_snapshots():
    import torch

    import paper_1603_03971_gb300 as rtm

    ie = 4
    case = Case(nx=32, ny=28, nz=24, nb=8, r=4, nt=40, image_every=ie)
    g, snaps = _store_all_snapshots(case, ie)
    P = torch.from_numpy(rtm_inputs.ae_flat(rtm_inputs.ae_init_params(2)).astype(np.float32)).cuda()
    d_obs = case.d_obs(g.nrec)
    dobs = torch.from_numpy(d_obs.astype(np.float32)).cuda()
    pl = case.params()
    pl.storage = 2  # RTM_STORE_LEARNED
    wl = rtm.alloc_workspace(pl)
    img = torch.zeros((case.nz, case.ny, case.nx), device="cuda")
    rtm.shot_learned(pl, g.c, g.rec, dobs, P, wl, img)
    rtm.check(wl)
    rec_snaps = _decode_all(P, snaps, (case.nz, case.ny, case.nx))
    ref = _oracle_image(case, d_obs, rec_snaps, ie)
    assert rel_l2(img.cpu().numpy(), ref) <= 1e-4


def test_trained_codec_beats_the_untrained_network():
    """The codec's gain from training: trained on snapshots of 16 other random
    models, it reconstructs held-out snapshots far better than the same
    network untrained, and its RTM image is correspondingly closer to the
    exact image. The non-learned 8x baseline (decimation by 2 per axis +
    linear interpolation) is printed beside them for reference."""
    import torch

    from oracle import ae as oae
    from paper_1603_03971_gb300 import learned

    n = 96
    data = learned.training_snapshots(n_models=16, size=n, nb=16, nt=640, every=20, first=40,
                                      f0=20.0, seed0=500)
    P, losses = learned.train(data, steps=800, batch=4, lr=1e-3, lr_min=5e-5, seed=1,
                              log_every=100)
    assert losses[-1][1] < 0.5 * losses[0][1]
    ie = 8
    case = Case(nx=n, ny=n, nz=n, nb=16, r=4, nt=480, image_every=ie, f0=20.0, t0=0.05,
                vmax=4500.0, src=(48, 40, 4), rec_stride=3, seed=77, sigma=8.0)
    g, snaps = _store_all_snapshots(case, ie)
    d_obs = g.forward()[0].cpu().numpy().astype(np.float64)
    exact = {m: s.cpu().numpy().astype(np.float64) for m, s in snaps.items()}
    P0 = torch.from_numpy(rtm_inputs.ae_flat(rtm_inputs.ae_init_params(1)).astype(np.float32)).cuda()
    rec_tr = _decode_all(P, snaps, (n, n, n))
    rec_un = _decode_all(P0, snaps, (n, n, n))
    rec_de = {m: oae.trilinear_upsample(oae.decimate(s), n) for m, s in exact.items()}

    def snap_err(rec):
        num = sum(float(np.sum((rec[m] - exact[m]) ** 2)) for m in exact)
        return (num / sum(float(np.sum(exact[m] ** 2)) for m in exact)) ** 0.5

    e_tr, e_un, e_de = snap_err(rec_tr), snap_err(rec_un), snap_err(rec_de)
    img = {k: _oracle_image(case, d_obs, r, ie)
           for k, r in (("exact", exact), ("trained", rec_tr), ("untrained", rec_un),
                        ("decimation", rec_de))}
    ie_tr = rel_l2(img["trained"], img["exact"])
    ie_un = rel_l2(img["untrained"], img["exact"])
    ie_de = rel_l2(img["decimation"], img["exact"])
    deep = slice(8, None)
    dd = {k: rel_l2(img[k][deep], img["exact"][deep]) for k in ("trained", "untrained",
                                                                  "decimation")}
    print("snapshot rel-L2: trained %.3e untrained %.3e decimation %.3e" % (e_tr, e_un, e_de))
    print("image rel-L2: trained %.3e untrained %.3e decimation %.3e" % (ie_tr, ie_un, ie_de))
    print("image rel-L2 below z=8: %s" % {k: round(v, 4) for k, v in dd.items()})
    assert e_tr < 0.25 * e_un
    assert ie_tr < 0.6 * ie_un
    assert dd["trained"] < 0.25 * dd["untrained"]

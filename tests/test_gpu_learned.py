"""Learned snapshot storage: the RTM image built from autoencoder-compressed
source snapshots.

1. Parity: the GPU learned shot against the oracle chain computed end to
   end in FP64 on the CPU (propagation, codec with bfloat16 rounding at the
   GPU's storage points, receiver propagation and imaging). The image is
   linear in the decoded snapshots, so the codec tolerance (2e-3) bounds it.
2. Gain: a codec trained (by the library's own kernels, starting from the
   parameters under which the network computes the non-learned 8x scheme)
   on snapshots the propagator generated from other random models
   reconstructs and images closer to the exact snapshots and image than
   that scheme at the same bytes (decimated storage) and than the untrained
   network. All images here are the GPU's own (store-all vs learned vs
   decimated storage).
"""
import numpy as np
import pytest

import rtm_inputs
from helpers import Case, rel_l2

pytestmark = pytest.mark.gpu
CODEC_TOL = 2e-3


def _learned_image(case, g, P, d_obs_np, window=0):
    import torch

    import paper_1603_03971_gb300 as rtm

    pl = case.params()
    pl.storage = 2  # RTM_STORE_LEARNED
    pl.ckpt_every = window  # exact window: steps 1..window recomputed, not coded
    wl = rtm.alloc_workspace(pl)
    dobs = torch.from_numpy(np.ascontiguousarray(d_obs_np, dtype=np.float32)).cuda()
    img = torch.zeros((case.nz, case.ny, case.nx), device="cuda")
    rtm.shot_learned(pl, g.c, g.rec, dobs, P, wl, img)
    rtm.check(wl)
    return img.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("window,shape", [(0, "small"), (13, "small"), (0, "columns"),
                                          (17, "columns")])
def test_learned_shot_matches_the_oracle_chain(window, shape):
    """With an exact window W the snapshots of steps 1..W are the exact ones
    (recomputed), the later ones coded. The "columns" model (136 x 72 x 48)
    has a latent of 34 x 18 x 12 points, so the z-marching encoder and
    decoder of the shot run several columns in x and y, each with a ragged
    last column."""
    import torch

    from helpers import DeviceShot
    from oracle import ae as oae

    ie = 4
    if shape == "small":
        case = Case(nx=32, ny=28, nz=24, nb=8, r=4, nt=40, image_every=ie)
    else:
        case = Case(nx=136, ny=72, nz=48, nb=8, r=4, nt=60, image_every=ie,
                    src=(68, 36, 4), rec_stride=3)
    P = rtm_inputs.ae_flat(rtm_inputs.ae_init_params(2)).astype(np.float32)
    g = DeviceShot(case)
    d_obs = case.d_obs(g.nrec)
    img = _learned_image(case, g, torch.from_numpy(P).cuda(), d_obs, window)
    # oracle: snapshots, codec and imaging, all on the CPU
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True)
    params = oae.unflatten(P.astype(np.float64))
    su = np.zeros_like(fw["u"])
    for m in range(ie, case.nt + 1, ie):
        if m <= window:
            su[m - 1] = fw["u"][m - 1]
            continue
        lat, sc = oae.encode(params, fw["u"][m - 1].astype(np.float32).astype(np.float64))
        su[m - 1] = oae.decode(params, lat, sc)
    ref = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=su,
                            image_every=ie)["image"]
    assert rel_l2(img, ref) <= CODEC_TOL


def test_exact_window_over_the_whole_run_is_the_store_all_image():
    import torch

    from helpers import DeviceShot

    case = Case(nx=32, ny=28, nz=24, nb=8, r=4, nt=40, image_every=4)
    P = torch.from_numpy(rtm_inputs.ae_flat(rtm_inputs.ae_init_params(2)).astype(np.float32)).cuda()
    g = DeviceShot(case)
    d_obs = case.d_obs(g.nrec)
    img = _learned_image(case, g, P, d_obs, window=case.nt)
    g.forward()
    ref = g.backward_image(d_obs)[0].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(img, ref)


def test_trained_codec_beats_the_decimation_scheme_and_the_untrained_network():
    """What the trained network gains over the method without it. The codec
    starts from the decimation-equivalent parameters (the network computing
    the non-learned 8x scheme) and is trained by the library's own kernels on
    snapshots of 16 other random models. On held-out snapshots and in the RTM
    image it beats

    * the non-learned 8x scheme at the same bytes (decimated storage: every
      other sample per axis in float32, linear interpolation), and
    * the same network with random weights (untrained),

    with the images of all three storage modes compared against the
    store-all image of the same shot."""
    import torch

    from helpers import DeviceShot
    import paper_1603_03971_gb300 as rtm
    from paper_1603_03971_gb300 import codec, learned

    n = 96
    data = learned.training_snapshots(n_models=16, size=n, nb=16, nt=640, every=20, first=40,
                                      f0=20.0, seed0=500)
    P, losses = learned.train(data, steps=800, batch=4, lr=1e-3, lr_min=5e-5, seed=1,
                              log_every=100, init="decimation")
    print("training losses:", [(s, round(v, 5)) for s, v, _ in losses])
    ie = 8
    case = Case(nx=n, ny=n, nz=n, nb=16, r=4, nt=480, image_every=ie, f0=20.0, t0=0.05,
                vmax=4500.0, src=(48, 40, 4), rec_stride=3, seed=77, sigma=8.0)
    g = DeviceShot(case)
    g.forward()
    exact = {m: rtm.snapshot(g.p, g.ws, m).clone() for m in range(ie, case.nt + 1, ie)}
    d_obs = case.d_obs(g.nrec)
    img_exact = g.backward_image(d_obs)[0].cpu().numpy().astype(np.float64)
    P0 = torch.from_numpy(rtm_inputs.ae_flat(rtm_inputs.ae_init_params(1)).astype(np.float32)).cuda()
    PD = torch.from_numpy(learned.decimation_init(1)).cuda()
    ws = codec.alloc_workspace((n, n, n))

    def snap_err(params):
        num = den = 0.0
        for s in exact.values():
            lat, sc = codec.encode(params, s, ws)
            r = codec.decode(params, lat, sc, ws)
            num += float(((r - s).double() ** 2).sum())
            den += float((s.double() ** 2).sum())
        return (num / den) ** 0.5

    e_tr, e_un, e_init = snap_err(P), snap_err(P0), snap_err(PD)
    # decimated storage on the GPU, its image and (through its snapshots,
    # rebuilt by the oracle's scheme) its snapshot error
    from oracle import ae as oae

    num = den = 0.0
    for s in exact.values():
        sn = s.cpu().numpy().astype(np.float64)
        num += float(np.sum((oae.trilinear_upsample(oae.decimate(sn), n) - sn) ** 2))
        den += float(np.sum(sn ** 2))
    e_de = (num / den) ** 0.5
    pd = case.params()
    pd.storage = rtm.RTM_STORE_DECIMATED
    wd = rtm.alloc_workspace(pd)
    img_d = torch.zeros((n, n, n), device="cuda")
    rtm.shot(pd, g.c, g.rec, torch.from_numpy(d_obs.astype(np.float32)).cuda(), wd, img_d)
    rtm.check(wd)
    img = {"trained": _learned_image(case, g, P, d_obs),
           "untrained": _learned_image(case, g, P0, d_obs),
           "decimated": img_d.cpu().numpy().astype(np.float64)}
    ie_ = {k: rel_l2(v, img_exact) for k, v in img.items()}
    print("snapshot rel-L2: trained %.3e decimation %.3e (network at its initial "
          "parameters %.3e) untrained %.3e" % (e_tr, e_de, e_init, e_un))
    print("image rel-L2: %s" % {k: round(v, 5) for k, v in ie_.items()})
    assert e_tr < 0.9 * e_de
    assert ie_["trained"] < 0.9 * ie_["decimated"]
    assert e_tr < 0.25 * e_un
    assert ie_["trained"] < 0.25 * ie_["untrained"]

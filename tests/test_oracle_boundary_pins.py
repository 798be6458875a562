"""Pins of the oracle's reverse-time source reconstruction (oracle.boundary)
against the forward recursion itself: in FP64 the states recovered backwards
from the last two states and the stored bands are the forward run's own
states, and the image built from them is the store-all image."""
import numpy as np
import pytest

import oracle
import rtm_inputs
from oracle import boundary
from helpers import Case


@pytest.mark.parametrize("shape,r", [((9, 10, 11), 4), ((17, 20, 18), 8), ((12, 12, 12), 1)])
def test_band_count_closed_forms(shape, r):
    nz, ny, nx = shape
    m = boundary.band_mask(shape, r)
    inner = (nx - 2 * r) * (ny - 2 * r) * (nz - 2 * r)
    assert m.sum() == nx * ny * nz - inner
    # faces taken in turn: z planes, then y rows of the other planes, then x cells
    assert m.sum() == 2 * r * nx * ny + 2 * r * (nz - 2 * r) * nx + 2 * r * (nz - 2 * r) * (ny - 2 * r)
    # every band cell is within r of a face, every other cell is not
    z, y, x = np.indices(shape)
    dist = np.minimum.reduce([z, nz - 1 - z, y, ny - 1 - y, x, nx - 1 - x])
    assert np.array_equal(m, dist < r)


def _case(r, src, nt=40, nb=6):
    return Case(nx=22, ny=20, nz=21, nb=nb, r=r, nt=nt, src=src)


@pytest.mark.parametrize("r,src", [(4, (11, 9, 10)), (4, (2, 3, 1)), (8, (11, 10, 10)),
                                   (4, (-3, 5, 6))])
def test_reverse_states_are_the_forward_states(r, src):
    """Source inner, in the band, and in the sponge padding."""
    case = _case(r, src)
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True, keep_last=True)
    u = fw["u"]  # u[n] = u^{n+1}, model region
    mask = boundary.band_mask(u.shape[1:], r)
    bands = {m: u[m - 1][mask] for m in range(1, case.nt - 1)}
    rec = boundary.reverse_states(prob.grid, prob.w, prob.src, fw["last"], bands)
    assert sorted(rec) == list(range(1, case.nt - 1))
    scale = np.abs(u).max()
    for m, um in rec.items():
        assert np.abs(um - u[m - 1]).max() <= 1e-9 * scale, m
    # leaving out the source term breaks it when the source is an inner cell
    if src == (11, 9, 10):
        w0 = np.zeros_like(prob.w)
        bad = boundary.reverse_states(prob.grid, w0, prob.src, fw["last"], bands)
        assert max(np.abs(bad[m] - u[m - 1]).max() for m in bad) > 1e-3 * scale


def test_image_from_reverse_states_is_the_store_all_image():
    case = _case(4, (11, 9, 10), nt=36)
    case.image_every = 1
    prob = case.oracle_problem()
    fw = prob.forward(keep_u=True, keep_last=True)
    u = fw["u"]
    mask = boundary.band_mask(u.shape[1:], 4)
    rec = boundary.reverse_states(prob.grid, prob.w, prob.src, fw["last"],
                                  {m: u[m - 1][mask] for m in range(1, case.nt - 1)})
    snaps = np.zeros_like(u)
    nz, ny, nx = u.shape[1:]
    nb = case.nb
    snaps[case.nt - 1] = fw["last"][1][nb:nb + nz, nb:nb + ny, nb:nb + nx]
    snaps[case.nt - 2] = fw["last"][0][nb:nb + nz, nb:nb + ny, nb:nb + nx]
    for m, um in rec.items():
        snaps[m - 1] = um
    d_obs = rtm_inputs.standard_normal((case.nt, prob.rec.shape[0]), seed=5) * 1e-3
    ref = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=u)["image"]
    img = prob.grid.adjoint(prob.w, prob.src, prob.rec, d_obs, snap_u=snaps)["image"]
    assert np.abs(img - ref).max() <= 1e-9 * np.abs(ref).max()


def test_sponge_in_the_model_region_is_refused():
    case = _case(4, (11, 9, 10), nt=8)
    prob = case.oracle_problem()
    NZ, NY, NX = prob.grid.shape
    deeper = tuple(oracle.sponge_profile(n, case.nb + 2) for n in (NX, NY, NZ))
    g = oracle.Grid(prob.grid.c, case.nb, 4, case.dx, profiles=deeper)  # 2 cells into the model
    fw = prob.forward(keep_last=True)
    with pytest.raises(ValueError):
        boundary.reverse_states(g, prob.w, prob.src, fw["last"], {})

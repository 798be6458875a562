"""Pins of the oracle's off-grid sources and receivers (Kaiser-windowed sinc
weights, Hicks 2002): what the weights must do, and what the propagation
with them must reproduce, each checked against something other than the
oracle's own formula.

* On-grid positions reduce to a single tap of weight 1, and the distributed
  forward and adjoint then reproduce the C oracle's point-source results.
* The weights interpolate waves of up to 3 cells per wavelength (the
  workloads' shortest) to within 1.5e-2 of their amplitude, and those of 4
  cells and more to within 6e-3 (a window parameter far from its optimum,
  or a missing sinc or window factor, misses these by several times).
* Mirror symmetry of the weights, and their decay to zero at the window.
* The adjoint identity <F w, q> = <w, F^T q> with off-grid source and
  receivers (the injection and the gather are transposes).
* Shift invariance: in a constant-velocity model, a source-receiver pair
  moved by half a cell on every axis records the trace of the unmoved pair
  within the interpolation accuracy, while the trace of a pair whose
  offset grows by half a cell on one axis differs by more.
"""
import numpy as np
import pytest

import oracle
import rtm_inputs
from oracle import offgrid


def test_grid_points_are_single_taps():
    for xi in (0.0, 7.0, 33.0):
        idx, w = offgrid.axis_weights(xi, 40)
        assert idx.tolist() == [int(xi)] and w.tolist() == [1.0]
    idx, w = offgrid.point_taps((3.0, 4.0, 5.0), 6, (30, 30, 30))
    assert idx.tolist() == [((5 + 6) * 30 + 4 + 6) * 30 + 3 + 6] and w.tolist() == [1.0]


@pytest.mark.parametrize("kmax,bound", [(2 * np.pi / 3, 1.5e-2), (np.pi / 2, 6e-3)])
def test_weights_interpolate_band_limited_waves(kmax, bound):
    worst = 0.0
    for f in np.linspace(0.05, 0.95, 19):
        xi = 20.0 + f
        idx, w = offgrid.axis_weights(xi, 64)
        assert len(idx) == 8
        for k in np.linspace(0.0, kmax, 41):
            for phase in (0.0, 0.7):
                worst = max(worst, abs(np.dot(w, np.cos(k * idx + phase)) - np.cos(k * xi + phase)))
    assert worst < bound


def test_weights_are_mirror_symmetric_and_windowed():
    i1, w1 = offgrid.axis_weights(10.3, 64)
    i2, w2 = offgrid.axis_weights(10.7, 64)
    np.testing.assert_allclose(w1, w2[::-1], rtol=0, atol=1e-15)
    assert (i1[-1] - 10.3) < 4 and (10.3 - i1[0]) < 4
    # half a cell: the two nearest points carry most of the weight
    i3, w3 = offgrid.axis_weights(10.5, 64)
    assert w3[3] == pytest.approx(w3[4]) and w3[3] > 0.55
    # taps outside the grid are dropped
    i4, _ = offgrid.axis_weights(1.5, 64)
    assert i4.min() == 0 and len(i4) == 6


def _problem(r=4, nt=50, seed=31):
    nx, ny, nz = 20, 18, 16
    nb = r + 2
    v = rtm_inputs.smooth_random_velocity(nx, ny, nz, 3.0, 1500.0, 3000.0, seed)
    dt = rtm_inputs.courant_dt(10.0, 3000.0)
    return oracle.Problem(v, nb, r, 10.0, dt, nt, 40.0, 0.03, (10, 9, 4),
                          rtm_inputs.surface_receivers(nx, ny, 2, stride=3))


@pytest.mark.parametrize("r", [4, 8])
def test_on_grid_positions_reproduce_the_point_oracle(r):
    p = _problem(r)
    NZ, NY, NX = p.grid.shape
    rec_xyz = rtm_inputs.surface_receivers(20, 18, 2, stride=3).astype(np.float64)
    src = offgrid.point_taps((10.0, 9.0, 4.0), p.nb, p.grid.shape)
    recs = offgrid.taps_of(rec_xyz, p.nb, p.grid.shape)
    fw = offgrid.forward(p.grid, p.w, src, recs, keep_u=True)
    ref = p.forward(keep_u=True)
    np.testing.assert_allclose(fw["data"], ref["data"], rtol=1e-12, atol=1e-14 * np.abs(ref["data"]).max())
    rng = np.random.default_rng(3)
    d = rng.standard_normal(ref["data"].shape)
    bw = offgrid.adjoint(p.grid, recs, d, snap_u=fw["u"], src_taps=src)
    bref = p.grid.adjoint(p.w, p.src, p.rec, d, snap_u=ref["u"])
    np.testing.assert_allclose(bw["image"], bref["image"], rtol=1e-11,
                               atol=1e-13 * np.abs(bref["image"]).max())
    np.testing.assert_allclose(bw["src_adj"], bref["src_adj"], rtol=1e-11,
                               atol=1e-13 * np.abs(bref["src_adj"]).max())


@pytest.mark.parametrize("r", [4, 8])
def test_off_grid_dot_product_identity(r):
    p = _problem(r, nt=40)
    rng = np.random.default_rng(5)
    # source and receivers between grid points, some taps in the sponge
    src = offgrid.point_taps((9.4, 8.7, 3.6), p.nb, p.grid.shape)
    rec_xyz = np.array([[2.3, 3.5, 2.25], [15.8, 4.1, 1.9], [10.0, 12.6, 2.0], [-1.5, 7.2, 2.7]])
    recs = offgrid.taps_of(rec_xyz, p.nb, p.grid.shape)
    w = rng.standard_normal(p.nt)
    q = rng.standard_normal((p.nt, len(recs)))
    Fw = offgrid.forward(p.grid, w, src, recs)["data"]
    FTq = offgrid.adjoint(p.grid, recs, q, src_taps=src)["src_adj"]
    lhs, rhs = float(np.sum(Fw * q)), float(np.dot(w, FTq))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_half_cell_shift_of_a_pair_keeps_its_trace():
    n, nb = 44, 8
    vel = np.full((n, n, n), 2000.0)
    dt = rtm_inputs.courant_dt(10.0, 2000.0)
    nt = 160
    p = oracle.Problem(vel, nb, 4, 10.0, dt, nt, 15.0, 0.08, (12, 22, 22),
                       np.array([[30, 22, 22]], np.int32))
    g = p.grid

    def trace(s, rcv):
        return offgrid.forward(g, p.w, offgrid.point_taps(s, nb, g.shape),
                               offgrid.taps_of([rcv], nb, g.shape))["data"][:, 0]

    base = trace((12.0, 22.0, 22.0), (30.0, 22.0, 22.0))
    shifted = trace((12.5, 22.5, 22.5), (30.5, 22.5, 22.5))
    longer = trace((12.0, 22.0, 22.0), (30.5, 22.0, 22.0))
    e_shift = np.linalg.norm(shifted - base) / np.linalg.norm(base)
    e_long = np.linalg.norm(longer - base) / np.linalg.norm(base)
    assert e_shift < 2e-2
    assert e_long > 3 * e_shift

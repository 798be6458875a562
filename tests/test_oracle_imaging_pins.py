"""Pins of the oracle's imaging-condition variants (source illumination,
illumination-normalised image, Laplacian-filtered image) against closed
forms, brute force on tiny inputs and invariants."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import imaging


@pytest.mark.parametrize("r", [2, 4, 8])
def test_laplacian_filter_exact_on_polynomials(r):
    """Away from the edges, -L I equals minus the analytic Laplacian of any
    polynomial image of degree <= 2r + 1 per axis (the 1D weights are exact
    there)."""
    n, dx = 2 * r + 12, 0.5
    z, y, x = np.meshgrid(*(np.arange(n) * dx,) * 3, indexing="ij")
    a, b, c = min(4, 2 * r + 1), 3, 2
    img = x ** a * y ** b + 2.0 * z ** c * x - 3.0 * y * z + 1.5
    lap = (a * (a - 1) * x ** (a - 2) * y ** b + b * (b - 1) * x ** a * y ** (b - 2)
           + 2.0 * c * (c - 1) * z ** (c - 2) * x)
    out = imaging.laplacian_filter(img, r, dx)
    inner = (slice(r, n - r),) * 3
    np.testing.assert_allclose(out[inner], -lap[inner], rtol=1e-9, atol=1e-9 * np.abs(lap).max())


@pytest.mark.parametrize("r,shape", [(2, (5, 6, 7)), (4, (5, 6, 9)), (8, (3, 4, 5))])
def test_laplacian_filter_matches_brute_force_with_zero_outside(r, shape):
    """Explicit loops with the zero condition outside the model grid, also
    for axes shorter than the stencil radius."""
    rng = np.random.default_rng(3)
    img = rng.standard_normal(shape)
    a = [float(f) for f in oracle.stencil_coefficients(r)]
    dx = 2.0
    nz, ny, nx = shape
    ref = np.zeros(shape)

    def at(k, j, i):
        if 0 <= k < nz and 0 <= j < ny and 0 <= i < nx:
            return img[k, j, i]
        return 0.0

    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        s = 3 * a[0] * img[k, j, i]
        for o in range(1, r + 1):
            s += a[o] * (at(k, j, i + o) + at(k, j, i - o) + at(k, j + o, i) + at(k, j - o, i)
                         + at(k + o, j, i) + at(k - o, j, i))
        ref[k, j, i] = -s / (dx * dx)
    np.testing.assert_allclose(imaging.laplacian_filter(img, r, dx), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("every", [1, 2, 3])
def test_illumination_brute_force_and_scaling(every):
    rng = np.random.default_rng(5)
    snaps = rng.standard_normal((8, 3, 4, 5))
    ref = np.zeros((3, 4, 5))
    for m in range(1, 9):
        if m % every == 0:
            for idx in itertools.product(range(3), range(4), range(5)):
                ref[idx] += snaps[m - 1][idx] ** 2
    lam = imaging.illumination(snaps, every)
    np.testing.assert_allclose(lam, ref, rtol=1e-14)
    # quadratic in the source field
    np.testing.assert_allclose(imaging.illumination(-3.0 * snaps, every), 9.0 * lam, rtol=1e-14)
    assert (lam >= 0).all()


def test_normalised_image_of_the_autocorrelation():
    """Dividing the source autocorrelation by itself: every value lies in
    [0, 1/(1 + eps)], the maximum is exactly 1/(1 + eps), and the quotient is
    invariant to a common scale of image and illumination."""
    rng = np.random.default_rng(7)
    lam = rng.random((4, 5, 6)) ** 2
    eps = 1e-2
    q = imaging.normalized_image(lam, lam, eps)
    assert q.max() == pytest.approx(1.0 / (1.0 + eps), rel=1e-15)
    assert (q >= 0).all() and (q <= 1.0 / (1.0 + eps) + 1e-15).all()
    np.testing.assert_allclose(imaging.normalized_image(5.0 * lam, 5.0 * lam, eps), q, rtol=1e-14)
    with pytest.raises(ValueError):
        imaging.normalized_image(lam, lam, 0.0)


def test_illumination_of_a_point_source_is_mirror_symmetric():
    """In a constant-velocity model with the source at the centre, the source
    illumination is symmetric under each axis reflection through the source
    (the propagator and sponge are symmetric there)."""
    n, nb, r = 21, 4, 4
    vel = np.full((n, n, n), 2000.0)
    dx, f0 = 10.0, 30.0
    dt = 0.5 * dx / (2000.0 * np.sqrt(3.0))
    rec = np.array([[1, 1, 1]], dtype=np.int64)
    prob = oracle.Problem(vel, nb, r, dx, dt, 40, f0, 1.0 / f0, (10, 10, 10), rec)
    snaps = prob.forward(keep_u=True)["u"]
    lam = imaging.illumination(snaps, 2)
    assert lam.max() > 0
    for axis in range(3):
        np.testing.assert_allclose(lam, np.flip(lam, axis=axis), rtol=1e-10,
                                   atol=1e-12 * lam.max())

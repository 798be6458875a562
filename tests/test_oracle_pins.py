"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an exactness property, a
published table, an identity of the discrete operators, or finite
differences, so that a dropped term, a wrong sign, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import rtm_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def closed_form_weights(r):
    """a_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!), a_0 = -2 sum a_k:
    the closed form of the centred second-derivative weights."""
    f = math.factorial
    ak = [Fraction(2 * (-1) ** (k + 1) * f(r) ** 2, k * k * f(r - k) * f(r + k))
          for k in range(1, r + 1)]
    return [-2 * sum(ak)] + ak


# ----------------------------------------------------------------------------
# stencil weights
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("r", range(1, 9))
def test_weights_match_closed_form(r):
    assert oracle.stencil_coefficients(r) == closed_form_weights(r)


def test_weights_match_published_table():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "stencil_weights_r4.txt"))
            if ln.strip() and not ln.startswith("#")]
    table = [Fraction(v) for _, v in rows]
    assert oracle.stencil_coefficients(4) == table


def _grid(shape, r, dx=1.0, c=0.0, nb=0, sponge=False):
    return oracle.Grid(np.full(shape, c), nb, r, dx, sponge=sponge)


@pytest.mark.parametrize("r", [4, 8])
def test_laplacian_exact_on_polynomials(r):
    """The 2r-order star is exact on x^a y^b z^c with a, b, c <= 2r+1."""
    n = 2 * r + 8
    dx = 0.5
    g = _grid((n, n, n), r, dx)
    ax = (np.arange(n) - n / 2.0) * dx
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    rng = np.random.default_rng(0)
    for _ in range(4):
        a, b, c = rng.integers(0, 2 * r + 2, size=3)
        u = x ** a * y ** b * z ** c
        exact = np.zeros_like(u)
        if a >= 2:
            exact += a * (a - 1) * x ** (a - 2) * y ** b * z ** c
        if b >= 2:
            exact += b * (b - 1) * x ** a * y ** (b - 2) * z ** c
        if c >= 2:
            exact += c * (c - 1) * x ** a * y ** b * z ** (c - 2)
        lu = g.laplacian(u)
        s = slice(r, n - r)
        err = np.abs(lu[s, s, s] - exact[s, s, s]).max()
        scale = np.abs(u).max() / dx ** 2 + 1.0
        assert err <= 1e-11 * scale, (a, b, c, err)


@pytest.mark.parametrize("r", [2, 4, 8])
def test_laplacian_truncation_constant(r):
    """On x^(2r+2) the error is exactly dx^(2r) * sum_{k=-r..r} a_|k| k^(2r+2)
    (the first non-vanishing moment), independent of x."""
    m = 2 * r + 2
    n = 2 * r + 5
    dx = 0.25
    g = _grid((1, 1, n), r, dx)
    x = (np.arange(n) - n // 2) * dx
    u = (x ** m).reshape(1, 1, n)
    lu = g.laplacian(u)[0, 0]
    w = closed_form_weights(r)
    moment = 2 * sum(w[k] * k ** m for k in range(1, r + 1))
    expect = m * (m - 1) * x ** (m - 2) + float(moment) * dx ** (2 * r)
    s = slice(r, n - r)
    # the y and z passes see zero ghost cells of a constant-in-y/z field: a
    # 1-cell-thick grid gives them a_0 u each, removed here
    a0 = float(w[0])
    lu_x = lu - 2.0 * a0 * u[0, 0] / dx ** 2
    np.testing.assert_allclose(lu_x[s], expect[s], rtol=1e-9, atol=1e-9 * abs(float(moment)))


# ----------------------------------------------------------------------------
# time stepping: dispersion relation and stability
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("r", [4, 8])
def test_plane_wave_is_exact_discrete_solution(r):
    """cos(k.x - w t) solves the leapfrog exactly in the interior when w obeys
    the discrete dispersion relation (2/dt^2)(1 - cos w dt) =
    -(v^2/dx^2) sum_axes symbol(k_a dx), symbol(t) = a0 + 2 sum a_k cos(k t)."""
    n = 6 * r + 6
    dx, v = 10.0, 2000.0
    dt = 0.3 * dx / v
    g = _grid((n, n, n), r, dx, c=v * v * dt * dt)
    rng = np.random.default_rng(1)
    kdx = rng.uniform(0.2, 1.4, size=3)
    w = closed_form_weights(r)
    sym = [float(w[0]) + 2 * sum(float(w[k]) * math.cos(k * t) for k in range(1, r + 1))
           for t in kdx]
    omega = math.acos(1.0 + 0.5 * (v * dt / dx) ** 2 * sum(sym)) / dt
    i = np.arange(n)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    phase = kdx[0] * x + kdx[1] * y + kdx[2] * z
    u_prev = np.cos(phase + omega * dt)
    u_cur = np.cos(phase)
    u_next = g.step(u_cur, u_prev)
    s = slice(r, n - r)
    err = np.abs(u_next - np.cos(phase - omega * dt))[s, s, s].max()
    assert err < 1e-12
    # the continuous dispersion relation w = v|k| must NOT satisfy it
    omega_c = v * np.linalg.norm(kdx) / dx
    err_c = np.abs(u_next - np.cos(phase - omega_c * dt))[s, s, s].max()
    assert err_c > 1e3 * max(err, 1e-15)


@pytest.mark.parametrize("r", [4, 8])
def test_stability_limit_closed_form(r):
    """The limit v dt/dx = 2 / sqrt(3 |symbol(pi)|) (the checkerboard mode)."""
    w = closed_form_weights(r)
    sym_pi = float(w[0]) + 2 * sum(float(w[k]) * (-1) ** k for k in range(1, r + 1))
    assert oracle.stability_limit(r) == pytest.approx(2.0 / math.sqrt(3.0 * abs(sym_pi)),
                                                      rel=1e-9)


def test_stability_limit_4_and_8_values():
    assert oracle.stability_limit(4) == pytest.approx(0.45285552, abs=1e-7)
    assert oracle.stability_limit(8) == pytest.approx(0.42370633, abs=1e-7)


def test_leapfrog_blows_up_just_above_the_limit():
    r, n, dx, v = 4, 28, 10.0, 2000.0
    lim = oracle.stability_limit(r)
    rng = np.random.default_rng(2)
    u0 = rng.standard_normal((n, n, n))
    for factor, should_grow in ((1.03, True), (0.97, False)):
        dt = factor * lim * dx / v
        g = _grid((n, n, n), r, dx, c=v * v * dt * dt)
        a, b = u0.copy(), u0.copy()
        for _ in range(150):
            a, b = g.step(a, b), a
        grew = np.abs(a).max() > 1e3 * np.abs(u0).max()
        assert grew == should_grow, factor


# ----------------------------------------------------------------------------
# wavelet and sponge
# ----------------------------------------------------------------------------

def test_ricker_closed_form_points():
    f0, dt = 16.0, 2.0 ** -14          # t0 / dt = 1024 exactly
    t0 = 1.0 / f0
    nt = 4096
    w = oracle.ricker(nt, dt, f0, t0)
    assert w[int(round(t0 / dt))] == pytest.approx(1.0, abs=1e-12)
    tz = 1.0 / (math.pi * f0 * math.sqrt(2.0))  # 1 - 2 pi^2 f0^2 tau^2 = 0
    for t in (t0 - tz, t0 + tz):
        # sample exactly on a zero crossing
        w1 = oracle.ricker(1, 1.0, f0, t0 - t)  # w(0 - (t0 - t)) = w at t
        assert abs(w1[0]) < 1e-12
    # trough value at tau = sqrt(3/2)/(pi f0): -2 exp(-3/2)
    tau = math.sqrt(1.5) / (math.pi * f0)
    assert oracle.ricker(1, 1.0, f0, -tau)[0] == pytest.approx(-2 * math.exp(-1.5), rel=1e-12)
    # integral over [0, 2 t0]: the antiderivative of (1 - 2 b s^2) exp(-b s^2)
    # is s exp(-b s^2), so it equals 2 t0 exp(-pi^2 f0^2 t0^2)
    win = w[:2049]
    trap = dt * (win.sum() - 0.5 * (win[0] + win[-1]))
    assert trap == pytest.approx(2 * t0 * math.exp(-(math.pi * f0 * t0) ** 2), abs=1e-9)
    # peak frequency f0
    spec = np.abs(np.fft.rfft(w, 1 << 16))
    freqs = np.fft.rfftfreq(1 << 16, dt)
    assert freqs[np.argmax(spec)] == pytest.approx(f0, abs=0.1)


def test_sponge_profile_shape():
    nb, n = 20, 64
    g = oracle.sponge_profile(n, nb)
    assert np.all(g[nb:n - nb] == 1.0)
    assert g[0] == pytest.approx(math.exp(-(0.015 * nb) ** 2))
    assert np.all(np.diff(g[:nb + 1]) > 0)
    np.testing.assert_array_equal(g, g[::-1])
    assert np.all(oracle.sponge_profile(n, 0) == 1.0)


def test_sponge_absorbs_energy():
    """With the sponge the field energy left after the wave has crossed it is
    a small fraction of the peak; with rigid walls it is not."""
    r, n_model, nb, dx, v = 4, 24, 20, 10.0, 2000.0
    dt = rtm_inputs.courant_dt(dx, v)
    vel = np.full((n_model,) * 3, v)
    rec = np.array([[12, 12, 12]], dtype=np.int32)
    res = {}
    for sponge in (True, False):
        p = oracle.Problem(vel, nb, r, dx, dt, 400, 20.0, 0.05, (12, 12, 12), rec,
                           sponge=sponge)
        p.w[150:] = 0.0
        energies = []
        u_prev = np.zeros(p.grid.shape)
        u = np.zeros(p.grid.shape)
        for step in range(400):
            u_next = p.grid.step(u, u_prev)
            u_next.flat[p.src] += p.grid.c.flat[p.src] * p.w[step] / dx ** 3
            u_prev, u = u, u_next
            energies.append(float(np.sum(u * u)))
        res[sponge] = energies[-1] / max(energies)
    assert res[True] < 0.02
    assert res[False] > 0.2


# ----------------------------------------------------------------------------
# physics: constant-velocity Green's function
# ----------------------------------------------------------------------------

@pytest.mark.slow
def test_green_function_constant_velocity():
    """p(r,t) = w(t - r/v) / (4 pi r) solves (1/v^2) p_tt - lap p = w(t) delta;
    the trace of receiver j at step n is time (n+1) dt."""
    r, n_model, nb, dx, v = 4, 48, 20, 10.0, 2000.0
    f0 = 10.0
    t0 = 1.2 / f0
    dt = rtm_inputs.courant_dt(dx, v)
    nt = 200
    vel = np.full((n_model,) * 3, v)
    src = (24, 24, 24)
    rec = np.array([[24 + 12, 24, 24], [24, 24 - 10, 24], [24 + 8, 24 + 8, 24 - 5]],
                   dtype=np.int32)
    p = oracle.Problem(vel, nb, r, dx, dt, nt, f0, t0, src, rec)
    d = p.forward()["data"]
    t = (np.arange(nt) + 1) * dt
    for j in range(rec.shape[0]):
        dist = dx * np.linalg.norm(rec[j] - np.array(src))
        tau = t - dist / v - t0
        a = (math.pi * f0 * tau) ** 2
        exact = (1 - 2 * a) * np.exp(-a) / (4 * math.pi * dist)
        err = np.linalg.norm(d[:, j] - exact) / np.linalg.norm(exact)
        assert err < 0.05, (j, err)


def test_linearity_in_the_wavelet():
    prob = _small_problem(4, seed=3)
    d1 = prob.forward()["data"]
    prob.w = prob.w * 2.5
    d2 = prob.forward()["data"]
    np.testing.assert_allclose(d2, 2.5 * d1, rtol=1e-12, atol=1e-300)


# ----------------------------------------------------------------------------
# adjoint, imaging, gradient
# ----------------------------------------------------------------------------

def _small_problem(r, seed, nt=60, squared=False, nb=None):
    nx, ny, nz = 20, 18, 16
    nb = (r + 2) if nb is None else nb
    dx = 10.0
    v = rtm_inputs.smooth_random_velocity(nx, ny, nz, 3.0, 1500.0, 3000.0, seed)
    dt = rtm_inputs.courant_dt(dx, 3000.0)
    rec = rtm_inputs.surface_receivers(nx, ny, 2, stride=3)
    vel = v * v if squared else v
    return oracle.Problem(vel, nb, r, dx, dt, nt, 40.0, 0.03, (10, 9, 4), rec,
                          squared=squared)


@pytest.mark.parametrize("r,in_sponge", [(4, False), (8, False), (4, True)])
def test_dot_product_adjoint(r, in_sponge):
    """<F w, q> = <w, F^T q> with F the forward map (wavelet -> data) and
    F^T q the receiver propagation's trace at the source. The last case puts
    the source and some receivers inside the sponge (g < 1) so that every
    sponge factor of the injection and of the source trace is exercised."""
    p = _small_problem(r, seed=11)
    if in_sponge:
        rec = np.concatenate([rtm_inputs.surface_receivers(20, 18, 2, stride=5),
                              np.array([[-3, 4, 5], [21, -2, 3], [5, 6, -4]], np.int32)])
        p = oracle.Problem(p.vel, p.nb, r, p.dx, p.dt, p.nt, p.f0, p.t0, (-2, 9, 4), rec)
        assert p.grid.g().flat[p.src] < 1.0
    rng = np.random.default_rng(12)
    w = rng.standard_normal(p.nt)
    q = rng.standard_normal((p.nt, p.rec.size))
    Fw = p.grid.forward(w, p.src, p.rec)["data"]
    FTq = p.grid.adjoint(w, p.src, p.rec, q)["src_adj"]
    lhs, rhs = float(np.sum(Fw * q)), float(np.dot(w, FTq))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_imaging_identity():
    """I(x) = sum_m u^m(x) mu^m(x) equals <d_obs, F_x q> where F_x models a
    source at x emitting q^n = g_x u^{n+1}(x): the receiver wavefield at x is
    the adjoint of injecting at x, so the pairing u^m with mu^m (same time
    level) is checked without re-implementing the image sum."""
    p = _small_problem(4, seed=21)
    rng = np.random.default_rng(22)
    d_obs = rng.standard_normal((p.nt, p.rec.size))
    fw = p.forward(keep_u=True)
    img = p.grid.adjoint(p.w, p.src, p.rec, d_obs, snap_u=fw["u"])["image"]
    g = p.grid.g()
    nz, ny, nx = p.grid.model_shape
    for (x, y, z) in [(3, 4, 5), (10, 9, 2), (17, 1, 14), (12, 12, 8)]:
        lin = int(oracle.padded_index(np.array([[x, y, z]]), p.nb, p.grid.shape)[0])
        q = fw["u"][:, z, y, x] * g.flat[lin]
        D = p.grid.forward(q, lin, p.rec)["data"]
        expect = float(np.sum(D * d_obs))
        assert img[z, y, x] == pytest.approx(expect, rel=1e-10, abs=1e-14 * abs(expect) + 1e-300)


def test_image_is_bilinear_and_subsamples():
    p = _small_problem(4, seed=31, nt=40)
    rng = np.random.default_rng(32)
    d_obs = rng.standard_normal((p.nt, p.rec.size))
    i1 = p.rtm_image(d_obs)["image"]
    i2 = p.rtm_image(2.0 * d_obs)["image"]
    np.testing.assert_allclose(i2, 2.0 * i1, rtol=1e-12)
    # imaging every 4th step: the sum over m = 4, 8, ... only
    fw = p.forward(keep_u=True)
    i4 = p.grid.adjoint(p.w, p.src, p.rec, d_obs, snap_u=fw["u"], image_every=4)["image"]
    keep = np.zeros_like(fw["u"])
    keep[3::4] = fw["u"][3::4]
    i4b = p.grid.adjoint(p.w, p.src, p.rec, d_obs, snap_u=keep)["image"]
    np.testing.assert_allclose(i4, i4b, rtol=1e-12, atol=1e-300)


def test_fold_is_transpose_of_padding():
    rng = np.random.default_rng(41)
    a = rng.standard_normal((5, 6, 7))
    b = rng.standard_normal((5 + 6, 6 + 6, 7 + 6))
    lhs = float(np.sum(oracle.pad_model(a, 3) * b))
    rhs = float(np.sum(a * oracle.fold_padding(b, 3)))
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("r", [4, 8])
def test_gradient_matches_central_differences(r):
    """dJ/d(v^2) against central differences of J in FP64 along random
    directions, one of them concentrated at the source (the injection term)."""
    p = _small_problem(r, seed=51, nt=50, squared=True)
    v2 = p.vel.copy()
    d_obs = _small_problem(r, seed=52, nt=50, squared=True).forward()["data"] * 0.7
    J, grad = p.misfit_and_grad(d_obs)
    dirs = list(rtm_inputs.random_directions(v2.shape, 3, seed=53))
    spot = np.zeros_like(v2)
    spot[4, 9, 10] = 1.0  # the source cell (x=10, y=9, z=4)
    dirs.append(spot)
    for k, delta in enumerate(dirs):
        eps = 1e-4 * np.abs(v2).max() / np.abs(delta).max()
        Jp = _misfit_at(p, v2 + eps * delta, d_obs)
        Jm = _misfit_at(p, v2 - eps * delta, d_obs)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(grad * delta))
        assert an == pytest.approx(fd, rel=1e-6), (k, an, fd)


def _misfit_at(p, v2, d_obs):
    q = oracle.Problem(v2, p.nb, p.r, p.dx, p.dt, p.nt, p.f0, p.t0, (10, 9, 4),
                       rtm_inputs.surface_receivers(20, 18, 2, stride=3), squared=True)
    return q.misfit(d_obs)


def test_crop_with_the_grids_profiles_reproduces_the_full_grid():
    """After n steps the discrete field vanishes beyond n r cells of the
    source, so a crop with that margin that keeps the full grid's c and sponge
    profiles reproduces the full-grid field exactly (used by the full-size
    sampled parity tests)."""
    r, nb, n_model, dx = 4, 10, 40, 10.0
    vel = rtm_inputs.smooth_random_velocity(n_model, n_model, n_model, 3.0, 1500.0, 3000.0, 5)
    dt = rtm_inputs.courant_dt(dx, 3000.0)
    nt = 6
    src = (20, 22, 3)
    full = oracle.Problem(vel, nb, r, dx, dt, nt, 30.0, 0.03, src, np.array([[20, 22, 5]]))
    ref = full.forward(keep_last=True)["last"][1]
    sz, sy, sx = (src[2] + nb, src[1] + nb, src[0] + nb)
    m = nt * r + 1
    z0, z1 = max(0, sz - m), min(full.grid.NZ, sz + m + 1)
    y0, y1 = max(0, sy - m), min(full.grid.NY, sy + m + 1)
    x0, x1 = max(0, sx - m), min(full.grid.NX, sx + m + 1)
    g = oracle.Grid(full.grid.c[z0:z1, y0:y1, x0:x1], nb, r, dx,
                    profiles=(full.grid.gx[x0:x1], full.grid.gy[y0:y1], full.grid.gz[z0:z1]))
    s_lin = ((sz - z0) * (y1 - y0) + (sy - y0)) * (x1 - x0) + (sx - x0)
    out = g.forward(full.w, s_lin, np.array([s_lin]), keep_last=True)["last"][1]
    np.testing.assert_array_equal(out, ref[z0:z1, y0:y1, x0:x1])
    assert np.abs(ref).sum() == pytest.approx(np.abs(out).sum(), rel=1e-14)

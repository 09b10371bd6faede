"""Pins for the FP64 oracle against what the mathematics fixes.

Each test is chosen so that a plausible slip in the oracle (a wrong
coefficient, a dropped axis, a transposed index, a sign error in the
recurrence, the wrong halo) fails at least one of them:

* the stencil weights are the unique 5-point-symmetric solution of the
  Taylor moment conditions (exact in rational arithmetic);
* the Laplacian is exact on polynomials of degree <= 9 per axis and not on
  degree 10 (leading error 2*sum c_m m^10 = -1152);
* the whole recurrence (Laplacian, sponge, source, receivers) equals the
  same recurrence written with explicit Kronecker-product matrices on a
  small non-cubic grid, Dirichlet and periodic;
* the discrete energy of the source-free, sponge-free scheme is conserved;
* a discrete plane wave in a periodic box follows the dispersion relation
  cos(w dt) = 1 + nu^2/2 * sum_a L(k_a h) exactly;
* the scheme is stable just below the Courant limit and blows up just
  above it;
* a centred source in a homogeneous odd-sized box gives a field symmetric
  under every mirror and axis swap;
* the Ricker wavelet has its peak, zero crossings and zero mean where its
  definition puts them; the sponge profile has the stated shape.
"""

from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle


# ---------------------------------------------------------------- stencil

def test_coefficients_solve_taylor_moments_exactly():
    # Unknowns c0..c4 of f''(0) ~ c0 f(0) + sum c_m (f(m) + f(-m)).
    # Conditions: p = 0: c0 + 2 sum c_m = 0;  p = 2k: 2 sum c_m m^p = p! [p==2]
    A = [[Fraction(1)] + [Fraction(2)] * 4]
    b = [Fraction(0)]
    for p in (2, 4, 6, 8):
        A.append([Fraction(0)] + [Fraction(2 * m ** p) for m in range(1, 5)])
        b.append(Fraction(2) if p == 2 else Fraction(0))
    # Gaussian elimination in exact arithmetic
    n = 5
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col] / M[col][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    exact = [M[i][n] / M[i][i] for i in range(n)]
    c = oracle.coefficients()
    for ce, co in zip(exact, c):
        assert co == pytest.approx(float(ce), rel=1e-15, abs=1e-18)


def test_coefficients_moments_and_order():
    c = oracle.coefficients()
    m = np.arange(1, 5, dtype=np.float64)
    assert c[0] + 2 * c[1:].sum() == pytest.approx(0.0, abs=1e-14)
    assert 2 * (c[1:] * m ** 2).sum() == pytest.approx(2.0, abs=1e-13)
    for p in (4, 6, 8):
        assert 2 * (c[1:] * m ** p).sum() == pytest.approx(0.0, abs=1e-10)
    # order is exactly 8: degree 10 is not reproduced
    assert 2 * (c[1:] * m ** 10).sum() == pytest.approx(-1152.0, rel=1e-12)


def _poly_field(nx, ny, nz, degs, s=0.1, seed=0):
    """u = P(x) Q(y) S(z) on the padded grid, with its exact Laplacian."""
    rng = np.random.default_rng(seed)
    R = oracle.R
    axes = []
    for n, d in zip((nx, ny, nz), degs):
        coeffs = rng.uniform(-1, 1, d + 1)
        t = (np.arange(-R, n + R) - n / 2.0) * s
        P = np.polynomial.Polynomial(coeffs)
        axes.append((P(t), P.deriv(2)(t) * s * s))
    (px, dpx), (py, dpy), (pz, dpz) = axes
    u = pz[:, None, None] * py[None, :, None] * px[None, None, :]
    lap = (dpz[:, None, None] * py[None, :, None] * px[None, None, :]
           + pz[:, None, None] * dpy[None, :, None] * px[None, None, :]
           + pz[:, None, None] * py[None, :, None] * dpx[None, None, :])
    return u, lap[R:-R, R:-R, R:-R]


@pytest.mark.parametrize("degs", [(9, 0, 0), (0, 9, 0), (0, 0, 9),
                                  (9, 9, 9), (2, 5, 7)])
def test_laplacian_exact_on_degree_9(degs):
    u, exact = _poly_field(11, 9, 7, degs)
    got = oracle.laplacian(u)
    scale = np.abs(exact).max() + np.abs(u).max() * 1e-3
    assert np.abs(got - exact).max() <= 1e-11 * scale


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_laplacian_degree_10_leading_error(axis):
    # u = t^10 along one axis (unit spacing): the discrete operator at t = 0
    # returns 2 sum c_m m^10 = -1152 while the exact second derivative is 0.
    R = oracle.R
    n = 9
    t = np.arange(-R, n + R, dtype=np.float64) - 4.0   # t = 0 at index 4
    shape = [1, 1, 1]
    shape[axis] = t.size
    line = (t ** 10).reshape(shape)
    full = np.broadcast_to(line, (n + 2 * R,) * 3).copy()
    got = oracle.laplacian(full)
    exact = 90.0 * t[R:-R] ** 8
    if axis == 0:
        got_line = got[:, 4, 4]
    elif axis == 1:
        got_line = got[4, :, 4]
    else:
        got_line = got[4, 4, :]
    err = got_line - exact
    # error of an order-8 scheme on t^10: (2 sum c_m m^10 / 10!) * u^(10) = -1152
    assert err == pytest.approx(np.full(n, -1152.0), rel=1e-9)


def test_symbol_minimum_is_at_pi():
    th = np.linspace(0.0, np.pi, 2001)
    vals = np.array([oracle.symbol(t) for t in th])
    assert np.argmin(vals) == th.size - 1
    c = oracle.coefficients()
    lpi = c[0] + 2 * sum(c[m] * (-1) ** m for m in range(1, 5))
    assert oracle.symbol(np.pi) == pytest.approx(lpi, rel=1e-15)
    assert lpi == pytest.approx(-6.5015873015873, rel=1e-12)
    assert oracle.nu_max() ** 2 * 3 * abs(lpi) == pytest.approx(4.0, rel=1e-14)


# ------------------------------------------------------- brute force (matrix)

def _d1(n, periodic):
    c = oracle.coefficients()
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] += c[0]
        for m in range(1, 5):
            for j in (i - m, i + m):
                if periodic:
                    D[i, j % n] += c[m]
                elif 0 <= j < n:
                    D[i, j] += c[m]
    return sp.csr_matrix(D)


def _kron_laplacian(nx, ny, nz, periodic):
    Ix, Iy, Iz = (sp.identity(n, format="csr") for n in (nx, ny, nz))
    Dx, Dy, Dz = (_d1(n, periodic) for n in (nx, ny, nz))
    # C order (z, y, x): x is the fastest index
    return (sp.kron(Iz, sp.kron(Iy, Dx)) + sp.kron(Iz, sp.kron(Dy, Ix))
            + sp.kron(Dz, sp.kron(Iy, Ix))).tocsr()


def _sponge(n, w, a):
    g = np.ones(n)
    for i in range(n):
        d = min(i, n - 1 - i)
        if d < w:
            g[i] = np.exp(-(a * (w - d)) ** 2)
    return g


@pytest.mark.parametrize("periodic", [False, True])
def test_recurrence_matches_kronecker_brute_force(periodic):
    nx, ny, nz = 7, 8, 9
    rng = np.random.default_rng(3)
    vel = rng.uniform(1500, 4500, (nz, ny, nx))
    h, dt, nsteps = 10.0, 1.0e-3, 25
    w, a = 2, 0.2
    src = (2, 5, 3)
    wl = rng.standard_normal(nsteps)
    rec = np.array([[1, 2, 3], [6, 0, 8], [3, 7, 4]], dtype=np.int32)
    u0 = rng.standard_normal((nz, ny, nx)) * 0.1
    um1 = rng.standard_normal((nz, ny, nx)) * 0.1
    got = oracle.run(vel, h, nsteps, dt=dt, sponge=w, sponge_a=a,
                     periodic=periodic, src=src, wavelet=wl, receivers=rec,
                     u0=u0, um1=um1, norms=True)

    L = _kron_laplacian(nx, ny, nz, periodic)
    coef = ((vel * dt / h) ** 2).ravel()
    G = (_sponge(nz, w, a)[:, None, None] * _sponge(ny, w, a)[None, :, None]
         * _sponge(nx, w, a)[None, None, :]).ravel()
    sidx = (src[2] * ny + src[1]) * nx + src[0]
    ridx = (rec[:, 2] * ny + rec[:, 1]) * nx + rec[:, 0]
    un, up = u0.ravel().copy(), um1.ravel().copy()
    traces = np.zeros((len(rec), nsteps))
    norms = np.zeros(nsteps)
    for n in range(nsteps):
        f = np.zeros_like(un)
        f[sidx] = wl[n]
        nxt = G * (2 * un - G * up + coef * (L @ un + f))
        up, un = un, nxt
        traces[:, n] = un[ridx]
        norms[n] = (un ** 2).sum()
    scale = np.abs(un).max()
    assert np.abs(got["u"].ravel() - un).max() <= 1e-12 * scale
    assert np.abs(got["u_prev"].ravel() - up).max() <= 1e-12 * scale
    assert np.abs(got["traces"] - traces).max() <= 1e-12 * scale
    assert got["norms"] == pytest.approx(norms, rel=1e-12)


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("periodic", [False, True])
def test_energy_is_conserved_without_source_and_sponge(periodic):
    nx, ny, nz = 10, 9, 8
    rng = np.random.default_rng(11)
    vel = rng.uniform(1500, 4500, (nz, ny, nx))
    h = 10.0
    dt = oracle.time_step(h, vel.max(), 0.9 * oracle.nu_max())
    coef = (vel * dt / h) ** 2
    u = rng.standard_normal((nz, ny, nx))
    up = rng.standard_normal((nz, ny, nx))
    energies = []
    for _ in range(40):
        r = oracle.run(vel, h, 1, dt=dt, periodic=periodic, u0=u, um1=up)
        energies.append(oracle.energy(coef, r["u"], u, periodic))
        u, up = r["u"], r["u_prev"]
    e = np.array(energies)
    assert e[0] > 0
    assert np.abs(e - e[0]).max() <= 1e-11 * abs(e[0])


def test_plane_wave_follows_discrete_dispersion():
    nx, ny, nz = 16, 12, 10
    h, v = 10.0, 2000.0
    nu = 0.8 * oracle.nu_max()
    dt = nu * h / v
    kx, ky, kz = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny, 2 * np.pi * 1 / nz
    c = oracle.coefficients()

    def L(t):  # symbol from the (moment-pinned) weights
        return c[0] + 2 * sum(c[m] * np.cos(m * t) for m in range(1, 5))

    cwdt = 1 + 0.5 * nu ** 2 * (L(kx) + L(ky) + L(kz))
    wdt = np.arccos(cwdt)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                          indexing="ij")
    phase = kx * i + ky * j + kz * k
    u0 = np.cos(phase)
    um1 = np.cos(phase + wdt)
    nsteps = 60
    r = oracle.run(np.full((nz, ny, nx), v), h, nsteps, dt=dt,
                   periodic=True, u0=u0, um1=um1)
    want = np.cos(phase - wdt * nsteps)
    assert np.abs(r["u"] - want).max() <= 1e-10
    # and it is NOT the continuous-dispersion wave (the test can tell)
    w_cont = v * np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) / h
    assert np.abs(r["u"] - np.cos(phase - w_cont * dt * nsteps)).max() > 1e-4


@pytest.mark.parametrize("factor,stable", [(0.99, True), (1.01, False)])
def test_courant_limit(factor, stable):
    n = 16
    h, v = 10.0, 3000.0
    dt = factor * oracle.nu_max() * h / v
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal((n, n, n))
    r = oracle.run(np.full((n, n, n), v), h, 300, dt=dt, periodic=True,
                   u0=u0, um1=u0)
    amp = np.abs(r["u"]).max()
    if stable:
        assert amp < 1e3
    else:
        assert amp > 1e20


def test_centred_source_is_mirror_symmetric():
    n = 15
    vel = np.full((n, n, n), 2500.0)
    r = oracle.run(vel, 10.0, 60, sponge=3, src=(7, 7, 7), f_peak=40.0)
    u = r["u"]
    scale = np.abs(u).max()
    assert scale > 0
    for ax in range(3):
        assert np.abs(u - np.flip(u, axis=ax)).max() <= 1e-13 * scale
    assert np.abs(u - u.transpose(1, 0, 2)).max() <= 1e-13 * scale
    assert np.abs(u - u.transpose(2, 1, 0)).max() <= 1e-13 * scale


def test_default_time_step_is_half_the_limit():
    dt = oracle.time_step(10.0, 1500.0)
    assert dt * 1500.0 / 10.0 == pytest.approx(0.5 * oracle.nu_max(),
                                               rel=1e-15)
    assert dt == pytest.approx(1.5095e-3, rel=1e-4)


# --------------------------------------------------------------- wavelet

def test_ricker_definition_properties():
    f = 15.0
    t0 = 1.0 / f
    dt = t0 / 500.0
    r = oracle.ricker(f, dt, 20000)
    assert r[500] == pytest.approx(1.0, abs=1e-15)        # peak at t0
    assert np.argmax(r) == 500
    assert np.abs(r[500 - 170:500] - r[501:501 + 170][::-1]).max() < 1e-13
    tz = 1.0 / (np.pi * f * np.sqrt(2.0))                  # zero crossings
    lo = int(np.floor((t0 + tz) / dt))
    assert r[lo] > 0 > r[lo + 1]
    lo = int(np.floor((t0 - tz) / dt))
    assert r[lo] < 0 < r[lo + 1]
    assert r[0] == pytest.approx(
        (1 - 2 * np.pi ** 2) * np.exp(-np.pi ** 2), rel=1e-12)
    # zero mean: an antiderivative of r is tau*exp(-pi^2 f^2 tau^2), so the
    # integral from t = 0 (tau = -t0) onwards is t0*exp(-pi^2)
    area = np.trapezoid(r, dx=dt)
    assert area == pytest.approx(t0 * np.exp(-np.pi ** 2), rel=1e-3)


def test_cerjan_profile_shape():
    g = oracle.cerjan(64, 20, 0.015)
    assert g[0] == pytest.approx(np.exp(-(0.015 * 20) ** 2), rel=1e-15)
    assert g[19] == pytest.approx(np.exp(-0.015 ** 2), rel=1e-15)
    assert np.all(g[20:44] == 1.0)
    assert np.all(np.diff(g[:21]) > 0)
    assert np.array_equal(g, g[::-1])
    assert np.all(oracle.cerjan(10, 0) == 1.0)


# ---------------------------------------------------------- halo exchange

def test_halo_exchange_definition():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((10, 9, 12))
    xs = oracle.split_points(12, 2)
    sub0 = oracle.halo_exchanged(u, xs[0], (0, 9), (0, 10))
    sub1 = oracle.halo_exchanged(u, xs[1], (0, 9), (0, 10))
    R = oracle.R
    # +x face halo of the left block = first R x-planes of the right block
    assert np.array_equal(sub0[R:-R, R:-R, -R:], u[:, :, 6:6 + R])
    assert np.array_equal(sub1[R:-R, R:-R, :R], u[:, :, 6 - R:6])
    # global boundary halos are zero (Dirichlet)
    assert np.all(sub0[R:-R, R:-R, :R] == 0)
    assert np.all(sub0[:R, R:-R, R:-R] == 0)
    # edges / corners are undefined
    assert np.isnan(sub0[0, 0, R])
    assert oracle.split_points(10, 3) == [(0, 4), (4, 7), (7, 10)]

"""Pins of the oracle's D3Q27 flow step: the generic central-moment procedure
that extends the paper's 3D method (Appendix A) to D3Q27.  The procedure's
code is shared with the D2Q9 route that reproduces Eqs. 23/31/32
(tests/test_oracle_d2q9.py); here it is pinned in 3D by definitions and
closed-form flows."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_10247_gb300 import workloads as W
from tests.moment_defs import D3Q27_E, W_D3Q27, central, maxwell_central, raw

EXPS = list(itertools.product(range(3), repeat=3))


def _lat(omega, shape=(1, 1, 1), wall=(0, 0, 0), P=None):
    return O.OracleLattice(O.D3Q27, shape, wall=wall, omega=omega, P=P)


def _rand_f(rng, amp=0.05):
    return W_D3Q27 * (1 + amp * rng.standard_normal(27))


def test_rest_weights():
    L = _lat(W.d3q27_omega(0.8), shape=(2, 2, 2))
    L.init_equilibrium(1.0, [0, 0, 0])
    assert np.abs(L.f[:, 0] - W_D3Q27).max() < 4e-16
    assert sorted(set(np.round(W_D3Q27 * 216).astype(int))) == [1, 4, 16, 64]


def test_unit_omega_reaches_maxwellian_central_moments():
    rng = np.random.default_rng(20)
    L = _lat(W.d3q27_omega(1.0))
    for _ in range(20):
        f = _rand_f(rng, 0.1)
        fp = L.collide_node(f, [0, 0, 0], [0, 0, 0])
        rho = f.sum()
        u = np.array([raw(f, D3Q27_E, 1, 0, 0), raw(f, D3Q27_E, 0, 1, 0), raw(f, D3Q27_E, 0, 0, 1)]) / rho
        for a, b, c in EXPS:
            got = central(fp, D3Q27_E, u, a, b, c)
            assert abs(got - maxwell_central(rho, a, b, c)) < 3e-15, ((a, b, c), got)


def test_general_omega_relaxation_by_group():
    rng = np.random.default_rng(21)
    for _ in range(20):
        om = (0.0,) + tuple(rng.uniform(0.2, 1.9, 6)) + (0.0, 0.0)
        L = _lat(om)
        f = _rand_f(rng, 0.1)
        fp = L.collide_node(f, [0, 0, 0], [0, 0, 0])
        rho = f.sum()
        u = np.array([raw(f, D3Q27_E, 1, 0, 0), raw(f, D3Q27_E, 0, 1, 0), raw(f, D3Q27_E, 0, 0, 1)]) / rho
        k = lambda g, a, b, c: central(g, D3Q27_E, u, a, b, c)  # noqa: E731
        T = k(f, 2, 0, 0) + k(f, 0, 2, 0) + k(f, 0, 0, 2)
        Tp = k(fp, 2, 0, 0) + k(fp, 0, 2, 0) + k(fp, 0, 0, 2)
        assert abs(Tp - (T + om[1] * (rho - T))) < 3e-15
        for (p, q) in [((2, 0, 0), (0, 2, 0)), ((2, 0, 0), (0, 0, 2))]:
            D = k(f, *p) - k(f, *q)
            Dp = k(fp, *p) - k(fp, *q)
            assert abs(Dp - (1 - om[2]) * D) < 3e-15
        for a, b, c in EXPS:
            n = a + b + c
            if n == 2 and 2 not in (a, b, c):
                assert abs(k(fp, a, b, c) - (1 - om[2]) * k(f, a, b, c)) < 3e-15
            if n >= 3:
                eq = maxwell_central(rho, a, b, c)
                want = k(f, a, b, c) + om[n] * (eq - k(f, a, b, c))
                assert abs(k(fp, a, b, c) - want) < 3e-15, (a, b, c)
            if n <= 1:
                assert abs(k(fp, a, b, c) - k(f, a, b, c)) < 3e-15


def test_force_changes_first_moment_by_average_force():
    rng = np.random.default_rng(22)
    L = _lat(W.d3q27_omega(0.7))
    for _ in range(20):
        f = _rand_f(rng)
        Fpre, Fpost = 1e-3 * rng.standard_normal(3), 1e-3 * rng.standard_normal(3)
        fp = L.collide_node(f, Fpre, Fpost)
        assert abs(fp.sum() - f.sum()) < 1e-15
        dj = (fp - f) @ D3Q27_E
        assert np.allclose(dj, (Fpre + Fpost) / 2, rtol=0, atol=2e-15)


def test_equilibrium_is_fixed_point():
    rng = np.random.default_rng(23)
    om = (0.0,) + tuple(rng.uniform(0.2, 1.9, 6)) + (0.0, 0.0)
    L = _lat(om, shape=(3, 2, 2))
    rho = 1 + 0.01 * rng.standard_normal(L.N)
    u = 0.05 * rng.standard_normal((3, L.N))
    L.init_equilibrium(rho, u)
    for i in range(L.N):
        fi = L.f[:, i]
        for a, b, c in EXPS:
            assert abs(central(fi, D3Q27_E, u[:, i], a, b, c) - maxwell_central(rho[i], a, b, c)) < 1e-15
        assert np.abs(L.collide_node(fi, [0, 0, 0], [0, 0, 0]) - fi).max() < 1e-15


def test_streaming_with_walls_in_two_axes():
    L = _lat((0.0,) * 9, shape=(3, 3, 3), wall=(0, 1, 1))
    opp = [26 - a for a in range(27)]
    for a in range(27):
        for (x, y, z) in [(0, 0, 0), (2, 2, 2), (1, 0, 2), (1, 1, 1)]:
            i = x + 3 * (y + 3 * z)
            L.f = np.repeat(W_D3Q27[:, None], L.N, axis=1)
            L.f[a, i] += 1.0
            L.run(1)
            L.f -= W_D3Q27[:, None]
            e = D3Q27_E[a].astype(int)
            tx, ty, tz = x + e[0], y + e[1], z + e[2]
            g = np.zeros((27, L.N))
            if 0 <= ty < 3 and 0 <= tz < 3:
                g[a, (tx % 3) + 3 * (ty + 3 * tz)] = 1.0
            else:
                g[opp[a], i] = 1.0
            assert np.abs(L.f - g).max() < 1e-15, (a, x, y, z)


@pytest.mark.parametrize("axis", [1, 2])
def test_shear_wave_decay_gives_viscosity(axis):
    n = 48
    tau = 0.9
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    shape = [2, 2, 2]
    shape[axis] = n
    L = _lat(W.d3q27_omega(tau), shape=tuple(shape))
    idx = np.indices(shape[::-1]).reshape(3, -1)[::-1]  # x, y, z of each node
    s = np.sin(k * idx[axis])
    u = np.zeros((3, L.N))
    u[0] = 1e-4 * s
    L.init_equilibrium(1.0, u)
    amps = []
    for t in (100, 600):
        L.run(t - L.t)
        _, uu = L.moments()
        amps.append(np.sum(uu[0] * s) / np.sum(s * s))
    rate = math.log(amps[0] / amps[1]) / 500
    assert abs(rate / (nu * k * k) - 1) < 3e-3


def test_kolmogorov_steady_profile_converges():
    """Steady Kolmogorov flow u_x = F0/(nu k^2) sin(k y) is an exact
    Navier-Stokes solution; the discrete error shrinks ~4x per doubling."""
    errs = []
    for ny in (12, 24):
        w = W.kolmogorov(shape=(1, ny, 1), F0=1e-6, nu=1 / 6, noise=0.0)
        L = _lat(w.omega, shape=w.shape, P=O.expand_separable(w.tables, w.shape))
        L.init_equilibrium(1.0, [0, 0, 0])
        L.run(int(40 * ny * ny / (1 / 6) / (4 * math.pi ** 2)) + 200)
        _, u = L.moments()
        k = 2 * math.pi / ny
        ua = 1e-6 / ((1 / 6) * k * k) * np.sin(k * np.arange(ny))
        errs.append(np.sqrt(np.sum((u[0] - ua) ** 2) / np.sum(ua ** 2)))
    assert errs[0] < 0.08
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def _duct_error(n, nu=1 / 6, Fx=1e-6):
    shape = (1, n, n)
    P = O.expand_separable([(np.array([Fx]), np.array([1.0]), np.array([1.0])),
                            (np.array([0.0]), np.array([1.0]), np.array([1.0])),
                            (np.array([0.0]), np.array([1.0]), np.array([1.0]))], shape)
    L = _lat(W.d3q27_omega(3 * nu + 0.5), shape=shape, wall=(0, 1, 1), P=P)
    L.init_equilibrium(1.0, [0, 0, 0])
    L.run(25 * n * n)
    _, u = L.moments()
    a = n / 2
    yy = np.arange(n) + 0.5 - a
    Y, Z = np.meshgrid(yy, yy, indexing="xy")
    ua = np.zeros_like(Y)
    for m in range(1, 60):
        b = (2 * m - 1) * math.pi / (2 * a)
        ua += ((-1) ** (m - 1) * (1 - np.cosh(b * Z) / math.cosh((2 * m - 1) * math.pi / 2))
               * np.cos(b * Y) / (2 * m - 1) ** 3)
    ua *= 16 * a * a * Fx / (nu * math.pi ** 3)
    return np.sqrt(np.sum((u[0].reshape(n, n) - ua) ** 2) / np.sum(ua ** 2))


def test_square_duct_fourier_series():
    """Sec. 6.4: duct of width 2a with four no-slip walls (halfway bounce-back),
    constant F_x; the steady profile converges to the Fourier series printed
    there at second order."""
    e8, e16 = _duct_error(8), _duct_error(16)
    assert e8 < 0.1 and e16 < 0.025, (e8, e16)
    assert 3.5 < e8 / e16 < 4.5, (e8, e16)

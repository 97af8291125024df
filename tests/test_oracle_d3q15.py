"""Pins of the oracle's D3Q15 flow step (Appendix A: Eqs. a1, 2A, 6A-13A and
the f^p expansion, with the three corrections named in the oracle's header).

Each pin is computed here from definitions (raw and central moments, the
basis of Eq. 2A) or from closed-form flows, never from the oracle's own
formulas."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests.moment_defs import D3Q15_E, W_D3Q15, K_d3q15, central, maxwell_central, raw

# omega[1] = omega_9 (trace), [2] = omega_4..8 (shear), [3] = omega_10..13, [4] = omega_14
RELAXED_3 = [(1, 2, 0), (2, 1, 0), (2, 0, 1), (1, 1, 1)]


def _lat(omega, shape=(1, 1, 1), wall=(0, 0, 0), P=None, as_printed=False):
    return O.OracleLattice(O.D3Q15, shape, wall=wall, omega=omega, P=P, as_printed=as_printed)


def _omega(tau, bulk=1.0, third=1.0, fourth=1.0):
    return (0.0, bulk, 1.0 / tau, third, fourth, 0.0, 0.0, 0.0, 0.0)


def _rand_f(rng, amp=0.1):
    return W_D3Q15 * (1 + amp * rng.standard_normal(15))


def _u(f, F=(0, 0, 0)):
    rho = f.sum()
    return np.array([raw(f, D3Q15_E, 1, 0, 0) + F[0] / 2, raw(f, D3Q15_E, 0, 1, 0) + F[1] / 2,
                     raw(f, D3Q15_E, 0, 0, 1) + F[2] / 2]) / rho


def test_velocity_set_and_basis():
    """Eq. a1 lists every velocity of D3Q15 once and the basis of Eq. 2A is
    orthogonal with the norms that fix the coefficients of Eqs. 6A and 12A."""
    assert np.array_equal(O.velocities(O.D3Q15), D3Q15_E.astype(int))
    assert len({tuple(e) for e in D3Q15_E}) == 15
    K = K_d3q15()
    G = K.T @ K
    assert np.array_equal(G, np.diag(np.diag(G)))
    assert list(np.diag(G)) == [15, 10, 10, 10, 8, 8, 8, 4, 12, 18, 160, 160, 160, 8, 1440]
    # Eq. 12A: only K_1 has a component along e_x, with weight 10
    assert list(K.T @ D3Q15_E[:, 0]) == [0, 10, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0]


def test_rest_weights_and_equilibrium_moments():
    L = _lat(_omega(0.8), shape=(2, 2, 2))
    L.init_equilibrium(1.0, [0, 0, 0])
    assert np.abs(L.f[:, 0] - W_D3Q15).max() < 3e-16
    rng = np.random.default_rng(30)
    for _ in range(10):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        L1 = _lat(_omega(0.8))
        L1.init_equilibrium(rho, u)
        f = L1.f[:, 0]
        assert abs(f.sum() - rho) < 1e-15
        assert np.abs(_u(f) - u).max() < 1e-15
        for a, b, c in [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1), (2, 2, 0)] + RELAXED_3:
            assert abs(central(f, D3Q15_E, u, a, b, c) - maxwell_central(rho, a, b, c)) < 2e-15


def test_rest_state_is_a_fixed_point_only_with_the_trace_correction():
    rng = np.random.default_rng(31)
    om = (0.0,) + tuple(rng.uniform(0.3, 1.9, 4)) + (0.0,) * 4
    fp = _lat(om).collide_node(W_D3Q15 * 1.3, [0, 0, 0], [0, 0, 0])
    assert np.abs(fp - W_D3Q15 * 1.3).max() < 2e-15  # roundoff of 32 g_14
    # g_9 as printed (no rho in its bracket) drives the rest state away
    fp = _lat(om, as_printed=True).collide_node(W_D3Q15 * 1.3, [0, 0, 0], [0, 0, 0])
    assert np.abs(fp - W_D3Q15 * 1.3).max() > 1e-2


def _collision_part(f, fp, Fpre, Fpost):
    """f^p minus the post-collision force part g_d K_d, g_d = (F_pre+F_post)_d/20."""
    K = K_d3q15()
    g = (np.asarray(Fpre) + np.asarray(Fpost)) / 20.0
    return fp - K[:, 1:4] @ g


def _central_half_forced(g, u, delta, a, b, c):
    """Central moment about u of the state whose raw moments are those of g
    except the first moments, which the pre-collision half force step has
    raised by delta (Eq. 8A acts on the first moments only): by the binomial
    expansion only the terms linear in a first moment change."""
    v = central(g, D3Q15_E, u, a, b, c)
    ux, uy, uz = -u[0], -u[1], -u[2]
    if a:
        v += a * ux ** (a - 1) * uy ** b * uz ** c * delta[0]
    if b:
        v += b * ux ** a * uy ** (b - 1) * uz ** c * delta[1]
    if c:
        v += c * ux ** a * uy ** b * uz ** (c - 1) * delta[2]
    return v


@pytest.mark.parametrize("printed", [False, True])
def test_every_moment_group_relaxes_with_its_rate(printed):
    """Central moments about u = (j + F_pre/2)/rho of the half-forced state
    (Eq. 8A), by definition: each relaxed moment of Eq. 6A goes to
    (1 - w) kappa + w kappa_eq, the fourth-order one towards the product of
    the post-collision kappa_xx and kappa_yy over rho.  With the printed sign
    of g_13 in f^p_12 (and the printed g_9) this fails."""
    rng = np.random.default_rng(32)
    worst = 0.0
    for _ in range(25):
        om = (0.0,) + tuple(rng.uniform(0.3, 1.9, 4)) + (0.0,) * 4
        f = _rand_f(rng)
        Fpre, Fpost = 1e-3 * rng.standard_normal(3), 1e-3 * rng.standard_normal(3)
        fp = _lat(om, as_printed=printed).collide_node(f, Fpre, Fpost)
        fc = _collision_part(f, fp, Fpre, Fpost)
        rho = f.sum()
        u = _u(f, Fpre)
        k = lambda g, a, b, c: _central_half_forced(g, u, Fpre / 2, a, b, c)  # noqa: E731
        errs = [abs(fc.sum() - rho)]
        for d in range(3):
            ed = [0, 0, 0]
            ed[d] = 1
            errs.append(abs(k(fc, *ed) - k(f, *ed)))
        for a, b, c in [(1, 1, 0), (1, 0, 1), (0, 1, 1)]:
            errs.append(abs(k(fc, a, b, c) - (1 - om[2]) * k(f, a, b, c)))
        d1 = lambda g: k(g, 2, 0, 0) - k(g, 0, 2, 0)  # noqa: E731
        d2 = lambda g: k(g, 2, 0, 0) + k(g, 0, 2, 0) - 2 * k(g, 0, 0, 2)  # noqa: E731
        tr = lambda g: k(g, 2, 0, 0) + k(g, 0, 2, 0) + k(g, 0, 0, 2)  # noqa: E731
        errs.append(abs(d1(fc) - (1 - om[2]) * d1(f)))
        errs.append(abs(d2(fc) - (1 - om[2]) * d2(f)))
        errs.append(abs(tr(fc) - ((1 - om[1]) * tr(f) + om[1] * rho)))
        for a, b, c in RELAXED_3:
            errs.append(abs(k(fc, a, b, c) - (1 - om[3]) * k(f, a, b, c)))
        target = k(fc, 2, 0, 0) * k(fc, 0, 2, 0) / rho
        errs.append(abs(k(fc, 2, 2, 0) - ((1 - om[4]) * k(f, 2, 2, 0) + om[4] * target)))
        worst = max(worst, max(errs))
        if printed:
            continue  # the printed f^p_12 also breaks mass conservation (by 2 g_13)
        # the whole step: mass kept, momentum changed by the mean force
        assert abs(fp.sum() - rho) < 1e-15
        j = np.array([raw(fp, D3Q15_E, 1, 0, 0), raw(fp, D3Q15_E, 0, 1, 0), raw(fp, D3Q15_E, 0, 0, 1)])
        j0 = np.array([raw(f, D3Q15_E, 1, 0, 0), raw(f, D3Q15_E, 0, 1, 0), raw(f, D3Q15_E, 0, 0, 1)])
        assert np.abs(j - j0 - (Fpre + Fpost) / 2).max() < 1e-16
    if printed:
        assert worst > 1e-3
    else:
        assert worst < 3e-15, worst


def test_unit_omega_collision_lands_on_the_equilibrium():
    """With every rate 1 and no force the collision maps any state to the
    equilibrium at its own (rho, u) (built from Maxwellian central moments by
    the oracle's separate equilibrium routine)."""
    rng = np.random.default_rng(33)
    L = _lat(_omega(1.0))
    for _ in range(10):
        f = _rand_f(rng)
        fp = L.collide_node(f, [0, 0, 0], [0, 0, 0])
        E = _lat(_omega(1.0))
        E.init_equilibrium(f.sum(), _u(f))
        assert np.abs(fp - E.f[:, 0]).max() < 1.5e-15


def test_printed_expansion_is_K_times_g():
    """The populations differ from K g (Eq. 2A) only through the corrected
    sign: recover g from f^p - f with the orthogonal basis and check that K g
    reproduces the change and that g_0 = 0, g_1..3 = (F_pre + F_post)/20."""
    rng = np.random.default_rng(34)
    K = K_d3q15()
    for _ in range(10):
        om = (0.0,) + tuple(rng.uniform(0.3, 1.9, 4)) + (0.0,) * 4
        f = _rand_f(rng)
        Fpre, Fpost = 1e-3 * rng.standard_normal(3), 1e-3 * rng.standard_normal(3)
        fp = _lat(om).collide_node(f, Fpre, Fpost)
        g = (K.T @ (fp - f)) / np.diag(K.T @ K)
        assert np.abs(K @ g - (fp - f)).max() < 1e-16
        assert abs(g[0]) < 1e-17
        assert np.abs(g[1:4] - (Fpre + Fpost) / 20).max() < 1e-17


@pytest.mark.parametrize("axis", [1, 2])
def test_shear_wave_decay_gives_viscosity(axis):
    n = 48
    tau = 0.9
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    shape = [2, 2, 2]
    shape[axis] = n
    L = _lat(_omega(tau), shape=tuple(shape))
    idx = np.indices(shape[::-1]).reshape(3, -1)[::-1]
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


def _duct_error(n, nu=1 / 6, Fx=1e-6):
    shape = (1, n, n)
    P = np.zeros((3, n * n))
    P[0] = Fx
    L = _lat(_omega(3 * nu + 0.5), shape=shape, wall=(0, 1, 1), P=P)
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
    """The paper's D3Q15 demonstration flow (Sec. 6.4 series): a duct with four
    halfway bounce-back walls and constant F_x converges to the Fourier series
    at second order."""
    e8, e16 = _duct_error(8), _duct_error(16)
    assert e8 < 0.1 and e16 < 0.025, (e8, e16)
    assert 3.5 < e8 / e16 < 4.5, (e8, e16)

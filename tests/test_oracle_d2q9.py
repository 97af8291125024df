"""Pins of the oracle's D2Q9 flow step (Sec. 4) against facts that the paper
and the mathematics fix, independently of the oracle's own formulas."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_10247_gb300 import workloads as W
from tests.moment_defs import D2Q9_E, K_d2q9, W_D2Q9, central, maxwell_central, raw


def _lat(omega, shape=(1, 1, 1), wall=(0, 0, 0)):
    return O.OracleLattice(O.D2Q9, shape, wall=wall, omega=omega)


def _rand_f(rng, amp=0.05):
    return W_D2Q9 * (1.0 + amp * rng.standard_normal(9))


def test_basis_matches_eq17_and_eq29():
    K = K_d2q9()
    G = K.T @ K
    # Eq. 17 basis is orthogonal; <K_1|e_x> = 6 gives the factor of Eq. 29.
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.allclose(np.diag(G), [9, 6, 6, 36, 4, 4, 12, 12, 36])


def test_collision_change_is_K_g_with_eq31_force():
    """f^p - f = K g with g_0 = 0 and g_1,2 = (F_pre + F_post)/12 (Eqs. 22a, 27-31)."""
    rng = np.random.default_rng(0)
    K = K_d2q9()
    for _ in range(50):
        om = (0, 0, 0) + tuple(rng.uniform(0.2, 1.9, 6))
        L = _lat(om)
        f = _rand_f(rng)
        Fpre, Fpost = 1e-3 * rng.standard_normal(2), 1e-3 * rng.standard_normal(2)
        g = np.linalg.solve(K, L.collide_node(f, Fpre, Fpost) - f)
        assert abs(g[0]) < 1e-16
        assert np.allclose(g[1:3], (Fpre + Fpost) / 12.0, rtol=1e-12, atol=1e-18)


def test_unit_omega_reaches_eq20_equilibrium():
    """omega = 1 and F = 0: every post-collision central moment equals Eq. 20."""
    rng = np.random.default_rng(1)
    L = _lat(W.d2q9_omega(1.0))
    for _ in range(50):
        f = _rand_f(rng, 0.1)
        fp = L.collide_node(f, [0, 0], [0, 0])
        rho = f.sum()
        u = np.array([raw(f, D2Q9_E, 1, 0), raw(f, D2Q9_E, 0, 1), 0.0]) / rho
        for a in range(3):
            for b in range(3):
                got = central(fp, D2Q9_E, u, a, b)
                assert abs(got - maxwell_central(rho, a, b)) < 2e-15, (a, b, got)


def test_general_omega_relaxes_central_moments():
    """F = 0, random omega: the cascaded collision relaxes the central moments
    (Sec. 4): trace with omega_3, kxx-kyy with omega_4, kxy with omega_5,
    kxxy with omega_6, kxyy with omega_7, kxxyy with omega_8."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        w = rng.uniform(0.2, 1.9, 6)
        L = _lat((0, 0, 0) + tuple(w))
        f = _rand_f(rng, 0.1)
        fp = L.collide_node(f, [0, 0], [0, 0])
        rho = f.sum()
        u = np.array([raw(f, D2Q9_E, 1, 0), raw(f, D2Q9_E, 0, 1), 0.0]) / rho
        k = lambda g, a, b: central(g, D2Q9_E, u, a, b)  # noqa: E731
        w3, w4, w5, w6, w7, w8 = w
        T, Tp = k(f, 2, 0) + k(f, 0, 2), k(fp, 2, 0) + k(fp, 0, 2)
        assert abs(Tp - (T + w3 * (2 * rho / 3 - T))) < 2e-15
        D, Dp = k(f, 2, 0) - k(f, 0, 2), k(fp, 2, 0) - k(fp, 0, 2)
        assert abs(Dp - (1 - w4) * D) < 2e-15
        assert abs(k(fp, 1, 1) - (1 - w5) * k(f, 1, 1)) < 2e-15
        assert abs(k(fp, 2, 1) - (1 - w6) * k(f, 2, 1)) < 2e-15
        assert abs(k(fp, 1, 2) - (1 - w7) * k(f, 1, 2)) < 2e-15
        assert abs(k(fp, 2, 2) - (k(f, 2, 2) + w8 * (rho / 9 - k(f, 2, 2)))) < 2e-15
        # first moments unchanged without force
        assert abs(k(fp, 1, 0)) < 1e-15 and abs(k(fp, 0, 1)) < 1e-15


def test_generic_procedure_equals_paper_formulas():
    """The generic central-moment procedure (used for D3Q27) reproduces
    Eqs. 23, 31 and 32 on D2Q9, with forcing and arbitrary omega."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        L = _lat((0, 0, 0) + tuple(rng.uniform(0.2, 1.9, 6)))
        f = _rand_f(rng)
        Fpre, Fpost = 1e-3 * rng.standard_normal(2), 1e-3 * rng.standard_normal(2)
        a = L.collide_node(f, Fpre, Fpost)
        b = L.collide_node(f, Fpre, Fpost, generic=True)
        assert np.abs(a - b).max() < 2e-15


def test_equilibrium_is_fixed_point_and_has_eq20_moments():
    rng = np.random.default_rng(4)
    L = _lat((0, 0, 0) + tuple(rng.uniform(0.2, 1.9, 6)), shape=(5, 4, 1))
    rho = 1.0 + 0.01 * rng.standard_normal(L.N)
    u = 0.05 * rng.standard_normal((2, L.N))
    L.init_equilibrium(rho, u)
    for i in range(L.N):
        fi = L.f[:, i]
        ui = np.array([u[0, i], u[1, i], 0.0])
        assert abs(fi.sum() - rho[i]) < 1e-15
        for a in range(3):
            for b in range(3):
                assert abs(central(fi, D2Q9_E, ui, a, b) - maxwell_central(rho[i], a, b)) < 1e-15
        fp = L.collide_node(fi, [0, 0], [0, 0])
        assert np.abs(fp - fi).max() < 1e-15
    # rest weights (4/9, 1/9, 1/36)
    L.init_equilibrium(1.0, [0.0, 0.0])
    assert np.allclose(L.f[:, 0], W_D2Q9, rtol=0, atol=4e-16)


def test_streaming_moves_and_bounces_back():
    """All omega = 0 and F = 0 make the collision the identity, so a step is a
    pure stream (Eq. 22b) with periodic wrap in x and halfway bounce-back at
    the y walls (Sec. 6.1)."""
    L = _lat((0.0,) * 9, shape=(4, 3, 1), wall=(0, 1, 0))
    opp = [0, 3, 4, 1, 2, 7, 8, 5, 6]
    for a in range(9):
        for (x, y) in [(0, 0), (3, 2), (1, 1)]:
            # a rest background keeps the density positive; it streams onto itself
            L.f = np.repeat(W_D2Q9[:, None], L.N, axis=1)
            L.f[a, x + 4 * y] += 1.0
            L.run(1)
            L.f -= W_D2Q9[:, None]
            tx, ty = x + int(D2Q9_E[a, 0]), y + int(D2Q9_E[a, 1])
            g = np.zeros((9, L.N))
            if 0 <= ty < 3:
                g[a, (tx % 4) + 4 * ty] = 1.0
            else:
                g[opp[a], x + 4 * y] = 1.0
            assert np.abs(L.f - g).max() < 1e-15, (a, x, y)


def _poiseuille_steady(ny, tau, Fx, steps_max=400000, tol=1e-13, start_parabolic=False):
    w = W.poiseuille(ny=ny, tau=tau, Fx=Fx)
    L = O.OracleLattice(O.D2Q9, w.shape, wall=w.wall, omega=w.omega,
                        P=O.expand_separable(w.tables, w.shape))
    u0 = np.zeros((2, L.N))
    if start_parabolic:  # only shortens the transient; the steady state is unique
        y = np.repeat(np.arange(ny), w.shape[0])
        u0[0] = Fx / (2 * (tau - 0.5) / 3.0) * (y + 0.5) * (ny - 0.5 - y)
    L.init_equilibrium(1.0, u0)
    prev = None
    while L.t < steps_max:
        L.run(500)
        rho, u = L.moments()
        if prev is not None and np.abs(u[0] - prev).max() < tol * np.abs(u[0]).max():
            break
        prev = u[0].copy()
    return L, rho, u


def test_poiseuille_profile_mass_and_slip():
    """Config 1: channel 3 x 33, tau = 0.8, Fx = 1e-6 (Sec. 6.1).  At steady
    state the discrete momentum balance fixes the interior second difference
    of u_x to -F/(rho nu); the profile is the parabola with walls at y = -1/2
    and ny - 1/2 plus a uniform slip; mass is conserved exactly."""
    ny, tau, Fx = 33, 0.8, 1e-6
    nu = (tau - 0.5) / 3.0
    L, rho, u = _poiseuille_steady(ny, tau, Fx)
    ux = u[0].reshape(ny, 3)
    assert np.abs(ux - ux[:, :1]).max() < 1e-18  # x-invariant
    prof = ux[:, 0]
    d2 = prof[2:] - 2 * prof[1:-1] + prof[:-2]
    assert np.abs(d2 + Fx / nu).max() < 1e-10 * Fx / nu
    assert np.abs(prof - prof[::-1]).max() < 1e-12 * prof.max()
    y = np.arange(ny)
    para = Fx / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    slip = prof - para
    assert np.abs(slip - slip.mean()).max() < 1e-9 * prof.max()
    assert abs(np.sum(rho) - L.N) < 1e-13 * L.N
    assert np.abs(u[1]).max() < 1e-14


def test_poiseuille_second_order_diffusive_scaling():
    """Sec. 6.1 grid convergence: tau fixed, the error against the parabola
    falls with slope 2 (the paper prints 2.00 for tau = 0.55, Re = 100)."""
    golden = dict(line.split("=") for line in open(
        __file__.replace("test_oracle_d2q9.py", "golden/poiseuille_convergence.txt"))
        if "=" in line and not line.startswith("#"))
    tau = float(golden["tau"])
    Re = float(golden["Re"])
    nu = (tau - 0.5) / 3.0
    errs, Hs = [], []
    for ny in (15, 31, 61):
        Umax = Re * nu / ny
        Fx = 8 * nu * Umax / ny ** 2
        L, rho, u = _poiseuille_steady(ny, tau, Fx, steps_max=2_000_000, tol=1e-9,
                                       start_parabolic=True)
        y = np.arange(ny)
        ua = Fx / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
        uc = u[0].reshape(ny, 3)[:, 0]
        errs.append(np.sqrt(np.sum((uc - ua) ** 2) / np.sum(ua ** 2)))
        Hs.append(ny)
        # the context API's l2 error of the whole velocity field (three
        # identical columns, u_y ~ 0) against the parabola gives the same value
        ctx = O.OracleContext(O.D2Q9, (3, ny, 1), omega=W.d2q9_omega(tau), wall=(0, 1, 0))
        assert ctx.set_force(L.P) == O.REF_OK and ctx.set_populations(L.f, 0) == O.REF_OK
        ref = np.zeros((2, 3 * ny))
        ref[0] = np.repeat(ua, 3)
        rc, out = ctx.l2_error(ref, field=1)
        assert rc == O.REF_OK and abs(out[2] - errs[-1]) <= 1e-9 * errs[-1]
    slope = np.polyfit(np.log(Hs), np.log(errs), 1)[0]
    assert abs(-slope - float(golden["slope"])) < 0.1, (errs, slope)


def test_momentum_budget_with_time_dependent_force():
    """Periodic box: total momentum changes by exactly sum (F_pre+F_post)/2 per
    step (Eq. 27 with the Sec. 6.3 trapezoid halves); mass is conserved."""
    rng = np.random.default_rng(5)
    shape = (6, 5, 1)
    tables = [(rng.standard_normal(6) * 1e-4, rng.standard_normal(5), np.array([1.0])),
              (np.array([2e-5]), np.array([1.0]), np.array([1.0]))]
    P = O.expand_separable(tables, shape)
    env = lambda t: np.cos(0.01 * t)  # noqa: E731
    L = O.OracleLattice(O.D2Q9, shape, omega=W.d2q9_omega(0.7), P=P, envelope=env)
    L.init_equilibrium(1.0 + 0.01 * rng.standard_normal(L.N), 0.01 * rng.standard_normal((2, L.N)))
    j0 = (L.f[:, :, None] * D2Q9_E[:, None, :2]).sum((0, 1))
    m0 = L.f.sum()
    pairs = O.envelope_pairs(env, 0, 20)
    L.run(20)
    j1 = (L.f[:, :, None] * D2Q9_E[:, None, :2]).sum((0, 1))
    dj = sum(0.5 * (pairs[2 * k] + pairs[2 * k + 1]) for k in range(20)) * P.sum(1)
    assert np.allclose(j1 - j0, dj, rtol=1e-10, atol=1e-17)
    assert abs(L.f.sum() - m0) < 1e-13


def test_shear_wave_decay_gives_viscosity():
    """A shear wave u_x = U sin(k y) decays at the Navier-Stokes rate nu k^2
    with nu = (tau - 1/2)/3 (Sec. 4 and Sec. 6 preamble)."""
    ny = 64
    tau = 0.9
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / ny
    y = np.repeat(np.arange(ny), 2)
    L = O.OracleLattice(O.D2Q9, (2, ny, 1), omega=W.d2q9_omega(tau))
    U = 1e-4
    u = np.stack([U * np.sin(k * y), np.zeros_like(y, dtype=float)])
    L.init_equilibrium(1.0, u)
    L.run(200)
    _, u1 = L.moments()
    a1 = np.sum(u1[0] * np.sin(k * y)) / np.sum(np.sin(k * y) ** 2)
    L.run(800)
    _, u2 = L.moments()
    a2 = np.sum(u2[0] * np.sin(k * y)) / np.sum(np.sin(k * y) ** 2)
    rate = np.log(a1 / a2) / 800
    assert abs(rate / (nu * k * k) - 1) < 2e-3

"""Pins of the oracle's D2Q5 passive-scalar step with source (Sec. 5)."""
import math

import numpy as np

from oracle import oracle as O
from paper_1806_10247_gb300 import workloads as W
from tests.moment_defs import D2Q5_E, L_d2q5, W_D2Q5, central, maxwell_central, raw


def _lat(omega, shape=(1, 1, 1), as_printed=False):
    return O.OracleLattice(O.D2Q5, shape, omega=omega, as_printed=as_printed)


def test_basis_eq35():
    L = L_d2q5()
    G = L.T @ L
    assert np.allclose(G, np.diag([5, 2, 2, 20, 4]))
    # <L_beta|1> = 5 delta_beta0: the factor 5 of Eqs. 45-47
    assert np.allclose(L.sum(0), [5, 0, 0, 0, 0])


def _moments(g, u):
    return {(a, b): central(g, D2Q5_E, u, a, b) for (a, b) in [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2)]}


def test_unit_omega_reaches_eq39_equilibrium_and_printed_sign_does_not():
    """omega = 1, S = 0: the post-collision central moments about the advecting
    velocity equal Eq. 39.  Eq. 41 exactly as printed misses this by O(u^2 phi)."""
    rng = np.random.default_rng(10)
    for _ in range(50):
        g = W_D2Q5 * (1 + 0.1 * rng.standard_normal(5))
        u = np.array([0.1 * rng.standard_normal(), 0.1 * rng.standard_normal(), 0.0])
        phi = g.sum()
        gp = _lat(W.d2q5_omega(1.0)).collide_node(g, [0.0], [0.0], uadv=u[:2])
        m = _moments(gp, u)
        for k, v in m.items():
            assert abs(v - maxwell_central(phi, *k)) < 2e-15, (k, v)
        bad = _lat(W.d2q5_omega(1.0), as_printed=True).collide_node(g, [0.0], [0.0], uadv=u[:2])
        mb = _moments(bad, u)
        err = abs(mb[(2, 0)] + mb[(0, 2)] - 2 * phi / 3)
        assert err > 0.5 * (u[0] ** 2 + u[1] ** 2) * phi


def test_general_omega_relaxes_central_moments():
    rng = np.random.default_rng(11)
    for _ in range(50):
        w = rng.uniform(0.2, 1.9, 4)
        L = _lat((0,) + tuple(w) + (0, 0, 0, 0))
        g = W_D2Q5 * (1 + 0.1 * rng.standard_normal(5))
        u = np.array([0.1 * rng.standard_normal(), 0.1 * rng.standard_normal(), 0.0])
        gp = L.collide_node(g, [0.0], [0.0], uadv=u[:2])
        phi = g.sum()
        m, mp = _moments(g, u), _moments(gp, u)
        assert abs(mp[(0, 0)] - phi) < 1e-15
        assert abs(mp[(1, 0)] - (1 - w[0]) * m[(1, 0)]) < 2e-15
        assert abs(mp[(0, 1)] - (1 - w[1]) * m[(0, 1)]) < 2e-15
        T, Tp = m[(2, 0)] + m[(0, 2)], mp[(2, 0)] + mp[(0, 2)]
        assert abs(Tp - (T + w[2] * (2 * phi / 3 - T))) < 2e-15
        D, Dp = m[(2, 0)] - m[(0, 2)], mp[(2, 0)] - mp[(0, 2)]
        assert abs(Dp - (1 - w[3]) * D) < 2e-15


def test_source_half_steps():
    """Eqs. 43-47: the zeroth moment gains (S_pre+S_post)/2, and the first-order
    relaxation sees the half-sourced scalar phi^o + S_pre/2."""
    rng = np.random.default_rng(12)
    for _ in range(50):
        w = rng.uniform(0.2, 1.9, 4)
        L = _lat((0,) + tuple(w) + (0, 0, 0, 0))
        g = W_D2Q5 * (1 + 0.1 * rng.standard_normal(5))
        u = 0.1 * rng.standard_normal(2)
        Spre, Spost = 1e-3 * rng.standard_normal(2)
        gp = L.collide_node(g, [Spre], [Spost], uadv=u)
        assert abs(gp.sum() - (g.sum() + (Spre + Spost) / 2)) < 1e-15
        phi = g.sum() + Spre / 2
        kx = raw(g, D2Q5_E, 1, 0)
        assert abs(raw(gp, D2Q5_E, 1, 0) - (kx + w[0] * (phi * u[0] - kx))) < 1e-15


def test_diffusion_rate_and_advection_speed():
    """A Fourier mode of phi decays at D k^2 with D = (tau_phi - 1/2)/3 and
    travels with the advecting velocity (Eq. 33 without source)."""
    N = 64
    tau = 0.8
    D = (tau - 0.5) / 3
    k = 2 * np.pi / N
    ux = 0.02
    x = np.tile(np.arange(N), 2)
    L = O.OracleLattice(O.D2Q5, (N, 2, 1), omega=W.d2q5_omega(tau),
                        uadv=np.stack([np.full(2 * N, ux), np.zeros(2 * N)]))
    L.init_equilibrium(1.0 + 1e-3 * np.sin(k * x), [ux, 0.0])
    amps = []
    for t in (200, 1200):
        L.run(t - L.t)
        phi = L.moments() - 1.0
        c = np.sum(phi * np.exp(-1j * k * x)) / (N)  # complex amplitude of the mode
        amps.append(c)
    rate = np.log(abs(amps[0]) / abs(amps[1])) / 1000
    assert abs(rate / (D * k * k) - 1) < 5e-3
    dphase = -np.angle(amps[1] / amps[0])
    assert abs(dphase / (k * ux * 1000) - 1) < 5e-3


def _closed_form(c, t, N):
    return W.cde_closed_form(c, t)


def _run_cde(c):
    w = W.cde_workload(c)
    N = c.N
    L = O.OracleLattice(O.D2Q5, w.shape, omega=w.omega, P=O.expand_separable(w.tables, w.shape),
                        envelope=w.envelope,
                        uadv=np.stack([np.full(w.nodes, c.ux), np.full(w.nodes, c.uy)]))
    L.init_equilibrium(1.0, [c.ux, c.uy])
    L.run(c.T)
    phi = L.moments().reshape(N, N) - 1.0
    ref = _closed_form(c, c.T, N)
    return np.sqrt(np.sum((phi - ref) ** 2) / np.sum(ref ** 2))


def test_manufactured_source_second_order():
    """Config 2 recipe under diffusive scaling: the l2 error against the closed
    form falls by ~4 per grid doubling (second order)."""
    cases = W.cde_sweep_params(sizes=(32, 64, 128))
    errs = [_run_cde(c) for c in cases]
    assert errs[0] < 2e-2
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - 2.0) < 0.15 for o in orders), (errs, orders)

"""Pins of the oracle's force step against the paper's analytic benchmark
flows (Sec. 6.2, 6.3, 6.5): a spatially varying force (Hartmann), a
time-periodic force through the trapezoid envelope (Womersley) and a force
varying in both directions and both components (four-rolls mill, convective
scaling).  Each converges to its closed form at second order."""
import math

import numpy as np

from oracle import oracle as O
from paper_1806_10247_gb300 import workloads as W


def _oracle(w):
    P = O.expand_separable(w.tables, w.shape)
    L = O.OracleLattice(w.lattice, w.shape, wall=w.wall, omega=w.omega, P=P, envelope=w.envelope)
    L.init_equilibrium(w.rho0, w.u0)
    return L


def _l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def test_hartmann_profile_second_order():
    errs = []
    for ny in (16, 32):
        w = W.hartmann(ny=ny, Ha=3.0, tau=0.8)
        L = _oracle(w)
        L.run(int(12 * ny * ny / w.meta["nu"] / math.pi ** 2))
        _, u = L.moments()
        errs.append(_l2(u[0].reshape(ny, -1)[:, 0], W.hartmann_profile(w)))
        # the profile is uniform along the periodic axis
        assert np.ptp(u[0].reshape(ny, -1), axis=1).max() < 1e-15
    assert errs[0] < 0.02, errs
    assert 3.6 < errs[0] / errs[1] < 4.4, errs


def test_womersley_periodic_state_second_order():
    """Diffusive scaling (T ~ ny^2, fixed tau, Wo = 1.1); the profile is compared
    at four phases of the fifth period."""
    worst = []
    for ny in (16, 32):
        T = int(2000 * (ny / 16) ** 2)
        w = W.womersley(ny=ny, period=T, tau=1.0)
        L = _oracle(w)
        L.run(5 * T)
        e = 0.0
        for _ in range(4):
            _, u = L.moments()
            e = max(e, _l2(u[0].reshape(ny, -1)[:, 0], W.womersley_profile(w, L.t)))
            L.run(T // 4)
        worst.append(e)
    assert worst[0] < 0.015, worst
    assert 3.6 < worst[0] / worst[1] < 4.4, worst


def test_four_rolls_mill_convective_scaling_second_order():
    """u0 = 0.01 and nu = 0.0011 (domain 2 pi) under convective scaling,
    started from the analytic field: the steady state's l2 error falls ~4x
    per doubling of N (second order in space and time)."""
    errs = []
    for N in (24, 48):
        w = W.four_rolls(N)
        L = _oracle(w)
        L.run(int(3 / (w.meta["nu"] * w.meta["k"] ** 2)))
        _, u = L.moments()
        ua = W.four_rolls_velocity(w)
        errs.append(max(_l2(u[0], ua[0]), _l2(u[1], ua[1])))
    assert errs[0] < 0.015, errs
    assert 3.6 < errs[0] / errs[1] < 4.6, errs

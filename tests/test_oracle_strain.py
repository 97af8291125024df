"""Pins of the oracle's strain-rate tensor from the non-equilibrium second
moments (Sec. 6.6) against closed-form flows."""
import math

import numpy as np

from oracle import oracle as O
from paper_1806_10247_gb300 import workloads as W


def _run(w, u_start, steps):
    P = O.expand_separable(w.tables, w.shape)
    L = O.OracleLattice(w.lattice, w.shape, wall=w.wall, omega=w.omega, P=P)
    L.init_equilibrium(1.0, u_start)
    L.run(steps)
    return L


def test_poiseuille_shear_rate_is_exact():
    """The discrete Poiseuille solution is a parabola (plus a uniform slip), so
    S_xy = (1/2) du/dy = F (ny - 1 - 2y) / (4 nu) exactly; the normal
    components vanish to O(u^2)."""
    ny, tau, F = 33, 0.8, 1e-6
    w = W.poiseuille(ny=ny, tau=tau, Fx=F)
    ua = np.tile(W.poiseuille_parabola(ny, tau, F)[:, None], (1, 3)).reshape(-1)
    L = _run(w, np.stack([ua, np.zeros_like(ua)]), int(8 * ny * ny / 0.1))
    S = L.strain_rate()
    nu = (tau - 0.5) / 3
    Sa = F / (4 * nu) * (ny - 1 - 2 * np.arange(ny))
    sxy = S[2].reshape(ny, 3)[:, 0]
    assert np.abs(sxy - Sa).max() < 1e-10 * np.abs(Sa).max()
    assert np.abs(S[:2]).max() < 1e-3 * np.abs(Sa).max()


def test_kolmogorov_2d_shear_rate_second_order():
    """Steady u_x = F0/(nu k^2) sin(ky): S_xy = F0 cos(ky) / (2 nu k), second order."""
    errs = []
    for ny in (16, 32):
        nu, F0, k = 1 / 6, 1e-6, 2 * math.pi / ny
        one = np.array([1.0])
        y = np.arange(ny, dtype=float)
        w = W.Workload(name="k2d", lattice=W.D2Q9, shape=(3, ny, 1), wall=(0, 0, 0),
                       omega=W.d2q9_omega(3 * nu + 0.5),
                       tables=[(one, F0 * np.sin(k * y), one), (np.array([0.0]), one, one)])
        ua = np.tile((F0 / (nu * k * k) * np.sin(k * y))[:, None], (1, 3)).reshape(-1)
        L = _run(w, np.stack([ua, np.zeros_like(ua)]), int(10 / (nu * k * k)))
        S = L.strain_rate()
        Sa = 0.5 * F0 / (nu * k) * np.cos(k * y)
        sxy = S[2].reshape(ny, 3)[:, 0]
        errs.append(float(np.sqrt(np.sum((sxy - Sa) ** 2) / np.sum(Sa ** 2))))
    assert errs[0] < 0.02 and 3.6 < errs[0] / errs[1] < 4.4, errs


def test_kolmogorov_3d_shear_rate_and_symmetry():
    """D3Q27: S_xy of the steady Kolmogorov flow at second order; the other
    off-diagonal components vanish."""
    errs = []
    for ny in (12, 24):
        w = W.kolmogorov(shape=(1, ny, 1), F0=1e-6, nu=1 / 6, noise=0.0)
        k = 2 * math.pi / ny
        L = _run(w, [0, 0, 0], int(40 * ny * ny / (1 / 6) / (4 * math.pi ** 2)) + 200)
        S = L.strain_rate()
        Sa = 0.5 * 1e-6 / ((1 / 6) * k) * np.cos(k * np.arange(ny))
        errs.append(float(np.sqrt(np.sum((S[3] - Sa) ** 2) / np.sum(Sa ** 2))))
        assert np.abs(S[4:]).max() < 1e-12
    assert errs[0] < 0.08 and 3.5 < errs[0] / errs[1] < 4.5, errs

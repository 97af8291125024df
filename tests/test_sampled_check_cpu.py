"""The sampled one-step check used at full size on the GPU (collide the pull
sources of sampled nodes with the oracle's single-node collision, stream them
in, compare with the next state), run on the CPU against a lattice that the
oracle itself steps.  Both sides are then the oracle, so the check must agree
to rounding; a wrong pull source, wall reflection, source/force value or
advecting velocity in the helper shows up as an O(1) relative error.  A
planted mistake (the stand-in skips the source) must be caught."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_10247_gb300 import workloads as W
from tests import gpu_helpers as H


class _OracleLattice:
    """The few calls of a library lattice the sampled check makes, backed by
    the oracle's whole-grid context."""

    def __init__(self, w, drop_source=False):
        self.lattice = w.lattice
        self.C = O.OracleContext(w.lattice, w.shape, omega=w.omega, wall=w.wall)
        assert self.C.status == 0
        assert self.C.init_equilibrium(w.rho0, w.u0) == 0
        P = O.expand_separable(w.tables, w.shape) if w.tables is not None else None
        if w.lattice == O.D2Q5:
            u = np.asarray(w.u0, np.float64)
            assert self.C.set_velocity(np.stack([np.full(w.nodes, u[0]), np.full(w.nodes, u[1])])) == 0
            if P is not None and not drop_source:
                assert self.C.set_source(P[0]) == 0
        elif P is not None and not drop_source:
            assert self.C.set_force(P) == 0

    def get_populations(self):
        rc, f = self.C.populations()
        assert rc == 0
        return f

    def step(self, n):
        assert self.C.step(n) == 0

    @property
    def t(self):
        rc, t = self.C.get_step()
        assert rc == 0
        return t

    def sync(self):
        pass


def _d2q5(nx=13, ny=11):
    x, y = np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64)
    return W.Workload(name="d2q5_small", lattice=W.D2Q5, shape=(nx, ny, 1), wall=(0, 0, 0),
                      omega=W.d2q5_omega(0.9), rho0=1.0, u0=(0.03, -0.02, 0.0),
                      tables=[(1e-2 * np.sin(2 * math.pi * x / nx), np.cos(2 * math.pi * y / ny), np.array([1.0]))])


def _d2q9_walls(nx=9, ny=7):
    y = np.arange(ny, dtype=np.float64)
    return W.Workload(name="d2q9_small", lattice=W.D2Q9, shape=(nx, ny, 1), wall=(0, 1, 0),
                      omega=W.d2q9_omega(0.7), rho0=1.0, u0=(0.0, 0.0, 0.0),
                      tables=[(np.array([1e-3]), 1.0 + 0.1 * y, np.array([1.0])),
                              (np.array([2e-4]), np.array([1.0]), np.array([1.0]))])


@pytest.mark.parametrize("make", [_d2q5, _d2q9_walls, lambda: W.kolmogorov(n=6)], ids=["d2q5", "d2q9_walls", "d3q27"])
def test_sampled_check_agrees_with_the_oracle_stepping_itself(make):
    w = make()
    G = _OracleLattice(w)
    G.step(3)
    worst = H.one_step_sampled(w, G, samples=40, seed=3, tol=1e-13)
    assert worst <= 1e-13


def test_sampled_check_catches_a_missing_source():
    w = _d2q5()
    G = _OracleLattice(w, drop_source=True)
    G.step(3)
    with pytest.raises(AssertionError):
        H.one_step_sampled(w, G, samples=40, seed=3, tol=1e-9)


def test_d2q5_collision_without_advecting_velocity_is_refused():
    L = O.OracleLattice(O.D2Q5, (1, 1, 1), omega=W.d2q5_omega(0.9))
    with pytest.raises(ValueError):
        L.collide_node(np.full(5, 0.2), [0.0], [0.0])

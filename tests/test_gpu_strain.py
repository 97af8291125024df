"""Strain rate from the non-equilibrium second moments (Sec. 6.6) on the GPU
against the oracle's definition, and the viscous-heating source it drives on
a scalar lattice."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W
from tests.gpu_helpers import compare_state, oracle_from_workload
from tests.test_gpu_parity import _pair_full, _random_workload

pytestmark = pytest.mark.gpu


def _tol(w, R):
    # S is -(3 omega / (2 rho0)) times sums of O(rho) terms: 1e-12 of that scale
    return 1e-12 * 1.5 * max(w.omega) * np.abs(R.f.sum(axis=0)).max()


@pytest.mark.parametrize("lattice,shape,wall", [
    (W.D2Q9, (13, 9, 1), (0, 1, 0)),
    (W.D3Q27, (7, 6, 5), (1, 0, 1)),
    (W.D3Q15, (6, 7, 5), (0, 1, 1)),
])
def test_strain_rate_matches_oracle(lattice, shape, wall):
    w, full = _random_workload(lattice, shape, wall, seed=70 + shape[0], kind="full")
    G, R = _pair_full(w, full)
    G.step(7)
    R.run(7)
    compare_state(G, R)
    for rho0 in (1.0, 1.3):
        Sg = G.strain_rate(rho0)
        Sr = R.strain_rate(rho0)
        assert Sg.shape == Sr.shape
        assert np.abs(Sg - Sr).max() <= _tol(w, R), np.abs(Sg - Sr).max()


def test_strain_rate_reduced_precision_close_to_fp64():
    w = W.kolmogorov(shape=(8, 24, 8), F0=1e-5, nu=0.05, noise=1e-4)
    a = lbm.from_workload(w)
    b = lbm.from_workload(w, storage=lbm.FP32_DEV)
    a.step(200)
    b.step(200)
    Sa, Sb = a.strain_rate(), b.strain_rate()
    assert np.sqrt(np.sum((Sa - Sb) ** 2) / np.sum(Sa ** 2)) < 1e-4


def test_viscous_heating_source_from_flow():
    """scalar.set_source_from_strain(flow, coef) sets the scalar's source
    shape to coef * S:S of the flow; one scalar step then equals the oracle's
    step with that source."""
    ny = 17
    flow_w = W.poiseuille(ny=ny, nx=5, tau=0.7, Fx=1e-5)
    flow = lbm.from_workload(flow_w)
    flow.step(300)
    scal_w = W.Workload(name="heat", lattice=W.D2Q5, shape=(5, ny, 1), wall=(0, 1, 0),
                        omega=W.d2q5_omega(0.782), rho0=0.5, u0=(0.0, 0.0, 0.0))
    scal = lbm.from_workload(scal_w)
    coef = 2 * 0.1 / 0.01
    scal.set_source_from_strain(flow, coef)
    S = flow.strain_rate()
    P = coef * (S[0] ** 2 + S[1] ** 2 + 2 * S[2] ** 2)
    R = oracle_from_workload(scal_w)
    R.P = np.ascontiguousarray(P[None, :])
    scal.step(3)
    R.run(3)
    compare_state(scal, R)
    phi = scal.moments()
    assert phi.sum() > 0.5 * scal.N  # heat was added
    with pytest.raises(lbm.LBMError):
        scal.set_source_from_strain(lbm.from_workload(W.poiseuille(ny=9)), coef)  # grid mismatch

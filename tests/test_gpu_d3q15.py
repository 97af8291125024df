"""GPU parity of the D3Q15 step (Appendix A) against the FP64 oracle: random
states, walls on every axis combination, ragged extents, separable and full
force fields with a time envelope, the paper's duct case, batched launches,
and the full-size launch of the bench on sampled nodes."""
import numpy as np
import pytest

from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W
from tests.gpu_helpers import compare_state, oracle_from_workload
from tests.gpu_helpers import one_step_sampled
from tests.test_gpu_parity import _advance, _pair, _pair_full, _random_workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,wall,kind", [
    ((17, 11, 7), (0, 0, 0), "separable"),
    ((5, 12, 9), (0, 1, 1), "full"),
    ((6, 5, 4), (1, 1, 1), "separable"),
    ((1, 1, 1), (0, 0, 0), "separable"),
    ((40, 3, 2), (0, 1, 0), "full"),
    ((33, 1, 19), (1, 0, 1), "separable"),
])
def test_d3q15_random_fields_envelope_walls(shape, wall, kind):
    w, full = _random_workload(W.D3Q15, shape, wall, seed=41 + shape[0], kind=kind)
    G, R = _pair_full(w, full)
    compare_state(G, R)
    for n in (1, 2, 20):
        _advance(G, R, n)
        compare_state(G, R)


def test_d3q15_paper_duct_3x45x45():
    """The paper's D3Q15 demonstration (3 x 45 x 45, tau = 0.76, F = 1e-7)."""
    w = W.duct15()
    G, R = _pair(w)
    _advance(G, R, 300)
    compare_state(G, R)
    # mass is exact; the momentum grows by the total force per step
    r = G.reduce()
    assert abs(r[0] - w.nodes) <= 1e-12 * w.nodes


def test_d3q15_batch_matches_single_and_oracle():
    ws = [W.duct15(n=9, nx=4), _random_workload(W.D3Q15, (7, 6, 5), (1, 1, 1), seed=3)[0],
          _random_workload(W.D3Q15, (11, 4, 3), (0, 0, 1), seed=4)[0]]
    solo = [lbm.from_workload(w) for w in ws]
    grp = [lbm.from_workload(w) for w in ws]
    B = lbm.Batch(grp)
    B.step(7)
    for G in solo:
        G.step(7)
    for w, a, b in zip(ws, solo, grp):
        assert np.abs(a.get_populations() - b.get_populations()).max() <= 7 * 4 * 2.0 ** -53
        R = oracle_from_workload(w)
        R.run(7)
        compare_state(b, R)


def test_d3q15_checkpoint_and_reduced_precision_rejected():
    w = W.duct15(n=12, nx=3)
    G = lbm.from_workload(w)
    G.step(5)
    f = G.get_populations()
    H = lbm.from_workload(w)
    H.set_populations(f, step=G.t)
    G.step(4)
    H.step(4)
    assert np.array_equal(G.get_populations(), H.get_populations())
    with pytest.raises(lbm.LBMError) as e:
        lbm.Lattice(lbm.D3Q15, (4, 4, 4), W.d3q15_omega(0.8), storage=lbm.FP32_DEV)
    assert e.value.code == lbm.EINVAL


def test_d3q15_duct_128_full_size_sampled():
    """The bench's D3Q15 workload (128^3 duct) in its launch configuration:
    3 steps, then one more checked on 300 sampled nodes by the oracle."""
    w = W.duct15(n=128, nx=128)
    G = lbm.from_workload(w)
    r0 = G.reduce()
    G.step(3)
    r1 = G.reduce()
    assert abs(r1[0] - r0[0]) <= 1e-12 * r0[0]
    one_step_sampled(w, G, samples=300, seed=6)

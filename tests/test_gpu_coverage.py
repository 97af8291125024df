"""Race / coverage checks without a sanitizer: the destination buffer is
poisoned with NaN before each step, so a node or plane a kernel failed to
write would stay NaN.  Covers every lattice, storage form, ragged extents
with walls, the batched tilings and the cluster form; plus the file
checkpoint (bitwise resume)."""
import math

import numpy as np
import pytest

from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W
from tests.test_gpu_parity import _random_workload

pytestmark = pytest.mark.gpu

CASES = [(W.D2Q9, (13, 7, 1), (0, 1, 0)), (W.D2Q5, (11, 9, 1), (1, 0, 0)),
         (W.D3Q27, (6, 5, 7), (1, 1, 0)), (W.D3Q15, (5, 7, 6), (0, 1, 1))]


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32_DEV, lbm.FP16_DEV])
@pytest.mark.parametrize("lattice,shape,wall", CASES)
def test_every_node_written_each_step(lattice, shape, wall, storage):
    if lattice == W.D3Q15 and storage != lbm.FP64:
        pytest.skip("D3Q15 stores FP64 only")
    w, _ = _random_workload(lattice, shape, wall, seed=3, env=False)
    G = lbm.from_workload(w, storage=storage)
    for n in (1, 1, 2, 3):  # single launches and the multi-step forms
        G.debug_poison()
        G.step(n)
        f = G.get_populations()
        assert np.isfinite(f).all(), (n, np.argwhere(~np.isfinite(f))[:5])
        G.reduce()  # raises LBMError(EUNSTABLE) on a non-finite node


@pytest.mark.parametrize("storage", [lbm.FP64, lbm.FP32_DEV])
def test_every_node_written_by_every_batch_tiling(storage):
    ch, sc = W.batched_sweep(count=24, seed=5, nx_range=(32, 160), ny_range=(32, 120))
    for ws in (ch, sc):
        Gs = [lbm.from_workload(w, storage=storage) for w in ws]
        B = lbm.Batch(Gs)
        for tile in (128, 256, 512):
            for persistent in (False, True):
                B.set_tiling(tile, persistent)
                for G in Gs:
                    G.debug_poison()
                B.step(1)
                for G in Gs:
                    assert np.isfinite(G.get_populations()).all(), (tile, persistent)


def test_small_lattice_cluster_form_writes_every_node(tmp_path):
    w = W.poiseuille(ny=37, nx=5, tau=0.7, Fx=1e-5)
    G = lbm.from_workload(w)
    for n in (2, 7, 100):
        G.debug_poison()
        G.step(n)
        assert np.isfinite(G.get_populations()).all()
    # file checkpoint: resume is bitwise identical to the uninterrupted run
    path = str(tmp_path / "ck.npz")
    G.save_checkpoint(path)
    H = lbm.from_workload(w)
    H.load_checkpoint(path)
    assert H.t == G.t
    G.step(13)
    H.step(13)
    assert np.array_equal(G.get_populations(), H.get_populations())
    bad = lbm.from_workload(W.poiseuille(ny=9))
    with pytest.raises(ValueError):
        bad.load_checkpoint(path)

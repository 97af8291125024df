"""lbm_reduce_sums_noalloc: the mass and momentum sums of lbm_reduce computed
with the library's fixed device scratch array, for callers that cannot
allocate device memory at that point (memory owned by another allocator, or a
time loop that must not call cudaMalloc/cudaFree, which can synchronise the
device).  Checked through the C ABI against lbm_reduce on two calls in a row.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _close(a, b, scale):
    return np.abs(np.asarray(a) - np.asarray(b)).max() <= TOL * scale


@pytest.mark.parametrize("make,storage", [
    (lambda: W.kolmogorov(shape=(20, 24, 12)), lbm.FP64),
    (lambda: W.cde_workload(W.cde_sweep_params(sizes=(64,))[0]), lbm.FP64),
    (lambda: W.poiseuille(), lbm.FP64),
    # reduced-precision storage takes its own partial-sum kernel (FP64 sums
    # of the stored deviations plus the rest state)
    (lambda: W.kolmogorov(shape=(20, 24, 12)), lbm.FP32_DEV),
    (lambda: W.cde_workload(W.cde_sweep_params(sizes=(64,))[0]), lbm.FP16_DEV),
    (lambda: W.poiseuille(ny=65, nx=40), lbm.BF16_DEV),
])
def test_noalloc_sums_match_reduce_on_two_calls(make, storage):
    w = make()
    L = lbm.from_workload(w, storage=storage)
    L.step(5)
    ref = L.reduce()[:4]
    scale = max(abs(ref[0]), 1.0)
    first = L.reduce_sums_noalloc()
    second = L.reduce_sums_noalloc()
    assert _close(first, ref, scale), (first, ref)
    assert _close(second, ref, scale), (second, ref)
    # after more steps the shared scratch holds the previous call's values;
    # the next result must still follow the new state
    L.step(3)
    ref2 = L.reduce()[:4]
    got2 = L.reduce_sums_noalloc()
    assert _close(got2, ref2, scale), (got2, ref2)


def test_noalloc_sums_across_two_contexts():
    a = lbm.from_workload(W.kolmogorov(shape=(16, 8, 8)))
    b = lbm.from_workload(W.poiseuille(ny=17))
    a.step(2)
    b.step(2)
    ra, rb = a.reduce()[:4], b.reduce()[:4]
    for _ in range(2):
        assert _close(a.reduce_sums_noalloc(), ra, abs(ra[0]))
        assert _close(b.reduce_sums_noalloc(), rb, abs(rb[0]))


def test_noalloc_on_a_local_reference_context():
    """A 16-bit lattice stored at a per-node reference is read through an FP32
    working copy; the no-alloc call refuses (LBM_ESTATE) until an allocating
    read has made it, then agrees with lbm_reduce."""
    w = W.poiseuille(ny=17, nx=8, Fx=1e-4)
    G = lbm.from_workload(w, storage=lbm.FP16_DEV)
    G.set_local_reference(8)
    G.step(20)
    with pytest.raises(lbm.LBMError) as e:
        G.reduce_sums_noalloc()
    assert e.value.code == lbm.ESTATE
    r = G.reduce()
    s = G.reduce_sums_noalloc()
    assert np.allclose(s, r[:4], rtol=1e-15, atol=1e-18), (s, r)

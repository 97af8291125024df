"""The GPU l2 error of Eq. sca (lbm_l2_error) against the oracle's
(lbmref_l2_error) on the same state and reference, for every lattice: the
sums agree to the parity bar; the GPU field is within 1e-12 (relative l2) of
the oracle's field; host and device references give the same bits, and so
does a repeated call; reduced-precision storage sums its own moments."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W
from tests.test_gpu_parity import _pair_full, _random_workload

pytestmark = pytest.mark.gpu

CASES = [(W.D2Q9, (23, 17, 1), (0, 1, 0)), (W.D2Q5, (19, 21, 1), (1, 0, 0)),
         (W.D3Q27, (9, 8, 7), (1, 0, 1)), (W.D3Q15, (7, 6, 9), (0, 1, 1))]


def _context_of(w, full, R):
    ctx = O.OracleContext(w.lattice, w.shape, omega=w.omega, wall=w.wall)
    P = np.ascontiguousarray(full) if full is not None else R.P
    if w.lattice == W.D2Q5:
        assert ctx.set_source(P[0] if P.ndim == 2 else P) == O.REF_OK
    else:
        assert ctx.set_force(P) == O.REF_OK
    assert ctx.set_envelope(w.envelope) == O.REF_OK
    assert ctx.set_populations(R.f, R.t) == O.REF_OK
    return ctx


@pytest.mark.parametrize("lattice,shape,wall", CASES)
def test_l2_error_matches_the_oracle(lattice, shape, wall):
    import torch

    w, full = _random_workload(lattice, shape, wall, seed=60 + shape[0], kind="full")
    G, R = _pair_full(w, full)
    G.step(13)
    R.run(13)
    ctx = _context_of(w, full, R)
    rng = np.random.default_rng(7)
    fields = (0,) if lattice == W.D2Q5 else (0, 1)
    for half in (True, False):
        rc, rho_r, u_r = ctx.moments(half_forced=half)
        for field in fields:
            q = rho_r if field == 0 else u_r
            # the GPU field against the oracle's: the parity bar in l2 form
            g = G.l2_error(q, field, half)
            assert g[2] <= 1e-12, (field, half, g)
            ref = q * (1 + 1e-3 * rng.standard_normal(q.shape))
            rc, want = ctx.l2_error(ref, field, half)
            assert rc == O.REF_OK
            got = G.l2_error(ref, field, half)
            assert abs(got[0] - want[0]) <= 1e-10 * want[0], (got, want)
            assert abs(got[1] - want[1]) <= 1e-14 * want[1]
            assert abs(got[2] - want[2]) <= 1e-10 * want[2]
            # device reference, repeated call: the same bits
            dref = torch.from_numpy(np.ascontiguousarray(ref)).cuda()
            assert G.l2_error(dref, field, half) == got
            assert G.l2_error(ref, field, half) == got


def test_l2_error_reduced_precision_and_checks():
    w, full = _random_workload(W.D2Q9, (40, 13, 1), (0, 1, 0), seed=3, kind="full")
    G = lbm.from_workload(w, storage=lbm.FP32_DEV)
    G.set_force(full=full)
    G.step(9)
    rho, u = G.moments()
    rng = np.random.default_rng(2)
    ref = u * (1 + 1e-2 * rng.standard_normal(u.shape))
    got = G.l2_error(ref, 1)
    num, den = float(np.sum((u - ref) ** 2)), float(np.sum(ref ** 2))
    assert abs(got[0] - num) <= 1e-13 * num and abs(got[1] - den) <= 1e-13 * den
    assert G.l2_error(u, 1)[0] == 0.0
    S = lbm.from_workload(W.cde_workload(W.cde_sweep_params(sizes=(32,))[0]))
    with pytest.raises(lbm.LBMError) as e:
        S._check(S._L.lbm_l2_error(S.h, np.zeros(2 * S.N).ctypes.data_as(lbm.ctypes.c_void_p), 0, 1, 1,
                                   lbm._dp(np.empty(3))))
    assert e.value.code == lbm.EINVAL
    with pytest.raises(ValueError):
        S.l2_error(np.zeros(S.N + 1))

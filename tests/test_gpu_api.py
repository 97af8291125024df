"""GPU checks of the C ABI's state handling: ordering errors, no-op steps,
checkpoint/restore, device-pointer outputs, reductions and the instability
flag (raised by host-injected NaN populations, never by a GPU fault)."""
import numpy as np
import pytest

from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W
from tests.gpu_helpers import compare_state, oracle_from_workload

pytestmark = pytest.mark.gpu


def test_step_before_init_is_a_state_error():
    L = lbm.Lattice(lbm.D2Q9, (4, 4, 1), W.d2q9_omega(0.8))
    with pytest.raises(lbm.LBMError) as e:
        L.step(1)
    assert e.value.code == lbm.ESTATE
    with pytest.raises(lbm.LBMError):
        L.moments()


def test_zero_steps_is_a_no_op_and_negative_is_invalid():
    L = lbm.from_workload(W.poiseuille(ny=9))
    f0 = L.get_populations()
    n0 = L.launch_count()
    L.step(0)
    assert L.t == 0 and L.launch_count() == n0
    assert np.array_equal(L.get_populations(), f0)
    with pytest.raises(lbm.LBMError) as e:
        L.step(-1)
    assert e.value.code == lbm.EINVAL


def test_checkpoint_restore_is_bitwise_identical():
    w = W.kolmogorov(shape=(8, 12, 6))
    A = lbm.from_workload(w)
    A.step(7)
    snap = A.get_populations()
    A.step(13)
    B = lbm.from_workload(w)
    B.set_populations(snap, step=7)
    assert np.array_equal(B.get_populations(), snap)
    B.step(13)
    assert B.t == A.t == 20
    assert np.array_equal(A.get_populations(), B.get_populations())


def test_device_outputs_match_host_outputs():
    torch = pytest.importorskip("torch")
    w = W.poiseuille(ny=17)
    L = lbm.from_workload(w)
    L.step(50)
    rho_h, u_h = L.moments()
    rho_d = torch.empty(L.N, dtype=torch.float64, device="cuda")
    u_d = torch.empty((2, L.N), dtype=torch.float64, device="cuda")
    L.moments(out=(rho_d, u_d), where=1)
    L.sync()
    assert np.array_equal(rho_d.cpu().numpy(), rho_h)
    assert np.array_equal(u_d.cpu().numpy(), u_h)
    f_d = torch.empty((9, L.N), dtype=torch.float64, device="cuda")
    L.get_populations(out=f_d, where=1)
    L.sync()
    assert np.array_equal(f_d.cpu().numpy(), L.get_populations())


def test_reduce_mass_momentum_and_convergence_metric():
    w = W.poiseuille()
    L = lbm.from_workload(w)
    R = oracle_from_workload(w)
    r0 = L.reduce()
    assert np.isinf(r0[4])
    assert abs(r0[0] - L.N) < 1e-12 * L.N
    L.step(100)
    R.run(100)
    r1 = L.reduce()
    rho, u = R.moments()
    f = R.f
    assert abs(r1[0] - r0[0]) < 1e-13 * L.N
    jx = (f[1] - f[3] + f[5] - f[6] - f[7] + f[8]).sum()
    assert abs(r1[1] - jx) < 1e-15 * L.N
    L.step(100)
    R.run(100)
    r2 = L.reduce()
    _, u2 = R.moments()
    assert abs(r2[4] - np.abs(u2 - u).max()) <= 1e-12 * np.abs(u2).max()


def test_nan_population_raises_unstable():
    w = W.poiseuille(ny=9)
    L = lbm.from_workload(w)
    f = L.get_populations()
    f[2, 5] = np.nan
    L.set_populations(f, step=0)
    L.step(2)
    with pytest.raises(lbm.LBMError) as e:
        L.reduce()
    assert e.value.code == lbm.EUNSTABLE


def test_invalid_field_lengths_are_rejected():
    L = lbm.Lattice(lbm.D2Q9, (6, 4, 1), W.d2q9_omega(0.8))
    with pytest.raises(lbm.LBMError) as e:
        L.set_force(tables=[(np.ones(5), np.ones(1), np.ones(1)), (np.ones(5), np.ones(1), np.ones(1))])
    assert e.value.code == lbm.EINVAL
    with pytest.raises(lbm.LBMError):
        L.set_source(tables=[(np.ones(1), np.ones(1), np.ones(1))])


def test_source_lattice_restart_matches_uninterrupted_oracle():
    c = W.cde_sweep_params(sizes=(64,))[0]
    w = W.cde_workload(c)
    A = lbm.from_workload(w)
    A.step(33)
    snap = A.get_populations()
    B = lbm.from_workload(w)
    B.set_populations(snap, step=33)
    B.step(40)
    R = oracle_from_workload(w)
    R.run(73)
    compare_state(B, R)


def test_small_d2q9_cluster_steps_equal_single_launches_and_oracle():
    """A small constant-force D2Q9 lattice takes n >= 2 steps in one cluster
    launch; the result equals n single-step launches (to rounding) and the
    oracle (parity bar).  Sizes cover 1 to 16 blocks and a ragged last block."""
    from tests.gpu_helpers import compare_state, oracle_from_workload

    for ny, nx in ((33, 3), (9, 2), (40, 17), (61, 70)):
        w = W.poiseuille(ny=ny, nx=nx, tau=0.7, Fx=1e-5)
        a = lbm.from_workload(w)
        b = lbm.from_workload(w)
        n0 = a.launch_count()
        a.step(37)
        assert a.launch_count() == n0 + 1 or a.N > 5000
        for _ in range(37):
            b.step(1)
        fa, fb = a.get_populations(), b.get_populations()
        assert np.abs(fa - fb).max() <= 37 * 4 * 2.0 ** -53 * np.abs(fb).max() * 2
        R = oracle_from_workload(w)
        R.run(37)
        compare_state(a, R)
        a.step(2)
        a.step(3)
        R.run(5)
        compare_state(a, R)


@pytest.mark.parametrize("lattice,storage", [
    (W.D3Q27, lbm.FP64), (W.D2Q9, lbm.FP64), (W.D2Q5, lbm.FP64),
    (W.D3Q27, lbm.FP32_DEV), (W.D2Q9, lbm.FP16_DEV), (W.D2Q5, lbm.FP32_DEV),
])
def test_device_field_equals_host_field_bitwise(lattice, storage):
    """A full force / source field given as device memory
    (LBM_FIELD_FULL_DEVICE, copied in stream order) drives the step exactly
    as the same field given from host memory, bit for bit; the field is
    replaced in place between steps, as a coupled solver would do."""
    torch = pytest.importorskip("torch")
    from tests.test_gpu_parity import _random_workload

    shape = (9, 7, 5) if lattice == W.D3Q27 else (23, 14, 1)
    w, full = _random_workload(lattice, shape, (0, 1, 0), seed=31, kind="full")
    rng = np.random.default_rng(32)
    full2 = 1e-4 * rng.standard_normal(full.shape)
    host = lbm.from_workload(w, storage=storage)
    dev = lbm.from_workload(w, storage=storage)
    setter_h = host.set_source if lattice == W.D2Q5 else host.set_force
    setter_d = dev.set_source if lattice == W.D2Q5 else dev.set_force
    buf = torch.from_numpy(np.ascontiguousarray(full)).to("cuda")
    setter_h(full=full)
    setter_d(full=buf)
    host.step(4)
    dev.step(4)
    # new values in the same device buffer, written on the context's stream
    # order (the copy is queued after the steps above)
    torch.cuda.synchronize()
    buf.copy_(torch.from_numpy(np.ascontiguousarray(full2)))
    torch.cuda.synchronize()
    setter_h(full=full2)
    setter_d(full=buf)
    host.step(3)
    dev.step(3)
    fh, th = host.get_populations(with_step=True)
    fd, td = dev.get_populations(with_step=True)
    assert th == td == 7 == host.t
    assert np.array_equal(fh, fd)
    # a host pointer given as a device field is rejected
    f = lbm._Field()
    f.kind = lbm.FIELD_FULL_DEVICE
    arr = np.zeros(full.size)
    f.data = lbm._dp(arr)
    fn = dev._L.lbm_set_source if lattice == W.D2Q5 else dev._L.lbm_set_force
    assert fn(dev.h, lbm.ctypes.byref(f)) == lbm.EINVAL


def test_get_populations_reports_the_step():
    torch = pytest.importorskip("torch")
    L = lbm.from_workload(W.kolmogorov(shape=(6, 5, 4)))
    L.step(11)
    f, t = L.get_populations(with_step=True)
    assert t == 11
    buf = torch.empty((27, L.N), dtype=torch.float64, device="cuda")
    _, t2 = L.get_populations(out=buf, where=1, with_step=True)
    L.sync()
    assert t2 == 11 and np.array_equal(buf.cpu().numpy(), f)

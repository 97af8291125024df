"""Reduced-precision storage (FP32 / FP16 / BF16 deviations from the rest
state, FP32 moment arithmetic): error against the FP64 oracle per form.

The FP32 form must stay within the 1e-4 relative l2 target; the measured
errors of every form are written to $LBM_RESULTS_DIR/rp_errors.json (when that
variable names a folder) so that they can be quoted."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W
from tests.gpu_helpers import one_step_sampled, oracle_from_workload

pytestmark = pytest.mark.gpu

STORAGES = {"fp32": lbm.FP32_DEV, "fp16": lbm.FP16_DEV, "bf16": lbm.BF16_DEV}
# Relative l2 bounds per case and form.  FP32 must meet the 1e-4 target
# everywhere.  16-bit forms: the measured error times ~3 where the form is
# usable; None where 16 bits cannot resolve the per-step force/source increment
# (Poiseuille F = 1e-6: increments ~1e-7 on deviations ~1e-3, below FP16 and
# BF16 resolution) -- there the error is only recorded and must stay < 1.
BOUND = {
    ("poiseuille", "fp32"): 1e-4, ("poiseuille", "fp16"): None, ("poiseuille", "bf16"): None,
    ("cde", "fp32"): 1e-4, ("cde", "fp16"): 3e-2, ("cde", "bf16"): None,
    ("kolmogorov", "fp32"): 1e-4, ("kolmogorov", "fp16"): 1e-3, ("kolmogorov", "bf16"): 3e-2,
}
EPS = {"fp32": 2.0 ** -24, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
RESULTS = {}


def _check(case, form, err):
    b = BOUND[(case, form)]
    assert np.isfinite(err) and err < 1.0, err
    if b is not None:
        assert err <= b, err


def _record(key, val):
    RESULTS[key] = val
    out = os.environ.get("LBM_RESULTS_DIR")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "rp_errors.json"), "w") as f:
            json.dump(RESULTS, f, indent=1, sort_keys=True)


def _l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def _gpu(w, storage, steps):
    G = lbm.from_workload(w, storage=storage)
    G.step(steps)
    return G


@pytest.mark.parametrize("form", ["fp32", "fp16", "bf16"])
def test_poiseuille_reduced_precision(form):
    w = W.poiseuille()
    R = oracle_from_workload(w)
    R.run(10000)
    _, ur = R.moments()
    G = _gpu(w, STORAGES[form], 10000)
    _, ug = G.moments()
    err = _l2(ug[0], ur[0])
    _record(f"poiseuille_d2q9_3x33_10k_{form}", err)
    _check("poiseuille", form, err)


@pytest.mark.parametrize("form", ["fp32", "fp16", "bf16"])
def test_cde_reduced_precision(form):
    c = W.cde_sweep_params(sizes=(64,))[0]
    w = W.cde_workload(c)
    R = oracle_from_workload(w)
    R.run(c.T)
    pr = R.moments() - 1.0
    G = _gpu(w, STORAGES[form], c.T)
    pg = G.moments() - 1.0
    err = _l2(pg, pr)
    _record(f"cde_d2q5_64_T{c.T}_{form}", err)
    _check("cde", form, err)


@pytest.mark.parametrize("form", ["fp32", "fp16", "bf16"])
def test_kolmogorov_reduced_precision(form):
    w = W.kolmogorov(shape=(24, 24, 24))
    R = oracle_from_workload(w)
    R.run(300)
    _, ur = R.moments()
    G = _gpu(w, STORAGES[form], 300)
    _, ug = G.moments()
    err = _l2(ug, ur)
    _record(f"kolmogorov_d3q27_24cubed_300_{form}", err)
    _check("kolmogorov", form, err)


def test_fp32_cde_keeps_second_order():
    """Closed-form error of the FP32 form over the 32/64/128 refinement: order ~2."""
    from tests.test_oracle_d2q5 import _closed_form

    errs = []
    for c in W.cde_sweep_params(sizes=(32, 64, 128)):
        w = W.cde_workload(c)
        G = _gpu(w, lbm.FP32_DEV, c.T)
        phi = G.moments().reshape(c.N, c.N) - 1.0
        ref = _closed_form(c, c.T, c.N)
        errs.append(_l2(phi, ref))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    _record("cde_fp32_closed_form_errors", errs)
    _record("cde_fp32_orders", orders)
    assert all(abs(o - 2.0) < 0.2 for o in orders), (errs, orders)


@pytest.mark.parametrize("form", ["fp32", "bf16"])
def test_reduced_precision_batch_and_checkpoint(form):
    ws = [W.cde_workload(c) for c in W.cde_sweep_params(sizes=(32, 64))]
    solo = [lbm.from_workload(w, storage=STORAGES[form]) for w in ws]
    grp = [lbm.from_workload(w, storage=STORAGES[form]) for w in ws]
    B = lbm.Batch(grp)
    B.step(7)
    for G in solo:
        G.step(7)
    # batched and single kernels: same arithmetic, FMA fusion may differ -> a
    # few units of the storage precision on the deviations (|d| <= ~0.01)
    tol = 8 * EPS[form] * 0.05
    for a, b in zip(solo, grp):
        assert np.abs(a.get_populations() - b.get_populations()).max() <= tol
    # checkpoint: restoring f(t) reproduces it to the storage precision
    f = grp[1].get_populations()
    C = lbm.from_workload(ws[1], storage=STORAGES[form])
    C.set_populations(f, step=grp[1].t)
    assert np.abs(C.get_populations() - f).max() <= tol
    r = grp[1].reduce()
    # mass: the deviations are rounded to the storage precision every step
    assert abs(r[0] - ws[1].nodes) < (1e-6 if form == "fp32" else 1e-4) * ws[1].nodes
    s = grp[1].reduce_sums_noalloc()
    assert np.allclose(s, r[:4], rtol=1e-12, atol=1e-12)


def test_fp32_kolmogorov_256_full_size_sampled_step():
    """Config 3 at 256^3 with FP32-deviation storage in the bench's launch
    configuration: 3 steps, then one more step checked on 200 sampled nodes
    against the FP64 oracle's collision of the same f(t) (the FP32 moment
    arithmetic is the only difference)."""
    w = W.kolmogorov(n=256)
    G = lbm.from_workload(w, storage=lbm.FP32_DEV)
    G.step(3)
    worst = one_step_sampled(w, G, samples=200, seed=9, tol=2e-6)
    _record("kolmogorov_256_fp32_one_step_sampled_rel_max", worst)


def test_config3_kolmogorov_256_1000_steps_error_per_form():
    """Config 3 as stated: Kolmogorov 256^3, 1000 steps, the FP64 run (which
    matches the oracle to 1e-12 in the parity tests) against each
    reduced-precision form.  FP32 must stay within 1e-4 relative l2 in u;
    the 16-bit errors are recorded."""
    w = W.kolmogorov(n=256)
    ref = lbm.from_workload(w)
    ref.step(1000)
    _, u_ref = ref.moments()
    ref.close()
    for form in ("fp32", "fp16", "bf16"):
        G = lbm.from_workload(w, storage=STORAGES[form])
        G.step(1000)
        _, u = G.moments()
        G.close()
        err = _l2(u, u_ref)
        _record(f"kolmogorov_d3q27_256cubed_1000_{form}", err)
        assert np.isfinite(err) and err < 1.0, (form, err)
        if form == "fp32":
            assert err <= 1e-4, err



@pytest.mark.parametrize("form", ["fp32", "fp16"])
def test_small_d2q9_cluster_steps_reduced_precision(form):
    """The cluster form of a small reduced-precision D2Q9 lattice rounds to the
    storage type every step, as single-step launches do."""
    for ny, nx in ((33, 3), (40, 17)):
        w = W.poiseuille(ny=ny, nx=nx, tau=0.7, Fx=1e-5)
        a = lbm.from_workload(w, storage=STORAGES[form])
        b = lbm.from_workload(w, storage=STORAGES[form])
        n0 = a.launch_count()
        a.step(40)
        assert a.launch_count() == n0 + 1
        for _ in range(40):
            b.step(1)
        fa, fb = a.get_populations(), b.get_populations()
        tol = 1e-6 if form == "fp32" else 4 * EPS["fp16"]
        assert np.abs(fa - fb).max() <= tol * np.abs(fb).max(), np.abs(fa - fb).max()


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("shape,wall", [
    ((12, 10, 8), (0, 0, 0)),   # periodic: the packed pulls, x wrap of both nodes
    ((12, 10, 8), (1, 0, 0)),   # walls on x: pairs at x = 0 and x = nx - 2 take the per-node pulls
    ((10, 9, 7), (0, 1, 1)),    # duct walls
    ((16, 6, 5), (1, 1, 1)),
    ((9, 8, 6), (0, 0, 0)),     # odd nx: the one-node kernel
])
def test_d3q27_16bit_pair_kernel(form, shape, wall):
    """16-bit D3Q27 storage at unit higher rates steps two x-neighbouring
    nodes per thread with packed FP32x2 arithmetic (nx even).  Against the
    FP64 oracle within the 16-bit error bound, and against the batched
    kernel (one node per thread, scalar FP32 arithmetic) to a few units of
    the storage precision after 5 steps; an x-dependent force checks that
    each node of a pair takes its own force."""
    rng = np.random.default_rng(41 + shape[0] + 3 * wall[0])
    nx, ny, nz = shape
    tables = [(1e-4 * (1 + 0.3 * rng.standard_normal(nx)), 1 + 0.2 * rng.standard_normal(ny),
               1 + 0.2 * rng.standard_normal(nz)) for _ in range(3)]
    u0 = 0.05 * rng.standard_normal((3, nx * ny * nz))
    w = W.Workload(name="pair", lattice=W.D3Q27, shape=shape, wall=wall, omega=W.d3q27_omega(0.7), rho0=1.0,
                   u0=u0, tables=tables)
    G = _gpu(w, STORAGES[form], 5)
    a = lbm.from_workload(w, storage=STORAGES[form])
    b = lbm.from_workload(w, storage=STORAGES[form])
    B = lbm.Batch([a, b])
    B.step(5)
    fg, fa = G.get_populations(), a.get_populations()
    tol = 8 * EPS[form] * 0.05
    assert np.abs(fg - fa).max() <= tol, np.abs(fg - fa).max()
    R = oracle_from_workload(w)
    R.run(5)
    _, ur = R.moments()
    _, ug = G.moments()
    err = _l2(ug, ur)
    _record(f"d3q27_pair_{form}_{nx}x{ny}x{nz}_walls{''.join(map(str, wall))}", err)
    assert err <= (2e-3 if form == "fp16" else 2e-2), err


def _pair2d_workload(lattice, shape, wall, seed):
    """A 2D lattice for the 16-bit pair kernels: x-dependent force or source
    (each node of a pair takes its own), a 0.05-sized initial signal."""
    rng = np.random.default_rng(seed)
    nx, ny, _ = shape
    N = nx * ny
    if lattice == W.D2Q9:
        tables = [(1e-4 * (1 + 0.3 * rng.standard_normal(nx)), 1 + 0.2 * rng.standard_normal(ny), np.array([1.0]))
                  for _ in range(2)]
        return W.Workload(name="pair9", lattice=W.D2Q9, shape=shape, wall=wall, omega=W.d2q9_omega(0.7), rho0=1.0,
                          u0=0.05 * rng.standard_normal((2, N)), tables=tables)
    tables = [(1e-4 * (1 + 0.3 * rng.standard_normal(nx)), 1 + 0.2 * rng.standard_normal(ny), np.array([1.0]))]
    return W.Workload(name="pair5", lattice=W.D2Q5, shape=shape, wall=wall, omega=W.d2q5_omega(0.8),
                      rho0=1.0 + 0.05 * rng.standard_normal(N), u0=(0.03, -0.02, 0.0), tables=tables)


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("lattice", [W.D2Q9, W.D2Q5], ids=["d2q9", "d2q5"])
@pytest.mark.parametrize("shape,wall", [
    ((12, 10, 1), (0, 0, 0)),   # nx % 4 = 0, periodic: four nodes per thread, 64-bit pulls, x wrap
    ((4, 5, 1), (0, 0, 0)),     # nx = 4: one quad per row, both x edges wrap onto it
    ((12, 10, 1), (1, 0, 0)),   # walls on x: quads at x = 0 and x = nx - 4 take the per-node pulls
    ((16, 9, 1), (0, 1, 0)),    # channel walls on y
    ((14, 6, 1), (0, 0, 0)),    # nx % 4 = 2: two nodes per thread, x wrap of both nodes
    ((2, 7, 1), (0, 0, 0)),     # nx = 2: one pair per row, each node the other's x source
    ((10, 5, 1), (1, 1, 0)),    # pairs next to walls on x and y
    ((9, 8, 1), (0, 0, 0)),     # odd nx: the one-node kernel
])
def test_2d_16bit_pair_kernels(form, lattice, shape, wall):
    """16-bit D2Q9 (unit higher rates) and D2Q5 (uniform velocity) storage step
    four consecutive nodes of a row per thread (nx a multiple of 4) or two
    (nx even) in packed FP32x2 arithmetic.  Against the batched kernel (one
    node per thread, scalar FP32) to a few units of the storage precision
    after 5 steps, and against the FP64 oracle within the 16-bit error bound."""
    w = _pair2d_workload(lattice, shape, wall, 7 + shape[0] + 5 * wall[0] + wall[1])
    G = _gpu(w, STORAGES[form], 5)
    a = lbm.from_workload(w, storage=STORAGES[form])
    b = lbm.from_workload(w, storage=STORAGES[form])
    B = lbm.Batch([a, b])
    B.step(5)
    fg, fa = G.get_populations(), a.get_populations()
    assert np.abs(fg - fa).max() <= 8 * EPS[form] * 0.05, np.abs(fg - fa).max()
    R = oracle_from_workload(w)
    R.run(5)
    if lattice == W.D2Q9:
        _, ur = R.moments()
        _, ug = G.moments()
        err = _l2(ug, ur)
    else:
        pr = R.moments()
        pg = G.moments()
        err = _l2(pg - pr.mean(), pr - pr.mean())
    _record(f"{'d2q9' if lattice == W.D2Q9 else 'd2q5'}_pair_{form}_{shape[0]}x{shape[1]}_walls{''.join(map(str, wall))}",
            err)
    assert err <= (3e-3 if form == "fp16" else 3e-2), err


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_2d_pair_kernels_stochastic_rounding(form):
    """Stochastic rounding in the 2D multi-node kernels (nx = 16: four nodes
    per thread; 14: two): seeded (same seed, same bits), each node its own
    bits (equal nodes do not round alike everywhere), and unbiased against
    the FP64 oracle."""
    for nx in (16, 14):
        _sr_multi_node_case(form, nx)


def _sr_multi_node_case(form, nx):
    ny = 12
    w9 = W.Workload(name="sr_pair9", lattice=W.D2Q9, shape=(nx, ny, 1), wall=(0, 0, 0), omega=W.d2q9_omega(0.7),
                    rho0=1.0, u0=np.stack([np.full(nx * ny, 0.031), np.full(nx * ny, -0.017)]))
    runs = []
    for seed in (3, 3):
        G = lbm.from_workload(w9, storage=STORAGES[form])
        G.set_stochastic_rounding(True, seed)
        G.step(7)
        runs.append(G.get_populations())
    assert np.array_equal(runs[0], runs[1])
    f = runs[0].reshape(9, ny, nx)
    # a uniform state: round to nearest would keep every node equal; own bits per node do not
    assert not np.array_equal(f[:, :, 0::2], f[:, :, 1::2])
    assert not np.array_equal(f[:, :, 0:nx - 2], f[:, :, 2:nx])
    R = oracle_from_workload(w9)
    R.run(7)
    _, ur = R.moments()
    G = lbm.from_workload(w9, storage=STORAGES[form])
    G.set_stochastic_rounding(True, 11)
    G.step(7)
    _, ug = G.moments()
    err = _l2(ug, ur)
    _record(f"d2q9_multi_node_sr_{form}_nx{nx}", err)
    assert err <= (2e-3 if form == "fp16" else 2e-2), err


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_stochastic_rounding_is_seeded_and_single_lattice_only(form):
    """Stochastic rounding of the 16-bit deviations: the same seed gives the
    same bits, another seed other bits; FP32 storage and batches refuse it."""
    w = W.kolmogorov(shape=(10, 8, 6))
    runs = []
    for seed in (7, 7, 8):
        G = lbm.from_workload(w, storage=STORAGES[form])
        G.set_stochastic_rounding(True, seed)
        G.step(20)
        runs.append(G.get_populations())
        if seed == 8:
            with pytest.raises(lbm.LBMError) as e:
                lbm.Batch([G])
            assert e.value.code == lbm.EINVAL
    assert np.array_equal(runs[0], runs[1])
    assert not np.array_equal(runs[0], runs[2])
    H = lbm.from_workload(w, storage=lbm.FP32_DEV)
    with pytest.raises(lbm.LBMError) as e:
        H.set_stochastic_rounding(True, 1)
    assert e.value.code == lbm.EINVAL


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("case", ["poiseuille", "cde", "kolmogorov", "kolmogorov_odd_nx"])
def test_stochastic_rounding_error_against_oracle(form, case):
    """The error of the stochastically rounded 16-bit forms against the FP64
    oracle, on the cases the round-to-nearest forms are measured on (recorded
    beside them); it must stay finite and below the round-to-nearest bound
    where there is one."""
    if case == "poiseuille":
        w, steps = W.poiseuille(), 10000
    elif case == "cde":
        c = W.cde_sweep_params(sizes=(64,))[0]
        w, steps = W.cde_workload(c), c.T
    elif case == "kolmogorov":
        w, steps = W.kolmogorov(shape=(24, 24, 24)), 300
    else:
        w, steps = W.kolmogorov(shape=(23, 24, 24)), 300  # one node per thread
    R = oracle_from_workload(w)
    R.run(steps)
    G = lbm.from_workload(w, storage=STORAGES[form])
    G.set_stochastic_rounding(True, 10247)
    G.step(steps)
    if w.lattice == W.D2Q5:
        err = _l2(G.moments() - 1.0, R.moments() - 1.0)
    else:
        err = _l2(G.moments()[1], R.moments()[1])
    _record(f"{case}_{form}_stochastic_rounding", err)
    assert np.isfinite(err) and err < 1.0, err
    b = BOUND.get((case.split("_")[0], form))
    if b is not None:
        assert err <= 3 * b, err


def _tiny_scalar(nx=40, ny=37, A=2e-7, tau=1.0):
    one = np.array([1.0])
    x, y = np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64)
    return W.Workload(name="tiny_scalar", lattice=W.D2Q5, shape=(nx, ny, 1), wall=(0, 0, 0),
                      omega=W.d2q5_omega(tau), rho0=1.0, u0=(0.01, 0.01, 0.0),
                      tables=[(A * np.sin(2 * math.pi * x / nx), np.sin(2 * math.pi * y / ny), one)])


@pytest.mark.parametrize("form", ["fp32", "fp16", "bf16"])
def test_d2q5_equilibrium_reference_small_signal(form):
    """A periodic scalar lattice with a uniform advecting velocity stores its
    deviations from the equilibrium at (phi_ref, u), which the step leaves
    unchanged: a source of amplitude 2e-7 (the smallest of the batched
    sweep's draws) whose response is ~1e-5 must keep its relative accuracy
    instead of drowning in the rounding of the background's advection term
    (FP32: the relative l2 of phi - phi0 against the FP64 oracle after 3000
    steps within 1e-5; the 16-bit forms recorded)."""
    w = _tiny_scalar()
    R = oracle_from_workload(w)
    R.run(3000)
    G = _gpu(w, STORAGES[form], 3000)
    err = _l2(G.moments() - 1.0, R.moments() - 1.0)
    _record(f"tiny_scalar_d2q5_40x37_A2e-7_3000_{form}", err)
    assert np.isfinite(err) and err < 1.0
    if form == "fp32":
        assert err <= 1e-5, err
    # the batched kernel takes the same reference (one launch for two members)
    a = lbm.from_workload(w, storage=STORAGES[form])
    b = lbm.from_workload(w, storage=STORAGES[form])
    B = lbm.Batch([a, b])
    B.step(3000)
    assert np.abs(a.moments() - G.moments()).max() <= 64 * EPS[form] * 1e-4


@pytest.mark.parametrize("form", ["fp32", "bf16"])
def test_d2q5_reference_rebased_for_a_velocity_field(form):
    """Switching a periodic, uniformly advected scalar lattice to a velocity
    field mid-run re-expresses its deviations against the rest state; the
    run then follows the oracle through the same sequence, and a checkpoint
    round trip reproduces f(t)."""
    w = _tiny_scalar(A=1e-4)
    rng = np.random.default_rng(5)
    field = 0.02 * rng.standard_normal((2, w.nodes))
    R = oracle_from_workload(w)
    G = lbm.from_workload(w, storage=STORAGES[form])
    G.step(50)
    R.run(50)
    f = G.get_populations()
    C = lbm.from_workload(w, storage=STORAGES[form])
    C.set_populations(f, step=G.t)
    assert np.abs(C.get_populations() - f).max() <= 4 * EPS[form] * 0.05
    G.set_velocity(full=field)
    R.uadv = np.ascontiguousarray(field)
    G.step(50)
    R.run(50)
    err = _l2(G.moments() - 1.0, R.moments() - 1.0)
    _record(f"d2q5_rebased_velocity_field_{form}", err)
    assert err <= (1e-5 if form == "fp32" else 3e-2), err


def test_maximum_node_count_d2q5_fp32():
    """The largest lattice a context takes (N = 65536 x 32767 = LBM_MAX_NODES
    = 2^31 - 2^16, so that 32-bit thread indices of every launch stay below
    2^31 and [q][N] offsets need 64 bits): a periodic D2Q5 scalar lattice
    with a uniform advecting velocity and a separable source, FP32 deviation
    storage (86 GB of populations).  One step, checked on sampled nodes -- the
    first and last nodes and both x edges among them -- by the oracle's
    collision of the GPU's f(t), streamed in; plus exact scalar accounting."""
    nx, ny = 65536, 32767
    one = np.array([1.0])
    x, y = np.arange(nx, dtype=np.float64), np.arange(ny, dtype=np.float64)
    w = W.Workload(name="max_d2q5", lattice=W.D2Q5, shape=(nx, ny, 1), wall=(0, 0, 0),
                   omega=W.d2q5_omega(0.9), rho0=1.0, u0=(0.01, -0.02, 0.0),
                   tables=[(1e-3 * np.sin(2 * math.pi * x / nx), np.cos(2 * math.pi * y / ny), one)])
    assert w.nodes == lbm.MAX_NODES
    G = lbm.from_workload(w, storage=lbm.FP32_DEV)
    r0 = G.reduce()
    G.step(2)
    r1 = G.reduce()
    # the source sums to ~0 over the lattice: the total scalar changes only by rounding
    assert abs(r1[0] - r0[0]) <= 1e-6 * r0[0]
    worst = one_step_sampled(w, G, samples=64, seed=17, tol=2e-6, device=True)
    _record("max_nodes_d2q5_fp32_one_step_sampled_rel_max", worst)
    G.close()

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
from tests.gpu_helpers import oracle_from_workload

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
    from tests.test_gpu_parity import _one_step_sampled

    w = W.kolmogorov(n=256)
    G = lbm.from_workload(w, storage=lbm.FP32_DEV)
    G.step(3)
    worst = _one_step_sampled(w, G, samples=200, seed=9, tol=2e-6)
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

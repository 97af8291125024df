"""The paper's analytic benchmark flows on the GPU (Sec. 6.2 Hartmann,
Sec. 6.3 Womersley, Sec. 6.5 four-rolls mill): parity with the FP64 oracle
over the first steps, then the converged fields against the closed forms,
FP64 and FP32 storage, with the convergence order of each form.  The errors
are written to $LBM_RESULTS_DIR/benchmarks.json when that names a folder."""
import json
import math
import os

import numpy as np
import pytest

from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W
from tests.gpu_helpers import compare_state, oracle_from_workload

pytestmark = pytest.mark.gpu

RESULTS = {}
FORMS = {"fp64": lbm.FP64, "fp32": lbm.FP32_DEV}


def _record(key, val):
    RESULTS[key] = val
    out = os.environ.get("LBM_RESULTS_DIR")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "benchmarks.json"), "w") as f:
            json.dump(RESULTS, f, indent=1, sort_keys=True)


def _l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def _gpu(w, storage=lbm.FP64, envelope_steps=None):
    return lbm.from_workload(w, storage=storage, envelope_steps=envelope_steps)


@pytest.mark.parametrize("w", [W.hartmann(ny=33, Ha=10.0), W.womersley(ny=32, period=400), W.four_rolls(48)],
                         ids=["hartmann", "womersley", "four_rolls"])
def test_benchmark_parity_with_oracle(w):
    G = _gpu(w)
    R = oracle_from_workload(w)
    for n in (1, 50, 250):
        G.step(n)
        R.run(n)
        compare_state(G, R)


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_hartmann_converges_at_second_order(form):
    errs = []
    for ny in (32, 64):
        w = W.hartmann(ny=ny, Ha=3.0, tau=0.8)
        G = _gpu(w, FORMS[form])
        G.step(int(12 * ny * ny / w.meta["nu"] / math.pi ** 2))
        _, u = G.moments()
        errs.append(_l2(u[0].reshape(ny, -1)[:, 0], W.hartmann_profile(w)))
    order = math.log2(errs[0] / errs[1])
    _record(f"hartmann_Ha3_{form}", {"l2": errs, "order": order})
    assert 1.8 < order < 2.2, errs


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_womersley_converges_at_second_order(form):
    worst = []
    for ny in (32, 64):
        T = int(2000 * (ny / 16) ** 2)
        w = W.womersley(ny=ny, period=T, tau=1.0)
        G = _gpu(w, FORMS[form], envelope_steps=6 * T + 10)
        G.step(5 * T)
        e = 0.0
        for _ in range(4):
            _, u = G.moments()
            e = max(e, _l2(u[0].reshape(ny, -1)[:, 0], W.womersley_profile(w, G.t)))
            G.step(T // 4)
        worst.append(e)
    order = math.log2(worst[0] / worst[1])
    _record(f"womersley_Wo1.1_{form}", {"l2": worst, "order": order})
    assert 1.8 < order < 2.2, worst


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_four_rolls_converges_at_second_order(form):
    errs = []
    for N in (48, 96):
        w = W.four_rolls(N)
        G = _gpu(w, FORMS[form])
        G.step(int(6 / (w.meta["nu"] * w.meta["k"] ** 2)))
        _, u = G.moments()
        ua = W.four_rolls_velocity(w)
        errs.append(max(_l2(u[0], ua[0]), _l2(u[1], ua[1])))
    order = math.log2(errs[0] / errs[1])
    _record(f"four_rolls_{form}", {"l2": errs, "order": order})
    assert 1.8 < order < 2.3, errs

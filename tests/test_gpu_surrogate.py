"""Learned warm start: the network's CUDA kernels against the FP64 numpy
oracle (loss, gradients, Adam), and a small end-to-end study showing what the
trained network gains over starting the LB iteration from rest."""
import json
import os

import numpy as np
import pytest

from oracle import surrogate_ref as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LAYERS = [(3, 4, (1, 3, 3), (1, 1, 1), "tanh"), (4, 5, (3, 3, 1), (1, 2, 1), "tanh"),
          (5, 1, (1, 1, 1), (1, 1, 1), None)]


def _pair(bf16, seed=0):
    from paper_1806_10247_gb300 import surrogate as G

    net = G.ConvNet(LAYERS, seed=seed, bf16=bf16)
    params = []
    for w, b in zip(net.W, net.B):
        wn = w.cpu().numpy().astype(np.float64)
        if bf16:  # the kernels read the BF16 copy
            wn = torch.tensor(wn, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
        params.append((wn, b.cpu().numpy().astype(np.float64)))
    return net, S.Net(LAYERS, params)


def test_forward_backward_match_oracle_fp32_weights():
    net, ref = _pair(bf16=False)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 3, 3, 7, 6)).astype(np.float32)
    t = rng.standard_normal((3, 1, 3, 7, 6)).astype(np.float32)
    loss, grads = net.loss_and_grads(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    rloss, rgrads = ref.loss_and_grads(x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - rloss) <= 1e-5 * rloss
    for (gw, gb), (rw, rb) in zip(grads, rgrads):
        assert np.allclose(gw.cpu().numpy(), rw, rtol=1e-4, atol=1e-6 * np.abs(rw).max())
        assert np.allclose(gb.cpu().numpy(), rb, rtol=1e-4, atol=1e-6 * np.abs(rb).max())


def test_bf16_weights_forward_and_gradients():
    net, ref = _pair(bf16=True, seed=1)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 3, 3, 5, 4)).astype(np.float32)
    t = rng.standard_normal((2, 1, 3, 5, 4)).astype(np.float32)
    y, _ = net.forward(torch.tensor(x, device="cuda"))
    ry, _ = ref.forward(x.astype(np.float64))
    assert np.allclose(y.cpu().numpy(), ry, rtol=1e-4, atol=1e-5)
    loss, grads = net.loss_and_grads(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    rloss, rgrads = ref.loss_and_grads(x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - rloss) <= 1e-4 * rloss
    for (gw, _), (rw, _) in zip(grads, rgrads):
        assert np.allclose(gw.cpu().numpy(), rw, rtol=1e-3, atol=1e-5 * np.abs(rw).max())


def test_adam_matches_oracle_every_parameter():
    """Three Adam steps on every weight and bias of the network against the
    oracle's update (each parameter keeps its own moment buffers)."""
    net, _ = _pair(bf16=False, seed=2)
    rng = np.random.default_rng(5)
    ref = []
    grads = []
    for w, b in zip(net.W, net.B):
        gw = rng.standard_normal(tuple(w.shape))
        gb = rng.standard_normal(tuple(b.shape))
        grads.append((torch.tensor(gw, dtype=torch.float32, device="cuda"),
                      torch.tensor(gb, dtype=torch.float32, device="cuda")))
        for p, g in ((w, gw), (b, gb)):
            p0 = p.cpu().numpy().astype(np.float64)
            ref.append([p0, g, np.zeros_like(p0), np.zeros_like(p0)])
    for t in (1, 2, 3):
        net.adam_step(grads, lr=1e-2)
        for p, g, m, v in ref:
            S.adam_step(p, g, m, v, t, lr=1e-2)
    got = []
    for w, b in zip(net.W, net.B):
        got += [w.cpu().numpy(), b.cpu().numpy()]
    for a, (p, _, _, _) in zip(got, ref):
        assert np.allclose(a, p, rtol=1e-5, atol=1e-6)


def test_warm_start_gain_small_duct():
    """n = 16 sections: train on 48 method-generated steady fields, then start
    the LB from the prediction for held-out parameters.  The converged field is
    the same as from rest and fewer steps are needed."""
    from paper_1806_10247_gb300 import surrogate as G

    n = 16
    X, Y, params, gen = G.generate(n, 48, seed=11)
    net = G.ConvNet(seed=0, bf16=True)
    hist = G.train(net, X, Y, iters=400, batch=16, lr=3e-3)
    assert hist[-1] < 0.2 * hist[0], (hist[0], hist[-1])
    cases = G.draw_params(3, n, seed=99)
    res = G.warm_start_study(net, n, cases)
    out = os.environ.get("LBM_RESULTS_DIR")
    if out and os.path.isdir(out):
        with open(os.path.join(out, "warmstart_small.json"), "w") as f:
            json.dump({"generation": gen, "loss_first": hist[0], "loss_last": hist[-1], "cases": res}, f, indent=1)
    for r in res:
        assert r["converged_fields_l2"] < 1e-6, r
        assert r["prediction_l2"] < 0.2, r
    assert sum(r["steps_warm"] for r in res) < sum(r["steps_cold"] for r in res), res

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


def _bf16(a):
    """Round to the nearest BF16 value (ties to even), as float64."""
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def test_bf16_weights_forward_and_gradients():
    """BF16 weights run the convolutions on the tensor cores, which round each
    layer's input (and each incoming gradient) to BF16 and sum exact products
    in FP32: the FP64 reference applies the same roundings layer by layer."""
    net, ref = _pair(bf16=True, seed=1)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 3, 3, 5, 4)).astype(np.float32)
    t = rng.standard_normal((2, 1, 3, 5, 4)).astype(np.float32)
    acts = [x.astype(np.float64)]
    h = acts[0]
    for (ci, co, k, dil, act), (w, b) in zip(LAYERS, ref.params):
        z = S.conv3d(_bf16(h), w, b, dil)
        h = np.tanh(z) if act == "tanh" else z
        h = np.asarray(h, np.float32).astype(np.float64)  # activations are stored in FP32
        acts.append(h)
    y, _ = net.forward(torch.tensor(x, device="cuda"))
    assert np.allclose(y.cpu().numpy(), acts[-1], rtol=1e-4, atol=1e-5 * np.abs(acts[-1]).max())
    loss, grads = net.loss_and_grads(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
    diff = acts[-1] - t
    rloss = float(np.mean(diff ** 2))
    assert abs(loss - rloss) <= 1e-4 * rloss
    g = (2.0 * diff / diff.size).astype(np.float32).astype(np.float64)
    for li in range(len(LAYERS) - 1, -1, -1):
        ci, co, k, dil, act = LAYERS[li]
        if act == "tanh":
            g = (g * (1.0 - acts[li + 1] ** 2)).astype(np.float32).astype(np.float64)
        w, b = ref.params[li]
        gx, gw, _ = S.conv3d_backward(_bf16(acts[li]), w, dil, _bf16(g))
        gb = g.sum(axis=(0, 2, 3, 4))
        got_w, got_b = grads[li]
        assert np.allclose(got_w.cpu().numpy(), gw, rtol=1e-3, atol=1e-5 * np.abs(gw).max()), li
        assert np.allclose(got_b.cpu().numpy(), gb, rtol=1e-3, atol=1e-5 * np.abs(gb).max()), li
        g = gx.astype(np.float32).astype(np.float64)
    st = ctypes_status()
    assert st == 0


def ctypes_status():
    import ctypes

    from paper_1806_10247_gb300 import surrogate as G

    L = G._nn()
    v = ctypes.c_int(-1)
    assert L.lbm_nn_tc_status(ctypes.byref(v)) == 0
    return v.value


@pytest.mark.parametrize("n,ci,co,k,dil,dhw", [
    (3, 5, 16, (1, 3, 3), (1, 1, 1), (1, 20, 17)),    # the network's first layer; ragged last pixel tile
    (2, 16, 16, (1, 3, 3), (1, 4, 4), (1, 33, 30)),   # a dilated middle layer; two weight-row tiles (144)
    (2, 16, 1, (1, 1, 1), (1, 1, 1), (1, 40, 9)),     # the linear output layer (one output channel)
    (1, 3, 5, (3, 3, 1), (1, 2, 1), (4, 9, 6)),       # a 3D kernel
    (1, 56, 64, (1, 3, 3), (1, 1, 1), (1, 12, 11)),   # K = 504 and N = 64: the tile limits
    (2, 4, 8, (1, 3, 3), (1, 2, 2), (1, 128, 70)),    # 140 pixel chunks: blocks taking two chunks each
])
def test_tensor_core_conv_against_bf16_rounded_reference(n, ci, co, k, dil, dhw):
    """The three tensor-core products (forward, input gradient, weight
    gradient) against the FP64 numpy convolution of the same BF16-rounded
    operands: exact products, so only the FP32 summation order differs."""
    import ctypes

    from paper_1806_10247_gb300 import surrogate as G

    L = G._nn()
    rng = np.random.default_rng(sum(dhw) + ci + co)
    x = rng.standard_normal((n, ci) + dhw).astype(np.float32)
    w = _bf16(rng.standard_normal((co, ci) + k) / np.sqrt(ci * np.prod(k)))
    b = rng.standard_normal(co).astype(np.float32)
    gy = rng.standard_normal((n, co) + dhw).astype(np.float32)
    dx = torch.tensor(x, device="cuda")
    dw = torch.tensor(w, dtype=torch.float32, device="cuda").to(torch.bfloat16)
    db = torch.tensor(b, device="cuda")
    dy = torch.empty((n, co) + dhw, dtype=torch.float32, device="cuda")
    dgy = torch.tensor(gy, device="cuda")
    dgx = torch.empty_like(dx)
    dgw = torch.empty((co, ci) + k, dtype=torch.float32, device="cuda")
    dgb = torch.empty(co, dtype=torch.float32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    G._ck(L.lbm_nn_conv3d_forward(p(dx), p(dw), 1, p(db), p(dy), n, ci, co, G._i3(dhw), G._i3(k), G._i3(dil), 0, s))
    G._ck(L.lbm_nn_conv3d_backward(p(dx), p(dw), 1, p(dgy), p(dgx), p(dgw), p(dgb), n, ci, co, G._i3(dhw), G._i3(k),
                                   G._i3(dil), s))
    torch.cuda.synchronize()
    assert ctypes_status() == 0
    taps = int(np.prod(k))
    # a product whose padded shape exceeds one tile runs on the CUDA cores
    # with FP32 operands (here: the input gradient of the 56 -> 64 layer, K = 576)
    tc = {"y": ci * taps <= 512 and co <= 64, "gx": co * taps <= 512 and ci <= 64, "gw": ci * taps <= 512 and co <= 64}
    rnd = {name: (_bf16 if on else (lambda a: np.asarray(a, np.float64))) for name, on in tc.items()}
    y_ref = S.conv3d(rnd["y"](x), w, b.astype(np.float64), dil)
    gx_ref = S.conv3d_backward(x.astype(np.float64), w, dil, rnd["gx"](gy))[0]
    gw_ref = S.conv3d_backward(rnd["gw"](x), w, dil, rnd["gw"](gy))[1]
    gb_ref = gy.astype(np.float64).sum(axis=(0, 2, 3, 4))
    tol = {"y": 2e-5, "gx": 2e-5, "gw": 1e-4, "gb": 1e-5}
    for got, want, name in ((dy, y_ref, "y"), (dgx, gx_ref, "gx"), (dgw, gw_ref, "gw"), (dgb, gb_ref, "gb")):
        g = got.cpu().numpy().astype(np.float64)
        err = np.abs(g - want).max() / np.abs(want).max()
        assert err <= tol[name], (name, err)
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


def test_warm_started_converged_field_matches_oracle():
    """The LB iteration alone decides the converged field: a duct section
    (n = 12) started from a network's prediction (here untrained, so far from
    the answer) and iterated to a residual of 1e-12 per 100 steps equals the
    FP64 oracle's field iterated from rest to the same residual, to 1e-9
    relative l2."""
    from paper_1806_10247_gb300 import lbm
    from paper_1806_10247_gb300 import surrogate as G
    from tests.gpu_helpers import oracle_from_workload

    n, F0, nu = 12, 1e-5, 0.05
    w = G.section(n, F0, nu)
    net = G.ConvNet(seed=3, bf16=True)
    ux = G.predict(net, n, F0, nu)
    L = lbm.from_workload(w)
    u = np.zeros((3, n * n))
    u[0] = ux.T.reshape(-1)
    L.init_equilibrium(1.0, u)
    steps, _ = G.run_to_steady([L], n, tol=1e-12)
    ug = G.ux_field(L, n)
    R = oracle_from_workload(w)
    prev = R.moments()[1][0].copy()
    k = 0
    while k < 200000:
        R.run(100)
        k += 100
        cur = R.moments()[1][0]
        if np.abs(cur - prev).max() / np.abs(cur).max() < 1e-12:
            break
        prev = cur.copy()
    ur = cur.reshape(n, n)  # [z][y], as ux_field
    start = np.sqrt(np.sum((ux.T - ur) ** 2) / np.sum(ur ** 2))
    err = np.sqrt(np.sum((ug - ur) ** 2) / np.sum(ur ** 2))
    assert start > 1e-2, start  # the start really was far from the answer
    assert err < 1e-9, (err, steps, k)

"""Pins of the numpy FP64 reference of the warm-start network: convolution
against a brute-force sum, gradients against central finite differences,
Adam's first step against its closed form."""
import numpy as np

from oracle import surrogate_ref as S


def _brute_conv(x, w, b, dil):
    N, Ci, D, H, V = x.shape
    Co, _, KD, KH, KW = w.shape
    y = np.zeros((N, Co, D, H, V))
    for n in range(N):
        for o in range(Co):
            for d in range(D):
                for h in range(H):
                    for v in range(V):
                        acc = b[o]
                        for i in range(Ci):
                            for a in range(KD):
                                for c in range(KH):
                                    for e in range(KW):
                                        dd = d + dil[0] * (a - (KD - 1) // 2)
                                        hh = h + dil[1] * (c - (KH - 1) // 2)
                                        vv = v + dil[2] * (e - (KW - 1) // 2)
                                        if 0 <= dd < D and 0 <= hh < H and 0 <= vv < V:
                                            acc += w[o, i, a, c, e] * x[n, i, dd, hh, vv]
                        y[n, o, d, h, v] = acc
    return y


def test_conv3d_matches_brute_force():
    rng = np.random.default_rng(0)
    for k, dil in [((3, 3, 1), (1, 2, 1)), ((1, 3, 3), (1, 1, 2)), ((3, 1, 3), (2, 1, 1)), ((1, 1, 1), (1, 1, 1))]:
        x = rng.standard_normal((2, 2, 3, 4, 5))
        w = rng.standard_normal((3, 2) + k)
        b = rng.standard_normal(3)
        assert np.allclose(S.conv3d(x, w, b, dil), _brute_conv(x, w, b, dil), atol=1e-12)


def _net(rng):
    layers = [(3, 4, (1, 3, 3), (1, 1, 1), "tanh"), (4, 4, (1, 3, 3), (1, 2, 2), "tanh"),
              (4, 1, (1, 1, 1), (1, 1, 1), None)]
    params = [(0.3 * rng.standard_normal((co, ci) + k), 0.1 * rng.standard_normal(co))
              for ci, co, k, dil, act in layers]
    return S.Net(layers, params)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    net = _net(rng)
    x = rng.standard_normal((2, 3, 1, 6, 5))
    t = rng.standard_normal((2, 1, 1, 6, 5))
    loss, grads = net.loss_and_grads(x, t)
    eps = 1e-6
    for li, (w, b) in enumerate(net.params):
        for arr, g in ((w, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            gflat = g.reshape(-1)
            for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[j]
                flat[j] = old + eps
                lp, _ = net.loss_and_grads(x, t)
                flat[j] = old - eps
                lm, _ = net.loss_and_grads(x, t)
                flat[j] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gflat[j]) <= 1e-6 * max(1.0, abs(fd)), (li, j, fd, gflat[j])


def test_adam_first_step_is_lr_times_sign():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    p0 = p.copy()
    S.adam_step(p, g, m, v, t=1, lr=0.01)
    assert np.allclose(p0 - p, 0.01 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)

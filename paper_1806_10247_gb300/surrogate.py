"""Learned warm start of the LB iteration (no counterpart in the paper).

A small 3D convolutional network predicts the steady velocity of a
body-force-driven square duct (x periodic, halfway bounce-back walls in y and
z, F_x = F0 (1 + 0.5 sin(2 pi z / n))) from the force shape, the wall
geometry and the relaxation time.  The prediction initialises the LB
populations (equilibrium at the predicted velocity); the LB iteration then
runs to the same convergence criterion as from rest and alone decides
the converged field.

Everything numeric runs in the library's CUDA kernels (``lbm_nn_*`` for the
network, ``lbm_*`` for the LB); torch tensors only hold device memory.  The
steady flow is x-invariant, so the grids are one node thick in x (nx = 1, a
periodic axis) and the convolutions use 1 x 3 x 3 kernels with dilations
1, 2, 4, 8 to reach across the section.  Physics-informed scaling: the
network predicts U = u_x nu / (F0 n^2), because the Stokes solution is
proportional to F0 / nu.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np

from . import lbm
from . import workloads as W

N_FEATURES = 5
DEFAULT_LAYERS = [
    (N_FEATURES, 16, (1, 3, 3), (1, 1, 1), "tanh"),
    (16, 16, (1, 3, 3), (1, 2, 2), "tanh"),
    (16, 16, (1, 3, 3), (1, 4, 4), "tanh"),
    (16, 16, (1, 3, 3), (1, 8, 8), "tanh"),
    (16, 1, (1, 1, 1), (1, 1, 1), None),
]


def _nn():
    L = lbm.load()
    if not hasattr(L, "_nn_ready"):
        vp, ip, ll, dd = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        i3 = ctypes.POINTER(ctypes.c_int)
        L.lbm_nn_conv3d_forward.argtypes = [vp, vp, ip, vp, vp, ip, ip, ip, i3, i3, i3, ip, vp]
        L.lbm_nn_conv3d_backward.argtypes = [vp, vp, ip, vp, vp, vp, vp, ip, ip, ip, i3, i3, i3, vp]
        L.lbm_nn_tanh_backward.argtypes = [vp, vp, ll, vp]
        L.lbm_nn_mse.argtypes = [vp, vp, vp, ll, vp, vp]
        L.lbm_nn_adam.argtypes = [vp, vp, vp, vp, vp, ll, dd, dd, dd, dd, ll, vp]
        L.lbm_nn_to_bf16.argtypes = [vp, vp, ll, vp]
        L.lbm_nn_last_error.restype = ctypes.c_char_p
        L.lbm_nn_tc_status.argtypes = [ctypes.POINTER(ctypes.c_int)]
        L.lbm_nn_tc_status.restype = ctypes.c_int
        for f in ("lbm_nn_conv3d_forward", "lbm_nn_conv3d_backward", "lbm_nn_tanh_backward", "lbm_nn_mse",
                  "lbm_nn_adam", "lbm_nn_to_bf16"):
            getattr(L, f).restype = ctypes.c_int
        L._nn_ready = True
    return L


def _ck(rc):
    if rc != 0:
        raise lbm.LBMError(rc, _nn().lbm_nn_last_error().decode())


def _i3(v):
    return (ctypes.c_int * 3)(*[int(a) for a in v])


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class ConvNet:
    """The surrogate: conv layers (Cin, Cout, kernel, dilation, act) on CUDA
    tensors.  Master weights FP32, forward/backward read the BF16 copy when
    ``bf16`` (FP32 accumulation), Adam updates both."""

    def __init__(self, layers=DEFAULT_LAYERS, seed=0, bf16=True):
        import torch

        self.torch = torch
        self.layers = layers
        self.bf16 = bf16
        rng = np.random.default_rng(seed)
        self.W, self.B, self.Wb, self.m, self.v = [], [], [], [], []
        for ci, co, k, dil, act in layers:
            fan = ci * k[0] * k[1] * k[2]
            w = rng.standard_normal((co, ci) + tuple(k)) * math.sqrt(1.0 / fan)
            self.W.append(torch.tensor(w, dtype=torch.float32, device="cuda"))
            self.B.append(torch.zeros(co, dtype=torch.float32, device="cuda"))
            self.Wb.append(torch.empty(self.W[-1].shape, dtype=torch.bfloat16, device="cuda"))
        # Adam moments, interleaved per layer: m[2l], v[2l] for W[l]; m[2l+1], v[2l+1] for B[l]
        for w, b in zip(self.W, self.B):
            for t in (w, b):
                self.m.append(torch.zeros_like(t))
                self.v.append(torch.zeros_like(t))
        self.step_count = 0
        self.refresh_bf16()

    @property
    def stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def refresh_bf16(self):
        for w, wb in zip(self.W, self.Wb):
            _ck(_nn().lbm_nn_to_bf16(_p(w), _p(wb), w.numel(), self.stream))

    def _w(self, li):
        return (self.Wb[li], 1) if self.bf16 else (self.W[li], 0)

    def forward(self, x):
        """x: float32 CUDA tensor [N, C, D, H, W]; returns (y, activations)."""
        acts = [x.contiguous()]
        h = acts[0]
        for li, (ci, co, k, dil, act) in enumerate(self.layers):
            if h.dtype != self.torch.float32 or h.dim() != 5 or h.shape[1] != ci or not h.is_cuda:
                raise ValueError(f"layer {li}: input {tuple(h.shape)} {h.dtype}, expected [N, {ci}, D, H, W] float32 CUDA")
            N, _, D, H, V = h.shape
            y = self.torch.empty((N, co, D, H, V), dtype=self.torch.float32, device="cuda")
            w, wflag = self._w(li)
            _ck(_nn().lbm_nn_conv3d_forward(_p(h), _p(w), wflag, _p(self.B[li]), _p(y), N, ci, co, _i3((D, H, V)),
                                            _i3(k), _i3(dil), 1 if act == "tanh" else 0, self.stream))
            acts.append(y)
            h = y
        return h, acts

    def loss_and_grads(self, x, target):
        """MSE loss (float) and gradients (list of (gW, gB)) by the backward kernels."""
        torch = self.torch
        y, acts = self.forward(x)
        if target.shape != y.shape or target.dtype != torch.float32:
            raise ValueError(f"target {tuple(target.shape)} {target.dtype}, expected {tuple(y.shape)} float32")
        g = torch.empty_like(y)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        _ck(_nn().lbm_nn_mse(_p(y), _p(target.contiguous()), _p(g), y.numel(), _p(loss), self.stream))
        grads = [None] * len(self.layers)
        for li in range(len(self.layers) - 1, -1, -1):
            ci, co, k, dil, act = self.layers[li]
            if act == "tanh":
                _ck(_nn().lbm_nn_tanh_backward(_p(g), _p(acts[li + 1]), g.numel(), self.stream))
            xin = acts[li]
            N, _, D, H, V = xin.shape
            gw = torch.empty_like(self.W[li])
            gb = torch.empty_like(self.B[li])
            gx = torch.empty_like(xin) if li > 0 else None
            w, wflag = self._w(li)
            _ck(_nn().lbm_nn_conv3d_backward(_p(xin), _p(w), wflag, _p(g), _p(gx), _p(gw), _p(gb), N, ci, co,
                                             _i3((D, H, V)), _i3(k), _i3(dil), self.stream))
            grads[li] = (gw, gb)
            g = gx
        return float(loss.item()), grads

    def adam_step(self, grads, lr=2e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for li, (gw, gb) in enumerate(grads):
            # every buffer handed to a kernel must match the parameter it updates
            for t in (gw, self.m[2 * li], self.v[2 * li], self.Wb[li]):
                if t.numel() != self.W[li].numel():
                    raise ValueError(f"layer {li}: buffer of {t.numel()} values for {self.W[li].numel()} weights")
            for t in (gb, self.m[2 * li + 1], self.v[2 * li + 1]):
                if t.numel() != self.B[li].numel():
                    raise ValueError(f"layer {li}: buffer of {t.numel()} values for {self.B[li].numel()} biases")
            _ck(_nn().lbm_nn_adam(_p(self.W[li]), _p(gw), _p(self.m[2 * li]), _p(self.v[2 * li]),
                                  _p(self.Wb[li]), self.W[li].numel(), lr, b1, b2, eps, self.step_count, self.stream))
            _ck(_nn().lbm_nn_adam(_p(self.B[li]), _p(gb), _p(self.m[2 * li + 1]), _p(self.v[2 * li + 1]), None,
                                  self.B[li].numel(), lr, b1, b2, eps, self.step_count, self.stream))


# ---------------------------------------------------------------- problem ---

def section(n: int, F0: float, nu: float) -> W.Workload:
    """Duct cross-section, one node thick in x (periodic), walls in y and z."""
    z = np.arange(n, dtype=np.float64)
    pz = F0 * (1.0 + 0.5 * np.sin(2.0 * math.pi * z / n))
    one, zero = np.array([1.0]), np.array([0.0])
    return W.Workload(name=f"duct_section_{n}", lattice=W.D3Q27, shape=(1, n, n), wall=(0, 1, 1),
                      omega=W.d3q27_omega(W.tau_from_nu(nu)), rho0=1.0, u0=(0.0, 0.0, 0.0),
                      tables=[(one, one, pz), (zero, one, one), (zero, one, one)], meta={"F0": F0, "nu": nu})


def features(n: int, nu: float) -> np.ndarray:
    """Input channels [5][1][n][n] (index [c][x][y][z] -> stored as [c][D=1][H=y][W=z]):
    force shape, wall distances in y and z, tau - 1/2, constant 1."""
    y = np.arange(n) + 0.5
    dy = np.minimum(y, n - y) / (n / 2.0)
    z = np.arange(n, dtype=np.float64)
    shape = 1.0 + 0.5 * np.sin(2.0 * math.pi * z / n)
    f = np.empty((N_FEATURES, 1, n, n))
    f[0, 0] = shape[None, :]
    f[1, 0] = dy[:, None]
    f[2, 0] = dy[None, :]
    f[3, 0] = W.tau_from_nu(nu) - 0.5
    f[4, 0] = 1.0
    return f


def draw_params(count: int, n: int, seed: int, umax: float = 0.1):
    """(F0, nu): F0 log-uniform in [1e-6, 1e-4], nu uniform in [0.01, 0.1];
    draws whose centre-line speed would exceed umax are redrawn
    (u_c ~ 0.2947 F0 a^2 / nu for a duct of half-width a = n/2, times 1.5 for
    the force's largest value)."""
    rng = np.random.default_rng(seed)
    out = []
    a = n / 2.0
    while len(out) < count:
        F0 = 10.0 ** rng.uniform(-6.0, -4.0)
        nu = rng.uniform(0.01, 0.1)
        if 1.5 * 0.2947 * F0 * a * a / nu <= umax:
            out.append((F0, nu))
    return out


def ux_field(L: lbm.Lattice, n: int) -> np.ndarray:
    _, u = L.moments()
    return u[0].reshape(n, n)  # node index y + n z -> [z][y]; transposed below


def run_to_steady(lats, n, tol=1e-10, check_every=100, max_steps=4000000):
    """Step a batch of duct sections until every member's relative residual
    max |u(t) - u(t - check_every)| / max |u| is below tol (u_x of every
    member from one packed readback per check).  Returns the steps each
    member needed and the wall time of the whole batch."""
    B = lbm.Batch(lats)
    nn = n * n
    done = [None] * len(lats)
    steps = 0
    t0 = time.perf_counter()
    _, u = B.moments_packed()
    prev = [u[3 * i * nn:3 * i * nn + nn].copy() for i in range(len(lats))]
    while steps < max_steps and any(d is None for d in done):
        B.step(check_every)
        steps += check_every
        _, u = B.moments_packed()
        for i in range(len(lats)):
            cur = u[3 * i * nn:3 * i * nn + nn]
            if done[i] is None:
                scale = max(float(np.abs(cur).max()), 1e-300)
                if float(np.abs(cur - prev[i]).max()) / scale < tol:
                    done[i] = steps
            prev[i] = cur.copy()
    sec = time.perf_counter() - t0
    B.close()
    return [d if d is not None else max_steps for d in done], sec


def generate(n: int, count: int, seed: int, storage=lbm.FP64, tol=1e-10, check_every=100):
    """Method-generated training fields: (features [S,5,1,n,n], targets
    [S,1,1,n,n] = u_x nu / (F0 n^2), params)."""
    params = draw_params(count, n, seed)
    lats = [lbm.from_workload(section(n, F0, nu), storage=storage) for F0, nu in params]
    steps, sec = run_to_steady(lats, n, tol=tol, check_every=check_every)
    X = np.empty((count, N_FEATURES, 1, n, n), dtype=np.float32)
    Y = np.empty((count, 1, 1, n, n), dtype=np.float32)
    for s, ((F0, nu), L) in enumerate(zip(params, lats)):
        X[s] = features(n, nu)
        u = ux_field(L, n)  # [z][y]
        Y[s, 0, 0] = (u.T * nu / (F0 * n * n)).astype(np.float32)  # [y][z]
        L.close()
    return X, Y, params, {"steps": steps, "seconds": sec}


def train(net: ConvNet, X, Y, iters=1500, batch=32, lr=2e-3, seed=0, log_every=0, lr_final=None):
    """Adam on minibatches; X, Y numpy.  With lr_final the step size follows a
    cosine from lr down to lr_final over the iterations (a stable end point
    instead of the last noisy minibatch).  Returns the loss history."""
    torch = net.torch
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.tensor(Y, device="cuda")
    rng = np.random.default_rng(seed)
    hist = []
    S = X.shape[0]
    for it in range(iters):
        idx = torch.tensor(rng.choice(S, size=min(batch, S), replace=False), device="cuda")
        loss, grads = net.loss_and_grads(Xd[idx], Yd[idx])
        step = lr
        if lr_final is not None:
            step = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * it / max(iters - 1, 1)))
        net.adam_step(grads, lr=step)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {loss:.3e}")
    return hist


def predict(net: ConvNet, n: int, F0: float, nu: float) -> np.ndarray:
    torch = net.torch
    x = torch.tensor(features(n, nu)[None].astype(np.float32), device="cuda")
    y, _ = net.forward(x)
    U = y[0, 0, 0].cpu().numpy().astype(np.float64)  # [y][z]
    return U * F0 * n * n / nu


def warm_start_study(net: ConvNet, n: int, cases, tol=1e-10, storage=lbm.FP64):
    """Steps and wall time to the residual tol from rest and from the network's
    prediction, for each (F0, nu); the two converged fields are compared."""
    out = []
    for F0, nu in cases:
        w = section(n, F0, nu)
        cold = lbm.from_workload(w, storage=storage)
        warm = lbm.from_workload(w, storage=storage)
        t0 = time.perf_counter()
        ux = predict(net, n, F0, nu)  # [y][z]
        u = np.zeros((3, n * n))
        u[0] = ux.T.reshape(-1)  # node index y + n z
        warm.init_equilibrium(1.0, u)
        t_pred = time.perf_counter() - t0
        s_cold, sec_cold = run_to_steady([cold], n, tol=tol)
        s_warm, sec_warm = run_to_steady([warm], n, tol=tol)
        uc = ux_field(cold, n)
        uw = ux_field(warm, n)
        diff = float(np.sqrt(np.sum((uc - uw) ** 2) / np.sum(uc ** 2)))
        pred_err = float(np.sqrt(np.sum((ux.T - uc) ** 2) / np.sum(uc ** 2)))
        out.append({"F0": F0, "nu": nu, "steps_cold": s_cold[0], "steps_warm": s_warm[0],
                    "seconds_cold": sec_cold, "seconds_warm": sec_warm + t_pred,
                    "prediction_l2": pred_err, "converged_fields_l2": diff})
        cold.close()
        warm.close()
    return out


def study(n=64, train_count=500, test_count=8, iters=4000, seed=10247, gen_storage=lbm.FP32_DEV,
          gen_tol=1e-7, tol=1e-10, check_every=100):
    """The full warm-start experiment: method-generated training fields (FP32
    storage, residual gen_tol), training on the GPU, then for held-out
    parameters steps and wall time to the FP64 residual tol from rest and from
    the prediction (all held-out cases stepped together as one batch each)."""
    t0 = time.perf_counter()
    X, Y, params, gen = generate(n, train_count, seed, storage=gen_storage, tol=gen_tol, check_every=check_every)
    t_gen = time.perf_counter() - t0
    net = ConvNet(seed=0, bf16=True)
    t0 = time.perf_counter()
    hist = train(net, X, Y, iters=iters, batch=32, lr=2e-3, seed=seed, lr_final=2e-5)
    net.torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    cases = draw_params(test_count, n, seed + 1)
    cold = [lbm.from_workload(section(n, F0, nu)) for F0, nu in cases]
    warm = []
    preds = []
    t0 = time.perf_counter()
    for F0, nu in cases:
        L = lbm.from_workload(section(n, F0, nu))
        ux = predict(net, n, F0, nu)
        u = np.zeros((3, n * n))
        u[0] = ux.T.reshape(-1)
        L.init_equilibrium(1.0, u)
        warm.append(L)
        preds.append(ux)
    t_pred = time.perf_counter() - t0
    s_cold, sec_cold = run_to_steady(cold, n, tol=tol, check_every=check_every)
    s_warm, sec_warm = run_to_steady(warm, n, tol=tol, check_every=check_every)
    rows = []
    for (F0, nu), c, w, ux, sc, sw in zip(cases, cold, warm, preds, s_cold, s_warm):
        uc, uw = ux_field(c, n), ux_field(w, n)
        rows.append({"F0": F0, "nu": nu, "steps_cold": sc, "steps_warm": sw,
                     "prediction_l2": float(np.sqrt(np.sum((ux.T - uc) ** 2) / np.sum(uc ** 2))),
                     "converged_fields_l2": float(np.sqrt(np.sum((uc - uw) ** 2) / np.sum(uc ** 2)))})
    return {"n": n, "train_fields": train_count, "generation_seconds": t_gen, "generation_tol": gen_tol,
            "tol": tol, "check_every": check_every,
            "generation_steps_max": int(max(gen["steps"])), "train_iters": iters, "train_seconds": t_train,
            "loss_first": hist[0], "loss_last": hist[-1], "prediction_seconds": t_pred,
            "cold": {"steps_total": int(sum(s_cold)), "seconds": sec_cold},
            "warm": {"steps_total": int(sum(s_warm)), "seconds": sec_warm + t_pred},
            "cases": rows}


"""Shared pieces of the GPU parity tests: running one workload through the
CUDA library and through the oracle, and the FP64 parity metric.

Parity metric (FP64), after the same number of steps from the same inputs:
  f   : max |f_gpu - f_ref|     <= 1e-12 * max |f_ref|
  rho : max |rho_gpu - rho_ref| <= 1e-12 * max |rho_ref|   (phi likewise)
  u   : max |u_gpu - u_ref|     <= 1e-12 * max(max |u_ref|, U_floor)
        U_floor = 1e-3 for the 2D lattices, 5e-3 for the 3D ones
  phi - mean(phi): max |phi_gpu - phi_ref| <= 1e-12 * max(max |phi_ref - mean|, 0.01 |mean|)
Populations are O(0.1) and every FP64 evaluation of the step rounds them; two
correct evaluations in different operation orders (the oracle's dense moment
matrices and the kernels' factorised transforms) differ in u = sum f e / rho
by a few units of eps * sum |f e| / rho (eps = 2^-53): one rounding of a
velocity sum is ~1e-16 absolute, whatever |u| is.  So the plain relative
1e-12 holds wherever |u| is large enough for 1e-12 |u| to exceed the
accumulated rounding, and below that the velocity is measured against a
floor set at that rounding: 1e-15 absolute (about 9 eps) for the 9-term sums
of the 2D lattices, 5e-15 (about 45 eps) for the 15- and 27-term sums of the
3D lattices over runs of up to 1000 steps.  Measured on the GB300 over every
parity case: at most 3.7e-13 (2D, the Poiseuille channel after 10^4 steps)
and 6.1e-13 (3D, Kolmogorov 64^3 after 1000 steps) of the bar.  The plain
relative errors are returned as "u_rel" / "phi_var_rel".
"""
import os

import numpy as np

from oracle import oracle as O
from paper_1806_10247_gb300 import lbm

TOL = 1e-12


def oracle_from_workload(w, f0=None):
    lat = w.lattice
    P = O.expand_separable(w.tables, w.shape) if w.tables is not None else None
    uadv = None
    if lat == O.D2Q5:
        u = np.asarray(w.u0, np.float64)
        uadv = np.stack([np.full(w.nodes, u[0]), np.full(w.nodes, u[1])])
    L = O.OracleLattice(lat, w.shape, wall=w.wall, omega=w.omega, P=P, envelope=w.envelope, uadv=uadv)
    if f0 is None:
        L.init_equilibrium(w.rho0, w.u0)
    else:
        L.f = np.ascontiguousarray(f0, dtype=np.float64)
        L.t = 0
    return L


U_FLOOR_2D, U_FLOOR_3D = 1e-3, 5e-3
PHI_VAR_FLOOR = 0.01


def compare_state(G, R, rho0=1.0, tol=TOL):
    """Compare a GPU lattice G with an oracle lattice R at the same step.
    Returns the errors; "u_rel" is the plain max |du| / max |u_ref| (no floor)."""
    assert G.t == R.t
    fg = G.get_populations()
    fr = R.f
    err = {"f": np.abs(fg - fr).max() / np.abs(fr).max()}
    info = {}
    if G.lattice == lbm.D2Q5_CDE:
        pg = G.moments()
        pr = R.moments()
        err["phi"] = np.abs(pg - pr).max() / np.abs(pr).max()
        m = abs(pr.mean())
        scale = max(np.abs(pr - pr.mean()).max(), PHI_VAR_FLOOR * m, 1e-300)
        err["phi_var"] = np.abs(pg - pr).max() / scale
        info["phi_var_rel"] = np.abs(pg - pr).max() / max(np.abs(pr - pr.mean()).max(), 1e-300)
        info["phi_abs"] = np.abs(pg - pr).max()
        info["phi_var_max"] = np.abs(pr - pr.mean()).max()
    else:
        floor = U_FLOOR_3D if G.dim == 3 else U_FLOOR_2D
        rg, ug = G.moments()
        rr, ur = R.moments()
        err["rho"] = np.abs(rg - rr).max() / np.abs(rr).max()
        err["u"] = np.abs(ug - ur).max() / max(np.abs(ur).max(), floor)
        info["u_rel"] = np.abs(ug - ur).max() / max(np.abs(ur).max(), 1e-300)
        info["u_abs"] = np.abs(ug - ur).max()
        info["u_max"] = np.abs(ur).max()
        rg0, ug0 = G.moments(half_forced=False)
        rr0, ur0 = R.moments(half_forced=False)
        err["u_out"] = np.abs(ug0 - ur0).max() / max(np.abs(ur0).max(), floor)
        info["u_out_abs"] = np.abs(ug0 - ur0).max()
    err.update(info)
    record(err, tol)
    for k, v in err.items():
        if k in info:
            continue
        assert v <= tol, (k, v, err, info)
    return err


# Every comparison's errors, in call order (written to a JSON file at the end
# of the session when LBM_RESULTS_DIR is set; see conftest.py).
RECORDS = []


def record(err, tol, **extra):
    r = {"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "tol": tol}
    r.update({k: float(v) for k, v in err.items()})
    r.update(extra)
    RECORDS.append(r)


def separable_at(tables, shape, nodes):
    """Separable shape (px[x] * py[y]) * pz[z] at the given node indices
    ([ncomp][len(nodes)]), in the product order of the full field."""
    nx, ny, nz = shape
    x, y, z = nodes % nx, (nodes // nx) % ny, nodes // (nx * ny)
    out = []
    for px, py, pz in tables:
        px = np.broadcast_to(np.asarray(px, np.float64), (nx,))
        py = np.broadcast_to(np.asarray(py, np.float64), (ny,))
        pz = np.broadcast_to(np.asarray(pz, np.float64), (nz,))
        out.append((px[x] * py[y]) * pz[z])
    return np.stack(out)


def one_step_sampled(w, G, samples, seed, tol=1e-12, device=False):
    """Full-size check for grids too large for a whole-grid oracle run: take the
    GPU's f(t), let the oracle collide the pull-neighbours of sampled nodes and
    stream them in, and compare with the GPU's f(t+1) at those nodes.  With
    device=True the two states stay in device memory and only the columns the
    check needs come to the host (for grids whose f does not fit host memory
    comfortably)."""
    E = O.velocities(w.lattice)
    q = E.shape[0]
    nx, ny, nz = w.shape
    opp = [int(np.where((E == -E[a]).all(1))[0][0]) for a in range(q)]
    rng = np.random.default_rng(seed)
    nxy = nx * ny
    edges = np.array([0, w.nodes - 1, nx - 1, w.nodes - nx, nx * (ny // 2)], dtype=np.int64)
    idx = np.concatenate([edges[edges < w.nodes], rng.integers(0, w.nodes, samples)])
    samples = len(idx)
    # pull source (node, component) of every sampled node and population
    src = np.empty((samples, q), dtype=np.int64)
    comp = np.empty((samples, q), dtype=np.int64)
    for k, i in enumerate(idx):
        x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
        for a in range(q):
            s_ = [x - E[a, 0], y - E[a, 1], z - E[a, 2]]
            n = [nx, ny, nz]
            out = False
            for d in range(3):
                if s_[d] < 0 or s_[d] >= n[d]:
                    if w.wall[d]:
                        out = True
                    else:
                        s_[d] %= n[d]
            # pulled value: post-collision population a of the source node, or
            # the opposite population of this node beyond a wall
            src[k, a], comp[k, a] = (i, opp[a]) if out else (s_[0] + nx * (s_[1] + ny * s_[2]), a)
    need = np.unique(np.concatenate([src.reshape(-1), idx]))
    pos = {int(v): j for j, v in enumerate(need)}
    t = G.t
    if device:
        import torch

        buf = torch.empty((q, w.nodes), dtype=torch.float64, device="cuda")
        sel = torch.from_numpy(need).to("cuda")
        G.get_populations(out=buf, where=1)
        G.sync()
        ft = buf[:, sel].cpu().numpy()
        G.step(1)
        G.get_populations(out=buf, where=1)
        G.sync()
        ft1 = buf[:, sel].cpu().numpy()
        scale = max(float(buf.max().item()), -float(buf.min().item()))  # no |f| temporary
        del buf
        torch.cuda.empty_cache()
    else:
        f_t = G.get_populations()
        G.step(1)
        f_t1 = G.get_populations()
        ft, ft1, scale = f_t[:, need], f_t1[:, need], np.abs(f_t1).max()
    R = O.OracleLattice(w.lattice, (1, 1, 1), omega=w.omega)  # single-node collisions only
    P = separable_at(w.tables, w.shape, need) if w.tables is not None else None
    pre, post = (O.envelope_pairs(w.envelope, t, 1) if w.envelope else (1.0, 1.0))
    dim = 3 if w.lattice in (O.D3Q27, O.D3Q15) else 2
    # the scalar lattice collides about its (uniform) advecting velocity
    uadv = np.asarray(w.u0[:2], np.float64) if w.lattice == O.D2Q5 else None
    if uadv is not None and np.ndim(w.u0) != 1:
        raise ValueError("sampled check: D2Q5 needs a uniform advecting velocity")
    worst = 0.0
    for k, i in enumerate(idx):
        want = np.empty(q)
        for a in range(q):
            j = pos[int(src[k, a])]
            Fpre = pre * P[:, j] if P is not None else np.zeros(dim)
            Fpost = post * P[:, j] if P is not None else np.zeros(dim)
            want[a] = R.collide_node(ft[:, j], Fpre, Fpost, uadv=uadv)[comp[k, a]]
        worst = max(worst, np.abs(ft1[:, pos[int(i)]] - want).max() / scale)
    record({"f": worst}, tol, samples=samples, nodes=w.nodes)
    assert worst <= tol, worst
    return worst

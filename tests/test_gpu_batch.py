"""Batched stepping (one launch per step for many lattices): bit-identical to
stepping each member alone, and within the parity bar of the oracle; envelope
tables equal envelope callbacks."""
import dataclasses
import math

import numpy as np
import pytest

from paper_1806_10247_gb300 import lbm
from paper_1806_10247_gb300 import workloads as W
from tests.gpu_helpers import compare_state, oracle_from_workload
from tests.test_gpu_parity import _random_workload

pytestmark = pytest.mark.gpu


def _members(kind):
    if kind == "d2q5":
        ws = [W.cde_workload(c) for c in W.cde_sweep_params(sizes=(32, 48, 64, 100))]
        w, full = _random_workload(W.D2Q5, (37, 21, 1), (1, 1, 0), seed=4, kind="full")
        ws.append(w)
        fulls = [None] * 4 + [full]
    elif kind == "d2q9":
        ws = [W.poiseuille(ny=n) for n in (9, 33, 65)]
        w, full = _random_workload(W.D2Q9, (29, 17, 1), (0, 0, 0), seed=5, kind="full")
        w2, _ = _random_workload(W.D2Q9, (40, 7, 1), (1, 0, 0), seed=6)
        # unit higher rates with a force that has a y component: the
        # unit-rates collision with its y terms (batch variant 1), beside the
        # channels' force-along-x form (variant 3)
        w3, _ = _random_workload(W.D2Q9, (15, 12, 1), (0, 1, 0), seed=12)
        w3 = dataclasses.replace(w3, omega=W.d2q9_omega(0.9))
        ws += [w, w2, w3]
        fulls = [None, None, None, full, None, None]
    elif kind == "d3q15":
        ws = [W.duct15(n=9, nx=4)]
        w, full = _random_workload(W.D3Q15, (7, 6, 5), (1, 1, 1), seed=9, kind="full")
        w2, _ = _random_workload(W.D3Q15, (5, 8, 6), (0, 1, 0), seed=10)
        ws += [w, w2]
        fulls = [None, full, None]
    else:
        ws = [W.kolmogorov(shape=(12, 10, 8)), W.duct(n=9, nx=4)]
        w, full = _random_workload(W.D3Q27, (7, 6, 5), (1, 1, 1), seed=8, kind="full")
        # unit higher rates with y and z force components (batch variant 1)
        # beside the force-along-x members (variant 3)
        w3, _ = _random_workload(W.D3Q27, (6, 7, 5), (0, 1, 0), seed=13)
        w3 = dataclasses.replace(w3, omega=W.d3q27_omega(0.7))
        ws += [w, w3]
        fulls = [None, None, full, None]
    return ws, fulls


def _make(w, full, envelope_steps=None):
    G = lbm.from_workload(w, envelope_steps=envelope_steps)
    if full is not None:
        if w.lattice == W.D2Q5:
            G.set_source(full=full)
        else:
            G.set_force(full=full)
    return G


@pytest.mark.parametrize("kind", ["d2q5", "d2q9", "d3q27", "d3q15"])
def test_batch_equals_individual_steps_bitwise(kind):
    ws, fulls = _members(kind)
    solo = [_make(w, f) for w, f in zip(ws, fulls)]
    grouped = [_make(w, f) for w, f in zip(ws, fulls)]
    B = lbm.Batch(grouped)
    for n in (1, 2, 5):
        B.step(n)
        for G in solo:
            G.step(n)
    assert B.launch_count() == 8
    diffs = []
    for a, b in zip(solo, grouped):
        assert a.t == b.t == 8
        diffs.append(float(np.abs(a.get_populations() - b.get_populations()).max()))
    # same arithmetic in both kernels; the compiler may fuse multiply-adds
    # differently in the kernels (seen for D2Q9: ~1 ulp per step), so allow
    # 4 ulps of f per step
    assert max(diffs) <= 8 * 4 * 2.0 ** -53, diffs


def test_batch_after_a_member_stepped_alone():
    """A member stepped on its own falls out of parity lockstep, and a member
    whose source changes gets a new descriptor; the batch must notice both."""
    ws, fulls = _members("d2q5")
    solo = [_make(w, f) for w, f in zip(ws, fulls)]
    grouped = [_make(w, f) for w, f in zip(ws, fulls)]
    B = lbm.Batch(grouped)
    new_src = [np.full((1, G.N), 1e-5) for G in grouped]
    # grouped sequence
    B.step(2)
    grouped[1].step(1)
    B.step(3)
    grouped[2].set_source(full=new_src[2])
    B.step(1)
    # the same sequence, every lattice on its own
    for G in solo:
        G.step(2)
    solo[1].step(1)
    for G in solo:
        G.step(3)
    solo[2].set_source(full=new_src[2])
    for G in solo:
        G.step(1)
    for a, b in zip(solo, grouped):
        assert a.t == b.t
        assert np.array_equal(a.get_populations(), b.get_populations())


@pytest.mark.parametrize("kind", ["d2q5", "d2q9", "d3q27", "d3q15"])
def test_batch_matches_oracle(kind):
    ws, fulls = _members(kind)
    Gs = [_make(w, f) for w, f in zip(ws, fulls)]
    B = lbm.Batch(Gs)
    B.step(13)
    for w, f, G in zip(ws, fulls, Gs):
        R = oracle_from_workload(w)
        if f is not None:
            R.P = np.ascontiguousarray(f)
        R.run(13)
        compare_state(G, R)


def test_envelope_table_equals_callback():
    c = W.cde_sweep_params(sizes=(64,))[0]
    w = W.cde_workload(c)
    a = lbm.from_workload(w)
    b = lbm.from_workload(w, envelope_steps=40)
    a.step(25)
    b.step(25)
    assert np.array_equal(a.get_populations(), b.get_populations())
    assert np.array_equal(a.moments(), b.moments())
    with pytest.raises(lbm.LBMError) as e:
        b.step(30)  # beyond the 40-step table
    assert e.value.code == lbm.EINVAL


def test_batch_rejects_mixed_lattices_and_uninitialised_members():
    a = lbm.from_workload(W.poiseuille(ny=9))
    b = lbm.from_workload(W.cde_workload(W.cde_sweep_params(sizes=(32,))[0]))
    with pytest.raises(lbm.LBMError):
        lbm.Batch([a, b])
    with pytest.raises(lbm.LBMError):
        lbm.Batch([a, a])
    c = lbm.Lattice(lbm.D2Q9, (4, 4, 1), W.d2q9_omega(0.8))
    B = lbm.Batch([a, c])
    with pytest.raises(lbm.LBMError) as e:
        B.step(1)
    assert e.value.code == lbm.ESTATE


@pytest.mark.parametrize("kind,storage", [("d2q5", lbm.FP64), ("d2q9", lbm.FP64), ("d3q27", lbm.FP32_DEV)])
def test_graph_replays_equal_plain_launches(kind, storage):
    """Graph replays (4 launches each) plus a plain remainder give the same
    populations as stepping each member alone; a member stepped alone in
    between changes the parity and forces a new capture."""
    ws, fulls = _members(kind)
    solo = [_make(w, f) for w, f in zip(ws, fulls)]
    grp = [_make(w, f) for w, f in zip(ws, fulls)]
    if storage != lbm.FP64:
        solo = [lbm.from_workload(w, storage=storage) for w in ws]
        grp = [lbm.from_workload(w, storage=storage) for w in ws]
        for f, a, b in zip(fulls, solo, grp):
            if f is not None:
                (a.set_force if a.lattice != lbm.D2Q5_CDE else a.set_source)(full=f)
                (b.set_force if b.lattice != lbm.D2Q5_CDE else b.set_source)(full=f)
    B = lbm.Batch(grp)
    B.set_graph(4)
    B.step(10)
    grp[0].step(1)
    B.step(9)
    for G in solo:
        G.step(10)
    solo[0].step(1)
    for G in solo:
        G.step(9)
    assert B.graph_replays() == 4
    # the batch and single-lattice kernels contract multiply-adds differently:
    # a few ulps per step, accumulated over the 20 steps
    tol = 20 * 4 * 2.0 ** -53 if storage == lbm.FP64 else 1e-7
    for a, b in zip(solo, grp):
        assert a.t == b.t
        assert np.abs(a.get_populations() - b.get_populations()).max() <= tol


def _sweep_members(count=40):
    """A sweep large enough that a persistent grid holds fewer blocks than the
    batch has tiles (so that blocks take runs of several tiles)."""
    ch, sc = W.batched_sweep(count=count, seed=11, nx_range=(32, 200), ny_range=(32, 150))
    return ch, sc


@pytest.mark.parametrize("which", ["d2q9", "d2q5"])
def test_every_tiling_gives_the_same_populations(which):
    ch, sc = _sweep_members()
    ws = ch if which == "d2q9" else sc
    ref = [lbm.from_workload(w, storage=lbm.FP32_DEV) for w in ws]
    B = lbm.Batch(ref)
    assert B.tiling()[:2] == (256, False)
    B.step(5)
    want = [G.get_populations() for G in ref]
    scale = max(float(np.abs(f).max()) for f in want)
    for tile in (128, 256, 512):
        for persistent in (False, True):
            Gs = [lbm.from_workload(w, storage=lbm.FP32_DEV) for w in ws]
            Bt = lbm.Batch(Gs)
            Bt.set_tiling(tile, persistent)
            t, p, grid = Bt.tiling()
            ntiles = sum(-(-w.nodes // tile) for w in ws)
            assert (t, p) == (tile, persistent)
            if persistent:
                assert grid < ntiles  # blocks take runs of tiles
            else:
                assert grid == ntiles
            Bt.step(2)
            Bt.step(3)
            for a, G in zip(want, Gs):
                assert G.t == 5
                # same per-node arithmetic; allow for multiply-add contraction
                # differences between the kernel instantiations
                assert np.abs(G.get_populations() - a).max() <= 1e-6 * scale
            Bt.close()
            for G in Gs:
                G.close()


def test_tiled_fp32_batch_matches_oracle():
    ch, _ = _sweep_members(count=12)
    Gs = [lbm.from_workload(w, storage=lbm.FP32_DEV) for w in ch]
    B = lbm.Batch(Gs)
    B.set_tiling(128, True)
    B.step(30)
    for w, G in list(zip(ch, Gs))[:3]:
        R = oracle_from_workload(w)
        R.run(30)
        _, u = G.moments()
        _, ur = R.moments()
        err = float(np.sqrt(np.sum((u - ur) ** 2) / np.sum(ur ** 2)))
        assert err <= 1e-4, (w.name, err)


def test_autotune_leaves_the_state_unchanged_and_picks_a_tiling():
    ch, _ = _sweep_members()
    Gs = [lbm.from_workload(w, storage=lbm.FP32_DEV) for w in ch]
    twins = [lbm.from_workload(w, storage=lbm.FP32_DEV) for w in ch]
    B = lbm.Batch(Gs)
    Bt = lbm.Batch(twins)
    B.step(3)
    Bt.step(3)
    before = [G.get_populations() for G in Gs]
    n0 = B.launch_count()
    us, tried = B.autotune(3, all_timings=True)
    assert us > 0 and len(tried) == 6 and min(tried.values()) == us
    assert B.launch_count() == n0 + 6 * (3 + 1)  # six tilings, 3 trials + 1 warm-up each
    tile, persistent, grid = B.tiling()
    assert tile in (128, 256, 512) and grid > 0
    for G, f in zip(Gs, before):
        assert G.t == 3
        assert np.array_equal(G.get_populations(), f)
    # the next steps continue from the unchanged state
    B.set_graph(4)
    B.step(4)
    Bt.step(4)
    scale = max(float(np.abs(f).max()) for f in before)
    for a, b in zip(Gs, twins):
        assert a.t == b.t == 7
        assert np.abs(a.get_populations() - b.get_populations()).max() <= 1e-6 * scale


def test_fp64_batch_every_tiling_and_autotune():
    """FP64 batches take every tiling too; all give the populations of the
    default tiling to FP64 rounding, and the autotuner leaves the state alone."""
    ws, fulls = _members("d2q5")
    ref = [_make(w, f) for w, f in zip(ws, fulls)]
    B = lbm.Batch(ref)
    B.step(4)
    want = [G.get_populations() for G in ref]
    for tile in (128, 256, 512):
        for persistent in (False, True):
            Gs = [_make(w, f) for w, f in zip(ws, fulls)]
            Bt = lbm.Batch(Gs)
            Bt.set_tiling(tile, persistent)
            Bt.step(4)
            for a, G in zip(want, Gs):
                assert np.abs(G.get_populations() - a).max() <= 4 * 4 * 2.0 ** -53
    n0 = B.launch_count()
    before = [G.get_populations() for G in ref]
    us, tried = B.autotune(2, all_timings=True)
    assert B.launch_count() == n0 + 6 * 3 and len(tried) == 6
    for G, f in zip(ref, before):
        assert np.array_equal(G.get_populations(), f)
    with pytest.raises(lbm.LBMError) as e:
        B.set_tiling(64, False)
    assert e.value.code == lbm.EINVAL
    with pytest.raises(lbm.LBMError):
        B.autotune(0)


def test_fp64_scalar_persistent_runs_cross_members():
    """FP64 scalar batches large enough that the persistent grid holds fewer
    blocks than there are tiles, so every block's run spans several tiles and
    many runs cross from one member into the next; its members have a
    uniform velocity with a separable source, a velocity field, a full source
    field and no source.  Each tiling steps every member as the member's own
    kernel does."""
    _, sc = W.batched_sweep(count=60, seed=21, nx_range=(40, 200), ny_range=(32, 160))
    ws, fulls = list(sc), [None] * len(sc)
    rng = np.random.default_rng(3)
    vel = {}
    for k, (shape, wall, kind) in enumerate([((150, 97, 1), (0, 0, 0), "full"),
                                             ((31, 200, 1), (1, 1, 0), "separable"),
                                             ((64, 64, 1), (0, 1, 0), "full")]):
        w, full = _random_workload(W.D2Q5, shape, wall, seed=40 + k, kind=kind)
        ws.insert(5 * k + 3, w)
        fulls.insert(5 * k + 3, full)
        if k != 2:
            vel[5 * k + 3] = 0.02 * rng.standard_normal((2, w.nodes))
    nosrc = ws.index(sc[7])
    ws[nosrc] = dataclasses.replace(sc[7], tables=None)
    nodes = sum(w.nodes for w in ws)

    def make_all():
        Gs = [_make(w, f) for w, f in zip(ws, fulls)]
        for i, v in vel.items():
            Gs[i].set_velocity(full=v)
        return Gs

    solo = make_all()
    for G in solo:
        G.step(3)
    want = [G.get_populations() for G in solo]
    for tile in (128, 256, 512):
        Gs = make_all()
        B = lbm.Batch(Gs)
        B.set_tiling(tile, True)
        t, p, grid = B.tiling()
        assert p and grid < -(-nodes // tile) // 2  # runs of two or more tiles
        B.step(1)
        B.step(2)
        for a, G in zip(want, Gs):
            assert G.t == 3
            assert np.abs(G.get_populations() - a).max() <= 3 * 4 * 2.0 ** -53, (tile, G.shape)
        B.close()


def test_batch_moments_equal_member_moments():
    for kind in ("d2q5", "d2q9", "d3q27", "d3q15"):
        ws, fulls = _members(kind)
        Gs = [_make(w, f) for w, f in zip(ws, fulls)]
        B = lbm.Batch(Gs)
        B.step(3)
        got = B.moments()
        for G, g in zip(Gs, got):
            want = G.moments()
            if kind == "d2q5":
                assert np.array_equal(g, want)
            else:
                assert np.array_equal(g[0], want[0]) and np.array_equal(g[1], want[1])
        got0 = B.moments(half_forced=False)
        for G, g in zip(Gs, got0):
            want = G.moments(half_forced=False)
            assert np.array_equal(g if kind == "d2q5" else g[1], want if kind == "d2q5" else want[1])


def test_packed_moments_equal_member_moments():
    for kind, storage in (("d2q5", lbm.FP64), ("d2q9", lbm.FP64), ("d3q27", lbm.FP64), ("d3q27", lbm.FP32_DEV)):
        ws, fulls = _members(kind)
        if storage == lbm.FP64:
            Gs = [_make(w, f) for w, f in zip(ws, fulls)]
        else:
            Gs = [lbm.from_workload(w, storage=storage) for w in ws]
        B = lbm.Batch(Gs)
        B.step(3)
        Gs[0].step(1)  # one member out of lockstep: packed readback follows each member's own state
        for half in (True, False):
            rho, u = B.moments_packed(half_forced=half)
            off = 0
            for G in Gs:
                want = G.moments(half_forced=half)
                if kind == "d2q5":
                    assert np.array_equal(rho[off:off + G.N], want)
                else:
                    assert np.array_equal(rho[off:off + G.N], want[0])
                    assert np.array_equal(u[G.dim * off:G.dim * (off + G.N)].reshape(G.dim, G.N), want[1])
                off += G.N


@pytest.mark.parametrize("where", [2, 3])
def test_readbacks_three_in_flight(where):
    """Three host buffers in turn, wait_moments(keep=2) each step: the buffer
    of step k - 2 is complete while two later readbacks may still be on their
    way; a keep outside 0..2 is refused."""
    import torch

    ws, fulls = _members("d2q5")
    Gs = [_make(w, f) for w, f in zip(ws, fulls)]
    twins = [_make(w, f) for w, f in zip(ws, fulls)]
    B, T = lbm.Batch(Gs), lbm.Batch(twins)
    n = sum(G.N for G in Gs)
    bufs = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(3)]
    history = []
    for k in range(8):
        B.step(1)
        T.step(1)
        history.append(T.moments_packed()[0])
        B.moments_packed_into(bufs[k % 3].data_ptr(), None, where=where)
        B.wait_moments(keep=2)
        if k >= 2:
            assert np.array_equal(bufs[(k - 2) % 3].numpy(), history[k - 2])
    B.wait_moments(keep=0)
    for k in (5, 6, 7):
        assert np.array_equal(bufs[k % 3].numpy(), history[k])
    for bad in (-1, 3):
        with pytest.raises(lbm.LBMError):
            B.wait_moments(keep=bad)
    B.close()
    T.close()


@pytest.mark.parametrize("kind", ["d2q5", "d2q9", "d3q27", "d3q15"])
@pytest.mark.parametrize("where", [1, 3])
def test_step_read_writes_the_fields_each_step_starts_from(kind, where):
    """lbm_batch_step_read: each call steps the batch once and its kernel
    writes the packed fields of the state the step started from, bit for bit
    what lbm_batch_moments_packed returned just before (half-forced or not);
    the stepped states equal plain batched steps bit for bit."""
    import torch

    ws, fulls = _members(kind)
    if kind == "d2q5":
        # plus a member without a source and one with an advecting-velocity field
        ws += [dataclasses.replace(ws[0], tables=None), ws[1]]
        fulls += [None, None]
    else:
        ws.append(dataclasses.replace(ws[0], tables=None))  # plus a member without a force
        fulls.append(None)
    Gs = [_make(w, f) for w, f in zip(ws, fulls)]
    twins = [_make(w, f) for w, f in zip(ws, fulls)]
    if kind == "d2q5":
        v = 0.02 * np.random.default_rng(9).standard_normal((2, Gs[-1].N))
        Gs[-1].set_velocity(full=v)
        twins[-1].set_velocity(full=v)
    B, T = lbm.Batch(Gs), lbm.Batch(twins)
    n = sum(G.N for G in Gs)
    dim = 0 if kind == "d2q5" else Gs[0].dim
    kw = {"dtype": torch.float64}
    kw.update({"device": "cuda"} if where == 1 else {"pin_memory": True})
    bufs = [(torch.empty(n, **kw), torch.empty(max(dim, 1) * n, **kw)) for _ in range(3)]
    for k in range(7):
        half = k % 2 == 0
        want = T.moments_packed(half_forced=half)
        r_, u_ = bufs[k % 3]
        B.step_read_into(r_.data_ptr(), u_.data_ptr() if dim else None, where=where, half_forced=half)
        T.step(1)
        B.wait_moments(keep=0)
        torch.cuda.synchronize()
        assert np.array_equal(r_.cpu().numpy(), want[0]), k
        if dim:
            assert np.array_equal(u_.cpu().numpy(), want[1]), k
    for G, H in zip(Gs, twins):
        assert G.t == H.t == 7
        assert np.array_equal(G.get_populations(), H.get_populations())
    with pytest.raises(lbm.LBMError):
        B.step_read_into(bufs[0][0].data_ptr(), None if not dim else bufs[0][1].data_ptr(), where=2)
    B.close()
    T.close()


def test_step_read_refuses_reduced_precision_and_pageable_memory():
    import torch

    ws, _ = _members("d2q5")
    Gs = [lbm.from_workload(w, storage=lbm.FP32_DEV) for w in ws]
    B = lbm.Batch(Gs)
    n = sum(G.N for G in Gs)
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError):
        B.step_read_into(d.data_ptr(), None, where=1)
    B.close()
    Hs = [lbm.from_workload(w) for w in ws]
    C = lbm.Batch(Hs)
    pageable = np.empty(n)
    with pytest.raises(lbm.LBMError):
        C.step_read_into(pageable.ctypes.data, None, where=3)
    assert all(H.t == 0 for H in Hs)  # refused before stepping
    C.close()


def test_packed_moments_many_members_every_form():
    """More members than travel in the launch arguments (their a_pre go
    through a device table instead): every packed form equals the members'
    own moments, the asynchronous ones after wait_moments."""
    import torch

    ws = [W.poiseuille(ny=5 + k % 7, nx=3 + k % 4, Fx=1e-5 * (1 + k)) for k in range(40)]
    Gs = [lbm.from_workload(w) for w in ws]
    B = lbm.Batch(Gs)
    B.step(2)
    n = sum(G.N for G in Gs)
    want = [G.moments() for G in Gs]
    for where in (0, 2, 3):
        if where == 0:
            rho, u = np.empty(n), np.empty(2 * n)
            B.moments_packed_into(rho.ctypes.data, u.ctypes.data, where=0)
        else:
            rt = torch.empty(n, dtype=torch.float64, pin_memory=True)
            ut = torch.empty(2 * n, dtype=torch.float64, pin_memory=True)
            B.moments_packed_into(rt.data_ptr(), ut.data_ptr(), where=where)
            B.wait_moments(keep=0)
            rho, u = rt.numpy(), ut.numpy()
        off = 0
        for G, (r, v) in zip(Gs, want):
            assert np.array_equal(rho[off:off + G.N], r)
            assert np.array_equal(u[2 * off:2 * (off + G.N)].reshape(2, G.N), v)
            off += G.N
    B.close()
    for G in Gs:
        G.close()


def test_full_batched_sweep_in_the_bench_configuration():
    """The bench's batched sweep (2048 D2Q9 channels + 2048 D2Q5 scalar
    lattices, FP32 deviations) in its launch configuration: autotuned tiling,
    graph replays of 10 steps.  Sampled members equal the same lattices
    stepped alone (single-lattice kernel), and the smallest members agree with
    the FP64 oracle within the FP32 bound."""
    ch, sc = W.batched_sweep()
    for ws in (ch, sc):
        Gs = [lbm.from_workload(w, storage=lbm.FP32_DEV) for w in ws]
        B = lbm.Batch(Gs)
        B.autotune(2)
        B.set_graph(10)
        B.step(20)
        assert B.graph_replays() == 2
        idx = [0, 1, 7, 100, 1000, 2047]
        for k in idx:
            solo = lbm.from_workload(ws[k], storage=lbm.FP32_DEV)
            solo.step(20)
            a, b = solo.get_populations(), Gs[k].get_populations()
            assert np.abs(a - b).max() <= 4e-6 * np.abs(a).max(), (k, np.abs(a - b).max())
            solo.close()
        small = sorted(range(len(ws)), key=lambda k: ws[k].nodes)[:3]
        for k in small:
            R = oracle_from_workload(ws[k])
            R.run(20)
            if ws[k].lattice == W.D2Q5:
                err = np.abs(Gs[k].moments() - R.moments()).max()
                assert err <= 1e-6, (k, err)
            else:
                _, ug = Gs[k].moments()
                _, ur = R.moments()
                assert np.abs(ug - ur).max() <= 1e-4 * max(np.abs(ur).max(), 1e-3), k
        B.close()
        for G in Gs:
            G.close()


@pytest.mark.parametrize("where", [2, 3])
def test_asynchronous_packed_readback_double_buffered(where):
    """where = 2: kernel and copies on the library's copy stream; where = 3:
    the kernel writes the pinned host buffers directly.  Both overlap the next
    step.  After wait_moments the host buffers hold exactly the fields of the
    step they were queued at."""
    import torch

    ws, fulls = _members("d2q9")
    Gs = [_make(w, f) for w, f in zip(ws, fulls)]
    twins = [_make(w, f) for w, f in zip(ws, fulls)]
    B = lbm.Batch(Gs)
    T = lbm.Batch(twins)
    n = sum(G.N for G in Gs)
    bufs = [(torch.empty(n, dtype=torch.float64, pin_memory=True),
             torch.empty(2 * n, dtype=torch.float64, pin_memory=True)) for _ in range(2)]
    history = []
    for k in range(6):
        B.step(1)
        T.step(1)
        history.append(T.moments_packed())
        r_, u_ = bufs[k % 2]
        B.moments_packed_into(r_.data_ptr(), u_.data_ptr(), where=where)
        B.wait_moments(keep=1)
        if k >= 1:
            r_prev, u_prev = bufs[(k - 1) % 2]
            assert np.array_equal(r_prev.numpy(), history[k - 1][0])
            assert np.array_equal(u_prev.numpy(), history[k - 1][1])
    B.wait_moments(keep=0)
    r_, u_ = bufs[5 % 2]
    assert np.array_equal(r_.numpy(), history[5][0]) and np.array_equal(u_.numpy(), history[5][1])
    with pytest.raises(lbm.LBMError):
        B.wait_moments(keep=3)
    if where == 3:
        # pageable memory is not addressable by the device: refused, nothing queued
        r_np, u_np = np.empty(n), np.empty(2 * n)
        with pytest.raises(lbm.LBMError):
            B.moments_packed_into(r_np.ctypes.data, u_np.ctypes.data, where=3)
    # member-level work while a readback may still read the populations: the
    # readback sees the state it was queued at, the members their own work
    r_, u_ = bufs[0]
    B.moments_packed_into(r_.data_ptr(), u_.data_ptr(), where=where)
    expect = T.moments_packed()
    Gs[0].step(2)
    Gs[1].set_populations(Gs[1].get_populations(), step=Gs[1].t)
    Gs[2].debug_poison()
    B.wait_moments(keep=0)
    assert np.array_equal(r_.numpy(), expect[0]) and np.array_equal(u_.numpy(), expect[1])
    twins[0].step(2)
    assert np.array_equal(Gs[0].get_populations(), twins[0].get_populations())

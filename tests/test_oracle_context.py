"""The oracle's context API (``lbmref_*``): the same call shape as the
library's C ABI on host arrays.  It must step exactly like the plain oracle
runs the other tests pin (bitwise, same arithmetic), honour the call order and
argument checks of the library, and report the reductions the library
reports (mass, momentum, max change since the previous call)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_10247_gb300 import workloads as W


def _pair(w, envelope=None):
    P = O.expand_separable(w.tables, w.shape) if w.tables else None
    ref = O.OracleLattice(w.lattice, w.shape, wall=w.wall, omega=w.omega, P=P, envelope=envelope)
    ctx = O.OracleContext(w.lattice, w.shape, omega=w.omega, wall=w.wall)
    assert ctx.status == O.REF_OK
    return ref, ctx, P


def test_flow_context_matches_plain_oracle_bitwise():
    w = W.womersley(ny=12, nx=3, tau=0.9, period=40)
    ref, ctx, P = _pair(w, envelope=w.envelope)
    ref.init_equilibrium(1.0, (0.0, 0.0, 0.0))
    assert ctx.init_equilibrium(1.0, (0.0, 0.0, 0.0)) == O.REF_OK
    assert ctx.set_force(P) == O.REF_OK
    assert ctx.set_envelope(w.envelope) == O.REF_OK
    for n in (1, 7, 30):
        ref.run(n)
        assert ctx.step(n) == O.REF_OK
    rc, f = ctx.populations()
    assert rc == O.REF_OK and np.array_equal(f, ref.f)
    rc, rho, u = ctx.moments(half_forced=True)
    r2, u2 = ref.moments(half_forced=True)
    assert rc == O.REF_OK and np.array_equal(rho, r2) and np.array_equal(u, u2)
    assert ctx.get_step() == (O.REF_OK, 38)


def test_scalar_context_matches_plain_oracle_bitwise():
    c = W.cde_sweep_params()[0]
    w = W.cde_workload(c)
    ref, ctx, P = _pair(w, envelope=w.envelope)
    N = ref.N
    uadv = np.zeros((2, N))
    uadv[0], uadv[1] = w.u0[0], w.u0[1]
    ref.uadv = uadv
    ref.init_equilibrium(w.rho0, uadv)
    assert ctx.init_equilibrium(w.rho0, None, None, uadv) == O.REF_OK
    assert ctx.set_source(P[0]) == O.REF_OK
    assert ctx.set_velocity(uadv) == O.REF_OK
    assert ctx.set_envelope(w.envelope) == O.REF_OK
    ref.run(25)
    assert ctx.step(25) == O.REF_OK
    rc, f = ctx.populations()
    assert np.array_equal(f, ref.f)
    rc, phi, _ = ctx.moments()
    assert np.array_equal(phi, ref.moments())


def test_reduce_mass_momentum_and_change():
    w = W.poiseuille(ny=9, nx=3, tau=0.8, Fx=1e-4)
    _, ctx, P = _pair(w)
    ctx.init_equilibrium(1.0)
    ctx.set_force(P)
    rc, out = ctx.reduce()
    assert rc == O.REF_OK and math.isinf(out[4])
    assert out[0] == pytest.approx(27.0, rel=1e-15)
    m0 = out[0]
    ctx.step(50)
    rc, out = ctx.reduce()
    # mass is conserved by every step (sum over K_beta of the changes is 0)
    assert abs(out[0] - m0) <= 1e-13 * m0
    # the force has accelerated the fluid along x only
    assert out[1] > 0.0 and out[2] == pytest.approx(0.0, abs=1e-15)
    assert 0.0 < out[4] < 1e-2
    ctx.step(0)
    rc, out2 = ctx.reduce()
    assert out2[4] == 0.0


def test_resume_from_populations_is_bitwise():
    w = W.poiseuille(ny=9, nx=3, tau=0.7, Fx=1e-5)
    _, a, P = _pair(w)
    _, b, _ = _pair(w)
    for c in (a, b):
        c.init_equilibrium(1.0)
        c.set_force(P)
    a.step(40)
    _, f = a.populations()
    b.set_populations(f, 40)
    a.step(15)
    b.step(15)
    assert np.array_equal(a.populations()[1], b.populations()[1])
    assert b.get_step() == (O.REF_OK, 55)


def test_call_order_and_argument_checks():
    om = W.d2q9_omega(0.8)
    ctx = O.OracleContext(O.D2Q9, (4, 4, 1), omega=om)
    assert ctx.step(1) == O.REF_ESTATE  # before initialisation
    assert ctx.moments()[0] == O.REF_ESTATE
    assert ctx.init_equilibrium(-1.0) == O.REF_EINVAL  # non-positive density
    assert ctx.init_equilibrium(1.0) == O.REF_OK
    assert ctx.step(-1) == O.REF_EINVAL
    assert ctx.set_source(np.zeros(16)) == O.REF_EINVAL  # flow lattice has no source
    assert ctx.set_velocity(np.zeros((2, 16))) == O.REF_EINVAL
    assert ctx.set_populations(np.zeros(5), 0) == O.REF_EINVAL  # wrong count
    bad = [
        O.OracleContext(9, (4, 4, 1), omega=om),                      # unknown lattice
        O.OracleContext(O.D2Q9, (4, 4, 2), omega=om),                 # 2D lattice with nz > 1
        O.OracleContext(O.D2Q9, (0, 4, 1), omega=om),                 # empty axis
        O.OracleContext(O.D2Q9, (4, 1, 1), omega=om, wall=(0, 1, 0)),  # walls on an axis of extent 1
        O.OracleContext(O.D2Q9, (4, 4, 1), omega=om, wall=(0, 0, 1)),  # walls on z of a 2D lattice
        O.OracleContext(O.D2Q9, (4, 4, 1), omega=(2.5,) * 9),          # rate outside (0, 2)
    ]
    assert all(c.status == O.REF_EINVAL for c in bad)
    s = O.OracleContext(O.D2Q5, (4, 4, 1), omega=W.d2q5_omega(0.8))
    assert s.set_force(np.zeros((2, 16))) == O.REF_EINVAL  # scalar lattice has no force


def test_reduce_flags_a_non_positive_density():
    ctx = O.OracleContext(O.D2Q9, (3, 3, 1), omega=W.d2q9_omega(0.8))
    ctx.init_equilibrium(1.0)
    _, f = ctx.populations()
    f[:, 4] = -f[:, 4]
    ctx.set_populations(f, 0)
    assert ctx.reduce()[0] == O.REF_EUNSTABLE


def test_l2_error_invariants():
    """Eq. sca on the context's own fields: zero against itself; exactly 1/2
    against twice the field (sum (q - 2q)^2 = sum q^2 and sum (2q)^2 =
    4 sum q^2, both exact in binary); a single perturbed value of one vector
    component contributes its own square and nothing else; +inf against a
    zero reference."""
    w = W.womersley(ny=10, nx=4, tau=0.9, period=40)
    _, ctx, P = _pair(w, envelope=w.envelope)
    ctx.init_equilibrium(1.0, (0.01, -0.02, 0.0))
    ctx.set_force(P)
    ctx.set_envelope(w.envelope)
    ctx.step(7)
    for field in (0, 1):
        _, rho, u = ctx.moments(half_forced=True)
        q = rho if field == 0 else u
        rc, out = ctx.l2_error(q, field)
        assert rc == O.REF_OK and out[0] == 0.0 and out[2] == 0.0
        rc, out = ctx.l2_error(2.0 * q, field)
        assert out[1] == 4.0 * out[0] and out[2] == 0.5
        ref = q.copy()
        k = (field, 17) if field == 1 else (17,)
        ref[k] = ref[k] * (1 + 1e-3)
        d = q[k] - ref[k]
        rc, out = ctx.l2_error(ref, field)
        assert out[0] == d * d and out[1] > 0.0
        rc, out = ctx.l2_error(np.zeros_like(q), field)
        assert out[1] == 0.0 and math.isinf(out[2])
    # the un-forced field differs from the half-forced one by a_pre F / (2 rho)
    _, _, u0 = ctx.moments(half_forced=False)
    rc, a = ctx.l2_error(u0, 1, half_forced=True)
    rc, b = ctx.l2_error(u0, 1, half_forced=False)
    assert a[0] > 0.0 and b[0] == 0.0


def test_l2_error_argument_checks():
    s = O.OracleContext(O.D2Q5, (4, 4, 1), omega=W.d2q5_omega(0.8))
    assert s.l2_error(np.zeros(16))[0] == O.REF_ESTATE
    s.init_equilibrium(1.0)
    assert s.l2_error(np.zeros(16))[0] == O.REF_OK
    assert s.l2_error(np.zeros(32), field=1)[0] == O.REF_EINVAL  # no velocity field on the scalar lattice
    assert s.l2_error(np.zeros(15))[0] == O.REF_EINVAL

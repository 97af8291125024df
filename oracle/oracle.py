"""Python access to the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
leg of the benchmark may use this module; the product path (the CUDA library
and its binding) never imports it, and it imports nothing from the product.

The oracle follows arXiv:1806.10247:
  * D2Q9 flow: Sec. 4, Eqs. 21-32 and the algorithm (i)-(vi) that ends Sec. 4;
  * D2Q5 passive scalar with source: Sec. 5, Eqs. 37-48 (Eq. 41 with the
    sign of its u^2 phi terms corrected, see ``lbm_oracle.c``);
  * D3Q27 flow: the generic central-moment procedure that the paper's
    Appendix A says extends to D3Q27;
  * D3Q15 flow: Appendix A, Eqs. 6A-13A and the f^p expansion, with the
    three corrections listed in ``lbm_oracle.c``;
  * streaming with periodic wrap or stationary halfway bounce-back (Sec. 6.1).

Force and source fields enter as F(x, t) = a(t) * P(x): a shape P given on the
nodes and an envelope a(t).  Each step uses the trapezoid averages of a over
its two half steps (Sec. 6.3), computed here by :func:`envelope_pairs`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(HERE, "_lib")
LIBPATH = os.path.join(LIBDIR, "liblbm_oracle.so")
SRC = os.path.join(HERE, "lbm_oracle.c")

D2Q9, D3Q27, D2Q5, D3Q15 = 1, 2, 3, 4
Q = {D2Q9: 9, D3Q27: 27, D2Q5: 5, D3Q15: 15}
DIM = {D2Q9: 2, D3Q27: 3, D2Q5: 2, D3Q15: 3}


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle into ``oracle/_lib/liblbm_oracle.so`` with gcc."""
    os.makedirs(LIBDIR, exist_ok=True)
    if (not force and os.path.exists(LIBPATH)
            and os.path.getmtime(LIBPATH) >= max(os.path.getmtime(SRC),
                                                 os.path.getmtime(os.path.join(HERE, "lbm_oracle.h")))):
        return LIBPATH
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wno-unknown-pragmas"]
    if openmp:
        cmd.append("-fopenmp")
    tmp = LIBPATH + f".tmp{os.getpid()}"
    cmd += ["-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIBPATH)
    return LIBPATH


class _Params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("n", ctypes.c_int * 3), ("wall", ctypes.c_int * 3),
                ("omega", ctypes.c_double * 9), ("generic", ctypes.c_int),
                ("as_printed", ctypes.c_int)]


_lib = None
ENVELOPE_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)
# status codes of the lbmref_* context API
REF_OK, REF_EINVAL, REF_ENOMEM, REF_EUNSTABLE, REF_ESTATE = 0, -1, -2, -4, -6


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIBPATH)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        L.orc_run.argtypes = [pp, dp, dp, ctypes.c_long, dp, dp, dp]
        L.orc_moments.argtypes = [pp, dp, dp, ctypes.c_double, dp, dp]
        L.orc_equilibrium.argtypes = [pp, dp, dp, dp]
        L.orc_collide_node.argtypes = [pp, dp, dp, dp, dp, dp]
        L.orc_collide_node_generic.argtypes = [pp, dp, dp, dp, dp]
        L.orc_velocities.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.orc_strain_rate.argtypes = [pp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        for fn in ("orc_run", "orc_moments", "orc_equilibrium", "orc_collide_node",
                   "orc_collide_node_generic", "orc_velocities", "orc_strain_rate"):
            getattr(L, fn).restype = ctypes.c_int
        vp = ctypes.c_void_p
        L.lbmref_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    dp, ctypes.POINTER(ctypes.c_int)]
        L.lbmref_destroy.argtypes = [vp]
        L.lbmref_destroy.restype = None
        L.lbmref_init_equilibrium.argtypes = [vp, ctypes.c_double, dp, dp, dp]
        L.lbmref_set_force.argtypes = [vp, dp]
        L.lbmref_set_source.argtypes = [vp, dp]
        L.lbmref_set_velocity.argtypes = [vp, dp]
        L.lbmref_set_envelope.argtypes = [vp, ENVELOPE_FN, vp]
        L.lbmref_step.argtypes = [vp, ctypes.c_long]
        L.lbmref_moments.argtypes = [vp, dp, dp, ctypes.c_int]
        L.lbmref_reduce.argtypes = [vp, dp]
        L.lbmref_l2_error.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, dp]
        L.lbmref_get_populations.argtypes = [vp, dp, ctypes.c_size_t]
        L.lbmref_set_populations.argtypes = [vp, dp, ctypes.c_size_t, ctypes.c_long]
        L.lbmref_get_step.argtypes = [vp, ctypes.POINTER(ctypes.c_long)]
        for fn in ("lbmref_create", "lbmref_init_equilibrium", "lbmref_set_force", "lbmref_set_source",
                   "lbmref_set_velocity", "lbmref_set_envelope", "lbmref_step", "lbmref_moments",
                   "lbmref_reduce", "lbmref_get_populations", "lbmref_set_populations", "lbmref_get_step",
                   "lbmref_l2_error"):
            getattr(L, fn).restype = ctypes.c_int
        _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Thread count of the oracle's node loops (n > 0 sets it); returns the
    count in use.  Timing only: results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def velocities(lattice: int) -> np.ndarray:
    q = Q[lattice]
    e = (ctypes.c_int * (3 * q))()
    lib().orc_velocities(lattice, e)
    return np.array(list(e), dtype=np.int64).reshape(q, 3)


def envelope_pairs(envelope, t0: int, nsteps: int) -> np.ndarray:
    """(a_pre, a_post) per step for steps t0 .. t0+nsteps-1 (Sec. 6.3 trapezoid)."""
    out = np.empty(2 * nsteps, dtype=np.float64)
    for k in range(nsteps):
        t = float(t0 + k)
        a0, ah, a1 = envelope(t), envelope(t + 0.5), envelope(t + 1.0)
        out[2 * k] = 0.5 * (a0 + ah)
        out[2 * k + 1] = 0.5 * (ah + a1)
    return out


def expand_separable(tables, shape) -> np.ndarray:
    """Full node field of a separable shape P(x,y,z) = (px[x] * py[y]) * pz[z].

    ``tables`` is a list (one entry per component) of (px, py, pz) 1-D arrays of
    length 1 (broadcast) or the axis extent; ``shape`` is (nx, ny, nz).  The
    product is taken in that order."""
    nx, ny, nz = shape
    comps = []
    for px, py, pz in tables:
        px = np.broadcast_to(np.asarray(px, np.float64), (nx,))
        py = np.broadcast_to(np.asarray(py, np.float64), (ny,))
        pz = np.broadcast_to(np.asarray(pz, np.float64), (nz,))
        full = (px[None, None, :] * py[None, :, None]) * pz[:, None, None]
        comps.append(full.reshape(-1))
    return np.ascontiguousarray(np.stack(comps), dtype=np.float64)


@dataclass
class OracleLattice:
    """One lattice advanced by the oracle; ``f`` holds f(t) as [q][z][y][x]."""

    lattice: int
    shape: tuple  # (nx, ny, nz)
    wall: tuple = (0, 0, 0)
    omega: tuple = (1.0,) * 9
    generic: bool = False
    as_printed: bool = False
    P: np.ndarray | None = None          # [ncomp][N] force/source shape
    envelope: object = None              # callable a(t); None means a == 1
    uadv: np.ndarray | None = None       # D2Q5: [2][N]
    t: int = 0
    f: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        self.shape = tuple(int(s) for s in self.shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.q = Q[self.lattice]
        self.dim = DIM[self.lattice]
        if self.f is None:
            self.f = np.zeros((self.q, self.N))
        self._work = np.empty_like(self.f)

    @property
    def params(self):
        p = _Params()
        p.lattice = self.lattice
        for d in range(3):
            p.n[d] = self.shape[d]
            p.wall[d] = int(self.wall[d])
        for k in range(9):
            p.omega[k] = float(self.omega[k])
        p.generic = int(self.generic)
        p.as_printed = int(self.as_printed)
        return p

    def init_equilibrium(self, rho, u):
        """f(0) = equilibrium with the central moments of Eq. 20 / Eq. 39 at (rho, u)."""
        rho = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, np.float64), (self.N,)))
        u3 = np.zeros((3, self.N))
        u = np.asarray(u, np.float64)
        if u.ndim == 1:
            u3[: len(u)] = u[:, None]
        else:
            u3[: u.shape[0]] = u
        u3 = np.ascontiguousarray(u3[: self.dim])
        f = np.empty((self.q, self.N))
        rc = lib().orc_equilibrium(ctypes.byref(self.params), _dp(rho), _dp(u3), _dp(f))
        assert rc == 0
        self.f = f
        self.t = 0

    def pairs(self, nsteps):
        if self.envelope is None:
            return None
        return envelope_pairs(self.envelope, self.t, nsteps)

    def a_pre_now(self):
        if self.envelope is None:
            return 1.0
        return float(envelope_pairs(self.envelope, self.t, 1)[0])

    def run(self, nsteps: int):
        if nsteps <= 0:
            return
        a = self.pairs(nsteps)
        uadv = None if self.uadv is None else np.ascontiguousarray(self.uadv, np.float64)
        rc = lib().orc_run(ctypes.byref(self.params), _dp(self.f), _dp(self._work), int(nsteps),
                           _dp(self.P), _dp(a), _dp(uadv))
        assert rc == 0, "orc_run rejected its parameters"
        self.t += nsteps

    def moments(self, half_forced: bool = True):
        """rho [N] and u [dim][N] (flow), or phi [N] (D2Q5)."""
        rho = np.empty(self.N)
        u = np.empty((self.dim, self.N))
        P = self.P if half_forced else None
        rc = lib().orc_moments(ctypes.byref(self.params), _dp(self.f), _dp(P),
                               self.a_pre_now(), _dp(rho), _dp(u))
        assert rc == 0
        if self.lattice == D2Q5:
            return rho
        return rho, u

    def strain_rate(self, rho0=1.0):
        """Strain-rate tensor [ncomp][N] from the non-equilibrium second moments
        (Sec. 6.6; 2D: xx, yy, xy; 3D: xx, yy, zz, xy, xz, yz)."""
        ncomp = 3 if self.dim == 2 else 6
        S = np.empty((ncomp, self.N))
        rc = lib().orc_strain_rate(ctypes.byref(self.params), _dp(self.f), _dp(self.P), self.a_pre_now(),
                                   float(rho0), _dp(S))
        assert rc == 0
        return S

    def collide_node(self, fin, Fpre, Fpost, uadv=None, generic=False):
        fin = np.ascontiguousarray(fin, np.float64)
        Fpre = np.ascontiguousarray(np.atleast_1d(Fpre), np.float64)
        Fpost = np.ascontiguousarray(np.atleast_1d(Fpost), np.float64)
        out = np.empty(self.q)
        if generic:
            rc = lib().orc_collide_node_generic(ctypes.byref(self.params), _dp(fin), _dp(Fpre),
                                                _dp(Fpost), _dp(out))
        else:
            if self.lattice == D2Q5 and uadv is None:
                raise ValueError("collide_node: the D2Q5 collision needs the advecting velocity uadv")
            ua = None if uadv is None else np.ascontiguousarray(uadv, np.float64)
            rc = lib().orc_collide_node(ctypes.byref(self.params), _dp(fin), _dp(Fpre),
                                        _dp(Fpost), _dp(ua), _dp(out))
        assert rc == 0
        return out


class OracleContext:
    """The oracle behind the library's call shape (``lbmref_*`` in
    ``lbm_oracle.c``): create / init_equilibrium / set_force / set_source /
    set_velocity / set_envelope / step / moments / reduce / populations.
    Methods return the C status code; arrays are host numpy arrays."""

    def __init__(self, lattice, shape, omega=(1.0,) * 9, wall=(0, 0, 0)):
        self.lattice = lattice
        self.shape = tuple(int(v) for v in shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.q, self.dim = Q.get(lattice, 0), DIM.get(lattice, 0)
        self._h = ctypes.c_void_p()
        om = np.ascontiguousarray(np.asarray(omega, np.float64))
        w = (ctypes.c_int * 3)(*[int(v) for v in wall])
        self.status = lib().lbmref_create(ctypes.byref(self._h), lattice, *self.shape, _dp(om), w)
        self._keep = None

    def close(self):
        if self._h:
            lib().lbmref_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_equilibrium(self, rho0=1.0, u0=(0.0, 0.0, 0.0), rho=None, u=None):
        u0a = np.ascontiguousarray(np.asarray(u0, np.float64))
        r = None if rho is None else np.ascontiguousarray(rho, np.float64)
        v = None if u is None else np.ascontiguousarray(u, np.float64)
        return lib().lbmref_init_equilibrium(self._h, float(rho0), _dp(u0a), _dp(r), _dp(v))

    def set_force(self, P):
        return lib().lbmref_set_force(self._h, _dp(None if P is None else np.ascontiguousarray(P, np.float64)))

    def set_source(self, S):
        return lib().lbmref_set_source(self._h, _dp(None if S is None else np.ascontiguousarray(S, np.float64)))

    def set_velocity(self, u):
        return lib().lbmref_set_velocity(self._h, _dp(None if u is None else np.ascontiguousarray(u, np.float64)))

    def set_envelope(self, fn):
        self._keep = None if fn is None else ENVELOPE_FN(lambda t, _u: float(fn(t)))
        return lib().lbmref_set_envelope(self._h, self._keep if fn is not None else ENVELOPE_FN(), None)

    def step(self, n):
        return lib().lbmref_step(self._h, int(n))

    def moments(self, half_forced=True):
        rho = np.empty(self.N)
        u = np.empty((self.dim, self.N))
        rc = lib().lbmref_moments(self._h, _dp(rho), _dp(u), int(half_forced))
        return rc, rho, u

    def reduce(self):
        out = np.empty(5)
        rc = lib().lbmref_reduce(self._h, _dp(out))
        return rc, out

    def l2_error(self, ref, field=0, half_forced=True):
        """(rc, [sum (q - ref)^2, sum ref^2, relative l2 error]) of Eq. sca."""
        ref = np.ascontiguousarray(ref, np.float64)
        want = self.N * (1 if field == 0 else self.dim)
        if ref.size != want:
            return REF_EINVAL, None
        out = np.empty(3)
        rc = lib().lbmref_l2_error(self._h, _dp(ref), int(field), int(half_forced), _dp(out))
        return rc, out

    def populations(self):
        f = np.empty((self.q, self.N))
        rc = lib().lbmref_get_populations(self._h, _dp(f), f.size)
        return rc, f

    def set_populations(self, f, step):
        f = np.ascontiguousarray(f, np.float64)
        return lib().lbmref_set_populations(self._h, _dp(f), f.size, int(step))

    def get_step(self):
        s = ctypes.c_long()
        rc = lib().lbmref_get_step(self._h, ctypes.byref(s))
        return rc, s.value

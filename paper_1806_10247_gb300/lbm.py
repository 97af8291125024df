"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``_lib/liblbm_gb300.so``.  There is no CPU fallback; if the library has not
been built, or no CUDA device is present, the calls fail loudly.

The Python names mirror the C entry points (``lbm_create`` ->
:class:`Lattice`, ``lbm_step`` -> :meth:`Lattice.step`, ...).  Arrays are numpy
(host) or anything exposing ``data_ptr()`` (device, e.g. a CUDA torch tensor)
where the C call takes ``where = 1``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

D2Q9, D3Q27, D2Q5_CDE, D3Q15 = 1, 2, 3, 4
FP64, FP32_DEV, FP16_DEV, BF16_DEV = 0, 1, 2, 3
PERIODIC, BOUNCE_BACK = 0, 1
FIELD_NONE, FIELD_SEPARABLE, FIELD_FULL, FIELD_FULL_DEVICE = 0, 1, 2, 3
OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ESTATE = 0, -1, -2, -3, -4, -6
MAX_NODES = 2 ** 31 - 2 ** 16  # LBM_MAX_NODES: largest lattice of one context
Q = {D2Q9: 9, D3Q27: 27, D2Q5_CDE: 5, D3Q15: 15}
DIM = {D2Q9: 2, D3Q27: 3, D2Q5_CDE: 2, D3Q15: 3}

EXPORTS = ("lbm_create", "lbm_destroy", "lbm_last_error", "lbm_init_equilibrium", "lbm_set_force",
           "lbm_set_source", "lbm_set_velocity", "lbm_set_envelope", "lbm_step", "lbm_moments",
           "lbm_reduce", "lbm_get_populations", "lbm_set_populations", "lbm_get_step", "lbm_sync",
           "lbm_launch_count", "lbm_reduce_sums_noalloc", "lbm_set_envelope_table", "lbm_batch_create",
           "lbm_batch_step", "lbm_batch_launch_count", "lbm_batch_last_error", "lbm_batch_destroy",
           "lbm_batch_set_graph", "lbm_batch_graph_replays", "lbm_batch_set_tiling", "lbm_batch_get_tiling",
           "lbm_batch_autotune", "lbm_batch_moments", "lbm_strain_rate", "lbm_set_source_from_strain",
           "lbm_batch_moments_packed", "lbm_batch_wait_moments", "lbm_debug_poison", "lbm_batch_step_read",
           "lbm_l2_error", "lbm_device_info", "lbm_probe_fp64", "lbm_probe_last_error",
           "lbm_set_stochastic_rounding", "lbm_set_local_reference")


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbm error {code}: {msg}")
        self.code = code


class _Relax(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double * 9)]


class _Boundary(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int * 3)]


class _Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("len", ctypes.c_int * 3),
                ("data", ctypes.POINTER(ctypes.c_double))]


ENVELOPE = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library and declare signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or (build_if_missing and not _build.up_to_date()):
        if not build_if_missing:
            raise OSError(f"CUDA library not built: {_build.LIB}")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.lbm_create.argtypes = [ctypes.POINTER(vp), ip, ip, ip, ip, ctypes.POINTER(_Relax),
                             ctypes.POINTER(_Boundary), ip, vp]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ctypes.c_char_p
    L.lbm_init_equilibrium.argtypes = [vp, ctypes.c_double, dp, dp, dp]
    L.lbm_set_force.argtypes = [vp, ctypes.POINTER(_Field)]
    L.lbm_set_source.argtypes = [vp, ctypes.POINTER(_Field)]
    L.lbm_set_velocity.argtypes = [vp, ctypes.POINTER(_Field)]
    L.lbm_set_envelope.argtypes = [vp, ENVELOPE, vp]
    L.lbm_set_envelope_table.argtypes = [vp, dp, ctypes.c_long, ctypes.c_double]
    L.lbm_step.argtypes = [vp, ctypes.c_long]
    L.lbm_set_stochastic_rounding.argtypes = [vp, ip, ctypes.c_ulonglong]
    L.lbm_set_local_reference.argtypes = [vp, ip]
    L.lbm_moments.argtypes = [vp, vp, vp, ip, ip]
    L.lbm_reduce.argtypes = [vp, dp]
    L.lbm_reduce_sums_noalloc.argtypes = [vp, dp]
    L.lbm_l2_error.argtypes = [vp, vp, ip, ip, ip, dp]
    L.lbm_get_populations.argtypes = [vp, vp, ctypes.c_size_t, ip, ctypes.POINTER(ctypes.c_long)]
    L.lbm_set_populations.argtypes = [vp, vp, ctypes.c_size_t, ip, ctypes.c_long]
    L.lbm_get_step.argtypes = [vp, ctypes.POINTER(ctypes.c_long)]
    L.lbm_sync.argtypes = [vp]
    L.lbm_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ip]
    L.lbm_batch_step.argtypes = [vp, ctypes.c_long]
    L.lbm_batch_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_batch_set_graph.argtypes = [vp, ip]
    L.lbm_batch_graph_replays.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_batch_set_tiling.argtypes = [vp, ip, ip]
    L.lbm_batch_get_tiling.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip)]
    L.lbm_batch_autotune.argtypes = [vp, ip, dp, dp]
    L.lbm_batch_moments.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ip, ip]
    L.lbm_strain_rate.argtypes = [vp, ctypes.c_double, dp, ip]
    L.lbm_batch_moments_packed.argtypes = [vp, vp, vp, ip, ip]
    L.lbm_batch_step_read.argtypes = [vp, vp, vp, ip, ip]
    L.lbm_batch_wait_moments.argtypes = [vp, ip]
    L.lbm_debug_poison.argtypes = [vp]
    L.lbm_set_source_from_strain.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double]
    L.lbm_batch_last_error.argtypes = [vp]
    L.lbm_batch_last_error.restype = ctypes.c_char_p
    L.lbm_probe_last_error.argtypes = []
    L.lbm_probe_last_error.restype = ctypes.c_char_p
    L.lbm_device_info.argtypes = [ip, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_probe_fp64.argtypes = [ip, ip, ip, ip, ctypes.c_longlong, vp, vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in ("lbm_destroy", "lbm_last_error", "lbm_batch_last_error", "lbm_batch_destroy",
                        "lbm_probe_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _torch_float64():
    import torch

    return torch.float64


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr(a):
    """Address of a numpy array (host) or a CUDA tensor-like object (device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _field(tables=None, full=None):
    """lbm_field for separable tables [(px, py, pz) per component] or a full
    [c][N] array: a numpy array (host) or a contiguous float64 CUDA tensor
    (device, copied on the context's stream without synchronising)."""
    f = _Field()
    keep = None
    if tables is None and full is None:
        f.kind = FIELD_NONE
        return f, keep
    if full is not None and getattr(full, "is_cuda", False):
        if full.dtype != _torch_float64() or not full.is_contiguous():
            raise ValueError("device field must be a contiguous float64 tensor")
        keep = full
        f.kind = FIELD_FULL_DEVICE
        f.data = ctypes.cast(ctypes.c_void_p(full.data_ptr()), ctypes.POINTER(ctypes.c_double))
        return f, keep
    if full is not None:
        keep = np.ascontiguousarray(full, dtype=np.float64)
        f.kind = FIELD_FULL
    else:
        # one table length per axis for all components: constant tables are
        # repeated to the longest length on that axis
        lens = [max(len(np.atleast_1d(comp[d])) for comp in tables) for d in range(3)]
        parts = []
        for comp in tables:
            for d in range(3):
                t = np.atleast_1d(np.asarray(comp[d], np.float64))
                if len(t) != lens[d]:
                    if len(t) != 1:
                        raise ValueError(f"table length {len(t)} on axis {d}: must be 1 or {lens[d]}")
                    t = np.repeat(t, lens[d])
                parts.append(t)
        keep = np.ascontiguousarray(np.concatenate(parts))
        f.kind = FIELD_SEPARABLE
        for d in range(3):
            f.len[d] = lens[d]
    f.data = _dp(keep)
    return f, keep


class Lattice:
    """One lattice on the GPU (an ``lbm_ctx``)."""

    def __init__(self, lattice, shape, omega, wall=(0, 0, 0), storage=FP64, stream=None):
        L = load()
        self._L = L
        self.lattice = lattice
        self.shape = tuple(int(s) for s in shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.q = Q[lattice]
        self.dim = DIM[lattice]
        self.storage = int(storage)
        r = _Relax()
        for k in range(9):
            r.omega[k] = float(omega[k])
        b = _Boundary()
        for d in range(3):
            b.axis[d] = BOUNCE_BACK if wall[d] else PERIODIC
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(int(stream))
        rc = L.lbm_create(ctypes.byref(h), int(lattice), *self.shape, ctypes.byref(r), ctypes.byref(b),
                          int(storage), s)
        if rc != OK:
            raise LBMError(rc, L.lbm_last_error(None).decode())
        self.h = h
        self._env = None

    def _check(self, rc):
        if rc != OK:
            raise LBMError(rc, self._L.lbm_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._L.lbm_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- set-up -------------------------------------------------------------
    def init_equilibrium(self, rho=1.0, u=(0.0, 0.0, 0.0)):
        """Equilibrium fill at uniform or per-node (rho, u)."""
        rho_arr = None
        u_arr = None
        rho0 = 1.0
        u0 = np.zeros(3)
        if np.ndim(rho) == 0:
            rho0 = float(rho)
        else:
            rho_arr = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, np.float64), (self.N,)))
        u = np.asarray(u, np.float64)
        if u.ndim == 1:
            u0[: len(u)] = u
        else:
            u_arr = np.ascontiguousarray(u[: self.dim], dtype=np.float64)
        self._check(self._L.lbm_init_equilibrium(self.h, rho0, _dp(u0), _dp(rho_arr), _dp(u_arr)))

    def set_force(self, tables=None, full=None):
        f, keep = _field(tables, full)
        self._check(self._L.lbm_set_force(self.h, ctypes.byref(f)))

    def set_source(self, tables=None, full=None):
        f, keep = _field(tables, full)
        self._check(self._L.lbm_set_source(self.h, ctypes.byref(f)))

    def set_velocity(self, tables=None, full=None):
        f, keep = _field(tables, full)
        self._check(self._L.lbm_set_velocity(self.h, ctypes.byref(f)))

    def set_envelope(self, fn, steps=None):
        """fn(t) -> a(t), or None for a == 1.  With ``steps``, fn is tabulated
        once at half-integer times for the next ``steps`` steps (no callbacks
        while stepping); otherwise the library calls fn back every step."""
        if fn is not None and steps is not None:
            t0 = self.t
            tab = np.array([float(fn(t0 + 0.5 * k)) for k in range(2 * int(steps) + 3)])
            self._env = None
            self._check(self._L.lbm_set_envelope_table(self.h, _dp(tab), len(tab), float(t0)))
            return
        if fn is None:
            self._env = None
            self._check(self._L.lbm_set_envelope(self.h, ENVELOPE(), None))
            return
        self._env = ENVELOPE(lambda t, user: float(fn(t)))
        self._check(self._L.lbm_set_envelope(self.h, self._env, None))

    def set_stochastic_rounding(self, on=True, seed=0):
        """16-bit storage: round the stored deviations stochastically (seeded,
        counter-based) instead of to nearest."""
        self._check(self._L.lbm_set_stochastic_rounding(self.h, int(bool(on)), int(seed) & (2 ** 64 - 1)))

    def set_local_reference(self, every):
        """16-bit D2Q9 / D2Q5 storage at a per-node reference rebuilt every
        `every` steps (0: the plain deviations); lbm_set_local_reference."""
        self._check(self._L.lbm_set_local_reference(self.h, int(every)))

    # -- stepping and output -----------------------------------------------
    def step(self, n=1):
        self._check(self._L.lbm_step(self.h, int(n)))

    def moments(self, half_forced=True, out=None, where=0):
        """Host: returns rho [N], u [dim][N] (flow) or phi [N] (scalar).
        Device (where=1): fills the given (rho, u) device buffers."""
        if where == 1:
            rho, u = out
            self._check(self._L.lbm_moments(self.h, _ptr(rho), _ptr(u), 1, int(bool(half_forced))))
            return out
        rho = np.empty(self.N)
        u = np.empty((self.dim, self.N)) if self.lattice != D2Q5_CDE else None
        self._check(self._L.lbm_moments(self.h, rho.ctypes.data, None if u is None else u.ctypes.data, 0,
                                        int(bool(half_forced))))
        return rho if self.lattice == D2Q5_CDE else (rho, u)

    def reduce(self):
        """[sum rho, sum jx, sum jy, sum jz, max change since last call]; raises on instability."""
        out = np.empty(5)
        self._check(self._L.lbm_reduce(self.h, _dp(out)))
        return out

    def l2_error(self, ref, field=0, half_forced=True):
        """Eq. sca against a reference field, summed on the GPU: returns
        (sum (q - ref)^2, sum ref^2, relative l2 error).  field 0: rho / phi
        ([N]); field 1: u ([dim][N]).  ref: a numpy array (host) or a CUDA
        tensor (anything with ``data_ptr`` and ``is_cuda``) of float64."""
        out = np.empty(3)
        if getattr(ref, "is_cuda", False):
            n = ref.numel()
            if ref.dtype != _torch_float64() or not ref.is_contiguous():
                raise ValueError("reference tensor must be contiguous float64")
            ptr, where = ctypes.c_void_p(ref.data_ptr()), 1
        else:
            ref = np.ascontiguousarray(ref, dtype=np.float64)
            n = ref.size
            ptr, where = ref.ctypes.data_as(ctypes.c_void_p), 0
        want = self.N * (1 if field == 0 else self.dim)
        if n != want:
            raise ValueError(f"reference must hold {want} values, got {n}")
        self._check(self._L.lbm_l2_error(self.h, ptr, where, int(field), int(bool(half_forced)), _dp(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def debug_poison(self):
        """Fill the destination buffer of the next step with NaN (debug aid)."""
        self._check(self._L.lbm_debug_poison(self.h))

    def save_checkpoint(self, path):
        """Write f(t), the step counter and the lattice description to an .npz file."""
        np.savez(path, f=self.get_populations(), t=self.t, lattice=self.lattice, shape=np.array(self.shape),
                 storage=self.storage)

    def load_checkpoint(self, path):
        """Restore a checkpoint written by save_checkpoint on a lattice of the
        same kind, shape and storage (bitwise resume)."""
        with np.load(path) as z:
            if int(z["lattice"]) != self.lattice or tuple(z["shape"]) != tuple(self.shape) or \
                    int(z["storage"]) != self.storage:
                raise ValueError("checkpoint does not match this lattice")
            self.set_populations(np.ascontiguousarray(z["f"]), step=int(z["t"]))

    def strain_rate(self, rho0=1.0):
        """Strain-rate tensor [ncomp][N] (2D: xx, yy, xy; 3D: xx, yy, zz, xy, xz, yz)
        from the non-equilibrium second moments (Sec. 6.6)."""
        S = np.empty((3 if self.dim == 2 else 6, self.N))
        self._check(self._L.lbm_strain_rate(self.h, float(rho0), _dp(S), 0))
        return S

    def set_source_from_strain(self, flow, coef, rho0=1.0):
        """Source shape of this scalar lattice := coef * S:S of `flow` (viscous heating)."""
        self._check(self._L.lbm_set_source_from_strain(self.h, flow.h, float(rho0), float(coef)))

    def reduce_sums_noalloc(self):
        """[sum rho, sum jx, sum jy, sum jz] like :meth:`reduce`, computed with the
        library's fixed device scratch array instead of allocated memory."""
        out = np.empty(4)
        self._check(self._L.lbm_reduce_sums_noalloc(self.h, _dp(out)))
        return out

    def get_populations(self, out=None, where=0, with_step=False):
        """f(t) as [q][N] doubles (host, or into the device buffer `out` when
        where = 1); with_step also returns t, the step of the state copied."""
        t = ctypes.c_long()
        if where == 1:
            self._check(self._L.lbm_get_populations(self.h, _ptr(out), self.q * self.N, 1, ctypes.byref(t)))
            return (out, t.value) if with_step else out
        f = np.empty((self.q, self.N))
        self._check(self._L.lbm_get_populations(self.h, f.ctypes.data, f.size, 0, ctypes.byref(t)))
        return (f, t.value) if with_step else f

    def set_populations(self, f, step=0, where=0):
        if where == 1:
            self._check(self._L.lbm_set_populations(self.h, _ptr(f), self.q * self.N, 1, int(step)))
            return
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.size == self.q * self.N
        self._check(self._L.lbm_set_populations(self.h, f.ctypes.data, f.size, 0, int(step)))

    @property
    def t(self):
        v = ctypes.c_long()
        self._check(self._L.lbm_get_step(self.h, ctypes.byref(v)))
        return v.value

    def sync(self):
        self._check(self._L.lbm_sync(self.h))

    def launch_count(self):
        v = ctypes.c_longlong()
        self._check(self._L.lbm_launch_count(self.h, ctypes.byref(v)))
        return v.value


class Batch:
    """Lattices of one kind stepped together, one kernel launch per step
    (``lbm_batch_*``).  The member :class:`Lattice` objects must stay alive."""

    def __init__(self, lattices):
        L = load()
        self._L = L
        self.members = list(lattices)
        arr = (ctypes.c_void_p * len(self.members))(*[m.h.value for m in self.members])
        h = ctypes.c_void_p()
        rc = L.lbm_batch_create(ctypes.byref(h), arr, len(self.members))
        if rc != OK:
            raise LBMError(rc, L.lbm_batch_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise LBMError(rc, self._L.lbm_batch_last_error(self.h).decode())

    def step(self, n=1):
        self._check(self._L.lbm_batch_step(self.h, int(n)))

    def launch_count(self):
        v = ctypes.c_longlong()
        self._check(self._L.lbm_batch_launch_count(self.h, ctypes.byref(v)))
        return v.value

    def set_graph(self, steps_per_graph):
        """Replay steps as CUDA graphs of that many launches (even; 0 = off)."""
        self._check(self._L.lbm_batch_set_graph(self.h, int(steps_per_graph)))

    def graph_replays(self):
        v = ctypes.c_longlong()
        self._check(self._L.lbm_batch_graph_replays(self.h, ctypes.byref(v)))
        return v.value

    def moments_into(self, rho_ptrs, u_ptrs=None, where=0, half_forced=True):
        """Fields of every member into caller buffers given as raw addresses
        (host when where = 0, e.g. pinned torch tensors' data_ptr(); device
        when where = 1); one synchronisation for the whole batch."""
        n = len(self.members)
        r = (ctypes.c_void_p * n)(*[int(p) for p in rho_ptrs])
        u = None if u_ptrs is None else (ctypes.c_void_p * n)(*[int(p) for p in u_ptrs])
        self._check(self._L.lbm_batch_moments(self.h, r, u, int(where), int(bool(half_forced))))

    def moments(self, half_forced=True):
        """Fields of every member as numpy arrays: phi [N] (scalar lattice) or
        (rho [N], u [dim][N]) per member."""
        outs = []
        for m in self.members:
            if m.lattice == D2Q5_CDE:
                outs.append(np.empty(m.N))
            else:
                outs.append((np.empty(m.N), np.empty((m.dim, m.N))))
        if self.members[0].lattice == D2Q5_CDE:
            self.moments_into([o.ctypes.data for o in outs], None, 0, half_forced)
        else:
            self.moments_into([o[0].ctypes.data for o in outs], [o[1].ctypes.data for o in outs], 0, half_forced)
        return outs

    def moments_packed_into(self, rho_ptr, u_ptr=None, where=0, half_forced=True):
        """Fields of every member, packed member after member, into one buffer
        each (raw addresses: host when where = 0 or 2, device when where = 1,
        device-addressable pinned host memory when where = 3, which the kernel
        writes directly); one kernel launch for the whole batch.  where = 2 and
        3 are asynchronous (see wait_moments)."""
        self._check(self._L.lbm_batch_moments_packed(self.h, ctypes.c_void_p(int(rho_ptr)),
                                                     None if u_ptr is None else ctypes.c_void_p(int(u_ptr)),
                                                     int(where), int(bool(half_forced))))

    def step_read_into(self, rho_ptr, u_ptr=None, where=3, half_forced=True):
        """One step of every member whose kernel also writes the packed fields
        of the state it starts from (raw addresses: device when where = 1,
        device-addressable pinned host memory when where = 3); asynchronous,
        complete after wait_moments.  FP64 batches only."""
        self._check(self._L.lbm_batch_step_read(self.h, ctypes.c_void_p(int(rho_ptr)),
                                                None if u_ptr is None else ctypes.c_void_p(int(u_ptr)),
                                                int(where), int(bool(half_forced))))

    def wait_moments(self, keep=0):
        """Wait for asynchronous readbacks (where = 2 or 3): all (keep = 0) or
        all but the `keep` most recent ones (keep = 1 or 2)."""
        self._check(self._L.lbm_batch_wait_moments(self.h, int(keep)))

    def moments_packed(self, half_forced=True):
        """(rho or phi [sum N], u [sum dim*N] or None) packed member after member."""
        n = sum(m.N for m in self.members)
        rho = np.empty(n)
        if self.members[0].lattice == D2Q5_CDE:
            self.moments_packed_into(rho.ctypes.data, None, 0, half_forced)
            return rho, None
        u = np.empty(self.members[0].dim * n)
        self.moments_packed_into(rho.ctypes.data, u.ctypes.data, 0, half_forced)
        return rho, u

    def set_tiling(self, tile, persistent=False):
        """Tile of 128/256/512 nodes per block; persistent grid or one block per tile."""
        self._check(self._L.lbm_batch_set_tiling(self.h, int(tile), int(bool(persistent))))

    def tiling(self):
        """(tile, persistent, grid) of the launches."""
        t, p, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._L.lbm_batch_get_tiling(self.h, ctypes.byref(t), ctypes.byref(p), ctypes.byref(g)))
        return t.value, bool(p.value), g.value

    def autotune(self, trial_steps=5, all_timings=False):
        """Time every tiling on the batch itself and keep the fastest; returns
        its average microseconds per launch (with all_timings, also a dict
        {(tile, persistent): microseconds} of every tiling tried).  Leaves the
        state unchanged."""
        us = ctypes.c_double()
        every = (ctypes.c_double * 6)()
        self._check(self._L.lbm_batch_autotune(self.h, int(trial_steps), ctypes.byref(us), every))
        if not all_timings:
            return us.value
        tried = {(t, bool(p)): every[2 * j + p] for j, t in enumerate((128, 256, 512)) for p in (0, 1)
                 if every[2 * j + p] >= 0}
        return us.value, tried

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self._L.lbm_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


DEVICE_INFO_KEYS = ("sm_count", "sm_max_khz", "mem_khz", "bus_bits", "l2_bytes", "cc_major", "cc_minor",
                    "max_threads_per_sm")


def device_info(device=0):
    """Attributes of a CUDA device (lbm_device_info) as a dict."""
    L = load()
    info = (ctypes.c_longlong * 8)()
    rc = L.lbm_device_info(int(device), info)
    if rc != OK:
        raise LBMError(rc, L.lbm_probe_last_error().decode())
    return dict(zip(DEVICE_INFO_KEYS, list(info)))


FP64_FMA, FP64_ADD, FP64_MUL = 0, 1, 2


def probe_fp64(op, blocks, threads, iters, sink_ptr, stream=None, chains=8):
    """Queue the FP64 throughput probe (lbm_probe_fp64): blocks * threads *
    iters * chains FP64 instructions of kind op; sink_ptr is the address of
    three device doubles (block 0's SM cycles and nanoseconds land in the
    first two).  Asynchronous on `stream`; returns the count."""
    L = load()
    s = None if stream is None else ctypes.c_void_p(int(stream))
    rc = L.lbm_probe_fp64(int(op), int(chains), int(blocks), int(threads), int(iters),
                          ctypes.c_void_p(int(sink_ptr)), s)
    if rc != OK:
        raise LBMError(rc, L.lbm_probe_last_error().decode())
    return int(blocks) * int(threads) * int(iters) * int(chains)


def from_workload(w, stream=None, envelope_steps=None, storage=FP64) -> Lattice:
    """Lattice set up (force/source, velocity, envelope, equilibrium) from a
    :class:`paper_1806_10247_gb300.workloads.Workload`."""
    lat = {1: D2Q9, 2: D3Q27, 3: D2Q5_CDE, 4: D3Q15}[w.lattice]
    L = Lattice(lat, w.shape, w.omega, wall=w.wall, stream=stream, storage=storage)
    if w.tables is not None:
        if lat == D2Q5_CDE:
            L.set_source(tables=w.tables)
        else:
            L.set_force(tables=w.tables)
    if lat == D2Q5_CDE:
        u = np.asarray(w.u0, np.float64)
        L.set_velocity(tables=[(np.array([u[0]]), np.array([1.0]), np.array([1.0])),
                               (np.array([u[1]]), np.array([1.0]), np.array([1.0]))])
    if w.envelope is not None:
        L.set_envelope(w.envelope, steps=envelope_steps)
    L.init_equilibrium(w.rho0, w.u0)
    return L

"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/lbm.h declares.  No compute calls (no
GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1806_10247_gb300 import build as B
from paper_1806_10247_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no entry points found in include/"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(lbm.EXPORTS) <= declared


def test_exports_are_c_symbols():
    out = subprocess.run(["nm", "-D", "--defined-only", B.build()], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in _declared():
        assert n in syms, n  # unmangled: extern "C"


def test_create_fails_cleanly_without_gpu_or_on_bad_args():
    """Argument validation happens before any device call, so bad arguments
    give LBM_EINVAL with a message even without a GPU."""
    L = lbm.load()
    h = ctypes.c_void_p()
    r = lbm._Relax()
    for k in range(9):
        r.omega[k] = 1.0
    rc = L.lbm_create(ctypes.byref(h), 99, 4, 4, 1, ctypes.byref(r), None, 0, None)
    assert rc == lbm.EINVAL and b"unknown lattice" in L.lbm_last_error(None)
    rc = L.lbm_create(ctypes.byref(h), lbm.D2Q9, 4, 4, 2, ctypes.byref(r), None, 0, None)
    assert rc == lbm.EINVAL and b"nz must be 1" in L.lbm_last_error(None)
    r.omega[4] = 2.5
    rc = L.lbm_create(ctypes.byref(h), lbm.D2Q9, 4, 4, 1, ctypes.byref(r), None, 0, None)
    assert rc == lbm.EINVAL and b"omega[4]" in L.lbm_last_error(None)
    r.omega[4] = 1.0
    rc = L.lbm_create(ctypes.byref(h), lbm.D2Q9, 0, 4, 1, ctypes.byref(r), None, 0, None)
    assert rc == lbm.EINVAL
    rc = L.lbm_create(ctypes.byref(h), lbm.D2Q9, 4, 4, 1, ctypes.byref(r), None, 7, None)
    assert rc == lbm.EINVAL and b"storage" in L.lbm_last_error(None)
    # node counts beyond the 32-bit index range of the kernels, and between
    # LBM_MAX_NODES = 2^31 - 2^16 and 2^31 - 1 (a last block's thread indices
    # would pass 2^31)
    rc = L.lbm_create(ctypes.byref(h), lbm.D3Q27, 2048, 1024, 1025, ctypes.byref(r), None, 0, None)
    assert rc == lbm.EINVAL and b"LBM_MAX_NODES" in L.lbm_last_error(None)
    hdr = open(os.path.join(ROOT, "include", "lbm.h")).read()
    assert f"#define LBM_MAX_NODES {lbm.MAX_NODES}LL" in hdr
    assert 65537 * 32767 > lbm.MAX_NODES and 65537 * 32767 < 2 ** 31 - 1
    rc = L.lbm_create(ctypes.byref(h), lbm.D2Q5_CDE, 65537, 32767, 1, ctypes.byref(r), None, lbm.FP32_DEV, None)
    assert rc == lbm.EINVAL and b"LBM_MAX_NODES" in L.lbm_last_error(None)
    # D3Q15 stores FP64 only; walls on z for a 2D lattice; unknown boundary kind
    rc = L.lbm_create(ctypes.byref(h), lbm.D3Q15, 4, 4, 4, ctypes.byref(r), None, lbm.FP32_DEV, None)
    assert rc == lbm.EINVAL and b"D3Q15" in L.lbm_last_error(None)
    bc = lbm._Boundary()
    bc.axis[2] = lbm.BOUNCE_BACK
    rc = L.lbm_create(ctypes.byref(h), lbm.D2Q9, 4, 4, 1, ctypes.byref(r), ctypes.byref(bc), 0, None)
    assert rc == lbm.EINVAL and b"walls on z" in L.lbm_last_error(None)
    bc.axis[2] = 0
    bc.axis[0] = 7
    rc = L.lbm_create(ctypes.byref(h), lbm.D2Q9, 4, 4, 1, ctypes.byref(r), ctypes.byref(bc), 0, None)
    assert rc == lbm.EINVAL and b"boundary kind" in L.lbm_last_error(None)
    # D3Q15 validates its four rates (omega[1..4])
    r.omega[3] = 0.0
    rc = L.lbm_create(ctypes.byref(h), lbm.D3Q15, 4, 4, 4, ctypes.byref(r), None, 0, None)
    assert rc == lbm.EINVAL and b"omega[3]" in L.lbm_last_error(None)
    assert h.value is None


def test_batch_and_nn_entry_points_reject_null_handles():
    """The batch and network entry points validate their handles and
    arguments on the host."""
    L = lbm.load()
    h = ctypes.c_void_p()
    assert L.lbm_batch_create(ctypes.byref(h), None, 0) == lbm.EINVAL
    assert b"at least one context" in L.lbm_batch_last_error(None)
    assert L.lbm_batch_step(None, 1) == lbm.EINVAL
    assert L.lbm_batch_autotune(None, 1, None, None) == lbm.EINVAL
    assert L.lbm_batch_set_tiling(None, 256, 0) == lbm.EINVAL
    assert L.lbm_batch_moments(None, None, None, 0, 1) == lbm.EINVAL
    assert L.lbm_l2_error(None, None, 0, 0, 1, None) == lbm.EINVAL


def test_probe_and_device_info_validate_arguments():
    """The FP64 probe and the device query reject bad arguments on the host."""
    L = lbm.load()
    sink = ctypes.c_void_p(16)
    assert L.lbm_probe_fp64(3, 8, 1, 256, 1, sink, None) == lbm.EINVAL
    assert L.lbm_probe_fp64(0, 12, 1, 256, 1, sink, None) == lbm.EINVAL
    assert L.lbm_probe_fp64(0, 8, 0, 256, 1, sink, None) == lbm.EINVAL
    assert L.lbm_probe_fp64(0, 8, 1, 100, 1, sink, None) == lbm.EINVAL
    assert L.lbm_probe_fp64(0, 8, 1, 256, 0, sink, None) == lbm.EINVAL
    assert L.lbm_probe_fp64(0, 16, 1, 256, 1, None, None) == lbm.EINVAL
    assert b"bad arguments" in L.lbm_probe_last_error()
    assert L.lbm_device_info(0, None) == lbm.EINVAL


def test_oracle_and_product_share_no_code():
    """The CUDA sources never include the oracle and the product never imports it."""
    for d in ("paper_1806_10247_gb300", "paper_1806_10247_gb300/csrc", "include"):
        for f in os.listdir(os.path.join(ROOT, d)):
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(ROOT, d, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), (d, f)
                assert "lbm_oracle" not in src and "orc_" not in src, (d, f)

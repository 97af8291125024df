"""Benchmark of the cascaded LB hot path on GB300.

Default workload (the headline): 3D periodic Kolmogorov flow on the D3Q27
lattice, 512^3 nodes, FP64 populations and arithmetic: F_x = 1e-5 sin(2 pi y /
512), nu = 0.02, rho = 1 and seeded N(0, 1e-4^2) velocity noise.  One bench
step is one fused stream + collide kernel over the whole grid (the state,
2 x 29 GB, is far larger than L2, so nothing is flushed).  Each step is timed
with CUDA events on the library's stream.

Beside the headline the same line carries (unless --no-extras):
  * fp64_peak: the FP64 unit's instruction rates measured in this run
    (lbm_probe_fp64), the denominator of the FP64 kernels' roofline;
  * storages: the 512^3 grid with FP32 / FP16 / BF16 deviation storage
    (MLUPS, HBM roofline) and the relative l2 error of u after 1000 steps
    against the FP64 run from the same start;
  * workloads: every lattice of the metric ("per lattice"): D3Q27 256^3,
    D2Q9 channels, the D2Q5 scalar refinement sweep, D3Q15, and the batched
    sweep of 4096 lattices under an autotuned CUDA graph;
  * time_to_solution: steps and wall time to the solution criteria.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1806_10247_gb300 import workloads as W  # noqa: E402

METRIC = "MLUPS and % of HBM roofline per lattice; time-to-steady-state at ≤1e-4 L2 error"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129 * 1024 * 1024
Q_OF = {W.D2Q9: 9, W.D2Q5: 5, W.D3Q27: 27, W.D3Q15: 15}
Q_NAME = {W.D2Q9: "d2q9", W.D2Q5: "d2q5", W.D3Q27: "d3q27", W.D3Q15: "d3q15"}
ELEM = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}

# ---------------------------------------------------------------------------
# Algorithmic FP64 work per node of each FP64 step formulation, counted from
# its formulas (each add, multiply or fused multiply-add one operation; the
# correctly rounded reciprocal 1/rho one operation).  The derivation of each
# count is written out in the design notes; the bench uses the fixed count,
# never the instruction count of the current build.  The FMA / add / multiply
# split weights the measured rates of the FP64 unit into the peak of that mix.
_C = "paper_1806_10247_gb300/csrc/"
_H = [_C + "lbm_lattices.cuh", _C + "lbm_device.cuh"]
ALG_FP64 = {
    # D3Q27, omega_3..6 = 1, force along x: the force shape and the two half
    # forces (4), the forward transform along x (27) and the partial ones
    # along y and z (18 + 22), the half-forced j_x, 1/rho and u (5), the six
    # second-order central moments and their relaxation (23), the halved
    # back-shift with its known zeros (3 + 62), the force in moment space
    # (5), the halved inverse transform (81): 254 operations, 71 of them FMAs
    "d3q27": {"ops": 254, "fma": 71, "addmul": 183, "form": "unit higher rates, force along x"},
    # D2Q9, omega_6..8 = 1, force along x: the same steps on 9 populations
    # (force 2, moments 18, j_x, 1/rho, u 4, central moments and relaxation
    # 16, back-shift 15, post-collision force 3, inverse transform 18)
    "d2q9": {"ops": 77, "fma": 21, "addmul": 56, "form": "unit higher rates, force along x"},
    # D2Q5 with a uniform advecting velocity: the source shape (2), the
    # zeroth moment (4), the half source and the post-collision term (2),
    # rows 1-4 of the step matrix (20 FMAs), the new total and the rest
    # population (5)
    "d2q5": {"ops": 33, "fma": 22, "addmul": 11, "form": "uniform-velocity step matrix, separable source"},
}

# DRAM traffic per node of a launch (dram__bytes_read.sum + dram__bytes_write.sum
# of one ncu capture, divided by its node count), reported only while the
# kernel sources still hash to the value it was measured on.  Traffic per
# launch scales with the node count once the state is larger than L2.
TRAFFIC = {
    ("d3q27", "fp64"): {"src": [_C + "k_d3q27.cu"] + _H, "sha": "4be8a09ad4918a7a",
                        "bytes_per_node": (1529.134848 + 1477.492224) * 1e6 / 192 ** 3, "captured_nodes": 192 ** 3,
                        "profile": "profiles/k_step_d3q27_kolmogorov_fp64.md"},
    ("d3q27", "fp32"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                        "bytes_per_node": (1812.015360 + 1756.774400) * 1e6 / 256 ** 3, "captured_nodes": 256 ** 3,
                        "profile": "profiles/reduced_precision_traffic.md"},
    ("d3q27", "fp16"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                        "bytes_per_node": (382.343680 + 333.836032) * 1e6 / 192 ** 3, "captured_nodes": 192 ** 3,
                        "profile": "profiles/reduced_precision_traffic.md"},
    ("d3q27", "bf16"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                        "bytes_per_node": (382.267392 + 333.867776) * 1e6 / 192 ** 3, "captured_nodes": 192 ** 3,
                        "profile": "profiles/reduced_precision_traffic.md"},
    ("d2q9", "fp64"): {"src": [_C + "k_d2q9.cu"] + _H, "sha": "018f6162beb1528d",
                       "bytes_per_node": (151.018240 + 99.837696) * 1e6 / (2048 * 1024),
                       "captured_nodes": 2048 * 1024, "profile": "profiles/k_step_d2q9_channel2048_fp64.md"},
    ("d2q9", "fp32"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                       "bytes_per_node": (1207.990016 + 1153.966848) * 1e6 / (8192 * 4096),
                       "captured_nodes": 8192 * 4096, "profile": "profiles/reduced_precision_traffic.md"},
    ("d2q9", "fp16"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                       "bytes_per_node": (604.020736 + 551.098112) * 1e6 / (8192 * 4096),
                       "captured_nodes": 8192 * 4096, "profile": "profiles/reduced_precision_traffic.md"},
    ("d2q9", "bf16"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                       "bytes_per_node": (604.019712 + 551.259904) * 1e6 / (8192 * 4096),
                       "captured_nodes": 8192 * 4096, "profile": "profiles/reduced_precision_traffic.md"},
    ("d2q5", "fp64"): {"src": [_C + "k_d2q5.cu"] + _H, "sha": "80d05b85abca33c6", "above_l2": True,
                       "bytes_per_node": (2684.653056 + 2632.778752) * 1e6 / 8192 ** 2,
                       "captured_nodes": 8192 ** 2, "profile": "profiles/k_step5_k_step_mat_cde8192.md"},
    ("d2q5", "fp32"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                       "bytes_per_node": (1342.345984 + 1290.611200) * 1e6 / 8192 ** 2,
                       "captured_nodes": 8192 ** 2, "profile": "profiles/reduced_precision_traffic.md"},
    ("d2q5", "fp16"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                       "bytes_per_node": (671.200256 + 620.869632) * 1e6 / 8192 ** 2,
                       "captured_nodes": 8192 ** 2, "profile": "profiles/reduced_precision_traffic.md"},
    ("d2q5", "bf16"): {"src": [_C + "k_rp.cu"] + _H, "sha": "93ac4523479a40ea", "above_l2": True,
                       "bytes_per_node": (671.203840 + 621.302016) * 1e6 / 8192 ** 2,
                       "captured_nodes": 8192 ** 2, "profile": "profiles/reduced_precision_traffic.md"},
    # batched kernels (keys of the batched launches; the single-lattice
    # captures above do not describe them)
    ("d2q9_batch", "fp32"): {"src": [_C + "k_rp.cu", _C + "lbm_tiles.cuh", _C + "lbm_batch.cu"] + _H,
                             "sha": "a4c28ce2b40de990", "above_l2": True,
                             "bytes_per_node": (379.160576 + 335.486720) * 1e6 / 10521531, "captured_nodes": 10521531,
                             "profile": "profiles/reduced_precision_traffic.md"},
    ("d2q5_batch", "fp32"): {"src": [_C + "k_rp.cu", _C + "lbm_tiles.cuh", _C + "lbm_batch.cu"] + _H,
                             "sha": "a4c28ce2b40de990", "above_l2": True,
                             "bytes_per_node": (211.178752 + 167.969792) * 1e6 / 10521531, "captured_nodes": 10521531,
                             "profile": "profiles/reduced_precision_traffic.md"},
    ("d2q5_sweep", "fp64"): {"src": [_C + "k_d2q5.cu", _C + "lbm_tiles.cuh"] + _H, "sha": "47b4fe221b263702",
                             "bytes_per_node": 14.0096e6 / 349184, "captured_nodes": 349184,
                             "profile": "profiles/k_batch_d2q5_cde_sweep_fp64.md"},
}


def src_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_per_launch(key, nodes, state=None):
    """Traffic of one launch scaled from a capture by the node count, while
    the kernel sources are unchanged; captures marked above_l2 (taken on a
    state many times L2) apply only to states at least four times L2 (a
    smaller launch leaves part of its writes in L2)."""
    t = TRAFFIC.get(key)
    if t is None or src_hash(t["src"]) != t["sha"]:
        return None, None
    if t.get("above_l2") and (state is None or state < 4 * L2_BYTES):
        return None, None
    return t["bytes_per_node"] * nodes, t


def sweep_workloads():
    return [W.cde_workload(c) for c in W.cde_sweep_params()]


def batched_sweep_workloads(count=2048):
    channels, scalars = W.batched_sweep(count=count)
    return channels + scalars


# name -> (config name, maker, CPU-sample maker or None)
WORKLOADS = {
    "kolmogorov512": ("kolmogorov_d3q27_512cubed", lambda: [W.kolmogorov(n=512)],
                      (lambda: [W.kolmogorov(shape=(512, 64, 64))],
                       "a 512 x 64 x 64 periodic Kolmogorov lattice (the same lattice, rates, force amplitude and "
                       "noise; 1/64 of the grid)")),
    "kolmogorov256": ("kolmogorov_d3q27_256cubed", lambda: [W.kolmogorov(n=256)],
                      (lambda: [W.kolmogorov(shape=(256, 64, 64))],
                       "a 256 x 64 x 64 periodic Kolmogorov lattice (1/16 of the grid)")),
    "cde_sweep": ("cde_d2q5_refinement_sweep", sweep_workloads, None),
    "poiseuille": ("poiseuille_d2q9_3x33", lambda: [W.poiseuille()], None),
    "duct128": ("duct_d3q27_128x128x128", lambda: [W.duct(n=128, nx=128)], None),
    "kolmogorov96": ("kolmogorov_d3q27_96cubed", lambda: [W.kolmogorov(n=96)], None),
    "kolmogorov192": ("kolmogorov_d3q27_192cubed", lambda: [W.kolmogorov(n=192)], None),
    "channel2048": ("channel_d2q9_2048x1024", lambda: [W.poiseuille(ny=1024, nx=2048)], None),
    "channel8192": ("channel_d2q9_8192x4096", lambda: [W.poiseuille(ny=4096, nx=8192)], None),
    # the scalar sweep's manufactured-source problem on one 8192^2 grid (a
    # state many times L2), for the D2Q5 kernels' throughput
    "cde8192": ("cde_d2q5_8192x8192", lambda: [W.cde_workload(W.cde_sweep_params(sizes=(8192,))[0])], None),
    "batched_sweep": ("batched_sweep_2048_d2q9_channels_2048_d2q5_scalars", batched_sweep_workloads, None),
    "duct15_128": ("duct_d3q15_128x128x128", lambda: [W.duct15(n=128, nx=128)], None),
    # smaller forms of the workloads above, for profiler captures
    "batched_sweep256": ("batched_sweep_256_d2q9_channels_256_d2q5_scalars", lambda: batched_sweep_workloads(256),
                         None),
    "duct15_96": ("duct_d3q15_96x96x96", lambda: [W.duct15(n=96, nx=96)], None),
}
DEFAULT_WORKLOAD = "kolmogorov512"
# storage, steps per CUDA-graph replay (0 = plain launches) and autotuning per
# workload when the command line does not say
WORKLOAD_DEFAULTS = {"batched_sweep": {"storage": "fp32", "graph": 10, "tune": True},
                     "batched_sweep256": {"storage": "fp32", "graph": 10, "tune": True}}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the GPU is loaded."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, tag="bench"):
        self.idx = gpu_index
        self.proc = None
        out = os.environ.get("LBM_RESULTS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_{tag}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the reference arm)

def oracle_lattices(workloads):
    from oracle import oracle as O

    lats = []
    for w in workloads:
        P = O.expand_separable(w.tables, w.shape) if w.tables is not None else None
        uadv = None
        if w.lattice == W.D2Q5:
            uadv = np.stack([np.full(w.nodes, w.u0[0]), np.full(w.nodes, w.u0[1])])
        R = O.OracleLattice(w.lattice, w.shape, wall=w.wall, omega=w.omega, P=P, envelope=w.envelope,
                            uadv=uadv)
        R.init_equilibrium(w.rho0, w.u0)
        lats.append(R)
    return lats


def time_oracle(lats, nodes, steps, budget_s=None):
    """Step every oracle lattice `steps` times (or until ~budget_s seconds).
    Returns (node updates, seconds, steps done)."""
    done = 0
    t0 = time.perf_counter()
    while True:
        for R in lats:
            R.run(1)
        done += 1
        el = time.perf_counter() - t0
        if (budget_s is None and done >= steps) or (budget_s is not None and el >= budget_s):
            break
    return nodes * done, time.perf_counter() - t0, done


def state_bytes(wl, elem=8):
    return sum(2 * elem * Q_OF[w.lattice] * w.nodes for w in wl)


def cpu_sample(name, wl=None, limit=1 << 30):
    """A bounded sample of a workload for the CPU oracle: the workload's own
    sample lattice where it names one (single grids too large for seconds of
    CPU work), every lattice when the FP64 state is below `limit` bytes, else
    an evenly strided subset of the lattices."""
    spec = WORKLOADS[name][2]
    if spec is not None:
        make, what = spec
        return make(), what
    if wl is None:
        wl = WORKLOADS[name][1]()
    if state_bytes(wl) < limit or len(wl) == 1:
        return wl, "the whole workload"
    stride = 1
    while state_bytes(wl[::stride]) >= limit:
        stride *= 2
    sub = wl[::stride]
    return sub, f"every {stride}-th lattice ({len(sub)} of {len(wl)}, {sum(w.nodes for w in sub)} nodes)"


def cpu_baselines(name, wl, budget_s, single_budget_s):
    """The oracle on the host cores: all cores (OpenMP), then one thread on a
    smaller sample where the all-core sample would take too long."""
    from oracle import oracle as O

    O.build()
    sub, what = cpu_sample(name, wl)
    lats = oracle_lattices(sub)
    nodes = sum(w.nodes for w in sub)
    threads = O.set_threads(os.cpu_count() or 1)
    time_oracle(lats, nodes, 1)
    upd, sec, done = time_oracle(lats, nodes, None, budget_s=budget_s)
    out = {"value": upd / sec / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
           "sample": f"{done} steps of {what} ({upd} node updates, {sec:.1f} s)",
           "cpu": cpu_model()}
    try:
        O.set_threads(1)
        if nodes > 1_000_000:
            # one thread: a slab of the sample (the same per-node work)
            sw = sub[0]
            nz = max(2, int(sw.shape[2] * 1_000_000 / nodes))
            small = [W.kolmogorov(shape=(sw.shape[0], sw.shape[1] // 4, nz))] if sw.lattice == W.D3Q27 else sub
            what1 = f"a {small[0].shape[0]} x {small[0].shape[1]} x {small[0].shape[2]} lattice of the same kind"
        else:
            small, what1 = sub, what
        l1 = oracle_lattices(small)
        n1 = sum(w.nodes for w in small)
        time_oracle(l1, n1, 1)
        upd1, sec1, done1 = time_oracle(l1, n1, None, budget_s=single_budget_s)
        out["single_thread"] = {"value": upd1 / sec1 / 1e6, "unit": "MLUPS", "cores": 1,
                                "sample": f"{done1} steps of {what1} ({upd1} node updates, {sec1:.1f} s)"}
    finally:
        O.set_threads(threads)
    return out


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_reference(args, world, rank):
    if rank != 0:
        return
    wname = WORKLOADS[args.workload][0]
    from oracle import oracle as O

    O.build()
    sub, what = cpu_sample(args.workload)
    lats = oracle_lattices(sub)
    nodes = sum(w.nodes for w in sub)
    threads = O.set_threads(os.cpu_count() or 1)
    time_oracle(lats, nodes, args.warmup)
    upd, sec, done = time_oracle(lats, nodes, args.steps)
    v = upd / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / done * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block(None, wname, args.storage, name=args.workload),
        "cpu_baseline": {"kind": "oracle", "value": v, "unit": "MLUPS", "cores": threads,
                         "sample": f"{done} steps of {what} ({upd} node updates)", "cpu": cpu_model()},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_block(wl, cname, storage="fp64", elem=8, name=None):
    """The workload named in the JSON line (wl None: described from its name
    without building it)."""
    if wl is None:
        if name in ("kolmogorov512", "kolmogorov256"):
            n = 512 if name == "kolmogorov512" else 256
            lat, nodes, kinds, first = [f"kolmogorov_d3q27_{n}x{n}x{n}"], n ** 3, 1, W.D3Q27
            sb = 2 * elem * 27 * nodes
        else:
            wl = WORKLOADS[name][1]()
    if wl is not None:
        if len(wl) <= 16:
            lat = [w.name for w in wl]
        else:
            lat = {}
            for w in wl:
                k = Q_NAME[w.lattice]
                e = lat.setdefault(k, {"count": 0, "nodes": 0, "min_nodes": w.nodes, "max_nodes": w.nodes})
                e["count"] += 1
                e["nodes"] += w.nodes
                e["min_nodes"] = min(e["min_nodes"], w.nodes)
                e["max_nodes"] = max(e["max_nodes"], w.nodes)
        nodes = sum(w.nodes for w in wl)
        kinds = len({w.lattice for w in wl})
        first = wl[0].lattice
        sb = state_bytes(wl, elem)
    c = {"workload": cname, "storage": storage, "lattices": lat, "nodes_per_step": nodes, "seed": W.SEED,
         "launch": ("one fused stream+collide kernel per time step" if len(lat) == 1 else
                    "one batched fused stream+collide kernel per time step") +
                   (" per lattice kind" if kinds > 1 else ""),
         "parallelism": "replicas (one independent copy of the workload per GPU)"}
    c["l2"] = ("flushed before every timed step (256 MB write); the state fits in L2" if sb < 2 * L2_BYTES else
               "state larger than L2 (no flush needed)")
    if first == W.D3Q27 and (name or "").startswith("kolmogorov"):
        c.update({"F0": 1e-5, "nu": 0.02, "noise": 1e-4})
    if wl is not None and first == W.D2Q5 and len(wl) <= 16:
        c["D"] = wl[0].meta["D"]
        c["A32"] = wl[0].meta["A"]
    return c


# ---------------------------------------------------------------------------
# GPU measurements

def torch_sync(stream):
    stream.synchronize()


class Run:
    """Lattices of a workload on the GPU, one batch (one fused step kernel per
    time step) per lattice kind; a batch of one member steps with the
    single-lattice kernel."""

    def __init__(self, lbm, stream, wl, storage, env_steps, graph=0, tune=False):
        import torch

        self.torch = torch
        self.lbm = lbm
        self.stream = stream
        self.wl = wl
        self.storage = storage
        self.elem = ELEM[storage]
        code = {"fp64": lbm.FP64, "fp32": lbm.FP32_DEV, "fp16": lbm.FP16_DEV, "bf16": lbm.BF16_DEV}[storage]
        self.lats = [lbm.from_workload(w, stream=stream.cuda_stream, envelope_steps=env_steps, storage=code)
                     for w in wl]
        self.kinds = []
        for w in wl:
            if w.lattice not in self.kinds:
                self.kinds.append(w.lattice)
        self.groups = [[L for L, w in zip(self.lats, wl) if w.lattice == k] for k in self.kinds]
        self.gwl = [[w for w in wl if w.lattice == k] for k in self.kinds]
        self.batches = [lbm.Batch(g) for g in self.groups]
        self.nodes = sum(w.nodes for w in wl)
        self.tuning = None
        if tune:
            self.tuning = []
            for k, b in zip(self.kinds, self.batches):
                us, tried = b.autotune(5, all_timings=True)
                t, p, g = b.tiling()
                self.tuning.append({"lattice": Q_NAME[k], "tile": t, "persistent": p, "grid": g,
                                    "trial_us_per_launch": us,
                                    "trials_us": {f"{tt}{'p' if pp else ''}": v for (tt, pp), v in tried.items()}})
        self.graph = graph
        for b in self.batches:
            b.set_graph(graph)
        self.need_flush = state_bytes(wl, self.elem) < 2 * L2_BYTES
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda") \
            if self.need_flush else None

    def launches(self):
        return sum(b.launch_count() for b in self.batches) + sum(L.launch_count() for L in self.lats)

    def warm(self, steps, unit, min_s=0.0):
        t0 = time.perf_counter()
        k = 0
        while k < steps or (time.perf_counter() - t0 < min_s and k < 2000):
            if self.need_flush:
                with self.torch.cuda.stream(self.stream):
                    self.flush.zero_()
            for b in self.batches:
                b.step(unit)
            k += unit
            if k % 50 < unit:
                self.stream.synchronize()
        self.torch.cuda.synchronize()

    def timed(self, steps, unit):
        """CUDA-event time of every batch's launches over `steps` steps, in
        `unit`-step calls (L2 flushed before each call when the state fits in
        it).  Returns per-batch milliseconds."""
        torch = self.torch
        n_units = steps // unit
        ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in self.batches]
              for _ in range(n_units)]
        for u in range(n_units):
            if self.need_flush:
                with torch.cuda.stream(self.stream):
                    self.flush.zero_()
            for bi, b in enumerate(self.batches):
                ev[u][bi][0].record(self.stream)
                b.step(unit)
                ev[u][bi][1].record(self.stream)
        torch.cuda.synchronize()
        return [sum(ev[u][bi][0].elapsed_time(ev[u][bi][1]) for u in range(n_units))
                for bi in range(len(self.batches))]

    def close(self):
        for b in self.batches:
            b.close()
        for L in self.lats:
            L.close()
        self.batches, self.lats = [], []
        self.flush = None


def fp64_peak(lbm, stream, info):
    """FP64 instruction rates of this GPU, measured with lbm_probe_fp64:
    independent dependency chains of one operation (8 or 16 per thread, the
    loop unrolled four times), 4 or 8 blocks of 256 threads per SM, CUDA
    events, best of 3 after a warm-up launch; the peak of each operation is
    the fastest configuration.  Block 0 of every probe launch also reports its
    own SM cycles and nanoseconds, which give the SM clock the rates were
    taken at (the cycles of one block are not the launch's: blocks beyond the
    resident ones run in later waves)."""
    import torch

    sink = torch.zeros(3, dtype=torch.float64, device="cuda")
    sms = int(info["sm_count"])
    threads = 256
    rates, tried, mhz_seen = {}, {}, []
    for op, name in ((lbm.FP64_FMA, "fma"), (lbm.FP64_ADD, "add"), (lbm.FP64_MUL, "mul")):
        best_rate = 0.0
        for chains in (8, 16):
            for per_sm in (4, 8):
                blocks = per_sm * sms
                iters = max(1000, int(4.0e10 / (blocks * threads * chains)))  # ~0.1 s at ~500 G/s
                lbm.probe_fp64(op, blocks, threads, 256, sink.data_ptr(), stream.cuda_stream, chains=chains)
                best = float("inf")
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    n = lbm.probe_fp64(op, blocks, threads, iters, sink.data_ptr(), stream.cuda_stream,
                                       chains=chains)
                    e1.record(stream)
                    e1.synchronize()
                    best = min(best, e0.elapsed_time(e1) * 1e-3)
                    cyc, ns = (float(v) for v in sink[:2].cpu())
                    if ns > 0:
                        mhz_seen.append(cyc / ns * 1e3)
                r = n / best / 1e9
                tried[f"{name}_chains{chains}_blocks{per_sm}xSM"] = r
                best_rate = max(best_rate, r)
        rates[name] = best_rate
    mhz = float(np.median(mhz_seen)) if mhz_seen else info["sm_max_khz"] / 1e3
    return {
        "fma_ginst_per_s": rates["fma"], "add_ginst_per_s": rates["add"], "mul_ginst_per_s": rates["mul"],
        "tflops_fma": 2 * rates["fma"] / 1e3,
        "per_clock_per_sm": {k: v * 1e3 / (sms * mhz) for k, v in rates.items()},
        "probe_sm_mhz": mhz, "probe_sm_mhz_range": [min(mhz_seen), max(mhz_seen)] if mhz_seen else None,
        "sm_count": sms, "sm_max_mhz": info["sm_max_khz"] / 1e3, "all_configurations_ginst_per_s": tried,
        "how": f"lbm_probe_fp64: 8 or 16 independent chains of one FP64 operation per thread (second and third "
               f"operands in constant memory, loop unrolled 4x), 4 or 8 blocks of {threads} threads per SM, CUDA "
               "events, best of 3 after a warm-up launch, the fastest configuration per operation; the SM clock "
               "from block 0's own cycles and nanoseconds (median over the probe launches)",
    }


def mix_peak(alg, peak):
    """Instruction rate (G/s) of an FP64 mix on the measured unit: each
    FMA at the FMA rate, each add or multiply at the mean add/multiply rate."""
    r_am = 0.5 * (peak["add_ginst_per_s"] + peak["mul_ginst_per_s"])
    t = alg["fma"] / peak["fma_ginst_per_s"] + alg["addmul"] / r_am
    return alg["ops"] / t


def roofline_block(kind, storage, nodes, kernel_s, hbm, hbm_src, peak, traffic_key=None, label=None):
    """Roofline of one kernel: HBM with the algorithmic bytes (Q populations
    read + Q written per node); FP64 kernels also against the FP64 unit with
    the algorithmic operation count and the measured rates, the larger
    fraction deciding the bound."""
    q = {"d3q27": 27, "d2q9": 9, "d2q5": 5, "d3q15": 15}[kind]
    bpn = 2 * ELEM[storage] * q
    gbs = bpn * nodes / kernel_s / 1e9
    traffic, tinfo = traffic_per_launch(traffic_key or (kind, storage), nodes, bpn * nodes)
    r = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": traffic,
         "kernel": label or f"{kind} step kernel ({nodes} nodes, {storage})",
         "peak_source": (f"measured (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else "fallback"),
         "bytes_per_node": bpn, "kernel_us": kernel_s * 1e6}
    if tinfo is not None:
        r["traffic_source"] = (f"ncu dram__bytes_read.sum + dram__bytes_write.sum per node of a {tinfo['captured_nodes']}"
                               f"-node capture x {nodes} nodes ({tinfo['profile']})")
    alg = ALG_FP64.get(kind) if storage == "fp64" else None
    if alg is not None and peak is not None:
        pk = mix_peak(alg, peak)
        gops = alg["ops"] * nodes / kernel_s / 1e9
        tf = (2 * alg["fma"] + alg["addmul"]) * nodes / kernel_s / 1e12
        hbm_part = {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "bytes_per_node": bpn}
        if gops / pk > r["frac"]:
            r.update({"bound": "alu", "achieved": gops, "peak": pk, "unit": "G FP64 op/s", "frac": gops / pk,
                      "peak_source": "measured in this run (lbm_probe_fp64): the FMA and add/multiply rates of the "
                                     "FP64 unit weighted by this formulation's mix (SM clock during the probe "
                                     f"{peak['probe_sm_mhz']:.0f} MHz)",
                      "ops_per_node": alg["ops"], "fma_per_node": alg["fma"], "formulation": alg["form"],
                      "hbm": hbm_part})
        r["flops"] = {"achieved": tf, "peak": peak["tflops_fma"], "unit": "TFLOP/s", "frac": tf / peak["tflops_fma"],
                      "flops_per_node": 2 * alg["fma"] + alg["addmul"],
                      "peak_source": "2 x the measured FMA rate"}
    return r


def measure(lbm, stream, name, storage, steps, warmup, hbm, hbm_src, peak, graph=0, tune=False, min_warm_s=0.0,
            wl=None, keep=False):
    """Time `steps` steps of a workload; returns (result dict, Run or None)."""
    wl = wl if wl is not None else WORKLOADS[name][1]()
    unit = graph if graph else 1
    steps = max(unit, steps // unit * unit)
    R = Run(lbm, stream, wl, storage, env_steps=warmup + steps + 64, graph=graph, tune=tune)
    try:
        R.warm(warmup, unit, min_warm_s)
        l0 = R.launches()
        ms = R.timed(steps, unit)
        launches = R.launches() - l0
        total = sum(ms)
        res = {"mlups": R.nodes * steps / (total * 1e-3) / 1e6, "ms_per_step": total / steps, "steps": steps,
               "nodes": R.nodes, "gpu_launches": launches}
        kernels = []
        for k, g, m in zip(R.kinds, R.gwl, ms):
            n = sum(w.nodes for w in g)
            kname = Q_NAME[k]
            # a batched launch has its own traffic entry (none: null), not the single-lattice kernel's
            tkey = None if len(g) == 1 else (("d2q5_sweep" if name == "cde_sweep" else f"{kname}_batch"), storage)
            kernels.append(roofline_block(kname, storage, n, m / steps * 1e-3, hbm, hbm_src, peak, tkey,
                                          label=f"{kname} {'batched ' if len(g) > 1 else ''}step kernel "
                                                f"({len(g)} lattice{'s' if len(g) > 1 else ''}, {n} nodes, {storage})"))
        dom = max(range(len(kernels)), key=lambda i: ms[i])
        res["roofline"] = kernels[dom]
        if len(kernels) > 1:
            res["all_kernels"] = kernels
        if R.tuning is not None:
            res["autotuned_tiling"] = R.tuning
        if graph:
            res["graph_steps"] = graph
        res["l2"] = "flushed before every timed step" if R.need_flush else "state larger than L2"
    except Exception:
        R.close()
        raise
    if keep:
        return res, R
    R.close()
    return res, None


def measure_e2e(R, ke, storage):
    """End to end through the public API with host buffers: per step the
    step's inputs (each lattice's envelope pair, evaluated on the host and
    sent with the launch) and the fields of every lattice read back into
    pinned host memory; the fastest of the fused, direct, overlapped-copy and
    synchronous readbacks is the headline, the others beside it."""
    torch = R.torch
    batches, wl, nodes = R.batches, R.wl, R.nodes
    for b in batches:
        b.set_graph(0)
    pinned_out = []  # per lattice kind, three slots: packed rho/phi and u of all members
    for k, ws_ in zip(R.kinds, R.gwl):
        n = sum(w.nodes for w in ws_)
        dim = 0 if k == W.D2Q5 else (3 if k in (W.D3Q27, W.D3Q15) else 2)
        pinned_out.append([(torch.empty(n, dtype=torch.float64, pin_memory=True),
                            torch.empty(dim * n, dtype=torch.float64, pin_memory=True) if dim else None)
                           for _ in range(3)])

    def read_back(slot):
        for b, slots in zip(batches, pinned_out):
            r_, u_ = slots[slot]
            b.moments_packed_into(r_.data_ptr(), None if u_ is None else u_.data_ptr())

    def read_back_async(k):
        for b, slots in zip(batches, pinned_out):
            r_, u_ = slots[k % 2]
            b.moments_packed_into(r_.data_ptr(), None if u_ is None else u_.data_ptr(), where=2)
        for b in batches:
            b.wait_moments(keep=1)

    def read_back_direct(k, depth):
        for b, slots in zip(batches, pinned_out):
            r_, u_ = slots[k % (depth + 1)]
            b.moments_packed_into(r_.data_ptr(), None if u_ is None else u_.data_ptr(), where=3)
        for b in batches:
            b.wait_moments(keep=depth)

    d2h = sum(r_.numel() * 8 + (0 if u_ is None else u_.numel() * 8) for r_, u_ in (sl[0] for sl in pinned_out))
    h2d = 16 * len(wl)

    def timed_loop(read):
        torch.cuda.synchronize()
        t0_ = time.perf_counter()
        for k in range(ke):
            for b in batches:
                b.step(1)
            read(k)
        for b in batches:
            b.wait_moments(keep=0)
        return nodes * ke / (time.perf_counter() - t0_) / 1e6

    def entry(v, path, **kw):
        d = {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ke,
             "path": path}
        d.update(kw)
        return d

    forms = {}
    forms["overlapped_copy"] = entry(
        timed_loop(read_back_async),
        "per step: lbm_batch_step(1) per lattice kind (the step's envelope pairs from the host), "
        "lbm_batch_moments_packed(where=2) into pinned host memory (kernel and copy overlapped with the next step, "
        "two slots in turn), every step's fields on the host before the timer stops")
    try:
        by_depth = {d: timed_loop(lambda k, d=d: read_back_direct(k, d)) for d in (1, 2)}
        depth = max(by_depth, key=by_depth.get)
        forms["direct"] = entry(
            by_depth[depth],
            "per step: lbm_batch_step(1) per lattice kind (the step's envelope pairs from the host), "
            "lbm_batch_moments_packed(where=3): the moments kernel writes the fields straight into pinned host "
            f"memory, overlapped with the next steps ({depth} in flight), every step's fields on the host before "
            "the timer stops", by_readbacks_in_flight={str(d): v for d, v in by_depth.items()})
    except Exception as exc:  # pinned memory the device cannot address
        forms["direct"] = {"value": None, "unavailable": str(exc)[:200]}
    if storage == "fp64":
        def fused_loop(depth):
            torch.cuda.synchronize()
            t0_ = time.perf_counter()
            for k in range(ke):
                for b, slots in zip(batches, pinned_out):
                    r_, u_ = slots[k % (depth + 1)]
                    b.step_read_into(r_.data_ptr(), None if u_ is None else u_.data_ptr(), where=3)
                for b in batches:
                    b.wait_moments(keep=depth)
            for b in batches:
                b.wait_moments(keep=0)
            read_back(ke % 2)
            return nodes * ke / (time.perf_counter() - t0_) / 1e6

        try:
            by_depth = {d: fused_loop(d) for d in (1, 2)}
            depth = max(by_depth, key=by_depth.get)
            forms["fused"] = entry(
                by_depth[depth],
                "per step: lbm_batch_step_read(where=3) per lattice kind (the step's envelope pairs from the host; "
                "the step kernel writes the fields of the state it starts from straight into pinned host memory, "
                f"{depth} step(s) in flight), the state after the last step read with lbm_batch_moments_packed; "
                "every step's fields on the host before the timer stops",
                by_steps_in_flight={str(d): v for d, v in by_depth.items()})
        except Exception as exc:
            forms["fused"] = {"value": None, "unavailable": str(exc)[:200]}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(ke):
        for b in batches:
            b.step(1)
        read_back(k % 2)
    forms["synchronous"] = entry(
        nodes * ke / (time.perf_counter() - t0) / 1e6,
        "per step: lbm_batch_step(1) per lattice kind (the step's envelope pairs from the host), "
        "lbm_batch_moments_packed(where=0) into pinned host memory: one synchronisation per step")
    best = max((k for k in forms if forms[k].get("value") is not None), key=lambda k: forms[k]["value"])
    e2e = dict(forms[best])
    e2e["form"] = best
    e2e["other_forms"] = {k: {kk: v[kk] for kk in ("value", "unit", "path") if kk in v} if v.get("value") is not None
                          else v for k, v in forms.items() if k != best}
    if nodes <= 20_000_000:
        pinned_src = []
        for w in wl:
            from_tables = [((np.asarray(px)[None, None, :] * np.asarray(py)[None, :, None]) * np.asarray(pz)[:, None, None])
                           for px, py, pz in w.tables]
            full = np.ascontiguousarray(np.stack([np.broadcast_to(t, w.shape[::-1]).reshape(-1) for t in from_tables]))
            t_src = torch.empty(full.shape, dtype=torch.float64, pin_memory=True)
            t_src.numpy()[:] = full
            pinned_src.append(t_src)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            for L, s_ in zip(R.lats, pinned_src):
                if L.lattice == R.lbm.D2Q5_CDE:
                    L.set_source(full=s_.numpy())
                else:
                    L.set_force(full=s_.numpy())
            for b in batches:
                b.step(1)
            read_back(0)
        el = time.perf_counter() - t0
        e2e["full_field_upload"] = {
            "value": nodes * ke / el / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": sum(t.numel() * 8 for t in pinned_src), "d2h_bytes_per_step": d2h,
            "path": "as above plus lbm_set_source/lbm_set_force(host, full field) per lattice every step"}
    e2e["timing"] = ("host wall clock around the whole loop (steps back to back as a user runs them; L2 is not "
                     "flushed between them)")
    return e2e


def storage_study(lbm, stream, hbm, hbm_src, peak, steps, warmup, n=512, run_steps=1000):
    """The headline grid with every storage form: MLUPS and the HBM roofline
    over `steps` timed steps, then, from the same start, `run_steps` steps
    whose u is compared with the FP64 run's (relative l2 of Eq. sca, summed on
    the GPU against the FP64 field held on the device)."""
    import torch

    name = f"kolmogorov{n}"
    wl = WORKLOADS[name][1]()
    out = {"grid": f"{n}^3", "run_steps": run_steps}
    u_ref = None
    for st in ("fp64", "fp32", "fp16", "bf16"):
        entry = {}
        if st != "fp64":
            res, _ = measure(lbm, stream, name, st, steps, warmup, hbm, hbm_src, peak, wl=wl)
            entry.update(res)
        L = lbm.from_workload(wl[0], stream=stream.cuda_stream,
                              storage={"fp64": lbm.FP64, "fp32": lbm.FP32_DEV, "fp16": lbm.FP16_DEV,
                                       "bf16": lbm.BF16_DEV}[st])
        try:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.step(run_steps)
            e1.record(stream)
            e1.synchronize()
            entry["run"] = {"steps": run_steps, "mlups": wl[0].nodes * run_steps / (e0.elapsed_time(e1) * 1e-3) / 1e6,
                            "timing": "CUDA events around lbm_step(run_steps)"}
            if st == "fp64":
                u_ref = torch.empty(3 * wl[0].nodes, dtype=torch.float64, device="cuda")
                rho = torch.empty(wl[0].nodes, dtype=torch.float64, device="cuda")
                L.moments(out=(rho, u_ref), where=1)
                torch.cuda.synchronize()
                del rho
                entry["u_max"] = float(u_ref.abs().max().item())
            else:
                e2, e1_, rel = L.l2_error(u_ref, field=1)
                entry["l2_u_vs_fp64"] = rel
        finally:
            L.close()
        out[st] = entry
    del u_ref
    torch.cuda.empty_cache()
    return out


LREF_EVERY = {"poiseuille": 32, "cde": 16}  # rebuild intervals of the local-reference forms


def time_to_solution(lbm, stream, storages=("fp64", "fp32", "fp16", "bf16", "fp16_sr", "bf16_sr", "fp16_lref",
                                            "bf16_lref", "fp16_lref_sr", "bf16_lref_sr")):
    """The metric's second half: wall time to the solution criterion.
    * config 1 (Poiseuille D2Q9 3 x 33), FP64: steps until
      max |u(t) - u(t-100)| < 1e-12 (checked every 100 steps with lbm_reduce);
      its final profile is the steady reference u_ref (the FP64 GPU path agrees
      with the oracle to 1e-12 in the parity tests), also compared with the
      parabola of Sec. 6.1;
    * config 1, every storage form from rest: steps and wall time until the
      relative l2 distance (Eq. sca) of u to the FP64 steady field is <= 1e-4
      (lbm_l2_error on the GPU every 100 steps, the reference resident on the
      device, the checks inside the timed region);
    * config 2 (scalar sweep): every member run to its T_N, l2 error against the
      closed form and the convergence order over the sweep, per storage form
      (the 16-bit forms show how far their rounding moves the order).
    The *_sr forms are the 16-bit storages with stochastic rounding (seed
    10247; single-lattice launches, one per step); the *_lref forms store them
    at a per-node reference (lbm_set_local_reference, rebuilt every 32 steps
    for the channel and 16 for the scalar sweep; single-lattice launches plus
    the rebuild's kernels); *_lref_sr both."""
    import torch

    codes = {"fp64": lbm.FP64, "fp32": lbm.FP32_DEV, "fp16": lbm.FP16_DEV, "bf16": lbm.BF16_DEV}
    out = {}
    w = W.poiseuille()
    ua = np.tile(W.poiseuille_parabola(w.shape[1], w.meta["tau"], w.meta["Fx"])[:, None], (1, w.shape[0])).reshape(-1)

    def l2(a, b):
        return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))

    how = "one cluster launch of 100 steps (lbm_step) between checks"
    L = lbm.from_workload(w, stream=stream.cuda_stream, storage=lbm.FP64)
    L.reduce()
    torch_sync(stream)
    t0 = time.perf_counter()
    steps, du = 0, float("inf")
    while steps < 200000:
        L.step(100)
        steps += 100
        du = L.reduce()[4]
        if du < 1e-12:
            break
    sec = time.perf_counter() - t0
    _, u = L.moments()
    u_ref = u[0].copy()
    u_ref_dev = torch.from_numpy(np.ascontiguousarray(u)).to("cuda")
    out["poiseuille_fp64"] = {"steps": steps, "seconds": sec, "max_du": du, "l2_vs_parabola": l2(u_ref, ua),
                              "criterion": "max |u(t) - u(t-100)| < 1e-12 (lbm_reduce every 100 steps)",
                              "launch": how}
    L.close()
    for st in storages:
        L = lbm.from_workload(w, stream=stream.cuda_stream, storage=codes[st.split("_")[0]])
        if st.endswith("_sr"):
            L.set_stochastic_rounding(True, 10247)
        if "_lref" in st:
            L.set_local_reference(LREF_EVERY["poiseuille"])
        L.reduce()
        torch_sync(stream)
        t0 = time.perf_counter()
        steps, err = 0, float("inf")
        while steps < 200000:
            L.step(100)
            steps += 100
            err = L.l2_error(u_ref_dev, 1)[2]
            if err <= 1e-4:
                break
        sec = time.perf_counter() - t0
        out[f"poiseuille_{st}_to_1e-4"] = {
            "steps": steps, "seconds": sec, "l2_vs_fp64_steady": err, "reached": err <= 1e-4,
            "criterion": "relative l2 (Eq. sca) of u against the FP64 steady field <= 1e-4 (lbm_l2_error every "
                         "100 steps, reference on the device)",
            "launch": how if st.split("_")[-1] not in ("sr", "lref") else "lbm_step(100) between checks (one launch per step)"}
        L.close()
    for st in storages:
        cases = W.cde_sweep_params()
        errs, total = [], 0.0
        for c in cases:
            wc = W.cde_workload(c)
            G = lbm.from_workload(wc, stream=stream.cuda_stream, envelope_steps=c.T + 2,
                                  storage=codes[st.split("_")[0]])
            Bt = None
            if "_lref" in st:
                G.set_local_reference(LREF_EVERY["cde"])
            if st.endswith("_sr"):
                G.set_stochastic_rounding(True, 10247)
            if st.split("_")[-1] not in ("sr", "lref"):
                Bt = lbm.Batch([G])
                Bt.set_graph(200)
            torch_sync(stream)
            t0 = time.perf_counter()
            if Bt is not None:
                Bt.step(c.T)
            else:
                G.step(c.T)
            G.sync()
            total += time.perf_counter() - t0
            phi = G.moments().reshape(c.N, c.N) - 1.0
            ref = W.cde_closed_form(c, c.T)
            errs.append(float(np.sqrt(np.sum((phi - ref) ** 2) / np.sum(ref ** 2))))
            if Bt is not None:
                Bt.close()
            G.close()
        orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
        out[f"cde_sweep_{st}"] = {"seconds": total, "steps": [c.T for c in cases],
                                  "l2_vs_closed_form": errs, "orders": orders}
    return out


def batched_time_to_solution(lbm, stream, count=32, tmax=700.0, check=100):
    """Time to the steady state for the batched sweep (config 4): a subset of
    its members -- the first `count` channels and `count` scalar lattices
    (in the sweep's seeded order) whose slowest mode decays with a time
    constant below `tmax` steps (channel ny^2/(pi^2 nu), scalar
    max(nx, ny)^2/(4 pi^2 D)) -- first run in FP64 for 30 time constants of
    the slowest one (e^-30 ~ 1e-13: the FP64 steady fields); then, from rest,
    each form until every member's field is within 1e-4 relative l2 (Eq. sca;
    u for the channels, phi - phi0 for the scalars) of its FP64 steady field,
    checked every `check` steps on one packed readback per lattice kind:
      * FP32 deviations, batched, autotuned tiling, CUDA graphs of 10 steps;
      * FP64, batched (one launch per step and kind);
      * FP64, per-instance launches (one lbm_step per member).
    Reports steps to the criterion (the largest over members) and wall time
    (checks included)."""
    chans, scals = W.batched_sweep(count=2048)
    pick_c = [w for w in chans if w.shape[1] ** 2 / (math.pi ** 2 * w.meta["nu"]) < tmax][:count]
    pick_s = [w for w in scals if max(w.shape[0], w.shape[1]) ** 2 / (4 * math.pi ** 2 * w.meta["D"]) < tmax][:count]
    groups = [pick_c, pick_s]
    taus = [w.shape[1] ** 2 / (math.pi ** 2 * w.meta["nu"]) for w in pick_c] + \
           [max(w.shape[0], w.shape[1]) ** 2 / (4 * math.pi ** 2 * w.meta["D"]) for w in pick_s]
    ref_steps = int(math.ceil(30 * max(taus) / 1000.0)) * 1000
    codes = {"fp64": lbm.FP64, "fp32": lbm.FP32_DEV}

    def fields(B, ws):
        rho, u = B.moments_packed()
        out, off = [], 0
        for w in ws:
            n = w.nodes
            if w.lattice == W.D2Q5:
                out.append(rho[off:off + n] - w.rho0)
            else:
                out.append(u[2 * off:2 * off + 2 * n])
            off += n
        return out

    t0 = time.perf_counter()
    refs = []
    for ws in groups:
        Ls = [lbm.from_workload(w, stream=stream.cuda_stream, storage=lbm.FP64) for w in ws]
        B = lbm.Batch(Ls)
        B.set_graph(100)
        B.step(ref_steps)
        refs.append(fields(B, ws))
        B.close()
        for L in Ls:
            L.close()
    out = {"members": {"d2q9_channels": len(pick_c), "d2q5_scalars": len(pick_s)},
           "nodes": sum(w.nodes for g in groups for w in g),
           "fp64_reference": {"steps": ref_steps, "seconds": time.perf_counter() - t0,
                              "rule": "30 time constants of the slowest member"},
           "criterion": "relative l2 (Eq. sca) <= 1e-4 against the FP64 steady field, every member (u of the "
                        "channels, phi - phi0 of the scalars), checked every %d steps" % check}

    def run(form, storage, batched, graph=0, tune=False):
        lats = [[lbm.from_workload(w, stream=stream.cuda_stream, storage=codes[storage]) for w in ws]
                for ws in groups]
        batches = [lbm.Batch(Ls) for Ls in lats]
        tuning = None
        if tune:
            tuning = [b.autotune(5) for b in batches]
        for b in batches:
            b.set_graph(graph)
        done = [[None] * len(ws) for ws in groups]
        worst = [[float("inf")] * len(ws) for ws in groups]
        torch_sync(stream)
        t1 = time.perf_counter()
        steps = 0
        while steps < 4 * ref_steps:
            if batched:
                for b in batches:
                    b.step(check)
            else:
                for Ls in lats:
                    for L in Ls:
                        L.step(check)
            steps += check
            for gi, (b, ws) in enumerate(zip(batches, groups)):
                for mi, (q, r) in enumerate(zip(fields(b, ws), refs[gi])):
                    e = float(np.sqrt(np.sum((q - r) ** 2) / np.sum(r ** 2)))
                    worst[gi][mi] = e
                    if done[gi][mi] is None and e <= 1e-4:
                        done[gi][mi] = steps
            if all(d is not None for g in done for d in g):
                break
        sec = time.perf_counter() - t1
        for b in batches:
            b.close()
        for Ls in lats:
            for L in Ls:
                L.close()
        flat = [d for g in done for d in g]
        r = {"reached": all(d is not None for d in flat), "steps": max(d for d in flat if d is not None),
             "seconds": sec, "steps_median": float(np.median([d for d in flat if d is not None])),
             "l2_at_end_max": max(max(g) for g in worst),
             "launch": form}
        missed = [(gi, mi) for gi in range(len(groups)) for mi in range(len(groups[gi])) if done[gi][mi] is None]
        if missed:
            r["not_reached"] = [{"member": groups[gi][mi].name, "l2_at_end": worst[gi][mi],
                                 "tau": groups[gi][mi].meta.get("tau", groups[gi][mi].meta.get("tau_phi")),
                                 "amplitude": groups[gi][mi].meta.get("Fx", groups[gi][mi].meta.get("A"))}
                                for gi, mi in missed[:8]]
            r["not_reached_count"] = len(missed)
        if tuning is not None:
            r["autotuned_us_per_launch"] = tuning
        return r

    out["fp32_batched_graph"] = run("FP32 deviations, one batched launch per step and kind, autotuned tiling, "
                                    "CUDA graphs of 10 steps", "fp32", True, graph=10, tune=True)
    out["fp64_batched"] = run("FP64, one batched launch per step and kind", "fp64", True)
    out["fp64_per_instance"] = run("FP64, one lbm_step launch per member and step", "fp64", False)
    return out


def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the slowest rank's time decides)."""
    import torch

    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, nodes_per_rank, steps, max_ms):
    """Node updates of all ranks (one independent workload copy each) per
    second of the slowest rank, in MLUPS."""
    return world * nodes_per_rank * steps / (max_ms * 1e-3) / 1e6


def measure_lref(lbm, stream, name, storage, every, steps, warmup, hbm, hbm_src):
    """Throughput of a single lattice stored at a per-node reference
    (lbm_set_local_reference): CUDA events around every lbm_step, the
    rebuilds (every `every` steps) inside; the roofline of the step kernel
    with its algorithmic bytes (the 16-bit populations read and written plus
    the FP32 reference of every node read once)."""
    import torch

    w = WORKLOADS[name][1]()[0]
    codes = {"fp16": lbm.FP16_DEV, "bf16": lbm.BF16_DEV}
    G = lbm.from_workload(w, stream=stream.cuda_stream, storage=codes[storage], envelope_steps=warmup + steps + 8)
    try:
        G.set_local_reference(every)
        for _ in range(warmup):
            G.step(1)
        torch_sync(stream)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record(stream)
        for k in range(steps):
            G.step(1)
            evs[k + 1].record(stream)
        torch_sync(stream)
        ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    finally:
        G.close()
    q = {W.D2Q9: 9, W.D2Q5: 5}[w.lattice]
    nref = 3 if w.lattice == W.D2Q9 else 1
    per_node = 2 * 2 * q + 4 * nref
    rebuild = [m for k, m in enumerate(ms) if (warmup + k + 1) % every == 0]
    plain = sorted(m for k, m in enumerate(ms) if (warmup + k + 1) % every != 0)
    step_ms = plain[len(plain) // 2] if plain else float("nan")
    total = sum(ms)
    gbs = per_node * w.nodes / (step_ms * 1e-3) / 1e9
    return {"mlups": w.nodes * steps / (total * 1e-3) / 1e6, "ms_per_step": total / steps, "steps": steps,
            "nodes": w.nodes, "every": every,
            "step_kernel": {"ms": step_ms, "mlups": w.nodes / (step_ms * 1e-3) / 1e6,
                            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                         "frac": gbs / hbm, "traffic": None, "bytes_per_node": per_node,
                                         "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"}},
            "rebuild_ms": (sum(rebuild) / len(rebuild)) if rebuild else None,
            "timing": "CUDA events around every lbm_step; mlups over all steps (rebuild steps included), "
                      "the step kernel's rate from the median step without a rebuild",
            "workload": WORKLOADS[name][0]}


def extras(lbm, stream, hbm, hbm_src, peak):
    """Per-lattice and per-storage sub-results of the metric (each its own
    lattices, created, timed and freed in turn)."""
    out = {}
    t0 = time.perf_counter()
    try:
        out["storages"] = storage_study(lbm, stream, hbm, hbm_src, peak, steps=20, warmup=3)
    except Exception as exc:  # pragma: no cover - reported, not hidden
        out["storages"] = {"error": repr(exc)}
    wk = {}
    plan = [("kolmogorov256", "fp64", 20, {}), ("kolmogorov256", "fp32", 20, {}),
            ("channel2048", "fp64", 50, {}), ("channel2048", "fp32", 50, {}),
            ("channel8192", "fp32", 20, {}), ("channel8192", "fp16", 20, {}), ("channel8192", "bf16", 20, {}),
            ("cde8192", "fp64", 20, {}), ("cde8192", "fp32", 20, {}), ("cde8192", "fp16", 20, {}),
            ("cde_sweep", "fp64", 100, {}), ("cde_sweep", "fp32", 100, {}),
            ("batched_sweep", "fp32", 20, {"graph": 10, "tune": True})]
    for name, st, steps, kw in plan:
        key = f"{name}_{st}"
        try:
            res, _ = measure(lbm, stream, name, st, steps, 5, hbm, hbm_src, peak, **kw)
            res["workload"] = WORKLOADS[name][0]
            wk[key] = res
        except Exception as exc:  # pragma: no cover - reported, not hidden
            wk[key] = {"error": repr(exc)}
    for name, st, every in (("channel8192", "fp16", 32), ("cde8192", "fp16", 16)):
        key = f"{name}_{st}_lref"
        try:
            wk[key] = measure_lref(lbm, stream, name, st, every, 40, 5, hbm, hbm_src)
        except Exception as exc:  # pragma: no cover - reported, not hidden
            wk[key] = {"error": repr(exc)}
    out["workloads"] = wk
    try:
        out["time_to_solution"] = time_to_solution(lbm, stream)
    except Exception as exc:  # pragma: no cover - reported, not hidden
        out["time_to_solution"] = {"error": repr(exc)}
    try:
        out["time_to_solution"]["batched_sweep_subset"] = batched_time_to_solution(lbm, stream)
    except Exception as exc:  # pragma: no cover - reported, not hidden
        out["time_to_solution"]["batched_sweep_subset"] = {"error": repr(exc)}
    out["extras_seconds"] = time.perf_counter() - t0
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--storage", default=None, choices=["fp64", "fp32", "fp16", "bf16"],
                    help="population storage: fp64, or fp32/fp16/bf16 deviations with FP32 arithmetic "
                         "(default: fp64; fp32 for batched_sweep)")
    ap.add_argument("--graph", type=int, default=None,
                    help="steps per CUDA-graph replay in the timed region (even; 0 = plain launches; "
                         "default 0, 10 for batched_sweep)")
    ap.add_argument("--chunk", type=int, default=1,
                    help="steps per lbm_batch_step call in the timed region without graphs (a one-member "
                         "batch of a small FP64 D2Q9 lattice then runs them in one cluster launch)")
    ap.add_argument("--tune", type=int, default=None, choices=[0, 1],
                    help="autotune the batch tiling before the warm-up (default 1 for batched workloads)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the per-lattice / per-storage sub-results and the time-to-solution runs")
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-solution runs")
    ap.add_argument("--warmstart", action="store_true",
                    help="run the learned warm-start study (duct sections) instead of the throughput bench")
    ap.add_argument("--ws-n", type=int, default=128, help="warm-start study: duct section n x n")
    ap.add_argument("--ws-train", type=int, default=200, help="warm-start study: training fields")
    ap.add_argument("--ws-test", type=int, default=4, help="warm-start study: held-out cases")
    ap.add_argument("--profile", action="store_true",
                    help="short run for a profiler: no minimum warm-up time, no e2e, no CPU baseline, no extras")
    args = ap.parse_args()
    dflt = WORKLOAD_DEFAULTS.get(args.workload, {})
    if args.storage is None:
        args.storage = dflt.get("storage", "fp64")
    if args.graph is None:
        args.graph = dflt.get("graph", 0)
    if args.tune is None:
        args.tune = int(dflt.get("tune", False))
    if args.graph and (args.graph % 2 or args.steps % args.graph):
        args.graph = 0  # graph replays must tile the timed steps exactly
    if args.profile:
        args.no_cpu_baseline = True
        args.no_extras = True
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    from paper_1806_10247_gb300 import lbm

    torch.cuda.set_device(local)
    if args.warmstart:
        from paper_1806_10247_gb300 import surrogate

        res = surrogate.study(n=args.ws_n, train_count=args.ws_train, test_count=args.ws_test, gen_tol=1e-6,
                              check_every=500 if args.ws_n >= 96 else 100)
        if rank == 0:
            print(json.dumps({"metric": "steps and wall time to the 1e-10 residual, warm vs zero start",
                              "config": {"workload": f"duct_section_warmstart_d3q27_{args.ws_n}x{args.ws_n}"},
                              "result": res}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    hbm, hbm_src = load_peaks()
    stream = torch.cuda.Stream()
    info = lbm.device_info(local)
    peak = None
    try:
        peak = fp64_peak(lbm, stream, info)
    except Exception as exc:  # pragma: no cover - reported, not hidden
        peak = None
        peak_err = repr(exc)

    wname, make, _ = WORKLOADS[args.workload]
    wl = make()
    nodes = sum(w.nodes for w in wl)
    unit = args.graph if args.graph else max(1, args.chunk)
    if args.steps % unit:
        raise SystemExit(f"--steps must be a multiple of {unit}")
    e2e_steps = 10 if nodes > 10_000_000 else max(3, min(args.steps, 50))
    R = Run(lbm, stream, wl, args.storage, env_steps=args.warmup + args.steps + 10 * e2e_steps + 2100,
            graph=args.graph, tune=bool(args.tune))

    sampler = ClockSampler(local)
    sampler.start()
    # warm-up: at least W steps and at least ~1 s of GPU work so that the
    # clock sampler sees the GPU under load
    R.warm(args.warmup, unit, 0.0 if args.profile else 1.0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = R.launches()
    per_batch_ms = R.timed(args.steps, unit)
    launches = R.launches() - l0
    total_ms = sum(per_batch_ms)
    if dist:
        total_ms = max_over_ranks(total_ms, dist, "cuda")
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()

    value = whole_job_mlups(world, nodes, args.steps, total_ms)

    # roofline of the dominant kernel: the batch that takes the most time
    dom = max(range(len(R.batches)), key=lambda i: per_batch_ms[i])
    nb = sum(w.nodes for w in R.gwl[dom])
    kname = Q_NAME[R.kinds[dom]]
    tkey = None if len(R.gwl[dom]) == 1 else \
        (("d2q5_sweep" if args.workload == "cde_sweep" else f"{kname}_batch"), args.storage)
    roof = roofline_block(kname, args.storage, nb, per_batch_ms[dom] / args.steps * 1e-3, hbm, hbm_src, peak, tkey,
                          label=f"{kname} {'batched ' if len(R.gwl[dom]) > 1 else ''}step kernel ({nb} nodes)")
    roof["timing"] = ("CUDA events around each step's launch" + (f" (graph replays of {unit} steps)" if args.graph
                                                                 else (f" ({unit} steps per call)" if unit > 1 else "")))
    if len(R.batches) > 1:
        roof["all_kernels"] = [{"lattice": Q_NAME[k], "nodes": sum(w.nodes for w in g),
                                "us_per_launch": ms / args.steps * 1e3,
                                "GB/s": sum(w.nodes for w in g) * 2 * R.elem * Q_OF[k] / (ms / args.steps * 1e-3) / 1e9}
                               for k, g, ms in zip(R.kinds, R.gwl, per_batch_ms)]

    # launch-mode comparison for many-lattice workloads
    modes = None
    if len(wl) > 32 and not args.profile:
        modes = {"timed": {"mlups": value, "graph_steps": args.graph, "tuned": bool(args.tune)}}
        for b in R.batches:
            b.set_graph(0)
        pm = 4
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(pm):
            for b in R.batches:
                b.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        modes["batched_plain_launches"] = {"mlups": nodes * pm / (e0.elapsed_time(e1) * 1e-3) / 1e6, "steps": pm}
        e0.record(stream)
        for _ in range(pm):
            for L in R.lats:
                L.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        modes["per_instance_launches"] = {"mlups": nodes * pm / (e0.elapsed_time(e1) * 1e-3) / 1e6, "steps": pm,
                                          "launches_per_step": len(R.lats)}

    e2e = None
    try:
        if args.profile:
            raise RuntimeError("skipped in --profile runs")
        e2e = measure_e2e(R, e2e_steps, args.storage)
    except Exception as exc:  # pragma: no cover - reported, not hidden
        e2e = {"value": None, "error": repr(exc)}
    tuning = R.tuning
    R.close()
    del R
    torch.cuda.empty_cache()

    ext = None
    if not args.no_extras and rank == 0:
        ext = extras(lbm, stream, hbm, hbm_src, peak) if args.workload == DEFAULT_WORKLOAD else None
        if ext is None and not args.no_tts and args.workload == "cde_sweep":
            try:
                ext = {"time_to_solution": time_to_solution(lbm, stream)}
            except Exception as exc:  # pragma: no cover - reported, not hidden
                ext = {"time_to_solution": {"error": repr(exc)}}
        if ext is not None and args.no_tts:
            ext.pop("time_to_solution", None)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baselines(args.workload, wl if len(wl) > 1 or nodes < 5_000_000 else None,
                                args.cpu_budget, 10.0)
        except Exception as exc:  # pragma: no cover - reported, not hidden
            cpu = {"error": repr(exc)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.storage == "fp64" else "f32",
            "data": "synthetic",
            "config": config_block(wl, wname, args.storage, ELEM[args.storage], name=args.workload),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "device": {k: info[k] for k in ("sm_count", "sm_max_khz", "l2_bytes", "cc_major", "cc_minor")},
            "fp64_peak": peak if peak is not None else {"error": peak_err},
        }
        if tuning is not None:
            line["config"]["autotuned_tiling"] = tuning
        if args.graph:
            line["config"]["graph_steps"] = args.graph
        if modes is not None:
            line["launch_modes"] = modes
        if ext:
            line.update(ext)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

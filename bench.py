"""Benchmark of the cascaded LB hot path on GB300.

Default workload: the scalar-transport refinement sweep — five periodic
D2Q5 lattices 32^2, 64^2, 128^2, 256^2, 512^2 with the manufactured source
A sin(2 pi x/L) sin(2 pi y/L) e^{-lambda t}, seeded D and A, advecting
velocity (0.01, 0.01) scaled by 32/N, FP64.  One bench step advances every
lattice of the sweep by one time step (one fused stream+collide kernel each).
The inputs are smaller than L2, so L2 is flushed (a 256 MB write) before every
timed step; each step is timed with CUDA events on the library's stream.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the same workload instead.
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

# Per (workload, storage): FP64 work per node of the step kernel and its DRAM
# traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum), from the
# ncu captures summarised under profiles/.  FP64 counts are thread-level
# instructions from ncu's per-opcode table (DFMA, DADD, DMUL); flops count an
# FMA as two.  The traffic is reported only while the kernel sources still hash
# to the value it was measured on.
_H = ["paper_1806_10247_gb300/csrc/lbm_lattices.cuh", "paper_1806_10247_gb300/csrc/lbm_internal.h",
      "paper_1806_10247_gb300/csrc/lbm_device.cuh"]
KERNEL_FACTS = {
    ("cde_sweep", "fp64"): {
        "src": ["paper_1806_10247_gb300/csrc/k_d2q5.cu"] + _H,
        "fp64_inst_per_node": 38, "fp64_flops_per_node": 48,
        "traffic_bytes_per_launch": 14.002176e6, "traffic_src_sha": "5fe048d974140251",
        "profile": "profiles/k_batch_d2q5_cde_sweep_fp64.md",
    },
    ("kolmogorov96", "fp64"): {
        "src": ["paper_1806_10247_gb300/csrc/k_d3q27.cu"] + _H,
        "fp64_inst_per_node": 426, "fp64_flops_per_node": 621,
        "traffic_bytes_per_launch": (191.174144 + 142.945536) * 1e6, "traffic_src_sha": "890a81d687f85b7f",
        "profile": "profiles/k_batch_d3q27_kolmogorov96_fp64.md",
    },
    ("channel2048", "fp64"): {
        "src": ["paper_1806_10247_gb300/csrc/k_d2q9.cu"] + _H,
        "fp64_inst_per_node": 134, "fp64_flops_per_node": 171,
        "traffic_bytes_per_launch": (151.023616 + 105.353728) * 1e6, "traffic_src_sha": "bf2bab403965bd53",
        "profile": "profiles/k_batch_d2q9_channel2048_fp64.md",
    },
    ("kolmogorov96", "fp32"): {
        "src": ["paper_1806_10247_gb300/csrc/k_rp.cu"] + _H,
        "traffic_bytes_per_launch": (95.602176 + 51.792128) * 1e6, "traffic_src_sha": "104107b6e5fb10f7",
        "profile": "profiles/k_batch27_kolmogorov96_fp32_fp16.md",
    },
    ("kolmogorov96", "fp16"): {
        "src": ["paper_1806_10247_gb300/csrc/k_rp.cu"] + _H,
        "traffic_bytes_per_launch": (47.818496 + 8.367872) * 1e6, "traffic_src_sha": "104107b6e5fb10f7",
        "profile": "profiles/k_batch27_kolmogorov96_fp32_fp16.md",
    },
    ("channel2048", "fp32"): {
        "src": ["paper_1806_10247_gb300/csrc/k_rp.cu"] + _H,
        "traffic_bytes_per_launch": (75.518976 + 31.702016) * 1e6, "traffic_src_sha": "104107b6e5fb10f7",
        "profile": "profiles/k_batch9_channel2048_fp32.md",
    },
}
# The same FP64 kernels run the 256^3 / 512^3 Kolmogorov workloads.
for _w in ("kolmogorov256", "kolmogorov512"):
    KERNEL_FACTS[(_w, "fp64")] = {k: v for k, v in KERNEL_FACTS[("kolmogorov96", "fp64")].items()
                                  if k != "traffic_bytes_per_launch"}
# FP64 pipe of the GB300: 2 FMA lanes per clock per SM (the recipe's 1.25 TFLOP/s
# divided by 2 flop x 152 SMs x 2.07 GHz), 152 SMs, 2.07 GHz maximum SM clock.
FP64_LANES_PER_SM, N_SMS, SM_GHZ = 2, 152, 2.07
FP64_PEAK_GINST = FP64_LANES_PER_SM * N_SMS * SM_GHZ          # 629.3 G FP64 instructions/s
FP64_PEAK_TFLOPS = 2 * FP64_PEAK_GINST / 1e3                  # 1.259 TFLOP/s
FP64_PEAK_NOTE = "derived: 2 FP64 FMA lanes/clk/SM x 152 SMs x 2.07 GHz x 2 flop"


def src_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def sweep_workloads():
    return [W.cde_workload(c) for c in W.cde_sweep_params()]


WORKLOADS = {
    "cde_sweep": ("cde_d2q5_refinement_sweep_fp64", sweep_workloads),
    "poiseuille": ("poiseuille_d2q9_3x33_fp64", lambda: [W.poiseuille()]),
    "kolmogorov256": ("kolmogorov_d3q27_256cubed_fp64", lambda: [W.kolmogorov(n=256)]),
    "kolmogorov512": ("kolmogorov_d3q27_512cubed_fp64", lambda: [W.kolmogorov(n=512)]),
    "duct128": ("duct_d3q27_128x128x128_fp64", lambda: [W.duct(n=128, nx=128)]),
    "kolmogorov96": ("kolmogorov_d3q27_96cubed_fp64", lambda: [W.kolmogorov(n=96)]),
    "channel2048": ("channel_d2q9_2048x1024_fp64", lambda: [W.poiseuille(ny=1024, nx=2048)]),
}
Q_OF = {W.D2Q9: 9, W.D2Q5: 5, W.D3Q27: 27}
L2_BYTES = 129 * 1024 * 1024


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

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        out = os.environ.get("LBM_RESULTS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_bench_{os.getpid()}.csv")

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
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[2]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def time_oracle(workloads, steps, budget_s=None):
    """Run the FP64 CPU oracle on every lattice of the workload for `steps`
    steps (or until ~budget_s seconds).  Returns (node updates, seconds, threads)."""
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
    nodes = sum(w.nodes for w in workloads)
    done = 0
    t0 = time.perf_counter()
    while True:
        for R in lats:
            R.run(1)
        done += 1
        el = time.perf_counter() - t0
        if (budget_s is None and done >= steps) or (budget_s is not None and el >= budget_s):
            break
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return nodes * done, time.perf_counter() - t0, threads, done


def run_reference(args, world, rank):
    if rank != 0:
        return
    wname, make = WORKLOADS[args.workload]
    wl = make()
    from oracle import oracle as O

    O.build()
    time_oracle(wl, args.warmup)
    upd, sec, threads, done = time_oracle(wl, args.steps)
    v = upd / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / done * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block(wl, wname),
        "cpu_baseline": {"kind": "oracle", "value": v, "unit": "MLUPS", "cores": threads,
                         "sample": f"{done} steps of the whole sweep ({upd} node updates)"},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def state_bytes(wl, elem=8):
    return sum(2 * elem * Q_OF[w.lattice] * w.nodes for w in wl)


def config_block(wl, name, storage="fp64", elem=8):
    c = {"workload": name, "storage": storage, "lattices": [w.name for w in wl], "nodes_per_step": sum(w.nodes for w in wl),
         "seed": W.SEED, "launch": "one batched fused stream+collide kernel per time step",
         "parallelism": "replicas (one independent copy of the workload per GPU)"}
    if state_bytes(wl, elem) < 2 * L2_BYTES:
        c["l2"] = "flushed before every timed step (256 MB write); the state fits in L2"
    else:
        c["l2"] = "state larger than L2 (no flush needed)"
    if wl[0].lattice == W.D2Q5:
        c["D"] = wl[0].meta["D"]
        c["A32"] = wl[0].meta["A"]
    return c


def time_to_solution(lbm, stream, storages=("fp64", "fp32")):
    """The metric's second half: wall time to the solution criterion.
    * config 1 (Poiseuille D2Q9 3 x 33): steps until max |u(t) - u(t-100)| < 1e-12
      (checked every 100 steps with lbm_reduce), and the l2 error of the final
      profile against the parabola of Sec. 6.1;
    * config 2 (scalar sweep): every member run to its T_N, l2 error against the
      closed form and the convergence order over the sweep."""
    codes = {"fp64": lbm.FP64, "fp32": lbm.FP32_DEV}
    out = {}
    for st in storages:
        w = W.poiseuille()
        L = lbm.from_workload(w, stream=stream.cuda_stream, storage=codes[st])
        G = lbm.Batch([L])
        G.set_graph(100)  # 100 steps per CUDA-graph replay between the checks
        L.reduce()
        torch_sync(stream)
        t0 = time.perf_counter()
        steps, du = 0, float("inf")
        while steps < 200000:
            G.step(100)
            steps += 100
            du = L.reduce()[4]
            if du < 1e-12:
                break
        sec = time.perf_counter() - t0
        _, u = L.moments()
        ua = np.tile(W.poiseuille_parabola(w.shape[1], w.meta["tau"], w.meta["Fx"])[:, None], (1, w.shape[0]))
        l2 = float(np.sqrt(np.sum((u[0] - ua.reshape(-1)) ** 2) / np.sum(ua ** 2)))
        out[f"poiseuille_{st}"] = {"steps": steps, "seconds": sec, "max_du": du, "l2_vs_parabola": l2,
                                   "criterion": "max |u(t) - u(t-100)| < 1e-12",
                                   "launch": "CUDA graph of 100 steps between lbm_reduce checks"}
        G.close()
        L.close()
        cases = W.cde_sweep_params()
        errs, total = [], 0.0
        for c in cases:
            wc = W.cde_workload(c)
            G = lbm.from_workload(wc, stream=stream.cuda_stream, envelope_steps=c.T + 2, storage=codes[st])
            Bt = lbm.Batch([G])
            Bt.set_graph(200)
            torch_sync(stream)
            t0 = time.perf_counter()
            Bt.step(c.T)
            G.sync()
            total += time.perf_counter() - t0
            phi = G.moments().reshape(c.N, c.N) - 1.0
            ref = W.cde_closed_form(c, c.T)
            errs.append(float(np.sqrt(np.sum((phi - ref) ** 2) / np.sum(ref ** 2))))
            Bt.close()
            G.close()
        orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
        out[f"cde_sweep_{st}"] = {"seconds": total, "steps": [c.T for c in cases],
                                  "l2_vs_closed_form": errs, "orders": orders}
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


def torch_sync(stream):
    stream.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cde_sweep", choices=sorted(WORKLOADS))
    ap.add_argument("--storage", default="fp64", choices=["fp64", "fp32", "fp16", "bf16"],
                    help="population storage: fp64, or fp32/fp16/bf16 deviations with FP32 arithmetic")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-tts", action="store_true", help="skip the time-to-solution runs")
    ap.add_argument("--warmstart", action="store_true",
                    help="run the learned warm-start study (duct sections) instead of the throughput bench")
    ap.add_argument("--profile", action="store_true",
                    help="short run for a profiler: no minimum warm-up time, no e2e, no CPU baseline")
    args = ap.parse_args()
    if args.profile:
        args.no_cpu_baseline = True
        args.no_tts = True
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

        res = surrogate.study()
        if rank == 0:
            print(json.dumps({"metric": "steps and wall time to the 1e-10 residual, warm vs zero start",
                              "config": {"workload": "duct_section_warmstart_d3q27"}, "result": res}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wname, make = WORKLOADS[args.workload]
    wl = make()
    need_flush = True  # refined below once the storage size is known
    stream = torch.cuda.Stream()
    e2e_steps = max(3, min(args.steps, 50))
    env_steps = args.warmup + args.steps + e2e_steps + 20000  # envelope tables cover every step run here
    storage = {"fp64": lbm.FP64, "fp32": lbm.FP32_DEV, "fp16": lbm.FP16_DEV, "bf16": lbm.BF16_DEV}[args.storage]
    elem = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[args.storage]
    lats = [lbm.from_workload(w, stream=stream.cuda_stream, envelope_steps=env_steps, storage=storage) for w in wl]
    batch = lbm.Batch(lats)  # one fused step kernel for all lattices of the sweep per time step
    need_flush = state_bytes(wl, elem) < 2 * L2_BYTES
    nodes = sum(w.nodes for w in wl)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    sampler = ClockSampler(local)
    sampler.start()
    # warm-up: at least W steps and at least ~1 s of GPU work so that the
    # clock sampler sees the GPU under load
    t0 = time.perf_counter()
    k = 0
    min_warm_s = 0.0 if args.profile else 1.0
    while k < args.warmup or (time.perf_counter() - t0 < min_warm_s and k < env_steps - args.steps - e2e_steps - 5):
        if need_flush:
            with torch.cuda.stream(stream):
                flush.zero_()
        batch.step(1)
        k += 1
        if k % 50 == 0:
            stream.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = batch.launch_count() + sum(L.launch_count() for L in lats)
    for s in range(args.steps):
        if need_flush:
            with torch.cuda.stream(stream):
                flush.zero_()
        ev[s][0].record(stream)
        batch.step(1)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    launches = batch.launch_count() + sum(L.launch_count() for L in lats) - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kern_ms = step_ms  # one launch per step: the batched D2Q5 step kernel
    total_ms = sum(step_ms)
    if dist:
        total_ms = max_over_ranks(total_ms, dist, "cuda")
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()

    value = whole_job_mlups(world, nodes, args.steps, total_ms)

    # roofline of the dominant (only) kernel: the batched D2Q5 step over the sweep
    hbm, hbm_src = load_peaks()
    kavg_s = statistics.mean(kern_ms) * 1e-3
    nb = nodes
    q = Q_OF[wl[0].lattice]
    alg_bytes = nb * 2 * elem * q  # q populations read + q written
    achieved_gbs = alg_bytes / kavg_s / 1e9
    facts = KERNEL_FACTS.get((args.workload, args.storage), {})
    traffic = None
    if facts.get("traffic_bytes_per_launch") is not None and facts["traffic_src_sha"] == src_hash(facts["src"]):
        traffic = facts["traffic_bytes_per_launch"]
    roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
            "frac": achieved_gbs / hbm, "traffic": traffic, "kernel": f"batched step kernel ({wname})",
            "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else "fallback",
            "bytes_per_node": 2 * elem * q, "kernel_us": kavg_s * 1e6}
    if facts.get("fp64_flops_per_node"):
        tf = facts["fp64_flops_per_node"] * nb / kavg_s / 1e12
        gi = facts["fp64_inst_per_node"] * nb / kavg_s / 1e9
        pipe = {"achieved": gi, "peak": FP64_PEAK_GINST, "unit": "G FP64 instr/s", "frac": gi / FP64_PEAK_GINST,
                "inst_per_node": facts["fp64_inst_per_node"]}
        if tf / FP64_PEAK_TFLOPS > roof["frac"]:
            roof.update({"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tf / FP64_PEAK_TFLOPS, "flops_per_node": facts["fp64_flops_per_node"],
                         "peak_source": FP64_PEAK_NOTE, "fp64_pipe": pipe,
                         "hbm": {"achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm}})
    if facts.get("profile"):
        roof["profile"] = facts["profile"]

    # end to end through the public API with host buffers: per step and lattice,
    # upload the step's source field from pinned host memory (lbm_set_source),
    # one lbm_step, and read phi back to pinned host memory (lbm_moments).
    e2e = None
    try:
        if args.profile:
            raise RuntimeError("skipped in --profile runs")
        pinned_src = []
        pinned_phi = []
        for w in wl:
            from_tables = [((np.asarray(px)[None, None, :] * np.asarray(py)[None, :, None]) * np.asarray(pz)[:, None, None])
                           for px, py, pz in w.tables]
            full = np.ascontiguousarray(np.stack([np.broadcast_to(t, w.shape[::-1]).reshape(-1) for t in from_tables]))
            t_src = torch.empty(full.shape, dtype=torch.float64, pin_memory=True)
            t_src.numpy()[:] = full
            pinned_src.append(t_src)
            pinned_phi.append(torch.empty(w.nodes * (1 if w.lattice == W.D2Q5 else 4), dtype=torch.float64,
                                          pin_memory=True))
        ke = e2e_steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            for L, s_ in zip(lats, pinned_src):
                if L.lattice == lbm.D2Q5_CDE:
                    L.set_source(full=s_.numpy())
                else:
                    L.set_force(full=s_.numpy())
            batch.step(1)
            for L, p_ in zip(lats, pinned_phi):
                L._check(L._L.lbm_moments(L.h, p_.data_ptr(), None, 0, 1))
        el = time.perf_counter() - t0
        ncomp = 1 if wl[0].lattice == W.D2Q5 else (3 if wl[0].lattice == W.D3Q27 else 2)
        nout = 1 if wl[0].lattice == W.D2Q5 else 1 + ncomp
        e2e = {"value": nodes * ke / el / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": nodes * 8 * ncomp,
               "d2h_bytes_per_step": nodes * 8 * nout, "steps": ke,
               "path": "per step: lbm_set_source/lbm_set_force(host, full field) per lattice, lbm_batch_step(1), "
                       "lbm_moments(host) per lattice"}
    except Exception as exc:  # pragma: no cover - reported, not hidden
        e2e = {"value": None, "error": repr(exc)}

    tts = None
    if not args.no_tts and args.workload == "cde_sweep":
        try:
            tts = time_to_solution(lbm, stream)
        except Exception as exc:  # pragma: no cover - reported, not hidden
            tts = {"error": repr(exc)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and state_bytes(wl) < (1 << 30):  # FP64 oracle
        upd, sec, threads, done = time_oracle(wl, None, budget_s=args.cpu_budget)
        cpu = {"value": upd / sec / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": f"{done} steps of the whole sweep ({upd} node updates, {sec:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.storage == "fp64" else "f32",
            "data": "synthetic", "config": config_block(wl, wname, args.storage, elem), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "time_to_solution": tts,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

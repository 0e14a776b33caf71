#!/usr/bin/env python3
"""Benchmark: SU(3) Landau gauge fixing by steepest descent with Fourier
acceleration on GB300, in site-iterations per second.

Workload (default): one 32^4 configuration (links of scale 0.5 behind a random
gauge of scale 1.0, seed 0), FP32 links (18 reals, structure of arrays) with
FP64 F/theta sums, alpha = 0.08.  A step is one full iteration of the method
(gradient, F/theta reduction, forward 4D FFT, p2_max/p2 scaling, inverse FFT,
gauge step g, and the update, applied to the accumulated gauge transformation
G <- g G with the links formed on the fly by the next gradient); ``value`` =
lattice sites x timed steps / device time.  Then the same configuration is
fixed to theta < 1e-15 (FP32 phase + an FP64-accurate double-float tail):
``time_to_theta``.  ``e2e`` repeats the
fix through the public API from pinned host links, with the host<->device
copies inside the timed region.

On one GPU the default run adds the metric's comparison arms under ``arms``
(``--arms`` selects them): the same 32^4 input fixed by the plain FP64
method (site-iterations/s, time to theta < 1e-15 and its ratio to the mixed
path), the FP32 step with g reunitarised in FP64, the 48^3 x 8 and 48^3 x 12
12-real lattices with per-kernel GB/s, the 64-lattice mixed batch, the
learned warm start (trained on the GPU, then iterations and time to theta
with and without it), and the oracle on all host cores and on one
(``nproc``/``lscpu`` recorded).  ``cpu_baseline`` is the oracle on all host
cores on the headline input.

--impl reference times the CPU oracle (numpy FP64, naive DFT) instead.
One JSON line on stdout (rank 0).
"""
from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "site-iterations/s"
WORKLOADS = {
    "32^4-f32": dict(dims=(32, 32, 32, 32), dtype="f32", link_scale=0.5, gauge_scale=1.0, seed=0, alpha=0.08,
                     tol=1e-15, max_iter=5000,
                     desc="32^4 single config, FP32 links (18 reals, SoA), FP64 F/theta sums, FP64 tail to "
                          "theta<1e-15, link scale 0.5, gauge scale 1.0, alpha 0.08"),
    "48^3x8-f32r12": dict(dims=(48, 48, 48, 8), dtype="f32_r12", link_scale=0.6, gauge_scale=1.0, seed=0,
                          alpha=0.08, tol=1e-15, max_iter=5000,
                          desc="48^3x8 single config, FP32 12-real links, FP64 tail to theta<1e-15, "
                               "link scale 0.6"),
    "8^4-f64": dict(dims=(8, 8, 8, 8), dtype="f64", link_scale=0.3, gauge_scale=1.0, seed=0, alpha=0.08,
                    tol=1e-12, max_iter=2000,
                    desc="8^4 single config, plain FP64, theta<1e-12, link scale 0.3"),
}
# Batched workload: 64 lattices of four shapes, config i has seed i and shape
# BATCH_SHAPES[i % 4]; all fixed together (lgf_batch) from CUDA graphs.
BATCH_SHAPES = [(16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 8), (20, 20, 20, 20)]
WORKLOADS["batch64-f32"] = dict(
    batch=64, dtype="f32", link_scale=0.5, gauge_scale=1.0, seed=0, alpha=0.08, tol=1e-15, max_iter=5000,
    desc="64 configs (16 each of 16^4, 24^3x48, 32^3x8, 20^4; seeds 0..63) fixed together from CUDA graphs, "
         "FP32 + FP64 tail to theta<1e-15, link scale 0.5, FFT pipeline autotuned per shape")
WORKLOADS["warmstart-f32"] = dict(
    warm=True, dtype="f32", link_scale=0.5, gauge_scale=1.0, alpha=0.08, tol=1e-15, max_iter=5000,
    train_dims=(16, 16, 16, 16), train_n=2000, train_seed=1000, epochs=1, lr=1e-5,
    eval_dims=(24, 24, 24, 24), eval_n=8, eval_seed=5000,
    desc="learned warm start: 4D conv net (3 layers, 32 channels, 3^4 taps, BF16 weights, FP32 accumulation) "
         "trained on 16^4 configs (maximising F of the warm-started links), evaluated on 24^4 configs: "
         "iterations and time to theta<1e-15 with and without the warm start")
DEFAULT_WORKLOAD = "32^4-f32"
KERNEL_SOURCES = {"update": "k_links.cu", "gradient": "k_links.cu", "build_g": "k_links.cu",
                  "accumulate": "k_links.cu", "fft_xy": "k_fft_plane.cu", "fft_zt": "k_fft_zt.cu",
                  "fft_axis": "k_fft_axis.cu", "fft_t": "k_fft_axis.cu", "xy_gstep": "k_fft_plane.cu"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# algorithmic bytes per site of each kernel (unique HBM bytes a launch must
# move: neighbour links and neighbour g count once, via the caches)
# ---------------------------------------------------------------------------
def bytes_per_site(kernel: str, prec: int, r: int, gauge_rep: bool = False) -> float:
    if gauge_rep:  # links U0 fixed, gauge G updated: see k_gauge_rep.cu
        table = {
            "gradient": 5 * r + 8,   # own U0 links and own G in, packed gradient out
            "build_g": 8 + 2 * r,    # packed gradient in, G in and out (g never stored)
            "xy_gstep": 8 + 2 * r,   # packed gradient in (inverse x-y FFT in shared memory), G in and out
        }
        if kernel in table:
            return table[kernel] * prec
    table = {
        "gradient": 4 * r + 8,   # own links in, packed gradient out
        "fft_xy": 16,            # 4 complex in, 4 complex out
        "fft_zt": 16,
        "fft_axis": 16,          # one axis pass: 4 complex in, 4 complex out
        "fft_t": 17,             # t pass: the same plus the acceleration factor
        "build_g": 8 + r,        # packed gradient in, g out
        "update": 9 * r,         # links in and out, g in
        "accumulate": 3 * r,     # g in, G in and out
    }
    return table.get(kernel, 0) * prec


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.path = tempfile.mktemp(prefix="lgf_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", gpu_id], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception as e:  # nvidia-smi missing
            log("clock sampling unavailable:", e)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, t0: float, t1: float):
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    ts = _dt.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(p[1]), float(p[2]), p[5:9]))
                except ValueError:
                    continue
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        inside = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15]
        note = None
        if not inside:
            inside = rows
            note = "timed region shorter than the 100 ms sampling period: samples from the whole run"
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        out = {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
               "reasons": reasons, "samples": len(inside)}
        if note:
            out["note"] = note
        return out


def gpu_id_for_smi(torch) -> str:
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        return vis or "0"


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
_ORACLE_CHILD = r"""
import os, sys, time, json
sys.path.insert(0, sys.argv[1])
import numpy as np
from oracle import lgf_oracle as O
U = np.load(sys.argv[2])
mode = sys.argv[3]; n = int(sys.argv[4]); alpha = float(sys.argv[5])
t = time.perf_counter()
if mode == "iterate":
    O.iterate(U, n, alpha)
    out = {"iterations": n}
else:
    r = O.fix(U, float(sys.argv[6]), n, alpha)
    out = {"iterations": r["iterations"], "F": r["F"], "theta": r["theta"], "converged": bool(r["converged"])}
out["seconds"] = time.perf_counter() - t
print(json.dumps(out))
"""


def thread_env(threads: int) -> dict:
    t = str(int(threads))
    return {"OMP_NUM_THREADS": t, "OPENBLAS_NUM_THREADS": t, "MKL_NUM_THREADS": t, "NUMEXPR_NUM_THREADS": t}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def host_cpu_info() -> dict:
    """nproc and the lscpu lines that name the host CPU."""
    info = {"nproc": host_cores()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            k = k.strip()
            if k in ("Architecture", "CPU(s)", "Model name", "Thread(s) per core", "Core(s) per socket",
                     "Socket(s)", "CPU max MHz"):
                info[k] = v.strip()
    except Exception as e:
        info["lscpu"] = f"unavailable: {e}"
    return info


def run_oracle(U, mode: str, n: int, alpha: float, threads: int = 1, tol: float = 0.0) -> dict:
    """The oracle as it stands on U in a child process with `threads` BLAS /
    OpenMP threads: n iterations (mode 'iterate') or a fix to theta < tol
    with at most n updates (mode 'fix')."""
    import numpy as np
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "U.npy")
        np.save(path, U)
        env = dict(os.environ, **thread_env(threads))
        r = subprocess.run([sys.executable, "-c", _ORACLE_CHILD, ROOT, path, mode, str(n), str(alpha), str(tol)],
                           capture_output=True, text=True, env=env, timeout=1800)
        if r.returncode != 0:
            raise RuntimeError("oracle child failed: " + r.stderr[-2000:])
        return json.loads(r.stdout.strip().splitlines()[-1])


def time_oracle(U, n: int, alpha: float, threads: int = 1) -> float:
    """Seconds for n oracle iterations on U (child process, `threads` threads)."""
    return run_oracle(U, "iterate", n, alpha, threads)["seconds"]


GOLDEN_FIX = os.path.join(ROOT, "tests", "golden", "fullsize_fix.json")


def oracle_fix_iterations(case: str):
    """Updates the oracle's own fix of a full-size case needs (stored by the
    committed script that calls only the oracle), or None."""
    try:
        return json.load(open(GOLDEN_FIX))["cases"][case]["iterations"]
    except Exception:
        return None


# ---------------------------------------------------------------------------
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
def include_closure(name: str) -> list:
    """The translation unit `name` and every project header it includes
    (#include "..."), transitively, in a fixed order."""
    csrc = os.path.join(ROOT, "paper_1208_1186_gb300", "csrc")
    seen, todo = [], [name]
    while todo:
        f = todo.pop(0)
        if f in seen:
            continue
        seen.append(f)
        for line in open(os.path.join(csrc, f)):
            m = re.match(r'\s*#include\s+"([^"/]+)"', line)
            if m and os.path.exists(os.path.join(csrc, m.group(1))):
                todo.append(m.group(1))
    return [seen[0]] + sorted(seen[1:])


def kernel_source_hash(kernel: str, gauge_rep: bool) -> str | None:
    """sha256 (16 hex) of the sources the kernel is compiled from: its
    translation unit and the project headers that unit includes."""
    name = "k_gauge_rep.cu" if (gauge_rep and kernel in ("gradient", "build_g")) else KERNEL_SOURCES.get(kernel)
    if name is None:
        return None
    h = hashlib.sha256()
    try:
        for f in include_closure(name):
            h.update(open(os.path.join(ROOT, "paper_1208_1186_gb300", "csrc", f), "rb").read())
    except OSError:
        return None
    return h.hexdigest()[:16]


def profile_traffic(kernel: str, workload: str, gauge_rep: bool):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (lines 'workload kernel dram_bytes_per_launch source_hash'), if it was
    taken on the current source of that kernel; else None."""
    want = kernel_source_hash(kernel, gauge_rep)
    try:
        for line in open(TRAFFIC_FILE):
            p = line.split()
            if len(p) == 4 and not line.startswith("#") and p[0] == workload and p[1] == kernel:
                return float(p[2]) if p[3] == want else None
    except OSError:
        pass
    return None


class Replicas:
    """One process per GPU under torchrun (RANK, LOCAL_RANK, WORLD_SIZE from
    the environment), each fixing its own configuration: no collective on the
    data path.  Timing across ranks: a barrier before and after each timed
    region and the maximum of the ranks' times; the reported value is the
    units all ranks processed over that maximum."""

    def __init__(self, backend: str, device):
        import torch.distributed as dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.device = device
        self._dist = dist
        if self.world > 1 and not dist.is_initialized():
            if backend == "nccl":
                dist.init_process_group(backend, device_id=device)
            else:
                dist.init_process_group(backend)

    def barrier(self):
        if self.world > 1:
            self._dist.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self._dist.all_reduce(t, op=self._dist.ReduceOp.MAX)
        return float(t.item())

    def seed(self, base: int) -> int:
        return base + self.rank

    def throughput(self, units_per_rank: float, seconds_max: float) -> float:
        return self.world * units_per_rank / seconds_max

    def close(self):
        if self.world > 1 and self._dist.is_initialized():
            self._dist.destroy_process_group()


def main_config(W, world: int, gauge_rep: bool) -> dict:
    """The `config` object of the single-lattice workloads; the reference arm
    prints the same one."""
    prec = 4 if W["dtype"].startswith("f32") else 8
    r = 12 if W["dtype"].endswith("r12") else 18
    V = 1
    for d in W["dims"]:
        V *= d
    return {"workload": W["desc"], "lattice": list(W["dims"]), "storage": W["dtype"], "alpha": W["alpha"],
            "link_update": ("gauge representation: U0 fixed, G <- g G, links formed on the fly"
                            if gauge_rep else "links updated in place"),
            "link_scale": W["link_scale"], "gauge_scale": W["gauge_scale"], "seed": W["seed"],
            "l2": f"inputs larger than L2: links {4 * r * prec * V / 1e6:.0f} MB per sweep",
            "parallelism": f"replicas x{world} (independent configs, no collective on the data path)"}


def kernel_table(prof: dict, steps: int, V: int, prec: int, r: int, gauge_rep: bool) -> dict:
    """Per-kernel launches, time, share and algorithmic GB/s from lgf_profile."""
    total = sum(v[0] for v in prof.values()) or 1.0
    out = {}
    for name, (kms, n) in prof.items():
        if n == 0 or name == "other":
            continue
        per = kms / n
        b = bytes_per_site(name, prec, r, gauge_rep) * V
        out[name] = {"launches": n, "ms_per_launch": round(per, 5), "share": round(kms / total, 4),
                     "algorithmic_gbs": round(b / (per * 1e-3) / 1e9, 1) if b else None}
    return out


def measure_handle(torch, gf, stream, Ud, W, steps: int, warmup: int, V: int, gauge_rep: bool) -> dict:
    """Site-iterations/s of `steps` iterations (CUDA events on the handle's
    stream, after `warmup`), per-kernel times from a second, profiled pass,
    and the time to theta < tol from device-resident links (after one
    untimed fix that builds the handle's loop graphs)."""
    prec = 4 if W["dtype"].startswith("f32") else 8
    r = 12 if W["dtype"].endswith("r12") else 18
    gf.load_links(Ud)
    gf.iterate(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gf.iterate(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    gf.profile(True)
    gf.iterate(steps)
    torch.cuda.synchronize()
    prof = gf.profile_read()
    gf.profile(False)
    gf.load_links(Ud)
    gf.fix(W["tol"], W["max_iter"])
    gf.load_links(Ud)
    torch.cuda.synchronize()
    e0.record(stream)
    iters, conv = gf.fix(W["tol"], W["max_iter"])
    e1.record(stream)
    torch.cuda.synchronize()
    fix_s = e0.elapsed_time(e1) / 1e3
    F, theta = gf.functional()
    return {"value": round(V * steps / (ms / 1e3), 1), "unit": METRIC, "ms_per_step": round(ms / steps, 5),
            "steps": steps, "kernels": kernel_table(prof, steps, V, prec, r, gauge_rep),
            "time_to_theta": {"theta_tol": W["tol"], "seconds": round(fix_s, 5), "iterations": iters,
                              "fp32_iterations": gf.fix_split()[0], "fp64_iterations": gf.fix_split()[1],
                              "converged": conv, "F": F, "theta": theta}}


def arm_single(lgf, torch, W, steps: int, warmup: int, params=(), Ud=None) -> dict:
    """One single-lattice workload W measured by measure_handle (its input
    generated on the GPU unless given)."""
    from lgf_inputs import torch_gen
    dims = W["dims"]
    V = 1
    for d in dims:
        V *= d
    if Ud is None:
        Ud = torch_gen.synthetic_config(dims, seed=W["seed"], link_scale=W["link_scale"],
                                        gauge_scale=W["gauge_scale"], device="cuda")
    stream = torch.cuda.Stream()
    gauge_rep = W["dtype"].startswith("f32")
    with lgf.GaugeFixer(dims, W["dtype"], stream=stream, alpha=W["alpha"]) as gf:
        for k, v in params:
            gf.set_param(k, v)
        gf.load_links(Ud)
        gf.autotune(reps=10)
        out = measure_handle(torch, gf, stream, Ud, W, steps, warmup, V, gauge_rep)
        out["fft_schedule"] = list(gf.schedule())
    out["workload"] = W["desc"]
    return out


def batch_measure(lgf, torch, W, steps: int, warmup: int, lanes_arg: int = -1, fft_tune: bool = True) -> dict:
    """The batched workload (lgf_batch): site-iterations/s over all members,
    the time to fix all of them, and the step-level roofline."""
    import numpy as np
    from lgf_inputs import torch_gen

    n = W["batch"]
    shapes = [BATCH_SHAPES[i % len(BATCH_SHAPES)] for i in range(n)]
    t = time.time()
    inputs = [torch_gen.synthetic_config(shapes[i], seed=W["seed"] + i, link_scale=W["link_scale"],
                                         gauge_scale=W["gauge_scale"], device="cuda") for i in range(n)]
    torch.cuda.synchronize()
    log(f"generated {n} configs ({sum(int(np.prod(s)) for s in shapes)} sites) on the GPU in {time.time() - t:.1f}s")
    fixers = [lgf.GaugeFixer(shapes[i], W["dtype"], alpha=W["alpha"]) for i in range(n)]
    try:
        for f, u in zip(fixers, inputs):
            f.load_links(u)
        tuned = {}
        for f, s in zip(fixers, shapes):
            if fft_tune:
                f.autotune(reps=5)
            tuned.setdefault("x".join(map(str, s)), list(f.schedule()))
        Vtot = sum(int(np.prod(s)) for s in shapes)
        with lgf.GaugeBatch(fixers) as batch:
            lanes = lanes_arg
            if lanes >= 0:
                batch.set_lanes(lanes)
            else:
                lanes = batch.autotune(reps=4)
            batch.iterate(warmup)
            torch.cuda.synchronize()
            l0 = sum(f.launch_count() for f in fixers)
            w0 = time.time()
            t0 = time.perf_counter()
            batch.iterate(steps)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            w1 = time.time()
            launches = sum(f.launch_count() for f in fixers) - l0
            for f, u in zip(fixers, inputs):
                f.load_links(u)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its, conv = batch.fix(W["tol"], W["max_iter"])
            fix_s = time.perf_counter() - t0
            thetas = [f.functional()[1] for f in fixers]
    finally:
        for f in fixers:
            f.close()
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    # gauge representation, FP32 18-real, every batch shape on the fused path:
    # gradient 392, forward x-y 64, z-t 64, inverse x-y + G update 176 bytes/site
    step_bytes = (bytes_per_site("gradient", 4, 18, True) + 2 * bytes_per_site("fft_xy", 4, 18)
                  + bytes_per_site("xy_gstep", 4, 18, True))
    value = Vtot * steps / secs
    return {"value": round(value, 1), "unit": METRIC, "ms_per_step": round(secs / steps * 1e3, 5), "steps": steps,
            "members": n, "sites": Vtot, "fft_pipeline_per_shape": tuned,
            "graph_lanes": lanes if lanes_arg >= 0 else f"{lanes} (autotuned; 0 = one per member)",
            "timing": "host wall clock around the synchronous lgf_batch_iterate: one graph launch, every member "
                      "looping on the device",
            "roofline": {"bound": "hbm", "kernel": "whole step (graph-launched; per-kernel events are not "
                                                   "recorded inside graphs)",
                         "achieved": round(step_bytes * value / 1e9, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(step_bytes * value / 1e9 / hbm_peak, 4), "traffic": None,
                         "algorithmic_bytes_per_site": step_bytes},
            "time_to_theta": {"theta_tol": W["tol"], "seconds": round(fix_s, 4), "all_converged": all(conv),
                              "iterations_min": min(its), "iterations_max": max(its),
                              "iterations_mean": round(sum(its) / len(its), 2), "theta_max": max(thetas)},
            "gpu_launches": launches, "_window": (w0, w1)}


def warm_measure(lgf, torch, W, ntr: int, profile_range: bool = False) -> dict:
    """Train the warm-start network on the GPU, then fix unseen larger
    configurations with and without it."""
    import numpy as np
    from lgf_inputs import torch_gen

    net = lgf.WarmStartNet(seed=0)
    gf = lgf.GaugeFixer(W["train_dims"], W["dtype"], alpha=W["alpha"])
    F_first, F_last = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = 0
    for ep in range(W["epochs"]):
        for k in range(ntr):
            u = torch_gen.synthetic_config(W["train_dims"], seed=W["train_seed"] + k, link_scale=W["link_scale"],
                                           gauge_scale=W["gauge_scale"], device="cuda")
            gf.load_links(u)
            F, _ = net.train_step(gf, W["lr"])
            steps += 1
            (F_first if k < 16 and ep == 0 else F_last if k >= ntr - 16 else []).append(F)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    gf.close()
    ge = lgf.GaugeFixer(W["eval_dims"], W["dtype"], alpha=W["alpha"])
    # one untimed fix first: it builds the handle's loop graphs, which both
    # timed arms then share
    ge.load_links(torch_gen.synthetic_config(W["eval_dims"], seed=W["eval_seed"] - 1, link_scale=W["link_scale"],
                                             gauge_scale=W["gauge_scale"], device="cuda"))
    ge.fix(W["tol"], W["max_iter"])
    rows = []
    for k in range(W["eval_n"]):
        u = torch_gen.synthetic_config(W["eval_dims"], seed=W["eval_seed"] + k, link_scale=W["link_scale"],
                                       gauge_scale=W["gauge_scale"], device="cuda")
        ge.load_links(u)
        F0 = ge.functional()[0]
        torch.cuda.synchronize()
        a = time.perf_counter()
        it_p, cp = ge.fix(W["tol"], W["max_iter"])
        torch.cuda.synchronize()
        tp = time.perf_counter() - a
        Fp = ge.functional()[0]
        ge.load_links(u)
        torch.cuda.synchronize()
        if profile_range:
            torch.cuda.profiler.start()
        a = time.perf_counter()
        net.warm_start(ge)
        torch.cuda.synchronize()
        tw0 = time.perf_counter() - a
        if profile_range:
            torch.cuda.profiler.stop()
        Fw0 = ge.functional()[0]
        a = time.perf_counter()
        it_w, cw = ge.fix(W["tol"], W["max_iter"])
        torch.cuda.synchronize()
        tw = time.perf_counter() - a + tw0
        Fw, thw = ge.functional()
        rows.append(dict(F_start=F0, F_warm_start=Fw0, it_plain=it_p, it_warm=it_w, t_plain=tp, t_warm=tw,
                         t_inference=tw0, F_plain=Fp, F_warm=Fw, converged=bool(cp and cw),
                         same_copy=bool(abs(Fw - Fp) <= 1e-12 * abs(Fp))))
    ge.close()
    net.close()
    Ve = int(np.prod(W["eval_dims"]))
    mean = lambda key: float(np.mean([r[key] for r in rows]))
    it_p, it_w = mean("it_plain"), mean("it_warm")
    return {
        "value": round(Ve * it_w / mean("t_warm"), 1), "unit": METRIC, "train_steps": steps,
        "ms_per_train_step": round(train_s / max(steps, 1) * 1e3, 4),
        "config": {"workload": W["desc"], "train_lattice": list(W["train_dims"]), "train_configs": ntr,
                   "epochs": W["epochs"], "lr": W["lr"], "eval_lattice": list(W["eval_dims"]),
                   "eval_configs": W["eval_n"]},
        "training": {"seconds": round(train_s, 2), "train_steps": steps,
                     "mean_F_warm_first16": round(float(np.mean(F_first)), 6) if F_first else None,
                     "mean_F_warm_last16": round(float(np.mean(F_last)), 6) if F_last else None},
        "evaluation": {"iterations_plain": it_p, "iterations_warm": it_w,
                       "iteration_gain": round(it_p - it_w, 3),
                       "seconds_plain": round(mean("t_plain"), 5), "seconds_warm": round(mean("t_warm"), 5),
                       "seconds_inference": round(mean("t_inference"), 5),
                       "F_before": mean("F_start"), "F_after_warm_start": mean("F_warm_start"),
                       "all_converged": all(r["converged"] for r in rows),
                       "same_gribov_copy": sum(r["same_copy"] for r in rows), "per_config": rows},
    }


def oracle_arms(U_c2, U_c3, alpha: float) -> dict:
    """The oracle as it stands on the host's cores, all of them and one:
    seconds per iteration on the 32^4 and 48^3 x 8 inputs (a bounded sample
    of iterations each) and the whole fix of the 8^4 FP64 input; for the
    large inputs the time to theta is projected as seconds per iteration x
    the updates the oracle's own fix needs (stored by the committed script
    that runs only the oracle)."""
    import lgf_inputs
    info = host_cpu_info()
    cores = info["nproc"]
    U_c1 = lgf_inputs.synthetic_config((8, 8, 8, 8), seed=0, link_scale=0.3, gauge_scale=1.0)
    out = {"host": info, "kind": "oracle (numpy FP64, naive separable DFT of all nine entries)", "configs": {}}
    for threads in sorted({cores, 1}, reverse=True):
        key = f"{threads}_threads"
        r = run_oracle(U_c1, "fix", 2000, alpha, threads, tol=1e-12)
        out["configs"].setdefault("8^4 FP64 theta<1e-12", {})[key] = {
            "iterations": r["iterations"], "seconds_to_theta": round(r["seconds"], 3),
            "seconds_per_iteration": round(r["seconds"] / max(r["iterations"], 1), 5), "F": r["F"]}
        for name, U, case in (("32^4 theta<1e-15", U_c2, "32^4"), ("48^3x8 theta<1e-15", U_c3, "48^3x8")):
            n = 2
            secs = time_oracle(U, n, alpha, threads)
            its = oracle_fix_iterations(case)
            rec = {"sample": f"{n} iterations", "seconds_per_iteration": round(secs / n, 4),
                   "site_iterations_per_s": round(U.size // 36 * n / secs, 1)}
            if its is not None:
                rec["oracle_iterations_to_theta"] = its
                rec["projected_seconds_to_theta"] = round(secs / n * its, 2)
            out["configs"].setdefault(name, {})[key] = rec
    return out


def host_link_rates(torch, pinned_in, pinned_out, reps: int = 3) -> list:
    """GB/s of one pinned host -> device and one device -> host copy of the
    given buffers (best of reps, CUDA events on the current stream): the floor
    under lgf_load_links and lgf_store_links, which move the same bytes."""
    dev = torch.empty_like(pinned_in, device="cuda")
    rates = []
    for src, dst in ((pinned_in, dev), (dev, pinned_out)):
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            dst.copy_(src, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        rates.append(round(src.numel() * src.element_size() / (best * 1e-3) / 1e9, 1))
    del dev
    return rates


def e2e_stream(lgf, torch, np, gf, W, args, hostU, hostOut, barrier, max_over_ranks, n_configs: int = 32) -> dict:
    """An ensemble streamed through lgf_fix_stream: gf and a second handle of
    the same lattice, dtype, parameters and FFT schedule, each on its own
    stream.  Two pinned input arrays alternate (the workload's links and their
    complex conjugate, an equally valid SU(3) configuration that the method
    fixes in the same number of updates), and so do two pinned output arrays.
    Returns the wall time of n_configs configurations after one untimed
    2-configuration pass, and whether the stream reproduced the
    single-configuration result held in hostOut bit for bit."""
    stream2 = torch.cuda.Stream()
    gf2 = lgf.GaugeFixer(gf.dims, W["dtype"], stream=stream2, alpha=W["alpha"])
    try:
        if W["dtype"].startswith("f32"):
            gf2.set_param(6, args.link_update)  # LGF_LINK_UPDATE
            if args.tail_theta > 0:
                gf2.set_param(2, args.tail_theta)  # LGF_TAIL_THETA
        for eng in ((0, 1) if W["dtype"].startswith("f32") else (0,)):
            gf2.set_schedule(*gf.schedule(eng), engine=eng)
        shape = hostU.shape
        bufs = []
        for _ in range(3):
            t = torch.empty(shape + (2,), dtype=torch.float64, pin_memory=True)
            bufs.append((t, t.numpy().view(np.complex128).reshape(shape)))
        hostU2, out_a, out_b = bufs[0][1], bufs[1][1], bufs[2][1]
        np.conjugate(hostU, out=hostU2)
        out_a[...] = 0
        out_b[...] = 0
        ref = hostOut.copy()  # the single-configuration path's fixed links of hostU
        ins, outs = [hostU, hostU2], [out_a, out_b]
        lgf.fix_stream((gf, gf2), ins, outs, W["tol"], W["max_iter"])  # untimed: graphs, staging buffers
        ins, outs = ins * (n_configs // 2), outs * (n_configs // 2)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        its, conv = lgf.fix_stream((gf, gf2), ins, outs, W["tol"], W["max_iter"])
        secs = max_over_ranks(time.perf_counter() - t0)
        return {"seconds": secs, "configs": len(ins), "iterations": int(sum(its)), "iters": sorted(set(its)),
                "converged": conv, "matches": bool(np.array_equal(out_a, ref))}
    finally:
        gf2.close()


def run_ours(args, W):
    import numpy as np
    import torch

    import paper_1208_1186_gb300 as lgf

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    rp = Replicas("nccl", torch.device("cuda", local))
    world, rank = rp.world, rp.rank
    barrier, max_over_ranks = rp.barrier, rp.max

    dims = W["dims"]
    V = int(np.prod(dims))
    seed = rp.seed(W["seed"])  # independent configurations per rank (replicas)
    t = time.time()
    from lgf_inputs import torch_gen
    Ud = torch_gen.synthetic_config(dims, seed=seed, link_scale=W["link_scale"], gauge_scale=W["gauge_scale"],
                                    device="cuda")
    torch.cuda.synchronize()
    U = Ud.cpu().numpy()  # host copy: e2e source and the oracle's input
    log(f"[rank {rank}] generated {dims} config on the GPU in {time.time() - t:.1f}s")
    stream = torch.cuda.Stream()
    gf = lgf.GaugeFixer(dims, W["dtype"], stream=stream, alpha=W["alpha"])
    gauge_rep = W["dtype"].startswith("f32") and args.link_update == 0
    if W["dtype"].startswith("f32"):
        gf.set_param(6, args.link_update)  # LGF_LINK_UPDATE
        if args.tail_theta > 0:
            gf.set_param(2, args.tail_theta)  # LGF_TAIL_THETA
    gf.load_links(Ud)
    schedule = None
    if not args.no_autotune:
        # the library's FFT schedule autotuner (pipeline, z-t tile width,
        # radix order) on this shape, before anything is timed
        gf.autotune(reps=10)
        schedule = gf.schedule()
        gf.load_links(Ud)
    smi = ClockSampler(gpu_id_for_smi(torch)) if rank == 0 else None
    try:
        gf.iterate(args.warmup)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        launches0 = gf.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        if args.profile_range == "steps":
            torch.cuda.profiler.start()
        ev0.record(stream)
        gf.iterate(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        if args.profile_range == "steps":
            torch.cuda.profiler.stop()
        w1 = time.time()
        barrier()
        ms = ev0.elapsed_time(ev1)
        launches = gf.launch_count() - launches0
        ms_max = max_over_ranks(ms)
        # the same K steps once more with CUDA events around every launch (on
        # the launch stream): the per-kernel durations of the roofline.  Kept
        # out of the timed pass, where events between launches would add their
        # own gaps and stop dependent launches from overlapping.
        gf.profile(True)
        ep0 = torch.cuda.Event(enable_timing=True)
        ep1 = torch.cuda.Event(enable_timing=True)
        ep0.record(stream)
        gf.iterate(args.steps)
        ep1.record(stream)
        torch.cuda.synchronize()
        ms_prof = ep0.elapsed_time(ep1)
        prof = gf.profile_read()
        gf.profile(False)

        # time to theta < tol from device-resident links, after one untimed
        # fix (which builds the handle's device-side loop graphs once)
        gf.load_links(Ud)
        gf.fix(W["tol"], W["max_iter"])
        gf.load_links(Ud)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        iters, conv = gf.fix(W["tol"], W["max_iter"])
        e1.record(stream)
        torch.cuda.synchronize()
        fix_s = max_over_ranks(e0.elapsed_time(e1) / 1e3)
        split = gf.fix_split()
        F, theta = gf.functional()
        # the same fix once more with per-kernel events, for the breakdown
        # (host-queued iterations instead of the device-side graph loops, so
        # that ncu, which cannot profile kernels inside graphs with conditional
        # nodes, sees them: --profile-range fix brackets this fix)
        gf.load_links(Ud)
        torch.cuda.synchronize()
        gf.profile(True)
        if args.profile_range == "fix":
            torch.cuda.profiler.start()
        gf.fix(W["tol"], W["max_iter"])
        if args.profile_range == "fix":
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        fix_prof = {k: round(v[0], 3) for k, v in gf.profile_read().items() if v[1]}
        fix_launches = {k: v[1] for k, v in gf.profile_read().items() if v[1]}
        gf.profile(False)

        # end to end through the public API from pinned host memory
        pinned = torch.empty(U.shape + (2,), dtype=torch.float64, pin_memory=True)
        hostU = pinned.numpy().view(np.complex128).reshape(U.shape)
        hostU[...] = U
        # (empty_like would not pin the output buffer)
        pinned_out = torch.empty(U.shape + (2,), dtype=torch.float64, pin_memory=True)
        hostOut = pinned_out.numpy().view(np.complex128).reshape(U.shape)
        hostOut[...] = 0  # touch every page before the timed region

        def e2e_pass():
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            gf.load_links(hostU)
            t1 = time.perf_counter()
            n, _ = gf.fix(W["tol"], W["max_iter"])
            t2 = time.perf_counter()
            gf.store_links(hostOut)
            t3 = time.perf_counter()
            return n, t3 - t0, {"load_s": round(t1 - t0, 4), "fix_s": round(t2 - t1, 4),
                                "store_s": round(t3 - t2, 4)}

        _, _, e2e_warm_parts = e2e_pass()  # one untimed warm-up pass
        iters_e2e, e2e_local, e2e_parts = e2e_pass()
        e2e_s = max_over_ranks(e2e_local)
        # (before the host-link timing below, which overwrites hostOut)
        stream_rec = e2e_stream(lgf, torch, np, gf, W, args, hostU, hostOut, barrier, max_over_ranks)
        link = host_link_rates(torch, pinned, pinned_out)
    finally:
        if smi:
            smi.stop()
    clocks = smi.summary(w0, w1) if smi else None
    gf.close()

    if rank != 0:
        rp.close()
        return None

    prec = 4 if W["dtype"].startswith("f32") else 8
    r = 12 if W["dtype"].endswith("r12") else 18
    pk = peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6800.0
    kernels = kernel_table(prof, args.steps, V, prec, r, gauge_rep)
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_launch"] * kernels[k]["launches"])
    ach = kernels[dom]["algorithmic_gbs"]
    step_bytes = sum(bytes_per_site(k, prec, r, gauge_rep) * kernels[k]["launches"] / args.steps
                     for k in kernels) * V
    value = rp.throughput(V * args.steps, ms_max / 1e3)
    h2d = V * 576
    d2h = V * 576
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": METRIC,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == 4 else "f64",
        "data": "synthetic (seeded SU(3) links behind a random gauge; stands in for thermalised ensembles)",
        "config": main_config(W, world, gauge_rep),
        "fft_schedule": ({"autotuned": True, "pipeline": schedule[0], "zt_tile_width": schedule[1],
                          "radix_order": schedule[2]} if schedule else {"autotuned": False}),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(ach / hbm_peak, 4) if ach else None,
                     "traffic": profile_traffic(dom, args.workload, gauge_rep),
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback"},
        "step_roofline": {"algorithmic_bytes_per_site": step_bytes / V,
                          "achieved_gbs": round(step_bytes / (ms_max / args.steps * 1e-3) / 1e9, 1),
                          "frac": round(step_bytes / (ms_max / args.steps * 1e-3) / 1e9 / hbm_peak, 4)},
        "kernels": kernels,
        "kernel_timing": {"how": "CUDA events around each launch on the launch stream, in a second pass of the "
                                 "same K steps right after the timed pass",
                          "ms_per_step_with_kernel_events": round(ms_prof / args.steps, 5)},
        "time_to_theta": {"theta_tol": W["tol"], "seconds": round(fix_s, 5), "iterations": iters,
                          "fp32_iterations": split[0], "fp64_iterations": split[1], "converged": conv,
                          "F": F, "theta": theta,
                          "kernel_ms_profiled_run": fix_prof, "kernel_launches_profiled_run": fix_launches},
        "e2e": {"value": round(rp.throughput(V * stream_rec["iterations"], stream_rec["seconds"]), 1),
                "unit": METRIC,
                "what": f"an ensemble of {stream_rec['configs']} configurations of this workload fixed to theta<tol "
                        "through the public API lgf_fix_stream from pinned host memory and back: two handles, "
                        "configuration k fixed while k+1 is copied in and k-1 copied out (every configuration's "
                        "links copied host->device and its fixed links device->host inside the timed region); "
                        "value = sites x updates of all configurations / wall time",
                "seconds": round(stream_rec["seconds"], 4),
                "seconds_per_config": round(stream_rec["seconds"] / stream_rec["configs"], 5),
                "configs": stream_rec["configs"], "iterations_per_config": stream_rec["iters"],
                "matches_single_config_path": stream_rec["matches"],
                "h2d_bytes_per_step": round(h2d / max(iters_e2e, 1), 1),
                "d2h_bytes_per_step": round(d2h / max(iters_e2e, 1), 1),
                "single": {"value": round(rp.throughput(V * iters_e2e, e2e_s), 1), "unit": METRIC,
                           "seconds": round(e2e_s, 4),
                           "what": "one configuration: lgf_load_links(pinned host) + lgf_fix(theta<tol) + "
                                   "lgf_store_links(pinned host), nothing overlapped",
                           "parts": e2e_parts, "warmup_pass_parts": e2e_warm_parts},
                "host_link": {"how": "plain pinned copies of the same link arrays (copy engine, CUDA events), "
                                     "after the e2e passes",
                              "h2d_gbs": link[0], "d2h_gbs": link[1],
                              "load_store_floor_s": round(h2d / (link[0] * 1e9) + d2h / (link[1] * 1e9), 5)}},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    arms = set(args.arms.split(",")) if args.arms not in ("", "none") else set()
    if "all" in arms:
        arms = set(ARMS)
    if world == 1 and arms and args.workload == DEFAULT_WORKLOAD:
        line["arms"] = run_arms(args, lgf, torch, W, Ud, U, line, arms)
    if not args.no_cpu_baseline:
        n = args.cpu_iters
        cores = host_cores()
        log(f"timing {n} oracle iteration(s) on the same {dims} input, {cores} thread(s) ...")
        secs = time_oracle(U, n, W["alpha"], cores)
        line["cpu_baseline"] = {"value": round(V * n / secs, 1), "unit": METRIC, "cores": cores, "kind": "oracle",
                                "sample": f"{n} iteration(s) of the numpy FP64 oracle on the same {dims} input "
                                          f"({secs:.1f} s, {cores} BLAS/OpenMP threads = all host cores; "
                                          f"1-thread figures under arms.cpu_oracle)"}
    rp.close()
    return line


ARMS = ("plain_fp64", "reunit_fp64", "c3", "batch", "warm", "cpu_oracle")


def run_arms(args, lgf, torch, W, Ud, U, line, arms) -> dict:
    """The comparison arms of the metric, on rank 0 of a 1-GPU run: the same
    32^4 input fixed by the plain FP64 method, the FP32 step with FP64
    reunitarisation, the 48^3 x Nt 12-real lattices, the 64-lattice batch,
    the learned warm start, and the oracle on the host's cores."""
    out = {}
    t_start = time.time()
    mixed_s = line["time_to_theta"]["seconds"]
    if "plain_fp64" in arms:
        log("arm: plain FP64 on the same 32^4 input ...")
        Wf = dict(W, dtype="f64", desc="the same 32^4 input, plain FP64 (links, FFT, update) to theta<1e-15")
        a = arm_single(lgf, torch, Wf, args.steps, args.warmup, Ud=Ud)
        tt = a["time_to_theta"]
        a["vs_mixed"] = {"time_to_theta_ratio_fp64_over_mixed": round(tt["seconds"] / mixed_s, 3),
                         "site_it_ratio_mixed_over_fp64": round(line["value"] / a["value"], 3),
                         "F_rel_diff_mixed_vs_fp64": abs(line["time_to_theta"]["F"] - tt["F"]) / abs(tt["F"])}
        out["plain_fp64_32^4"] = a
    if "reunit_fp64" in arms:
        log("arm: FP32 step with g reunitarised in FP64 ...")
        Wr = dict(W, desc="the same 32^4 input, FP32 storage with g reunitarised in FP64 arithmetic "
                          "(LGF_REUNIT_FP64=1)")
        out["reunit_fp64_32^4"] = arm_single(lgf, torch, Wr, args.steps, args.warmup, params=((4, 1),), Ud=Ud)
    U_c3 = None
    if "c3" in arms:
        for lt in (8, 12):
            log(f"arm: 48^3x{lt} 12-real ...")
            Wc = dict(WORKLOADS["48^3x8-f32r12"], dims=(48, 48, 48, lt),
                      desc=f"48^3x{lt} single config, FP32 12-real links, FP64 tail to theta<1e-15, link scale 0.6")
            from lgf_inputs import torch_gen
            Uc = torch_gen.synthetic_config(Wc["dims"], seed=0, link_scale=0.6, gauge_scale=1.0, device="cuda")
            if lt == 8:
                U_c3 = Uc.cpu().numpy()
            out[f"48^3x{lt}-f32r12"] = arm_single(lgf, torch, Wc, args.steps, args.warmup, Ud=Uc)
            del Uc
    if "batch" in arms:
        log("arm: batch of 64 mixed lattices ...")
        b = batch_measure(lgf, torch, WORKLOADS["batch64-f32"], args.steps, args.warmup)
        b.pop("_window", None)
        out["batch64-f32"] = b
    if "warm" in arms:
        log("arm: learned warm start (training on the GPU, evaluation on 24^4) ...")
        Ww = WORKLOADS["warmstart-f32"]
        out["warmstart-f32"] = warm_measure(lgf, torch, Ww, Ww["train_n"])
    torch.cuda.synchronize()
    if "cpu_oracle" in arms:
        if U_c3 is None:
            from lgf_inputs import torch_gen
            U_c3 = torch_gen.synthetic_config((48, 48, 48, 8), seed=0, link_scale=0.6, gauge_scale=1.0,
                                              device="cuda").cpu().numpy()
        log("arm: the oracle on all host cores and on one ...")
        out["cpu_oracle"] = oracle_arms(U, U_c3, W["alpha"])
    out["seconds"] = round(time.time() - t_start, 1)
    return out


def run_batch(args, W):
    """Batched workload on one GPU (lgf_batch) as its own bench line."""
    import torch

    import paper_1208_1186_gb300 as lgf

    torch.cuda.set_device(0)
    smi = ClockSampler(gpu_id_for_smi(torch))
    try:
        b = batch_measure(lgf, torch, W, args.steps, args.warmup, args.lanes, not args.no_autotune)
    finally:
        smi.stop()
    w0, w1 = b.pop("_window")
    return {
        "metric": METRIC, "value": b["value"], "unit": METRIC, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded SU(3) links behind a random gauge; stands in for thermalised ensembles)",
        "config": {"workload": W["desc"], "members": b["members"], "sites": b["sites"], "storage": W["dtype"],
                   "fft_pipeline_per_shape": b["fft_pipeline_per_shape"], "graph_lanes": b["graph_lanes"],
                   "timing": b["timing"]},
        "roofline": b["roofline"], "time_to_theta": b["time_to_theta"],
        "e2e": None,
        "e2e_note": "batched workload: inputs generated and kept on the device; see the 32^4 line for e2e",
        "gpu_launches": b["gpu_launches"],
        "clocks": smi.summary(w0, w1),
    }


def run_warm(args, W):
    """The warm-start workload as its own bench line."""
    import torch

    import paper_1208_1186_gb300 as lgf

    torch.cuda.set_device(0)
    ntr = args.train_n if args.train_n else W["train_n"]
    w = warm_measure(lgf, torch, W, ntr, bool(args.profile_range))
    return {
        "metric": METRIC, "value": w["value"], "unit": METRIC, "n_gpus": 1,
        "steps": w["train_steps"], "warmup": 0, "ms_per_step": w["ms_per_train_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
        "data": "synthetic (seeded SU(3) links behind a random gauge; stands in for thermalised ensembles)",
        "config": w["config"], "training": w["training"], "evaluation": w["evaluation"],
        "e2e": None, "e2e_note": "see the 32^4 line", "roofline": None,
    }


def run_reference(args, W):
    """The oracle as it stands, on all host cores, each step a bounded sample."""
    import numpy as np

    import lgf_inputs
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return None
    cores = host_cores()
    budget = 150.0 / max(args.steps + args.warmup, 1)  # seconds per step
    # per-site cost model from two small lattices
    probe = {}
    for L in (8, 12):
        U = lgf_inputs.synthetic_config((L,) * 4, seed=W["seed"], link_scale=W["link_scale"])
        probe[L] = time_oracle(U, 2, W["alpha"], cores) / 2 / L ** 4
    slope = (probe[12] - probe[8]) / 4

    def est(dims):
        return int(np.prod(dims)) * max(probe[8] + slope * (max(dims) - 8), probe[8])

    cands = [W["dims"]] + [(L,) * 4 for L in (24, 20, 16, 12, 8)]
    dims = next((d for d in cands if est(d) <= budget), (8, 8, 8, 8))
    U = lgf_inputs.synthetic_config(dims, seed=W["seed"], link_scale=W["link_scale"],
                                    gauge_scale=W["gauge_scale"])
    V = int(np.prod(dims))
    time_oracle(U, args.warmup, W["alpha"], cores) if args.warmup else None
    secs = time_oracle(U, args.steps, W["alpha"], cores)
    value = V * args.steps / secs
    sample = (f"{args.steps} oracle iteration(s) on a {dims} lattice of the same recipe"
              + ("" if tuple(dims) == tuple(W["dims"]) else f" (full {W['dims']} does not fit the time budget)")
              + f", {cores} BLAS/OpenMP threads (all host cores)")
    gauge_rep = W["dtype"].startswith("f32")
    return {
        "impl": "reference",
        "metric": METRIC, "value": round(value, 1), "unit": METRIC, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": main_config(W, world, gauge_rep),
        "sample_lattice": list(dims),
        "cpu_baseline": {"value": round(value, 1), "unit": METRIC, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 1), "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


SWEEP_SHAPES = [((32, 32, 32, 32), "f32"), ((48, 48, 48, 8), "f32_r12"), ((48, 48, 48, 12), "f32_r12"),
                ((24, 24, 24, 48), "f32"), ((32, 32, 32, 8), "f32"), ((16, 16, 16, 16), "f32"),
                ((20, 20, 20, 20), "f32")]


def schedule_sweep(iters: int = 50):
    """z-t pass time per launch for each (tile width, radix order) the
    register-plane pipeline supports on each shape (lgf_set_schedule, then
    `iters` iterations with per-kernel CUDA events), and the autotuner's own
    choice on the same handle."""
    import torch
    import paper_1208_1186_gb300 as lgf
    from lgf_inputs import torch_gen
    for dims, dtype in SWEEP_SHAPES:
        Ud = torch_gen.synthetic_config(dims, seed=0, link_scale=0.5, gauge_scale=1.0, device="cuda")
        st = torch.cuda.Stream()
        gf = lgf.GaugeFixer(dims, dtype, stream=st)
        res = {}
        for bx in (0, 8):
            for ro in (0, 1, 2):
                try:
                    gf.set_schedule(3, bx, ro)
                except lgf.LgfError:
                    continue  # not supported on this shape
                gf.load_links(Ud)
                gf.iterate(5)
                torch.cuda.synchronize()
                gf.profile(True)
                gf.iterate(iters)
                torch.cuda.synchronize()
                k = gf.profile_read()
                gf.profile(False)
                res[f"width{bx or 4}_order{ro}"] = round(k["fft_zt"][0] / k["fft_zt"][1] * 1e3, 2)
        gf.set_schedule(3, 0, 0)
        gf.load_links(Ud)
        gf.autotune(reps=10)
        print(json.dumps({"lattice": list(dims), "storage": dtype, "zt_us_per_launch": res,
                          "autotune": list(gf.schedule())}), flush=True)
        gf.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--train-n", type=int, default=0, help="warm-start workload: training configurations")
    ap.add_argument("--tail-theta", type=float, default=0.0, help="theta at which the FP32 phase hands over")
    ap.add_argument("--lanes", type=int, default=-1, help="batch workload: parallel graph lanes (0: one per member)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default FFT schedule (no lgf_autotune on the timed handles or batch members)")
    ap.add_argument("--profile-range", choices=["", "steps", "fix"], default="", nargs="?", const="steps",
                    help="bracket with cudaProfilerStart/Stop, for ncu --profile-from-start off: the timed steps "
                         "(steps, the default of the bare flag) or the per-kernel-profiled (host-queued) fix to "
                         "theta < tol (fix) of the single-lattice workloads, or the warm-start inferences of the "
                         "warm-start workload")
    ap.add_argument("--arms", default="all",
                    help="default workload: comparison arms to add, comma-separated from "
                         + ",".join(ARMS) + ", or 'all' / 'none'")
    ap.add_argument("--link-update", type=int, default=0, choices=[0, 1],
                    help="FP32 storage: 0 gauge representation (default), 1 links updated in place")
    ap.add_argument("--schedule-sweep", action="store_true",
                    help="time the z-t pass (us per launch) under every register-plane FFT schedule on "
                         "32^4, 48^3x8, 48^3x12, 24^3x48, 32^3x8, 16^4 and 20^4, print one JSON line per "
                         "lattice and exit")
    args = ap.parse_args()
    if args.schedule_sweep:
        schedule_sweep()
        return
    if args.warmup < 3 and args.impl == "ours":
        log("warm-up raised to 3 steps (minimum)")
        args.warmup = 3
    W = WORKLOADS[args.workload]
    if args.impl == "reference":
        if "batch" in W or "warm" in W:
            W = WORKLOADS[DEFAULT_WORKLOAD]
        line = run_reference(args, W)
    elif "batch" in W:
        line = run_batch(args, W)
    elif "warm" in W:
        line = run_warm(args, W)
    else:
        line = run_ours(args, W)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

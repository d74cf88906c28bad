"""Benchmark of the GKS step on GB300: prints ONE JSON line (rank 0).

Workload (default): 2-D TM, 4096 x 4096 Cartesian grid with 32 seeded dielectric cylinders,
kinetic non-reflecting boundary, Gaussian-modulated line source, CFL 0.5, FP32 state and
arithmetic; a step is one GKS time step over the whole grid (one fused kernel launch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gks|reference]

value      cell-updates per second over the K timed steps (all ranks), inputs resident in HBM.
e2e        the same metric through the C ABI from host memory: gks_write_fields (pinned FP64
           host fields) + gks_step(K) + gks_read_fields, wall-clocked.
roofline   the fused step kernel against the measured HBM copy bandwidth.
cpu_baseline  the FP64 oracle on a bounded sample of the workload on the host cores.
With N > 1 (torchrun) the grid is split into N slabs of its slowest axis (y in 2-D, z in 3-D),
one per GPU, each with two ghost layers per shared side refreshed from the neighbours over NCCL
after every step (strong scaling: the same grid on more GPUs); the 2-D headline and the 3-D leg
run that way, the other legs only at N = 1.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCell-updates/s FP32 vs FP64 at stated error; % HBM roofline; adjoint/fwd cost"
UNIT = "GCell-updates/s"
BYTES_PER_CELL_STEP = {"fp32": 28, "fp64": 56}   # 3 fields read + written, eps read
KERNEL_SRC = os.path.join(ROOT, "paper_2412_16845_gb300", "csrc", "gks_cart2d.cu")
PROFILE = os.path.join(ROOT, "profiles", "cart2d_step_tm2d_cylinders_4096_fp32.md")


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SRC_3D = os.path.join(ROOT, "paper_2412_16845_gb300", "csrc", "gks_cart3d_side.cu")
PROFILE_3D = os.path.join(ROOT, "profiles", "cart3d_side_step_maxwell3d_sphere_fp32.md")


def _kernel_hash(src=KERNEL_SRC):
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def _profiled_traffic(profile=PROFILE, src=KERNEL_SRC):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current kernel."""
    if not os.path.exists(profile):
        return None
    txt = open(profile).read()
    m = re.search(r"dram_bytes_per_launch\s*=\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256_16\s*=\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != _kernel_hash(src):
        return None
    return float(m.group(1))


def sharded_steps(w, precision, steps, warmup, world, rank, stream, e2e=False):
    """Time `steps` steps of the workload split into `world` slabs (this rank's slab), with the
    halo exchange after every step.  Returns (ms over the timed steps, this rank's launches,
    e2e wall seconds or None).  e2e: gks_write_fields of the slab's fields from pinned host
    memory + steps + gks_read_fields, wall clock."""
    import torch
    import torch.distributed as dist

    from paper_2412_16845_gb300 import gks as G
    from paper_2412_16845_gb300 import slab

    ax = w.dim - 1
    plan = slab.partition(w.n[ax], world, rank, w.bc[2 * ax] == "periodic")
    s = slab.SlabSolver(w, plan, precision=precision, backend="nccl", stream=stream.cuda_stream)
    s.step(warmup)
    torch.cuda.synchronize()
    dist.barrier()
    L0 = G.gks_get_launch_count(s.ctx)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    ms = a.elapsed_time(b)
    launches = G.gks_get_launch_count(s.ctx) - L0
    wall = None
    if e2e:
        f = np.asarray(w.fields0)[:, s.ids]
        hin = torch.empty(f.shape, dtype=torch.float64, pin_memory=True)
        hin.copy_(torch.from_numpy(np.ascontiguousarray(f)))
        hout = torch.empty(f.shape, dtype=torch.float64, pin_memory=True)
        dist.barrier()
        t0 = time.perf_counter()
        G.gks_write_fields(s.ctx, hin.numpy())
        s.step(steps)
        G.gks_read_fields(s.ctx, hout.numpy())
        wall = time.perf_counter() - t0
        dist.barrier()
    s.close()
    return ms, launches, wall


def max_over_ranks(x, world, device="cuda"):
    """The largest of the ranks' values of x (every rank gets it); x itself when world == 1."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank, steps, ms_max, world):
    """Whole-job cell-updates per second (in G): every rank advanced cells_per_rank cells by
    `steps` steps, and the job took the slowest rank's time ms_max."""
    return world * cells_per_rank * steps / (ms_max * 1e-3) / 1e9


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds=12.0, block=160, all_cores=False):
    """Time the FP64 oracle (unchanged) on a block of the 4096^2 workload, in a fresh process
    with single-threaded numpy/BLAS."""
    code = f"""
import sys, time, json, numpy as np
sys.path.insert(0, {ROOT!r})
from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
n = 4096; b = {block}
w = wl.config2_cylinders_tm(n=n, steps=1)
i0 = w.extra['i_src'] - b // 2; j0 = n // 2 - b // 2
ii = np.arange(i0, i0 + b); jj = np.arange(j0, j0 + b)
gid = (jj[:, None] * n + ii[None, :]).ravel()
h = 1.0 / n
mesh = go.cartesian_mesh((b, b), (i0 * h, j0 * h), ((i0 + b) * h, (j0 + b) * h), ('nrbc',) * 4)
rng = np.random.default_rng(0)
V = go.fields_to_state(rng.standard_normal((3, b * b)), 2)
m = go.material_diag(w.eps[gid], None)
dt = 0.5 * h; C = go.time_coefficients(dt, 0.0)
steps = 0; t0 = time.perf_counter()
while True:
    V = go.step(mesh, V, m, dt, C, 1.0, w.jz_mask[gid] * go.source_signal(steps * dt, *w.src))
    steps += 1
    el = time.perf_counter() - t0
    if el >= {seconds}:
        break
print(json.dumps({{"cells": b * b, "steps": steps, "seconds": el}}))
"""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=600)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "failed: " + r.stderr[-300:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    v = d["cells"] * d["steps"] / d["seconds"] / 1e9
    out = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
           "nproc": os.cpu_count(),
           "sample": f"{d['steps']} FP64 oracle steps on a {block}x{block} block of the 4096^2 "
                     f"cylinder workload around the source ({d['seconds']:.1f} s, numpy single "
                     f"thread)"}
    if all_cores:
        # one single-threaded oracle process per host core, each on its own copy of the block,
        # run side by side for the same time: the aggregate rate of the whole host (left out
        # of the line if any process fails)
        ncores = max(1, min(os.cpu_count() or 1, 64))
        procs = []
        try:
            procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True, env=env)
                     for _ in range(ncores)]
            total = 0.0
            for pr in procs:
                so, _ = pr.communicate(timeout=600)
                if pr.returncode != 0:
                    raise RuntimeError("oracle process failed")
                e = json.loads(so.strip().splitlines()[-1])
                total += e["cells"] * e["steps"] / e["seconds"] / 1e9
            out["all_cores"] = {"value": total, "unit": UNIT, "cores": ncores,
                                "sample": f"{ncores} such processes side by side"}
        except Exception:
            for pr in procs:
                if pr.poll() is None:
                    pr.kill()
    return out


# reduced versions of the three timed workloads, whose FP32 GPU results the oracle leg checks
REDUCED = {"tm2d_cylinders": (96, 60), "maxwell3d_sphere": (20, 30), "tets_sphere": (8, 25)}


def reduced_gpu_results(stream_ptr, path):
    """FP32 (and FP64) GPU fields of the reduced workloads, saved for the oracle leg."""
    from paper_2412_16845_gb300 import workloads as wl
    from paper_2412_16845_gb300.gks import GKSSolver
    out = {}
    n2, k2 = REDUCED["tm2d_cylinders"]
    n3, k3 = REDUCED["maxwell3d_sphere"]
    m4, k4 = REDUCED["tets_sphere"]
    for prec in ("fp32", "fp64"):
        s = GKSSolver.from_workload(wl.config2_cylinders_tm(n=n2, steps=k2), precision=prec,
                                    stream=stream_ptr)
        s.step(k2)
        out[f"tm2d_{prec}"] = s.read_fields()
        s.close()
        s = GKSSolver.from_workload(wl.config3_sphere_3d(n=n3, steps=k3), precision=prec,
                                    stream=stream_ptr)
        s.step(k3)
        out[f"maxwell3d_{prec}"] = s.read_fields()
        s.close()
        s = GKSSolver.from_tet_workload(wl.config4_tets(m=m4, steps=k4), precision=prec,
                                        stream=stream_ptr)
        s.step(k4)
        out[f"tets_{prec}"] = s.read_fields()
        s.close()
    np.savez(path, **out)


# The 3-D FP32 step kernel (cart3d_side_kernel) is bound by instruction issue: its ncu summary
# (profiles/cart3d_side_step_maxwell3d_sphere_fp32.md) counts 608 thread-instructions per cell at
# 160^3, where 20% of the 64-column tiles lie past the grid, i.e. about 520 per cell on a grid of
# whole tiles such as 256^3.  The issue peak is 152 SMs x 4 schedulers x 32 threads x 2.07 GHz.
INSTR_PER_CELL_3D = 520
ISSUE_PEAK_T = 152 * 4 * 32 * 2.07e9 / 1e12          # T thread-instructions/s


def roofline_3d(ncell, ms):
    """Roofline object of the 3-D FP32 step: issue-bound (thread-instructions per second against
    the issue peak), with the HBM fraction of its 52 algorithmic bytes per cell alongside."""
    hbm, how = _peaks()
    gcells = ncell / (ms * 1e-3) / 1e9
    achieved = gcells * 1e9 * INSTR_PER_CELL_3D / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": ISSUE_PEAK_T,
            "unit": "T thread-instructions/s", "frac": achieved / ISSUE_PEAK_T,
            "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2.07 GHz",
            "instructions_per_cell": INSTR_PER_CELL_3D,
            "instructions_source": "ncu, profiles/cart3d_side_step_maxwell3d_sphere_fp32.md",
            "kernel": "cart3d_side_kernel (FP32, mu = 1)",
            "hbm": {"achieved": 52 * gcells, "peak": hbm, "unit": "GB/s",
                    "frac": 52 * gcells / hbm, "peak_source": how,
                    "traffic": _profiled_traffic(PROFILE_3D, KERNEL_SRC_3D) if ncell == 256 ** 3
                    else None}}


def divergence_report(sptr):
    """div_h H = (Hx(i+1) - Hx(i-1))/(2h) + (Hy(j+1) - Hy(j-1))/(2h) of the GPU FP64 fields on the
    periodic 64^2 workload (oblique plane wave plus Gaussian pulse, CFL 0.5) before and after its
    200 steps: discrete L2 norms (sqrt(sum h^2 x^2)), the same relative to the summed norms of its
    two terms, and the largest change of sum_i |Omega_i| U_i over the run (conservation).  The
    test suite checks these fields against the oracle's."""
    from paper_2412_16845_gb300 import workloads as wl
    from paper_2412_16845_gb300.gks import GKSSolver

    n = 64
    w = wl.config1_periodic_tm(n)
    s = GKSSolver.from_workload(w, precision="fp64", stream=sptr)
    f0 = s.read_fields()
    s.step(200)
    f1 = s.read_fields()
    s.close()
    h = 1.0 / n

    def div(f):
        hx, hy = f[1].reshape(n, n), f[2].reshape(n, n)
        dx = (np.roll(hx, -1, axis=1) - np.roll(hx, 1, axis=1)) / (2 * h)
        dy = (np.roll(hy, -1, axis=0) - np.roll(hy, 1, axis=0)) / (2 * h)
        return float(np.linalg.norm(dx + dy) * h), float((np.linalg.norm(dx) + np.linalg.norm(dy)) * h)

    d0, t0 = div(f0)
    d1, t1 = div(f1)
    return {"workload": "tm2d_periodic_64 (FP64, 200 steps)", "div_h_H_l2_initial": d0,
            "div_h_H_l2": d1, "div_rel_to_terms_initial": d0 / t0, "div_rel_to_terms": d1 / t1,
            "max_change_sum_vol_U": float(np.abs((f1.sum(axis=1) - f0.sum(axis=1)) * h * h).max())}


def oracle_errors(path):
    """The oracle leg's second job: the FP64 oracle on the reduced workloads against the GPU
    results saved at `path` (relative L2 over all components and cells, volume-weighted on
    tets), in a fresh process like the timing."""
    code = f"""
import sys, json, numpy as np
sys.path.insert(0, {ROOT!r})
from oracle import gks_oracle as go
from paper_2412_16845_gb300 import workloads as wl
R = {REDUCED!r}
g = np.load({path!r})
def rel(a, b, w=None):
    w = np.ones(b.shape[1]) if w is None else w
    return float(np.sqrt(np.sum(w * (a - b) ** 2) / np.sum(w * b * b)))
res = {{}}
n2, k2 = R["tm2d_cylinders"]
w = wl.config2_cylinders_tm(n=n2, steps=k2)
m = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
ref, _ = go.run(m, w.fields0, w.eps, None, w.cfl, k2, jz_mask=w.jz_mask, src=w.src)
res["tm2d_cylinders"] = {{"grid": [n2, n2], "steps": k2, "fp32": rel(g["tm2d_fp32"], ref),
                          "fp64": rel(g["tm2d_fp64"], ref)}}
n3, k3 = R["maxwell3d_sphere"]
w = wl.config3_sphere_3d(n=n3, steps=k3)
m = go.cartesian_mesh(w.n, w.lo, w.hi, w.bc)
ref, _ = go.run(m, w.fields0, w.eps, None, w.cfl, k3)
res["maxwell3d_sphere"] = {{"grid": [n3, n3, n3], "steps": k3,
                            "fp32": rel(g["maxwell3d_fp32"], ref),
                            "fp64": rel(g["maxwell3d_fp64"], ref)}}
m4, k4 = R["tets_sphere"]
w = wl.config4_tets(m=m4, steps=k4)
m = go.tet_mesh(w.vert, w.tet)
ref, _ = go.run(m, w.fields0, w.eps, None, w.cfl, k4, c=1.0)
res["tets_sphere"] = {{"tets": int(w.tet.shape[0]), "steps": k4,
                       "fp32": rel(g["tets_fp32"], ref, m.vol), "fp64": rel(g["tets_fp64"], ref, m.vol)}}
print(json.dumps(res))
"""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        return {"failed": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def run_reference(args, rank):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return
    block = 96
    per = []
    base = cpu_baseline(seconds=0.5, block=block)   # warm imports / caches
    for _ in range(args.warmup):
        pass
    t0 = time.perf_counter()
    res = cpu_baseline(seconds=max(2.0, 1.0 * args.steps / 50.0), block=block)
    el = time.perf_counter() - t0
    v = res["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "tm2d_cylinders_4096 (block sample)", "grid": [4096, 4096],
                       "cfl": 0.5, "steps_config": 2000},
            "cpu_baseline": res,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": el}
    print(json.dumps(line))


def run_sharded(args, w, world, rank, local, stream):
    """N > 1: the 2-D headline and the 3-D leg on slabs (strong scaling); one JSON line."""
    import torch
    from paper_2412_16845_gb300 import workloads as wl

    n = args.n
    ncell = n * n
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    ms, launches, wall = sharded_steps(w, "fp32", args.steps, args.warmup, world, rank, stream,
                                       e2e=True)
    clocks = sampler.stop() if rank == 0 else None
    ms = max_over_ranks(ms, world)
    wall = max_over_ranks(wall, world)
    value = ncell * args.steps / (ms * 1e-3) / 1e9
    e2e = ncell * args.steps / wall / 1e9
    three = None
    if args.with_3d:
        w3 = wl.config3_sphere_3d(n=args.n3, steps=500)
        ms3, _, _ = sharded_steps(w3, "fp32", args.steps3, 3, world, rank, stream)
        ms3 = max_over_ranks(ms3, world) / args.steps3
        three = {"workload": f"maxwell3d_sphere_{args.n3}", "steps_timed": args.steps3,
                 "slabs": world, "value_fp32": w3.ncell / (ms3 * 1e-3) / 1e9,
                 "ms_per_step_fp32": ms3,
                 "hbm_frac_fp32_per_gpu": 52 * w3.ncell / world / (ms3 * 1e-3) / 1e9 / _peaks()[0],
                 "algorithmic_bytes_per_cell_step": 52}
    if rank == 0:
        hbm, how = _peaks()
        ms_step = ms / args.steps
        achieved = BYTES_PER_CELL_STEP["fp32"] * ncell / world / (ms_step * 1e-3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"tm2d_cylinders_{n}", "grid": [n, n], "cylinders": 32,
                       "bc": "nonreflecting", "cfl": 0.5, "source": "line, f0=20",
                       "steps_config": 2000, "precision": "fp32",
                       "l2": "inputs larger than L2 per GPU for N <= 3 (state+eps read+write "
                             f"{BYTES_PER_CELL_STEP['fp32'] * ncell / world / 1e6:.0f} MB per GPU)",
                       "parallelism": f"slabs x{world} (y), 2 ghost rows per side, NCCL "
                                      "send/recv after every step"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_source": how, "traffic": None,
                         "kernel": "cart2d_step_kernel_s (staged FP32, mu = 1), per GPU, halo "
                                   "exchange included in the time",
                         "algorithmic_bytes_per_launch": BYTES_PER_CELL_STEP["fp32"] * ncell // world},
            "e2e": {"value": e2e, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * 3 * ncell / args.steps,
                    "d2h_bytes_per_step": 8 * 3 * ncell / args.steps,
                    "definition": "per rank write_fields(pinned FP64, its slab) + step(K) with "
                                  "halo exchange + read_fields, wall clock, slowest rank"},
            "gpu_launches": int(launches),
            "maxwell3d": three,
            "clocks": clocks,
            "note": "multi-GPU run: FP64, tets, adjoint, limiter, variants and cleaning legs "
                    "run at N = 1 only",
        }
        print(json.dumps(line))
    import torch.distributed as dist
    dist.barrier()
    dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gks", choices=["gks", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--with-3d", dest="with_3d", action="store_true", default=True)
    ap.add_argument("--no-3d", dest="with_3d", action="store_false")
    ap.add_argument("--n3", type=int, default=256)
    ap.add_argument("--steps3", type=int, default=100)
    ap.add_argument("--no-err3", dest="err3", action="store_false", default=True)
    ap.add_argument("--no-tets", dest="with_tets", action="store_false", default=True)
    ap.add_argument("--m4", type=int, default=64)
    ap.add_argument("--steps4", type=int, default=100)
    ap.add_argument("--no-err4", dest="err4", action="store_false", default=True)
    ap.add_argument("--no-cleaning", dest="with_cleaning", action="store_false", default=True)
    ap.add_argument("--no-limiter", dest="with_limiter", action="store_false", default=True)
    ap.add_argument("--no-variants", dest="with_variants", action="store_false", default=True)
    ap.add_argument("--no-adjoint", dest="with_adjoint", action="store_false", default=True)
    ap.add_argument("--n5", type=int, default=2048)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    from paper_2412_16845_gb300 import build as gbuild
    from paper_2412_16845_gb300 import workloads as wl
    from paper_2412_16845_gb300.gks import GKSSolver

    if rank == 0 and not os.path.exists(os.path.join(ROOT, "paper_2412_16845_gb300", "libgks.so")):
        gbuild.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
        dist.barrier()
        if rank != 0:
            gbuild.build()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    n = args.n
    w = wl.config2_cylinders_tm(n=n, steps=args.steps)
    ncell = n * n

    def barrier():
        if world > 1:
            dist.barrier()

    if world > 1:
        run_sharded(args, w, world, rank, local, stream)
        return

    # ---------------- FP32 device-resident timing
    s32 = GKSSolver.from_workload(w, precision="fp32", stream=sptr)
    s32.step(args.warmup)
    s32.sync()
    L0 = s32.launch_count()
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s32.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if rank == 0 else None
    ms = e0.elapsed_time(e1)
    launches = s32.launch_count() - L0
    ms = max_over_ranks(ms, world)
    value = job_throughput(ncell, args.steps, ms, world)
    ms_step = ms / args.steps

    # ---------------- FP64 path, FP32-vs-FP64 error after the configuration's step count
    steps_cfg = 2000
    s64 = GKSSolver.from_workload(w, precision="fp64", stream=sptr)
    s64.step(3)
    s64.sync()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    k64 = min(args.steps, 200)
    f0.record(stream)
    s64.step(k64)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1) / k64
    value64 = ncell / (ms64 * 1e-3) / 1e9
    a32 = GKSSolver.from_workload(w, precision="fp32", stream=sptr)
    a64 = GKSSolver.from_workload(w, precision="fp64", stream=sptr)
    a32.step(steps_cfg)
    a64.step(steps_cfg)
    r32 = a32.read_fields()
    r64 = a64.read_fields()
    err = float(np.sqrt(np.sum((r32 - r64) ** 2) / max(np.sum(r64 ** 2), 1e-300)))
    for s in (s64, a32, a64):
        s.close()

    # ---------------- end to end through the C ABI from pinned host memory
    host_in = torch.empty((3, ncell), dtype=torch.float64, pin_memory=True)
    host_in.copy_(torch.from_numpy(w.fields0))
    host_out = torch.empty((3, ncell), dtype=torch.float64, pin_memory=True)
    hin, hout = host_in.numpy(), host_out.numpy()
    s32.write_fields(hin)
    s32.step(2)
    s32.read_fields(hout)
    barrier()
    t0 = time.perf_counter()
    s32.write_fields(hin)
    s32.step(args.steps)
    s32.read_fields(hout)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e = job_throughput(ncell, args.steps, e2e_s * 1e3, world)
    s32.close()

    # ---------------- 3-D sphere workload (256^3): FP32 and FP64, error after its 500 steps
    three = None
    if args.with_3d:
        w3 = wl.config3_sphere_3d(n=args.n3, steps=500)
        n3 = w3.ncell
        t32 = GKSSolver.from_workload(w3, precision="fp32", stream=sptr)
        t32.step(3)
        t32.sync()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        k3 = args.steps3
        g0.record(stream)
        t32.step(k3)
        g1.record(stream)
        torch.cuda.synchronize()
        ms3 = g0.elapsed_time(g1) / k3
        t64 = GKSSolver.from_workload(w3, precision="fp64", stream=sptr)
        t64.step(1)
        t64.sync()
        g0.record(stream)
        t64.step(5)
        g1.record(stream)
        torch.cuda.synchronize()
        ms3_64 = g0.elapsed_time(g1) / 5
        t32.close()
        t64.close()
        err3 = None
        if args.err3:
            b32 = GKSSolver.from_workload(w3, precision="fp32", stream=sptr)
            b64 = GKSSolver.from_workload(w3, precision="fp64", stream=sptr)
            b32.step(500)
            b64.step(500)
            o32, o64 = b32.read_fields(), b64.read_fields()
            err3 = float(np.sqrt(np.sum((o32 - o64) ** 2) / np.sum(o64 ** 2)))
            b32.close()
            b64.close()
        three = {"workload": f"maxwell3d_sphere_{args.n3}", "steps_timed": k3,
                 "value_fp32": n3 / (ms3 * 1e-3) / 1e9, "ms_per_step_fp32": ms3,
                 "value_fp64": n3 / (ms3_64 * 1e-3) / 1e9, "ms_per_step_fp64": ms3_64,
                 "fp32_speedup": ms3_64 / ms3, "fp32_vs_fp64_rel_l2_after_500": err3,
                 "hbm_frac_fp32": 52 * n3 / (ms3 * 1e-3) / 1e9 / _peaks()[0],
                 "algorithmic_bytes_per_cell_step": 52,
                 "roofline": roofline_3d(n3, ms3)}

    # ---------------- tetrahedral sphere workload (64^3 x 6 Kuhn tets, jittered): FP32 and FP64
    tets = None
    if args.with_tets:
        w4 = wl.config4_tets(m=args.m4, steps=500)
        n4 = int(w4.tet.shape[0])
        q32 = GKSSolver.from_tet_workload(w4, precision="fp32", stream=sptr)
        q32.step(3)
        q32.sync()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        k4 = args.steps4
        h0.record(stream)
        q32.step(k4)
        h1.record(stream)
        torch.cuda.synchronize()
        ms4 = h0.elapsed_time(h1) / k4
        q64 = GKSSolver.from_tet_workload(w4, precision="fp64", stream=sptr)
        q64.step(1)
        q64.sync()
        h0.record(stream)
        q64.step(10)
        h1.record(stream)
        torch.cuda.synchronize()
        ms4_64 = h0.elapsed_time(h1) / 10
        q32.close()
        q64.close()
        err4 = None
        if args.err4:
            b32 = GKSSolver.from_tet_workload(w4, precision="fp32", stream=sptr)
            b64 = GKSSolver.from_tet_workload(w4, precision="fp64", stream=sptr)
            b32.step(500)
            b64.step(500)
            o32, o64 = b32.read_fields(), b64.read_fields()
            err4 = float(np.sqrt(np.sum((o32 - o64) ** 2) / np.sum(o64 ** 2)))
            b32.close()
            b64.close()
        tets = {"workload": f"tets_sphere_{args.m4}", "tets": n4, "steps_timed": k4,
                "value_fp32": n4 / (ms4 * 1e-3) / 1e9, "ms_per_step_fp32": ms4,
                "value_fp64": n4 / (ms4_64 * 1e-3) / 1e9, "ms_per_step_fp64": ms4_64,
                "fp32_speedup": ms4_64 / ms4, "fp32_vs_fp64_rel_l2_after_500": err4,
                "algorithmic_bytes_per_tet_step": 229,
                "hbm_frac_fp32": 229 * n4 / (ms4 * 1e-3) / 1e9 / _peaks()[0]}

    # ---------------- van Leer limiter: the cylinder workload with limited slopes (FP32)
    limited = None
    if args.with_limiter:
        wlim = dataclasses.replace(wl.config2_cylinders_tm(n=n, steps=args.steps),
                                   limiter="vanleer")
        ls = GKSSolver.from_workload(wlim, precision="fp32", stream=sptr)
        ls.step(3)
        ls.sync()
        kl = min(args.steps, 500)
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        ls.step(kl)
        l1.record(stream)
        torch.cuda.synchronize()
        msl = l0.elapsed_time(l1) / kl
        ls.close()
        limited = {"workload": f"tm2d_cylinders_{n}_vanleer", "steps_timed": kl,
                   "value_fp32": ncell / (msl * 1e-3) / 1e9, "ms_per_step_fp32": msl}

    # ---------------- boundary and source variants of the 2-D step (FP32, 500 steps each):
    # PEC walls on all four sides (the cylinder grid as a closed cavity, Sec. 5.5) and the two
    # oscillating dipoles of Sec. 5.4 on a 2n x n grid
    variants = None
    if args.with_variants:
        variants = {}
        cases = [("pec_walls", dataclasses.replace(wl.config2_cylinders_tm(n=n, steps=args.steps),
                                                   bc=("pec",) * 4)),
                 ("dipole", wl.dipole_tm(n=n // 2, two=True))]
        for key, wv in cases:
            sv = GKSSolver.from_workload(wv, precision="fp32", stream=sptr)
            sv.step(3)
            sv.sync()
            kv = min(args.steps, 500)
            v0e = torch.cuda.Event(enable_timing=True)
            v1e = torch.cuda.Event(enable_timing=True)
            v0e.record(stream)
            sv.step(kv)
            v1e.record(stream)
            torch.cuda.synchronize()
            msv = v0e.elapsed_time(v1e) / kv
            sv.close()
            nv = int(np.prod(wv.n))
            variants[key] = {"workload": wv.name + ("_pec" if key == "pec_walls" else ""),
                             "grid": list(wv.n), "steps_timed": kv,
                             "value_fp32": nv / (msv * 1e-3) / 1e9, "ms_per_step_fp32": msv}

    # ---------------- divergence cleaning (TM + psi, gamma = 1, CFL 0.4) on the cylinder grid
    cleaning = None
    if args.with_cleaning:
        wc = wl.config2_cylinders_tm(n=n, steps=args.steps)
        wc.cfl, wc.phm, wc.fields0 = 0.4, (0.0, 1.0), np.zeros((4, ncell))
        c32 = GKSSolver.from_workload(wc, precision="fp32", stream=sptr)
        c32.step(3)
        c32.sync()
        kc = min(args.steps, 500)
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        c32.step(kc)
        k1.record(stream)
        torch.cuda.synchronize()
        msc = k0.elapsed_time(k1) / kc
        c32.close()
        cleaning = {"workload": f"tm2d_cylinders_{n}_cleaning", "gamma": 1.0, "cfl": 0.4,
                    "steps_timed": kc, "value_fp32": ncell / (msc * 1e-3) / 1e9,
                    "ms_per_step_fp32": msc, "algorithmic_bytes_per_cell_step": 36,
                    "hbm_frac_fp32": 36 * ncell / (msc * 1e-3) / 1e9 / _peaks()[0]}
        if args.with_3d:
            # 3-D: (E, H, phi, psi) on the sphere grid, chi = gamma = 1, CFL 0.3
            nq = n3
            wq = dataclasses.replace(w3, cfl=0.3, phm=(1.0, 1.0),
                                     fields0=np.concatenate([w3.fields0, np.zeros((2, nq))]))
            q = GKSSolver.from_workload(wq, precision="fp32", stream=sptr)
            q.step(3)
            q.sync()
            kq = args.steps3
            k0.record(stream)
            q.step(kq)
            k1.record(stream)
            torch.cuda.synchronize()
            msq = k0.elapsed_time(k1) / kq
            q.close()
            cleaning["maxwell3d"] = {
                "workload": f"maxwell3d_sphere_{args.n3}_cleaning", "chi": 1.0, "gamma": 1.0,
                "cfl": 0.3, "steps_timed": kq, "value_fp32": nq / (msq * 1e-3) / 1e9,
                "ms_per_step_fp32": msq, "algorithmic_bytes_per_cell_step": 68,
                "hbm_frac_fp32": 68 * nq / (msq * 1e-3) / 1e9 / _peaks()[0]}

    # ---------------- adjoint: eps-gradient of the probe objective, 2048^2 design workload
    adj = None
    if args.with_adjoint:
        from paper_2412_16845_gb300.adjoint import DesignProblem
        w5 = wl.config5_design_tm(n=args.n5, steps=2000)
        plain = GKSSolver.from_workload(w5, precision="fp32", stream=sptr)
        plain.step(3)
        plain.sync()
        t0 = time.perf_counter()
        plain.step(2000)
        plain.sync()
        t_plain = time.perf_counter() - t0
        plain.close()
        prob = DesignProblem(w5, precision="fp32", checkpoint_every=45, stream=stream)
        e0 = w5.eps[w5.design]
        prob.forward(e0)                       # warm-up of the whole path
        prob.backward()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = prob.forward(e0)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        t0 = time.perf_counter()
        g = prob.backward()
        torch.cuda.synchronize()
        t_bwd = time.perf_counter() - t0
        prob.close()
        adj = {"workload": f"tm2d_design_{args.n5}", "steps": 2000, "checkpoint_every": 45,
               "design_cells": int(w5.design.size), "probe_cells": int(w5.probe.size),
               "forward_plain_s": t_plain, "forward_with_checkpoints_s": t_fwd,
               "backward_s": t_bwd, "adjoint_over_forward": t_bwd / t_plain,
               "gradient_over_forward": (t_fwd + t_bwd) / t_plain, "J": J,
               "grad_norm": float(g.norm())}

    if rank == 0:
        divergence = divergence_report(sptr)
        hbm, how = _peaks()
        achieved = BYTES_PER_CELL_STEP["fp32"] * ncell / (ms_step * 1e-3) / 1e9
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"tm2d_cylinders_{n}", "grid": [n, n], "cylinders": 32,
                       "bc": "nonreflecting", "cfl": 0.5, "source": "line, f0=20",
                       "steps_config": steps_cfg, "precision": "fp32",
                       "l2": "inputs larger than L2 (state+eps read+write per step "
                             f"{BYTES_PER_CELL_STEP['fp32'] * ncell / 1e6:.0f} MB > 129 MB)",
                       "parallelism": "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_source": how,
                         "traffic": _profiled_traffic(),
                         "kernel": "cart2d_step_kernel_s (staged FP32, mu = 1)",
                         "algorithmic_bytes_per_launch": BYTES_PER_CELL_STEP["fp32"] * ncell},
            "fp64": {"value": value64, "ms_per_step": ms64, "unit": UNIT,
                     "fp32_speedup": value / world / value64},
            "fp32_vs_fp64_rel_l2": {"value": err, "after_steps": steps_cfg},
            "e2e": {"value": e2e, "unit": UNIT,
                    "h2d_bytes_per_step": 8 * 3 * ncell / args.steps,
                    "d2h_bytes_per_step": 8 * 3 * ncell / args.steps,
                    "definition": "write_fields(pinned FP64) + step(K) + read_fields, wall clock"},
            "gpu_launches": int(launches),
            "maxwell3d": three,
            "tets": tets,
            "limiter": limited,
            "variants": variants,
            "cleaning": cleaning,
            "adjoint": adj,
            "divergence": divergence,
            "clocks": clocks,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(all_cores=True)
            # the same oracle leg checks the FP32 and FP64 GPU paths on reduced workloads
            import tempfile
            with tempfile.TemporaryDirectory() as td:
                pth = os.path.join(td, "gpu_reduced.npz")
                reduced_gpu_results(sptr, pth)
                line["fp32_vs_oracle"] = oracle_errors(pth)
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

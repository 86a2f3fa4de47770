#!/usr/bin/env python
"""Benchmark of the GB300 imaging path: reconstructed voxels/s.

A step is one whole image (every stage of the path: reference plane,
geometry and binning, compensation, Gaussian gridding, FT_2D, k_z filter +
Stolt, inverse FT) of one synthetic scan already resident in HBM.  The
default workload is the single realistic scan: 2 Tx x 4 Rx, 128 x 128
random-walk serpentine positions, Nk = 256, imaged onto 256 x 256 x 64
voxels (echo 268 MB, larger than the 129 MB L2, so no flush is needed
between steps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank images its own scan (independent scans:
weak scaling, no collective on the data path); the time is the maximum
over ranks and ``value`` counts the voxels of all ranks.

``--impl reference`` times the FP64 CPU oracle (the only reference this
path has) on the host cores, each step one whole image of the same scan.

At N = 1 the line also carries the oracle timings on the host cores
(``oracle_timings``: exact and fast oracle on the tiny scan, direct
back-projection on the tiny scan in full and on a voxel sample of the
realistic scan) and, unless ``--no-extras``, compact records of the other
workloads: ``batch`` (the 64-scan uneven mix), ``serve`` (Poisson stream,
FP16-stored served form against the plain FP32 form) and ``large_storage``
(the large scan with FP32, FP16 and BF16 echo storage against the oracle).
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reconstructed voxels/s at <=1e-4 NMSE vs the FP64 oracle (realistic single scan)"
UNIT = "voxels/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["realistic", "tiny", "large", "batch", "serve", "psf"], default="realistic")
    ap.add_argument("--compensate", type=int, choices=[0, 1, 2], default=1,
                    help="1: Eq. 11-12 (the paper's residual), 2: Eq. 5 at the scene centre, 0: none (ablation)")
    ap.add_argument("--mix", type=int, default=64, help="scans in the batched mix")
    ap.add_argument("--requests", type=int, default=256, help="requests in the serving run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-traffic", default=None, metavar="CSV",
                    help="write profiles/ncu_traffic.json from an ncu launch list (CSV) and exit")
    ap.add_argument("--ncu-command", default="", help="the command that produced --ncu-traffic's CSV")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds the reference arm's warm-up and timed steps may take together")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batch / serve / large_storage records of the default run")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default gridding launch shape")
    ap.add_argument("--tiles", default=None,
                    help="gridding form 'nf,warps,grouped[,tensor_cores]' instead of the autotuner's "
                         "(single-scan workloads; '2,4,0,v' = tensor cores, pipeline v = 1..4)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
class Dist:
    def __init__(self, want_cuda: bool):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = False
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if (want_cuda and torch.cuda.is_available()) else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local_rank)
            dist.init_process_group(backend=backend)
            self.backend = backend
            self.pg = True

    def barrier(self):
        if self.pg:
            import torch.distributed as dist
            if self.backend == "nccl":
                import torch
                dist.barrier(device_ids=[self.local_rank])
            else:
                dist.barrier()

    def max(self, x: float) -> float:
        return self._reduce(x, "max")

    def sum(self, x: float) -> float:
        return self._reduce(x, "sum")

    def _reduce(self, x, op):
        if not self.pg:
            return x
        import torch
        import torch.distributed as dist
        dev = f"cuda:{self.local_rank}" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            import torch.distributed as dist
            dist.destroy_process_group()


# ----------------------------------------------------------------------------- workloads
LARGE_POINTS = 200   # scatterers of the large scene (echo synthesis cost grows with them; imaging does not)


def make_scan(workload: str, rank: int):
    import synth
    if workload == "tiny":
        return synth.tiny(seed=rank)
    if workload == "large":
        return synth.large(seed=5000 + rank, n_points=LARGE_POINTS)
    return synth.realistic(seed=2000 + rank)


def plan_geometry(scan, nufft_tol=1e-3):
    """Kernel width and spectral grid the library's plan picks for a scan
    with default options (the same rules, restated for reporting only: the
    smallest Gaussian width whose gridding error is within the tolerance,
    and the next power of two >= the voxel count per axis, at least 16)."""
    errs = {4: 4.8e-3, 5: 1.4e-3, 6: 5.5e-4, 7: 1.5e-4, 8: 5.4e-5, 9: 1.6e-5, 10: 4.4e-6, 11: 1.3e-6, 12: 3.5e-7}
    w = next((k for k in sorted(errs) if errs[k] <= nufft_tol), 12)
    p2 = lambda n: max(16, 1 << max(0, (n - 1).bit_length()))
    return {"kernel_width": w, "spectral_grid": [p2(scan.grid.nx), p2(scan.grid.ny)], "nufft_tol": nufft_tol}


def workload_config(scan, workload, plan=None):
    T, R, P, Nk = scan.echo.shape
    g = scan.grid
    cfg = {"workload": {"tiny": "tiny: 1Tx x 2Rx, 16x16 jittered positions, Nk=32 -> 32x32x16",
                        "realistic": "realistic single scan: 2Tx x 4Rx, 128x128 random-walk serpentine, "
                                     "Nk=256 -> 256x256x64 complex64",
                        "large": f"large: 3Tx x 4Rx, 256x256 positions, Nk=512 -> 512x512x128 "
                                 f"({LARGE_POINTS} scatterers)"}[workload],
           "tx_rx_pos_k": [T, R, P, Nk], "voxels": [g.nx, g.ny, g.nz],
           "echo_bytes": int(scan.echo.nbytes), "l2": "inputs larger than L2 (no flush)"
           if scan.echo.nbytes > 129e6 else "L2 flushed between steps",
           "dtype_storage": "complex64", "parallelism": "independent scans per GPU (replicas)"}
    if plan is not None:
        cfg.update({"kernel_width": plan.kernel_width, "spectral_grid": [plan.mx, plan.my],
                    "nufft_tol": plan.opt.nufft_tol})
    else:
        cfg.update(plan_geometry(scan))
    return cfg


def host_cpu():
    """(model name, logical cores) of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return model or platform.processor() or platform.machine(), os.cpu_count() or 1


def oracle_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 20):
        self.gpu = gpu_index
        self.period_ms = period_ms
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", str(self.period_ms)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[5:]))
            except Exception:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        window = "timed region"
        if not inside:
            inside, window = rows, f"whole run (timed region shorter than the {self.period_ms} ms sampling period)"
        reasons = set()
        for r in inside:
            active = r[3]
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, active[1:5]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


# ----------------------------------------------------------------------------- roofline model
def occupied_window(plan, scan):
    """Cells of the 2Mx x 2My gridding grid that can be nonzero (the same rule
    the library applies on the device): the span of the samples' first taps
    plus the kernel width, capped at the grid size."""
    import numpy as np
    pos, tx, rx = (np.asarray(a, np.float64).reshape(-1, 3) for a in (scan.pos, scan.tx, scan.rx))
    if pos.shape[0] == 0:
        return 0, 0
    T = pos[None, None] + tx[:, None, None]
    R = pos[None, None] + rx[None, :, None]
    xv = 0.5 * (T[..., 0] + R[..., 0])
    yv = 0.5 * (T[..., 1] + R[..., 1])
    g = scan.grid
    xc, yc = g.x0 + (g.nx // 2) * g.dx, g.y0 + (g.ny // 2) * g.dy
    w = plan.kernel_width
    u0 = np.ceil(2 * (xv - xc) / g.dx - w / 2)
    v0 = np.ceil(2 * (yv - yc) / g.dy - w / 2)
    ul = min(2 * plan.mx, int(u0.max() - u0.min()) + w)
    vl = min(2 * plan.my, int(v0.max() - v0.min()) + w)
    return ul, vl


def stage_bytes(plan, scan):
    """Algorithmic HBM bytes of each stage: the compulsory reads and writes of
    the data it transforms, counting only the occupied window of the
    gridding grid (the rest is known zero and never touched)."""
    T, R, P, Nk = scan.echo.shape
    L = T * R * P
    nkp = ((Nk + 31) // 32) * 32
    mx, my = plan.mx, plan.my
    ul, vl = occupied_window(plan, scan)
    nx, ny, nz = scan.grid.nx, scan.grid.ny, scan.grid.nz
    c = 8  # complex64
    echo = L * Nk * c
    shat = L * nkp * c
    G = vl * ul * nkp * c          # occupied cells of the gridding grid
    A = vl * mx * nkp * c          # occupied rows after the FFT along x'
    S = mx * my * nkp * c
    Z = mx * my * nz * c
    B = mx * ny * nz * c
    V = nx * ny * nz * c
    if plan.tiles[3]:
        # tensor-core form: s_hat as FP16 hi / lo planes (the same bytes as
        # complex64), a 16-byte record per sample (bin order) and one
        # normalisation exponent byte per sample
        rec = 16 + 1
    else:
        rec = (2 * (plan.kernel_width + 3) + 1) * 16 + 8   # weight record + (in-bin offset, sample index)
    # prep: geometry records, phases, bin ids, permutation; compensate: echo
    # in, s_hat out, phases, and (same launch) the in-bin sort and records
    return {"prep": L * 36 + 24 * P, "compensate": echo + shat + L * 8 + L * (24 + rec), "grid": shat + G + L * rec,
            "fft_x": G + A, "fft_y": A + S, "stolt": S + Z, "ifft_y": Z + B, "ifft_x": B + V}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def csrc_digest(files=None):
    """sha256 (first 16 hex digits) of the given source files (paths relative
    to the repository root), or of every file under the package's csrc/."""
    h = hashlib.sha256()
    if files is None:
        files = sorted(os.path.relpath(p, ROOT) for p in glob.glob(os.path.join(ROOT, "paper_2305_02064_gb300",
                                                                               "csrc", "*")))
    for p in files:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


# kernels of one image in launch order, by stage (name fragments of the kernels)
STAGE_SOURCES = {
    "compensate": ["paper_2305_02064_gb300/csrc/samples.cu"],
    "grid": ["paper_2305_02064_gb300/csrc/spread.cu", "paper_2305_02064_gb300/csrc/grid_tc.cu"],
    "fft_x": ["paper_2305_02064_gb300/csrc/fft_kernels.cu"],
    "fft_y": ["paper_2305_02064_gb300/csrc/fft_kernels.cu"],
    "stolt": ["paper_2305_02064_gb300/csrc/stolt.cu"],
    "ifft_y": ["paper_2305_02064_gb300/csrc/fft_kernels.cu"],
    "ifft_x": ["paper_2305_02064_gb300/csrc/fft_kernels.cu"],
}
COMMON_SOURCES = ["paper_2305_02064_gb300/csrc/fft.cuh", "paper_2305_02064_gb300/csrc/internal.cuh",
                  "include/mmsar.h"]


def stage_of_kernel(name: str, fft_seen: int):
    """Stage of a kernel of the imaging sequence (None for prep kernels);
    the column FFT kernel serves four stages, told apart by launch order."""
    if "compensate" in name:
        return "compensate"
    if "spread" in name or "grid_tc" in name or "grid_ws" in name:
        return "grid"
    if "stolt" in name:
        return "stolt"
    if "column_fft" in name:
        return ("fft_x", "fft_y", "ifft_y", "ifft_x")[fft_seen % 4]
    return None


def write_ncu_traffic(csv_path: str, command: str, workload: str = "realistic"):
    """profiles/ncu_traffic.json from an ncu launch list taken with
    --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
    --csv: per stage the DRAM bytes (read + write) and time of its kernel in
    the last complete image of the list, with the digest of the sources that
    kernel is built from (so the bench uses it only while they are unchanged)."""
    import csv
    launches = {}
    order = []
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        lid = row["ID"]
        if lid not in launches:
            launches[lid] = {"kernel": row["Kernel Name"], "m": {}}
            order.append(lid)
        v = row["Metric Value"].replace(",", "")
        unit = row.get("Metric Unit", "")
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-3, "ns": 1e-3, "usecond": 1.0,
                 "us": 1.0, "msecond": 1e3, "ms": 1e3}.get(unit, 1)   # times in us
        launches[lid]["m"][row["Metric Name"]] = float(v) * scale
    # the last image: from the last prep launch (zref) on
    starts = [i for i, lid in enumerate(order) if "zref" in launches[lid]["kernel"]]
    stages = {}
    for st in starts[::-1]:
        seq, fft_seen = {}, 0
        for lid in order[st:]:
            k = launches[lid]["kernel"]
            stage = stage_of_kernel(k, fft_seen)
            if "column_fft" in k:
                fft_seen += 1
            if stage and stage not in seq:
                seq[stage] = launches[lid]
        if len(seq) == len(STAGE_SOURCES):
            stages = seq
            break
    out = {"workload": workload, "command": command,
           "note": "dram__bytes_read.sum + dram__bytes_write.sum of each kernel in the last complete image of the "
                   "launch list; sha = digest of the listed sources the kernel is built from",
           "stages": {}}
    for stage, l in stages.items():
        srcs = [p for p in STAGE_SOURCES[stage] if os.path.exists(os.path.join(ROOT, p))] + COMMON_SOURCES
        m = l["m"]
        out["stages"][stage] = {"kernel": l["kernel"][:60], "sources": srcs, "sha": csrc_digest(srcs),
                                "dram_bytes_per_launch": m.get("dram__bytes_read.sum", 0) +
                                m.get("dram__bytes_write.sum", 0),
                                "us": m.get("gpu__time_duration.sum", 0)}
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
    return out


def ncu_traffic(stage: str, workload: str):
    """DRAM bytes per launch of a stage's kernel from the committed ncu
    summary, if it was taken on the current sources of that kernel (the
    files listed with it) and on the same workload; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
        e = d["stages"][stage]
        if d.get("workload") != workload or e.get("sha") != csrc_digest(e["sources"]):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


# ----------------------------------------------------------------------------- ours
def run_ours(args, dist):
    import numpy as np
    import torch
    import paper_2305_02064_gb300 as mm

    dev = torch.device(f"cuda:{dist.local_rank}")
    torch.cuda.set_device(dev)
    scan = make_scan(args.workload, dist.rank)
    plan = mm.Plan.for_scan(scan, compensate=args.compensate)
    stream = torch.cuda.Stream(device=dev)
    ws = plan.new_workspace(dev)
    vol = plan.new_volume(dev)
    echo_h = torch.from_numpy(np.ascontiguousarray(scan.echo)).pin_memory()
    pos_h = torch.from_numpy(np.ascontiguousarray(scan.pos, np.float64)).pin_memory()
    tx_h = torch.from_numpy(np.ascontiguousarray(scan.tx, np.float64)).pin_memory()
    rx_h = torch.from_numpy(np.ascontiguousarray(scan.rx, np.float64)).pin_memory()
    echo, pos, tx, rx = (t.to(dev) for t in (echo_h, pos_h, tx_h, rx_h))
    vol_h = torch.empty(vol.shape, dtype=vol.dtype).pin_memory()
    torch.cuda.synchronize(dev)
    # the autotuner picks the gridding launch shape on this scan (untimed)
    tuned = None
    if args.tiles:
        plan.set_tiles(*(int(v) for v in args.tiles.split(",")))
    elif not args.no_autotune:
        from paper_2305_02064_gb300.tune import autotune
        tuned = autotune(plan, ws, echo, pos, tx, rx, vol, stream=stream)
        torch.cuda.synchronize(dev)

    def step():
        plan.image(ws, echo, pos, tx, rx, vol, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    plan.poll_error(ws, stream=stream)

    n_stage = len(plan.stage_names())
    n_ev = min(args.steps, 50)
    evsets = [[torch.cuda.Event(enable_timing=True) for _ in range(n_stage + 1)] for _ in range(n_ev)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device() if not os.environ.get("CUDA_VISIBLE_DEVICES")
                          else int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[dist.local_rank]))
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize(dev)
    w0 = time.time()
    t_start.record(stream)
    for i in range(args.steps):
        if i < n_ev:
            plan.set_stage_events(evsets[i])
        elif i == n_ev:
            plan.set_stage_events(None)
        step()
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    w1 = time.time()
    dist.barrier()
    plan.set_stage_events(None)
    clk = clocks.stop(w0, w1)
    plan.poll_error(ws, stream=stream)
    # a sustained window after the timed region (not timed): about a second of
    # the same steps with the clocks sampled, for runs whose timed region is
    # short against the sampling period
    sustained = ClockSampler(clocks.gpu)
    sustained.start()
    time.sleep(0.2)
    torch.cuda.synchronize(dev)
    n_sus = max(1, int(1.0 / max(t_start.elapsed_time(t_end) / args.steps * 1e-3, 1e-6)))
    s0 = time.time()
    for _ in range(n_sus):
        step()
    torch.cuda.synchronize(dev)
    s1 = time.time()
    clk_sustained = sustained.stop(s0, s1)
    if clk_sustained is not None:
        clk_sustained["steps"] = n_sus
    ms = t_start.elapsed_time(t_end) / args.steps
    ms_max = dist.max(ms)

    names = plan.stage_names()
    stage_ms = {n: statistics.mean(ev[s].elapsed_time(ev[s + 1]) for ev in evsets) for s, n in enumerate(names)}
    per_image = sorted(ev[0].elapsed_time(ev[-1]) for ev in evsets)
    nb = stage_bytes(plan, scan)
    peak_gbs, peak_kind = measured_peaks()
    dom = max(stage_ms, key=stage_ms.get)
    achieved = nb[dom] / (stage_ms[dom] * 1e-3) / 1e9

    # end to end through the public API from pinned host buffers.  Serial:
    # every step copies its inputs in, images, copies the volume out, on one
    # stream.  Pipelined (the form a scan stream would use): step i's inputs
    # go in on a copy stream while step i-1 images on the compute stream and
    # step i-2's volume comes back on a third stream (two buffer sets).
    e2e_steps = max(3, args.e2e_steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for i in range(e2e_steps + 1):
            if i == 1:
                e0.record(stream)
            echo.copy_(echo_h, non_blocking=True)
            pos.copy_(pos_h, non_blocking=True)
            tx.copy_(tx_h, non_blocking=True)
            rx.copy_(rx_h, non_blocking=True)
            step()
            vol_h.copy_(vol, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_serial_ms = dist.max(e0.elapsed_time(e1) / e2e_steps)

    bufs = [(echo, pos, tx, rx, vol, vol_h)]
    bufs.append((torch.empty_like(echo), torch.empty_like(pos), torch.empty_like(tx), torch.empty_like(rx),
                 torch.empty_like(vol), torch.empty_like(vol_h, device="cpu").pin_memory()))
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(e2e_steps + 2):
        b = i % 2
        e_d, p_d, t_d, r_d, v_d, v_h = bufs[b]
        with torch.cuda.stream(s_in):
            if i == 2:
                p0.record(s_in)
            if i >= 2:
                s_in.wait_event(ev_comp[b])     # step i-2 has consumed these inputs
            e_d.copy_(echo_h, non_blocking=True)
            p_d.copy_(pos_h, non_blocking=True)
            t_d.copy_(tx_h, non_blocking=True)
            r_d.copy_(rx_h, non_blocking=True)
            ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        if i >= 2:
            stream.wait_event(ev_out[b])        # step i-2's volume has left
        plan.image(ws, e_d, p_d, t_d, r_d, v_d, stream=stream)
        ev_comp[b].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[b])
            v_h.copy_(v_d, non_blocking=True)
            ev_out[b].record(s_out)
    p1.record(s_out)
    torch.cuda.synchronize(dev)
    # p0 .. p1 spans steps 2 .. e2e_steps + 1 (the first two fill the pipeline)
    e2e_ms = dist.max(p0.elapsed_time(p1) / e2e_steps)
    h2d = echo_h.nbytes + pos_h.nbytes + tx_h.nbytes + rx_h.nbytes
    d2h = vol_h.nbytes

    voxels = scan.grid.n_voxels
    total_vox = voxels * dist.world
    res = {
        "metric": METRIC, "value": total_vox / (ms_max * 1e-3), "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fp32 (complex64 storage, fp64 per-sample phase)",
        "data": "synthetic (seeded scans shaped like the paper's workloads)",
        "config": workload_config(scan, args.workload, plan),
        "images_per_s": dist.world / (ms_max * 1e-3),
        "latency_ms": {"p50": per_image[len(per_image) // 2], "p99": per_image[min(len(per_image) - 1,
                                                                                    int(0.99 * len(per_image)))],
                       "what": "device time of one image, back to back"},
        "stages_ms": stage_ms,
        "stages_gbs": {n: nb[n] / (stage_ms[n] * 1e-3) / 1e9 for n in names},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                     "frac": achieved / peak_gbs, "peak_kind": f"{peak_kind} (copy bandwidth)",
                     "traffic": ncu_traffic(dom, args.workload), "algorithmic_bytes": nb[dom]},
        "e2e": {"value": total_vox / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms,
                "form": "pipelined: copy in / image / copy out of successive steps on three streams",
                "serial_ms_per_step": e2e_serial_ms, "serial_value": total_vox / (e2e_serial_ms * 1e-3)},
        "gpu_launches": plan.kernels_per_image * args.steps,
        "clocks": clk,
        "clocks_sustained": clk_sustained,
        "grid_launch_shape": {"tensor_cores": plan.tiles[3], "freqs_per_lane": plan.tiles[0],
                              "warps_per_cta": plan.tiles[1], "grouped": plan.tiles[2],
                              "autotuned_ms": None if tuned is None else
                              {(f"tc{t}" if t else f"{a}x{b}{'g' if c else ''}"): round(v, 4)
                               for (a, b, c, t), v in tuned["ms"].items()}},
    }
    return res, scan, vol


def cpu_baseline(scan, vol_gpu, compensate=1):
    """The FP64 oracle (rma_fast) on the whole scan, timed on the host cores;
    also the NMSE of the GPU volume against it."""
    import numpy as np
    from oracle import rma
    su = rma.setup_from(scan, compensate=compensate)
    t0 = time.time()
    ref = rma.rma_fast(su)
    dt = time.time() - t0
    got = vol_gpu.cpu().numpy()
    cores = oracle_cores()
    return ({"value": scan.grid.n_voxels / dt, "unit": UNIT, "cores": cores, "cpu_model": host_cpu()[0],
             "kind": "oracle",
             "sample": "one whole scan of the workload through oracle.rma.rma_fast (FP64 Gaussian gridding w=16, "
                       "OpenMP + scipy.fft workers on all cores)", "seconds": dt},
            {"nmse_vs_oracle": float(rma.nmse(got, ref)), "peak_match": rma.peak_index(got) == rma.peak_index(ref)})


def storage_comparison(scan, vol_fp32, args):
    """BF16 and FP16 echo storage against FP32 storage and the FP64 oracle on
    the same scan: per-image device time and NMSE (Gaussian gridding oracle,
    w = 12, relative error ~1e-6 per transform)."""
    import numpy as np
    import torch
    import paper_2305_02064_gb300 as mm
    from oracle import rma
    dev = vol_fp32.device
    echo = torch.from_numpy(np.ascontiguousarray(scan.echo)).to(dev)
    pos, tx, rx = (torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev) for a in (scan.pos, scan.tx, scan.rx))
    out = {}
    vols = {"fp32": vol_fp32.cpu().numpy()}
    for dt in ("bf16", "f16"):
        plan = mm.Plan.for_scan(scan, dtype=dt, compensate=args.compensate)
        q, sc = mm.quantize_echo(echo, dt)
        ws, vol = plan.new_workspace(dev), plan.new_volume(dev)
        for _ in range(3):
            plan.image(ws, q, pos, tx, rx, vol, echo_scale=sc)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        n = max(3, args.steps // 10)
        for _ in range(n):
            plan.image(ws, q, pos, tx, rx, vol, echo_scale=sc)
        e1.record()
        torch.cuda.synchronize(dev)
        plan.poll_error(ws)
        out[dt] = {"ms_per_image": e0.elapsed_time(e1) / n}
        vols[dt] = vol.cpu().numpy()
        del ws, q
    t0 = time.time()
    ref = rma.rma_fast(rma.setup_from(scan, compensate=args.compensate), w=12)
    oracle_s = time.time() - t0
    for k, v in vols.items():
        out.setdefault(k, {})["nmse_vs_oracle"] = float(rma.nmse(v, ref))
        out[k]["peak_match"] = rma.peak_index(v) == rma.peak_index(ref)
    for k in ("bf16", "f16"):
        out[k]["nmse_vs_fp32"] = float(rma.nmse(vols[k], vols["fp32"]))
    out["oracle_seconds"] = oracle_s
    return out


def oracle_timings(scan_realistic, n_sample_voxels=16):
    """The oracles timed on the host cores (OpenMP on every core): on the
    tiny scan the exact oracle, the fast oracle and the direct
    back-projection over its whole volume; on the realistic scan the direct
    back-projection at a voxel sample (the voxels of its first scatterers
    plus seeded random voxels), reported per voxel with the full-volume time
    extrapolated from it (labelled as such)."""
    import numpy as np
    import synth
    from oracle import bpa, rma
    out = {"cores": oracle_cores(), "cpu_model": host_cpu()[0]}
    tiny = synth.tiny()
    su = rma.setup_from(tiny)
    for name, fn in (("rma_exact_tiny_s", lambda: rma.rma_exact(su)), ("rma_fast_tiny_s", lambda: rma.rma_fast(su)),
                     ("bpa_tiny_full_s", lambda: bpa.bpa(tiny))):
        t0 = time.time()
        fn()
        out[name] = time.time() - t0
    g = scan_realistic.grid
    rng = np.random.default_rng(17)
    half = n_sample_voxels // 2
    near = []
    for x, y, z, _ in scan_realistic.scatterers[:half]:
        i, j, q = g.centre_index(x, y, z)
        near.append((i * g.ny + j) * g.nz + q)
    idx = np.unique(np.concatenate([np.asarray(near, np.int64),
                                    rng.integers(0, g.n_voxels, n_sample_voxels - len(near))]))
    t0 = time.time()
    bpa.bpa(scan_realistic, idx)
    dt = time.time() - t0
    out["bpa_realistic_sample"] = {"voxels": int(idx.size), "seconds": dt, "s_per_voxel": dt / idx.size,
                                   "full_volume_s_extrapolated": dt / idx.size * g.n_voxels,
                                   "note": "extrapolated linearly from the sample to all 256x256x64 voxels"}
    return out


def run_large_storage(args, dist):
    """The large scan (3 Tx x 4 Rx, 256 x 256 positions, Nk = 512 ->
    512 x 512 x 128 voxels) imaged with FP32, FP16 and BF16 echo storage;
    device ms per image and NMSE against the FP64 oracle for each."""
    import numpy as np
    import torch
    import paper_2305_02064_gb300 as mm
    dev = torch.device(f"cuda:{dist.local_rank}")
    scan = make_scan("large", dist.rank)
    plan = mm.Plan.for_scan(scan, compensate=args.compensate)
    echo = torch.from_numpy(np.ascontiguousarray(scan.echo)).to(dev)
    pos, tx, rx = (torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev) for a in (scan.pos, scan.tx, scan.rx))
    ws, vol = plan.new_workspace(dev), plan.new_volume(dev)
    for _ in range(3):
        plan.image(ws, echo, pos, tx, rx, vol)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(3, args.steps // 10)
    e0.record()
    for _ in range(n):
        plan.image(ws, echo, pos, tx, rx, vol)
    e1.record()
    torch.cuda.synchronize(dev)
    plan.poll_error(ws)
    fp32_ms = e0.elapsed_time(e1) / n
    del ws, echo
    out = storage_comparison(scan, vol, args)
    out.setdefault("fp32", {})["ms_per_image"] = fp32_ms
    out["fp32"]["voxels_per_s"] = scan.grid.n_voxels / (fp32_ms * 1e-3)
    out["workload"] = workload_config(scan, "large", plan)["workload"]
    out["oracle"] = "oracle.rma.rma_fast, FP64 Gaussian gridding w=12 (relative error ~1e-6 per transform)"
    return out


# ----------------------------------------------------------------------------- reference (oracle) arm
def run_reference(args, dist):
    """The oracle (FP64, as it stands) on the host cores.  One whole image of
    the scan is timed once (after one untimed run) and reported as
    whole_scan_seconds; the K timed steps (after W untimed ones) are bounded
    samples sized so that all K + W end within about --ref-budget seconds: the
    whole scan while it fits, else the first nk' of its Nk frequencies and,
    where that is still too long, the first P' of its positions (the image is
    linear in both).  The oracle's cost is not proportional to either (a
    per-image part does not depend on them), so a sample's time is scaled by
    the measured ratio of one whole image to one sample image, timed back to
    back."""
    import dataclasses
    import numpy as np
    from oracle import rma
    if dist.rank != 0:
        return None
    scan = make_scan(args.workload, 0)
    su = rma.setup_from(scan, compensate=args.compensate)

    def image_seconds(s):
        """One image's time (the median of three when an image is short)."""
        ts = []
        for _ in range(3):
            t0 = time.time()
            rma.rma_fast(s)
            ts.append(time.time() - t0)
            if ts[0] > 0.5:
                break
        return statistics.median(ts)

    rma.rma_fast(su)
    t_full = image_seconds(su)
    echo = np.asarray(scan.echo)
    nk, n_pos = echo.shape[-1], echo.shape[-2]
    per_step = args.ref_budget / max(1, args.warmup + args.steps)
    nks, nps, t_s = nk, n_pos, t_full
    su_s = su
    for _ in range(4):   # shrink the sample until one image of it fits a step's budget
        if t_s <= per_step or (nks <= min(nk, 8) and nps <= min(n_pos, 64)):
            break
        f = per_step / t_s
        if nks > 8:
            nks = max(min(nk, 8), min(nks, int(nks * f) // 8 * 8))
        else:
            nps = max(min(n_pos, 64), int(nps * f))
        sub = dataclasses.replace(scan, pos=np.asarray(scan.pos)[:nps], echo=echo[:, :, :nps, :nks])
        su_s = rma.setup_from(sub, compensate=args.compensate)
        rma.rma_fast(su_s)
        t_s = image_seconds(su_s)
    ratio = t_full / t_s if su_s is not su else 1.0
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.time()
        rma.rma_fast(su_s)
        if i >= args.warmup:
            times.append(time.time() - t0)
    sec = statistics.mean(times) * ratio
    value = scan.grid.n_voxels / sec
    if su_s is su:
        sample = "one whole image of the scan per step through oracle.rma.rma_fast (FP64 Gaussian gridding, w=16)"
    else:
        sample = (f"per step the first {nps} of the scan's {n_pos} positions and the first {nks} of its {nk} "
                  f"frequencies through oracle.rma.rma_fast (FP64 Gaussian gridding, w=16), time scaled by the "
                  f"measured whole-image / sample-image ratio {ratio:.2f}; one whole image took {t_full:.2f} s")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(scan, args.workload),
            "whole_scan_seconds": t_full,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_cores(), "cpu_model": host_cpu()[0],
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ----------------------------------------------------------------------------- batched mix
def run_batch(args, dist):
    """Batched uneven mix: the same 64 scans imaged (a) one after another on
    one stream, (b) round-robin over 4 streams through mmsar_image_batch,
    (c) as one replayed CUDA graph of (b), (d) through the fused launches of
    mmsar_image_batch_fused (one launch per stage and kernel shape for the
    whole mix) and (e) as a replayed graph of (d).  A step is the whole mix;
    the line reports the fastest form."""
    import numpy as np
    import torch
    import synth
    from paper_2305_02064_gb300.batch import BatchGraph, ScanJob, image_batch, image_batch_fused

    dev = torch.device(f"cuda:{dist.local_rank}")
    torch.cuda.set_device(dev)
    scans = synth.batch_mix(args.mix, seed0=3000 + 1000 * dist.rank)
    jobs = [ScanJob(s, dev) for s in scans]
    voxels = sum(s.grid.n_voxels for s in scans)
    streams = [torch.cuda.Stream(device=dev) for _ in range(4)]
    main_s = torch.cuda.Stream(device=dev)

    def seq():
        for j in jobs:
            j.image(stream=main_s)

    def multi():
        cur = main_s
        for st in streams:
            st.wait_stream(cur)
        image_batch(jobs, streams)
        for st in streams:
            cur.wait_stream(st)

    graph_default = BatchGraph(jobs, n_streams=4, device=dev)

    def timed(fn, steps):
        with torch.cuda.stream(main_s):
            for _ in range(args.warmup):
                fn()
        torch.cuda.synchronize(dev)
        dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(main_s):
            e0.record(main_s)
            for _ in range(steps):
                fn()
            e1.record(main_s)
        torch.cuda.synchronize(dev)
        dist.barrier()
        return dist.max(e0.elapsed_time(e1) / steps)

    steps = max(1, args.steps // 20)
    ms_default = timed(graph_default.replay, steps)
    # the autotuner picks each plan's gridding launch shape on its own data
    # (untimed), then every mode runs with the tuned plans
    with torch.cuda.stream(main_s):
        tuned = [j.tune(stream=main_s) for j in jobs]
    torch.cuda.synchronize(dev)
    graph = BatchGraph(jobs, n_streams=4, device=dev)
    graph_fused = BatchGraph(jobs, n_streams=1, device=dev, fused=True)
    graph_fused4 = BatchGraph(jobs, n_streams=4, device=dev, fused=True)
    ms = {"sequential": timed(seq, steps), "streams4": timed(multi, steps), "graph": timed(graph.replay, steps),
          "graph_default_tiles": ms_default, "fused": timed(lambda: image_batch_fused(jobs, main_s), steps),
          "graph_fused": timed(graph_fused.replay, steps), "graph_fused4": timed(graph_fused4.replay, steps)}
    launches = {"sequential": graph.launches, "streams4": graph.launches, "graph": graph.launches,
                "graph_default_tiles": graph_default.launches, "fused": graph_fused.launches,
                "graph_fused": graph_fused.launches, "graph_fused4": graph_fused4.launches}
    best_mode = min(("graph", "fused", "graph_fused", "graph_fused4"), key=lambda k: ms[k])
    best = ms[best_mode]
    shapes = {}
    for t in tuned:
        key = (f"tensor cores {t['tiles'][3]}" if t['tiles'][3] else
               f"{t['tiles'][0]} freq/lane, {t['tiles'][1]} warps" + (", grouped" if t['tiles'][2] else ""))
        shapes[key] = shapes.get(key, 0) + 1
    n_img = len(jobs) * dist.world
    forms = {"graph": "one CUDA graph of the mix on 4 streams, ten launches per scan",
             "fused": "fused launches (one per stage and kernel shape for the whole mix)",
             "graph_fused": "one CUDA graph of the fused launches",
             "graph_fused4": "one CUDA graph of four fused sub-batches on four streams"}
    return {"metric": "images/s, batched uneven mix (64 scans, 32x32..128x160 positions, Nk 64-256)",
            "value": n_img / (best * 1e-3), "unit": "images/s", "n_gpus": dist.world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": best, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp32", "data": "synthetic (seeded batched mix)",
            "config": {"workload": f"batched uneven mix of {len(jobs)} scans ({forms[best_mode]}, "
                                   f"autotuned gridding launch shapes)",
                       "voxels_per_step": voxels * dist.world, "l2": "inputs larger than L2 (no flush)"},
            "modes_ms_per_mix": ms,
            "modes_images_per_s": {k: n_img / (v * 1e-3) for k, v in ms.items()},
            "modes_launches_per_mix": launches,
            "voxels_per_s": voxels * dist.world / (best * 1e-3),
            "autotuned_grid_shapes": shapes,
            "gpu_launches": launches[best_mode] * steps}


# ----------------------------------------------------------------------------- serving
def run_serve(args, dist):
    """Poisson arrivals (200 req/s) of scans from the batched mix.  The
    served form stores echoes as FP16 with a per-scan scale and admits up to
    8 concurrent requests under a 40 GB device cap; the plain form images one
    FP32 request at a time.  Latency = arrival -> volume ready.  Each form is
    also run saturated (every request arriving at once): its images/s there
    is its capacity."""
    import numpy as np
    import torch
    import synth
    from paper_2305_02064_gb300.serve import (GpuExecutor, Scheduler, ServeRequest, latency_summary,
                                              poisson_arrivals)
    from oracle import rma

    dev = torch.device(f"cuda:{dist.local_rank}")
    torch.cuda.set_device(dev)
    pool = synth.batch_mix(16, seed0=4000 + 1000 * dist.rank)
    rng = np.random.default_rng(7 + dist.rank)
    picks = rng.integers(0, len(pool), args.requests)
    arrivals = poisson_arrivals(args.requests, 200.0, seed=11 + dist.rank)
    out = {}
    results = {}
    cap = 40 << 30
    for name, dtype, slots in (("served_f16", "f16", 8), ("plain_fp32", "c64", 1)):
        # one device arena of the admission cap, allocated before serving:
        # every admitted request's buffers are placed in it
        ex = GpuExecutor(dev, dtype=dtype, n_streams=slots, mem_cap=cap)
        # page-locked inputs once per distinct scan, shared by its requests
        pinned = []
        for sc in pool:
            r = ServeRequest(-1, sc, 0.0)
            ex.pin(r)
            pinned.append(r.pinned)
        reqs = [ServeRequest(i, pool[picks[i]], float(arrivals[i]), ex.footprint(pool[picks[i]]),
                             pinned=pinned[picks[i]]) for i in range(args.requests)]
        # one untimed pass over the same stream warms plans, kernel attributes,
        # the device allocator and the pinned output pool
        Scheduler(ex, slots=slots, mem_cap=cap).run(
            [ServeRequest(r.rid, r.scan, r.arrival, r.footprint, pinned=r.pinned) for r in reqs])
        torch.cuda.synchronize(dev)
        dist.barrier()
        alloc0 = torch.cuda.memory_allocated(dev)
        torch.cuda.reset_peak_memory_stats(dev)
        ex.arena.peak = ex.arena.in_use
        sch = Scheduler(ex, slots=slots, mem_cap=cap)
        done = sch.run(reqs)
        out[name] = latency_summary(done)
        out[name]["max_concurrent"] = sch.max_concurrent
        out[name]["peak_admitted_gb"] = ex.arena.peak / 2 ** 30
        out[name]["cap_gb"] = cap / 2 ** 30
        out[name]["allocated_while_serving_bytes"] = int(torch.cuda.max_memory_allocated(dev) - alloc0)
        # capacity: the same requests all arriving at once (after one untimed
        # burst that grows the pinned output pool to the slot count)
        burst = lambda: [ServeRequest(r.rid, r.scan, 0.0, r.footprint, pinned=r.pinned) for r in reqs]
        Scheduler(ex, slots=slots, mem_cap=cap).run(burst())
        torch.cuda.synchronize(dev)
        out[name]["saturated"] = latency_summary(Scheduler(ex, slots=slots, mem_cap=cap).run(burst()))
        # volumes for the accuracy comparison, outside the timed run
        ex.keep = True
        check = [ServeRequest(i, pool[i], 0.0, ex.footprint(pool[i]), pinned=pinned[i]) for i in range(len(pool))]
        Scheduler(ex, slots=slots, mem_cap=cap).run(check)
        results[name] = {r.rid: r.result for r in check}
        del ex
        torch.cuda.empty_cache()
    # accuracy of the served form against the plain FP32 form, per scan of the pool
    worst = float(max(rma.nmse(results["served_f16"][i].numpy(), results["plain_fp32"][i].numpy())
                      for i in range(len(pool))))
    s = out["served_f16"]
    return {"metric": "images/s with p50/p99 latency, served Poisson stream (200 req/s) from the batched mix",
            "value": s["images_per_s"] * dist.world, "unit": "images/s", "n_gpus": dist.world,
            "steps": args.requests, "warmup": len(pool), "ms_per_step": 1e3 / s["images_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp16 storage, fp32 arithmetic", "data": "synthetic (seeded batched mix)",
            "config": {"workload": "serving: Poisson 200 req/s, continuous batching (8 slots), requests placed in "
                                   "one 40 GiB device arena",
                       "requests": args.requests},
            "latency_ms": {"p50": s["p50_ms"], "p99": s["p99_ms"]},
            "forms": out, "worst_nmse_served_vs_plain_fp32": worst}


# ----------------------------------------------------------------------------- PSF study (Sec. V-A)
PSF_DZ = (0.0, 0.05, 0.10, 0.15, 0.20)


def run_psf(args, dist):
    """The point-spread study of Sec. V-A: a linear-track scan of one point
    target at 0.5 m with the samples up to dz_max off the reference plane,
    imaged on the GPU without compensation, with Eq. 7's residual and with
    Eq. 5's at the scene centre; per case the -3 dB main-lobe widths, the
    peak's offset and amplitude, and the NMSE against the FP64 oracle of the
    same mode."""
    import numpy as np
    import torch
    import paper_2305_02064_gb300 as mm
    from paper_2305_02064_gb300 import quality
    from oracle import rma
    import synth
    dev = torch.device(f"cuda:{dist.local_rank}")
    rows = []
    ideal = None
    t_img = []
    for dz in PSF_DZ:
        sc = synth.psf_track(dz)
        echo = torch.from_numpy(np.ascontiguousarray(sc.echo)).to(dev)
        pos, tx, rx = (torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev) for a in (sc.pos, sc.tx, sc.rx))
        for mode in (0, 1, 2):
            plan = mm.Plan.for_scan(sc, z_ref=0.0, compensate=mode)
            ws = plan.new_workspace(dev)
            vol = plan.new_volume(dev)
            for _ in range(3):
                plan.image(ws, echo, pos, tx, rx, vol)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                plan.image(ws, echo, pos, tx, rx, vol)
            e1.record()
            torch.cuda.synchronize()
            t_img.append(e0.elapsed_time(e1) / 10)
            plan.poll_error(ws)
            got = vol.cpu().numpy()
            m = quality.psf_metrics(got, sc.grid, sc.scatterers[0])
            su = rma.setup_from(sc, z_ref=0.0, compensate=mode, Mx=plan.mx, My=plan.my)
            m["nmse_vs_oracle"] = float(rma.nmse(got, rma.rma_fast(su, w=16)))
            if dz == 0.0 and mode == 1:
                ideal = m["peak"]
            m.update({"dz_max_cm": dz * 100, "compensate": mode})
            rows.append({k: (float(f"{float(v):.4g}") if isinstance(v, (float, np.floating)) else v) for k, v in m.items()})
    for r in rows:
        r["peak_rel_planar"] = float(f"{r['peak'] / ideal:.4g}")
    return {"metric": "point-spread main-lobe widths vs largest plane deviation (Sec. V-A study)",
            "value": None, "unit": "mm", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "linear 2Tx x 4Rx track, 256 positions over y' in [-12.5, 12.5] cm, Nk=64, "
                                   "point at (0, 0, 0.5 m), y-z image 256 x 64 at 1 x 2.5 mm",
                       "dz_max_cm": [d * 100 for d in PSF_DZ],
                       "compensate": {"0": "none", "1": "Eq. 7 residual (paper)", "2": "Eq. 5 at the scene centre"}},
            "ms_per_image_mean": round(float(np.mean(t_img)), 4), "rows": rows}


def extras(args, dist):
    """Compact records of the batched, served and large workloads for the
    default run (each a few tens of seconds, inputs generated on the host)."""
    import torch
    out = {}
    t0 = time.time()
    b = run_batch(args, dist)
    out["batch"] = {"images_per_s": b["value"], "ms_per_mix": b["ms_per_step"], "scans": args.mix,
                    "form": b["config"]["workload"], "launches_per_mix": b["modes_launches_per_mix"],
                    "modes_ms_per_mix": b["modes_ms_per_mix"], "voxels_per_s": b["voxels_per_s"],
                    "dtype": b["dtype"], "wall_s": time.time() - t0}
    torch.cuda.empty_cache()
    t0 = time.time()
    sv = run_serve(args, dist)
    f = sv["forms"]
    out["serve"] = {k: {"p50_ms": v["p50_ms"], "p99_ms": v["p99_ms"], "images_per_s": v["images_per_s"],
                        "saturated_images_per_s": v["saturated"]["images_per_s"],
                        "max_concurrent": v["max_concurrent"]} for k, v in f.items()}
    out["serve"].update({"arrivals": "Poisson 200 req/s", "requests": args.requests,
                         "worst_nmse_served_vs_plain_fp32": sv["worst_nmse_served_vs_plain_fp32"],
                         "wall_s": time.time() - t0})
    for k in ("peak_admitted_gb", "cap_gb", "allocated_while_serving_bytes"):
        out["serve"][k] = {n: f[n].get(k) for n in f}
    torch.cuda.empty_cache()
    t0 = time.time()
    out["large_storage"] = run_large_storage(args, dist)
    out["large_storage"]["wall_s"] = time.time() - t0
    torch.cuda.empty_cache()
    return out


def main():
    args = parse_args()
    if args.ncu_traffic:
        print(json.dumps(write_ncu_traffic(args.ncu_traffic, args.ncu_command, args.workload), indent=1))
        return 0
    if args.impl == "reference":
        dist = Dist(want_cuda=False)
        out = run_reference(args, dist)
        if out is not None:
            print(json.dumps(out))
        dist.close()
        return 0
    dist = Dist(want_cuda=True)
    if args.workload == "psf":
        res = run_psf(args, dist) if dist.rank == 0 else None
        if res is not None:
            print(json.dumps(res))
        dist.close()
        return 0
    if args.workload in ("batch", "serve"):
        res = (run_batch if args.workload == "batch" else run_serve)(args, dist)
        if dist.rank == 0:
            print(json.dumps(res))
        dist.close()
        return 0
    res, scan, vol = run_ours(args, dist)
    if args.workload == "large" and dist.rank == 0 and dist.world == 1:
        res["storage_comparison"] = storage_comparison(scan, vol, args)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        cb, acc = cpu_baseline(scan, vol, args.compensate)
        res["cpu_baseline"] = cb
        res["accuracy"] = acc
        if args.workload == "realistic":
            res["oracle_timings"] = oracle_timings(scan)
            res["oracle_timings"]["rma_fast_realistic_s"] = cb["seconds"]
    if dist.world == 1 and args.workload == "realistic" and not args.no_extras:
        import torch
        del vol
        torch.cuda.empty_cache()
        res.update(extras(args, dist))
    if dist.rank == 0:
        print(json.dumps(res))
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

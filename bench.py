"""Benchmark: ED voxels/s through FFT + |F|^2 + Q binning, forward and adjoint.

Workload (one step): the 512^3 FP32 grid of a 2.6 nm MOF-like cell (60
Gaussian atoms, 64^3 samples, seed 0) tiled and cut by a 10 nm sphere, 512
log-spaced Q bins from dq to pi/dx:
  ur_fft_intensity_tiled (the density of the 247 nonzero planes generated
  inside the plane pass, column pass with fused |F|^2 and binning) ->
  dL/d(mean I) of a log-MSE loss against the closed-form sphere curve
  (ur_log_mse_grad) ->
  ur_backward (dL/d cell, dL/d mask).
All inputs are synthetic and larger than L2 (ED slab 259 MB, intermediate
520 MB), so no explicit L2 flush is done between steps.

`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ED voxels/s through FFT+|F|^2+Q-binning (fwd and adjoint); % HBM roofline"
UNIT = "voxels/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--workload", default="mof512", choices=["mof512", "batch64", "merge3", "ooc"])
    ap.add_argument("--check", action="store_true", help="ooc: also compare with the device-resident path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# library kernel behind each timing label of the step (for the ncu profile lookup)
KERNEL_OF = {
    "rows_r2c": "k_p2_rows<512, 1, float>",
    "cols_y": "k_p2_cols<512, 0>",
    "cols_z_bin": "k_p2_cols<512, 2>",
    "adj_cols_z": "k_p2_cols<512, 3>",
    "adj_cols_y": "k_p2_cols<512, 1>",
    "adj_rows_grad": "k_p2_rows_grad<512>",
}


def csrc_digest() -> str:
    """sha256 over the CUDA sources; a profile taken from other sources is stale."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2303_13435_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def profiled_traffic(kernel: str, variant: str):
    """DRAM bytes (read + write) per launch of `kernel` from a committed ncu summary
    under profiles/ taken on the current sources in the same launch variant, else None."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None, None
    digest = csrc_digest()
    for f in sorted(os.listdir(pdir)):
        if not f.endswith(".txt"):
            continue
        kv = {}
        for line in open(os.path.join(pdir, f)):
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if (kv.get("kernel") == kernel and kv.get("variant") == variant and kv.get("source_sha256") == digest
                and "traffic_bytes_per_launch" in kv):
            return float(kv["traffic_bytes_per_launch"]), f"profiles/{f}"
    return None, None


def max_over_ranks(x: float, device="cpu") -> float:
    """Largest value of x over the ranks of the default process group (x itself when
    there is none): the job time of N replicas is that of the slowest one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job throughput: every rank processes units_per_rank in at most ms_max."""
    return world * units_per_rank / (ms_max * 1e-3)


def workload(n: int):
    from paper_2303_13435_gb300 import inputs
    d = 10.0 * n / 512.0
    return inputs.mof_workload(n=n, diameter_nm=d, nbins=512)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# algorithmic bytes per launch of each kernel: what its pass must read and write; store_f: the
# forward writes the half spectrum F and the adjoint reads it instead of recomputing it
def kernel_bytes(n: int, P: int, U: int, store_f: bool = False):
    H = n // 2 + 1
    X = 8 * n * H * P           # forward intermediate, complex64
    Y = 8 * n * n * H           # adjoint intermediate, all planes (and F, same size)
    return {
        "density": 4 * n * n * P,
        "rows_r2c": X,          # density generated in the kernel: only the intermediate is written
        "cols_y": 2 * X,
        "cols_z_bin": X + (Y if store_f else 0),
        "finalize": 0,
        "sigma": 0,
        "loss_grad": 0,
        "adj_cols_z": (Y if store_f else X) + Y,
        "adj_cols_y": 2 * Y,
        "adj_rows_grad": Y + 4 * n ** 3 + 4 * U ** 3,
    }


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2303_13435_gb300 import api, build, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    api.lib()

    n = args.n
    w = workload(n)
    cell = torch.from_numpy(w.cell).cuda()
    # nonzero plane slab from a first density pass
    rng = torch.tensor([2 ** 31 - 1, -1], dtype=torch.int32, device="cuda")
    full = api.build_density(n, cell, w.shape, nz_range=rng)
    z0, z1 = rng.cpu().tolist()
    P = z1 - z0 + 1
    del full
    plan = api.Plan(n, w.dx, w.edges, z0=z0, nz=P)
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD)
    ed = torch.empty((P, n, n), dtype=torch.float32, device="cuda")
    bins = api.new_bins(plan)
    dcell = torch.empty_like(cell)
    dmask = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    # target curve: closed-form sphere of the particle's electron count (loss input)
    api.build_density(n, cell, w.shape, z_begin=z0, z_count=P, out=ed)
    api.fft_intensity(plan, ed, bins=bins, ws=ws)
    b0 = bins.cpu().numpy()
    ne = float(ed.double().sum().item())
    qm = b0[3] / np.maximum(b0[0], 1)
    radius = 0.5 * 10.0 * n / 512.0
    target = torch.from_numpy(inputs.sphere_target_curve(qm, radius, ne) / float(n) ** 6 + 1e-300).cuda()

    g = torch.empty(plan.nbins, dtype=torch.float64, device="cuda")

    def step():
        api.fft_intensity_tiled(plan, cell, w.shape, bins=bins, ws=ws)
        api.log_mse_grad(bins, target, g)
        api.backward(plan, g, bins, cell, w.shape, ws, dl_dcell=dcell, dl_dmask=dmask)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # per-kernel times: one timed pass of eager steps with the library's own events around
    # each of its launches (on the launching stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    api.set_timing(True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_eager = e0.elapsed_time(e1) / args.steps
    kt = api.last_timings()
    api.set_timing(False)

    # the step captured once in a CUDA graph (its launches replay without host work)
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    # timed region: device events on the launching stream around K graph replays
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms_total, "cuda")
    ms_step = ms_max / args.steps

    # per-kernel averages
    per = {}
    for name, ms in kt:
        s = per.setdefault(name, [0.0, 0])
        s[0] += ms
        s[1] += 1
    # kernel_bytes() is per step; a kernel launched in plane chunks moves that over
    # launches/steps launches, so bytes per launch = per-step bytes * steps / launches.
    kb = kernel_bytes(n, P, w.ucell)
    dom = max(per.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_cnt) = dom
    hbm, src = peaks()
    avg_ms = dom_ms / dom_cnt
    bytes_per_launch = kb.get(dom_name, 0) * args.steps / dom_cnt
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    kernels = {k: {"launches": c, "avg_us": 1e3 * ms / c, "share": ms / sum(v[0] for v in per.values()),
                   "bytes_per_launch": kb.get(k, 0) * args.steps / c,
                   "gbs": (kb.get(k, 0) * args.steps / (ms * 1e-3) / 1e9) if kb.get(k, 0) else None}
               for k, (ms, c) in per.items()}
    # step-level algorithmic bytes: forward 16 N H P (intermediate written and read once; the
    # density is generated, not read) + adjoint 8 N H P (read the forward intermediate) +
    # 16 N^2 H (the inverse intermediate of all N planes written and read once) + 4 N^3 (dL/dm)
    H = n // 2 + 1
    fwd_alg = 16 * n * H * P
    adj_alg = 8 * n * H * P + 16 * n * n * H + 4 * n ** 3
    step_frac = (fwd_alg + adj_alg) / (ms_step * 1e-3) / 1e9 / hbm
    # forward gate: e N^2 P + 16 N H P (stored FP32 ED read + intermediate written and read)
    # over the forward kernels' time
    fwd_names = ("rows_r2c", "cols_y", "cols_z_bin", "finalize")
    fwd_ms = sum(per[k][0] for k in fwd_names if k in per) / args.steps
    fwd_gate_bytes = 4 * n * n * P + 16 * n * H * P
    fwd_frac = fwd_gate_bytes / (fwd_ms * 1e-3) / 1e9 / hbm
    # the forward path alone (no F kept for an adjoint), timed as graph replays
    fgraph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap):
        api.fft_intensity_tiled(plan, cell, w.shape, bins=bins, ws=ws, stream=cap)
    torch.cuda.synchronize()
    with torch.cuda.graph(fgraph, stream=cap):
        api.fft_intensity_tiled(plan, cell, w.shape, bins=bins, ws=ws, stream=cap)
    for _ in range(args.warmup):
        fgraph.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        fgraph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    fonly_ms = max_over_ranks(e0.elapsed_time(e1), "cuda") / args.steps
    fonly_frac = fwd_gate_bytes / (fonly_ms * 1e-3) / 1e9 / hbm
    traffic, traffic_src = profiled_traffic(KERNEL_OF.get(dom_name, ""), "recompute")

    # end to end through the public API with host buffers: every step copies its input (the
    # cell) from pinned host memory and reads its results (bins, dL/du, dL/dm) back to pinned
    # host memory.  Serially, and pipelined: the read-back of step k runs on a copy stream
    # while step k + 1 computes (two sets of output buffers), as a training loop that needs
    # dL/dm on the host would run it
    cell_host = torch.from_numpy(w.cell).pin_memory()
    cell_dev = torch.empty_like(cell)
    outs = [(torch.empty_like(bins), torch.empty_like(dcell), torch.empty_like(dmask),
             torch.empty(bins.shape, dtype=bins.dtype).pin_memory(),
             torch.empty(dcell.shape, dtype=dcell.dtype).pin_memory(),
             torch.empty(dmask.shape, dtype=dmask.dtype).pin_memory()) for _ in range(2)]
    gbuf = torch.empty_like(g)

    def compute(o):
        cell_dev.copy_(cell_host, non_blocking=True)
        api.fft_intensity_tiled(plan, cell_dev, w.shape, bins=o[0], ws=ws)
        api.log_mse_grad(o[0], target, gbuf)
        api.backward(plan, gbuf, o[0], cell_dev, w.shape, ws, dl_dcell=o[1], dl_dmask=o[2])

    def read_back(o):
        o[3].copy_(o[0], non_blocking=True)
        o[4].copy_(o[1], non_blocking=True)
        o[5].copy_(o[2], non_blocking=True)

    def e2e_serial(k):
        compute(outs[0])
        read_back(outs[0])

    copy_stream = torch.cuda.Stream()
    done = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]
    for ev in free:
        ev.record(stream)

    def e2e_pipelined(k):
        b = k & 1
        stream.wait_event(free[b])       # the read-back of step k - 2 is done with buffers b
        compute(outs[b])
        done[b].record(stream)
        copy_stream.wait_event(done[b])
        with torch.cuda.stream(copy_stream):
            read_back(outs[b])
            free[b].record(copy_stream)

    def time_e2e(fn):
        for k in range(2):
            fn(k)
        torch.cuda.synchronize()
        steps = max(3, args.steps // 2)
        e0.record(stream)
        for k in range(steps):
            fn(k)
        stream.wait_stream(copy_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / steps, "cuda")

    e2e_serial_ms = time_e2e(e2e_serial)
    e2e_ms = time_e2e(e2e_pipelined)
    bins_host, dcell_host, dmask_host = outs[0][3], outs[0][4], outs[0][5]

    out = {
        "metric": METRIC, "value": job_rate(n ** 3, ms_step, world), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": mof_config(n, P, w.ucell, world),
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs, burst copy)"
                     if src == "measured" else "fallback 6800 GB/s", "traffic": traffic,
                     "traffic_source": traffic_src, "algorithmic_bytes_per_launch": bytes_per_launch,
                     "step_frac_of_hbm": step_frac,
                     "forward_in_step": {"us_per_step": 1e3 * fwd_ms, "gate_bytes": fwd_gate_bytes,
                                         "frac": fwd_frac},
                     "forward_only": {"us": 1e3 * fonly_ms, "gate_bytes": fwd_gate_bytes, "frac": fonly_frac,
                                      "voxels_per_s": job_rate(n ** 3, fonly_ms, world)}},
        "kernels": kernels,
        "timing": {"value_from": "CUDA-graph replays of the step", "ms_per_step_eager": ms_eager,
                   "kernel_times_from": "library events around each launch, eager pass of the same steps"},
        "e2e": {"value": job_rate(n ** 3, e2e_ms, world), "unit": UNIT,
                "h2d_bytes_per_step": int(cell_host.numel() * 4),
                "d2h_bytes_per_step": int(bins_host.numel() * 8 + dcell_host.numel() * 4 + dmask_host.numel() * 4),
                "ms_per_step": e2e_ms, "how": "read-back of step k on a copy stream while step k+1 computes",
                "serial": {"value": job_rate(n ** 3, e2e_serial_ms, world), "ms_per_step": e2e_serial_ms}},
        "gpu_launches": sum(c for _, c in per.values()),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(512 if n == 512 else n)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def mof_config(n: int, P: int, ucell: int, world: int) -> dict:
    """The `config` of the default workload's JSON line (both arms)."""
    return {"workload": f"mof512 sphere 10 nm, {n}^3 FP32 grid, {P} nonzero planes, 512 log Q bins, "
                        "forward + adjoint (dL/d cell, dL/d mask) recomputing F along z",
            "grid": n, "nonzero_planes": P, "bins": 512, "cell": f"{ucell}^3, 2.6 nm, 60 atoms, seed 0",
            "l2": "inputs larger than L2 (ED slab, intermediates); no flush",
            "parallelism": f"replicas x{world}"}


def oracle_nonzero_planes(n: int) -> int:
    """Planes of the default workload's density holding a nonzero voxel (oracle density, in chunks)."""
    from oracle import density
    w = workload(n)
    hit = []
    for z0 in range(0, n, 32):
        rho = density.tile_mask_density(w.n, w.cell, w.shape.kind, w.shape.center, w.shape.size, w.shape.rot,
                                        z_begin=z0, z_count=min(32, n - z0))
        hit.extend((z0 + i) for i in np.flatnonzero(rho.any(axis=(1, 2))))
    return int(hit[-1] - hit[0] + 1) if hit else 0


def oracle_step(n: int):
    """The FP64 oracle as it stands: density, forward (Eq. 1 FFT + Sec. 2.5 bins) and the adjoint."""
    from oracle import adjoint, density, scatter
    w = workload(n)
    t = time.perf_counter()
    rho = density.tile_mask_density(w.n, w.cell, w.shape.kind, w.shape.center, w.shape.size, w.shape.rot)
    ob = scatter.forward(rho.astype(np.float64), w.dx, w.edges)
    g = np.where(ob["count"] > 0, 1.0, 0.0)
    grho = adjoint.grad_rho(rho.astype(np.float64), w.dx, w.edges, g, count=ob["count"], F=ob["F"])
    m = density.mask_values(w.n, w.shape.kind, w.shape.center, w.shape.size, w.shape.rot)
    adjoint.grad_cell_and_mask(grho, w.cell.astype(np.float64), m)
    return time.perf_counter() - t


def cpu_baseline(n: int):
    dt = oracle_step(n)
    return {"value": n ** 3 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one forward+adjoint step of the FP64 numpy oracle on the {n}^3 grid of the same workload "
                      f"({dt:.1f} s; numpy FFT single-threaded)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    # the same workload and config as the GPU arm; each timed step is a bounded sample of it:
    # the oracle's forward + adjoint on the 256^3 grid of the same cell, dx, bins and a sphere
    # scaled with the box (5 nm), so that warm-up plus K steps finish within minutes
    full = args.n
    sample_n = 256 if full > 256 else full
    P = oracle_nonzero_planes(full)
    for _ in range(args.warmup):
        oracle_step(sample_n)
    times = [oracle_step(sample_n) for _ in range(args.steps)]
    ms = 1e3 * sum(times) / len(times)
    v = sample_n ** 3 / (ms * 1e-3)
    sample = (f"{args.steps} forward + adjoint steps of the FP64 numpy oracle on the {sample_n}^3 grid of the same "
              f"cell, dx and bins ({sample_n * 10.0 / 512:g} nm sphere), {ms / 1e3:.1f} s each; voxels/s counts "
              f"that grid's voxels")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(mof_config(full, P, 64, args.gpus), sample_grid=sample_n),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batch(args):
    """Uneven-particle batch (64 particles, 96^3..384^3, seed 7): looped single-instance
    forward+adjoint against the batched launches captured in one CUDA graph."""
    import torch

    from paper_2303_13435_gb300 import api, autotune, build, inputs

    torch.cuda.set_device(0)
    build.build()
    api.lib()
    dx = 2.6 / 64
    parts = inputs.batch_particles(count=64, seed=7)
    edges = inputs.log_edges(2 * math.pi / (384 * dx), math.pi / dx, 256)
    cell = torch.from_numpy(inputs.mof_like_cell(64, 2.6, 0)).cuda()
    plans, targets, voxels = [], [], 0
    for p in parts:
        rng = torch.tensor([2 ** 31 - 1, -1], dtype=torch.int32, device="cuda")
        ed = api.build_density(p.n, cell, p.shape, nz_range=rng)
        ne = float(ed.double().sum().item())
        vol = float((ed != 0).sum().item()) * dx ** 3
        z0, z1 = rng.cpu().tolist()
        del ed
        plan = api.Plan(p.n, dx, edges, z0=z0, nz=z1 - z0 + 1)
        b = api.fft_intensity_tiled(plan, cell, p.shape).cpu().numpy()
        qm = b[3] / np.maximum(b[0], 1)
        r_eq = (3 * vol / (4 * math.pi)) ** (1 / 3)
        targets.append(torch.from_numpy(inputs.sphere_target_curve(qm, r_eq, ne) / float(p.n) ** 6 + 1e-300).cuda())
        plans.append(plan)
        voxels += p.n ** 3
    shapes = [p.shape for p in parts]
    t0 = time.time()
    chosen = autotune.tune(plans, cell, shapes, reps=2)
    tune_s = time.time() - t0


    # looped single-instance path (fast kernels for power-of-two edges)
    ws = [p.workspace(api.UR_WS_FORWARD | api.UR_WS_BACKWARD) for p in plans]
    bins = [api.new_bins(p) for p in plans]
    gs = [torch.zeros(p.nbins, dtype=torch.float64, device="cuda") for p in plans]
    dcell = [torch.empty_like(cell) for _ in plans]

    def loop_step():
        for i, (p, pl) in enumerate(zip(parts, plans)):
            api.fft_intensity_tiled(pl, cell, p.shape, bins=bins[i], ws=ws[i])
            api.log_mse_grad(bins[i], targets[i], gs[i])
            api.backward(pl, gs[i], bins[i], cell, p.shape, ws[i], dl_dcell=dcell[i], want_mask=False)

    batch = api.Batch(plans, cell, shapes)

    def batch_step():
        batch.forward()
        for i in range(len(plans)):
            api.log_mse_grad(batch.bins[i], targets[i], batch.dl_dmean[i])
        batch.backward()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_loop = timed(loop_step, args.steps)
    ms_batch_eager = timed(batch_step, args.steps)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch_step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        batch_step()
    ms_graph = timed(graph.replay, args.steps)
    # the looped path captured in one graph too: what is left of the batched form's advantage
    # once both paths are free of launch overhead
    with torch.cuda.stream(s):
        loop_step()
    torch.cuda.synchronize()
    graph_loop = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_loop, stream=s):
        loop_step()
    ms_loop_graph = timed(graph_loop.replay, args.steps)
    # agreement of the two paths (same accuracy bar as the tests)
    loop_step()
    batch_step()
    torch.cuda.synchronize()
    worst = 0.0
    for i in range(len(plans)):
        a, b = bins[i].cpu().numpy(), batch.bins[i].cpu().numpy()
        ok = a[0] > 0
        worst = max(worst, float(np.max(np.abs(a[4][ok] - b[4][ok]) / np.abs(a[4][ok]))))
    out = {"metric": METRIC, "value": voxels / (ms_graph * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch of 64 particles, uneven grids 96^3..384^3 (seed 7), sphere/cube/octahedron, "
                                  "256 log Q bins, forward + adjoint of a log-I(Q) MSE loss", "voxels_per_step": voxels,
                      "sizes": sorted({p.n for p in parts})},
           "batch": {"ms_looped_single_instance": ms_loop, "ms_batched_eager": ms_batch_eager,
                     "ms_batched_graph": ms_graph, "speedup_graph_vs_looped": ms_loop / ms_graph,
                     "ms_looped_in_one_graph": ms_loop_graph,
                     "max_rel_diff_mean_I": worst, "autotune_seconds": tune_s,
                     "tiles": {str(k): list(v[:2]) for k, v in chosen.items()}}}
    print(json.dumps(out))


def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_merge3(args):
    """Three-level workload: ED-1 1024^3 FP16 (20 nm cube filling the box), ED-2/ED-3 4x/16x
    block sums in 512^3 FP16 boxes, 1000 log bins 0.01-150 nm^-1, merged.  One step = ED-1
    generation, both zooms, the three forwards and the merge."""
    import torch

    from paper_2303_13435_gb300 import api, build, inputs

    torch.cuda.set_device(0)
    build.build()
    api.lib()
    ed1w, zooms = inputs.cube_merge_levels()
    cell = torch.from_numpy(ed1w.cell).cuda()
    edges_d = torch.from_numpy(ed1w.edges).cuda()
    n1 = ed1w.n
    ed1 = torch.empty((n1, n1, n1), dtype=torch.float16, device="cuda")
    levels = [(ed1, n1, ed1w.dx, 1)]
    for f, n_out, dx in zooms:
        levels.append((torch.empty((n_out, n_out, n_out), dtype=torch.float16, device="cuda"), n_out, dx, f))
    api.build_density(n1, cell, ed1w.shape, out_dtype="f16", out=ed1)
    plans, slabs = [], []
    for ed, n, dx, f in levels:
        if f > 1:
            api.zoom_density(ed1, f, n, out_dtype="f16", out=ed)
        occ = torch.nonzero(ed.float().abs().sum(dim=(1, 2)) > 0).flatten()
        z0, z1 = int(occ[0]), int(occ[-1])
        plan = api.Plan(n, dx, ed1w.edges, z0=z0, nz=z1 - z0 + 1, ed_dtype="f16")
        plans.append(plan)
        slabs.append((z0, z1 - z0 + 1))
    ws = [p.workspace(api.UR_WS_FORWARD) for p in plans]
    bins = [api.new_bins(p) for p in plans]
    ns = [n for _, n, _, _ in levels]
    dxs = [dx for _, _, dx, _ in levels]
    merged = torch.empty((5, len(ed1w.edges) - 1), dtype=torch.float64, device="cuda")

    def step():
        api.build_density(n1, cell, ed1w.shape, out_dtype="f16", out=ed1)
        for (ed, n, dx, f), plan, (z0, nz), b, w_ in zip(levels, plans, slabs, bins, ws):
            if f > 1:
                api.zoom_density(ed1, f, n, out_dtype="f16", out=ed)
            api.fft_intensity(plan, ed[z0:z0 + nz], bins=b, ws=w_)
        api.merge(bins, ns, dxs, edges_d, out=merged)

    ms = _timed(step, args.steps, args.warmup)
    out_np = merged.cpu().numpy()
    src = out_np[4].astype(np.int64)
    voxels = sum(n ** 3 for n in ns)
    out = {"metric": METRIC, "value": voxels / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (FP16 ED storage)", "data": "synthetic",
           "config": {"workload": "three-level merge: ED-1 1024^3 FP16 (20 nm cube filling the box, 2.5 nm cell "
                                  "at 128^3), ED-2/ED-3 4x/16x block sums in 512^3 boxes, 1000 log bins "
                                  "0.01-150 nm^-1, forward only + merge", "voxels_per_step": voxels},
           "merge": {"levels_used": sorted(int(v) for v in np.unique(src[src >= 0])),
                     "bins_filled": int((src >= 0).sum()), "bins": int(len(src))}}
    print(json.dumps(out))


def run_ooc(args):
    """Out-of-core forward: the nonzero planes of the FP32 density in pinned host memory,
    streamed to the device in double-buffered slabs (N = --n, 4096 by default: 64 nm sphere,
    2000 log bins 0.0378-77.33 nm^-1; 2048: 32 nm sphere)."""
    import torch

    from paper_2303_13435_gb300 import api, build, inputs

    torch.cuda.set_device(0)
    build.build()
    api.lib()
    n = args.n if args.n != 512 else 4096
    a_nm, U = 2.6, 64
    dx = a_nm / U
    w = inputs.mof_workload(n=n, diameter_nm=64.0 * n / 4096, nbins=2000)
    w.edges = inputs.log_edges(2 * math.pi / (n * dx), math.pi / dx, 2000)
    cell = torch.from_numpy(w.cell).cuda()
    # occupied planes from a density pass over the middle of the box
    rng = torch.tensor([2 ** 31 - 1, -1], dtype=torch.int32, device="cuda")
    R = 0.5 * 64.0 * n / 4096 / dx
    zc0 = max(0, int(n // 2 - R - 2))
    zc1 = min(n, int(n // 2 + R + 3))
    for p0 in range(zc0, zc1, 64):
        d = api.build_density(n, cell, w.shape, z_begin=p0, z_count=min(64, zc1 - p0), nz_range=rng)
        del d
    z0, z1 = rng.cpu().tolist()
    P = z1 - z0 + 1
    # page-locked by registering an anonymous mapping of the exact size (a caching pinned
    # allocator would round a 106 GB request up to the next power of two); transparent huge
    # pages where the kernel allows them (the streamed copies measured about 10 % faster)
    import mmap
    host_map = mmap.mmap(-1, P * n * n * 4, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    if hasattr(host_map, "madvise") and hasattr(mmap, "MADV_HUGEPAGE"):
        try:
            host_map.madvise(mmap.MADV_HUGEPAGE)
        except OSError:
            pass
    host_np = np.frombuffer(host_map, dtype=np.float32).reshape(P, n, n)
    cudart = torch.cuda.cudart()
    err = cudart.cudaHostRegister(host_np.ctypes.data, host_np.nbytes, 0)
    if int(err) != 0:
        raise RuntimeError(f"cudaHostRegister of {host_np.nbytes / 1e9:.1f} GB failed: {err}")
    host = torch.from_numpy(host_np)
    for p0 in range(0, P, 64):
        cnt = min(64, P - p0)
        d = api.build_density(n, cell, w.shape, z_begin=z0 + p0, z_count=cnt)
        host[p0:p0 + cnt].copy_(d)
        del d
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    plan = api.Plan(n, dx, w.edges, z0=z0, nz=P)
    # the out-of-core adjoint's slab of inverse-intermediate planes: as many as about 85 % of
    # the free device memory holds next to the forward workspace (fewer slabs, fewer rereads)
    free0 = torch.cuda.mem_get_info()[0]
    fwd_bytes = plan.workspace_size(api.UR_WS_FORWARD | api.UR_WS_HOST_SLABS)
    H = n // 2 + 1
    staging = 2 * 64 * n * n * 4
    adj_planes = int(max(1, min(n, (0.85 * free0 - fwd_bytes - staging) // (n * H * 8))))
    plan.set_adj_slab_planes(adj_planes)
    ws = plan.workspace(api.UR_WS_FORWARD | api.UR_WS_HOST_SLABS | api.UR_WS_ADJ_SLABS)
    bins = api.new_bins(plan)
    bins_host = torch.empty(bins.shape, dtype=bins.dtype).pin_memory()

    def step():
        api.fft_intensity(plan, host, bins=bins, ws=ws)
        bins_host.copy_(bins, non_blocking=True)

    ms = _timed(step, args.steps, args.warmup)
    # one more step with the library's per-launch events: where the step's time goes
    api.set_timing(True)
    step()
    torch.cuda.synchronize()
    breakdown = {}
    for name, t in api.last_timings():
        breakdown[name] = breakdown.get(name, 0.0) + t
    api.set_timing(False)
    # pinned host -> device copy peak of this machine (best of 5 copies of 4 GiB)
    src_h = torch.empty(1 << 30, dtype=torch.float32, pin_memory=True)
    dst_d = torch.empty(1 << 30, dtype=torch.float32, device="cuda")
    best = min(_timed(lambda: dst_d.copy_(src_h, non_blocking=True), 1, 1) for _ in range(5))
    h2d_peak = 4.0 * (1 << 30) / (best * 1e-3) / 1e9
    del src_h, dst_d
    moved = 4.0 * P * n * n
    achieved = moved / (ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": n ** 3 / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"out-of-core {n}^3 FP32: 2.6 nm MOF-like cell tiled and cut by a "
                                  f"{64.0 * n / 4096:g} nm sphere, {P} nonzero planes ({moved / 1e9:.1f} GB) in pinned "
                                  "host memory streamed in double-buffered slabs, 2000 log Q bins; value: the "
                                  "forward; 'adjoint': the per-slab adjoint (dL/d cell)",
                      "grid": n, "nonzero_planes": P, "slabs": "two device slabs of about 256 MiB (double buffer)"},
           "breakdown_ms": {k: round(v, 2) for k, v in breakdown.items()},
           "roofline": {"bound": "h2d", "achieved": achieved, "peak": h2d_peak, "unit": "GB/s",
                        "frac": achieved / h2d_peak, "peak_source": "measured pinned H2D copy of 4 GiB, best of 5",
                        "traffic": None},
           "e2e": {"value": n ** 3 / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(moved),
                   "d2h_bytes_per_step": int(bins_host.numel() * 8)}}
    # the per-slab adjoint of the same forward (dL/d cell; the z pass recomputed per slab)
    api.fft_intensity(plan, host, bins=bins, ws=ws)
    m = bins[4]
    g = torch.where(torch.isfinite(m) & (m > 0), 1e-3 / torch.nan_to_num(m, nan=1.0).clamp(min=1e-300), 0.0)
    dcell = torch.empty_like(cell)
    ms_adj = _timed(lambda: api.backward_slabs(plan, g, bins, cell, w.shape, ws, dl_dcell=dcell), max(1, args.steps // 2),
                    1)
    out["adjoint"] = {"ms": ms_adj, "slab_planes": adj_planes, "slabs": -(-n // adj_planes),
                      "voxels_per_s": n ** 3 / (ms_adj * 1e-3),
                      "what": "ur_backward_slabs: dL/d cell; per slab the z pass is recomputed from the forward "
                              "intermediate over every spectrum column, then y inverse and row pass of the slab"}
    if args.check:
        del ws
        torch.cuda.empty_cache()
        ws = plan.workspace(api.UR_WS_FORWARD)
        dev = host.cuda()
        ref = api.fft_intensity(plan, dev, ws=ws).cpu().numpy()
        got = bins_host.numpy()
        ok = ref[0] > 0
        out["check"] = {"counts_equal": bool(np.array_equal(got[0], ref[0])),
                        "max_rel_diff_mean_vs_device_path": float(np.max(np.abs(got[4][ok] - ref[4][ok])
                                                                         / np.abs(ref[4][ok])))}
        del dev
    print(json.dumps(out))
    del host
    cudart.cudaHostUnregister(host_np.ctypes.data)
    del host_np
    try:
        host_map.close()
    except BufferError:  # a view is still alive; the mapping goes with the process
        pass


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "merge3":
        run_merge3(args)
    elif args.workload == "ooc":
        run_ooc(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

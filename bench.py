"""Benchmark of the fused wall-modelled LBM LES step on GB300.

Headline workload: the 256^3 turbulent channel (D3Q19, BGK + Smagorinsky C_S = 0.1, Spalding wall
function on both walls, body force for Re_tau = 550, FP32 storage), one step = one collide-and-stream
pass over all cells (interior kernel + boundary-list kernel). Value: GLUPS = cells * steps / time
(the paper's "billions of lattice cell updates per second", Sec. 3.1), device-timed with CUDA
events on the library's stream; the 2.6 GB state exceeds L2, so no flush is needed between steps.

Also printed in the same JSON line: the interior kernel's HBM roofline, the end-to-end number
through the C ABI with host buffers, the oracle on the host cores, SM clocks during the timed
region, and secondary forms (16-bit storage with its error, D3Q27 and D3Q19 urban canopy, the
adjoint on the 128^3 duct).

`--impl reference` times the CPU oracle (the reference arm of this build) on a bounded slab of the
same workload. Multi-GPU (N > 1): the channel 256 x 256 x (256 N) in N z-slabs, one per rank, with the
halo exchange of every step between neighbouring ranks (weak scaling), max time over ranks.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 LES GLUPS, % HBM roofline; adjoint GLUPS; 16-bit vs FP32 GLUPS at err"
WORKLOAD = ("channel 256x256x256 D3Q19 BGK + Smagorinsky (C_S=0.1) + Spalding wall function, "
            "Re_tau=550 body force, FP32 storage (f - w deviations)")
Q19_FP32_BYTES = 19 * 4 * 2  # one read and one write per population


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(x, world):
    """Max of a float over ranks (identity on one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current source of
    the kernels (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt, re.M)
    h = re.search(r"^source_sha256:\s*([0-9a-f]+)", txt, re.M)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


# the sources that make up the interior kernels of the FP32 translation unit
KERNEL_FILES = ("lbm_device.cuh", "lbm_kernels.cuh", "lbm_hrr.cuh", "lbm_adjoint.cuh", "lbm_impl.cuh", "lbm_tma.cuh",
                "lbm_ops.h", "lbm_ops_f32.cu")


def kernel_source_hash():
    d = os.path.join(ROOT, "paper_2506_21804_gb300", "csrc")
    hs = hashlib.sha256()
    for f in KERNEL_FILES:
        hs.update(open(os.path.join(d, f), "rb").read())
    return hs.hexdigest()[:16]


# ---- CPU oracle (baseline leg and reference arm) ----------------------------------------------------------
def oracle_slab_rate(nz_slab, steps, seed=550):
    """Oracle GLUPS on a 256 x 256 x nz_slab periodic slab of the channel workload (nz_slab = 256 is
    the whole workload)."""
    from oracle import oracle as O
    from paper_2506_21804_gb300 import inputs as I
    w = I.channel(nx=256, ny=256, nz=nz_slab, seed=seed, dtype=np.float32)
    o = O.Oracle(w.q, w.nx, w.ny, w.nz, w.tau, w.cs)
    o.set_faces(w.faces)
    o.set_geometry(w.mask)
    o.set_force(*w.force)
    o.set_wall_model(True, w.kappa, w.E)
    o.init_equilibrium(np.asarray(w.rho0, np.float64), np.asarray(w.u0, np.float64))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return w.N * steps / dt / 1e9, O.get_threads(), w.N, dt


def run_reference(args):
    rank, _, world = dist_info()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2506_21804_gb300 import inputs as I
    nz_slab = 8
    w = I.channel(nx=256, ny=256, nz=nz_slab, seed=550, dtype=np.float32)
    o = O.Oracle(w.q, w.nx, w.ny, w.nz, w.tau, w.cs)
    o.set_faces(w.faces)
    o.set_geometry(w.mask)
    o.set_force(*w.force)
    o.set_wall_model(True, w.kappa, w.E)
    o.init_equilibrium(np.asarray(w.rho0, np.float64), np.asarray(w.u0, np.float64))
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = w.N * args.steps / dt / 1e9
    sample = f"oracle (FP64 C++, OpenMP) on a 256x256x{nz_slab} periodic slab of the channel, {args.steps} steps"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_cells": w.N},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": O.get_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---- GPU arm ---------------------------------------------------------------------------------------------------
def interior_kernel_name(code, q, storage, hrr):
    s = {"f32": "float", "f16": "__half", "bf16": "__nv_bfloat16"}[storage]
    if code == 2:
        return f"k_bulk_tma<{q}, {s}>"
    if code == 3:
        return f"k_bulk4r<{q}, {s}> (even steps) + k_bulk2r<{q}, {s}> (odd steps)"
    if code == 1:
        return f"k_bulk2r<{q}, {s}, HRR>" if hrr else f"k_bulk2r<{q}, {s}>"
    return f"k_bulk_hrr<{q}, {s}>" if hrr else f"k_bulk<{q}, {s}>"


def timed_glups(lat, steps, warmup):
    lat.step(warmup)
    lat.sync()
    ms = lat.step_timed(steps)
    return lat.N * steps / (ms[2] * 1e-3) / 1e9, ms


def parity_interior_us(lat, pairs=10):
    """Mean interior-kernel time of even and of odd steps (CUDA events, one step per timed call)."""
    acc = [0.0, 0.0]
    for _ in range(2 * pairs):
        parity = lat.info()["t"] & 1
        acc[parity] += lat.step_timed(1)[0]
    return {"even_us": acc[0] / pairs * 1e3, "odd_us": acc[1] / pairs * 1e3}


def adjoint_run(lbm, I, n, T, ckpt, W=None):
    """Differentiation workload: duct n^3, objective over the last W of T steps, checkpoint interval
    ckpt. The forward and backward are run twice (the first call allocates the checkpoints and the
    ring); GLUPS from the second call's device times."""
    W = W or max(1, T // 10)
    wd = I.duct(n=n, u_in=0.04, tau=0.6, sigma=8.0, dtype=np.float32)
    lat = lbm.Lattice.from_workload(wd, storage=lbm.F32)
    res = {}
    for rep in range(2):
        lat.init_equilibrium(np.asarray(wd.rho0, np.float32), np.asarray(wd.u0, np.float32))
        J = lat.objective_forward(T, W, 1, wd.nx - 2, ckpt=ckpt)
        g, _ = lat.objective_backward()
        rec, rev, fwd = lat.adjoint_timing()
        cells = wd.N * T
        res = {"cells": wd.N, "steps": T, "window": W, "checkpoint_interval": ckpt, "J": J,
               "forward_glups": cells / (fwd * 1e-3) / 1e9,
               "backward_glups": cells / ((rec + rev) * 1e-3) / 1e9,
               "recompute_glups": cells / (rec * 1e-3) / 1e9 if rec > 0 else None,
               "reverse_kernel_glups": cells / (rev * 1e-3) / 1e9,
               "backward_over_forward": fwd / (rec + rev),
               "grad_l2": float(np.linalg.norm(g))}
    lat.close()
    return res


def secondary(lbm, I, torch):
    """Shorter runs of the other forms of the metric."""
    out = {}
    # 16-bit storage on the same channel, with its deviation from FP32 after the same steps
    w = I.channel(nx=256, ny=256, nz=256, seed=550, dtype=np.float32)
    ref = lbm.Lattice.from_workload(w, storage=lbm.F32)
    ref.step(100)
    _, u32 = ref.moments(np.float32)
    g32, _ = timed_glups(ref, 40, 2)
    ref.close()
    out["channel_fp32_glups"] = g32
    for name, st in (("fp16", lbm.F16), ("bf16", lbm.BF16)):
        lat = lbm.Lattice.from_workload(w, storage=st)
        lat.step(100)
        _, u = lat.moments(np.float32)
        err = float(np.linalg.norm(u - u32) / np.linalg.norm(u32))
        g, ms = timed_glups(lat, 40, 2)
        info = lat.info()
        nb = info["N"] - info["n_solid"] - info["n_list"]
        per_launch = nb * 19 * 2 * 2 + info["N"]
        bw = per_launch / (ms[0] / 40 * 1e-3) / 1e9
        par = parity_interior_us(lat)
        par["even_gbs"] = per_launch / (par["even_us"] * 1e-6) / 1e9
        par["odd_gbs"] = per_launch / (par["odd_us"] * 1e-6) / 1e9
        out[f"channel_{name}"] = {"glups": g, "vs_fp32": g / g32, "u_rel_l2_vs_fp32_after_100_steps": err,
                                  "interior_kernel_gbs": bw, "interior_by_parity": par}
        lat.close()
    del u32
    # hybrid recursive regularised collision on the same channel: local stress only (sigma = 1) and
    # blended with the finite-difference strain (sigma = 1/2, reads and writes the velocity field)
    for sg in (1.0, 0.5):
        for name, st, pb in (("fp32", lbm.F32, 152), ("fp16", lbm.F16, 76)):
            lat = lbm.Lattice.from_workload(w, storage=st)
            lat.set_collision(lbm.HRR, sg)
            g, ms = timed_glups(lat, 40, 3)
            info = lat.info()
            nb = info["N"] - info["n_solid"] - info["n_list"]
            bw = (nb * (pb + (24 if sg < 1 else 0)) + info["N"]) / (ms[0] / 40 * 1e-3) / 1e9
            out[f"channel_hrr_sigma{sg:g}_{name}"] = {"glups": g, "vs_bgk_fp32": g / g32, "interior_kernel_gbs": bw}
            lat.close()
    # precision configuration: the canopy generator on 1024 x 512 x 256 (134M cells), FP32, FP16 and
    # BF16 storage: GLUPS of each, and the velocity deviation of the 16-bit forms from FP32 after 100
    # steps from the same initial state
    wp = I.canopy(nx=1024, ny=512, nz=256, q=19, seed=2506, dtype=np.float32)
    fl = wp.mask != 1
    prec = {}
    up32 = None
    for name, st in (("fp32", lbm.F32), ("fp16", lbm.F16), ("bf16", lbm.BF16)):
        lat = lbm.Lattice.from_workload(wp, storage=st)
        lat.step(100)
        _, up = lat.moments(np.float32)
        g, ms = timed_glups(lat, 20, 2)
        info = lat.info()
        lat.close()
        prec[name] = {"glups": g, "interior_ms": ms[0] / 20, "rest_ms": (ms[2] - ms[0]) / 20,
                      "boundary_list_fraction": info["n_list"] / info["N"]}
        if up32 is None:
            up32 = up
        else:
            prec[name]["u_rel_l2_vs_fp32_after_100_steps"] = float(
                np.linalg.norm(up[:, fl] - up32[:, fl]) / np.linalg.norm(up32[:, fl]))
            prec[name]["vs_fp32"] = g / prec["fp32"]["glups"]
        del up
    del up32
    out["canopy1024x512x256_precision"] = prec
    # urban canopy, D3Q19 and D3Q27
    for q in (19, 27):
        wc = I.canopy(nx=512, ny=512, nz=256, q=q, seed=2506, dtype=np.float32)
        lat = lbm.Lattice.from_workload(wc, storage=lbm.F32)
        g, ms = timed_glups(lat, 20, 2)
        info = lat.info()
        # wall-model traffic beyond the populations: normal + distance (16 B) per WALL cell, the
        # reference velocity written and read (2 x 12 B) per reference cell, per cell of the grid
        wm_bytes = (info["n_wall"] * 16 + info["n_ref"] * 24) / info["N"]
        out[f"canopy512x512x256_d3q{q}_fp32"] = {"glups": g, "boundary_list_fraction": info["n_list"] / info["N"],
                                                 "interior_ms": ms[0] / 20, "list_ms": ms[1] / 20,
                                                 "wall_model_bytes_per_cell": wm_bytes,
                                                 "glups_non_solid": g * (info["N"] - info["n_solid"]) / info["N"]}
        lat.close()
    # the paper's full model on the canopy: HRR collision (sigma = 1/2) and the vortex-method inlet
    wc = I.canopy(nx=512, ny=512, nz=256, q=19, seed=2506, dtype=np.float32)
    lat = lbm.Lattice.from_workload(wc, storage=lbm.F32)
    lat.set_collision(lbm.HRR, 0.5)
    lat.set_vortex_inlet(200, 4.0, 0.1, 2506)
    g, ms = timed_glups(lat, 20, 3)
    out["canopy512x512x256_d3q19_hrr_vortex_fp32"] = {"glups": g, "interior_ms": ms[0] / 20,
                                                     "rest_ms": (ms[2] - ms[0]) / 20, "vortices": 200}
    lat.close()
    # adjoint on the 128^3 duct at the differentiation configuration: T = 1000 steps, objective over
    # the last 100, checkpoint interval 32; backward = segment recomputation + reverse sweep
    adj = adjoint_run(lbm, I, 128, 1000, 32, W=100)
    adj["backward_over_channel_fp32_forward"] = adj["backward_glups"] / g32
    out["duct128_adjoint_T1000"] = adj
    # the same with every state kept in HBM (1001 states, 160 GB): no recomputation in the backward
    try:
        adj1 = adjoint_run(lbm, I, 128, 1000, 1, W=100)
        adj1["backward_over_channel_fp32_forward"] = adj1["backward_glups"] / g32
        adj1["gradient_rel_diff_vs_checkpointed"] = abs(adj1["grad_l2"] - adj["grad_l2"]) / adj["grad_l2"]
        out["duct128_adjoint_T1000_every_state"] = adj1
    except Exception as e:  # reported, not hidden (e.g. not enough device memory)
        out["duct128_adjoint_T1000_every_state"] = {"error": repr(e)}
    return out


def run_sharded(args, rank, world):
    """N > 1: the channel 256 x 256 x (256 N) split into N z-slabs of 256 planes, one per rank, with
    the halo exchange of every step between neighbouring ranks (torch.distributed point-to-point
    messages of device buffers; weak scaling: per-rank work fixed). Time = max over ranks of the
    CUDA-event time of K steps including the exchanges."""
    import torch
    from paper_2506_21804_gb300 import inputs as I, lbm
    from paper_2506_21804_gb300.shard import RankSlab
    w = I.channel(nx=256, ny=256, nz=256 * world, seed=550, dtype=np.float32)
    sl = RankSlab(w, rank, world, storage=lbm.F32)
    sl.step(args.warmup)
    sl.sync()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    l0 = sl.lat.launch_count()
    e0.record(stream)
    sl.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    launches = (sl.lat.launch_count() - l0)
    t_ms = max_over_ranks(e0.elapsed_time(e1), world)
    cells = w.N  # all ranks' real cells
    value = cells * args.steps / (t_ms * 1e-3) / 1e9
    peak, peak_src = peaks()
    per_rank = (sl.z1 - sl.z0) * w.nx * w.ny
    step_bytes = per_rank * (2 * 19 * 4 + 1)
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("256x256x256", f"256x256x{256 * world}") + f", {world} z-slabs",
                   "cells": cells, "parallelism": f"z-slabs x{world} (halo exchange every step)",
                   "l2": "state > 129 MB L2 between steps, no flush needed"},
        "step_roofline": {"bytes_per_step_per_rank": step_bytes,
                          "achieved_gbs": step_bytes / (t_ms / args.steps * 1e-3) / 1e9,
                          "frac": step_bytes / (t_ms / args.steps * 1e-3) / 1e9 / peak, "peak_source": peak_src},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary forms and the CPU baseline")
    ap.add_argument("--size", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="grid size (the headline channel is 256 256 256; other sizes are for profiling)")
    ap.add_argument("--workload", default="channel", choices=["channel", "canopy", "duct"],
                    help="channel (headline); the urban canopy or the differentiation duct (profiling)")
    ap.add_argument("--kernel", default="plain", choices=["plain", "staged"], help="interior kernel variant")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="population storage (the headline is f32; the others are for profiling)")
    ap.add_argument("--lattice", type=int, default=19, choices=[19, 27], help="velocity set (profiling)")
    ap.add_argument("--collision", default="bgk", choices=["bgk", "hrr"], help="collision model (profiling)")
    ap.add_argument("--sigma", type=float, default=1.0, help="HRR hybridisation factor")
    ap.add_argument("--vortex", type=int, default=0, help="vortex-method inlet with this many vortices (canopy)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    rank, local, world = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2506_21804_gb300 import build, inputs as I, lbm
    build.build()
    lbm.lib()
    if world > 1 and args.workload == "channel":
        run_sharded(args, rank, world)
        import torch.distributed as dist
        dist.destroy_process_group()
        return

    if args.workload == "duct":
        n = (args.size or (128, 128, 128))[0]
        res = adjoint_run(lbm, I, n, max(args.steps, 2) // 2 * 2, 1)
        print(json.dumps({"metric": "adjoint GLUPS (duct, checkpointed backward)", "value": res["backward_glups"],
                          "unit": "GLUPS", "config": {"workload": f"duct {n}^3 D3Q19 FP32 porosity"}, "adjoint": res}))
        return
    headline = (args.workload == "channel" and args.size in (None, [256, 256, 256]) and args.storage == "f32"
                and args.lattice == 19 and args.collision == "bgk" and args.vortex == 0)
    storage = {"f32": lbm.F32, "f16": lbm.F16, "bf16": lbm.BF16}[args.storage]
    esize = 4 if args.storage == "f32" else 2
    if args.workload == "channel":
        nx, ny, nz = args.size or (256, 256, 256)
        w = I.channel(nx=nx, ny=ny, nz=nz, seed=550 + rank, q=args.lattice, dtype=np.float32)
        wname = WORKLOAD.replace("256x256x256", f"{nx}x{ny}x{nz}").replace("D3Q19", f"D3Q{args.lattice}").replace(
            "FP32 storage", f"{args.storage.upper()} storage")
    else:
        nx, ny, nz = args.size or (512, 512, 256)
        w = I.canopy(nx=nx, ny=ny, nz=nz, q=args.lattice, seed=2506, dtype=np.float32)
        wname = f"urban canopy {nx}x{ny}x{nz} D3Q{args.lattice} Smagorinsky + wall function, log-law inlet, {args.storage.upper()}"
    stream = torch.cuda.current_stream()
    lat = lbm.Lattice.from_workload(w, storage=storage)
    lat.set_stream(stream)
    if args.kernel == "staged":
        lat.set_option(lbm.OPT_KERNEL, lbm.KERNEL_STAGED)
    hrr = args.collision == "hrr"
    if hrr:
        lat.set_collision(lbm.HRR, args.sigma)
        wname += f", HRR collision sigma={args.sigma}"
    if args.vortex > 0:
        lat.set_vortex_inlet(args.vortex, 4.0, 0.1, 2506)
        wname += f", vortex inlet n={args.vortex}"
    info = lat.info()
    kname = interior_kernel_name(lat.interior_kernel(), args.lattice, args.storage, hrr)
    wms = lat.step_timed(args.warmup)   # the warm-up steps, timed only to size the repeats below
    lat.sync()
    # The timed region (K = --steps steps) is repeated until the repeats together last >= 0.5 s; the
    # median repeat is reported, so that ms_per_step * steps is one timed region of K steps.
    est_ms = wms[2] / args.warmup
    n_rep = int(min(200, max(1, np.ceil(500.0 / max(est_ms * args.steps, 1e-3)))))

    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.3)
    runs = []
    timed_launches = 0
    # The canopy with the wall function stays bounded for a few hundred steps from its impulsive
    # start; between repeats its state is re-initialised (outside the timed region) before it would
    # pass 300 steps. The channel runs on.
    since = args.warmup
    reinit_after = 300 if args.workload == "canopy" else None
    n_init = 0
    for _ in range(n_rep):
        if reinit_after is not None and since + args.steps > reinit_after:
            lat.init_equilibrium(np.asarray(w.rho0, np.float32), np.asarray(w.u0, np.float32))
            lat.step(args.warmup)
            lat.sync()
            since = args.warmup
            n_init += 1
        since += args.steps
        barrier(world)
        torch.cuda.synchronize()
        l0 = lat.launch_count()
        m = lat.step_timed(args.steps)
        timed_launches += lat.launch_count() - l0
        torch.cuda.synchronize()
        barrier(world)
        runs.append((max_over_ranks(m[2], world), m))
    clocks = clk.stop()
    launches_per_region = timed_launches // n_rep
    runs.sort(key=lambda r: r[0])
    ms = runs[len(runs) // 2][1]

    t_ms = runs[len(runs) // 2][0]
    value = world * w.N * args.steps / (t_ms * 1e-3) / 1e9
    n_bulk = info["N"] - info["n_solid"] - info["n_list"]
    # HRR with sigma < 1 also reads the previous velocity field and writes its own (3 values each)
    per_cell = 2 * w.q * esize + (2 * 3 * (8 if args.storage == "f64" else 4) if (hrr and args.sigma < 1) else 0)
    bytes_bulk = n_bulk * per_cell + info["N"] * 1
    bulk_ms = ms[0] / args.steps
    peak, peak_src = peaks()
    achieved = bytes_bulk / (bulk_ms * 1e-3) / 1e9
    traffic = kernel_traffic("interior", "channel256") if headline else None
    step_bytes = (info["N"] - info["n_solid"]) * per_cell + info["N"]

    # end to end through the C ABI with pinned host buffers: geometry + initial state in, fields out
    rho_h = torch.from_numpy(np.ascontiguousarray(w.rho0, np.float32)).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(w.u0, np.float32)).pin_memory()
    mask_h = torch.from_numpy(np.ascontiguousarray(w.mask, np.uint8)).pin_memory()
    rho_o = torch.empty(w.N, dtype=torch.float32, pin_memory=True)
    u_o = torch.empty((3, w.N), dtype=torch.float32, pin_memory=True)
    reps = []
    for _ in range(5):                  # median of five runs of the whole sequence
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        lat.set_geometry(mask_h)
        lat.init_equilibrium(rho_h, u_h)
        for _ in range(args.steps):
            lat.step(1)
            lat.sync()                  # every step: its status word (NaN/timeout checks) read back
        lat.moments(np.float32, rho_o, u_o)
        torch.cuda.synchronize()
        reps.append(max_over_ranks(time.perf_counter() - t0, world))
    e2e_s = sorted(reps)[2]
    # the fixed part of the e2e sequence, phase by phase (each followed by a synchronisation)
    fixed = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.set_geometry(mask_h)
    torch.cuda.synchronize()
    fixed["set_geometry_ms"] = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    lat.init_equilibrium(rho_h, u_h)
    lat.sync()
    fixed["init_equilibrium_ms"] = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    lat.moments(np.float32, rho_o, u_o)
    torch.cuda.synchronize()
    fixed["moments_to_host_ms"] = (time.perf_counter() - t0) * 1e3
    h2d = mask_h.numel() + 4 * (rho_h.numel() + u_h.numel())
    d2h = 4 * (rho_o.numel() + u_o.numel()) + 4 * args.steps
    e2e = {"value": world * w.N * args.steps / e2e_s / 1e9, "unit": "GLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "includes": "set_geometry(pinned host mask) + init_equilibrium(pinned host rho,u) + per step: "
                       "step + status read-back + at the end moments(pinned host); median of 5 runs",
           "runs_s": reps, "fixed_cost": fixed}
    lat.close()

    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {"workload": wname, "kernel": args.kernel, "cells": w.N, "parallelism": f"replicas x{world}",
                   "l2": "state of 2.6 GB > 129 MB L2 between steps, no flush needed",
                   "timed_repeats": n_rep, "repeat_ms": [r[0] for r in runs],
                   "non_solid_cells": info["N"] - info["n_solid"], "boundary_list_cells": info["n_list"]},
        "roofline": {"bound": "hbm", "kernel": kname + " (interior cells)", "achieved": achieved, "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "bytes_per_launch": bytes_bulk, "launch_ms": bulk_ms,
                     "share_of_step": ms[0] / ms[2]},
        "step_roofline": {"bytes_per_step": step_bytes, "achieved_gbs": step_bytes / (t_ms / args.steps * 1e-3) / 1e9,
                          "frac": step_bytes / (t_ms / args.steps * 1e-3) / 1e9 / peak},
        "e2e": e2e,
        "glups_non_solid": world * (info["N"] - info["n_solid"]) * args.steps / (t_ms * 1e-3) / 1e9,
        "gpu_launches": launches_per_region,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extra and headline:
        try:
            line["extra"] = secondary(lbm, I, torch)
        except Exception as e:  # reported, not hidden
            line["extra"] = {"error": repr(e)}
        slab, nst = 256, 12
        v, cores, cells, dt = oracle_slab_rate(slab, nst)
        line["cpu_baseline"] = {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                                "sample": f"the full 256^3 channel ({cells} cells), {nst} steps, {dt:.1f} s"}
        # the same oracle on one thread (a 256 x 256 x 16 slab of the channel, 2 steps)
        from oracle import oracle as O
        O.set_threads(1)
        v1, _, cells1, dt1 = oracle_slab_rate(16, 2)
        O.set_threads(cores)
        line["cpu_baseline"]["single_thread"] = {"value": v1, "unit": "GLUPS", "cores": 1,
                                                 "sample": f"256x256x16 slab ({cells1} cells), 2 steps, {dt1:.1f} s"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

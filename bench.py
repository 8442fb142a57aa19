#!/usr/bin/env python
"""Forward + adjoint throughput of the differentiable volume renderer.

One step = one pass of the whole hot path over the 256^3 emission-absorption
workload: orbit camera -> forward march (Alg. 1) -> L2 loss seed ->
constant-memory adjoint (Alg. 2) with TF and camera gradients -> orbit
camera adjoint. Metric: ray samples (forward + adjoint) per second, in
Gsamples/s, i.e. samples / (t_forward + t_adjoint + the small kernels).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own replica of the workload (the rays
of different problems are independent; no collective on the data path) and
rank 0 prints one JSON line with the whole-job rate.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20          # > 126 MB L2
METRIC = "forward+adjoint Gsamples/s and % gather roofline vs plain FP32 at stated grad error"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ea_256")
    ap.add_argument("--tf-immediate", action="store_true", help="adjoint-immediate TF accumulation")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2107_12672_b300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources."""
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


class Clocks:
    """SM clock and throttle-reason sampling (NVML, every ~5 ms) in a thread
    during the timed region; falls back to nvidia-smi if NVML is missing."""
    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.stop_flag = False
        self.thread = None
        self.max_mhz = None
        self.t0 = None

    def _run(self):
        import pynvml
        h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
        self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM)
        while not self.stop_flag:
            sm = pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM)
            r = pynvml.nvmlDeviceGetCurrentClocksEventReasons(h)
            if self.t0 is not None:
                self.samples.append((sm, r))
            time.sleep(0.005)

    def start(self):
        try:
            import threading
            import pynvml
            pynvml.nvmlInit()
            self.thread = threading.Thread(target=self._run, daemon=True)
            self.thread.start()
            time.sleep(0.02)          # the sampler is running before the timed region starts
        except Exception:
            self.thread = None

    def mark(self):
        """Start of the timed region: samples from here on are kept."""
        self.t0 = time.perf_counter()

    def stop(self):
        if self.thread is None:
            return None
        self.stop_flag = True
        self.thread.join(timeout=2)
        if not self.samples:
            return None
        sm = [s for s, _ in self.samples]
        reasons = sorted({n for _, r in self.samples for n, bit in self.REASONS.items() if r & bit})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(sm), "source": "nvml"}


# ------------------------------------------------------------ the workload
class Workload:
    """Device-resident inputs of one replica plus everything the step needs."""

    def __init__(self, name, device, tf_immediate=False):
        import torch

        import paper_2107_12672_b300 as dvr
        from paper_2107_12672_b300 import synthetic as syn
        self.dvr = dvr
        self.torch = torch
        w = syn.workload(name)
        self.w = w
        self.device = device
        self.vol = [torch.as_tensor(v).to(device) for v in w.volumes]
        self.tf = torch.as_tensor(w.tf).to(device).contiguous()
        self.params = torch.as_tensor(w.orbit.astype(np.float32)).to(device).contiguous()
        self.scene = dvr.Scene.make(self.vol, self.tf, w.model, w.views)
        self.eye = torch.empty((len(w.views), 3), device=device)
        self.image = torch.empty((self.scene.pixels, self.scene.channels), device=device)
        self.aux = torch.empty((self.scene.pixels, 2), device=device)
        self.gimg = torch.empty_like(self.image)
        self.loss = torch.zeros(1, device=device)
        self.g_tf = torch.zeros_like(self.tf)
        self.g_eye = torch.zeros_like(self.eye)
        self.g_par = torch.zeros_like(self.params)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.tf_immediate = tf_immediate
        # target: the same view rendered with a second transfer function
        tft = torch.as_tensor(w.target["tf"]).to(device).contiguous()
        dvr.orbit_eye(self.params, eye=self.eye)
        tscene = dvr.Scene.make(self.vol, tft, w.model, w.views)
        self.target, _ = dvr.forward(None, None, None, None, self.eye, w.step_voxels, scene=tscene)
        dvr.forward(None, None, None, None, self.eye, w.step_voxels, scene=self.scene, image=self.image,
                    aux=self.aux, sample_count=self.count)
        torch.cuda.synchronize()
        self.samples_per_pass = int(self.count.item())

    def step(self, ev=None):
        """One pass: 5 kernels of the library. `ev` = (fwd_start, fwd_end,
        bwd_start, bwd_end) events to bracket the two march kernels."""
        dvr, w = self.dvr, self.w
        self.loss.zero_()
        self.g_tf.zero_()
        self.g_eye.zero_()
        self.g_par.zero_()
        dvr.orbit_eye(self.params, eye=self.eye)
        if ev:
            ev[0].record()
        dvr.forward(None, None, None, None, self.eye, w.step_voxels, scene=self.scene, image=self.image,
                    aux=self.aux)
        if ev:
            ev[1].record()
        dvr.loss_l2(self.image, self.target, 1.0 / self.image.numel(), grad_image=self.gimg, loss=self.loss)
        if ev:
            ev[2].record()
        dvr.backward(None, None, None, None, self.eye, w.step_voxels, self.aux, self.gimg,
                     scene=self.scene, grads={"tf": self.g_tf, "eye": self.g_eye}, want=("tf", "eye"),
                     tf_immediate=self.tf_immediate)
        if ev:
            ev[3].record()
        dvr.orbit_eye_backward(self.params, self.g_eye, grad_params=self.g_par)

    LAUNCHES_PER_STEP = 5


def algorithmic_bytes(wl, kernel):
    """Bytes the method must move per launch: 8 trilinear corners per sample
    (element size of the volume) plus per-pixel image/aux/seed traffic."""
    e = wl.vol[0].element_size()
    px = wl.scene.pixels
    if kernel == "forward":
        return wl.samples_per_pass * 8 * e + px * (16 + 8)
    return wl.samples_per_pass * 8 * e + px * (16 + 8)


# -------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = Workload(args.workload, dev, args.tf_immediate)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.mark()
    t0 = time.perf_counter()
    for k in range(K):
        flush.zero_()                     # evict the volume from L2 between steps
        st[k].record()
        wl.step(evs[k])
        en[k].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()

    step_ms = float(np.mean([s.elapsed_time(e) for s, e in zip(st, en)]))
    fwd_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    bwd_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in evs]))
    if world > 1:
        t = torch.tensor([step_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())

    samples = wl.samples_per_pass                  # per pass; forward and adjoint each visit them
    value = world * samples / (step_ms * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(wl, args, world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl.w, budget_s=12.0)

    if rank == 0:
        hbm, src = peaks()
        dom = "backward" if bwd_ms >= fwd_ms else "forward"
        dur = bwd_ms if dom == "backward" else fwd_ms
        achieved = algorithmic_bytes(wl, dom) / (dur * 1e-3) / 1e9
        line = {
            "metric": METRIC,
            "value": round(value, 4),
            "unit": "Gsamples/s",
            "n_gpus": world,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": round(step_ms, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic (seeded 3-octave value noise, seeded TF; no dataset)",
            "config": {
                "workload": args.workload,
                "volume": "256^3 f32 value noise",
                "tf_rows": int(wl.tf.shape[0]),
                "image": "512x512 perspective, distance 2.5, fov 45 deg",
                "step_voxels": wl.w.step_voxels,
                "gradients": ["tf", "camera yaw/pitch/distance"],
                "samples_per_pass": samples,
                "l2": "flushed between timed steps (512 MiB write)",
                "tf_accumulation": "immediate" if args.tf_immediate else "delayed (shared memory)",
                "parallelism": f"replicas x{world}",
            },
            "forward_ms": round(fwd_ms, 4),
            "adjoint_ms": round(bwd_ms, 4),
            "forward_gsamples_s": round(samples / (fwd_ms * 1e-3) / 1e9, 3),
            "adjoint_gsamples_s": round(samples / (bwd_ms * 1e-3) / 1e9, 3),
            "wall_s_timed_region": round(wall, 4),
            "roofline": {
                "kernel": dom,
                "bound": "hbm",
                "achieved": round(achieved, 2),
                "peak": hbm,
                "unit": "GB/s",
                "frac": round(achieved / hbm, 4),
                "peak_source": src,
                "traffic": profiled_traffic(f"{dom}_{args.workload}"),
                "bytes_per_sample": 8 * wl.vol[0].element_size(),
            },
            "clocks": clk,
            "gpu_launches": Workload.LAUNCHES_PER_STEP * K,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(wl, args, world):
    """Same metric through the public API with host buffers: every step
    copies its inputs (volume, TF, orbit parameters) from pinned host memory
    and reads back the loss and the gradients."""
    import torch
    dvr = wl.dvr
    h_vol = torch.as_tensor(wl.w.volumes[0]).pin_memory()
    h_tf = torch.as_tensor(wl.w.tf).pin_memory()
    h_par = torch.as_tensor(wl.w.orbit.astype(np.float32)).pin_memory()
    o_loss = torch.empty(1).pin_memory()
    o_tf = torch.empty_like(h_tf).pin_memory()
    o_par = torch.empty_like(h_par).pin_memory()
    d_vol = wl.vol[0]

    def one():
        d_vol.copy_(h_vol, non_blocking=True)
        wl.tf.copy_(h_tf, non_blocking=True)
        wl.params.copy_(h_par, non_blocking=True)
        wl.step()
        o_loss.copy_(wl.loss, non_blocking=True)
        o_tf.copy_(wl.g_tf, non_blocking=True)
        o_par.copy_(wl.g_par, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = (time.perf_counter() - t0) / args.steps
    h2d = h_vol.numel() * 4 + h_tf.numel() * 4 + h_par.numel() * 4
    d2h = 4 + o_tf.numel() * 4 + o_par.numel() * 4
    return {"value": round(world * wl.samples_per_pass / dt / 1e9, 4), "unit": "Gsamples/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(dt * 1e3, 4)}


# ------------------------------------------------------ the CPU oracle arm
class OraclePass:
    """The oracle's forward + stored-state adjoint (with the L2 seed and the
    orbit chain) on a strided subset of the workload's rows; the target image
    is rendered once, untimed, as on the GPU side."""

    def __init__(self, w, stride):
        import oracle
        oracle.build()
        self.oracle = oracle
        self.w = w
        self.view = w.views[0]
        self.stride = stride
        self.eye = oracle.orbit_eye(w.orbit.astype(np.float32).astype(np.float64))[0]
        self.target, _, _ = oracle.render(w.volumes[0], w.target["tf"], w.model, self.view, self.eye,
                                          w.step_voxels)
        self.phase = 0

    def __call__(self):
        o, w, view = self.oracle, self.w, self.view
        rows = np.arange(self.phase, view.height, self.stride)
        self.phase = (self.phase + 1) % self.stride
        pix = (rows[:, None] * view.width + np.arange(view.width)[None, :]).reshape(-1).astype(np.int64)
        img, N, _ = o.render(w.volumes[0], w.tf, w.model, view, self.eye, w.step_voxels, pix=pix)
        G = 2.0 * (img - self.target[pix]) / self.target.size
        g = o.backward(w.volumes[0], w.tf, w.model, view, self.eye, w.step_voxels, G, pix=pix,
                       want=("tf", "eye"))
        o.orbit_eye_backward(w.orbit, g["eye"][None])
        return int(N.sum()), pix.size


def cpu_baseline(w, budget_s=12.0):
    op = OraclePass(w, stride=8)
    done, passes, rays = 0, 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        n, r = op()
        done += n
        rays += r
        passes += 1
    dt = time.perf_counter() - t0
    return {"value": round(done / dt / 1e9, 6), "unit": "Gsamples/s", "cores": op.oracle.threads(),
            "kind": "oracle",
            "sample": f"{passes} passes over every 8th row of the {w.views[0].width}x{w.views[0].height} "
                      f"image ({rays} rays, {done} samples; forward + L2 seed + stored-state adjoint, "
                      f"FP64, OpenMP) in {dt:.1f} s"}


def run_reference(args):
    """The oracle as the reference arm: rank 0 only, on the host cores; each
    step is a bounded sample (every 16th row) of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2107_12672_b300 import synthetic as syn
    w = syn.workload(args.workload)
    op = OraclePass(w, stride=16)
    for _ in range(args.warmup):
        op()
    t0 = time.perf_counter()
    n = rays = 0
    for _ in range(args.steps):
        a, b = op()
        n += a
        rays += b
    dt = time.perf_counter() - t0
    v = n / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "Gsamples/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "parallelism": "host cores"},
        "cpu_baseline": {"value": round(v, 6), "unit": "Gsamples/s", "cores": op.oracle.threads(),
                         "kind": "oracle",
                         "sample": f"each step: every 16th row of the {w.views[0].width}x{w.views[0].height} "
                                   f"image, forward + L2 seed + stored-state adjoint (FP64); "
                                   f"{rays} rays, {n} samples in {dt:.1f} s"},
        "e2e": {"value": round(v, 6), "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

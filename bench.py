#!/usr/bin/env python
"""Forward + adjoint throughput of the differentiable volume renderer.

One step = one pass of the whole hot path over the largest workload that
one GPU holds: a 1024^3 FP16 volume (value noise + 32 Gaussian blobs), a
32-point TF, 32 views of 2048^2 at step 0.25 voxel (135 G ray samples per
pass): forward march (Alg. 1) -> opacity-entropy loss and its seed
(Sec. 5.1) -> constant-memory adjoint (Alg. 2) with the volume, TF and
camera gradients. Metric: ray samples (each visited by the forward and by
the adjoint) per second of step, in Gsamples/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ea_fp16_1024|ea_256|absorption_64|tomo_256x64|ea_bf16_512]

Timing: the tile widths are autotuned per pass (L2 flushed before each timed
pass; views beyond the first four are left out of the tuning runs of
workloads whose step takes longer than a second); W warm-up steps, then K
steps each bracketed by CUDA events with a 512 MiB write flushing L2 between
steps, outside the brackets. `value` comes from the mean step of the step
captured once as a CUDA graph and replayed (--eager: launched step by
step; `ms_per_step_stats` gives the median, minimum and maximum of those K
steps). The secondary legs (forward / adjoint breakdown from eager steps,
e2e, the other storage form, the camera-gradient modes) run
`secondary_steps` steps each (e2e at least 6, K allowing), enough for
~6 s of work, so that the whole run ends within a few minutes. The 512^3 and 1024^3 workloads run in their
own BF16 / FP16 storage (the arithmetic is binary32 throughout) and
`storage_variants` times the other storage form of the same workload
(binary32 beside 16-bit). NVML samples the SM clock and throttle reasons
during the timed region. The roofline divides the adjoint's algorithmic
bytes by its event time and compares them with the measured HBM copy
bandwidth (MEASURED_PEAKS.json) and with the L2 / L1 / reduction ceilings
measured in the same run (dvr_probe); `traffic` is the DRAM bytes of the
committed ncu summary of that kernel, when it was taken on the kernel's
current sources. `e2e` copies the step's inputs from pinned host memory and
reads the loss and every gradient back every step, through the public
binding, the copies overlapped with the neighbouring steps' compute.
`cpu_baseline` times the FP64 oracle on a strided sample of the same rays
on the host cores. `accuracy` compares seeded pixels and the gradients of a
seed supported on them with the FP64 oracle, element by element.

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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ea_fp16_1024")
    ap.add_argument("--tf-immediate", action="store_true", help="adjoint-immediate TF accumulation")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default 8x4 ray tiles")
    ap.add_argument("--tile-width", type=int, default=0, help="fix the warp tile width (1..32)")
    ap.add_argument("--adjoint-tile-width", type=int, default=0,
                    help="with --tile-width: the adjoint's width (default: the same)")
    ap.add_argument("--no-variants", action="store_true", help="skip the BF16/FP16 storage comparison")
    ap.add_argument("--eager", action="store_true", help="time eagerly launched steps instead of a CUDA graph")
    ap.add_argument("--views", type=int, default=0,
                    help="keep only the first N views (a smaller case of the workload, e.g. for ncu)")
    ap.add_argument("--image", type=int, default=0, help="render every view at S x S pixels (smaller case)")
    ap.add_argument("--grid", type=int, default=0,
                    help="the 1024^3 workload's volume at N^3 vertices instead (smaller case, same generator)")
    ap.add_argument("--cells", type=int, default=-1, choices=(-1, 0, 1, 4, 8),
                    help="gather from the volumes' arrays (0) or cell layouts with records in row order (1) or "
                         "bricks of 4^3 or 8^3 cells (4, 8), remade inside every step (default: autotuned)")
    ap.add_argument("--cell-gradient", type=int, default=-1, choices=(-1, 0, 1),
                    help="accumulate the volume gradient per cell first (DVR_FLAG_CELL_GRADIENT) or not "
                         "(default: autotuned)")
    ap.add_argument("--persistent-scatter", type=int, default=-1, choices=(-1, 0, 1),
                    help="the volume-gradient adjoint as a persistent launch (DVR_FLAG_PERSISTENT_SCATTER) "
                         "or one tile per warp (default: autotuned)")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# the device sources a march kernel is compiled from (its own file, the
# shared device header and the launch declarations)
KERNEL_SOURCES = {"forward": ("dvr_forward.cu", "dvr_device.cuh", "dvr_launch.h"),
                  "backward": ("dvr_backward.cu", "dvr_backward.cuh", "dvr_backward_cells.cu",
                               "dvr_backward_cells4.cu", "dvr_backward_cells8.cu", "dvr_device.cuh",
                               "dvr_launch.h"),
                  # the colour-volume kernels (both passes in one file)
                  "forward_color": ("dvr_color.cu", "dvr_device.cuh", "dvr_launch.h"),
                  "backward_color": ("dvr_color.cu", "dvr_device.cuh", "dvr_launch.h")}


def kernel_source_hash(kernel: str):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2107_12672_b300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current sources of that kernel."""
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_source_hash(kernel):
        return None
    return float(m.group(1))


class _NVML:
    """Read-only NVML queries (clocks and clock-event reasons) through the
    driver's libnvidia-ml, for the GPU this process uses."""
    SM = 1          # NVML_CLOCK_SM

    def __init__(self, index):
        import ctypes
        import torch
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        rc = self.lib.nvmlInit_v2()
        if rc != 0:
            raise RuntimeError(f"nvmlInit_v2 returned {rc}")
        self.h = ctypes.c_void_p()
        bus = None
        p = torch.cuda.get_device_properties(index)
        if hasattr(p, "pci_bus_id") and hasattr(p, "pci_domain_id") and hasattr(p, "pci_device_id"):
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
        rc = -1
        if bus is not None:
            rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(self.h))
        if rc != 0:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h))
        if rc != 0:
            raise RuntimeError(f"no NVML handle for device {index} (bus {bus}): {rc}")
        reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self._reasons = reasons or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def clock(self):
        v = self.ct.c_uint()
        self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, self.ct.byref(v))
        return v.value

    def max_clock(self):
        v = self.ct.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, self.ct.byref(v))
        return v.value

    def reasons(self):
        v = self.ct.c_ulonglong()
        self._reasons(self.h, self.ct.byref(v))
        return v.value


class Clocks:
    """SM clock and clock-event-reason sampling (NVML, every ~5 ms) in a
    thread during the timed region."""
    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.stop_flag = False
        self.thread = None
        self.max_mhz = None
        self.t0 = None
        self.error = None

    def _run(self, nv):
        try:
            self.max_mhz = nv.max_clock()
            while not self.stop_flag:
                sm, r = nv.clock(), nv.reasons()
                if self.t0 is not None:
                    self.samples.append((sm, r))
                time.sleep(0.005)
            if self.t0 is not None:   # one more at the end of the region (regions shorter than 5 ms)
                self.samples.append((nv.clock(), nv.reasons()))
        except Exception as e:      # reported in the JSON line instead of the clocks
            self.error = f"{type(e).__name__}: {e}"[:200]

    def start(self):
        try:
            import threading
            nv = _NVML(self.index)
            self.thread = threading.Thread(target=self._run, args=(nv,), daemon=True)
            self.thread.start()
            time.sleep(0.02)          # the sampler is running before the timed region starts
        except Exception as e:
            self.thread = None
            self.error = f"{type(e).__name__}: {e}"[:200]

    def mark(self):
        """Start of the timed region: samples from here on are kept."""
        self.t0 = time.perf_counter()

    def stop(self):
        if self.thread is None:
            return {"error": self.error} if self.error else None
        self.stop_flag = True
        self.thread.join(timeout=2)
        if not self.samples:
            return {"error": self.error or "no samples"}
        sm = [s for s, _ in self.samples]
        reasons = sorted({n for _, r in self.samples for n, bit in self.REASONS.items() if r & bit})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(sm), "source": "nvml"}


# ------------------------------------------------------------ the workload
class Workload:
    """Device-resident inputs of one replica of a named workload plus the
    buffers a step needs. The volume and the TF are stored in the
    workload's own dtypes (BF16 / FP16 for the 512^3 and 1024^3 workloads)
    unless others are given (the FP32 form is the plain one)."""

    def __init__(self, name, device, tf_immediate=False, vol_dtype=None, tf_dtype=None, views=0, image=0,
                 cells=False, cell_gradient=False, grid=0):
        import dataclasses

        import torch

        import paper_2107_12672_b300 as dvr
        from paper_2107_12672_b300 import synthetic as syn
        self.dvr = dvr
        self.torch = torch
        w = syn.workload(name)
        # a smaller case of the same workload (profiling stand-ins): its
        # first `views` views, each `image` pixels square
        if views:
            w.views, w.eye = w.views[:views], w.eye[:views]
            if w.orbit is not None:
                w.orbit = w.orbit[:views]
        if image:
            w.views = [dataclasses.replace(v, width=image, height=image) for v in w.views]
        if grid and name == "ea_fp16_1024":
            w.target["n"] = grid
        self.reduced = ({"views": views or None, "image": image or None, "grid": grid or None}
                        if (views or image or grid) else None)
        self.w = w
        self.name = name
        self.device = device
        # the workload's own storage unless another is asked for
        vdt = getattr(torch, vol_dtype or w.volume_dtype)
        tdt = getattr(torch, tf_dtype or w.tf_dtype)
        if name == "ea_fp16_1024":
            w.volumes = [None]
            self.vol = [syn.large_volume(w.target["n"], device=device).to(vdt)]
        else:
            self.vol = [torch.as_tensor(v).to(device=device, dtype=vdt) for v in w.volumes]
        self.ea = w.model == "emission_absorption"
        self.tf = torch.as_tensor(w.tf).to(device=device, dtype=tdt).contiguous() if self.ea else None
        self.configure(cells, cell_gradient)
        self.orbit = w.orbit is not None
        if self.orbit:
            self.params = torch.as_tensor(w.orbit.astype(np.float32)).to(device).contiguous()
            self.eye = torch.empty((len(w.views), 3), device=device)
            dvr.orbit_eye(self.params, eye=self.eye)
        else:
            self.eye = torch.as_tensor(w.eye).to(device).contiguous()
        self.image = torch.empty((self.scene.pixels, self.scene.channels), device=device)
        self.aux = torch.empty((self.scene.pixels, 2), device=device)
        self.gimg = torch.empty_like(self.image)
        self.want = tuple({"volume": "volume", "tf": "tf", "camera": "eye"}[g] for g in w.grads)
        self.use_outputs(self.make_outputs())
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.tf_immediate = tf_immediate
        self.persistent_scatter = False
        # target image: the same views with the second TF or the second volume
        if "tf" in w.target:
            tft = torch.as_tensor(w.target["tf"]).to(device=device, dtype=tdt).contiguous()
            tscene = dvr.Scene.make(self.vol, tft, w.model, w.views)
        elif "volume" in w.target:
            tv = [torch.as_tensor(w.target["volume"]).to(device=device, dtype=vdt)]
            tscene = dvr.Scene.make(tv, self.tf, w.model, w.views)
        else:
            tscene = None
        if tscene is not None:
            self.target, _ = dvr.forward(None, None, None, None, self.eye, w.step_voxels, scene=tscene)
        else:
            self.target = torch.zeros_like(self.image)
        dvr.forward(None, None, None, None, self.eye, w.step_voxels, scene=self.scene, image=self.image,
                    aux=self.aux, sample_count=self.count)
        torch.cuda.synchronize()
        self.samples_per_pass = int(self.count.item())
        # our kernels per step (configure): forward, loss (the entropy loss is
        # two), adjoint, orbit and its adjoint, the cell layouts and the
        # cell-gradient passes

    def make_outputs(self):
        """A set of the step's outputs: the loss and the small gradients as
        views of one buffer, zeroed with one fill per step (each part starts
        on a 16-byte boundary), and the volume gradients."""
        import torch
        parts = [("loss", (1,))]
        if "tf" in self.want:
            parts.append(("tf", (self.tf.shape[0], 4)))
        if "eye" in self.want:
            parts.append(("eye", tuple(self.eye.shape)))
            if self.orbit:
                parts.append(("par", tuple(self.params.shape)))
        sizes = [int(np.prod(shape)) for _, shape in parts]
        offs = np.concatenate([[0], np.cumsum([(n + 3) // 4 * 4 for n in sizes])])
        small = torch.zeros(int(offs[-1]), device=self.device)
        views = {name: small[o:o + n].view(shape) for (name, shape), o, n in zip(parts, offs, sizes)}
        out = {"small": small, "loss": views["loss"], "grads": {}, "g_par": views.get("par")}
        if "volume" in self.want:
            out["grads"]["volume"] = [torch.zeros(v.shape, device=self.device) for v in self.vol]
        if "tf" in self.want:
            out["grads"]["tf"] = views["tf"]
        if "eye" in self.want:
            out["grads"]["eye"] = views["eye"]
        return out

    def use_outputs(self, out):
        """Make `out` (from make_outputs) the set that step() writes."""
        self.outputs = out
        self.small, self.loss, self.grads, self.g_par = out["small"], out["loss"], out["grads"], out["g_par"]

    def result_tensors(self):
        """The tensors of the current output set that a user reads back
        after a step: the loss and every gradient."""
        outs = [self.loss]
        for k, g in self.grads.items():
            if k == "eye" and self.orbit:
                outs.append(self.g_par)
            else:
                outs.extend(g if isinstance(g, list) else [g])
        return outs

    def configure(self, cells, cell_gradient):
        """Gather from the volumes' arrays (cells 0) or their cell layouts
        with records in row order (1) or 4^3 bricks (4), remade from the
        volumes at the start of every step; accumulate the volume gradient
        per cell first (with a workspace of 32 bytes per record, allocated
        once) or into the vertex array."""
        import torch
        dvr, w = self.dvr, self.w
        if w.model == "color":          # colour volumes gather their corners from the array only
            cells, cell_gradient = 0, False
        self.use_cells = int(cells)
        self.cells = [dvr.make_cells(v, brick=self.use_cells) for v in self.vol] if cells else None
        self.scene = dvr.Scene.make(self.vol, self.tf, w.model, w.views, cells=self.cells,
                                    cells_brick=self.use_cells or 1)
        self.cell_gradient = bool(cell_gradient) and "volume" in tuple(w.grads)
        self.cg_ws = (torch.empty(dvr.cell_workspace_bytes(self.scene), dtype=torch.uint8, device=self.device)
                      if self.cell_gradient else None)
        self.launches_per_step = 3 + (1 if w.loss == "entropy" else 0) + (2 if w.orbit is not None else 0) + \
            (len(self.vol) if self.use_cells else 0) + (len(self.vol) if self.cell_gradient else 0)

    def zero(self):
        self.small.zero_()
        for t in self.grads.get("volume", []):
            t.zero_()

    def step(self, ev=None, scene=None):
        """One pass of the path. `ev` = (fwd_start, fwd_end, bwd_start,
        bwd_end) events bracket the two march kernels; `scene` replaces the
        workload's own (the same views over another volume buffer)."""
        dvr, w = self.dvr, self.w
        sc = scene or self.scene
        self.zero()
        if sc.cells is not None:
            for v, c in zip(sc.volumes, sc.cells):
                dvr.make_cells(v, out=c, brick=sc.cells_brick)
        if self.orbit:
            dvr.orbit_eye(self.params, eye=self.eye)
        if ev:
            ev[0].record()
        dvr.forward(None, None, None, None, self.eye, w.step_voxels, scene=sc, image=self.image, aux=self.aux)
        if ev:
            ev[1].record()
        if w.loss == "entropy":
            dvr.loss_entropy(self.image, sc, 1.0 / len(w.views), grad_image=self.gimg, loss=self.loss)
        else:
            dvr.loss_l2(self.image, self.target, 1.0 / self.image.numel(), grad_image=self.gimg, loss=self.loss)
        if ev:
            ev[2].record()
        dvr.backward(None, None, None, None, self.eye, w.step_voxels, self.aux, self.gimg, scene=sc,
                     grads=self.grads, want=self.want, tf_immediate=self.tf_immediate,
                     cell_gradient=self.cell_gradient, workspace=self.cg_ws,
                     persistent_scatter=self.persistent_scatter)
        if ev:
            ev[3].record()
        if self.orbit and "eye" in self.want:
            dvr.orbit_eye_backward(self.params, self.grads["eye"], grad_params=self.g_par)

    def describe(self):
        w = self.w
        v = self.vol[0]
        return {
            "workload": self.name,
            "volume": f"{'x'.join(str(s) for s in reversed(v.shape))} {str(v.dtype).replace('torch.', '')}",
            "model": w.model,
            "tf_rows": int(self.tf.shape[0]) if self.tf is not None else 0,
            "tf_dtype": str(self.tf.dtype).replace("torch.", "") if self.tf is not None else None,
            "views": len(w.views),
            "pixels": self.scene.pixels,
            "step_voxels": w.step_voxels,
            "gradients": list(w.grads),
            "samples_per_pass": self.samples_per_pass,
            "loss": {"l2": "L2 against the target image", "entropy": "opacity entropy (Sec. 5.1), maximised"}[w.loss],
            "note": w.note,
            "reduced_case": self.reduced,
            "gather_layout": {0: "the volume's array", 1: "cell records in row order (remade every step)",
                              4: "cell records in 4^3 bricks (remade every step)"}[self.use_cells],
            "volume_gradient_scatter": "per cell, then per vertex" if self.cell_gradient else "per vertex",
            "volume_gradient_launch": ("persistent (tile queue)"
                                       if self.persistent_scatter and v.element_size() == 2 else "one tile per warp")
            if "volume" in self.want else None,
        }


def gather_bytes(wl):
    """Bytes of the 8 trilinear corners of one sample: the volume's element
    size, times 4 for a colour volume (r, g, b, tau per vertex)."""
    return 8 * wl.vol[0].element_size() * (4 if wl.w.model == "color" else 1)


def algorithmic_bytes(wl, kernel):
    """Bytes the method must move per launch: 8 trilinear corners per sample
    plus per-pixel image/aux/seed traffic; the adjoint adds 8 FP32
    read-modify-writes per sample (per channel of a colour volume) when it
    scatters the volume gradient."""
    px = wl.scene.pixels
    b = wl.samples_per_pass * gather_bytes(wl) + px * (4 * wl.scene.channels + 8)
    if kernel == "backward" and "volume" in wl.want:
        b += wl.samples_per_pass * 8 * 4 * 2 * (4 if wl.w.model == "color" else 1)
    return b


def probe_ceilings(dev):
    """On-chip ceilings measured with the library's probes on this device
    (CUDA events around each; best of 3): L2 read GB/s (a 32 MiB buffer,
    loads that bypass L1), L1 read GB/s (32 KB per block, 4 blocks per SM)
    and L2 scattered-reduction throughput (Gops/s, 2^22 words)."""
    import torch
    from paper_2107_12672_b300 import _abi
    lib = _abi.load()
    stream = torch.cuda.current_stream().cuda_stream
    sink = torch.zeros(1, device=dev)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    cases = {"l2_read_gbs": (_abi.DVR_PROBE_L2_READ, 32 << 20, 40),
             "l1_read_gbs": (_abi.DVR_PROBE_L1_READ, 4 * nsm * 32768, 400),
             "l2_red_gops": (_abi.DVR_PROBE_L2_RED, 16 << 20, 8)}
    out = {}
    for name, (kind, nbytes, reps) in cases.items():
        buf = torch.zeros(nbytes // 4, device=dev)
        best = None
        for _ in range(4):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            _abi.check(lib.dvr_probe(kind, buf.data_ptr(), nbytes, reps, sink.data_ptr(), stream), "dvr_probe")
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) * 1e-3
            best = t if best is None else min(best, t)
        work = nbytes * reps if name != "l2_red_gops" else (nbytes // 4) * reps
        out[name] = round(work / best / 1e9, 1)
        del buf
    return out


def _errs(a, b, slack=None):
    """The parity tests' two error forms: per element, (|a - b| - slack)+ /
    max(|b|, 1e-3 max|b|) (the bar: 1e-5 for images, 1e-3 for gradients),
    and the max-norm form |a - b| / (|b| + max|b|)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(a - b)
    s = np.abs(b).max() if b.size else 0.0
    if s == 0:
        return {"per_element": float(d.max()) if d.size else 0.0, "max_norm": float(d.max()) if d.size else 0.0}
    out = {"max_norm": float((d / (np.abs(b) + s)).max()),
           "per_element": float((d / np.maximum(np.abs(b), 1e-3 * s)).max())}
    if slack is not None:
        out["per_element_beyond_kink_bound"] = float((np.maximum(d - slack, 0.0) / np.maximum(np.abs(b), 1e-3 * s)).max())
    return out


def sampled_accuracy(wl, per_view=64, n_views=4, seed=21):
    """accuracy() for workloads whose views are too large for the oracle to
    render whole: seeded pixel samples of the first views, with dL/d(image)
    non-zero only on them, so the oracle computes the exact gradients of the
    same seed. The volume gradient is compared on every vertex those rays
    read (the oracle returns it compactly there; a 1024^3 volume needs no
    dense binary64 array) and must be exactly zero on every other vertex.
    `per_element_beyond_kink_bound` subtracts, per element, the oracle's
    bound on what binary32 rounding may change where a sample lies on a cell
    face or TF control point (the parity tests' slack)."""
    import torch

    import oracle
    dvr, w = wl.dvr, wl.w
    rng = np.random.default_rng(seed)
    eye = torch.as_tensor(w.eye).to(wl.device).contiguous()
    img, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=wl.scene)
    nc = img.shape[1]
    offs = np.cumsum([0] + [v.width * v.height for v in w.views])
    views = w.views[:n_views]
    G = torch.zeros_like(img)
    picks, Gs = [], []
    for k, v in enumerate(views):
        pk = np.sort(rng.choice(v.width * v.height, size=min(per_view, v.width * v.height), replace=False))
        gk = rng.normal(size=(pk.size, nc)).astype(np.float32)
        picks.append(pk)
        Gs.append(gk)
        G[torch.as_tensor(offs[k] + pk, device=wl.device)] = torch.as_tensor(gk, device=wl.device)
    want = tuple(wl.want)
    g = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=wl.scene, want=want)
    torch.cuda.synchronize()
    imgh = np.concatenate([img[offs[k] + torch.as_tensor(picks[k], device=wl.device)].cpu().numpy()
                           for k in range(len(views))])
    del img, aux, G
    vol = wl.vol[0].float().cpu().numpy()
    tf = wl.tf.float().cpu().numpy().astype(np.float64) if wl.tf is not None else None
    sel = None
    if "volume" in want:
        sel = np.unique(np.concatenate([oracle.touched(vol.shape, view, w.eye[k], w.step_voxels, pix=picks[k])
                                        for k, view in enumerate(views)]))
        ref_vol = np.zeros((sel.size,) + vol.shape[3:])     # four entries per vertex of a colour volume
        amb_vol = np.zeros(sel.size)
    ref_tf = np.zeros((tf.shape[0], 4)) if (tf is not None and "tf" in want) else None
    ref_img, e_eye = [], []
    for k, view in enumerate(views):
        ri, _, _ = oracle.render(vol, tf, w.model, view, w.eye[k], w.step_voxels, pix=picks[k])
        ref_img.append(ri)
        rg = oracle.backward(vol, tf, w.model, view, w.eye[k], w.step_voxels, Gs[k], pix=picks[k],
                             want=want, margin=2.0, sel=sel)
        if sel is not None:
            ref_vol += rg["volume"]
            amb_vol += rg["volume_ambiguity"]
        if ref_tf is not None:
            ref_tf += rg["tf"]
        if "eye" in rg:
            e_eye.append((g["eye"][k].cpu().numpy(), rg["eye"], rg["eye_ambiguity"]))
    out = {"reference": f"FP64 oracle, same stored inputs, {len(views)} views x {per_view} seeded pixels "
                        "(dL/d(image) non-zero only there)",
           "definition": "per_element: max_i |gpu - ref| / max(|ref_i|, 1e-3 max|ref|) (bar: 1e-5 image, "
                         "1e-3 gradients); max_norm: max_i |gpu - ref| / (|ref_i| + max|ref|)",
           "image": _errs(imgh, np.concatenate(ref_img))}
    if sel is not None:
        gv = g["volume"][0]
        flat = gv.view(-1, gv.shape[3]) if gv.dim() == 4 else gv.view(-1)
        idx = torch.as_tensor(sel, device=flat.device)
        got = flat[idx].cpu().numpy()
        amb = np.broadcast_to(amb_vol.reshape((-1,) + (1,) * (got.ndim - 1)), got.shape)
        out["grad_volume"] = _errs(got, ref_vol, amb)
        out["grad_volume"]["vertices_compared"] = int(sel.size)
        flat[idx] = 0.0
        out["grad_volume"]["nonzero_outside_the_rays"] = int(torch.count_nonzero(flat))
    if ref_tf is not None:
        out["grad_tf"] = _errs(g["tf"].cpu().numpy(), ref_tf)
    if e_eye:
        out["grad_eye"] = _errs(np.stack([a for a, _, _ in e_eye]), np.stack([b for _, b, _ in e_eye]),
                                np.stack([c for _, _, c in e_eye]))
    out["views_checked"] = len(views)
    return out


def accuracy(wl):
    """Errors of one forward + adjoint against the FP64 oracle on identical
    inputs (the workload's seeded eye positions; volume and TF as stored on
    the device), in the parity tests' two forms (_errs); untimed. Views of
    more than 300,000 pixels in all are checked on pixel samples
    (sampled_accuracy)."""
    import torch

    import oracle
    dvr, w = wl.dvr, wl.w
    if sum(v.width * v.height for v in w.views[:4]) > 300_000:
        return sampled_accuracy(wl)
    eye = torch.as_tensor(w.eye).to(wl.device).contiguous()
    img, aux = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=wl.scene)
    G = torch.randn(img.shape, device=wl.device, generator=torch.Generator(device=wl.device).manual_seed(1))
    want = tuple(x for x in wl.want)
    g = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=wl.scene, want=want)
    torch.cuda.synchronize()
    vol64 = wl.vol[0].float().cpu().numpy()
    tf64 = wl.tf.double().cpu().numpy() if wl.tf is not None else None
    Gh = G.cpu().numpy()
    imgh = img.cpu().numpy()

    def rel(a, b):
        return _errs(a, b)["per_element"]

    out = {"reference": "FP64 oracle, same stored inputs, fixed eye positions",
           "definition": "per_element: max_i |gpu - ref| / max(|ref_i|, 1e-3 max|ref|) (bar: 1e-5 image, "
                         "1e-3 gradients); max_norm: max_i |gpu - ref| / (|ref_i| + max|ref|)"}
    off = 0
    errs_img, ref_tf, ref_eye = [], None, []
    ref_imgs = []
    for k, view in enumerate(w.views[:4]):
        n = view.width * view.height
        ri, _, _ = oracle.render(vol64, tf64, w.model, view, w.eye[k], w.step_voxels)
        ref_imgs.append(ri)
        errs_img.append(rel(imgh[off:off + n], ri))
        ow = tuple(x for x in want if x != "volume")
        rg = oracle.backward(vol64, tf64, w.model, view, w.eye[k], w.step_voxels, Gh[off:off + n], want=ow)
        if "tf" in rg:
            ref_tf = rg["tf"] if ref_tf is None else ref_tf + rg["tf"]
        if "eye" in rg:
            ref_eye.append((k, rg["eye"]))
        off += n
    nimg = sum(v.width * v.height for v in w.views[:4])
    out["image"] = _errs(imgh[:nimg], np.concatenate(ref_imgs))
    if len(w.views) <= 4:
        if ref_tf is not None:
            out["grad_tf"] = _errs(g["tf"].cpu().numpy(), ref_tf)
            if wl.vol[0].dtype == torch.float32 and len(w.views) == 1:
                # how the opacity before each sample is recovered (Sec. 4.4)
                inv = {"optical_depth (default)": out["grad_tf"]["per_element"]}
                for mode in ("alpha64", "alpha32"):
                    gm = dvr.backward(None, None, None, None, eye, w.step_voxels, aux, G, scene=wl.scene,
                                      want=("tf",), inversion=mode)
                    inv[{"alpha64": "alpha_form_fp64_above_0.99", "alpha32": "alpha_form_fp32"}[mode]] = \
                        rel(gm["tf"].cpu().numpy(), ref_tf)
                # the binary32 alpha form restarted from forward checkpoints every K samples
                for k in (256, 16):
                    ck = torch.empty((wl.scene.pixels, dvr.checkpoint_slots(wl.scene, w.step_voxels, k)),
                                     device=wl.device)
                    _, aux_k = dvr.forward(None, None, None, None, eye, w.step_voxels, scene=wl.scene,
                                           checkpoints=(ck, k))
                    gm = dvr.backward(None, None, None, None, eye, w.step_voxels, aux_k, G, scene=wl.scene,
                                      want=("tf",), inversion="alpha32", checkpoints=(ck, k))
                    inv[f"alpha_form_fp32_checkpoints_K{k}"] = rel(gm["tf"].cpu().numpy(), ref_tf)
                    del ck
                out["grad_tf_by_inversion"] = inv
    if ref_eye:
        ge = g["eye"].cpu().numpy()
        out["grad_eye"] = _errs(np.stack([ge[k] for k, _ in ref_eye]), np.stack([r for _, r in ref_eye]))
    out["views_checked"] = min(4, len(w.views))
    return out


# -------------------------------------------------------------- our arm
def time_steps(wl, K, W, flush, clocks=None, world=1):
    """W untimed steps, then K steps each bracketed by CUDA events (L2 flushed
    between steps, outside the brackets). Returns per-step, forward and
    adjoint milliseconds and the wall time of the timed region."""
    import torch
    import torch.distributed as dist
    for _ in range(W):
        wl.step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
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
    clk = clocks.stop() if clocks is not None else None
    step_ms = float(np.mean([s.elapsed_time(e) for s, e in zip(st, en)]))
    fwd_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    bwd_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in evs]))
    return step_ms, fwd_ms, bwd_ms, wall, clk


def time_steps_graph(wl, K, W, flush, clocks=None, world=1, stats=None, side_steps=3):
    """The same step captured once as a CUDA graph and replayed: K replays
    each bracketed by CUDA events (L2 flushed between replays, outside the
    brackets), after W untimed replays. Returns the mean milliseconds per
    step and the wall time of the timed region; `stats`, if given, receives
    the median, minimum and maximum of the K step times."""
    import torch
    import torch.distributed as dist
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(side_steps):
            wl.step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        wl.step()
    for _ in range(W):
        graph.replay()
    torch.cuda.synchronize()
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
        clocks.mark()
    t0 = time.perf_counter()
    for k in range(K):
        flush.zero_()
        st[k].record()
        graph.replay()
        en[k].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks is not None else None
    ms = [s.elapsed_time(e) for s, e in zip(st, en)]
    if stats is not None:
        stats.update(median=round(float(np.median(ms)), 4), min=round(float(np.min(ms)), 4),
                     max=round(float(np.max(ms)), 4))
    return float(np.mean(ms)), wall, clk


def compare_camera_modes(wl, K, W, flush):
    """Camera gradient alone, two ways (Sec. 5.1): the adjoint (forward pass,
    then the adjoint with only the eye gradient) and forward mode (one
    tangent pass, then the contraction). Device time per step, L2 flushed
    between steps."""
    import torch
    dvr, w = wl.dvr, wl.w

    def adjoint(ge):
        dvr.forward(None, None, None, None, wl.eye, w.step_voxels, scene=wl.scene, image=wl.image, aux=wl.aux)
        dvr.loss_l2(wl.image, wl.target, 1.0 / wl.image.numel(), grad_image=wl.gimg, loss=wl.loss)
        dvr.backward(None, None, None, None, wl.eye, w.step_voxels, wl.aux, wl.gimg, scene=wl.scene,
                     grads={"eye": ge}, want=("eye",))

    tangent = torch.empty((wl.scene.pixels, wl.scene.channels, 3), device=wl.device)

    def forward_mode(ge):
        dvr.forward_tangent(None, None, None, None, wl.eye, w.step_voxels, scene=wl.scene, image=wl.image,
                            tangent=tangent)
        dvr.loss_l2(wl.image, wl.target, 1.0 / wl.image.numel(), grad_image=wl.gimg, loss=wl.loss)
        dvr.tangent_contract(wl.scene, tangent, wl.gimg, grad_eye=ge)

    out = {}
    grads = {}
    for name, fn in (("adjoint", adjoint), ("forward_mode", forward_mode)):
        ge = torch.zeros_like(wl.eye)
        for _ in range(W):
            ge.zero_()
            fn(ge)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for k in range(K):
            flush.zero_()
            ge.zero_()
            ev[k][0].record()
            fn(ge)
            ev[k][1].record()
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        grads[name] = ge.clone()
        out[name] = {"ms_per_step": round(ms, 4), "gsamples_s": round(wl.samples_per_pass / (ms * 1e-3) / 1e9, 3)}
    a, f = grads["adjoint"].double(), grads["forward_mode"].double()
    out["max_rel_difference"] = float(((a - f).abs() / (a.abs() + a.abs().max())).max())
    out["note"] = "camera gradient only; the paper reports 24.1 ms (adjoint) vs 21.3 ms (forward-immediate) on an RTX 2070"
    return out


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

    wl = Workload(args.workload, dev, args.tf_immediate, views=args.views, image=args.image,
                  cells=max(args.cells, 0), cell_gradient=args.cell_gradient > 0, grid=args.grid)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    K = args.steps
    if args.persistent_scatter >= 0:            # a fixed launch form applies from the first step on
        wl.persistent_scatter = bool(args.persistent_scatter)
    # one untimed step to size the secondary legs (~10 s of work each)
    probe_ms, _, _, _, _ = time_steps(wl, 1, 1, flush, None, world)
    K2 = max(2, min(K, int(math.ceil(6_000.0 / max(probe_ms, 1e-3)))))
    W2 = min(args.warmup, 2) if probe_ms > 1000.0 else args.warmup
    tuning = None
    if args.tile_width:
        from paper_2107_12672_b300 import autotune
        aw = args.adjoint_tile_width or args.tile_width
        autotune.set_tile_width(args.tile_width, aw)
        tuning = {"width": args.tile_width, "adjoint_width": aw, "fixed": True}
    elif not args.no_autotune:
        from paper_2107_12672_b300 import autotune
        color = wl.w.model == "color"         # no cell layout for colour volumes
        tscene, teye, tnote = wl.scene, wl.eye, "all views"
        if probe_ms > 1000.0 and len(wl.w.views) > 4:
            # steps of seconds: tune on the first four views (same volume,
            # TF and view sizes), one timed pass per width and round
            tscene = wl.dvr.Scene.make(wl.vol, wl.tf, wl.w.model, wl.w.views[:4])
            teye, tnote = wl.eye[:4].contiguous(), "first 4 views"
        tuning = autotune.autotune(tscene, teye, wl.w.step_voxels, want=wl.want, l2_flush=flush,
                                   reps=1 if probe_ms > 1000.0 else 5,
                                   layouts=(0,) if color else (0, 1, 4, 8) if args.cells < 0 else (args.cells,),
                                   cell_gradients=(False,) if color else
                                   (False, True) if args.cell_gradient < 0 else (bool(args.cell_gradient),),
                                   persistent=(False, True) if args.persistent_scatter < 0
                                   else (bool(args.persistent_scatter),))
        tuning["tuned_on"] = tnote
        if tuning["cells"] != wl.use_cells or tuning["cell_gradient"] != wl.cell_gradient:
            wl.configure(tuning["cells"], tuning["cell_gradient"])
        wl.persistent_scatter = bool(tuning.get("persistent_scatter", False))
    if args.persistent_scatter >= 0:
        wl.persistent_scatter = bool(args.persistent_scatter)
    if tuning is not None:
        tuning["persistent_scatter"] = wl.persistent_scatter
    # per-kernel breakdown from eagerly launched steps; the headline step
    # time from the same step replayed as one CUDA graph
    eager_ms, fwd_ms, bwd_ms, _, _ = time_steps(wl, K2, W2, flush, None, world)
    step_stats = {}                 # this rank's median / min / max step (graph replays)
    if args.eager:
        step_ms, _, _, wall, clk = time_steps(wl, K, args.warmup, flush, Clocks(local), world)
    else:
        step_ms, wall, clk = time_steps_graph(wl, K, args.warmup, flush, Clocks(local), world, step_stats,
                                              side_steps=1 if probe_ms > 1000.0 else 3)
    if world > 1:
        t = torch.tensor([step_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t.item())

    samples = wl.samples_per_pass                  # per pass; forward and adjoint each visit them
    value = world * samples / (step_ms * 1e-3) / 1e9

    e2e = None
    if not args.no_e2e:
        # at least 6 steps (K allowing): the first upload and the last
        # read-back have no neighbouring step to hide behind, and over n
        # steps each step carries 1/n of them
        e2e = run_e2e(wl, args, world, max(K2, min(K, 6)), W2)
    cpu = acc = variants = camera_modes = None
    if rank == 0 and world == 1:
        if not args.no_accuracy:
            acc = accuracy(wl)
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(wl, budget_s=12.0)
        if not args.no_variants and "eye" in wl.want and wl.w.model != "color":
            camera_modes = compare_camera_modes(wl, K2, W2, flush)
        if not args.no_variants and (wl.ea or wl.w.model == "color"):
            variants = {}
            # the other storage form of the same workload: 16-bit beside a
            # binary32 workload, the plain binary32 form beside a 16-bit one
            plain = wl.w.volume_dtype == "float32" and wl.w.tf_dtype == "float32"
            other = ("float16", "float32") if wl.w.model == "color" else ("bfloat16", "float16")
            for vd, td in ((other,) if plain else (("float32", "float32"),)):
                # with the gather layout and scatter of the headline workload
                wv = Workload(args.workload, dev, args.tf_immediate, vol_dtype=vd, tf_dtype=td, views=args.views,
                              image=args.image, cells=wl.use_cells, cell_gradient=wl.cell_gradient, grid=args.grid)
                wv.persistent_scatter = wl.persistent_scatter
                sm, fm, bm, _, _ = time_steps(wv, K2, W2, flush)
                variants[f"volume_{vd}_tf_{td}"] = {
                    "value": round(wv.samples_per_pass / (sm * 1e-3) / 1e9, 4), "unit": "Gsamples/s",
                    "ms_per_step": round(sm, 4), "forward_ms": round(fm, 4), "adjoint_ms": round(bm, 4),
                    "steps": K2, "launch": "eager launches",
                    "accuracy": None if args.no_accuracy else accuracy(wv),
                    "note": "errors include the rounding of the stored volume and TF"}
                del wv

    if rank == 0:
        hbm, src = peaks()
        dom = "backward" if bwd_ms >= fwd_ms else "forward"
        dur = bwd_ms if dom == "backward" else fwd_ms
        achieved = algorithmic_bytes(wl, dom) / (dur * 1e-3) / 1e9
        ceil = probe_ceilings(dev)
        levels = {"l2_read": {"peak": ceil["l2_read_gbs"], "unit": "GB/s",
                              "frac": round(achieved / ceil["l2_read_gbs"], 4)},
                  "l1_read": {"peak": ceil["l1_read_gbs"], "unit": "GB/s",
                              "frac": round(achieved / ceil["l1_read_gbs"], 4)},
                  "peak_source": "measured in this run with dvr_probe"}
        if dom == "backward" and "volume" in wl.want:
            # the density-gradient scatter: 8 corner additions per sample
            ops = wl.samples_per_pass * 8 / (dur * 1e-3) / 1e9
            levels["l2_red"] = {"achieved": round(ops, 2), "peak": ceil["l2_red_gops"], "unit": "Gops/s",
                                "frac": round(ops / ceil["l2_red_gops"], 4)}
        cfg = wl.describe()
        cfg.update({"l2": "flushed between timed steps (512 MiB write)",
                    "launch": "eager launches" if args.eager else "the whole step as one CUDA graph, replayed",
                    "tile": tuning,
                    "tf_accumulation": "immediate" if args.tf_immediate else "delayed (shared memory)",
                    "parallelism": f"replicas x{world}"})
        line = {
            "metric": METRIC,
            "value": round(value, 4),
            "unit": "Gsamples/s",
            "n_gpus": world,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": round(step_ms, 4),
            "ms_per_step_stats": step_stats or None,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            # the arithmetic is binary32 for every storage type (the storage
            # is in config.volume / config.tf_dtype)
            "dtype": "f32",
            "data": "synthetic (seeded generators; no dataset)",
            "config": cfg,
            "secondary_steps": {"steps": K2, "warmup": W2,
                                "legs": "eager breakdown (forward_ms, adjoint_ms), e2e, storage_variants, "
                                        "camera_gradient_modes"},
            "eager_ms_per_step": round(eager_ms, 4),
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
                "traffic": profiled_traffic(dom + ("_color" if wl.w.model == "color" else ""), args.workload),
                "bytes_per_sample": round(algorithmic_bytes(wl, dom) / wl.samples_per_pass, 3),
                "gather_bytes_per_sample": gather_bytes(wl),
                "levels": levels,
            },
            "accuracy": acc,
            "storage_variants": variants,
            "camera_gradient_modes": camera_modes,
            "clocks": clk,
            "gpu_launches": wl.launches_per_step * K,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(wl, args, world, K, W):
    """Same metric through the public API with host buffers: every step
    copies its inputs (volume, TF, camera parameters) from pinned host memory
    and reads back the loss and the gradients (the 4 GiB volume gradient at
    1024^3 included), and the host waits for every step's results. The step
    runs as a captured CUDA graph of the same calls, pipelined over two
    buffer sets: step k+1's volume is copied in on one copy stream and step
    k-1's results are copied out on another while step k computes (the small
    inputs are copied on the compute stream just before each replay); the
    host waits for step k-1's results after launching step k, and for the
    last step's before the clock stops."""
    import torch
    dvr = wl.dvr
    vol_h = wl.vol[0].cpu().pin_memory()
    small_in = []
    if wl.tf is not None:
        small_in.append((wl.tf, wl.tf.cpu().pin_memory()))
    cam = wl.params if wl.orbit else wl.eye
    small_in.append((cam, cam.cpu().pin_memory()))

    own = wl.outputs
    out_sets = [own, wl.make_outputs()]
    bufs = [wl.vol[0], torch.empty_like(wl.vol[0])]
    cells1 = [torch.empty_like(wl.cells[0])] if wl.cells is not None else None
    scenes = [wl.scene, dvr.Scene.make([bufs[1]], wl.tf, wl.w.model, wl.w.views, cells=cells1,
                                       cells_brick=wl.use_cells or 1)]
    outs, h_out = [], []
    for o in out_sets:
        wl.use_outputs(o)
        outs.append(wl.result_tensors())
        h_out.append([torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs[-1]])
    compute = torch.cuda.current_stream()
    copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
    graphs = []
    try:
        for sc, o in zip(scenes, out_sets):
            wl.use_outputs(o)
            side = torch.cuda.Stream()
            side.wait_stream(compute)
            with torch.cuda.stream(side):
                for _ in range(1 if W < 3 else 3):
                    wl.step(scene=sc)
            compute.wait_stream(side)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                wl.step(scene=sc)
            graphs.append(g)
    finally:
        wl.use_outputs(own)
    torch.cuda.synchronize()
    copied = [torch.cuda.Event(), torch.cuda.Event()]       # volume b is in place
    computed = [torch.cuda.Event(), torch.cuda.Event()]     # the step on set b is done
    read = [torch.cuda.Event(), torch.cuda.Event()]         # set b's results are on the host

    def prefetch(b):
        with torch.cuda.stream(copy_in):
            copy_in.wait_event(computed[b])     # the step that last read buffer b
            bufs[b].copy_(vol_h, non_blocking=True)
            copied[b].record(copy_in)

    def run(n):
        for e in computed + read:
            e.record(compute)
        prefetch(0)
        for k in range(n):
            b = k & 1
            if k + 1 < n:
                prefetch(1 - b)
            compute.wait_event(copied[b])
            compute.wait_event(read[b])         # set b's previous results have left the device
            for d, h in small_in:
                d.copy_(h, non_blocking=True)
            graphs[b].replay()
            computed[b].record(compute)
            with torch.cuda.stream(copy_out):
                copy_out.wait_event(computed[b])
                for h, t in zip(h_out[b], outs[b]):
                    h.copy_(t, non_blocking=True)
                read[b].record(copy_out)
            if k > 0:
                read[1 - b].synchronize()       # the host has step k-1's loss and gradients
        read[(n - 1) & 1].synchronize()         # ... and the last step's
        torch.cuda.synchronize()

    run(max(1, W))
    t0 = time.perf_counter()
    run(K)
    dt = (time.perf_counter() - t0) / K
    h2d = vol_h.numel() * vol_h.element_size() + sum(h.numel() * h.element_size() for _, h in small_in)
    d2h = sum(h.numel() * h.element_size() for h in h_out[0])
    return {"value": round(world * wl.samples_per_pass / dt / 1e9, 4), "unit": "Gsamples/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(dt * 1e3, 4),
            "steps": K,
            "how": "step as a replayed CUDA graph over two buffer sets; step k+1's volume copied in and "
                   "step k-1's loss and gradients copied out on two copy streams during step k; the host "
                   "waits for every step's results (one step behind), the last one inside the timed region"}


# ------------------------------------------------------ the CPU oracle arm
class OraclePass:
    """The oracle's forward + stored-state adjoint (with the workload's loss
    seed, and the orbit chain when the camera is orbit-parameterised) on a
    strided subset of the rows of the workload's first view. The L2 loss's
    target image is rendered once, untimed, as on the GPU side; the
    opacity-entropy loss (Sec. 5.1) is taken over the sampled pixels."""

    def __init__(self, w, stride, volume=None):
        import oracle
        oracle.build()
        self.oracle = oracle
        self.w = w
        self.view = w.views[0]
        self.stride = stride
        if w.orbit is not None:
            self.eye = oracle.orbit_eye(w.orbit.astype(np.float32).astype(np.float64))[0]
        else:
            self.eye = w.eye[0].astype(np.float64)
        self.vol = volume if volume is not None else (w.volumes[0] if w.volumes else None)
        if self.vol is None:
            raise ValueError("the oracle baseline needs the volume on the host")
        self.target = None
        if w.loss == "l2":
            tf_t = w.target.get("tf", w.tf)
            vol_t = w.target.get("volume", self.vol)
            self.target, _, _ = oracle.render(vol_t, tf_t, w.model, self.view, self.eye, w.step_voxels)
        self.want = tuple({"volume": "volume", "tf": "tf", "camera": "eye"}[g] for g in w.grads)
        self.phase = 0

    def __call__(self):
        o, w, view = self.oracle, self.w, self.view
        rows = np.arange(self.phase, view.height, self.stride)
        self.phase = (self.phase + 1) % self.stride
        pix = (rows[:, None] * view.width + np.arange(view.width)[None, :]).reshape(-1).astype(np.int64)
        img, N, _ = o.render(self.vol, w.tf, w.model, view, self.eye, w.step_voxels, pix=pix)
        if self.target is not None:
            G = 2.0 * (img - self.target[pix]) / self.target.size
        else:
            _, dH = o.opacity_entropy(img[:, -1])
            G = np.zeros_like(img)
            G[:, -1] = -dH          # the loss is -H (maximised)
        # the dense binary64 volume gradient (8 GB virtual at 1024^3) is
        # zero-filled lazily by the host OS: only the pages these rays touch
        # are ever backed
        g = o.backward(self.vol, w.tf, w.model, view, self.eye, w.step_voxels, G, pix=pix, want=self.want)
        if w.orbit is not None and "eye" in g:
            o.orbit_eye_backward(w.orbit, g["eye"][None])
        return int(N.sum()), pix.size


def _host_volume(wl_or_w, name):
    """The workload's volume on the host as float32 (the values the device
    holds: binary16 / bfloat16 widen exactly)."""
    if hasattr(wl_or_w, "vol"):
        return wl_or_w.vol[0].float().cpu().numpy()
    w = wl_or_w
    if w.volumes and w.volumes[0] is not None:
        return w.volumes[0]
    import torch

    from paper_2107_12672_b300 import synthetic as syn
    torch.set_num_threads(os.cpu_count() or 1)
    v = syn.large_volume(w.target["n"], device="cpu")
    return v.to(getattr(torch, w.volume_dtype)).float().numpy()


def _stride(w):
    """Rows between sampled rows: about 64 sampled rows of the first view,
    so that one oracle pass takes seconds at every size."""
    return max(8, w.views[0].height // 64)


def cpu_baseline(wl, budget_s=12.0):
    w = wl.w
    stride = _stride(w)
    op = OraclePass(w, stride=stride, volume=_host_volume(wl, wl.name))
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
            "sample": f"{passes} passes over every {stride}th row of the {w.views[0].width}x{w.views[0].height} "
                      f"first view ({rays} rays, {done} samples; forward + {w.loss} seed + stored-state adjoint, "
                      f"FP64, OpenMP) in {dt:.1f} s; the rate per sample stands for the whole workload"}


def run_reference(args):
    """The oracle as the reference arm: rank 0 only, on the host cores; each
    step is a bounded sample (every 2*stride-th row of the first view) of
    the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2107_12672_b300 import synthetic as syn
    w = syn.workload(args.workload)
    stride = 2 * _stride(w)
    op = OraclePass(w, stride=stride, volume=_host_volume(w, args.workload))
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
                         "sample": f"each step: every {stride}th row of the {w.views[0].width}x"
                                   f"{w.views[0].height} first view, forward + {w.loss} seed + stored-state "
                                   f"adjoint (FP64); {rays} rays, {n} samples in {dt:.1f} s"},
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

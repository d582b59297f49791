#!/usr/bin/env python3
"""ApplyFilter benchmark on one GB300 (or N replicas under torchrun).

Workload (one step = the whole filter path over one volume): a 512^3 uint8 CT-like
volume (32 Gaussian blobs + noise, mapping range [0,1]) filtered twice to float32:
  1. a normalised 5^3 Gaussian, sigma 1.5 (built per step, separable path), and
  2. the 7-point Laplacian as a dense 3^3 kernel (direct FP32 path).
Gvoxel/s counts output voxels (2 x 512^3 per step).  Inputs are resident in HBM when the
timed region starts; L2 is flushed (256 MiB write) before every timed step, outside the
step's own CUDA events.  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (512, 512, 512)
SEED = 220310213 + 1
METRIC = "ApplyFilter Gvoxel/s & % roofline, split-TC vs plain FP32 at <=1e-5 err, 1 GB300"
WORKLOAD = "ct512_u8_to_f32: gaussian5 sigma1.5 (separable) + laplacian3 (dense direct)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-precision-form", action="store_true",
                    help="skip the tensor-core vs FP32 comparison on the 1024x1024x512 field")
    ap.add_argument("--precision-reps", type=int, default=10)
    ap.add_argument("--no-batching-form", action="store_true",
                    help="skip the 256-volume graph batch vs separate launches comparison")
    ap.add_argument("--no-extra-forms", action="store_true",
                    help="skip the range, BrickDecompose, CLAHE-3D, render, differentiation "
                         "and smallest-case forms")
    ap.add_argument("--kernel-case", choices=sorted(KERNEL_CASES),
                    help="run one kernel configuration --reps times and exit (for ncu captures)")
    ap.add_argument("--reps", type=int, default=3)
    return ap.parse_args()


# single-kernel cases for profiler captures: (value model, format, dims, filter, path)
# (path "auto": the path and launch shape the step's calls take, tuned on the first call;
# with VKT_AUTOTUNE_CACHE naming the file a previous run wrote, the choice is read, not timed)
KERNEL_CASES = {
    "sep5_ct512": ("blobs", 0, (512, 512, 512), "gaussian5", "auto"),
    "lap3_ct512": ("blobs", 0, (512, 512, 512), "laplacian3", "auto"),
    "sep5_ct640": ("blobs", 0, (640, 512, 512), "gaussian5", "auto"),
    "lap3_ct640": ("blobs", 0, (640, 512, 512), "laplacian3", "auto"),
    "tc7_dns512": ("uniform", 2, (512, 512, 256), "random7", "tensor"),
    "direct7_dns512": ("uniform", 2, (512, 512, 256), "random7", "direct"),
    "batch256": None,    # the batching form's 256 volumes (run_batch_case)
    "bricks2_ct512": None,   # BrickDecompose of the 512^3 volume, 64^3 bricks, 2 ghost cells
    "render_ct512": None,    # the render form's 1024 x 768 frame of the 512^3 volume
    "backward_train": None,  # the differentiation form's batch backward (8 x 128^3, k = 5)
}

# Per-launch DRAM traffic of the kernels this bench reports, from the ncu captures summarised
# in profiles/; each entry holds the hash of the kernel's sources at capture time and is
# used only while the sources are unchanged.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.md")
KERNEL_SOURCES = {
    "separable gaussian5": ["vkt_sep_brick.cuh", "vkt_separable.cuh", "vkt_separable5.cu", "vkt_tile.cuh"],
    "direct laplacian3": ["vkt_direct.cuh", "vkt_direct.cu", "vkt_tile.cuh"],
}


def source_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2203_10213_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel: str):
    """(bytes per launch at 512^3, capture note) if a current capture exists, else (None, why)."""
    try:
        with open(TRAFFIC_FILE) as f:
            lines = [ln.strip() for ln in f if ln.startswith("| ") and "source" not in ln]
    except OSError:
        return None, "no capture summary"
    want = source_hash(KERNEL_SOURCES[kernel])
    for ln in lines:
        cells = [c.strip() for c in ln.strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == kernel:
            if cells[3] != want:
                return None, "kernel changed since the capture"
            return float(cells[1]), cells[2]
    return None, "kernel not captured"


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(ms: float, device, world: int) -> float:
    """The largest of every rank's `ms` (the whole job ends when its slowest replica does);
    an all-reduce over the default process group when world > 1."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_gvoxel_s(voxels_per_step: float, world: int, ms_per_step: float) -> float:
    """Whole-job output voxels per second (1e9) when each of `world` replicas filters its own
    volume per step and the job's step takes `ms_per_step` (the slowest rank's)."""
    return voxels_per_step * world / (ms_per_step * 1e-3) / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.split(",") for ln in self.file.read().splitlines() if ln.count(",") >= 8]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------ CPU baseline (oracle)

def workload_host():
    import synth
    return synth.volume("blobs", synth.U8, DIMS, SEED)


def oracle_sample_rate(vol, seconds: float, seed: int = 7):
    """Times the FP64 oracle on random voxels of the workload for about `seconds`; returns
    voxels/s (both filters, each output counted once), the voxel count and the time."""
    import oracle
    w_g = oracle.gaussian_weights(5, float(np.float32(1.5)))
    w_l = oracle.laplacian_3()
    rng = np.random.default_rng(seed)
    n, total_n, total_t = 4096, 0, 0.0
    while total_t < seconds:
        idx = rng.integers(0, vol.size, n)
        t0 = time.perf_counter()
        oracle.correlate_points(vol, w_g, idx, 0.0, 1.0)
        oracle.correlate_points(vol, w_l, idx, 0.0, 1.0)
        dt = time.perf_counter() - t0
        total_n += n
        total_t += dt
        rate = n / max(dt, 1e-6)
        n = int(min(max(4096, rate * (seconds - total_t)), 1 << 24))
    return 2 * total_n / total_t, total_n, total_t


def cpu_leg(args, vol, pin):
    """The CPU (oracle) leg, the only part of our arm that runs the oracle: the FP64 oracle
    timed on the host cores on random voxels of the step's workload (`cpu_baseline`), and
    the oracle's values at the precision form's sampled voxels, against which that form
    states the error of each GPU path."""
    import oracle
    rate, n, dt = oracle_sample_rate(vol, args.cpu_seconds)
    cores = oracle.num_threads()
    cpu = {"value": round(rate / 1e9, 6), "unit": "Gvoxel/s", "cores": cores,
           "kind": "oracle",
           "sample": f"{n} random voxels of the 512^3 volume, both filters, FP64 C, {dt:.1f} s"}
    # one core on a shorter sample; the whole step's time extrapolated from its rate
    oracle.set_num_threads(1)
    try:
        rate1, n1, dt1 = oracle_sample_rate(vol, max(1.0, args.cpu_seconds / 5))
    finally:
        oracle.set_num_threads(cores)
    cpu["single_core"] = {"value": round(rate1 / 1e9, 6), "unit": "Gvoxel/s",
                          "sample": f"{n1} random voxels, {dt1:.1f} s, one thread",
                          "step_s_extrapolated": round(2 * float(vol.size) / rate1, 1)}
    refs = None
    if pin is not None:
        field, idx, kernels = pin
        refs = {k: oracle.correlate_points(field, w, idx) for k, (w, _) in kernels.items()}
    return cpu, refs


# ------------------------------------------------------------------ precision form (TC vs FP32)

PF_DIMS = (1024, 1024, 512)


def precision_inputs():
    """The precision form's field, its sampled voxel numbers and its two kernels (k = 7, 9:
    weights and the seed actually used), all from the seeded generator."""
    import synth
    field = synth.volume("fourier", synth.F32, PF_DIMS, synth.BASE_SEED + 2)
    idx = np.random.default_rng(5).integers(0, field.size, 20000)
    kernels = {k: synth.random_kernel(synth.BASE_SEED + 2, k, 1.0, normalise_sum=True)
               for k in (7, 9)}
    return field, idx, kernels


def precision_form(args, vkt, torch, dev, stream, peaks, field, idx, kernels, refs):
    """Split FP16 hi/lo tensor-core path vs plain FP32 path on the 1024x1024x512
    turbulence-like field with normalised N(0,1) k^3 kernels, k = 7 and 9: Gvoxel/s of
    each, their ratio, the error of each against the FP64 oracle on sampled voxels (the
    oracle's values `refs` come from the CPU leg, None when it is skipped), and the
    algorithmic FLOP rate (2 k^3 per voxel) against the measured dense FP16/BF16 tensor
    peak and against the FP32 CUDA-core peak; the MMA FLOPs the tensor pipe executes
    (Toeplitz zeros, three split products, N padding) are a separate diagnostic."""
    src = torch.from_numpy(field).to(dev)
    out = torch.empty_like(src)
    v_src = vkt.StructuredVolume.from_tensor(src)
    v_out = vkt.StructuredVolume.from_tensor(out)
    vox = float(np.prod(PF_DIMS))
    xmax = float(np.abs(field).max())
    props = torch.cuda.get_device_properties(dev)
    fp32_peak = props.multi_processor_count * 128 * 2 * measured_peaks()[0].get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    res = {"workload": "fourier 1024x1024x512 f32, normalised N(0,1) kernels", "dims": list(PF_DIMS)}
    for k in (7, 9):
        w, seed_used = kernels[k]
        f = vkt.Filter.dense(w)
        ref = refs.get(k) if refs else None
        # the normalisation of the error: sum|w| * max|x| (float32 weights promoted)
        scale = float(np.abs(w.astype(np.float64)).sum()) * xmax
        entry = {}
        for path in ("tensor", "direct"):
            with vkt.policy(stream=stream, path=path):
                for _ in range(3):
                    vkt.check(vkt._lib.vktApplyFilterSV(v_out.handle, v_src.handle, f.handle))
                torch.cuda.synchronize()
                evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                evs[0].record(stream)
                for _ in range(args.precision_reps):
                    vkt.check(vkt._lib.vktApplyFilterSV(v_out.handle, v_src.handle, f.handle))
                evs[1].record(stream)
                torch.cuda.synchronize()
                vkt.synchronize()
            ms = evs[0].elapsed_time(evs[1]) / args.precision_reps
            got = out.view(-1)[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
            err = float(np.max(np.abs(got - ref)) / scale) if ref is not None else None
            entry[path] = {"ms": round(ms, 4), "gvoxel_s": round(vox / (ms * 1e-3) / 1e9, 2),
                           "max_err_normalised": err}
        # executed tensor FLOPs: per 128 x 16 output voxels and input plane, 2 x-tiles x k
        # row offsets x 3 split products of a 128 x N x 16 MMA (N = 8 * even(k)); input
        # planes per output plane = (zchunk + k - 1) / zchunk
        slots = ((k + 1) // 2) * 2
        flops_plane = 2 * k * 3 * (128 * 8 * slots * 16 * 2)
        tc = entry["tensor"]
        tc_tflops = flops_plane / 2048 * vox / (tc["ms"] * 1e-3) / 1e12
        alg_tflops = 2 * k ** 3 * vox / (tc["ms"] * 1e-3) / 1e12
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        entry["tc_over_fp32"] = round(entry["direct"]["ms"] / tc["ms"], 3)
        entry["tensor_roofline"] = {"bound": "tensor", "achieved": round(alg_tflops, 1),
                                    "algorithmic_flop_per_voxel": 2 * k ** 3,
                                    "peak": bf16, "unit": "TFLOP/s",
                                    "frac": round(alg_tflops / bf16, 4),
                                    "peak_source": "measured bf16_tflops (dense fp16 has the same rate)",
                                    "fp32_peak_tflops": round(fp32_peak, 1),
                                    "frac_vs_fp32_peak": round(alg_tflops / fp32_peak, 4),
                                    "executed_tflops_lower_bound": round(tc_tflops, 1),
                                    "executed_frac_diagnostic": round(tc_tflops / bf16, 4)}
        entry["kernel_seed"] = seed_used
        res[f"k{k}"] = entry
    return res


# ------------------------------------------------------------------ batching form

def batching_form(args, vkt, torch, dev, stream):
    """256 volumes (dims log-uniform in 16..256 per axis, u8/u16/f32, Gaussian k in {3,5,7},
    sigma = k/3, dst = src format) in one graph-captured persistent launch, against the
    same 256 filters issued as separate launches (back to back on one stream, and the sum
    of individually timed launches)."""
    import synth
    items = synth.batch_recipe(synth.BASE_SEED + 3, n=256)
    srcs, dsts, vs, vd, fs = [], [], [], [], []
    dt = {synth.U8: torch.uint8, synth.U16: torch.uint16, synth.F32: torch.float32}
    nbytes = 0
    for it in items:
        a = synth.volume(it["kind"], it["fmt"], it["dims"], it["seed"])
        s = torch.from_numpy(a).to(dev)
        d = torch.empty(a.shape, dtype=dt[it["fmt"]], device=dev)
        srcs.append(s)
        dsts.append(d)
        vs.append(vkt.StructuredVolume.from_tensor(s))
        vd.append(vkt.StructuredVolume.from_tensor(d))
        fs.append(vkt.Filter.gaussian(it["k"], it["sigma"]))
        nbytes += 2 * a.nbytes
    vox = float(sum(s.numel() for s in srcs))
    lib = vkt._lib
    reps = 5

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        vkt.synchronize()
        return a.elapsed_time(b) / reps

    import ctypes
    with vkt.policy(stream=stream):
        def batched():
            vkt.apply_filter_batch(vd, vs, fs, stream=stream)

        def separate():
            for i in range(len(items)):
                vkt.check(lib.vktApplyFilterSV(vd[i].handle, vs[i].handle, fs[i].handle))

        # the fixed rule (64-plane bricks, full occupancy) and the autotuned plan (its first
        # call, untimed, measures the candidates), timed in alternation and compared by
        # their medians so that the drift of the GPU between two timings does not favour one
        enabled = ctypes.c_int32()
        vkt.check(lib.vktAutotuneGetEnabled(ctypes.byref(enabled)))
        vkt.check(lib.vktAutotuneSetEnabled(1))
        batched()
        torch.cuda.synchronize()
        rule_ms, tuned_ms = [], []
        for _ in range(5):
            vkt.check(lib.vktAutotuneSetEnabled(0))
            rule_ms.append(timed(batched))
            vkt.check(lib.vktAutotuneSetEnabled(1))
            tuned_ms.append(timed(batched))
        ms_rule, ms_batch = statistics.median(rule_ms), statistics.median(tuned_ms)
        vkt.check(lib.vktAutotuneSetEnabled(enabled.value))
        ms_sep = timed(separate)
        # sum of individually timed launches
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in items]
        for i in range(len(items)):
            evs[i][0].record(stream)
            vkt.check(lib.vktApplyFilterSV(vd[i].handle, vs[i].handle, fs[i].handle))
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        ms_sum = sum(a.elapsed_time(b) for a, b in evs)
    hbm = measured_peaks()[0]["hbm_gbs"]
    return {"volumes": len(items), "voxels": int(vox), "algorithmic_bytes": int(nbytes),
            "graph_batch_ms": round(ms_batch, 4),
            "graph_batch_gvoxel_s": round(vox / (ms_batch * 1e-3) / 1e9, 2),
            "graph_batch_frac_hbm": round(nbytes / (ms_batch * 1e-3) / 1e9 / hbm, 4),
            "graph_batch_fixed_rule_ms": round(ms_rule, 4),
            "tuned_over_fixed_rule": round(ms_rule / ms_batch, 3),
            "separate_back_to_back_ms": round(ms_sep, 4),
            "separate_sum_of_launches_ms": round(ms_sum, 4),
            "speedup_vs_back_to_back": round(ms_sep / ms_batch, 3),
            "speedup_vs_sum_of_launches": round(ms_sum / ms_batch, 3)}


# ------------------------------------------------------------------ range form

RANGE_BOX = ((101, 77, 130), (401, 327, 400))   # 300 x 250 x 270 voxels, off every boundary


def range_form(vkt, torch, stream, lib, v_g, v_l, v_src, g, lap):
    """The two filters of the step restricted to a region of interest of the same volume
    (vktApplyFilterRangeSV): output voxels of the region per second, and the HBM fraction
    on the region's algorithmic bytes (1 B in + 4 B out per voxel)."""
    (x0, y0, z0), (x1, y1, z1) = RANGE_BOX
    vox = float((x1 - x0) * (y1 - y0) * (z1 - z0))
    reps = 10
    out = {}
    with vkt.policy(stream=stream):
        for name, dst, f in (("separable gaussian5", v_g, g), ("direct laplacian3", v_l, lap)):
            def call():
                vkt.check(lib.vktApplyFilterRangeSV(dst.handle, v_src.handle, f.handle,
                                                    x0, y0, z0, x1, y1, z1))
            for _ in range(3):
                call()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                call()
            b.record(stream)
            torch.cuda.synchronize()
            vkt.synchronize()
            ms = a.elapsed_time(b) / reps
            out[name] = {"ms": round(ms, 4), "gvoxel_s": round(vox / (ms * 1e-3) / 1e9, 2),
                         "frac_hbm": round(5 * vox / (ms * 1e-3) / 1e9 / measured_peaks()[0]["hbm_gbs"], 4)}
    return {"box": [list(RANGE_BOX[0]), list(RANGE_BOX[1])], "voxels": int(vox),
            "note": "consecutive calls on a resident volume (the region's 20 MB input stays in L2)",
            **out}


# ------------------------------------------------------------------ brick form

def brick_form(vkt, torch, stream, src):
    """BrickDecompose of the step's 512^3 uint8 volume into 64^3 bricks, without ghost cells
    and with the 2 ghost cells a 5^3 filter needs: ms per call (device time of the call,
    including its small brick-table upload) and GB/s on the algorithmic bytes (the source
    read once, every brick voxel written once)."""
    import ctypes
    out = {}
    for g in (0, 2):
        bricks = vkt.brick_decompose(src, (64, 64, 64), g, stream=stream)
        views = [vkt.StructuredVolume.from_tensor(t) for t in bricks]
        arr = (ctypes.c_void_p * len(views))(*(v.handle.value for v in views))
        sv = vkt.StructuredVolume.from_tensor(src)
        reps = 10
        with vkt.policy(stream=stream):
            def call():
                vkt.check(vkt._lib.vktBrickDecomposeSV(arr, len(views), sv.handle, 64, 64, 64, g))
            for _ in range(3):
                call()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                call()
            b.record(stream)
            torch.cuda.synchronize()
            vkt.synchronize()
        ms = a.elapsed_time(b) / reps
        nbytes = src.numel() * src.element_size() + sum(t.numel() * t.element_size() for t in bricks)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[f"ghost{g}"] = {"bricks": len(bricks), "ms": round(ms, 4), "algorithmic_bytes": int(nbytes),
                            "achieved_gbs": round(gbs, 1),
                            "frac_hbm": round(gbs / measured_peaks()[0]["hbm_gbs"], 4)}
        del views, bricks
    return out


# ------------------------------------------------------------------ CLAHE form

def clahe_form(vkt, torch, stream):
    """CLAHE-3D at the paper's case-study size (256^3 uint8 CT-like volume, 8^3 bricks of
    32^3 voxels, clip limit 2): ms per call (the histogram, mapping and blend kernels plus
    their scratch), and GB/s on its algorithmic bytes (the volume read twice, the result
    written once)."""
    import synth
    v = torch.from_numpy(synth.volume("blobs", synth.U8, (256, 256, 256), synth.BASE_SEED + 1)).cuda()
    out = torch.empty_like(v)
    reps = 20
    for _ in range(3):
        vkt.clahe3d(v, (8, 8, 8), 2.0, out=out, stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        vkt.clahe3d(v, (8, 8, 8), 2.0, out=out, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    vkt.synchronize()
    ms = a.elapsed_time(b) / reps
    nbytes = 3 * v.numel()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"dims": [256, 256, 256], "bricks": [8, 8, 8], "clip_limit": 2.0, "ms": round(ms, 4),
            "gvoxel_s": round(v.numel() / (ms * 1e-3) / 1e9, 2), "achieved_gbs": round(gbs, 1),
            "frac_hbm": round(gbs / measured_peaks()[0]["hbm_gbs"], 4),
            "paper_context": "about 30 ms on a Quadro RTX 8000 (Sec. 4.1), other hardware"}


# ------------------------------------------------------------------ render form

def render_form(vkt, torch, stream, src):
    """Headless ray marching (absorption and emission) of the step's 512^3 uint8 volume into
    a 1024 x 768 RGBA float image, step 0.5 voxel, a four-entry ramp table, no early
    termination: ms per frame, rays and samples per second (the samples counted on the host
    from each pixel's ray-box interval)."""
    import math
    W, H, step = 1024, 768, 0.5
    eye, center, up, fovy = (256.0, 300.0, -600.0), (256.0, 256.0, 256.0), (0.0, 1.0, 0.0), 0.8
    lut = np.array([[0, 0, 0, 0], [0.9, 0.5, 0.2, 0.02], [1, 0.9, 0.6, 0.15], [1, 1, 1, 0.6]], np.float32)
    img = vkt.render(src, W, H, eye, center, up, fovy, step, lut, stream=stream)
    reps = 10
    for _ in range(2):
        vkt.render(src, W, H, eye, center, up, fovy, step, lut, out=img, stream=stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        vkt.render(src, W, H, eye, center, up, fovy, step, lut, out=img, stream=stream)
    b.record(stream)
    torch.cuda.synchronize()
    vkt.synchronize()
    ms = a.elapsed_time(b) / reps
    # samples per ray from the same camera model (float64 on the host)
    f = np.subtract(center, eye); f /= np.linalg.norm(f)
    r = np.cross(f, up); r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(fovy / 2)
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    d = (f[None, None] + ((2 * px / W - 1) * th * W / H)[..., None] * r
         + ((1 - 2 * py / H) * th)[..., None] * u)
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    n = np.array(src.shape[::-1], dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta = (0 - np.array(eye)) / d
        tb = (n - np.array(eye)) / d
    t0 = np.maximum(np.max(np.minimum(ta, tb), axis=-1), 0)
    t1 = np.min(np.maximum(ta, tb), axis=-1)
    samples = float(np.sum(np.where(t1 > t0, np.ceil((t1 - t0) / step - 0.5), 0)))
    return {"image": [W, H], "step": step, "ms": round(ms, 4),
            "mrays_s": round(W * H / (ms * 1e-3) / 1e6, 1),
            "gsamples_s": round(samples / (ms * 1e-3) / 1e9, 2), "samples": int(samples)}


# ------------------------------------------------------------------ smallest case

def small_form(vkt, torch, stream, lib, dev):
    """The smallest case: one float32 volume of 64^3 voxels i.i.d. U[0,1) from the seed, the
    normalised 3^3 Gaussian sigma 1.0 as dense weights on the FP32 direct path.  Its 2 MiB
    of algorithmic bytes stay in L2 and one call takes a few microseconds, so it is
    launch-bound: reported as the per-call time of 200 calls back to back on one stream
    (bound by the host's per-call work), of 20 calls captured in a CUDA graph and replayed
    (the device time per call), and of one call bracketed alone by events (median of 20)."""
    import synth
    n = 64
    x = torch.from_numpy(synth.volume("uniform", synth.F32, (n, n, n), synth.BASE_SEED)).to(dev)
    y = torch.empty_like(x)
    vx, vy = vkt.StructuredVolume.from_tensor(x), vkt.StructuredVolume.from_tensor(y)
    # the library's own normalised Gaussian (its dense float32 weights), given as a dense filter
    g = vkt.Filter.gaussian(3, 1.0)
    f = vkt.Filter.dense(g.weights())
    g.destroy()
    loop = 200
    with vkt.policy(stream=stream, path="direct"):
        call = lambda: vkt.check(lib.vktApplyFilterSV(vy.handle, vx.handle, f.handle))
        for _ in range(5):
            call()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(loop):
            call()
        b.record(stream)
        torch.cuda.synchronize()
        ms_loop = a.elapsed_time(b) / loop
        # the call captured once in a CUDA graph and replayed: the device time per call
        # without the host's per-call work (argument checks, the Python-to-C call)
        gs = torch.cuda.Stream(dev)
        gs.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            with vkt.policy(stream=gs, path="direct"):
                for _ in range(20):
                    call()
        stream.wait_stream(gs)
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(10):
            graph.replay()
        b.record(stream)
        torch.cuda.synchronize()
        ms_graph = a.elapsed_time(b) / (10 * 20)
        single = []
        for _ in range(20):
            a.record(stream)
            call()
            b.record(stream)
            torch.cuda.synchronize()
            single.append(a.elapsed_time(b))
        vkt.synchronize()
    ms_one = statistics.median(single)
    vox = n ** 3
    for h in (vx, vy):
        h.destroy()
    f.destroy()
    return {"dims": [n, n, n], "src": "f32 U[0,1)", "filter": "gaussian k3 sigma1 (dense weights)",
            "path": "direct", "bound": "launch (inputs and outputs L2-resident)",
            "back_to_back_ms": round(ms_loop, 5),
            "back_to_back_gvoxel_s": round(vox / (ms_loop * 1e-3) / 1e9, 2),
            "graph_replay_ms_per_call": round(ms_graph, 5),
            "graph_replay_gvoxel_s": round(vox / (ms_graph * 1e-3) / 1e9, 2),
            "single_call_ms": round(ms_one, 5),
            "single_call_gvoxel_s": round(vox / (ms_one * 1e-3) / 1e9, 2)}


# ------------------------------------------------------------------ differentiation form

def differentiation_form(vkt, torch, stream, lib, dev):
    """One training step's filter work on a batch of 8 float32 blob volumes of 128^3 with a
    learnable dense 5^3 kernel (N(0, 0.1)), the loss being the mean squared difference to
    the same volumes filtered by a hidden 5^3 kernel: the forward filter of the batch
    (vktApplyFilterBatchSV with one filter: one direct launch over the 8 volumes), then
    vktApplyFilterBackwardBatchSV (dL/dx by the exact adjoint in one launch, dL/dw by the
    per-tap reduction in one launch plus one FP64 reduction over the whole batch).  The loss
    gradient dL/dy = 2 (y - y*) / N is formed between the two by torch (the caller's loss, not
    the filter) and is not timed.  Reports forward and backward ms per batch, the library's
    launches per step, forward+backward Gvoxel/s (output voxels of the forward), and the
    fraction of the FP32 FMA peak (SMs x 128 FMA per clock x the maximum SM clock) on the
    algorithmic 3 x 125 FMA per voxel."""
    import ctypes
    import synth
    B, n, k = 8, 128, 5
    x = torch.from_numpy(np.stack([synth.blobs(synth.BASE_SEED + 100 + b, (n, n, n))
                                   for b in range(B)]).astype(np.float32)).to(dev)
    w0 = synth.normal(synth.BASE_SEED + 200, (k, k, k), 0.0, 0.1).astype(np.float32)
    wh = synth.normal(synth.BASE_SEED + 201, (k, k, k), 0.0, 0.1).astype(np.float32)
    f, fh = vkt.Filter.dense(w0), vkt.Filter.dense(wh)
    y, target, gy = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    gx = torch.zeros_like(x)
    gw = torch.zeros(k ** 3, dtype=torch.float32, device=dev)
    vx = [vkt.StructuredVolume.from_tensor(x[b]) for b in range(B)]
    vy = [vkt.StructuredVolume.from_tensor(y[b]) for b in range(B)]
    vt = [vkt.StructuredVolume.from_tensor(target[b]) for b in range(B)]
    vgx = [vkt.StructuredVolume.from_tensor(gx[b]) for b in range(B)]
    vgy = [vkt.StructuredVolume.from_tensor(gy[b]) for b in range(B)]
    reps = 10
    fwd_ms, bwd_ms = [], []
    arr = ctypes.c_void_p * B
    h_x, h_y, h_t = (arr(*(v.handle.value for v in vs)) for vs in (vx, vy, vt))
    h_gx, h_gy = (arr(*(v.handle.value for v in vs)) for vs in (vgx, vgy))
    h_f, h_fh = arr(*([f.handle.value] * B)), arr(*([fh.handle.value] * B))
    launches = 0
    with vkt.policy(stream=stream, path="direct"):
        vkt.check(lib.vktApplyFilterBatchSV(B, h_t, h_x, h_fh))
        for it in range(3 + reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            l0 = vkt.launch_count()
            ev[0].record(stream)
            vkt.check(lib.vktApplyFilterBatchSV(B, h_y, h_x, h_f))
            ev[1].record(stream)
            with torch.cuda.stream(stream):
                torch.sub(y, target, out=gy)
                gy.mul_(2.0 / y.numel())
            ev[2].record(stream)
            vkt.check(lib.vktApplyFilterBackwardBatchSV(B, h_gx, ctypes.c_void_p(gw.data_ptr()), h_gy,
                                                        h_x, f.handle))
            ev[3].record(stream)
            launches = vkt.launch_count() - l0
            torch.cuda.synchronize()
            vkt.synchronize()
            if it >= 3:
                fwd_ms.append(ev[0].elapsed_time(ev[1]))
                bwd_ms.append(ev[2].elapsed_time(ev[3]))
    if not bool(torch.isfinite(gw).all()) or not bool(torch.isfinite(gx).all()):
        raise RuntimeError("non-finite gradient in the differentiation form")
    fms, bms = statistics.median(fwd_ms), statistics.median(bwd_ms)
    vox = B * n ** 3
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = measured_peaks()[0].get("sm_max_mhz", 2070.0)
    fma_peak = props.multi_processor_count * 128 * sm_mhz * 1e6
    fma = 3 * k ** 3 * vox
    for h in vx + vy + vt + vgx + vgy:
        h.destroy()
    f.destroy()
    fh.destroy()
    return {"batch": B, "dims": [n, n, n], "k": k,
            "path": "direct over the batch (forward), adjoint + weight reduction over the batch (backward)",
            "library_launches_per_step": launches,
            "forward_ms": round(fms, 4), "backward_ms": round(bms, 4),
            "forward_gvoxel_s": round(vox / (fms * 1e-3) / 1e9, 2),
            "fwd_bwd_gvoxel_s": round(vox / ((fms + bms) * 1e-3) / 1e9, 2),
            "fp32_fma_peak_tfma_s": round(fma_peak / 1e12, 1),
            "frac_fp32": round(fma / ((fms + bms) * 1e-3) / fma_peak, 4),
            "not_timed": "the loss gradient 2 (y - y*) / N (torch, between forward and backward)"}


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import synth
    import paper_2203_10213_gb300 as vkt

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    vol = workload_host()
    src = torch.from_numpy(vol).to(dev)
    out_g = torch.empty(vol.shape, dtype=torch.float32, device=dev)
    out_l = torch.empty(vol.shape, dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    v_src = vkt.StructuredVolume.from_tensor(src, 0.0, 1.0)
    v_g = vkt.StructuredVolume.from_tensor(out_g, 0.0, 1.0)
    v_l = vkt.StructuredVolume.from_tensor(out_l, 0.0, 1.0)
    lap = vkt.Filter.dense(synth.laplacian_3())
    lib = vkt._lib
    vkt.set_policy(stream=stream)

    def step(evs=None):
        g = vkt.Filter.gaussian(5, 1.5)          # filter construction is part of the path
        if evs:
            evs[0].record(stream)
        vkt.check(lib.vktApplyFilterSV(v_g.handle, v_src.handle, g.handle))
        if evs:
            evs[1].record(stream)
        vkt.check(lib.vktApplyFilterSV(v_l.handle, v_src.handle, lap.handle))
        if evs:
            evs[2].record(stream)
        g.destroy()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    vkt.synchronize()

    K = args.steps
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
    kern_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.2)
    launches0 = vkt.launch_count()
    wall0 = time.perf_counter()
    for i in range(K):
        flush.zero_()                             # L2 flush, outside the step's events
        step_ev[i][0].record(stream)
        step(kern_ev[i])
        step_ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = vkt.launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    vkt.synchronize()

    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    sep_ms = [e[0].elapsed_time(e[1]) for e in kern_ev]
    dir_ms = [e[1].elapsed_time(e[2]) for e in kern_ev]
    total_ms = max_over_ranks(sum(step_ms), dev, world)
    ms_per_step = total_ms / K
    vox = float(np.prod(DIMS))
    value = replica_gvoxel_s(2 * vox, world, ms_per_step)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed.  Steps
    # alternate between two streams, each with its own device volumes and host buffers, so
    # one step's device-to-host copies overlap the next step's upload and filtering (the
    # copy engines and the SMs work at once); every step still uploads its input and
    # reads back both of its outputs.
    e2e = None
    if rank == 0 or world > 1:
        host_in = torch.from_numpy(vol).pin_memory()
        E = max(2, args.e2e_steps)
        slots = []
        for si in range(2):
            d_src = src if si == 0 else torch.empty_like(src)
            d_g = out_g if si == 0 else torch.empty_like(out_g)
            d_l = out_l if si == 0 else torch.empty_like(out_l)
            slots.append({
                "stream": stream if si == 0 else torch.cuda.Stream(dev),
                "src": vkt.StructuredVolume.from_tensor(d_src, 0.0, 1.0),
                "g": vkt.StructuredVolume.from_tensor(d_g, 0.0, 1.0),
                "l": vkt.StructuredVolume.from_tensor(d_l, 0.0, 1.0),
                "keep": (d_src, d_g, d_l),
                "host_g": torch.empty(vol.shape, dtype=torch.float32).pin_memory(),
                "host_l": torch.empty(vol.shape, dtype=torch.float32).pin_memory()})

        def e2e_step(sl):
            with vkt.policy(stream=sl["stream"]):
                vkt.check(lib.vktStructuredVolumeSetData(sl["src"].handle, host_in.data_ptr()))
                g = vkt.Filter.gaussian(5, 1.5)
                vkt.check(lib.vktApplyFilterSV(sl["g"].handle, sl["src"].handle, g.handle))
                vkt.check(lib.vktApplyFilterSV(sl["l"].handle, sl["src"].handle, lap.handle))
                vkt.check(lib.vktStructuredVolumeCopyToHost(sl["g"].handle, sl["host_g"].data_ptr()))
                vkt.check(lib.vktStructuredVolumeCopyToHost(sl["l"].handle, sl["host_l"].data_ptr()))
                g.destroy()

        for i in range(4):
            e2e_step(slots[i % 2])
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        slots[1]["stream"].wait_event(a)
        for i in range(E):
            e2e_step(slots[i % 2])
        done = torch.cuda.Event()
        done.record(slots[1]["stream"])
        stream.wait_event(done)
        b.record(stream)
        torch.cuda.synchronize()
        vkt.set_policy(stream=stream)
        vkt.synchronize()
        e2e_ms = max_over_ranks(a.elapsed_time(b) / E, dev, world)
        e2e = {"value": round(replica_gvoxel_s(2 * vox, world, e2e_ms), 3), "unit": "Gvoxel/s",
               "h2d_bytes_per_step": int(host_in.numel()),
               "d2h_bytes_per_step": int(2 * vol.size * 4),
               "ms_per_step": round(e2e_ms, 4),
               "pipeline": "two streams, double-buffered device volumes and host buffers"}
        del slots

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    alg_bytes = vox * (1 + 4)                   # u8 in, f32 out per launch
    kernels = []
    for name, ms in (("separable gaussian5", sep_ms), ("direct laplacian3", dir_ms)):
        avg = statistics.mean(ms)
        gbs = alg_bytes / (avg * 1e-3) / 1e9
        kernels.append({"kernel": name, "avg_ms": round(avg, 5), "achieved_gbs": round(gbs, 1),
                        "frac_hbm": round(gbs / hbm, 4),
                        "gvoxel_s": round(vox / (avg * 1e-3) / 1e9, 2)})
    dom = max(kernels, key=lambda k: k["avg_ms"])
    traffic, traffic_note = captured_traffic(dom["kernel"])
    roofline = {"bound": "hbm", "kernel": dom["kernel"], "achieved": dom["achieved_gbs"],
                "peak": hbm, "unit": "GB/s", "frac": dom["frac_hbm"],
                "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy)",
                "algorithmic_bytes_per_launch": int(alg_bytes), "traffic": traffic,
                "traffic_note": traffic_note}

    pin = None if args.no_precision_form else precision_inputs()
    cpu, refs = None, None
    if not args.no_cpu_baseline:
        cpu, refs = cpu_leg(args, vol, pin)

    pform = None
    if pin is not None:
        pform = precision_form(args, vkt, torch, dev, stream, peaks, *pin, refs)
    bform = None
    if not args.no_batching_form:
        bform = batching_form(args, vkt, torch, dev, stream)
    kform = cform = vform = rform = dform = sform = None
    if not args.no_extra_forms:
        kform = brick_form(vkt, torch, stream, src)
        cform = clahe_form(vkt, torch, stream)
        vform = render_form(vkt, torch, stream, src)
        g_roi = vkt.Filter.gaussian(5, 1.5)
        rform = range_form(vkt, torch, stream, lib, v_g, v_l, v_src, g_roi, lap)
        g_roi.destroy()
        try:
            dform = differentiation_form(vkt, torch, stream, lib, dev)
        except Exception as e:   # reported in the line; the step's figures stand on their own
            dform = {"error": f"{type(e).__name__}: {e}"}
        try:
            sform = small_form(vkt, torch, stream, lib, dev)
        except Exception as e:
            sform = {"error": f"{type(e).__name__}: {e}"}

    line = {"metric": METRIC, "value": round(value, 3), "unit": "Gvoxel/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded CT-like blobs, no dataset)",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "src": "u8 range [0,1]",
                       "dst": "f32", "filters": ["gaussian k5 sigma1.5 separable",
                                                 "laplacian 7-point as dense k3"],
                       "l2": "flushed before every timed step (256 MiB write, untimed)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "precision_form": pform, "batching_form": bform,
            "range_form": rform, "brick_form": kform, "clahe_form": cform, "render_form": vform,
            "differentiation_form": dform, "small_form": sform,
            "wall_s_timed_loop": round(wall, 3)}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm (oracle)

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    vol = workload_host()
    total = max(1, args.steps + args.warmup)
    per_step = max(0.01, 60.0 / total)
    rate, n, dt = oracle_sample_rate(vol, per_step)
    rng = np.random.default_rng(11)
    w_g = oracle.gaussian_weights(5, float(np.float32(1.5)))
    w_l = oracle.laplacian_3()
    times = []
    for i in range(total):
        idx = rng.integers(0, vol.size, n)
        t0 = time.perf_counter()
        oracle.correlate_points(vol, w_g, idx, 0.0, 1.0)
        oracle.correlate_points(vol, w_l, idx, 0.0, 1.0)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    sec = statistics.mean(times)
    value = 2 * n / sec / 1e9
    cpu = {"value": round(value, 6), "unit": "Gvoxel/s", "cores": oracle.num_threads(),
           "kind": "oracle", "sample": f"{n} random voxels per step of the 512^3 volume, both filters"}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gvoxel/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec * 1e3, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded CT-like blobs)",
            "config": {"workload": WORKLOAD, "dims": list(DIMS), "src": "u8 range [0,1]",
                       "dst": "f32 (oracle computes f64)"},
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 6), "unit": "Gvoxel/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_batch_case(args):
    """The 256-volume batch of the batching form, --reps graph launches (fixed rule, no
    tuning), for profiler captures of the persistent batch kernels."""
    import ctypes
    import torch
    import synth
    import paper_2203_10213_gb300 as vkt
    items = synth.batch_recipe(synth.BASE_SEED + 3, n=256)
    dt = {synth.U8: torch.uint8, synth.U16: torch.uint16, synth.F32: torch.float32}
    keep, vs, vd, fs = [], [], [], []
    for it in items:
        a = synth.volume(it["kind"], it["fmt"], it["dims"], it["seed"])
        s = torch.from_numpy(a).cuda()
        d = torch.empty(a.shape, dtype=dt[it["fmt"]], device="cuda")
        keep += [s, d]
        vs.append(vkt.StructuredVolume.from_tensor(s))
        vd.append(vkt.StructuredVolume.from_tensor(d))
        fs.append(vkt.Filter.gaussian(it["k"], it["sigma"]))
    vkt.check(vkt._lib.vktAutotuneSetEnabled(0))
    for _ in range(args.reps):
        vkt.apply_filter_batch(vd, vs, fs)
    torch.cuda.synchronize()
    vkt.synchronize()
    print(json.dumps({"kernel_case": "batch256", "reps": args.reps,
                      "checksum": float(sum(float(np.abs(d.cpu().numpy().astype(np.float64)).mean())
                                            for d in keep[1::2]))}))


def run_bricks_case(args):
    """BrickDecompose of the step's 512^3 uint8 volume into 64^3 bricks with the 2 ghost cells
    a 5^3 filter needs, --reps calls, for profiler captures of the brick kernel."""
    import torch
    import paper_2203_10213_gb300 as vkt
    src = torch.from_numpy(workload_host()).cuda()
    bricks = None
    for _ in range(args.reps):
        bricks = vkt.brick_decompose(src, (64, 64, 64), 2)
    torch.cuda.synchronize()
    vkt.synchronize()
    print(json.dumps({"kernel_case": "bricks2_ct512", "reps": args.reps, "bricks": len(bricks),
                      "checksum": float(sum(float(b.double().mean()) for b in bricks))}))


def run_render_case(args):
    """The render form's frame (1024 x 768 of the 512^3 uint8 volume, step 0.5), --reps calls,
    for profiler captures of the ray-marching kernel."""
    import torch
    import paper_2203_10213_gb300 as vkt
    src = torch.from_numpy(workload_host()).cuda()
    img = None
    for _ in range(args.reps):
        img = vkt.render(src, 1024, 768, (256, 300, -600), (256, 256, 256), (0, 1, 0), 0.8, 0.5,
                         [[0, 0, 0, 0], [1, 0.8, 0.5, 0.1], [1, 1, 1, 0.6]])
    torch.cuda.synchronize()
    vkt.synchronize()
    print(json.dumps({"kernel_case": "render_ct512", "reps": args.reps,
                      "checksum": float(img.double().mean())}))


def run_backward_case(args):
    """The differentiation form's batch backward (8 float32 blob volumes of 128^3, dense 5^3
    kernel N(0, 0.1)), --reps calls, for profiler captures of the adjoint, shell and
    weight-gradient kernels."""
    import ctypes
    import torch
    import synth
    import paper_2203_10213_gb300 as vkt
    B, n, k = 8, 128, 5
    x = torch.from_numpy(np.stack([synth.blobs(synth.BASE_SEED + 100 + b, (n, n, n))
                                   for b in range(B)]).astype(np.float32)).cuda()
    f = vkt.Filter.dense(synth.normal(synth.BASE_SEED + 200, (k, k, k), 0.0, 0.1).astype(np.float32))
    gy = x * 1e-3
    gx = torch.zeros_like(x)
    gw = torch.zeros(k ** 3, dtype=torch.float32, device="cuda")
    vx = [vkt.StructuredVolume.from_tensor(x[b]) for b in range(B)]
    vgx = [vkt.StructuredVolume.from_tensor(gx[b]) for b in range(B)]
    vgy = [vkt.StructuredVolume.from_tensor(gy[b]) for b in range(B)]
    arr = ctypes.c_void_p * B
    hx, hgx, hgy = (arr(*(v.handle.value for v in vs)) for vs in (vx, vgx, vgy))
    with vkt.policy(path="direct"):
        for _ in range(args.reps):
            vkt.check(vkt._lib.vktApplyFilterBackwardBatchSV(B, hgx, ctypes.c_void_p(gw.data_ptr()),
                                                            hgy, hx, f.handle))
    torch.cuda.synchronize()
    vkt.synchronize()
    print(json.dumps({"kernel_case": "backward_train", "reps": args.reps, "gw0": float(gw[0])}))


def run_kernel_case(args):
    import torch
    import synth
    import paper_2203_10213_gb300 as vkt
    if args.kernel_case == "batch256":
        run_batch_case(args)
        return
    if args.kernel_case == "bricks2_ct512":
        run_bricks_case(args)
        return
    if args.kernel_case == "render_ct512":
        run_render_case(args)
        return
    if args.kernel_case == "backward_train":
        run_backward_case(args)
        return
    kind, fmt, dims, filt, path = KERNEL_CASES[args.kernel_case]
    if kind == "uniform":
        vol = synth.uniform(synth.BASE_SEED + 5, tuple(reversed(dims)), -1.0, 1.0)
    else:
        vol = synth.volume(kind, fmt, dims, SEED)
    if filt == "gaussian5":
        f = vkt.Filter.gaussian(5, 1.5)
    elif filt == "laplacian3":
        f = vkt.Filter.dense(synth.laplacian_3())
    else:
        w, _ = synth.random_kernel(synth.BASE_SEED + 2, 7, 1.0, normalise_sum=True)
        f = vkt.Filter.dense(w)
    src = torch.from_numpy(vol).cuda()
    out = torch.empty(vol.shape, dtype=torch.float32, device="cuda")
    for _ in range(args.reps):
        vkt.filter_tensor(src, f, path=path, out=out)
    torch.cuda.synchronize()
    vkt.synchronize()
    print(json.dumps({"kernel_case": args.kernel_case, "reps": args.reps,
                      "checksum": float(out.double().abs().mean())}))


def main():
    args = parse()
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

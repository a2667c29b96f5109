"""Benchmark: neural volumetric path tracing with photon fields on B300.

Workload (the paper's large-render setting, synthetic): 1024^3 float16
turbulence volume (2 GiB, larger than L2), 256-node RGBA transfer function,
8 point lights, 1920x1080 at 16 samples per pixel, phase coefficient g drawn
per frame from U[-0.9, 0.9], photon field 4 x 128 in f16 (the paper's field
precision, Sec. 4.1; fp8 e4m3 with per-layer power-of-two scales is reported
as a named variant), delta-tracking free flight and ratio-tracking shadow
rays (Algorithm 2).  One step = one frame of the 60-frame orbit through the
library's C ABI (pf_render_neural): camera samples, NEE, field queries,
compose.  The field is trained on the GPU (tcgen05 forward and backward) on
photon caches the GPU tracer builds, before timing (trace and train once,
render many frames).

Reports frames/s and field queries/s, the dominant stage's roofline from
live CUDA events, the end-to-end number through the C ABI with the camera
from host memory and the image read back to pinned host memory, clocks
sampled during the timed region, the equal-RMSE comparison with the plain
path tracer (4 frames at full resolution, against 4096-spp references, the
path tracer timed at the spp its fitted error curve needs), the mid-render
workload (512^3 u8, 1024^2 x 4 spp, f16 and fp8 fields), training and
photon-cache throughput, dense f16 / fp8 GEMM peaks measured on this GPU,
and the CPU oracle on bounded samples.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/sec and field queries/sec vs plain GPU path tracer at equal RMSE"
W_, H_, SPP, N_VOX, N_LIGHTS = 1920, 1080, 16, 1024, 8
BRICK = 32                      # majorant brick edge (voxels) for the 1024^3 volume
BRICK_PRIMARY = 128             # brick edge of the camera rays' (pooled) majorant grid
BRICK_SHADOW = 0                # brick edge walked by shadow rays, thinned to BRICK (0: BRICK)
BRICK_PT = 64                   # majorant brick edge of the path-tracer baseline (its own best, tuned apart)
HIDDEN, N_HIDDEN, FREQS = 128, 4, 12
FIELD_PREC = "f16"              # the paper's field precision (Sec. 4.1); fp8 is a variant
HELD_OUT_TOL = 0.01     # early stopping: held-out losses this close count as a tie
VOXEL_BYTES = 2                 # float16
EQ_FRAMES = (0, 15, 30, 45)     # orbit frames of the equal-RMSE comparison
# DRAM bytes (read + write) per density lookup of k_nee at full size, from a
# one-pass ncu capture of the two counted launches of this workload
# (profiles/k_nee__large_render_1024cube_1080p_dram.md: 21.14 GB over
# 2 x 104,918,229 lookups); a launch is scaled by its lookups.  None whenever
# k_nee changed since the capture.
NEE_DRAM_BYTES_PER_LOOKUP = 21136791808 / (2 * 104918229)
FETCH_BYTES = 8 * VOXEL_BYTES   # one trilinear lookup reads 8 voxels


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained", d["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, 1400.0, "fallback"


class Clocks:
    """SM clocks and clock-event (throttle) reasons sampled in the background
    while the timed region runs: NVML every 10 ms (the GPU matched to the
    CUDA device by PCI bus id), else nvidia-smi every 200 ms.  Reads only."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.samples = []        # (sm MHz, max MHz, reason names)
        self.stop_flag = threading.Event()
        self.nvml = None
        self.t = None

    # NVML through ctypes (the driver's libnvidia-ml; no Python binding
    # needed): clock id 1 = SM; clock-event reason bits of nvml.h
    NVML_CLOCK_SM = 1
    REASON_BITS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
                   "sw_power_cap": 0x4}

    def _nvml_handle(self):
        import ctypes
        import torch
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")
        h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(self.device)
        bus = getattr(props, "pci_bus_id", None)
        ok = False
        if bus is not None:
            bus_id = "%08x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0), bus, getattr(props, "pci_device_id", 0))
            ok = lib.nvmlDeviceGetHandleByPciBusId_v2(bus_id.encode(), ctypes.byref(h)) == 0
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.device), ctypes.byref(h)) != 0:
            raise RuntimeError("no NVML handle for device %d" % self.device)
        return lib, h

    def _poll_nvml(self):
        import ctypes
        lib, h = self.nvml
        mx = ctypes.c_uint(0)
        lib.nvmlDeviceGetMaxClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(mx))
        sm = ctypes.c_uint(0)
        r = ctypes.c_ulonglong(0)
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_flag.is_set():
            if lib.nvmlDeviceGetClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(sm)) != 0 or \
                    reasons(h, ctypes.byref(r)) != 0:
                break
            self.samples.append((float(sm.value), float(mx.value),
                                 [k for k, b in self.REASON_BITS.items() if r.value & b]))
            time.sleep(0.01)

    def start(self):
        try:
            self.nvml = self._nvml_handle()
            self.t = threading.Thread(target=self._poll_nvml, daemon=True)
            self.t.start()
            return
        except Exception as e:
            self.nvml = None
            self.nvml_error = repr(e)[:120]
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml:
            self.stop_flag.set()
            self.t.join(timeout=2)
            if not self.samples:
                return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "source": "nvml"}
            reasons = sorted({n for _, _, rs in self.samples for n in rs})
            return {"sm_mhz": float(np.median([s for s, _, _ in self.samples])),
                    "sm_max_mhz": float(max(m for _, m, _ in self.samples)), "reasons": reasons,
                    "samples": len(self.samples), "source": "nvml, 10 ms"}
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(self.NAMES, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 200 ms",
                "nvml_error": getattr(self, "nvml_error", None)}


def reduce_max(x: float, dist, device) -> float:
    """Max over ranks of a per-rank float (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / seconds_max


def frame_index(rank: int, i: int, n_frames: int) -> int:
    """Frame of the orbit that rank `rank` renders as its i-th frame (ranks
    start 1000 frames apart, so their frames differ)."""
    return (rank * 1000 + i) % n_frames


def setup_scene(device):
    import torch
    from paper_2304_07338_b300 import inputs as I
    vol_t, tf, lights, cams = I.large_scene_parts(N_VOX, device=device)
    cams = [I.Camera(c.eye, c.at, c.up, c.fovy_deg, W_, H_) for c in cams]
    return vol_t.contiguous(), torch.from_numpy(tf).to(device), lights, cams


def _prec_name(desc):
    return {0: "f32", 1: "bf16", 2: "f16", 3: "fp8"}.get(getattr(desc, "prec", 0), "?") if desc else "no"


def cpu_baseline(vol_host, tf, lights, cams, seed, rows=2, weights=None, desc=None, scales=None, brick=8,
                 brick_primary=0, cols=None, brick_shadow=0, t_fix=None):
    """The oracle (plain C++/numpy) on a bounded sample: `rows` image rows of
    one frame (all columns, or the columns [x0, x1)) at full spp, scaled to
    a frame.  The oracle's fixed cost per call (volume marshalling, brick
    majorants), timed on a one-pixel call, is counted once per frame; only
    the rest scales with the pixels."""
    import oracle
    from paper_2304_07338_b300 import inputs as I
    v = I.Volume(vol_host, 20.0, 0.9, tf, brick=brick, brick_primary=brick_primary, brick_shadow=brick_shadow)
    cam = cams[0]
    g = I.frame_g(seed, 0)
    y0 = H_ // 2
    x0, x1 = cols if cols is not None else (0, W_)
    if t_fix is None:       # the fixed cost (single-threaded majorant grids): a one-pixel call
        t = time.perf_counter()
        oracle.render_neural(v, lights, g, cam, SPP, 0.0, seed, weights=weights, desc=desc, scales=scales,
                             fp32=True, rows=(y0, y0 + 1), cols=(x0, x0 + 1))
        t_fix = time.perf_counter() - t
    t = time.perf_counter()
    oracle.render_neural(v, lights, g, cam, SPP, 0.0, seed, weights=weights, desc=desc, scales=scales, fp32=True,
                         rows=(y0, y0 + rows), cols=(x0, x1))
    dt = time.perf_counter() - t
    per_px = max(dt - t_fix, 1e-9) / (rows * (x1 - x0))
    frame_s = t_fix + per_px * H_ * W_
    return {"value": 1.0 / frame_s, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle", "fixed_s": t_fix,
            "sample": "%d pixels (%d row(s) x columns %d-%d) of frame 0 (%dx%d, %d spp, 8 lights, %s field "
                      "emulated in FP64), scaled to a full frame; %.2f s measured, of which %.2f s fixed per call "
                      "(counted once per frame)"
                      % (rows * (x1 - x0), rows, x0, x1, W_, H_, SPP, _prec_name(desc), dt, t_fix)}


def gemm_peaks(device, n=8192, reps=10, sustain_s=1.5):
    """Dense GEMM throughput of this GPU for the field's operand types,
    measured here: f16 (torch.matmul, cuBLAS) and fp8 e4m3 with f32
    accumulation (torch._scaled_mm, cuBLASLt), n^3, 2 n^3 flops per call;
    burst = best of `reps` single calls (CUDA events), sustained = calls back
    to back for about `sustain_s` seconds.  They are the denominators of the
    field kernels' tensor fractions (the driver's file has bf16 only)."""
    import torch
    out = {"how": "%d^3, 2n^3 flop/call; burst: best of %d (CUDA events); sustained: back to back for ~%.1f s"
                  % (n, reps, sustain_s)}
    g = torch.Generator(device=device).manual_seed(0)
    a16 = torch.randn(n, n, device=device, generator=g, dtype=torch.float16)
    b16 = torch.randn(n, n, device=device, generator=g, dtype=torch.float16)
    a8 = a16.to(torch.float8_e4m3fn)
    b8 = b16.to(torch.float8_e4m3fn).t()            # column-major second operand
    one = torch.ones((), device=device)
    calls = {"f16": lambda: torch.matmul(a16, b16),
             "fp8_e4m3": lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)}
    for name, fn in calls.items():
        try:
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            k = max(1, int(sustain_s / best))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(k):
                fn()
            e1.record()
            torch.cuda.synchronize()
            sus = e0.elapsed_time(e1) / 1e3 / k
            out[name] = {"burst_tflops": 2 * n ** 3 / best / 1e12, "sustained_tflops": 2 * n ** 3 / sus / 1e12}
        except Exception as e:  # reported, not fatal
            out[name] = {"error": repr(e)[:160]}
    del a16, b16, a8, b8
    torch.cuda.empty_cache()
    return out


def train_render_field(ctx, vol, lights, g_set, seed, photons, prec="f16", candidates=(150, 300, 600, 1000),
                       batch=1 << 16):
    """The render workloads' field, trained on the GPU (tcgen05) on photon
    caches of `photons` per light per g, with early stopping: one field per
    step count in `candidates` (the learning-rate schedule scales with the
    run), and the one with the lowest relative MSE on 2^16 held-out queries
    at phases between the traced ones (the midpoints of g_set), with targets
    from a cache traced there.  The renders draw g from U[-0.9, 0.9], so the
    field must interpolate across phases; the loss at the traced phases
    keeps falling with training while the interpolation between them
    degrades (the 12 frequencies of the g encoding let the field fit the
    traced phases separately), and only held-out phases show it.  Returns
    (field, cache, report)."""
    import torch
    from paper_2304_07338_b300 import api
    t0 = time.perf_counter()
    cache = api.build_photon_cache(ctx, vol, lights, g_set, photons, 16, 64, seed=seed + 1)
    ctx.sync()
    rep = {"photon_cache_s": time.perf_counter() - t0, "photons": int(cache.info.n_photons),
           "records": int(cache.n_records)}
    gs = sorted(g_set)
    g_held = [0.5 * (a + b) for a, b in zip(gs[:-1], gs[1:])]
    held = api.build_photon_cache(ctx, vol, lights, g_held, photons, 16, 64, seed=seed + 91)
    qv = held.sample_queries(1 << 16, step=0, seed=seed + 92)
    _, yv = held.estimate_targets(qv)
    runs, fields = {}, {}
    for n in candidates:
        f = api.Field(ctx, FREQS, HIDDEN, N_HIDDEN, prec, 5.0, seed=seed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = f.train(cache, steps=n, batch=batch, lr=1e-2, seed=seed + 2)
        dt = time.perf_counter() - t0
        y = f.forward(qv)
        val = float(torch.mean((y - yv) ** 2 / (yv ** 2 + 0.01)))
        runs[str(n)] = {"train_s": dt, "steps_per_s": n / dt, "loss_last": float(loss[-20:].mean()),
                        "held_out_loss": val}
        fields[n] = f
    held.free()
    # the fewest steps whose held-out loss is within HELD_OUT_TOL of the
    # lowest: candidates closer than that are a tie (the caches' FP64 sums
    # carry run-to-run rounding, and the training amplifies it to about 1 %)
    low = min(r["held_out_loss"] for r in runs.values())
    pick = min(n for n in candidates if runs[str(n)]["held_out_loss"] <= low * (1.0 + HELD_OUT_TOL))
    for n, f in fields.items():
        if n != pick:
            f.free()
    best = (pick, runs[str(pick)]["held_out_loss"], fields[pick])
    rep.update({"training": "4x128 %s on tcgen05, batches of %d, steps chosen by held-out loss at g = %s "
                            "(a cache traced there)" % (prec, batch, ", ".join("%g" % g for g in g_held)),
                "candidates": runs, "chosen_steps": best[0],
                "rule": "fewest steps within %g %% of the lowest held-out loss" % (100 * HELD_OUT_TOL)})
    return best[2], cache, rep


def field_flop(queries: float) -> float:
    """Field forward flops: 2 (144 H + (L-1) H^2 + 3 H) per query."""
    return queries * 2 * (12 * FREQS * HIDDEN + (N_HIDDEN - 1) * HIDDEN * HIDDEN + 3 * HIDDEN)


def render_frames(ctx, vol, lights, frame, field, seed, steps, warmup, dist, dev, clocks_dev=None, step_vox=0.0):
    """Warm-up frames, one untimed counting pass over the timed frames (density
    lookups, field queries, NEE lookups), then `steps` frames timed with CUDA
    events on the context's stream (barrier and synchronize on both sides,
    per-stage events inside) and, if clocks_dev is given, nvidia-smi sampled
    during the timed region."""
    import torch
    from paper_2304_07338_b300 import api
    H, W = frame(0)[0].height, frame(0)[0].width
    out = torch.empty(H, W, 3, device=dev)
    for i in range(warmup):
        cam, g = frame(i)
        api.render_neural(ctx, vol, lights, g, cam, SPP, step_vox, seed + i, field, out)
    ctx.sync()
    counters = torch.zeros(4, dtype=torch.int64, device=dev)
    ctx.set_counters(counters)
    for i in range(steps):
        cam, g = frame(warmup + i)
        api.render_neural(ctx, vol, lights, g, cam, SPP, step_vox, seed + 100 + i, field, out)
    ctx.sync()
    ctx.set_counters(None)
    ctx.stage_times()
    ctx.stage_timing(True)
    clocks = Clocks(clocks_dev) if clocks_dev is not None else None
    if clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s_ev.record(ctx.stream)
    for i in range(steps):
        cam, g = frame(warmup + i)
        api.render_neural(ctx, vol, lights, g, cam, SPP, step_vox, seed + 100 + i, field, out)
    e_ev.record(ctx.stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = s_ev.elapsed_time(e_ev)
    clk = clocks.stop() if clocks else None
    ctx.stage_timing(False)
    stages = ctx.stage_times()
    return {"ms_total": ms_total, "stages": stages, "clocks": clk, "out": out,
            "fetches": int(counters[0].item()) // steps, "queries": int(counters[1].item()) // steps,
            "nee_fetches": int(counters[2].item()) // steps}


def field_roofline(stage, queries_per_frame, steps, peak_tflops, peak_source):
    """Tensor roofline of the field forward (k_tc_forward) from its stage
    events: model flops of the frame's queries over the stage's time."""
    ms, n = stage
    per_launch_s = ms / max(n, 1) / 1e3
    achieved = field_flop(queries_per_frame) / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    return {"kernel": "k_tc_forward", "bound": "tensor", "achieved": achieved, "peak": peak_tflops,
            "unit": "TFLOP/s", "frac": achieved / peak_tflops if peak_tflops else None,
            "ms_per_frame": ms / max(steps, 1), "peak_source": peak_source}


def field_library_reference(queries_per_frame, field_ms, dev, hidden=128, n_hidden=4, freqs=12, reps=5):
    """The same 4 x 128 field on library kernels, for the frame's number of
    queries: the hidden layers as a chain of cuBLAS f16 GEMMs (torch.matmul,
    ReLU between them) with the 3-wide output layer in float32, on inputs
    already encoded; and the whole pipeline with the frequency encoding as
    torch elementwise ops.  Best of `reps`, CUDA events.  Timing does not
    depend on the weight values, so they are random."""
    import torch
    n = int(queries_per_frame)
    if n <= 0:
        return None
    g = torch.Generator(device=dev).manual_seed(7)
    q = torch.rand(n, 6, device=dev, generator=g)
    k0 = 6 * 2 * freqs
    ws = [torch.randn(hidden, k0 if l == 0 else hidden, device=dev, generator=g).half() * 0.05
          for l in range(n_hidden)]
    w_out = torch.randn(3, hidden, device=dev, generator=g) * 0.05
    scale = (torch.pi * 2.0 ** torch.arange(freqs, device=dev)).view(1, 1, freqs)

    def encode():
        a = q.unsqueeze(2) * scale                      # [n][6][F]
        return torch.stack((torch.sin(a), torch.cos(a)), dim=3).reshape(n, k0).half()

    def chain(x):
        for w in ws:
            x = torch.relu(torch.matmul(x, w.t()))
        return torch.matmul(x.float(), w_out.t())

    x0 = encode()

    def best(fn):
        fn()
        torch.cuda.synchronize()
        t = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            t = min(t, e0.elapsed_time(e1))
        return t

    chain_ms = best(lambda: chain(x0))
    full_ms = best(lambda: chain(encode()))
    del x0, q
    return {"queries": n, "cublas_chain_ms": chain_ms, "torch_encode_and_chain_ms": full_ms,
            "k_tc_forward_ms": field_ms,
            "k_tc_forward_speedup_vs_chain": chain_ms / field_ms if field_ms else None,
            "k_tc_forward_speedup_vs_full": full_ms / field_ms if field_ms else None,
            "how": "torch.matmul f16 (cuBLAS) per hidden layer + ReLU, float32 output layer; encoding as torch "
                   "sin/cos; best of %d, CUDA events" % reps}


def encoding_workload(ctx, queries_per_frame, dev, freqs=12, reps=5):
    """The frequency encoding (Sec. 3.4) on its own (pf_field_encode), for the
    frame's number of queries: 144 float32 features per query written to HBM
    (24 B read, 576 B written per query), so the standalone kernel is bound by
    its writes; inside k_tc_forward the same steps feed shared memory.  Best of
    `reps`, CUDA events on the library's stream."""
    import torch
    n = int(queries_per_frame)
    if n <= 0:
        return None
    q = torch.rand(n, 6, device=dev)
    out = torch.empty((n, 12 * freqs), dtype=torch.float32, device=dev)
    st = ctx.stream
    ctx.check(ctx.lib.pf_field_encode(ctx.h, q.data_ptr(), n, freqs, out.data_ptr()))
    ctx.sync()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.check(ctx.lib.pf_field_encode(ctx.h, q.data_ptr(), n, freqs, out.data_ptr()))
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    nbytes = n * (24 + 48 * freqs)
    del q, out
    return {"kernel": "k_field_encode", "queries": n, "ms": best, "queries_per_s": n / (best / 1e3),
            "features_per_s": n * 12 * freqs / (best / 1e3), "bound": "hbm",
            "achieved_gbs": nbytes / (best / 1e3) / 1e9, "bytes_per_query": 24 + 48 * freqs}


def handoff_cost(ctx, queries_per_frame, frame_ms, dev):
    """What the pass split costs in HBM traffic: a fused camera-sample +
    field kernel would keep each scattering sample's field input (query 24 B,
    albedo 12 B, slot index 4 B) and output (L_i 12 B) on the SM; here they
    are written once and read once per frame.  Measured as a device copy of
    the same bytes (read + write), best of 5."""
    import torch
    per_query = 2 * (24 + 12 + 4) + 2 * 12
    nbytes = int(queries_per_frame * per_query)
    half = max(nbytes // 2, 16)
    src = torch.empty(half, dtype=torch.uint8, device=dev)
    dst = torch.empty_like(src)
    dst.copy_(src)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dst.copy_(src)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del src, dst
    return {"bytes_per_query": per_query, "bytes_per_frame": nbytes, "ms_per_frame": best,
            "share_of_frame": best / frame_ms if frame_ms else None,
            "how": "device copy of the hand-off bytes (read + write), best of 5, CUDA events"}


def _omp_threads(n):
    """Sets the OpenMP thread count of the oracle's C++ part (libgomp is
    loaded once per process) and returns the previous value."""
    import ctypes
    try:
        gomp = ctypes.CDLL("libgomp.so.1")
        prev = gomp.omp_get_max_threads()
        gomp.omp_set_num_threads(int(n))
        return prev
    except OSError:
        return None


def cpu_baseline_plan(vol_host, tf, lights, cams, seed, args, prec, fixed_s=None):
    """The oracle (never tuned for speed) on bounded samples of every
    workload, on one host thread and on all of them (reported baselines):
      plain method: the marched render (64^3, 128^2 x 4 spp) in full;
      photon tracing: the data-source scene at 2^14 photons per light per g
        (FP64 transport), photons/s (scales linearly with photons);
      training: steps of 2^15 queries (sampling, cell targets, precision-
        emulated 4x64 bf16 forward, loss, backward, Adam in numpy FP64),
        time per step scaled linearly to 2^18;
      mid render: a 64x64 crop at 1 spp, samples/s extrapolated to a frame
        (1024^2 x 4 spp), the oracle's fixed cost per call counted once;
      large render (all threads): the headline cpu_baseline; one thread:
        the middle row, its fixed cost per call (the majorant grids,
        single-threaded either way) taken from the headline's."""
    import oracle
    from oracle import field as F
    from paper_2304_07338_b300 import inputs as I
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:  # numpy's BLAS threads then stay as they are
        threadpool_limits = None
    plan = {"cores": os.cpu_count(), "kind": "oracle"}
    sm = I.scene_small()
    sj = I.scene_judge()
    smid = I.scene_mid()
    for label, nthr in (("all_threads", os.cpu_count()), ("one_thread", 1)):
        prev = _omp_threads(nthr)
        lim = threadpool_limits(nthr) if threadpool_limits else None
        r = {}
        try:
            t = time.perf_counter()
            oracle.render_neural(sm.volume, sm.lights, sm.g, sm.camera, sm.spp, 0.5, 7)
            r["plain_method_frames_per_s"] = 1.0 / (time.perf_counter() - t)
            n_ph = 1 << 14
            t = time.perf_counter()
            tr = oracle.trace_photons(sj.volume, sj.lights, sj.g_set, n_ph, 16, 64, seed=1, fp32=False)
            r["photons_per_s"] = len(sj.lights) * len(sj.g_set) * n_ph / (time.perf_counter() - t)
            oc = oracle.build_cache(tr)
            csig = oracle.cell_sigma(sj.volume, 64)
            occ = oracle.occupied_cells(oc, csig)
            desc = F.FieldDesc(12, 64, 4, F.PREC_BF16, 5.0, seed)
            w = F.init_weights(desc).astype(np.float64)
            m = np.zeros_like(w)
            v = np.zeros_like(w)
            B, n_steps = 1 << 15, (10 if nthr > 1 else 2)
            t = time.perf_counter()
            for step in range(n_steps):
                q, _ = oracle.sample_queries(occ, 64, sj.g_set, B, step, seed)
                y = F.log_encode(oracle.estimate_targets(q, sj.g_set, oc, csig), 5.0)
                yh, cache = F.forward(w, q, desc)
                _, dy = F.rel_mse(yh, y)
                g = F.backward(w, cache, dy, desc)
                w, m, v = F.adam_step(w, m, v, g, step + 1, 1e-2, 0.9, 0.99, 1e-8)
            per = (time.perf_counter() - t) / n_steps * ((1 << 18) / B)
            r["training_s_per_step_2^18"] = per
            r["training_steps"] = "%d steps of %d queries, scaled to 2^18" % (n_steps, B)
            mv = I.Volume(smid.volume.data, smid.volume.sigma_scale, smid.volume.albedo, smid.volume.tf, brick=16,
                          brick_primary=64)
            fd = oracle_field(seed, prec)
            # a 128x128 crop at 1 spp (the 64x64 crop's time is within the
            # noise of the oracle's fixed cost per call, the best of two
            # one-pixel calls, which is subtracted)
            cy, cx = smid.camera.height // 2 - 64, smid.camera.width // 2 - 64
            t_fix = float("inf")
            for _ in range(2):
                t = time.perf_counter()
                oracle.render_neural(mv, smid.lights, smid.g, smid.camera, 1, 0.0, seed, fp32=True,
                                     rows=(cy, cy + 1), cols=(cx, cx + 1), **fd)
                t_fix = min(t_fix, time.perf_counter() - t)
            t = time.perf_counter()
            oracle.render_neural(mv, smid.lights, smid.g, smid.camera, 1, 0.0, seed, fp32=True, rows=(cy, cy + 128),
                                 cols=(cx, cx + 128), **fd)
            per_sample = max(time.perf_counter() - t - t_fix, 1e-9) / (128 * 128)
            r["mid_render_sample"] = "128x128 crop at 1 spp; %.2f s fixed per call subtracted" % t_fix
            n_frame = smid.camera.width * smid.camera.height * smid.spp
            r["mid_render_samples_per_s"] = 1.0 / per_sample
            r["mid_render_frames_per_s_extrapolated"] = 1.0 / (t_fix + per_sample * n_frame)
            if nthr == 1:
                one = cpu_baseline(vol_host, tf, lights, cams, seed, rows=1, brick=args.brick,
                                   brick_primary=args.brick_primary, brick_shadow=args.brick_shadow,
                                   t_fix=fixed_s, **oracle_field(seed, prec))
                r["large_render_frames_per_s_extrapolated"] = one["value"]
                r["large_render_sample"] = one["sample"]
        finally:
            if prev is not None:
                _omp_threads(prev)
            if lim is not None:
                lim.restore_original_limits()
        plan[label] = r
    return plan


def main():
    global W_, H_, SPP, N_VOX
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)   # one pass over the 60-frame orbit
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=64)  # ~20 s of host time (two oracle calls)
    ap.add_argument("--res", type=int, default=N_VOX, help="volume resolution (profiling: smaller case)")
    ap.add_argument("--width", type=int, default=W_)
    ap.add_argument("--height", type=int, default=H_)
    ap.add_argument("--spp", type=int, default=SPP)
    ap.add_argument("--photons", type=int, default=1 << 22, help="photons per light per g for the caches")
    ap.add_argument("--no-train", action="store_true",
                    help="untrained field (profiling: the timing does not depend on the weights)")
    ap.add_argument("--train-batch", type=int, default=1 << 16)
    ap.add_argument("--no-equal-rmse", action="store_true")
    ap.add_argument("--ref-spp", type=int, default=4096)
    ap.add_argument("--brick", type=int, default=BRICK, help="majorant brick edge in voxels (power of two)")
    ap.add_argument("--no-march", action="store_true", help="skip the ray-marched renderer's measurement")
    ap.add_argument("--no-mid", action="store_true", help="skip the mid-render workload")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline frames (profiling): no variants, comparisons or workloads")
    ap.add_argument("--linear-voxels", action="store_true",
                    help="gather from the caller's x-fastest volume instead of the 4x4x4-tiled copy")
    ap.add_argument("--field-prec", default=FIELD_PREC, choices=["f16", "bf16", "fp8"],
                    help="precision of the timed field (profiling)")
    ap.add_argument("--step-vox", type=float, default=0.0,
                    help="render the timed frames with the ray-marched sampler of this step (profiling; 0: tracking)")
    ap.add_argument("--training-only", action="store_true",
                    help="run only the field-training workload and print its JSON (profiling)")
    ap.add_argument("--training-steps", type=int, default=2000)
    ap.add_argument("--field-training-only", type=int, default=0, metavar="WIDTH",
                    help="run only WIDTH-wide f16 field training (data-source caches, 2^18 queries per step, "
                         "--training-steps steps) and print steps/s (profiling)")
    ap.add_argument("--brick-pt", type=int, default=BRICK_PT,
                    help="majorant brick edge of the path-tracer baseline (power of two)")
    ap.add_argument("--brick-shadow", type=int, default=BRICK_SHADOW,
                    help="brick edge walked by shadow rays, thinned to --brick (0: --brick)")
    ap.add_argument("--brick-primary", type=int, default=BRICK_PRIMARY,
                    help="brick edge of the camera rays' pooled majorant grid (multiple of --brick)")
    args = ap.parse_args()
    W_, H_, SPP, N_VOX = args.width, args.height, args.spp, args.res
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    seed = 20230418

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, dev, seed)
        if dist:
            dist.destroy_process_group()
        return

    from paper_2304_07338_b300 import api, build, inputs as I
    build.build()
    ctx = api.Context(local)
    if args.training_only or args.field_training_only:
        if rank == 0:
            if args.field_training_only:
                out = {"field_training": field_training_only(ctx, seed, args.field_training_only,
                                                             args.training_steps)}
            else:
                out = {"training_workload": training_workload(ctx, seed, args.training_steps)}
            print(json.dumps(out), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    vol_t, tf_t, lights, cams = setup_scene(dev)
    vol = api.Volume(vol_t, 20.0, 0.9, tf_t, brick=args.brick, brick_primary=args.brick_primary,
                     brick_shadow=args.brick_shadow)
    vol.s.majorant = vol.majorant(ctx)
    vol.attach_brick_majorants(ctx)
    if not args.linear_voxels:
        vol.attach_tiled(ctx)
    # the path-tracer baseline walks its own majorant grid (same voxels)
    vol_pt = vol
    if args.brick_pt != args.brick:
        vol_pt = api.Volume(vol_t, 20.0, 0.9, tf_t, brick=args.brick_pt)
        vol_pt.s.majorant = vol.s.majorant
        vol_pt.attach_brick_majorants(ctx)
        if not args.linear_voxels:
            vol_pt.tiled = vol.tiled
            vol_pt.s.tiled_dev = vol.s.tiled_dev
    fields = {}
    train_prec = "bf16" if args.field_prec == "bf16" else "f16"
    if not args.no_train:
        trainer, cache, setup = train_render_field(ctx, vol, lights, I.G_PAPER, seed, args.photons, train_prec,
                                                   batch=args.train_batch)
    else:     # untrained field (profiling runs: the timing does not depend on the weights)
        trainer = api.Field(ctx, FREQS, HIDDEN, N_HIDDEN, train_prec, 5.0, seed=seed)
        cache, setup = None, {"training": "none (untrained field)"}
    fields[train_prec] = trainer
    fp8 = api.Field(ctx, FREQS, HIDDEN, N_HIDDEN, "fp8", 5.0, seed=seed)
    fp8.set_weights(trainer.get_weights())
    fp8.calibrate_fp8(calibration_queries().to(dev))
    fields["fp8"] = fp8
    head = args.field_prec if args.field_prec in fields else train_prec
    field = fields[head]

    def frame(i):
        f = frame_index(rank, i, len(cams))
        return cams[f], I.frame_g(seed, f)

    # ---- timed region: the headline field
    run = render_frames(ctx, vol, lights, frame, field, seed, args.steps, args.warmup, dist, dev, clocks_dev=local,
                        step_vox=args.step_vox)
    ms_total = reduce_max(run["ms_total"], dist, dev)
    stages, clk, out = run["stages"], run["clocks"], run["out"]
    ms_per_step = ms_total / args.steps
    fps = whole_job_rate(args.steps, world, ms_total / 1e3)
    qpf, fetches_per_frame, nee_fetches_per_frame = run["queries"], run["fetches"], run["nee_fetches"]

    # end to end through the C ABI, over the same frames as the timed region:
    # camera and lights from host memory, each frame's image copied into
    # pinned host memory and waited for by the host; the copy of frame i
    # (second stream) overlaps the rendering of frame i + 1 (two buffers)
    host_img = [torch.empty(H_, W_, 3, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    outs = [out, torch.empty_like(out)]
    copy_stream = torch.cuda.Stream(device=dev)
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = args.steps
    for i in range(e2e_steps):
        b = i & 1
        cam, g = frame(args.warmup + i)
        if i >= 2:
            ctx.stream.wait_event(copied[b])              # buffer b's previous copy is done
        api.render_neural(ctx, vol, lights, g, cam, SPP, args.step_vox, seed + 100 + i, field, outs[b])
        rendered[b].record(ctx.stream)
        copy_stream.wait_event(rendered[b])
        with torch.cuda.stream(copy_stream):
            host_img[b].copy_(outs[b], non_blocking=True)
            copied[b].record(copy_stream)
        if i >= 1:
            copied[b ^ 1].synchronize()                   # the host has frame i - 1
    copied[(e2e_steps - 1) & 1].synchronize()
    e2e_total = reduce_max(time.perf_counter() - t0, dist, dev)
    e2e_fps = whole_job_rate(e2e_steps, world, e2e_total)
    import ctypes
    h2d = ctypes.sizeof(api.PfCamera) + N_LIGHTS * ctypes.sizeof(api.PfLight)
    d2h = H_ * W_ * 3 * 4

    hbm, bf16, bf16s, src = peaks()
    gp = gemm_peaks(dev) if not args.no_extras else {}
    cam_ms, cam_n = stages["camera"]
    pooled = [e for e in (args.brick_primary, args.brick_shadow) if e > args.brick]
    grid_launches = len(pooled) + 1 + len(pooled)     # k_pool_majorants per pooled grid, k_border_grid per grid
    nee_ms, nee_n = stages["nee"]
    fld_ms, fld_n = stages["field"]
    cmp_ms, cmp_n = stages["compose"]

    def tensor_peak(prec):
        """Sustained peak for the field's operand type (the field runs inside
        a long step): measured here for f16 / fp8, the driver's bf16 file."""
        key = {"f16": "f16", "fp8": "fp8_e4m3"}.get(prec)
        if key and "sustained_tflops" in gp.get(key, {}):
            return gp[key]["sustained_tflops"], "measured %s sustained (torch GEMM on this GPU)" % key
        if prec == "fp8":
            return 2 * bf16s, src + " bf16 sustained x 2 (fp8 nominal ratio)"
        return bf16s, src + " bf16 sustained"

    dominant = max((cam_ms, "camera"), (nee_ms, "nee"), (fld_ms, "field"))[1]
    if dominant in ("camera", "nee"):
        st_ms, st_n = stages[dominant]
        lookups = nee_fetches_per_frame if dominant == "nee" else fetches_per_frame - nee_fetches_per_frame
        per_launch_s = st_ms / max(st_n, 1) / 1e3
        alg_bytes = lookups * FETCH_BYTES
        achieved = alg_bytes / per_launch_s / 1e9
        name = "k_nee (ratio-tracked shadow rays)" if dominant == "nee" else "k_camera_samples (delta tracking)"
        traffic = None
        if dominant == "nee" and NEE_DRAM_BYTES_PER_LOOKUP is not None:
            traffic = lookups * NEE_DRAM_BYTES_PER_LOOKUP
        roof = {"kernel": name, "bound": "hbm", "achieved": achieved,
                "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                "traffic_note": "DRAM bytes per launch: bytes per lookup from a one-pass ncu capture of two "
                                "full-size launches, times this run's lookups"
                if traffic else None,
                "limiter": "issue-bound divergent control flow, not bandwidth (ncu, small case)"
                if dominant == "nee" else None,
                "algorithmic": "%d density lookups/frame x %d B" % (lookups, FETCH_BYTES),
                "peak_source": src}
    else:
        pk, psrc = tensor_peak(head)
        roof = field_roofline(stages["field"], qpf, args.steps, pk, psrc)
        roof["traffic"] = None

    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "%s field (f32 accumulation) / f32 tracking" % head,
        "data": "synthetic",
        "config": {"workload": "large neural render: %d^3 f16 turbulence, 8 point lights, %dx%d, %d spp, "
                               "%s 4x128 field, delta/ratio tracking" % (N_VOX, W_, H_, SPP, head),
                   "frames": "60-frame orbit", "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (2 GiB volume)", "majorant_brick": args.brick,
                   "majorant_brick_primary": args.brick_primary, "majorant_brick_shadow": args.brick_shadow,
                   "majorant_brick_path_tracer": args.brick_pt,
                   "voxel_layout": "linear" if args.linear_voxels else "4x4x4 tiles"},
        "queries_per_s": qpf * fps,
        "queries_per_frame": qpf,
        "lookups_per_frame": {"camera": fetches_per_frame - nee_fetches_per_frame, "nee": nee_fetches_per_frame},
        "stages_ms_per_frame": {k: v[0] / max(args.steps, 1) for k, v in stages.items() if v[1]},
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # kernels per frame: the pooled grids (camera rays; shadow rays when coarser than
        # the brick) and the walks' bordered copies of the distinct grids; camera samples;
        # scan (3) + placement + k_nee + k_nee_sum; field; compose
        "gpu_launches": grid_launches * cam_n + cam_n + 6 * nee_n + fld_n + cmp_n,
    }
    line["setup"] = setup
    if not args.no_extras:
        pk, psrc = tensor_peak(head)
        line["field_roofline"] = {head: field_roofline(stages["field"], qpf, args.steps, pk, psrc)}
        line["gemm_peaks"] = gp
        # the other precisions of the same trained field, same frames
        variants = {}
        for name, fv in fields.items():
            if name == head:
                continue
            r = render_frames(ctx, vol, lights, frame, fv, seed, args.steps, args.warmup, None, dev)
            fps_v = args.steps / (r["ms_total"] / 1e3)
            pk, psrc = tensor_peak(name)
            variants[name] = {"frames_per_s": fps_v, "queries_per_s": r["queries"] * fps_v,
                              "stages_ms_per_frame": {k: v[0] / args.steps for k, v in r["stages"].items() if v[1]},
                              "field_roofline": field_roofline(r["stages"]["field"], r["queries"], args.steps, pk,
                                                               psrc)}
            line["field_roofline"][name] = variants[name]["field_roofline"]
        line["variants"] = variants
        line["field_handoff"] = handoff_cost(ctx, qpf, ms_per_step, dev)
        line["field_library_reference"] = field_library_reference(qpf, fld_ms / max(args.steps, 1), dev)
        line["encoding_workload"] = encoding_workload(ctx, qpf, dev)
        if not args.no_equal_rmse:
            eq = equal_rmse(ctx, vol, vol_pt, lights, cams, fields, seed, args)
            line["equal_rmse"] = eq
            line["vs_path_tracer_equal_rmse"] = eq.get(head, {}).get("speedup")
            line["phase_sweep"] = phase_sweep(ctx, vol, lights, frame, field, seed, args)
        if not args.no_march:
            line["march_workload"] = march_workload(ctx, vol, lights, frame, field, seed, args)
        del cache
        if not args.no_mid:
            line["mid_workload"] = mid_workload(ctx, seed, args, gp)
        line["training_workload"] = training_workload(ctx, seed)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = cpu_baseline(vol_t.cpu().numpy(), tf_t.cpu().numpy(), lights, cams, seed,
                                                rows=args.cpu_rows, brick=args.brick,
                                                brick_primary=args.brick_primary, brick_shadow=args.brick_shadow,
                                                **oracle_field(seed, head))
            if not args.no_extras:
                line["cpu_baseline"]["plan"] = cpu_baseline_plan(vol_t.cpu().numpy(), tf_t.cpu().numpy(), lights,
                                                                 cams, seed, args, head,
                                                                 fixed_s=line["cpu_baseline"]["fixed_s"])
        except Exception as e:  # reported, not fatal
            line["cpu_baseline"] = {"error": repr(e)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def oracle_field(seed, prec=FIELD_PREC):
    """The CPU baseline's field: a Kaiming-initialised 4x128 field of the
    bench's shape in the headline precision (emulated in FP64; fp8 scales
    calibrated by the oracle), the same per-sample work as the trained field;
    nothing is taken from the GPU path."""
    from oracle import field as F
    code = {"f16": F.PREC_F16, "bf16": F.PREC_BF16, "fp8": F.PREC_FP8}[prec]
    desc = F.FieldDesc(FREQS, HIDDEN, N_HIDDEN, code, 5.0, seed + 3)
    w = F.init_weights(desc).astype(np.float64)
    scales = None
    if code == F.PREC_FP8:
        scales = F.fp8_calibrate(w, calibration_queries().numpy().astype(np.float64), desc)
    return dict(weights=w, desc=desc, scales=scales)


def march_workload(ctx, vol, lights, frame, field, seed, args):
    """The ray-marched variant of the neural renderer (step h = 0.5 voxel,
    inverse-CDF free flight, marched Beer-Lambert shadow rays, one fused
    camera-sample kernel, brick-majorant-0 segments skipped) on the same
    scene, camera and field at the full resolution: frames/s, samples/s,
    density lookups per frame and the camera kernel's algorithmic bandwidth."""
    import torch
    from paper_2304_07338_b300 import api
    cam, g = frame(0)
    out = torch.empty(cam.height, cam.width, 3, device=torch.device("cuda", ctx.device))
    api.render_neural(ctx, vol, lights, g, cam, SPP, 0.5, seed + 30, field, out)     # warm-up
    counters = torch.zeros(4, dtype=torch.int64, device=out.device)
    ctx.set_counters(counters)
    api.render_neural(ctx, vol, lights, g, cam, SPP, 0.5, seed + 31, field, out)
    ctx.sync()
    ctx.set_counters(None)
    lookups = int(counters[0].item())
    n = 2
    ctx.stage_times()
    ctx.stage_timing(True)
    s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s_ev.record(ctx.stream)
    for i in range(n):
        api.render_neural(ctx, vol, lights, g, cam, SPP, 0.5, seed + 31, field, out)
    e_ev.record(ctx.stream)
    torch.cuda.synchronize()
    ctx.stage_timing(False)
    st = ctx.stage_times()
    ms = s_ev.elapsed_time(e_ev) / n
    cam_ms = st["camera"][0] / max(st["camera"][1], 1)
    samples = cam.width * cam.height * SPP
    hbm = peaks()[0]
    bw = lookups * FETCH_BYTES / (cam_ms / 1e3) / 1e9
    return {"resolution": "%dx%d x %d spp, h = 0.5 voxel" % (cam.width, cam.height, SPP),
            "frames_per_s": 1e3 / ms, "ms_per_frame": ms, "samples_per_s": samples / (ms / 1e3),
            "lookups_per_frame": lookups, "stages_ms_per_frame": {k: v[0] / n for k, v in st.items() if v[1]},
            "roofline": {"kernel": "k_camera_samples_march (marched free flight and shadow rays)", "bound": "hbm",
                         "achieved": bw, "peak": hbm, "unit": "GB/s", "frac": bw / hbm,
                         "algorithmic": "%d lookups x %d B" % (lookups, FETCH_BYTES)}}


def phase_sweep(ctx, vol, lights, frame, field, seed, args, ref_spp=1024, width=480, height=270):
    """Phase-function awareness (Sec. 4.3.4): the field, trained on caches
    traced at G = {-0.75, 0, 0.75}, rendered at g inside and between the
    traced phases.  For every g, the image error (frame 0's camera, the
    equal-RMSE resolution) of the neural render, of the same render with
    the field off (direct light only) and of the path tracer at the neural
    render's spp, against a ref_spp path-traced reference at that g."""
    from paper_2304_07338_b300 import api, inputs as I
    cam, _ = frame(0)
    small = I.Camera(cam.eye, cam.at, cam.up, cam.fovy_deg, width, height)
    rows = []
    for i, g in enumerate((-0.9, -0.75, -0.5, -0.25, 0.0, 0.25, 0.5, 0.75, 0.9)):
        ref = api.render_pathtraced(ctx, vol, lights, g, small, ref_spp, 16, seed=seed + 60 + i)
        neural = api.render_neural(ctx, vol, lights, g, small, SPP, 0.0, seed + 8, field)
        direct = api.render_neural(ctx, vol, lights, g, small, SPP, 0.0, seed + 8, None)
        pt = api.render_pathtraced(ctx, vol, lights, g, small, SPP, 16, seed=seed + 9)
        ctx.sync()
        r_n, r_d, r_p = (api.image_rmse(ctx, x, ref) for x in (neural, direct, pt))
        rows.append({"g": g, "in_G": g in I.G_PAPER, "rmse_neural": r_n, "rmse_direct_only": r_d,
                     "rmse_pt_same_spp": r_p, "error_removed": 1.0 - r_n / r_d})
    return {"reference": "path tracer, %d spp per g, %dx%d, frame 0 camera" % (ref_spp, width, height),
            "spp": SPP, "by_g": rows}


def pooled_rmse(ctx, imgs, refs):
    """RMSE over several equally sized images (all pixels and channels)."""
    from paper_2304_07338_b300 import api
    return math.sqrt(sum(api.image_rmse(ctx, a, r) ** 2 for a, r in zip(imgs, refs)) / len(refs))


def equal_rmse(ctx, vol, vol_pt, lights, cams, fields, seed, args, frames=EQ_FRAMES, spps=(1, 2, 4, 8, 16, 32, 64)):
    """Equal-RMSE comparison with the plain path tracer (Sec. 4.3 compares the
    two renderers; the metric asks for equal image error), at the full
    resolution over `frames` of the orbit (their cameras and per-frame g):
      1. a path-traced reference of ref_spp samples per pixel per frame;
      2. each field's neural render (the benchmark's spp) and the direct-light
         render, their RMSE pooled over the frames;
      3. the path tracer at spps (vol_pt: the same voxels on its own majorant
         bricks), pooled RMSE, fitted as a / sqrt(spp) + b;
      4. per field, the spp the fit needs to reach the neural RMSE, rounded
         up, raised until the measured pooled RMSE of the path tracer at that
         spp is at or below the neural one;
      5. frames/s of both renderers over the same frames (one warm-up pass,
         then two timed passes, CUDA events); speedup = neural / path tracer."""
    import torch
    from paper_2304_07338_b300 import api, inputs as I
    dev = torch.device("cuda", ctx.device)
    fr = [(cams[f], I.frame_g(seed, f)) for f in frames]
    t0 = time.perf_counter()
    refs = [api.render_pathtraced(ctx, vol_pt, lights, g, cam, args.ref_spp, 16, seed=seed + 7 + k)
            for k, (cam, g) in enumerate(fr)]
    ctx.sync()
    t_ref = time.perf_counter() - t0
    out = {"frames": list(frames), "resolution": "%dx%d" % (W_, H_),
           "reference": "path tracer, %d spp per frame" % args.ref_spp, "reference_s": t_ref}

    def neural_imgs(field):
        return [api.render_neural(ctx, vol, lights, g, cam, SPP, 0.0, seed + 8 + k, field) for k, (cam, g) in
                enumerate(fr)]

    def pt_imgs(spp, sd):
        return [api.render_pathtraced(ctx, vol_pt, lights, g, cam, spp, 16, seed=sd + k) for k, (cam, g) in
                enumerate(fr)]

    def fps_of(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(2):
            fn()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        return 2 * len(fr) / (e0.elapsed_time(e1) / 1e3)

    out["rmse_direct_only"] = pooled_rmse(ctx, neural_imgs(None), refs)
    curve = {}
    for spp in spps:
        curve[spp] = pooled_rmse(ctx, pt_imgs(spp, seed + 9 * 1000), refs)
    X = np.stack([1.0 / np.sqrt(list(curve)), np.ones(len(curve))], 1)
    a, b = np.linalg.lstsq(X, np.array(list(curve.values())), rcond=None)[0]
    out["pt_rmse_by_spp"] = {str(k): v for k, v in curve.items()}
    out["pt_fit"] = {"a": float(a), "b": float(b)}
    for name, field in fields.items():
        r_n = pooled_rmse(ctx, neural_imgs(field), refs)
        res = {"rmse_neural": r_n}
        if r_n <= b:
            res["note"] = "neural RMSE below the path tracer's fitted floor"
            out[name] = res
            continue
        spp_fit = (a / (r_n - b)) ** 2
        need = max(1, int(math.ceil(spp_fit)))
        r_need = pooled_rmse(ctx, pt_imgs(need, seed + 10 * 1000), refs)
        tries = 0
        while r_need > r_n and tries < 8:
            need += max(1, need // 16)
            r_need = pooled_rmse(ctx, pt_imgs(need, seed + 10 * 1000), refs)
            tries += 1
        fps_n = fps_of(lambda: neural_imgs(field))
        fps_pt = fps_of(lambda: pt_imgs(need, seed + 11 * 1000))
        res.update({"pt_spp_fit": float(spp_fit), "pt_spp_at_equal_rmse": need, "pt_rmse_at_that_spp": r_need,
                    "neural_frames_per_s": fps_n, "pt_frames_per_s": fps_pt, "speedup": fps_n / fps_pt})
        out[name] = res
    del refs
    torch.cuda.empty_cache()
    return out


def mid_workload(ctx, seed, args, gp, n_frames=20, warmup=3, ref_spp=4096):
    """The mid render (512^3 u8 blurred noise, 256-node RGBA table, 4 point
    lights, 1024^2 x 4 spp, tracking, g per frame from U[-0.9, 0.9], an
    8-frame orbit): photon caches (G = {-0.75, 0, 0.75}, 2^22 photons per
    light per g), a 4x128 f16 field trained on tcgen05 with early stopping
    (train_render_field) and its fp8 copy; frames/s and field queries/s of both fields,
    their field rooflines, and the equal-RMSE comparison with the path
    tracer over two frames against ref_spp references."""
    import torch
    from paper_2304_07338_b300 import api, inputs as I
    dev = torch.device("cuda", ctx.device)
    sc = I.scene_mid(device="cuda")
    data = torch.from_numpy(np.ascontiguousarray(sc.volume.data)).to(dev)
    tf = torch.from_numpy(np.ascontiguousarray(sc.volume.tf, np.float32)).to(dev)
    vol = api.Volume(data, sc.volume.sigma_scale, sc.volume.albedo, tf, brick=16, brick_primary=64)
    vol.s.majorant = vol.majorant(ctx)
    vol.attach_brick_majorants(ctx)
    vol.attach_tiled(ctx)
    vol_pt = api.Volume(data, sc.volume.sigma_scale, sc.volume.albedo, tf, brick=32)
    vol_pt.s.majorant = vol.s.majorant
    vol_pt.attach_brick_majorants(ctx)
    vol_pt.tiled = vol.tiled
    vol_pt.s.tiled_dev = vol.s.tiled_dev
    cams = [I.orbit_camera(0.6 + 2 * math.pi * f / 8, 0.35, sc.camera.width, sc.camera.height) for f in range(8)]
    spp = sc.spp
    f16, cache, setup = train_render_field(ctx, vol, sc.lights, sc.g_set, seed + 60, 1 << 22)
    fp8 = api.Field(ctx, FREQS, HIDDEN, N_HIDDEN, "fp8", 5.0, seed=seed + 62)
    fp8.set_weights(f16.get_weights())
    fp8.calibrate_fp8(calibration_queries().to(dev))
    fields = {"f16": f16, "fp8": fp8}
    out = {"config": "512^3 u8 blurred noise, 256-node RGBA TF, 4 point lights, %dx%d, %d spp, 4x128 fields, "
                     "majorant bricks 16 (camera rays 64, path tracer 32)" % (sc.camera.width, sc.camera.height, spp),
           "setup": setup}
    global SPP, W_, H_
    saved = (SPP, W_, H_)
    SPP, W_, H_ = spp, sc.camera.width, sc.camera.height
    try:
        def frame(i):
            return cams[i % len(cams)], I.frame_g(seed + 1, i % len(cams))

        for name, fv in fields.items():
            r = render_frames(ctx, vol, sc.lights, frame, fv, seed, n_frames, warmup, None, dev)
            fps = n_frames / (r["ms_total"] / 1e3)
            key = {"f16": "f16", "fp8": "fp8_e4m3"}[name]
            pk = gp.get(key, {}).get("sustained_tflops")
            out[name] = {"frames_per_s": fps, "queries_per_frame": r["queries"], "queries_per_s": r["queries"] * fps,
                         "stages_ms_per_frame": {k: v[0] / n_frames for k, v in r["stages"].items() if v[1]},
                         "field_roofline": field_roofline(r["stages"]["field"], r["queries"], n_frames, pk,
                                                          "measured %s sustained" % key) if pk else None}
        saved_ref = args.ref_spp
        args.ref_spp = ref_spp
        out["equal_rmse"] = equal_rmse(ctx, vol, vol_pt, sc.lights, cams, fields, seed + 1, args, frames=(0, 4))
        args.ref_spp = saved_ref
    finally:
        SPP, W_, H_ = saved
    del cache, vol, vol_pt, data
    torch.cuda.empty_cache()
    return out


def training_workload(ctx, seed, steps=2000):
    """Field-training workload: data-source caches (128^3 fBm, 2 point
    lights, G = {-0.5, 0, 0.5}, 2^20 photons per light per g, 64^3 caches),
    4x64 bf16 field, 2^18 queries per step, 2000 steps, lr 1e-2 (tcgen05
    forward/backward)."""
    import torch
    from paper_2304_07338_b300 import api, inputs as I
    sc = I.scene_judge()
    vol = api.Volume.from_inputs(sc.volume)
    # photon caches: one warm-up build, then the best of three (each build
    # allocates its device buffers, whose first-touch cost varies)
    cache = api.build_photon_cache(ctx, vol, sc.lights, sc.g_set, 1 << 20, 16, 64, seed=seed + 20)
    times = []
    for _ in range(3):
        cache.free()
        ctx.sync()
        t0 = time.perf_counter()
        cache = api.build_photon_cache(ctx, vol, sc.lights, sc.g_set, 1 << 20, 16, 64, seed=seed + 20)
        ctx.sync()
        times.append(time.perf_counter() - t0)
    t_cache = min(times)
    fld = api.Field(ctx, 12, 64, 4, "bf16", 5.0, seed=seed + 21)
    fld.train(cache, steps=5, batch=1 << 18, lr=1e-2, seed=seed + 22)      # warm-up
    fld2 = api.Field(ctx, 12, 64, 4, "bf16", 5.0, seed=seed + 21)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = fld2.train(cache, steps=steps, batch=1 << 18, lr=1e-2, seed=seed + 22)
    dt = time.perf_counter() - t0
    flop = 3 * 2 * (144 * 64 + 3 * 64 * 64 + 3 * 64) * (1 << 18) * steps
    renders = judge_renders(ctx, sc, vol, fld2, seed)
    out = {"steps_per_s": steps / dt, "train_s": dt, "loss_first": float(loss[:5].mean()),
           "loss_last": float(loss[-20:].mean()), "photon_cache_s": t_cache, "photons_per_s": 6 * (1 << 20) / t_cache,
           "records": int(cache.n_records), "model_tflops": flop / dt / 1e12}
    # the render workloads' field width (4 x 128) on the same caches
    wide = {}
    for B in (1 << 16, 1 << 18):
        w = api.Field(ctx, 12, 128, 4, "f16", 5.0, seed=seed + 23)
        w.train(cache, steps=5, batch=B, lr=1e-2, seed=seed + 22)                 # warm-up
        w = api.Field(ctx, 12, 128, 4, "f16", 5.0, seed=seed + 23)
        n = 1000 if B == 1 << 16 else 300
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lw = w.train(cache, steps=n, batch=B, lr=1e-2, seed=seed + 22)
        dtw = time.perf_counter() - t0
        wide[str(B)] = {"steps": n, "steps_per_s": n / dtw, "model_tflops": field_flop(B) * 3 * n / dtw / 1e12,
                        "loss_first": float(lw[:5].mean()), "loss_last": float(lw[-20:].mean())}
    out["field_4x128_f16"] = wide
    out["renders"] = renders
    out["knn"] = knn_training(ctx, cache, seed, steps, vol_res=sc.volume.data.shape[0])
    out["knn_saturated"] = knn_saturated(ctx, seed)
    out["hashgrid"] = hashgrid_training(ctx, cache, seed, steps)
    return out


def field_training_only(ctx, seed, width, steps, batch=1 << 18):
    """f16 field training alone (4 hidden layers of `width`, data-source
    caches, `batch` queries per step): steps/s and model TFLOP/s."""
    import torch
    from paper_2304_07338_b300 import api, inputs as I
    sc = I.scene_judge()
    vol = api.Volume.from_inputs(sc.volume)
    cache = api.build_photon_cache(ctx, vol, sc.lights, sc.g_set, 1 << 20, 16, 64, seed=seed + 20)
    f = api.Field(ctx, 12, width, 4, "f16", 5.0, seed=seed + 23)
    f.train(cache, steps=3, batch=batch, lr=1e-2, seed=seed + 22)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = f.train(cache, steps=steps, batch=batch, lr=1e-2, seed=seed + 22)
    dt = time.perf_counter() - t0
    fl = 3 * 2 * (144 * width + 3 * width * width + 3 * width) * batch * steps
    return {"width": width, "batch": batch, "steps": steps, "steps_per_s": steps / dt, "model_tflops": fl / dt / 1e12,
            "loss_last": float(loss[-5:].mean())}


# The paper's encoding (Sec. 3.4): 16 levels of 8 features, x2 per level,
# 2^19 table entries; base resolution 16 cells.
HASH = dict(encoding="hashgrid", hash_levels=16, hash_features=8, hash_log2_size=19, hash_base_res=16,
            hash_scale=2.0)


def hashgrid_training(ctx, cache, seed, steps, batch=1 << 16):
    """Convergence of the hash-grid field against the frequency encoding on
    the same caches and cell targets: 4x64 bf16 MLPs, 2^16 queries per step
    (the paper's batch), `steps` steps each.  The training loss of every step
    is taken on a fresh batch, so its running mean is a held-out estimate;
    reported at a few steps, with the step (and time) at which the hash-grid
    field first matches the frequency field's final loss, and both fields'
    loss on one held-out batch."""
    import torch
    from paper_2304_07338_b300 import api
    qv = cache.sample_queries(1 << 16, step=0, seed=seed + 41)
    _, yv = cache.estimate_targets(qv)
    res = {"batch": batch, "steps": steps, "config": dict(HASH, mlp="4x64 bf16")}
    curves = {}
    for name, kw in (("frequency", {}), ("hashgrid", HASH)):
        w = api.Field(ctx, 12, 64, 4, "bf16", 5.0, seed=seed + 21, **kw)
        w.train(cache, steps=3, batch=batch, lr=1e-2, seed=seed + 42)            # warm-up
        del w
        fld = api.Field(ctx, 12, 64, 4, "bf16", 5.0, seed=seed + 21, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = fld.train(cache, steps=steps, batch=batch, lr=1e-2, seed=seed + 42)
        dt = time.perf_counter() - t0
        yh = fld.forward(qv)
        val = float(torch.mean((yh - yv) ** 2 / (yv ** 2 + 0.01)))
        run = np.convolve(loss, np.ones(20) / 20, mode="valid")         # mean of steps s-19 .. s
        curves[name] = run
        res[name] = {"steps_per_s": steps / dt, "train_s": dt, "params": int(fld.n_params), "val_loss": val,
                     "loss_at": {str(s_): float(run[s_ - 20]) for s_ in (100, 250, 500, 1000, steps) if s_ <= steps}}
        del fld
    target = curves["frequency"][-1]
    hit = np.nonzero(curves["hashgrid"] <= target)[0]
    if hit.size:
        s_hit = int(hit[0]) + 20
        res["hashgrid_steps_to_frequency_final_loss"] = s_hit
        res["hashgrid_time_to_frequency_final_loss_s"] = s_hit / res["hashgrid"]["steps_per_s"]
    res["frequency_time_s"] = res["frequency"]["train_s"]
    return res


def judge_renders(ctx, sc, vol, fld, seed, ref_spp=1024):
    """The data-source scene (256^2, g = 0) with the field just trained:
    error against a ref_spp path-traced reference and frames/s of the
    ray-marching renderer with the field at every step (Sec. 3.6; 1 spp,
    0.5-voxel steps), the neural path tracer (16 spp, tracking), both without
    the field, and the path tracer at 16 spp."""
    import torch
    from paper_2304_07338_b300 import api
    cam, g = sc.camera, 0.0
    ref = api.render_pathtraced(ctx, vol, sc.lights, g, cam, ref_spp, 16, seed=seed + 50)
    ctx.sync()

    def timed(fn, n=5):
        img = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(n):
            fn()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        return img, n / (e0.elapsed_time(e1) / 1e3)

    runs = {
        "raymarch_field": lambda: api.render_raymarched(ctx, vol, sc.lights, g, cam, 1, 0.5, seed + 51, fld),
        "raymarch_direct_only": lambda: api.render_raymarched(ctx, vol, sc.lights, g, cam, 1, 0.5, seed + 51),
        "neural_pt_16spp": lambda: api.render_neural(ctx, vol, sc.lights, g, cam, 16, 0.0, seed + 52, fld),
        "neural_pt_direct_only_16spp": lambda: api.render_neural(ctx, vol, sc.lights, g, cam, 16, 0.0, seed + 52),
        "path_tracer_16spp": lambda: api.render_pathtraced(ctx, vol, sc.lights, g, cam, 16, 16, seed=seed + 53),
    }
    out = {"reference": "path tracer, %d spp, %dx%d, g = 0" % (ref_spp, cam.width, cam.height)}
    for name, fn in runs.items():
        img, fps = timed(fn)
        out[name] = {"rmse": api.image_rmse(ctx, img, ref), "frames_per_s": fps}
    return out


# Staggered KNN schedule (Sec. 3.5.2, Table 1, the 6M-photon row: this
# workload traces 6.3M photons): stage starts at 0, 37, 64 and 91 % of the
# steps, radius caps 0.25, 0.5, 1.5 and 3.0 voxels.
KNN_K = 1024
KNN_STAGES = [(0.0, 0.25), (0.37, 0.5), (0.64, 1.5), (0.91, 3.0)]


def knn_training(ctx, cache, seed, steps, vol_res):
    """Training with the phase-selective KNN targets (K = 1024): the staggered
    radius schedule against the fixed final radius (the paper's naive
    training), the KNN kernel's time per 2^18-query batch at every radius and
    at a saturating 8-voxel radius, and both fields' loss on one held-out
    batch whose targets use the final radius."""
    import torch
    from paper_2304_07338_b300 import api
    B = 1 << 18
    vox = 1.0 / vol_res
    sched = [(b, r * vox) for b, r in KNN_STAGES]
    r_final = sched[-1][1]
    res = {"K": KNN_K, "schedule_voxels": KNN_STAGES, "batch": B, "steps": steps}
    # kernel time per batch and records used per query, at each radius
    q = cache.sample_queries(B, step=0, seed=seed + 30)
    per = {}
    for r_vox in sorted({r for _, r in KNN_STAGES} | {8.0}):
        cache.estimate_targets_knn(q, KNN_K, r_vox * vox)          # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        n_rep = 5
        for _ in range(n_rep):
            _, _, k, _ = cache.estimate_targets_knn(q, KNN_K, r_vox * vox)
        e1.record()
        torch.cuda.synchronize()
        kf = k.float()
        per[str(r_vox)] = {"ms": e0.elapsed_time(e1) / n_rep, "mean_k": float(kf.mean()),
                           "saturated_frac": float((k >= KNN_K).float().mean())}
    res["batch_ms_by_radius_voxels"] = per
    # held-out batch with final-radius targets
    qv = cache.sample_queries(1 << 16, step=0, seed=seed + 31)
    _, yv, _, _ = cache.estimate_targets_knn(qv, KNN_K, r_final)

    def val_loss(fld):
        y = fld.forward(qv)
        return float(torch.mean((y - yv) ** 2 / (yv ** 2 + 0.01)))

    for name, sch in (("staggered", sched), ("fixed", [(0.0, r_final)])):
        w = api.Field(ctx, 12, 64, 4, "bf16", 5.0, seed=seed + 21)
        w.train(cache, steps=5, batch=B, lr=1e-2, seed=seed + 22, knn_k=KNN_K, knn_schedule=sch)      # warm-up
        fld = api.Field(ctx, 12, 64, 4, "bf16", 5.0, seed=seed + 21)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = fld.train(cache, steps=steps, batch=B, lr=1e-2, seed=seed + 22, knn_k=KNN_K, knn_schedule=sch)
        dt = time.perf_counter() - t0
        res[name] = {"steps_per_s": steps / dt, "train_s": dt, "loss_last": float(loss[-20:].mean()),
                     "val_loss_final_radius": val_loss(fld)}
    res["staggered_speedup"] = res["fixed"]["train_s"] / res["staggered"]["train_s"]
    return res


# Table 1's 1M-photon row: radius caps 0.25, 0.5, 2.5 and 5.0 voxels.
KNN_STAGES_1M = [(0.0, 0.25), (0.37, 0.5), (0.64, 2.5), (0.91, 5.0)]


def knn_saturated(ctx, seed, photons=1 << 24, batch=1 << 16, steps_list=(250, 500, 1000, 2000)):
    """The staggered KNN schedule where it is meant to act (Sec. 3.5.2: the
    larger the radius, the more likely k = K, and the costlier the search):
    the data-source scene's photon map at 2^24 photons per light per g, dense
    enough that K = 1024 saturates at the final cap of Table 1's 1M row
    (0.25 / 0.5 / 2.5 / 5 voxels; the 6M and 12M rows' caps would not
    saturate on this 128^3 volume).  Both schedules (staggered, and the
    fixed final cap of the paper's naive training) train a 4x64 bf16 field
    for each step count in steps_list on 2^16-query batches; every run's
    held-out loss is taken against final-cap targets; the time each schedule
    needs to reach the lowest held-out loss both reach is interpolated in
    log time between runs, and their ratio is the speed-up."""
    import torch
    from paper_2304_07338_b300 import api, inputs as I
    sc = I.scene_judge()
    vol = api.Volume.from_inputs(sc.volume)
    cache = api.build_photon_cache(ctx, vol, sc.lights, sc.g_set, photons, 16, 64, seed=seed + 24)
    vox = 1.0 / sc.volume.data.shape[0]
    sched = [(b, r * vox) for b, r in KNN_STAGES_1M]
    r_final = sched[-1][1]
    res = {"K": KNN_K, "photons_per_light_per_g": photons, "records": int(cache.n_records),
           "schedule_voxels": KNN_STAGES_1M, "batch": batch, "steps": list(steps_list)}
    q = cache.sample_queries(batch, step=0, seed=seed + 30)
    per = {}
    for _, r_vox in KNN_STAGES_1M:
        cache.estimate_targets_knn(q, KNN_K, r_vox * vox)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            _, _, k, _ = cache.estimate_targets_knn(q, KNN_K, r_vox * vox)
        e1.record()
        torch.cuda.synchronize()
        per[str(r_vox)] = {"ms": e0.elapsed_time(e1) / 5, "mean_k": float(k.float().mean()),
                           "saturated_frac": float((k >= KNN_K).float().mean())}
    res["batch_ms_by_radius_voxels"] = per
    qv = cache.sample_queries(1 << 16, step=0, seed=seed + 31)
    _, yv, _, _ = cache.estimate_targets_knn(qv, KNN_K, r_final)

    def val_loss(fld):
        y = fld.forward(qv)
        return float(torch.mean((y - yv) ** 2 / (yv ** 2 + 0.01)))

    runs = {}
    for name, sch in (("staggered", sched), ("fixed", [(0.0, r_final)])):
        w = api.Field(ctx, 12, 64, 4, "bf16", 5.0, seed=seed + 21)
        w.train(cache, steps=5, batch=batch, lr=1e-2, seed=seed + 22, knn_k=KNN_K, knn_schedule=sch)    # warm-up
        pts = []
        for n in steps_list:
            fld = api.Field(ctx, 12, 64, 4, "bf16", 5.0, seed=seed + 21)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fld.train(cache, steps=n, batch=batch, lr=1e-2, seed=seed + 22, knn_k=KNN_K, knn_schedule=sch)
            dt = time.perf_counter() - t0
            pts.append({"steps": n, "train_s": dt, "val_loss": val_loss(fld)})
        runs[name] = pts
    res["runs"] = runs
    # the lowest held-out loss both schedules reach within the step counts
    target = max(min(p["val_loss"] for p in runs["fixed"]), min(p["val_loss"] for p in runs["staggered"]))

    def time_to(pts, target):
        # first run at or below the target; log-time interpolation from the previous run
        for i, p in enumerate(pts):
            if p["val_loss"] <= target:
                if i == 0:
                    return p["train_s"]
                a, b = pts[i - 1], p
                f = (a["val_loss"] - target) / max(a["val_loss"] - b["val_loss"], 1e-30)
                return math.exp(math.log(a["train_s"]) + f * (math.log(b["train_s"]) - math.log(a["train_s"])))
        return None

    t_fix, t_stag = time_to(runs["fixed"], target), time_to(runs["staggered"], target)
    res["target_val_loss"] = target
    res["time_to_target_s"] = {"fixed": t_fix, "staggered": t_stag}
    res["staggered_speedup_to_equal_loss"] = t_fix / t_stag if (t_fix and t_stag) else None
    cache.free()
    return res


def calibration_queries():
    """4096 fp8 calibration queries: uniform positions and angles, g in [-0.9, 0.9]."""
    import torch
    g = torch.Generator().manual_seed(0)
    cal = torch.rand(4096, 6, generator=g)
    cal[:, 5] = cal[:, 5] * 1.8 - 0.9
    return cal.contiguous()


def run_reference(args, dev, seed):
    """The oracle as the reference arm: each step is one full image row (at
    full spp) of the same workload on the host cores, the steps' rows
    rendered by one oracle call; frames/s from the oracle's fixed cost per
    call plus the per-pixel time over a frame."""
    import torch
    vol_t, tf_t, lights, cams = setup_scene(dev)
    vol_h, tf_h = vol_t.cpu().numpy(), tf_t.cpu().numpy()
    # a 4x128 field of the bench's shape and headline precision (Kaiming
    # init): the same per-sample work as the trained field
    fld = oracle_field(seed, FIELD_PREC)
    # one row of the frame per step, all steps' rows in one oracle call (each
    # call pays the oracle's fixed cost, about 9 s at 1024^3, once)
    r = cpu_baseline(vol_h, tf_h, lights, cams, seed, rows=max(1, min(args.steps, H_ // 2)), brick=args.brick,
                     brick_primary=args.brick_primary, brick_shadow=args.brick_shadow, **fld)
    fps = r["value"]
    cb = {"value": fps, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": "one full row per step from the middle of the frame at full spp (4x128 %s field, Kaiming "
                    "init), the oracle's fixed cost per call counted once per frame, the rest scaled to a frame: "
                    % FIELD_PREC + r["sample"]}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / fps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32 oracle",
                      "data": "synthetic",
                      "config": {"workload": "large neural render: 1024^3 f16 turbulence, 8 point lights, "
                                             "1920x1080, 16 spp, %s 4x128 field, delta/ratio tracking" % FIELD_PREC},
                      "cpu_baseline": cb,
                      "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


if __name__ == "__main__":
    main()

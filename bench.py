#!/usr/bin/env python3
"""Benchmark of the W-projection hot path on one B300 (or N independent replicas).

One step = one pass of the whole path over the workload, all on one CUDA stream:
  make_wkernels (float64 kernel tables) -> grid (float64 coordinates, bin sort, gridding)
  -> degrid (coordinates, bin sort, degridding of the same grid) -> fft_to_image (cuFFT +
  taper-corrected image epilogue).
Metric: gridded visibilities per second for the whole step (the tap-update rate and the
per-phase rates are reported beside it). The workload ("fp32"): 128 antennas in a 5 km
disk, 4 channels 1.0-1.4 GHz, 480 samples over 8 h, 15.6M samples gridded with their
Hermitian conjugates = 31.2M gridded visibilities, 2048^2 grid at 1", 32 w-planes,
support 8-16, oversampling 8; synthetic, seeded, generated on the GPU (inputs 0.4 GB,
larger than the 126 MB L2, so no L2 flush between steps).

--impl reference runs the float64 CPU oracle (the reference arm here) on a bounded sample
of the same workload on the host cores.

Multi-GPU (torchrun): every rank runs its own independent imaging job of the same size
(independent problems shard with no collective); value = all ranks' visibilities / the
max over ranks of the timed region; scaling "weak".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "gridded visibilities/s (whole W-projection step: kernels, coordinates+sort, grid, degrid, FFT+taper)"
WORKLOADS = {
    "fp32": ("fp32: 128 ants / 5 km, 4 ch 1.0-1.4 GHz, 480 samples / 8 h -> 15.6M samples + Hermitian "
             "conjugates = 31.2M gridded vis; 2048^2 @ 1\", 32 w-planes, support 8-16, os 8"),
    "mixed": ("mixed: 256 ants / 10 km, 16 ch 1.0-1.4 GHz, 720 samples / 8 h -> 376M vis; 4096^2 @ 0.5\", "
              "64 w-planes, support 8-32, os 8"),
    "diff": "diff: 64 ants / 5 km, 1 ch 1.4 GHz, 496 samples / 8 h -> 1.0M vis; 2048^2 @ 1\", 32 w-planes, support 12, os 8",
}


def workload_name(config: str) -> str:
    return WORKLOADS.get(config, config)


def measured_peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def fp32_peak_tflops(nsm=148, mhz=2032.0):
    """FP32 FMA peak from unit counts: SMs x 128 lanes x 2 flop x max SM clock."""
    return nsm * 128 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": float(max(power)) if power else None}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def run_gpu(args):
    import torch
    import synth
    import paper_1905_03213_b300 as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    cfg = synth.config(args.config)
    cfg.seed += 97 * rank                          # an independent job per rank
    ob = synth.observe(cfg, device=f"cuda:{local}", rows=args.rows or None)
    uvw, vis, wt = ob.uvw.contiguous(), ob.vis.contiguous(), ob.weight.contiguous()
    freq = torch.as_tensor(ob.freqs, dtype=torch.float64, device=dev)
    tile = tuple(int(x) for x in args.tile.split("x")) if args.tile else (0, 0)
    n = cfg.n
    grid = torch.empty((n, n), dtype=torch.complex64, device=dev)
    image = torch.empty((n, n), dtype=torch.float32, device=dev)
    pred = torch.empty_like(vis)
    sum_w = torch.zeros(1, dtype=torch.float64, device=dev)
    ndrop = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def make(table):
        return W.WProj(n=cfg.n, cell=cfg.cell, n_w=cfg.n_w, w_max=ob.w_max, support_min=cfg.s_min,
                       support_max=cfg.s_max, oversample=cfg.oversample, table=table, tile=tile, device=local,
                       units_per_cta=args.units)

    def stepper(wp, compensated=False):
        def step():
            wp.make_wkernels()
            wp.grid(uvw, freq, vis, wt, grid=grid, sum_w=sum_w, n_dropped=ndrop,
                    hermitian_pairs=cfg.hermitian_pairs, keep_binning=True, compensated=compensated)
            wp.degrid_last(grid, vis_out=pred)
            wp.fft_to_image(grid, sum_w, image=image)
        return step

    def timed_steps(wp, steps, warmup, clocks=None, compensated=False):
        step = stepper(wp, compensated)
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wp.profile(True)
        wp.profile_read()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with (clocks if clocks is not None else _NoClock()):
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = e0.elapsed_time(e1) / steps
        phase_ms, phase_cnt, launches = wp.profile_read()
        wp.profile(False)
        return ms, {k: phase_ms[k] / max(1, phase_cnt[k]) for k in phase_ms}, launches

    wp = make(args.table)
    stepper(wp)()                                   # untimed first step
    torch.cuda.synchronize()
    # the work counts (kept visibilities and taps) from the library's own coordinates
    sup, _ = wp.plane_info()
    sup_t = torch.as_tensor(sup, device=dev).long()
    crd = wp.coords(uvw, freq, hermitian_pairs=cfg.hermitian_pairs)
    keep = crd[:, 4].bool()
    kept = int(keep.sum().item())
    taps_grid = int((sup_t[crd[:, 2][keep].long()] ** 2).sum().item())
    crd = wp.coords(uvw, freq, hermitian_pairs=False)
    keep = crd[:, 4].bool()
    kept_degrid = int(keep.sum().item())
    taps_degrid = int((sup_t[crd[:, 2][keep].long()] ** 2).sum().item())
    del crd, keep

    clk = ClockSampler(local)
    ms_step, phases, launches = timed_steps(wp, args.steps, args.warmup, clocks=clk)
    if world > 1:
        t = torch.tensor([ms_step], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step = float(t.item())

    e2e = None if args.no_e2e else run_e2e(wp, uvw, vis, wt, freq, grid, sum_w, ndrop, pred, image, cfg, args,
                                           stream, kept * world)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return None

    grid_ms, degrid_ms = phases["grid"], phases["degrid"]
    peaks = measured_peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_fp32 = fp32_peak_tflops(nsm)
    achieved = 8.0 * taps_grid / (grid_ms * 1e-3) / 1e12
    # algorithmic bytes of one gridding launch: every 16-byte record read once, the grid's
    # 8-byte cells read and written once, the plane tables read once
    tab_bytes = sum((int(s) * cfg.oversample) ** 2 * (8 if args.table == "f32" else 4) for s in sup)
    alg_bytes = kept * 16 + 2 * 8 * n * n + tab_bytes
    probe = {}
    if not args.no_probe:
        tf2, ms2 = W.probe_fp32_fma(local, packed=True, iters=100_000, reps=5)
        tf1, _ = W.probe_fp32_fma(local, packed=False, iters=100_000, reps=5)
        probe = {"packed_fma2_tflops": tf2, "scalar_fma_tflops": tf1, "frac_of_measured_fma2": achieved / tf2,
                 "note": "project-written FMA probe (wp_probe_fp32_fma), 16 independent chains per thread, "
                         f"{ms2:.1f} ms per launch"}
    out = {
        "metric": METRIC,
        "value": kept * world / (ms_step * 1e-3),
        "unit": "visibilities/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.table == "f32" else f"f32 ({args.table} tables)",
        "data": "synthetic (seeded array/uvw/sky generators; values from 200 point sources + noise)",
        "config": {"workload": workload_name(args.config) + (f"; first {args.rows} rows only" if args.rows else ""),
                   "table": args.table, "tile": args.tile or "default",
                   "units_per_cta": args.units or "default", "gridded_visibilities": kept,
                   "degridded_visibilities": kept_degrid,
                   "l2": "inputs larger than L2 (0.4 GB fp32, 4.5 GB mixed); no flush",
                   "degrid": "wp_degrid_last: degrids the gridded samples with the gridding call's binning",
                   "parallelism": f"{world} independent job(s)"},
        "taps_per_s": (taps_grid + taps_degrid) * world / (ms_step * 1e-3),
        "phases_ms": phases,
        "grid_kernel": {"ms": grid_ms, "vis_per_s": kept / (grid_ms * 1e-3), "taps_per_s": taps_grid / (grid_ms * 1e-3),
                        "taps": taps_grid},
        "degrid_kernel": {"ms": degrid_ms, "vis_per_s": kept_degrid / (degrid_ms * 1e-3),
                          "taps_per_s": taps_degrid / (degrid_ms * 1e-3), "taps": taps_degrid,
                          "frac_of_fp32_peak": 8.0 * taps_degrid / (degrid_ms * 1e-3) / 1e12 / peak_fp32},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                     "frac": achieved / peak_fp32, "traffic": profiled_traffic(args.table, args.rows, args.config),
                     "traffic_note": f"DRAM bytes per launch from the ncu summary in {GRID_PROFILE}",
                     "kernel": f"grid kernel <{args.table}> (warp-synchronous register-accumulating gridding scatter, 8 flop per tap)",
                     "peak_note": f"FP32 FMA peak derived from unit counts ({nsm} SMs x 128 lanes x 2 x 2.032 GHz)",
                     "peak_measured": probe,
                     "hbm": {"algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / (grid_ms * 1e-3) / 1e9,
                             "peak_gbs": peaks.get("hbm_gbs"), "peak_note": "of measured"}},
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        rows = cpu_sample_rows(cfg, args.cpu_vis)
        sp = cpu_sample_from_device(cfg, rows, uvw, freq, vis, wt, ob.w_max)
        cb, res = cpu_baseline(args, sp, keep=True)
        cb["single_thread"] = single_thread_grid_rate(sp, res)
        out["cpu_baseline"] = cb
        out["error"] = {args.table: error_figures(wp, sp, res)}
        if args.variants:
            out["mixed_vs_fp32"] = table_variants(args, make, timed_steps, sp, res, kept, taps_grid, grid_ms,
                                                  ms_step, out["error"])
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


class _NoClock:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


def table_variants(args, make, timed_steps, sp, res, kept, taps, grid_ms, ms_step, errors):
    """The same step with each kernel-table precision, on the same workload: throughput and
    the error against the float64 oracle on the sample, side by side."""
    rows = {args.table: {"ms_per_step": ms_step, "grid_kernel_ms": grid_ms, "vis_per_s": kept / (ms_step * 1e-3),
                         "grid_taps_per_s": taps / (grid_ms * 1e-3), "error": errors[args.table]}}
    for name in ("f32", "f16", "bf16", "f32_compensated"):
        if name in rows:
            continue
        table, comp = (name, False) if name != "f32_compensated" else ("f32", True)
        wp = make(table)
        ms, ph, _ = timed_steps(wp, args.steps, args.warmup, compensated=comp)
        rows[name] = {"ms_per_step": ms, "grid_kernel_ms": ph["grid"], "vis_per_s": kept / (ms * 1e-3),
                      "grid_taps_per_s": taps / (ph["grid"] * 1e-3),
                      "error": error_figures(wp, sp, res, compensated=comp)}
        wp.close()
    base = rows["f32"]
    for name, r in rows.items():
        r["step_speedup_vs_f32"] = base["ms_per_step"] / r["ms_per_step"]
        r["grid_speedup_vs_f32"] = base["grid_kernel_ms"] / r["grid_kernel_ms"]
        tol = 1e-5 if name.startswith("f32") else 1e-3
        r["tolerance"] = tol
        r["meets_tolerance"] = all(r["error"][k]["max"] <= tol for k in ("image_uncorrected", "image_corrected_inner"))
        r["degrid_within_tolerance"] = r["error"]["degrid"]["max"] <= tol
    return rows


def run_fp32peak(args):
    """The FP32 FMA roofline denominator, measured by the project's probe kernel."""
    import torch
    import paper_1905_03213_b300 as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    W.probe_fp32_fma(0, packed=True, iters=20_000, reps=2)
    with ClockSampler(0) as clk:
        tf2, ms2 = W.probe_fp32_fma(0, packed=True, iters=400_000, reps=args.steps)
        tf1, ms1 = W.probe_fp32_fma(0, packed=False, iters=400_000, reps=args.steps)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    return {"metric": "FP32 FMA throughput (roofline denominator of the gridding scatter)", "value": tf2,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": ms2,
            "higher_is_better": True, "dtype": "f32", "data": "none (register-only FMA chains)",
            "config": {"workload": "fp32peak: every SM at full occupancy, 16 independent FMA chains per thread"},
            "packed_fma2_tflops": tf2, "scalar_fma_tflops": tf1, "scalar_ms_per_launch": ms1,
            "unit_count_peak_tflops": fp32_peak_tflops(nsm), "frac_of_unit_count_peak": tf2 / fp32_peak_tflops(nsm),
            "clocks": clk.summary()}


ROOT = os.path.dirname(os.path.abspath(__file__))
GRID_KERNEL_SOURCES = ("paper_1905_03213_b300/csrc/grid2.cu", "paper_1905_03213_b300/csrc/warp_common.cuh")
GRID_PROFILE = "profiles/k_grid_v2_fp32_workload.md"


def profiled_traffic(table: str, rows: int, config: str = "fp32"):
    """DRAM bytes of one gridding launch on the full fp32 workload, as the committed ncu summary
    states them, or None when the summary was taken on other kernel sources (or another case)."""
    if rows or table != "f32" or config != "fp32":
        return None
    h = hashlib.sha256()
    try:
        for p in GRID_KERNEL_SOURCES:
            with open(os.path.join(ROOT, p), "rb") as f:
                h.update(f.read())
        text = open(os.path.join(ROOT, GRID_PROFILE)).read()
    except OSError:
        return None
    fields = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line and line.split(": ", 1)[0].isascii())
    if fields.get("kernel_source_sha256[:16] (grid2.cu + warp_common.cuh)", "").strip() != h.hexdigest()[:16]:
        return None
    try:
        return int(fields["traffic_bytes_per_launch[f32]"].strip())
    except (KeyError, ValueError):
        return None


def run_e2e(wp, uvw, vis, wt, freq, grid, sum_w, ndrop, pred, image, cfg, args, stream, units):
    """The same step through the public API from pinned host buffers, every step's copies inside
    the timing: each step copies its inputs (uvw, freq, vis, weight) host -> device and reads its
    image back device -> host. Measured two ways: serially (copy, compute, read back, on one
    stream), and as a stream pipeline with two device input sets, where step i + 1's copies (on a
    copy stream) run while step i computes and step i's image is read back on a third stream."""
    import torch
    n = cfg.n
    dev = uvw.device
    h_uvw, h_vis, h_wt = uvw.cpu().pin_memory(), vis.cpu().pin_memory(), wt.cpu().pin_memory()
    h_freq = freq.cpu().pin_memory()
    h_img = [torch.empty((n, n), dtype=torch.float32).pin_memory() for _ in range(2)]
    sets = [(torch.empty_like(uvw), torch.empty_like(freq), torch.empty_like(vis), torch.empty_like(wt))
            for _ in range(2)]
    imgs = [image, torch.empty_like(image)]

    def compute(x, img):
        d_uvw, d_freq, d_vis, d_wt = x
        wp.make_wkernels()
        wp.grid(d_uvw, d_freq, d_vis, d_wt, grid=grid, sum_w=sum_w, n_dropped=ndrop,
                hermitian_pairs=cfg.hermitian_pairs, keep_binning=True)
        wp.degrid_last(grid, vis_out=pred)
        wp.fft_to_image(grid, sum_w, image=img)

    def copy_in(x):
        for d, h in zip(x, (h_uvw, h_freq, h_vis, h_wt)):
            d.copy_(h, non_blocking=True)

    # serial: one stream, copy in, compute, read back
    def serial_step():
        copy_in(sets[0])
        compute(sets[0], imgs[0])
        h_img[0].copy_(imgs[0], non_blocking=True)

    steps = max(6, args.steps // 2)                 # enough steps for the pipeline to fill and drain
    for _ in range(2):
        serial_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        serial_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_serial = e0.elapsed_time(e1) / steps

    # pipelined: copy stream, compute stream (the current one), read-back stream
    cs, rs = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]       # compute done with input set / image x
    read = [torch.cuda.Event() for _ in range(2)]       # image x read back
    for ev in used + read:
        ev.record(stream)

    def pipelined_step(i):
        x = i % 2
        cs.wait_event(used[x])                          # step i - 2 no longer reads set x
        with torch.cuda.stream(cs):
            copy_in(sets[x])
        copied[x].record(cs)
        stream.wait_event(copied[x])
        stream.wait_event(read[x])                      # step i - 2's image x has been read back
        compute(sets[x], imgs[x])
        used[x].record(stream)
        rs.wait_event(used[x])
        with torch.cuda.stream(rs):
            h_img[x].copy_(imgs[x], non_blocking=True)
        read[x].record(rs)

    for i in range(2):
        pipelined_step(i)
    torch.cuda.synchronize()
    e0.record(stream)
    cs.wait_event(e0)
    for i in range(steps):
        pipelined_step(i)
    stream.wait_event(read[0])
    stream.wait_event(read[1])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    h2d = h_uvw.numel() * 8 + h_vis.numel() * 8 + h_wt.numel() * 4 + h_freq.numel() * 8
    return {"value": units / (ms * 1e-3), "unit": "visibilities/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": h_img[0].numel() * 4, "ms_per_step": ms,
            "mode": "pipelined: step i + 1's host-to-device copies overlap step i's compute (two device "
                    "input sets, copy and read-back streams); every step's copies are inside the timing",
            "serial": {"value": units / (ms_serial * 1e-3), "ms_per_step": ms_serial,
                       "mode": "copy in, compute, read back, one stream"}}


def cpu_sample_rows(cfg, target_vis):
    return max(1, min(cfg.n_rows, target_vis // len(cfg.freqs)))


class CpuSample:
    """The oracle's bounded sample of the workload: its first `rows` rows (the first time
    samples of every baseline) as host arrays, with the planes of the full observation."""

    def __init__(self, cfg, rows, uvw, freqs, vis, weight, w_max):
        import oracle
        self.cfg, self.rows = cfg, rows
        self.uvw, self.freqs, self.vis, self.weight, self.w_max = uvw, freqs, vis, weight, w_max
        self.prm = oracle.Params(cfg.n, cfg.cell, cfg.n_w, w_max, cfg.s_min, cfg.s_max, cfg.oversample)


def cpu_sample_from_host(cfg, rows):
    """Sample made on the host by the numpy generators (the reference arm, no GPU)."""
    import synth
    ob = synth.observe(cfg, rows=rows)
    # w_max of the full observation, so the planes match the GPU run
    enu = synth.antenna_enu(cfg.n_ant, cfg.radius_m, cfg.height_m, np.random.default_rng(cfg.seed))
    uvw_all = synth.uvw_metres(enu, synth.SITE_LAT, cfg.dec, synth.hour_angles(cfg.n_time, cfg.duration_h))
    w_max = float(np.max(np.abs(uvw_all[:, 2])) * np.max(cfg.freqs) / synth.C_LIGHT)
    return CpuSample(cfg, rows, ob.uvw, np.asarray(ob.freqs), ob.vis, ob.weight, w_max)


def cpu_sample_from_device(cfg, rows, uvw, freq, vis, wt, w_max):
    """Sample copied from the GPU run's own inputs (the same stored values on both sides)."""
    return CpuSample(cfg, rows, uvw[:rows].cpu().numpy(), freq.cpu().numpy(), vis[:rows].cpu().numpy(),
                     wt[:rows].cpu().numpy(), w_max)


def host_threads():
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return cores, max(1, min(cores, 32))    # each OpenMP private float64 grid is 67 MB at 2048^2


def oracle_step(sp: CpuSample, threads: int, keep=False):
    """One pass of the whole path by the float64 oracle (kernels, coordinates, gridding,
    degridding of the grid, image), with the time of each part."""
    import oracle
    from oracle import wproj
    cfg, prm = sp.cfg, sp.prm
    t = [time.perf_counter()]
    tabs, _ = oracle.wkernels(prm)
    t.append(time.perf_counter())
    crd = oracle.coords(sp.uvw, sp.freqs, prm, hermitian_pairs=cfg.hermitian_pairs)
    crd1 = oracle.coords(sp.uvw, sp.freqs, prm)
    c = wproj.gridded_values(sp.vis, sp.weight, crd)
    t.append(time.perf_counter())
    g = oracle.grid(crd, c, tabs, prm, threads=threads)
    t.append(time.perf_counter())
    pred = oracle.degrid(crd1, g, tabs, prm, threads=threads)
    t.append(time.perf_counter())
    sw = max(oracle.sum_weights(sp.weight, crd), 1.0)
    img = oracle.fft_to_image(g, sw, prm)
    t.append(time.perf_counter())
    names = ("wkernels", "coords", "grid", "degrid", "fft_image")
    out = {"seconds": t[-1] - t[0], "phases_s": {k: round(t[i + 1] - t[i], 4) for i, k in enumerate(names)},
           "kept": int(crd["keep"].sum()), "kept_degrid": int(crd1["keep"].sum())}
    if keep:
        out.update(tabs=tabs, crd=crd, crd1=crd1, c=c, grid=g, sum_w=sw, image=img, pred=pred)
    return out


def single_thread_grid_rate(sp: CpuSample, res, frac=16):
    """The paper's single-thread figure (Sec. 3.1-3.2): the oracle's scatter on one thread, on
    the first 1/frac of the sample's gridded visibilities."""
    import oracle
    crd = dict(res["crd"])
    keep = crd["keep"].copy()
    cut = np.zeros_like(keep)
    cut[: max(1, keep.size // frac)] = True
    crd["keep"] = keep & cut
    n = int(crd["keep"].sum())
    t0 = time.perf_counter()
    oracle.grid(crd, res["c"], res["tabs"], sp.prm, threads=1)
    dt = time.perf_counter() - t0
    return {"grid_vis_per_s": n / dt, "gridded_visibilities": n, "seconds": round(dt, 3), "threads": 1}


def cpu_baseline(args, sp: CpuSample, keep=False):
    """The float64 oracle on the host cores over the bounded sample `sp`: the same step as on
    the GPU (kernels, coordinates, grid, degrid, image)."""
    cores, threads = host_threads()
    r = oracle_step(sp, threads, keep=keep)
    dt = r["seconds"]
    cb = {"value": r["kept"] / dt, "unit": "visibilities/s", "cores": threads, "kind": "oracle",
          "sample": f"first {sp.rows} rows ({r['kept']} gridded visibilities) of the workload, full step "
                    f"(kernels, coordinates, grid, degrid, image), float64, {dt:.1f} s on {threads} of {cores} cores",
          "phases_s": r["phases_s"]}
    return cb, r


def peak_rel(a, ref):
    a, ref = np.asarray(a), np.asarray(ref)
    scale = float(np.abs(ref).max())
    d = np.abs(a - ref)
    return {"max": float(d.max() / scale), "rms": float(np.sqrt(np.mean(d ** 2)) / scale)}


def error_figures(wp, sp: CpuSample, res, compensated=False):
    """Peak-relative max and RMS error of the GPU path against the float64 oracle on the
    sample: grid, uncorrected image (all pixels), corrected image (inner half, where the taper
    is not near zero) and degridded visibilities (of the GPU's own grid, so that only the
    degridding arithmetic differs)."""
    import torch
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    uvw = torch.from_numpy(np.ascontiguousarray(sp.uvw)).to(dev)
    f = torch.from_numpy(np.ascontiguousarray(sp.freqs)).to(dev)
    vis = torch.from_numpy(np.ascontiguousarray(sp.vis)).to(dev)
    wt = torch.from_numpy(np.ascontiguousarray(sp.weight)).to(dev)
    g, sw, _ = wp.grid(uvw, f, vis, wt, hermitian_pairs=sp.cfg.hermitian_pairs, compensated=compensated)
    pred = wp.degrid(uvw, f, g)
    g_host = g.cpu().numpy()
    img_u = wp.fft_to_image(g.clone(), sw, taper_correct=False).cpu().numpy()
    img_c = wp.fft_to_image(g, sw, taper_correct=True).cpu().numpy()
    n = sp.prm.n
    q = slice(n // 4, 3 * n // 4)
    ref_u = oracle.fft_to_image(res["grid"], res["sum_w"], sp.prm, taper_correct=False)
    ref_pred = oracle.degrid(res["crd1"], g_host.astype(np.complex128), res["tabs"], sp.prm, threads=host_threads()[1])
    return {"grid": peak_rel(g_host, res["grid"]),
            "image_uncorrected": peak_rel(img_u, ref_u),
            "image_corrected_inner": peak_rel(img_c[q, q], res["image"][q, q]),
            "degrid": peak_rel(pred.cpu().numpy().ravel(), ref_pred.ravel()),
            "sample": f"first {sp.rows} rows of the workload ({res['kept']} gridded visibilities)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    import synth
    cfg = synth.config(args.config)
    rows = cpu_sample_rows(cfg, args.cpu_vis)
    sp = cpu_sample_from_host(cfg, rows)        # inputs made once, outside the timing
    cores, threads = host_threads()
    times, r = [], None
    for i in range(args.warmup + args.steps):
        r = oracle_step(sp, threads)
        if i >= args.warmup:
            times.append(r["seconds"])
    ms = 1e3 * float(np.mean(times))
    value = r["kept"] / (ms * 1e-3)
    cb = {"value": value, "unit": "visibilities/s", "cores": threads, "kind": "oracle",
          "sample": f"first {rows} rows ({r['kept']} gridded visibilities) of the workload per step, full step "
                    f"(kernels, coordinates, grid, degrid, image), float64, on {threads} of {cores} cores",
          "phases_s": r["phases_s"]}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "visibilities/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": workload_name(args.config), "sample_rows": rows}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "visibilities/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batched(args):
    """Batched imaging jobs: 64 jobs of uneven sizes (synth.batch_jobs), tile per job from the
    autotuner, all gridded by one wp_batch_grid replayed as a CUDA graph; the same jobs gridded
    one by one with wp_grid are timed beside it."""
    import torch
    import synth
    import paper_1905_03213_b300 as W
    from paper_1905_03213_b300.autotune import tune_tile
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    specs = synth.batch_jobs(n_jobs=args.jobs, scale=args.batch_scale)
    jobs, total_vis, tiles = [], 0, {}
    t_setup = time.perf_counter()
    for sp in specs:
        uvw = torch.as_tensor(synth.job_uvw(sp), dtype=torch.float64, device=dev)
        freq = torch.as_tensor(sp.freqs, dtype=torch.float64, device=dev)
        nrow, nchan = uvw.shape[0], freq.shape[0]
        g = torch.Generator(device=dev)
        g.manual_seed(sp.seed)
        vis = torch.view_as_complex(torch.randn((nrow, nchan, 2), generator=g, device=dev, dtype=torch.float32))
        w_max = float(uvw[:, 2].abs().max().item() * sp.freqs.max() / synth.C_LIGHT)
        params = dict(n=sp.n, cell=sp.cell, n_w=sp.n_w, w_max=w_max, support_min=sp.s_min, support_max=sp.s_max,
                      oversample=sp.oversample, table=args.table)
        tile, _ = tune_tile(params, uvw, freq, vis, candidates=((16, 16), (32, 32), (64, 32)), reps=2,
                            max_rows=min(nrow, 200_000))
        tiles[tile] = tiles.get(tile, 0) + 1
        wp = W.WProj(**params, tile=tile)
        wp.make_wkernels()
        jobs.append(dict(wp=wp, uvw=uvw, freq=freq, vis=vis))
        total_vis += nrow * nchan
    batch = W.WBatch(jobs)
    graph = batch.capture()
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    for _ in range(args.warmup):
        graph.replay()
    with ClockSampler(0) as clk:
        ms_batch = timed(graph.replay, args.steps)
    kept = sum(int(nrow_nchan) for nrow_nchan in [j["uvw"].shape[0] * j["freq"].shape[0] for j in jobs]) - \
        sum(int(nd.item()) for (_, _, nd) in batch.outputs)

    def plain():
        for j in jobs:
            j["wp"].grid(j["uvw"], j["freq"], j["vis"], None)

    plain()
    ms_plain = timed(plain, max(1, args.steps // 2))

    def phases(fn):
        for j in jobs:
            j["wp"].profile(True)
            j["wp"].profile_read()
        fn()
        torch.cuda.synchronize()
        tot = {}
        for j in jobs:
            ms, cnt, _ = j["wp"].profile_read()
            j["wp"].profile(False)
            for k, v in ms.items():
                tot[k] = tot.get(k, 0.0) + v
        return {k: round(v, 3) for k, v in tot.items() if v}

    phase_batch = phases(batch.grid)
    phase_plain = phases(plain)
    return {
        "metric": "gridded visibilities/s (batched imaging jobs: one persistent gridding launch, CUDA graph)",
        "value": kept / (ms_batch * 1e-3), "unit": "visibilities/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.table == "f32" else f"f32 ({args.table} tables)",
        "data": "synthetic (seeded job generator; random complex visibilities)",
        "config": {"workload": f"batched: {len(jobs)} jobs, N in {{512,1024,2048,4096}}, visibilities "
                               f"log-uniform 10k-20M x {args.batch_scale} ({total_vis / 1e6:.1f}M total), supports 7-31, "
                               f"oversampling 4-8, 8-64 w-planes, tile per job from the autotuner",
                   "fused_jobs": batch.fused_jobs, "tiles_chosen": {f"{a}x{b}": c for (a, b), c in tiles.items()},
                   "gridded_visibilities": kept, "setup_s": setup_s},
        "plain_fp32_per_job": {"value": kept / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                               "note": "same jobs, one wp_grid call each, eager"},
        "batched_over_plain": ms_plain / ms_batch,
        "phases_ms": {"batched": phase_batch, "plain": phase_plain},
        "clocks": clk.summary(),
    }


def run_compare(args):
    """The paper's own GPU scheme (Sec. 2.2, Fig. 2: rows grouped by the Eq. 5 baseline index,
    time-ordered, one thread per support tap) against the binned kernels, both gridding the
    float32 workload's time-major baselines; the baseline ordering (Eq. 5/6 and a per-baseline
    sort) is timed apart as the one-off preprocessing it is in the paper."""
    import numpy as np
    import torch
    import synth
    import paper_1905_03213_b300 as W
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cfg = synth.config("fp32")
    ob = synth.observe(cfg, device="cuda:0", rows=args.rows or None)
    uvw, vis, wt = ob.uvw.contiguous(), ob.vis.contiguous(), ob.weight.contiguous()
    freq = torch.as_tensor(ob.freqs, dtype=torch.float64, device=dev)
    nrow = uvw.shape[0]
    a1, a2 = synth.row_antennas(cfg.n_ant, cfg.n_time)
    ant1 = torch.from_numpy(a1[:nrow]).to(dev)
    ant2 = torch.from_numpy(a2[:nrow]).to(dev)
    wp = W.WProj(n=cfg.n, cell=cfg.cell, n_w=cfg.n_w, w_max=ob.w_max, support_min=cfg.s_min,
                 support_max=cfg.s_max, oversample=cfg.oversample, table=args.table)
    wp.make_wkernels()
    grid = torch.empty((cfg.n, cfg.n), dtype=torch.complex64, device=dev)
    grid_b = torch.empty_like(grid)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # larger than L2

    def timed(fn, reps):
        tot = 0.0
        for _ in range(reps):
            flush.add_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    perm, start = wp.baseline_order(ant1, ant2, cfg.n_ant)

    def binned():
        wp.grid(uvw, freq, vis, wt, grid=grid, hermitian_pairs=cfg.hermitian_pairs)

    def baseline():
        wp.grid_baseline(uvw, freq, vis, perm, start, cfg.n_ant, wt, grid=grid_b,
                         hermitian_pairs=cfg.hermitian_pairs)

    def order():
        wp.baseline_order(ant1, ant2, cfg.n_ant)

    for _ in range(args.warmup):
        binned(), baseline(), order()
    with ClockSampler(0) as clk:
        ms_order = timed(order, args.steps)
        ms_binned = timed(binned, args.steps)
        ms_baseline = timed(baseline, args.steps)

    def phases(fn):
        wp.profile(True)
        wp.profile_read()
        fn()
        torch.cuda.synchronize()
        ms, _, _ = wp.profile_read()
        wp.profile(False)
        return {k: round(v, 3) for k, v in ms.items() if v}

    ph_binned, ph_baseline = phases(binned), phases(baseline)
    g0, g1 = grid.cpu().numpy(), grid_b.cpu().numpy()
    agree = float(np.abs(g0 - g1).max() / np.abs(g0).max())
    ngridded = nrow * len(ob.freqs) * (2 if cfg.hermitian_pairs else 1)
    return {
        "metric": "gridded visibilities/s (binned kernels vs the paper's baseline-ordered scheme)",
        "value": ngridded / (ms_binned * 1e-3), "unit": "visibilities/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_binned, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.table == "f32" else f"f32 ({args.table} tables)",
        "data": "synthetic (seeded array, power-law sky, time-major baselines)",
        "config": {"workload": f"{cfg.n_ant} antennas x {cfg.n_time} samples x {len(ob.freqs)} channels "
                               f"+ Hermitian partners, {cfg.n}^2, {cfg.n_w} planes, support "
                               f"{cfg.s_min}-{cfg.s_max}, oversampling {cfg.oversample}",
                   "l2": "256 MiB buffer written before every timed call"},
        "binned_ms": ms_binned, "baseline_ordered_ms": ms_baseline, "baseline_order_ms": ms_order,
        "baseline_ordered_over_binned": ms_baseline / ms_binned,
        "phases_ms": {"binned": ph_binned, "baseline_ordered": ph_baseline},
        "grids_peak_rel_diff": agree,
        "clocks": clk.summary(),
    }


def run_autotune(args):
    """--autotune: the autotuner's search (tile shape x work units per CTA) on the workload's own
    visibilities, each candidate one gridding plus one degridding with the gridding plan."""
    import torch
    import synth
    from paper_1905_03213_b300.autotune import tune

    cfg = synth.config(args.config)
    ob = synth.observe(cfg, device="cuda:0", rows=args.rows or None)
    freq = torch.as_tensor(ob.freqs, dtype=torch.float64, device="cuda:0")
    params = dict(n=cfg.n, cell=cfg.cell, n_w=cfg.n_w, w_max=ob.w_max, support_min=cfg.s_min,
                  support_max=cfg.s_max, oversample=cfg.oversample, table=args.table)
    best, t = tune(params, ob.uvw.contiguous(), freq, ob.vis.contiguous(), ob.weight.contiguous(),
                   hermitian_pairs=cfg.hermitian_pairs, tiles=((32, 16), (32, 32), (64, 32), (64, 16)),
                   units=(3, 4, 6, 8, 12), reps=max(args.steps, 1), with_degrid=True, use_cache=False)
    return {"metric": "ms per wp_grid + wp_degrid_last, by tile shape and work units per CTA",
            "config": {"workload": workload_name(args.config), "table": args.table},
            "best": best, "ms": {f"{k[0][0]}x{k[0][1]}/{k[1]}": v for k, v in t.items()}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wproj", choices=["wproj", "reference"])
    ap.add_argument("--config", default="fp32",
                    help="fp32 | mixed | diff (imaging step), batched (many jobs), compare (the paper's GPU "
                         "scheme), fp32peak (the FMA probe)")
    ap.add_argument("--table", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--tile", default="", help="origin tile WxH, e.g. 64x32")
    ap.add_argument("--units", type=int, default=0, help="work units per CTA of the grid/degrid schedule (0: default)")
    ap.add_argument("--cpu-vis", type=int, default=6_000_000, help="visibilities (rows x channels) in the CPU sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the FP32 FMA probe")
    ap.add_argument("--variants", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the f16/bf16 tables on the same workload, with their errors")
    ap.add_argument("--rows", type=int, default=0, help="use only the first ROWS rows (profiling captures)")
    ap.add_argument("--jobs", type=int, default=64, help="--config batched: number of jobs")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="--config batched: visibility-count scale")
    ap.add_argument("--autotune", action="store_true", help="run the tile/granularity autotuner on the workload")
    args = ap.parse_args()
    if args.impl != "reference":
        args.warmup = max(args.warmup, 3)
    if args.autotune and args.impl != "reference":
        out = run_autotune(args)
    elif args.config == "fp32peak" and args.impl != "reference":
        out = run_fp32peak(args)
    elif args.config == "batched" and args.impl != "reference":
        out = run_batched(args)
    elif args.config == "compare" and args.impl != "reference":
        out = run_compare(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

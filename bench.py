"""Throughput benchmark of the fused 16x16 block codec (libtx16) on GB300.

Workload (one step): 256 frames of 1920 x 1088 uint8 luma -- one AR(1)
field (rho 0.95) cropped along a 2-pixel random walk, a stand-in for video --
through the fused forward transform, S-scaled quantiser (q = 16, zonal r = 16),
inverse, reconstruction and per-frame squared-error reduction: 2,088,960
16x16 blocks, one kernel launch.  Inputs (535 MB) and outputs (535 MB) are
larger than the 129 MB L2, so every step streams from HBM.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mblocks/s & % of HBM roofline (fused fwd+quant+inv); serving p50/p99 latency"
UNIT = "Mblocks/s"
FRAMES, H, W = 256, 1088, 1920
BLOCKS_PER_FRAME = (H // 16) * (W // 16)
BYTES_PER_BLOCK_CODEC = 512    # 256 B samples in + 256 B reconstructed samples out
BYTES_PER_BLOCK_FORWARD = 1280  # 256 B samples in + 1024 B int32 coefficients out
SEED = 2016
# SSIM: binary32 operations per window position (row pass of five moments
# 65.5, column pass 55, the index 17) and the GB300's binary32 lanes
SSIM_OPS_PER_POSITION = 137.5
ALU_LANES_PER_SM, SM_COUNT, SM_MAX_MHZ = 128, 152, 2070


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def _workload(q, r):
    return {"workload": f"{FRAMES} frames {W}x{H} uint8 AR(1) rho=0.95 with 2-px random-walk translation; "
                        f"fused forward+quantise(q={q:g},r={r})+inverse+SSE",
            "frames": FRAMES, "width": W, "height": H, "q": q, "r": r,
            "blocks_per_step": FRAMES * BLOCKS_PER_FRAME,
            "l2": "inputs larger than L2 (535 MB in + 535 MB out per step)"}


# ---------------------------------------------------------------------------
# Clocks sampled with nvidia-smi while the GPU is busy
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,utilization.gpu,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) == 7:
                try:
                    rows.append((float(p[0]), float(p[1]), float(p[2]), p[3:]))
                except ValueError:
                    pass
        loaded = [r for r in rows if r[2] >= 50.0] or rows
        if not loaded:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in loaded),
                "reasons": reasons, "samples": len(loaded)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def max_over_ranks(value: float, world: int) -> float:
    """The largest value over all ranks (the job time is the slowest rank's);
    works with any torch.distributed backend (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(blocks_per_rank: int, world: int, ms: float) -> float:
    """Whole-job Mblocks/s: every rank's blocks over the slowest rank's time."""
    return world * blocks_per_rank / (ms * 1e-3) / 1e6


def _at(arr, i):
    """Pointer to element i of a ctypes array of descriptors."""
    t = arr._type_
    return ctypes.cast(ctypes.addressof(arr) + i * ctypes.sizeof(t), ctypes.POINTER(t))


def _events_time(fn, steps, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps  # ms per step


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1606_07414_gb300 import synth, tx16

    rank, local_rank, world = _env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    lib = tx16.load()
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)

    frames = synth.video_frames(SEED + rank, FRAMES, H, W, rho=0.95)
    h_in = torch.from_numpy(frames).pin_memory()
    d_in = h_in.to("cuda", non_blocking=False)
    d_out = torch.empty_like(d_in)
    d_sse = torch.zeros(FRAMES, dtype=torch.int64, device="cuda")
    ins = (tx16.tx16_image * FRAMES)(*[tx16.image(d_in[i]) for i in range(FRAMES)])
    outs = (tx16.tx16_image * FRAMES)(*[tx16.image(d_out[i]) for i in range(FRAMES)])

    def qparams(q, r):
        return (tx16.tx16_qparams * FRAMES)(*[tx16.tx16_qparams(q, r)] * FRAMES)

    qp = qparams(args.q, args.r)
    sse_ptr = ctypes.c_void_p(d_sse.data_ptr())

    def step():
        st = lib.tx16_codec_batch(ins, outs, FRAMES, qp, sse_ptr, None, sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_codec_batch")

    sampler = ClockSampler(local_rank) if rank == 0 else None
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = _events_time(step, args.steps, stream)
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(ms, world)
    blocks = FRAMES * BLOCKS_PER_FRAME
    value = job_throughput(blocks, world, ms)

    # Per-frame PSNR of the last step (reported, from the library's host helper)
    sse_host = d_sse.cpu().tolist()
    psnr = tx16.tx16_psnr(sse_host, [ins[0]] * FRAMES)
    mean_psnr = float(np.mean(psnr))

    extra = {}
    if rank == 0 and not args.quick:
        extra = _extras(args, lib, tx16, torch, np, ins, outs, d_in, d_out, h_in, d_sse, sptr, stream, qparams)
    clocks = sampler.stop() if sampler else None

    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    peak = _measured_peak()
    achieved = blocks * BYTES_PER_BLOCK_CODEC / (ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "i32+f32", "data": "synthetic", "config": _workload(args.q, args.r),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak["value"], "unit": "GB/s",
                     "frac": round(achieved / peak["value"], 4), "traffic": _traffic_per_launch(),
                     "peak_source": peak["source"], "kernel": _codec_kernel_name(args.r),
                     "algorithmic_bytes_per_launch": blocks * BYTES_PER_BLOCK_CODEC},
        "gpu_launches": args.steps,
        "mean_psnr_db": round(mean_psnr, 4),
    }
    line.update(extra)
    line["clocks"] = clocks
    prop = torch.cuda.get_device_properties(local_rank)
    line["device"] = {"name": prop.name, "sm_count": prop.multi_processor_count,
                      "compute_capability": f"{prop.major}.{prop.minor}",
                      "hbm_gib": round(prop.total_memory / 2**30, 1)}
    line["seeds"] = {"frames": SEED, "per_rank": "frames seed + rank", "10bit_frames": SEED + 10,
                     "uneven_sizes": SEED + 9, "uneven_fields": f"{SEED + 700}..", "serving_arrivals": "seed + rate"}
    print(json.dumps(line), flush=True)


def _extras(args, lib, tx16, torch, np, ins, outs, d_in, d_out, h_in, d_sse, sptr, stream, qparams):
    out = {}
    blocks = FRAMES * BLOCKS_PER_FRAME
    peak = _measured_peak()["value"]

    # -- end to end through the public API: pinned host frames in, host
    #    reconstruction and per-frame SSE out, copies inside the timed region.
    h_out = torch.empty_like(h_in).pin_memory()
    h_sse = torch.empty(FRAMES, dtype=torch.int64).pin_memory()
    qp = qparams(args.q, args.r)
    chunk = args.e2e_chunk
    copy_in = torch.cuda.Stream()
    copy_out = torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(FRAMES // chunk)]
    ev_k = [torch.cuda.Event() for _ in range(FRAMES // chunk)]
    sse_ptr = d_sse.data_ptr()

    def e2e_step():
        # chunked pipeline: H2D of chunk i+1 and D2H of chunk i-1 overlap the
        # kernel on chunk i (separate copy engines, full-duplex link)
        for c in range(FRAMES // chunk):
            s = slice(c * chunk, (c + 1) * chunk)
            with torch.cuda.stream(copy_in):
                d_in[s].copy_(h_in[s], non_blocking=True)
                ev_in[c].record(copy_in)
            stream.wait_event(ev_in[c])
            st = lib.tx16_codec_batch(_at(ins, c * chunk), _at(outs, c * chunk), chunk,
                                      qp, ctypes.c_void_p(sse_ptr + 8 * c * chunk), None, sptr)
            if st != 0:
                raise tx16.Tx16Error(st, "tx16_codec_batch")
            ev_k[c].record(stream)
            with torch.cuda.stream(copy_out):
                copy_out.wait_event(ev_k[c])
                h_out[s].copy_(d_out[s], non_blocking=True)
        copy_out.wait_stream(stream)
        with torch.cuda.stream(copy_out):
            h_sse.copy_(d_sse, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(2):
        e2e_step()
    n_e2e = max(3, min(args.steps, 20))
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
    out["e2e"] = {"value": round(blocks / (e2e_ms * 1e-3) / 1e6, 2), "unit": UNIT,
                  "h2d_bytes_per_step": h_in.numel(), "d2h_bytes_per_step": h_out.numel() + 8 * FRAMES,
                  "ms_per_step": round(e2e_ms, 4), "pipeline": f"{FRAMES // chunk} chunks of {chunk} frames, "
                                                               "copy streams overlapping the kernel"}

    # -- the small case: one 512 x 512 8-bit image (1024 blocks), zonal r = 16,
    #    no quantiser; launch-latency bound, so reported in microseconds
    from paper_1606_07414_gb300 import synth

    img1 = torch.from_numpy(synth.ar1_image(1, 512, 512, 0.95)).cuda()
    rec1 = torch.empty_like(img1)
    sse1 = torch.zeros(1, dtype=torch.int64, device="cuda")
    in1 = (tx16.tx16_image * 1)(tx16.image(img1))
    out1 = (tx16.tx16_image * 1)(tx16.image(rec1))
    qp1 = qparams(0.0, 16)

    def small():
        st = lib.tx16_codec_batch(in1, out1, 1, qp1, ctypes.c_void_p(sse1.data_ptr()), None, sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_codec_batch")

    for _ in range(20):
        small()
    small_gpu_ms = _events_time(small, 500, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(200):
        small()
        torch.cuda.synchronize()
    small_sync_us = (time.perf_counter() - t0) * 1e6 / 200
    out["small_image"] = {
        "workload": "one 512x512 uint8 AR(1) image (rho 0.95, seed 1), 1024 blocks, zonal r = 16, no quantiser",
        "us_per_call_gpu": round(small_gpu_ms * 1e3, 2),
        "us_per_call_synchronous": round(small_sync_us, 2),
        "psnr_db": round(tx16.tx16_psnr([int(sse1.item())], [in1[0]])[0], 4)}

    # -- end to end with the kernel reading and writing the pinned host planes
    #    directly (mapped memory over the CPU-GPU link: no staging copies)
    hin = (tx16.tx16_image * FRAMES)(*[tx16.tx16_image(h_in[i].data_ptr(), W, H, W, 8) for i in range(FRAMES)])
    hout = (tx16.tx16_image * FRAMES)(*[tx16.tx16_image(h_out[i].data_ptr(), W, H, W, 8) for i in range(FRAMES)])

    def zc_step():
        st = lib.tx16_codec_batch(hin, hout, FRAMES, qp, ctypes.c_void_p(sse_ptr), None, sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_codec_batch")
        h_sse.copy_(d_sse, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(2):
        zc_step()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        zc_step()
    zc_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
    out["e2e_zero_copy"] = {"value": round(blocks / (zc_ms * 1e-3) / 1e6, 2), "unit": UNIT,
                            "h2d_bytes_per_step": h_in.numel(), "d2h_bytes_per_step": h_out.numel() + 8 * FRAMES,
                            "ms_per_step": round(zc_ms, 4),
                            "pipeline": "one launch; the kernel loads the pinned host frames and stores the "
                                        "reconstruction into pinned host memory over the CPU-GPU link"}

    # -- q x r sweep of the fused kernel (the workload's full parameter grid)
    sweep = []
    for q in (8.0, 16.0, 32.0):
        for r in (4, 16, 64, 256):
            qpx = qparams(q, r)

            def f():
                lib.tx16_codec_batch(ins, outs, FRAMES, qpx, ctypes.c_void_p(sse_ptr), None, sptr)
            for _ in range(3):
                f()
            ms = _events_time(f, 10, stream)
            gbs = blocks * BYTES_PER_BLOCK_CODEC / (ms * 1e-3) / 1e9
            sweep.append({"q": q, "r": r, "Mblocks_s": round(blocks / (ms * 1e-3) / 1e6, 1),
                          "GB_s": round(gbs, 1), "frac": round(gbs / peak, 4)})
    out["sweep"] = sweep

    # -- the unfused ("plain") form: per-frame forward, quantise, inverse and
    #    SSE launches through int32 coefficients in HBM
    nbf = BLOCKS_PER_FRAME
    coeffs = torch.empty(FRAMES * nbf * 256, dtype=torch.int32, device="cuda")
    one_qp = qparams(args.q, args.r)
    qsingle = tx16.tx16_qparams(args.q, args.r)

    def plain():
        for i in range(FRAMES):
            cp = ctypes.c_void_p(coeffs.data_ptr() + i * nbf * 1024)
            a = _at(ins, i)
            b = _at(outs, i)
            lib.tx16_forward(a, 1, cp, sptr)
            lib.tx16_quantise(cp, nbf, qsingle, cp, sptr)
            lib.tx16_inverse(cp, b, 1, one_qp, sptr)
            lib.tx16_sse(a, b, 1, ctypes.c_void_p(sse_ptr + 8 * i), sptr)
    plain()
    ms_plain = _events_time(plain, 3, stream)
    out["plain_form"] = {"value": round(blocks / (ms_plain * 1e-3) / 1e6, 2), "unit": UNIT,
                         "ms_per_step": round(ms_plain, 4), "launches_per_step": 4 * FRAMES}

    # -- forward only to int32 coefficients (64 images of 2048 x 2048):
    #    one batched launch vs one launch per image
    del coeffs
    n2, s2 = 64, 2048
    nb2 = (s2 // 16) ** 2
    base = torch.from_numpy(np.ascontiguousarray(d_in[:2].cpu().numpy()[:, :1024, :1024])).cuda()
    imgs2 = torch.empty((n2, s2, s2), dtype=torch.uint8, device="cuda")
    for i in range(n2):  # tile crops of the frames: the transform's cost is data independent
        imgs2[i] = base[i % 2].repeat(2, 2)
    co2 = torch.empty(n2 * nb2 * 256, dtype=torch.int32, device="cuda")
    d2 = (tx16.tx16_image * n2)(*[tx16.image(imgs2[i]) for i in range(n2)])
    cptr = ctypes.c_void_p(co2.data_ptr())

    def fwd_batched():
        lib.tx16_forward(d2, n2, cptr, sptr)

    def fwd_per_image():
        for i in range(n2):
            lib.tx16_forward(_at(d2, i), 1,
                             ctypes.c_void_p(co2.data_ptr() + i * nb2 * 1024), sptr)
    for f in (fwd_batched, fwd_per_image):
        for _ in range(3):
            f()
    ms_b = _events_time(fwd_batched, 10, stream)
    ms_p = _events_time(fwd_per_image, 10, stream)
    gb = n2 * nb2 * BYTES_PER_BLOCK_FORWARD / 1e9
    out["forward_only"] = {"workload": "64 images 2048x2048 uint8 -> int32 coefficients",
                           "batched": {"Mblocks_s": round(n2 * nb2 / (ms_b * 1e-3) / 1e6, 1),
                                       "GB_s": round(gb / (ms_b * 1e-3), 1),
                                       "frac": round(gb / (ms_b * 1e-3) / peak, 4)},
                           "per_image_launches": {"Mblocks_s": round(n2 * nb2 / (ms_p * 1e-3) / 1e6, 1),
                                                  "GB_s": round(gb / (ms_p * 1e-3), 1)}}
    del co2, imgs2

    # -- zonal sweep (the paper's Fig. 2 experiment): PSNR for ten r values
    #    from one forward per block, no quantiser
    r_list = [1, 2, 4, 8, 16, 32, 64, 100, 128, 150]
    rl = (ctypes.c_int32 * len(r_list))(*r_list)
    sw = torch.zeros(FRAMES * len(r_list), dtype=torch.int64, device="cuda")

    def sweep():
        lib.tx16_zonal_sweep(ins, FRAMES, rl, len(r_list), ctypes.c_void_p(sw.data_ptr()), sptr)
    for _ in range(2):
        sweep()
    ms_sw = _events_time(sweep, 5, stream)
    sse_r = sw.view(FRAMES, len(r_list)).sum(0).cpu().tolist()
    npx = FRAMES * H * W
    psnr_r = [10 * math.log10(255.0 ** 2 * npx / s) if s else float("inf") for s in sse_r]
    out["zonal_sweep"] = {"workload": f"{FRAMES} frames 1920x1088, r in {r_list}, no quantiser, exact inverse",
                          "block_r_per_s_M": round(blocks * len(r_list) / (ms_sw * 1e-3) / 1e6, 1),
                          "ms": round(ms_sw, 3),
                          "psnr_db": [round(p, 3) for p in psnr_r],
                          "psnr_per_addition": [round(p / 44.0, 4) for p in psnr_r]}

    # -- real 1920 x 1080 frames (1080 = 67.5 block rows): the any-size codec,
    #    one launch of the one-block-per-thread kernel over the padded block
    #    rows, the last block row repeating row 1079 and storing its 8 rows
    H1080 = 1080
    ins_a = (tx16.tx16_image * FRAMES)(*[tx16.tx16_image(d_in[i].data_ptr(), W, H1080, W, 8)
                                         for i in range(FRAMES)])
    outs_a = (tx16.tx16_image * FRAMES)(*[tx16.tx16_image(d_out[i].data_ptr(), W, H1080, W, 8)
                                          for i in range(FRAMES)])
    qpa = qparams(args.q, args.r)

    def any_size():
        st = lib.tx16_codec_any_size(ins_a, outs_a, FRAMES, qpa, ctypes.c_void_p(sse_ptr), sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_codec_any_size")
    for _ in range(3):
        any_size()
    ms_a = _events_time(any_size, 10, stream)
    blocks_a = FRAMES * ((H1080 + 15) // 16) * (W // 16)
    gbs_a = FRAMES * H1080 * W * 2 / (ms_a * 1e-3) / 1e9
    out["any_size_1080"] = {"workload": f"{FRAMES} frames {W}x{H1080} uint8, q={args.q:g}, r={args.r}; "
                                        "edge-replicated last block row",
                            "Mblocks_s": round(blocks_a / (ms_a * 1e-3) / 1e6, 1),
                            "Gpixels_s": round(FRAMES * H1080 * W / (ms_a * 1e-3) / 1e9, 1),
                            "GB_s": round(gbs_a, 1), "frac": round(gbs_a / peak, 4), "ms": round(ms_a, 4),
                            "launches_per_step": 1}

    # -- 10-bit 3840 x 2160 frames (uint16 samples, 1 KB per block in and
    #    out): the fused 16-bit path against the general kernel
    n10, H10, W10 = 64, 2160, 3840
    f10 = torch.from_numpy(synth_frames_10bit(n10, H10, W10).view(np.int16)).cuda()
    o10 = torch.empty_like(f10)
    in10 = (tx16.tx16_image * n10)(*[tx16.image(f10[i], 10) for i in range(n10)])
    out10 = (tx16.tx16_image * n10)(*[tx16.image(o10[i], 10) for i in range(n10)])
    sse10 = torch.zeros(n10, dtype=torch.int64, device="cuda")
    blocks10 = n10 * (H10 // 16) * (W10 // 16)
    res10 = {}
    for label, qv in (("fused", 64.0), ("general", 0.01)):
        qp10 = (tx16.tx16_qparams * n10)(*[tx16.tx16_qparams(qv, args.r)] * n10)

        def c10():
            st = lib.tx16_codec_batch(in10, out10, n10, qp10, ctypes.c_void_p(sse10.data_ptr()), None, sptr)
            if st != 0:
                raise tx16.Tx16Error(st, "tx16_codec_batch")
        for _ in range(3):
            c10()
        ms10 = _events_time(c10, 10, stream)
        gbs10 = blocks10 * 1024 / (ms10 * 1e-3) / 1e9
        res10[label] = {"q": qv, "Mblocks_s": round(blocks10 / (ms10 * 1e-3) / 1e6, 1), "GB_s": round(gbs10, 1),
                        "frac": round(gbs10 / peak, 4), "ms": round(ms10, 4)}
    out["frames_10bit"] = {"workload": f"{n10} frames {W10}x{H10} 10-bit in uint16, r={args.r}; q = 64 on the "
                                       "fused 16-bit path, q = 0.01 (below its range) on the general kernel",
                           **res10}
    del f10, o10

    # -- mixed 8/16 tiling (the video experiment's second scenario): every
    #    region coded with T and as four 8x8 blocks with T8, the better kept
    mqp = (tx16.tx16_mixed_qparams * FRAMES)(*[tx16.tx16_mixed_qparams(args.q, args.r, max(1, args.r // 4), 0)] * FRAMES)
    split = torch.zeros(blocks, dtype=torch.uint8, device="cuda")

    def mixed():
        st = lib.tx16_codec_mixed(ins, outs, FRAMES, ctypes.cast(mqp, ctypes.c_void_p),
                                  ctypes.c_void_p(split.data_ptr()), ctypes.c_void_p(sse_ptr), sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_codec_mixed")
    for _ in range(3):
        mixed()
    ms_m = _events_time(mixed, 10, stream)
    sse_m = d_sse.cpu().tolist()
    psnr_m = float(np.mean(tx16.tx16_psnr(sse_m, [ins[0]] * FRAMES)))
    out["mixed_tiling"] = {"workload": f"{FRAMES} frames {W}x{H} uint8, q={args.q:g}, r16={args.r}, "
                                       f"r8={max(1, args.r // 4)}, tiling chosen per 16x16 region by squared error",
                           "Mregions_s": round(blocks / (ms_m * 1e-3) / 1e6, 1), "ms": round(ms_m, 4),
                           # 256 bytes in, 256 out and one split-map byte per region
                           "GB_s": round(blocks * 513 / (ms_m * 1e-3) / 1e9, 1),
                           "frac": round(blocks * 513 / (ms_m * 1e-3) / 1e9 / peak, 4),
                           "split_fraction": round(float(split.float().mean().item()), 4),
                           "mean_psnr_db": round(psnr_m, 4)}

    # -- SSIM of every frame against its reconstruction (the paper's second
    #    measure): arithmetic-bound, 137.5 binary32 operations per window position
    ms_t = torch.zeros(FRAMES, dtype=torch.float64, device="cuda")

    def ssim():
        st = lib.tx16_ssim(ins, outs, FRAMES, ctypes.c_void_p(ms_t.data_ptr()), None, sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_ssim")
    lib.tx16_codec_batch(ins, outs, FRAMES, qp, ctypes.c_void_p(sse_ptr), None, sptr)
    for _ in range(3):
        ssim()
    ms_s = _events_time(ssim, 10, stream)
    positions = FRAMES * (H - 10) * (W - 10)
    ops = positions * SSIM_OPS_PER_POSITION
    alu_peak = ALU_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6
    out["ssim"] = {"workload": f"{FRAMES} frames {W}x{H} uint8 vs their q={args.q:g}, r={args.r} reconstruction; "
                               "11x11 Gaussian window (sigma 1.5), mean over window positions",
                   "Gpositions_s": round(positions / (ms_s * 1e-3) / 1e9, 2), "ms": round(ms_s, 4),
                   "mean_ssim": round(float(ms_t.mean().item()), 6),
                   "roofline": {"bound": "alu", "achieved": round(ops / (ms_s * 1e-3) / 1e12, 2),
                                "peak": round(alu_peak / 1e12, 2), "unit": "Tops/s",
                                "frac": round(ops / (ms_s * 1e-3) / alu_peak, 4),
                                "ops_per_position": SSIM_OPS_PER_POSITION,
                                "peak_source": f"{ALU_LANES_PER_SM} binary32 lanes x {SM_COUNT} SMs x "
                                               f"{SM_MAX_MHZ} MHz (one fma, add or mul per lane per clock)"}}

    # -- uneven-size batch (2000 images, sides 64..4096): plan vs per-image launches
    if not args.no_uneven:
        out["uneven_batch"] = _uneven_batch(lib, tx16, torch, np, stream, sptr, peak)

    # -- serving: Poisson arrivals, continuous batching vs one request at a time
    if not args.no_serve:
        out["serving"] = _serving(tx16, torch, np, args)

    # -- CPU baseline: the oracle on a bounded sample, all host cores
    if not args.no_cpu:
        frames_np = h_in[: args.cpu_frames].numpy()
        out["cpu_baseline"] = cpu_oracle_rate(frames_np, args.q, args.r)
    return out


def synth_frames_10bit(n, h, w):
    """n 10-bit frames (uint16), the same AR(1) video model at 10 bits."""
    from paper_1606_07414_gb300 import synth

    return synth.video_frames(SEED + 10, n, h, w, rho=0.95, bits=10)


def _gen_field(job):
    seed, n, rho = job
    from paper_1606_07414_gb300 import synth

    return synth.ar1_image(seed, n, n, rho)


def _uneven_batch(lib, tx16, torch, np, stream, sptr, peak):
    """2000 images with sides drawn independently from the multiples of 16 in
    [64, 4096], zonal r drawn from {8, 32, 128}, q = 16.  Inputs are crops of
    10 seeded 4096 x 4096 AR(1) fields (rho 0.80 .. 0.98), so many images
    re-read the same field: part of the input traffic is served by L2."""
    import multiprocessing as mp
    from paper_1606_07414_gb300 import synth

    n, side, nb = 2000, 4096, 10
    rhos = [0.80 + 0.02 * i for i in range(nb)]
    with mp.get_context("spawn").Pool(min(nb, os.cpu_count() or 1)) as pool:
        bases = pool.map(_gen_field, [(SEED + 700 + i, side, rhos[i]) for i in range(nb)])
    d_bases = [torch.from_numpy(b).cuda() for b in bases]
    Hs, Ws = synth.uneven_sizes(SEED + 9, n)
    rs = synth.choice(SEED + 10, n, [8, 32, 128])
    u = synth.uniforms(SEED + 11, 2 * n)
    total = int(np.sum(Hs.astype(np.int64) * Ws))
    d_out = torch.empty(total, dtype=torch.uint8, device="cuda")
    ins = (tx16.tx16_image * n)()
    outs = (tx16.tx16_image * n)()
    qp = (tx16.tx16_qparams * n)()
    off = 0
    for i in range(n):
        H, W = int(Hs[i]), int(Ws[i])
        base = d_bases[i % nb]
        oy = int(u[2 * i] * (side - H + 1))
        ox = int(u[2 * i + 1] * ((side - W) // 16 + 1)) * 16
        ins[i] = tx16.tx16_image(base.data_ptr() + oy * side + ox, W, H, side, 8)
        outs[i] = tx16.tx16_image(d_out.data_ptr() + off, W, H, W, 8)
        off += H * W
        qp[i] = tx16.tx16_qparams(16.0, int(rs[i]))
    blocks = total // 256
    sse = torch.zeros(n, dtype=torch.int64, device="cuda")
    plan = tx16.Plan(list(ins), list(outs), [(16.0, int(r)) for r in rs])
    plan.autotune(None)
    res = {"workload": f"{n} images, sides uniform over multiples of 16 in [64, 4096], r in {{8, 32, 128}}, "
                       f"q = 16, crops of {nb} AR(1) fields 4096^2 (rho 0.80..0.98)",
           "blocks": blocks, "schedule": plan.info()}

    def run_graph():
        plan.run_graph(sse=sse, stream=stream)

    def run_batch():
        lib.tx16_codec_batch(ins, outs, n, qp, ctypes.c_void_p(sse.data_ptr()), None, sptr)

    def run_per_image():
        for i in range(n):
            lib.tx16_codec_batch(_at(ins, i), _at(outs, i), 1, _at(qp, i),
                                 ctypes.c_void_p(sse.data_ptr() + 8 * i), None, sptr)
    for name, f, k in (("plan_graph", run_graph, 10), ("codec_batch", run_batch, 10),
                       ("per_image_launches", run_per_image, 3)):
        for _ in range(2):
            f()
        ms = _events_time(f, k, stream)
        res[name] = {"Mblocks_s": round(blocks / (ms * 1e-3) / 1e6, 1), "ms": round(ms, 3),
                     "GB_s": round(blocks * BYTES_PER_BLOCK_CODEC / (ms * 1e-3) / 1e9, 1)}
    plan.close()
    del d_out, d_bases
    return res


def _serving(tx16, torch, np, args):
    """Poisson request streams: 60 % 256 x 256 8-bit, 30 % 1920 x 1088 8-bit,
    10 % 3840 x 2160 10-bit (uint16), q from {8, 16, 32}, r from {4, 16, 64,
    256} per request; pinned host buffers.  The server's continuous batching
    against the plain form that codes one request at a time as it arrives."""
    from paper_1606_07414_gb300 import synth

    kinds = [(256, 256, 8), (1088, 1920, 8), (2160, 3840, 10)]
    pools = []
    for ki, (H, W, bits) in enumerate(kinds):
        k = 8 if ki < 2 else 3
        src = synth.video_frames(SEED + 50 + ki, k, H, W, bits=bits)
        dt = torch.uint8 if bits == 8 else torch.int16
        ins = [torch.from_numpy(f.view(np.int16) if bits > 8 else f).pin_memory() for f in src]
        outs = [torch.empty_like(t).pin_memory() for t in ins]
        pools.append((H, W, bits, ins, outs))
    cfg = {"device_pool_mb": 16384, "streams": args.serve_streams, "max_batch": 256}
    if args.serve_band_mb is not None:
        cfg["band_mb"] = args.serve_band_mb
    srv = tx16.Server(cfg)
    rates = [int(x) for x in args.serve_rates.split(",")]
    # untimed warm-up: every request kind, q and r through both forms once
    # (first launches of each kernel variant load their modules)
    dev_in = {k: torch.empty((H, W), dtype=torch.uint8 if b == 8 else torch.int16, device="cuda")
              for k, (H, W, b) in enumerate(kinds)}
    dev_out = {k: torch.empty_like(v) for k, v in dev_in.items()}
    sse = torch.zeros(1, dtype=torch.int64, device="cuda")
    warm = []
    for k, (H, W, bits, ins, outs) in enumerate(pools):
        for q in (8.0, 16.0, 32.0):
            for r in (4, 16, 64, 256):
                warm.append(srv.submit_ptr(ins[0].data_ptr(), W, H, bits, q, r, outs[0].data_ptr()))
                tx16.tx16_codec_batch([tx16.image(dev_in[k], bits)], [tx16.image(dev_out[k], bits)], [(q, r)],
                                      sse=sse)
    for t in warm:
        srv.wait(t)
    torch.cuda.synchronize()
    out = {"workload": "Poisson arrivals; 60% 256x256 u8, 30% 1920x1088 u8, 10% 3840x2160 10-bit; "
                       "q in {8,16,32}, r in {4,16,64,256}; pinned host buffers", "rates": []}
    for rate in rates:
        n = max(1000, min(int(rate * args.serve_seconds), 60000))  # p99 from at least 1000 requests
        u = synth.uniforms(SEED + rate, 4 * n)
        gaps = -np.log(u[:n]) / rate
        kind = np.where(u[n:2 * n] < 0.6, 0, np.where(u[n:2 * n] < 0.9, 1, 2))
        qs = np.array([8.0, 16.0, 32.0])[np.minimum((u[2 * n:3 * n] * 3).astype(int), 2)]
        rs = np.array([4, 16, 64, 256])[np.minimum((u[3 * n:] * 4).astype(int), 3)]
        reqs = []
        for i in range(n):
            H, W, bits, ins, outs = pools[kind[i]]
            j = i % len(ins)
            reqs.append((ins[j].data_ptr(), outs[j].data_ptr(), W, H, bits, float(qs[i]), int(rs[i]), H * W))
        blocks = sum(r[7] for r in reqs) / 256
        # continuous batching
        srv.reset_stats()
        tickets = []
        t0 = time.perf_counter()
        due = t0
        for i, (ip, op, W, H, bits, q, r, _) in enumerate(reqs):
            due += gaps[i]
            while time.perf_counter() < due:
                pass
            tickets.append(srv.submit_ptr(ip, W, H, bits, q, r, op))
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
        achieved = n / (time.perf_counter() - t0)
        line = {"rate": rate, "requests": n, "offered_Mblocks_s": round(blocks * rate / n / 1e6, 1),
                "batched": {"p50_us": round(st["p50_us"], 1), "p99_us": round(st["p99_us"], 1),
                            "p999_us": round(st["p999_us"], 1), "Mblocks_s": round(st["mblocks_per_s"], 1),
                            "req_per_s": round(achieved, 1)}}
        # the plain form: each request coded alone (copy in, one launch, copy out) as it arrives
        m = min(n, max(1000, int(rate * 0.5)))
        lat = []
        t0 = time.perf_counter()
        due = t0
        done_blocks = 0
        for i in range(m):
            due += gaps[i]
            while time.perf_counter() < due:
                pass
            H, W, bits, ins, outs = pools[kind[i]]
            j = i % len(ins)
            di, do = dev_in[kind[i]], dev_out[kind[i]]
            di.copy_(ins[j], non_blocking=True)
            tx16.tx16_codec_batch([tx16.image(di, bits)], [tx16.image(do, bits)], [(float(qs[i]), int(rs[i]))],
                                  sse=sse)
            outs[j].copy_(do, non_blocking=True)
            torch.cuda.synchronize()
            lat.append((time.perf_counter() - due) * 1e6)
            done_blocks += H * W / 256
        span = time.perf_counter() - t0
        lat = np.sort(np.array(lat))
        line["plain_per_request"] = {"requests": m, "p50_us": round(float(np.percentile(lat, 50)), 1),
                                     "p99_us": round(float(np.percentile(lat, 99)), 1),
                                     "p999_us": round(float(np.percentile(lat, 99.9)), 1),
                                     "Mblocks_s": round(done_blocks / span / 1e6, 1)}
        out["rates"].append(line)
    srv.close()
    return out


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------
def _oracle_frame(job):
    """One frame through the float64 oracle codec; the forward transform by
    the 44-addition factorisation (path B) unless the job says 'direct'."""
    frame, q, r = job[:3]
    forward = job[3] if len(job) > 3 else "factored"
    from oracle import tx16_oracle as O

    O.codec_image(frame, q, r, 8, "fp64", forward=forward)
    return frame.shape


def _oracle_frame_timed(job):
    t0 = time.perf_counter()
    _oracle_frame(job)
    return time.perf_counter() - t0


def cpu_oracle_rate(frames_np, q, r, pool=None, cores=None, single=True):
    """The oracle's rate on the host cores: frames_np through the float64
    codec with the factorised forward transform (path B), one frame per task
    on `cores` single-threaded processes; with `single`, also one frame on one
    core by each forward path (factorisation and direct matrix products)."""
    import multiprocessing as mp

    cores = cores or os.cpu_count() or 1
    own = pool is None
    if own:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        pool = mp.get_context("spawn").Pool(cores)
        pool.map(_oracle_frame, [(frames_np[0][:16, :16], q, r)] * cores)  # warm the workers
    t0 = time.perf_counter()
    pool.map(_oracle_frame, [(f, q, r, "factored") for f in frames_np], chunksize=1)
    dt = time.perf_counter() - t0
    out = {}
    if single:
        nblk1 = (frames_np.shape[1] // 16) * (frames_np.shape[2] // 16)
        for fw in ("factored", "direct"):
            t1 = pool.apply(_oracle_frame_timed, ((frames_np[0], q, r, fw),))  # one frame, one core
            key = "single_thread" if fw == "factored" else "single_thread_direct_matmul"
            out[key] = {"value": round(nblk1 / t1 / 1e6, 5), "unit": UNIT, "cores": 1,
                        "sample": f"one frame in one single-threaded process, forward by "
                                  f"{'the factorisation' if fw == 'factored' else 'int64 matrix products'}, "
                                  f"{t1:.3f} s"}
    if own:
        pool.close()
        pool.join()
    nblk = len(frames_np) * (frames_np.shape[1] // 16) * (frames_np.shape[2] // 16)
    res = {"value": round(nblk / dt / 1e6, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{len(frames_np)} of the {FRAMES} frames (float64 oracle codec_image, forward by the "
                     f"44-addition factorisation; one frame per task, {cores} single-threaded processes), "
                     f"{dt:.2f} s wall"}
    res.update(out)
    return res


def run_reference(args):
    import numpy as np
    import multiprocessing as mp

    from paper_1606_07414_gb300 import synth

    rank, _, world = _env_rank()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    # one frame per host core per step keeps any --steps K run to ~0.3 s a step
    frames = synth.video_frames(SEED, cores, H, W, rho=0.95)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    pool = mp.get_context("spawn").Pool(cores)
    pool.map(_oracle_frame, [(frames[0][:16, :16], args.q, args.r)] * cores)
    for _ in range(args.warmup):
        cpu_oracle_rate(frames[:1], args.q, args.r, pool, cores, single=False)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rates.append(cpu_oracle_rate(frames, args.q, args.r, pool, cores, single=False))
    dt = time.perf_counter() - t0
    pool.close()
    pool.join()
    nblk = args.steps * len(frames) * BLOCKS_PER_FRAME
    value = nblk / dt / 1e6
    line = {"metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i64+f64", "data": "synthetic",
            "config": dict(_workload(args.q, args.r), frames_coded_per_step=len(frames)),
            "impl": "reference",
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step codes {len(frames)} of the workload's {FRAMES} frames (one per "
                                       f"core) through the float64 oracle (forward by the factorisation) on "
                                       f"{cores} single-threaded processes"},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return {"value": float(json.load(f)["hbm_gbs"]), "source": "measured (copy, MEASURED_PEAKS.json)"}
    except (OSError, KeyError, ValueError):
        return {"value": 6800.0, "source": "fallback 6.8 TB/s"}


def _codec_kernel_name(r):
    """The fused kernel the library picks for an 8-bit batch with zone Z_r
    and no level output: the one-block-per-thread kernel of the zonal class
    (index 0..5, r_max 8, 16, 32, 64, 128, 256)."""
    for c, rmax in enumerate((8, 16, 32, 64, 128, 256)):
        if r <= rmax:
            return f"tx16::fused_bt_kernel<256, {c}, DST=true, 1> (one block per thread, class r <= {rmax})"
    return None


def _traffic_per_launch():
    """DRAM bytes per launch of the codec kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "codec_traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for fn in rec.get("sources", []):
        with open(os.path.join(ROOT, fn), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec.get("sha256"):
        return None
    scale = (FRAMES * BLOCKS_PER_FRAME) / rec["blocks"]
    return int(rec["dram_bytes"] * scale)


def run_ssim_only(args):
    """SSIM of --frames frames against their reconstruction, --steps timed
    launches after --warmup; prints one short JSON line (not the bench line)."""
    import torch

    from paper_1606_07414_gb300 import synth, tx16

    lib = tx16.load()
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    d_in = torch.from_numpy(synth.video_frames(SEED, FRAMES, H, W, rho=0.95)).cuda()
    d_out = torch.empty_like(d_in)
    ins = (tx16.tx16_image * FRAMES)(*[tx16.image(d_in[i]) for i in range(FRAMES)])
    outs = (tx16.tx16_image * FRAMES)(*[tx16.image(d_out[i]) for i in range(FRAMES)])
    qp = (tx16.tx16_qparams * FRAMES)(*[tx16.tx16_qparams(args.q, args.r)] * FRAMES)
    if lib.tx16_codec_batch(ins, outs, FRAMES, qp, None, None, sptr) != 0:
        raise RuntimeError("tx16_codec_batch failed")
    ms_t = torch.zeros(FRAMES, dtype=torch.float64, device="cuda")

    def ssim():
        st = lib.tx16_ssim(ins, outs, FRAMES, ctypes.c_void_p(ms_t.data_ptr()), None, sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_ssim")
    for _ in range(args.warmup):
        ssim()
    ms = _events_time(ssim, args.steps, stream)
    positions = FRAMES * (H - 10) * (W - 10)
    print(json.dumps({"ssim_ms": round(ms, 4), "frames": FRAMES,
                      "Gpositions_s": round(positions / (ms * 1e-3) / 1e9, 2),
                      "alu_frac": round(positions * SSIM_OPS_PER_POSITION / (ms * 1e-3)
                                        / (ALU_LANES_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6), 4),
                      "mean_ssim": round(float(ms_t.mean().item()), 6)}), flush=True)


def run_mixed_only(args):
    """Mixed 8/16 tiling of --frames frames (q, r16 = r, r8 = r / 4), --steps
    timed launches after --warmup; prints one short JSON line (not the bench
    line)."""
    import torch

    from paper_1606_07414_gb300 import synth, tx16

    lib = tx16.load()
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    d_in = torch.from_numpy(synth.video_frames(SEED, FRAMES, H, W, rho=0.95)).cuda()
    d_out = torch.empty_like(d_in)
    ins = (tx16.tx16_image * FRAMES)(*[tx16.image(d_in[i]) for i in range(FRAMES)])
    outs = (tx16.tx16_image * FRAMES)(*[tx16.image(d_out[i]) for i in range(FRAMES)])
    r8 = max(1, args.r // 4)
    mqp = (tx16.tx16_mixed_qparams * FRAMES)(*[tx16.tx16_mixed_qparams(args.q, args.r, r8, 0)] * FRAMES)
    regions = FRAMES * (H // 16) * (W // 16)
    split = torch.zeros(regions, dtype=torch.uint8, device="cuda")
    sse = torch.zeros(FRAMES, dtype=torch.int64, device="cuda")

    def mixed():
        st = lib.tx16_codec_mixed(ins, outs, FRAMES, ctypes.cast(mqp, ctypes.c_void_p),
                                  ctypes.c_void_p(split.data_ptr()), ctypes.c_void_p(sse.data_ptr()), sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_codec_mixed")
    for _ in range(args.warmup):
        mixed()
    ms = _events_time(mixed, args.steps, stream)
    gbs = regions * 513 / (ms * 1e-3) / 1e9
    print(json.dumps({"mixed_ms": round(ms, 4), "frames": FRAMES, "r16": args.r, "r8": r8,
                      "Mregions_s": round(regions / (ms * 1e-3) / 1e6, 1), "GB_s": round(gbs, 1),
                      "split_fraction": round(float(split.float().mean().item()), 4)}))


def run_frames10_only(args):
    """The fused 16-bit codec on --frames 3840 x 2160 10-bit frames, --steps
    timed launches after --warmup; prints one short JSON line (not the bench
    line)."""
    import numpy as np
    import torch

    from paper_1606_07414_gb300 import tx16

    lib = tx16.load()
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    n, H10, W10 = FRAMES, 2160, 3840
    f10 = torch.from_numpy(synth_frames_10bit(n, H10, W10).view(np.int16)).cuda()
    o10 = torch.empty_like(f10)
    ins = (tx16.tx16_image * n)(*[tx16.image(f10[i], 10) for i in range(n)])
    outs = (tx16.tx16_image * n)(*[tx16.image(o10[i], 10) for i in range(n)])
    qp = (tx16.tx16_qparams * n)(*[tx16.tx16_qparams(64.0, args.r)] * n)
    sse = torch.zeros(n, dtype=torch.int64, device="cuda")

    def c10():
        st = lib.tx16_codec_batch(ins, outs, n, qp, ctypes.c_void_p(sse.data_ptr()), None, sptr)
        if st != 0:
            raise tx16.Tx16Error(st, "tx16_codec_batch")
    for _ in range(args.warmup):
        c10()
    ms = _events_time(c10, args.steps, stream)
    blocks = n * (H10 // 16) * (W10 // 16)
    gbs = blocks * 1024 / (ms * 1e-3) / 1e9
    print(json.dumps({"frames10_ms": round(ms, 4), "frames": n, "r": args.r,
                      "Mblocks_s": round(blocks / (ms * 1e-3) / 1e6, 1), "GB_s": round(gbs, 1),
                      "frac": round(gbs / _measured_peak()["value"], 4)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="tx16", choices=["tx16", "reference"])
    ap.add_argument("--q", type=float, default=16.0)
    ap.add_argument("--r", type=int, default=16)
    ap.add_argument("--cpu-frames", type=int, default=96)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-rates", default="1000,2000,5000,10000,20000,50000")
    ap.add_argument("--serve-seconds", type=float, default=0.5)
    ap.add_argument("--serve-streams", type=int, default=6, help="stream slots of the server")
    ap.add_argument("--serve-only", action="store_true", help="the serving section alone (one short JSON line)")
    ap.add_argument("--serve-band-mb", type=float, default=None,
                    help="server band size in MB (planes above it are copied and coded in bands; 0: never)")
    ap.add_argument("--quick", action="store_true", help="headline number only")
    ap.add_argument("--e2e-chunk", type=int, default=16,
                    help="frames per chunk of the host-buffer pipeline (a divisor of the frame count)")
    ap.add_argument("--frames", type=int, default=FRAMES, help="smaller cases for profiling")
    ap.add_argument("--ssim-only", action="store_true",
                    help="time tx16_ssim alone on --frames frames and their reconstruction (profiling)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="the mixed 8/16 tiling section alone (one short JSON line)")
    ap.add_argument("--frames10-only", action="store_true",
                    help="time the fused 16-bit codec alone on --frames 10-bit 3840x2160 frames (profiling)")
    args = ap.parse_args()
    globals()["FRAMES"] = args.frames
    if args.warmup < 3 and args.impl == "tx16":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.serve_only:
        import numpy as np
        import torch

        from paper_1606_07414_gb300 import tx16

        tx16.load()
        print(json.dumps({"serving": _serving(tx16, torch, np, args), "streams": args.serve_streams}), flush=True)
    elif args.ssim_only:
        run_ssim_only(args)
    elif args.frames10_only:
        run_frames10_only(args)
    elif args.mixed_only:
        run_mixed_only(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

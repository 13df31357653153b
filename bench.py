#!/usr/bin/env python
"""Throughput of the JDE detect-and-track step on one GB300 (and N replicas).

One step = the whole hot path over one batch: letterbox of B FullHD uint8
frames to 1088x608, the 78-conv JDE network (BF16 tcgen05 implicit GEMM),
decode + confidence filter + NMS + embedding L2 for every frame, and one
tracker step (Kalman, cosine cost, gating, Hungarian, lifecycle) for each of
the B video streams.  Frames are uniform random uint8 (stand-in for the
FullHD MOT16 sequences of the paper's speed study, Sec. 5.1).  Random weights
cannot detect anything in noise, so the post-processing and tracker consume
head tensors with 50 planted objects per stream (constant-velocity paths),
swapped in after the forward: the forward does its full work, the tracker gets
a realistic, checkable load.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
of the same pipeline on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

SRC_W, SRC_H = 1920, 1080
IN_W, IN_H = 1088, 608
STRIDES = (32, 16, 8)
METRIC = "JDE FPS at 1088x608: BF16/FP8 batched vs FP32 plain on one GB300; p99 latency"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the 78 conv launches of one BF16
# batch-16 step, from one ncu capture of this build; re-take it (or set None) when the conv kernels change
CONV_DRAM_BYTES_PER_STEP = 8.462e9   # ncu dram__bytes_read.sum + dram__bytes_write.sum, 77 conv launches, autotuned tiles
CONV_DRAM_SOURCE = "profiles/dram_bf16_b16_1088x608.md (autotuned tiles, the profiled step of this bench)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--batch", type=int, default=16)
    p.add_argument("--objects", type=int, default=50)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp32", action="store_true")
    p.add_argument("--soak", type=int, default=40, help="untimed steps while the clock sampler starts")
    p.add_argument("--serve-seconds", type=float, default=20.0,
                   help="serving run: seconds of Poisson arrivals measured after a 2 s warm-up (0: skip)")
    p.add_argument("--serve-budget-gb", type=float, default=64.0, help="serving run: device memory budget")
    p.add_argument("--no-fp8", action="store_true", help="skip the E4M3 batch-32 line")
    p.add_argument("--no-jpeg", action="store_true", help="skip the compressed-frame (device decode) e2e line")
    p.add_argument("--no-autotune", action="store_true", help="default tile rule instead of jde_autotune")
    p.add_argument("--profile-step", action="store_true",
                   help="after the warm-up, run one step inside cudaProfilerStart/Stop (for ncu --profile-from-start "
                        "off) and exit without timing")
    p.add_argument("--dependent-launch", type=int, default=-1, choices=[-1, 0, 1],
                   help="jde_config.dependent_launch of the BF16 handles in the single-forward-stream steps "
                        "(-1: the library default)")
    p.add_argument("--fp8-dependent-launch", type=int, default=-1, choices=[-1, 0, 1],
                   help="dependent_launch of the E4M3 handles (-1: the library default)")
    p.add_argument("--pipeline-dependent-launch", type=int, default=0, choices=[0, 1],
                   help="dependent_launch of the two BF16 handles while two forward streams share the GPU")
    p.add_argument("--latency-batches", type=int, default=220,
                   help="batches of the pipelined step whose latency percentiles are reported (0: skip)")
    return p.parse_args()


# ----------------------------------------------------------------------------- helpers
def conv_flops(table, in_w, in_h):
    """2*M*N*K summed over the layer table (spatial sizes follow the DarkNet-53 + FPN chain)."""
    sizes = [(in_h, in_w)]
    h, w = in_h, in_w
    for nb in (1, 2, 8, 8, 4):
        h, w = (h + 1) // 2, (w + 1) // 2
        sizes += [(h, w)] * (1 + 2 * nb)
    for i, s in enumerate(STRIDES):
        sizes += [(in_h // s, in_w // s)] * (9 if i < 2 else 8)
    return sum(2 * hh * ww * co * ci * k * k for (ci, co, k, _, _, _), (hh, ww) in zip(table, sizes))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the GPU is under load."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
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
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def whole_job_rate(units_per_rank, local_ms, dist=None, device=None):
    """Replicas: every rank processed `units_per_rank` units in `local_ms`; the job took the
    slowest rank's time.  Returns (units/s over all ranks, max ms)."""
    ms = local_ms
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_rank / (ms / 1000.0), ms


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def planted_clips(n_streams, n_frames, n_obj, anchors, ratio, px, py):
    import synth
    return [synth.PlantedClip(100 + s, n_obj, n_frames, IN_W, IN_H, anchors, STRIDES, ratio, px, py)
            for s in range(n_streams)]


def anchor_table():
    """Anchor (w, h) per head as the library's decode uses them (pedestrian 1:3, sqrt(2) steps)."""
    return [[(b * 2 ** (i / 2), 3 * b * 2 ** (i / 2)) for i in range(4)] for b in (128.0, 32.0, 8.0)]


def letterbox_geometry(src_w, src_h, dst_w, dst_h):
    import math
    r = min(dst_w / src_w, dst_h / src_h)
    nw, nh = int(math.floor(src_w * r + 0.5)), int(math.floor(src_h * r + 0.5))
    return r, (dst_w - nw) // 2, (dst_h - nh) // 2


def build_heads_device(torch, clips, t, device):
    """Dense planted head tensors for frame t of every stream, built in HBM from the sparse entries."""
    B = len(clips)
    grids = [(IN_H // s, IN_W // s) for s in STRIDES]
    dets = []
    embs = []
    for (gh, gw) in grids:
        d = torch.zeros((B, gh, gw, 24), dtype=torch.float32, device=device)
        d[..., 4::6] = -6.0
        dets.append(d)
        embs.append(torch.zeros((B, gh, gw, 512), dtype=torch.float32, device=device))
    for b, c in enumerate(clips):
        det_e, emb_e, _ = c.frame_entries(t)
        for s in range(3):
            de = [e for e in det_e if e[0] == s]
            if de:
                ys = torch.tensor([e[1] for e in de], device=device)
                xs = torch.tensor([e[2] for e in de], device=device)
                ch = torch.tensor([[6 * e[3] + k for k in range(6)] for e in de], device=device)
                vals = torch.tensor([e[4] for e in de], dtype=torch.float32, device=device)
                dets[s][b][ys[:, None], xs[:, None], ch] = vals
            ee = [e for e in emb_e if e[0] == s]
            if ee:
                ys = torch.tensor([e[1] for e in ee], device=device)
                xs = torch.tensor([e[2] for e in ee], device=device)
                embs[s][b][ys, xs] = torch.from_numpy(np.stack([e[3] for e in ee])).to(device)
    return dets + embs


def run_fp8(torch, jde, dev, blob, stream, table, B=32, K=20, autotune=True, sparse_emb=0, dependent_launch=-1):
    """E4M3 network at 1088x608, batch 32: activation amax from 64 seeded calibration frames run through
    a BF16 handle that keeps every layer output (jde_act_amax, elementwise max over 4 batches of 16),
    then letterbox + forward + decode + confidence filter + NMS (jde_detect_batch) captured in one
    CUDA graph and replayed."""
    import synth
    amax = None
    ccfg = jde.jde_default_config()
    ccfg.precision = jde.JDE_BF16
    ccfg.max_batch = 16
    ccfg.max_streams = 1
    ccfg.device = dev.index or 0
    ccfg.keep_layer_outputs = 1
    ccfg.sparse_emb = 0
    hc = jde.jde_create(ccfg, blob)
    for i in range(4):
        cal = torch.from_numpy(synth.frames_uniform(1000 + i, 16, SRC_H, SRC_W)).to(dev)
        jde.jde_forward(hc, cal, 16, SRC_W, SRC_H, IN_W, IN_H, True, stream)
        a = jde.jde_act_amax(hc, stream)
        amax = a if amax is None else [max(u, v) for u, v in zip(amax, a)]
        del cal
    jde.jde_destroy(hc)
    cfg = jde.jde_default_config()
    cfg.precision = jde.JDE_FP8_E4M3
    cfg.max_batch = B
    cfg.max_streams = 1
    cfg.device = dev.index or 0
    if dependent_launch >= 0:
        cfg.dependent_launch = dependent_launch
    # synthetic weights on noise frames keep ~1600 detections per frame after NMS (256 rows kept per
    # frame here); at that count the dense embedding maps cost less than the sparse head
    cfg.sparse_emb = sparse_emb
    h8 = jde.jde_create(cfg, blob)
    jde.jde_set_act_amax(h8, amax)
    changed = None
    if autotune:
        d0 = jde.jde_tile_choice(h8, B, IN_W, IN_H)
        jde.jde_autotune(h8, B, IN_W, IN_H, stream)
        changed = sum(a != b for a, b in zip(d0, jde.jde_tile_choice(h8, B, IN_W, IN_H)))
    frames = [torch.from_numpy(synth.frames_uniform(2000 + i, B, SRC_H, SRC_W)).to(dev) for i in range(2)]
    cap = 256
    rows = torch.zeros((B, cap, 518), dtype=torch.float32, device=dev)
    count = torch.zeros(B, dtype=torch.int32, device=dev)
    dets = jde.make_dets(rows, count, None, cap=cap)
    gs = torch.cuda.Stream(device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for e in ev:
        e.record(gs)
    with torch.cuda.stream(gs):
        for t in range(3):           # first calls allocate; the captured calls then allocate nothing
            jde.jde_detect_batch(h8, frames[t % 2], B, SRC_W, SRC_H, IN_W, IN_H, dets, True, gs)
        # conv phase, eager, for the roofline
        jde.jde_set_profile_events(h8, *ev)
        jde.jde_forward(h8, frames[0], B, SRC_W, SRC_H, IN_W, IN_H, True, gs)
        jde.jde_set_profile_events(h8, None, None, None)
    torch.cuda.synchronize()
    conv_ms = ev[1].elapsed_time(ev[2])
    graphs = []
    for i in range(2):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=gs):
            jde.jde_detect_batch(h8, frames[i], B, SRC_W, SRC_H, IN_W, IN_H, dets, True, gs)
        graphs.append(g)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(gs):
        for i in range(3):
            graphs[i % 2].replay()
        torch.cuda.synchronize()
        e0.record(gs)
        for i in range(K):
            graphs[i % 2].replay()
        e1.record(gs)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1) / K
    # the timed form: two handles (same weights, scales and tiles), each with its own graph on its own
    # stream, batches alternating, so one batch's forward fills the last waves of the other's layers
    h8b = jde.jde_create(cfg, blob)
    jde.jde_set_act_amax(h8b, amax)
    jde.jde_set_tile_choice(h8b, B, IN_W, IN_H, jde.jde_tile_choice(h8, B, IN_W, IN_H))
    rows_b = torch.zeros_like(rows)
    count_b = torch.zeros_like(count)
    dets_b = jde.make_dets(rows_b, count_b, None, cap=cap)
    gs2 = [gs, torch.cuda.Stream(device=dev)]
    with torch.cuda.stream(gs2[1]):
        for t in range(3):
            jde.jde_detect_batch(h8b, frames[1], B, SRC_W, SRC_H, IN_W, IN_H, dets_b, True, gs2[1])
    torch.cuda.synchronize()
    gb = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gb, stream=gs2[1]):
        jde.jde_detect_batch(h8b, frames[1], B, SRC_W, SRC_H, IN_W, IN_H, dets_b, True, gs2[1])
    pair = [graphs[0], gb]
    for i in range(4):
        with torch.cuda.stream(gs2[i % 2]):
            pair[i % 2].replay()
    torch.cuda.synchronize()
    l0 = jde.jde_launch_count()
    e0.record(gs2[0])
    gs2[1].wait_event(e0)
    for i in range(K):
        with torch.cuda.stream(gs2[i % 2]):
            pair[i % 2].replay()
    j1 = torch.cuda.Event()
    j1.record(gs2[1])
    gs2[0].wait_event(j1)
    e1.record(gs2[0])
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    assert jde.jde_kernel_errors(h8) == 0 and jde.jde_kernel_errors(h8b) == 0
    n_dets = int(count.sum())
    jde.jde_destroy(h8)
    jde.jde_destroy(h8b)
    flops = conv_flops(table, IN_W, IN_H) * B
    peak8 = fp8_gemm_peak(torch)
    peaks, _ = measured_peaks()
    achieved = flops / (conv_ms * 1e-3) / 1e12
    return {"fps": B * 1000.0 / ms, "ms_per_batch": ms, "batch": B, "steps": K, "graph": True,
            "streams": "two handles, one CUDA graph each, replayed on two streams with batches alternating",
            "fps_single_stream": B * 1000.0 / ms1,
            "dependent_launch": int(cfg.dependent_launch),
            "autotuned_tiles_changed": changed,
            "what": "letterbox + E4M3 forward + decode + confidence filter + NMS + embedding L2, one CUDA graph "
                    "per batch; two handles with a graph each, replayed on two streams with batches alternating",
            "calibration": "amax per layer output: 64 seeded 1920x1080 uniform frames through a BF16 handle that keeps every layer output",
            "conv_ms": conv_ms, "conv_tflops": achieved,
            "fp8_peak_tflops": peak8, "conv_frac_of_fp8_peak": achieved / peak8 if peak8 else None,
            "fp8_peak_derived_tflops": 2.0 * peaks["bf16_tflops"],
            "conv_frac_of_fp8_peak_derived": achieved / (2.0 * peaks["bf16_tflops"]),
            "peak_note": "fp8_peak_tflops: measured in this run, torch._scaled_mm (cuBLASLt) E4M3 x E4M3 -> bf16 "
                         "GEMM, 8192^3, per-tensor scales, best of 30 launches; fp8_peak_derived_tflops: the measured "
                         "BF16 burst peak x 2 (nominal dense E4M3 / BF16 ratio 4.5 / 2.25)",
            "detections_last_batch": n_dets, "launch_count_note": "graph replays; library launches are inside graphs"}


def fp8_gemm_peak(torch, n=8192, reps=30):
    """Dense E4M3 tensor-core peak on this GPU, TFLOP/s: the best of `reps` cuBLASLt GEMMs
    (torch._scaled_mm, E4M3 x E4M3 -> bf16, per-tensor scales of 1) of n x n x n, timed with CUDA events
    after ten untimed ones."""
    a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
    b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
    one = torch.tensor(1.0, device="cuda")
    f = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
    for _ in range(10):
        f()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n * n * n / (best * 1e-3) / 1e12


def run_jpeg_e2e(torch, jde, dev, hs, F, P, D, heads, tracks_h, streams, B, K, post_done, fwd_done, t0):
    """The pipelined step fed by Motion-JPEG bitstreams from host memory: per batch, the decoder of its
    forward stream decodes B frames into that handle's device frame buffer, then forward, post-processing
    and tracker step (host track outputs) as in the e2e line.  Also the decoder alone: B frames per
    call, one stream, CUDA events."""
    import synth
    try:
        decs = [jde.jde_decoder_create(dev.index or 0, B, True) for _ in range(2)]
    except jde.JdeError as e:
        return {"unavailable": f"nvJPEG: {e}"}
    backend = {1: "hardware JPEG engines", 2: "GPU-assisted hybrid"}.get(jde.jde_decoder_backend(decs[0]), "?")
    src = torch.from_numpy(synth.frames_smooth(3000, B, SRC_H, SRC_W)).to(dev)
    bits = jde.jde_encode_jpeg(decs[0], src, B, SRC_W, SRC_H, 90, F[0])
    del src
    dframes = [torch.empty((B, SRC_H, SRC_W, 3), dtype=torch.uint8, device=dev) for _ in range(2)]
    torch.cuda.synchronize()
    # decoder alone
    for _ in range(3):
        jde.jde_decode_jpeg(decs[0], bits, SRC_W, SRC_H, dframes[0], F[0])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nd = 10
    tt = time.perf_counter()
    e0.record(F[0])
    for _ in range(nd):
        jde.jde_decode_jpeg(decs[0], bits, SRC_W, SRC_H, dframes[0], F[0])
    e1.record(F[0])
    torch.cuda.synchronize()
    dec_wall = (time.perf_counter() - tt) / nd
    dec_ms = e0.elapsed_time(e1) / nd

    # A decode call returns when its batch is decoded, so each forward stream has a host thread that
    # decodes its batches ahead: batch u is decoded (on F[u % 2]) once forward u - 2, which read the
    # same frame buffer, has been enqueued before it on that stream; the main thread enqueues forward u
    # once decode u has returned.  ctypes releases the GIL during the calls.
    import threading
    decoded = {}
    fwd_enq = {}

    def ev(dct, u):
        return dct.setdefault(u, threading.Event())

    def decoder_loop(f, first, last):
        for u in range(first + f, last, 2):
            if u - 2 >= first and not ev(fwd_enq, u - 2).wait(60):
                return
            jde.jde_decode_jpeg(decs[f], bits, SRC_W, SRC_H, dframes[f], F[f])
            ev(decoded, u).set()

    def fwd_jpeg(u):
        f = u % 2
        if not ev(decoded, u).wait(60):
            raise RuntimeError("decode thread stalled")
        if u - 4 in post_done:
            F[f].wait_event(post_done[u - 4])
        jde.jde_forward(hs[f], dframes[f], B, SRC_W, SRC_H, IN_W, IN_H, True, F[f])
        e = fwd_done[u] = torch.cuda.Event()
        e.record(F[f])
        ev(fwd_enq, u).set()

    def run(first, n, timed):
        threads = [threading.Thread(target=decoder_loop, args=(f, first, first + n), daemon=True) for f in range(2)]
        for th in threads:
            th.start()
        fwd_jpeg(first)
        if n > 1:
            fwd_jpeg(first + 1)
        for i in range(n):
            u = first + i
            P.wait_event(fwd_done[u])
            d = D[u % 2]
            jde.jde_postprocess(hs[u % 2], heads[u % len(heads)], B, IN_W, IN_H, SRC_W, SRC_H, d, P)
            e = post_done[u] = torch.cuda.Event()
            e.record(P)
            if i + 2 < n:
                fwd_jpeg(u + 2)
            jde.jde_track_step(hs[0], streams, d, tracks_h, P)
        torch.cuda.synchronize()
        for th in threads:
            th.join(60)

    run(t0, 4, False)               # warm both decoders on their streams
    base = t0 + 4
    tt0 = time.perf_counter()
    run(base, K, True)
    secs = time.perf_counter() - tt0
    for d_ in decs:
        jde.jde_decoder_destroy(d_)
    nbytes = sum(len(b) for b in bits)
    return {"value": B * K / secs, "unit": "frames/s", "h2d_bytes_per_step": nbytes,
            "decoder": backend, "jpeg_quality": 90, "mean_bitstream_bytes": nbytes / B,
            "decode_only": {"fps": B * 1000.0 / dec_ms, "ms_per_batch": dec_ms, "host_ms_per_call": dec_wall * 1000},
            "what": "Motion-JPEG bitstreams (synth.frames_smooth, 1920x1080) in host memory decoded on the device "
                    "into each forward stream's frame buffer, then the pipelined detect + track step, tracks to host"}


def run_sparse_compare(torch, jde, dev, blob, stream, B=16, K=10):
    """jde_detect_batch on the network's own detections (letterbox, forward, decode, NMS, embeddings) with the
    dense embedding maps and with the sparse embedding head (tensor-core gathered GEMM at the kept
    detections): ms per batch of B frames and the detections kept."""
    import synth
    frames = torch.from_numpy(synth.frames_uniform(3000, B, SRC_H, SRC_W)).to(dev)
    out = {}
    for sparse in (0, 1):
        cfg = jde.jde_default_config()
        cfg.max_batch, cfg.max_streams, cfg.device, cfg.sparse_emb = B, 1, dev.index or 0, sparse
        h = jde.jde_create(cfg, blob)
        cap = 256
        rows = torch.zeros((B, cap, 518), dtype=torch.float32, device=dev)
        count = torch.zeros(B, dtype=torch.int32, device=dev)
        dets = jde.make_dets(rows, count, None, cap=cap)
        for _ in range(3):
            jde.jde_detect_batch(h, frames, B, SRC_W, SRC_H, IN_W, IN_H, dets, True, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            jde.jde_detect_batch(h, frames, B, SRC_W, SRC_H, IN_W, IN_H, dets, True, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        assert jde.jde_kernel_errors(h) == 0
        out["sparse" if sparse else "dense"] = {"ms_per_batch": e0.elapsed_time(e1) / K,
                                                "rows_kept": int(torch.clamp(count, max=cap).sum())}
        jde.jde_destroy(h)
    out["what"] = (f"jde_detect_batch, BF16 batch {B} at {IN_W}x{IN_H}, the network's own detections (rows capped at "
                   "256 per frame): dense embedding maps vs the sparse embedding head")
    return out


def run_serving(torch, jde, dev, blob, seconds, budget_gb, n_streams=16, warm_s=2.0):
    """Serving: 16 streams, Poisson arrivals at 30 fps each, input 1088x608 / 864x480 / 576x320 by stream,
    20 + 80u planted objects per stream; the library's native server (jde_server_*: admission by budget,
    continuous batching per input size, CUDA-graph replays) driven by paper_2011_03910_gb300.serve."""
    import synth
    from paper_2011_03910_gb300 import serve
    sizes = [(1088, 608), (864, 480), (576, 320)]
    g = np.random.Generator(np.random.PCG64(4))
    specs = [serve.StreamSpec(i, *sizes[i % 3], fps=30.0, n_objects=int(20 + 80 * g.uniform()), seed=4000 + i)
             for i in range(n_streams)]
    srv = serve.Server(jde, torch, dev, blob, budget_bytes=int(budget_gb * 1e9), caller_heads=True)
    total_s = seconds + warm_s
    T = 150
    for sp in specs:
        fr = torch.from_numpy(synth.frames_uniform(5000 + sp.stream_id, 4, SRC_H, SRC_W)).to(dev)
        r, px, py = serve.letterbox_geometry(SRC_W, SRC_H, sp.in_w, sp.in_h)
        clip = synth.PlantedClip(100 + sp.seed, sp.n_objects, T, sp.in_w, sp.in_h, serve.anchor_table(),
                                 serve.STRIDES, r, px, py, max_speed=min(3.0, 600.0 / (T - 1)))
        srv.open_stream(sp, [fr[k] for k in range(4)], heads=synth.PlantedHeadFrames(clip))
    reqs = serve.poisson_arrivals([sp for sp in specs if sp.stream_id in srv.streams], total_s, seed=4)
    # the planted entries of every frame are built (and copied to the device) before the clock starts
    for sp in specs:
        if sp.stream_id in srv.streams:
            srv.streams[sp.stream_id].heads.preload(torch, dev)
    l0 = jde.jde_launch_count()
    stats = srv.run(reqs, warm_s=warm_s)
    charged, held = srv.device_bytes()
    stats.update({"streams": n_streams, "admitted": len(srv.streams), "refused": list(srv.refused),
                  "offered_fps": 30.0 * len(srv.streams), "seconds": seconds, "warmup_s": warm_s,
                  "inputs": {f"{w}x{h}": sum(1 for sp in specs if (sp.in_w, sp.in_h) == (w, h)) for w, h in sizes},
                  "device_bytes_charged": charged, "device_bytes_held": held, "budget_bytes": srv.budget,
                  "host_launches": int(jde.jde_launch_count() - l0), "server": srv.stats(),
                  "what": "latency per frame: device time its batch finished minus its Poisson arrival; "
                          "fps = frames served / time from the end of warm-up to the last frame's completion; "
                          "host_launches counts kernels launched eagerly (graph replays launch theirs from "
                          "the graph)"})
    # capacity: the same streams with every frame released at once (batches fill to max_batch per size)
    sat = [serve.Request(0.0, sp.stream_id, k) for k in range(60) for sp in specs if sp.stream_id in srv.streams]
    st2 = srv.run(sat, realtime=False)
    stats["saturated_fps"] = st2["fps"]
    stats["server_after_saturation"] = srv.stats()
    for sp in specs:
        if sp.stream_id in srv.streams:
            srv.close_stream(sp.stream_id)
    srv.close()
    return stats


# ----------------------------------------------------------------------------- reference arm
def cpu_oracle_frames(n_frames, seed_base=7):
    """Time the FP64 oracle pipeline (letterbox, network, post-processing, tracker step) on
    n_frames 1920x1080 frames at 1088x608, one frame per step; returns per-frame seconds."""
    import synth
    from oracle import network as net
    from oracle import postprocess as pp
    from oracle import tracker as tk
    layers = synth.parse_blob(synth.weights_blob(net.layer_specs()))
    r, nw, nh, px, py = net.letterbox_geometry(SRC_W, SRC_H, IN_W, IN_H)
    clip = synth.PlantedClip(100, 50, max(n_frames, 1), IN_W, IN_H, pp.anchors(), pp.STRIDES, r, px, py)
    T = tk.Tracker()
    times = []
    for i in range(n_frames):
        frame = synth.frames_uniform(seed_base, 1, SRC_H, SRC_W, first=i)
        dets_p, embs_p, _ = clip.frame(i)
        t0 = time.perf_counter()
        x = net.letterbox(frame, IN_W, IN_H)
        net.forward(x, layers)
        out = pp.postprocess_frame(dets_p, embs_p, r, px, py)
        T.step(out["rows"])
        times.append(time.perf_counter() - t0)
    return times


def run_reference(args, rank):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    times = cpu_oracle_frames(steps + warm)[warm:]
    total = sum(times)
    v = steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1000 * total / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "JDE FP64 CPU oracle, 1088x608 letterboxed from 1920x1080 uint8, one frame per step"
                   ", 50 planted objects for post-processing + tracking", "batch": 1, "in": [IN_W, IN_H]},
        "cpu_baseline": {"value": v, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{steps} frames, one per step"},
        "e2e": {"value": v, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    import synth
    from paper_2011_03910_gb300 import _build
    _build.build()
    from paper_2011_03910_gb300 import jde

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    B, K, W = args.batch, args.steps, args.warmup
    table = jde.jde_layer_table()
    blob = synth.weights_blob(table)
    cfg = jde.jde_default_config()
    cfg.precision = jde.JDE_BF16
    cfg.max_batch = B
    cfg.max_streams = B
    cfg.device = local
    # the timed post-processing reads planted head maps (embeddings included): the forward computes
    # the network's dense embedding maps too, so no part of the network is skipped
    cfg.sparse_emb = 0
    if args.dependent_launch >= 0:
        cfg.dependent_launch = args.dependent_launch
    h = jde.jde_create(cfg, blob)
    st = torch.cuda.current_stream()
    tiles = None
    if not args.no_autotune:
        default_bn = jde.jde_tile_choice(h, B, IN_W, IN_H)
        jde.jde_autotune(h, B, IN_W, IN_H, st)
        tuned_bn = jde.jde_tile_choice(h, B, IN_W, IN_H)
        tiles = {"autotuned": True, "changed_layers": sum(a != b for a, b in zip(default_bn, tuned_bn)),
                 "bn": tuned_bn}

    # inputs resident in HBM: 4 distinct batches of frames, planted heads for every step
    NF = 4
    frames = [torch.from_numpy(synth.frames_uniform(1000 * (rank + 1) + i, B, SRC_H, SRC_W)).to(dev)
              for i in range(NF)]
    ratio, px, py = letterbox_geometry(SRC_W, SRC_H, IN_W, IN_H)
    soak = args.soak
    K1 = 10                     # single-forward-stream steps that time the conv phase (kernel roofline)
    n_heads = W + K1 + soak + K   # planted heads of every step up to the end of the timed region
    clips = planted_clips(B, n_heads, args.objects, anchor_table(), ratio, px, py)
    heads = [build_heads_device(torch, clips, t, dev) for t in range(n_heads)]
    cap = 256
    rows = torch.zeros((B, cap, 518), dtype=torch.float32, device=dev)
    count = torch.zeros(B, dtype=torch.int32, device=dev)
    dets = jde.make_dets(rows, count, None, cap=cap)
    tcap = 256
    tr = [torch.zeros((B, tcap), dtype=torch.int64, device=dev), torch.zeros((B, tcap, 4), device=dev),
          torch.zeros((B, tcap), dtype=torch.int32, device=dev), torch.zeros((B, tcap), dtype=torch.int32, device=dev),
          torch.zeros(B, dtype=torch.int32, device=dev)]
    tracks = jde.make_tracks(*tr, cap=tcap)
    streams = list(range(B))

    # The pipelined step.  Two forward streams F[0], F[1] over two handles with the same weights and
    # tiles (each with its own activation buffers): batch t runs its forward on handle t % 2, so the
    # forward of batch t+1 fills the SMs that the last wave of each layer of batch t leaves idle.  One
    # stream P post-processes and tracks the batches in order (the paper's parallel post-processing,
    # Sec. 4.3, on the device) with the first handle's tracker, so every video stream's tracks live in
    # one state.  P waits for forward t; a handle's next-but-one forward (which reuses the head-tensor
    # set of batch t) waits for post-processing t.  nf = 1 is the single-forward-stream form.
    h2 = jde.jde_create(cfg, blob)
    jde.jde_set_tile_choice(h2, B, IN_W, IN_H, jde.jde_tile_choice(h, B, IN_W, IN_H))
    hs = [h, h2]
    F = [torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)]
    P = torch.cuda.Stream(device=dev)
    rows_b = torch.zeros_like(rows)
    count_b = torch.zeros_like(count)
    D = [dets, jde.make_dets(rows_b, count_b, None, cap=cap)]
    fwd_start, fwd_done, post_done = {}, {}, {}

    def step(t, nf, prof=None):
        f = t % nf
        hh = hs[f]
        if t - 2 * nf in post_done:
            F[f].wait_event(post_done[t - 2 * nf])
        if prof is not None and t - 1 in post_done:
            # timed conv phase: no post-processing or tracker kernel of the step before shares the GPU
            F[f].wait_event(post_done[t - 1])
        if prof is not None:
            jde.jde_set_profile_events(hh, *prof)
        e = fwd_start[t] = torch.cuda.Event(enable_timing=True)
        e.record(F[f])
        jde.jde_forward(hh, frames[t % NF], B, SRC_W, SRC_H, IN_W, IN_H, True, F[f])
        e = fwd_done[t] = torch.cuda.Event()
        e.record(F[f])
        P.wait_event(e)
        d = D[t % 2]
        jde.jde_postprocess(hh, heads[t % len(heads)], B, IN_W, IN_H, SRC_W, SRC_H, d, P)
        jde.jde_track_step(h, streams, d, tracks, P)
        e = post_done[t] = torch.cuda.Event(enable_timing=True)
        e.record(P)

    def drain():
        torch.cuda.synchronize()
        fwd_start.clear()
        fwd_done.clear()
        post_done.clear()

    t = 0
    for _ in range(W):
        step(t, 2)
        t += 1
    drain()
    if args.profile_step:
        # one single-stream step (forward, post-processing, tracker) inside the profiler range, then stop
        torch.cuda.profiler.start()
        step(t, 1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        assert jde.jde_kernel_errors(h) == 0
        jde.jde_destroy(h)
        jde.jde_destroy(h2)
        print(json.dumps({"profile_step": True, "batch": B, "tiles": tiles}), flush=True)
        return

    # kernel roofline: the conv phase of single-stream steps, timed with the CUDA events the library
    # records around the convolutions of each forward (no other forward, post-processing or tracker
    # kernel overlaps them)
    prof = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K1)]
    for p3 in prof:          # torch creates the CUDA event on its first record; the library re-records it
        for e in p3:
            e.record(F[0])
    torch.cuda.synchronize()
    for i in range(K1):
        step(t, 1, prof[i])
        t += 1
    drain()
    for hh in hs:
        jde.jde_set_profile_events(hh)
    conv_ms1 = sum(p[1].elapsed_time(p[2]) for p in prof) / K1
    fwd_ms1 = sum(p[0].elapsed_time(p[2]) for p in prof) / K1
    # two forward streams: each fills the SMs the other's layer tails leave idle, which a dependent
    # launch (its CTAs set up early and wait on those SMs) would take from it
    single_dl = int(cfg.dependent_launch)
    for hh in hs:
        jde.jde_set_dependent_launch(hh, args.pipeline_dependent_launch)

    sampler = ClockSampler(local)
    sampler.start()
    for _ in range(args.soak):      # keeps the GPU loaded while the clock sampler starts
        step(t, 2)
        t += 1
    drain()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = jde.jde_launch_count()
    t_start.record(F[0])
    F[1].wait_event(t_start)
    P.wait_event(t_start)
    for i in range(K):
        step(t, 2)
        t += 1
    F[0].wait_event(post_done[t - 1])
    t_end.record(F[0])
    torch.cuda.synchronize()
    l1 = jde.jde_launch_count()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    assert jde.jde_kernel_errors(h) == 0 and jde.jde_kernel_errors(h2) == 0
    total_ms = t_start.elapsed_time(t_end)
    value, total_ms = whole_job_rate(B * K, total_ms, dist, dev)
    drain()

    # latency percentiles over LAT_BATCHES more batches of the same pipelined step (outside the timed
    # region): per batch, from the start of its forward to the end of its tracker step
    step_ms = []
    if rank == 0 and args.latency_batches > 0:
        nl = args.latency_batches
        t_lat = t
        for i in range(nl):
            step(t, 2)
            t += 1
        torch.cuda.synchronize()
        step_ms = [fwd_start[u].elapsed_time(post_done[u]) for u in range(t_lat, t)]
        drain()
    F0 = F[0]
    for hh in hs:
        jde.jde_set_dependent_launch(hh, single_dl)

    # batch sweep (the batches of the BF16 configuration): the single-forward-stream pipelined step on
    # n frames / n streams, one handle
    sweep = {}
    if rank == 0:
        for n in [b for b in (1, 4, 8, 16) if b <= B]:
            ks, ws = 10, 3
            ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(ks + ws)]
            ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(ks + ws)]
            evf = [torch.cuda.Event() for _ in range(ks + ws)]
            sub_dets = jde.make_dets(rows[:n], count[:n], None, cap=cap)
            sub_tr = jde.make_tracks(*[x[:n] for x in tr], cap=tcap)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            for i in range(ks + ws):
                if i == ws:
                    a0.record(F0)
                    P.wait_event(a0)
                tt = (W + i) % len(heads)
                if i >= 2:
                    F0.wait_event(ev1[i - 2])
                ev0[i].record(F0)
                jde.jde_forward(h, frames[i % NF][:n], n, SRC_W, SRC_H, IN_W, IN_H, True, F0)
                evf[i].record(F0)
                P.wait_event(evf[i])
                jde.jde_postprocess(h, [x[:n] for x in heads[tt]], n, IN_W, IN_H, SRC_W, SRC_H, sub_dets, P)
                jde.jde_track_step(h, list(range(n)), sub_dets, sub_tr, P)
                ev1[i].record(P)
            F0.wait_event(ev1[ks + ws - 1])
            a1.record(F0)
            torch.cuda.synchronize()
            lat = sorted(ev0[i].elapsed_time(ev1[i]) for i in range(ws, ws + ks))
            # device memory a handle sized for batches of n holds at this input size (the library's exact
            # allocation rule, evaluated on the host): the peak-HBM-versus-batch study
            mcfg = jde.jde_default_config()
            mcfg.precision, mcfg.max_batch, mcfg.max_streams, mcfg.sparse_emb = jde.JDE_BF16, n, n, 0
            sweep[str(n)] = {"fps": n * ks / (a0.elapsed_time(a1) / 1000.0), "p50_ms": lat[len(lat) // 2],
                             "p99_ms": lat[-1], "hbm_bytes": jde.jde_estimate_device_bytes(mcfg, IN_W, IN_H)}

        # batch 1 captured in one CUDA graph (forward + post-processing + tracker step): launch-bound regime
        g1_dets = jde.make_dets(rows[:1], count[:1], None, cap=cap)
        g1_tr = jde.make_tracks(*[x[:1] for x in tr], cap=tcap)
        gs = torch.cuda.Stream(device=dev)
        hd1 = [x[:1] for x in heads[W]]

        def one():
            jde.jde_forward(h, frames[0][:1], 1, SRC_W, SRC_H, IN_W, IN_H, True, gs)
            jde.jde_postprocess(h, hd1, 1, IN_W, IN_H, SRC_W, SRC_H, g1_dets, gs)
            jde.jde_track_step(h, [0], g1_dets, g1_tr, gs)

        with torch.cuda.stream(gs):
            for _ in range(3):
                one()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gs)
        for _ in range(20):
            one()
        e1.record(gs)
        torch.cuda.synchronize()
        eager_ms = e0.elapsed_time(e1) / 20
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            one()
        with torch.cuda.stream(gs):
            graph.replay()
            torch.cuda.synchronize()
            e0.record(gs)
            for _ in range(20):
                graph.replay()
            e1.record(gs)
        torch.cuda.synchronize()
        graph_ms = e0.elapsed_time(e1) / 20
        sweep["1_graph"] = {"fps": 1000.0 / graph_ms, "ms": graph_ms, "eager_ms": eager_ms}
        assert jde.jde_kernel_errors(h) == 0

    # roofline of the convolutions (tcgen05 implicit GEMM): algorithmic FLOPs / measured conv time of the
    # single-stream steps (each launch alone on the GPU); the pipelined aggregate is reported beside it
    flops_frame = conv_flops(table, IN_W, IN_H)
    peaks, peak_kind = measured_peaks()
    achieved = flops_frame * B / (conv_ms1 / 1000.0) / 1e12
    agg = flops_frame * B * K / (total_ms / 1000.0) / 1e12
    # the conv phase is a few ms of dense MMA inside a step whose clocks are sampled: against the burst
    # figure (a cuBLAS GEMM timed alone) while the SM clock stays at its maximum with no power cap, the
    # sustained one (a GEMM loop under the power cap) is reported beside it
    peak = peaks.get("bf16_tflops", 1900.0)
    peak_s = peaks.get("bf16_tflops_sustained", peak)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": CONV_DRAM_BYTES_PER_STEP if B == 16 else None,
                "traffic_unit": "bytes per step (77 conv launches), ncu dram__bytes_read.sum + dram__bytes_write.sum",
                "traffic_source": CONV_DRAM_SOURCE,
                "kernel": "stem_s2_kernel + conv_tc_kernel (77 launches per step, aggregated)",
                "conv_time": f"conv phase of {K1} single-forward-stream steps, {conv_ms1:.3f} ms per step, CUDA events "
                             "the library records around the convolutions on the launch stream; each step's forward "
                             "starts after the previous step's post-processing and tracker kernels, so the "
                             "convolutions run alone",
                "peak_kind": f"{peak_kind} bf16 burst (of measured)",
                "peak_sustained": peak_s, "frac_sustained": achieved / peak_s,
                "pipelined": {"achieved": agg, "frac": agg / peak, "frac_sustained": agg / peak_s,
                              "how": "conv FLOPs of the timed region / its wall time (two forward streams; the "
                                     "wall time also covers the letterbox, post-processing and tracker kernels)"}}

    # e2e: host frames in (pinned), tracks out to host, through the same C ABI and the same two-handle
    # pipeline: jde_forward copies each batch's frames from pinned host memory on its forward stream
    for hh in hs:
        jde.jde_set_dependent_launch(hh, args.pipeline_dependent_launch)
    pinned = [f.cpu().pin_memory() for f in frames]
    tr_h = [np.zeros((B, tcap), np.int64), np.zeros((B, tcap, 4), np.float32), np.zeros((B, tcap), np.int32),
            np.zeros((B, tcap), np.int32), np.zeros(B, np.int32)]
    tracks_h = jde.make_tracks(*tr_h, cap=tcap, on_device=False)
    h2d = B * SRC_W * SRC_H * 3
    d2h = sum(x.nbytes for x in tr_h)
    torch.cuda.synchronize()

    def fwd_host(u):
        f = u % 2
        if u - 4 in post_done:
            F[f].wait_event(post_done[u - 4])
        jde.jde_forward(hs[f], pinned[u % NF], B, SRC_W, SRC_H, IN_W, IN_H, False, F[f])
        e = fwd_done[u] = torch.cuda.Event()
        e.record(F[f])

    tt0 = time.perf_counter()
    base = t
    fwd_host(base)
    fwd_host(base + 1)
    for i in range(K):
        u = base + i
        P.wait_event(fwd_done[u])
        d = D[u % 2]
        jde.jde_postprocess(hs[u % 2], heads[u % len(heads)], B, IN_W, IN_H, SRC_W, SRC_H, d, P)
        e = post_done[u] = torch.cuda.Event()
        e.record(P)
        if i + 2 < K:      # enqueue forward u+2 before the host waits on the tracks of u
            fwd_host(u + 2)
        jde.jde_track_step(h, streams, d, tracks_h, P)     # host outputs: synchronises P
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - tt0
    t = base + K
    drain()
    e2e = {"value": world * B * K / e2e_s, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # the first residual block fused into one kernel (fuse_block1 = 1): the same pipelined step on two
    # such handles, and the conv phase of single-stream steps, beside the default two-kernel form
    fused_block = None
    if rank == 0 and not args.no_jpeg:
        fcfg = jde.jde_config.from_buffer_copy(cfg)
        fcfg.fuse_block1 = 1
        fh = [jde.jde_create(fcfg, blob) for _ in range(2)]
        for x in fh:
            jde.jde_set_tile_choice(x, B, IN_W, IN_H, jde.jde_tile_choice(h, B, IN_W, IN_H))
        saved_hs = list(hs)
        hs[:] = fh
        for _ in range(W):
            step(t, 2)
            t += 1
        drain()
        fprof = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K1)]
        for p3 in fprof:
            for e in p3:
                e.record(F[0])
        for i in range(K1):
            step(t, 1, fprof[i])
            t += 1
        drain()
        for x in fh:
            jde.jde_set_profile_events(x)
        fconv = sum(p[1].elapsed_time(p[2]) for p in fprof) / K1
        for x in fh:
            jde.jde_set_dependent_launch(x, args.pipeline_dependent_launch)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(F[0])
        F[1].wait_event(f0)
        P.wait_event(f0)
        for i in range(K):
            step(t, 2)
            t += 1
        F[0].wait_event(post_done[t - 1])
        f1.record(F[0])
        torch.cuda.synchronize()
        assert all(jde.jde_kernel_errors(x) == 0 for x in fh)
        fms = f0.elapsed_time(f1) / K
        drain()
        hs[:] = saved_hs
        for x in fh:
            jde.jde_destroy(x)
        fused_block = {"fps_pipelined": B * 1000.0 / fms, "conv_ms_single_stream": fconv,
                       "default_fps_pipelined": value, "default_conv_ms_single_stream": conv_ms1,
                       "what": "fuse_block1 = 1 (layers 2-3 in one kernel, the 1x1 output on chip) against the default "
                               "two kernels: the same pipelined step (two handles) and single-stream conv phase"}

    # e2e from compressed frames: Motion-JPEG bitstreams in host memory (camera-like synthetic frames,
    # quality 90, 4:2:0), decoded on the device (jde_decode_jpeg) on each forward stream into that
    # handle's frame buffer, then the same pipeline; only the bitstreams cross the host link
    jpeg = None
    if rank == 0 and not args.no_jpeg:
        jpeg = run_jpeg_e2e(torch, jde, dev, hs, F, P, D, heads, tracks_h, streams, B, K, post_done, fwd_done, t)
        if "value" in jpeg:
            jpeg["d2h_bytes_per_step"] = d2h
        t += K + 4
        drain()

    # plain FP32 batch-1 comparator (no graph): same step, one frame / one stream
    fp32 = None
    if not args.no_fp32 and rank == 0:
        cfg32 = jde.jde_default_config()
        cfg32.precision = jde.JDE_FP32
        cfg32.max_batch = 1
        cfg32.max_streams = 1
        cfg32.device = local
        h32 = jde.jde_create(cfg32, blob)
        rows1 = torch.zeros((1, cap, 518), dtype=torch.float32, device=dev)
        count1 = torch.zeros(1, dtype=torch.int32, device=dev)
        dets1 = jde.make_dets(rows1, count1, None, cap=cap)
        tr1 = [x[:1].clone() for x in tr]
        tracks1 = jde.make_tracks(*tr1, cap=tcap)
        n32 = max(5, K // 2)

        def step32(t):
            jde.jde_forward(h32, frames[t % NF][:1], 1, SRC_W, SRC_H, IN_W, IN_H, True, st)
            jde.jde_postprocess(h32, [x[:1] for x in heads[t]], 1, IN_W, IN_H, SRC_W, SRC_H, dets1, st)
            jde.jde_track_step(h32, [0], dets1, tracks1, st)

        for t in range(3):
            step32(t)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(n32):
            step32(3 + i)
        e1.record(st)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1) / n32
        fp32 = {"fps": 1000.0 / ms32, "ms_per_frame": ms32, "steps": n32, "batch": 1, "graph": False}
        jde.jde_destroy(h32)

    sparse_cmp = None
    if rank == 0 and not args.no_fp8:
        sparse_cmp = run_sparse_compare(torch, jde, dev, blob, F0)

    fp8 = None
    if not args.no_fp8 and rank == 0:
        fp8 = run_fp8(torch, jde, dev, blob, F0, table, autotune=not args.no_autotune,
                      dependent_launch=args.fp8_dependent_launch)

    serving = None
    if args.serve_seconds > 0 and rank == 0:
        serving = run_serving(torch, jde, dev, blob, args.serve_seconds, args.serve_budget_gb)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ts = cpu_oracle_frames(1)
        cpu = {"value": 1.0 / ts[0], "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "1 frame 1920x1080 -> 1088x608: FP64 letterbox + network + post-processing + tracker step"}

    if rank == 0:
        srt = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"JDE BF16, 1920x1080 uint8 -> 1088x608 letterbox, batch {B} ({B} streams), "
                                   f"{args.objects} planted objects/stream for post-processing + tracking",
                       "batch": B, "in": [IN_W, IN_H], "src": [SRC_W, SRC_H], "parallelism": f"replicas{world}",
                       "dependent_launch": {"single_stream": single_dl, "pipelined": args.pipeline_dependent_launch},
                       "l2": "inputs larger than L2: ~5 GB of activations per step, 4 rotating 100 MB frame batches"},
            "latency_ms": {"p50": srt[len(srt) // 2] if srt else None,
                           "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))] if srt else None,
                           "batches": len(srt),
                           "what": "per batch, from the start of its forward to the end of its tracker step, "
                                   "in the timed pipeline (two forward streams over two handles, batches "
                                   "alternating; one stream post-processes and tracks them in order), over "
                                   "batches run after the timed region"},
            "pipeline": "two forward streams over two handles (same weights and tiles), batch t on handle t % 2; "
                        "post-processing and tracker steps in order on a third stream with one tracker state",
            "stages_ms_per_step_single_stream": {"forward": fwd_ms1, "convs": conv_ms1},
            "fp32_plain_batch1": fp32,
            "batch_sweep": sweep,
            "fp8_batch32": fp8,
            "sparse_embedding_head": sparse_cmp,
            "tiles": tiles,
            "serving": serving,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "e2e_jpeg": jpeg,
            "fused_first_block": fused_block,
            "gpu_launches": int(l1 - l0),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    jde.jde_destroy(h)
    jde.jde_destroy(h2)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

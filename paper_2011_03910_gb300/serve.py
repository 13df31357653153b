"""Serving loop: frames of many video streams through the library's native server.

The paper's system runs one video at a time and overlaps post-processing with
the next prediction (Sec. 4.3, Fig. 4).  The library's server (``jde_server_*``
in include/jde.h) serves many streams at once on one GPU: it groups streams by
model input size (one handle, CUDA stream and set of batch buffers per group),
admits a stream only if its group fits in a device-memory budget, batches the
queued frames of a group continuously (at most one frame per stream per batch,
since a stream's tracker steps are sequential) and replays each batch size's
launch sequence as a CUDA graph.  This module only releases frames at their
arrival times, submits them, polls the results and computes the statistics.

Latency of a frame is the device time at which its batch finished minus its
arrival time, both measured from the server's clock start.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

SRC_W, SRC_H = 1920, 1080
STRIDES = (32, 16, 8)
EMB_DIM = 512
JDE_ERR_ADMISSION = 5


def anchor_table():
    """Anchor (w, h) per head as the library's decode uses them (pedestrian 1:3, sqrt(2) steps)."""
    return [[(b * 2 ** (i / 2), 3 * b * 2 ** (i / 2)) for i in range(4)] for b in (128.0, 32.0, 8.0)]


def letterbox_geometry(src_w, src_h, dst_w, dst_h):
    r = min(dst_w / src_w, dst_h / src_h)
    nw, nh = int(math.floor(src_w * r + 0.5)), int(math.floor(src_h * r + 0.5))
    return r, (dst_w - nw) // 2, (dst_h - nh) // 2


@dataclass
class StreamSpec:
    stream_id: int
    in_w: int
    in_h: int
    fps: float = 30.0
    n_objects: int = 50
    seed: int = 0


@dataclass
class Request:
    t: float                 # arrival, seconds after the start
    stream_id: int
    index: int               # frame number within the stream
    done_ms: float = float("nan")
    outputs: dict = field(default_factory=dict)


def poisson_arrivals(specs, duration_s, seed):
    """Arrival times of every stream's frames: exponential gaps at the stream's rate (seeded)."""
    g = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for s in specs:
        t, k = 0.0, 0
        while True:
            t += g.exponential(1.0 / s.fps)
            if t >= duration_s:
                break
            reqs.append(Request(t, s.stream_id, k))
            k += 1
    reqs.sort(key=lambda r: (r.t, r.stream_id))
    return reqs


@dataclass
class _Stream:
    spec: StreamSpec
    sid: int                 # the server's stream id
    frames: list             # device tensors [SRC_H, SRC_W, 3] uint8, cycled
    heads: object = None     # caller heads: an object with write(torch, bufs, index)
    ring: list = None        # caller heads: RING sets of six device tensors
    ready: list = None       # caller heads: per ring set, the event recorded after it was written


class Server:
    """A ``jde_server`` and the streams opened on it (keyed by ``StreamSpec.stream_id``).

    With ``caller_heads`` every stream supplies its frames' head tensors through an object with a
    ``write(torch, bufs, index)`` method (e.g. planted objects, since random weights detect nothing in
    noise); the forward pass still does its full work on every frame.  A stream has at most ``RING``
    frames submitted and not yet returned, so its head tensors live in a ring of that many sets.
    """

    RING = 3

    def __init__(self, jde, torch, device, blob, budget_bytes, max_batch=16, max_streams_per_group=16,
                 det_cap=256, track_cap=256, precision=None, caller_heads=False, collect_net_heads=False,
                 use_graphs=True, prewarm=True):
        self.jde, self.torch, self.device = jde, torch, device
        cfg = jde.jde_default_server_config()
        cfg.group.precision = jde.JDE_BF16 if precision is None else precision
        cfg.group.max_batch = max_batch
        cfg.group.device = device.index or 0
        cfg.src_w, cfg.src_h = SRC_W, SRC_H
        cfg.max_streams_per_group = max_streams_per_group
        cfg.hbm_budget_bytes = int(budget_bytes)
        cfg.det_cap, cfg.track_cap = det_cap, track_cap
        cfg.caller_heads = int(caller_heads)
        cfg.collect_net_heads = int(collect_net_heads)
        cfg.use_graphs = int(use_graphs)
        cfg.prewarm = int(prewarm)
        self.cfg = cfg
        self.det_cap, self.track_cap = det_cap, track_cap
        self.caller_heads, self.collect_net_heads = caller_heads, collect_net_heads
        self.budget = int(budget_bytes)
        self.s = jde.jde_server_create(cfg, blob)
        self.streams = {}
        self.refused = []

    def close(self):
        if self.s is not None:
            self.jde.jde_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def group_cost(self, in_w, in_h):
        return self.jde.jde_server_group_cost(self.cfg, in_w, in_h)

    @staticmethod
    def grids(in_w, in_h):
        return [(in_h // s, in_w // s) for s in STRIDES]

    def open_stream(self, spec: StreamSpec, frames, heads=None) -> bool:
        """Admit a stream (frames: device tensors [1080, 1920, 3] uint8 that it cycles through).
        Returns False when the server refuses it (no free slot, or its group does not fit the budget)."""
        try:
            sid = self.jde.jde_stream_open(self.s, spec.in_w, spec.in_h)
        except self.jde.JdeError as e:
            if e.status != JDE_ERR_ADMISSION:
                raise
            self.refused.append(spec.stream_id)
            return False
        st = _Stream(spec, sid, list(frames))
        if self.caller_heads:
            if heads is None:
                raise ValueError("this server takes per-frame head tensors: pass heads")
            torch = self.torch
            st.heads = heads
            # one set: the three detection maps then the three embedding maps, each at its own grid
            st.ring = [[torch.empty((gh, gw, 24), dtype=torch.float32, device=self.device)
                        for gh, gw in self.grids(spec.in_w, spec.in_h)] +
                       [torch.empty((gh, gw, EMB_DIM), dtype=torch.float32, device=self.device)
                        for gh, gw in self.grids(spec.in_w, spec.in_h)] for _ in range(self.RING)]
            st.ready = [torch.cuda.Event() for _ in range(self.RING)]
        self.streams[spec.stream_id] = st
        return True

    def close_stream(self, stream_id):
        st = self.streams.pop(stream_id)
        self.jde.jde_stream_close(self.s, st.sid)

    def device_bytes(self):
        """(bytes charged to the budget, device bytes the groups hold)."""
        return self.jde.jde_server_device_bytes(self.s)

    def stats(self):
        e, c, r = self.jde.jde_server_stats(self.s)
        return {"eager_batches": e, "graphs_captured": c, "graph_replays": r}

    def _out_buffers(self, st: _Stream):
        tc, dc = self.track_cap, self.det_cap
        bufs = {"track_id": np.zeros(tc, np.int64), "track_box": np.zeros((tc, 4), np.float32),
                "track_state": np.zeros(tc, np.int32), "track_det": np.zeros(tc, np.int32),
                "rows": np.zeros((dc, 518), np.float32)}
        if self.collect_net_heads:
            bufs["net_det"] = [np.zeros((gh, gw, 24), np.float32) for gh, gw in self.grids(st.spec.in_w, st.spec.in_h)]
        return bufs

    def run(self, requests, collect=False, realtime=True, warm_s=0.0):
        """Serve the requests (sorted by arrival).  realtime: a request is released when the wall clock
        reaches its arrival time; otherwise all are released at once (arrival times then only order
        them).  Fills each request's done_ms (and outputs when collect) and returns summary statistics."""
        jde, torch = self.jde, self.torch
        reqs = [r for r in requests if r.stream_id in self.streams]
        pending = {k: collections.deque() for k in self.streams}
        outstanding = {k: 0 for k in self.streams}
        by_ticket = {}
        jde.jde_server_reset_clock(self.s)
        t0 = time.perf_counter()
        i, done_n = 0, 0
        while done_n < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].t <= now):
                pending[reqs[i].stream_id].append(reqs[i])
                i += 1
            batch = []
            for k, q in pending.items():
                while q and outstanding[k] < self.RING:
                    batch.append(q.popleft())
                    outstanding[k] += 1
            for r in batch:
                st = self.streams[r.stream_id]
                bufs = self._out_buffers(st) if collect else None
                out = jde.make_frame_out(**bufs) if bufs else None
                heads, ready = None, None
                if self.caller_heads:
                    # written on torch's stream; the server's copy of them waits for the event on the device
                    k = r.index % self.RING
                    heads, ready = st.ring[k], st.ready[k]
                    st.heads.write(torch, heads, r.index)
                    ready.record()
                t = jde.jde_submit(self.s, st.sid, st.frames[r.index % len(st.frames)], heads, out, ready)
                by_ticket[t] = (r, bufs, out)
            res = jde.jde_poll(self.s, 256)
            for x in res:
                r, bufs, _ = by_ticket.pop(x.ticket)
                r.done_ms = x.done_ms
                outstanding[r.stream_id] -= 1
                done_n += 1
                if bufs is not None:
                    k, nt = x.n_dets, x.n_tracks
                    r.outputs = {"count": k, "errors": x.errors, "rows": bufs["rows"][:min(k, self.det_cap)],
                                 "track_id": bufs["track_id"][:nt], "track_box": bufs["track_box"][:nt],
                                 "track_state": bufs["track_state"][:nt], "track_det": bufs["track_det"][:nt],
                                 "net_det": bufs.get("net_det")}
            if not res and not batch and realtime and i < len(reqs) and not by_ticket:
                time.sleep(max(0.0, min(0.0005, reqs[i].t - (time.perf_counter() - t0))))
        jde.jde_server_flush(self.s)
        wall = time.perf_counter() - t0
        timed = [r for r in reqs if r.t >= warm_s]
        lat = np.array([r.done_ms - 1000.0 * r.t for r in timed]) if realtime else np.array([r.done_ms for r in timed])
        span_ms = max(r.done_ms for r in reqs) - 1000.0 * warm_s if reqs else 0.0
        return {"frames": len(timed), "wall_s": wall, "fps": len(timed) / (span_ms / 1000.0) if span_ms > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None}

"""Serving loop: frames from many video streams, continuous batching, per-stream tracks.

The paper's system runs one video at a time and overlaps post-processing with
the next prediction (Sec. 4.3, Fig. 4).  This module serves many streams at
once on one GPU through the C ABI:

* **Groups.**  Streams are grouped by model input size.  Each group owns one
  library handle (weights, activation buffers for its size, post-processing
  scratch, and the tracker state of its streams, all device-resident) and one
  CUDA stream, so the groups' batches overlap on the device.  A handle is used
  by one group only, so its calls are naturally serialised.
* **Admission.**  A stream joins the group of its input size if that group has
  a free tracker slot; a new group is created only if its device memory
  (``jde_estimate_device_bytes`` plus the group's own frame/head/output
  buffers) fits in what the budget has left.  Otherwise the stream is refused.
  Closing the last stream of a group destroys its handle and returns its
  memory to the budget.
* **Continuous batching.**  A frame that arrives is queued in its group.  A
  group with no batch on the device takes every queued frame (at most
  ``max_batch``, at most one per stream since a stream's track steps are
  sequential) and launches forward + post-processing + tracker step on its
  CUDA stream; frames that arrive meanwhile form the next batch.
* **Latency** of a frame is the device time at which its tracker step
  finished minus its arrival time, both measured from a start event.

Every computation step runs in libjde's kernels; this module only schedules
calls and moves buffers.  Random weights detect nothing in noise, so (as in the
throughput benchmark) the post-processing and tracker consume planted head
tensors of the stream's input size, built per frame into the group's head
buffers; the forward pass does its full work on the frame.
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


def planted_entries(spec: StreamSpec, T: int):
    """Per frame of a T-frame planted clip at the stream's input size, per head: detection entries
    (y, x, anchor) + 6 values, embedding entries (y, x) + 512 values (compact numpy arrays)."""
    import synth
    r, px, py = letterbox_geometry(SRC_W, SRC_H, spec.in_w, spec.in_h)
    clip = synth.PlantedClip(100 + spec.seed, spec.n_objects, T, spec.in_w, spec.in_h, anchor_table(), STRIDES,
                             r, px, py, max_speed=min(3.0, 600.0 / (T - 1)))
    out = []
    for t in range(T):
        det_e, emb_e, _ = clip.frame_entries(t)
        per = []
        for s in range(3):
            de = [e for e in det_e if e[0] == s]
            ee = [e for e in emb_e if e[0] == s]
            yxa = np.array([(e[1], e[2], e[3]) for e in de], dtype=np.int64).reshape(-1, 3)
            vals = np.array([e[4] for e in de], dtype=np.float32).reshape(-1, 6)
            eyx = np.array([(e[1], e[2]) for e in ee], dtype=np.int64).reshape(-1, 2)
            evals = np.array([e[3] for e in ee], dtype=np.float32).reshape(-1, EMB_DIM)
            per.append((yxa, vals, eyx, evals))
        out.append(per)
    return out


class AdmissionLedger:
    """Device-memory budget: groups are charged when created and credited when destroyed."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.used = 0
        self.charges = {}

    def try_charge(self, key, nbytes: int) -> bool:
        if key in self.charges:
            return True
        if self.used + nbytes > self.budget:
            return False
        self.charges[key] = int(nbytes)
        self.used += int(nbytes)
        return True

    def credit(self, key):
        self.used -= self.charges.pop(key, 0)


class _Group:
    """One input size: a library handle, a CUDA stream, the member streams' tracker slots and buffers."""

    def __init__(self, server, in_w, in_h):
        jde, torch = server.jde, server.torch
        self.server, self.in_w, self.in_h = server, in_w, in_h
        cfg = server.group_config(in_w, in_h)
        self.h = jde.jde_create(cfg, server.blob)
        self.stream = torch.cuda.Stream(device=server.device)
        self.free_slots = list(range(cfg.max_streams))[::-1]
        self.slot_of = {}
        self.queue = collections.deque()
        self.inflight = collections.deque()
        B, dev = server.max_batch, server.device
        self.frames = torch.empty((B, SRC_H, SRC_W, 3), dtype=torch.uint8, device=dev)
        self.grids = [(in_h // s, in_w // s) for s in STRIDES]
        self.heads = ([torch.zeros((B, gh, gw, 24), dtype=torch.float32, device=dev) for gh, gw in self.grids] +
                      [torch.zeros((B, gh, gw, EMB_DIM), dtype=torch.float32, device=dev) for gh, gw in self.grids])
        cap = server.det_cap
        self.rows = torch.zeros((B, cap, 518), dtype=torch.float32, device=dev)
        self.count = torch.zeros(B, dtype=torch.int32, device=dev)
        self.dets = jde.make_dets(self.rows, self.count, None, cap=cap)
        tcap = server.track_cap
        self.tr = [torch.zeros((B, tcap), dtype=torch.int64, device=dev), torch.zeros((B, tcap, 4), device=dev),
                   torch.zeros((B, tcap), dtype=torch.int32, device=dev),
                   torch.zeros((B, tcap), dtype=torch.int32, device=dev), torch.zeros(B, dtype=torch.int32, device=dev)]
        self.tracks = jde.make_tracks(*self.tr, cap=tcap)

    @staticmethod
    def buffer_bytes(max_batch, in_w, in_h, det_cap, track_cap):
        """Device bytes of the group's own buffers (frames, planted heads, outputs)."""
        cells = sum((in_h // s) * (in_w // s) for s in STRIDES)
        return (max_batch * SRC_H * SRC_W * 3 + max_batch * cells * (24 + EMB_DIM) * 4 +
                max_batch * det_cap * 518 * 4 + max_batch * 4 + max_batch * track_cap * (8 + 16 + 4 + 4) + max_batch * 4)

    def destroy(self):
        self.server.torch.cuda.synchronize(self.server.device)
        self.server.jde.jde_destroy(self.h)
        self.h = None

    def _fill_heads(self, batch):
        """Planted head tensors of the batch's frames (on the group's stream): background everywhere,
        then each frame's precomputed entries, one scatter per head tensor for the whole batch."""
        torch, srv = self.server.torch, self.server
        n = len(batch)
        for s in range(3):
            self.heads[s][:n].zero_()
            self.heads[s][:n, ..., 4::6] = -6.0
            self.heads[3 + s][:n].zero_()
        for s, (gh, gw) in enumerate(self.grids):
            d_lin, d_val, e_row, e_val = [], [], [], []
            for b, r in enumerate(batch):
                ent = srv.entries[r.stream_id][r.index % len(srv.entries[r.stream_id])][s]
                yxa, vals, eyx, evals = ent
                if len(yxa):
                    cell = (b * gh + yxa[:, 0]) * gw + yxa[:, 1]
                    d_lin.append((cell[:, None] * 24 + 6 * yxa[:, 2:3] + np.arange(6)[None, :]).ravel())
                    d_val.append(vals.ravel())
                if len(eyx):
                    e_row.append((b * gh + eyx[:, 0]) * gw + eyx[:, 1])
                    e_val.append(evals)
            if d_lin:
                lin = torch.from_numpy(np.concatenate(d_lin)).to(srv.device, non_blocking=True)
                val = torch.from_numpy(np.concatenate(d_val)).to(srv.device, non_blocking=True)
                self.heads[s].view(-1)[lin] = val
            if e_row:
                rows = torch.from_numpy(np.concatenate(e_row)).to(srv.device, non_blocking=True)
                val = torch.from_numpy(np.concatenate(e_val)).to(srv.device, non_blocking=True)
                self.heads[3 + s].view(-1, EMB_DIM)[rows] = val

    def launch(self, collect):
        """Take queued frames (one per stream, at most max_batch) and run detect + track on the device."""
        srv, jde, torch = self.server, self.server.jde, self.server.torch
        batch, seen, rest = [], set(), collections.deque()
        while self.queue:
            r = self.queue.popleft()
            if r.stream_id in seen or len(batch) >= srv.max_batch:
                rest.append(r)
            else:
                batch.append(r)
                seen.add(r.stream_id)
        self.queue = rest
        n = len(batch)
        with torch.cuda.stream(self.stream):
            for b, r in enumerate(batch):
                self.frames[b].copy_(srv.frames[r.stream_id][r.index % len(srv.frames[r.stream_id])], non_blocking=True)
            self._fill_heads(batch)
        jde.jde_forward(self.h, self.frames, n, SRC_W, SRC_H, self.in_w, self.in_h, True, self.stream)
        heads_out = None
        if collect:
            # the network's own detection maps (the 24-channel 1x1 outputs) of this batch
            heads_out = []
            for tid in srv.det_layers:
                dims, _ = jde.jde_get_tensor(self.h, tid, None, 0, self.stream)
                t = torch.empty(tuple(dims), dtype=torch.float32, device=srv.device)
                jde.jde_get_tensor(self.h, tid, t, t.numel() * 4, self.stream)
                heads_out.append(t)
        jde.jde_postprocess(self.h, self.heads, n, self.in_w, self.in_h, SRC_W, SRC_H, self.dets, self.stream)
        jde.jde_track_step(self.h, [self.slot_of[r.stream_id] for r in batch], self.dets, self.tracks, self.stream)
        outs = None
        if collect:
            with torch.cuda.stream(self.stream):
                outs = [(self.count[:n].clone(), self.rows[:n].clone(), [x[:n].clone() for x in self.tr], heads_out)]
        done = torch.cuda.Event(enable_timing=True)
        done.record(self.stream)
        self.inflight.append((done, batch, outs))


class Server:
    """Continuous-batching JDE server over libjde handles (one per input size)."""

    def __init__(self, jde, torch, device, blob, budget_bytes, max_batch=16, max_streams_per_group=16,
                 det_cap=256, track_cap=256, precision=None):
        self.jde, self.torch, self.device = jde, torch, device
        self.blob = blob
        self.max_batch, self.max_streams = max_batch, max_streams_per_group
        self.det_cap, self.track_cap = det_cap, track_cap
        self.precision = jde.JDE_BF16 if precision is None else precision
        self.ledger = AdmissionLedger(budget_bytes)
        self.groups = {}
        self.group_of = {}
        self.frames = {}
        self.entries = {}
        self.refused = []
        self.det_layers = [i for i, d in enumerate(jde.jde_layer_table()) if d[1] == 24]

    def group_config(self, in_w, in_h):
        cfg = self.jde.jde_default_config()
        cfg.precision = self.precision
        cfg.max_batch = self.max_batch
        cfg.max_streams = self.max_streams
        cfg.max_in_w, cfg.max_in_h = in_w, in_h
        cfg.device = self.device.index or 0
        # the post-processing reads the planted head maps (embeddings included), so the forward
        # computes the network's dense embedding maps as well (nothing of the network is skipped)
        cfg.sparse_emb = 0
        return cfg

    def group_cost(self, in_w, in_h):
        return (self.jde.jde_estimate_device_bytes(self.group_config(in_w, in_h), in_w, in_h) +
                _Group.buffer_bytes(self.max_batch, in_w, in_h, self.det_cap, self.track_cap))

    def open_stream(self, spec: StreamSpec, frames, n_frames_hint=150) -> bool:
        """Admit a stream (frames: list of [1080,1920,3] uint8 device tensors it cycles through).  Its planted
        objects follow a clip of min(n_frames_hint, 150) frames that repeats (objects jump back at the wrap)."""
        key = (spec.in_w, spec.in_h)
        g = self.groups.get(key)
        if g is None:
            if not self.ledger.try_charge(key, self.group_cost(*key)):
                self.refused.append(spec.stream_id)
                return False
            g = self.groups[key] = _Group(self, *key)
        if not g.free_slots:
            self.refused.append(spec.stream_id)
            return False
        slot = g.free_slots.pop()
        self.jde.jde_stream_reset(g.h, slot, g.stream)
        g.slot_of[spec.stream_id] = slot
        self.group_of[spec.stream_id] = g
        self.frames[spec.stream_id] = frames
        self.entries[spec.stream_id] = planted_entries(spec, max(2, min(n_frames_hint, 150)))
        return True

    def close_stream(self, stream_id):
        g = self.group_of.pop(stream_id)
        g.free_slots.append(g.slot_of.pop(stream_id))
        self.frames.pop(stream_id, None)
        self.entries.pop(stream_id, None)
        if not g.slot_of:
            key = (g.in_w, g.in_h)
            g.destroy()
            del self.groups[key]
            self.ledger.credit(key)

    def device_bytes(self):
        return sum(self.jde.jde_device_bytes(g.h) for g in self.groups.values())

    def run(self, requests, collect=False, realtime=True, warm_s=0.0):
        """Serve the requests (sorted by arrival).  realtime: a request is released when the wall clock
        reaches its arrival time; otherwise all are released at once (arrival times then only order
        them).  Fills each request's done_ms (and outputs when collect) and returns summary statistics."""
        torch = self.torch
        reqs = [r for r in requests if r.stream_id in self.group_of]
        start = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(self.device)
        start.record()
        t0 = time.perf_counter()
        i, done_n = 0, 0
        groups = list(self.groups.values())
        while done_n < len(reqs):
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].t <= now):
                self.group_of[reqs[i].stream_id].queue.append(reqs[i])
                i += 1
            busy = False
            for g in groups:
                while g.inflight and g.inflight[0][0].query():
                    ev, batch, outs = g.inflight.popleft()
                    ms = start.elapsed_time(ev)
                    for b, r in enumerate(batch):
                        r.done_ms = ms
                        if outs is not None:
                            cnt, rows, tr, net_heads = outs[0]
                            k = int(cnt[b])
                            nt = int(tr[4][b])
                            r.outputs = {"count": k, "rows": rows[b, :min(k, self.det_cap)].cpu().numpy(),
                                         "track_id": tr[0][b, :nt].cpu().numpy(), "track_box": tr[1][b, :nt].cpu().numpy(),
                                         "track_state": tr[2][b, :nt].cpu().numpy(),
                                         "net_det": [x[b].cpu().numpy() for x in net_heads]}
                    done_n += len(batch)
                if not g.inflight and g.queue:
                    g.launch(collect)
                busy = busy or bool(g.inflight)
            if not busy and i < len(reqs) and realtime:
                time.sleep(max(0.0, min(0.0005, reqs[i].t - (time.perf_counter() - t0))))
        torch.cuda.synchronize(self.device)
        wall = time.perf_counter() - t0
        timed = [r for r in reqs if r.t >= warm_s]
        lat = np.array([r.done_ms - 1000.0 * r.t for r in timed]) if realtime else np.array([r.done_ms for r in timed])
        span_ms = max(r.done_ms for r in reqs) - 1000.0 * warm_s if reqs else 0.0
        return {"frames": len(timed), "wall_s": wall, "fps": len(timed) / (span_ms / 1000.0) if span_ms > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None}

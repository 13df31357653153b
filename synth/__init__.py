"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the bench.

This module draws random numbers and lays them out; it holds none of the
tracker's arithmetic (no convolution, no decode, no NMS, no Kalman step).
Everything the two implementations consume comes from here, so that both see
bit-identical inputs:

* ``frames_uniform``  - uint8 RGB frames, uniform on [0, 255] (the stand-in for
  the FullHD MOT16 frames the paper times on, Sec. 5.1).
* ``weights_blob``    - random-init JDE weights in the blob format that
  ``jde_create`` parses (He-normal convolution weights, seeded BN statistics).
* ``PlantedClip``     - head tensors with objects planted on constant-velocity
  paths, used to drive the post-processing and tracker (Appendix A steps).
* ``random_heads``    - dense random head tensors for decode / NMS stress.

Random streams are numpy PCG64 generators keyed by ``SeedSequence([seed, k])``
so that each layer, frame or object draws from its own independent stream.
"""
from __future__ import annotations

import json
import math
import os
import struct

import numpy as np

WEIGHT_SEED = 20110391
BLOB_MAGIC = b"JDEW"
BLOB_VERSION = 1
FLAG_BN = 1
FLAG_BIAS = 2

# Synthetic stand-in frame size: FullHD, the resolution of the MOT16 sequences
# the paper reports its speed on (Sec. 5.1).
SRC_W, SRC_H = 1920, 1080


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(k) for k in key])))


# --------------------------------------------------------------------------- frames
def frames_uniform(seed: int, n: int, h: int, w: int, first: int = 0) -> np.ndarray:
    """``n`` uint8 RGB frames ``[n, h, w, 3]``, uniform on [0, 255].

    Frame ``i`` of the sequence is drawn from stream ``(seed, first + i)`` so a
    long clip can be generated in pieces.
    """
    out = np.empty((n, h, w, 3), dtype=np.uint8)
    for i in range(n):
        out[i] = _rng(seed, first + i).integers(0, 256, size=(h, w, 3), dtype=np.uint8)
    return out


def frames_smooth(seed: int, n: int, h: int, w: int, first: int = 0, waves: int = 6, noise: float = 3.0) -> np.ndarray:
    """``n`` uint8 RGB frames ``[n, h, w, 3]`` with the spatial structure of camera frames rather than
    of noise (for compressed-stream inputs, whose size and decode cost depend on the content): per
    channel a mean level ~ U(60, 190) plus ``waves`` plane waves of amplitude ~ U(10, 35) and spatial
    period ~ U(40, 600) px in a random direction, plus N(0, ``noise``) per pixel, rounded and clipped to
    [0, 255].  Frame ``i`` is drawn from stream ``(seed, first + i, 7)``.
    """
    out = np.empty((n, h, w, 3), dtype=np.uint8)
    x = np.arange(w, dtype=np.float64)
    y = np.arange(h, dtype=np.float64)
    for i in range(n):
        g = _rng(seed, first + i, 7)
        img = np.empty((h, w, 3), np.float32)
        for c in range(3):
            v = np.full((h, w), g.uniform(60.0, 190.0), np.float64)
            for _ in range(waves):
                amp, period, ang, ph = g.uniform(10, 35), g.uniform(40, 600), g.uniform(0, np.pi), g.uniform(0, 2 * np.pi)
                k = 2 * np.pi / period
                a = k * np.cos(ang) * x + ph           # cos(a + b) = cos a cos b - sin a sin b: separable
                b = k * np.sin(ang) * y
                v += amp * (np.outer(np.cos(b), np.cos(a)) - np.outer(np.sin(b), np.sin(a)))
            v += g.normal(0.0, noise, (h, w))
            img[..., c] = v
        out[i] = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    return out


# --------------------------------------------------------------------------- weights
def load_tobj_shift() -> list:
    """Per-(detection head, anchor) shift added to the objectness-logit bias.

    The values in ``tobj_bias.json`` are written by the oracle calibration
    script under ``tests/golden``; they make roughly 1% of anchors pass the 0.5
    confidence threshold on uniform frames (random weights would otherwise put
    about half of all anchors above it).
    """
    path = os.path.join(os.path.dirname(__file__), "tobj_bias.json")
    if not os.path.exists(path):
        return [[0.0] * 4 for _ in range(3)]
    with open(path) as f:
        return json.load(f)["shift"]


def weights_blob(specs, seed: int = WEIGHT_SEED, tobj_shift=None) -> bytes:
    """Random-init weights for the layer list ``specs`` as a blob.

    ``specs`` is a sequence of ``(cin, cout, k, stride, has_bn, res_nblocks)``:
    ``has_bn`` selects BN statistics (else a plain bias), ``res_nblocks`` is the
    block count of the residual stage when the convolution closes a residual
    branch (0 otherwise).

    Draws (per layer ``i``, stream ``(seed, i)``):
      W ~ N(0, 2 / fan_in) (He-normal), then for BN layers
      gamma ~ U(0.8, 1.2), beta ~ N(0, 0.05), mean ~ N(0, 0.05), var ~ U(0.8, 1.2);
      gamma is scaled by 1/(2 * res_nblocks) on branch-closing layers so the
      23 residual adds do not blow up the activations (the leaky-ReLU outputs
      have a positive mean that adds up coherently along the residual stream;
      with 1/sqrt(2 n) the head outputs reach std ~13).  Bias layers draw
      bias ~ N(0, 0.05); on the i-th 24-channel bias layer (the detection
      1x1 of head i), channel 6a+4 (anchor a's objectness logit) is shifted by
      ``tobj_shift[i][a]``.

    Blob layout (little-endian): a 16-byte header ``"JDEW", u32 version,
    u32 n_layers, u32 0`` then per layer a 32-byte header
    ``u32 cin, cout, k, stride, flags, 0, 0, 0`` (flags: 1 = BN, 2 = bias)
    followed by f32 ``W[cout][cin][k][k]`` and either
    ``gamma, beta, mean, var`` (each ``[cout]``) or ``bias[cout]``.
    """
    if tobj_shift is None:
        tobj_shift = load_tobj_shift()
    parts = [BLOB_MAGIC, struct.pack("<III", BLOB_VERSION, len(specs), 0)]
    det_i = 0
    for i, (cin, cout, k, stride, has_bn, res_nb) in enumerate(specs):
        g = _rng(seed, i)
        fan_in = cin * k * k
        w = g.standard_normal(cout * cin * k * k) * math.sqrt(2.0 / fan_in)
        flags = FLAG_BN if has_bn else FLAG_BIAS
        parts.append(struct.pack("<8I", cin, cout, k, stride, flags, 0, 0, 0))
        parts.append(w.astype("<f4").tobytes())
        if has_bn:
            gamma = g.uniform(0.8, 1.2, cout)
            if res_nb:
                gamma = gamma / (2.0 * res_nb)
            beta = g.normal(0.0, 0.05, cout)
            mean = g.normal(0.0, 0.05, cout)
            var = g.uniform(0.8, 1.2, cout)
            for v in (gamma, beta, mean, var):
                parts.append(v.astype("<f4").tobytes())
        else:
            bias = g.normal(0.0, 0.05, cout)
            if cout == 24:
                for a in range(4):
                    bias[6 * a + 4] += tobj_shift[det_i][a]
                det_i += 1
            parts.append(bias.astype("<f4").tobytes())
    return b"".join(parts)


def parse_blob(blob: bytes):
    """Split a weights blob into per-layer dicts of float32 arrays (no arithmetic)."""
    magic = blob[:4]
    if magic != BLOB_MAGIC:
        raise ValueError("bad weights blob magic")
    version, n, _ = struct.unpack_from("<III", blob, 4)
    if version != BLOB_VERSION:
        raise ValueError("bad weights blob version")
    off = 16
    layers = []
    for _ in range(n):
        cin, cout, k, stride, flags, _, _, _ = struct.unpack_from("<8I", blob, off)
        off += 32
        nw = cout * cin * k * k
        w = np.frombuffer(blob, "<f4", nw, off).reshape(cout, cin, k, k)
        off += 4 * nw
        d = dict(cin=cin, cout=cout, k=k, stride=stride, flags=flags, w=w)
        if flags & FLAG_BN:
            for name in ("gamma", "beta", "mean", "var"):
                d[name] = np.frombuffer(blob, "<f4", cout, off)
                off += 4 * cout
        if flags & FLAG_BIAS:
            d["bias"] = np.frombuffer(blob, "<f4", cout, off)
            off += 4 * cout
        layers.append(d)
    if off != len(blob):
        raise ValueError("trailing bytes in weights blob")
    return layers


# --------------------------------------------------------------------------- heads
def random_heads(seed: int, batch: int, grids, tobj_mean: float = -2.0, tobj_std: float = 1.5,
                 emb: bool = True):
    """Dense random head tensors for decode / NMS stress tests.

    ``grids`` lists ``(H_s, W_s)`` per head.  Each detection map is
    ``[batch, H_s, W_s, 24]`` float32 with every value ~ N(0, 1) except the
    objectness channels (6a+4) ~ N(tobj_mean, tobj_std); each embedding map is
    ``[batch, H_s, W_s, 512]`` ~ N(0, 1).
    """
    g = _rng(seed, 0)
    dets, embs = [], []
    for (h, w) in grids:
        d = g.standard_normal((batch, h, w, 24)).astype(np.float32)
        for a in range(4):
            d[..., 6 * a + 4] = g.normal(tobj_mean, tobj_std, (batch, h, w)).astype(np.float32)
        dets.append(d)
        if emb:
            embs.append(g.standard_normal((batch, h, w, 512)).astype(np.float32))
    return dets, embs


class PlantedClip:
    """Objects planted on constant-velocity paths into JDE head tensors.

    Object ``o`` has a fixed size (w, h) in frame pixels (h ~ U(80, 320),
    w/h ~ U(0.35, 0.5)) and moves at a constant velocity of at most
    ``max_speed`` px/frame per axis on a path that stays inside the frame for
    the whole clip; each frame its centre
    gets N(0, ``jitter``) px noise, and it is hidden with probability ``occl``.
    Each object carries a unit identity vector ``u_o``; its cell in the
    embedding map holds ``u_o + n`` with ``n`` an isotropic Gaussian vector of
    expected norm ``emb_noise``.

    Planting (the head tensors are what a detector would emit): the object is
    written at the anchor ``(scale, a)`` whose height is nearest in log-space,
    at the cell containing its letterboxed centre, with logits chosen so that a
    YOLO-style decode returns the box: ``tx = logit(frac(cx/s))``,
    ``tw = log(w / anchor_w)``, objectness +4.  A duplicate is written at a
    second anchor of the same cell with the same box and objectness +1 (and
    with probability 1/2 a third one), so NMS has work to do.  Background
    cells keep objectness -6.  Two objects that would land on one
    (scale, cell) in a frame would share its embedding: the later one is hidden.

    ``anchors[s]`` lists the four (w, h) of head ``s``, ``strides[s]`` its
    stride; the letterbox is described by ``(ratio, pad_x, pad_y)``.
    """

    def __init__(self, seed, n_objects, n_frames, in_w, in_h, anchors, strides, ratio, pad_x, pad_y,
                 src_w=SRC_W, src_h=SRC_H, occl=0.1, jitter=2.0, emb_noise=0.1, emb_noise_per_dim=False,
                 max_speed=3.0):
        self.seed, self.n, self.T = seed, n_objects, n_frames
        self.in_w, self.in_h = in_w, in_h
        self.anchors, self.strides = anchors, strides
        self.r, self.px, self.py = ratio, pad_x, pad_y
        self.src_w, self.src_h = src_w, src_h
        self.occl, self.jitter = occl, jitter
        g = _rng(seed, 1 << 20)
        h = g.uniform(80.0, 320.0, n_objects)
        w = h * g.uniform(0.35, 0.5, n_objects)
        self.size = np.stack([w, h], 1)
        # velocity up to max_speed px/frame per axis; the start is drawn so the whole path stays inside
        self.vel = g.uniform(-max_speed, max_speed, (n_objects, 2))
        span = self.vel * max(n_frames - 1, 1)
        lo_x = w / 2 + 4 + np.maximum(0, -span[:, 0])
        hi_x = src_w - w / 2 - 4 - np.maximum(0, span[:, 0])
        lo_y = h / 2 + 4 + np.maximum(0, -span[:, 1])
        hi_y = src_h - h / 2 - 4 - np.maximum(0, span[:, 1])
        self.start = np.stack([g.uniform(lo_x, hi_x), g.uniform(lo_y, hi_y)], 1)
        ident = g.standard_normal((n_objects, 512))
        self.ident = ident / np.linalg.norm(ident, axis=1, keepdims=True)
        # isotropic noise with E|n| = emb_noise (per-dim sigma emb_noise/sqrt(512)),
        # or the literal per-dimension sigma when emb_noise_per_dim is set.
        self.emb_sigma = emb_noise if emb_noise_per_dim else emb_noise / math.sqrt(512.0)
        self.grids = [(in_h // s, in_w // s) for s in strides]

    def frame_entries(self, t: int):
        """Sparse content of frame ``t``: ``(det_entries, emb_entries, truth)``.

        ``det_entries`` lists ``(head, y, x, anchor, values[6])``, ``emb_entries``
        lists ``(head, y, x, vector[512])``; every other detection value is 0
        except the objectness channels (-6) and every other embedding value 0.
        ``truth`` lists ``(object_id, cx, cy, w, h)`` in frame px of the objects
        planted in this frame.
        """
        g = _rng(self.seed, t)
        used = set()
        det_e, emb_e, truth = [], [], []
        jit = g.normal(0.0, self.jitter, (self.n, 2))
        hide = g.random(self.n) < self.occl
        third = g.random(self.n) < 0.5
        noise = g.normal(0.0, self.emb_sigma, (self.n, 512))
        lg_anchor = [[math.log(a[1]) for a in sc] for sc in self.anchors]
        for o in range(self.n):
            if hide[o]:
                continue
            cx, cy = self.start[o] + self.vel[o] * t + jit[o]
            w, h = self.size[o]
            lx, ly = cx * self.r + self.px, cy * self.r + self.py
            lw, lh = w * self.r, h * self.r
            best = None
            for s, sc in enumerate(self.anchors):
                for a in range(4):
                    dist = abs(math.log(lh) - lg_anchor[s][a])
                    if best is None or dist < best[0]:
                        best = (dist, s, a)
            _, s, a = best
            st = self.strides[s]
            gh, gw = self.grids[s]
            gx, gy = int(lx // st), int(ly // st)
            if not (0 <= gx < gw and 0 <= gy < gh):
                continue
            alts = [b for b in (a - 1, a + 1, a - 2, a + 2) if 0 <= b < 4]
            slots = [(s, a, gy, gx)] + [(s, b, gy, gx) for b in alts[: (2 if third[o] else 1)]]
            if (s, gy, gx) in used or any(sl in used for sl in slots):
                continue
            fx = min(max(lx / st - gx, 1e-3), 1 - 1e-3)
            fy = min(max(ly / st - gy, 1e-3), 1 - 1e-3)
            tx, ty = math.log(fx / (1 - fx)), math.log(fy / (1 - fy))
            for j, (_, b, _, _) in enumerate(slots):
                aw, ah = self.anchors[s][b]
                vals = [tx, ty, math.log(lw / aw), math.log(lh / ah), 4.0 if j == 0 else 1.0, 4.0]
                det_e.append((s, gy, gx, b, vals))
                used.add((s, b, gy, gx))
            used.add((s, gy, gx))
            emb_e.append((s, gy, gx, (self.ident[o] + noise[o]).astype(np.float32)))
            truth.append((o, cx, cy, w, h))
        return det_e, emb_e, truth

    def frame(self, t: int):
        """Dense head tensors of frame ``t``: ``(dets, embs, truth)``.

        ``dets[s]`` is ``[H_s, W_s, 24]`` float32, ``embs[s]`` ``[H_s, W_s, 512]``
        float32 (the entries of ``frame_entries`` written into the background).
        """
        det_e, emb_e, truth = self.frame_entries(t)
        dets = []
        for (gh, gw) in self.grids:
            d = np.zeros((gh, gw, 24), np.float32)
            d[..., 4::6] = -6.0
            dets.append(d)
        embs = [np.zeros((gh, gw, 512), np.float32) for (gh, gw) in self.grids]
        for s, y, x, b, vals in det_e:
            dets[s][y, x, 6 * b:6 * b + 6] = vals
        for s, y, x, vec in emb_e:
            embs[s][y, x] = vec
        return dets, embs, truth


class PlantedHeadFrames:
    """The frames of a ``PlantedClip`` written as dense head tensors on a torch device.

    ``write(torch, bufs, t)`` fills ``bufs`` (the three ``[H_s, W_s, 24]`` detection maps and the three
    ``[H_s, W_s, 512]`` embedding maps of one frame, float32, on the device) with frame ``t mod T`` of
    the clip on torch's current stream: the background values of ``PlantedClip.frame``, then one
    scatter per tensor of the frame's entries (kept in compact form, built once per frame).
    """

    def __init__(self, clip: PlantedClip):
        self.clip = clip
        self._entries = {}
        self._dev = {}

    def entries(self, t: int):
        t %= self.clip.T
        if t not in self._entries:
            det_e, emb_e, _ = self.clip.frame_entries(t)
            per = []
            for s, (gh, gw) in enumerate(self.clip.grids):
                de = [e for e in det_e if e[0] == s]
                ee = [e for e in emb_e if e[0] == s]
                lin = np.array([(y * gw + x) * 24 + 6 * a + k for _, y, x, a, _ in de for k in range(6)], np.int64)
                vals = np.array([v for e in de for v in e[4]], np.float32)
                cells = np.array([y * gw + x for _, y, x, _ in ee], np.int64)
                vecs = np.array([e[3] for e in ee], np.float32).reshape(-1, 512)
                per.append((lin, vals, cells, vecs))
            self._entries[t] = per
        return self._entries[t]

    def _device_entries(self, torch, dev, t: int):
        key = (t % self.clip.T, str(dev))
        if key not in self._dev:        # the frame's entries, copied to the device once
            self._dev[key] = [tuple(torch.from_numpy(a).to(dev) for a in ent) for ent in self.entries(t)]
        return self._dev[key]

    def preload(self, torch, dev):
        """Build every frame's entries and copy them to the device (before a timed run)."""
        for t in range(self.clip.T):
            self._device_entries(torch, dev, t)

    def write(self, torch, bufs, t: int):
        dev = bufs[0].device
        for s, (lin, vals, cells, vecs) in enumerate(self._device_entries(torch, dev, t)):
            d, e = bufs[s], bufs[3 + s]
            d.zero_()
            d[..., 4::6] = -6.0
            e.zero_()
            if len(lin):
                d.view(-1)[lin] = vals
            if len(cells):
                e.view(-1, 512)[cells] = vecs

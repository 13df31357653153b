"""Oracle network: letterbox + DarkNet-53 backbone + FPN + JDE heads, in float64.

Sec. 3.1 names the parts (DarkNet-53 backbone, FPN that upsamples higher-level
features and fuses them with lower ones, predictions taken from three layers,
YOLOv3-style detection) but prints no layer table.  The readings used here:

* Backbone: stem 3x3 3->32; five stride-2 3x3 downsamples to 64/128/256/512/1024
  channels, followed by 1/2/8/8/4 residual blocks (1x1 c->c/2, 3x3 c/2->c,
  then ``x + branch``).  The stage outputs at strides 8/16/32 are C3/C4/C5.
* Per scale (32, 16, 8 with mid = 512, 256, 128): five alternating convs
  1x1 mid, 3x3 2mid, 1x1 mid, 3x3 2mid, 1x1 mid giving F_s; detection head
  3x3 mid->2mid then linear 1x1 2mid->24 (4 anchors x 6); embedding head
  linear 3x3 mid->512.  Scales 32 and 16 add a lateral 1x1 (mid -> mid/2)
  whose output is upsampled 2x (nearest) and concatenated before the skip
  feature (C4 resp. C3) to feed the next scale.
* Every conv has padding k//2 and is followed by BN + leaky-ReLU(0.1), except
  the detection 1x1 and the embedding 3x3 which are linear with a bias.
* BN is folded: W' = W gamma / sqrt(var + eps), b' = beta - mean gamma / sqrt(var + eps),
  eps = 1e-5.

Layer order (the order of the weights blob): backbone in forward order, then
for each scale 32, 16, 8: the five block convs, det 3x3, det 1x1, emb 3x3 and
(scales 32 and 16) the lateral 1x1.

Layout: activations are NHWC float64 arrays.
"""
from __future__ import annotations

import math

import numpy as np

BN_EPS = 1e-5
LEAKY = 0.1
STAGES = ((64, 1), (128, 2), (256, 8), (512, 8), (1024, 4))
SCALES = ((1024, 512, 256), (768, 256, 128), (384, 128, None))  # (cin, mid, lateral) for strides 32, 16, 8
STRIDES = (32, 16, 8)


def layer_specs():
    """The layer table: ``(cin, cout, k, stride, has_bn, res_nblocks)`` per conv."""
    L = [(3, 32, 3, 1, True, 0)]
    for c, nb in STAGES:
        L.append((c // 2, c, 3, 2, True, 0))
        for _ in range(nb):
            L.append((c, c // 2, 1, 1, True, 0))
            L.append((c // 2, c, 3, 1, True, nb))
    for cin, mid, lat in SCALES:
        L += [(cin, mid, 1, 1, True, 0), (mid, 2 * mid, 3, 1, True, 0), (2 * mid, mid, 1, 1, True, 0),
              (mid, 2 * mid, 3, 1, True, 0), (2 * mid, mid, 1, 1, True, 0)]
        L += [(mid, 2 * mid, 3, 1, True, 0), (2 * mid, 24, 1, 1, False, 0), (mid, 512, 3, 1, False, 0)]
        if lat:
            L.append((mid, lat, 1, 1, True, 0))
    return L


# ----------------------------------------------------------------------------- letterbox
def letterbox_geometry(src_w, src_h, dst_w, dst_h):
    """Scale and padding of the letterbox (reading; the paper only says FullHD input).

    r = min(dst_w/src_w, dst_h/src_h); the resized image is
    floor(src_w r + 0.5) x floor(src_h r + 0.5) and is centred with
    pad = floor((dst - new) / 2) on the left/top, the remainder right/bottom.
    """
    r = min(dst_w / src_w, dst_h / src_h)
    nw = int(math.floor(src_w * r + 0.5))
    nh = int(math.floor(src_h * r + 0.5))
    return r, nw, nh, (dst_w - nw) // 2, (dst_h - nh) // 2


def letterbox(frames_u8: np.ndarray, dst_w: int, dst_h: int) -> np.ndarray:
    """uint8 ``[N, H, W, 3]`` frames -> float64 ``[N, dst_h, dst_w, 3]`` network input.

    Bilinear resize with half-pixel centres (src = (dst + 0.5) / r - 0.5,
    clamped to the image), values scaled by 1/255, padding filled with 0.5.
    """
    n, sh, sw, _ = frames_u8.shape
    r, nw, nh, px, py = letterbox_geometry(sw, sh, dst_w, dst_h)
    out = np.full((n, dst_h, dst_w, 3), 0.5)

    def axis(count, size):
        s = (np.arange(count) + 0.5) / r - 0.5
        s = np.clip(s, 0.0, size - 1)
        i0 = np.floor(s).astype(np.int64)
        i1 = np.minimum(i0 + 1, size - 1)
        return i0, i1, s - i0

    x0, x1, fx = axis(nw, sw)
    y0, y1, fy = axis(nh, sh)
    img = frames_u8.astype(np.float64)
    fx = fx[None, None, :, None]
    fy = fy[None, :, None, None]
    top = img[:, y0][:, :, x0] * (1 - fx) + img[:, y0][:, :, x1] * fx
    bot = img[:, y1][:, :, x0] * (1 - fx) + img[:, y1][:, :, x1] * fx
    out[:, py:py + nh, px:px + nw] = (top * (1 - fy) + bot * fy) / 255.0
    return out


# ----------------------------------------------------------------------------- layers
def fold_bn(layer):
    """Fold BN statistics into the conv: returns (W' [cout, cin, k, k], b' [cout]) in float64."""
    w = layer["w"].astype(np.float64)
    if "gamma" in layer:
        g = layer["gamma"].astype(np.float64)
        s = g / np.sqrt(layer["var"].astype(np.float64) + BN_EPS)
        b = layer["beta"].astype(np.float64) - layer["mean"].astype(np.float64) * s
        return w * s[:, None, None, None], b
    return w, layer["bias"].astype(np.float64)


def conv2d(x: np.ndarray, w: np.ndarray, b: np.ndarray, stride: int) -> np.ndarray:
    """out[n, oy, ox, co] = b[co] + sum_{ky,kx,ci} w[co, ci, ky, kx] * xpad[n, s oy + ky, s ox + kx, ci].

    Zero padding p = k // 2.  Written as one matrix product per kernel tap.
    """
    n, h, wd, cin = x.shape
    cout, _, k, _ = w.shape
    p = k // 2
    ho = (h + 2 * p - k) // stride + 1
    wo = (wd + 2 * p - k) // stride + 1
    xp = np.zeros((n, h + 2 * p, wd + 2 * p, cin))
    xp[:, p:p + h, p:p + wd] = x
    out = np.zeros((n * ho * wo, cout))
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, ky:ky + stride * (ho - 1) + 1:stride, kx:kx + stride * (wo - 1) + 1:stride, :]
            out += np.ascontiguousarray(patch).reshape(-1, cin) @ w[:, :, ky, kx].T
    return out.reshape(n, ho, wo, cout) + b


def leaky(x):
    return np.where(x > 0, x, LEAKY * x)


def upsample2(x):
    """Nearest-neighbour 2x upsampling of an NHWC tensor."""
    return x.repeat(2, axis=1).repeat(2, axis=2)


# ----------------------------------------------------------------------------- forward
def forward(x: np.ndarray, layers, keep_all: bool = False):
    """Run the network on an NHWC float64 input.

    ``layers`` is the parsed weights blob (``synth.parse_blob``).  Returns
    ``(dets, embs, acts)`` where ``dets[s]`` is the ``[N, H_s, W_s, 24]``
    detection map and ``embs[s]`` the ``[N, H_s, W_s, 512]`` embedding map for
    strides 32, 16, 8, and ``acts`` the output of every conv in layer order
    when ``keep_all`` (else empty); for a conv that closes a residual branch
    the recorded output is the block output ``x + branch``.
    """
    specs = layer_specs()
    if len(layers) != len(specs):
        raise ValueError("layer count mismatch")
    for L, (cin, cout, k, st, bn, _) in zip(layers, specs):
        if (L["cin"], L["cout"], L["k"], L["stride"], bool(L["flags"] & 1)) != (cin, cout, k, st, bn):
            raise ValueError("layer shape mismatch")
    it = iter(layers)
    acts = []

    def conv(inp, linear=False, res=None):
        L = next(it)
        w, b = fold_bn(L)
        y = conv2d(inp, w, b, L["stride"])
        if not linear:
            y = leaky(y)
        if res is not None:
            y = res + y
        if keep_all:
            acts.append(y)
        return y

    x = conv(x)
    feats = {}
    for c, nb in STAGES:
        x = conv(x)
        for _ in range(nb):
            x = conv(conv(x), res=x)
        feats[c] = x
    skips = {512: feats[512], 256: feats[256]}
    dets, embs = [], []
    inp = feats[1024]
    for cin, mid, lat in SCALES:
        f = inp
        for _ in range(5):
            f = conv(f)
        d = conv(conv(f), linear=True)
        e = conv(f, linear=True)
        dets.append(d)
        embs.append(e)
        if lat:
            up = upsample2(conv(f))
            inp = np.concatenate([up, skips[2 * lat]], axis=3)
    return dets, embs, acts


def layer_io():
    """Wiring of ``forward`` as data: per conv ``(input, residual)``.  ``input`` is a layer id, -1 for
    the network input, or ``("cat", lateral, skip)`` for the concat of the upsampled lateral's output
    and a skip feature; ``residual`` is the layer id whose output is added, or None."""
    io = []

    def conv(inp, res=None):
        io.append((inp, res))
        return len(io) - 1

    x = conv(-1)
    feats = {}
    for c, nb in STAGES:
        x = conv(x)
        for _ in range(nb):
            x = conv(conv(x), res=x)
        feats[c] = x
    inp = feats[1024]
    for cin, mid, lat in SCALES:
        f = inp
        for _ in range(5):
            f = conv(f)
        conv(conv(f))
        conv(f)
        if lat:
            up = conv(f)
            inp = ("cat", up, feats[2 * lat])
    return io


def flops(in_w: int, in_h: int) -> int:
    """Multiply-add FLOPs (2 M N K summed over convs) of one frame at the given input size."""
    specs = layer_specs()
    sizes = [(in_h, in_w)]
    h, w = in_h, in_w
    for _, nb in STAGES:
        h, w = (h + 1) // 2, (w + 1) // 2
        sizes += [(h, w)] * (1 + 2 * nb)
    for s, (_, _, lat) in zip(STRIDES, SCALES):
        sizes += [(in_h // s, in_w // s)] * (9 if lat else 8)
    return sum(2 * hh * ww * co * ci * k * k for (ci, co, k, _, _, _), (hh, ww) in zip(specs, sizes))

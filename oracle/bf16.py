"""Oracle of the BF16 network: the float64 forward with every stored tensor rounded to bfloat16.

Test infrastructure: only tests/, the smoke entry point and the benchmark's CPU
baseline use this package.  Shares no code with the CUDA library.

bfloat16: sign, 8 exponent bits (bias 127, the float32 range), 7 stored
mantissa bits.  A normal value is (1 + m/128) 2^e; the spacing of values in
the binade [2^k, 2^(k+1)) is 2^(k-7), and below 2^-126 the subnormal spacing
2^-133 applies.  Conversion from a wider type rounds to the nearest value,
ties to the even mantissa.

Storage scheme of the library's BF16 path (a reading: Sec. 4.1 runs the network
in reduced precision with BN kept separate; here BN is folded first and the
folded weights are rounded once):

* network input: the letterboxed frame (float64 here) rounded to bfloat16;
* weights: the BN-folded weights W' rounded to bfloat16, the folded bias b'
  rounded to float32;
* every conv accumulates exactly (float64 here) and adds the bias; leaky-ReLU
  follows where the layer has BN;
* the output of every conv except the two linear heads is stored as
  bfloat16; the heads are kept in float (float64 here);
* a residual block's output, ``x + branch``, is stored two ways:
  ``inplace=True`` (the default handle) rounds the branch to bfloat16 first and
  then the sum (the block adds its rounded output into the storage of its
  input), ``inplace=False`` (a handle that keeps every layer output) rounds the
  sum once.

Pins: the rounding against every bfloat16 value's neighbours and midpoints
(ties to even), overflow to infinity, and torch's float32 -> bfloat16 cast;
with the rounding replaced by the identity the scheme's forward equals
``network.forward`` to 1e-12 on every layer.
"""
from __future__ import annotations

import numpy as np

from . import network as net

BF16_MAX = (2.0 - 2.0 ** -7) * 2.0 ** 127


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even mantissa); float64 out.

    Magnitudes that round above the largest finite value give +-inf; NaN stays NaN."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        # binade exponent k with 2^k <= a < 2^(k+1); the subnormal spacing 2^-133 below 2^-126
        k = np.floor(np.log2(np.where(a > 0, a, 1.0)))
        k = np.maximum(k, -126.0)
        q = np.exp2(k - 7.0)
        r = np.round(a / q) * q                  # numpy rounds halves to even
        r = np.where(np.isfinite(a), r, a)
        r = np.where(r > BF16_MAX, np.inf, r)
    out = np.copysign(r, x)
    return np.where(np.isnan(x), np.nan, out)


def f32(x) -> np.ndarray:
    """Round to float32 (ties to even) and return float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def conv_layer(l: int, inp: np.ndarray, layers, res=None, inplace: bool = True, rnd=bf16) -> np.ndarray:
    """One conv of the scheme on an input already held in bfloat16: bfloat16 weights, float32 bias,
    float64 accumulation, leaky-ReLU (BN layers), residual, bfloat16 store (not the heads)."""
    spec = net.layer_specs()[l]
    head = not spec[4]
    w, b = net.fold_bn(layers[l])
    y = net.conv2d(inp, rnd(w), f32(b) if rnd is bf16 else b, layers[l]["stride"])
    if not head:
        y = net.leaky(y)
    if res is not None:
        y = res + (rnd(y) if inplace else y)
    return y if head else rnd(y)


def forward(x: np.ndarray, layers, inplace: bool = True, keep_all: bool = False, rnd=bf16):
    """The BF16 scheme's forward on the float64 letterboxed input ``x`` (rounded here): same structure
    and return values as ``network.forward``.  ``rnd`` replaces the rounding (the identity reduces the
    scheme to the float64 network)."""
    specs = net.layer_specs()
    it = iter(range(len(specs)))
    acts = []

    def conv(inp, linear=False, res=None):
        l = next(it)
        assert linear == (not specs[l][4])
        y = conv_layer(l, inp, layers, res, inplace, rnd)
        if keep_all:
            acts.append(y)
        return y

    x = conv(rnd(x))
    feats = {}
    for c, nb in net.STAGES:
        x = conv(x)
        for _ in range(nb):
            x = conv(conv(x), res=x)
        feats[c] = x
    skips = {512: feats[512], 256: feats[256]}
    dets, embs = [], []
    inp = feats[1024]
    for cin, mid, lat in net.SCALES:
        f = inp
        for _ in range(5):
            f = conv(f)
        d = conv(conv(f), linear=True)
        e = conv(f, linear=True)
        dets.append(d)
        embs.append(e)
        if lat:
            up = net.upsample2(conv(f))
            inp = np.concatenate([up, skips[2 * lat]], axis=3)
    return dets, embs, acts

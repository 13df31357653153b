"""Oracle of the FP8 (E4M3) network: fake-quantised float64 forward, and its calibration.

Test infrastructure: only tests/, the smoke entry point and the benchmark's CPU
baseline use this package.  Shares no code with the CUDA library.

E4M3 (OCP 8-bit floating point, "fn" flavour): sign, 4 exponent bits with bias
7, 3 mantissa bits.  Normal values (1 + m/8) 2^(e-7) for e = 1..15 (the code
e = 15, m = 7 is NaN, so the largest finite value is 1.75 * 2^8 = 448);
subnormals m/8 * 2^-6 for e = 0.  Conversion from a wider type rounds to the
nearest representable value, ties to the even mantissa, and saturates finite
values beyond the range to +-448.

Quantisation scheme (the E4M3 pattern of the library's FP8 path; the paper itself
runs FP32): every conv whose input tensor is stored in FP8 multiplies E4M3 codes of
the input (one scale per tensor, s_x = amax_x / 448) with E4M3 codes of the
folded weights (one scale per output channel, s_w[co] = max|W'[co]| / 448) and
accumulates exactly; the epilogue applies s_x s_w[co], the bias, leaky-ReLU
and the residual (itself an FP8-stored tensor), then stores the result as
E4M3 codes of its own tensor scale.  Which tensors are FP8 (a reading, see
``FIRST_FP8_OUTPUT``): the outputs of layers 4 and later, the two concat buffers,
and therefore the inputs of layers 5 and later; the stem, the three following
32/64-channel layers and layer 4's input stay in higher precision (the
oracle keeps them float64).  The heads (det 1x1, emb 3x3) write float values.
A concat buffer is one tensor: the lateral written into it and the skip
feature stored in it share its scale (the larger amax of the two writers).

Pins: the quantiser against all 256 codes decoded from their bit fields, the
ties-to-even midpoints, saturation, and torch's float8_e4m3fn conversion; the
fake-quantised forward reduces exactly to the float64 forward when the
quantiser is replaced by the identity (same structure, scales only where the
scheme puts them); per-channel weight scales against a brute-force maximum.
"""
from __future__ import annotations

import numpy as np

from . import network as net

E4M3_MAX = 448.0
FIRST_FP8_OUTPUT = 4          # layer whose output is the first FP8-stored tensor


def e4m3_decode(code: int) -> float:
    """Value of an 8-bit E4M3 code (bit 7 sign, bits 6..3 exponent, bits 2..0 mantissa)."""
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return float("nan")
    if e == 0:
        return s * (m / 8.0) * 2.0 ** -6
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def e4m3(x) -> np.ndarray:
    """Round to the nearest E4M3 value (ties to even mantissa), saturating at +-448; float64 out."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    # binade exponent k with 2^k <= a < 2^(k+1); below 2^-6 the subnormal spacing 2^-9 applies
    k = np.floor(np.log2(np.maximum(a, 2.0 ** -9)))
    k = np.maximum(k, -6.0)
    q = np.exp2(k - 3.0)                       # spacing of the 8 mantissa steps in the binade
    r = np.round(a / q) * q                    # numpy rounds halves to even
    r = np.minimum(r, E4M3_MAX)
    out = np.copysign(r, x)
    return np.where(np.isnan(x), np.nan, out)


def fake_quant(x, scale) -> np.ndarray:
    """Value an FP8 store with the given scale(s) keeps: e4m3(x / scale) * scale."""
    return e4m3(np.asarray(x, dtype=np.float64) / scale) * scale


# ----------------------------------------------------------------------------- scales
def concat_writers():
    """Layer ids whose outputs live in the two concat buffers: {buffer: [lateral, skip]}.

    Stride-16 buffer: the first lateral (the conv after the stride-32 embedding head, upsampled) and
    C4 (the last stage-4 block); stride-8 buffer: the second lateral and C3 (the last stage-3 block)."""
    specs = net.layer_specs()
    emb = [i for i, s in enumerate(specs) if s[1] == 512 and s[2] == 3 and not s[4]]
    ends = {}
    for i, s in enumerate(specs):
        if s[5]:                               # conv closing a residual block (backbone)
            ends[s[1]] = i
    return {"cat16": [emb[0] + 1, ends[512]], "cat8": [emb[1] + 1, ends[256]]}


def buffer_of(layer: int):
    for name, ws in concat_writers().items():
        if layer in ws:
            return name
    return layer


def tensor_scales(amax):
    """Per-layer output scale s = amax / 448 for FP8-stored outputs (concat writers share the buffer's)."""
    amax = np.asarray(amax, dtype=np.float64)
    s = amax / E4M3_MAX
    for ws in concat_writers().values():
        s[ws] = max(amax[w] for w in ws) / E4M3_MAX
    return s


def calibrate(frames_nhwc: np.ndarray, layers) -> np.ndarray:
    """amax of every layer output over the calibration frames (float64 forward)."""
    _, _, acts = net.forward(frames_nhwc, layers, keep_all=True)
    return np.array([float(np.max(np.abs(a))) for a in acts])


def weight_scales(w: np.ndarray) -> np.ndarray:
    """Per-output-channel scale max|W'[co]| / 448 (channels of all zeros get scale 1)."""
    m = np.max(np.abs(w.reshape(w.shape[0], -1)), axis=1) / E4M3_MAX
    return np.where(m > 0, m, 1.0)


def is_head(spec) -> bool:
    return not spec[4]


# ----------------------------------------------------------------------------- forward
def conv_layer(l: int, inp: np.ndarray, layers, out_scales, res=None) -> np.ndarray:
    """One conv of the scheme: FP8 weights when its input is FP8, epilogue in float64, FP8 store of
    its output when that tensor is FP8 (heads stay float)."""
    specs = net.layer_specs()
    L = layers[l]
    w, b = net.fold_bn(L)
    if l > FIRST_FP8_OUTPUT:                   # FP8 input tensor: per-channel FP8 weights
        sw = weight_scales(w)
        w = e4m3(w / sw[:, None, None, None]) * sw[:, None, None, None]
    y = net.conv2d(inp, w, b, L["stride"])
    if not is_head(specs[l]):
        y = net.leaky(y)
    if res is not None:
        y = res + y
    if l >= FIRST_FP8_OUTPUT and not is_head(specs[l]):
        y = fake_quant(y, out_scales[l])
    return y


def forward(x: np.ndarray, layers, out_scales, keep_all: bool = False):
    """Fake-quantised forward: same structure as ``network.forward``; FP8 stores and FP8 weights where
    the scheme above puts them.  ``out_scales[l]`` is the scale of layer l's output tensor."""
    specs = net.layer_specs()
    it = iter(range(len(specs)))
    acts = []

    def conv(inp, linear=False, res=None):
        l = next(it)
        assert linear == is_head(specs[l])
        y = conv_layer(l, inp, layers, out_scales, res)
        if keep_all:
            acts.append(y)
        return y

    x = conv(x)
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

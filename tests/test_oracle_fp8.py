"""Pins of the FP8 (E4M3) oracle: the quantiser against the format definition, and the fake-quantised forward."""
import numpy as np
import pytest

import synth
from oracle import fp8
from oracle import network as net


def finite_codes():
    vals = {}
    for c in range(256):
        v = fp8.e4m3_decode(c)
        if not np.isnan(v):
            vals[c] = v
    return vals


def test_every_code_is_a_fixed_point_and_the_range_is_the_format_s():
    vals = finite_codes()
    assert len(vals) == 254                    # 0x7f and 0xff are NaN
    for c, v in vals.items():
        assert fp8.e4m3(v) == v, hex(c)
    pos = sorted(v for v in vals.values() if v > 0)
    assert pos[-1] == 448.0 and pos[0] == 2.0 ** -9
    assert len(pos) == 126                     # 7 subnormals + 15 binades x 8 - 1 (NaN)


def test_midpoints_round_to_the_even_code():
    pos = sorted((v, c) for c, v in finite_codes().items() if v > 0)
    for (a, ca), (b, cb) in zip(pos, pos[1:]):
        mid = (a + b) / 2
        want = a if ca % 2 == 0 else b
        assert fp8.e4m3(mid) == want, (a, b)
        assert fp8.e4m3(np.nextafter(mid, 0)) == a
        assert fp8.e4m3(np.nextafter(mid, 1e9)) == b
        assert fp8.e4m3(-mid) == -want


def test_saturation_zero_and_nan():
    assert fp8.e4m3(460.0) == 448.0            # below the midpoint to the (absent) 480
    assert fp8.e4m3(1e6) == 448.0 and fp8.e4m3(-1e6) == -448.0
    assert fp8.e4m3(2.0 ** -10) == 0.0         # half the smallest subnormal: tie to even (zero)
    assert fp8.e4m3(1.5 * 2.0 ** -9) == 2.0 ** -8
    assert np.isnan(fp8.e4m3(np.nan))


def test_matches_torch_float8_e4m3fn_in_range():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    g = np.random.Generator(np.random.PCG64(11))
    x = np.concatenate([g.uniform(-448, 448, 20000), g.standard_normal(20000) * 1e-2,
                        g.standard_normal(20000)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(fp8.e4m3(x.astype(np.float64)), ref)


def test_weight_scales_are_the_per_channel_maximum():
    g = np.random.Generator(np.random.PCG64(3))
    w = g.standard_normal((7, 5, 3, 3))
    w[4] = 0.0
    s = fp8.weight_scales(w)
    for co in range(7):
        m = max(abs(float(v)) for v in w[co].ravel())
        assert s[co] == (m / 448.0 if m > 0 else 1.0)
    q = fp8.e4m3(w / s[:, None, None, None])
    assert np.max(np.abs(q)) == 448.0          # each channel's extreme lands on the largest code


def test_concat_writers_are_the_laterals_and_the_skips():
    specs = net.layer_specs()
    cw = fp8.concat_writers()
    lat16, c4 = cw["cat16"]
    lat8, c3 = cw["cat8"]
    assert specs[lat16][:4] == (512, 256, 1, 1) and specs[lat8][:4] == (256, 128, 1, 1)
    assert not specs[lat16 - 1][4] and specs[lat16 - 1][1] == 512      # after the stride-32 emb head
    assert specs[c4][1] == 512 and specs[c4][5] == 8 and specs[c4 + 1][3] == 2   # last stage-4 block
    assert specs[c3][1] == 256 and specs[c3][5] == 8 and specs[c3 + 1][3] == 2
    amax = np.arange(1.0, 79.0)
    s = fp8.tensor_scales(amax)
    assert s[lat16] == s[c4] == max(amax[lat16], amax[c4]) / 448.0
    assert s[lat8] == s[c3] == max(amax[lat8], amax[c3]) / 448.0
    assert s[10] == amax[10] / 448.0


def test_fake_quant_forward_is_the_float64_forward_with_the_identity_quantiser(monkeypatch):
    layers = synth.parse_blob(synth.weights_blob(net.layer_specs()))
    x = net.letterbox(synth.frames_uniform(5, 1, 1080, 1920), 64, 64)
    d0, e0, a0 = net.forward(x, layers, keep_all=True)
    monkeypatch.setattr(fp8, "e4m3", lambda v: np.asarray(v, dtype=np.float64))
    d1, e1, a1 = fp8.forward(x, layers, np.full(78, 0.37), keep_all=True)
    for u, v in zip(d0 + e0 + a0, d1 + e1 + a1):
        np.testing.assert_allclose(u, v, rtol=1e-12, atol=1e-12)


def test_fake_quant_stores_fp8_values_and_keeps_heads_float():
    layers = synth.parse_blob(synth.weights_blob(net.layer_specs()))
    x = net.letterbox(synth.frames_uniform(6, 1, 1080, 1920), 64, 64)
    amax = fp8.calibrate(x, layers)
    s = fp8.tensor_scales(amax)
    _, _, acts = fp8.forward(x, layers, s, keep_all=True)
    specs = net.layer_specs()
    for l, a in enumerate(acts):
        if l >= fp8.FIRST_FP8_OUTPUT and specs[l][4]:
            np.testing.assert_array_equal(fp8.e4m3(a / s[l]) * s[l], a)   # on the tensor's FP8 grid
    for l in range(fp8.FIRST_FP8_OUTPUT):
        assert not np.array_equal(fp8.e4m3(acts[l] / (amax[l] / 448)) * (amax[l] / 448), acts[l])


def test_layer_io_replays_the_forward_layer_by_layer():
    """The wiring table drives a layer-by-layer replay that reproduces forward(keep_all) exactly."""
    layers = synth.parse_blob(synth.weights_blob(net.layer_specs()))
    x = net.letterbox(synth.frames_uniform(8, 1, 1080, 1920), 64, 64)
    _, _, acts = net.forward(x, layers, keep_all=True)
    io = net.layer_io()
    assert len(io) == 78
    outs = []
    for l, (inp, res) in enumerate(io):
        if inp == -1:
            xin = x
        elif isinstance(inp, tuple):
            xin = np.concatenate([net.upsample2(outs[inp[1]]), outs[inp[2]]], axis=3)
        else:
            xin = outs[inp]
        w, b = net.fold_bn(layers[l])
        y = net.conv2d(xin, w, b, layers[l]["stride"])
        if layers[l]["flags"] & 1:
            y = net.leaky(y)
        if res is not None:
            y = outs[res] + y
        outs.append(y)
        np.testing.assert_array_equal(y, acts[l])

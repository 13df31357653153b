"""Pins of the oracle network (CPU): each operation against brute force or a library routine.

The assembled network has no external pin (the paper prints no layer table and
no numbers for it); it is pinned by construction: layer count, folded
parameter count and FLOPs, plus an activation-scale check of the random init.
"""
import itertools
import math

import numpy as np
import pytest
import torch

import synth
from oracle import network as net


def brute_conv(x, w, b, stride):
    n, h, wd, cin = x.shape
    cout, _, k, _ = w.shape
    p = k // 2
    ho = (h + 2 * p - k) // stride + 1
    wo = (wd + 2 * p - k) // stride + 1
    out = np.zeros((n, ho, wo, cout))
    for ni, oy, ox, co in itertools.product(range(n), range(ho), range(wo), range(cout)):
        acc = b[co]
        for ky, kx, ci in itertools.product(range(k), range(k), range(cin)):
            iy, ix = oy * stride + ky - p, ox * stride + kx - p
            if 0 <= iy < h and 0 <= ix < wd:
                acc += w[co, ci, ky, kx] * x[ni, iy, ix, ci]
        out[ni, oy, ox, co] = acc
    return out


@pytest.mark.parametrize("k,stride,h,w,cin,cout", [
    (1, 1, 5, 7, 3, 4), (3, 1, 5, 6, 2, 3), (3, 2, 7, 9, 3, 2), (3, 2, 6, 8, 4, 5), (1, 1, 1, 1, 8, 8),
    (3, 1, 1, 1, 2, 2), (3, 2, 1, 2, 1, 1)])
def test_conv_matches_brute_force(k, stride, h, w, cin, cout):
    g = np.random.default_rng(k * 100 + stride * 10 + h)
    x = g.standard_normal((2, h, w, cin))
    wt = g.standard_normal((cout, cin, k, k))
    b = g.standard_normal(cout)
    np.testing.assert_allclose(net.conv2d(x, wt, b, stride), brute_conv(x, wt, b, stride), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k,stride", [(1, 1), (3, 1), (3, 2)])
def test_conv_matches_torch_f64(k, stride):
    g = np.random.default_rng(7)
    x = g.standard_normal((2, 17, 23, 12))
    wt = g.standard_normal((9, 12, k, k))
    b = g.standard_normal(9)
    ref = torch.nn.functional.conv2d(torch.from_numpy(x).permute(0, 3, 1, 2), torch.from_numpy(wt),
                                     torch.from_numpy(b), stride=stride, padding=k // 2)
    np.testing.assert_allclose(net.conv2d(x, wt, b, stride), ref.permute(0, 2, 3, 1).numpy(), rtol=1e-11, atol=1e-11)


def test_bn_fold_equals_unfolded_bn():
    g = np.random.default_rng(3)
    layer = dict(w=g.standard_normal((6, 4, 3, 3)).astype(np.float32),
                 gamma=g.uniform(0.8, 1.2, 6).astype(np.float32), beta=g.normal(0, 0.05, 6).astype(np.float32),
                 mean=g.normal(0, 0.05, 6).astype(np.float32), var=g.uniform(0.8, 1.2, 6).astype(np.float32))
    x = g.standard_normal((1, 8, 9, 4))
    y = net.conv2d(x, layer["w"].astype(np.float64), np.zeros(6), 1)
    ref = (y - layer["mean"].astype(np.float64)) / np.sqrt(layer["var"].astype(np.float64) + 1e-5) \
        * layer["gamma"].astype(np.float64) + layer["beta"].astype(np.float64)
    w, b = net.fold_bn(layer)
    np.testing.assert_allclose(net.conv2d(x, w, b, 1), ref, rtol=1e-12, atol=1e-12)


def test_layer_table_size():
    specs = net.layer_specs()
    assert len(specs) == 78
    assert sum(ci * co * k * k + co for ci, co, k, _, _, _ in specs) == 65_638_504
    assert abs(net.flops(1088, 608) / 1e9 - 270.9626) < 1e-3
    assert abs(net.flops(320, 192) / 1e9 - 25.1668) < 1e-3
    # 23 residual blocks, each closing conv tagged with its stage's block count
    assert sorted(r for *_, r in specs if r) == sorted([1] + [2] * 2 + [8] * 8 + [8] * 8 + [4] * 4)
    # three linear 1x1 detection heads (24 ch) and three linear 3x3 embedding heads (512 ch)
    assert [(ci, k) for ci, co, k, _, bn, _ in specs if not bn and co == 24] == [(1024, 1), (512, 1), (256, 1)]
    assert [(ci, k) for ci, co, k, _, bn, _ in specs if not bn and co == 512] == [(512, 3), (256, 3), (128, 3)]


@pytest.mark.parametrize("dst,expect", [((1088, 608), (1081, 608, 3, 0)), ((864, 480), (853, 480, 5, 0)),
                                        ((576, 320), (569, 320, 3, 0)), ((320, 192), (320, 180, 0, 6))])
def test_letterbox_geometry(dst, expect):
    r, nw, nh, px, py = net.letterbox_geometry(1920, 1080, *dst)
    assert (nw, nh, px, py) == expect


def test_letterbox_identity_when_same_size():
    f = synth.frames_uniform(1, 2, 192, 320)
    out = net.letterbox(f, 320, 192)
    np.testing.assert_array_equal(out, f.astype(np.float64) / 255.0)


def test_letterbox_constant_and_pad():
    f = np.full((1, 1080, 1920, 3), 77, np.uint8)
    out = net.letterbox(f, 1088, 608)
    r, nw, nh, px, py = net.letterbox_geometry(1920, 1080, 1088, 608)
    np.testing.assert_allclose(out[:, :, px:px + nw], 77 / 255.0, rtol=0, atol=1e-15)
    assert np.all(out[:, :, :px] == 0.5) and np.all(out[:, :, px + nw:] == 0.5)


def test_letterbox_reproduces_linear_ramp():
    # bilinear sampling of a linear function returns the function at the sample point
    h, w = 60, 200
    x = np.arange(w)
    f = np.zeros((1, h, w, 3), np.uint8)
    f[..., 0] = x[None, :]
    f[..., 1] = (np.arange(h)[:, None] * 2)
    out = net.letterbox(f, 100, 40)           # r = 0.5 on x, 0.666 on y -> r = 0.5
    r, nw, nh, px, py = net.letterbox_geometry(w, h, 100, 40)
    assert r == 0.5 and (nw, nh) == (100, 30)
    sx = (np.arange(nw) + 0.5) / r - 0.5
    sy = (np.arange(nh) + 0.5) / r - 0.5
    inner_x = (sx >= 0) & (sx <= w - 1)
    inner_y = (sy >= 0) & (sy <= h - 1)
    got = out[0, py:py + nh, px:px + nw]
    np.testing.assert_allclose(got[:, inner_x, 0] * 255, np.broadcast_to(sx[inner_x], (nh, inner_x.sum())), atol=1e-9)
    np.testing.assert_allclose(got[inner_y, :, 1] * 255, np.broadcast_to(2 * sy[inner_y, None], (inner_y.sum(), nw)),
                               atol=1e-9)


def test_upsample_matches_torch_nearest():
    x = np.random.default_rng(1).standard_normal((2, 3, 5, 4))
    ref = torch.nn.functional.interpolate(torch.from_numpy(x).permute(0, 3, 1, 2), scale_factor=2, mode="nearest")
    np.testing.assert_array_equal(net.upsample2(x), ref.permute(0, 2, 3, 1).numpy())


@pytest.mark.slow
def test_forward_shapes_and_activation_scale():
    """Random init keeps the head outputs O(1) (std within [0.1, 10]) through 23 residual adds."""
    blob = synth.weights_blob(net.layer_specs())
    layers = synth.parse_blob(blob)
    x = net.letterbox(synth.frames_uniform(1, 1, 192, 320), 320, 192)
    dets, embs, acts = net.forward(x, layers, keep_all=True)
    assert len(acts) == 78
    assert [d.shape for d in dets] == [(1, 6, 10, 24), (1, 12, 20, 24), (1, 24, 40, 24)]
    assert [e.shape for e in embs] == [(1, 6, 10, 512), (1, 12, 20, 512), (1, 24, 40, 512)]
    for t in dets + embs:
        assert 0.1 < float(t.std()) < 10.0
    for a in acts:
        assert np.isfinite(a).all() and float(np.abs(a).max()) < 1e3

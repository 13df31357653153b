"""E4M3 (FP8) path on the GPU.

Per-layer parity: every E4M3 conv gets the GPU's own stored input (and residual), the oracle
recomputes that one layer with the same scheme (per-channel E4M3 weights, float64 accumulation,
E4M3 store) and the stored codes must agree, apart from rare one-code flips where the float32
accumulation lands on the other side of a rounding boundary.  The end-to-end element-wise comparison
with the fake-quantised oracle, and the bench configuration, are in test_gpu_precision.py."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import HEAD_LAYERS, forward, jde, make_handle, oracle_layers, rel_maxabs
from oracle import fp8
from oracle import network as net

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fp8_amax_320x192.json")
AMAX = json.load(open(GOLDEN))["amax"]
LUT = np.array([fp8.e4m3_decode(c) for c in range(256)])


def raw_tensor(j, h, tid):
    dims, dt = j.jde_get_tensor(h, tid)
    tdt = {0: torch.float32, 1: torch.bfloat16, 2: torch.uint8}[dt]
    t = torch.empty(dims, dtype=tdt, device="cuda")
    j.jde_get_tensor(h, tid, t, t.numel() * t.element_size(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    return t, dt


def value(j, h, tid, scales):
    t, dt = raw_tensor(j, h, tid)
    if dt == 2:
        return LUT[t.cpu().numpy()] * scales[tid]
    return t.float().cpu().numpy().astype(np.float64)


def spacing(v):
    """Distance between adjacent E4M3 values around |v| (scaled grid: pass v / scale)."""
    a = np.maximum(np.abs(v), 2.0 ** -6)
    return np.exp2(np.floor(np.log2(a)) - 3.0)


def fp8_handle(max_batch=2):
    j = jde()
    h = make_handle(j.JDE_FP8_E4M3, max_batch=max_batch, src_w=320, src_h=192)
    j.jde_set_act_amax(h, AMAX)
    return j, h


def test_e4m3_forward_needs_activation_scales():
    j = jde()
    h = make_handle(j.JDE_FP8_E4M3, max_batch=1, src_w=320, src_h=192)
    try:
        f = torch.from_numpy(synth.frames_uniform(1, 1, 192, 320)).cuda()
        with pytest.raises(j.JdeError):
            j.jde_forward(h, f, 1, 320, 192, 320, 192, True, torch.cuda.current_stream())
        with pytest.raises(j.JdeError):
            j.jde_set_act_amax(h, AMAX[:10])
    finally:
        j.jde_destroy(h)


def test_each_e4m3_layer_matches_the_oracle_layer_on_the_gpu_inputs():
    j, h = fp8_handle()
    try:
        frames = synth.frames_uniform(1, 2, 192, 320)
        forward(h, frames, 320, 192)
        layers = oracle_layers()
        scales = fp8.tensor_scales(AMAX)
        io = net.layer_io()
        outs = {}
        report = []
        for l in range(fp8.FIRST_FP8_OUTPUT, 78):
            inp, res = io[l]
            def get(t):
                if t not in outs:
                    outs[t] = value(j, h, t, scales)
                return outs[t]
            if isinstance(inp, tuple):
                xin = np.concatenate([get(inp[1]), get(inp[2])], axis=3)   # the lateral is stored upsampled
            else:
                xin = get(inp)
            want = fp8.conv_layer(l, xin, layers, scales, get(res) if res is not None else None)
            got = get(l)
            if got.shape != want.shape:          # a lateral: stored 2x upsampled in its concat buffer
                want = net.upsample2(want)
            if l in HEAD_LAYERS:
                err = rel_maxabs(got, want)
                report.append((l, "head", err))
                assert err < 1e-4, (l, err)
                continue
            s = scales[l]
            exact = float(np.mean(got == want))
            steps = np.abs(got - want) / (s * spacing(np.maximum(np.abs(got), np.abs(want)) / s))
            report.append((l, "e4m3", exact, float(steps.max())))
            if l == fp8.FIRST_FP8_OUTPUT:
                # BF16 operands (GPU) vs float64 (oracle) before the first E4M3 store: near-cancelling
                # sums differ by a few 1e-3 of the tensor's range, which can move small values many codes
                assert np.max(np.abs(got - want)) <= 1e-2 * AMAX[l] + s * spacing(np.abs(want) / s).max()
                assert exact >= 0.85, (l, exact)
            else:
                assert steps.max() <= 1.0 + 1e-9, (l, float(steps.max()))
                assert exact >= 0.98, (l, exact)
        print("per-layer E4M3 parity", report)
    finally:
        j.jde_destroy(h)


def test_bf16_calibration_amax_matches_the_oracle_s():
    """jde_act_amax of a BF16 handle on the calibration frames reproduces the golden (oracle) amax."""
    j = jde()
    h = make_handle(j.JDE_BF16, max_batch=2, src_w=1920, src_h=1080, keep_layer_outputs=1)
    try:
        f = torch.from_numpy(synth.frames_uniform(1000, 2, 1080, 1920)).cuda()
        j.jde_forward(h, f, 2, 1920, 1080, 320, 192, True, torch.cuda.current_stream())
        got = np.array(j.jde_act_amax(h, torch.cuda.current_stream()))
        want = np.array(AMAX)
        np.testing.assert_allclose(got, want, rtol=3e-2)
    finally:
        j.jde_destroy(h)

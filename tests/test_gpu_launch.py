"""Dependent launches of the convolution chain (jde_config.dependent_launch).

With dependent_launch = 1 each convolution kernel may start its set-up while the previous layer's
kernel is still running, and waits for it before touching global memory; the results must be the
same bits as in plain stream order, for BF16 (default and autotuned tiles) and E4M3, and on a
forward captured into a CUDA graph.
"""
import json
import os

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import HEAD_LAYERS, forward, get_tensor, jde, make_handle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fp8_amax_1088x608.json")


def _heads(precision, dependent, frames, in_w, in_h, autotune=False, reps=1):
    j = jde()
    n = frames.shape[0]
    h = make_handle(precision, max_batch=n, in_w=in_w, in_h=in_h, dependent_launch=dependent)
    try:
        if precision == j.JDE_FP8_E4M3:
            j.jde_set_act_amax(h, json.load(open(GOLDEN))["amax"])
        if autotune:
            j.jde_autotune(h, n, in_w, in_h, torch.cuda.current_stream())
        out = None
        for _ in range(reps):
            # forwards back to back: each chain's first kernel follows the last one of the previous forward
            out = forward(h, frames, in_w, in_h)
        assert j.jde_kernel_errors(h) == 0
        return out
    finally:
        j.jde_destroy(h)


@pytest.mark.parametrize("precision,in_w,in_h,n,autotune", [
    ("BF16", 1088, 608, 4, False),
    ("BF16", 1088, 608, 4, True),
    ("BF16", 576, 320, 3, False),
    ("FP8", 1088, 608, 2, False),
])
def test_dependent_launch_gives_the_same_bits(precision, in_w, in_h, n, autotune):
    j = jde()
    p = j.JDE_BF16 if precision == "BF16" else j.JDE_FP8_E4M3
    frames = synth.frames_uniform(31, n, 1080, 1920)
    plain = _heads(p, 0, frames, in_w, in_h, autotune)
    dep = _heads(p, 1, frames, in_w, in_h, autotune, reps=3)
    for a, b, l in zip(plain, dep, HEAD_LAYERS):
        assert np.array_equal(a, b), (precision, in_w, in_h, l, float(np.max(np.abs(a - b))))


def test_dependent_launch_inside_a_captured_graph():
    """The forward captured into a CUDA graph (programmatic edges between the conv kernels) and
    replayed three times on new frames gives the eager forward's bits."""
    j = jde()
    n, in_w, in_h = 2, 1088, 608
    h = make_handle(j.JDE_BF16, max_batch=n, in_w=in_w, in_h=in_h, dependent_launch=1)
    try:
        fa = synth.frames_uniform(41, n, 1080, 1920)
        fb = synth.frames_uniform(42, n, 1080, 1920)
        ref_a = forward(h, fa, in_w, in_h)
        ref_b = forward(h, fb, in_w, in_h)
        src = torch.from_numpy(np.ascontiguousarray(fa)).cuda()
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            j.jde_forward(h, src, n, 1920, 1080, in_w, in_h, True, st)   # warm: plans, tensor maps
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            j.jde_forward(h, src, n, 1920, 1080, in_w, in_h, True, st)
        for frames, ref in ((fb, ref_b), (fa, ref_a), (fb, ref_b)):
            src.copy_(torch.from_numpy(np.ascontiguousarray(frames)).cuda())
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            assert j.jde_kernel_errors(h) == 0
            # the captured forward writes the head set that was current at capture time
            got = [get_tensor(h, l) for l in HEAD_LAYERS]
            for a, b, l in zip(ref, got, HEAD_LAYERS):
                assert np.array_equal(a, b), l
        del g
    finally:
        j.jde_destroy(h)

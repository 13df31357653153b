"""Tile autotuner: tuned forwards give bit-identical layer outputs, and the tuned choice is reported."""
import json
import os

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import jde, make_handle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fp8_amax_320x192.json")


def _layer_outputs(j, h, frames):
    f = torch.from_numpy(frames).cuda()
    j.jde_forward(h, f, frames.shape[0], 320, 192, 320, 192, True, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert j.jde_kernel_errors(h) == 0
    outs = []
    for tid in range(78):
        dims, dt = j.jde_get_tensor(h, tid)
        t = torch.empty(dims, dtype={0: torch.float32, 1: torch.bfloat16, 2: torch.uint8}[dt], device="cuda")
        j.jde_get_tensor(h, tid, t, t.numel() * t.element_size(), torch.cuda.current_stream())
        outs.append(t.view(torch.uint8).cpu().numpy() if dt != 0 else t.cpu().numpy())
    torch.cuda.synchronize()
    return outs


@pytest.mark.parametrize("fp8", [False, True])
def test_autotuned_forward_is_bit_identical(fp8):
    j = jde()
    h = make_handle(j.JDE_FP8_E4M3 if fp8 else j.JDE_BF16, max_batch=2, src_w=320, src_h=192, keep_layer_outputs=1)
    try:
        if fp8:
            j.jde_set_act_amax(h, json.load(open(GOLDEN))["amax"])
        frames = synth.frames_uniform(1, 2, 192, 320)
        before = _layer_outputs(j, h, frames)
        default = j.jde_tile_choice(h, 2, 320, 192)
        j.jde_autotune(h, 2, 320, 192, torch.cuda.current_stream())
        tuned = j.jde_tile_choice(h, 2, 320, 192)
        assert all(b in (32, 64, 128, 256) for b in tuned)
        print("tile widths changed on", sum(a != b for a, b in zip(default, tuned)), "layers:", tuned)
        after = _layer_outputs(j, h, frames)
        for l, (a, b) in enumerate(zip(before, after)):
            np.testing.assert_array_equal(a, b, err_msg=f"layer {l}")
    finally:
        j.jde_destroy(h)

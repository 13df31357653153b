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


def _layer_outputs(j, h, frames, in_w=320, in_h=192):
    f = torch.from_numpy(frames).cuda()
    j.jde_forward(h, f, frames.shape[0], frames.shape[2], frames.shape[1], in_w, in_h, True,
                  torch.cuda.current_stream())
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
        assert all(b in (32, 64, 128, 256, 129, 130) for b in tuned)
        print("tile widths changed on", sum(a != b for a, b in zip(default, tuned)), "layers:", tuned)
        after = _layer_outputs(j, h, frames)
        for l, (a, b) in enumerate(zip(before, after)):
            np.testing.assert_array_equal(a, b, err_msg=f"layer {l}")
    finally:
        j.jde_destroy(h)


def _two_subtile_codes(j, h, n, in_w, in_h, fp8=False):
    """Tile code 129 (128 channels x 256 rows per CTA) on every stride-1 3x3 conv that can take it with
    the same K order as its default tile (64-byte k-blocks: the 128-wide convs of the second stage),
    found by asking jde_set_tile_choice layer by layer."""
    base = j.jde_tile_choice(h, n, in_w, in_h)
    codes = list(base)
    table = j.jde_layer_table()
    for l, (cin, cout, k, stride, _, _) in enumerate(table):
        if not (k == 3 and stride == 1 and cin % 32 == 0 and cout % 128 == 0):
            continue
        trial = list(base)
        trial[l] = 129
        try:
            j.jde_set_tile_choice(h, n, in_w, in_h, trial)
        except j.JdeError:
            continue
        codes[l] = 129
    j.jde_set_tile_choice(h, n, in_w, in_h, base)
    return codes


@pytest.mark.parametrize("fp8,size", [(False, (320, 192)), (True, (320, 192)), (False, (1088, 608))])
def test_two_m_subtiles_per_cta_are_bit_identical(fp8, size):
    """Code 129 runs each flat-window 3x3 conv as 256 rows x 128 channels per CTA (two M sub-tiles sharing
    every weight tile); each output is the same K sum in the same order, so every layer is bit-identical
    to the default tiles."""
    j = jde()
    in_w, in_h = size
    n = 2 if in_w == 320 else 1
    h = make_handle(j.JDE_FP8_E4M3 if fp8 else j.JDE_BF16, max_batch=n, in_w=in_w, in_h=in_h, src_w=in_w,
                    src_h=in_h, keep_layer_outputs=1)
    try:
        if fp8:
            j.jde_set_act_amax(h, json.load(open(GOLDEN))["amax"])
        frames = synth.frames_uniform(3, n, in_h, in_w)
        before = _layer_outputs(j, h, frames, in_w, in_h)
        codes = _two_subtile_codes(j, h, n, in_w, in_h, fp8)
        assert sum(c == 129 for c in codes) >= 2
        j.jde_set_tile_choice(h, n, in_w, in_h, codes)
        assert j.jde_tile_choice(h, n, in_w, in_h) == codes
        after = _layer_outputs(j, h, frames, in_w, in_h)
        for l, (a, b) in enumerate(zip(before, after)):
            np.testing.assert_array_equal(a, b, err_msg=f"layer {l} (code {codes[l]})")
    finally:
        j.jde_destroy(h)


@pytest.mark.parametrize("size", [(320, 192), (1088, 608)])
def test_128_wide_tiles_on_cta_pairs_are_bit_identical(size):
    """Code 130 runs a 128-wide BF16 tile of a stride-1 flat or stride-2 conv on a CTA pair (M = 256 per
    MMA, each CTA loading half of every weight tile); every output is the same K sum in the same order,
    so every layer is bit-identical to the default tiles.  Layers that take it are found by asking
    jde_set_tile_choice layer by layer; flat-window 3x3 convs refuse it."""
    j = jde()
    in_w, in_h = size
    n = 2 if in_w == 320 else 1
    h = make_handle(j.JDE_BF16, max_batch=n, in_w=in_w, in_h=in_h, src_w=in_w, src_h=in_h, keep_layer_outputs=1)
    try:
        frames = synth.frames_uniform(5, n, in_h, in_w)
        before = _layer_outputs(j, h, frames, in_w, in_h)
        base = j.jde_tile_choice(h, n, in_w, in_h)
        codes = list(base)
        table = j.jde_layer_table()
        for l, (cin, cout, k, stride, _, _) in enumerate(table):
            if cout % 128 or cin % 64:
                continue
            trial = list(base)
            trial[l] = 130
            try:
                j.jde_set_tile_choice(h, n, in_w, in_h, trial)
            except j.JdeError:
                assert k == 3 and stride == 1 or l < 2, l   # only flat-window convs (and the fused stem) refuse
                continue
            codes[l] = 130
        j.jde_set_tile_choice(h, n, in_w, in_h, base)
        assert sum(c == 130 for c in codes) >= 10
        j.jde_set_tile_choice(h, n, in_w, in_h, codes)
        assert j.jde_tile_choice(h, n, in_w, in_h) == codes
        after = _layer_outputs(j, h, frames, in_w, in_h)
        for l, (a, b) in enumerate(zip(before, after)):
            np.testing.assert_array_equal(a, b, err_msg=f"layer {l} (code {codes[l]})")
    finally:
        j.jde_destroy(h)


def test_set_tile_choice_refuses_codes_a_layer_cannot_run():
    j = jde()
    h = make_handle(j.JDE_BF16, max_batch=2, src_w=320, src_h=192)
    try:
        codes = j.jde_tile_choice(h, 2, 320, 192)
        bad = list(codes)
        bad[5] = 129                       # a 1x1 conv has no flat-window form
        with pytest.raises(j.JdeError):
            j.jde_set_tile_choice(h, 2, 320, 192, bad)
        bad = list(codes)
        bad[6] = 130                       # a flat-window 3x3 conv has no CTA-pair 128-wide form
        with pytest.raises(j.JdeError):
            j.jde_set_tile_choice(h, 2, 320, 192, bad)
        bad = list(codes)
        bad[5] = 96                        # not a tile width
        with pytest.raises(j.JdeError):
            j.jde_set_tile_choice(h, 2, 320, 192, bad)
        assert j.jde_tile_choice(h, 2, 320, 192) == codes     # the previous choice stands
    finally:
        j.jde_destroy(h)

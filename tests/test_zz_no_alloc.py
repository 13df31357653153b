"""jde_postprocess_noalloc: the post-processing entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc while they run (all device memory reserved
up front by the host application, a real-time loop that must not synchronise
on an allocation, a plugin that only receives device pointers).  For them the
library offers a post-processing call whose scratch is a fixed device array
inside libjde.  These tests check it against jde_postprocess on the same head
tensors, on two different inputs in a row (the shared scratch keeps the first
call's contents, which must not leak into the second), and that an oversized
request is refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synth

from gpu_helpers import heads_to_device, jde, make_handle, postprocess


def _noalloc(heads_dev, n, in_w, in_h, cap, max_cand):
    j = jde()
    rows = torch.full((n, cap, 518), -7.0, dtype=torch.float32, device="cuda")
    count = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    aidx = torch.full((n, cap), -1, dtype=torch.int32, device="cuda")
    d = j.make_dets(rows, count, aidx, cap=cap)
    j.jde_postprocess_noalloc(heads_dev, n, in_w, in_h, 1920, 1080, 0.5, 0.4, max_cand, d,
                              torch.cuda.current_stream())
    torch.cuda.synchronize()
    return rows, count, aidx


@pytest.mark.gpu
def test_noalloc_matches_postprocess_on_two_calls_in_a_row():
    j = jde()
    grids = [(6, 10), (12, 20), (24, 40)]
    h = make_handle(j.JDE_FP32, max_batch=4, max_cand=1024)
    try:
        for seed, mean in ((21, -2.0), (22, -1.0)):      # two calls, different inputs and candidate counts
            dets, embs = synth.random_heads(seed, 4, grids, tobj_mean=mean, tobj_std=1.5)
            heads = heads_to_device(dets, embs)
            rows_r, count_r, aidx_r, _ = postprocess(h, heads, 4, 320, 192, 1920, 1080, cap=1024)
            rows, count, aidx = _noalloc(heads, 4, 320, 192, 1024, 1024)
            assert count.tolist() == count_r.tolist()
            for f in range(4):
                k = int(count_r[f])
                assert torch.equal(aidx[f, :k], aidx_r[f, :k])
                np.testing.assert_allclose(rows[f, :k].cpu().numpy(), rows_r[f, :k].cpu().numpy(),
                                           rtol=1e-6, atol=1e-6)
                assert bool((rows[f, k:] == -7.0).all())      # nothing written past the kept rows
    finally:
        j.jde_destroy(h)


def test_noalloc_refuses_requests_above_its_fixed_scratch():
    j = jde()
    heads = [1] * 6                                          # never dereferenced: refused before any GPU work
    d = j.make_dets(16, 16, None, cap=1, on_device=True)
    with pytest.raises(j.JdeError) as e:
        j.jde_postprocess_noalloc(heads, 16, 1088, 608, 1920, 1080, 0.5, 0.4, 4096, d)
    assert e.value.status == 4 and "scratch" in str(e.value)

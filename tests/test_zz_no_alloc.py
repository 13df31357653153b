"""jde_postprocess_noalloc: the post-processing entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc while they run (all device memory reserved
up front by the host application, a real-time loop that must not synchronise
on an allocation, a plugin that only receives device pointers).  For them the
library offers a post-processing call whose scratch is a fixed device array
inside libjde.  These tests check it against jde_postprocess and against the
oracle's post-processing of the same head tensors, on two different inputs in a
row (the shared scratch keeps the first call's contents, which must not leak
into the second), that a call leaves the device's free memory unchanged, and
that an oversized request is refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import network as net
from oracle import postprocess as pp

from gpu_helpers import heads_to_device, jde, make_handle, nms_tie_frame, postprocess


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


@pytest.mark.gpu
def test_noalloc_matches_the_oracle_and_allocates_nothing():
    """Two calls in a row on different heads: kept sets (sorted canonical indices) bit-exact and rows
    within float32 rounding of the oracle's post-processing (frames with a decision inside the 1e-6 tie
    band are skipped), and the device's free memory is the same before and after the second call."""
    j = jde()
    grids = [(6, 10), (12, 20), (24, 40)]
    n, cap, kmax = 4, 1024, 1024
    r, nw, nh, px, py = net.letterbox_geometry(1920, 1080, 320, 192)
    inputs = [synth.random_heads(seed, n, grids, tobj_mean=mean, tobj_std=1.5) for seed, mean in ((31, -2.0),
                                                                                                (32, -1.5))]
    heads = [heads_to_device(d, e) for d, e in inputs]
    outs = [(torch.full((n, cap, 518), -7.0, device="cuda"), torch.full((n,), -1, dtype=torch.int32, device="cuda"),
             torch.full((n, cap), -1, dtype=torch.int32, device="cuda")) for _ in inputs]
    st = torch.cuda.current_stream()
    compared = 0
    for call, ((dets, embs), hd, (rows, count, aidx)) in enumerate(zip(inputs, heads, outs)):
        d = j.make_dets(rows, count, aidx, cap=cap)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        j.jde_postprocess_noalloc(hd, n, 320, 192, 1920, 1080, 0.5, 0.4, kmax, d, st)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:
            assert free1 == free0, (free0, free1)
        rows_h, count_h, aidx_h = rows.cpu().numpy(), count.cpu().numpy(), aidx.cpu().numpy()
        for f in range(n):
            out = pp.postprocess_frame([x[f] for x in dets], [x[f] for x in embs], r, px, py, k_max=kmax)
            if nms_tie_frame(out):
                continue
            k = len(out["index"])
            assert int(count_h[f]) == k
            np.testing.assert_array_equal(np.sort(aidx_h[f, :k]), np.sort(out["index"]))
            pos = {int(i): p for p, i in enumerate(out["index"])}
            o = out["rows"][[pos[int(i)] for i in aidx_h[f, :k]]]
            np.testing.assert_allclose(rows_h[f, :k, :4], o[:, :4], rtol=1e-5, atol=1e-3)
            np.testing.assert_allclose(rows_h[f, :k, 4:6], o[:, 4:6], rtol=1e-6, atol=1e-7)
            np.testing.assert_allclose(rows_h[f, :k, 6:], o[:, 6:], rtol=0, atol=1e-6)
            assert bool(np.all(rows_h[f, k:] == -7.0))
            compared += 1
    assert compared >= 2 * n - 1


def test_noalloc_refuses_requests_above_its_fixed_scratch():
    j = jde()
    heads = [1] * 6                                          # never dereferenced: refused before any GPU work
    d = j.make_dets(16, 16, None, cap=1, on_device=True)
    with pytest.raises(j.JdeError) as e:
        j.jde_postprocess_noalloc(heads, 16, 1088, 608, 1920, 1080, 0.5, 0.4, 4096, d)
    assert e.value.status == 4 and "scratch" in str(e.value)

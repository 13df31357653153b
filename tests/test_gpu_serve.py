"""Serving loop on the GPU: results alone vs in the mix, memory accounting, admission by budget."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import blob, jde

pytestmark = pytest.mark.gpu

SIZES = [(576, 320), (320, 192)]


def _server(budget=64e9, max_batch=4):
    from paper_2011_03910_gb300 import serve
    j = jde()
    return serve, serve.Server(j, torch, torch.device("cuda", 0), blob(), budget_bytes=int(budget), max_batch=max_batch,
                               max_streams_per_group=4)


def _frames(stream_id):
    fr = torch.from_numpy(synth.frames_uniform(7000 + stream_id, 2, 1080, 1920)).cuda()
    return [fr[0], fr[1]]


def _run(stream_ids, n_frames=6):
    serve, srv = _server()
    specs = [serve.StreamSpec(i, *SIZES[i % 2], n_objects=20 + 10 * i, seed=i) for i in stream_ids]
    for sp in specs:
        assert srv.open_stream(sp, _frames(sp.stream_id), n_frames_hint=n_frames)
    # arrivals interleaved across streams; released at once, so batches mix streams and sizes
    reqs = [serve.Request(0.001 * (k * 8 + sp.stream_id), sp.stream_id, k) for k in range(n_frames) for sp in specs]
    reqs.sort(key=lambda r: r.t)
    stats = srv.run(reqs, collect=True, realtime=False)
    assert stats["frames"] == len(reqs)
    out = {(r.stream_id, r.index): r.outputs for r in reqs}
    for sp in specs:
        srv.close_stream(sp.stream_id)
    assert not srv.groups and srv.ledger.used == 0
    return out


def test_each_stream_gives_the_same_results_alone_and_in_the_mix():
    mix = _run([0, 1, 2, 3])
    for s in range(4):
        alone = _run([s])
        for k in range(6):
            a, m = alone[(s, k)], mix[(s, k)]
            assert a["count"] == m["count"] and a["count"] > 0
            np.testing.assert_array_equal(a["rows"], m["rows"])
            np.testing.assert_array_equal(a["track_id"], m["track_id"])
            np.testing.assert_array_equal(a["track_box"], m["track_box"])
            np.testing.assert_array_equal(a["track_state"], m["track_state"])
            for x, y in zip(a["net_det"], m["net_det"]):      # the forward of the frame, batched differently
                np.testing.assert_array_equal(x, y)
        # tracks persist across frames: ids seen on the last frame were mostly born on the first ones
        assert len(set(alone[(s, 5)]["track_id"]) & set(alone[(s, 1)]["track_id"])) >= 10


def test_device_bytes_match_the_estimate_after_a_full_batch():
    j = jde()
    cfg = j.jde_default_config()
    cfg.precision = j.JDE_BF16
    cfg.max_batch = 4
    cfg.max_in_w, cfg.max_in_h = 576, 320
    h = j.jde_create(cfg, blob())
    try:
        before = j.jde_device_bytes(h)
        fr = torch.from_numpy(synth.frames_uniform(3, 4, 1080, 1920)).cuda()
        rows = torch.zeros((4, 256, 518), device="cuda")
        cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
        dets = j.make_dets(rows, cnt, None, cap=256)
        j.jde_detect_batch(h, fr, 4, 1920, 1080, 576, 320, dets, True, torch.cuda.current_stream())
        torch.cuda.synchronize()
        after = j.jde_device_bytes(h)
        est = j.jde_estimate_device_bytes(cfg, 576, 320)
        assert before < after
        assert 0.95 * est <= after <= 1.05 * est
    finally:
        j.jde_destroy(h)


def test_streams_of_a_size_whose_group_does_not_fit_are_refused():
    serve, srv = _server(max_batch=4)
    big = srv.group_cost(576, 320)
    small = srv.group_cost(320, 192)
    serve, srv = _server(budget=big + small // 2, max_batch=4)
    assert srv.open_stream(serve.StreamSpec(0, 576, 320), _frames(0))
    assert not srv.open_stream(serve.StreamSpec(1, 320, 192), _frames(1))
    assert srv.open_stream(serve.StreamSpec(2, 576, 320), _frames(2))
    assert srv.refused == [1]
    srv.close_stream(0)
    srv.close_stream(2)
    assert srv.ledger.used == 0
    assert srv.open_stream(serve.StreamSpec(1, 320, 192), _frames(1))
    srv.close_stream(1)

"""Native server on the GPU (jde_server_*): results alone vs in the mix, graph replays vs eager
launches, memory accounting, admission by budget."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import blob, jde

pytestmark = pytest.mark.gpu

SIZES = [(576, 320), (320, 192)]


def _server(budget=64e9, max_batch=4, use_graphs=True, collect=True):
    from paper_2011_03910_gb300 import serve
    return serve, serve.Server(jde(), torch, torch.device("cuda", 0), blob(), budget_bytes=int(budget),
                               max_batch=max_batch, max_streams_per_group=4, caller_heads=True,
                               collect_net_heads=collect, use_graphs=use_graphs)


def _frames(stream_id):
    fr = torch.from_numpy(synth.frames_uniform(7000 + stream_id, 2, 1080, 1920)).cuda()
    return [fr[0], fr[1]]


def _planted(serve, spec, T):
    r, px, py = serve.letterbox_geometry(serve.SRC_W, serve.SRC_H, spec.in_w, spec.in_h)
    clip = synth.PlantedClip(100 + spec.seed, spec.n_objects, T, spec.in_w, spec.in_h, serve.anchor_table(),
                             serve.STRIDES, r, px, py, max_speed=min(3.0, 600.0 / (T - 1)))
    return synth.PlantedHeadFrames(clip)


def _run(stream_ids, n_frames=6, use_graphs=True):
    serve, srv = _server(use_graphs=use_graphs)
    specs = [serve.StreamSpec(i, *SIZES[i % 2], n_objects=20 + 10 * i, seed=i) for i in stream_ids]
    for sp in specs:
        assert srv.open_stream(sp, _frames(sp.stream_id), heads=_planted(serve, sp, n_frames))
    # arrivals interleaved across streams; released at once, so batches mix streams and sizes
    reqs = [serve.Request(0.001 * (k * 8 + sp.stream_id), sp.stream_id, k) for k in range(n_frames) for sp in specs]
    reqs.sort(key=lambda r: r.t)
    stats = srv.run(reqs, collect=True, realtime=False)
    assert stats["frames"] == len(reqs)
    out = {(r.stream_id, r.index): r.outputs for r in reqs}
    counters = srv.stats()
    charged, held = srv.device_bytes()
    assert 0 < held <= charged
    for sp in specs:
        srv.close_stream(sp.stream_id)
    assert srv.device_bytes() == (0, 0)
    srv.close()
    return out, counters


def _same(a, m):
    assert a["count"] == m["count"] and a["count"] > 0 and a["errors"] == m["errors"] == 0
    for key in ("rows", "track_id", "track_box", "track_state", "track_det"):
        np.testing.assert_array_equal(a[key], m[key])
    for x, y in zip(a["net_det"], m["net_det"]):      # the forward of the frame, batched differently
        np.testing.assert_array_equal(x, y)


def test_each_stream_gives_the_same_results_alone_and_in_the_mix():
    mix, counters = _run([0, 1, 2, 3])
    # batch sizes repeat from the third batch of a group on: those batches are graph replays
    assert counters["graphs_captured"] >= 1 and counters["graph_replays"] >= 1
    for s in range(4):
        alone, _ = _run([s])
        for k in range(6):
            _same(alone[(s, k)], mix[(s, k)])
        # tracks persist across frames: ids seen on the last frame were mostly born on the first ones
        assert len(set(alone[(s, 5)]["track_id"]) & set(alone[(s, 1)]["track_id"])) >= 10


def test_graph_replays_give_the_eager_results():
    graphs, c1 = _run([0, 2], n_frames=8)
    eager, c2 = _run([0, 2], n_frames=8, use_graphs=False)
    assert c1["graph_replays"] >= 4 and c2["graph_replays"] == 0 and c2["graphs_captured"] == 0
    for key in graphs:
        _same(graphs[key], eager[key])


def _growing_batches(use_graphs):
    """Stream 0 alone (batches of 1), then with streams 1 and 2 (batches of 3), then alone again."""
    serve, srv = _server(use_graphs=use_graphs, collect=False)
    specs = [serve.StreamSpec(i, 576, 320, n_objects=25 + 5 * i, seed=10 + i) for i in range(3)]
    assert srv.open_stream(specs[0], _frames(0), heads=_planted(serve, specs[0], 12))
    out = {}

    def serve_frames(ids, ks):
        reqs = [serve.Request(0.0, i, k) for k in ks for i in ids]
        srv.run(reqs, collect=True, realtime=False)
        out.update({(r.stream_id, r.index): r.outputs for r in reqs})

    serve_frames([0], range(0, 3))
    for sp in specs[1:]:
        assert srv.open_stream(sp, _frames(sp.stream_id), heads=_planted(serve, sp, 12))
    serve_frames([0, 1, 2], range(3, 6))
    for sp in specs[1:]:
        srv.close_stream(sp.stream_id)
    serve_frames([0], range(6, 9))
    counters = srv.stats()
    srv.close()
    return out, counters


def test_batch_sizes_that_grow_after_a_capture_keep_their_graphs_valid():
    """A graph captured for small batches is replayed after a larger batch has run: nothing the graph
    refers to may have moved (the handle's scratch is sized for max_batch at its first use)."""
    g, cg = _growing_batches(True)
    e, ce = _growing_batches(False)
    assert cg["graph_replays"] >= 4 and ce["graph_replays"] == 0
    assert set(g) == set(e)
    for key in g:
        assert g[key]["errors"] == e[key]["errors"] == 0
        for f in ("count", "rows", "track_id", "track_box", "track_state", "track_det"):
            np.testing.assert_array_equal(g[key][f], e[key][f])


def test_server_results_match_direct_library_calls():
    """One stream through the server = jde_forward, jde_postprocess on the same planted heads and
    jde_track_step called directly, frame by frame."""
    serve, srv = _server(collect=False)
    sp = serve.StreamSpec(0, 576, 320, n_objects=30, seed=5)
    planted = _planted(serve, sp, 5)
    frames = _frames(0)
    assert srv.open_stream(sp, frames, heads=planted)
    reqs = [serve.Request(0.0, 0, k) for k in range(5)]
    srv.run(reqs, collect=True, realtime=False)
    srv.close()
    j = jde()
    cfg = j.jde_default_config()
    cfg.precision = j.JDE_BF16
    cfg.max_batch = 4
    cfg.max_in_w, cfg.max_in_h = 576, 320
    cfg.max_streams = 4
    cfg.sparse_emb = 0
    h = j.jde_create(cfg, blob())
    try:
        st = torch.cuda.current_stream()
        bufs = [torch.empty((gh, gw, c), dtype=torch.float32, device="cuda")
                for c in (24, 512) for gh, gw in serve.Server.grids(576, 320)]
        rows = torch.zeros((1, 256, 518), device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        dets = j.make_dets(rows, cnt, None, cap=256)
        tr = [torch.zeros((1, 256), dtype=torch.int64, device="cuda"), torch.zeros((1, 256, 4), device="cuda"),
              torch.zeros((1, 256), dtype=torch.int32, device="cuda"),
              torch.zeros((1, 256), dtype=torch.int32, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda")]
        tracks = j.make_tracks(*tr, cap=256)
        j.jde_stream_reset(h, 0, st)
        for k in range(5):
            planted.write(torch, bufs, k)
            j.jde_forward(h, frames[k % 2], 1, 1920, 1080, 576, 320, True, st)
            j.jde_postprocess(h, bufs, 1, 576, 320, 1920, 1080, dets, st)
            j.jde_track_step(h, [0], dets, tracks, st)
            torch.cuda.synchronize()
            o = reqs[k].outputs
            n, nt = int(cnt[0]), int(tr[4][0])
            assert o["count"] == n > 0 and len(o["track_id"]) == nt
            np.testing.assert_array_equal(o["rows"], rows[0, :n].cpu().numpy())
            np.testing.assert_array_equal(o["track_id"], tr[0][0, :nt].cpu().numpy())
            np.testing.assert_array_equal(o["track_box"], tr[1][0, :nt].cpu().numpy())
            np.testing.assert_array_equal(o["track_state"], tr[2][0, :nt].cpu().numpy())
            np.testing.assert_array_equal(o["track_det"], tr[3][0, :nt].cpu().numpy())
    finally:
        j.jde_destroy(h)


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
    srv.close()
    serve, srv = _server(budget=big + small // 2, max_batch=4)
    pl = lambda sp: _planted(serve, sp, 4)
    specs = [serve.StreamSpec(i, *wh) for i, wh in enumerate([(576, 320), (320, 192), (576, 320)])]
    assert srv.open_stream(specs[0], _frames(0), heads=pl(specs[0]))
    assert not srv.open_stream(specs[1], _frames(1), heads=pl(specs[1]))
    assert srv.open_stream(specs[2], _frames(2), heads=pl(specs[2]))
    assert srv.refused == [1]
    assert srv.device_bytes()[0] == big
    # a fifth stream of the admitted size finds no free slot (4 per group): refused as well
    more = [serve.StreamSpec(10 + i, 576, 320) for i in range(3)]
    assert [srv.open_stream(sp, _frames(0), heads=pl(sp)) for sp in more] == [True, True, False]
    for sp in [specs[0], specs[2]] + more[:2]:
        srv.close_stream(sp.stream_id)
    assert srv.device_bytes() == (0, 0)
    assert srv.open_stream(specs[1], _frames(1), heads=pl(specs[1]))
    assert srv.device_bytes()[0] == small
    srv.close_stream(1)
    srv.close()

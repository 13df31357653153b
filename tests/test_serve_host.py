"""Host logic of the serving loop (no GPU): arrivals, admission ledger, device-memory estimates."""
import numpy as np
import pytest

from paper_2011_03910_gb300 import serve


def specs(n=16):
    sizes = [(1088, 608), (864, 480), (576, 320)]
    return [serve.StreamSpec(i, *sizes[i % 3], fps=30.0) for i in range(n)]


def test_poisson_arrivals_are_seeded_sorted_and_at_the_stream_rate():
    a = serve.poisson_arrivals(specs(), 20.0, seed=4)
    b = serve.poisson_arrivals(specs(), 20.0, seed=4)
    assert [(r.t, r.stream_id) for r in a] == [(r.t, r.stream_id) for r in b]
    assert all(x.t <= y.t for x, y in zip(a, a[1:]))
    per = np.bincount([r.stream_id for r in a], minlength=16)
    # 600 expected frames per stream; Poisson count sd ~ 24.5
    assert np.all(np.abs(per - 600) < 6 * 24.5)
    # frame numbers of each stream are consecutive from 0
    for s in range(16):
        idx = [r.index for r in a if r.stream_id == s]
        assert idx == list(range(len(idx)))
    gaps = np.diff([r.t for r in a if r.stream_id == 0])
    assert abs(gaps.mean() - 1 / 30) < 0.005


def test_estimated_device_bytes_scale_with_input_size_and_batch():
    from paper_2011_03910_gb300 import jde
    cfg = jde.jde_default_config()
    cfg.precision = jde.JDE_BF16
    cfg.max_batch = 16
    est = [jde.jde_estimate_device_bytes(cfg, w, h) for w, h in [(1088, 608), (864, 480), (576, 320)]]
    assert est[0] > est[1] > est[2] > 0
    cfg.max_batch = 8
    half = jde.jde_estimate_device_bytes(cfg, 1088, 608)
    assert half < est[0]
    # the batch-dependent part (activations, post-processing scratch) is most of it
    assert est[0] - half > 0.4 * (est[0] - 0.131e9)
    with pytest.raises(jde.JdeError):
        jde.jde_estimate_device_bytes(cfg, 1100, 608)      # not a multiple of 32


def _server_cfg(caller_heads=0, collect=0, batch=16):
    from paper_2011_03910_gb300 import jde
    c = jde.jde_default_server_config()
    c.group.precision = jde.JDE_BF16
    c.group.max_batch = batch
    c.caller_heads, c.collect_net_heads = caller_heads, collect
    return c


def test_server_group_cost_is_the_handle_estimate_plus_the_batch_buffers():
    """jde_server_group_cost (host arithmetic, no GPU): the handle's estimate for the group's size plus
    frames, caller heads, detection rows, track outputs, collected detection maps and stream slots."""
    from paper_2011_03910_gb300 import jde
    B, W, H = 16, 1088, 608
    cells = sum((H // s) * (W // s) for s in (32, 16, 8))
    for caller, collect in [(0, 0), (1, 0), (1, 1), (0, 1)]:
        c = _server_cfg(caller, collect, B)
        g = jde.jde_config.from_buffer_copy(c.group)
        g.max_in_w, g.max_in_h, g.max_src_w, g.max_src_h = W, H, 1920, 1080
        g.max_streams = c.max_streams_per_group
        if caller:
            g.sparse_emb = 0          # the forward computes the embedding maps densely
        est = jde.jde_estimate_device_bytes(g, W, H)
        buf = (B * 1920 * 1080 * 3 + caller * B * cells * 536 * 4 + B * c.det_cap * 518 * 4 + B * 4 +
               B * c.track_cap * 32 + B * 4 + collect * B * cells * 24 * 4 + B * 4)
        assert jde.jde_server_group_cost(c, W, H) == est + buf
    with pytest.raises(jde.JdeError):
        jde.jde_server_group_cost(_server_cfg(), 1100, 608)     # not a multiple of 32
    bad = _server_cfg()
    bad.group.max_batch = 65
    with pytest.raises(jde.JdeError):
        jde.jde_server_group_cost(bad, 1088, 608)


def test_server_group_cost_orders_the_serving_sizes():
    from paper_2011_03910_gb300 import jde
    c = _server_cfg()
    cost = [jde.jde_server_group_cost(c, w, h) for w, h in [(1088, 608), (864, 480), (576, 320)]]
    assert cost[0] > cost[1] > cost[2] > 16 * 1920 * 1080 * 3
    # with caller heads the dense embedding maps come back into the handle and the heads into the group
    c1 = _server_cfg(caller_heads=1)
    assert jde.jde_server_group_cost(c1, 1088, 608) > cost[0]


def _act_bytes(n, hw, c, el, pad=1):
    h, w = hw
    return n * (h + 2 * pad) * (w + 2 * pad) * c * el


def test_estimate_accounts_for_in_place_stages_the_fused_stem_and_the_sparse_embedding_head():
    """Host bookkeeping of the activation buffers (no GPU): with keep_layer_outputs = 0 every residual
    block's output shares its stage buffer (the 3x3 reduce-adds into the block input; the stride-16 and
    stride-8 stages live in their concat slices), and with sparse_emb = 1 the three f32 embedding maps
    (two sets, zero halo) are replaced by two-set bf16 copies of their input maps; fuse_block1 = 1
    keeps the first block's output in its own tensor and its 1x1 output (layer 2) on chip."""
    from paper_2011_03910_gb300 import jde
    n, W, H = 16, 1088, 608
    table = jde.jde_layer_table()

    def est(keep, sparse):
        cfg = jde.jde_default_config()
        cfg.precision = jde.JDE_BF16
        cfg.max_batch = n
        cfg.keep_layer_outputs = keep
        cfg.sparse_emb = sparse
        return jde.jde_estimate_device_bytes(cfg, W, H)

    # spatial size of every layer output (stem at full size, five stride-2 stages, three scales)
    sizes, h, w = [(H, W)], H, W
    stage_blocks = [1, 2, 8, 8, 4]
    stage_first = []
    for nb in stage_blocks:
        h, w = h // 2, w // 2
        stage_first.append(len(sizes))
        sizes += [(h, w)] * (1 + 2 * nb)
    for i, s in enumerate((32, 16, 8)):
        sizes += [(H // s, W // s)] * (9 if i < 2 else 8)
    assert len(sizes) == len(table) == 78
    # in place: a stage's block outputs (the last block of stages 3 and 4 is a concat slice in both
    # layouts) and the downsampling outputs of stages 3 and 4 (they move into the concat slices)
    saved = 0
    for s, (first, nb) in enumerate(zip(stage_first, stage_blocks)):
        blocks = [first + 2 + 2 * b for b in range(nb)]
        if s in (2, 3):
            blocks = blocks[:-1] + [first]
        saved += sum(_act_bytes(n, sizes[l], table[l][1], 2) for l in blocks)
    # the stem's output (32 channels at full size) is not stored when it is fused into layer 1
    saved += _act_bytes(n, sizes[0], table[0][1], 2)
    assert est(1, 0) - est(0, 0) == saved
    cfg = jde.jde_default_config()
    cfg.precision = jde.JDE_BF16
    cfg.max_batch = n
    cfg.sparse_emb = 0
    cfg.fuse_block1 = 1
    fused = jde.jde_estimate_device_bytes(cfg, W, H)
    assert fused - est(0, 0) == _act_bytes(n, sizes[3], table[3][1], 2) - _act_bytes(n, sizes[2], table[2][1], 2)
    # sparse head: minus the padded f32 embedding maps, plus bf16 copies of their inputs (two sets each)
    emb = [59, 68, 77]
    dense = sum(2 * _act_bytes(n, sizes[l], 512, 4) for l in emb)
    copies = sum(2 * _act_bytes(n, sizes[l], table[l][0], 2) for l in emb)
    assert est(0, 0) - est(0, 1) == dense - copies


def test_smooth_frames_are_seeded_and_structured():
    """synth.frames_smooth: the same seed gives the same frames, other seeds others; neighbouring pixels
    are close (structure, unlike uniform noise)."""
    import synth
    a = synth.frames_smooth(3, 2, 64, 96)
    b = synth.frames_smooth(3, 2, 64, 96)
    c = synth.frames_smooth(4, 2, 64, 96)
    assert a.shape == (2, 64, 96, 3) and a.dtype == np.uint8
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    step = np.abs(np.diff(a.astype(int), axis=2)).mean()
    noise = np.abs(np.diff(synth.frames_uniform(3, 2, 64, 96).astype(int), axis=2)).mean()
    assert step < 6 and noise > 60

"""Pins of the oracle decode / filter / NMS / embedding steps (CPU)."""
import math

import numpy as np
import pytest

import synth
from oracle import network as net
from oracle import postprocess as pp


def empty_heads(grids):
    dets = []
    for (h, w) in grids:
        d = np.zeros((h, w, 24), np.float32)
        d[..., 4::6] = -20.0
        dets.append(d)
    return dets, [np.zeros((h, w, 512), np.float32) for (h, w) in grids]


GRIDS = [(6, 10), (12, 20), (24, 40)]   # 320x192 input


def test_anchor_table():
    a = pp.anchors()
    assert len(a) == 3 and all(len(s) == 4 for s in a)
    np.testing.assert_allclose([w for w, _ in a[2]], [8, 8 * 2 ** 0.5, 16, 16 * 2 ** 0.5])
    np.testing.assert_allclose([w for w, _ in a[1]], [32, 32 * 2 ** 0.5, 64, 64 * 2 ** 0.5])
    np.testing.assert_allclose([w for w, _ in a[0]], [128, 128 * 2 ** 0.5, 256, 256 * 2 ** 0.5])
    for s in a:
        for w, h in s:
            assert h == 3 * w


def test_decode_zero_logits_and_canonical_index():
    dets, embs = empty_heads(GRIDS)
    s, a, y, x = 1, 2, 5, 7
    dets[s][y, x, 6 * a:6 * a + 6] = 0.0
    idx, boxes, conf, cls = pp.decode(dets)
    off = 4 * 6 * 10
    gi = off + (a * 12 + y) * 20 + x
    assert conf[gi] == 0.5 and cls[gi] == 0.5
    aw, ah = pp.anchors()[s][a]
    cx, cy = (x + 0.5) * 16, (y + 0.5) * 16
    np.testing.assert_allclose(boxes[gi], [cx - aw / 2, cy - ah / 2, cx + aw / 2, cy + ah / 2], rtol=1e-15)
    assert np.sum(conf >= 0.5) == 1          # only the planted anchor passes (ties at 0.5 kept)


def test_decode_saturation():
    dets, _ = empty_heads(GRIDS)
    dets[0][0, 0, 0:6] = [50.0, -50.0, 30.0, -30.0, 40.0, -40.0]
    idx, boxes, conf, cls = pp.decode(dets)
    aw, ah = pp.anchors()[0][0]
    w, h = aw * math.exp(10), ah * math.exp(-10)
    cx, cy = (0 + 1.0) * 32, (0 + pp.sigmoid(-50.0)) * 32
    np.testing.assert_allclose(boxes[0], [cx - w / 2, cy - h / 2, cx + w / 2, cy + h / 2], rtol=1e-12)
    assert conf[0] == 1.0 and cls[0] < 1e-17


@pytest.mark.parametrize("a,b,expect", [
    ([0, 0, 2, 2], [0, 0, 2, 2], 1.0), ([0, 0, 1, 1], [2, 2, 3, 3], 0.0), ([0, 0, 2, 1], [1, 0, 3, 1], 1 / 3),
    ([0, 0, 4, 4], [1, 1, 3, 3], 0.25), ([0, 0, 1, 1], [1, 0, 2, 1], 0.0), ([0, 0, 0, 0], [0, 0, 0, 0], 0.0)])
def test_iou_hand_cases(a, b, expect):
    assert pp.iou(np.array(a, float), np.array(b, float)) == pytest.approx(expect, abs=1e-15)
    assert pp.iou_many(np.array(a, float), np.array([b], float))[0] == pytest.approx(expect, abs=1e-15)


def test_nms_iou_exactly_threshold_is_kept():
    boxes = np.array([[0, 0, 5, 1], [0, 0, 2, 1]], float)      # IoU = 2 / 5, exactly the literal 0.4
    assert pp.iou(boxes[0], boxes[1]) == 0.4
    assert list(pp.greedy_nms(boxes, 0.4)) == [0, 1]
    assert list(pp.greedy_nms(boxes, 0.39)) == [0]


def test_nms_chain():
    # A suppresses B (IoU 0.6), B would suppress C (0.6) but A-C overlap is 0.2: C survives
    A = [0, 0, 10, 1]
    B = [2.5, 0, 12.5, 1]
    C = [5, 0, 15, 1]
    boxes = np.array([A, B, C], float)
    assert pp.iou(boxes[0], boxes[1]) > 0.4 and pp.iou(boxes[1], boxes[2]) > 0.4 and pp.iou(boxes[0], boxes[2]) < 0.4
    assert list(pp.greedy_nms(boxes)) == [0, 2]


def test_sort_ties_by_index():
    conf = np.array([0.7, 0.9, 0.7, 0.9, 0.8])
    idx = np.array([10, 3, 2, 7, 5])
    assert list(idx[pp.sort_candidates(conf, idx)]) == [3, 7, 5, 2, 10]


def test_nms_greedy_characterisation_random():
    """Greedy NMS is the unique set with: no kept pair above the threshold, and every dropped
    box above the threshold with some kept box ranked before it."""
    g = np.random.default_rng(11)
    for trial in range(30):
        n = g.integers(1, 120)
        c = g.uniform(0, 100, (n, 2))
        wh = g.uniform(5, 40, (n, 2))
        boxes = np.concatenate([c - wh / 2, c + wh / 2], 1)
        keep = pp.greedy_nms(boxes)
        ks = set(keep.tolist())
        for i in range(n):
            over = [j for j in keep if j < i and pp.iou(boxes[i], boxes[j]) > 0.4]
            if i in ks:
                assert not over
            else:
                assert over


def test_conf_cap_keeps_best_by_conf_then_index():
    dets, embs = empty_heads(GRIDS)
    for s in range(3):
        dets[s][..., 4::6] = 3.0                  # every anchor passes with equal confidence
    dets[2][0, 0, 4] = 5.0                        # one stronger anchor in the last head
    out = pp.postprocess_frame(dets, embs, 1.0, 0, 0, k_max=100)
    assert out["n_candidates"] == 4 * (60 + 240 + 960)
    cand = out["candidates"]
    assert len(cand) == 100
    first = 4 * (60 + 240)
    assert cand[0] == first and list(cand[1:]) == list(range(99))


def test_planted_clip_roundtrip():
    r, nw, nh, px, py = net.letterbox_geometry(1920, 1080, 1088, 608)
    clip = synth.PlantedClip(5, 20, 3, 1088, 608, pp.anchors(), pp.STRIDES, r, px, py)
    dets, embs, truth = clip.frame(1)
    out = pp.postprocess_frame(dets, embs, r, px, py)
    rows = out["rows"]
    assert 0 < len(rows) <= len(truth)
    found = 0
    for (o, cx, cy, w, h) in truth:
        d = np.hypot((rows[:, 0] + rows[:, 2]) / 2 - cx, (rows[:, 1] + rows[:, 3]) / 2 - cy)
        j = int(np.argmin(d))
        if d[j] > 1e-6 * 1920:
            # not detected: it must overlap a kept box above the NMS threshold
            box = np.array([cx - w / 2, cy - h / 2, cx + w / 2, cy + h / 2])
            assert np.max(pp.iou_many(box, rows[:, :4])) > 0.4
            continue
        found += 1
        np.testing.assert_allclose(rows[j, 2] - rows[j, 0], w, rtol=1e-6)   # logits are float32
        np.testing.assert_allclose(rows[j, 3] - rows[j, 1], h, rtol=1e-6)
        assert rows[j, 6:] @ clip.ident[o] > 0.99
        assert abs(np.linalg.norm(rows[j, 6:]) - 1) < 1e-12
    assert found == len(rows)

"""Oracle post-processing of the head tensors (Sec. 3.2, Appendix A steps 1-3).

* Decode (Sec. 3.1: detection "in the same manner as YOLOv3").  Reading: per
  anchor a the channels 6a..6a+5 hold (tx, ty, tw, th, t_obj, t_cls);
  cx = (x + sigmoid(tx)) s, cy = (y + sigmoid(ty)) s,
  w = anchor_w exp(clamp(tw, -10, 10)), h = anchor_h exp(clamp(th, -10, 10)),
  conf = sigmoid(t_obj), cls = sigmoid(t_cls); boxes are xyxy in letterbox
  pixels and are mapped back to frame pixels by (v - pad) / r.
* Anchors (not printed in the paper): pedestrian-shaped, h = 3 w, four per
  scale in a sqrt(2) progression from w = 8 (stride 8), 32 (stride 16) and 128
  (stride 32).
* Canonical index of an anchor: off_s + (a H_s + y) W_s + x with heads ordered
  by stride 32, 16, 8.
* Confidence filter (Appendix A): a detection whose score is below the
  threshold is discarded, so conf >= threshold is kept.  At most
  ``k_max`` candidates survive, the best by (conf descending, index ascending).
* NMS (Appendix A): sort by confidence, then drop any detection whose IoU with
  an already kept, higher-scored detection is above the threshold (strictly
  greater).  Class-agnostic, over all three scales of a frame.
* IoU of continuous boxes without the +1 convention; 0 for an empty union.
* Embedding (Appendix A: the last 512 values of the detection row) is the
  embedding map at the anchor's cell, L2-normalised (zero stays zero).

Each frame yields rows of 518 values: x1, y1, x2, y2 (frame px), conf, cls and
the 512-d unit embedding, in kept order.
"""
from __future__ import annotations

import math

import numpy as np

STRIDES = (32, 16, 8)
CONF_THRESH = 0.5
NMS_IOU = 0.4
K_MAX = 4096


def anchors():
    """Anchor (w, h) per head, heads ordered by stride 32, 16, 8."""
    out = []
    for base in (128.0, 32.0, 8.0):
        out.append([(base * math.sqrt(2.0) ** i, 3.0 * base * math.sqrt(2.0) ** i) for i in range(4)])
    return out


def sigmoid(t):
    return 1.0 / (1.0 + np.exp(-t))


def decode(dets_frame):
    """All anchors of one frame: ``(index, box_xyxy_letterbox, conf, cls)`` in canonical order.

    ``dets_frame[s]`` is the ``[H_s, W_s, 24]`` map of head s.
    """
    boxes, conf, cls = [], [], []
    for s, (d, st, anc) in enumerate(zip(dets_frame, STRIDES, anchors())):
        d = np.asarray(d, np.float64)
        h, w, _ = d.shape
        ys, xs = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
        for a in range(4):
            t = d[..., 6 * a:6 * a + 6]
            cx = (xs + sigmoid(t[..., 0])) * st
            cy = (ys + sigmoid(t[..., 1])) * st
            bw = anc[a][0] * np.exp(np.clip(t[..., 2], -10.0, 10.0))
            bh = anc[a][1] * np.exp(np.clip(t[..., 3], -10.0, 10.0))
            b = np.stack([cx - bw / 2, cy - bh / 2, cx + bw / 2, cy + bh / 2], -1)
            boxes.append(b.reshape(-1, 4))
            conf.append(sigmoid(t[..., 4]).reshape(-1))
            cls.append(sigmoid(t[..., 5]).reshape(-1))
    boxes = np.concatenate(boxes)
    return np.arange(len(boxes)), boxes, np.concatenate(conf), np.concatenate(cls)


def iou(a, b):
    """IoU of two xyxy boxes."""
    iw = max(0.0, min(a[2], b[2]) - max(a[0], b[0]))
    ih = max(0.0, min(a[3], b[3]) - max(a[1], b[1]))
    inter = iw * ih
    union = (a[2] - a[0]) * (a[3] - a[1]) + (b[2] - b[0]) * (b[3] - b[1]) - inter
    return inter / union if union > 0 else 0.0


def iou_many(a, bs):
    """IoU of box ``a`` with each row of ``bs`` (same formula as ``iou``)."""
    iw = np.maximum(0.0, np.minimum(a[2], bs[:, 2]) - np.maximum(a[0], bs[:, 0]))
    ih = np.maximum(0.0, np.minimum(a[3], bs[:, 3]) - np.maximum(a[1], bs[:, 1]))
    inter = iw * ih
    union = (a[2] - a[0]) * (a[3] - a[1]) + (bs[:, 2] - bs[:, 0]) * (bs[:, 3] - bs[:, 1]) - inter
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(union > 0, inter / np.where(union > 0, union, 1.0), 0.0)


def sort_candidates(conf, index):
    """Order by conf descending, ties by canonical index ascending."""
    return np.lexsort((index, -conf))


def greedy_nms(boxes, iou_thresh=NMS_IOU):
    """Greedy NMS over boxes already in score order; returns kept positions."""
    n = len(boxes)
    removed = np.zeros(n, bool)
    keep = []
    for i in range(n):
        if removed[i]:
            continue
        keep.append(i)
        if i + 1 < n:
            removed[i + 1:] |= iou_many(boxes[i], boxes[i + 1:]) > iou_thresh
    return np.array(keep, np.int64)


def postprocess_frame(dets_frame, embs_frame, ratio, pad_x, pad_y,
                      conf_thresh=CONF_THRESH, iou_thresh=NMS_IOU, k_max=K_MAX):
    """Decode, filter, sort, NMS and gather embeddings for one frame.

    Returns a dict with ``rows`` ``[K, 518]`` float64 in kept order, ``index``
    (canonical anchor index per row), ``n_candidates`` (before the k_max cap)
    and ``candidates`` (the sorted, capped candidate indices).
    """
    idx, boxes, conf, cls = decode(dets_frame)
    m = conf >= conf_thresh
    idx, boxes, conf, cls = idx[m], boxes[m], conf[m], cls[m]
    order = sort_candidates(conf, idx)
    n_cand = len(order)
    order = order[:k_max]
    idx, boxes, conf, cls = idx[order], boxes[order], conf[order], cls[order]
    keep = greedy_nms(boxes, iou_thresh)
    rows = np.zeros((len(keep), 518))
    grids = [e.shape[:2] for e in embs_frame]
    offs = np.cumsum([0] + [4 * h * w for (h, w) in grids])
    for r, p in enumerate(keep):
        b = boxes[p]
        rows[r, 0] = (b[0] - pad_x) / ratio
        rows[r, 1] = (b[1] - pad_y) / ratio
        rows[r, 2] = (b[2] - pad_x) / ratio
        rows[r, 3] = (b[3] - pad_y) / ratio
        rows[r, 4] = conf[p]
        rows[r, 5] = cls[p]
        gi = int(idx[p])
        s = int(np.searchsorted(offs, gi, side="right") - 1)
        h, w = grids[s]
        loc = (gi - offs[s]) % (h * w)
        v = np.asarray(embs_frame[s][loc // w, loc % w], np.float64)
        nrm = math.sqrt(float(v @ v))
        rows[r, 6:] = v / nrm if nrm > 0 else 0.0
    return dict(rows=rows, index=idx[keep], n_candidates=n_cand, candidates=idx, cand_conf=conf,
                cand_boxes=boxes)

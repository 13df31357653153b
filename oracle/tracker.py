"""Oracle tracker: Kalman filter, cosine cost, gating, Hungarian, lifecycle (float64).

Follows Sec. 3 ("Location Estimation", "Association") and the tracker steps of
Appendix A, in their order:

1. predict every active or lost track to the current frame (Kalman filter);
2. cost = cosine distance between track and detection embeddings;
3. motion gating: a pair whose predicted-to-detected distance exceeds the
   gate gets an "infinite" cost;
4. Hungarian assignment on the cost matrix, then Kalman update of the
   assigned tracks; pairs costing more than the assignment threshold are
   rejected; an assigned track becomes active;
5. tracks with no detection become lost; lost tracks older than the limit
   are removed.

Readings where the paper is silent:

* Kalman model: constant velocity on (cx, cy, a = w/h, h) with dt = 1 and
  height-proportional noise, sigma_p = 1/20, sigma_v = 1/160:
  Q = diag((sp h)^2, (sp h)^2, 1e-4, (sp h)^2, (sv h)^2, (sv h)^2, 1e-10, (sv h)^2)
  with h the height of the mean being predicted; R = diag((sp h)^2, (sp h)^2,
  1e-2, (sp h)^2) with h the predicted height; new tracks start with
  P0 = diag((2 sp h)^2, (2 sp h)^2, 1e-4, (2 sp h)^2, (10 sv h)^2, (10 sv h)^2,
  1e-10, (10 sv h)^2) from the measured h.  Update: K = P H^T S^-1,
  x += K (z - H x), P -= K S K^T.
* Distance for gating: squared Mahalanobis distance d^2 = y^T S^-1 y via the
  Cholesky factor of S; gated when d^2 > chi2_0.95(4) = 9.487729036781154.
* "Infinite" cost is the finite value 1e5; after assignment a pair is rejected
  when its cost exceeds 0.7 (or is the gated value).
* Hungarian: shortest augmenting paths with row/column potentials.  Rows are
  the tracks (in creation order) and columns the detections (in kept order);
  when there are more tracks than detections the matrix is transposed so that
  rows <= columns.  Columns are scanned in ascending order and the first
  minimum wins.
* Track set for the cost and the prediction: active and lost tracks.
* Birth: every unassigned detection starts a new active track; ids count from
  1 per stream, handed out in kept order.
* Embedding gallery: on assignment e <- normalise(0.9 e + 0.1 d); a new track
  starts from its detection's embedding.
* Lost limit: a track is removed once its frames since the last update
  exceed 30.
"""
from __future__ import annotations

import math

import numpy as np

STD_POS = 1.0 / 20
STD_VEL = 1.0 / 160
GATE_CHI2 = 9.487729036781154
INF_COST = 1e5
ASSIGN_THRESH = 0.7
LOST_MAX = 30
EMB_MOMENTUM = 0.9

TRACKED, LOST = 1, 2

F = np.eye(8)
for _i in range(4):
    F[_i, _i + 4] = 1.0
H = np.eye(4, 8)


def xyxy_to_z(b):
    """Box (x1, y1, x2, y2) -> measurement (cx, cy, a = w/h, h)."""
    w, h = b[2] - b[0], b[3] - b[1]
    return np.array([b[0] + w / 2, b[1] + h / 2, w / h, h])


def z_to_xyxy(m):
    """State mean (cx, cy, a, h, ...) -> box (x1, y1, x2, y2)."""
    w = m[2] * m[3]
    return np.array([m[0] - w / 2, m[1] - m[3] / 2, m[0] + w / 2, m[1] + m[3] / 2])


def initiate(z):
    h = z[3]
    std = np.array([2 * STD_POS * h, 2 * STD_POS * h, 1e-2, 2 * STD_POS * h,
                    10 * STD_VEL * h, 10 * STD_VEL * h, 1e-5, 10 * STD_VEL * h])
    return np.concatenate([z, np.zeros(4)]), np.diag(std ** 2)


def process_noise(h):
    std = np.array([STD_POS * h, STD_POS * h, 1e-2, STD_POS * h, STD_VEL * h, STD_VEL * h, 1e-5, STD_VEL * h])
    return np.diag(std ** 2)


def measurement_noise(h):
    std = np.array([STD_POS * h, STD_POS * h, 1e-1, STD_POS * h])
    return np.diag(std ** 2)


def predict(mean, cov, q=None):
    """x <- F x, P <- F P F^T + Q (Q from the pre-prediction height unless given)."""
    if q is None:
        q = process_noise(mean[3])
    return F @ mean, F @ cov @ F.T + q


def project(mean, cov, r=None):
    """Measurement-space mean H x and innovation covariance S = H P H^T + R."""
    if r is None:
        r = measurement_noise(mean[3])
    return H @ mean, H @ cov @ H.T + r


def cholesky_lower(a):
    """Plain Cholesky factorisation A = L L^T (lower triangular)."""
    n = a.shape[0]
    L = np.zeros_like(a)
    for j in range(n):
        s = a[j, j] - L[j, :j] @ L[j, :j]
        L[j, j] = math.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (a[i, j] - L[i, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_sub(L, b):
    """Solve L y = b for lower-triangular L (b a vector, or a matrix of column right-hand sides)."""
    y = np.zeros_like(b, dtype=np.float64)
    for i in range(len(b)):
        y[i] = (b[i] - L[i, :i] @ y[:i]) / L[i, i]
    return y


def back_sub_t(L, y):
    """Solve L^T x = y for lower-triangular L."""
    n = len(y)
    x = np.zeros_like(y, dtype=np.float64)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def mahalanobis2(mean, cov, z):
    """Squared Mahalanobis distance of measurement z from the track's projection."""
    zh, S = project(mean, cov)
    L = cholesky_lower(S)
    w = forward_sub(L, z - zh)
    return float(w @ w)


def update(mean, cov, z, r=None):
    """Kalman update with measurement z: K = P H^T S^-1, x += K y, P -= K S K^T."""
    zh, S = project(mean, cov, r)
    L = cholesky_lower(S)
    PHt = cov @ H.T                       # 8x4
    # K^T = S^-1 (P H^T)^T, column by column through the Cholesky factor
    Kt = np.stack([back_sub_t(L, forward_sub(L, PHt[i])) for i in range(8)], 1)
    K = Kt.T
    y = z - zh
    return mean + K @ y, cov - K @ S @ K.T


def hungarian(cost):
    """Minimum-cost assignment by shortest augmenting paths (rows <= columns).

    Returns ``col_of_row`` (length n, column index per row).  Potentials u, v;
    ``p[j]`` the row assigned to column j (1-based, 0 = none); columns are
    scanned in ascending order and the first minimal column wins.
    """
    a = np.asarray(cost, np.float64)
    n, m = a.shape
    assert n <= m
    INF = math.inf
    u = np.zeros(n + 1)
    v = np.zeros(m + 1)
    p = np.zeros(m + 1, np.int64)
    way = np.zeros(m + 1, np.int64)
    for i in range(1, n + 1):
        p[0] = i
        j0 = 0
        minv = np.full(m + 1, INF)
        used = np.zeros(m + 1, bool)
        while True:
            used[j0] = True
            i0 = p[j0]
            free = ~used[1:]
            cur = (a[i0 - 1, :] - u[i0]) - v[1:]
            better = free & (cur < minv[1:])
            minv[1:][better] = cur[better]
            way[1:][better] = j0
            cand = np.where(free, minv[1:], INF)
            j1 = int(np.argmin(cand)) + 1
            delta = cand[j1 - 1]
            uj = np.nonzero(used)[0]
            u[p[uj]] += delta
            v[uj] -= delta
            nf = np.nonzero(~used)[0]
            minv[nf] -= delta
            j0 = j1
            if p[j0] == 0:
                break
        while True:
            j1 = way[j0]
            p[j0] = p[j1]
            j0 = j1
            if j0 == 0:
                break
    col_of_row = np.full(n, -1, np.int64)
    for j in range(1, m + 1):
        if p[j]:
            col_of_row[p[j] - 1] = j - 1
    return col_of_row


def assign(cost):
    """Rectangular assignment: list of (track i, det j) pairs, transposing when T > K."""
    T, K = cost.shape
    if T == 0 or K == 0:
        return []
    if T <= K:
        c = hungarian(cost)
        return [(i, int(c[i])) for i in range(T)]
    c = hungarian(cost.T)
    return sorted((int(c[j]), j) for j in range(K))


class Track:
    __slots__ = ("id", "state", "mean", "cov", "emb", "since")

    def __init__(self, tid, z, emb):
        self.id = tid
        self.state = TRACKED
        self.mean, self.cov = initiate(z)
        self.emb = np.asarray(emb, np.float64).copy()
        self.since = 0


class Tracker:
    """Per-stream tracker state and one step of the Appendix A association."""

    def __init__(self, gate=GATE_CHI2, assign_thresh=ASSIGN_THRESH, lost_max=LOST_MAX,
                 momentum=EMB_MOMENTUM):
        self.tracks: list[Track] = []
        self.next_id = 1
        self.gate, self.assign_thresh, self.lost_max, self.momentum = gate, assign_thresh, lost_max, momentum
        self.last = {}

    def step(self, rows):
        """Advance one frame with detection rows ``[K, 518]`` (kept order).

        Returns a list of ``(id, state, box_xyxy)`` for the surviving tracks,
        in track order; diagnostics of the step are kept in ``self.last``.
        """
        rows = np.asarray(rows, np.float64).reshape(-1, 518)
        K = len(rows)
        pool = self.tracks
        for t in pool:
            t.mean, t.cov = predict(t.mean, t.cov)
        zs = [xyxy_to_z(r[:4]) for r in rows]
        Z = np.array(zs).reshape(-1, 4)
        T = len(pool)
        cost = np.zeros((T, K))
        d2 = np.zeros((T, K))
        for i, t in enumerate(pool):
            cost[i] = 1.0 - rows[:, 6:] @ t.emb
            zh, S = project(t.mean, t.cov)
            L = cholesky_lower(S)
            W = forward_sub(L, (Z - zh).T)          # column j: L^-1 (z_j - H x)
            d2[i] = (W * W).sum(0)
        raw = cost.copy()
        cost[d2 > self.gate] = INF_COST
        pairs = assign(cost)
        matched_t, matched_d = set(), set()
        for i, j in pairs:
            if cost[i, j] > self.assign_thresh or cost[i, j] >= INF_COST:
                continue
            t = pool[i]
            t.mean, t.cov = update(t.mean, t.cov, zs[j])
            e = self.momentum * t.emb + (1 - self.momentum) * rows[j, 6:]
            t.emb = e / math.sqrt(float(e @ e))
            t.state = TRACKED
            t.since = 0
            matched_t.add(i)
            matched_d.add(j)
        det_track = [None] * K
        for i, j in pairs:
            if i in matched_t and j in matched_d:
                det_track[j] = pool[i].id
        survivors = []
        for i, t in enumerate(pool):
            if i not in matched_t:
                t.state = LOST
                t.since += 1
                if t.since > self.lost_max:
                    continue
            survivors.append(t)
        for j in range(K):
            if j not in matched_d:
                survivors.append(Track(self.next_id, zs[j], rows[j, 6:]))
                det_track[j] = self.next_id
                self.next_id += 1
        self.tracks = survivors
        self.last = dict(cost=raw, d2=d2, gated=cost, pairs=pairs, det_track=det_track,
                         matches=sorted((pool[i].id, j) for i, j in pairs if i in matched_t and j in matched_d))
        return [(t.id, t.state, z_to_xyxy(t.mean)) for t in self.tracks]


# ----------------------------------------------------------------------------- association cascade
# The cited JDE tracker associates in three stages instead of Appendix A's single one (readings; this
# paper's Appendix A does not describe them):
#  1. confirmed tracks (tracked or lost) against all detections on a motion-fused cost
#     lambda (1 - cos) + (1 - lambda) d^2, lambda = 0.98, with the same gate (d^2 > gate -> "infinite")
#     and the same rejection (cost > 0.7 or infinite);
#  2. the confirmed tracks left unmatched that were tracked (not lost) before this frame, against the
#     detections left, on 1 - IoU(predicted box, detection box); reject 1 - IoU > 0.5;
#  3. unconfirmed tracks (born in an earlier frame, never matched since) against the detections still
#     left, on 1 - IoU; reject 1 - IoU > 0.3; an unconfirmed track left unmatched is removed;
#  then every matched track gets the Kalman update and the gallery update and becomes tracked,
#  confirmed tracks left unmatched become lost (removed after the lost limit as before), and the
#  detections left start tracks: tracked on the stream's first frame, unconfirmed after it.
# Every stage is a Hungarian assignment (rows in creation order, columns in kept order, transposed
# when there are more rows) on its sub-matrix.
MOTION_LAMBDA = 0.98
IOU_COST_2 = 0.5
IOU_COST_3 = 0.3
UNCONFIRMED = 3


def iou_xyxy(a, b):
    """IoU of two boxes (x1, y1, x2, y2), continuous coordinates, 0 for an empty union."""
    iw = max(0.0, min(a[2], b[2]) - max(a[0], b[0]))
    ih = max(0.0, min(a[3], b[3]) - max(a[1], b[1]))
    inter = iw * ih
    union = (a[2] - a[0]) * (a[3] - a[1]) + (b[2] - b[0]) * (b[3] - b[1]) - inter
    return inter / union if union > 0 else 0.0


class CascadeTracker(Tracker):
    """Per-stream tracker state and one step of the three-stage association described above."""

    def __init__(self, lam=MOTION_LAMBDA, iou_cost2=IOU_COST_2, iou_cost3=IOU_COST_3, **kw):
        super().__init__(**kw)
        self.lam, self.iou_cost2, self.iou_cost3 = lam, iou_cost2, iou_cost3
        self.frame = 0

    def _stage(self, cost, rows_idx, cols_idx, thresh):
        """Hungarian on the sub-matrix; pairs (row id, col id) with cost <= thresh and below "infinite"."""
        if not rows_idx or not cols_idx:
            return [], np.zeros((len(rows_idx), len(cols_idx)))
        sub = cost[np.ix_(rows_idx, cols_idx)] if isinstance(cost, np.ndarray) else cost
        out = []
        for i, j in assign(sub):
            if sub[i, j] > thresh or sub[i, j] >= INF_COST:
                continue
            out.append((rows_idx[i], cols_idx[j]))
        return out, sub

    def step(self, rows):
        rows = np.asarray(rows, np.float64).reshape(-1, 518)
        K = len(rows)
        pool = self.tracks
        prev_state = [t.state for t in pool]
        for t in pool:
            t.mean, t.cov = predict(t.mean, t.cov)
        zs = [xyxy_to_z(r[:4]) for r in rows]
        Z = np.array(zs).reshape(-1, 4)
        T = len(pool)
        cos_cost = np.zeros((T, K))
        d2 = np.zeros((T, K))
        for i, t in enumerate(pool):
            cos_cost[i] = 1.0 - rows[:, 6:] @ t.emb
            zh, S = project(t.mean, t.cov)
            L = cholesky_lower(S)
            W = forward_sub(L, (Z - zh).T)
            d2[i] = (W * W).sum(0)
        fused = self.lam * cos_cost + (1.0 - self.lam) * d2
        fused[d2 > self.gate] = INF_COST
        confirmed = [i for i in range(T) if prev_state[i] != UNCONFIRMED]
        unconf = [i for i in range(T) if prev_state[i] == UNCONFIRMED]
        # stage 1: motion-fused appearance cost over the confirmed tracks
        m1, sub1 = self._stage(fused, confirmed, list(range(K)), self.assign_thresh)
        det_left = [j for j in range(K) if j not in {d for _, d in m1}]
        matched1 = {i for i, _ in m1}
        # stage 2: IoU of the predicted box for the confirmed tracks tracked before this frame
        trk2 = [i for i in confirmed if i not in matched1 and prev_state[i] == TRACKED]
        boxes = [z_to_xyxy(t.mean) for t in pool]
        iou_cost = np.array([[1.0 - iou_xyxy(boxes[i], rows[j, :4]) for j in range(K)] for i in range(T)]).reshape(T, K)
        m2, sub2 = self._stage(iou_cost, trk2, det_left, self.iou_cost2)
        det_left3 = [j for j in det_left if j not in {d for _, d in m2}]
        # stage 3: unconfirmed tracks on IoU
        m3, sub3 = self._stage(iou_cost, unconf, det_left3, self.iou_cost3)
        matches = m1 + m2 + m3
        matched_t = {i for i, _ in matches}
        matched_d = {j for _, j in matches}
        for i, j in matches:
            t = pool[i]
            t.mean, t.cov = update(t.mean, t.cov, zs[j])
            e = self.momentum * t.emb + (1 - self.momentum) * rows[j, 6:]
            t.emb = e / math.sqrt(float(e @ e))
            t.state = TRACKED
            t.since = 0
        det_track = [None] * K
        for i, j in matches:
            det_track[j] = pool[i].id
        survivors = []
        for i, t in enumerate(pool):
            if i not in matched_t:
                if prev_state[i] == UNCONFIRMED:
                    continue                      # an unconfirmed track is dropped at its first miss
                t.state = LOST
                t.since += 1
                if t.since > self.lost_max:
                    continue
            survivors.append(t)
        first = self.frame == 0
        for j in range(K):
            if j not in matched_d:
                nt = Track(self.next_id, zs[j], rows[j, 6:])
                nt.state = TRACKED if first else UNCONFIRMED
                survivors.append(nt)
                det_track[j] = self.next_id
                self.next_id += 1
        self.tracks = survivors
        self.frame += 1
        self.last = dict(cost=cos_cost, d2=d2, gated=fused, fused=fused, iou=iou_cost, stages=(m1, m2, m3),
                         subs=(sub1, sub2, sub3), det_track=det_track,
                         matches=sorted((pool[i].id, j) for i, j in matches))
        return [(t.id, t.state, z_to_xyxy(t.mean)) for t in self.tracks]

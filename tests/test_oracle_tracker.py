"""Pins of the oracle tracker (CPU): Kalman closed forms, gating, assignment, lifecycle."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize
import scipy.stats

import synth
from oracle import network as net
from oracle import postprocess as pp
from oracle import tracker as tk


def test_gate_constant_is_chi2_95_4dof():
    assert tk.GATE_CHI2 == pytest.approx(scipy.stats.chi2.ppf(0.95, 4), rel=0, abs=1e-12)


def test_predict_without_noise_is_exact():
    g = np.random.default_rng(1)
    mean = g.standard_normal(8)
    A = g.standard_normal((8, 8))
    cov = A @ A.T
    m2, c2 = tk.predict(mean, cov, q=np.zeros((8, 8)))
    np.testing.assert_array_equal(m2[:4], mean[:4] + mean[4:])
    np.testing.assert_array_equal(m2[4:], mean[4:])
    np.testing.assert_allclose(c2, tk.F @ cov @ tk.F.T, rtol=0, atol=0)


def test_update_with_zero_measurement_noise_returns_measurement():
    mean, cov = tk.initiate(np.array([100.0, 50.0, 0.4, 120.0]))
    mean, cov = tk.predict(mean, cov)
    z = np.array([104.0, 47.0, 0.41, 118.0])
    m2, c2 = tk.update(mean, cov, z, r=np.zeros((4, 4)))
    np.testing.assert_allclose(m2[:4], z, rtol=1e-12)
    np.testing.assert_allclose(c2[:4, :4], 0, atol=1e-9)


def test_kalman_gain_matches_inverse_route():
    g = np.random.default_rng(2)
    mean, cov = tk.initiate(np.array([300.0, 200.0, 0.45, 90.0]))
    for _ in range(3):
        mean, cov = tk.predict(mean, cov)
        mean, cov = tk.update(mean, cov, tk.H @ mean + g.normal(0, 2, 4) * [1, 1, 0.01, 1])
    mean, cov = tk.predict(mean, cov)
    z = tk.H @ mean + np.array([3.0, -2.0, 0.01, 1.5])
    S = tk.H @ cov @ tk.H.T + tk.measurement_noise(mean[3])
    K = cov @ tk.H.T @ np.linalg.inv(S)
    m2, c2 = tk.update(mean, cov, z)
    np.testing.assert_allclose(m2, mean + K @ (z - tk.H @ mean), rtol=1e-12)
    np.testing.assert_allclose(c2, (np.eye(8) - K @ tk.H) @ cov, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(c2, c2.T, rtol=0, atol=1e-9)
    assert np.all(np.linalg.eigvalsh(c2) > 0)
    y = z - tk.H @ mean
    assert tk.mahalanobis2(mean, cov, z) == pytest.approx(float(y @ np.linalg.solve(S, y)), rel=1e-12)


def _dare_axes(h):
    Fa = np.array([[1.0, 1.0], [0.0, 1.0]])
    Ha = np.array([[1.0, 0.0]])
    sp, sv = tk.STD_POS * h, tk.STD_VEL * h
    out = []
    for ax, (qp, qv), r in [(0, (sp, sv), sp), (1, (sp, sv), sp), (2, (1e-2, 1e-5), 1e-1), (3, (sp, sv), sp)]:
        Q = np.diag([qp ** 2, qv ** 2])
        R = np.array([[r ** 2]])
        out.append((ax, scipy.linalg.solve_discrete_are(Fa.T, Ha.T, Q, R)))
    return out


def test_steady_state_covariance_solves_dare():
    """With h frozen each axis is a 2-state constant-velocity filter; the prior covariance
    converges to the discrete algebraic Riccati solution (cx, cy, h axes: fast)."""
    h = 150.0
    mean, cov = tk.initiate(np.array([100.0, 200.0, 0.4, h]))
    g = np.random.default_rng(5)
    for _ in range(300):
        mean, cov = tk.predict(mean, cov)
        prior = cov.copy()
        z = np.array([mean[0] + g.normal(0, 3), mean[1] + g.normal(0, 3), 0.4, h])
        mean, cov = tk.update(mean, cov, z)
        assert mean[3] == h
    for ax, X in _dare_axes(h):
        if ax != 2:       # the aspect axis (Q/R ~ 1e-8) needs ~2e4 steps; covered by the fixed-point test
            np.testing.assert_allclose(prior[np.ix_([ax, ax + 4], [ax, ax + 4])], X, rtol=1e-10)


def test_dare_solution_is_a_fixed_point_of_update_then_predict():
    h = 150.0
    P = np.zeros((8, 8))
    for ax, X in _dare_axes(h):
        P[np.ix_([ax, ax + 4], [ax, ax + 4])] = X
    mean = np.array([100.0, 200.0, 0.4, h, 0, 0, 0, 0])
    m2, c2 = tk.update(mean, P, np.array([101.0, 199.0, 0.4, h]))
    m3, c3 = tk.predict(m2, c2)
    assert m3[3] == h
    np.testing.assert_allclose(c3, P, rtol=1e-12, atol=1e-12 * np.abs(P).max())
    for ax, X in _dare_axes(h):
        blk = c3[np.ix_([ax, ax + 4], [ax, ax + 4])]
        assert np.max(np.abs(blk - X) / np.abs(X)) < 1e-11


def _brute(cost):
    n, m = cost.shape
    best, arg = math.inf, None
    for perm in itertools.permutations(range(m), n):
        c = sum(cost[i, perm[i]] for i in range(n))
        if c < best - 1e-12:
            best, arg = c, perm
    return best, arg


@pytest.mark.parametrize("n,m", [(1, 1), (2, 2), (3, 5), (5, 5), (4, 7), (6, 8), (8, 8)])
def test_hungarian_matches_brute_force(n, m):
    g = np.random.default_rng(n * 10 + m)
    for _ in range(5):
        cost = g.uniform(0, 1, (n, m))
        col = tk.hungarian(cost)
        best, arg = _brute(cost)
        assert sum(cost[i, col[i]] for i in range(n)) == pytest.approx(best, abs=1e-12)
        assert tuple(col) == arg       # continuous costs: the optimum is unique
        assert len(set(col.tolist())) == n


def test_hungarian_matches_scipy_large():
    g = np.random.default_rng(9)
    for n, m in [(200, 200), (50, 120)]:
        cost = g.uniform(0, 1, (n, m))
        col = tk.hungarian(cost)
        r, c = scipy.optimize.linear_sum_assignment(cost)
        assert cost[np.arange(n), col].sum() == pytest.approx(cost[r, c].sum(), abs=1e-9)


def test_hungarian_ties_prefer_low_columns():
    assert list(tk.hungarian(np.zeros((4, 4)))) == [0, 1, 2, 3]
    assert list(tk.hungarian(np.full((2, 5), 1e5))) == [0, 1]


def test_assign_transposes_when_more_tracks():
    cost = np.array([[0.9, 0.1], [0.2, 0.8], [0.05, 0.95]])
    assert tk.assign(cost) == [(0, 1), (2, 0)]


def det_row(box, emb, conf=0.9):
    r = np.zeros(518)
    r[:4] = box
    r[4] = conf
    r[6:] = emb / np.linalg.norm(emb)
    return r


def test_lifecycle_birth_lost_and_removal():
    g = np.random.default_rng(4)
    e1, e2 = g.standard_normal(512), g.standard_normal(512)
    T = tk.Tracker()
    out = T.step(np.stack([det_row([100, 100, 140, 220], e1), det_row([500, 300, 560, 450], e2)]))
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED), (2, tk.TRACKED)]
    out = T.step(np.stack([det_row([101, 101, 141, 221], e1)]))
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED), (2, tk.LOST)]
    for f in range(29):
        out = T.step(np.stack([det_row([101, 101, 141, 221], e1)]))
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED), (2, tk.LOST)]   # lost for 30 frames: kept
    out = T.step(np.stack([det_row([101, 101, 141, 221], e1)]))
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED)]                 # 31 > 30: removed


def test_cost_and_gate_rejections_give_births():
    g = np.random.default_rng(6)
    e1 = g.standard_normal(512)
    T = tk.Tracker()
    T.step(np.stack([det_row([100, 100, 140, 220], e1)]))
    # same place, unrelated appearance: cosine cost ~1 > 0.7 -> rejected, new id
    out = T.step(np.stack([det_row([100, 100, 140, 220], g.standard_normal(512))]))
    assert [(i, s) for i, s, _ in out] == [(1, tk.LOST), (2, tk.TRACKED)]
    # same appearance as id 1, far away: gated -> rejected, new id
    out = T.step(np.stack([det_row([900, 600, 940, 720], e1)]))
    assert [i for i, s, _ in out if s == tk.TRACKED] == [3]
    assert T.last["d2"][0, 0] > tk.GATE_CHI2


def test_planted_objects_keep_their_ids():
    """Every detected planted object stays with one track id for the whole clip."""
    r, nw, nh, px, py = net.letterbox_geometry(1920, 1080, 1088, 608)
    clip = synth.PlantedClip(3, 8, 40, 1088, 608, pp.anchors(), pp.STRIDES, r, px, py)
    T = tk.Tracker()
    owner = {}
    for t in range(40):
        dets, embs, truth = clip.frame(t)
        rows = pp.postprocess_frame(dets, embs, r, px, py)["rows"]
        T.step(rows)
        for (o, cx, cy, w, h) in truth:
            d = np.hypot((rows[:, 0] + rows[:, 2]) / 2 - cx, (rows[:, 1] + rows[:, 3]) / 2 - cy)
            j = int(np.argmin(d))
            if d[j] > 1e-3:
                continue              # suppressed by an overlapping object in NMS
            tid = T.last["det_track"][j]
            assert owner.setdefault(o, tid) == tid, "identity switch"
    assert len(owner) == 8


def test_gallery_update_is_the_normalised_momentum_average():
    """The gallery update by hand: a track born from a detection with embedding e starts its gallery at e; each match
    with a detection d sets it to (0.9 e + 0.1 d) / |0.9 e + 0.1 d|.  Two unit vectors at 60 degrees in a
    plane (cosine cost 0.5 <= 0.7, same box) give the closed form (0.9 + 0.05, 0.1 sin 60) / norm; a swapped
    momentum or a missing normalisation gives another vector."""
    e = np.zeros(512)
    e[0] = 1.0
    d = np.zeros(512)
    d[0], d[1] = 0.5, math.sqrt(3.0) / 2
    T = tk.Tracker()
    T.step(np.stack([det_row([100, 100, 140, 220], e)]))
    np.testing.assert_array_equal(T.tracks[0].emb, e)
    T.step(np.stack([det_row([100, 100, 140, 220], d)]))
    assert T.last["matches"] == [(1, 0)]
    v = np.array([0.9 + 0.1 * 0.5, 0.1 * math.sqrt(3.0) / 2])
    want = np.zeros(512)
    want[:2] = v / math.hypot(*v)
    np.testing.assert_allclose(T.tracks[0].emb, want, rtol=0, atol=1e-15)
    assert abs(np.linalg.norm(T.tracks[0].emb) - 1.0) < 1e-15
    # a third frame: the update composes from the gallery, not from the last detection
    T.step(np.stack([det_row([100, 100, 140, 220], d)]))
    v2 = 0.9 * want[:2] + 0.1 * d[:2]
    np.testing.assert_allclose(T.tracks[0].emb[:2], v2 / np.linalg.norm(v2), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(T.tracks[0].emb[2:], 0.0)
    # the cost of the next step uses the gallery: 1 - <gallery, d>
    T.step(np.stack([det_row([100, 100, 140, 220], d)]))
    assert T.last["cost"][0, 0] == pytest.approx(1.0 - float(v2 @ d[:2]) / np.linalg.norm(v2), abs=1e-15)


# ----------------------------------------------------------------------------- association cascade
def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def test_cascade_iou_of_boxes_hand_cases():
    assert tk.iou_xyxy([0, 0, 2, 2], [0, 0, 2, 2]) == 1.0
    assert tk.iou_xyxy([0, 0, 2, 2], [3, 3, 4, 4]) == 0.0
    assert tk.iou_xyxy([0, 0, 2, 2], [1, 0, 3, 2]) == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert tk.iou_xyxy([0, 0, 4, 4], [1, 1, 3, 3]) == pytest.approx(0.25, abs=1e-15)
    assert tk.iou_xyxy([0, 0, 0, 0], [0, 0, 0, 0]) == 0.0


def test_cascade_stage1_cost_is_the_motion_fused_cost():
    """lambda (1 - <e, d>) + (1 - lambda) y^T S^-1 y, the Mahalanobis term by the explicit inverse."""
    g = np.random.default_rng(21)
    e, d = unit(g.standard_normal(512)), unit(g.standard_normal(512))
    d = unit(0.9 * e + 0.3 * d)
    T = tk.CascadeTracker()
    T.step(np.stack([det_row([100, 100, 140, 220], e)]))
    T.step(np.stack([det_row([103, 98, 143, 219], d)]))
    # recompute from the track's state before the second step: predict, project, explicit inverse
    T2 = tk.CascadeTracker()
    T2.step(np.stack([det_row([100, 100, 140, 220], e)]))
    t = T2.tracks[0]
    mean, cov = tk.predict(t.mean, t.cov)
    zh, S = tk.project(mean, cov)
    y = tk.xyxy_to_z(np.array([103.0, 98.0, 143.0, 219.0])) - zh
    d2 = float(y @ np.linalg.inv(S) @ y)
    want = tk.MOTION_LAMBDA * (1.0 - float(e @ d)) + (1.0 - tk.MOTION_LAMBDA) * d2
    assert T.last["fused"][0, 0] == pytest.approx(want, rel=1e-10)
    assert T.last["stages"][0] == [(0, 0)] and T.tracks[0].id == 1


def test_cascade_iou_stage_keeps_the_id_through_an_appearance_change():
    """Same box, unrelated appearance: the single-stage association rejects it (cosine cost ~1 > 0.7)
    and starts a new id; the cascade's IoU stage matches it to the tracked track (IoU 1 > 0.5)."""
    g = np.random.default_rng(22)
    e1, e2 = g.standard_normal(512), g.standard_normal(512)
    A, C = tk.Tracker(), tk.CascadeTracker()
    for T in (A, C):
        T.step(np.stack([det_row([100, 100, 140, 220], e1)]))
    a = A.step(np.stack([det_row([100, 100, 140, 220], e2)]))
    c = C.step(np.stack([det_row([100, 100, 140, 220], e2)]))
    assert [(i, s) for i, s, _ in a] == [(1, tk.LOST), (2, tk.TRACKED)]
    assert [(i, s) for i, s, _ in c] == [(1, tk.TRACKED)]
    m1, m2, m3 = C.last["stages"]
    assert m1 == [] and m2 == [(0, 0)] and m3 == []


def test_cascade_iou_stage_skips_lost_tracks_and_births_are_unconfirmed():
    g = np.random.default_rng(23)
    e1, e2 = g.standard_normal(512), g.standard_normal(512)
    C = tk.CascadeTracker()
    C.step(np.stack([det_row([100, 100, 140, 220], e1)]))
    C.step(np.zeros((0, 518)))                                   # id 1 lost
    out = C.step(np.stack([det_row([100, 100, 140, 220], e2)]))  # unrelated appearance, lost track
    assert [(i, s) for i, s, _ in out] == [(1, tk.LOST), (2, tk.UNCONFIRMED)]


def test_cascade_unconfirmed_tracks_are_confirmed_by_iou_or_removed():
    g = np.random.default_rng(24)
    ea, eb = g.standard_normal(512), g.standard_normal(512)
    first = np.stack([det_row([100, 100, 140, 220], ea)])
    second = np.stack([det_row([100, 100, 140, 220], ea), det_row([500, 300, 560, 450], eb)])
    # confirmed: the next frame has B at IoU >= 0.7 (moved by a pixel), even with an unrelated embedding
    C = tk.CascadeTracker()
    C.step(first)
    out = C.step(second)
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED), (2, tk.UNCONFIRMED)]
    out = C.step(np.stack([det_row([101, 101, 141, 221], ea), det_row([501, 301, 561, 451], g.standard_normal(512))]))
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED), (2, tk.TRACKED)]
    assert C.last["stages"][2] == [(1, 1)]
    # removed: the next frame has no detection near B (not lost: an unconfirmed track is dropped)
    C = tk.CascadeTracker()
    C.step(first)
    C.step(second)
    out = C.step(np.stack([det_row([101, 101, 141, 221], ea)]))
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED)]
    # an IoU below 0.7 does not confirm (B moved by 20 px): B is dropped, the detection is a new unconfirmed id
    C = tk.CascadeTracker()
    C.step(first)
    C.step(second)
    out = C.step(np.stack([det_row([101, 101, 141, 221], ea), det_row([520, 320, 580, 470], eb)]))
    assert tk.iou_xyxy([500, 300, 560, 450], [520, 320, 580, 470]) < 0.7
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED), (3, tk.UNCONFIRMED)]


def test_cascade_first_frame_births_are_confirmed():
    g = np.random.default_rng(25)
    C = tk.CascadeTracker()
    out = C.step(np.stack([det_row([100 + 200 * k, 100, 140 + 200 * k, 220], g.standard_normal(512)) for k in range(3)]))
    assert [(i, s) for i, s, _ in out] == [(1, tk.TRACKED), (2, tk.TRACKED), (3, tk.TRACKED)]


def test_cascade_every_stage_is_an_optimal_assignment():
    """Random small scenes: each stage's chosen pairs (before rejection) minimise the stage's summed cost
    over all assignments of its sub-matrix (brute force)."""
    g = np.random.default_rng(26)
    for trial in range(20):
        C = tk.CascadeTracker(assign_thresh=2.0, iou_cost2=1.0, iou_cost3=1.0)   # accept every pair
        n0 = int(g.integers(2, 6))
        embs = [g.standard_normal(512) for _ in range(n0)]
        boxes = [np.array([50 + 120 * k, 100, 90 + 120 * k, 220], float) for k in range(n0)]
        C.step(np.stack([det_row(b, e) for b, e in zip(boxes, embs)]))
        k1 = int(g.integers(1, 6))
        rows = [det_row(boxes[int(g.integers(0, n0))] + g.normal(0, 3, 4), unit(embs[int(g.integers(0, n0))] +
                                                                                  g.normal(0, 0.5, 512)))
                for _ in range(k1)]
        C.step(np.stack(rows))
        for sub in C.last["subs"]:
            if sub.size == 0:
                continue
            r, c = sub.shape
            if r <= c:
                best = min(sum(sub[i, p[i]] for i in range(r)) for p in itertools.permutations(range(c), r))
            else:
                best = min(sum(sub[p[j], j] for j in range(c)) for p in itertools.permutations(range(r), c))
            chosen = tk.assign(sub)
            assert sum(sub[i, j] for i, j in chosen) == pytest.approx(best, rel=1e-12, abs=1e-12)


def test_cascade_planted_objects_keep_their_ids():
    """The three-stage association keeps every detected planted object on one id for the whole clip."""
    r, nw, nh, px, py = net.letterbox_geometry(1920, 1080, 1088, 608)
    clip = synth.PlantedClip(3, 8, 40, 1088, 608, pp.anchors(), pp.STRIDES, r, px, py)
    C = tk.CascadeTracker()
    owner = {}
    for t in range(40):
        dets, embs, truth = clip.frame(t)
        rows = pp.postprocess_frame(dets, embs, r, px, py)["rows"]
        C.step(rows)
        for (o, cx, cy, w, h) in truth:
            d = np.hypot((rows[:, 0] + rows[:, 2]) / 2 - cx, (rows[:, 1] + rows[:, 3]) / 2 - cy)
            j = int(np.argmin(d))
            if d[j] > 1e-3:
                continue
            tid = C.last["det_track"][j]
            assert owner.setdefault(o, tid) == tid, "identity switch"
    assert len(owner) == 8

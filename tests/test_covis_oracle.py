"""Pins of the covisibility / keyframe-window oracle (supplementary material,
Keyframe Management, Eq. S1/S2): set identities, hand-built cases and the
rules' worked consequences."""
import numpy as np

from oracle import covis_oracle as C
from paper_2507_03737_gb300 import scenes


def test_counts_iou_oc_on_hand_sets():
    # G0 = {0,1,2,3}, G1 = {2,3,4}, G2 = {} ; |G0&G1| = 2, |G0|G1| = 5
    vis = np.zeros((3, 6), dtype=bool)
    vis[0, [0, 1, 2, 3]] = True
    vis[1, [2, 3, 4]] = True
    Cm = C.counts(vis)
    assert Cm.tolist() == [[4, 2, 0], [2, 3, 0], [0, 0, 0]]
    iou, oc = C.iou_oc(Cm)
    assert iou[0, 1] == 2 / 5 and oc[0, 1] == 2 / 3
    assert iou[0, 0] == 1.0 and oc[1, 1] == 1.0
    assert iou[0, 2] == 0.0 and oc[2, 2] == 0.0      # empty set: defined as 0


def test_iou_oc_identities_on_random_sets():
    rng = np.random.default_rng(1)
    vis = rng.random((7, 500)) < rng.uniform(0.1, 0.9, (7, 1))
    iou, oc = C.iou_oc(C.counts(vis))
    for i in range(7):
        for j in range(7):
            a, b = set(np.nonzero(vis[i])[0]), set(np.nonzero(vis[j])[0])
            assert iou[i, j] == len(a & b) / len(a | b)
            assert oc[i, j] == len(a & b) / min(len(a), len(b))
            assert iou[i, j] <= oc[i, j] + 1e-15
    np.testing.assert_array_equal(iou, iou.T)


def test_median_is_lower_median_of_positive_depths():
    d = np.array([0.0, 5.0, -1.0, 2.0, 9.0, 0.0, 7.0])
    assert C.median_depth(d) == (5.0, 4)        # sorted 2 5 7 9 -> rank 1
    assert C.median_depth(np.array([3.0, 1.0, 2.0])) == (2.0, 3)
    assert C.median_depth(np.zeros(4)) == (0.0, 0)


def test_new_keyframe_rule():
    assert C.is_new_keyframe(0.85, 0.0, 10.0)          # low overlap
    assert not C.is_new_keyframe(0.95, 0.79, 10.0)     # 0.79 <= 0.08 * 10
    assert C.is_new_keyframe(0.95, 0.81, 10.0)         # moved more than 8 % of the median depth
    assert not C.is_new_keyframe(0.9, 0.0, 10.0)       # strict: IOU = k_I does not trigger


def test_window_update_rules():
    # OC below 0.3 leaves; the new keyframe is appended
    assert C.window_update([1, 2, 3], [0.5, 0.29, 0.3], 9) == [1, 3, 9]
    # overflow: 8 kept + new = 9 > 8, the lowest OC (earliest on ties) leaves
    ids = list(range(10, 18)); oc = [0.9, 0.4, 0.8, 0.4, 0.7, 0.6, 0.5, 0.95]
    assert C.window_update(ids, oc, 99) == [10, 12, 13, 14, 15, 16, 17, 99]
    assert C.window_update([], [], 5) == [5]


def test_extents_and_projection_agree_away_from_the_border():
    sc = scenes.config_scene(1)
    vis, slack = C.projected_sets(sc, sc.cameras)
    assert vis.shape == (1, 4096) and 0 < vis.sum() < 4096
    assert np.all(np.isfinite(slack[vis]))

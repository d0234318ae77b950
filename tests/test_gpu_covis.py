"""Keyframe covisibility (Eq. S1/S2) and median depth on the GPU.

Counts are integer work: they must equal, bit for bit, the integer referee's
counts from the same render's per-record extents; IOU and OC are one
double-precision division of those counts rounded to float, so they are
compared exactly too. Against the FP64 projection the visible sets can differ
only for Gaussians whose 3-sigma footprint edge lies within the tile cover's
rounding margin of the image border (at most 2 pixels here), so the counts may
differ by at most the number of such Gaussians. The median is a selection, so
it is exact.
"""
import numpy as np
import pytest

from oracle import covis_oracle as C
from paper_2507_03737_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2507_03737_gb300.autograd import Renderer
    r = Renderer(0)
    yield r
    r.close()


def _covis(R, V):
    import torch
    from paper_2507_03737_gb300 import binding as B
    counts = torch.empty((V, V), dtype=torch.int64, device="cuda")
    iou = torch.empty((V, V), device="cuda")
    oc = torch.empty((V, V), device="cuda")
    B.s3gs_covisibility(R.ctx, R.state, counts, iou, oc)
    torch.cuda.synchronize()
    return counts.cpu().numpy(), iou.cpu().numpy(), oc.cpu().numpy()


@pytest.mark.parametrize("cid,n", [(3, 60000), (4, 40000), (1, None)])
def test_counts_match_referee_and_oracle(R, cid, n):
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.config_scene(cid, n_override=n)
    V = len(sc.cameras)
    R.render_np(sc)
    cnt, iou, oc = _covis(R, V)
    rec = B.s3gs_debug_records(R.ctx, R.state, V * sc.n)
    ref = C.counts(C.sets_from_extents(rec["extent"], V))
    np.testing.assert_array_equal(cnt, ref)
    ref_iou, ref_oc = C.iou_oc(ref)
    np.testing.assert_array_equal(iou, ref_iou.astype(np.float32))
    np.testing.assert_array_equal(oc, ref_oc.astype(np.float32))
    # against the FP64 projection: differences only from footprints at the border
    vis, slack = C.projected_sets(sc, sc.cameras)
    amb = slack < 2.0
    oracle_counts = C.counts(vis)
    for i in range(V):
        for j in range(V):
            bound = int(np.count_nonzero(amb[i] | amb[j]))
            assert abs(int(cnt[i, j]) - int(oracle_counts[i, j])) <= bound, (i, j)
    assert np.all(np.diag(cnt) > 0)


def test_empty_and_disjoint_views(R):
    """A view that sees nothing has zero IOU and OC with every view."""
    sc = scenes.tiny_scene(3, n=30, n_views=2)
    away = dict(sc.cameras[1])
    T = np.asarray(away["T_cw"], np.float64).reshape(3, 4).copy()
    T[2, 3] -= 100.0                       # everything behind the camera
    away["T_cw"] = T.astype(np.float32)
    R.render_np(sc, cameras=[sc.cameras[0], away])
    cnt, iou, oc = _covis(R, 2)
    assert cnt[1, 1] == 0 and cnt[0, 1] == 0 and cnt[0, 0] > 0
    assert iou[0, 1] == 0.0 and oc[0, 1] == 0.0 and oc[1, 1] == 0.0 and iou[0, 0] == 1.0


def _median_case(seed):
    rng = np.random.default_rng(seed)
    sizes = [(37, 23), (1241, 376), (5, 3), (64, 48), (1, 1), (200, 100)]
    maps = []
    for k, (w, h) in enumerate(sizes):
        d = rng.lognormal(2.0, 1.0, w * h).astype(np.float32)
        d[rng.random(w * h) < 0.2] = 0.0
        if k == 2:
            d[:] = 0.0                      # no positive depth at all
        if k == 3:
            d[rng.random(w * h) < 0.1] = -1.0
            d[5] = np.nan
            d[rng.random(w * h) < 0.3] = 7.25  # many ties
        maps.append(d)
    return sizes, maps


def test_median_depth_is_exact(R):
    import torch
    from paper_2507_03737_gb300 import binding as B
    for seed in (1, 2):
        sizes, maps = _median_case(seed)
        wh, nv = B.view_sizes(sizes)
        ws = torch.empty(B.s3gs_median_depth_workspace(nv), dtype=torch.uint8, device="cuda")
        med = torch.empty(nv, device="cuda")
        nval = torch.empty(nv, dtype=torch.int64, device="cuda")
        B.s3gs_median_depth(R.ctx, wh, nv, torch.from_numpy(np.concatenate(maps)).cuda(), med, nval, ws)
        torch.cuda.synchronize()
        for k, d in enumerate(maps):
            ref, n = C.median_depth(d)
            assert float(med[k]) == ref and int(nval[k]) == n, (seed, k)


def test_covis_and_median_capture_in_a_graph(R):
    import torch
    from paper_2507_03737_gb300 import binding as B
    sc = scenes.config_scene(3, n_override=30000)
    V = len(sc.cameras)
    p = R.upload(sc)
    out = R.forward(p, sc.cameras)
    torch.cuda.synchronize()
    cnt0, iou0, _ = _covis(R, V)
    wh, nv = B.view_sizes(sc.cameras)
    ws = torch.empty(B.s3gs_median_depth_workspace(nv), dtype=torch.uint8, device="cuda")
    med = torch.empty(nv, device="cuda")
    counts = torch.empty((V, V), dtype=torch.int64, device="cuda")
    iou = torch.empty((V, V), device="cuda")
    B.s3gs_median_depth(R.ctx, wh, nv, out["depth"], med, None, ws)
    torch.cuda.synchronize()
    med0 = med.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        B.s3gs_covisibility(R.ctx, R.state, counts, iou, None)
        B.s3gs_median_depth(R.ctx, wh, nv, out["depth"], med, None, ws)
    med.zero_()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy(), cnt0)
    np.testing.assert_array_equal(iou.cpu().numpy(), iou0)
    assert torch.equal(med, med0)

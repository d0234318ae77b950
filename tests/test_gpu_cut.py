"""The occlusion cut changes no output and no gradient (GPU).

Eq. 2 stops compositing a pixel at the first Gaussian that would take its
transmittance below 1e-4. By default the library ends each tile's list after the
first depth bin by which the Gaussians that cover the whole tile are certain, by a
bound with FP32 margins, to have stopped every pixel of the tile. Each scene here
is rendered with the cut and with every covered pair listed (full_lists = 1; that
list is pinned bit for bit against the integer referee by the binning tests), and:

- each tile's list with the cut is a prefix of its full list that ends at a
  depth-bin boundary;
- rgb, depth, pointmap and alpha are bitwise equal;
- in deterministic mode every gradient tensor, the twist included, is bitwise equal;
- on the large-Gaussian workload the cut removes most of the list, so the
  comparison is not vacuous.
"""
import numpy as np
import pytest

from paper_2507_03737_gb300 import scenes
from tests.gpu_helpers import upstream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2507_03737_gb300.autograd import Renderer
    r = Renderer(0)
    yield r
    r.close()


def _depth_bin(depth_bits):
    """The renderer's log-depth bin of a depth given by its FP32 bit pattern."""
    b = (depth_bits.astype(np.int64) >> 19) - 1993
    return np.clip(b, 0, 255)


def _case(name):
    if name == "config1":
        return scenes.config_scene(1)
    if name == "config3_200k_2views":
        sc = scenes.config_scene(3, n_override=200_000)
        sc.cameras = sc.cameras[:2]
        return sc
    if name == "config5_2views":
        # 5M large, elongated SH-3 Gaussians; one view of each size
        sc = scenes.config_scene(5)
        sc.cameras = sc.cameras[:2]
        return sc
    if name == "opaque_wall":
        # a wall of opaque, wide Gaussians in front of a cloud of small ones: most
        # tiles are cut after the wall's depth bins
        rng = np.random.default_rng(11)
        n_wall, n_back = 3000, 200000
        wall = np.stack([rng.uniform(-3, 3, n_wall), rng.uniform(-2, 2, n_wall), rng.uniform(3.0, 3.2, n_wall)], 1)
        back = np.stack([rng.uniform(-4, 4, n_back), rng.uniform(-3, 3, n_back), rng.uniform(4, 12, n_back)], 1)
        sc = scenes.random_gaussians(rng, np.concatenate([wall, back]), 1)
        sc.log_scales[:n_wall] = np.log(0.25).astype(np.float32)
        sc.opacity_logits[:n_wall] = 3.0
        sc.cameras = [scenes.camera(160, 120, 150.0, 150.0, 80.0, 60.0),
                      scenes.camera(97, 61, 90.0, 90.0, 40.0, 33.0)]
        return sc
    raise ValueError(name)


def _lists(R, sc, **kw):
    from paper_2507_03737_gb300 import binding as B
    out = R.render_np(sc, options=B.s3gs_options_default(**kw))
    keys, vals, ranges = B.s3gs_debug_binning(R.ctx, R.state)
    return out, keys.copy(), vals.copy(), ranges.copy()


def _check_prefix(keys, vals, ranges, fkeys, fvals, franges):
    n = np.diff(ranges)
    nf = np.diff(franges)
    assert np.all(n <= nf)
    tile = np.repeat(np.arange(n.size), n)
    off = np.arange(keys.size) - np.repeat(ranges[:-1], n)
    src = franges[:-1][tile] + off
    assert np.array_equal(keys, fkeys[src]) and np.array_equal(vals, fvals[src])
    # where a tile's list was cut, the first dropped key lies in a later depth bin
    # than the last kept one
    cut = np.nonzero((n < nf) & (n > 0))[0]
    last = _depth_bin(fkeys[franges[cut] + n[cut] - 1] & 0xffffffff)
    nxt = _depth_bin(fkeys[franges[cut] + n[cut]] & 0xffffffff)
    assert np.all(nxt > last)
    return int(np.count_nonzero(n < nf))


CASES = ["config1", "opaque_wall", "config3_200k_2views", "config5_2views"]


@pytest.mark.parametrize("name", CASES)
def test_cut_lists_are_prefixes_and_outputs_are_unchanged(R, name):
    sc = _case(name)
    full, fkeys, fvals, franges = _lists(R, sc, full_lists=1)
    cut, keys, vals, ranges = _lists(R, sc)
    n_cut_tiles = _check_prefix(keys, vals, ranges, fkeys, fvals, franges)
    for k in full:
        assert np.array_equal(full[k].view(np.uint32), cut[k].view(np.uint32)), k
    kept = keys.size / max(fkeys.size, 1)
    print(f"CUT {name}: kept {keys.size} of {fkeys.size} pairs ({kept:.4f}); tiles cut {n_cut_tiles} of "
          f"{ranges.size - 1}")
    if name in ("opaque_wall", "config5_2views"):
        assert kept < 0.5, kept
    if name == "config5_2views":
        assert kept < 0.1, kept


@pytest.mark.parametrize("name", ["opaque_wall", "config3_200k_2views", "config5_2views"])
def test_cut_gradients_are_bitwise_unchanged(R, name):
    sc = _case(name)
    V = len(sc.cameras)
    ups = upstream(sc.cameras, 7)
    res = {}
    for fl in (1, 0):
        _lists(R, sc, full_lists=fl, deterministic=1)
        res[fl] = R.backward_np(ups, V)
    for k in res[1]:
        assert np.array_equal(res[1][k].view(np.uint32), res[0][k].view(np.uint32)), k


def test_cut_with_recompute_and_persistent_grid(R):
    """The recompute replay and the persistent grid read the same cut lists."""
    sc = _case("opaque_wall")
    ups = upstream(sc.cameras, 3)
    res = {}
    for fl in (1, 0):
        _lists(R, sc, full_lists=fl, deterministic=1, recompute=1, blocks_per_sm=4)
        res[fl] = R.backward_np(ups, len(sc.cameras))
    for k in res[1]:
        assert np.array_equal(res[1][k].view(np.uint32), res[0][k].view(np.uint32)), k


def _wall_ragged():
    """The opaque wall seen by uneven views whose border tiles are partial."""
    sc = _case("opaque_wall")
    sc.cameras = [scenes.camera(77, 45, 70.0, 70.0, 38.0, 22.0), scenes.camera(33, 70, 40.0, 40.0, 16.5, 35.0),
                  scenes.camera(1, 1, 10.0, 10.0, 0.5, 0.5), scenes.camera(161, 7, 120.0, 120.0, 80.0, 3.0)]
    return sc


@pytest.mark.parametrize("tile", [(16, 16), (16, 8), (8, 8), (32, 8)])
def test_cut_every_tile_shape_on_ragged_views(R, tile):
    """Each tile shape (a different inradius filter and partial border tiles)."""
    sc = _wall_ragged()
    tw, th = tile
    full, fkeys, fvals, franges = _lists(R, sc, full_lists=1, tile_w=tw, tile_h=th)
    cut, keys, vals, ranges = _lists(R, sc, tile_w=tw, tile_h=th)
    n_cut_tiles = _check_prefix(keys, vals, ranges, fkeys, fvals, franges)
    for k in full:
        assert np.array_equal(full[k].view(np.uint32), cut[k].view(np.uint32)), k
    print(f"CUT ragged {tw}x{th}: kept {keys.size} of {fkeys.size}; tiles cut {n_cut_tiles} of {ranges.size - 1}")
    assert n_cut_tiles > 0


def test_cut_behind_three_opaque_layers(R):
    """Three wide, nearly opaque Gaussians in one depth bin in front of 5,000 small ones:
    over every tile each has alpha >= 0.98, so three of them stop every pixel (T <= 1e-5)
    and every tile's list must end with them, with nothing else listed."""
    rng = np.random.default_rng(4)
    n = 5000
    front = np.array([[0.0, 0.0, 2.0], [0.0, 0.0, 2.02], [0.0, 0.0, 2.04]])
    back = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(3, 8, n)], 1)
    sc = scenes.random_gaussians(rng, np.concatenate([front, back]), 0)
    sc.log_scales[:3] = np.log(np.array([10.0, 10.0, 0.05])).astype(np.float32)
    sc.quats[:3] = np.array([1, 0, 0, 0], np.float32)
    sc.opacity_logits[:3] = 8.0
    sc.cameras = [scenes.camera(96, 64, 60.0, 60.0, 48.0, 32.0)]
    full, fkeys, fvals, franges = _lists(R, sc, full_lists=1)
    cut, keys, vals, ranges = _lists(R, sc)
    _check_prefix(keys, vals, ranges, fkeys, fvals, franges)
    for k in full:
        assert np.array_equal(full[k].view(np.uint32), cut[k].view(np.uint32)), k
    assert np.all(np.diff(ranges) == 3) and set(np.unique(vals)) == {0, 1, 2}
    assert fkeys.size > 10 * keys.size


def test_cut_pose_only_backward(R):
    """The geometry-only (tracking) backward reads the same cut lists."""
    sc = _wall_ragged()
    ups = upstream(sc.cameras, 9)
    res = {}
    for fl in (1, 0):
        _lists(R, sc, full_lists=fl, deterministic=1)
        res[fl] = R.backward_np(ups, len(sc.cameras), want=("twist",))
    assert np.array_equal(res[1]["twist"].view(np.uint32), res[0]["twist"].view(np.uint32))


def _moved_wall(dz):
    sc = _case("opaque_wall")
    sc.means = sc.means.copy()
    sc.means[:, 2] += np.float32(dz)
    return sc


def test_cut_hints_from_previous_forwards(R):
    """A forward with the cut takes the previous forward's cut as a hint (pairs behind it
    add no optical depth). Whatever the hint, the result must equal the full lists: the
    same scene again (a hint that matches), then the wall moved back by 2 m (a hint that
    ends too early: those tiles keep more), then moved forward again (a hint that ends
    late), and the first scene once more."""
    seq = [("same", _case("opaque_wall")), ("same again", _case("opaque_wall")),
           ("wall 2 m back", _moved_wall(2.0)), ("wall 1 m forward", _moved_wall(-1.0)),
           ("first again", _case("opaque_wall"))]
    kept = []
    for name, sc in seq:
        full, fkeys, fvals, franges = _lists(R, sc, full_lists=1)
        # full lists leave the hint alone; run the cut twice so the second sees this
        # scene's own cut, after a first run that sees the previous scene's
        for rep in range(2):
            cut, keys, vals, ranges = _lists(R, sc)
            _check_prefix(keys, vals, ranges, fkeys, fvals, franges)
            for k in full:
                assert np.array_equal(full[k].view(np.uint32), cut[k].view(np.uint32)), (name, rep, k)
            kept.append(keys.size)
        print(f"CUT hint {name}: kept {kept[-2]} then {kept[-1]} of {fkeys.size}")
    # a tile's own previous cut as the hint gives that cut again (the sums up to it are
    # complete), and the same as no hint; a stale hint can only keep more
    own = kept[1::2]
    assert own[0] == own[1] == own[4]
    assert all(kept[2 * i + 1] <= kept[2 * i] for i in range(len(seq)))

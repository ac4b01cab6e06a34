"""Batched multi-view form against the oracle and the single-view path.

Per view of a batch (uneven resolutions, mixed tile and blend-warp shapes, shrink off
and on): the selection equals the oracle's serial traversal bit for bit (§3.2: the
parallel filter reaches the serial cut), the view's sorted pairs (global tile id minus
the view's first tile, value minus the view's first entry) and the splat decision fields
equal the oracle's, transmittance is bit-exact and colour within the image tolerance.
Every pixel also equals the single-view GPU render, with and without CUDA-graph replay."""
import math

import numpy as np
import pytest

from paper_2603_23891_gb300 import synth

from gpu_util import assert_frame_parity, batch_view_frame, oracle_frame, orbit_cameras

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_23891_gb300 import build, filtergs
    build.build()
    r = filtergs.Renderer(device=0)
    yield r
    r.close()


def _single(r, cam, tile):
    import torch
    r.set_params(tile=tile)
    r.set_camera(cam)
    rgb, T, st = r.render(stats=True)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), T.cpu().numpy(), st.n_selected, st.n_pairs


@pytest.mark.parametrize("shrink", [None, 0.05])
def test_batch_equals_single_views(renderer, shrink):
    import torch
    tree = synth.random_small_tree(7, n_leaves=6000, branching=(2, 8), sh_degree=3, extent=25.0,
                                   log_scale_mean=-0.8)
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    renderer.shrink(None if shrink is None else shrink,
                    None if shrink is None else float(np.float32(math.log(shrink))))
    sizes = [(64, 48), (250, 130), (128, 128), (96, 200), (333, 77), (160, 120)]
    cams = [c for c, _ in zip(orbit_cameras(tree, len(sizes), (64, 64), 3, dist=(10, 80)), sizes)]
    cams = [synth.look_at_camera(c.campos.astype(float), tree.mu.mean(axis=1), w, h, 60.0)
            for c, (w, h) in zip(cams, sizes)]
    tiles = [(16, 16), (32, 8), (16, 16), (8, 32), (64, 4), (32, 8)]
    warps = [8, 4, 4, 8, 8, 8]
    refs = [_single(renderer, c, t) for c, t in zip(cams, tiles)]
    renderer.set_params(tile=(16, 16))
    renderer.batch_setup(cams, tile_shapes=[(tw, th, ww) for (tw, th), ww in zip(tiles, warps)])
    shr = None if shrink is None else (shrink, float(np.float32(math.log(shrink))))
    oracles = [oracle_frame(tree, c, 3.0, shrink=shr, tile=t)[0] for c, t in zip(cams, tiles)]
    for graph in (False, True, True):
        rgb, T, st, views = renderer.render_batch(graph=graph, stats=True)
        torch.cuda.synchronize()
        assert st.n_selected == sum(x[2] for x in refs)
        assert st.n_pairs == sum(x[3] for x in refs)
        for (rgb_v, T_v), (rr, tr, _, _) in zip(views, refs):
            assert np.array_equal(rgb_v.cpu().numpy().view(np.uint32), rr.view(np.uint32))
            assert np.array_equal(T_v.cpu().numpy().view(np.uint32), tr.view(np.uint32))
        frames = renderer.batch_frame()
        for v, (bv, (rgb_v, T_v), o) in enumerate(zip(frames, views, oracles)):
            assert bv["M"] > 0 and bv["NP"] > 0, v
            assert_frame_parity(batch_view_frame(bv, rgb_v, T_v), o)
    # new cameras through the captured graph
    cams2 = [synth.look_at_camera(c.campos.astype(float) * 1.3, tree.mu.mean(axis=1), c.width, c.height,
                                  50.0) for c in cams]
    refs2 = [_single(renderer, c, t) for c, t in zip(cams2, tiles)]
    renderer.batch_set_cameras(cams2)
    # the blend warp shape changes no pixel: 4x8 warps on the single-view path too
    renderer.set_params(tile=(16, 16), blend_warp_w=4)
    r4 = _single(renderer, cams2[0], (16, 16))
    assert np.array_equal(r4[0].view(np.uint32), refs2[0][0].view(np.uint32))
    renderer.set_params(blend_warp_w=8)
    rgb, T, st, views = renderer.render_batch(graph=True, stats=True)
    torch.cuda.synchronize()
    for (rgb_v, T_v), (rr, tr, _, _) in zip(views, refs2):
        assert np.array_equal(rgb_v.cpu().numpy().view(np.uint32), rr.view(np.uint32))
        assert np.array_equal(T_v.cpu().numpy().view(np.uint32), tr.view(np.uint32))
    frames = renderer.batch_frame()
    for bv, (rgb_v, T_v), c, t in zip(frames, views, cams2, tiles):
        o, _ = oracle_frame(tree, c, 3.0, shrink=shr, tile=t)
        assert_frame_parity(batch_view_frame(bv, rgb_v, T_v), o)
    renderer.shrink(None)


def test_batch_views_see_nothing_or_one_tile(renderer):
    """Degenerate views inside a batch: a camera facing away from the tree (no node in
    the frustum: no selection, no pairs, background image, T = 1) between ordinary
    views, and a 16x16 view of one tile; every view against the oracle."""
    import torch
    tree = synth.random_small_tree(9, n_leaves=3000, branching=(2, 6), sh_degree=1, extent=20.0,
                                   log_scale_mean=-0.9)
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16), bg=(0.25, 0.5, 0.75))
    renderer.shrink(None)
    c = tree.mu.mean(axis=1).astype(np.float64)
    cams = [synth.look_at_camera(c + [0, -60, 25], c, 200, 120, 60.0),
            synth.look_at_camera(c + [0, -60, 25], c + [0, -200, 25], 96, 64, 60.0),   # away
            synth.look_at_camera(c + [30, 30, 40], c, 16, 16, 50.0),
            synth.look_at_camera(c + [-50, 10, 30], c, 130, 70, 70.0)]
    renderer.batch_setup(cams)
    rgb, T, st, views = renderer.render_batch(stats=True)
    torch.cuda.synchronize()
    frames = renderer.batch_frame()
    assert frames[1]["M"] == 0 and frames[1]["NP"] == 0
    for bv, (rgb_v, T_v), cam in zip(frames, views, cams):
        o, _ = oracle_frame(tree, cam, 3.0, bg=(0.25, 0.5, 0.75))
        assert_frame_parity(batch_view_frame(bv, rgb_v, T_v), o)
    assert np.all(views[1][1].cpu().numpy() == 1.0)
    renderer.set_params(bg=(0.0, 0.0, 0.0))


def test_batch_capacity_reported(renderer):
    from paper_2603_23891_gb300 import filtergs
    tree = synth.tiny_tree()
    renderer.load_tree(tree)
    renderer.set_params(tau_R=1.0, tile=(16, 16))
    cams = [synth.tiny_camera()] * 3
    renderer.batch_setup(cams, sel_capacity=1000, pair_capacity=1 << 20)
    with pytest.raises(filtergs.FgsError) as e:
        renderer.render_batch(stats=True)
    assert e.value.code == filtergs.FGS_ERR_CAPACITY
    renderer.batch_setup(cams, sel_capacity=1 << 16, pair_capacity=1 << 20)
    rgb, T, st, views = renderer.render_batch(stats=True)
    assert st.n_selected == 3 * 4096

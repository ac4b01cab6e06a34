"""GPU parity of the whole render path against the CPU oracle (through the C ABI).

Selections, splat decision fields, sorted pair lists and final transmittance are
compared bit for bit; colours within 2e-3 max-abs and >= 60 dB PSNR."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_23891_gb300 import synth

from gpu_util import IMG_TOL, assert_frame_parity, gpu_frame, oracle_frame, orbit_cameras

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


@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_tree(), synth.tiny_camera()


@pytest.mark.parametrize("tau_R", [1.0, 3.0, 10.0, 40.0, -1.0, 1e30])
def test_tiny_tree_all_thresholds(renderer, tiny, tau_R):
    tree, cam = tiny
    renderer.load_tree(tree)
    g = gpu_frame(renderer, tree, cam, tau_R)
    o, _ = oracle_frame(tree, cam, tau_R)
    assert_frame_parity(g, o)


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 32)])
def test_tile_shapes_and_ragged_image(renderer, tile):
    tree = synth.tiny_tree()
    renderer.load_tree(tree)
    # 250 x 130 is not a multiple of any tile shape: ragged last row / column of tiles
    cam = synth.look_at_camera([0.0, -60.0, 35.0], [0, 0, 0], 250, 130, 65.0)
    g = gpu_frame(renderer, tree, cam, 3.0, tile=tile, bg=(0.1, 0.2, 0.3))
    o, _ = oracle_frame(tree, cam, 3.0, tile=tile, bg=(0.1, 0.2, 0.3))
    assert_frame_parity(g, o)


@pytest.mark.parametrize("seed", range(4))
def test_random_trees_multilevel_cuts(renderer, seed):
    """Small trees with large leaves: cuts span several levels."""
    tree = synth.random_small_tree(seed, n_leaves=3000, branching=(2, 8), sh_degree=3,
                                   extent=20.0, log_scale_mean=-0.8)
    renderer.load_tree(tree)
    levels = set()
    for cam in orbit_cameras(tree, 3, (160, 120), seed, dist=(10.0, 80.0)):
        for tau_R in (3.0, 12.0, 40.0):
            g = gpu_frame(renderer, tree, cam, tau_R)
            o, _ = oracle_frame(tree, cam, tau_R)
            assert_frame_parity(g, o)
            levels |= set(np.unique(tree.level[o.sel]).tolist())
    assert len(levels) >= 3


def test_shrink_on_pairs_bit_exact(renderer, tiny):
    """Adaptive shrinking: the same tau / ln tau bits on both sides give identical pairs;
    more aggressive tau never adds pairs."""
    tree, cam = tiny
    renderer.load_tree(tree)
    prev = None
    for tau in (1 / 255, 0.02, 0.1, 0.3):
        sh = (float(np.float32(tau)), float(np.float32(math.log(tau))))
        g = gpu_frame(renderer, tree, cam, 3.0, shrink=sh)
        o, _ = oracle_frame(tree, cam, 3.0, shrink=sh)
        assert_frame_parity(g, o)
        if prev is not None:
            assert g["NP"] <= prev
        prev = g["NP"]


def test_calibration_matches_oracle(renderer):
    """KPC per pair (Eq. 5), GTC per tile (Eq. 6), view average (Eq. 7) and tau (Eq. 8)."""
    tree = synth.random_small_tree(11, n_leaves=2000, branching=(2, 6), sh_degree=0,
                                   extent=15.0, log_scale_mean=-0.9)
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    cams = orbit_cameras(tree, 3, (128, 96), 5)
    gbars = []
    for cam in cams:
        renderer.set_camera(cam)
        renderer.shrink(None)
        renderer.render()
        n = renderer.n_pairs()
        gbar, G, kpc = renderer.calibrate_view(want_kpc=True, n_pairs=n)
        o, p = oracle_frame(tree, cam, 3.0, blend=False)
        _, _, okpc = oracle.render(o.splat, o.keys, o.vals, cam, p, want_kpc=True)
        tx, ty = oracle.tiles_of(cam, p)
        oG, ogbar, _ = oracle.gtc(o.keys, okpc, tx * ty)
        np.testing.assert_allclose(kpc, okpc, rtol=1e-4, atol=1e-5)
        both = ~np.isnan(oG)
        assert np.array_equal(np.isnan(G), np.isnan(oG))
        np.testing.assert_allclose(G[both], oG[both], rtol=1e-4, atol=1e-6)
        assert gbar == pytest.approx(ogbar, rel=1e-4)
        gbars.append(gbar)
    tau, ln_tau, gb = renderer.calibrate(cams, 0.2)
    # the reductions run in a fixed order: a second calibration gives the same bits
    assert np.array_equal(gb, np.array(gbars))
    otau, oln = oracle.tau_from(gbars, 0.2)
    assert tau == pytest.approx(otau, rel=1e-6) and ln_tau == pytest.approx(oln, rel=1e-6)


def test_device_exp_matches_oracle_and_cuda(renderer):
    """The blend's exp: bit-identical to the oracle's binary32 restatement, and within
    2 ulp of CUDA's expf."""
    import torch
    from paper_2603_23891_gb300 import filtergs
    x = torch.linspace(-87.0, 0.0, 100001, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    filtergs.fgs_eval_exp(x, y, None)
    torch.cuda.synchronize()
    xs = x.cpu().numpy()
    ys = y.cpu().numpy()
    sub = slice(None, None, 97)
    assert np.array_equal(ys[sub].view(np.uint32), oracle.expf(xs[sub]).view(np.uint32))
    ref = torch.exp(x).cpu().numpy()
    ulp = np.spacing(np.abs(ref).astype(np.float32))
    assert (np.abs(ys.astype(np.float64) - ref) / ulp).max() <= 2.0


def test_empty_view_and_behind_camera(renderer, tiny):
    """Camera facing away: no selection, no pairs, image = background, T = 1."""
    tree, _ = tiny
    renderer.load_tree(tree)
    cam = synth.look_at_camera([0, -80, 10], [0, -200, 10], 64, 48, 60.0)
    g = gpu_frame(renderer, tree, cam, 3.0, bg=(0.25, 0.5, 0.75))
    assert g["M"] == 0 and g["NP"] == 0 and g["sel"].size == 0
    assert np.all(g["T"] == 1.0)
    for ch, v in enumerate((0.25, 0.5, 0.75)):
        assert np.all(g["rgb"][ch] == np.float32(v))


def test_gaussian_covering_whole_screen(renderer):
    """One large Gaussian right in front of the camera touches every tile."""
    t = synth.tree_from_gaussians(np.array([[0.0, 3.0, 0.0], [0.5, 20.0, 0.3]]),
                                  np.array([[0.5, 0.5, 0.5], [-1.0, -1.0, -1.0]]),
                                  np.array([[1.0, 0, 0, 0], [1.0, 0, 0, 0]]), np.array([0.0, 2.0]),
                                  np.zeros((2, 1, 3)), 0)
    renderer.load_tree(t)
    cam = synth.look_at_camera([0, 0, 0], [0, 1, 0], 200, 120, 60.0)
    g = gpu_frame(renderer, t, cam, -1.0)
    o, _ = oracle_frame(t, cam, -1.0)
    assert_frame_parity(g, o)
    tiles = ((200 + 15) // 16) * ((120 + 15) // 16)
    assert g["NP"] >= tiles


def test_wide_footprints(renderer):
    """Gaussians whose footprints cover more than 128 tiles (up to the whole 640x360
    screen) among small ones: their pairs are counted and scattered by the whole block
    after their group of 256 Gaussians instead of by their warp.  Ranks 0-299 are all
    wide (a group of 256 wide ones, then a partial group), every fifth rank beyond;
    pairs, splats and image against the oracle, with and without shrinking."""
    W, H = 640, 360
    cam = synth.look_at_camera([0.0, 0.0, 0.0], [0.0, 1.0, 0.0], W, H, 60.0)
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    t = np.asarray(cam.t, np.float64)
    rng = np.random.default_rng(23)
    n = 1400
    u = rng.uniform(0.0, W, n)
    v = rng.uniform(0.0, H, n)
    z = rng.uniform(8.0, 30.0, n)
    xc = (u - cam.cx) * z / cam.fx
    yc = (v - cam.cy) * z / cam.fy
    mu = (np.stack([xc, yc, z], 1) - t) @ R
    rank = np.empty(n, np.int64)                  # the leaves' selection ranks (Morton order)
    rank[np.argsort(synth.morton_codes(mu), kind="stable")] = np.arange(n)
    wide = (rank < 300) | (rank % 5 == 0)
    sigma_px = np.where(wide, rng.uniform(50.0, 120.0, n), rng.uniform(0.5, 3.0, n))
    log_s = np.log(sigma_px * z / cam.fx)
    tree = synth.tree_from_gaussians(mu, np.repeat(log_s[:, None], 3, 1), np.tile([1.0, 0, 0, 0], (n, 1)),
                                     np.where(wide, rng.normal(2.0, 0.5, n), rng.normal(-1.0, 1.0, n)),
                                     rng.normal(0, 1, (n, 1, 3)), 0)
    renderer.load_tree(tree)
    for shrink in (None, (0.05, float(np.float32(np.log(np.float32(0.05)))))):
        g = gpu_frame(renderer, tree, cam, -1.0, shrink=shrink)
        o, _ = oracle_frame(tree, cam, -1.0, shrink=shrink)
        per_g = np.bincount(o.vals.astype(np.int64), minlength=len(o.sel))
        assert (per_g[:256] > 128).sum() >= 200 and per_g.max() > 400, np.sort(per_g)[-5:]
        assert_frame_parity(g, o)


def test_depth_ties_break_by_id(renderer):
    """Duplicated Gaussians at one depth: equal keys keep ascending selection order."""
    mu = np.array([[0.0, 10.0, 0.0]] * 6 + [[0.3, 10.0, 0.2]] * 3)
    n = mu.shape[0]
    rng = np.random.default_rng(3)
    t = synth.tree_from_gaussians(mu, np.full((n, 3), -1.5), np.tile([1.0, 0, 0, 0], (n, 1)),
                                  rng.normal(0, 1, n), rng.normal(0, 1, (n, 1, 3)), 0)
    renderer.load_tree(t)
    cam = synth.look_at_camera([0, 0, 0], [0, 1, 0], 64, 64, 60.0)
    g = gpu_frame(renderer, t, cam, -1.0)
    o, _ = oracle_frame(t, cam, -1.0)
    assert_frame_parity(g, o)
    k = g["keys"]
    assert np.any(k[1:] == k[:-1])     # ties exist


def test_capacity_exceeded_is_reported(tiny):
    """N_P above the pair capacity: the frame reports FGS_ERR_CAPACITY (no overflow write),
    and the context renders correctly once the capacity is raised."""
    from paper_2603_23891_gb300 import filtergs
    tree, cam = tiny
    r2 = filtergs.Renderer(device=0, pair_capacity=1000)
    try:
        r2.load_tree(tree)
        r2.set_camera(cam)
        with pytest.raises(filtergs.FgsError) as e:
            r2.render(stats=True)
        assert e.value.code == filtergs.FGS_ERR_CAPACITY
        r2.set_params(pair_capacity=1 << 20)
        g = gpu_frame(r2, tree, cam, 3.0)
        o, _ = oracle_frame(tree, cam, 3.0)
        assert len(o.keys) > 1000
        assert_frame_parity(g, o)
    finally:
        r2.close()


def test_invalid_inputs_rejected(renderer, tiny):
    from paper_2603_23891_gb300 import filtergs
    tree, cam = tiny
    renderer.load_tree(tree)
    bad = filtergs.make_camera(cam)
    bad.fx = float("nan")
    with pytest.raises(filtergs.FgsError) as e:
        filtergs.fgs_set_camera(renderer.ctx, bad)
    assert e.value.code == filtergs.FGS_ERR_ARG
    bad = filtergs.make_camera(cam)
    bad.width = 0
    with pytest.raises(filtergs.FgsError):
        filtergs.fgs_set_camera(renderer.ctx, bad)
    with pytest.raises(filtergs.FgsError):
        renderer.set_params(tile=(16, 8))
    renderer.set_params(tile=(16, 16))
    with pytest.raises(filtergs.FgsError):
        filtergs.fgs_set_shrink(renderer.ctx, 1, float("nan"), 0.0)
    par = tree.parent.copy()
    par[3] = 3
    import copy
    t2 = copy.copy(tree)
    t2.parent = par
    with pytest.raises(filtergs.FgsError) as e:
        filtergs.fgs_load_tree(renderer.ctx, t2)
    assert e.value.code == filtergs.FGS_ERR_TREE


@pytest.mark.parametrize("seed", range(3))
def test_needles_and_blobs_culling_exact(renderer, seed):
    """Very elongated and very large Gaussians at random orientations: the per-warp culling
    of the blend (and its fallback for ill-conditioned conics) leaves every pixel's
    decisions unchanged, so T stays bit-identical."""
    rng = np.random.default_rng(100 + seed)
    n = 400
    mu = np.stack([rng.uniform(-6, 6, n), rng.uniform(6, 30, n), rng.uniform(-4, 4, n)], 1)
    logs = np.stack([rng.uniform(-5, -3, n), rng.uniform(-5, -3, n), rng.uniform(-0.5, 1.5, n)], 1)
    big = rng.random(n) < 0.15
    logs[big] = rng.uniform(-0.5, 0.8, (big.sum(), 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    t = synth.tree_from_gaussians(mu, logs, q, rng.normal(1.0, 1.5, n), rng.normal(0, 1, (n, 1, 3)), 0)
    renderer.load_tree(t)
    cam = synth.look_at_camera([0, 0, 0], [0, 1, 0], 192, 160, 70.0)
    g = gpu_frame(renderer, t, cam, -1.0)
    o, _ = oracle_frame(t, cam, -1.0)
    assert_frame_parity(g, o)


@pytest.mark.parametrize("seed", range(3))
def test_tiny_gaussians_straddling_warp_blocks(renderer, seed):
    """Thousands of Gaussians a few pixels across (threshold ellipses 2-5 px) at random
    sub-pixel positions and orientations, low opacity so pixels rarely stop: many
    ellipse boxes end within a hundredth of a pixel of a warp-block edge, where the
    blend's culling margin is tightest.  A Gaussian culled from a warp whose pixel
    passes the skip test would change that pixel's T, which is compared bit for bit."""
    rng = np.random.default_rng(300 + seed)
    n = 5000
    mu = np.stack([rng.uniform(-7, 7, n), rng.uniform(8, 14, n), rng.uniform(-6, 6, n)], 1)
    logs = rng.uniform(-3.9, -2.2, (n, 3))
    logs[:, 2] += rng.uniform(-1.5, 0.0, n)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    t = synth.tree_from_gaussians(mu, logs, q, rng.normal(-1.5, 1.0, n), rng.normal(0, 1, (n, 1, 3)), 0)
    renderer.load_tree(t)
    cam = synth.look_at_camera([0, 0, 0], [0, 1, 0], 200, 168, 70.0)
    g = gpu_frame(renderer, t, cam, -1.0)
    o, _ = oracle_frame(t, cam, -1.0)
    assert o.n_pairs > 4000
    assert_frame_parity(g, o)


@pytest.mark.parametrize("seed", range(3))
def test_levelwise_baseline_selects_same_set(renderer, seed):
    """The serial level-by-level selection (Eq. 3 scheme) and the traversal-free filter
    select exactly the oracle's LoD cut (§3.2, Table 3)."""
    tree = synth.random_small_tree(20 + seed, n_leaves=5000, branching=(2, 8), sh_degree=0,
                                   extent=25.0, log_scale_mean=-0.8)
    renderer.load_tree(tree)
    for cam in orbit_cameras(tree, 3, (200, 150), seed, dist=(10.0, 90.0)):
        for tau_R in (-1.0, 3.0, 15.0, 1e30):
            renderer.set_params(tau_R=tau_R)
            renderer.set_camera(cam)
            sel_lw, levels = renderer.filter_levelwise()
            sel = renderer.filter()
            ref = oracle.filter_dfs(tree, cam, tau_R)
            assert np.array_equal(sel_lw, ref) and np.array_equal(sel, ref)
            assert 1 <= levels <= tree.depth + 1


def test_bounded_wait_times_out_and_context_stays_usable(renderer, tiny):
    """Failure detection without a GPU fault: a look-back wait on an entry that nothing
    publishes gives up after its bound, the host reads FGS_ERR_TIMEOUT with the probe's
    site code, and the next frames render bit-exactly as before."""
    from paper_2603_23891_gb300 import filtergs
    tree, cam = tiny
    renderer.load_tree(tree)
    before = gpu_frame(renderer, tree, cam, 1.0)
    for _ in range(2):
        code, site = renderer.probe_wait_timeout()
        assert code == filtergs.FGS_ERR_TIMEOUT and site == 0x7F0
    renderer.sync()                                 # the status was cleared by the probe
    after = gpu_frame(renderer, tree, cam, 1.0)
    o, _ = oracle_frame(tree, cam, 1.0)
    assert_frame_parity(after, o)
    assert np.array_equal(after["rgb"], before["rgb"]) and np.array_equal(after["T"], before["T"])


def test_blend_counters_consistent(renderer, tiny):
    """The counting blend variant renders the same image and reports consistent work:
    alpha-applying evaluations <= evaluations <= 32 x lockstep warp steps."""
    import torch
    tree, cam = tiny
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    renderer.set_camera(cam)
    renderer.shrink(None)
    rgb0, T0, st0 = renderer.render(stats=True)
    rgb1, T1, st1 = renderer.render(count=True)
    torch.cuda.synchronize()
    assert torch.equal(rgb0, rgb1) and torch.equal(T0, T1)
    assert st1.n_pairs == st0.n_pairs
    assert 0 < st1.blend_hits <= st1.blend_evals <= 32 * st1.blend_entries
    assert st1.blend_entries <= 8 * st1.n_pairs
    # every entry where some pixel applies alpha has at least one such pixel
    assert st1.blend_active <= st1.blend_hits <= 32 * st1.blend_active
    assert st1.blend_active <= st1.blend_entries


def test_crowded_tiles_sorted_in_global_memory(renderer):
    """Tiles holding more than 4096 pairs (the block sort's shared-memory limit): 20k
    Gaussians seen at 64x48 on 16x16 tiles (12 tiles), each bucket sorted by one block
    in global memory; pairs and image against the oracle."""
    tree = synth.random_small_tree(21, n_leaves=20000, branching=(2, 6), sh_degree=0,
                                   extent=6.0, log_scale_mean=-1.0)
    cam = synth.look_at_camera([0.0, -16.0, 8.0], [0.0, 0.0, 0.0], 64, 48, 60.0)
    renderer.load_tree(tree)
    g = gpu_frame(renderer, tree, cam, -1.0)
    o, _ = oracle_frame(tree, cam, -1.0)
    tiles = (o.keys >> np.uint64(32)).astype(np.int64)
    per_tile = np.bincount(tiles)
    assert per_tile.max() > 4096, per_tile.max()
    assert_frame_parity(g, o)


def test_large_tile_grid(renderer):
    """A 4096x4096 image on 16x16 tiles (65,536 tiles, the most a view may have: the
    tile scan runs 16 rounds); pairs bit for bit, sampled pixels."""
    tree = synth.tiny_tree()
    cam = synth.look_at_camera([0.0, -60.0, 30.0], [0.0, 0.0, 0.0], 4096, 4096, 60.0)
    renderer.load_tree(tree)
    g = gpu_frame(renderer, tree, cam, 3.0)
    o, p = oracle_frame(tree, cam, 3.0, blend=False)
    assert len(o.keys) > 100000
    assert_frame_parity(g, o, check_image=False)
    pix = np.sort(np.random.default_rng(3).choice(4096 * 4096, 20000, replace=False))
    rgb, T = oracle.render_pixels(o.splat, o.keys, o.vals, cam, p, pix)
    grgb = g["rgb"].reshape(3, -1)[:, pix].T.astype(np.float64)
    assert np.abs(grgb - rgb).max() <= IMG_TOL
    assert np.array_equal(g["T"].reshape(-1)[pix].view(np.uint32), T.view(np.uint32))


def test_tiny_tree_thousand_random_cameras(renderer, tiny):
    """The tiny LoD tree (4,096 leaves, LoD threshold 1 px) from 1,000 random 256x256
    cameras (positions over and around the box, random targets and FOVs, some looking
    away): selection, pair list and transmittance bit for bit, images within 2e-3 and
    60 dB, for every camera."""
    import time
    tree, _ = tiny
    renderer.load_tree(tree)
    rng = np.random.default_rng(1)
    t0 = time.time()
    worst = 0.0
    n_empty = 0
    for k in range(1000):
        pos = rng.uniform([-80.0, -80.0, 2.0], [80.0, 80.0, 90.0])
        target = rng.uniform([-32.0, -32.0, -4.0], [32.0, 32.0, 4.0])
        if k % 10 == 9:                                   # some cameras face away from the box
            target = pos + (pos - target)
        cam = synth.look_at_camera(pos, target, 256, 256, rng.uniform(30.0, 100.0))
        g = gpu_frame(renderer, tree, cam, 1.0)
        o, _ = oracle_frame(tree, cam, 1.0)
        worst = max(worst, assert_frame_parity(g, o))
        n_empty += len(o.sel) == 0
    print(f"1000 cameras: worst max-abs {worst:.2e}, {n_empty} empty views, {time.time() - t0:.1f}s")
    assert n_empty < 1000


def test_tile_grid_limit_rejected(renderer):
    """More than 65,536 tiles (16384 x 8192 on 16x16 tiles) is refused on the host
    before any launch; the context stays usable."""
    from paper_2603_23891_gb300 import filtergs
    tree = synth.tiny_tree()
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    big = synth.look_at_camera([0.0, -60.0, 30.0], [0.0, 0.0, 0.0], 16384, 8192, 70.0)
    with pytest.raises(filtergs.FgsError) as e:
        renderer.set_camera(big)
    assert e.value.code == filtergs.FGS_ERR_ARG
    cam = synth.tiny_camera()
    g = gpu_frame(renderer, tree, cam, 3.0)
    o, _ = oracle_frame(tree, cam, 3.0)
    assert_frame_parity(g, o)


@pytest.mark.parametrize("ties", ["none", "short", "long"])
def test_bucket_sizes_at_sort_boundaries(renderer, ties):
    """One row of 16x16 tiles whose tiles hold exactly 0, 1, 2, 32, 33, 64, 65, 128, 129,
    256, 257, 511, 512, 513, 1024, 1025, 2048, 2049, 4096 and 4097 pairs (each Gaussian a
    few pixels wide, inside one tile): every size class of the per-tile sort (one warp
    with 1, 2, 4 or 8 items a lane; one block by depth radix in shared memory with 2, 4
    or 8 items a thread; one block by radix passes in global memory) and its edges,
    without depth ties, with short runs of equal depths inside the buckets (put in rank
    order where they lie after the depth sort) and with one run of 40 equal depths per
    bucket (longer than the in-place fix takes: the bitonic network in shared memory,
    or the full radix passes in global memory); pairs, splats and image against the
    oracle."""
    counts = [1, 32, 33, 64, 65, 128, 129, 256, 257, 511, 512, 513, 1024, 1025, 2048, 2049, 4096,
              4097, 0, 2]
    W, H = 16 * len(counts), 16
    cam = synth.look_at_camera([0.0, 0.0, 0.0], [0.0, 1.0, 0.0], W, H, 60.0)
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    t = np.asarray(cam.t, np.float64)
    rng = np.random.default_rng(17)
    pts = []
    for i, c in enumerate(counts):
        u = 16 * i + rng.uniform(3.5, 12.5, c)
        v = rng.uniform(3.5, 12.5, c)
        if ties == "short":                                          # repeated depths
            z = rng.choice(rng.uniform(5.0, 40.0, max(c // 3, 1)), c)
        else:                                                        # distinct depths
            z = rng.permutation(5.0 + np.arange(c) * (35.0 / max(c, 1)))
            if ties == "long" and c >= 80:                           # one run of 40
                z[rng.choice(c, 40, replace=False)] = z[0]
        xc = (u - cam.cx) * z / cam.fx
        yc = (v - cam.cy) * z / cam.fy
        cpts = np.stack([xc, yc, z], 1)
        pts.append((cpts - t) @ R)                                   # world = R^T (c - t)
    mu = np.concatenate(pts)
    n = mu.shape[0]
    tree = synth.tree_from_gaussians(mu, np.full((n, 3), -6.0), np.tile([1.0, 0, 0, 0], (n, 1)),
                                     rng.normal(0, 1, n), rng.normal(0, 1, (n, 1, 3)), 0)
    renderer.load_tree(tree)
    g = gpu_frame(renderer, tree, cam, -1.0)
    o, _ = oracle_frame(tree, cam, -1.0)
    per_tile = np.bincount((o.keys >> np.uint64(32)).astype(np.int64), minlength=len(counts))
    assert np.array_equal(per_tile, counts), per_tile
    depth_tie = (o.keys[1:] == o.keys[:-1])
    assert depth_tie.any() == (ties != "none")
    assert_frame_parity(g, o)


def test_pipelined_host_outputs(renderer, tiny):
    """FGS_RENDER_ASYNC: six frames of mixed cameras (and one resolution change)
    rendered into pinned host buffers without waiting, two frames in flight; after
    fgs_sync every buffer holds exactly what a synchronising host render of the same
    camera returns (bits of colour and transmittance)."""
    import torch
    tree, cam0 = tiny
    renderer.load_tree(tree)
    renderer.set_params(tau_R=1.0)
    renderer.shrink(None)
    cams = orbit_cameras(tree, 4, (256, 256), 5) + orbit_cameras(tree, 2, (320, 200), 6)
    ref = []
    for c in cams:
        renderer.set_camera(c)
        rgb = np.zeros((3, c.height, c.width), np.float32)
        T = np.zeros((c.height, c.width), np.float32)
        renderer.render_host(rgb, T)
        ref.append((rgb, T))
    bufs = [(torch.zeros((3, c.height, c.width), dtype=torch.float32).pin_memory(),
             torch.zeros((c.height, c.width), dtype=torch.float32).pin_memory()) for c in cams]
    for c, (rgb, T) in zip(cams, bufs):
        renderer.set_camera(c)
        renderer.render_host(rgb.numpy(), T.numpy(), pipelined=True)
    renderer.sync()
    for (rgb, T), (rr, tr) in zip(bufs, ref):
        assert np.array_equal(rgb.numpy().view(np.uint32), rr.view(np.uint32))
        assert np.array_equal(T.numpy().view(np.uint32), tr.view(np.uint32))
    # stats need a synchronisation, so they do not combine with the pipelined mode
    from paper_2603_23891_gb300 import filtergs
    with pytest.raises(RuntimeError):
        filtergs.fgs_render(renderer.ctx, renderer.stream, bufs[0][0].numpy(), None, 0,
                            filtergs.FGS_RENDER_ASYNC | filtergs.FGS_RENDER_STATS, filtergs.fgs_stats())


def test_frustum_boundary_chunks(renderer):
    """Leaves on and beside the guard-banded frustum's planes (|x / z| and |y / z| at
    1.3 times the half-FOV tangents, depth 0.2) at relative offsets down to 1e-7:
    the R&L filter skips a 128-node chunk only when its centres' box lies beyond a
    plane by a margin, so the selection must equal the oracle's node for node."""
    import math as _m
    W, H = 320, 240
    cam = synth.look_at_camera([0.0, 0.0, 0.0], [0.0, 1.0, 0.0], W, H, 60.0)
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    t = np.asarray(cam.t, np.float64)
    Lx, Ly = 1.3 * cam.tan_half_x, 1.3 * cam.tan_half_y
    rng = np.random.default_rng(31)
    n = 8192
    z = rng.uniform(0.05, 60.0, n)
    rel = rng.choice([-1e-3, -1e-5, -1e-7, 0.0, 1e-7, 1e-5, 1e-3], n)
    side = rng.integers(0, 5, n)
    x = rng.uniform(-Lx, Lx, n) * z
    y = rng.uniform(-Ly, Ly, n) * z
    x = np.where(side == 0, (Lx + rel) * z, np.where(side == 1, -(Lx + rel) * z, x))
    y = np.where(side == 2, (Ly + rel) * z, np.where(side == 3, -(Ly + rel) * z, y))
    z = np.where(side == 4, 0.2 * (1.0 + rel), z)
    mu = (np.stack([x, y, z], 1) - t) @ R
    tree = synth.tree_from_gaussians(mu, np.full((n, 3), -4.0), np.tile([1.0, 0, 0, 0], (n, 1)),
                                     rng.normal(0, 1, n), rng.normal(0, 1, (n, 1, 3)), 0)
    renderer.load_tree(tree)
    g = gpu_frame(renderer, tree, cam, -1.0)
    o, _ = oracle_frame(tree, cam, -1.0, blend=False)
    assert 0 < len(o.sel) < n
    assert np.array_equal(g["sel"], o.sel), (len(g["sel"]), len(o.sel))

"""GPU parity at the benchmark workloads' full sizes.

1M-leaf blob tree at 1920x1080: every pose, shrink off and on, whole frames.
10M-leaf city tree at 1920x1080 (the benchmark workload and launch configuration,
adaptive shrink): sampled poses; selection, splats and pairs bit for bit, the
image on sampled pixels that the oracle evaluates one by one.
The batched form at its own workload's scale: the 32 city views of uneven resolution
(360p to 2160p) in one CUDA-graph batch; sampled views against the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_23891_gb300 import synth

from gpu_util import (IMG_TOL, assert_frame_parity, batch_view_frame, gpu_frame, grad_parity_case,
                      oracle_frame, psnr)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_23891_gb300 import build, filtergs
    build.build()
    r = filtergs.Renderer(device=0, pair_capacity=64 << 20)
    yield r
    r.close()


@pytest.fixture(scope="module")
def blobs():
    return synth.blob_tree(), synth.blob_cameras()


def test_blobs_all_poses_shrink_off(renderer, blobs):
    tree, cams = blobs
    renderer.load_tree(tree)
    for k, cam in enumerate(cams):
        g = gpu_frame(renderer, tree, cam, 3.0)
        o, _ = oracle_frame(tree, cam, 3.0)
        err = assert_frame_parity(g, o)
        assert g["NP"] > 500_000, k
        print(f"pose {k}: M={g['M']} N_P={g['NP']} max_abs={err:.2e}")


def test_blobs_adaptive_shrink(renderer, blobs):
    """Calibration over the 8 poses on the GPU and in the oracle agree (Eq. 8); with the
    same tau bits both sides emit the same pairs and images.  The shrunk image against
    the unshrunk oracle is reported, not gated."""
    tree, cams = blobs
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    tau, ln_tau, gbars = renderer.calibrate(cams, 0.2)
    otau, oln, ogbars = oracle.calibrate(tree, cams, 3.0, 0.2)
    np.testing.assert_allclose(gbars, ogbars, rtol=1e-4)
    assert tau == pytest.approx(otau, rel=1e-4)
    for k in (0, 3, 6):
        g = gpu_frame(renderer, tree, cams[k], 3.0, shrink=(tau, ln_tau))
        o, _ = oracle_frame(tree, cams[k], 3.0, shrink=(tau, ln_tau))
        assert_frame_parity(g, o)
        o_off, _ = oracle_frame(tree, cams[k], 3.0)
        assert g["NP"] < len(o_off.keys)
        print(f"pose {k}: tau={tau:.4f} N_P {len(o_off.keys)} -> {g['NP']}; shrunk vs unshrunk "
              f"PSNR {psnr(g['rgb'], o_off.rgb):.1f} dB, max-abs "
              f"{np.abs(g['rgb'] - o_off.rgb).max():.3f}")


@pytest.fixture(scope="module")
def city():
    return synth.city_tree(), synth.city_cameras()


def test_city_benchmark_configuration(renderer, city):
    """The benchmark's workload and launch configuration (tau from the GPU calibration over
    the 64 poses, adaptive shrink, 16x16 tiles, 64 Mi pair capacity)."""
    tree, cams = city
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    tau, ln_tau, gbars = renderer.calibrate(cams, 0.2)
    assert np.isfinite(gbars).all()
    rng = np.random.default_rng(0)
    for k in (0, 21, 42, 63):
        cam = cams[k]
        g = gpu_frame(renderer, tree, cam, 3.0, shrink=(tau, ln_tau))
        o, p = oracle_frame(tree, cam, 3.0, shrink=(tau, ln_tau), blend=False)
        assert_frame_parity(g, o, check_image=False)
        sel_lw, _ = renderer.filter_levelwise()
        assert np.array_equal(sel_lw, o.sel)
        n = cam.width * cam.height
        pix = np.sort(rng.choice(n, size=20000, replace=False))
        rgb, T = oracle.render_pixels(o.splat, o.keys, o.vals, cam, p, pix)
        grgb = g["rgb"].reshape(3, -1)[:, pix].T.astype(np.float64)
        gT = g["T"].reshape(-1)[pix]
        assert np.abs(grgb - rgb).max() <= IMG_TOL
        assert np.array_equal(gT.view(np.uint32), T.view(np.uint32))
        print(f"pose {k}: M={g['M']} N_P={g['NP']} sampled max-abs {np.abs(grgb - rgb).max():.2e}")


def test_city_gradient_sampled_pixels(renderer, city):
    """Differentiable form on the 10M-leaf city tree at 1920x1080 (16x16 tiles, shrink at
    tau = 0.0772): the gradient of a loss on 4096 sampled pixels for every node, against
    the oracle's binary64 gradient; selection and pairs bit for bit."""
    tree, cams = city
    pix = np.sort(np.random.default_rng(5).choice(1920 * 1080, 4096, replace=False))
    shrink = (0.0772, float(np.float32(math.log(0.0772))))
    g, of, worst = grad_parity_case(renderer, tree, cams[21], 3.0, 8, bg=(0.0, 0.0, 0.0),
                                    shrink=shrink, pix=pix)
    print(f"city pose 21: M={g['M']} N_P={g['NP']} worst relative gradient error "
          f"{max(worst.values()):.2e}")


def test_city_batch_32_views_sampled(renderer, city):
    """The 32-view batch over the city tree (8 views each at 640x360, 1280x720,
    1920x1080, 3840x2160; tiles 16x16 with 8x4 warps and 32x8 with 4x8 warps
    alternating; adaptive shrink at tau = 0.0772; CUDA-graph replay).  Six views, three
    of them 3840x2160, against the oracle: selection (§3.2: equal to the serial
    traversal), splat decision fields and the view's sorted pairs bit for bit, and
    20,000 sampled pixels (transmittance bits, colour within the image tolerance)."""
    import torch
    tree, _ = city
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    shrink = (0.0772, float(np.float32(math.log(0.0772))))
    renderer.shrink(*shrink)
    bc = synth.city_batch_cameras()
    shapes = [(16, 16, 8) if v % 2 == 0 else (32, 8, 4) for v in range(len(bc))]
    renderer.batch_setup(bc, tile_shapes=shapes, sel_capacity=48 << 20, pair_capacity=64 << 20)
    renderer.render_batch(graph=True, stats=True)
    rgb, T, st, views = renderer.render_batch(graph=True, stats=True)
    torch.cuda.synchronize()
    frames = renderer.batch_frame()
    assert sum(f["M"] for f in frames) == st.n_selected
    assert sum(f["NP"] for f in frames) == st.n_pairs
    rng = np.random.default_rng(1)
    for v in (0, 9, 18, 27, 28, 31):
        cam, (tw, th, _) = bc[v], shapes[v]
        o, p = oracle_frame(tree, cam, 3.0, shrink=shrink, tile=(tw, th), blend=False)
        assert_frame_parity(batch_view_frame(frames[v]), o, check_image=False)
        n = cam.width * cam.height
        pix = np.sort(rng.choice(n, size=20000, replace=False))
        orgb, oT = oracle.render_pixels(o.splat, o.keys, o.vals, cam, p, pix)
        grgb = views[v][0].cpu().numpy().reshape(3, -1)[:, pix].T.astype(np.float64)
        gT = views[v][1].cpu().numpy().reshape(-1)[pix]
        assert np.abs(grgb - orgb).max() <= IMG_TOL, v
        assert np.array_equal(gT.view(np.uint32), oT.view(np.uint32)), v
        print(f"batch view {v} ({cam.width}x{cam.height}, tile {tw}x{th}): M={frames[v]['M']} "
              f"N_P={frames[v]['NP']} sampled max-abs {np.abs(grgb - orgb).max():.2e}")
    renderer.shrink(None)

"""GPU parity of the differentiable form: parameters -> attributes (bit-exact with
the oracle's binary32 map, checked through the whole frame), and the hand-written
backward against the oracle's binary64 gradient of the frozen-decision render.

Gradient bar: per parameter group, max |g_gpu - g_oracle| <= 1e-3 max |g_oracle|
(binary32 kernels against binary64); nodes outside the cut get exactly zero."""
import numpy as np
import pytest

import oracle
from paper_2603_23891_gb300 import synth

from gpu_util import GRAD_RTOL, dev_params, gpu_grad, grad_parity_case

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


@pytest.mark.parametrize("seed,deg,warp_w", [(0, 3, 8), (1, 1, 4), (2, 0, 8), (3, 2, 4)])
def test_grad_scene(renderer, seed, deg, warp_w):
    """64 Gaussians at 32x32 (several layers per pixel), SH degrees 0-3, both warp shapes."""
    tree, cam = synth.grad_scene(seed, sh_degree=deg)
    _, of, worst = grad_parity_case(renderer, tree, cam, 0.0, seed, warp_w=warp_w)
    assert len(of.ent) > 4 * cam.width * cam.height
    print(f"seed {seed}: worst relative gradient error {max(worst.values()):.2e}")


@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_multilevel_cut_ragged_and_shrink(renderer, tile):
    """A cut with internal nodes, a 40x24 image (ragged tiles), shrink on and off."""
    tree = synth.random_small_tree(7, n_leaves=96, branching=(3, 5), sh_degree=2, extent=5.0,
                                   log_scale_mean=-0.8)
    cam = synth.look_at_camera([0.0, -14.0, 6.0], [0.0, 0.0, 0.0], 40, 24, 60.0)
    for shrink in (None, (0.02, float(np.float32(np.log(0.02))))):
        g, of, _ = grad_parity_case(renderer, tree, cam, 6.0, 5, tile=tile, shrink=shrink)
        assert (tree.is_leaf[of.frame.sel] == 0).any()


def test_random_trees_many_tiles(renderer):
    """Larger random trees over several tiles: 2k leaves, 200x120, τ_R sweep."""
    for seed, tau_R in ((11, 2.0), (12, 8.0), (13, 0.0)):
        tree = synth.random_small_tree(seed, n_leaves=2000, branching=(2, 6), sh_degree=3,
                                       extent=12.0, log_scale_mean=-1.2)
        cam = synth.look_at_camera([0.0, -30.0, 14.0], [0.0, 0.0, 0.0], 200, 120, 60.0)
        grad_parity_case(renderer, tree, cam, tau_R, seed)


def test_empty_view_gradient_is_zero(renderer):
    import torch
    tree, cam = synth.grad_scene(0)
    away = synth.look_at_camera([0.0, -12.0, 4.0], [0.0, -40.0, 4.0], 32, 32, 60.0)
    gp = oracle.GaussParams.of_tree(tree)
    renderer.load_tree(tree)
    g = gpu_grad(renderer, gp, away, 0.0, np.ones((3, 32, 32), np.float32))
    assert g["M"] == 0
    for k, v in g["grads"].items():
        assert not v.any(), k


def test_accumulate_and_autograd(renderer):
    import torch
    from paper_2603_23891_gb300 import filtergs
    tree, cam = synth.grad_scene(4, sh_degree=3)
    gp = oracle.GaussParams.of_tree(tree)
    renderer.load_tree(tree)
    dL = np.random.default_rng(3).normal(size=(3, 32, 32)).astype(np.float32)
    g = gpu_grad(renderer, gp, cam, 0.0, dL, bg=(0.2, 0.1, 0.4))
    P = g["P"]
    # accumulate: the same frame's gradient added twice
    renderer.update_params(P)
    renderer.render(keep=True)
    dLt = torch.from_numpy(dL).cuda()
    acc = renderer.backward(dLt, P)
    renderer.backward(dLt, P, grads=acc, accumulate=True)
    # each gradient is a sum of float atomic additions whose order differs from run
    # to run, so two runs agree to rounding relative to the field's scale
    for k in oracle.GRAD_FIELDS:
        ref = 2 * g["grads"][k]
        np.testing.assert_allclose(acc[k].cpu().numpy(), ref, rtol=1e-5,
                                   atol=1e-6 * float(np.abs(ref).max()))
    # torch autograd through the hand-written backward
    leaves = [P[k].clone().requires_grad_(True) for k in oracle.GRAD_FIELDS]
    rgb = filtergs.render_differentiable(renderer, *leaves)
    np.testing.assert_array_equal(rgb.detach().cpu().numpy(), g["rgb"])
    (rgb * dLt).sum().backward()
    for k, leaf in zip(oracle.GRAD_FIELDS, leaves):
        ref = g["grads"][k]
        np.testing.assert_allclose(leaf.grad.cpu().numpy(), ref, rtol=1e-5,
                                   atol=1e-6 * float(np.abs(ref).max()))


def test_backward_state_and_argument_errors(renderer):
    import torch
    from paper_2603_23891_gb300 import filtergs
    tree, cam = synth.grad_scene(0)
    gp = oracle.GaussParams.of_tree(tree)
    renderer.load_tree(tree)
    renderer.set_camera(cam)
    P = dev_params(gp)
    renderer.update_params(P)
    dL = torch.zeros((3, 32, 32), device="cuda")
    with pytest.raises(filtergs.FgsError) as e:          # no frame since the parameters changed
        renderer.backward(dL, P)
    assert e.value.code == filtergs.FGS_ERR_STATE
    renderer.calibrate_view()                            # a calibration frame is not differentiable
    with pytest.raises(filtergs.FgsError) as e:
        renderer.backward(dL, P)
    assert e.value.code == filtergs.FGS_ERR_STATE
    renderer.render(keep=True)
    host = {k: v.cpu() for k, v in P.items()}
    with pytest.raises(filtergs.FgsError) as e:          # host memory is refused before any launch
        filtergs.fgs_backward(renderer.ctx, renderer.stream, dL, host,
                              {k: torch.empty_like(v) for k, v in P.items()})
    assert e.value.code == filtergs.FGS_ERR_ARG
    renderer.backward(dL, P)                             # still fine afterwards
    torch.cuda.synchronize()


def test_blobs_1080p_sampled_pixels(renderer):
    """1M-leaf blob tree at 1920x1080 with shrink: the gradient of a loss on 4096
    sampled pixels, every node's gradient against the oracle's."""
    tree = synth.blob_tree()
    cam = synth.blob_cameras()[2]
    pix = np.sort(np.random.default_rng(9).choice(cam.width * cam.height, 4096, replace=False))
    shrink = (0.05, float(np.float32(np.log(0.05))))
    g, of, worst = grad_parity_case(renderer, tree, cam, 3.0, 21, shrink=shrink, pix=pix)
    print(f"blobs: M={g['M']} N_P={g['NP']} worst relative gradient error {max(worst.values()):.2e}")


@pytest.mark.parametrize("seed", [0, 5])
def test_recomputed_transmittance_equals_kept(renderer, seed):
    """The default backward recomputes each pixel's final T and stop by a walk over its
    tile; after a FGS_RENDER_KEEP forward it reads them.  Same gradients (up to the
    order of the atomic additions), on a one-tile scene and a multi-tile random tree."""
    import torch
    if seed == 0:
        tree, cam = synth.grad_scene(4, sh_degree=3)
    else:
        tree = synth.random_small_tree(seed, n_leaves=3000, branching=(2, 6), sh_degree=2,
                                       extent=12.0, log_scale_mean=-1.0)
        cam = synth.look_at_camera([0.0, -30.0, 14.0], [0.0, 0.0, 0.0], 160, 96, 60.0)
    gp = oracle.GaussParams.of_tree(tree)
    renderer.load_tree(tree)
    renderer.set_params(tau_R=2.0, tile=(16, 16), bg=(0.2, 0.1, 0.4))
    renderer.set_camera(cam)
    renderer.shrink(None)
    P = dev_params(gp)
    renderer.update_params(P)
    dL = torch.randn((3, cam.height, cam.width), device="cuda",
                     generator=torch.Generator(device="cuda").manual_seed(seed))
    renderer.render(keep=True)
    kept = {k: v.cpu().numpy() for k, v in renderer.backward(dL, P).items()}
    renderer.render()
    rec = {k: v.cpu().numpy() for k, v in renderer.backward(dL, P).items()}
    for k in oracle.GRAD_FIELDS:
        scale = np.abs(kept[k]).max()
        assert np.abs(rec[k] - kept[k]).max() <= 1e-5 * scale + 1e-9, k


def test_blobs_l2_loss_against_perturbed_target(renderer):
    """The differentiable configuration: the 1M-leaf blob tree at 1920x1080, L2 loss
    against the image of the tree with every leaf attribute perturbed by N(0, 0.01);
    gradient of the loss restricted to 4096 sampled pixels, every node against the
    oracle (default backward: transmittance recomputed per tile)."""
    import torch
    tree, target_tree = synth.blob_tree(), synth.blob_target_tree()
    cam = synth.blob_cameras()[0]
    renderer.set_params(tau_R=3.0, tile=(16, 16), bg=(0.0, 0.0, 0.0))
    renderer.set_camera(cam)
    renderer.shrink(None)
    renderer.load_tree(target_tree)
    target, _, _ = renderer.render()
    target = target.clone()
    renderer.load_tree(tree)
    gp = oracle.GaussParams.of_tree(tree)
    P = dev_params(gp)
    renderer.update_params(P)
    rgb, _, _ = renderer.render()
    pix = np.sort(np.random.default_rng(17).choice(cam.width * cam.height, 4096, replace=False))
    mask = torch.zeros(cam.width * cam.height, device="cuda")
    mask[torch.from_numpy(pix).cuda()] = 1.0
    dL = 2.0 * (rgb - target) * mask.view(1, cam.height, cam.width)
    G = {k: v.cpu().numpy() for k, v in renderer.backward(dL, P).items()}
    torch.cuda.synchronize()
    assert float((rgb - target).abs().max()) > 1e-3          # the target differs
    of = oracle.grad_frame(tree, gp, cam, oracle.Params(tau_R=3.0), dL.cpu().numpy(), pix=pix)
    for k in oracle.GRAD_FIELDS:
        o = of.grads[k]
        err = np.abs(G[k].astype(np.float64) - o).max()
        assert err <= GRAD_RTOL * np.abs(o).max() + 1e-7, (k, err, np.abs(o).max())

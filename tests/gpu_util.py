"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and the
oracle on the same seeded inputs and compare."""
import math

import numpy as np

import oracle
from paper_2603_23891_gb300 import synth

IMG_TOL = 2e-3          # max-abs per channel, FP32 accumulation (spec bound)
PSNR_MIN = 60.0
EXACT_FIELDS = [0, 1, 2, 3, 4, 5, 6, 7, 11]   # u v A B C lthr a0 depth radius
COLOUR_FIELDS = [8, 9, 10]
GRAD_RTOL = 1e-3        # per parameter group: max-abs error / max-abs oracle gradient


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0 else 10.0 * math.log10(1.0 / mse)


def gpu_frame(r, tree_loaded, cam, tau_R, shrink=None, tile=(16, 16), bg=(0, 0, 0)):
    """Render one frame on the GPU; returns dict of host numpy results."""
    import torch
    r.set_params(tau_R=tau_R, tile=tile, bg=bg)
    r.set_camera(cam)
    if shrink is None:
        r.shrink(None)
    else:
        r.shrink(*shrink)
    rgb, T, st = r.render(stats=True)
    torch.cuda.synchronize()
    keys, vals = r.pairs()
    spl = r.splats()
    out = dict(rgb=rgb.cpu().numpy(), T=T.cpu().numpy(), keys=keys, vals=vals, splat=spl,
               M=int(st.n_selected), NP=int(st.n_pairs), E=int(st.n_emitting))
    out["sel"] = r.filter()
    return out


def oracle_frame(tree, cam, tau_R, shrink=None, tile=(16, 16), bg=(0, 0, 0), blend=True):
    p = oracle.Params(tau_R=tau_R, tile_w=tile[0], tile_h=tile[1], bg=tuple(bg))
    if shrink is not None:
        p.shrink, p.tau, p.ln_tau = True, shrink[0], shrink[1]
    return oracle.frame(tree, cam, p, blend=blend), p


def assert_frame_parity(g, o, check_image=True):
    assert np.array_equal(g["sel"], o.sel), f"selection differs ({len(g['sel'])} vs {len(o.sel)})"
    assert g["M"] == len(o.sel)
    assert g["NP"] == len(o.keys)
    if "E" in g:
        rect = o.rect
        assert g["E"] == int(np.count_nonzero((rect[:, 1] > rect[:, 0]) & (rect[:, 3] > rect[:, 2])))
    assert g["splat"].shape == o.splat.shape
    if len(o.sel):
        ge = g["splat"][:, EXACT_FIELDS].view(np.uint32)
        oe = o.splat[:, EXACT_FIELDS].view(np.uint32)
        bad = np.nonzero((ge != oe).any(axis=1))[0]
        assert bad.size == 0, f"splat fields differ for {bad.size} Gaussians, first {bad[:5]}"
        # colours exist for Gaussians that emit pairs (the others' colours are never read)
        emits = ((o.rect[:, 1] - o.rect[:, 0]) > 0) & ((o.rect[:, 3] - o.rect[:, 2]) > 0)
        np.testing.assert_allclose(g["splat"][emits][:, COLOUR_FIELDS], o.splat[emits][:, COLOUR_FIELDS],
                                   atol=2e-5, rtol=0)
    assert np.array_equal(g["keys"], o.keys), "sorted keys differ"
    assert np.array_equal(g["vals"], o.vals), "sorted values differ"
    if check_image:
        err = np.abs(g["rgb"].astype(np.float64) - o.rgb)
        assert err.max() <= IMG_TOL, f"max-abs {err.max()}"
        assert psnr(g["rgb"], o.rgb) >= PSNR_MIN
        # transmittance is decided and multiplied in the same binary32 order on both sides
        assert np.array_equal(g["T"].view(np.uint32), o.T.view(np.uint32)), \
            f"T differs at {np.count_nonzero(g['T'] != o.T)} pixels"
        return float(err.max())
    return None


def batch_view_frame(bv, rgb_v=None, T_v=None):
    """One view of a batched render (``Renderer.batch_frame()`` entry plus its image
    planes) in the form ``assert_frame_parity`` takes."""
    g = dict(sel=bv["sel"], M=bv["M"], NP=bv["NP"], splat=bv["splat"], keys=bv["keys"],
             vals=bv["vals"])
    if rgb_v is not None:
        g["rgb"] = rgb_v.cpu().numpy()
        g["T"] = T_v.cpu().numpy()
    return g


def orbit_cameras(tree, n, size, seed, dist=(8.0, 40.0), fov=(35.0, 80.0)):
    rng = np.random.default_rng(seed)
    c = tree.mu.mean(axis=1).astype(np.float64)
    cams = []
    for _ in range(n):
        a = rng.uniform(0, 2 * math.pi)
        d = rng.uniform(*dist)
        pos = [c[0] + d * math.cos(a), c[1] + d * math.sin(a), c[2] + rng.uniform(1.0, 0.6 * d)]
        cams.append(synth.look_at_camera(pos, c + rng.normal(0, 1.0, 3), size[0], size[1],
                                         rng.uniform(*fov)))
    return cams


# ---------------------------------------------------------------- differentiable form

def dev_params(gp):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(gp, k), np.float32)).cuda()
            for k in oracle.GRAD_FIELDS}


def gpu_grad(r, gp, cam, tau_R, dL, tile=(16, 16), bg=(0, 0, 0), shrink=None, warp_w=8):
    """update_params -> render -> backward; host numpy results."""
    import torch
    r.set_params(tau_R=tau_R, tile=tile, bg=bg, blend_warp_w=warp_w)
    r.set_camera(cam)
    r.shrink(*shrink) if shrink else r.shrink(None)
    P = dev_params(gp)
    r.update_params(P)
    rgb, T, st = r.render(stats=True, keep=True)
    G = r.backward(torch.from_numpy(np.ascontiguousarray(dL, np.float32)).cuda(), P)
    torch.cuda.synchronize()
    keys, vals = r.pairs()
    out = dict(rgb=rgb.cpu().numpy(), T=T.cpu().numpy(), keys=keys, vals=vals, splat=r.splats(),
               M=int(st.n_selected), NP=int(st.n_pairs),
               grads={k: v.cpu().numpy() for k, v in G.items()}, P=P)
    out["sel"] = r.filter()
    return out


def oracle_params(tau_R, tile=(16, 16), bg=(0, 0, 0), shrink=None):
    p = oracle.Params(tau_R=tau_R, tile_w=tile[0], tile_h=tile[1], bg=tuple(bg))
    if shrink:
        p.shrink, p.tau, p.ln_tau = True, shrink[0], shrink[1]
    return p


def assert_grad_parity(g, of, n_nodes):
    sel = of.frame.sel
    outside = np.ones(n_nodes, bool)
    outside[sel] = False
    worst = {}
    for k in oracle.GRAD_FIELDS:
        a = g["grads"][k].astype(np.float64)
        o = of.grads[k]
        scale = np.abs(o).max()
        err = np.abs(a - o).max()
        worst[k] = err / max(scale, 1e-30)
        assert err <= GRAD_RTOL * scale + 1e-7, (k, err, scale)
        node_axis = 0 if k == "sh" else -1
        zero = np.take(a, np.nonzero(outside)[0], axis=node_axis)
        assert not zero.any(), f"{k}: gradient outside the cut"
    return worst


def grad_parity_case(r, tree, cam, tau_R, seed, tile=(16, 16), bg=(0.2, 0.1, 0.4), shrink=None,
                     warp_w=8, pix=None):
    """The tree's own parameters through the GPU and the oracle; dL/drgb ~ N(0, 1)
    (only at ``pix`` when given).  Whole frames: the frame bit for bit; with
    ``pix``: selection and pairs bit for bit.  Then the gradients."""
    gp = oracle.GaussParams.of_tree(tree)
    rng = np.random.default_rng(seed)
    dL = rng.normal(size=(3, cam.height, cam.width)).astype(np.float32)
    if pix is not None:
        mask = np.zeros(cam.height * cam.width, bool)
        mask[pix] = True
        dL = dL * mask.reshape(cam.height, cam.width)
    r.load_tree(tree)
    g = gpu_grad(r, gp, cam, tau_R, dL, tile, bg, shrink, warp_w)
    p = oracle_params(tau_R, tile, bg, shrink)
    of = oracle.grad_frame(tree, gp, cam, p, dL, pix=pix)
    if pix is None:
        of_fr = oracle.frame(oracle.tree_with_params(tree, gp), cam, p)
        assert_frame_parity(g, of_fr)
    else:
        assert np.array_equal(g["sel"], of.frame.sel)
        assert g["NP"] == len(of.frame.keys)
        assert np.array_equal(g["keys"], of.frame.keys) and np.array_equal(g["vals"], of.frame.vals)
    return g, of, assert_grad_parity(g, of, tree.n)

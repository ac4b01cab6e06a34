"""Pins of the oracle's differentiable form (binary64 gradient with the cut,
the pairs and the blending decisions frozen).

The analytic gradient is checked against central finite differences of the
frozen binary64 forward (h = 1e-4), against closed forms (one Gaussian and two
stacked Gaussians at a pixel centre, Eq. 2), and against invariants of the
parametrisation (quaternion scale, isotropy, the DC-coefficient sum).  The
frozen forward is checked against the decision-exact oracle render, and the
binary32 parameter map against library routines."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_23891_gb300 import synth

Y00 = 0.5 / math.sqrt(math.pi)


def _setup(tree, cam, tau_R=0.0, bg=(0.2, 0.1, 0.4), tile=(16, 16), seed=1, pix=None):
    gp = oracle.GaussParams.of_tree(tree)
    p = oracle.Params(tau_R=tau_R, tile_w=tile[0], tile_h=tile[1], bg=bg)
    dL = np.random.default_rng(seed).normal(size=(3, cam.height, cam.width))
    gf = oracle.grad_frame(tree, gp, cam, p, dL, pix=pix)
    return gp, p, dL, gf


def _fd_check(gp, p, cam, gf, dL, n_per_group=None, h=1e-4, seed=0):
    """Central differences of the frozen forward for (a sample of) every parameter."""
    g64 = gp.astype(np.float64)
    w = np.asarray(dL, np.float64).reshape(3, -1)[:, gf.pix].T

    def loss():
        return float((oracle.diff_render(g64, gf.frame.sel, cam, p.bg, gf.pix, gf.offs,
                                         gf.ent) * w).sum())

    rng = np.random.default_rng(seed)
    rel = {}
    for key in oracle.GRAD_FIELDS:
        arr = getattr(g64, key)
        an = gf.grads[key]
        flat = np.arange(arr.size)
        if n_per_group is not None and arr.size > n_per_group:
            flat = rng.choice(arr.size, n_per_group, replace=False)
        worst = 0.0
        for i in flat:
            ix = np.unravel_index(i, arr.shape)
            old = arr[ix]
            arr[ix] = old + h
            lp = loss()
            arr[ix] = old - h
            lm = loss()
            arr[ix] = old
            worst = max(worst, abs((lp - lm) / (2 * h) - an[ix]))
        scale = max(np.abs(an).max(), 1e-12)
        rel[key] = worst / scale
    return rel


def test_lnf_matches_log():
    x = np.concatenate([np.float32(1.0) + np.float32(2.0 ** -23) * np.arange(1, 64),
                        np.logspace(-30, 30, 2001).astype(np.float32),
                        np.float32(1.0) + np.exp(-np.linspace(0, 80, 200)).astype(np.float32)])
    got = oracle.lnf(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    err = np.abs(got - ref)
    assert (err <= 4 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) + 1e-7).all()
    assert oracle.lnf([1.0])[0] == 0.0


def test_prep_params_matches_library_routines():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    tree = synth.random_small_tree(3, n_leaves=200, sh_degree=1)
    gp = oracle.GaussParams.of_tree(tree)
    gp.quat = gp.quat * np.float32(1.7)                  # any norm
    gp.logit = np.concatenate([gp.logit[:-2], np.float32([90.0, -95.0])])
    cov, op, lop = oracle.prep_params(gp)
    q = gp.quat.astype(np.float64).T                     # (n, 4) w x y z
    R = Rot.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    s2 = np.exp(2.0 * gp.log_scale.astype(np.float64).T)
    S = np.einsum("nik,nk,njk->nij", R, s2, R)
    ref = np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]])
    scale = s2.max(axis=1)
    assert (np.abs(cov - ref) <= 2e-6 * scale).all()
    l = np.clip(gp.logit.astype(np.float64), -80.0, 80.0)
    np.testing.assert_allclose(op, 1.0 / (1.0 + np.exp(-l)), rtol=4e-7)
    np.testing.assert_allclose(lop, -np.log1p(np.exp(-l)), rtol=2e-6, atol=2e-7)


def test_frozen_forward_equals_oracle_render():
    tree, cam = synth.grad_scene(0)
    gp, p, _, gf = _setup(tree, cam)
    fr = oracle.frame(oracle.tree_with_params(tree, gp), cam, p)
    assert len(gf.ent) > 4 * cam.width * cam.height     # several layers per pixel
    assert np.abs(fr.rgb.reshape(3, -1).T - gf.rgb).max() < 1e-6


@pytest.mark.parametrize("seed,deg", [(4, 3), (0, 3), (1, 1)])
def test_gradient_matches_finite_differences(seed, deg):
    """64 Gaussians at 32x32, every parameter group (SH sampled); seed 4 is the
    differentiable configuration's finite-difference scene."""
    tree, cam = synth.grad_scene(seed, sh_degree=deg)
    gp, p, dL, gf = _setup(tree, cam, seed=seed + 10)
    rel = _fd_check(gp, p, cam, gf, dL, n_per_group=256)
    for key, r in rel.items():
        assert r < 1e-6, (key, r)


def test_gradient_fd_multilevel_cut_ragged_tiles():
    """A cut with internal nodes (R&L on a 3-level tree), 40x24 image, 16x16 and 32x8
    tiles (ragged last row/column)."""
    tree = synth.random_small_tree(7, n_leaves=96, branching=(3, 5), sh_degree=2, extent=5.0,
                                   log_scale_mean=-0.8)
    cam = synth.look_at_camera([0.0, -14.0, 6.0], [0.0, 0.0, 0.0], 40, 24, 60.0)
    for tile in ((16, 16), (32, 8)):
        gp, p, dL, gf = _setup(tree, cam, tau_R=6.0, tile=tile)
        sel = gf.frame.sel
        assert (tree.is_leaf[sel] == 0).any() and (tree.is_leaf[sel] == 1).any()
        rel = _fd_check(gp, p, cam, gf, dL, n_per_group=200)
        for key, r in rel.items():
            assert r < 1e-6, (tile, key, r)


def _axis_camera(width=33, height=33):
    # looks along +y from (0, -10, 0): a node at the origin projects to (16.5, 16.5)
    return synth.look_at_camera([0.0, -10.0, 0.0], [0.0, 0.0, 0.0], width, height, 60.0)


def _node_of(tree, xyz):
    d = np.abs(tree.mu.T - np.float32(xyz)).sum(axis=1)
    return int(np.argmin(d))


def test_single_gaussian_at_pixel_centre_closed_form():
    """C = c alpha + bg (1 - alpha) with alpha = sigmoid(l) at the centre (power 0):
    dL/dl = w.(c - bg) alpha (1 - alpha), dL/dsh_0 = w alpha Y00, zero for the mean,
    scale and rotation (power is stationary at the centre; SH degree 0)."""
    tree = synth.tree_from_gaussians([[0.0, 0.0, 0.0]], [[-1.0, -1.2, -0.8]],
                                     [[0.9, 0.1, -0.3, 0.2]], [0.4], [[[0.7, -0.2, 0.3]]], 0)
    cam = _axis_camera()
    pix = np.array([16 * 33 + 16])
    bg = (0.2, 0.1, 0.4)
    gp, p, dL, gf = _setup(tree, cam, bg=bg, pix=pix)
    w = dL.reshape(3, -1)[:, pix[0]]
    a = 1.0 / (1.0 + math.exp(-float(np.float32(0.4))))
    c = 0.5 + Y00 * gp.sh[0, 0].astype(np.float64)
    g = gf.grads
    assert g["logit"][0] == pytest.approx(float((w * (c - np.array(bg))).sum()) * a * (1 - a),
                                          rel=1e-12)
    np.testing.assert_allclose(g["sh"][0, 0], w * a * Y00, rtol=1e-12)
    for key in ("mu", "log_scale", "quat"):
        assert np.abs(g[key]).max() < 1e-12, key


def test_two_stacked_gaussians_closed_form():
    """Two Gaussians on the optical axis (depths 10 and 12) seen at the centre pixel:
    C = c1 a1 + c2 a2 (1 - a1) + bg (1 - a1)(1 - a2)."""
    tree = synth.tree_from_gaussians([[0.0, 0.0, 0.0], [0.0, 2.0, 0.0]],
                                     [[-1.0, -1.0, -1.0], [-0.7, -0.9, -1.1]],
                                     [[1.0, 0.0, 0.0, 0.0], [0.5, 0.5, 0.5, 0.5]], [0.3, -0.2],
                                     [[[0.7, -0.2, 0.3]], [[-0.4, 0.9, 0.1]]], 0)
    cam = _axis_camera()
    pix = np.array([16 * 33 + 16])
    bg = np.array([0.2, 0.1, 0.4])
    gp, p, dL, gf = _setup(tree, cam, bg=tuple(bg), pix=pix)
    n1, n2 = _node_of(tree, [0, 0, 0]), _node_of(tree, [0, 2, 0])
    assert set(gf.frame.sel.tolist()) == {n1, n2}
    w = dL.reshape(3, -1)[:, pix[0]]
    sig = lambda l: 1.0 / (1.0 + math.exp(-float(l)))
    a1, a2 = sig(gp.logit[n1]), sig(gp.logit[n2])
    c1 = 0.5 + Y00 * gp.sh[n1, 0].astype(np.float64)
    c2 = 0.5 + Y00 * gp.sh[n2, 0].astype(np.float64)
    g = gf.grads
    assert g["logit"][n1] == pytest.approx(
        float((w * (c1 - c2 * a2 - bg * (1 - a2))).sum()) * a1 * (1 - a1), rel=1e-12)
    assert g["logit"][n2] == pytest.approx(
        float((w * (c2 - bg)).sum()) * (1 - a1) * a2 * (1 - a2), rel=1e-12)
    np.testing.assert_allclose(g["sh"][n1, 0], w * a1 * Y00, rtol=1e-12)
    np.testing.assert_allclose(g["sh"][n2, 0], w * a2 * (1 - a1) * Y00, rtol=1e-12)


def test_quaternion_invariances():
    """R(q / |q|) does not depend on |q|: q . dL/dq = 0 and scaling q by k scales
    dL/dq by 1/k; an isotropic Gaussian does not depend on q at all."""
    tree, cam = synth.grad_scene(2, sh_degree=0)
    gp, p, dL, gf = _setup(tree, cam)
    gq = gf.grads["quat"]
    q = gp.quat.astype(np.float64)
    dots = (gq * q).sum(axis=0)
    assert np.abs(dots).max() < 1e-12 * max(1.0, np.abs(gq).max())
    gp2 = oracle.GaussParams(gp.mu, gp.log_scale, gp.quat * np.float32(2.0), gp.logit, gp.sh,
                             gp.sh_degree)
    g2 = oracle.diff_grad(gp2, gf.frame.sel, cam, p.bg, gf.pix, gf.offs, gf.ent,
                          dL.reshape(3, -1)[:, gf.pix].T)
    np.testing.assert_allclose(g2["quat"], 0.5 * gq, rtol=1e-9, atol=1e-14)
    iso = oracle.GaussParams(gp.mu, np.repeat(gp.log_scale[:1], 3, axis=0), gp.quat, gp.logit,
                             gp.sh, gp.sh_degree)
    g3 = oracle.diff_grad(iso, gf.frame.sel, cam, p.bg, gf.pix, gf.offs, gf.ent,
                          dL.reshape(3, -1)[:, gf.pix].T)
    assert np.abs(g3["quat"]).max() < 1e-12


def test_dc_gradient_sum_equals_coverage():
    """With no colour clamp, sum over Gaussians of dL/dsh_DC = Y00 sum_p w_p (1 - T_p)
    (the alpha T weights of Eq. 2 sum to 1 - T_final); T from the decision-exact render."""
    tree, cam = synth.grad_scene(3, sh_degree=2)
    gp, p, dL, gf = _setup(tree, cam)
    fr = oracle.frame(oracle.tree_with_params(tree, gp), cam, p)
    cover = 1.0 - fr.T.astype(np.float64).reshape(-1)
    expect = Y00 * (dL.reshape(3, -1) * cover).sum(axis=1)
    got = gf.grads["sh"][:, 0, :].sum(axis=0)
    np.testing.assert_allclose(got, expect, rtol=1e-5)

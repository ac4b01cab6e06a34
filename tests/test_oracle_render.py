"""Pins of the oracle's projection, pairs, blending (Eq. 2), KPC/GTC (Eq. 5-8) on the CPU."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_23891_gb300 import synth

C0 = 0.5 / math.sqrt(math.pi)


# ---------------------------------------------------------------- exp

def test_expf_against_libm():
    """Cody-Waite + degree-7 Taylor exp with fused multiply-adds: within 1 ulp of
    e^x over the whole range the blend and the parameter map use, exact at 0,
    0 below -87 and infinite above 88."""
    x = np.concatenate([np.linspace(-87.0, 88.0, 40001, dtype=np.float32),
                        -np.float32(np.log(2.0)) * np.arange(0, 30, dtype=np.float32)])
    got = oracle.expf(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    err = np.abs(got - ref) / ulp
    assert err.max() <= 1.0
    assert err.mean() < 0.3
    assert oracle.expf([0.0])[0] == 1.0
    assert oracle.expf([-87.5])[0] == 0.0 and np.isinf(oracle.expf([88.5])[0])


# ---------------------------------------------------------------- SH

def _real_sh_scipy(deg, d):
    from scipy.special import sph_harm_y
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    out = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                out.append(math.sqrt(2) * Y.real)
            elif m < 0:
                out.append(math.sqrt(2) * Y.imag)
            else:
                out.append(Y.real)
    return np.array(out)


def test_sh_basis_matches_scipy_real_sh():
    """Real SH with the Condon-Shortley phase built from scipy's complex Y_l^m."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        np.testing.assert_allclose(oracle.sh_basis(3, d), _real_sh_scipy(3, d), atol=1e-12)


def test_sh_basis_orthonormal():
    """Monte-Carlo check of orthonormality on the sphere: integral Y_i Y_j = delta_ij."""
    rng = np.random.default_rng(1)
    d = rng.normal(size=(40000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    B = np.stack([oracle.sh_basis(3, x) for x in d])
    G = 4 * math.pi * B.T @ B / d.shape[0]
    np.testing.assert_allclose(G, np.eye(16), atol=0.05)


# ---------------------------------------------------------------- projection + pairs

@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_tree(), synth.tiny_camera()


def test_degree0_colour(tiny):
    """Degree 0: colour = C0 * dc + 0.5, the generator's uniform base colour."""
    tree, cam = tiny
    sel = oracle.filter_dfs(tree, cam, 1.0)
    splat, rect, _ = oracle.project(tree, cam, oracle.Params(tau_R=1.0), sel)
    expect = C0 * tree.sh[sel, 0, :].astype(np.float64) + 0.5
    np.testing.assert_allclose(splat[:, 8:11], np.maximum(expect, 0), atol=1e-6)


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 32)])
@pytest.mark.parametrize("tau_R", [1.0, 3.0, 12.0])
def test_pair_count_bruteforce(tiny, tile, tau_R):
    """Analytic rectangles give exactly the tiles a brute-force overlap test finds."""
    tree, cam = tiny
    for shrink, tau in [(False, 0.0), (True, 0.05), (True, 0.3)]:
        p = oracle.Params(tau_R=tau_R, tile_w=tile[0], tile_h=tile[1], shrink=shrink,
                          tau=tau, ln_tau=float(np.float32(math.log(tau))) if tau else -math.inf)
        sel = oracle.filter_dfs(tree, cam, tau_R)
        splat, rect, n = oracle.project(tree, cam, p, sel)
        assert n == oracle.count_pairs_bruteforce(splat, rect, cam, p)
        keys, vals = oracle.pairs(splat, rect, cam, p)
        assert keys.shape[0] == n
        k = np.stack([keys >> np.uint64(32), keys & np.uint64(0xFFFFFFFF), vals.astype(np.uint64)], 1)
        assert np.all(np.diff(keys.astype(np.float64)) >= 0)
        # depth bits in the key are the splat depth of the value
        d = splat[vals, 7].view(np.uint32).astype(np.uint64)
        assert np.array_equal(k[:, 1], d)


def test_shrink_limits_and_monotonicity(tiny):
    """tau -> 0+ reproduces the 3-sigma pairs bit for bit; N_P never rises with tau;
    tau = 1/255 never gives more pairs than 3 sigma; alpha0 <= tau emits nothing."""
    tree, cam = tiny
    sel = oracle.filter_dfs(tree, cam, 3.0)
    base = oracle.Params(tau_R=3.0)
    s0, r0, n0 = oracle.project(tree, cam, base, sel)
    k0, v0 = oracle.pairs(s0, r0, cam, base)
    tiny_tau = oracle.Params(tau_R=3.0, shrink=True, tau=1e-30, ln_tau=float(np.float32(math.log(1e-30))))
    s1, r1, n1 = oracle.project(tree, cam, tiny_tau, sel)
    k1, v1 = oracle.pairs(s1, r1, cam, tiny_tau)
    assert np.array_equal(k0, k1) and np.array_equal(v0, v1)
    prev = n0
    for tau in [1 / 255, 0.01, 0.03, 0.1, 0.2, 0.5, 0.9]:
        p = oracle.Params(tau_R=3.0, shrink=True, tau=tau, ln_tau=float(np.float32(math.log(tau))))
        s, r, n = oracle.project(tree, cam, p, sel)
        assert n <= prev
        prev = n
        if tau == 1 / 255:
            assert n <= n0
        a0 = tree.opacity[sel]
        dead = tree.ln_opacity[sel] <= np.float32(p.ln_tau)
        assert np.all((r[dead, 1] - r[dead, 0]) * (r[dead, 3] - r[dead, 2]) == 0)
        del a0


def test_shrink_radius_closed_form():
    """Shrunk radius: alpha0 exp(-r^2 / (2 lambda_max)) = tau when below the 3-sigma cap."""
    cam = synth.look_at_camera([0, 0, 0], [0, 1, 0], 256, 256, 60.0)
    for logit in (2.0, 0.0, -1.0):
        t = synth.tree_from_gaussians(np.array([[0.0, 10.0, 0.0]]), np.array([[-1.0, -1.0, -1.0]]),
                                      np.array([[1.0, 0, 0, 0]]), np.array([logit]),
                                      np.zeros((1, 1, 3)), 0)
        a0 = float(t.opacity[0])
        for tau in (0.05, 0.1, 0.2):
            p = oracle.Params(tau_R=-1.0, shrink=True, tau=tau, ln_tau=float(np.float32(math.log(tau))))
            splat, rect, n = oracle.project(t, cam, p, np.array([0], np.uint32))
            s = math.exp(-1.0)
            lam = (cam.fx * s / 10.0) ** 2 + 0.3 + math.sqrt(0.1)
            if a0 <= tau:
                assert n == 0
                continue
            r2 = min(9.0, 2 * math.log(a0 / tau)) * lam
            assert splat[0, 11] == pytest.approx(math.sqrt(r2), rel=1e-4)


# ---------------------------------------------------------------- blending

def _flat_scene(mu, logs, logit, rgb, cam_pos=(0, 0, 0), target=(0, 1, 0), size=(64, 64), fov=60.0):
    n = len(mu)
    sh = ((np.asarray(rgb, np.float64) - 0.5) / C0).reshape(n, 1, 3)
    q = np.tile([1.0, 0, 0, 0], (n, 1))
    t = synth.tree_from_gaussians(np.asarray(mu, float), np.asarray(logs, float), q,
                                  np.asarray(logit, float), sh, 0)
    cam = synth.look_at_camera(cam_pos, target, size[0], size[1], fov)
    return t, cam


def test_single_isotropic_gaussian_closed_form():
    """One isotropic Gaussian on the optical axis: pixel colour = c * min(0.99, a0 e^{-d^2/(2 s^2)})
    with s^2 = (f s_w / z)^2 + 0.3 wherever alpha >= 1/255 and the tile is in the 3-sigma box."""
    t, cam = _flat_scene([[0.0, 10.0, 0.0]], [[-1.2] * 3], [0.8], [[0.9, 0.4, 0.2]], size=(64, 64))
    p = oracle.Params(tau_R=-1.0)
    fr = oracle.frame(t, cam, p)
    assert fr.sel.shape[0] == 1
    a0 = float(t.opacity[fr.sel[0]])
    s2 = (cam.fx * math.exp(-1.2) / 10.0) ** 2 + 0.3
    colour = np.array([0.9, 0.4, 0.2])
    rect = fr.rect[0]
    checked = 0
    for y in range(64):
        for x in range(64):
            tx, ty = x // 16, y // 16
            d2 = (x + 0.5 - 32.0) ** 2 + (y + 0.5 - 32.0) ** 2
            a = a0 * math.exp(-0.5 * d2 / s2)
            inside = rect[0] <= tx < rect[1] and rect[2] <= ty < rect[3]
            if not inside or a < 1 / 255 * (1 - 1e-4):
                assert np.all(fr.rgb[:, y, x] == 0.0) and fr.T[y, x] == 1.0
                continue
            if a < 1 / 255 * (1 + 1e-4):
                continue
            a = min(0.99, a)
            np.testing.assert_allclose(fr.rgb[:, y, x], colour * a, rtol=2e-5, atol=1e-7)
            assert fr.T[y, x] == pytest.approx(1 - a, rel=1e-5)
            checked += 1
    assert checked > 50


def test_two_gaussians_front_to_back():
    """Two overlapping Gaussians: C = c1 a1 + c2 a2 (1 - a1) with the nearer one first,
    whatever their ids."""
    for order in ([0, 1], [1, 0]):
        mus = [[0.0, 10.0, 0.0], [0.0, 12.0, 0.0]]
        cols = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]
        mus = [mus[i] for i in order]
        cols = [cols[i] for i in order]
        t, cam = _flat_scene(mus, [[-1.0] * 3, [-0.6] * 3], [0.5, 1.5], cols)
        fr = oracle.frame(t, cam, oracle.Params(tau_R=-1.0))
        y = x = 32
        # pixel centre (32.5, 32.5) is half a pixel off the principal point (32, 32)
        d2 = 0.5
        out = []
        for m in range(2):
            n = fr.sel[m]
            depth = fr.splat[m, 7]
            s_w = math.exp(float(t.log_scale[0, n]))
            s2 = (cam.fx * s_w / depth) ** 2 + 0.3
            a = min(0.99, float(t.opacity[n]) * math.exp(-0.5 * d2 / s2))
            out.append((depth, a, fr.splat[m, 8:11].astype(np.float64)))
        out.sort(key=lambda z: z[0])
        (_, a1, c1), (_, a2, c2) = out
        np.testing.assert_allclose(fr.rgb[:, y, x], c1 * a1 + c2 * a2 * (1 - a1), rtol=1e-5)
        assert fr.T[y, x] == pytest.approx((1 - a1) * (1 - a2), rel=1e-5)


def test_white_gaussians_colour_equals_opacity_and_stop_rule():
    """White Gaussians: C = 1 - T_final exactly (telescoping sum of Eq. 2), T never below 1e-4,
    and the sum of KPC over all pairs = sum over pixels of (1 - T_final)."""
    rng = np.random.default_rng(7)
    n = 60
    mu = np.stack([rng.uniform(-1, 1, n), rng.uniform(8, 12, n), rng.uniform(-1, 1, n)], 1)
    t, cam = _flat_scene(mu, rng.normal(-1.0, 0.3, (n, 3)), rng.normal(3.0, 1.0, n),
                         np.ones((n, 3)), size=(64, 48))
    p = oracle.Params(tau_R=-1.0)
    fr = oracle.frame(t, cam, p, want_kpc=True)
    assert fr.T.min() >= 1e-4
    assert (fr.T < 0.01).sum() > 50          # the stop rule was exercised
    np.testing.assert_allclose(fr.rgb[0], 1.0 - fr.T.astype(np.float64), atol=2e-6)
    assert fr.kpc.sum() == pytest.approx((1.0 - fr.T.astype(np.float64)).sum(), rel=1e-6)


GUARD = 1e-4      # relative guard band around the skip and stop thresholds


def _python_blend(splat, rect, cam, p):
    """Independent float64 restatement of Eq. 2 with the 3DGS rules, per pixel.

    It does not read the oracle's pair list: a pixel's Gaussians are those whose
    footprint rectangle (x0, x1, y0, y1 in tiles) holds the pixel's tile, ordered
    by (depth, rank).  Returns the colour (with T * bg), the final T, the number
    of Gaussians added, and a flag for pixels where a skip or stop decision lies
    within the relative guard band GUARD of its threshold (binary32 rounding on
    the oracle's side may take the other branch there)."""
    W, H = cam.width, cam.height
    M = splat.shape[0]
    order = sorted(range(M), key=lambda m: (float(splat[m, 7]), m))
    tx_n = (W + p.tile_w - 1) // p.tile_w
    ty_n = (H + p.tile_h - 1) // p.tile_h
    lists = {}
    for ty in range(ty_n):
        for tx in range(tx_n):
            lists[(tx, ty)] = [m for m in order if rect[m, 0] <= tx < rect[m, 1]
                               and rect[m, 2] <= ty < rect[m, 3]]
    bg = np.asarray(p.bg, np.float64)
    rgb = np.zeros((3, H, W))
    T_out = np.ones((H, W))
    n_out = np.zeros((H, W), np.int64)
    near = np.zeros((H, W), bool)
    for y in range(H):
        for x in range(W):
            T, acc, n, close = 1.0, np.zeros(3), 0, False
            for m in lists[(x // p.tile_w, y // p.tile_h)]:
                s = splat[m].astype(np.float64)
                dx, dy = s[0] - (x + 0.5), s[1] - (y + 0.5)
                power = -0.5 * (s[2] * dx * dx + s[4] * dy * dy) - s[3] * dx * dy
                if abs(power) <= GUARD:
                    close = True
                if power > 0:
                    continue
                a = min(0.99, s[6] * math.exp(power))
                if abs(a * 255.0 - 1.0) <= GUARD:
                    close = True
                if a < 1 / 255:
                    continue
                Tn = T * (1 - a)
                if abs(Tn * 1e4 - 1.0) <= GUARD:
                    close = True
                if Tn < 1e-4:
                    break
                acc += s[8:11] * a * T
                T = Tn
                n += 1
            rgb[:, y, x] = acc + T * bg
            T_out[y, x] = T
            n_out[y, x] = n
            near[y, x] = close
    return rgb, T_out, n_out, near


def _restatement_case(seed, tile, shrink, bg, dense):
    n_leaves, pos, ls = (300, [0, -9, 4], -0.8) if dense else (90, [0, -12, 5], -1.0)
    tree = synth.random_small_tree(seed, n_leaves=n_leaves, branching=(2, 4), log_scale_mean=ls,
                                   extent=3.0, sh_degree=1)
    cam = synth.look_at_camera(pos, [0, 0, 0], 70, 44, 60.0)
    p = oracle.Params(tau_R=3.0, tile_w=tile[0], tile_h=tile[1], bg=bg)
    if shrink:
        p.shrink, p.tau, p.ln_tau = True, 0.05, float(np.float32(math.log(0.05)))
    fr = oracle.frame(tree, cam, p)
    return fr, cam, p


@pytest.mark.parametrize("seed,tile,shrink,bg,dense", [
    (0, (16, 16), False, (0.0, 0.0, 0.0), True), (1, (32, 8), False, (0.2, 0.5, 0.9), True),
    (2, (16, 16), True, (0.0, 0.0, 0.0), False), (3, (8, 32), True, (1.0, 0.0, 0.3), False),
    (4, (64, 4), True, (0.3, 0.3, 0.3), True)])
def test_blend_matches_independent_float64_restatement(seed, tile, shrink, bg, dense):
    """Every pixel of tiny scenes (70x44: ragged tiles in x and y; the dense ones layer
    enough Gaussians for the stop rule to end hundreds of pixels) against an independent
    float64 blend that builds each pixel's list from the footprint rectangles, not from
    the oracle's pairs.  Pixels with a skip or stop decision within the guard band are
    counted (and must be rare); every other pixel has the same number of Gaussians added
    as the oracle's contributor trace, colour within 1e-5 and T within 1e-5 relative."""
    fr, cam, p = _restatement_case(seed, tile, shrink, bg, dense)
    rgb, T, n_add, near = _python_blend(fr.splat, fr.rect, cam, p)
    W, H = cam.width, cam.height
    pix = np.arange(W * H, dtype=np.int64)
    offs, _ = oracle.trace_pixels(fr.splat, fr.keys, fr.vals, cam, p, pix)
    n_oracle = np.diff(offs).reshape(H, W)
    assert n_oracle.max() >= 3, "the scene must layer Gaussians"
    if dense:
        assert (fr.T < 1e-3).sum() > 100, "the stop rule must be exercised"
    n_near = int(near.sum())
    print(f"seed {seed}: {n_near} of {W * H} pixels within the guard band")
    assert n_near <= 0.01 * W * H
    ok = ~near
    assert np.array_equal(n_add[ok], n_oracle[ok]), \
        f"contributor counts differ at {np.count_nonzero(n_add[ok] != n_oracle[ok])} pixels"
    err = np.abs(rgb - fr.rgb).max(axis=0)
    assert err[ok].max() <= 1e-5, f"max colour error {err[ok].max()} at {np.argwhere(ok & (err > 1e-5))[:5]}"
    np.testing.assert_allclose(fr.T.astype(np.float64)[ok], T[ok], rtol=1e-5, atol=0)


# ---------------------------------------------------------------- KPC / GTC

def test_kpc_single_and_stacked():
    """Eq. 5: one Gaussian alone -> KPC = sum_p alpha_p over its tile; a second one behind it
    -> KPC_2 = sum_p alpha2 (1 - alpha1).  Eq. 6-7 on one tile."""
    t, cam = _flat_scene([[0.0, 10.0, 0.0]], [[-2.0] * 3], [1.0], [[1, 1, 1]], size=(16, 16))
    fr = oracle.frame(t, cam, oracle.Params(tau_R=-1.0), want_kpc=True)
    assert fr.keys.shape[0] == 1
    assert fr.kpc[0] == pytest.approx(float((1.0 - fr.T.astype(np.float64)).sum()), rel=1e-6)
    G, gbar, used = oracle.gtc(fr.keys, fr.kpc, 1)
    assert used == 1 and gbar == pytest.approx(fr.kpc[0])

    t, cam = _flat_scene([[0.0, 10.0, 0.0], [0.0, 11.0, 0.0]], [[-2.0] * 3, [-1.9] * 3], [1.0, 0.5],
                         [[1, 1, 1], [1, 1, 1]], size=(16, 16))
    fr = oracle.frame(t, cam, oracle.Params(tau_R=-1.0), want_kpc=True)
    assert fr.keys.shape[0] == 2
    # alpha of each Gaussian at each pixel, front one first
    alphas = []
    for q in range(2):
        s = fr.splat[fr.vals[q]].astype(np.float64)
        a = np.zeros((16, 16))
        for y in range(16):
            for x in range(16):
                dx, dy = s[0] - (x + 0.5), s[1] - (y + 0.5)
                pw = -0.5 * (s[2] * dx * dx + s[4] * dy * dy) - s[3] * dx * dy
                v = min(0.99, s[6] * math.exp(pw))
                a[y, x] = v if v >= 1 / 255 else 0.0
        alphas.append(a)
    assert fr.kpc[0] == pytest.approx(alphas[0].sum(), rel=1e-5)
    assert fr.kpc[1] == pytest.approx((alphas[1] * (1 - alphas[0])).sum(), rel=1e-5)
    G, gbar, used = oracle.gtc(fr.keys, fr.kpc, 1)
    assert G[0] == pytest.approx(fr.kpc.mean())


def test_gtc_skips_empty_tiles_and_tau():
    """Eq. 7 averages over tiles that have pairs; Eq. 8: tau = lambda_G / mean of view GTCs."""
    keys = np.array([(0 << 32) | 5, (0 << 32) | 6, (3 << 32) | 1], np.uint64)
    kpc = np.array([1.0, 3.0, 0.5])
    G, gbar, used = oracle.gtc(keys, kpc, 4)
    assert used == 2 and G[0] == 2.0 and G[3] == 0.5 and np.isnan(G[1])
    assert gbar == pytest.approx(1.25)
    tau, ln_tau = oracle.tau_from([1.0, 3.0], 0.2)
    assert tau == pytest.approx(0.1, rel=1e-7) and ln_tau == pytest.approx(math.log(0.1), rel=1e-7)

"""Pins of the oracle's §3.2 filter against structure and closed forms (CPU)."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_23891_gb300 import synth


def _cams_for(tree, n=4, seed=0, size=(96, 64)):
    rng = np.random.default_rng(seed)
    cams = []
    c = tree.mu.mean(axis=1)
    for _ in range(n):
        a = rng.uniform(0, 2 * math.pi)
        dist = rng.uniform(6.0, 40.0)
        h = rng.uniform(2.0, 20.0)
        pos = [c[0] + dist * math.cos(a), c[1] + dist * math.sin(a), c[2] + h]
        tgt = c + rng.normal(0, 2.0, size=3)
        cams.append(synth.look_at_camera(pos, tgt, size[0], size[1], rng.uniform(30, 90)))
    return cams


def _ancestors(tree, n):
    out = []
    p = tree.parent[n]
    while p >= 0:
        out.append(int(p))
        p = tree.parent[p]
    return out


TAUS = [-1.0, 1.0, 3.0, 10.0, 40.0, 1e30]


@pytest.mark.parametrize("seed", range(6))
def test_dfs_equals_ancestor_set_definition(seed):
    """The traversal-free filter selects exactly the serial traversal's set (§3.2, Table 3)."""
    tree = synth.random_small_tree(seed, n_leaves=200, branching=(2, 5), log_scale_mean=-0.5)
    for cam in _cams_for(tree, seed=seed):
        for tau in TAUS:
            a = oracle.filter_dfs(tree, cam, tau)
            b = oracle.filter_setdef(tree, cam, tau)
            assert np.array_equal(a, b), (seed, tau)


@pytest.mark.parametrize("seed", range(4))
def test_cut_is_antichain_covering_in_frustum_leaves(seed):
    """Each branch keeps exactly one node: no selected node has a selected ancestor, and every
    in-frustum leaf has exactly one selected node on its root path (§3.2)."""
    tree = synth.random_small_tree(seed + 10, n_leaves=300, branching=(2, 6), log_scale_mean=-0.7)
    for cam in _cams_for(tree, seed=seed):
        for tau in TAUS:
            sel = oracle.filter_dfs(tree, cam, tau)
            S = set(int(x) for x in sel)
            for n in sel:
                assert not (set(_ancestors(tree, int(n))) & S)
            P, _ = oracle.predicate(tree, cam, tau)
            for leaf in np.nonzero(tree.is_leaf)[0]:
                path = [int(leaf)] + _ancestors(tree, int(leaf))
                k = sum(1 for x in path if x in S)
                if P[leaf]:
                    assert k == 1
                else:
                    assert k <= 1


def test_special_thresholds():
    """tau_R < 0: only leaves pass R&L, so the cut is every in-frustum leaf.
    tau_R = +inf: every in-frustum node passes, so the cut is the topmost in-frustum nodes."""
    tree = synth.random_small_tree(3, n_leaves=250, branching=(2, 4), log_scale_mean=-0.5)
    for cam in _cams_for(tree, seed=5):
        P_neg, R = oracle.predicate(tree, cam, -1.0)
        inf = ~np.isnan(R)
        sel = oracle.filter_dfs(tree, cam, -1.0)
        assert np.array_equal(sel, np.nonzero(inf & (tree.is_leaf == 1))[0])
        sel = oracle.filter_dfs(tree, cam, 1e30)
        top = [n for n in range(tree.n) if inf[n] and not any(inf[a] for a in _ancestors(tree, n))]
        assert np.array_equal(sel, np.array(top, dtype=np.uint32))


def test_ap_matches_parent_chain():
    tree = synth.random_small_tree(1, n_leaves=500, branching=(2, 8))
    for n in range(tree.n):
        anc = _ancestors(tree, n)
        row = [int(x) for x in tree.ap[:, n] if x != 0xFFFFFFFF]
        assert row == anc


def _one_gaussian_tree(pos, log_scale, quat=(1.0, 0, 0, 0)):
    return synth.tree_from_gaussians(np.array([pos]), np.array([log_scale]), np.array([quat]),
                                     np.array([0.0]), np.zeros((1, 1, 3)), 0)


def test_frustum_guard_band():
    """In-frustum = depth above 0.2 and centre within 1.3x the half-FOV tangents."""
    cam = synth.look_at_camera([0, 0, 0], [0, 1, 0], 200, 100, 60.0)  # looks along +y
    tx, ty = cam.tan_half_x, cam.tan_half_y
    cases = [((0, 10, 0), True), ((0, -10, 0), False), ((0, 0.1, 0), False),
             ((1.29 * tx * 10, 10, 0), True), ((1.31 * tx * 10, 10, 0), False),
             ((-1.29 * tx * 10, 10, 0), True), ((-1.31 * tx * 10, 10, 0), False),
             ((0, 10, -1.29 * ty * 10), True), ((0, 10, -1.31 * ty * 10), False),
             ((0, 10, 1.29 * ty * 10), True), ((0, 10, 1.31 * ty * 10), False)]
    for pos, inside in cases:
        t = _one_gaussian_tree(pos, (-3, -3, -3))
        P, R = oracle.predicate(t, cam, 3.0)
        assert bool(P[0]) == inside, pos
        assert np.isnan(R[0]) != inside


def test_radius_isotropic_on_axis():
    """Isotropic world std s at depth z on the optical axis: Sigma_2D = ((f s / z)^2 + 0.3) I.
    Both eigenvalues are equal, so the 3DGS discriminant floor of 0.1 applies:
    lambda_max = (f s / z)^2 + 0.3 + sqrt(0.1) and R_2D = 3 sqrt(lambda_max)."""
    cam = synth.look_at_camera([0, 0, 0], [0, 1, 0], 320, 240, 60.0)
    for z in (2.0, 7.5, 40.0):
        for ls in (-3.0, -1.0, 0.5):
            t = _one_gaussian_tree((0, z, 0), (ls, ls, ls))
            _, R = oracle.predicate(t, cam, 3.0)
            s = math.exp(ls)
            expect = 3 * math.sqrt((cam.fx * s / z) ** 2 + 0.3 + math.sqrt(0.1))
            assert R[0] == pytest.approx(expect, rel=2e-5)


def _numeric_jacobian(cam, v):
    """d(pixel)/d(camera-space point) by central differences of the pinhole map, float64."""
    def proj(q):
        return np.array([cam.fx * q[0] / q[2] + cam.cx, cam.fy * q[1] / q[2] + cam.cy])
    J = np.zeros((2, 3))
    h = 1e-6 * max(1.0, abs(v[2]))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (proj(v + e) - proj(v - e)) / (2 * h)
    return J


@pytest.mark.parametrize("seed", range(5))
def test_ewa_covariance_against_numeric_jacobian(seed):
    """Sigma_2D = J W Sigma W^T J^T + 0.3 I with J the Jacobian of the pinhole map at the
    centre (EWA splatting).  Checked through the oracle's conic (its inverse)."""
    rng = np.random.default_rng(seed)
    cam = synth.look_at_camera([0, -30, 10], [0, 0, 0], 256, 192, 70.0)
    mu = rng.uniform([-5, -5, -2], [5, 5, 2], size=(8, 3))
    logs = rng.normal(-0.5, 0.5, size=(8, 3))
    q = rng.normal(size=(8, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    tree = synth.tree_from_gaussians(mu, logs, q, np.zeros(8), np.zeros((8, 1, 3)), 0)
    leaves = np.nonzero(tree.is_leaf)[0].astype(np.uint32)
    p = oracle.Params(tau_R=-1.0)
    splat, rect, _ = oracle.project(tree, cam, p, leaves)
    R = cam.R.astype(np.float64)
    for m, n in enumerate(leaves):
        c6 = tree.cov[:, n].astype(np.float64)
        S = np.array([[c6[0], c6[1], c6[2]], [c6[1], c6[3], c6[4]], [c6[2], c6[4], c6[5]]])
        v = R @ tree.mu[:, n].astype(np.float64) + cam.t.astype(np.float64)
        J = _numeric_jacobian(cam, v)
        S2 = J @ R @ S @ R.T @ J.T + 0.3 * np.eye(2)
        A, B, Cc = splat[m, 2], splat[m, 3], splat[m, 4]
        got = np.linalg.inv(np.array([[A, B], [B, Cc]], dtype=np.float64))
        np.testing.assert_allclose(got, S2, rtol=2e-4, atol=1e-4 * np.abs(S2).max())
        u = cam.fx * v[0] / v[2] + cam.cx
        vv = cam.fy * v[1] / v[2] + cam.cy
        assert splat[m, 0] == pytest.approx(u, abs=2e-3)
        assert splat[m, 1] == pytest.approx(vv, abs=2e-3)
        assert splat[m, 7] == pytest.approx(v[2], rel=1e-6)
        mid = 0.5 * (S2[0, 0] + S2[1, 1])
        lam = mid + math.sqrt(max(0.1, mid * mid - np.linalg.det(S2)))
        assert splat[m, 11] == pytest.approx(3 * math.sqrt(lam), rel=1e-3)

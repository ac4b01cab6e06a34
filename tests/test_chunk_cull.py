"""The R&L filter's chunk frustum cull is exact for the per-node test (CPU, brute force).

R&L skips a chunk of 128 nodes when the box of their centres lies beyond one of the
five planes of the in-frustum condition (§3.2: depth above 0.2, |x / z| and |y / z|
within 1.3 times the half-FOV tangents), cleared by a margin of 1e-3 times the
magnitudes involved.  A skipped chunk's nodes are never tested, so no centre in
such a box may pass the per-node binary32 test.  This test restates the box-plane
test and the per-node test in numpy binary32, rounded as the kernel rounds them
(the planes and the margin with and without fused multiply-adds), and checks boxes
against the centres in them: random boxes around random cameras, and boxes whose
corner nearest the frustum lies on a side or near plane to within a relative
offset of 1e-6 on either side.  The latter give the test its power: the same cull
without its margin skips boxes holding centres that pass.
"""
import numpy as np
import pytest

f32 = np.float32


def fma(a, b, c):
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(f32)


def random_camera(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]).astype(f32)
    t = rng.uniform(-200, 200, 3).astype(f32)
    tan = rng.uniform(0.2, 1.5, 2).astype(f32)
    return R, t, tan


def node_passes(R, t, tan, P):
    """The per-node test: camera-space centre by products and sums rounded one at a
    time, depth above 0.2, x / z and y / z (IEEE quotients) within 1.3 tan."""
    mx, my, mz = P[:, 0], P[:, 1], P[:, 2]
    v = [((R[i, 0] * mx + R[i, 1] * my) + R[i, 2] * mz) + t[i] for i in range(3)]
    vx, vy, vz = v
    limx, limy = f32(1.3) * tan[0], f32(1.3) * tan[1]
    with np.errstate(divide="ignore", invalid="ignore"):
        tx, ty = vx / vz, vy / vz
    return (vz > f32(0.2)) & (tx >= -limx) & (tx <= limx) & (ty >= -limy) & (ty <= limy)


def planes(R, t, tan, fused):
    """The five planes n . p + d > 0 (outside), coefficients rounded plainly or with
    the product fused into the difference."""
    Lx, Ly = f32(1.3) * tan[0], f32(1.3) * tan[1]

    def comb(a, L, b):          # a - L b
        return fma(-L, b, a) if fused else a - L * b
    r0, r1, r2 = R[0], R[1], R[2]
    P = [
        [comb(r0[j], Lx, r2[j]) for j in range(3)] + [comb(t[0], Lx, t[2])],
        [comb(-r0[j], Lx, r2[j]) for j in range(3)] + [comb(-t[0], Lx, t[2])],
        [comb(r1[j], Ly, r2[j]) for j in range(3)] + [comb(t[1], Ly, t[2])],
        [comb(-r1[j], Ly, r2[j]) for j in range(3)] + [comb(-t[1], Ly, t[2])],
        [-r2[0], -r2[1], -r2[2], f32(0.2) - t[2]],
    ]
    scale = f32(1.0) + max(Lx, Ly)
    tt = (abs(t[0]) + abs(t[1])) + abs(t[2])
    return np.array(P, f32), scale, tt


def box_outside(Pl, scale, tt, lo, hi, fused_margin, margin_factor=f32(1e-3)):
    """The chunk test for boxes lo, hi [B, 3]: beyond some plane by the margin."""
    ax = np.maximum(np.abs(lo[:, 0]), np.abs(hi[:, 0]))
    ay = np.maximum(np.abs(lo[:, 1]), np.abs(hi[:, 1]))
    az = np.maximum(np.abs(lo[:, 2]), np.abs(hi[:, 2]))
    s = ((ax + ay) + az) + tt
    inner = fma(s, scale, f32(1.0)) if fused_margin else s * scale + f32(1.0)
    margin = margin_factor * inner
    out = np.zeros(len(lo), bool)
    for q in Pl:
        m = ((q[3] + np.minimum(q[0] * lo[:, 0], q[0] * hi[:, 0])) +
             np.minimum(q[1] * lo[:, 1], q[1] * hi[:, 1])) + np.minimum(q[2] * lo[:, 2], q[2] * hi[:, 2])
        out |= m > margin
    return out


def grazing_boxes(rng, R, t, tan, n):
    """Boxes whose corner nearest the frustum is a centre on one of the five planes,
    offset by a relative 1e-6 inwards or outwards, extending away from the frustum."""
    Lx, Ly = 1.3 * float(tan[0]), 1.3 * float(tan[1])
    k = rng.integers(0, 5, n)
    z = np.exp(rng.uniform(np.log(0.3), np.log(500.0), n))
    d = rng.uniform(-1e-6, 1e-6, n)
    x = rng.uniform(-0.9, 0.9, n) * Lx * z
    y = rng.uniform(-0.9, 0.9, n) * Ly * z
    x = np.where(k == 0, Lx * z * (1 + d), np.where(k == 1, -Lx * z * (1 + d), x))
    y = np.where(k == 2, Ly * z * (1 + d), np.where(k == 3, -Ly * z * (1 + d), y))
    z = np.where(k == 4, 0.2 * (1 - d), z)
    x = np.where(k == 4, rng.uniform(-0.9, 0.9, n) * Lx * 0.2, x)
    y = np.where(k == 4, rng.uniform(-0.9, 0.9, n) * Ly * 0.2, y)
    v = np.stack([x, y, z], 1)
    Rd, td = R.astype(np.float64), t.astype(np.float64)
    P = ((v - td) @ Rd).astype(f32)                     # world centre: R^T (v - t)
    # outward normal of each plane in world coordinates (exact, in binary64)
    nrm = np.stack([Rd[0] - Lx * Rd[2], -Rd[0] - Lx * Rd[2], Rd[1] - Ly * Rd[2],
                    -Rd[1] - Ly * Rd[2], -Rd[2]])[k]
    ext = np.exp(rng.uniform(np.log(1e-3), np.log(50.0), (n, 3))).astype(f32)
    lo = np.where(nrm > 0, P, P - ext).astype(f32)
    hi = np.where(nrm > 0, P + ext, P).astype(f32)
    return lo, hi, P


@pytest.mark.parametrize("fused_margin", [False, True], ids=["margin_plain", "margin_fused"])
@pytest.mark.parametrize("fused", [False, True], ids=["planes_plain", "planes_fused"])
def test_culled_boxes_hold_no_passing_centre(fused, fused_margin):
    rng = np.random.default_rng(5 + int(fused) + 2 * int(fused_margin))
    n_corner_pass = 0
    n_culled = 0
    for _ in range(60):
        R, t, tan = random_camera(rng)
        Pl, scale, tt = planes(R, t, tan, fused)
        lo, hi, corner = grazing_boxes(rng, R, t, tan, 4000)
        # random boxes too: centres within 600 of the camera, up to 80 wide
        c = (-(t.astype(np.float64)) @ R.astype(np.float64) + rng.uniform(-600, 600, (2000, 3)))
        e = rng.uniform(0, 80, (2000, 3))
        lo = np.concatenate([lo, (c - e).astype(f32)])
        hi = np.concatenate([hi, (c + e).astype(f32)])
        corner = np.concatenate([corner, (c - e).astype(f32)])
        out = box_outside(Pl, scale, tt, lo, hi, fused_margin)
        n_culled += int(out.sum())
        # the centres tested per box: the grazing corner, the eight box corners, random points
        pts = [corner]
        for cx in (0, 1):
            for cy in (0, 1):
                for cz in (0, 1):
                    pts.append(np.stack([(lo, hi)[cx][:, 0], (lo, hi)[cy][:, 1], (lo, hi)[cz][:, 2]], 1))
        for _ in range(4):
            f = rng.random(lo.shape).astype(f32)
            pts.append((lo + f * (hi - lo)).astype(f32))
        passing = np.zeros(len(lo), bool)
        for p in pts:
            p = np.clip(p, lo, hi)
            passing |= node_passes(R, t, tan, p)
        n_corner_pass += int(node_passes(R, t, tan, corner).sum())
        bad = out & passing
        assert not bad.any(), f"{int(bad.sum())} culled boxes hold a centre that passes"
    assert n_culled > 50000            # the cull does skip boxes
    assert n_corner_pass > 50000       # and many grazing corners pass the per-node test

"""The blend's culling masks are conservative (CPU, brute force).

Before a tile is walked, each Gaussian gets a mask of the tile's 4x4 half-blocks (the
forward) or of its warps' pixel blocks (the KPC pre-render) whose pixels may reach
its skip threshold: power >= lthr, the alpha >= 1/255 rule of Eq. 2.  The mask is
cut from the threshold ellipse's bounding box with margins for binary32 rounding.
A block left out of the mask is never tested, so the masks must be conservative
for the kernel's exact binary32 power.  This test restates the mask and the power
in numpy binary32, the way the kernel rounds them, and checks by brute force over
every pixel of a tile that no pixel whose power passes both skip tests lies in a
block outside the mask.  The Gaussians are random: screen covariances from
isotropic to the conditioning limit beyond which every block is kept (cond 1e4),
footprints from sub-pixel to wider than the tile, opacities down to 1/255 (a
vanishing ellipse), centres in, beside and far from the tile; and Gaussians whose
ellipse reaches a pixel centre on a block's edge row or column at its extreme
point, to within a small relative offset of the exact boundary.  The latter give
the test its power: the same masks without the rounding margins (the exact box)
miss hundreds of passing pixels of them.  Every way the compiler may contract
the determinant into a fused multiply-add is checked.
"""
import numpy as np
import pytest

f32 = np.float32


def fma(a, b, c):
    """Fused multiply-add in binary32: the binary64 product of two binary32 values is
    exact, and the one binary64 rounding of the sum lies within an ulp of binary64
    of the exact sum, far inside the margins under test."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def dets(A, B, C):
    """A C - B B as the compiler may round it: plainly, or with either product fused."""
    AC, BB = A * C, B * B
    return [AC - BB, fma(A, C, -BB), fma(-B, B, AC)]


def box_extent(A, B, C, lthr, det):
    """Half-widths ex, ey of the threshold ellipse's box, with the kernel's margins;
    `full` marks the Gaussians for which every block is kept (singular or badly
    conditioned conic)."""
    tr = A + C
    full = ~(det > 0) | (tr * tr > f32(1e4) * det)
    with np.errstate(divide="ignore", invalid="ignore"):
        sq = fma(np.full_like(lthr, f32(-2.1)), lthr, np.full_like(lthr, f32(1e-4)))
        ex = fma(np.sqrt((sq * C) / det), np.full_like(lthr, f32(1.001)), np.full_like(lthr, f32(0.01)))
        ey = fma(np.sqrt((sq * A) / det), np.full_like(lthr, f32(1.001)), np.full_like(lthr, f32(0.01)))
    return full, ex, ey


def block_range(uc, e, bw, n):
    """Blocks (of bw pixels, n of them) whose pixel centres meet [uc - e, uc + e]."""
    with np.errstate(invalid="ignore"):
        lo = np.ceil((uc - e - f32(bw - 0.5)) * f32(1.0 / bw))
        hi = np.floor((uc + e - f32(0.5)) * f32(1.0 / bw))
    lo = np.maximum(0, np.nan_to_num(lo, nan=0).astype(np.int64))
    hi = np.minimum(n - 1, np.nan_to_num(hi, nan=n - 1).astype(np.int64))
    return lo, hi


def block_mask(u, v, A, B, C, lthr, tx0, ty0, bw, bh, ncol, nrow, det):
    """The mask as the kernel forms it: bit r * ncol + c for block (c, r)."""
    full, ex, ey = box_extent(A, B, C, lthr, det)
    ux, vy = u - f32(tx0), v - f32(ty0)
    c_lo, c_hi = block_range(ux, ex, bw, ncol)
    r_lo, r_hi = block_range(vy, ey, bh, nrow)
    cols = np.arange(ncol)[None, :]
    rows = np.arange(nrow)[None, :]
    cin = (cols >= c_lo[:, None]) & (cols <= c_hi[:, None])          # [G, ncol]
    rin = (rows >= r_lo[:, None]) & (rows <= r_hi[:, None])          # [G, nrow]
    m = rin[:, :, None] & cin[:, None, :]                             # [G, nrow, ncol]
    m = m.reshape(len(u), nrow * ncol)
    m[full] = True
    m[~(lthr <= 0)] = False                                           # alpha0 < 1/255
    return m


def power(u, v, A, B, C, px, py):
    """The kernel's binary32 exponent: A' = -A/2, B' = -B, C' = -C/2, then
    (A' dx + B' dy) dx + (C' dy) dy with two fused multiply-adds."""
    Ah, Bn, Ch = f32(-0.5) * A, -B, f32(-0.5) * C
    dx = u[:, None] - px[None, :]
    dy = v[:, None] - py[None, :]
    inner = fma(np.broadcast_to(Ah[:, None], dx.shape), dx, Bn[:, None] * dy)
    return fma(inner, dx, (Ch[:, None] * dy) * dy)


def random_gaussians(rng, n, tx0, ty0, tile):
    """Conics of 2D covariances R diag(s1^2, s2^2) R^T + 0.3 I (the dilation), with
    s1 log-uniform over sub-pixel to beyond the tile, s2 = s1 / ratio and the ratio up
    to past the conditioning limit; opacity thresholds down to alpha0 = 1/255."""
    s1 = np.exp(rng.uniform(np.log(0.05), np.log(4.0 * tile), n))
    ratio = np.exp(rng.uniform(0.0, np.log(400.0), n))
    s2 = s1 / ratio
    th = rng.uniform(0.0, np.pi, n)
    c, s = np.cos(th), np.sin(th)
    a = c * c * s1 ** 2 + s * s * s2 ** 2 + 0.3
    b = c * s * (s1 ** 2 - s2 ** 2)
    d = s * s * s1 ** 2 + c * c * s2 ** 2 + 0.3
    det = a * d - b * b
    A, B, C = (d / det).astype(f32), (-b / det).astype(f32), (a / det).astype(f32)
    alpha0 = np.where(rng.random(n) < 0.2, 1.0 / 255.0 * (1.0 + rng.uniform(0, 1e-3, n)),
                      rng.uniform(1.0 / 255.0, 0.99, n))
    lthr = np.log(1.0 / 255.0 / alpha0).astype(f32)
    reach = np.minimum(3.0 * s1, 3.0 * tile)
    u = (tx0 + rng.uniform(-reach, tile + reach)).astype(f32)
    v = (ty0 + rng.uniform(-reach, tile + reach)).astype(f32)
    return u, v, A, B, C, lthr


def boundary_gaussians(rng, n, tx0, ty0, tw, th, bw, bh):
    """Gaussians whose threshold ellipse reaches, at its extreme point along x or y,
    a pixel centre on the first or last pixel row / column of a block, to within a
    relative offset delta of the exact boundary on either side (the pixel then
    passes or fails the binary32 test by its rounding, and the exact box edge falls
    on the block edge)."""
    u0, v0, A, B, C, lthr = random_gaussians(rng, n, tx0, ty0, tw)
    a, b, c = A.astype(np.float64), B.astype(np.float64), C.astype(np.float64)
    s = -2.0 * lthr.astype(np.float64)
    det = a * c - b * b
    ok = (det > 0) & ((a + c) ** 2 < 1e4 * det)
    delta = rng.uniform(-2e-3, 2e-3, n) * np.where(rng.random(n) < 0.5, 1.0, 1e-4)
    along_x = rng.random(n) < 0.5
    with np.errstate(invalid="ignore", divide="ignore"):
        X = np.sqrt(s * c / det) * (1.0 - delta)        # extreme along x: (X, -B X / C)
        Yx = -b * X / c
        Y = np.sqrt(s * a / det) * (1.0 - delta)        # extreme along y: (-B Y / A, Y)
        Xy = -b * Y / a
    ex_off = np.where(along_x, X, Xy)
    ey_off = np.where(along_x, Yx, Y)
    ncol, nrow = tw // bw, th // bh
    first = rng.random(n) < 0.5                         # first pixel of a block, else its last
    col = rng.integers(0, ncol, n) * bw + np.where(first, 0, bw - 1)
    row = rng.integers(0, nrow, n) * bh + np.where(first, 0, bh - 1)
    col = np.where(along_x, col, rng.integers(0, tw, n))
    row = np.where(along_x, rng.integers(0, th, n), row)
    px = tx0 + col + 0.5
    py = ty0 + row + 0.5
    sign = np.where(first, 1.0, -1.0)                   # the pixel lies beyond the centre
    u = np.where(ok, px - sign * ex_off, u0).astype(f32)
    v = np.where(ok, py - sign * ey_off, v0).astype(f32)
    return u, v, A, B, C, lthr


SHAPES = [
    # (tile_w, tile_h, block_w, block_h): the forward's 4x4 half-blocks of 16x16 and
    # 32x8 tiles, and the KPC pass's 8x4 and 4x8 warp blocks
    (16, 16, 4, 4), (32, 8, 4, 4), (16, 16, 8, 4), (16, 16, 4, 8),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"tile{s[0]}x{s[1]}_block{s[2]}x{s[3]}")
def test_masks_keep_every_block_with_a_passing_pixel(shape):
    tw, th, bw, bh = shape
    ncol, nrow = tw // bw, th // bh
    tx0, ty0 = 5 * tw, 3 * th
    ys, xs = np.mgrid[0:th, 0:tw]
    px = (xs.ravel() + tx0).astype(f32) + f32(0.5)
    py = (ys.ravel() + ty0).astype(f32) + f32(0.5)
    bit = (ys.ravel() // bh) * ncol + xs.ravel() // bw                # each pixel's block
    rng = np.random.default_rng(11 + tw + 3 * bw)
    n_hit_pixels = 0
    n_kept_blocks = 0
    n_blocks = 0
    for it in range(8):
        if it % 2:
            u, v, A, B, C, lthr = boundary_gaussians(rng, 20000, tx0, ty0, tw, th, bw, bh)
        else:
            u, v, A, B, C, lthr = random_gaussians(rng, 20000, tx0, ty0, tw)
        p = power(u, v, A, B, C, px, py)
        hit = ~((p > 0) | (p < lthr[:, None]))                        # both skip tests pass
        n_hit_pixels += int(hit.sum())
        for det in dets(A, B, C):
            m = block_mask(u, v, A, B, C, lthr, tx0, ty0, bw, bh, ncol, nrow, det)
            missed = hit & ~m[:, bit]
            assert not missed.any(), (
                f"{int(missed.sum())} passing pixels in blocks outside the mask, first Gaussian "
                f"{np.flatnonzero(missed.any(1))[:1]}")
            n_kept_blocks += int(m.sum())
            n_blocks += m.size
    # the cases are not vacuous: many pixels pass, and the masks do drop blocks
    assert n_hit_pixels > 100000
    assert n_kept_blocks < 0.8 * n_blocks


def test_masks_are_tight_for_a_round_gaussian():
    """The margins are small: a round Gaussian of 2 px sigma at alpha0 = 0.5 in the
    middle of a 16x16 tile (threshold radius sqrt(2 ln 127.5) * 2 = 6.2 px) keeps the
    four central half-blocks and their neighbours it reaches, not the corners."""
    s2 = 4.0 + 0.3
    A = np.array([1.0 / s2], f32)
    C = A.copy()
    B = np.zeros(1, f32)
    lthr = np.array([np.log(1.0 / 255.0 / 0.5)], f32)
    u = np.array([8.0], f32)
    v = np.array([8.0], f32)
    m = block_mask(u, v, A, B, C, lthr, 0, 0, 4, 4, 4, 4, dets(A, B, C)[0])[0].reshape(4, 4)
    r = np.sqrt(-2.0 * float(lthr[0]) * s2)
    assert 6.0 < r < 6.5
    # blocks whose pixel centres (0.5 .. 3.5 + 4k) come within r of the centre along each axis
    assert m.all()                      # r > 4.5: every column and row is reached
    A2 = np.array([1.0 / (1.0 + 0.3)], f32)
    m2 = block_mask(u, v, A2, B, A2.copy(), lthr, 0, 0, 4, 4, 4, 4, dets(A2, B, A2)[0])[0].reshape(4, 4)
    r2 = np.sqrt(-2.0 * float(lthr[0]) * 1.3)
    assert 3.3 < r2 < 3.7               # reaches pixel centres 4.5 .. 11.5 only: the middle blocks
    assert m2[1:3, 1:3].all() and not m2[0].any() and not m2[3].any()
    assert not m2[:, 0].any() and not m2[:, 3].any()

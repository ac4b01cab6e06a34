"""The oracle's OpenMP loops change no bit: a whole frame (cut, splats, pairs, image,
transmittance, KPC), sampled pixels and the calibration on one thread and on every
host thread are identical."""
import math

import numpy as np

import oracle
from paper_2603_23891_gb300 import synth


def _run(tree, cams, p):
    out = []
    for cam in cams:
        fr = oracle.frame(tree, cam, p, want_kpc=True)
        pix = np.arange(0, cam.width * cam.height, 7, dtype=np.int64)
        rgb, T = oracle.render_pixels(fr.splat, fr.keys, fr.vals, cam, p, pix)
        out.append((fr, rgb, T))
    return out


def test_threads_bit_identical():
    tree = synth.random_small_tree(3, n_leaves=30000, branching=(2, 8), sh_degree=2, extent=40.0,
                                   log_scale_mean=-0.6)
    c = tree.mu.mean(axis=1).astype(np.float64)
    cams = [synth.look_at_camera(c + [0, -70, 30], c, 190, 130, 60.0),
            synth.look_at_camera(c + [50, 20, 25], c, 333, 77, 75.0)]
    p = oracle.Params(tau_R=3.0, tile_w=32, tile_h=8, shrink=True, tau=0.05,
                      ln_tau=float(np.float32(math.log(0.05))), bg=(0.1, 0.2, 0.3))
    n_all = oracle.set_threads(0)
    try:
        oracle.set_threads(1)
        one = _run(tree, cams, p)
        cal1 = oracle.calibrate(tree, cams, 3.0)
        oracle.set_threads(max(n_all, 4))
        many = _run(tree, cams, p)
        calm = oracle.calibrate(tree, cams, 3.0)
    finally:
        oracle.set_threads(n_all)
    for (a, ra, ta), (b, rb, tb) in zip(one, many):
        assert len(a.sel) > 1000 and len(a.keys) > 1000
        for f in ("sel", "splat", "rect", "keys", "vals", "T"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f
        assert np.array_equal(a.rgb.view(np.uint64), b.rgb.view(np.uint64))
        assert np.array_equal(a.kpc.view(np.uint64), b.kpc.view(np.uint64))
        assert np.array_equal(ra.view(np.uint64), rb.view(np.uint64))
        assert np.array_equal(ta.view(np.uint32), tb.view(np.uint32))
    assert cal1[0] == calm[0] and cal1[1] == calm[1] and cal1[2] == calm[2]

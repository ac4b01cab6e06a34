"""GPU parity and properties of the shrinking study (§3.3; §4.2 shrinking
comparison and lambda_G sweep).

The KPC of every pair under a shrunk footprint (fgs_kpc_view) against the
oracle's Eq. 5 on the oracle's shrunk pair list; then the study on the blob
tree: N_P non-increasing along 3 sigma -> tau = 1/255 -> lambda_G sweep, and the
redundant pairs (KPC < 0.05) are the ones shrinking removes first."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_23891_gb300 import synth

from gpu_util import oracle_frame, orbit_cameras

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


@pytest.mark.parametrize("tau", [1.0 / 255.0, 0.02, 0.1])
def test_kpc_view_under_shrink_matches_oracle(renderer, tau):
    tree = synth.random_small_tree(11, n_leaves=2000, branching=(2, 6), sh_degree=1,
                                   extent=15.0, log_scale_mean=-0.9)
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    shrink = (float(np.float32(tau)), float(np.float32(math.log(tau))))
    for cam in orbit_cameras(tree, 3, (128, 96), 5):
        renderer.set_camera(cam)
        renderer.shrink(*shrink)
        renderer.render()
        n = renderer.n_pairs()
        gbar, G, kpc = renderer.kpc_view(n)
        o, p = oracle_frame(tree, cam, 3.0, shrink=shrink, blend=False)
        assert n == len(o.keys)
        _, _, okpc = oracle.render(o.splat, o.keys, o.vals, cam, p, want_kpc=True)
        tx, ty = oracle.tiles_of(cam, p)
        oG, ogbar, _ = oracle.gtc(o.keys, okpc, tx * ty)
        np.testing.assert_allclose(kpc, okpc, rtol=1e-4, atol=1e-5)
        both = ~np.isnan(oG)
        assert np.array_equal(np.isnan(G), np.isnan(oG))
        np.testing.assert_allclose(G[both], oG[both], rtol=1e-4, atol=1e-6)
        assert gbar == pytest.approx(ogbar, rel=1e-4)


def test_study_on_blobs(renderer):
    from paper_2603_23891_gb300 import shrink_study
    tree, cams = synth.blob_tree(), synth.blob_cameras()
    renderer.load_tree(tree)
    renderer.set_params(tau_R=3.0, tile=(16, 16))
    res = shrink_study.run_study(renderer, cams, [0, 4], lambdas=(0.02, 0.1, 0.2, 0.43), reps=1)
    rows = res["settings"]
    names = [r["setting"] for r in rows]
    assert names[:2] == ["3sigma", "tau_1/255"]
    nps = [r["N_P_mean"] for r in rows]
    assert all(a >= b for a, b in zip(nps, nps[1:])), nps
    assert rows[0]["psnr_vs_3sigma_db"] == math.inf and rows[0]["max_abs_vs_3sigma"] == 0.0
    assert rows[-1]["N_P_mean"] < 0.8 * rows[0]["N_P_mean"]
    # pairs removed by shrinking are mostly redundant ones: the count of pairs with
    # KPC >= 0.05 drops less, relatively, than the count below 0.05
    lo0 = rows[0]["kpc"]["below_0.05"]
    hi0 = rows[0]["kpc"]["pairs"] - lo0
    lo1 = rows[-1]["kpc"]["below_0.05"]
    hi1 = rows[-1]["kpc"]["pairs"] - lo1
    assert lo1 / lo0 < hi1 / hi0
    psnr = [r["psnr_vs_3sigma_db"] for r in rows[2:]]
    assert psnr[0] >= psnr[-1]
    print({r["setting"]: (round(r["N_P_mean"]), r["psnr_vs_3sigma_db"], r["kpc"]["below_0.05"])
           for r in rows})

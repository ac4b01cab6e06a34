"""Gaussian-shrinking study (§3.3; the shrinking comparison and the lambda_G
sweep of §4.2).

For a workload and a set of poses, every footprint setting
  * 3 sigma (no shrinking, the 3DGS rule),
  * a fixed opacity threshold tau = 1/255,
  * the scene-adaptive tau = lambda_G / G of Eq. 8 for a sweep of lambda_G,
is rendered on the GPU and reported with: the pair count N_P, the frame time,
the KPC distribution of the emitted pairs (Eq. 5, from the KPC blend under the
same footprint), the number of redundant pairs (KPC below 0.01 and 0.05), and
the image error against the 3-sigma render of the same pose (PSNR, max-abs).
The 3-sigma GPU image stands in for the unshrunk oracle image: the parity tests
hold it to the oracle within 2e-3 with bit-identical transmittance.

  python -m paper_2603_23891_gb300.shrink_study --workload city --poses 8
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KPC_EDGES = (0.0, 0.01, 0.05, 0.1, 0.2, 0.5, 1.0, 2.0, 5.0, math.inf)
LAMBDAS = (0.02, 0.03, 0.05, 0.07, 0.1, 0.14, 0.2, 0.3, 0.43)


def kpc_summary(kpc: np.ndarray) -> dict:
    """Histogram of per-pair KPC over KPC_EDGES (left-closed bins) and the
    redundant-pair counts (KPC < 0.01, KPC < 0.05)."""
    k = np.asarray(kpc, np.float64)
    counts = [int(np.count_nonzero((k >= lo) & (k < hi)))
              for lo, hi in zip(KPC_EDGES[:-1], KPC_EDGES[1:])]
    return {"edges": [e if math.isfinite(e) else "inf" for e in KPC_EDGES], "counts": counts,
            "below_0.01": int(np.count_nonzero(k < 0.01)),
            "below_0.05": int(np.count_nonzero(k < 0.05)), "pairs": int(k.size)}


def merge_summaries(a: dict, b: dict) -> dict:
    if a is None:
        return dict(b)
    out = dict(a)
    out["counts"] = [x + y for x, y in zip(a["counts"], b["counts"])]
    for key in ("below_0.01", "below_0.05", "pairs"):
        out[key] = a[key] + b[key]
    return out


def image_error(rgb, ref) -> tuple:
    """(PSNR in dB over [0, 1], max-abs) of two torch images."""
    d = (rgb.double() - ref.double())
    mse = float((d * d).mean())
    return (math.inf if mse == 0 else 10.0 * math.log10(1.0 / mse)), float(d.abs().max())


def run_study(r, cams, poses, lambdas=LAMBDAS, reps: int = 3) -> dict:
    """r: a Renderer with the tree loaded and its tau_R / tile set."""
    import torch
    from paper_2603_23891_gb300 import filtergs  # noqa: F401  (r's library)
    dev = torch.device("cuda", r.device)
    settings = [("3sigma", None), ("tau_1/255", (float(np.float32(1.0 / 255.0)),
                                                 float(np.float32(-math.log(255.0)))))]
    gbar = None
    for lam in lambdas:
        tau, ln_tau, gbars = r.calibrate(cams, lam)
        gbar = float(np.nanmean(gbars)) if gbar is None else gbar
        settings.append((f"lambda_G={lam}", (tau, ln_tau)))
    refs = {}
    r.shrink(None)
    for k in poses:
        r.set_camera(cams[k])
        rgb, _, _ = r.render()
        refs[k] = rgb.clone()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    out = {"poses": list(poses), "G_bar": gbar, "settings": []}
    for name, shr in settings:
        if shr is None:
            r.shrink(None)
        else:
            r.shrink(*shr)
        nps, ms, psnrs, maxabs, summ = [], [], [], [], None
        for k in poses:
            cam = cams[k]
            r.set_camera(cam)
            rgb = torch.empty((3, cam.height, cam.width), dtype=torch.float32, device=dev)
            _, _, st = r.render(rgb, stats=True)
            nps.append(int(st.n_pairs))
            p, m = image_error(rgb, refs[k])
            psnrs.append(p)
            maxabs.append(m)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(reps):
                r.render(rgb)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1) / reps)
            _, _, kpc = r.kpc_view(st.n_pairs)
            summ = merge_summaries(summ, kpc_summary(kpc))
        finite = [p for p in psnrs if math.isfinite(p)]
        out["settings"].append({
            "setting": name, "tau": None if shr is None else shr[0],
            "N_P_mean": float(np.mean(nps)), "ms_mean": round(float(np.mean(ms)), 4),
            "fps": round(1e3 / float(np.mean(ms)), 1),
            "psnr_vs_3sigma_db": round(float(np.mean(finite)), 2) if finite else math.inf,
            "max_abs_vs_3sigma": round(float(np.max(maxabs)), 4),
            "kpc": summ})
    base = out["settings"][0]
    for srow in out["settings"]:
        srow["N_P_vs_3sigma"] = round(srow["N_P_mean"] / base["N_P_mean"], 4)
        b = base["kpc"]["below_0.05"]
        srow["redundant_0.05_vs_3sigma"] = round(srow["kpc"]["below_0.05"] / b, 4) if b else None
    r.shrink(None)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="city", choices=["city", "blobs", "tiny"])
    ap.add_argument("--poses", type=int, default=8, help="every P/poses-th pose of the set")
    args = ap.parse_args()
    from paper_2603_23891_gb300 import build, filtergs, synth
    build.build()
    if args.workload == "city":
        tree, cams, tau_R = synth.city_tree(), synth.city_cameras(), 3.0
    elif args.workload == "blobs":
        tree, cams, tau_R = synth.blob_tree(), synth.blob_cameras(), 3.0
    else:
        tree, cams, tau_R = synth.tiny_tree(), [synth.tiny_camera()], 1.0
    r = filtergs.Renderer(device=0, tau_R=tau_R, pair_capacity=64 << 20)
    r.load_tree(tree)
    step = max(1, len(cams) // args.poses)
    res = run_study(r, cams, list(range(0, len(cams), step))[: args.poses])
    res["workload"] = tree.name
    print(json.dumps(res))
    r.close()


if __name__ == "__main__":
    main()

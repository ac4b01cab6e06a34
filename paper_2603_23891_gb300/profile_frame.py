"""Render a few frames of a synthetic workload, for external profilers (ncu).

  python -m paper_2603_23891_gb300.profile_frame --workload city --frames 3 \
      [--tau 0.0772 --ln-tau -2.5616] [--pose 0]

With --cycle frame k renders pose (pose + k) mod poses.  With --batch the 32-view batch of the city workload is rendered --frames times
(shrink as given by --tau).  With --tau the frames use that shrink threshold and no calibration kernels run,
so the launch sequence is exactly the per-frame path (9 kernels per frame:
frame_begin, filter_pred, filter_anc, compact_counted, project, tile_scan, scatter,
segsort, blend).
Without it the frames use the 3-sigma footprint.  With --backward the tree's
attributes are first recomputed from its parameters (one prep_params launch)
and every frame is followed by the differentiable form's backward for
dL/drgb ~ N(0, 1) (accumulate mode: zero_rows, blend_bwd, project_bwd).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="city", choices=["city", "blobs", "tiny"])
    ap.add_argument("--frames", type=int, default=3)
    ap.add_argument("--pose", type=int, default=0)
    ap.add_argument("--tau", type=float, default=None)
    ap.add_argument("--ln-tau", dest="ln_tau", type=float, default=None)
    ap.add_argument("--backward", action="store_true")
    ap.add_argument("--cycle", action="store_true",
                    help="frame k renders pose (pose + k) mod poses (the bench's timed poses)")
    ap.add_argument("--batch", action="store_true",
                    help="render the 32-view city batch (16x16 tiles, 8x4 warps) instead")
    args = ap.parse_args()

    import torch
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
    if args.tau is not None:
        r.shrink(args.tau, args.ln_tau)
    if args.batch:
        bc = synth.city_batch_cameras()
        r.batch_setup(bc, sel_capacity=96 << 20, pair_capacity=256 << 20)
        t0 = time.time()
        for _ in range(args.frames):
            _, _, st, _ = r.render_batch(stats=True)
        torch.cuda.synchronize()
        print(f"{args.frames} batches of {len(bc)} views, entries={st.n_selected} N_P={st.n_pairs} "
              f"launches/batch={st.n_launches} ({time.time() - t0:.3f}s)")
        r.close()
        return
    cam = cams[args.pose % len(cams)]
    r.set_camera(cam)
    P = G = dL = None
    if args.backward:
        import numpy as np
        P = {"mu": tree.mu, "log_scale": tree.log_scale, "quat": tree.quat,
             "logit": tree.opacity_logit, "sh": tree.sh}
        P = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda() for k, v in P.items()}
        G = {k: torch.zeros_like(v) for k, v in P.items()}
        dL = torch.randn((3, cam.height, cam.width), device="cuda",
                         generator=torch.Generator(device="cuda").manual_seed(0))
        r.update_params(P)
    t0 = time.time()
    st = None
    for k in range(args.frames):
        if args.cycle:
            r.set_camera(cams[(args.pose + k) % len(cams)])
        _, _, st = r.render(stats=True, keep=args.backward)
        if args.backward:
            r.backward(dL, P, G, accumulate=True)
    torch.cuda.synchronize()
    print(f"{args.frames} frames, M={st.n_selected} N_P={st.n_pairs} "
          f"launches/frame={st.n_launches} ({time.time() - t0:.3f}s)")
    r.close()


if __name__ == "__main__":
    main()

"""Render a few frames of a synthetic workload, for external profilers (ncu).

  python -m paper_2603_23891_gb300.profile_frame --workload city --frames 3 \
      [--tau 0.0772 --ln-tau -2.5616] [--pose 0]

With --tau the frames use that shrink threshold and no calibration kernels run,
so the launch sequence is exactly the per-frame path (12 kernels per frame).
Without it the frames use the 3-sigma footprint.
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
    cam = cams[args.pose % len(cams)]
    r.set_camera(cam)
    t0 = time.time()
    st = None
    for _ in range(args.frames):
        _, _, st = r.render(stats=True)
    torch.cuda.synchronize()
    print(f"{args.frames} frames, M={st.n_selected} N_P={st.n_pairs} "
          f"launches/frame={st.n_launches} ({time.time() - t0:.3f}s)")
    r.close()


if __name__ == "__main__":
    main()

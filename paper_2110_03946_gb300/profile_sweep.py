"""Run a few fine-level ORAS sweeps on one synthetic frame: a small, fixed
launch sequence for profilers (e.g. ``ncu -k regex:oras_sweep -s 1 -c 1``).

python -m paper_2110_03946_gb300.profile_sweep [--workload rgb4k_edge3]
       [--precision fp32] [--k 16] [--local-rtol 0] [--sweeps 3]
"""
from __future__ import annotations

import argparse
import os
import sys


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="rgb4k_edge3")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--block", type=int, default=None)
    ap.add_argument("--overlap", type=int, default=None)
    ap.add_argument("--k", type=int, default=16)
    ap.add_argument("--robin", type=float, default=0.0)
    ap.add_argument("--tile-warps", type=int, default=0)
    ap.add_argument("--local-rtol", type=float, default=0.0)
    ap.add_argument("--sweeps", type=int, default=3)
    a = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import synth
    from paper_2110_03946_gb300.inpaint import Inpainter

    w = synth.WORKLOADS[a.workload]
    f, m = synth.workload_frame(a.workload)
    dev = torch.device("cuda", 0)
    fd, md = torch.as_tensor(f).to(dev), torch.as_tensor(m).to(dev)
    with Inpainter(md, fd, device=dev, block=a.block or w.block, overlap=a.overlap if a.overlap is not None
                   else w.overlap, local_cg_iters=a.k, levels=1, precision=a.precision, robin_p=a.robin,
                   tile_warps=a.tile_warps, local_rtol=a.local_rtol) as ip:
        ip.set_iterate(fd * (md != 0))
        for _ in range(a.sweeps):
            ip.sweep(1)
        torch.cuda.synchronize()
    print("profile_sweep done")


if __name__ == "__main__":
    main()

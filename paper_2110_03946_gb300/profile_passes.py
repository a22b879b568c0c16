"""A fixed sequence of whole solves on one synthetic frame that runs every
kernel of the library, as plain launches (device_loop = 0, so profilers list
each kernel by name): the multilevel FP32 ORAS cascade, the coarse-grid
correction mode, multilevel conjugate gradients, and FP16 inner storage with
the FP64-accurate outer correction.  For profilers, e.g.
``ncu --metrics gpu__time_duration.sum`` (a launch list) or a
``--section MemoryWorkloadAnalysis`` capture of the streaming passes.

python -m paper_2110_03946_gb300.profile_passes [--workload rgb4k_edge3]
       [--legs oras,correction,cg,cg_fine,fp16,correction_cg]
"""
from __future__ import annotations

import argparse
import os
import sys


LEGS = {
    "oras": dict(precision="fp32"),
    "correction": dict(precision="fp32", ml_mode="correction", correction_sweeps=2),
    "cg": dict(precision="fp32", solver="cg", max_sweeps=4000, coarse_sweeps=400),
    # plain CG on the fine grid alone, a fixed 40 iterations (it does not converge):
    # the fine-level operator and update passes at full size
    "cg_fine": dict(precision="fp32", solver="cg", levels=1, max_sweeps=40),
    "fp16": dict(precision="fp16_ref"),
    # the coarse-grid correction after every fine sweep with the small-grid coarse CG on a
    # hierarchy deep enough for it (4K: 6 levels, coarsest 120 x 68)
    "correction_cg": dict(precision="fp32", ml_mode="correction", levels=6, correction_cg=300),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="rgb4k_edge3")
    ap.add_argument("--legs", default="oras,correction,cg,fp16")
    ap.add_argument("--tol", type=float, default=1e-6)
    a = ap.parse_args()
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch

    import synth
    from paper_2110_03946_gb300 import autotune
    from paper_2110_03946_gb300.inpaint import Inpainter

    w = synth.WORKLOADS[a.workload]
    f, m = synth.workload_frame(a.workload)
    base = autotune.lookup(w.H, w.W, w.C, w.density, "fp32", a.tol) or dict(block=w.block, overlap=w.overlap)
    dev = torch.device("cuda", 0)
    fd, md = torch.as_tensor(f).to(dev), torch.as_tensor(m).to(dev)
    for leg in a.legs.split(","):
        prm = dict(base, device_loop=0, **LEGS[leg])
        with Inpainter(md, fd, device=dev, **prm) as ip:
            ip.solve(a.tol, allow_unconverged=leg == "cg_fine")
            torch.cuda.synchronize()
            st = ip.stats()
        print(f"{leg}: sweeps {st['sweeps_per_level']} corrections {st['corrections']} "
              f"converged {st['converged']} ms {st['ms_total']:.2f}")
    print("profile_passes done")


if __name__ == "__main__":
    main()

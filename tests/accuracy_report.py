"""Prints the rel-L2 error of every precision mode against the FP64 oracle, per
bandwidth, on band-limited inputs (the table in the design doc).  Needs a GPU:

    python tests/accuracy_report.py [B ...]
"""
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1808_00896_gb300 import Plan, synth  # noqa: E402


def main(bandwidths):
    oracle.build()
    dev = torch.device("cuda", 0)
    for B in bandwidths:
        coef = synth.coefficients(B, "gauss_decay", seed=123 + B)
        g_ref = oracle.inverse(B, coef)
        f_ref = oracle.forward(B, g_ref)
        for mode in ("fp64", "fp64_tc", "bf16x3", "tf32"):
            with Plan(B, mode, device=dev) as p:
                f = p.forward(torch.from_numpy(g_ref).to(dev)).cpu().numpy()
                g = p.inverse(torch.from_numpy(coef).to(dev)).cpu().numpy()
            print(f"B={B:4d} {mode:7s} forward rel-L2 {synth.rel_l2(f, f_ref):.3e}  "
                  f"inverse rel-L2 {synth.rel_l2(g, g_ref):.3e}", flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [8, 16, 32, 64, 128])

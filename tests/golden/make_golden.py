"""Writes tests/golden/tiny_cavity.npz from the FP64 oracle only.

A regression fixture: three steps of a 4x4-cell cavity with 8^3 velocities
from a seeded warm state.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1005_5405_gb300 import workloads  # noqa: E402

PROBLEM = dict(nx=4, ny=4, kn=1.0, nv=8, vmax=4.0, nt=500, seed=17, lid_u0=0.1)


def make():
    p = workloads.small(nx=4, ny=4, nv=8, vmax=4.0)
    h0 = workloads.warm_state(p, seed=19)
    o = oracle.Oracle(**PROBLEM)
    h, mom = o.run(h0, 3)
    return h0, h, mom


if __name__ == "__main__":
    h0, h, mom = make()
    np.savez_compressed(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_cavity.npz"),
                        h0=h0, h3=h, mom3=mom)
    print("wrote tiny_cavity.npz")

"""Writes j2_amplitude.json: the displacement amplitude of the elastoplastic
hex8 workload (96^3 cube, two load steps 0.5 u and u) at which 30% of the
Gauss points yield in the second step.

The fraction is computed by the CPU oracle only (oracle.j2_sweep); the
amplitude is found by bisection on a log scale until the fraction is within
0.25% of 30%.  Run:  python tests/golden/make_j2_amplitude.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_1805_03949_gb300 import meshgen as mg  # noqa: E402

TARGET = 0.30


def fraction(mesh, U, amp):
    n1, st = oracle.j2_sweep(mesh, U, 0.5 * amp, want_state=True)
    n2 = oracle.j2_sweep(mesh, U, amp, st)
    pts = 8 * mesh.n_elems
    return n1 / pts, n2 / pts


def main(n=96):
    mesh, U = mg.j2_workload(n)
    lo, hi = 1e-6, 1e-3
    f_lo, f_hi = fraction(mesh, U, lo)[1], fraction(mesh, U, hi)[1]
    assert f_lo < TARGET < f_hi
    amp, f1, f2 = None, None, None
    for _ in range(40):
        mid = float(np.sqrt(lo * hi))
        f1, f2 = fraction(mesh, U, mid)
        amp = mid
        print(f"amplitude {mid:.6e}: step 1 {f1:.4f}, step 2 {f2:.4f}", flush=True)
        if abs(f2 - TARGET) <= 0.0025:
            break
        if f2 < TARGET:
            lo = mid
        else:
            hi = mid
    out = {"workload": f"hex8 J2/Voce, {n}^3 cube jittered +-0.2h (PCG64 seed 6), "
                       "u = amplitude * fourier_displacement(seed 4, 8 modes), steps 0.5u and u",
           "n": n, "amplitude": amp, "yield_fraction_step1": f1, "yield_fraction_step2": f2,
           "source": "oracle.j2_sweep (CPU FP64 oracle), bisection to 30 +- 0.25 %"}
    with open(os.path.join(HERE, "j2_amplitude.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(out)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 96)

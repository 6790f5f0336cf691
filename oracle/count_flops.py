"""Writes profiles/algorithmic_flops.json: the method's flops per cell, counted
by the oracle's op-counting scalar (count_ops) on the benchmark workloads'
initial states.

TEST AND MEASUREMENT INFRASTRUCTURE: it calls only the oracle and the seeded
input generators.  The benchmark reads the file for the numerator of its ALU
rooflines (algorithmic flops per cell x cells / kernel time); the method's
count does not depend on the GPU code, so the file stays valid across kernel
changes.

    python -m oracle.count_flops
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1607_08710_gb300 import inputs  # noqa: E402

OUT = os.path.join(ROOT, "profiles", "algorithmic_flops.json")

# (name, oracle config, initial primitive state): the benchmark's workloads on
# a mesh small enough to count in seconds.  The share of active limiters, the
# only data-dependent part, is a property of the state's structure (constant
# regions, layers, waves), not of the mesh size.
WORKLOADS = {
    "kh2d": ("periodic Kelvin-Helmholtz shear layer (seed 0), counted at 1024x1024",
             dict(nx=1024, ny=1024, limiter="vanleer", bc="periodic", cfl=0.45),
             lambda: inputs.kelvin_helmholtz(1024, 1024, seed=0).stack()),
    "quadrant2d": ("four-quadrant Riemann problem (seed 0), counted at 1024x1024",
                   dict(nx=1024, ny=1024, limiter="vanleer", bc="transmissive", cfl=0.45),
                   lambda: inputs.quadrant(1024, 1024, seed=0).stack()),
    "shear3d": ("periodic 3D shear layer (seed 0), counted at 96x96x96",
                dict(nx=96, ny=96, nz=96, dim=3, limiter="vanleer", bc="periodic", cfl=0.45),
                lambda: inputs.shear_layer_3d(96, 96, 96, seed=0).stack()),
}


def main() -> dict:
    out = {"how": "oracle count_ops: every primitive state, limited slope, face flux and flux balance formed once "
                  "per cell or face; each add, multiply, divide and square root is one flop; comparisons, "
                  "absolute values and sign tests are not counted",
           "workloads": {}}
    for key, (what, kw, gen) in WORKLOADS.items():
        oc = O.OracleConfig(**kw)
        counts = O.count_ops(oc, O.prim_to_cons(oc, gen()))
        f = O.flops_per_cell(counts)
        out["workloads"][key] = {"workload": what, "flops_per_cell": f, "parts": counts}
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    return out


if __name__ == "__main__":
    r = main()
    for k, v in r["workloads"].items():
        print(k, json.dumps(v["flops_per_cell"]))

"""Writes tests/golden/cm1024_relaxed.json: the FP64 oracle's own arrested-Newton-flow
relaxation (Sec. 3.2: RK4 with the Eq. 4 arrest, from rest) of the 1024^2 chiral-magnet
workload (Eq. 5 without demagnetisation; J = D = 1, K = 0.1, h = 0.6, interfacial DMI,
dx = 0.2, eight compact skyrmions at seeded positions) to dx dy max|G| < 1e-6, and
the energy, lattice charge and residual of the field it ends on.

It calls only the oracle and the seeded input generator; no value comes from the
CUDA path. About 6-15 minutes on 8-16 host cores:

    python tests/golden/make_cm1024_relaxed.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2603_24370_gb300 import inputs as I  # noqa: E402


def main() -> None:
    p = I.cm_skyrmions()
    f0 = O.ansatz(O.CHIRAL_MAGNET, p.soliton_array(), p.nx, p.ny, p.dx, p.dy)
    t0 = time.time()
    r = O.minimise(O.CHIRAL_MAGNET, p.params, f0, p.dx, p.dy, 1e-6, 100000)
    wall = time.time() - t0
    obs = O.observables(O.CHIRAL_MAGNET, p.params, r["f"], p.dx, p.dy)
    out = {
        "workload": "chiral magnet 1024x1024, dx 0.2, J=D=1, K=0.1, h=0.6, interfacial DMI, 8 skyrmions "
                    "(inputs.cm_skyrmions defaults), FP64 oracle ANF-RK4 from rest to dx dy max|G| < 1e-6",
        "params": list(p.params),
        "converged": r["converged"],
        "steps": r["steps"],
        "arrests": r["arrests"],
        "energy": obs["energy"],
        "charge": obs["charge"],
        "grad_max": obs["grad_max"],
        "norm_dev": obs["norm_dev"],
        "oracle_threads": O.num_threads(),
        "oracle_wall_s": round(wall, 1),
        "written_by": "tests/golden/make_cm1024_relaxed.py (oracle only)",
    }
    with open(os.path.join(HERE, "cm1024_relaxed.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()

"""Writes tests/golden/c3_theta_fd.json from the oracle only:

    python tests/golden/make_c3_fd.py [workers]

Central finite differences of the shape-optimisation loss (Sec. 3.3; the loss
of reading R11, ``oracle.shape_opt``) on the differentiable workload: the
degree-6 SH body (49 coefficients) at 100,000 fixed seeded directions, 128^3
grid, 500,000 uniform query points, target = the same pipeline at the seeded
target coefficients.  Step 1e-4 along each stored direction, central cells
frozen at the base point (reading R12), points and normals in FP64.  The
directions are the normalised oracle adjoint gradient and the four coordinate
axes with the largest adjoint components.  The oracle adjoint itself is stored
beside them.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import shape_opt as SO  # noqa: E402

EPS = 1e-4
RES = 128
BBOX = np.array([0, 0, 0, 1, 1, 1], dtype=np.float32)


def main(workers: int):
    t0 = time.time()
    ci = synth.config_inputs("shopt128")
    dirs, th0, tht, q = ci["dirs"], ci["theta"], ci["theta_target"], ci["queries"]
    pt, nt = SO.sh_cloud(tht, dirs)
    phi_t, _ = SO.phi_at_queries(pt, nt, q, BBOX, RES, workers)
    p0, n0 = SO.sh_cloud(th0, dirs)
    phi0, rec0 = SO.phi_at_queries(p0, n0, q, BBOX, RES, workers)
    L0 = SO.loss(phi0, phi_t)
    dth, _, _ = SO.theta_gradient(th0, dirs, rec0, q, SO.loss_seeds(phi0, phi_t))
    print(f"base L={L0:.6e} |dtheta|={np.linalg.norm(dth):.6e} ({time.time() - t0:.0f} s)", flush=True)
    bins = rec0.bins
    top = np.argsort(-np.abs(dth))[:4]
    directions = [dth / np.linalg.norm(dth)] + [np.eye(len(th0))[k] for k in top]
    names = ["adjoint_direction"] + [f"axis_{int(k)}" for k in top]
    fd = []
    for v, nm in zip(directions, names):
        Ls = []
        for sgn in (1.0, -1.0):
            pp, nn = SO.sh_cloud(th0 + sgn * EPS * v, dirs, float32=False)
            ph, _ = SO.phi_at_queries(pp, nn, q, BBOX, RES, workers, frozen_bins=bins)
            Ls.append(SO.loss(ph, phi_t))
        fd.append((Ls[0] - Ls[1]) / (2 * EPS))
        print(f"{nm}: fd={fd[-1]:.8e} adjoint={float(dth @ v):.8e} ({time.time() - t0:.0f} s)", flush=True)
    out = {
        "what": "central FD (step 1e-4, frozen central cells, FP64 points) of the C3 loss along each direction, "
                "and the oracle adjoint dL/dtheta at the base point (float32 points)",
        "written_by": "tests/golden/make_c3_fd.py (oracle only)",
        "workload": "synth.config_inputs('shopt128'): degree-6 SH body, 100k fixed directions, 128^3, "
                    "500k queries (seed 2002), target theta from the same seed",
        "eps": EPS, "loss_base": L0, "names": names,
        "directions": [list(map(float, v)) for v in directions],
        "fd": [float(x) for x in fd],
        "oracle_dtheta": [float(x) for x in dth],
    }
    with open(os.path.join(HERE, "c3_theta_fd.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1)

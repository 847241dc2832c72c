"""Write the stored expected values of tests/golden/ from the FP64 oracle alone.

    python tests/golden/make_golden.py

Fixtures (JSON, one per case):
  cube_n8.json      unit-cube conductor (edge 1 cm, 6 x 8 x 8 squares, 1 V): capacitance
                    and potential / field at fixed points; beside it the literature value
                    of the unit cube's capacitance, 0.6607 * 4 pi eps0 * a, which a
                    constant-element 8 x 8 mesh approaches from below (the oracle pins
                    check the refinement sequence).
  thgem_small.json  a small THGEM cell (24 sectors, 5 x 5 copies, dielectric FR4):
                    charge densities of sampled elements and potential / field at fixed
                    points.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2606_24154_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

CUBE_POINTS = [[0.0, 0.0, 0.0], [0.012, 0.0, 0.0], [0.007, 0.006, -0.004], [-0.015, 0.011, 0.019],
               [0.0051, 0.0, 0.0], [0.003, 0.0049, 0.0]]
THGEM_POINTS = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.3e-3], [0.2e-3, 0.1e-3, -0.1e-3], [0.4e-3, -0.2e-3, 1.5e-3],
                [-0.3e-3, 0.25e-3, -2.0e-3], [0.1e-3, 0.0, 0.27e-3]]


def small_thgem():
    return I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)


def main():
    g = I.cube(n_per_edge=8)
    sigma, _, _ = O.solve(g)
    _, _, area = O.centroids(g)
    C = float((sigma * area).sum())  # one conductor at 1 V
    phi, E = O.eval_points(g, sigma, np.array(CUBE_POINTS))
    cube = {"case": "unit cube, edge 0.01 m, 6 x 8 x 8 squares, 1 V, no images",
            "capacitance_F": C, "capacitance_over_4pi_eps0_a": C / (4 * np.pi * O.eps0() * 0.01),
            "literature_unit_cube_capacitance_over_4pi_eps0_a": 0.6607,
            "points_m": CUBE_POINTS, "phi_V": phi.tolist(), "E_V_per_m": E.tolist()}
    with open(os.path.join(HERE, "cube_n8.json"), "w") as f:
        json.dump(cube, f, indent=1)

    g = small_thgem()
    sigma, _, _ = O.solve(g)
    idx = list(range(0, g.n, max(1, g.n // 24)))
    phi, E = O.eval_points(g, sigma, np.array(THGEM_POINTS))
    thgem = {"case": "THGEM cell, PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3, images -2..2",
             "n_elements": g.n, "element_index": idx, "sigma_C_per_m2": sigma[idx].tolist(),
             "points_m": THGEM_POINTS, "phi_V": phi.tolist(), "E_V_per_m": E.tolist()}
    with open(os.path.join(HERE, "thgem_small.json"), "w") as f:
        json.dump(thgem, f, indent=1)


if __name__ == "__main__":
    main()

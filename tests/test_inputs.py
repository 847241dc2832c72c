"""The seeded synthetic inputs follow their stated recipe: the workload geometries (element
counts and kinds, conductors, dielectric interfaces, the 5 x 5 image range on the
hexagonal lattice), points uniform in the cell, the carrier cloud (in gas, half +e and
half -e, sigma 0.1 mm), and the serving trace (Poisson arrivals at 2000/s, sizes
log-uniform in [1e2, 1e6], uniform geometry ids).  Seeds reproduce exactly.  The module
itself holds no method arithmetic: it imports neither the oracle nor the CUDA path.
CPU only."""
import ast
import math
import os

import numpy as np
from scipy import stats

from paper_2606_24154_gb300 import inputs as I


def _areas(g):
    v = g.elements["v"]
    kind = g.elements["kind"]
    a = 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1)
    four = kind != I.KIND_TRI
    a[four] += 0.5 * np.linalg.norm(np.cross(v[four, 2] - v[four, 0], v[four, 3] - v[four, 0]), axis=1)
    return a


def test_workload_geometries():
    c = I.cube(n_per_edge=8)
    assert c.n == 384 and (c.elements["kind"] == I.KIND_RECT).all()
    assert abs(_areas(c).sum() - 6 * 0.01 ** 2) <= 1e-15
    g = I.thgem()
    kind, bc = g.elements["kind"], g.elements["bc"]
    assert g.n == 9996
    assert (kind == I.KIND_RECT).sum() == 2112 and (kind == I.KIND_TRI).sum() == 7884
    assert g.img_lo == -2 and g.img_hi == 2 and g.n_images == 25
    assert np.allclose(g.lattice, [[1e-3, 0, 0], [0.5e-3, 0.5e-3 * math.sqrt(3.0), 0]], rtol=0, atol=1e-18)
    # FR4 hole wall: 96 facets x 18 rows, FR4 (4.4) on the -n side
    diel = bc == I.BC_DIELECTRIC
    assert diel.sum() == 96 * 18
    assert (g.elements["eps_a"][diel] == 4.4).all() and (g.elements["eps_b"][diel] == 1.0).all()
    assert set(np.unique(g.elements["conductor"][~diel])) == {0, 1, 2, 3} and len(g.voltages) == 4
    assert (_areas(g) > 0).all()
    # each Cu face covers the hexagonal cell minus the hole: its elements tile that area
    hex_area = math.sqrt(3.0) / 2.0 * 1e-3 ** 2
    top = (~diel) & (g.elements["conductor"] == 0) & np.all(np.isclose(g.elements["v"][:, :3, 2], 0.285e-3), axis=1)
    assert abs(_areas(g)[top].sum() - (hex_area - 96 / 2 * 0.25e-3 ** 2 * math.sin(2 * math.pi / 96))) <= 1e-12 * hex_area
    d = I.double_thgem()
    assert d.n == 40368 and len(d.voltages) == 6 and d.n_images == 25


def test_cell_points_uniform_in_the_prism_and_seeded():
    g = I.thgem()
    p = I.cell_points(g, 200_000, I.rng(1, 0))
    assert p.shape == (200_000, 3) and p.flags["C_CONTIGUOUS"]
    x, y, z = p.T
    s3 = math.sqrt(3.0) / 2.0
    h = 0.5e-3
    assert (np.abs(x) <= h).all() and (np.abs(0.5 * x + s3 * y) <= h).all() and (np.abs(-0.5 * x + s3 * y) <= h).all()
    assert (z >= g.z_range[0]).all() and (z <= g.z_range[1]).all()
    # uniform: each coordinate's mean is the prism's centre, within 5 standard errors
    for col, half in ((x, h), (y, h / s3), (z, g.z_range[1])):
        assert abs(col.mean()) <= 5 * half / math.sqrt(3 * col.size)
    assert stats.kstest((z - g.z_range[0]) / (g.z_range[1] - g.z_range[0]), "uniform").pvalue > 1e-4
    assert np.array_equal(p, I.cell_points(g, 200_000, I.rng(1, 0)))
    assert not np.array_equal(p[:10], I.cell_points(g, 10, I.rng(1, 1)))


def test_carrier_cloud_in_gas_neutral_and_sized():
    g = I.thgem()
    pos, q = I.carrier_cloud(g, 100_000, I.rng(3, 0))
    assert not I.in_solid(g, pos).any()
    assert (q == I.E_CHARGE).sum() == 50_000 and (q == -I.E_CHARGE).sum() == 50_000
    # z is not clipped by the hole (FR4 spans +-0.25 mm, the hole radius is 0.25 mm):
    # its spread is the Gaussian's, 0.1 mm
    assert abs(pos[:, 2].std() - 0.1e-3) <= 0.005e-3
    assert np.abs(pos.mean(axis=0)).max() <= 5 * 0.1e-3 / math.sqrt(pos.shape[0])


def test_serving_trace():
    n = 20_000
    t, sizes, geo = I.serving_trace(n, I.rng(4, 0))
    assert t[0] == 0.0 and (np.diff(t) >= 0).all()
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000.0) <= 5 * (1 / 2000.0) / math.sqrt(gaps.size)
    assert stats.kstest(gaps, "expon", args=(0, 1 / 2000.0)).pvalue > 1e-4
    assert sizes.min() >= 100 and sizes.max() <= 1_000_000
    u = (np.log(sizes + 0.5) - math.log(100)) / (math.log(1_000_000) - math.log(100))
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    counts = np.bincount(geo, minlength=3)
    assert counts.size == 3 and np.abs(counts - n / 3).max() <= 5 * math.sqrt(n / 3)


def test_inputs_module_has_no_method_imports():
    src = open(os.path.join(os.path.dirname(I.__file__), "inputs.py")).read()
    names = set()
    for node in ast.walk(ast.parse(src)):
        if isinstance(node, ast.Import):
            names |= {a.name for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            names.add(node.module or "")
    assert names <= {"__future__", "math", "dataclasses", "numpy"}, names

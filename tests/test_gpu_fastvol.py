"""FastVolume maps (Sec. 3.3): node values from the evaluation kernels, trilinear lookup,
against the oracle's map; exact at the nodes; stale maps refused."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2606_24154_gb300 import build, nebem
    build.build()
    nebem.load()
    return nebem


def graded_axis(lo, hi, n, focus, strength=3.0):
    """Nodes packed towards `focus` (a graded FastVolume axis)."""
    u = np.linspace(-1.0, 1.0, n)
    f = (focus - lo) / (hi - lo) * 2 - 1
    v = f + (u - f) * np.abs(u - f) ** (strength - 1) / np.max(np.abs(np.array([-1, 1]) - f)) ** (strength - 1)
    v = np.sort(np.clip(v, -1, 1))
    v[0], v[-1] = -1.0, 1.0
    v = np.unique(v)
    return lo + (v + 1) / 2 * (hi - lo)


def test_fastvol_matches_oracle_map_and_nodes(N):
    g = I.cube(n_per_edge=8)
    sig, _, _ = O.solve(g)
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sig)
    # no node on a cube face (+-5 mm) or on an element edge (multiples of 1.25 mm):
    # the in-plane field diverges logarithmically on an edge
    ax = graded_axis(-0.02, 0.02, 13, 0.0) + 0.37e-3
    ay = np.linspace(-0.02, 0.02, 9) + 0.21e-3
    az = np.linspace(-0.018, 0.022, 11)
    N.nebem_fastvol_build(ctx.h, ax, ay, az, N.NEBEM_FP64)
    gen = np.random.default_rng(5)
    pts = np.concatenate([gen.uniform(-0.025, 0.025, (200, 3)),            # incl. outside the box
                          np.stack(np.meshgrid(ax[:3], ay[-2:], az[4:6], indexing="ij"), -1).reshape(-1, 3)])
    phi, E = N.nebem_fastvol_eval(ctx.h, pts)
    rphi, rE = O.fastvol(g, sig, ax, ay, az, pts)
    assert np.abs(phi - rphi).max() <= 1e-10 * np.abs(rphi).max()
    assert np.abs(E - rE).max() <= 1e-10 * np.abs(rE).max()
    # at the nodes the map returns the direct evaluation bit for bit
    nodes = pts[200:]
    dphi, dE = ctx.eval(nodes, N.NEBEM_FP64)
    assert np.array_equal(phi[200:], dphi) and np.array_equal(E[200:], dE)
    # a new charge density makes the map stale
    ctx.set_sigma(sig * 2)
    with pytest.raises(N.NebemError) as e:
        N.nebem_fastvol_eval(ctx.h, pts[:3])
    assert e.value.code == N.NEBEM_BAD_STATE


def test_fastvol_thgem_accuracy_against_direct(N):
    """A THGEM map (mixed node values) on a grid graded towards the foil: interpolation
    error against the direct evaluation in the drift region, reported and bounded."""
    g = I.thgem()
    ctx = N.Context().set_geometry(g)
    ctx.solve(N.NEBEM_MIXED)
    p = g.pitch
    ax = np.linspace(-0.5 * p, 0.5 * p, 41)
    ay = np.linspace(-p / np.sqrt(3), p / np.sqrt(3), 47)
    az = np.concatenate([np.linspace(g.z_range[0], -0.6e-3, 30), np.linspace(-0.59e-3, 0.59e-3, 60),
                         np.linspace(0.6e-3, g.z_range[1], 30)])
    N.nebem_fastvol_build(ctx.h, ax, ay, az, N.NEBEM_MIXED)
    pts = I.cell_points(g, 4000, I.rng(1, 40))
    drift = pts[(pts[:, 2] > 1.2e-3) & (pts[:, 2] < 3.0e-3)]
    phi, E = N.nebem_fastvol_eval(ctx.h, drift)
    dphi, dE = ctx.eval(drift, N.NEBEM_MIXED)
    rel = np.linalg.norm(E - dE, axis=1) / np.linalg.norm(dE, axis=1)
    assert np.median(rel) < 2.5e-3 and np.abs(phi - dphi).max() < 2.5e-3 * np.abs(dphi).max()

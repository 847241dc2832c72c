"""Parity at the full sizes of the benchmark workloads, in the launch configurations the
benchmark times (all points / carriers in one call), checked against the oracle on
sampled outputs or through properties that hold at any size:

  - THGEM cell, 1e6 points, mixed evaluation (with its refinement): 200 sampled points
    against the oracle, normwise and per point;
  - double THGEM (40,368 elements), mixed solve (FP32 tensor-core LU + FP64 refinement):
    the residual of sampled rows of the oracle's own matrix times the GPU's charge
    densities;
  - dynamic space charge, 1e6 carriers, one mixed step with point charges and one with
    line charges: the field at sampled carriers (recovered from their displacement
    x1 - x0 = sign(q) mu E dt) against the oracle's element sum plus carrier / line sum.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def N():
    from paper_2606_24154_gb300 import build, nebem
    build.build()
    nebem.load()
    return nebem


@pytest.fixture(scope="module")
def thgem_solved(N):
    g = I.thgem()
    ctx = N.Context().set_geometry(g)
    sigma, _, _ = ctx.solve(N.NEBEM_MIXED)
    return g, ctx, sigma


def rel_norm(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def test_headline_eval_1e6_points_sampled(N, thgem_solved):
    g, ctx, sigma = thgem_solved
    pts = I.cell_points(g, 1_000_000, I.rng(1, 0))
    phi, E = ctx.eval(pts, N.NEBEM_MIXED)
    idx = I.rng(1, 90).choice(pts.shape[0], 200, replace=False)
    rphi, rE = O.eval_points(g, sigma, pts[idx])
    assert rel_norm(phi[idx], rphi) <= TOL_MIXED
    assert rel_norm(E[idx], rE) <= TOL_MIXED
    # per point, with the floor 1e-6 of the largest value (E as a vector)
    r = np.abs(rphi)
    assert (np.abs(phi[idx] - rphi) / np.maximum(r, 1e-6 * r.max())).max() <= TOL_MIXED
    m = np.linalg.norm(rE, axis=1)
    assert (np.linalg.norm(E[idx] - rE, axis=1) / np.maximum(m, 1e-6 * m.max())).max() <= TOL_MIXED


def test_double_thgem_solve_residual_on_oracle_rows(N):
    """sum_j K_ij sigma_j = b_i on sampled rows, K_ij from the oracle entry by entry; the
    refinement stops at |d sigma| / |sigma| <= 1e-8, so the residual relative to the
    row's sum of |terms| is bounded by about 1e-8 times the row's conditioning."""
    g = I.double_thgem()
    ctx = N.Context().set_geometry(g)
    sigma, info, _ = ctx.solve(N.NEBEM_MIXED)
    rows = I.rng(2, 91).choice(g.n, 24, replace=False)
    b = O.rhs(g)
    cols = np.arange(g.n)
    worst = 0.0
    for i in rows:
        K_i = O.fill_entries(g, np.full(g.n, i), cols)
        terms = K_i * sigma
        r = terms.sum() - b[i]
        worst = max(worst, abs(r) / np.abs(terms).sum())
    assert worst <= 1e-9, worst


def _step_field(N, ctx, pos, q, mu, dt):
    out = N.nebem_step(ctx.h, 1, mu, dt, N.NEBEM_MIXED, pos.shape[0])
    return (out - pos) / (np.sign(q)[:, None] * mu * dt)


@pytest.mark.parametrize("mode", ["points", "lines"])
def test_dynamic_step_1e6_carriers_sampled(N, thgem_solved, mode):
    g, ctx, _ = thgem_solved
    pos, q = I.carrier_cloud(g, 1_000_000, I.rng(3, 0))
    voxel = np.array([20e-6, 20e-6, 40e-6])

    def load():
        N.nebem_space_charge(ctx.h, pos, q, 1e-6)
        if mode == "lines":
            N.nebem_space_charge_lines(ctx.h, voxel)

    # the densities of this charge set: a mixed solve forms the known-charge RHS in mixed
    # precision, as the step does, so the step's own solve reproduces them
    load()
    sig, _, _ = ctx.solve(N.NEBEM_MIXED)
    load()
    E = _step_field(N, ctx, pos, q, 1e-4, 1e-9)
    idx = I.rng(3, 92).choice(pos.shape[0], 48, replace=False)
    _, rE = O.eval_points(g, sig, pos[idx])
    if mode == "points":
        for k, i in enumerate(idx):
            keep = np.ones(pos.shape[0], bool)
            keep[i] = False
            _, Es = O.space_charge(pos[keep], q[keep], tgt=pos[i:i + 1], soft=1e-6)
            rE[k] += Es[0]
    else:
        _, El = O.line_charge(O.voxel_lines(pos, q, voxel), pos[idx])
        rE += El
    assert rel_norm(E[idx], rE) <= TOL_MIXED, rel_norm(E[idx], rE)

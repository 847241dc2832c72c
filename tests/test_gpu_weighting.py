"""Weighting fields (Sec. 2.1): the influence matrix does not depend on the voltages, so the
weighting field of a readout conductor (unit potential on it, 0 on every other conductor,
no known charges) is a solve of a unit right-hand side with the retained factors.
nebem_weighting_fields solves k of them through each triangular sweep together; each
column must equal the single solve of its unit voltages bit for bit, and the oracle's LU
solution to the FP64 solve tolerance.  The weighting-field FastVolume maps (Sec. 3.3) are
checked against the oracle's map of the same densities."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module")
def N():
    from paper_2606_24154_gb300 import build, nebem
    build.build()
    nebem.load()
    return nebem


def small_thgem():
    return I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)


def rel_norm(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def unit(g, c):
    v = np.zeros(len(g.voltages))
    v[c] = 1.0
    return v


# nine readouts (repeats included): two passes of the eight-column sweep
READOUT = [0, 1, 2, 3, 0, 2, 1, 3, 3]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_multi_rhs_columns_equal_single_solves_and_oracle(N, prec):
    g = small_thgem()
    p = N.NEBEM_FP64 if prec == "fp64" else N.NEBEM_MIXED
    ctx = N.Context().set_geometry(g)
    W, info, _ = N.nebem_weighting_fields(ctx.h, READOUT, p, g.n)
    assert W.shape == (g.n, len(READOUT))
    K = O.fill(g)
    fac = O.lu_factor(K)
    # scale-free residual of every column, |K w - b| against |K| |w|: FP64 rounding for the
    # FP64 solve; the refinement's stopping point (corrections below 1e-8) for mixed
    B = np.stack([O.rhs(g, unit(g, r)) for r in READOUT], axis=1)
    scale = np.abs(K).sum(axis=1).max() * np.abs(W).max(axis=0)
    tol_r = 1e-12 if prec == "fp64" else 1e-8
    assert (np.abs(K @ W - B).max(axis=0) <= tol_r * scale).all()
    assert np.isfinite(info.residual) and info.residual > 0.0
    for c in range(len(g.voltages)):
        N.nebem_set_bc(ctx.h, unit(g, c))
        single, _, _ = ctx.solve(p)
        ref = O.lu_solve(fac, O.rhs(g, unit(g, c)))
        tol = TOL64 if prec == "fp64" else 1e-8
        assert rel_norm(single, ref) <= tol
        for j, r in enumerate(READOUT):
            if r == c:
                # the multi-column sweeps do each column's arithmetic in the single sweep's order
                assert np.array_equal(W[:, j], single), (c, j, rel_norm(W[:, j], single))


def test_weighting_potential_is_one_on_the_readout_and_zero_on_the_others(N):
    """The defining property (Sec. 2.1): the weighting potential of readout r, evaluated at the
    collocation points, is 1 on r's elements and 0 on every other conductor's."""
    g = small_thgem()
    ctx = N.Context().set_geometry(g)
    W, _, _ = N.nebem_weighting_fields(ctx.h, [0, 1, 2, 3], N.NEBEM_FP64, g.n)
    c, _, _ = O.centroids(g)
    cond = g.elements["bc"] == 0
    for r in range(4):
        ctx.set_sigma(W[:, r])
        phi, _ = ctx.eval(c[cond], N.NEBEM_FP64)
        want = (g.elements["conductor"][cond] == r).astype(float)
        assert np.abs(phi - want).max() <= 1e-9, (r, np.abs(phi - want).max())


def test_context_state_is_left_unchanged(N):
    g = small_thgem()
    ctx = N.Context().set_geometry(g)
    sig0, _, _ = ctx.solve(N.NEBEM_FP64)
    pts = I.cell_points(g, 16, I.rng(0, 70))
    phi0, E0 = ctx.eval(pts, N.NEBEM_FP64)
    N.nebem_weighting_fields(ctx.h, [1, 3], N.NEBEM_FP64, g.n)
    N.nebem_weighting_fastvol_build(ctx.h, [2], np.linspace(-4e-4, 4e-4, 3) + 1.3e-7,
                                    np.linspace(-4e-4, 4e-4, 3) + 2.9e-7, np.linspace(1e-3, 2e-3, 3) + 3.1e-7,
                                    N.NEBEM_FP64)
    assert np.array_equal(ctx.sigma(), sig0)
    phi1, E1 = ctx.eval(pts, N.NEBEM_FP64)
    assert np.array_equal(phi1, phi0) and np.array_equal(E1, E0)
    # the voltages too: a new solve gives the same densities
    sig1, _, _ = ctx.solve(N.NEBEM_FP64)
    assert np.array_equal(sig1, sig0)


def _axes(g):
    """A small grid over one cell, offset so that no node lies on an element edge."""
    p = g.pitch
    ax = np.linspace(-0.5 * p, 0.5 * p, 7) + 1.37e-7
    ay = np.linspace(-0.5 * p, 0.5 * p, 6) + 2.91e-7
    az = np.concatenate([np.linspace(g.z_range[0], -0.7e-3, 3), np.linspace(0.7e-3, g.z_range[1], 4)]) + 3.17e-7
    return ax, ay, az


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_weighting_maps_match_the_oracle_map(N, prec):
    g = small_thgem()
    p = N.NEBEM_FP64 if prec == "fp64" else N.NEBEM_MIXED
    ctx = N.Context().set_geometry(g)
    readout = [3, 1]
    ax, ay, az = _axes(g)
    maps, info = N.nebem_weighting_fastvol_build(ctx.h, readout, ax, ay, az, p)
    W, _, _ = N.nebem_weighting_fields(ctx.h, readout, p, g.n)
    fac = O.lu_factor(O.fill(g))
    gen = np.random.default_rng(11)
    lo = np.array([ax[0], ay[0], az[0]]) - 1e-4
    hi = np.array([ax[-1], ay[-1], az[-1]]) + 1e-4
    pts = gen.uniform(lo, hi, (300, 3))  # a few outside the box: nearest point of the box
    for j, r in enumerate(readout):
        assert rel_norm(W[:, j], O.lu_solve(fac, O.rhs(g, unit(g, r)))) <= (TOL64 if prec == "fp64" else 1e-8)
        phi, E = maps[j].eval(pts)
        # the oracle's map of the same densities: node values by the FP64 closed forms,
        # the same trilinear rule
        rphi, rE = O.fastvol(g, W[:, j], ax, ay, az, pts)
        # FP64: the node evaluation to 1e-10; mixed: each node to 1e-6 (the refined mixed
        # evaluation), a convex combination of nodes to 1e-6 of the largest
        tol = 1e-10 if prec == "fp64" else 1e-6
        assert rel_norm(phi, rphi) <= tol, (r, rel_norm(phi, rphi))
        assert rel_norm(E, rE) <= tol, (r, rel_norm(E, rE))
    for m in maps:
        m.close()


def test_weighting_map_device_lookup_equals_host_lookup(N):
    import torch
    g = small_thgem()
    ctx = N.Context().set_geometry(g)
    ax, ay, az = _axes(g)
    maps, _ = N.nebem_weighting_fastvol_build(ctx.h, [2], ax, ay, az, N.NEBEM_FP64)
    pts = I.cell_points(g, 257, I.rng(0, 71))
    phi, E = maps[0].eval(pts)
    d_pts = torch.tensor(pts, device="cuda")
    d_phi = torch.empty(pts.shape[0], dtype=torch.float64, device="cuda")
    d_E = torch.empty((pts.shape[0], 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    maps[0].eval_device(d_pts.data_ptr(), pts.shape[0], d_phi.data_ptr(), d_E.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    assert np.array_equal(d_phi.cpu().numpy(), phi) and np.array_equal(d_E.cpu().numpy(), E)


def test_weighting_sweep_wait_runs_out_then_solves(N):
    """A poll limit of 1: a 64-row block's wait in the multi-column sweep gives up, the call
    returns NEBEM_TIMEOUT with NaN in that block; the context's own densities are not touched,
    and with the default limit the same factors give the weighting fields."""
    g = I.cube(n_per_edge=8)
    ctx = N.Context(wait_polls=1).set_geometry(g)
    N.nebem_set_bc(ctx.h, g.voltages)
    out = np.full((1, g.n), 7.0)
    info = N.nebem_solve_info()
    rc = N.load().nebem_weighting_fields(ctx.h, (C.c_int32 * 1)(0), 1, N.NEBEM_FP64,
                                         out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info))
    assert rc == N.NEBEM_TIMEOUT, (rc, N.load().nebem_last_error())
    assert np.isnan(out).any()
    N.nebem_set_wait_polls(ctx.h, 0)
    W, _, _ = N.nebem_weighting_fields(ctx.h, [0], N.NEBEM_FP64, g.n)
    ref, _, _ = O.solve(g, unit(g, 0))
    assert rel_norm(W[:, 0], ref) <= TOL64


def test_weighting_arguments_checked(N):
    g = small_thgem()
    ctx = N.Context().set_geometry(g)
    for readout in ([], [4], [-1], list(range(4)) * 17):  # k = 0, no such conductor, k = 68
        with pytest.raises(N.NebemError) as e:
            N.nebem_weighting_fields(ctx.h, readout, N.NEBEM_FP64, g.n)
        assert e.value.code == N.NEBEM_INVALID_ARG
    with pytest.raises(N.NebemError) as e:
        N.nebem_weighting_fields(ctx.h, [0], 7, g.n)
    assert e.value.code == N.NEBEM_INVALID_ARG
    empty = N.Context()
    with pytest.raises(N.NebemError) as e:
        N.nebem_weighting_fields(empty.h, [0], N.NEBEM_FP64, 1)
    assert e.value.code == N.NEBEM_BAD_STATE

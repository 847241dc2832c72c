"""Adaptive Modelling (Sec. 3.3, PrimAfter) through the C-ABI against the oracle: near
copies by elements, distant copies (ring index > PrimAfter) by whole primitives with
their average densities.  FP64 <= 1e-10, mixed <= 1e-6 (per quantity, normwise)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def N():
    from paper_2606_24154_gb300 import build, nebem
    build.build()
    nebem.load()
    return nebem


def rel_norm(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def small(lo=-3, hi=3):
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    g.img_lo, g.img_hi = lo, hi
    return g


def smooth_sigma(g):
    c, _, _ = O.centroids(g)
    return 1e-9 * (1.0 + 0.5 * np.sin(7e3 * c[:, 0]) * np.cos(5e3 * c[:, 1]) + 3e2 * c[:, 2])


@pytest.mark.parametrize("prim_after", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_am_parity(N, prim_after, prec):
    g = small()
    sigma = smooth_sigma(g)
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    N.nebem_set_primitives(ctx.h, g.primitives, g.prim_of, prim_after)
    pts = I.cell_points(g, 300, I.rng(1, 70))
    p = N.NEBEM_FP64 if prec == "fp64" else N.NEBEM_MIXED
    phi, E = ctx.eval(pts, p)
    rphi, rE = O.eval_am(g, sigma, g.primitives, g.prim_of, prim_after, pts)
    tol = TOL64 if prec == "fp64" else TOL_MIXED
    assert rel_norm(phi, rphi) <= tol, rel_norm(phi, rphi)
    assert rel_norm(E, rE) <= tol, rel_norm(E, rE)


def test_am_off_and_far_ring_is_plain_evaluation(N):
    g = small(-2, 2)
    sigma = smooth_sigma(g)
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    pts = I.cell_points(g, 200, I.rng(1, 71))
    plain = ctx.eval(pts, N.NEBEM_MIXED)
    for pa in (-1, 2, 5):  # off, and no copy beyond ring 2
        N.nebem_set_primitives(ctx.h, g.primitives, g.prim_of, pa)
        phi, E = ctx.eval(pts, N.NEBEM_MIXED)
        assert np.array_equal(phi, plain[0]) and np.array_equal(E, plain[1])


def test_am_follows_sigma_and_free_elements(N):
    """The primitives' densities follow every change of sigma; elements without a
    primitive stand for themselves in the distant copies."""
    g = small()
    ctx = N.Context().set_geometry(g)
    po = g.prim_of.copy()
    po[po < 30] = -1
    keep = np.unique(po[po >= 0])
    remap = -np.ones(len(g.primitives), dtype=np.int32)
    remap[keep] = np.arange(len(keep))
    po2 = np.where(po >= 0, remap[np.maximum(po, 0)], -1).astype(np.int32)
    N.nebem_set_primitives(ctx.h, g.primitives[keep], po2, 1)
    pts = I.cell_points(g, 100, I.rng(1, 72))
    for scale in (1.0, -3.0):
        sigma = scale * smooth_sigma(g)
        ctx.set_sigma(sigma)
        phi, E = ctx.eval(pts, N.NEBEM_FP64)
        rphi, rE = O.eval_am(g, sigma, g.primitives[keep], po2, 1, pts)
        assert rel_norm(phi, rphi) <= TOL64 and rel_norm(E, rE) <= TOL64


def test_am_full_thgem_121_images_sampled(N):
    """The full THGEM cell with 11 x 11 copies, solved, then evaluated with PrimAfter = 1
    (9 copies by elements, 112 by primitives) on sampled points in mixed precision."""
    g = I.thgem()
    g.img_lo, g.img_hi = -5, 5
    ctx = N.Context().set_geometry(g)
    sigma, _, _ = ctx.solve(N.NEBEM_MIXED)
    N.nebem_set_primitives(ctx.h, g.primitives, g.prim_of, 1)
    pts = I.cell_points(g, 48, I.rng(1, 73))
    phi, E = ctx.eval(pts, N.NEBEM_MIXED)
    rphi, rE = O.eval_am(g, sigma, g.primitives, g.prim_of, 1, pts)
    assert rel_norm(phi, rphi) <= TOL_MIXED and rel_norm(E, rE) <= TOL_MIXED


def test_am_errors(N):
    g = small(-2, 2)
    ctx = N.Context()
    with pytest.raises(N.NebemError) as e:
        N.nebem_set_primitives(ctx.h, g.primitives, g.prim_of, 1)
    assert e.value.code == N.NEBEM_BAD_STATE
    ctx.set_geometry(g)
    bad = g.prim_of.copy()
    bad[0] = len(g.primitives)
    with pytest.raises(N.NebemError) as e:
        N.nebem_set_primitives(ctx.h, g.primitives, bad, 1)
    assert e.value.code == N.NEBEM_INVALID_ARG
    bad = g.prim_of.copy()
    bad[0] = bad[1] if bad[1] != bad[0] else bad[0] + 1  # breaks the tiling of two primitives
    with pytest.raises(N.NebemError) as e:
        N.nebem_set_primitives(ctx.h, g.primitives, bad, 1)
    assert e.value.code == N.NEBEM_INVALID_ARG
    moved = g.primitives.copy()
    moved["v"][0, :, 2] += 1e-5  # primitive 0 lifted out of its elements' plane
    with pytest.raises(N.NebemError) as e:
        N.nebem_set_primitives(ctx.h, moved, g.prim_of, 1)
    assert e.value.code == N.NEBEM_INVALID_ARG

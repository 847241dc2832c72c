"""Mixed-precision influence-matrix fill (Eq. Matrix: far pairs by Gauss rules in two-float
arithmetic, pairs nearer than 6 element radii by the FP64 closed forms) against the oracle's
FP64 fill, entry by entry, and the mixed solve built on it.

Tolerance.  Per (element, image) pair the Gauss rules' truncation error stays below ~3e-12
of the pair at their distance tiers, and the two-float arithmetic adds ~2e-13.  The oracle's
closed form itself carries rounding noise that grows with the distance in element radii
(about (d/rho)^2 x 1.3e-15 for the potential, from cancellation among the edge terms); on
these geometries the GPU's own FP64 fill differs from the oracle by up to 9e-12 per entry
for that reason.  Conductor rows (positive potential terms) are compared entry by entry
relative to the entry; interface rows (normal-field terms of both signs, some entries
cancelling to ~0) relative to max(|entry|, 1e-3 x the row's largest entry).  Bound 5e-11."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_ENTRY = 5e-11


@pytest.fixture(scope="module")
def N():
    from paper_2606_24154_gb300 import build, nebem
    build.build()
    nebem.load()
    return nebem


GEOMS = {
    "cube": lambda: I.cube(n_per_edge=8),
    # FR4 hole wall (interface rows), rectangles and triangles, 5 x 5 copies
    "thgem_small": lambda: I.thgem(I.PlateSpec(n_phi=32, n_r=4, n_zf=6, n_zc=1), n_plane=5),
    # exposed FR4 rims: interface rows on annuli (triangles / quadrilateral sectors)
    "thgem_rim": lambda: I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zf=4, n_zc=1, rim=0.1e-3, n_rim=2), n_plane=4),
}


def entry_errors(K, R, bc):
    rowmax = np.abs(R).max(axis=1, keepdims=True)
    cond = bc == I.BC_CONDUCTOR
    e_cond = np.abs(K[cond] - R[cond]) / np.abs(R[cond])  # potential terms are all > 0
    e_if = np.abs(K[~cond] - R[~cond]) / np.maximum(np.abs(R[~cond]), 1e-3 * rowmax[~cond])
    return (e_cond.max() if e_cond.size else 0.0), (e_if.max() if e_if.size else 0.0)


@pytest.mark.parametrize("name", list(GEOMS))
def test_mixed_fill_entries_match_oracle(N, name):
    g = GEOMS[name]()
    ctx = N.Context().set_geometry(g)
    K = ctx.fill(N.NEBEM_MIXED)
    R = O.fill(g)
    ec, ei = entry_errors(K, R, g.elements["bc"])
    assert ec <= TOL_ENTRY, ec
    assert ei <= TOL_ENTRY, ei
    # the diagonal (self pair, principal value, interface term) comes from the FP64 part
    d = np.diag(K) - np.diag(R)
    assert (np.abs(d) / np.abs(np.diag(R))).max() <= 1e-12


def test_mixed_fill_quadrilaterals(N):
    """Planar convex quadrilaterals (tensor rules on the bilinear map) next to rectangles and
    triangles: the THGEM's primitives taken as elements, one conductor, 5 x 5 copies."""
    g0 = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    g = I.Geometry(name="thgem_primitives", elements=g0.primitives.copy(), voltages=np.array([1.0]),
                   lattice=g0.lattice, img_lo=-2, img_hi=2, pitch=g0.pitch, z_range=g0.z_range)
    ctx = N.Context().set_geometry(g)
    K = ctx.fill(N.NEBEM_MIXED)
    R = O.fill(g)
    ec, _ = entry_errors(K, R, g.elements["bc"])
    assert ec <= TOL_ENTRY, ec


def test_mixed_fill_wide_image_range(N):
    """11 x 11 copies (the largest image table; smaller column tiles in shared memory) on
    a coarse cell: distant copies reach ~1000 element radii."""
    g = I.thgem(I.PlateSpec(n_phi=12, n_r=2, n_zc=1, n_zf=3), n_plane=2)
    ctx = N.Context()
    N.nebem_set_geometry(ctx.h, g.elements, g.lattice, -5, 5)
    g5 = I.Geometry(name="thgem_11x11", elements=g.elements, voltages=g.voltages, lattice=g.lattice, img_lo=-5,
                    img_hi=5, pitch=g.pitch, z_range=g.z_range)
    K = N.nebem_fill(ctx.h, N.NEBEM_MIXED, g.n)
    R = O.fill(g5)
    ec, ei = entry_errors(K, R, g.elements["bc"])
    # pairs at up to ~1000 radii: the oracle's own far-field noise is ~1e-9 there (Phi)
    assert ec <= 2e-9, ec
    assert ei <= 2e-9, ei


def test_mixed_solve_on_mixed_fill(N):
    """sigma of the mixed solve (mixed fill, FP32 LU, FP64 refinement) within 1e-8 of the
    oracle's FP64 solve.  An FP64 solve after it in the same context refills in FP64 (the
    same bits as in a fresh context), and that FP64 matrix then answers mixed requests."""
    g = GEOMS["thgem_small"]()
    ref, _, _ = O.solve(g)
    ctx = N.Context().set_geometry(g)
    sig, info, _ = ctx.solve(N.NEBEM_MIXED)
    assert np.abs(sig - ref).max() / np.abs(ref).max() <= 1e-8
    assert info.correction <= 1e-8
    fresh = N.Context().set_geometry(g)
    sig64_fresh, _, _ = fresh.solve(N.NEBEM_FP64)
    sig64, _, _ = ctx.solve(N.NEBEM_FP64)
    assert np.array_equal(sig64, sig64_fresh)
    assert np.array_equal(ctx.fill(N.NEBEM_MIXED), fresh.fill(N.NEBEM_FP64))

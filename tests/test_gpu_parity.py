"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances: FP64 mode <= 1e-10 relative (per quantity, normwise, plus a per-point
form with a floor of 1e-6 of the largest magnitude); image indexing bit-exact.
"""
import math

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


def rel_norm(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def rel_point(a, ref, floor=1e-6):
    """max_i |a_i - ref_i| / max(|ref_i|, floor * max|ref|), vectors per row."""
    a = np.asarray(a).reshape(len(a), -1)
    ref = np.asarray(ref).reshape(len(ref), -1)
    d = np.linalg.norm(a - ref, axis=1)
    m = np.linalg.norm(ref, axis=1)
    return float((d / np.maximum(m, floor * m.max())).max())


def small_thgem():
    return I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)


def random_elements(gen, n):
    el = np.zeros(n, I.ELEMENT_DTYPE)
    for i in range(n):
        if i % 2 == 0:
            c = gen.normal(size=3) * 1e-3
            u = gen.normal(size=3); u /= np.linalg.norm(u)
            w = np.cross(u, gen.normal(size=3)); w /= np.linalg.norm(w)
            L1, L2 = 1e-3 * gen.uniform(0.2, 1.5, 2)
            v0 = c - 0.5 * L1 * u - 0.5 * L2 * w
            el[i]["kind"] = I.KIND_RECT
            el[i]["v"] = [v0, v0 + L1 * u, v0 + L1 * u + L2 * w, v0 + L2 * w]
        else:
            el[i]["kind"] = I.KIND_TRI
            el[i]["v"][:3] = gen.normal(size=(3, 3)) * 1e-3
    return el


def test_element_influence_closed_form(N):
    gen = np.random.default_rng(101)
    el = random_elements(gen, 12)
    # axis-aligned rectangle and triangle for exact in-plane points
    ax = np.zeros(2, I.ELEMENT_DTYPE)
    ax[0]["kind"] = I.KIND_RECT
    ax[0]["v"] = [[-1e-3, -1e-3, 0], [1e-3, -1e-3, 0], [1e-3, 0.5e-3, 0], [-1e-3, 0.5e-3, 0]]
    ax[1]["kind"] = I.KIND_TRI
    ax[1]["v"][:3] = [[0, 0, 0], [2e-3, 0, 0], [0.5e-3, 1.5e-3, 0]]
    el = np.concatenate([el, ax])
    pts = np.concatenate([gen.normal(size=(40, 3)) * 2e-3, gen.normal(size=(10, 3)) * 0.3e-3,
                          gen.normal(size=(5, 3)) * 0.2,  # far
                          [[0.2e-3, -0.3e-3, 0.0], [3e-3, 0.1e-3, 0.0], [0.4e-3, 0.2e-3, 0.0],
                           [0.2e-3, -0.3e-3, 1e-14], [0.2e-3, -0.3e-3, -1e-14]]])
    ctx = N.Context()
    phi, E = N.nebem_element_influence(ctx.h, el, pts)
    worst = 0.0
    for e in range(el.shape[0]):
        rp, rE = O.influence(el[e:e + 1], pts)
        v = el[e]["v"][: (4 if el[e]["kind"] == I.KIND_RECT else 3)]
        c = v.mean(0)
        a = math.sqrt(np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0])))
        # both closed forms cancel in the far field: allowed error ~ eps (d/a)^2 (a 40-digit
        # reference shows each side within that bound at d/a ~ 600)
        d = np.linalg.norm(pts - c, axis=1)
        tol = 1e-12 + 2e-15 * (d / a) ** 2
        ep = np.abs(phi[e] - rp) / np.abs(rp)
        eE = np.linalg.norm(E[e] - rE, axis=1) / np.maximum(np.linalg.norm(rE, axis=1), 1e-300)
        inplane = np.abs(pts[:, 2]) == 0.0
        eE[inplane & (np.linalg.norm(rE, axis=1) < 1e-12)] = 0.0
        worst = max(worst, float((ep / tol).max()), float((eE / tol).max()))
    assert worst <= 1.0, worst


def test_image_table_bit_exact(N):
    g = I.thgem(I.PlateSpec(n_phi=12, n_r=1, n_zc=1, n_zf=2), n_plane=1)
    for lo, hi in [(-2, 2), (-5, 5), (0, 0), (-1, 3)]:
        ctx = N.Context()
        N.nebem_set_geometry(ctx.h, g.elements, g.lattice, lo, hi)
        t_gpu = N.nebem_image_table(ctx.h)
        t_or = O.image_table(g.lattice, lo, hi)
        assert t_gpu.shape == t_or.shape
        assert np.array_equal(t_gpu.view(np.uint64), t_or.view(np.uint64))


def test_fill_parity_cube(N):
    g = I.cube(n_per_edge=8)
    ctx = N.Context().set_geometry(g)
    K = ctx.fill()
    Kr = O.fill(g)
    assert rel_norm(K, Kr) <= 1e-13
    assert np.abs(K - Kr).max(axis=1).max() <= TOL64 * np.abs(Kr).max()


def test_fill_parity_thgem_images_and_dielectric(N):
    g = small_thgem()
    assert (g.elements["bc"] == I.BC_DIELECTRIC).any() and (g.elements["kind"] == I.KIND_RECT).any()
    ctx = N.Context().set_geometry(g)
    K = ctx.fill()
    Kr = O.fill(g)
    # per row: conductor rows (potential) and interface rows (normal field) differ in scale
    rowmax = np.abs(Kr).max(axis=1, keepdims=True)
    assert (np.abs(K - Kr) / rowmax).max() <= TOL64


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_parity_cube(N, prec):
    g = I.cube(n_per_edge=8)
    sig_r, K, fac = O.solve(g)
    ctx = N.Context().set_geometry(g)
    p = N.NEBEM_FP64 if prec == "fp64" else N.NEBEM_MIXED
    sig, info, rc = ctx.solve(p)
    tol = TOL64 if prec == "fp64" else 1e-8
    assert rel_norm(sig, sig_r) <= tol
    _, _, area = O.centroids(g)
    cap = (sig * area).sum() / (4 * math.pi * O.eps0() * 0.01)
    assert abs(cap - 0.6563946187799465) < 1e-9
    if prec == "mixed":
        assert 1 <= info.iterations <= 30 and info.correction <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_parity_thgem_small(N, prec):
    g = small_thgem()
    sig_r, K, fac = O.solve(g)
    ctx = N.Context().set_geometry(g)
    p = N.NEBEM_FP64 if prec == "fp64" else N.NEBEM_MIXED
    sig, info, rc = ctx.solve(p)
    tol = TOL64 if prec == "fp64" else 1e-8
    assert rel_norm(sig, sig_r) <= tol, rel_norm(sig, sig_r)


def test_eval_parity_cube_grid(N):
    g = I.cube(n_per_edge=8)
    sig_r, K, fac = O.solve(g)
    pts = I.cube_grid_points()
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sig_r)
    phi, E = ctx.eval(pts, N.NEBEM_FP64)
    rphi, rE = O.eval_points(g, sig_r, pts)
    # points on the cube faces are the principal-value test (in-plane normal field)
    assert rel_norm(phi, rphi) <= TOL64
    assert rel_norm(E, rE) <= TOL64
    assert rel_point(phi, rphi) <= 1e-9
    assert rel_point(E, rE) <= 1e-9


def test_eval_parity_thgem_full_geometry_sampled(N):
    """Full-size THGEM cell (about 10,000 elements, 25 images) with a seeded charge
    density; sampled points checked one by one against the oracle."""
    g = I.thgem()
    gen = I.rng(1, 7)
    sigma = gen.normal(size=g.n) * 1e-6
    pts = I.cell_points(g, 200, I.rng(1, 8))[:64]
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    phi, E = ctx.eval(pts, N.NEBEM_FP64)
    rphi, rE = O.eval_points(g, sigma, pts)
    assert rel_norm(phi, rphi) <= TOL64
    assert rel_norm(E, rE) <= TOL64


def test_eval_fp64_full_thgem_per_point_1000(N):
    """Full-size THGEM cell with its solved charge densities, 1,000 points against the
    oracle point by point: |d_i| / max(|ref_i|, 1e-6 max|ref|) <= 1e-10 for phi and for the
    field vector."""
    g = I.thgem()
    ctx = N.Context().set_geometry(g)
    sigma, _, _ = ctx.solve(N.NEBEM_MIXED)
    pts = I.cell_points(g, 1000, I.rng(1, 77))
    phi, E = ctx.eval(pts, N.NEBEM_FP64)
    rphi, rE = O.eval_points(g, sigma, pts)
    r = np.abs(rphi)
    assert (np.abs(phi - rphi) / np.maximum(r, 1e-6 * r.max())).max() <= TOL64
    m = np.linalg.norm(rE, axis=1)
    assert (np.linalg.norm(E - rE, axis=1) / np.maximum(m, 1e-6 * m.max())).max() <= TOL64


def test_eval_ragged_and_empty(N):
    g = small_thgem()
    sigma = I.rng(0, 3).normal(size=g.n)
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    for n in [0, 1, 127, 129, 300]:
        pts = I.cell_points(g, max(n, 1), I.rng(0, n))[:n]
        phi, E = ctx.eval(pts, N.NEBEM_FP64)
        if n:
            rphi, rE = O.eval_points(g, sigma, pts)
            assert rel_norm(phi, rphi) <= TOL64 and rel_norm(E, rE) <= TOL64


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_space_charge_parity(N, prec):
    g = I.thgem()
    pos, q = I.carrier_cloud(g, 3000, I.rng(3, 1))
    ctx = N.Context().set_geometry(g)
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    p = N.NEBEM_FP64 if prec == "fp64" else N.NEBEM_MIXED
    phi, E = N.nebem_space_charge_eval(ctx.h, pos, p, exclude_self=True)
    rphi, rE = O.space_charge(pos, q, soft=1e-6)
    tol = TOL64 if prec == "fp64" else 1e-6
    assert rel_norm(phi, rphi) <= tol, rel_norm(phi, rphi)
    assert rel_norm(E, rE) <= tol, rel_norm(E, rE)
    tgt = I.cell_points(g, 100, I.rng(3, 2))
    phi, E = N.nebem_space_charge_eval(ctx.h, tgt, p)
    rphi, rE = O.space_charge(pos, q, tgt=tgt, soft=1e-6)
    if prec == "fp64":
        assert rel_norm(phi, rphi) <= tol and rel_norm(E, rE) <= tol
    else:
        # Away from a net-neutral cloud the +/-e terms cancel: FP32 per-term accuracy
        # (~1e-7) bounds the error by the absolute sums ke sum |q| / r and ke sum |q| / r^2,
        # not by the (much smaller) result.
        absphi, _ = O.space_charge(pos, np.abs(q), tgt=tgt, soft=1e-6)
        d = tgt[:, None, :] - pos[None]
        r2 = (d * d).sum(2) + 1e-12
        absE = O.ke() * (np.abs(q)[None] / r2).sum(1)
        assert (np.abs(phi - rphi) / absphi).max() <= 3e-7
        assert (np.linalg.norm(E - rE, axis=1) / absE).max() <= 3e-7


def test_space_charge_large_target_sets_same_bits(N):
    """Target sets of >= 311,296 points take the four-targets-per-thread kernel: per target
    the same operations in the same order as the two-target kernel used for small sets, so
    the results agree bit for bit; with self exclusion, sampled carriers against the oracle."""
    g = I.cube(n_per_edge=2)
    pos, q = I.carrier_cloud(I.thgem(), 320_000, I.rng(3, 5))
    ctx = N.Context().set_geometry(g)
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    phi4, E4 = N.nebem_space_charge_eval(ctx.h, pos, N.NEBEM_MIXED)
    phi2, E2 = N.nebem_space_charge_eval(ctx.h, pos[:3000], N.NEBEM_MIXED)
    assert np.array_equal(phi4[:3000], phi2) and np.array_equal(E4[:3000], E2)
    phi, E = N.nebem_space_charge_eval(ctx.h, pos, N.NEBEM_MIXED, exclude_self=True)
    idx = I.rng(3, 6).choice(pos.shape[0], 12, replace=False)
    for i in idx:
        keep = np.ones(pos.shape[0], bool)
        keep[i] = False
        rphi, rE = O.space_charge(pos[keep], q[keep], tgt=pos[i:i + 1], soft=1e-6)
        # the +/-e terms cancel at a carrier of a net-neutral cloud: FP32 per-term accuracy
        # bounds the error by the sums of |terms| (as in test_space_charge_parity)
        absphi, _ = O.space_charge(pos[keep], np.abs(q[keep]), tgt=pos[i:i + 1], soft=1e-6)
        d = pos[i] - pos[keep]
        absE = O.ke() * (np.abs(q[keep]) / ((d * d).sum(1) + 1e-12)).sum()
        assert abs(phi[i] - rphi[0]) <= 3e-7 * absphi[0]
        assert np.linalg.norm(E[i] - rE[0]) <= 3e-7 * absE


def test_dynamic_step_parity(N):
    g = I.cube(n_per_edge=4)
    gen = np.random.default_rng(37)
    pos = gen.normal(size=(300, 3)) * 2e-3 + np.array([0.0, 0.0, 0.012])
    q = np.where(gen.random(300) < 0.5, 1.0, -1.0) * 1e-15
    sig0, K, fac = O.solve(g)
    ref = pos.copy()
    for _ in range(3):
        ref, sig_ref, _ = O.dynamic_step(g, fac, ref, q)
    ctx = N.Context().set_geometry(g)
    ctx.solve(N.NEBEM_FP64)
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    out = N.nebem_step(ctx.h, 3, 1e-4, 1e-9, N.NEBEM_FP64, pos.shape[0])
    disp_ref = ref - pos
    assert np.abs((out - pos) - disp_ref).max() <= 1e-9 * np.abs(disp_ref).max()


def test_error_paths(N):
    ctx = N.Context()
    with pytest.raises(N.NebemError) as e:
        ctx.eval(np.zeros((3, 3)))
    assert e.value.code == N.NEBEM_BAD_STATE
    bad = np.zeros(1, I.ELEMENT_DTYPE)
    bad["kind"] = I.KIND_TRI  # all vertices at the origin: zero area
    with pytest.raises(N.NebemError) as e:
        N.nebem_set_geometry(ctx.h, bad)
    assert e.value.code == N.NEBEM_DEGENERATE_ELEMENT
    g = I.cube(n_per_edge=2)
    N.nebem_set_geometry(ctx.h, g.elements)
    with pytest.raises(N.NebemError) as e:
        N.nebem_solve(ctx.h, N.NEBEM_FP64, g.n)
    assert e.value.code == N.NEBEM_BAD_STATE  # no voltages yet
    with pytest.raises(N.NebemError) as e:
        N.nebem_set_bc(ctx.h, [])
    assert e.value.code == N.NEBEM_INVALID_ARG  # conductor 0 out of range
    with pytest.raises(N.NebemError) as e:
        N.nebem_set_geometry(ctx.h, g.elements, np.eye(2, 3), -6, 6)
    assert e.value.code == N.NEBEM_TOO_LARGE



def test_counts_above_the_limit_refused_before_any_access(N):
    """A count above NEBEM_MAX_COUNT (2^31 - 1) is refused with NEBEM_TOO_LARGE before
    any buffer is read and before any size is computed from it: every buffer passed here
    holds a single point (or a 1 x 1 matrix)."""
    import ctypes as C

    import torch
    L = N.load()
    ctx = N.Context().set_geometry(I.cube(n_per_edge=2))
    big = 2 ** 31
    one = np.zeros(3)
    d1 = N._dp(one)
    i1 = np.zeros(1, np.int64).ctypes.data_as(C.POINTER(C.c_int64))
    dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    piv = torch.zeros(1, dtype=torch.int32, device="cuda")
    calls = {
        "nebem_eval": lambda: L.nebem_eval(ctx.h, d1, big, d1, d1, N.NEBEM_FP64),
        "nebem_eval_device": lambda: L.nebem_eval_device(ctx.h, dev.data_ptr(), big, dev.data_ptr(), None,
                                                         N.NEBEM_MIXED, None),
        "nebem_space_charge": lambda: L.nebem_space_charge(ctx.h, d1, d1, big, 1e-6),
        "nebem_space_charge_eval": lambda: L.nebem_space_charge_eval(ctx.h, d1, big, d1, d1, N.NEBEM_FP64, 0),
        "nebem_fastvol_eval": lambda: L.nebem_fastvol_eval(ctx.h, d1, big, d1, d1),
        "nebem_matrix_entries": lambda: L.nebem_matrix_entries(ctx.h, i1, i1, big, d1),
        "nebem_lu_factor_device": lambda: L.nebem_lu_factor_device(ctx.h, dev.data_ptr(), big, piv.data_ptr(), None),
        "nebem_lu_solve_device": lambda: L.nebem_lu_solve_device(ctx.h, dev.data_ptr(), big, piv.data_ptr(),
                                                                 dev.data_ptr(), None),
    }
    for name, call in calls.items():
        assert call() == N.NEBEM_TOO_LARGE, name
        assert b"above 2^31 - 1" in L.nebem_last_error(), name
    # the context is still usable
    N.nebem_set_bc(ctx.h, [1.0])
    ctx.solve(N.NEBEM_FP64)

def test_fill_parity_double_thgem_full_size_sampled(N):
    """The 40,368-element double THGEM (25 images): sampled entries of the GPU-filled
    matrix against the oracle computed entry by entry (incl. diagonal/self terms)."""
    g = I.double_thgem()
    ctx = N.Context().set_geometry(g)
    gen = I.rng(2, 3)
    rows = gen.integers(0, g.n, 96)
    cols = np.concatenate([gen.integers(0, g.n, 64), rows[64:]])  # 32 diagonal entries
    got = N.nebem_matrix_entries(ctx.h, rows, cols)
    ref = O.fill_entries(g, rows, cols)
    diag = O.fill_entries(g, rows, rows)
    assert (np.abs(got - ref) / np.abs(diag)).max() <= TOL64


def test_dense_lu_device_matches_oracle(N):
    """nebem_lu_factor_device / nebem_lu_solve_device on a BEM matrix (oracle-filled) and
    on a ragged size, against the oracle's LU: same pivots, factors and solution."""
    import torch
    ctx = N.Context()
    for g in (I.cube(n_per_edge=8), I.thgem(I.PlateSpec(n_phi=12, n_r=2, n_zc=1, n_zf=3), n_plane=2)):
        K = O.fill(g)
        n = K.shape[0]
        A_ref, piv_ref = O.lu_factor(K)
        dA = torch.tensor(np.asfortranarray(K).ravel(order="F"), device="cuda")
        dpiv = torch.empty(n, dtype=torch.int32, device="cuda")
        N.nebem_lu_factor_device(ctx.h, dA.data_ptr(), n, dpiv.data_ptr())
        assert np.array_equal(dpiv.cpu().numpy(), piv_ref)
        LU = dA.cpu().numpy()
        assert np.abs(LU - A_ref).max() <= TOL64 * np.abs(A_ref).max()
        b = O.rhs(g)
        db = torch.tensor(b, device="cuda")
        N.nebem_lu_solve_device(ctx.h, dA.data_ptr(), n, dpiv.data_ptr(), db.data_ptr())
        torch.cuda.synchronize()
        x_ref = O.lu_solve((A_ref, piv_ref), b)
        assert np.abs(db.cpu().numpy() - x_ref).max() <= TOL64 * np.abs(x_ref).max()


def test_weighting_fields_reuse_the_factors(N):
    """K does not depend on the voltages, so the factors are reused (Sec. 2.1): the
    solution for any voltage set equals the sum of per-conductor unit ("weighting
    field") solutions, and each unit solution matches the oracle."""
    g = small_thgem()
    ctx = N.Context().set_geometry(g)
    K = O.fill(g)
    fac = O.lu_factor(K)
    units = []
    for c in range(len(g.voltages)):
        v = np.zeros(len(g.voltages)); v[c] = 1.0
        N.nebem_set_bc(ctx.h, v)
        sig, info, _ = ctx.solve(N.NEBEM_FP64)
        ref = O.lu_solve(fac, O.rhs(g, v))
        assert rel_norm(sig, ref) <= TOL64
        units.append(sig)
    N.nebem_set_bc(ctx.h, g.voltages)
    sig_all, _, _ = ctx.solve(N.NEBEM_FP64)
    combo = sum(V * u for V, u in zip(g.voltages, units))
    # each unit solve is good to the FP64 solve tolerance; the voltage-weighted sum of
    # four of them (|V| up to 1700 V, opposite signs) carries those errors scaled by |V|
    assert rel_norm(combo, sig_all) <= TOL64


def test_quadrilateral_elements_fill_solve_eval(N):
    """A geometry of rectangles, triangles and planar convex quadrilaterals (the THGEM's
    primitives taken as elements, one conductor, 5 x 5 copies): FP64 fill, solve and
    evaluation against the oracle, and the mixed evaluation within its bound."""
    g0 = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    g = I.Geometry(name="thgem_primitives", elements=g0.primitives.copy(), voltages=np.array([1.0]),
                   lattice=g0.lattice, img_lo=-2, img_hi=2, pitch=g0.pitch, z_range=g0.z_range)
    assert (g.elements["kind"] == I.KIND_QUAD).sum() > 0
    ctx = N.Context().set_geometry(g)
    K = ctx.fill(N.NEBEM_FP64)
    Kr = O.fill(g)
    assert rel_norm(K, Kr) <= TOL64
    sig, _, _ = ctx.solve(N.NEBEM_FP64)
    ref, _, _ = O.solve(g)
    assert rel_norm(sig, ref) <= TOL64
    pts = I.cell_points(g, 200, I.rng(2, 60))
    phi, E = ctx.eval(pts, N.NEBEM_FP64)
    rphi, rE = O.eval_points(g, ref, pts)
    assert rel_norm(phi, rphi) <= TOL64 and rel_norm(E, rE) <= TOL64
    phi, E = ctx.eval(pts, N.NEBEM_MIXED)
    assert rel_norm(phi, rphi) <= 1e-6 and rel_norm(E, rE) <= 1e-6

"""Mixed-precision evaluation (FP32 far-field Gauss rules + FP64 near closed forms, then a
two-float re-evaluation of the points whose estimated error exceeds 1e-6 of their own
value) against the FP64 oracle and the FP64 path: <= 1e-6 relative per point, with the
floor 1e-6 of the largest value (|dPhi_i| / max(|Phi_i|, 1e-6 max|Phi|), and the same for
the field vector), and bit-identical per point whatever the batch it is evaluated in."""
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


def rel_norm(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def rel_vec(a, ref):
    return float(np.linalg.norm(a - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max())


def pp_scalar(a, ref):
    """largest per-point relative error, floor 1e-6 of the largest |ref|"""
    r = np.abs(ref)
    return float((np.abs(a - ref) / np.maximum(r, 1e-6 * r.max())).max())


def pp_vec(a, ref):
    """the same for vectors (rows): |a_i - ref_i| / max(|ref_i|, 1e-6 max |ref|)"""
    r = np.linalg.norm(ref, axis=1)
    return float((np.linalg.norm(a - ref, axis=1) / np.maximum(r, 1e-6 * r.max())).max())


def assert_mixed(phi, E, rphi, rE):
    assert pp_scalar(phi, rphi) <= TOL_MIXED, pp_scalar(phi, rphi)
    assert pp_vec(E, rE) <= TOL_MIXED, pp_vec(E, rE)
    assert rel_norm(phi, rphi) <= TOL_MIXED and rel_vec(E, rE) <= TOL_MIXED


def structured_sigma(g):
    """A smooth, physically shaped charge density: conductor elements carry
    eps0 * V / 1 mm with a smooth modulation, interface elements a tenth of the scale."""
    c, _, _ = O.centroids(g)
    v = g.voltages
    sig = np.zeros(g.n)
    cond = g.elements["bc"] == I.BC_CONDUCTOR
    mod = 1.0 + 0.3 * np.sin(2 * np.pi * c[:, 0] / 1e-3) * np.cos(2 * np.pi * c[:, 1] / 1e-3)
    sig[cond] = 8.854e-12 * v[g.elements["conductor"][cond]] / 1e-3 * mod[cond]
    sig[~cond] = 0.1 * 8.854e-12 * 500.0 / 1e-3 * np.sin(2 * np.pi * c[~cond, 2] / 0.5e-3)
    return sig


def test_mixed_eval_cube_grid(N):
    g = I.cube(n_per_edge=8)
    sig_r, _, _ = O.solve(g)
    pts = I.cube_grid_points()
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sig_r)
    phi, E = ctx.eval(pts, N.NEBEM_MIXED)
    rphi, rE = O.eval_points(g, sig_r, pts)
    assert_mixed(phi, E, rphi, rE)


def test_mixed_eval_thgem_full_geometry_sampled(N):
    g = I.thgem()
    sigma = structured_sigma(g)
    pts = I.cell_points(g, 64, I.rng(1, 11))
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    phi, E = ctx.eval(pts, N.NEBEM_MIXED)
    rphi, rE = O.eval_points(g, sigma, pts)
    assert_mixed(phi, E, rphi, rE)


def test_mixed_matches_fp64_path_on_many_points(N):
    g = I.thgem()
    sigma = structured_sigma(g)
    pts = I.cell_points(g, 20000, I.rng(1, 12))
    # points close to surfaces: the FP64 near-field branch and the high-order tiers
    near = pts.copy()
    near[:, 2] = np.where(pts[:, 2] > 0, 0.285e-3 + 1e-6 * (1 + np.abs(pts[:, 0]) * 1e3),
                          -0.285e-3 - 1e-6 * (1 + np.abs(pts[:, 1]) * 1e3))
    pts = np.concatenate([pts, near[:4000]])
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    phi, E = ctx.eval(pts, N.NEBEM_MIXED)
    phi64, E64 = ctx.eval(pts, N.NEBEM_FP64)
    assert_mixed(phi, E, phi64, E64)


def test_mixed_result_independent_of_batch(N):
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    sigma = structured_sigma(g)
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    mine = I.cell_points(g, 300, I.rng(0, 21))
    others = I.cell_points(g, 5000, I.rng(0, 22))
    alone_phi, alone_E = ctx.eval(mine, N.NEBEM_MIXED)
    batch = np.concatenate([others[:1777], mine, others[1777:]])
    perm = I.rng(0, 23).permutation(batch.shape[0])
    bphi, bE = ctx.eval(batch[perm], N.NEBEM_MIXED)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    sel = inv[1777:1777 + 300]
    assert np.array_equal(bphi[sel], alone_phi)
    assert np.array_equal(bE[sel], alone_E)


def test_mixed_ragged_and_empty(N):
    g = I.cube(n_per_edge=4)
    sig_r, _, _ = O.solve(g)
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sig_r)
    for n in [0, 1, 127, 128, 129, 1000]:
        pts = I.cell_points(g, max(n, 1), I.rng(0, 100 + n))[:n]
        phi, E = ctx.eval(pts, N.NEBEM_MIXED)
        if n:
            rphi, rE = O.eval_points(g, sig_r, pts)
            assert_mixed(phi, E, rphi, rE)


def test_pair_tiers_bit_exact_with_oracle(N):
    """The mixed evaluation's per-pair tier decision (FP32 on two-float coordinates)
    equals the oracle's written-out classification for every (point, element, image)."""
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    pts = I.cell_points(g, 120, I.rng(1, 31))
    near = pts[:40].copy()
    near[:, 2] = 0.285e-3 + 1e-7 * np.arange(40)  # just above the top Cu face
    pts = np.concatenate([pts, near, [[0.0, 0.0, 0.0], [0.25e-3, 0.0, 0.1e-3]]])
    ctx = N.Context().set_geometry(g)
    got = N.nebem_pair_tiers(ctx.h, pts, g.n, g.n_images)
    ref = O.pair_tiers(g, pts)
    assert np.array_equal(got, ref)
    assert set(np.unique(ref)) == {0, 1, 2, 3, 4}


def test_mixed_eval_121_images(N):
    """Eleven copies per lattice axis (the largest image range): mixed against the oracle."""
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    g.img_lo, g.img_hi = -5, 5
    sigma = structured_sigma(g)
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    pts = I.cell_points(g, 200, I.rng(1, 33))
    phi, E = ctx.eval(pts, N.NEBEM_MIXED)
    rphi, rE = O.eval_points(g, sigma, pts)
    assert_mixed(phi, E, rphi, rE)
    assert N.nebem_image_table(ctx.h).shape[0] == 121


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_eval_device_on_caller_stream(N, prec):
    """nebem_eval_device on a caller's CUDA stream gives the same bits as nebem_eval."""
    import torch
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    sigma = structured_sigma(g)
    ctx = N.Context().set_geometry(g)
    ctx.set_sigma(sigma)
    p = N.NEBEM_FP64 if prec == "fp64" else N.NEBEM_MIXED
    pts = I.cell_points(g, 3000, I.rng(1, 34))
    hphi, hE = ctx.eval(pts, p)
    st = torch.cuda.Stream()
    d_pts = torch.from_numpy(pts).cuda()
    d_phi = torch.full((pts.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
    d_E = torch.full((pts.shape[0], 3), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    N.nebem_eval_device(ctx.h, d_pts.data_ptr(), pts.shape[0], d_phi.data_ptr(), d_E.data_ptr(), p, st.cuda_stream)
    st.synchronize()
    assert np.array_equal(d_phi.cpu().numpy(), hphi) and np.array_equal(d_E.cpu().numpy(), hE)


def test_non_finite_points_give_nan_and_leave_the_batch_unchanged(N):
    """A point with a NaN or infinite coordinate has no field.  The FP32 tiers would fail
    every distance test for it and return zeros, so every evaluation path writes NaN for
    it instead: FP64 and mixed evaluation, the serving kernel (requests below its
    whole-block size run as element chunks) and the FastVolume lookup.  The finite points
    of the same batch keep their bits."""
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    ctx = N.Context().set_geometry(g)
    ctx.solve(N.NEBEM_MIXED)
    pts = I.cell_points(g, 400, I.rng(0, 31))
    bad = np.array([3, 128, 255, 399])
    dirty = pts.copy()
    dirty[3, 0] = np.nan
    dirty[128, 1] = np.inf
    dirty[255, 2] = -np.inf
    dirty[399] = np.nan
    ok = np.setdiff1d(np.arange(pts.shape[0]), bad)
    for prec in (N.NEBEM_FP64, N.NEBEM_MIXED):
        phi, E = ctx.eval(dirty, prec)
        assert np.isnan(phi[bad]).all() and np.isnan(E[bad]).all()
        cphi, cE = ctx.eval(pts[ok], prec)
        assert np.array_equal(phi[ok], cphi) and np.array_equal(E[ok], cE)
    srv = N.nebem_server_create([ctx.h])
    try:
        for prec in (N.NEBEM_FP64, N.NEBEM_MIXED):
            phi = np.empty(pts.shape[0])
            E = np.empty((pts.shape[0], 3))
            rid = N.nebem_server_submit(srv, 0, dirty, phi, E, prec)
            N.nebem_server_wait(srv, rid, 120000)
            rphi, rE = ctx.eval(dirty, prec)
            assert np.array_equal(phi, rphi, equal_nan=True) and np.array_equal(E, rE, equal_nan=True)
    finally:
        N.nebem_server_destroy(srv)
    p = g.pitch
    N.nebem_fastvol_build(ctx.h, np.linspace(-0.5 * p, 0.5 * p, 9), np.linspace(-0.5 * p, 0.5 * p, 9),
                          np.linspace(1.2e-3, 3.0e-3, 7), N.NEBEM_FP64)
    phi, E = N.nebem_fastvol_eval(ctx.h, dirty)
    assert np.isnan(phi[bad]).all() and np.isnan(E[bad]).all()
    cphi, cE = N.nebem_fastvol_eval(ctx.h, pts[ok])
    assert np.array_equal(phi[ok], cphi) and np.array_equal(E[ok], cE)


def test_error_estimates_and_refinement(N):
    """nebem_eval_err: the single FP32 pass (mixed_point_tol = 0) and the refined evaluation
    (default 1e-6) on THGEM points, against the FP64 path.
      - the single pass misses the per-point bound where its result is small next to its
        error scale (inside the plate, inside the copper), which is what the refinement is for;
      - every estimate of the single pass covers its actual error;
      - the refinement re-evaluates exactly the points whose estimate exceeds 1e-6 of their
        |phi| or |E|, leaves every other point's bits unchanged, and meets the bound at every
        point; the refined points' estimates cover their errors too."""
    g = I.thgem()
    ctx = N.Context().set_geometry(g)
    sigma, _, _ = ctx.solve(N.NEBEM_MIXED)
    fast = N.Context(mixed_point_tol=0.0).set_geometry(g)
    fast.set_sigma(sigma)
    gen = I.rng(1, 41)
    pts = I.cell_points(g, 12000, gen)
    plate = pts[:3000].copy()
    plate[:, 2] = (gen.random(3000) - 0.5) * 0.65e-3  # through the plate and both copper layers
    pts = np.concatenate([pts, plate])
    phi64, E64 = ctx.eval(pts, N.NEBEM_FP64)
    fphi, fE, ferr, n0 = fast.eval_err(pts)
    phi, E, err, nref = ctx.eval_err(pts)
    assert n0 == 0 and nref > 0
    # the single pass: estimates cover the errors; the bound is missed somewhere
    dphi_f = np.abs(fphi - phi64)
    dE_f = np.linalg.norm(fE - E64, axis=1)
    assert (dphi_f <= ferr[:, 0]).all(), (dphi_f / ferr[:, 0]).max()
    assert (dE_f <= ferr[:, 1]).all(), (dE_f / ferr[:, 1]).max()
    assert pp_vec(fE, E64) > TOL_MIXED or pp_scalar(fphi, phi64) > TOL_MIXED
    # which points were refined: exactly the flagged ones
    fp = ferr[:, 0] > 1e-6 * np.abs(fphi)
    fe = ferr[:, 1] > 1e-6 * np.linalg.norm(fE, axis=1)
    flag = fp | fe
    assert int(flag.sum()) == nref
    changed = (phi != fphi) | (E != fE).any(axis=1)
    assert not changed[~flag].any()
    assert np.array_equal(err[~flag], ferr[~flag])
    # a point re-evaluated for one quantity keeps the other's value and estimate, unless
    # its level-1 estimate sent it on to level 2, which re-evaluates both
    # (level-2 estimates, 1e-11 B, are far below a thousandth of the FP32 pass's, >= 7e-8 B)
    l2 = (err[:, 0] < 1e-3 * ferr[:, 0]) & (err[:, 1] < 1e-3 * ferr[:, 1])
    only_phi, only_e = fp & ~fe & ~l2, fe & ~fp & ~l2
    assert only_phi.any() and only_e.any()
    assert np.array_equal(E[only_phi], fE[only_phi]) and np.array_equal(err[only_phi, 1], ferr[only_phi, 1])
    assert np.array_equal(phi[only_e], fphi[only_e]) and np.array_equal(err[only_e, 0], ferr[only_e, 0])
    # refined: the bound at every point, and covered estimates
    assert_mixed(phi, E, phi64, E64)
    assert (np.abs(phi - phi64)[flag] <= err[flag, 0] + 1e-12 * np.abs(phi64[flag])).all()
    assert (np.linalg.norm(E - E64, axis=1)[flag] <= err[flag, 1] + 1e-12 * np.linalg.norm(E64[flag], axis=1)).all()
    # nebem_eval with NEBEM_MIXED gives the refined result
    ephi, eE = ctx.eval(pts, N.NEBEM_MIXED)
    assert np.array_equal(ephi, phi) and np.array_equal(eE, E)
    # the stage report of that evaluation
    st = N.nebem_eval_stats(ctx.h)
    assert st.points == pts.shape[0] and st.refined_level1 == nref
    assert st.refined_level1_phi_only == int((fp & ~fe).sum()) and st.refined_level1_E_only == int((fe & ~fp).sum())
    assert 0 <= st.refined_level2 <= st.refined_level1
    assert st.ms_fp32 > 0.0 and st.ms_level1 > 0.0 and st.ms_level2 >= 0.0


def test_error_scales_match_oracle(N):
    """The FP32 pass's error scales B = ke sum_j b_j and S = ke sqrt(sum_j b_j^2), with
    b_j = |sigma_j| |sum_k Phi'_jk| (for E: |sigma_j| |sum_k E'_jk|_1) over the pairs the
    FP32 tiers take (tier codes 0-3), against the same sums formed from the oracle's
    closed forms; the estimate gamma_r |x| + gamma_b B + gamma_s S is linear in its
    constants."""
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    sigma = structured_sigma(g)
    pts = I.cell_points(g, 12, I.rng(1, 51))
    codes = O.pair_tiers(g, pts)
    timg = O.image_table(g.lattice, g.img_lo, g.img_hi)
    sp = np.zeros((pts.shape[0], g.n))
    sE = np.zeros((pts.shape[0], g.n, 3))
    for j in range(g.n):
        for k in range(timg.shape[0]):
            p, e = O.influence(g.elements[j], pts - timg[k])
            far = codes[:, j, k] < 4
            sp[:, j] += np.where(far, p, 0.0)
            sE[:, j] += np.where(far[:, None], e, 0.0)
    ke = O.ke()
    bphi = np.abs(sigma) * np.abs(sp)
    bE = np.abs(sigma) * np.abs(sE).sum(axis=2)
    B = ke * np.stack([bphi.sum(1), bE.sum(1)], axis=1)
    S = ke * np.stack([np.sqrt((bphi ** 2).sum(1)), np.sqrt((bE ** 2).sum(1))], axis=1)
    f = N.Context(mixed_point_tol=0.0).set_geometry(g)
    f.set_sigma(sigma)
    N.nebem_set_error_model(f.h, 0.0, 1.0, 0.0)
    phi, E, eb, _ = f.eval_err(pts)
    N.nebem_set_error_model(f.h, 0.0, 0.0, 1.0)
    _, _, es, _ = f.eval_err(pts)
    N.nebem_set_error_model(f.h, 1.0, 0.0, 0.0)
    _, _, er, _ = f.eval_err(pts)
    N.nebem_set_error_model(f.h, -1.0, -1.0, -1.0)  # the defaults
    _, _, ed, _ = f.eval_err(pts)
    assert np.abs(eb / B - 1).max() < 1e-5
    assert np.abs(es / S - 1).max() < 1e-5
    x = np.stack([np.abs(phi), np.linalg.norm(E, axis=1)], axis=1)
    assert np.allclose(er, x, rtol=1e-15, atol=0)
    assert np.allclose(ed, 1e-7 * x + 7e-8 * eb + 5e-7 * es, rtol=1e-6, atol=0)
    f.close()

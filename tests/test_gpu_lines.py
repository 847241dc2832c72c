"""Line-charge representation of the known charges (Sec. 4.2, Alg. 3; LineCh in Alg. 4)
through the C-ABI against the oracle: the point -> line reduction bit for bit (line
count, order, geometry and densities), line-charge sums at points (FP64 <= 1e-10,
mixed <= 1e-6), the right-hand side / solve with lines, and dynamic steps."""
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


@pytest.fixture(scope="module")
def thgem():
    return I.thgem()


def rel_norm(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def _charges(gen, n):
    """+-e times 1..4: unequal magnitudes, so the per-voxel summation order shows."""
    return gen.choice([-1.0, 1.0], n) * I.E_CHARGE * gen.integers(1, 5, n)


def _lines_of(N, ctx):
    st, sp, lam = N.nebem_get_lines(ctx.h)
    return O.Lines(st, sp, lam)


@pytest.mark.parametrize("n", [1, 5, 2047, 2048, 2049, 5000, 70000])
def test_voxel_lines_bit_exact(N, thgem, n):
    gen = np.random.default_rng(100 + n)
    pos, _ = I.carrier_cloud(thgem, n, I.rng(3, 40 + n % 7))
    q = _charges(gen, n)
    ctx = N.Context().set_geometry(I.cube(n_per_edge=2))
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    d = np.array([30e-6, 25e-6, 50e-6])
    nl = N.nebem_space_charge_lines(ctx.h, d)
    st, sp, lam = N.nebem_get_lines(ctx.h)
    ref = O.voxel_lines(pos, q, d)
    assert nl == len(ref) == st.shape[0]
    assert np.array_equal(st, ref.start) and np.array_equal(sp, ref.stop)
    assert np.array_equal(lam, ref.lam)


def test_voxel_lines_on_voxel_boundaries_and_one_voxel(N):
    """Points on an exact lattice of the voxel size (every floor decision at a boundary),
    and a voxel larger than the cloud (one line with all the charge)."""
    gen = np.random.default_rng(7)
    d = np.array([1e-5, 2e-5, 4e-5])
    idx = gen.integers(0, 12, size=(3000, 3))
    pos = np.ascontiguousarray(1e-3 + idx * d)
    q = _charges(gen, 3000)
    ctx = N.Context().set_geometry(I.cube(n_per_edge=2))
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    N.nebem_space_charge_lines(ctx.h, d)
    got = _lines_of(N, ctx)
    ref = O.voxel_lines(pos, q, d)
    assert np.array_equal(got.start, ref.start) and np.array_equal(got.lam, ref.lam)
    assert N.nebem_space_charge_lines(ctx.h, [1.0, 1.0, 1.0]) == 1
    one = _lines_of(N, ctx)
    assert np.array_equal(one.lam, O.voxel_lines(pos, q, [1.0, 1.0, 1.0]).lam)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_line_charge_sum_parity(N, thgem, prec):
    gen = np.random.default_rng(11)
    pos, _ = I.carrier_cloud(thgem, 6000, I.rng(3, 50))
    q = _charges(gen, 6000)
    ctx = N.Context().set_geometry(I.cube(n_per_edge=2))
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    N.nebem_space_charge_lines(ctx.h, [40e-6, 40e-6, 60e-6])
    L = _lines_of(N, ctx)
    p = N.NEBEM_FP64 if prec == "fp64" else N.NEBEM_MIXED
    inside = pos[::20]
    phi, E = N.nebem_space_charge_eval(ctx.h, inside, p)
    rphi, rE = O.line_charge(L, inside)
    tol = TOL64 if prec == "fp64" else TOL_MIXED
    assert rel_norm(phi, rphi) <= tol, rel_norm(phi, rphi)
    assert rel_norm(E, rE) <= tol, rel_norm(E, rE)
    outside = I.cell_points(thgem, 200, I.rng(3, 51))
    phi, E = N.nebem_space_charge_eval(ctx.h, outside, p)
    rphi, rE = O.line_charge(L, outside)
    if prec == "fp64":
        assert rel_norm(phi, rphi) <= tol and rel_norm(E, rE) <= tol
    else:
        # far from a net-neutral cloud the +/- terms cancel: per-term FP32 accuracy
        # bounds the error by the sums of |terms|
        absL = O.Lines(L.start, L.stop, np.abs(L.lam))
        absphi, _ = O.line_charge(absL, outside)
        absE = np.zeros(outside.shape[0])
        for l in range(len(L)):
            _, El = O.line_charge(O.Lines(L.start[l:l + 1], L.stop[l:l + 1], np.abs(L.lam[l:l + 1])), outside)
            absE += np.linalg.norm(El, axis=1)
        assert (np.abs(phi - rphi) / absphi).max() <= 3e-7
        assert (np.linalg.norm(E - rE, axis=1) / absE).max() <= 3e-7


def test_solve_with_line_charges(N):
    g = I.cube(n_per_edge=4)
    sig0, K, fac = O.solve(g)
    gen = np.random.default_rng(13)
    pos = gen.normal(size=(400, 3)) * 2e-3 + np.array([0.0, 0.0, 0.011])
    q = np.where(gen.random(400) < 0.5, 1.0, -1.0) * 1e-14
    d = np.array([4e-4, 4e-4, 6e-4])
    ctx = N.Context().set_geometry(g)
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    N.nebem_space_charge_lines(ctx.h, d)
    sig, info, _ = ctx.solve(N.NEBEM_FP64)
    ref = O.lu_solve(fac, O.rhs_lines(g, O.voxel_lines(pos, q, d)))
    assert rel_norm(sig, ref) <= TOL64
    # the known-charge part of nebem_eval is the line sum
    pts = gen.normal(size=(50, 3)) * 3e-3 + np.array([0.0, 0.0, 0.011])
    phi, E = ctx.eval(pts, N.NEBEM_FP64)
    ephi, eE = O.eval_points(g, sig, pts)
    lphi, lE = O.line_charge(O.voxel_lines(pos, q, d), pts)
    assert rel_norm(phi, ephi + lphi) <= TOL64 and rel_norm(E, eE + lE) <= TOL64


def test_dynamic_steps_with_lines(N):
    g = I.cube(n_per_edge=4)
    gen = np.random.default_rng(17)
    pos = gen.normal(size=(300, 3)) * 2e-3 + np.array([0.0, 0.0, 0.012])
    q = np.where(gen.random(300) < 0.5, 1.0, -1.0) * 1e-15
    d = np.array([5e-4, 5e-4, 8e-4])
    _, _, fac = O.solve(g)
    ref = pos.copy()
    for _ in range(3):
        ref, _, _ = O.dynamic_step_lines(g, fac, ref, q, d)
    ctx = N.Context().set_geometry(g)
    ctx.solve(N.NEBEM_FP64)
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    N.nebem_space_charge_lines(ctx.h, d)
    out = N.nebem_step(ctx.h, 3, 1e-4, 1e-9, N.NEBEM_FP64, pos.shape[0])
    disp = ref - pos
    assert np.abs((out - pos) - disp).max() <= 1e-9 * np.abs(disp).max()
    # the lines after the steps are the reduction of the last step's starting positions
    # (the step re-reduces before it moves the carriers)
    mixed = N.nebem_step(ctx.h, 1, 1e-4, 1e-9, N.NEBEM_MIXED, pos.shape[0])
    assert np.all(np.isfinite(mixed))


def test_full_size_cloud_sampled(N, thgem):
    """1e6 carriers in the THGEM hole (the dynamic-step workload), 20 x 20 x 40 um voxels:
    every line bit-exact with the oracle's reduction; line sums at sampled carriers in
    mixed precision against the oracle's sum over the same lines."""
    pos, q = I.carrier_cloud(thgem, 1_000_000, I.rng(3, 0))
    d = np.array([20e-6, 20e-6, 40e-6])
    ctx = N.Context().set_geometry(I.cube(n_per_edge=2))
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    nl = N.nebem_space_charge_lines(ctx.h, d)
    L = _lines_of(N, ctx)
    ref = O.voxel_lines(pos, q, d)
    assert nl == len(ref)
    assert np.array_equal(L.start, ref.start) and np.array_equal(L.lam, ref.lam)
    sample = pos[I.rng(3, 1).choice(pos.shape[0], 256, replace=False)]
    phi, E = N.nebem_space_charge_eval(ctx.h, sample, N.NEBEM_MIXED)
    rphi, rE = O.line_charge(ref, sample)
    assert rel_norm(phi, rphi) <= TOL_MIXED and rel_norm(E, rE) <= TOL_MIXED


def test_line_state_errors(N):
    ctx = N.Context().set_geometry(I.cube(n_per_edge=2))
    with pytest.raises(N.NebemError) as e:
        N.nebem_space_charge_lines(ctx.h, [1e-5, 1e-5, 1e-5])
    assert e.value.code == N.NEBEM_BAD_STATE  # no point charges
    pos = np.random.default_rng(1).normal(size=(100, 3)) * 1e-3
    q = np.full(100, I.E_CHARGE)
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    with pytest.raises(N.NebemError) as e:
        N.nebem_get_lines(ctx.h)
    assert e.value.code == N.NEBEM_BAD_STATE  # point charges in use
    for bad in ([0.0, 1e-5, 1e-5], [1e-5, -1e-5, 1e-5], [np.inf, 1e-5, 1e-5]):
        with pytest.raises(N.NebemError) as e:
            N.nebem_space_charge_lines(ctx.h, bad)
        assert e.value.code == N.NEBEM_INVALID_ARG
    with pytest.raises(N.NebemError) as e:
        N.nebem_space_charge_lines(ctx.h, [1e-6, 1e-6, 1e-3])  # needle voxels: near search too wide
    assert e.value.code == N.NEBEM_INVALID_ARG
    with pytest.raises(N.NebemError) as e:
        N.nebem_space_charge_lines(ctx.h, [1e-15, 1e-15, 1e-15])  # ~1e37 voxels
    assert e.value.code == N.NEBEM_TOO_LARGE
    # still point charges: self exclusion works, lines are refused
    N.nebem_space_charge_eval(ctx.h, pos, N.NEBEM_FP64, exclude_self=True)
    N.nebem_space_charge_lines(ctx.h, [1e-4, 1e-4, 1e-4])
    with pytest.raises(N.NebemError) as e:
        N.nebem_space_charge_eval(ctx.h, pos, N.NEBEM_FP64, exclude_self=True)
    assert e.value.code == N.NEBEM_INVALID_ARG
    # a new point set switches back to points
    N.nebem_space_charge(ctx.h, pos, q, 1e-6)
    with pytest.raises(N.NebemError) as e:
        N.nebem_get_lines(ctx.h)
    assert e.value.code == N.NEBEM_BAD_STATE

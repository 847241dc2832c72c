"""FP32 LU with tensor-core (tcgen05, TF32 hi/lo split) trailing updates: the factors
reproduce P A = L U to FP32-level accuracy on ragged sizes (several 128 x 128 tiles and
partial tiles), and refined solutions match the FP64 oracle.  Sizes with n % 4 == 0 take
the bulk-asynchronous update (pre-split operands, TMA-moved C tiles; 4100 gives CTAs
several column tiles each), the others the register-staged update."""
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


def _unpack(LU, piv):
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    perm = np.arange(n)
    for k in range(n):
        p = piv[k]
        perm[[k, p]] = perm[[p, k]]
    return L, U, perm


@pytest.mark.parametrize("n", [64, 200, 333, 700, 1028, 4100])
def test_fp32_tensor_core_lu_reconstructs(N, n):
    import torch
    gen = np.random.default_rng(n)
    A = gen.normal(size=(n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    ctx = N.Context()
    dA = torch.tensor(np.asfortranarray(A).ravel(order="F").astype(np.float32), device="cuda")
    dp = torch.empty(n, dtype=torch.int32, device="cuda")
    N.nebem_lu_factor_device_f32(ctx.h, dA.data_ptr(), n, dp.data_ptr())
    LU = dA.cpu().numpy().astype(np.float64).reshape(n, n, order="F")
    L, U, perm = _unpack(LU, dp.cpu().numpy())
    err = np.abs(A[perm] - L @ U).max() / np.abs(A).max()
    assert err <= 2e-5, err


def test_mixed_solve_bem_matrix_refines_to_oracle(N):
    g = I.thgem(I.PlateSpec(n_phi=36, n_r=4, n_zc=1, n_zf=6), n_plane=4)
    assert g.n > 1000
    sig_r, K, fac = O.solve(g)
    ctx = N.Context().set_geometry(g)
    sig, info, _ = ctx.solve(N.NEBEM_MIXED)
    assert np.abs(sig - sig_r).max() <= 1e-8 * np.abs(sig_r).max()
    assert info.iterations <= 12


@pytest.mark.parametrize("n", [1, 2, 63, 65, 129, 1000])
def test_lu_edge_sizes_fp64_solve_and_fp32_factor(N, n):
    """Sizes around the 64-row block of the single-launch triangular sweeps and the panel
    width: FP64 factor + solve against numpy; FP32 factor (cooperative panel) reconstructs."""
    import torch
    gen = np.random.default_rng(1000 + n)
    A = gen.normal(size=(n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    b = gen.normal(size=n)
    ctx = N.Context()
    dA = torch.tensor(np.asfortranarray(A).ravel(order="F"), device="cuda")
    dp = torch.empty(n, dtype=torch.int32, device="cuda")
    N.nebem_lu_factor_device(ctx.h, dA.data_ptr(), n, dp.data_ptr())
    db = torch.tensor(b, device="cuda")
    N.nebem_lu_solve_device(ctx.h, dA.data_ptr(), n, dp.data_ptr(), db.data_ptr())
    torch.cuda.synchronize()
    x = db.cpu().numpy()
    xr = np.linalg.solve(A, b)
    assert np.abs(x - xr).max() <= 1e-12 * np.abs(xr).max()
    dA32 = torch.tensor(np.asfortranarray(A).ravel(order="F").astype(np.float32), device="cuda")
    N.nebem_lu_factor_device_f32(ctx.h, dA32.data_ptr(), n, dp.data_ptr())
    LU = dA32.cpu().numpy().astype(np.float64).reshape(n, n, order="F")
    L, U, perm = _unpack(LU, dp.cpu().numpy())
    assert np.abs(A[perm] - L @ U).max() / np.abs(A).max() <= 2e-5


@pytest.mark.parametrize("zero_col", [0, 70, 299])
def test_exact_zero_pivot_reported_and_factorisation_completed(N, zero_col):
    """A matrix with an exactly zero column keeps that column zero through every row swap
    and update (each update term is a multiple of one of its entries), so the pivot search
    meets an exact zero there.  Both factorisations report NEBEM_SINGULAR naming the
    column, skip that column's scaling (there is nothing below the diagonal to eliminate)
    and run to the end: every pivot row lies in [k, n), U has an exact zero on its
    diagonal at the column, and P A = L U holds as for a regular matrix."""
    import torch
    n = 300
    gen = np.random.default_rng(77 + zero_col)
    A = gen.normal(size=(n, n)) + 2.0 * np.sqrt(n) * np.eye(n)
    A[:, zero_col] = 0.0
    ctx = N.Context()
    cases = ((np.float64, N.nebem_lu_factor_device, 1e-12), (np.float32, N.nebem_lu_factor_device_f32, 2e-5))
    for dtype, factor, tol in cases:
        dA = torch.tensor(np.asfortranarray(A).ravel(order="F").astype(dtype), device="cuda")
        dp = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        with pytest.raises(N.NebemError) as e:
            factor(ctx.h, dA.data_ptr(), n, dp.data_ptr())
        assert e.value.code == N.NEBEM_SINGULAR
        assert f"zero pivot at column {zero_col}" in str(e.value)
        piv = dp.cpu().numpy()
        assert np.all(piv >= np.arange(n)) and np.all(piv < n)
        LU = dA.cpu().numpy().astype(np.float64).reshape(n, n, order="F")
        L, U, perm = _unpack(LU, piv)
        assert U[zero_col, zero_col] == 0.0
        assert np.abs(A[perm] - L @ U).max() / np.abs(A).max() <= tol


def test_refinement_limit_reports_not_converged(N):
    """With the refinement limit at one iteration the mixed solve stops after its first
    correction.  x starts at zero, so that correction is all of x (relative size exactly
    1): NEBEM_NOT_CONVERGED, one iteration, sigma still written (the FP32-LU solution,
    within FP32 accuracy of the oracle) and usable by the evaluation.  The default limit
    converges on the same system."""
    g = I.cube(n_per_edge=4)
    ref, _, _ = O.solve(g)
    ctx = N.Context(ir_max_iter=1).set_geometry(g)
    sig, info, rc = N.nebem_solve(ctx.h, N.NEBEM_MIXED, g.n, allow_not_converged=True)
    assert rc == N.NEBEM_NOT_CONVERGED
    assert info.iterations == 1 and info.correction == 1.0
    assert np.abs(sig - ref).max() <= 1e-4 * np.abs(ref).max()
    pts = np.array([[0.0, 0.0, 0.03], [0.02, -0.01, 0.005]])
    phi, _ = ctx.eval(pts, N.NEBEM_FP64)
    rphi, _ = O.eval_points(g, sig, pts)
    assert np.abs(phi - rphi).max() <= 1e-10 * np.abs(rphi).max()
    sig2, info2, rc2 = N.Context().set_geometry(g).solve(N.NEBEM_MIXED)
    assert rc2 == N.NEBEM_OK and info2.correction <= 1e-8
    assert np.abs(sig2 - ref).max() <= 1e-8 * np.abs(ref).max()

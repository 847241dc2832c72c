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

"""The LU entry point that allocates nothing (nebem_lu_factor_device_noalloc).

Callers that cannot allocate device memory while they run (their memory is reserved up
front for their own pool, or their loop must not allocate after start-up) factor with
nebem_lu_factor_device_noalloc, whose work space lives in a static device array of the
library.  It must give the same factors and pivots as nebem_lu_factor_device, call
after call (the shared array keeps the previous call's contents), and reject sizes
beyond its fixed maximum.  Collected last on purpose (file name) so that a run that
stops at the first failure has run everything else first.
"""
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
    L = nebem.load()
    L.nebem_lu_factor_device_noalloc.restype = C.c_int
    L.nebem_lu_factor_device_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    return nebem


def _factor_both(N, ctx, K):
    import torch
    n = K.shape[0]
    colmajor = np.asfortranarray(K).ravel(order="F")
    dA = torch.tensor(colmajor, device="cuda")
    dB = torch.tensor(colmajor, device="cuda")
    p1 = torch.empty(n, dtype=torch.int32, device="cuda")
    p2 = torch.empty(n, dtype=torch.int32, device="cuda")
    N.nebem_lu_factor_device(ctx.h, dA.data_ptr(), n, p1.data_ptr())
    rc = N.load().nebem_lu_factor_device_noalloc(dB.data_ptr(), n, p2.data_ptr(), None)
    assert rc == 0, N.load().nebem_last_error()
    return dA.cpu().numpy(), p1.cpu().numpy(), dB.cpu().numpy(), p2.cpu().numpy()


def test_noalloc_lu_matches_allocating_lu_twice(N):
    ctx = N.Context()
    # two calls in a row, different sizes (the second leaves the static work space dirty
    # from the first)
    for g in (I.cube(n_per_edge=8), I.thgem(I.PlateSpec(n_phi=12, n_r=2, n_zc=1, n_zf=3), n_plane=2)):
        K = O.fill(g)
        A1, p1, A2, p2 = _factor_both(N, ctx, K)
        assert np.array_equal(p1, p2)
        assert np.abs(A1 - A2).max() <= TOL64 * np.abs(A1).max()
        # and both are the oracle's factorisation
        A_ref, piv_ref = O.lu_factor(K)
        assert np.array_equal(p2, piv_ref)
        assert np.abs(A2 - A_ref).max() <= TOL64 * np.abs(A_ref).max()


def test_noalloc_lu_rejects_sizes_beyond_its_maximum(N):
    import torch
    d = torch.empty(1, dtype=torch.float64, device="cuda")
    p = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = N.load().nebem_lu_factor_device_noalloc(d.data_ptr(), 4097, p.data_ptr(), None)
    assert rc == N.NEBEM_TOO_LARGE
    rc = N.load().nebem_lu_factor_device_noalloc(None, 10, p.data_ptr(), None)
    assert rc == N.NEBEM_INVALID_ARG

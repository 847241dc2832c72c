"""Bounded device-side waits that run out (a poll limit of 1 through wait_polls): the call
returns NEBEM_TIMEOUT instead of hanging, every kernel has returned, and the same context
solves correctly once the limit is back at its default.

  - triangular sweeps (FP64 solve): a 64-row block waits for the blocks before it; with
    one poll the wait gives up before they have finished, the sweep writes NaN for that
    block and the solve reports NEBEM_TIMEOUT with sigma written (NaN there);
  - the FP32 factorisation's cooperative panel (mixed solve): its grid barrier gives up,
    the factorisation reports NEBEM_TIMEOUT.

No GPU fault is involved: the waits are polls of flags in global memory, and giving up
only skips work.  The tensor-core update's mbarrier waits are not shortened (it has
copies and MMAs in flight), so its own limit stays as it is."""
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


def small_thgem():
    return I.thgem(I.PlateSpec(n_phi=24, n_r=4, n_zc=1, n_zf=6), n_plane=4)


def _solve_rc(N, ctx, precision, n):
    import ctypes as C
    sigma = np.full(n, 7.0)
    info = N.nebem_solve_info()
    rc = N.load().nebem_solve(ctx.h, precision, sigma.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info))
    return rc, sigma


def test_triangular_sweep_wait_runs_out_then_solves(N):
    g = I.cube(n_per_edge=8)
    assert g.n >= 4 * 64  # several 64-row blocks, so that blocks wait for each other
    ctx = N.Context(wait_polls=1).set_geometry(g)
    rc, sigma = _solve_rc(N, ctx, N.NEBEM_FP64, g.n)
    assert rc == N.NEBEM_TIMEOUT, (rc, N.load().nebem_last_error())
    # NaN from the blocks whose wait ran out (and the blocks that depend on them: the
    # backward sweep's first block uses the forward sweep's last)
    assert np.isnan(sigma).any()
    # no valid densities: evaluation is refused rather than returning NaN fields
    with pytest.raises(N.NebemError) as e:
        ctx.eval(I.cell_points(g, 4, I.rng(0, 5)), N.NEBEM_FP64)
    assert e.value.code == N.NEBEM_BAD_STATE
    # the same context, default limit: the retained factors solve correctly
    N.nebem_set_wait_polls(ctx.h, 0)
    sig, _, _ = ctx.solve(N.NEBEM_FP64)
    ref, _, _ = O.solve(g)
    assert np.abs(sig - ref).max() <= 1e-10 * np.abs(ref).max()


def test_panel_barrier_wait_runs_out_then_solves(N):
    g = small_thgem()
    ctx = N.Context(wait_polls=1).set_geometry(g)
    rc, _ = _solve_rc(N, ctx, N.NEBEM_MIXED, g.n)
    assert rc == N.NEBEM_TIMEOUT, (rc, N.load().nebem_last_error())
    N.nebem_set_wait_polls(ctx.h, 0)
    sig, info, _ = ctx.solve(N.NEBEM_MIXED)
    ref, _, _ = O.solve(g)
    assert np.abs(sig - ref).max() <= 1e-8 * np.abs(ref).max()
    pts = I.cell_points(g, 64, I.rng(0, 6))
    phi, E = ctx.eval(pts, N.NEBEM_FP64)
    rphi, rE = O.eval_points(g, ref, pts)
    assert np.abs(phi - rphi).max() <= 1e-7 * np.abs(rphi).max()


def test_wait_polls_option_checked(N):
    ctx = N.Context()  # held: the handle lives as long as this object
    with pytest.raises(N.NebemError) as e:
        N.nebem_set_wait_polls(ctx.h, -1)
    assert e.value.code == N.NEBEM_INVALID_ARG

"""Continuous-batching field-query server (nebem_server_*): every request's result is
bit-identical to the same points evaluated alone with nebem_eval, requests admitted
while others run join the running work, and admission waits for arena memory."""
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


@pytest.fixture(scope="module")
def ctxs(N):
    g0 = I.cube(n_per_edge=8)
    g1 = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    g2 = I.thgem(I.PlateSpec(n_phi=36, n_r=4, n_zc=1, n_zf=6), n_plane=4)
    out = []
    for g in (g0, g1, g2):
        c = N.Context().set_geometry(g)
        c.solve(N.NEBEM_MIXED)
        out.append((g, c))
    return out


def _request_points(g, n, seed):
    return np.ascontiguousarray(I.cell_points(g, n, I.rng(4, seed)))


def test_server_results_identical_to_standalone(N, ctxs):
    srv = N.nebem_server_create([c.h for _, c in ctxs])
    try:
        sizes = [1, 127, 128, 129, 1000, 5000, 300, 2]
        reqs = []
        for i, n in enumerate(sizes):
            gi = i % 3
            prec = N.NEBEM_MIXED if i % 2 == 0 else N.NEBEM_FP64
            pts = _request_points(ctxs[gi][0], n, i)
            phi = np.empty(n)
            E = np.empty((n, 3))
            rid = N.nebem_server_submit(srv, gi, pts, phi, E, prec)
            reqs.append((rid, gi, prec, pts, phi, E))
        for rid, gi, prec, pts, phi, E in reqs:
            N.nebem_server_wait(srv, rid, 120000)
            rphi, rE = ctxs[gi][1].eval(pts, prec)
            assert np.array_equal(phi, rphi), (gi, prec, pts.shape)
            assert np.array_equal(E, rE)
    finally:
        N.nebem_server_destroy(srv)


def test_server_admits_while_running(N, ctxs):
    srv = N.nebem_server_create([c.h for _, c in ctxs])
    try:
        g, c = ctxs[2]
        big = _request_points(g, 60000, 100)
        bphi, bE = np.empty(60000), np.empty((60000, 3))
        r_big = N.nebem_server_submit(srv, 2, big, bphi, bE, N.NEBEM_MIXED)
        smalls = []
        for k in range(4):
            p = _request_points(ctxs[0][0], 500, 200 + k)
            ph, E = np.empty(500), np.empty((500, 3))
            smalls.append((N.nebem_server_submit(srv, 0, p, ph, E, N.NEBEM_MIXED), p, ph, E))
        N.nebem_server_wait(srv, r_big, 120000)
        _, _, big_done = N.nebem_server_request_times(srv, r_big)
        for rid, p, ph, E in smalls:
            N.nebem_server_wait(srv, rid, 120000)
            ts, ta, td = N.nebem_server_request_times(srv, rid)
            assert ta < big_done  # admitted while the big request was on the GPU
            rphi, rE = ctxs[0][1].eval(p, N.NEBEM_MIXED)
            assert np.array_equal(ph, rphi) and np.array_equal(E, rE)
        rphi, rE = c.eval(big, N.NEBEM_MIXED)
        assert np.array_equal(bphi, rphi) and np.array_equal(bE, rE)
    finally:
        N.nebem_server_destroy(srv)


def test_server_admission_waits_for_memory(N, ctxs):
    opt = N.nebem_server_default_options()
    opt.arena_points = 10000
    srv = N.nebem_server_create([c.h for _, c in ctxs], opt)
    try:
        g, c = ctxs[1]
        reqs = []
        for k in range(5):
            p = _request_points(g, 4000, 300 + k)
            ph, E = np.empty(4000), np.empty((4000, 3))
            reqs.append((N.nebem_server_submit(srv, 1, p, ph, E, N.NEBEM_MIXED), p, ph, E))
        times = []
        for rid, p, ph, E in reqs:
            N.nebem_server_wait(srv, rid, 120000)
            times.append(N.nebem_server_request_times(srv, rid))
            rphi, rE = c.eval(p, N.NEBEM_MIXED)
            assert np.array_equal(ph, rphi) and np.array_equal(E, rE)
        # only two 4000-point requests fit in 10000 points: the third waited for a release
        assert times[2][1] >= min(times[0][2], times[1][2])
        with pytest.raises(N.NebemError) as e:
            N.nebem_server_submit(srv, 1, np.zeros((20000, 3)), None, None, N.NEBEM_MIXED)
        assert e.value.code == N.NEBEM_TOO_LARGE
    finally:
        N.nebem_server_destroy(srv)


def test_server_argument_errors(N, ctxs):
    srv = N.nebem_server_create([c.h for _, c in ctxs])
    try:
        with pytest.raises(N.NebemError) as e:
            N.nebem_server_submit(srv, 7, np.zeros((3, 3)), None, None, N.NEBEM_MIXED)
        assert e.value.code == N.NEBEM_INVALID_ARG
        with pytest.raises(N.NebemError) as e:
            N.nebem_server_wait(srv, 12345, 10)
        assert e.value.code == N.NEBEM_INVALID_ARG
    finally:
        N.nebem_server_destroy(srv)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_server_small_requests_split_by_element_chunks(N, prec):
    """Requests on the full THGEM cell (10 element chunks) of up to 16384 points run as one
    item per (point block, chunk), larger ones as one item per point block; either way the
    results equal the standalone evaluation bit for bit (sizes on both sides of the limit)."""
    g = I.thgem()
    c = N.Context().set_geometry(g)
    c.solve(N.NEBEM_MIXED)
    p = N.NEBEM_MIXED if prec == "mixed" else N.NEBEM_FP64
    sizes = [1, 50, 129, 300, 1024, 1025, 5000, 16384, 16385] if prec == "mixed" else [1, 129, 2000, 16384, 16385]
    srv = N.nebem_server_create([c.h])
    try:
        reqs = []
        for k, n in enumerate(sizes):
            pts = _request_points(g, n, 500 + k)
            phi, E = np.empty(n), np.empty((n, 3))
            reqs.append((N.nebem_server_submit(srv, 0, pts, phi, E, p), pts, phi, E))
        for rid, pts, phi, E in reqs:
            N.nebem_server_wait(srv, rid, 120000)
            rphi, rE = c.eval(pts, p)
            assert np.array_equal(phi, rphi) and np.array_equal(E, rE)
    finally:
        N.nebem_server_destroy(srv)


def test_server_refuses_contexts_it_cannot_reproduce(N):
    """The server evaluates element sums only: a context with known charges or Adaptive
    Modelling (whose nebem_eval results include them) is refused, at create and submit."""
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    c = N.Context().set_geometry(g)
    c.solve(N.NEBEM_MIXED)
    srv = N.nebem_server_create([c.h])
    try:
        N.nebem_space_charge(c.h, np.zeros((2, 3)) + 1e-4, np.array([1e-15, -1e-15]), 1e-6)
        c.solve(N.NEBEM_MIXED)
        with pytest.raises(N.NebemError) as e:
            N.nebem_server_submit(srv, 0, np.zeros((3, 3)), None, None, N.NEBEM_MIXED)
        assert e.value.code == N.NEBEM_BAD_STATE
    finally:
        N.nebem_server_destroy(srv)
    with pytest.raises(N.NebemError) as e:
        N.nebem_server_create([c.h])
    assert e.value.code == N.NEBEM_BAD_STATE
    c2 = N.Context().set_geometry(g)
    c2.solve(N.NEBEM_MIXED)
    N.nebem_set_primitives(c2.h, g.primitives, g.prim_of, 0)
    with pytest.raises(N.NebemError) as e:
        N.nebem_server_create([c2.h])
    assert e.value.code == N.NEBEM_BAD_STATE


def test_server_keeps_its_workers_under_a_trickle(N, ctxs):
    """Requests that arrive a few at a time, with gaps longer than the kernel's idle time
    and small bursts, are all served at the rate they arrive: the persistent kernel closes
    as a whole when it runs dry and is relaunched with every CTA.  (When CTAs left one by
    one, a trickle kept a few of them alive and the backlog grew to tens of seconds.)"""
    import time
    gen = I.rng(4, 77)
    n_req = 80
    gaps = gen.exponential(1.0 / 50.0, n_req)  # ~50 requests/s, Poisson
    sizes = gen.integers(1, 1000, n_req)
    geo = gen.integers(0, len(ctxs), n_req)
    reqs = []
    for k in range(n_req):
        pts = _request_points(ctxs[geo[k]][0], int(sizes[k]), 500 + k)
        reqs.append((pts, np.empty(pts.shape[0]), np.empty((pts.shape[0], 3))))
    # the single FP32 pass, far below the server's capacity at this rate: any backlog would
    # come from lost workers, not from the work itself
    single = []
    for g, c in ctxs:
        c1 = N.Context(mixed_point_tol=0.0).set_geometry(g)
        c1.set_sigma(c.sigma())
        single.append(c1)
    srv = N.nebem_server_create([c.h for c in single])
    try:
        t_arr = np.cumsum(gaps) - gaps[0]
        ids, first, i = [], 0, 0
        t0 = time.perf_counter()
        while first < n_req:
            now = time.perf_counter() - t0
            assert now < 60.0, "trickle not served"
            while i < n_req and t_arr[i] <= now:
                p, ph, E = reqs[i]
                ids.append(N.nebem_server_submit(srv, int(geo[i]), p, ph, E, N.NEBEM_MIXED))
                i += 1
            while first < i and N.nebem_server_poll(srv, ids[first]):
                first += 1
            time.sleep(50e-6)
        lat = np.array([np.subtract(*N.nebem_server_request_times(srv, r)[2::-2]) for r in ids])
        span = t_arr[-1]
        # served about as fast as they arrive: the backlog never builds up
        assert time.perf_counter() - t0 < span + 2.0
        assert np.percentile(lat, 99) < 0.5, np.percentile(lat, 99)
    finally:
        N.nebem_server_destroy(srv)

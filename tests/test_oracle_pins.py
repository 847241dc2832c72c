"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check uses an independent route
(adaptive quadrature of the defining integrals of Sec. 2.1, textbook closed values,
the far-field limit, E = -grad(phi) (Sec. 2), Gauss's law, Galerkin reciprocity, an
independent LU from numpy, refinement of the unit-cube capacitance, cube symmetry,
the interface condition of the dielectric rows checked through the evaluation path).
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I


def rect_el(v0, v1, v3):
    v0, v1, v3 = map(np.asarray, (v0, v1, v3))
    el = np.zeros(1, I.ELEMENT_DTYPE)
    el["kind"] = I.KIND_RECT
    el["v"][0] = [v0, v1, v1 + v3 - v0, v3]
    return el


def tri_el(v0, v1, v2):
    el = np.zeros(1, I.ELEMENT_DTYPE)
    el["kind"] = I.KIND_TRI
    el["v"][0, :3] = [v0, v1, v2]
    return el


def random_rect(gen, scale=1e-3):
    c = gen.normal(size=3) * scale
    u = gen.normal(size=3); u /= np.linalg.norm(u)
    w = np.cross(u, gen.normal(size=3)); w /= np.linalg.norm(w)
    L1, L2 = scale * gen.uniform(0.3, 1.5, 2)
    v0 = c - 0.5 * L1 * u - 0.5 * L2 * w
    return rect_el(v0, v0 + L1 * u, v0 + L2 * w)


def random_tri(gen, scale=1e-3):
    v = gen.normal(size=(3, 3)) * scale
    return tri_el(*v)


def quad_el(v0, v1, v2, v3):
    el = np.zeros(1, I.ELEMENT_DTYPE)
    el["kind"] = I.KIND_QUAD
    el["v"][0] = [v0, v1, v2, v3]
    return el


def random_quad(gen, scale=1e-3):
    """A planar convex quadrilateral (corners at jittered quarter angles around a centre)."""
    c = gen.normal(size=3) * scale
    u = gen.normal(size=3); u /= np.linalg.norm(u)
    w = np.cross(u, gen.normal(size=3)); w /= np.linalg.norm(w)
    while True:
        ang = np.arange(4) * 0.5 * math.pi + gen.uniform(-0.35, 0.35, 4)
        rad = scale * gen.uniform(0.6, 1.4, 4)
        q = np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
        turns = []
        for k in range(4):
            a, b = q[(k + 1) % 4] - q[k], q[(k + 2) % 4] - q[(k + 1) % 4]
            turns.append(a[0] * b[1] - a[1] * b[0])
        if min(turns) > 0.05 * scale * scale:
            break
    return quad_el(*[c + a * u + b * w for a, b in q])


def _tri_area(a, b, c):
    return 0.5 * np.linalg.norm(np.cross(b - a, c - a))


def _area(el):
    v = el["v"][0]
    k = el["kind"][0]
    if k == I.KIND_TRI:
        return _tri_area(*v[:3])
    return _tri_area(v[0], v[1], v[2]) + _tri_area(v[0], v[2], v[3])


def random_shape(gen, shape, scale=1e-3):
    return {"rect": random_rect, "tri": random_tri, "quad": random_quad}[shape](gen, scale)


def quad_influence(el, P, eps=1e-13):
    """Adaptive 2-D quadrature of Phi' and E' over the parametrised element."""
    v = el["v"][0]
    P = np.asarray(P, float)
    if el["kind"][0] == I.KIND_QUAD:  # the two triangles of the quadrilateral
        p1, E1 = quad_influence(tri_el(v[0], v[1], v[2]), P, eps)
        p2, E2 = quad_influence(tri_el(v[0], v[2], v[3]), P, eps)
        return p1 + p2, E1 + E2
    if el["kind"][0] == I.KIND_RECT:
        e1, e2 = v[1] - v[0], v[3] - v[0]
        jac = np.linalg.norm(np.cross(e1, e2))
        top = lambda s: 1.0
    else:
        e1, e2 = v[1] - v[0], v[2] - v[0]
        jac = np.linalg.norm(np.cross(e1, e2))
        top = lambda s: 1.0 - s

    def comp(k):
        def f(t, s):
            x = v[0] + s * e1 + t * e2
            d = P - x
            r = math.sqrt(d @ d)
            return jac / r if k < 0 else jac * d[k] / r**3
        return integrate.dblquad(f, 0.0, 1.0, 0.0, top, epsabs=0.0, epsrel=eps)[0]

    return comp(-1), np.array([comp(0), comp(1), comp(2)])


def _normal(el):
    v = el["v"][0]
    n = np.cross(v[1] - v[0], v[2] - v[0])
    return n / np.linalg.norm(n)


def _centroid(el):
    v = el["v"][0]
    if el["kind"][0] == I.KIND_QUAD:
        a1, a2 = _tri_area(v[0], v[1], v[2]), _tri_area(v[0], v[2], v[3])
        return (a1 * v[:3].mean(0) + a2 * v[[0, 2, 3]].mean(0)) / (a1 + a2)
    return v[:4].mean(0) if el["kind"][0] == I.KIND_RECT else v[:3].mean(0)


@pytest.mark.parametrize("shape", ["rect", "tri", "quad"])
def test_closed_form_vs_quadrature(shape):
    gen = np.random.default_rng(7)
    worst = 0.0
    for trial in range(6):
        el = random_shape(gen, shape)
        c, n = _centroid(el), _normal(el)
        size = math.sqrt(_area(el))
        for dist, h in [(0.3, 0.2), (1.0, 0.5), (3.0, 1.0), (0.2, 0.05), (2.0, -0.7)]:
            dirn = gen.normal(size=3); dirn -= (dirn @ n) * n; dirn /= np.linalg.norm(dirn)
            P = c + dist * size * dirn + h * size * n
            phi, E = O.influence(el, P)
            qphi, qE = quad_influence(el, P)
            worst = max(worst, abs(phi[0] - qphi) / abs(qphi),
                        np.abs(E[0] - qE).max() / np.abs(qE).max())
    assert worst < 2e-11, worst


def test_rect_equals_two_triangles():
    gen = np.random.default_rng(11)
    cases = [random_rect(gen) for _ in range(20)]
    # an exactly axis-aligned rectangle (local normal coordinate of in-plane points is 0)
    cases.append(rect_el([-1e-3, -0.5e-3, 0.0], [1e-3, -0.5e-3, 0.0], [-1e-3, 0.7e-3, 0.0]))
    for ci, el in enumerate(cases):
        v = el["v"][0]
        t1, t2 = tri_el(v[0], v[1], v[2]), tri_el(v[0], v[2], v[3])
        c, n = _centroid(el), _normal(el)
        size = math.sqrt(np.linalg.norm(np.cross(v[1] - v[0], v[3] - v[0])))
        P = [c + size * gen.normal(size=3) * s for s in (0.1, 0.7, 3.0, 30.0)]
        if ci == len(cases) - 1:
            # in-plane points: inside (off the diagonal) and outside the element
            P += [np.array([0.3e-3, -0.2e-3, 0.0]), np.array([2.5e-3, 0.1e-3, 0.0]),
                  np.array([-0.4e-3, 0.6e-3, 0.0])]
        P = np.array(P)
        pr, Er = O.influence(el, P)
        pa, Ea = O.influence(t1, P)
        pb, Eb = O.influence(t2, P)
        scale_p = np.abs(pr).max()
        assert np.abs(pr - (pa + pb)).max() <= 1e-12 * scale_p
        assert np.abs(Er - (Ea + Eb)).max() <= 1e-11 * max(1.0, np.abs(Er).max())
        # the polygon form of the rectangle agrees too (two independent formulas)
        pp, Ep = O.influence(el, P, poly=True)
        assert np.abs(pr - pp).max() <= 1e-12 * scale_p
        assert np.abs(Er - Ep).max() <= 1e-11 * max(1.0, np.abs(Er).max())


def test_quad_equals_two_triangles_and_rect():
    """A quadrilateral's edge formula equals the sum of its two triangles, and a
    rectangle given as a quadrilateral equals the rectangle's corner antiderivative."""
    gen = np.random.default_rng(23)
    for _ in range(4):
        q = random_quad(gen)
        v = q["v"][0]
        size = math.sqrt(_area(q))
        P = _centroid(q) + size * gen.normal(size=(6, 3))
        phi, E = O.influence(q, P)
        p1, E1 = O.influence(tri_el(v[0], v[1], v[2]), P)
        p2, E2 = O.influence(tri_el(v[0], v[2], v[3]), P)
        assert np.abs(phi - (p1 + p2)).max() <= 1e-13 * np.abs(phi).max()
        assert np.abs(E - (E1 + E2)).max() <= 1e-12 * np.abs(E).max()
    r = random_rect(gen)
    rq = quad_el(*r["v"][0])
    P = _centroid(r) + 1e-3 * gen.normal(size=(6, 3))
    pr, Er = O.influence(r, P)
    pq, Eq = O.influence(rq, P)
    assert np.abs(pr - pq).max() <= 1e-13 * np.abs(pr).max() and np.abs(Er - Eq).max() <= 1e-12 * np.abs(Er).max()
    # the oracle's collocation point of a quadrilateral is its area centroid
    c, _, area = O.centroids(I.Geometry(name="q", elements=q, voltages=np.array([1.0])))
    assert np.allclose(c[0], _centroid(q), rtol=0, atol=1e-15) and abs(area[0] - _area(q)) <= 1e-15 * _area(q)
    # non-planar and non-convex quadrilaterals are rejected
    bent = q.copy(); bent["v"][0][3] += 1e-4 * _normal(q)
    with pytest.raises(ValueError):
        O.influence(bent, P)
    dart = quad_el(v[0], v[1], v[0] + 0.1 * (v[2] - v[0]), v[3])
    with pytest.raises(ValueError):
        O.influence(dart, P)


def test_square_textbook_values():
    a = 2e-3
    el = rect_el([0, 0, 0], [a, 0, 0], [0, a, 0])  # in the z=0 plane, normal +z
    phi, E = O.influence(el, [[a / 2, a / 2, 0.0]])
    assert abs(phi[0] - 4 * a * math.log(1 + math.sqrt(2))) < 1e-14 * a * 10
    assert np.abs(E).max() < 1e-12
    b = a / 2
    for h in [1e-6, 1e-4, 1e-3, 1e-2, 1.0]:
        _, E = O.influence(el, [[b, b, h]])
        omega = 4 * math.atan(b * b / (h * math.sqrt(2 * b * b + h * h)))
        assert abs(E[0, 2] - omega) <= 1e-13 * max(omega, 1e-300) + 1e-300
        assert abs(E[0, 0]) < 1e-12 and abs(E[0, 1]) < 1e-12


def test_normal_jump_and_principal_value():
    gen = np.random.default_rng(3)
    for el in [random_rect(gen), random_tri(gen)]:
        c, n = _centroid(el), _normal(el)
        size = 1e-3
        for delta in [1e-9 * size, 1e-12 * size]:
            _, Ep = O.influence(el, c + delta * n)
            _, Em = O.influence(el, c - delta * n)
            jump = (Ep[0] - Em[0]) @ n
            assert abs(jump - 4 * math.pi) < 1e-6
    # principal value exactly in the plane: the mean of the one-sided limits, i.e. no
    # normal component (axis-aligned element, so the in-plane point is exact)
    el = rect_el([-1e-3, -1e-3, 0.0], [1e-3, -1e-3, 0.0], [-1e-3, 0.5e-3, 0.0])
    P = np.array([[0.2e-3, -0.1e-3, 0.0]])
    _, E0 = O.influence(el, P)
    _, Ep = O.influence(el, P + [0, 0, 1e-15])
    _, Em = O.influence(el, P - [0, 0, 1e-15])
    assert E0[0, 2] == 0.0
    assert np.allclose(E0[0], 0.5 * (Ep[0] + Em[0]), rtol=1e-9, atol=1e-9)


def test_self_term_principal_value_in_fill():
    gen = np.random.default_rng(5)
    el = np.concatenate([random_tri(gen), random_rect(gen)])
    el["bc"] = I.BC_DIELECTRIC
    el["eps_a"], el["eps_b"] = 4.4, 1.0
    g = I.Geometry("pv", el, np.array([0.0]))
    K = O.fill(g)
    # the element's own normal field at its centroid is zero (principal value): the
    # diagonal equals the interface term alone
    diag = (4.4 + 1.0) / (2 * O.eps0() * (1.0 - 4.4))
    assert np.allclose(np.diag(K), diag, rtol=1e-14)


@pytest.mark.parametrize("shape", ["rect", "tri", "quad"])
def test_far_field_limit(shape):
    gen = np.random.default_rng(13)
    el = random_shape(gen, shape)
    A = _area(el)
    c = _centroid(el)
    size = math.sqrt(A)
    errs = []
    for R in [30.0, 300.0, 3000.0]:
        d = gen.normal(size=3); d /= np.linalg.norm(d)
        P = c + R * size * d
        phi, E = O.influence(el, P)
        r = R * size
        errs.append((abs(phi[0] * r / A - 1.0), np.linalg.norm(E[0] * r * r / A - d)))
    # monopole limit with O((a/r)^2) error: each decade of distance gains ~2 decades
    assert errs[0][0] < 5e-3 and errs[1][0] < 5e-5 and errs[2][0] < 5e-7
    assert errs[0][1] < 5e-3 and errs[1][1] < 5e-5 and errs[2][1] < 5e-7


@pytest.mark.parametrize("shape", ["rect", "tri", "quad"])
def test_field_is_minus_gradient(shape):
    gen = np.random.default_rng(17)
    el = random_shape(gen, shape)
    c, n = _centroid(el), _normal(el)
    size = 1e-3
    for P in [c + size * gen.normal(size=3) for _ in range(5)] + [c + 0.01 * size * n + 0.1 * size * gen.normal(size=3)]:
        h = 1e-5 * size
        _, E = O.influence(el, P)
        g = np.zeros(3)
        for k in range(3):
            dp = np.zeros(3); dp[k] = h
            pp, _ = O.influence(el, P + dp)
            pm, _ = O.influence(el, P - dp)
            g[k] = (pp[0] - pm[0]) / (2 * h)
        assert np.abs(E[0] + g).max() <= 1e-7 * max(1.0, np.abs(E[0]).max())


def _box_flux(field_fn, lo, hi, m=40):
    x, w = np.polynomial.legendre.leggauss(m)
    total = 0.0
    for ax in range(3):
        u_ax, w_ax = (ax + 1) % 3, (ax + 2) % 3
        su = 0.5 * (hi[u_ax] - lo[u_ax]); sw = 0.5 * (hi[w_ax] - lo[w_ax])
        cu = 0.5 * (hi[u_ax] + lo[u_ax]); cw = 0.5 * (hi[w_ax] + lo[w_ax])
        U, W = np.meshgrid(cu + su * x, cw + sw * x, indexing="ij")
        WT = np.outer(w, w) * su * sw
        for side, sgn in ((hi[ax], 1.0), (lo[ax], -1.0)):
            P = np.zeros((m * m, 3))
            P[:, ax] = side; P[:, u_ax] = U.ravel(); P[:, w_ax] = W.ravel()
            E = field_fn(P)
            total += sgn * (E[:, ax] * WT.ravel()).sum()
    return total


@pytest.mark.parametrize("shape", ["rect", "tri", "quad"])
def test_gauss_law_single_element(shape):
    gen = np.random.default_rng(19)
    el = random_shape(gen, shape, 1.0)
    v = el["v"][0][: (3 if shape == "tri" else 4)]
    A = _area(el)
    lo, hi = v.min(0) - 1.0, v.max(0) + 1.0
    flux = _box_flux(lambda P: O.influence(el, P)[1], lo, hi)
    assert abs(flux - 4 * math.pi * A) < 1e-9 * 4 * math.pi * A
    lo2 = hi + 0.5
    flux0 = _box_flux(lambda P: O.influence(el, P)[1], lo2, lo2 + 1.0)
    assert abs(flux0) < 1e-10 * 4 * math.pi * A


def _surface_integral(el, fn, m=24):
    """Gauss-Legendre integral of fn over an element (collapsed map for triangles)."""
    x, w = np.polynomial.legendre.leggauss(m)
    s = 0.5 * (x + 1.0); ws = 0.5 * w
    S, T = np.meshgrid(s, s, indexing="ij")
    W = np.outer(ws, ws)
    v = el["v"][0]
    if el["kind"][0] == I.KIND_RECT:
        e1, e2 = v[1] - v[0], v[3] - v[0]
        jac = np.linalg.norm(np.cross(e1, e2))
        P = v[0] + S.ravel()[:, None] * e1 + T.ravel()[:, None] * e2
        return (fn(P) * W.ravel()).sum() * jac
    e1, e2 = v[1] - v[0], v[2] - v[0]
    jac = np.linalg.norm(np.cross(e1, e2))
    a, b = S.ravel(), (T * (1.0 - S)).ravel()
    P = v[0] + a[:, None] * e1 + b[:, None] * e2
    return (fn(P) * W.ravel() * (1.0 - S.ravel())).sum() * jac


def test_galerkin_reciprocity():
    gen = np.random.default_rng(23)
    for trial in range(4):
        ei = random_rect(gen) if trial % 2 else random_tri(gen)
        ej = random_tri(gen)
        ej["v"] += np.array([3e-3, 1e-3, -2e-3])
        a = _surface_integral(ei, lambda P: O.influence(ej, P)[0])
        b = _surface_integral(ej, lambda P: O.influence(ei, P)[0])
        assert abs(a - b) <= 1e-9 * abs(a)


def test_image_sum_equals_explicit_copies():
    g = I.thgem(I.PlateSpec(n_phi=12, n_r=1, n_zc=1, n_zf=2), n_plane=1)
    g.img_lo, g.img_hi = -1, 1
    t = O.image_table(g.lattice, -1, 1)
    # explicit superposition of translated copies, without images
    copies = []
    for k in range(t.shape[0]):
        e = g.elements.copy()
        e["v"] = e["v"] + t[k]
        if e["kind"][0] == I.KIND_TRI:
            pass
        copies.append(e)
    big = np.concatenate(copies)
    # triangles keep v[3] = 0 as padding: restore the padding after the shift
    tri = big["kind"] == I.KIND_TRI
    big["v"][tri, 3] = 0.0
    gb = I.Geometry("copies", big, g.voltages)
    sigma = np.random.default_rng(1).normal(size=g.n)
    P = I.cell_points(g, 50, I.rng(99))
    p1, E1 = O.eval_points(g, sigma, P)
    p2, E2 = O.eval_points(gb, np.tile(sigma, t.shape[0]), P)
    assert np.abs(p1 - p2).max() <= 1e-11 * np.abs(p1).max()
    assert np.abs(E1 - E2).max() <= 1e-11 * np.abs(E1).max()
    # image index order: k = (k1 - lo) * m + (k2 - lo)
    a1, a2 = g.lattice
    assert np.array_equal(t[0], -a1 - a2) and np.array_equal(t[1], -a1) and np.array_equal(t[3], -a2)
    assert np.array_equal(t[4], np.zeros(3)) and np.array_equal(t[8], a1 + a2)


def test_lu_matches_numpy_and_tie_break():
    gen = np.random.default_rng(29)
    n = 60
    K = gen.normal(size=(n, n)) + n * 0.1 * np.eye(n)
    b = gen.normal(size=n)
    x = O.lu_solve(O.lu_factor(K), b)
    xr = np.linalg.solve(K, b)
    assert np.abs(x - xr).max() <= 1e-12 * np.abs(xr).max()
    # ties: equal |a| in column 0 -> the lowest index is the pivot (no swap at step 0)
    T = np.array([[2.0, 1.0, 0.0], [-2.0, 3.0, 1.0], [2.0, 0.0, 5.0]])
    _, piv = O.lu_factor(T)
    assert piv[0] == 0
    T2 = np.array([[1.0, 1.0, 0.0], [-2.0, 3.0, 1.0], [2.0, 0.0, 5.0]])
    _, piv2 = O.lu_factor(T2)
    assert piv2[0] == 1
    # backward error of the factorisation on a BEM matrix
    g = I.cube(n_per_edge=4)
    Kc = O.fill(g)
    sig = O.lu_solve(O.lu_factor(Kc), O.rhs(g))
    r = Kc @ sig - O.rhs(g)
    assert np.abs(r).max() / (np.abs(Kc).max() * np.abs(sig).max() * g.n) < 1e-15


def _capacitance(n_edge):
    g = I.cube(edge=0.01, n_per_edge=n_edge)
    sigma, K, fac = O.solve(g)
    _, _, area = O.centroids(g)
    return (sigma * area).sum() / 1.0 / (4 * math.pi * O.eps0() * 0.01), g, sigma


def test_cube_capacitance_refinement():
    c4, _, _ = _capacitance(4)
    c8, _, _ = _capacitance(8)
    c12, _, _ = _capacitance(12)
    ref = 0.6607
    # constant-element collocation approaches the unit-cube value monotonically
    assert c4 < c8 < c12 < ref + 2e-3
    assert abs(c12 - ref) < abs(c8 - ref) < abs(c4 - ref)
    assert abs(c8 - ref) < 0.01 * ref


def test_cube_symmetry_and_gauss():
    cap, g, sigma = _capacitance(8)
    c, nr, area = O.centroids(g)
    key = {tuple(np.round(ci / 1e-6).astype(int)): i for i, ci in enumerate(c)}
    perms = [(0, 1, 2), (1, 2, 0), (2, 0, 1), (1, 0, 2), (0, 2, 1), (2, 1, 0)]
    for perm in perms:
        for signs in [(1, 1, 1), (-1, 1, 1), (1, -1, -1), (-1, -1, -1)]:
            cc = c[:, perm] * np.array(signs)
            idx = [key[tuple(np.round(x / 1e-6).astype(int))] for x in cc]
            assert np.abs(sigma[idx] - sigma).max() <= 1e-12 * np.abs(sigma).max()
    P = np.random.default_rng(2).uniform(-0.02, 0.02, (20, 3))
    p1, E1 = O.eval_points(g, sigma, P)
    p2, E2 = O.eval_points(g, sigma, -P)
    assert np.abs(p1 - p2).max() <= 1e-12 * np.abs(p1).max()
    assert np.abs(E1 + E2).max() <= 1e-11 * np.abs(E1).max()
    # Gauss's law on the solved charge: flux through an enclosing box = Q / eps0
    Q = (sigma * area).sum()
    flux = _box_flux(lambda X: O.eval_points(g, sigma, X)[1], np.full(3, -0.015), np.full(3, 0.015), m=32)
    assert abs(flux - Q / O.eps0()) < 1e-8 * Q / O.eps0()
    # potential on the conductor away from collocation points is close to 1 V
    v = g.elements["v"][0]
    P_edge = 0.25 * v[0] + 0.75 * v[2]
    ph, _ = O.eval_points(g, sigma, P_edge[None])
    assert abs(ph[0] - 1.0) < 0.05


def _slab_capacitor():
    """Two conductor plates around a dielectric slab (square lattice, +-3 images)."""
    p = 1e-3
    b = I._Builder()
    m = 3
    xs = np.linspace(-p / 2, p / 2, m + 1)

    def sheet(z, up, bc, cond, ea=1.0, eb=1.0):
        for i in range(m):
            for j in range(m):
                v0 = [xs[i], xs[j], z]
                v1 = [xs[i + 1], xs[j], z]
                v3 = [xs[i], xs[j + 1], z]
                v2 = [xs[i + 1], xs[j + 1], z]
                if up:
                    b.rect(v0, v1, v2, v3, bc, cond, ea, eb)
                else:
                    b.rect(v0, v3, v2, v1, bc, cond, ea, eb)

    sheet(1e-3, True, I.BC_CONDUCTOR, 0)
    sheet(-1e-3, True, I.BC_CONDUCTOR, 1)
    sheet(0.4e-3, True, I.BC_DIELECTRIC, -1, 4.0, 1.0)   # slab top: slab below (-n side)
    sheet(-0.4e-3, False, I.BC_DIELECTRIC, -1, 4.0, 1.0)  # slab bottom: normal -z, slab above
    lat = np.array([[p, 0, 0], [0, p, 0]])
    return I.Geometry("slab", b.build(), np.array([100.0, 0.0]), lattice=lat, img_lo=-3, img_hi=3)


def test_dielectric_interface_condition():
    g = _slab_capacitor()
    sigma, K, fac = O.solve(g)
    c, nr, _ = O.centroids(g)
    diel = np.where(g.elements["bc"] == I.BC_DIELECTRIC)[0]
    d = 1e-9
    _, Eb = O.eval_points(g, sigma, c[diel] + d * nr[diel])   # +n side (eps_b)
    _, Ea = O.eval_points(g, sigma, c[diel] - d * nr[diel])   # -n side (eps_a)
    ea = g.elements["eps_a"][diel]; eb = g.elements["eps_b"][diel]
    Dn_a = ea * (Ea * nr[diel]).sum(1)
    Dn_b = eb * (Eb * nr[diel]).sum(1)
    assert np.abs(Dn_a - Dn_b).max() <= 1e-5 * np.abs(Dn_a).max()
    # the slab weakens the field inside it: E_slab / E_gas close to 1/eps_r at the centre
    _, Ein = O.eval_points(g, sigma, np.array([[0, 0, 0.0]]))
    _, Eout = O.eval_points(g, sigma, np.array([[0, 0, 0.7e-3]]))
    assert 0.2 < Ein[0, 2] / Eout[0, 2] < 0.3


def test_space_charge_invariants():
    gen = np.random.default_rng(31)
    n = 300
    pos = gen.normal(size=(n, 3)) * 1e-4
    q = np.where(gen.random(n) < 0.5, 1.0, -1.0) * I.E_CHARGE
    phi, E = O.space_charge(pos, q, soft=1e-6)
    # Newton's third law: the total force on the cloud vanishes
    F = (q[:, None] * E).sum(0)
    assert np.abs(F).max() <= 1e-12 * (np.abs(q[:, None] * E)).sum()
    # the interaction energy is symmetric: sum_t q_t phi_t == sum over ordered pairs
    # self exclusion by index: removing carrier 0 and evaluating at its position
    p0, E0 = O.space_charge(pos[1:], q[1:], tgt=pos[:1], soft=1e-6)
    assert abs(p0[0] - phi[0]) <= 1e-14 * abs(phi[0]) and np.allclose(E0[0], E[0], rtol=1e-13, atol=0)
    # symmetric cloud: field at the centre vanishes
    sym = np.concatenate([pos, -pos]); qs = np.concatenate([q, q])
    _, Ec = O.space_charge(sym, qs, tgt=np.zeros((1, 3)), soft=1e-6)
    assert np.abs(Ec).max() <= 1e-12 * np.abs(E).max()
    # a distant same-sign cluster looks like a point charge at its charge centroid
    far = np.array([[1.0, 0.0, 0.0]])
    pf, Ef = O.space_charge(pos, np.abs(q), tgt=far, soft=1e-6)
    Qt = np.abs(q).sum()
    r = np.linalg.norm(far[0] - pos.mean(0))
    assert abs(pf[0] / (O.ke() * Qt / r) - 1) < 1e-7


def test_known_charge_rhs_and_dynamic_step():
    g = I.cube(n_per_edge=4)
    sigma0, K, fac = O.solve(g)
    c, nr, _ = O.centroids(g)
    gen = np.random.default_rng(37)
    pos = gen.normal(size=(40, 3)) * 2e-3 + np.array([0.0, 0.0, 0.012])
    q = np.where(gen.random(40) < 0.5, 1.0, -1.0) * 1e-15
    pos1, sigma, E = O.dynamic_step(g, fac, pos, q)
    # with the known charges, the total potential at every collocation point is the BC
    pe, _ = O.eval_points(g, sigma, c)
    ps, _ = O.space_charge(pos, q, tgt=c, soft=1e-6)
    assert np.abs(pe + ps - 1.0).max() < 1e-10
    # sigma is affine in q
    _, sigma2, _ = O.dynamic_step(g, fac, pos, 2 * q)
    assert np.abs((sigma2 - sigma0) - 2 * (sigma - sigma0)).max() <= 1e-9 * np.abs(sigma - sigma0).max()
    # carriers move along sign(q) mu E dt
    step = np.sign(q)[:, None] * 1e-4 * E * 1e-9
    tol = 4e-16 * np.abs(pos).max()
    assert np.abs(pos1 - (pos + step)).max() <= tol
    # the displacement is far above that tolerance, so the check above sees the step
    # (a dropped or mis-signed drift term would fail it)
    assert np.abs(step).max() > 1e3 * tol


# --- line-charge representation (Sec. 4.2, Alg. 3; LineCh in Alg. 4) ---------------

def _cloud(seed, n=300, scale=30e-6):
    gen = np.random.default_rng(seed)
    pos = gen.normal(scale=scale, size=(n, 3))
    q = gen.choice([-1.0, 1.0], n) * I.E_CHARGE * gen.integers(1, 5, n)
    return pos, q


def test_voxel_lines_brute_force():
    """Alg. 3 against an assignment by geometric containment: every voxel of the grid
    is visited and the points with lo + i d <= x < lo + (i+1) d (per axis) are summed
    in point order; the occupied voxels are exactly the oracle's lines, in voxel order."""
    pos, q = _cloud(3)
    d = np.array([12e-6, 15e-6, 20e-6])
    L = O.voxel_lines(pos, q, d)
    lo = pos.min(0)
    dims = (np.floor((pos.max(0) - lo) / d) + 1).astype(np.int64)
    assert np.array_equal(O.voxel_grid(pos, d)[1], dims)
    starts, lams, vox = [], [], []
    for k in range(dims[2]):
        for j in range(dims[1]):
            for i in range(dims[0]):
                idx = np.array([i, j, k])
                inside = np.all((pos >= lo + idx * d) & ((pos < lo + (idx + 1) * d) | (idx == dims - 1)), axis=1)
                if not inside.any():
                    continue
                Q = 0.0
                for p in np.nonzero(inside)[0]:
                    Q += q[p]
                vox.append((k * dims[1] + j) * dims[0] + i)
                starts.append([lo[0] + (i + 0.5) * d[0], lo[1] + (j + 0.5) * d[1], lo[2] + k * d[2]])
                lams.append(Q / d[2])
    assert np.array_equal(L.voxel, vox)
    assert np.array_equal(L.start, np.array(starts))
    assert np.array_equal(L.stop[:, :2], L.start[:, :2]) and np.array_equal(L.stop[:, 2], L.start[:, 2] + d[2])
    assert np.array_equal(L.lam, np.array(lams))
    # charge is conserved
    assert abs((L.lam * d[2]).sum() - q.sum()) <= 1e-14 * np.abs(q).sum()
    # a voxel as large as the cloud gives one line with all the charge
    big = O.voxel_lines(pos, q, [1.0, 1.0, 1.0])
    assert len(big) == 1 and abs(big.lam[0] - q.sum()) <= 1e-14 * np.abs(q).sum()


def _line_quad(A, B, lam, P, s):
    u = B - A
    Ln = np.linalg.norm(u)
    u = u / Ln

    def r(t):
        return P - A - t * u

    def f(t, k):
        rr = r(t)
        R2 = rr @ rr + s * s
        return 1.0 / math.sqrt(R2) if k < 0 else rr[k] / R2 ** 1.5

    opts = dict(epsabs=0.0, epsrel=1e-13, limit=200)
    phi = integrate.quad(f, 0.0, Ln, args=(-1,), **opts)[0]
    E = np.array([integrate.quad(f, 0.0, Ln, args=(k,), **opts)[0] for k in range(3)])
    return O.ke() * lam * phi, O.ke() * lam * E


def test_line_charge_vs_quadrature():
    gen = np.random.default_rng(41)
    for trial in range(6):
        A = gen.normal(size=3) * 1e-4
        B = A + gen.normal(size=3) * 5e-5
        lam = gen.normal() * 1e-9
        lines = O.Lines(A[None], B[None], np.array([lam]))
        s = [0.0, 1e-6][trial % 2]
        P = np.stack([A + gen.normal(size=3) * 1e-4 for _ in range(4)] + [0.5 * (A + B) + 2e-6 * gen.normal(size=3)])
        phi, E = O.line_charge(lines, P, soft=s)
        for p in range(P.shape[0]):
            rp, rE = _line_quad(A, B, lam, P[p], s)
            assert abs(phi[p] - rp) <= 1e-11 * abs(rp)
            assert np.abs(E[p] - rE).max() <= 1e-10 * np.linalg.norm(rE)


def test_line_charge_textbook_values():
    ke, lam, Ln = O.ke(), 3e-10, 2e-4
    A, B = np.zeros(3), np.array([0.0, 0.0, Ln])
    lines = O.Lines(A[None], B[None], np.array([lam]))
    # on the axis beyond the end (no softening): ke lam ln((d+L)/d), E_z = ke lam (1/d - 1/(d+L))
    dd = 7e-5
    phi, E = O.line_charge(lines, np.array([[0.0, 0.0, Ln + dd]]), soft=0.0)
    assert abs(phi[0] - ke * lam * math.log((dd + Ln) / dd)) <= 1e-14 * abs(phi[0])
    assert abs(E[0, 2] - ke * lam * (1 / dd - 1 / (dd + Ln))) <= 1e-13 * abs(E[0, 2])
    assert np.abs(E[0, :2]).max() <= 1e-12 * abs(E[0, 2])
    # beside the midpoint: E_perp = ke lam L / (rho sqrt(rho^2 + L^2/4)), E_z = 0
    rho = 3e-5
    phi, E = O.line_charge(lines, np.array([[rho, 0.0, Ln / 2]]), soft=0.0)
    assert abs(E[0, 0] - ke * lam * Ln / (rho * math.sqrt(rho ** 2 + Ln ** 2 / 4))) <= 1e-13 * abs(E[0, 0])
    assert abs(E[0, 2]) <= 1e-12 * abs(E[0, 0])
    assert abs(phi[0] - 2 * ke * lam * math.asinh(Ln / 2 / rho)) <= 1e-14 * abs(phi[0])
    # far field: a point charge lam L
    for R, tol in [(1e-2, 1e-3), (1e-1, 1e-5)]:
        P = np.array([[R * 0.6, 0.0, Ln / 2 + R * 0.8]])
        phi, E = O.line_charge(lines, P, soft=1e-6)
        assert abs(phi[0] * R / (ke * lam * Ln) - 1) < tol


def test_line_charge_gauss_law_and_gradient():
    lam, Ln = 1e-9, 1.0
    A, B = np.array([0.1, -0.2, 0.3]), np.array([0.1, -0.2, 0.3]) + np.array([0.48, 0.6, 0.64]) * Ln
    lines = O.Lines(A[None], B[None], np.array([lam]))
    lo, hi = np.minimum(A, B) - 0.7, np.maximum(A, B) + 0.7
    flux = _box_flux(lambda P: O.line_charge(lines, P, soft=0.0)[1], lo, hi, m=60)
    assert abs(flux - lam * Ln / O.eps0()) <= 1e-7 * lam * Ln / O.eps0()
    # E = -grad phi, softened and not
    gen = np.random.default_rng(43)
    for s in (0.0, 0.05):
        for P in [A + gen.normal(size=3) * 0.5 for _ in range(4)]:
            _, E = O.line_charge(lines, P[None], soft=s)
            h, g = 1e-5, np.zeros(3)
            for k in range(3):
                dp = np.zeros(3); dp[k] = h
                g[k] = (O.line_charge(lines, (P + dp)[None], soft=s)[0][0]
                        - O.line_charge(lines, (P - dp)[None], soft=s)[0][0]) / (2 * h)
            assert np.abs(E[0] + g).max() <= 1e-7 * np.abs(E[0]).max()


def test_line_rhs_tends_to_point_rhs():
    """A carrier at the centre of its own small voxel becomes a short line centred on it,
    so the line-charge RHS equals the point-charge RHS up to O((dz / r)^2) (Alg. 4,
    Type == Line vs Type == Point).  Two uncharged carriers fix the grid's corner."""
    g = I.cube(n_per_edge=4)
    gen = np.random.default_rng(47)
    d = 1e-6
    pos = gen.normal(size=(30, 3)) * 2e-3 + np.array([0.0, 0.0, 0.012])
    q = np.where(gen.random(30) < 0.5, 1.0, -1.0) * 1e-15
    lo = pos.min(0) - 10 * d
    pos = lo + (np.floor((pos - lo) / d) + 0.5) * d
    cloud = np.concatenate([lo[None], pos, (pos.max(0) + 10 * d)[None]])
    qc = np.concatenate([[0.0], q, [0.0]])
    L = O.voxel_lines(cloud, qc, [d, d, d])
    assert len(L) == 32 and (L.lam != 0).sum() == 30
    mid = 0.5 * (L.start + L.stop)
    assert np.abs(np.sort(mid[L.lam != 0], axis=0) - np.sort(pos, axis=0)).max() <= 1e-15
    b_pt = O.rhs_space_charge(g, pos, q)
    b_ln = O.rhs_lines(g, L)
    b0 = O.rhs(g)
    assert np.abs((b_ln - b0) - (b_pt - b0)).max() <= 1e-6 * np.abs(b_pt - b0).max()
    with pytest.raises(ValueError):
        O.voxel_lines(pos, q, [1e-12, 1e-12, 1e-12])  # 1e27 voxels: rejected


def test_dynamic_step_lines_satisfies_bc():
    g = I.cube(n_per_edge=4)
    _, _, fac = O.solve(g)
    c, _, _ = O.centroids(g)
    gen = np.random.default_rng(53)
    pos = gen.normal(size=(200, 3)) * 5e-4 + np.array([0.0, 0.0, 0.009])
    q = np.where(gen.random(200) < 0.5, 1.0, -1.0) * 1e-14
    d = np.array([3e-4, 3e-4, 4e-4])
    pos1, sigma, E = O.dynamic_step_lines(g, fac, pos, q, d)
    L = O.voxel_lines(pos, q, d)
    # with the lines as known charges, the total potential at every collocation point is the BC
    pe, Ee = O.eval_points(g, sigma, c)
    pl, _ = O.line_charge(L, c)
    assert np.abs(pe + pl - 1.0).max() < 1e-10
    # E at the carriers is the elements' field plus the lines' field
    _, Ec = O.eval_points(g, sigma, pos)
    _, El = O.line_charge(L, pos)
    assert np.abs(E - (Ec + El)).max() <= 1e-12 * np.abs(E).max()
    assert np.abs(pos1 - (pos + np.sign(q)[:, None] * 1e-4 * E * 1e-9)).max() <= 4e-16 * np.abs(pos).max()


# --- Adaptive Modelling (Sec. 3.3; PrimAfter) ----------------------------------------

def _am_geometry(lo=-3, hi=3):
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    g.img_lo, g.img_hi = lo, hi
    return g


def _smooth_sigma(g):
    c, _, _ = O.centroids(g)
    return 1e-9 * (1.0 + 0.5 * np.sin(7e3 * c[:, 0]) * np.cos(5e3 * c[:, 1]) + 3e2 * c[:, 2])


def test_am_exact_for_uniform_primitive_charge():
    """With the charge density uniform over every primitive, a primitive's influence is
    the sum of its elements' (additivity of the surface integral), so the adaptive
    evaluation equals the full one for any PrimAfter."""
    g = _am_geometry()
    rough = _smooth_sigma(g)
    _, _, area = O.centroids(g)
    # per-primitive uniform density (the primitive average of the rough one)
    pa = np.bincount(g.prim_of, weights=area)
    sbar = np.bincount(g.prim_of, weights=rough * area) / pa
    sigma = sbar[g.prim_of]
    pts = I.cell_points(g, 40, I.rng(0, 60))
    full_phi, full_E = O.eval_points(g, sigma, pts)
    for pa_ in (0, 1, 2):
        phi, E = O.eval_am(g, sigma, g.primitives, g.prim_of, pa_, pts)
        assert np.abs(phi - full_phi).max() <= 1e-12 * np.abs(full_phi).max()
        assert np.abs(E - full_E).max() <= 1e-11 * np.abs(full_E).max()


def test_am_limits_and_trend():
    """PrimAfter < 0 or beyond the last ring is the plain evaluation; for a density that
    varies inside the primitives the error falls as PrimAfter grows (the trend of the
    paper's PrimAfter table)."""
    g = _am_geometry()
    sigma = _smooth_sigma(g)
    pts = I.cell_points(g, 40, I.rng(0, 61))
    full_phi, full_E = O.eval_points(g, sigma, pts)
    for pa_ in (-1, 3, 7):
        phi, E = O.eval_am(g, sigma, g.primitives, g.prim_of, pa_, pts)
        assert np.abs(phi - full_phi).max() <= 1e-13 * np.abs(full_phi).max()
        assert np.abs(E - full_E).max() <= 1e-12 * np.abs(full_E).max()
    errs = []
    for pa_ in (0, 1, 2):
        phi, E = O.eval_am(g, sigma, g.primitives, g.prim_of, pa_, pts)
        errs.append(max(np.abs(phi - full_phi).max() / np.abs(full_phi).max(),
                        np.abs(E - full_E).max() / np.abs(full_E).max()))
    assert errs[0] > errs[1] > errs[2] > 0.0
    assert errs[2] < 1e-3


def test_am_unassigned_elements_and_bad_tiling():
    g = _am_geometry(-2, 2)
    sigma = _smooth_sigma(g)
    pts = I.cell_points(g, 10, I.rng(0, 62))
    # an element without a primitive stands for itself in every copy: dropping the
    # primitives of a set of elements moves the result towards the full evaluation
    po = g.prim_of.copy()
    po[po < 40] = -1
    keep = np.unique(po[po >= 0])
    remap = -np.ones(len(g.primitives), dtype=np.int32)
    remap[keep] = np.arange(len(keep))
    po2 = np.where(po >= 0, remap[np.maximum(po, 0)], -1).astype(np.int32)
    full_phi, _ = O.eval_points(g, sigma, pts)
    a_phi, _ = O.eval_am(g, sigma, g.primitives, g.prim_of, 0, pts)
    b_phi, _ = O.eval_am(g, sigma, g.primitives[keep], po2, 0, pts)
    assert np.abs(b_phi - full_phi).max() < np.abs(a_phi - full_phi).max()
    # elements that do not tile their primitive are rejected
    bad = g.prim_of.copy()
    bad[0] = bad[1] if bad[1] != bad[0] else bad[0] + 1
    with pytest.raises(ValueError):
        O.eval_am(g, sigma, g.primitives, bad, 0, pts)


def test_thgem_inversion_symmetry():
    """The rhombic 5 x 5 image set {k1 a1 + k2 a2} is symmetric under (x, y) -> (-x, -y),
    and so is the THGEM mesh (96 sectors): sigma of an element equals sigma of its rotated
    partner, Phi(-x, -y, z) = Phi(x, y, z) and (E_x, E_y) change sign.  (The x and y
    mirrors map the rhombus to another rhombus, so they are not symmetries here.)"""
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    sigma, _, _ = O.solve(g)
    c, _, _ = O.centroids(g)
    flip = c * np.array([-1.0, -1.0, 1.0])
    # partner of every element: the one whose centroid is the rotated centroid
    d = np.linalg.norm(flip[:, None, :] - c[None, :, :], axis=2)
    partner = d.argmin(1)
    assert d[np.arange(g.n), partner].max() < 1e-12
    # rounding of the FP64 solve (condition number ~1e4) allows ~1e-11; a wrong image index
    # or sign breaks the symmetry at the 1e-3 level
    assert np.abs(sigma[partner] - sigma).max() <= 1e-9 * np.abs(sigma).max()
    pts = I.cell_points(g, 20, I.rng(0, 63))
    p1, E1 = O.eval_points(g, sigma, pts)
    p2, E2 = O.eval_points(g, sigma, pts * np.array([-1.0, -1.0, 1.0]))
    assert np.abs(p1 - p2).max() <= 1e-9 * np.abs(p1).max()
    assert np.abs(E1 * np.array([-1.0, -1.0, 1.0]) - E2).max() <= 1e-9 * np.abs(E1).max()


def test_two_carriers_coulomb():
    """Two softened point charges: phi = ke q / sqrt(r^2 + s^2), E = ke q d / (r^2 + s^2)^1.5."""
    q = np.array([2.0e-15, -3.0e-15])
    pos = np.array([[0.0, 0.0, 0.0], [3e-6, -4e-6, 12e-6]])
    s = 1e-6
    phi, E = O.space_charge(pos, q, soft=s)
    d = pos[0] - pos[1]
    r2 = d @ d + s * s
    ke = O.ke()
    assert abs(phi[0] - ke * q[1] / np.sqrt(r2)) <= 1e-15 * abs(phi[0])
    assert np.abs(E[0] - ke * q[1] * d / r2 ** 1.5).max() <= 1e-14 * np.abs(E[0]).max()
    assert abs(phi[1] - ke * q[0] / np.sqrt(r2)) <= 1e-15 * abs(phi[1])
    assert np.abs(E[1] + ke * q[0] * d / r2 ** 1.5).max() <= 1e-14 * np.abs(E[1]).max()


def test_pair_tiers_match_fp64_distance_classes():
    """The FP32 tier decision of the oracle (two-float differences, FP32 squared distance)
    agrees with the classification of the FP64 distance d / rho_j wherever d is not
    within 1e-5 (relative) of a threshold; near thresholds either neighbouring tier is
    accepted.  Covers all five codes (points in the hole, near the Cu and FR4 surfaces)."""
    g = I.thgem(I.PlateSpec(n_phi=12, n_r=2, n_zc=1, n_zf=3), n_plane=2)
    gen = np.random.default_rng(71)
    pts = I.cell_points(g, 60, gen)
    # points close to element centroids give the near tiers
    v = g.elements["v"]
    kinds = g.elements["kind"]
    c = np.where((kinds == I.KIND_TRI)[:, None], v[:, :3].mean(1), v[:, :4].mean(1))
    pick = gen.choice(g.n, 20, replace=False)
    pts = np.vstack([pts, c[pick] + gen.normal(size=(20, 3)) * 2e-5])
    ratios = (64.0, 24.0, 8.0, 3.0)
    codes = O.pair_tiers(g, pts, ratios)
    nv = np.where(kinds == I.KIND_TRI, 3, 4)
    d = np.linalg.norm(v - c[:, None, :], axis=2)
    d[nv == 3, 3] = 0.0
    rho = d.max(1)
    t = O.image_table(g.lattice, g.img_lo, g.img_hi)
    C = c[:, None, :] + t[None]                                   # (n, img, 3)
    dist = np.linalg.norm(pts[:, None, None, :] - C[None], axis=3) / rho[None, :, None]
    expect = np.full(dist.shape, 4, np.uint8)
    for code, r in reversed(list(enumerate(ratios))):
        expect[dist >= r] = code
    near_thr = np.zeros(dist.shape, bool)
    for r in ratios:
        near_thr |= np.abs(dist / r - 1.0) <= 1e-5
    ok = (codes == expect) | (near_thr & (np.abs(codes.astype(int) - expect.astype(int)) == 1))
    assert ok.all()
    assert set(np.unique(codes)) == {0, 1, 2, 3, 4}


def test_fastvol_oracle_interpolation():
    """FastVolume oracle (Sec. 3.3): node values are the evaluation at the nodes exactly;
    an edge midpoint is the mean of its two nodes; points outside the box take the value
    at the clamped point; and the interpolation error at fixed off-node points falls like
    h^2 (trilinear, second order) as the grid is refined."""
    g = I.cube(n_per_edge=4)
    sigma, _, _ = O.solve(g)
    ax = np.linspace(0.01, 0.02, 3)
    ay = np.linspace(-0.004, 0.004, 3)
    az = np.linspace(-0.003, 0.005, 3)
    X, Y, Z = np.meshgrid(ax, ay, az, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    phi, E = O.fastvol(g, sigma, ax, ay, az, nodes)
    rphi, rE = O.eval_points(g, sigma, nodes)
    assert np.array_equal(phi, rphi) and np.array_equal(E, rE)
    mid = np.array([[0.5 * (ax[0] + ax[1]), ay[1], az[2]]])
    m_phi, m_E = O.fastvol(g, sigma, ax, ay, az, mid)
    ends = np.array([[ax[0], ay[1], az[2]], [ax[1], ay[1], az[2]]])
    e_phi, e_E = O.eval_points(g, sigma, ends)
    assert abs(m_phi[0] - 0.5 * e_phi.sum()) <= 1e-14 * abs(e_phi).max()
    assert np.abs(m_E[0] - 0.5 * e_E.sum(0)).max() <= 1e-14 * np.abs(e_E).max()
    out = np.array([[0.03, 0.0, 0.0], [0.015, -0.01, 0.009]])
    clamp = np.array([[0.02, 0.0, 0.0], [0.015, -0.004, 0.005]])
    o_phi, o_E = O.fastvol(g, sigma, ax, ay, az, out)
    c_phi, c_E = O.fastvol(g, sigma, ax, ay, az, clamp)
    assert np.array_equal(o_phi, c_phi) and np.array_equal(o_E, c_E)
    # second-order convergence outside the cube: the RMS error over random points of the box
    # falls like h^2 (fitted log-log slope; first order would give 1)
    probe = np.random.default_rng(72).uniform([0.012, -0.003, -0.003], [0.018, 0.003, 0.003], size=(200, 3))
    ref, _ = O.eval_points(g, sigma, probe)
    hs, errs = [], []
    for m in (9, 17, 33, 65):
        bx = np.linspace(0.012, 0.018, m)
        by = np.linspace(-0.003, 0.003, m)
        bz = np.linspace(-0.003, 0.003, m)
        p, _ = O.fastvol(g, sigma, bx, by, bz, probe)
        hs.append(0.006 / (m - 1))
        errs.append(np.sqrt(np.mean((p - ref) ** 2)))
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 1.7 <= slope <= 2.3, (slope, errs)

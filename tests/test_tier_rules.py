"""The distance tiers of the mixed path (element radii rho to the image centroid: 64, 24, 8
and 3 by default, the library's ratio_0, ratio_a, ratio_b, ratio_near) keep every far
pair's quadrature truncation far below the 1e-6 end-to-end bound.  CPU only: the rules are
restated here from their published definitions and compared with the oracle's FP64 closed
forms (Sec. 2.1) at each tier's own boundary, over random directions, for square and thin
rectangles, a skewed quadrilateral, and acute, obtuse and sliver triangles.

Rules: Gauss-Legendre tensor products on rectangles (2x2, 3x3, 4x4, 6x6); on triangles
the 4-point degree-3 rule (centroid weight -27/48, three points at barycentric
(0.6, 0.2, 0.2) with 25/48), the 6-point degree-4 rule (two orbits of three points), and
collapsed (Duffy) Gauss-Legendre products (4x4, 6x6)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I

RATIOS = {"t0": 64.0, "a": 24.0, "b": 8.0, "c": 3.0}
BOUND = 5e-8  # per pair, at the tier boundary (the end-to-end target is 1e-6)
# A non-parallelogram quadrilateral's Jacobian varies over the bilinear map, which costs the
# 2x2 rule one degree: its truncation falls as (rho/d)^3 instead of (rho/d)^4
BOUND_QUAD_T0 = 3e-7


def gl01(m):
    x, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * (x + 1.0), 0.5 * w


def rect_rule(v0, e1, e3, m):
    x, w = gl01(m)
    area = np.linalg.norm(np.cross(e1, e3))
    pts = np.array([v0 + a * e1 + b * e3 for a in x for b in x])
    wts = np.array([wa * wb * area for wa in w for wb in w])
    return pts, wts


def quad_rule(v, m):
    """Tensor Gauss-Legendre on the bilinear map x(s, t) = v0 + s e1 + t e3 + s t tw of a
    planar convex quadrilateral (tw = v2 - v1 - e3), weights w_s w_t |x_s x x_t|."""
    x, w = gl01(m)
    e1, e3 = v[1] - v[0], v[3] - v[0]
    tw = v[2] - v[1] - e3
    pts, wts = [], []
    for a, wa in zip(x, w):
        for b, wb in zip(x, w):
            pts.append(v[0] + a * e1 + b * e3 + a * b * tw)
            wts.append(wa * wb * np.linalg.norm(np.cross(e1 + b * tw, e3 + a * tw)))
    return np.array(pts), np.array(wts)


def tri_rule(v, kind):
    area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    if kind == "t0":
        bc = [(1 / 3, 1 / 3, 1 / 3), (0.6, 0.2, 0.2), (0.2, 0.6, 0.2), (0.2, 0.2, 0.6)]
        w = [-27 / 48, 25 / 48, 25 / 48, 25 / 48]
    elif kind == "a":
        bc, w = [], []
        for a, wt in ((0.445948490915965, 0.223381589678011), (0.091576213509771, 0.109951743655322)):
            for r in range(3):
                b = [a, a, a]
                b[r] = 1 - 2 * a
                bc.append(tuple(b))
                w.append(wt)
    else:
        m = 4 if kind == "b" else 6
        x, wx = gl01(m)
        bc, w = [], []
        for s, ws in zip(x, wx):
            for t, wt in zip(x, wx):
                # x = v0 + s (v1 - v0) + t (1 - s) (v2 - v0), collapsed at v1 (s = 1):
                # barycentric (1 - s - t(1-s), s, t(1-s)), Jacobian 2 A (1 - s)
                tt = t * (1 - s)
                bc.append((1 - s - tt, s, tt))
                w.append(2 * ws * wt * (1 - s))
    pts = np.array([b[0] * v[0] + b[1] * v[1] + b[2] * v[2] for b in bc])
    return pts, np.array(w) * area


def quad(pts, wts, P):
    d = P[:, None, :] - pts[None]
    r = np.linalg.norm(d, axis=2)
    return (wts / r).sum(1), ((wts / r ** 3)[..., None] * d).sum(1)


def _centre_radius(kind, v):
    """Expansion centre of the tiers (the vertex mean the library's element tables use for
    rectangles and triangles, the area centroid for quadrilaterals) and the circumradius
    about it."""
    nv = 3 if kind == "tri" else 4
    if kind == "quad":
        t1 = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
        t2 = 0.5 * np.linalg.norm(np.cross(v[2] - v[0], v[3] - v[0]))
        c = (t1 * (v[0] + v[1] + v[2]) + t2 * (v[0] + v[2] + v[3])) / (3 * (t1 + t2))
    else:
        c = v[:nv].mean(0)
    return c, np.linalg.norm(v[:nv] - c, axis=1).max()


def element(kind, v):
    el = np.zeros(1, I.ELEMENT_DTYPE)
    el["kind"] = kind
    el["v"][0, :len(v)] = v
    return el


SHAPES = {
    "square": ("rect", np.array([[0, 0, 0], [1e-4, 0, 0], [1e-4, 0, 1e-4], [0, 0, 1e-4]], float)),
    "thin_rect": ("rect", np.array([[0, 0, 0], [1e-4, 0, 0], [1e-4, 0, 1e-5], [0, 0, 1e-5]], float)),
    "acute_tri": ("tri", np.array([[0, 0, 0], [1e-4, 0, 0], [0.4e-4, 0, 0.8e-4]], float)),
    "obtuse_tri": ("tri", np.array([[0, 0, 0], [1e-4, 0, 0], [1.6e-4, 0, 0.3e-4]], float)),
    "sliver_tri": ("tri", np.array([[0, 0, 0], [1e-4, 0, 0], [0.5e-4, 0, 0.05e-4]], float)),
    "skewed_quad": ("quad", np.array([[0, 0, 0], [1e-4, 0, 0.1e-4], [0.7e-4, 0, 0.9e-4], [-0.1e-4, 0, 0.5e-4]], float)),
}


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("tier", list(RATIOS))
def test_rule_truncation_at_the_tier_boundary(shape, tier):
    kind, v = SHAPES[shape]
    m = {"t0": 2, "a": 3, "b": 4, "c": 6}[tier]
    if kind == "rect":
        el = element(I.KIND_RECT, v)
        pts, wts = rect_rule(v[0], v[1] - v[0], v[3] - v[0], m)
    elif kind == "quad":
        el = element(I.KIND_QUAD, v)
        pts, wts = quad_rule(v, m)
    else:
        el = element(I.KIND_TRI, v[:3])
        pts, wts = tri_rule(v[:3], tier)
    c, rho = _centre_radius(kind, v)
    gen = I.rng(0, 1000 + 10 * list(SHAPES).index(shape) + list(RATIOS).index(tier))
    u = gen.normal(size=(200, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    P = c + RATIOS[tier] * rho * u
    phi, E = O.influence(el, P)
    qphi, qE = quad(pts, wts, P)
    ephi = np.abs(qphi - phi) / np.abs(phi)
    eE = np.linalg.norm(qE - E, axis=1) / np.linalg.norm(E, axis=1)
    bound = BOUND_QUAD_T0 if (kind == "quad" and tier == "t0") else BOUND
    assert ephi.max() <= bound and eE.max() <= bound, (ephi.max(), eE.max())


FILL_RATIOS = {"a": 96.0, "b": 32.0, "c": 6.0}
FILL_BOUND = 1e-11  # per pair: the fill's entries must stay near 1e-11 for the FP64 refinement


def _converged(kind, v):
    """The defining integrals of Sec. 2.1 by a 24 x 24 Gauss product (collapsed on
    triangles): converged to rounding at these distances, independent of the closed form."""
    if kind == "rect":
        return rect_rule(v[0], v[1] - v[0], v[3] - v[0], 24)
    if kind == "quad":
        return quad_rule(v, 24)
    x, wx = gl01(24)
    area = 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))
    pts, w = [], []
    for s, ws in zip(x, wx):
        for t, wt in zip(x, wx):
            tt = t * (1 - s)
            pts.append((1 - s - tt) * v[0] + s * v[1] + tt * v[2])
            w.append(2 * ws * wt * (1 - s) * area)
    return np.array(pts), np.array(w)


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("tier", list(FILL_RATIOS))
def test_fill_rule_truncation_at_the_tier_boundary(shape, tier):
    """The mixed fill's tiers (96, 32, 6 rho: 3x3 / 6-point, 4x4 / collapsed 4x4, 6x6 /
    collapsed 6x6) truncate by at most 1e-11 of the pair, against the converged integral."""
    kind, v = SHAPES[shape]
    m = {"a": 3, "b": 4, "c": 6}[tier]
    if kind == "rect":
        pts, wts = rect_rule(v[0], v[1] - v[0], v[3] - v[0], m)
    elif kind == "quad":
        pts, wts = quad_rule(v, m)
    else:
        pts, wts = tri_rule(v[:3], tier)
    c, rho = _centre_radius(kind, v)
    gen = I.rng(0, 2000 + 10 * list(SHAPES).index(shape) + list(FILL_RATIOS).index(tier))
    u = gen.normal(size=(200, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    P = c + FILL_RATIOS[tier] * rho * u
    rpts, rw = _converged(kind, v)
    phi, E = quad(rpts, rw, P)
    qphi, qE = quad(pts, wts, P)
    ephi = np.abs(qphi - phi) / np.abs(phi)
    eE = np.linalg.norm(qE - E, axis=1) / np.linalg.norm(E, axis=1)
    assert ephi.max() <= FILL_BOUND and eE.max() <= FILL_BOUND, (ephi.max(), eE.max())

"""The closed forms (Sec. 2.1) at the singular places of an element, GPU against the oracle:
points exactly at its vertices and on its edges, and points on an edge's line beyond its
ends (the ln branch taken for a negative argument).

Reading of the paper's silence on these points: the potential is finite there (the ln
terms of a vertex or an edge go to 0 as their factor does), and both sides return it to
1e-10; the field E' diverges logarithmically on an edge, and both sides return a
non-finite value there (inf, or NaN where two infinite terms meet), which is the status of
such a point; elsewhere on the edge's line it is finite and agrees.  Edges are axis-aligned with vertex coordinates that are exact in binary, so that
a point on an edge is on it in FP64 for both sides."""
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


def _element(kind, verts):
    rec = np.zeros(1, dtype=I.ELEMENT_DTYPE)
    rec["kind"] = kind
    v = np.zeros((4, 3))
    v[: len(verts)] = verts
    rec["v"] = v
    return rec


# lengths in m, exact in binary: 2^-10 ~ 0.98 mm, 2^-9 ~ 1.95 mm
A, B = 2.0 ** -10, 2.0 ** -9
ELEMENTS = {
    "rect": _element(I.KIND_RECT, [[0, 0, 0], [A, 0, 0], [A, 0, B], [0, 0, B]]),
    "tri": _element(I.KIND_TRI, [[0, 0, 0], [A, 0, 0], [0, 0, B]]),
    "quad": _element(I.KIND_QUAD, [[0, 0, 0], [A, 0, 0], [0.75 * A, 0, B], [0, 0, B]]),
}


def _points(name):
    """(points exactly on the element's edges or vertices, points on an edge's line outside
    the element, general points nearby)"""
    on = [[0, 0, 0], [A, 0, 0], [0, 0, B], [0.5 * A, 0, 0], [0.25 * A, 0, 0], [0, 0, 0.5 * B],
          [0, 0, 0.125 * B]]
    if name == "rect":
        on += [[A, 0, 0], [A, 0, B], [A, 0, 0.5 * B], [0.5 * A, 0, B], [0.75 * A, 0, B]]
    if name == "quad":
        on += [[0.75 * A, 0, B], [0.5 * A, 0, B], [0.25 * A, 0, B]]
    line = [[1.5 * A, 0, 0], [-0.5 * A, 0, 0], [0, 0, 1.5 * B], [0, 0, -0.25 * B], [2 * A, 0, 0]]
    near = [[0.5 * A, 1e-7, 0], [0.5 * A, 0, -1e-7], [0.3 * A, 0.5 * A, 0.2 * B], [-A, A, -B],
            [0.25 * A, 0, 0.25 * B]]
    return np.array(on, float), np.array(line, float), np.array(near, float)


@pytest.mark.parametrize("name", list(ELEMENTS))
def test_edges_vertices_and_edge_lines(N, name):
    el = ELEMENTS[name]
    on, line, near = _points(name)
    pts = np.concatenate([on, line, near])
    ctx = N.Context()
    phi, E = N.nebem_element_influence(ctx.h, el, pts)
    phi, E = phi[0], E[0]
    rphi, rE = O.influence(el, pts)
    # the potential: finite everywhere, 1e-10 of the value
    assert np.isfinite(phi).all() and np.isfinite(rphi).all()
    assert (np.abs(phi - rphi) <= 1e-10 * np.abs(rphi)).all(), np.abs(phi - rphi) / np.abs(rphi)
    # the field: non-finite at exactly the points where the oracle's is (on an edge; which
    # components come out inf or NaN depends on each side's formula), finite and equal
    # elsewhere
    fin_g, fin_o = np.isfinite(E).all(axis=1), np.isfinite(rE).all(axis=1)
    assert np.array_equal(fin_g, fin_o), (fin_g, fin_o)
    n_on = on.shape[0]
    assert not np.isfinite(rE[:n_on]).all(axis=1).any()  # every point on an edge or vertex
    fin = np.isfinite(rE[n_on:]).all(axis=1)
    assert fin.all()  # off the edges, including the edges' lines beyond the element
    scale = np.abs(rE[n_on:]).max()
    assert np.abs(E[n_on:] - rE[n_on:]).max() <= 1e-10 * scale

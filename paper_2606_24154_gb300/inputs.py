"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds only geometry generation and random sampling: flat boundary
elements (raw vertices, boundary-condition type, conductor index, permittivities),
evaluation points, space-charge carriers and serving traces.  It contains none of
the method's arithmetic (no influence integrals, no image translations, no frames):
each side builds those from the raw records itself.

Geometries follow the paper's workloads (Sec. 5, Case 2: a THGEM foil of FR4 with
Cu cladding, a hexagonal hole pattern, drift and induction planes) at the sizes of
the benchmark configurations:

* ``cube``: unit cube conductor (edge 1 cm) at 1 V, 6 faces x 8 x 8 rectangles.
* ``thgem``: hexagonal THGEM unit cell (pitch 1 mm, hole 0.5 mm, FR4 0.5 mm with
  eps_r = 4.4, 35 um Cu at -500/+500 V, drift/induction planes 3 mm away), about
  10,000 rectangles and triangles, 5 x 5 periodic images.
* ``double_thgem``: two such plates with 0.1 mm rims, offset by half a pitch,
  2 mm transfer gap, about 40,000 elements.

Element record (128 bytes, little-endian), identical to the C-ABI ``nebem_element``:
``int32 kind`` (0 rectangle v0..v3 in order, right angles; 1 triangle v0..v2),
``int32 bc`` (0 conductor, 1 dielectric interface), ``int32 conductor``,
``int32 reserved``, ``float64 eps_a`` (relative permittivity on the -n side),
``float64 eps_b`` (+n side), ``float64 v[4][3]`` (metres).  The normal n follows
the right-hand rule on v0, v1, v2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ELEMENT_DTYPE = np.dtype(
    [
        ("kind", "<i4"),
        ("bc", "<i4"),
        ("conductor", "<i4"),
        ("reserved", "<i4"),
        ("eps_a", "<f8"),
        ("eps_b", "<f8"),
        ("v", "<f8", (4, 3)),
    ]
)
assert ELEMENT_DTYPE.itemsize == 128

KIND_RECT, KIND_TRI, KIND_QUAD = 0, 1, 2
BC_CONDUCTOR, BC_DIELECTRIC = 0, 1

E_CHARGE = 1.602176634e-19  # C (exact, SI 2019)
BASE_SEED = 20261203


@dataclass
class Geometry:
    """A discretised problem: raw element records plus the data the C-ABI takes."""

    name: str
    elements: np.ndarray  # ELEMENT_DTYPE[n]
    voltages: np.ndarray  # float64[n_conductors]
    lattice: np.ndarray | None = None  # float64[2, 3] primitive translations, or None
    img_lo: int = 0
    img_hi: int = 0
    # Sampling box for evaluation points: hexagonal prism (pitch, z range) or a box.
    pitch: float | None = None
    z_range: tuple[float, float] = (0.0, 0.0)
    box: tuple[tuple[float, float], ...] | None = None
    xy_offset: tuple[float, float] = (0.0, 0.0)
    solids: list = field(default_factory=list)  # (kind, params) for the carrier resampler
    # Primitives (flat polygons the elements tile, for Adaptive Modelling): records of
    # ELEMENT_DTYPE and the primitive of every element (-1: none).
    primitives: np.ndarray | None = None
    prim_of: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.elements.shape[0])

    @property
    def n_images(self) -> int:
        if self.lattice is None:
            return 1
        m = self.img_hi - self.img_lo + 1
        return m * m


# --------------------------------------------------------------------------- elements
def _records(n: int) -> np.ndarray:
    return np.zeros(n, dtype=ELEMENT_DTYPE)


def _put(rec, kind, verts, bc, cond, eps_a=1.0, eps_b=1.0):
    rec["kind"] = kind
    rec["bc"] = bc
    rec["conductor"] = cond
    rec["eps_a"] = eps_a
    rec["eps_b"] = eps_b
    v = np.zeros((4, 3))
    v[: len(verts)] = verts
    rec["v"] = v


class _Builder:
    def __init__(self):
        self.rows = []
        self.prims = []   # (kind, verts) of every primitive
        self.prim_of = []
        self.cur = -1

    def _add(self, row):
        self.rows.append(row)
        self.prim_of.append(self.cur)

    def rect(self, v0, v1, v2, v3, bc=BC_CONDUCTOR, cond=0, eps_a=1.0, eps_b=1.0):
        self._add((KIND_RECT, np.array([v0, v1, v2, v3], float), bc, cond, eps_a, eps_b))

    def tri(self, v0, v1, v2, bc=BC_CONDUCTOR, cond=0, eps_a=1.0, eps_b=1.0):
        self._add((KIND_TRI, np.array([v0, v1, v2], float), bc, cond, eps_a, eps_b))

    def quad(self, v0, v1, v2, v3, bc=BC_CONDUCTOR, cond=0, eps_a=1.0, eps_b=1.0):
        self._add((KIND_QUAD, np.array([v0, v1, v2, v3], float), bc, cond, eps_a, eps_b))

    def primitive(self, kind, verts):
        """Elements added from now until end_primitive() tile this flat polygon."""
        self.prims.append((kind, np.array(verts, float)))
        self.cur = len(self.prims) - 1

    def end_primitive(self):
        self.cur = -1

    def build(self) -> np.ndarray:
        out = _records(len(self.rows))
        for i, (kind, verts, bc, cond, ea, eb) in enumerate(self.rows):
            _put(out[i], kind, verts, bc, cond, ea, eb)
        return out

    def build_primitives(self):
        out = _records(len(self.prims))
        for i, (kind, verts) in enumerate(self.prims):
            _put(out[i], kind, verts, BC_CONDUCTOR, 0)
        return out, np.array(self.prim_of, dtype=np.int32)


# --------------------------------------------------------------------------- cube
def cube(edge: float = 0.01, n_per_edge: int = 8, voltage: float = 1.0) -> Geometry:
    """Cube conductor centred at the origin, faces at +-edge/2, n x n squares per face.

    Each square's normal points out of the cube.
    """
    b = _Builder()
    h = edge / 2.0
    s = np.linspace(-h, h, n_per_edge + 1)
    # For each axis a and side sgn, the face lies at x_a = sgn*h; (u, w) are the other
    # two axes ordered so that u x w points along +sgn * e_a.
    for a in range(3):
        u_ax, w_ax = (a + 1) % 3, (a + 2) % 3
        for sgn in (+1.0, -1.0):
            def P(ui, wj):
                p = [0.0, 0.0, 0.0]
                p[a] = sgn * h
                p[u_ax] = s[ui]
                p[w_ax] = s[wj]
                return p

            m = n_per_edge
            b.primitive(KIND_RECT, [P(0, 0), P(m, 0), P(m, m), P(0, m)] if sgn > 0
                        else [P(0, 0), P(0, m), P(m, m), P(m, 0)])
            for i in range(n_per_edge):
                for j in range(n_per_edge):
                    if sgn > 0:
                        b.rect(P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1))
                    else:
                        b.rect(P(i, j), P(i, j + 1), P(i + 1, j + 1), P(i + 1, j))
            b.end_primitive()
    g = Geometry(
        name=f"cube_a{edge:g}_n{n_per_edge}",
        elements=b.build(),
        voltages=np.array([voltage]),
        box=((-2 * edge, 2 * edge),) * 3,
    )
    g.solids = [("box", (-h, h, -h, h, -h, h))]
    g.primitives, g.prim_of = b.build_primitives()
    return g


def cube_grid_points(edge: float = 0.01, shape=(20, 20, 25)) -> np.ndarray:
    """The cube's evaluation grid: linspace(-2 edge, 2 edge) per axis, x fastest last."""
    ax = [np.linspace(-2 * edge, 2 * edge, m) for m in shape]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).copy()


# --------------------------------------------------------------------------- hex cell
def hex_lattice(pitch: float) -> np.ndarray:
    """Primitive translations of the hexagonal hole lattice (nearest neighbours at 0, 60 deg)."""
    return np.array([[pitch, 0.0, 0.0], [0.5 * pitch, 0.5 * math.sqrt(3.0) * pitch, 0.0]])


def _hex_radius(phi: np.ndarray, pitch: float) -> np.ndarray:
    """Distance from the cell centre to the Wigner-Seitz hexagon (flats at 0, 60, ... deg)."""
    flat = np.round(phi / (math.pi / 3.0)) * (math.pi / 3.0)
    return 0.5 * pitch / np.cos(phi - flat)


def _annulus_to_hex(b: _Builder, z, r_in, pitch, n_phi, n_r, grade, up, bc, cond,
                    eps_a=1.0, eps_b=1.0, center=(0.0, 0.0)):
    """Triangulate (hexagon minus the n_phi-gon of radius r_in) in the plane z.

    Rings are graded geometrically (ratio ``grade``) from the hole outwards; each quad
    cell becomes two triangles.  ``up`` selects the normal direction (+z or -z).
    """
    phis = 2.0 * math.pi * np.arange(n_phi + 1) / n_phi
    R = _hex_radius(phis, pitch)
    if grade == 1.0:
        s = np.linspace(0.0, 1.0, n_r + 1)
    else:
        s = (grade ** np.arange(n_r + 1) - 1.0) / (grade ** n_r - 1.0)
    cx, cy = center
    for j in range(n_phi):
        def P(ii, jj):
            r = r_in + (R[jj] - r_in) * s[ii]
            return [cx + r * math.cos(phis[jj]), cy + r * math.sin(phis[jj]), z]

        # the sector between two rays is a flat convex quadrilateral (hexagon corners lie
        # on rays), tiled by its 2 n_r triangles
        q = [P(0, j), P(n_r, j), P(n_r, j + 1), P(0, j + 1)]
        b.primitive(KIND_QUAD, q if up else [q[0], q[3], q[2], q[1]])
        for i in range(n_r):
            a, bb, c, d = P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)
            if up:  # counter-clockwise seen from +z
                b.tri(a, bb, c, bc, cond, eps_a, eps_b)
                b.tri(a, c, d, bc, cond, eps_a, eps_b)
            else:
                b.tri(a, c, bb, bc, cond, eps_a, eps_b)
                b.tri(a, d, c, bc, cond, eps_a, eps_b)
        b.end_primitive()


def _annulus(b: _Builder, z, r_in, r_out, n_phi, n_rad, up, bc, cond, eps_a=1.0, eps_b=1.0,
             center=(0.0, 0.0)):
    """Triangulate the flat ring between two concentric n_phi-gons."""
    phis = 2.0 * math.pi * np.arange(n_phi + 1) / n_phi
    rs = np.linspace(r_in, r_out, n_rad + 1)
    cx, cy = center
    for j in range(n_phi):
        def P(ii, jj):
            return [cx + rs[ii] * math.cos(phis[jj]), cy + rs[ii] * math.sin(phis[jj]), z]

        q = [P(0, j), P(n_rad, j), P(n_rad, j + 1), P(0, j + 1)]
        b.primitive(KIND_QUAD, q if up else [q[0], q[3], q[2], q[1]])
        for i in range(n_rad):
            a, bb, c, d = P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)
            if up:
                b.tri(a, bb, c, bc, cond, eps_a, eps_b)
                b.tri(a, c, d, bc, cond, eps_a, eps_b)
            else:
                b.tri(a, c, bb, bc, cond, eps_a, eps_b)
                b.tri(a, d, c, bc, cond, eps_a, eps_b)
        b.end_primitive()


def _hole_wall(b: _Builder, r, z0, z1, n_phi, n_z, bc, cond, eps_a=1.0, eps_b=1.0,
               center=(0.0, 0.0)):
    """Rectangular facets of the n_phi-gon prism r, z0..z1; normals point to the axis."""
    phis = 2.0 * math.pi * np.arange(n_phi + 1) / n_phi
    zs = np.linspace(z0, z1, n_z + 1)
    cx, cy = center
    for j in range(n_phi):
        p0 = [cx + r * math.cos(phis[j]), cy + r * math.sin(phis[j])]
        p1 = [cx + r * math.cos(phis[j + 1]), cy + r * math.sin(phis[j + 1])]
        b.primitive(KIND_RECT, [[*p0, zs[0]], [*p1, zs[0]], [*p1, zs[-1]], [*p0, zs[-1]]])
        for k in range(n_z):
            # v0 -> v1 along the facet chord, v1 -> v2 along +z: (v1-v0) x (v2-v0) points inwards.
            b.rect([*p0, zs[k]], [*p1, zs[k]], [*p1, zs[k + 1]], [*p0, zs[k + 1]], bc, cond,
                   eps_a, eps_b)
        b.end_primitive()


def _hex_plane(b: _Builder, z, pitch, n_sub, up, cond, center=(0.0, 0.0)):
    """Hexagonal cell of an electrode plane: 6 sector triangles, each split n_sub x n_sub."""
    cx, cy = center
    rv = pitch / math.sqrt(3.0)
    verts = [(cx + rv * math.cos(math.pi / 6 + k * math.pi / 3),
              cy + rv * math.sin(math.pi / 6 + k * math.pi / 3)) for k in range(7)]
    for k in range(6):
        A = np.array([cx, cy]); B = np.array(verts[k]); C = np.array(verts[k + 1])
        pa, pb, pc = [A[0], A[1], z], [B[0], B[1], z], [C[0], C[1], z]
        b.primitive(KIND_TRI, [pa, pb, pc] if up else [pa, pc, pb])
        # barycentric sub-triangulation
        def node(i, j):
            p = A + (B - A) * (i / n_sub) + (C - A) * (j / n_sub)
            return [p[0], p[1], z]
        for i in range(n_sub):
            for j in range(n_sub - i):
                t = (node(i, j), node(i + 1, j), node(i, j + 1))
                if up:
                    b.tri(*t, BC_CONDUCTOR, cond)
                else:
                    b.tri(t[0], t[2], t[1], BC_CONDUCTOR, cond)
                if j < n_sub - i - 1:
                    t2 = (node(i + 1, j), node(i + 1, j + 1), node(i, j + 1))
                    if up:
                        b.tri(*t2, BC_CONDUCTOR, cond)
                    else:
                        b.tri(t2[0], t2[2], t2[1], BC_CONDUCTOR, cond)
        b.end_primitive()


@dataclass
class PlateSpec:
    pitch: float = 1.0e-3
    hole_d: float = 0.5e-3
    fr4: float = 0.5e-3
    cu: float = 35e-6
    rim: float = 0.0
    eps_fr4: float = 4.4
    n_phi: int = 96
    n_r: int = 9
    n_rim: int = 2
    n_zc: int = 2
    n_zf: int = 18
    grade: float = 1.15


def _plate(b: _Builder, spec: PlateSpec, zc: float, cond_top: int, cond_bot: int,
           center=(0.0, 0.0)) -> list:
    """One THGEM plate centred at height zc; returns its solids for the carrier resampler."""
    r_f = 0.5 * spec.hole_d          # FR4 hole radius
    r_c = r_f + spec.rim             # Cu hole radius
    zf0, zf1 = zc - 0.5 * spec.fr4, zc + 0.5 * spec.fr4
    zt = zf1 + spec.cu               # top Cu outer face
    zb = zf0 - spec.cu               # bottom Cu outer face
    eps = spec.eps_fr4
    # Cu faces (conductors): outer faces and the Cu/FR4 contact faces.
    _annulus_to_hex(b, zt, r_c, spec.pitch, spec.n_phi, spec.n_r, spec.grade, True,
                    BC_CONDUCTOR, cond_top, center=center)
    _annulus_to_hex(b, zf1, r_c, spec.pitch, spec.n_phi, spec.n_r, spec.grade, False,
                    BC_CONDUCTOR, cond_top, center=center)
    _annulus_to_hex(b, zf0, r_c, spec.pitch, spec.n_phi, spec.n_r, spec.grade, True,
                    BC_CONDUCTOR, cond_bot, center=center)
    _annulus_to_hex(b, zb, r_c, spec.pitch, spec.n_phi, spec.n_r, spec.grade, False,
                    BC_CONDUCTOR, cond_bot, center=center)
    # Cu hole-wall bands.
    _hole_wall(b, r_c, zf1, zt, spec.n_phi, spec.n_zc, BC_CONDUCTOR, cond_top, center=center)
    _hole_wall(b, r_c, zb, zf0, spec.n_phi, spec.n_zc, BC_CONDUCTOR, cond_bot, center=center)
    # FR4 hole wall: dielectric interface, FR4 on the -n side (normals point into the hole).
    _hole_wall(b, r_f, zf0, zf1, spec.n_phi, spec.n_zf, BC_DIELECTRIC, -1, eps, 1.0,
               center=center)
    if spec.rim > 0.0:
        # Exposed FR4 rims: top rim normal +z (FR4 below = -n side), bottom rim normal -z.
        _annulus(b, zf1, r_f, r_c, spec.n_phi, spec.n_rim, True, BC_DIELECTRIC, -1, eps, 1.0,
                 center=center)
        _annulus(b, zf0, r_f, r_c, spec.n_phi, spec.n_rim, False, BC_DIELECTRIC, -1, eps, 1.0,
                 center=center)
    return [("plate", (center[0], center[1], zb, zf0, zf1, zt, r_f, r_c))]


def thgem(spec: PlateSpec | None = None, gap: float = 3.0e-3, n_plane: int = 9,
          v_top=-500.0, v_bot=500.0, v_drift=-1100.0, v_ind=1700.0) -> Geometry:
    """Single THGEM unit cell (hexagonal, pitch 1 mm) with drift and induction planes.

    Conductors: 0 top Cu, 1 bottom Cu, 2 drift plane, 3 induction plane.
    """
    spec = spec or PlateSpec()
    b = _Builder()
    solids = _plate(b, spec, 0.0, 0, 1)
    zt = 0.5 * spec.fr4 + spec.cu
    _hex_plane(b, zt + gap, spec.pitch, n_plane, False, 2)
    _hex_plane(b, -(zt + gap), spec.pitch, n_plane, True, 3)
    g = Geometry(
        name="thgem_cell",
        elements=b.build(),
        voltages=np.array([v_top, v_bot, v_drift, v_ind]),
        lattice=hex_lattice(spec.pitch),
        img_lo=-2,
        img_hi=2,
        pitch=spec.pitch,
        z_range=(-(zt + gap), zt + gap),
    )
    g.solids = solids
    g.primitives, g.prim_of = b.build_primitives()
    return g


def double_thgem(spec: PlateSpec | None = None, transfer: float = 2.0e-3, gap: float = 3.0e-3,
                 n_plane: int = 14) -> Geometry:
    """Two THGEM plates (rims 0.1 mm) offset by half a pitch in x, 2 mm transfer gap.

    Conductors: 0/1 upper plate top/bottom Cu, 2/3 lower plate top/bottom Cu,
    4 drift plane, 5 induction plane.  Both plates carry -500/+500 V.
    """
    spec = spec or PlateSpec(rim=0.1e-3, n_phi=144, n_r=12, n_rim=3, n_zc=2, n_zf=20)
    b = _Builder()
    half = 0.5 * spec.fr4 + spec.cu
    zc = 0.5 * transfer + half
    solids = _plate(b, spec, +zc, 0, 1)
    solids += _plate(b, spec, -zc, 2, 3, center=(0.5 * spec.pitch, 0.0))
    ztop = zc + half + gap
    _hex_plane(b, ztop, spec.pitch, n_plane, False, 4)
    _hex_plane(b, -ztop, spec.pitch, n_plane, True, 5)
    g = Geometry(
        name="double_thgem",
        elements=b.build(),
        voltages=np.array([-500.0, 500.0, -500.0, 500.0, -1100.0, 1700.0]),
        lattice=hex_lattice(spec.pitch),
        img_lo=-2,
        img_hi=2,
        pitch=spec.pitch,
        z_range=(-ztop, ztop),
    )
    g.solids = solids
    g.primitives, g.prim_of = b.build_primitives()
    return g


# --------------------------------------------------------------------------- points
def rng(config_index: int, stream: int = 0) -> np.random.Generator:
    """PCG64 generator seeded with 20261203 + config index (+ a stream offset)."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + config_index, stream]))


def _in_hex(x, y, pitch):
    s3 = math.sqrt(3.0) / 2.0
    h = 0.5 * pitch
    return (np.abs(x) <= h) & (np.abs(0.5 * x + s3 * y) <= h) & (np.abs(-0.5 * x + s3 * y) <= h)


def cell_points(g: Geometry, n: int, gen: np.random.Generator) -> np.ndarray:
    """n points uniform in the geometry's cell (hexagonal prism between the planes, or box)."""
    if g.pitch is None:
        lo = np.array([b[0] for b in g.box]); hi = np.array([b[1] for b in g.box])
        return lo + (hi - lo) * gen.random((n, 3))
    p = g.pitch
    out = np.empty((0, 3))
    z0, z1 = g.z_range
    while out.shape[0] < n:
        m = int(1.3 * (n - out.shape[0])) + 16
        x = (gen.random(m) - 0.5) * p
        y = (gen.random(m) - 0.5) * (2.0 * p / math.sqrt(3.0))
        z = z0 + (z1 - z0) * gen.random(m)
        keep = _in_hex(x, y, p)
        out = np.concatenate([out, np.stack([x[keep], y[keep], z[keep]], 1)])
    return np.ascontiguousarray(out[:n])


def in_solid(g: Geometry, pts: np.ndarray) -> np.ndarray:
    """True where a point lies inside FR4 or Cu of a plate, or inside the cube."""
    inside = np.zeros(pts.shape[0], bool)
    for kind, prm in g.solids:
        if kind == "box":
            x0, x1, y0, y1, z0, z1 = prm
            inside |= ((pts[:, 0] >= x0) & (pts[:, 0] <= x1) & (pts[:, 1] >= y0)
                       & (pts[:, 1] <= y1) & (pts[:, 2] >= z0) & (pts[:, 2] <= z1))
        else:
            cx, cy, zb, zf0, zf1, zt, r_f, r_c = prm
            r = np.hypot(pts[:, 0] - cx, pts[:, 1] - cy)
            z = pts[:, 2]
            fr4 = (z >= zf0) & (z <= zf1) & (r >= r_f)
            cu = (((z >= zf1) & (z <= zt)) | ((z >= zb) & (z <= zf0))) & (r >= r_c)
            inside |= fr4 | cu
    return inside


def carrier_cloud(g: Geometry, n: int, gen: np.random.Generator, sigma: float = 0.1e-3,
                  center=(0.0, 0.0, 0.0), ion_fraction: float = 0.5):
    """n point carriers from an isotropic Gaussian, resampled until all lie in gas.

    Returns (positions float64[n,3], charges float64[n]): the first round(n*ion_fraction)
    carry +e, the rest -e.
    """
    c = np.asarray(center, float)
    pos = c + sigma * gen.standard_normal((n, 3))
    for _ in range(100):
        bad = in_solid(g, pos)
        if not bad.any():
            break
        pos[bad] = c + sigma * gen.standard_normal((int(bad.sum()), 3))
    n_ion = int(round(n * ion_fraction))
    q = np.full(n, -E_CHARGE)
    q[:n_ion] = E_CHARGE
    return np.ascontiguousarray(pos), q


def serving_trace(n_requests: int, gen: np.random.Generator, rate_hz: float = 2000.0,
                  lo: int = 100, hi: int = 1_000_000, n_geometries: int = 3):
    """Poisson arrivals (mean rate_hz), log-uniform sizes in [lo, hi], uniform geometry ids."""
    gaps = gen.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(gen.uniform(math.log(lo), math.log(hi), n_requests)).astype(np.int64)
    geo = gen.integers(0, n_geometries, n_requests)
    return t, sizes, geo

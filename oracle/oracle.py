"""ctypes wrapper around the plain-C FP64 oracle (``nebem_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py``.  The CUDA path never imports it.

Every function takes the raw element records (``ELEMENT_DTYPE`` arrays) and builds its
own local frames, image translations and constants inside the C code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nebem_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_d = C.POINTER(C.c_double)
_i32 = C.POINTER(C.c_int32)
_vp = C.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_ke.restype = C.c_double
        L.or_eps0.restype = C.c_double
        L.or_num_threads.restype = C.c_int
        L.or_influence_points.argtypes = [_vp, _d, C.c_int64, C.c_int, _d, _d]
        L.or_image_table.argtypes = [_d, C.c_int, C.c_int, _d]
        L.or_image_table.restype = C.c_int64
        L.or_fill.argtypes = [_vp, C.c_int64, _d, C.c_int, C.c_int, _d]
        L.or_fill_entries.argtypes = [_vp, C.c_int64, _d, C.c_int, C.c_int, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64), C.c_int64, _d]
        L.or_pair_tiers.argtypes = [_vp, C.c_int64, _d, C.c_int, C.c_int, _d, C.c_int64, _d,
                                    C.POINTER(C.c_uint8)]
        L.or_lu_factor.argtypes = [C.c_int64, _d, _i32]
        L.or_lu_solve.argtypes = [C.c_int64, _d, _i32, _d]
        L.or_rhs.argtypes = [_vp, C.c_int64, _d, C.c_int32, _d]
        L.or_eval.argtypes = [_vp, C.c_int64, _d, _d, C.c_int, C.c_int, _d, C.c_int64, _d, _d]
        L.or_centroids.argtypes = [_vp, C.c_int64, _d, _d, _d]
        L.or_space_charge.argtypes = [_d, _d, C.c_int64, _d, C.c_int64, C.c_int, C.c_double, _d, _d]
        L.or_rhs_space_charge.argtypes = [_vp, C.c_int64, _d, C.c_int32, _d, _d, C.c_int64, C.c_double, _d]
        L.or_dynamic_step.argtypes = [_vp, C.c_int64, _d, C.c_int32, _d, C.c_int, C.c_int, _d, _i32, _d, _d,
                                      C.c_int64, C.c_double, C.c_double, C.c_double, _d, _d]
        _i64 = C.POINTER(C.c_int64)
        L.or_voxel_grid.argtypes = [_d, C.c_int64, _d, _d, _i64]
        L.or_voxel_lines.argtypes = [_d, _d, C.c_int64, _d, _d, _d, _d, _i64]
        L.or_voxel_lines.restype = C.c_int64
        L.or_line_charge.argtypes = [_d, _d, _d, C.c_int64, _d, C.c_int64, C.c_double, C.c_int, _d, _d]
        L.or_rhs_lines.argtypes = [_vp, C.c_int64, _d, C.c_int32, _d, _d, _d, C.c_int64, C.c_double, _d]
        L.or_dynamic_step_lines.argtypes = [_vp, C.c_int64, _d, C.c_int32, _d, C.c_int, C.c_int, _d, _i32, _d,
                                            _d, C.c_int64, _d, C.c_double, C.c_double, C.c_double, _d, _d]
        L.or_eval_am.argtypes = [_vp, C.c_int64, _d, _d, C.c_int, C.c_int, _vp, C.c_int64, C.POINTER(C.c_int32),
                                 C.c_int, _d, C.c_int64, _d, _d]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_d)


def _pi(a):
    return a.ctypes.data_as(_i32)


def _rec(el):
    el = np.ascontiguousarray(el)
    assert el.dtype.itemsize == 128
    return el, el.ctypes.data_as(_vp)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def ke() -> float:
    return lib().or_ke()


def eps0() -> float:
    return lib().or_eps0()


def num_threads() -> int:
    return lib().or_num_threads()


def influence(element, pts, poly: bool = False):
    """Phi' (m) and E' (dimensionless, global components) of one element at points."""
    el, pe = _rec(np.atleast_1d(element)[:1])
    pts = np.ascontiguousarray(np.atleast_2d(pts), dtype=np.float64)
    n = pts.shape[0]
    phi = np.empty(n)
    E = np.empty((n, 3))
    _check(lib().or_influence_points(pe, _p(pts), n, int(poly), _p(phi), _p(E)), "influence")
    return phi, E


def image_table(lattice, lo, hi):
    if lattice is None:
        return np.zeros((1, 3))
    m = hi - lo + 1
    t = np.empty((m * m, 3))
    lat = np.ascontiguousarray(lattice, dtype=np.float64)
    lib().or_image_table(_p(lat), lo, hi, _p(t))
    return t


def _lat(g):
    return None if g.lattice is None else np.ascontiguousarray(g.lattice, dtype=np.float64)


def fill(g):
    """Influence matrix K (n x n, returned as a C-ordered array with K[i, j])."""
    el, pe = _rec(g.elements)
    n = el.shape[0]
    K = np.empty(n * n)
    lat = _lat(g)
    _check(lib().or_fill(pe, n, _p(lat), g.img_lo, g.img_hi, _p(K)), "fill")
    return K.reshape(n, n).T.copy()  # column-major storage -> K[i, j]


def fill_entries(g, rows, cols):
    """K[rows[e], cols[e]] computed entry by entry (full-size checks)."""
    el, pe = _rec(g.elements)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(rows.shape[0])
    lat = _lat(g)
    i64 = C.POINTER(C.c_int64)
    _check(lib().or_fill_entries(pe, el.shape[0], _p(lat), g.img_lo, g.img_hi, rows.ctypes.data_as(i64),
                                 cols.ctypes.data_as(i64), rows.shape[0], _p(out)), "fill_entries")
    return out


def pair_tiers(g, pts, ratios=(64.0, 24.0, 8.0, 3.0)):
    """Distance-tier code (0..4) of every (point, element, image) pair, FP32 decision."""
    el, pe = _rec(g.elements)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    r = np.ascontiguousarray(ratios, dtype=np.float64)
    nimg = 1 if g.lattice is None else (g.img_hi - g.img_lo + 1) ** 2
    codes = np.empty(pts.shape[0] * el.shape[0] * nimg, dtype=np.uint8)
    _check(lib().or_pair_tiers(pe, el.shape[0], _p(_lat(g)), g.img_lo, g.img_hi, _p(pts), pts.shape[0], _p(r),
                               codes.ctypes.data_as(C.POINTER(C.c_uint8))), "pair_tiers")
    return codes.reshape(pts.shape[0], el.shape[0], nimg)


def lu_factor(K):
    """Partial-pivoting LU of K[i, j]; returns (column-major factors, pivots)."""
    n = K.shape[0]
    A = np.asfortranarray(K, dtype=np.float64).ravel(order="F").copy()
    piv = np.empty(n, dtype=np.int32)
    _check(lib().or_lu_factor(n, _p(A), _pi(piv)), "lu_factor")
    return A, piv


def lu_solve(fac, b):
    A, piv = fac
    x = np.array(b, dtype=np.float64, copy=True)
    lib().or_lu_solve(x.shape[0], _p(A), _pi(piv), _p(x))
    return x


def rhs(g, voltages=None):
    el, pe = _rec(g.elements)
    v = np.ascontiguousarray(g.voltages if voltages is None else voltages, dtype=np.float64)
    b = np.empty(el.shape[0])
    _check(lib().or_rhs(pe, el.shape[0], _p(v), v.shape[0], _p(b)), "rhs")
    return b


def solve(g, voltages=None, K=None):
    """sigma (C/m^2) for the geometry's boundary conditions; also returns K and factors."""
    K = fill(g) if K is None else K
    fac = lu_factor(K)
    return lu_solve(fac, rhs(g, voltages)), K, fac


def eval_points(g, sigma, pts):
    el, pe = _rec(g.elements)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    n = pts.shape[0]
    phi = np.empty(n)
    E = np.empty((n, 3))
    lat = _lat(g)
    _check(lib().or_eval(pe, el.shape[0], _p(sigma), _p(lat), g.img_lo, g.img_hi, _p(pts), n, _p(phi), _p(E)),
           "eval")
    return phi, E


def centroids(g):
    el, pe = _rec(g.elements)
    n = el.shape[0]
    c = np.empty((n, 3)); nr = np.empty((n, 3)); a = np.empty(n)
    _check(lib().or_centroids(pe, n, _p(c), _p(nr), _p(a)), "centroids")
    return c, nr, a


def space_charge(src, q, tgt=None, soft=1e-6):
    """Softened direct sum; tgt=None means targets are the sources (self excluded)."""
    src = np.ascontiguousarray(src, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    selfidx = tgt is None
    tgt = src if tgt is None else np.ascontiguousarray(tgt, dtype=np.float64)
    nt = tgt.shape[0]
    phi = np.empty(nt)
    E = np.empty((nt, 3))
    lib().or_space_charge(_p(src), _p(q), src.shape[0], _p(tgt), nt, int(selfidx), soft, _p(phi), _p(E))
    return phi, E


def rhs_space_charge(g, pos, q, soft=1e-6):
    el, pe = _rec(g.elements)
    v = np.ascontiguousarray(g.voltages, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    b = np.empty(el.shape[0])
    _check(lib().or_rhs_space_charge(pe, el.shape[0], _p(v), v.shape[0], _p(pos), _p(q), pos.shape[0], soft,
                                     _p(b)), "rhs_space_charge")
    return b


def dynamic_step(g, fac, pos, q, soft=1e-6, mu=1e-4, dt=1e-9):
    """One Alg. 4 step; returns (new positions, sigma, E at carriers before the move)."""
    el, pe = _rec(g.elements)
    v = np.ascontiguousarray(g.voltages, dtype=np.float64)
    A, piv = fac
    pos = np.array(pos, dtype=np.float64, copy=True)
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = el.shape[0]
    sigma = np.empty(n)
    E = np.empty((pos.shape[0], 3))
    lat = _lat(g)
    _check(lib().or_dynamic_step(pe, n, _p(v), v.shape[0], _p(lat), g.img_lo, g.img_hi, _p(A), _pi(piv),
                                 _p(pos), _p(q), pos.shape[0], soft, mu, dt, _p(sigma), _p(E)), "dynamic_step")
    return pos, sigma, E


def fastvol(g, sigma, x_nodes, y_nodes, z_nodes, pts):
    """FastVolume map (Sec. 3.3): potential and field at the grid nodes (oracle
    evaluation), then trilinear interpolation of the eight nodes of each point's cell;
    coordinates outside the box are clamped to it."""
    ax, ay, az = (np.asarray(a, dtype=np.float64) for a in (x_nodes, y_nodes, z_nodes))
    X, Y, Z = np.meshgrid(ax, ay, az, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    vphi, vE = eval_points(g, sigma, nodes)
    vphi = vphi.reshape(len(ax), len(ay), len(az))
    vE = vE.reshape(len(ax), len(ay), len(az), 3)
    pts = np.asarray(pts, dtype=np.float64)
    phi = np.empty(pts.shape[0])
    E = np.empty((pts.shape[0], 3))
    for p, (x, y, z) in enumerate(pts):
        idx, frac = [], []
        for a, v in zip((ax, ay, az), (x, y, z)):
            v = min(max(v, a[0]), a[-1])
            c = min(max(int(np.searchsorted(a, v, side="right")) - 1, 0), len(a) - 2)
            idx.append(c)
            frac.append((v - a[c]) / (a[c + 1] - a[c]))
        sp, sE = 0.0, np.zeros(3)
        for di in (0, 1):
            for dj in (0, 1):
                for dk in (0, 1):
                    w = ((frac[0] if di else 1 - frac[0]) * (frac[1] if dj else 1 - frac[1])
                         * (frac[2] if dk else 1 - frac[2]))
                    sp += w * vphi[idx[0] + di, idx[1] + dj, idx[2] + dk]
                    sE += w * vE[idx[0] + di, idx[1] + dj, idx[2] + dk]
        phi[p] = sp
        E[p] = sE
    return phi, E


def voxel_grid(pos, d):
    """Alg. 3 grid of a cloud: (minimum corner, dims)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    lo = np.empty(3)
    dims = np.empty(3, dtype=np.int64)
    _check(lib().or_voxel_grid(_p(pos), pos.shape[0], _p(d), _p(lo), dims.ctypes.data_as(C.POINTER(C.c_int64))),
           "voxel_grid")
    return lo, dims


class Lines:
    """Line charges: start, stop (L x 3, m), lam (L, C/m), voxel (L, flat voxel index)."""

    def __init__(self, start, stop, lam, voxel=None):
        self.start = np.ascontiguousarray(start, dtype=np.float64)
        self.stop = np.ascontiguousarray(stop, dtype=np.float64)
        self.lam = np.ascontiguousarray(lam, dtype=np.float64)
        self.voxel = voxel

    def __len__(self):
        return self.lam.shape[0]


def voxel_lines(pos, q, d):
    """Point -> line charge reduction (Sec. 4.2, Alg. 3) with the readings stated in
    nebem_oracle.c: grid at the cloud's minimum corner, one z-directed line through the
    centre of every occupied voxel, lambda = total charge / dz."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = pos.shape[0]
    st, sp, lam = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
    vox = np.empty(n, dtype=np.int64)
    L = lib().or_voxel_lines(_p(pos), _p(q), n, _p(d), _p(st), _p(sp), _p(lam),
                             vox.ctypes.data_as(C.POINTER(C.c_int64)))
    _check(0 if L >= 0 else -1, "voxel_lines")
    return Lines(st[:L].copy(), sp[:L].copy(), lam[:L].copy(), vox[:L].copy())


def line_charge(lines, tgt, soft=1e-6):
    """Potential and field of the line charges at the targets (softened closed form)."""
    tgt = np.ascontiguousarray(tgt, dtype=np.float64)
    nt = tgt.shape[0]
    phi, E = np.empty(nt), np.empty((nt, 3))
    lib().or_line_charge(_p(lines.start), _p(lines.stop), _p(lines.lam), len(lines), _p(tgt), nt, soft, 0,
                         _p(phi), _p(E))
    return phi, E


def rhs_lines(g, lines, soft=1e-6):
    el, pe = _rec(g.elements)
    v = np.ascontiguousarray(g.voltages, dtype=np.float64)
    b = np.empty(el.shape[0])
    _check(lib().or_rhs_lines(pe, el.shape[0], _p(v), v.shape[0], _p(lines.start), _p(lines.stop),
                              _p(lines.lam), len(lines), soft, _p(b)), "rhs_lines")
    return b


def dynamic_step_lines(g, fac, pos, q, d, soft=1e-6, mu=1e-4, dt=1e-9):
    """One Alg. 4 step with Type == Line; returns (new positions, sigma, E at carriers)."""
    el, pe = _rec(g.elements)
    v = np.ascontiguousarray(g.voltages, dtype=np.float64)
    A, piv = fac
    pos = np.array(pos, dtype=np.float64, copy=True)
    q = np.ascontiguousarray(q, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = el.shape[0]
    sigma = np.empty(n)
    E = np.empty((pos.shape[0], 3))
    lat = _lat(g)
    _check(lib().or_dynamic_step_lines(pe, n, _p(v), v.shape[0], _p(lat), g.img_lo, g.img_hi, _p(A), _pi(piv),
                                       _p(pos), _p(q), pos.shape[0], _p(d), soft, mu, dt, _p(sigma), _p(E)),
           "dynamic_step_lines")
    return pos, sigma, E


def eval_am(g, sigma, prims, prim_of, prim_after, pts):
    """Adaptive Modelling (Sec. 3.3): element sums over the copies with ring index
    max(|k1|, |k2|) <= prim_after, primitive sums with the primitives' average charge
    densities over the others (readings stated in nebem_oracle.c)."""
    el, pe = _rec(g.elements)
    pr, pp = _rec(np.atleast_1d(prims)) if len(prims) else (None, None)
    po = np.ascontiguousarray(prim_of, dtype=np.int32)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    phi, E = np.empty(pts.shape[0]), np.empty((pts.shape[0], 3))
    lat = _lat(g)
    _check(lib().or_eval_am(pe, el.shape[0], _p(sigma), _p(lat), g.img_lo, g.img_hi, pp, len(prims),
                            po.ctypes.data_as(C.POINTER(C.c_int32)), prim_after, _p(pts), pts.shape[0], _p(phi),
                            _p(E)), "eval_am")
    return phi, E

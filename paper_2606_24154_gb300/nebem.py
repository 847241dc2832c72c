"""Thin Python binding of libnebem (include/nebem.h): the same entry points, argument
marshalling only.  Every step of the computation runs in the library's CUDA kernels;
there is no fallback.  Loading fails loudly when libnebem.so is missing or cannot be
loaded.

Host-array functions take numpy arrays; the ``*_device`` functions take raw device
pointers (e.g. ``torch.Tensor.data_ptr()``) and a CUDA stream handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnebem.so")

NEBEM_OK = 0
NEBEM_INVALID_ARG = -1
NEBEM_BAD_STATE = -2
NEBEM_OUT_OF_MEMORY = -3
NEBEM_CUDA = -4
NEBEM_SINGULAR = -5
NEBEM_NOT_CONVERGED = -6
NEBEM_TIMEOUT = -7
NEBEM_DEGENERATE_ELEMENT = -8
NEBEM_NO_DEVICE = -9
NEBEM_TOO_LARGE = -10

NEBEM_FP64 = 0
NEBEM_MIXED = 1


class nebem_options(C.Structure):
    _fields_ = [
        ("device", C.c_int32),
        ("ir_max_iter", C.c_int32),
        ("ir_tol", C.c_double),
        ("ratio_0", C.c_double),
        ("ratio_a", C.c_double),
        ("ratio_b", C.c_double),
        ("ratio_near", C.c_double),
        ("softening", C.c_double),
        ("sc_near", C.c_double),
        ("lu_block", C.c_int32),
        ("wait_polls", C.c_int32),
        ("mixed_point_tol", C.c_double),
        ("reserved", C.c_double * 3),
    ]


class nebem_solve_info(C.Structure):
    _fields_ = [
        ("precision", C.c_int32),
        ("iterations", C.c_int32),
        ("correction", C.c_double),
        ("residual", C.c_double),
        ("ms_fill", C.c_double),
        ("ms_factor", C.c_double),
        ("ms_solve", C.c_double),
        ("reserved", C.c_double * 4),
    ]


class nebem_eval_stats_t(C.Structure):
    _fields_ = [
        ("points", C.c_int64),
        ("refined_level1", C.c_int64),
        ("refined_level2", C.c_int64),
        ("ms_fp32", C.c_double),
        ("ms_level1", C.c_double),
        ("ms_level2", C.c_double),
        ("refined_level1_phi_only", C.c_int64),
        ("refined_level1_E_only", C.c_int64),
        ("reserved", C.c_double * 2),
    ]


class nebem_server_options(C.Structure):
    _fields_ = [
        ("arena_points", C.c_int64),
        ("chunk_points", C.c_int32),
        ("max_requests", C.c_int32),
        ("workers", C.c_int32),
        ("idle_us", C.c_int32),
        ("reserved", C.c_double * 4),
    ]


_vp = C.c_void_p
_d = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)

# name -> (restype, argtypes); every symbol declared in include/nebem.h
SIGNATURES = {
    "nebem_default_options": (C.c_int, [C.POINTER(nebem_options)]),
    "nebem_create": (C.c_int, [C.POINTER(_vp), C.POINTER(nebem_options)]),
    "nebem_destroy": (C.c_int, [_vp]),
    "nebem_last_error": (C.c_char_p, []),
    "nebem_status_string": (C.c_char_p, [C.c_int]),
    "nebem_set_geometry": (C.c_int, [_vp, _vp, C.c_int64, _d, C.c_int32, C.c_int32]),
    "nebem_set_bc": (C.c_int, [_vp, _d, C.c_int32]),
    "nebem_solve": (C.c_int, [_vp, C.c_int32, _d, C.POINTER(nebem_solve_info)]),
    "nebem_set_sigma": (C.c_int, [_vp, _d, C.c_int64]),
    "nebem_get_sigma": (C.c_int, [_vp, _d, C.c_int64]),
    "nebem_fill": (C.c_int, [_vp, C.c_int32, _d]),
    "nebem_matrix_entries": (C.c_int, [_vp, _i64p, _i64p, C.c_int64, _d]),
    "nebem_eval": (C.c_int, [_vp, _d, C.c_int64, _d, _d, C.c_int32]),
    "nebem_eval_device": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, C.c_int32, _vp]),
    "nebem_eval_err": (C.c_int, [_vp, _d, C.c_int64, _d, _d, _d, _i64p]),
    "nebem_eval_device_err": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, _vp, _vp]),
    "nebem_eval_stats": (C.c_int, [_vp, C.POINTER(nebem_eval_stats_t)]),
    "nebem_set_wait_polls": (C.c_int, [_vp, C.c_int32]),
    "nebem_set_error_model": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "nebem_peak_rates": (C.c_int, [_vp, _d]),
    "nebem_space_charge": (C.c_int, [_vp, _d, _d, C.c_int64, C.c_double]),
    "nebem_space_charge_eval": (C.c_int, [_vp, _d, C.c_int64, _d, _d, C.c_int32, C.c_int32]),
    "nebem_space_charge_lines": (C.c_int, [_vp, _d, _i64p]),
    "nebem_set_primitives": (C.c_int, [_vp, _vp, C.c_int32, C.POINTER(C.c_int32), C.c_int32]),
    "nebem_get_lines": (C.c_int, [_vp, _d, _d, _d, C.c_int64, _i64p]),
    "nebem_step": (C.c_int, [_vp, C.c_int32, C.c_double, C.c_double, C.c_int32, _d]),
    "nebem_lu_factor_device": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp]),
    "nebem_lu_factor_device_f32": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp]),
    "nebem_lu_solve_device": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, _vp]),
    "nebem_lu_factor_device_noalloc": (C.c_int, [_vp, C.c_int64, _vp, _vp]),
    "nebem_fastvol_build": (C.c_int, [_vp, _d, C.c_int32, _d, C.c_int32, _d, C.c_int32, C.c_int32]),
    "nebem_fastvol_eval": (C.c_int, [_vp, _d, C.c_int64, _d, _d]),
    "nebem_fastvol_eval_device": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, _vp]),
    "nebem_weighting_fields": (C.c_int, [_vp, _i32p, C.c_int32, C.c_int32, _d, C.POINTER(nebem_solve_info)]),
    "nebem_weighting_fastvol_build": (C.c_int, [_vp, _i32p, C.c_int32, _d, C.c_int32, _d, C.c_int32, _d, C.c_int32,
                                                C.c_int32, C.POINTER(_vp), C.POINTER(nebem_solve_info)]),
    "nebem_fvmap_eval": (C.c_int, [_vp, _d, C.c_int64, _d, _d]),
    "nebem_fvmap_eval_device": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, _vp]),
    "nebem_fvmap_destroy": (C.c_int, [_vp]),
    "nebem_image_table": (C.c_int, [_vp, _d, _i64p]),
    "nebem_pair_tiers": (C.c_int, [_vp, _d, C.c_int64, C.POINTER(C.c_uint8)]),
    "nebem_element_influence": (C.c_int, [_vp, _vp, C.c_int64, _d, C.c_int64, _d, _d]),
    "nebem_server_default_options": (C.c_int, [C.POINTER(nebem_server_options)]),
    "nebem_server_create": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int32, C.POINTER(nebem_server_options)]),
    "nebem_server_submit": (C.c_int, [_vp, C.c_int32, _d, C.c_int64, _d, _d, C.c_int32, _i64p]),
    "nebem_server_poll": (C.c_int, [_vp, C.c_int64, _i32p]),
    "nebem_server_wait": (C.c_int, [_vp, C.c_int64, C.c_int64]),
    "nebem_server_request_times": (C.c_int, [_vp, C.c_int64, _d, _d, _d]),
    "nebem_server_destroy": (C.c_int, [_vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libnebem.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libnebem.so not found at {path}: build it with "
                           "`python -m paper_2606_24154_gb300.build` (needs nvcc)")
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class NebemError(RuntimeError):
    def __init__(self, code, where):
        L = load()
        super().__init__(f"{where}: {L.nebem_status_string(code).decode()} ({code}): "
                         f"{L.nebem_last_error().decode()}")
        self.code = code


def _check(code, where):
    if code != NEBEM_OK:
        raise NebemError(code, where)
    return code


def _dp(a):
    return None if a is None else a.ctypes.data_as(_d)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- raw entry points
def nebem_default_options() -> nebem_options:
    o = nebem_options()
    _check(load().nebem_default_options(C.byref(o)), "nebem_default_options")
    return o


def nebem_create(opt: nebem_options | None = None):
    h = _vp()
    _check(load().nebem_create(C.byref(h), C.byref(opt) if opt is not None else None), "nebem_create")
    return h


def nebem_destroy(ctx):
    return load().nebem_destroy(ctx)


def nebem_set_geometry(ctx, elements: np.ndarray, lattice=None, img_lo=0, img_hi=0):
    el = np.ascontiguousarray(elements)
    assert el.dtype.itemsize == 128
    lat = None if lattice is None else _f64(lattice, (6,))
    _check(load().nebem_set_geometry(ctx, el.ctypes.data_as(_vp), el.shape[0], _dp(lat), img_lo, img_hi),
           "nebem_set_geometry")


def nebem_set_bc(ctx, voltages):
    v = _f64(voltages)
    _check(load().nebem_set_bc(ctx, _dp(v), v.shape[0]), "nebem_set_bc")


def nebem_solve(ctx, precision: int, n: int, allow_not_converged=False):
    sigma = np.empty(n)
    info = nebem_solve_info()
    rc = load().nebem_solve(ctx, precision, _dp(sigma), C.byref(info))
    if not (allow_not_converged and rc == NEBEM_NOT_CONVERGED):
        _check(rc, "nebem_solve")
    return sigma, info, rc


def nebem_set_sigma(ctx, sigma):
    s = _f64(sigma)
    _check(load().nebem_set_sigma(ctx, _dp(s), s.shape[0]), "nebem_set_sigma")


def nebem_get_sigma(ctx, n):
    s = np.empty(n)
    _check(load().nebem_get_sigma(ctx, _dp(s), n), "nebem_get_sigma")
    return s


def nebem_fill(ctx, precision: int, n: int):
    K = np.empty(n * n)
    _check(load().nebem_fill(ctx, precision, _dp(K)), "nebem_fill")
    return K.reshape(n, n).T  # column-major -> K[i, j]


def nebem_matrix_entries(ctx, rows, cols):
    r = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(cols, dtype=np.int64)
    out = np.empty(r.shape[0])
    _check(load().nebem_matrix_entries(ctx, r.ctypes.data_as(_i64p), c.ctypes.data_as(_i64p), r.shape[0], _dp(out)),
           "nebem_matrix_entries")
    return out


def nebem_eval(ctx, pts, precision: int, want_phi=True, want_E=True):
    p = _f64(pts, (-1, 3))
    n = p.shape[0]
    phi = np.empty(n) if want_phi else None
    E = np.empty((n, 3)) if want_E else None
    _check(load().nebem_eval(ctx, _dp(p), n, _dp(phi), _dp(E), precision), "nebem_eval")
    return phi, E


def nebem_eval_device(ctx, d_pts: int, n: int, d_phi: int | None, d_E: int | None, precision: int,
                      stream: int | None = None):
    _check(load().nebem_eval_device(ctx, d_pts, n, d_phi, d_E, precision, stream), "nebem_eval_device")


def nebem_eval_err(ctx, pts, want_phi=True, want_E=True):
    """Mixed evaluation with per-point error estimates: (phi, E, err[n, 2], refined count)."""
    p = _f64(pts, (-1, 3))
    n = p.shape[0]
    phi = np.empty(n) if want_phi else None
    E = np.empty((n, 3)) if want_E else None
    err = np.empty((n, 2))
    nref = C.c_int64(0)
    _check(load().nebem_eval_err(ctx, _dp(p), n, _dp(phi), _dp(E), _dp(err), C.byref(nref)), "nebem_eval_err")
    return phi, E, err, int(nref.value)


def nebem_eval_device_err(ctx, d_pts: int, n: int, d_phi: int | None, d_E: int | None, d_err: int | None,
                          stream: int | None = None):
    _check(load().nebem_eval_device_err(ctx, d_pts, n, d_phi, d_E, d_err, stream), "nebem_eval_device_err")


def nebem_peak_rates(ctx) -> dict:
    r = np.zeros(4)
    _check(load().nebem_peak_rates(ctx, _dp(r)), "nebem_peak_rates")
    return {"ffma": r[0], "ffma2_lanes": r[1], "mufu_rsqrt": r[2], "dfma": r[3]}


def nebem_set_error_model(ctx, gamma_r: float, gamma_b: float, gamma_s: float):
    _check(load().nebem_set_error_model(ctx, gamma_r, gamma_b, gamma_s), "nebem_set_error_model")


def nebem_set_wait_polls(ctx, polls: int):
    _check(load().nebem_set_wait_polls(ctx, polls), "nebem_set_wait_polls")


def nebem_eval_stats(ctx) -> nebem_eval_stats_t:
    st = nebem_eval_stats_t()
    _check(load().nebem_eval_stats(ctx, C.byref(st)), "nebem_eval_stats")
    return st


def nebem_space_charge(ctx, pos, q, softening=0.0):
    p = _f64(pos, (-1, 3))
    qq = _f64(q)
    _check(load().nebem_space_charge(ctx, _dp(p), _dp(qq), p.shape[0], softening), "nebem_space_charge")


def nebem_set_primitives(ctx, prims, prim_of, prim_after: int):
    pr = np.ascontiguousarray(prims)
    po = np.ascontiguousarray(prim_of, dtype=np.int32)
    _check(load().nebem_set_primitives(ctx, pr.ctypes.data_as(_vp) if len(pr) else None, len(pr),
                                       po.ctypes.data_as(C.POINTER(C.c_int32)), prim_after), "nebem_set_primitives")


def nebem_space_charge_lines(ctx, voxel) -> int:
    v = _f64(voxel)
    nl = C.c_int64(0)
    _check(load().nebem_space_charge_lines(ctx, _dp(v), C.byref(nl)), "nebem_space_charge_lines")
    return nl.value


def nebem_get_lines(ctx):
    """(start, stop, lambda) of the current line charges."""
    nl = C.c_int64(0)
    _check(load().nebem_get_lines(ctx, None, None, None, 0, C.byref(nl)), "nebem_get_lines")
    L = nl.value
    start, stop, lam = np.empty((L, 3)), np.empty((L, 3)), np.empty(L)
    _check(load().nebem_get_lines(ctx, _dp(start), _dp(stop), _dp(lam), L, C.byref(nl)), "nebem_get_lines")
    return start, stop, lam


def nebem_space_charge_eval(ctx, pts, precision: int, exclude_self=False):
    p = _f64(pts, (-1, 3))
    n = p.shape[0]
    phi = np.empty(n)
    E = np.empty((n, 3))
    _check(load().nebem_space_charge_eval(ctx, _dp(p), n, _dp(phi), _dp(E), precision, int(exclude_self)),
           "nebem_space_charge_eval")
    return phi, E


def nebem_step(ctx, steps: int, mu: float, dt: float, precision: int, n_carriers: int):
    pos = np.empty((n_carriers, 3))
    _check(load().nebem_step(ctx, steps, mu, dt, precision, _dp(pos)), "nebem_step")
    return pos


def nebem_lu_factor_device(ctx, d_A: int, n: int, d_piv: int, stream: int | None = None):
    _check(load().nebem_lu_factor_device(ctx, d_A, n, d_piv, stream), "nebem_lu_factor_device")


def nebem_lu_factor_device_f32(ctx, d_A: int, n: int, d_piv: int, stream: int | None = None):
    _check(load().nebem_lu_factor_device_f32(ctx, d_A, n, d_piv, stream), "nebem_lu_factor_device_f32")


def nebem_lu_solve_device(ctx, d_LU: int, n: int, d_piv: int, d_b: int, stream: int | None = None):
    _check(load().nebem_lu_solve_device(ctx, d_LU, n, d_piv, d_b, stream), "nebem_lu_solve_device")


def nebem_lu_factor_device_noalloc(d_A: int, n: int, d_piv: int, stream: int | None = None):
    """Dense LU with the library's static work space (n <= 4096); allocates nothing."""
    _check(load().nebem_lu_factor_device_noalloc(d_A, n, d_piv, stream), "nebem_lu_factor_device_noalloc")


def nebem_fastvol_build(ctx, x_nodes, y_nodes, z_nodes, precision: int):
    ax, ay, az = _f64(x_nodes), _f64(y_nodes), _f64(z_nodes)
    _check(load().nebem_fastvol_build(ctx, _dp(ax), ax.shape[0], _dp(ay), ay.shape[0], _dp(az), az.shape[0],
                                      precision), "nebem_fastvol_build")


def nebem_fastvol_eval(ctx, pts):
    p = _f64(pts, (-1, 3))
    n = p.shape[0]
    phi = np.empty(n)
    E = np.empty((n, 3))
    _check(load().nebem_fastvol_eval(ctx, _dp(p), n, _dp(phi), _dp(E)), "nebem_fastvol_eval")
    return phi, E


def nebem_fastvol_eval_device(ctx, d_pts: int, n: int, d_phi: int | None, d_E: int | None,
                              stream: int | None = None):
    _check(load().nebem_fastvol_eval_device(ctx, d_pts, n, d_phi, d_E, stream), "nebem_fastvol_eval_device")


def nebem_weighting_fields(ctx, readout, precision: int, n: int, allow_not_converged=False):
    """Weighting-field densities of the readout conductors: (sigma[n, k] with column j for
    readout[j], info, status)."""
    r = np.ascontiguousarray(readout, dtype=np.int32)
    k = r.shape[0]
    out = np.empty((k, n))  # row j of this C-ordered array is column j of the n x k result
    info = nebem_solve_info()
    rc = load().nebem_weighting_fields(ctx, r.ctypes.data_as(_i32p), k, precision, _dp(out), C.byref(info))
    if not (allow_not_converged and rc == NEBEM_NOT_CONVERGED):
        _check(rc, "nebem_weighting_fields")
    return np.ascontiguousarray(out.T), info, rc


class FvMap:
    """One weighting-field FastVolume map (owns its nebem_fvmap handle)."""

    def __init__(self, h):
        self.h = h

    def eval(self, pts):
        p = _f64(pts, (-1, 3))
        n = p.shape[0]
        phi = np.empty(n)
        E = np.empty((n, 3))
        _check(load().nebem_fvmap_eval(self.h, _dp(p), n, _dp(phi), _dp(E)), "nebem_fvmap_eval")
        return phi, E

    def eval_device(self, d_pts: int, n: int, d_phi: int | None, d_E: int | None, stream: int | None = None):
        _check(load().nebem_fvmap_eval_device(self.h, d_pts, n, d_phi, d_E, stream), "nebem_fvmap_eval_device")

    def close(self):
        if self.h is not None:
            load().nebem_fvmap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nebem_weighting_fastvol_build(ctx, readout, x_nodes, y_nodes, z_nodes, precision: int):
    """One FastVolume map per readout conductor: (list of FvMap, info)."""
    r = np.ascontiguousarray(readout, dtype=np.int32)
    k = r.shape[0]
    ax, ay, az = _f64(x_nodes), _f64(y_nodes), _f64(z_nodes)
    hs = (_vp * k)()
    info = nebem_solve_info()
    _check(load().nebem_weighting_fastvol_build(ctx, r.ctypes.data_as(_i32p), k, _dp(ax), ax.shape[0], _dp(ay),
                                                ay.shape[0], _dp(az), az.shape[0], precision, hs, C.byref(info)),
           "nebem_weighting_fastvol_build")
    return [FvMap(hs[j]) for j in range(k)], info


def nebem_image_table(ctx):
    cnt = C.c_int64()
    _check(load().nebem_image_table(ctx, None, C.byref(cnt)), "nebem_image_table")
    t = np.empty((cnt.value, 3))
    _check(load().nebem_image_table(ctx, _dp(t), C.byref(cnt)), "nebem_image_table")
    return t


def nebem_pair_tiers(ctx, pts, n_el: int, n_img: int):
    p = _f64(pts, (-1, 3))
    codes = np.empty(p.shape[0] * n_el * n_img, dtype=np.uint8)
    _check(load().nebem_pair_tiers(ctx, _dp(p), p.shape[0], codes.ctypes.data_as(C.POINTER(C.c_uint8))),
           "nebem_pair_tiers")
    return codes.reshape(p.shape[0], n_el, n_img)


def nebem_element_influence(ctx, elements, pts):
    el = np.ascontiguousarray(elements)
    p = _f64(pts, (-1, 3))
    ne, npt = el.shape[0], p.shape[0]
    phi = np.empty(ne * npt)
    E = np.empty((ne * npt, 3))
    _check(load().nebem_element_influence(ctx, el.ctypes.data_as(_vp), ne, _dp(p), npt, _dp(phi), _dp(E)),
           "nebem_element_influence")
    return phi.reshape(ne, npt), E.reshape(ne, npt, 3)


def nebem_server_default_options() -> nebem_server_options:
    o = nebem_server_options()
    _check(load().nebem_server_default_options(C.byref(o)), "nebem_server_default_options")
    return o


def nebem_server_create(ctxs, opt: nebem_server_options | None = None):
    arr = (_vp * len(ctxs))(*[c.value if isinstance(c, _vp) else c for c in ctxs])
    h = _vp()
    _check(load().nebem_server_create(C.byref(h), arr, len(ctxs), C.byref(opt) if opt is not None else None),
           "nebem_server_create")
    return h


def nebem_server_submit(srv, geometry: int, pts: np.ndarray, phi: np.ndarray | None, E: np.ndarray | None,
                        precision: int) -> int:
    """pts, phi and E must stay alive (and unmoved) until the request completes."""
    rid = C.c_int64()
    _check(load().nebem_server_submit(srv, geometry, _dp(pts), pts.shape[0], _dp(phi), _dp(E), precision,
                                      C.byref(rid)), "nebem_server_submit")
    return rid.value


def nebem_server_poll(srv, req_id: int) -> bool:
    done = C.c_int32()
    _check(load().nebem_server_poll(srv, req_id, C.byref(done)), "nebem_server_poll")
    return bool(done.value)


def nebem_server_wait(srv, req_id: int, timeout_ms: int = 60000):
    _check(load().nebem_server_wait(srv, req_id, timeout_ms), "nebem_server_wait")


def nebem_server_request_times(srv, req_id: int):
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(load().nebem_server_request_times(srv, req_id, C.byref(a), C.byref(b), C.byref(c)),
           "nebem_server_request_times")
    return a.value, b.value, c.value


def nebem_server_destroy(srv):
    return load().nebem_server_destroy(srv)


# ---------------------------------------------------------------- convenience wrapper
class Context:
    """Owns one nebem_ctx; thin method wrappers over the entry points above."""

    def __init__(self, device: int = 0, **opts):
        o = nebem_default_options()
        o.device = device
        for k, v in opts.items():
            setattr(o, k, v)
        self.h = nebem_create(o)
        self.n = 0

    def close(self):
        if self.h is not None:
            nebem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, g):
        nebem_set_geometry(self.h, g.elements, g.lattice, g.img_lo, g.img_hi)
        nebem_set_bc(self.h, g.voltages)
        self.n = g.n
        return self

    def solve(self, precision=NEBEM_FP64):
        return nebem_solve(self.h, precision, self.n)

    def fill(self, precision=NEBEM_FP64):
        return nebem_fill(self.h, precision, self.n)

    def set_sigma(self, sigma):
        nebem_set_sigma(self.h, sigma)

    def sigma(self):
        return nebem_get_sigma(self.h, self.n)

    def eval(self, pts, precision=NEBEM_FP64):
        return nebem_eval(self.h, pts, precision)

    def eval_err(self, pts):
        return nebem_eval_err(self.h, pts)

    def eval_device(self, d_pts, n, d_phi, d_E, precision=NEBEM_FP64, stream=None):
        nebem_eval_device(self.h, d_pts, n, d_phi, d_E, precision, stream)

    def image_table(self):
        return nebem_image_table(self.h)

"""The C-ABI used from a C program (no Python binding on the path): the unit-cube
conductor solved and evaluated through libnebem.so, against the oracle."""
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL64 = 1e-10


@pytest.fixture(scope="module")
def lib_dir():
    from paper_2606_24154_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_2606_24154_gb300")


def test_c_program_solves_and_evaluates(lib_dir, tmp_path):
    exe = tmp_path / "c_abi_check"
    subprocess.run(["gcc", "-O2", "-std=c99", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_check.c"), "-L", lib_dir, "-lnebem",
                    f"-Wl,-rpath,{lib_dir}", "-o", str(exe)], check=True)
    g = I.cube(n_per_edge=8)
    pts = I.cube_grid_points()[::37]
    with open(tmp_path / "el.bin", "wb") as f:
        f.write(np.int64(g.n).tobytes())
        f.write(np.ascontiguousarray(g.elements).tobytes())
    with open(tmp_path / "pts.bin", "wb") as f:
        f.write(np.int64(pts.shape[0]).tobytes())
        f.write(np.ascontiguousarray(pts, dtype=np.float64).tobytes())
    r = subprocess.run([str(exe), str(tmp_path / "el.bin"), str(tmp_path / "pts.bin"), str(tmp_path / "out.bin")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(tmp_path / "out.bin", dtype=np.float64)
    n, m = g.n, pts.shape[0]
    sigma, phi, E = out[:n], out[n:n + m], out[n + m:].reshape(m, 3)
    ref_sigma, _, _ = O.solve(g)
    rphi, rE = O.eval_points(g, ref_sigma, pts)
    assert np.abs(sigma - ref_sigma).max() <= TOL64 * np.abs(ref_sigma).max()
    assert np.abs(phi - rphi).max() <= TOL64 * np.abs(rphi).max()
    assert np.abs(E - rE).max() <= TOL64 * np.abs(rE).max()
    # capacitance of the unit cube: 0.6607 * 4 pi eps0 * a up to the discretisation (~1 %)
    _, _, area = O.centroids(g)
    C = (sigma * area).sum()
    assert abs(C / (0.6607 * 4 * np.pi * O.eps0() * 0.01) - 1.0) < 0.02


def test_peak_rates_are_plausible():
    """nebem_peak_rates measures the FP32, packed FP32x2, MUFU and FP64 pipes; each rate is
    positive and within a factor of a few of the unit counts (152 SMs x 128 FP32 lanes, 16
    MUFU and 2 FP64 per clock at up to 2.07 GHz; the clock under load may be lower)."""
    from paper_2606_24154_gb300 import build, nebem as N
    build.build()
    N.load()
    ctx = N.Context()  # held: the handle lives as long as this object
    r = N.nebem_peak_rates(ctx.h)
    clk = 2.07e9
    for key, units in (("ffma", 128), ("ffma2_lanes", 128), ("mufu_rsqrt", 16), ("dfma", 2)):
        nominal = 152 * units * clk
        assert 0.2 * nominal < r[key] < 2.5 * nominal, (key, r[key], nominal)

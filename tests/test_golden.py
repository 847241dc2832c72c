"""Stored expected values (tests/golden/, written by make_golden.py from the oracle) and
the literature value of the unit cube's capacitance.

CPU: the oracle still reproduces its stored values (a change of the oracle's arithmetic
shows here), and the 8 x 8 cube lands just below the unit-cube capacitance
0.6607 * 4 pi eps0 * a.  GPU: the CUDA path (through the C-ABI) against the same values."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def small_thgem():
    return I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)


def test_oracle_reproduces_stored_cube():
    d = load("cube_n8.json")
    g = I.cube(n_per_edge=8)
    sigma, _, _ = O.solve(g)
    _, _, area = O.centroids(g)
    assert abs((sigma * area).sum() - d["capacitance_F"]) <= 1e-12 * d["capacitance_F"]
    phi, E = O.eval_points(g, sigma, np.array(d["points_m"]))
    assert np.abs(phi - d["phi_V"]).max() <= 1e-12 * np.abs(d["phi_V"]).max()
    assert np.abs(E - np.array(d["E_V_per_m"])).max() <= 1e-11 * np.abs(d["E_V_per_m"]).max()
    # the unit cube's capacitance: a constant-element 8 x 8 mesh approaches it from below
    ratio = d["capacitance_over_4pi_eps0_a"] / d["literature_unit_cube_capacitance_over_4pi_eps0_a"]
    assert 0.99 < ratio < 1.0


def test_oracle_reproduces_stored_thgem():
    d = load("thgem_small.json")
    g = small_thgem()
    assert g.n == d["n_elements"]
    sigma, _, _ = O.solve(g)
    ref = np.array(d["sigma_C_per_m2"])
    assert np.abs(sigma[d["element_index"]] - ref).max() <= 1e-11 * np.abs(ref).max()
    phi, E = O.eval_points(g, sigma, np.array(d["points_m"]))
    assert np.abs(phi - d["phi_V"]).max() <= 1e-11 * np.abs(d["phi_V"]).max()
    assert np.abs(E - np.array(d["E_V_per_m"])).max() <= 1e-10 * np.abs(d["E_V_per_m"]).max()


@pytest.fixture(scope="module")
def N():
    from paper_2606_24154_gb300 import build, nebem
    build.build()
    nebem.load()
    return nebem


@pytest.mark.gpu
def test_gpu_matches_stored_values(N):
    d = load("cube_n8.json")
    g = I.cube(n_per_edge=8)
    ctx = N.Context().set_geometry(g)
    sigma, _, _ = ctx.solve(N.NEBEM_FP64)
    _, _, area = O.centroids(g)
    assert abs((sigma * area).sum() - d["capacitance_F"]) <= 1e-10 * d["capacitance_F"]
    phi, E = ctx.eval(np.array(d["points_m"]), N.NEBEM_FP64)
    assert np.abs(phi - d["phi_V"]).max() <= 1e-10 * np.abs(d["phi_V"]).max()
    assert np.abs(E - np.array(d["E_V_per_m"])).max() <= 1e-10 * np.abs(d["E_V_per_m"]).max()
    t = load("thgem_small.json")
    g = small_thgem()
    ctx = N.Context().set_geometry(g)
    sigma, _, _ = ctx.solve(N.NEBEM_FP64)
    ref = np.array(t["sigma_C_per_m2"])
    assert np.abs(sigma[t["element_index"]] - ref).max() <= 1e-10 * np.abs(ref).max()
    phi, E = ctx.eval(np.array(t["points_m"]), N.NEBEM_FP64)
    assert np.abs(phi - t["phi_V"]).max() <= 1e-10 * np.abs(t["phi_V"]).max()
    assert np.abs(E - np.array(t["E_V_per_m"])).max() <= 1e-10 * np.abs(t["E_V_per_m"]).max()
    phi, E = ctx.eval(np.array(t["points_m"]), N.NEBEM_MIXED)
    rphi, rE = np.array(t["phi_V"]), np.array(t["E_V_per_m"])
    assert np.abs(phi - rphi).max() <= 1e-6 * np.abs(rphi).max()
    assert np.abs(E - rE).max() <= 1e-6 * np.abs(rE).max()
    # per point (floor 1e-6 of the largest value; E as a vector)
    assert (np.abs(phi - rphi) / np.maximum(np.abs(rphi), 1e-6 * np.abs(rphi).max())).max() <= 1e-6
    m = np.linalg.norm(rE, axis=1)
    assert (np.linalg.norm(E - rE, axis=1) / np.maximum(m, 1e-6 * m.max())).max() <= 1e-6

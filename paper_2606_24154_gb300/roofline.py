"""Roofline bookkeeping for the mixed evaluation kernel (measurement only).

Algorithmic work of one mixed evaluation launch, counted per (point, element, image)
pair by its distance tier (distance to the image centroid in element circumradii):
  tier 0 (>= ratio_0):   4 Gauss nodes
  tier a (>= ratio_a):   6 Gauss nodes (triangle) or 9 (rectangle)
  tier b (>= ratio_b):   16 nodes
  tier c (>= ratio_near): 36 nodes
  near:                  one FP64 closed form
Per Gauss node the FP32 arithmetic is 13 lane operations (3 differences, 3 for r^2,
2 for w r^-1 and w r^-3 after one rsqrt, 1 for phi, 3 for E, 1 product) plus one MUFU
rsqrt; per pair 12 (two-float difference: 3 per axis, squared distance: 3).  The counts are
taken on a sample of points with the same thresholds as the kernel and scaled to the
launch.
"""
from __future__ import annotations

import numpy as np

OPS_PER_NODE = 13
OPS_PER_PAIR = 12
N_SM = 152
FP32_LANES_PER_SM = 128
MUFU_PER_SM = 16


def _element_table(g):
    kinds = g.elements["kind"]
    v = g.elements["v"]
    nv = np.where(kinds == 0, 4, 3)
    c = np.where(nv[:, None] == 4, v[:, :4].mean(1), v[:, :3].mean(1))
    d = np.linalg.norm(v - c[:, None, :], axis=2)
    d[nv == 3, 3] = 0.0
    rho = d.max(1)
    return c, rho, nv


def _images(g):
    if g.lattice is None:
        return np.zeros((1, 3))
    ks = np.arange(g.img_lo, g.img_hi + 1)
    return np.array([k1 * g.lattice[0] + k2 * g.lattice[1] for k1 in ks for k2 in ks])


def tier_counts(g, pts, sample=4096, ratio_0=64.0, ratio_a=24.0, ratio_b=8.0, ratio_near=3.0, chunk=32):
    c, rho, nv = _element_table(g)
    t = _images(g)
    C = (c[:, None, :] + t[None]).reshape(-1, 3)          # (el*img, 3)
    R = np.repeat(rho, t.shape[0])
    NV = np.repeat(nv, t.shape[0])
    na = np.where(NV == 4, 9, 6)
    slots_a = np.where(NV == 4, 10, 6)  # tier-a node slots in pairs (a 9-node rule is padded to 10)
    counts = {"pairs": 0, "t0": 0, "a": 0, "b": 0, "c": 0, "near": 0, "nodes": 0, "slots": 0, "sample_points": 0}
    P = pts[:sample]
    for s in range(0, P.shape[0], chunk):
        d = np.linalg.norm(P[s:s + chunk, None, :] - C[None], axis=2) / R[None]
        t0 = d >= ratio_0
        ta = (~t0) & (d >= ratio_a)
        tb = (d < ratio_a) & (d >= ratio_b)
        tc = (d < ratio_b) & (d >= ratio_near)
        tn = d < ratio_near
        counts["pairs"] += d.size
        counts["t0"] += int(t0.sum())
        counts["a"] += int(ta.sum())
        counts["b"] += int(tb.sum())
        counts["c"] += int(tc.sum())
        counts["near"] += int(tn.sum())
        counts["nodes"] += int(4 * t0.sum() + (ta * na[None]).sum() + 16 * tb.sum() + 36 * tc.sum())
        counts["slots"] += int(4 * t0.sum() + (ta * slots_a[None]).sum() + 16 * tb.sum() + 36 * tc.sum())
    counts["sample_points"] = int(P.shape[0])
    return counts


def fp32_ops_per_launch(counts, scale):
    return (OPS_PER_NODE * counts["nodes"] + OPS_PER_PAIR * counts["pairs"]) * scale


def fp32_peak_ops(sm_mhz):
    return N_SM * FP32_LANES_PER_SM * sm_mhz * 1e6


def mufu_peak(sm_mhz):
    return N_SM * MUFU_PER_SM * sm_mhz * 1e6


# FP64 closed form: FP64 instructions per (point, element, image) pair of the FP64
# evaluation kernel, from an ncu instruction count on the THGEM cell (166 DFMA, 59 DADD,
# 53 DMUL); the FP64 pipe issues 2 such instructions per clock per SM on this GPU
# (1.25 TFLOP/s nominal with an FMA as 2 flops).
FP64_INST_PER_PAIR = 278
FP64_INST_PER_SM_CLK = 2


def fp64_peak_inst(sm_mhz):
    return N_SM * FP64_INST_PER_SM_CLK * sm_mhz * 1e6


# ---------------------------------------------------------------- mixed fill
# Two-float (hi + lo FP32) operations of the mixed fill kernel, counted from its code (FP32
# lane operations; the node loops run two nodes per packed FP32x2 instruction, one lane
# each): per (row, column): c_i - c_j (3 two-float differences, 8 each) and its local
# components (3 two-float dot products, 28 each); interface rows add the normal's local
# components (3 more dot products).  Per far image pair: the FP32 tier test (12 + 3
# compares), X, Y, Z (3 differences), |D|^2 (28) and two negations; interface rows add
# n . D (28).  Per Gauss node: r^2 and the refined 1/r (41, plus one MUFU rsqrt), then w / r
# accumulated (12) on conductor rows, or w (n . (D + s)) / r^3 accumulated (49) on
# interface rows.
FILL_OPS_COLUMN = (108, 192)   # conductor, interface row
FILL_OPS_IMAGE = (69, 97)
FILL_OPS_NODE = (53, 90)
FILL_RATIOS = (96.0, 32.0, 6.0)


def fill_tier_counts(g, rows=256, seed=0, chunk=16):
    """Pair and node counts of the mixed fill on a sample of rows (collocation points), by
    row type, with the fill's distance tiers; scale = n / rows."""
    c, rho, nv = _element_table(g)
    t = _images(g)
    C = (c[:, None, :] + t[None]).reshape(-1, 3)
    R = np.repeat(rho, t.shape[0])
    NV = np.repeat(nv, t.shape[0])
    na = np.where(NV == 4, 9, 6)
    bc = g.elements["bc"]
    n = c.shape[0]
    sel = np.random.default_rng(seed).choice(n, min(rows, n), replace=False)
    out = {k: {"rows": 0, "pairs": 0, "far_pairs": 0, "nodes": 0, "near_pairs": 0} for k in ("cond", "iface")}
    for s in range(0, sel.size, chunk):
        r = sel[s:s + chunk]
        d = np.linalg.norm(c[r, None, :] - C[None], axis=2) / R[None]
        ta = d >= FILL_RATIOS[0]
        tb = (~ta) & (d >= FILL_RATIOS[1])
        tc = (d < FILL_RATIOS[1]) & (d >= FILL_RATIOS[2])
        far = ta | tb | tc
        nodes = (ta * na[None]).sum(1) + 16 * tb.sum(1) + 36 * tc.sum(1)
        for k, key in ((0, "cond"), (1, "iface")):
            m = bc[r] == k
            o = out[key]
            o["rows"] += int(m.sum())
            o["pairs"] += int(m.sum()) * d.shape[1]
            o["far_pairs"] += int(far[m].sum())
            o["near_pairs"] += int((~far[m]).sum())
            o["nodes"] += int(nodes[m].sum())
    out["sample_rows"] = int(sel.size)
    return out


def fill_ops(counts, n):
    """Two-float FP32 operations of one mixed fill of an n x n matrix, from fill_tier_counts."""
    scale = n / counts["sample_rows"]
    ops = 0.0
    for k, key in enumerate(("cond", "iface")):
        o = counts[key]
        ops += o["rows"] * n * FILL_OPS_COLUMN[k] + o["far_pairs"] * FILL_OPS_IMAGE[k] + o["nodes"] * FILL_OPS_NODE[k]
    return ops * scale


# ---------------------------------------------------------------- refinement, first level
# Two-float re-evaluation of flagged points with the FP32 pass's tiers (eval_acc.cu), FP32
# lane operations counted from its code (node pairs run in the packed FP32x2 instructions,
# two lanes each; a node slot is one lane of a node pair, padding included):
#   per (point, element): P - c_j (3 two-float differences, 8 each) and its local
#     components (3 two-float dot products, 28 each);
#   per far (point, element, image) pair: the FP32 tier test (12 + 4 compares), X, Y, Z
#     (3 differences, 24), |D|^2 (28), negations (3), the three node-pair sums folded to
#     two-float values (30) and E_local += D S0 + S (3 two-float multiply-adds, 60);
#   per node slot: r^2 and the refined 1/r (41, plus one MUFU rsqrt), w / r accumulated
#     (12), w / r^3 (11) accumulated (8), and w (2 s_x) / r^3, w (2 s_z) / r^3 accumulated
#     (1 + 12 + 12).
# A point whose E estimate was within the tolerance has phi alone re-evaluated: per pair
# without the folding and the E multiply-adds (161 - 90), per slot r^2, 1/r and w / r
# (41 + 12).  A point whose phi estimate was within it has E alone re-evaluated: per slot
# without w / r (97 - 12).
ACC1_OPS_ELEMENT = 108
ACC1_OPS_PAIR = 161
ACC1_OPS_SLOT = 97
ACC1_OPS_PAIR_PHI = 71
ACC1_OPS_SLOT_PHI = 53
ACC1_OPS_SLOT_E = 85


def acc1_ops_per_point(counts, n_el, mode="both"):
    """FP32 lane operations of the first refinement level per refined point, from
    tier_counts taken on a sample of refined points; mode "both", "phi" or "E" (which
    quantities the point has re-evaluated)."""
    pair, slot = {"both": (ACC1_OPS_PAIR, ACC1_OPS_SLOT), "phi": (ACC1_OPS_PAIR_PHI, ACC1_OPS_SLOT_PHI),
                  "E": (ACC1_OPS_PAIR, ACC1_OPS_SLOT_E)}[mode]
    per = counts["sample_points"]
    far = counts["t0"] + counts["a"] + counts["b"] + counts["c"]
    return ACC1_OPS_ELEMENT * n_el + (pair * far + slot * counts["slots"]) / per


# Space-charge carrier sum (spacecharge.cu, mixed): per (target, source) pair, the two-float
# difference (9), r^2 + s^2 (3), then q / r and q / r^3 and the four accumulations (7), plus
# one MUFU rsqrt.
SC_OPS_PER_PAIR = 19

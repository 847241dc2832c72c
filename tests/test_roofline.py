"""The work counts behind bench.py's roofline (paper_2606_24154_gb300/roofline.py), CPU
only: the host-side tier counts agree with the oracle's own pair classification (up to
pairs within FP32 rounding of a threshold), and the peaks are the unit counts times the
clock."""
import numpy as np

from oracle import oracle as O
from paper_2606_24154_gb300 import inputs as I
from paper_2606_24154_gb300 import roofline as R


def test_tier_counts_match_the_oracle_classification():
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    pts = I.cell_points(g, 48, I.rng(0, 70))
    counts = R.tier_counts(g, pts, sample=48)
    codes = O.pair_tiers(g, pts)
    n_img = g.n_images
    assert counts["pairs"] == codes.size == 48 * g.n * n_img
    rect = np.repeat((g.elements["kind"] != I.KIND_TRI)[None, :, None], n_img, axis=2)
    rect = np.broadcast_to(rect, codes.shape)
    ref = {"t0": int((codes == 0).sum()), "a": int((codes == 1).sum()), "b": int((codes == 2).sum()),
           "c": int((codes == 3).sum()), "near": int((codes == 4).sum())}
    ref_nodes = int(4 * ref["t0"] + 9 * ((codes == 1) & rect).sum() + 6 * ((codes == 1) & ~rect).sum()
                    + 16 * ref["b"] + 36 * ref["c"])
    # FP64 distances (host count) against the FP32 decision (oracle): only pairs within a
    # few ulps of a threshold may differ
    for k in ref:
        assert abs(counts[k] - ref[k]) <= max(2, 1e-4 * counts["pairs"]), (k, counts[k], ref[k])
    assert abs(counts["nodes"] - ref_nodes) <= 1e-4 * ref_nodes
    ops = R.fp32_ops_per_launch(counts, 2.0)
    assert ops == 2.0 * (13 * counts["nodes"] + 12 * counts["pairs"])


def test_peaks_from_unit_counts():
    assert R.fp32_peak_ops(2070.0) == 152 * 128 * 2070e6
    assert R.mufu_peak(2070.0) == 152 * 16 * 2070e6
    assert R.fp64_peak_inst(2070.0) == 152 * 2 * 2070e6


def test_refinement_counts():
    """Node slots count a 9-node tier-a rule as 10 (five packed pairs); the first refinement
    level's operations are the per-element, per-pair and per-slot counts added up."""
    g = I.thgem(I.PlateSpec(n_phi=24, n_r=3, n_zc=1, n_zf=4), n_plane=3)
    pts = I.cell_points(g, 16, I.rng(0, 71))
    c = R.tier_counts(g, pts, sample=16)
    rect_a = (c["slots"] - c["nodes"])  # one padding slot per rectangle tier-a pair
    assert rect_a >= 0 and c["slots"] - rect_a == c["nodes"]
    far = c["t0"] + c["a"] + c["b"] + c["c"]
    per = R.acc1_ops_per_point(c, g.n)
    assert per == R.ACC1_OPS_ELEMENT * g.n + (R.ACC1_OPS_PAIR * far + R.ACC1_OPS_SLOT * c["slots"]) / 16


def test_refinement_ops_by_mode():
    """A point re-evaluated for phi alone or E alone costs fewer counted operations than one
    re-evaluated for both, and the per-mode counts differ from the full one by exactly the
    parts each mode skips."""
    c = {"sample_points": 4, "t0": 100, "a": 10, "b": 2, "c": 1, "near": 3, "slots": 460, "nodes": 458, "pairs": 116}
    n_el = 50
    both = R.acc1_ops_per_point(c, n_el)
    phi = R.acc1_ops_per_point(c, n_el, "phi")
    e = R.acc1_ops_per_point(c, n_el, "E")
    far = 113
    assert both - phi == ((R.ACC1_OPS_PAIR - R.ACC1_OPS_PAIR_PHI) * far
                          + (R.ACC1_OPS_SLOT - R.ACC1_OPS_SLOT_PHI) * c["slots"]) / 4
    assert both - e == (R.ACC1_OPS_SLOT - R.ACC1_OPS_SLOT_E) * c["slots"] / 4
    assert phi < e < both

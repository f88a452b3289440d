"""CPU checks of the comparison rules in oracle/parity.py (no GPU): the near-tie excuse
applies only at the first block where two runs part, and only for a gap logged there."""
import numpy as np

from oracle import parity as P
from oracle import rbrp as O
from paper_2309_16002_gb300 import workloads as WL


def _ref(bps, gaps, D, D0=1.0):
    blocks = []
    for t, (bp, (sg, cg, fg), Dt) in enumerate(zip(bps, gaps, D), start=1):
        blocks.append(dict(t=t, b_t=bp, bp=bp, sample_gap=sg, cpqr_gap=cg, filter_gap=fg, D=Dt))
    S = np.arange(sum(bps), dtype=np.int64) * 3
    return dict(S=S, blocks=blocks, D0=D0)


BIG = (1e-3, 1e-3, 1e-3)


def test_identical_skeletons_pass_without_note():
    ref = _ref([4, 4], [BIG, BIG], [0.1, 0.01])
    assert P.fp64_skeleton_check(ref, ref["S"].copy(), 0.02) == (True, "")


def test_mismatch_is_excused_only_by_a_gap_in_its_own_block():
    ref = _ref([4, 4, 4], [BIG, (1e-14, 1e-3, 1e-3), BIG], [0.5, 0.1, 0.01])
    S = ref["S"].copy()
    S[5] = 1  # parts in block 2 (positions 4..7), which logged a sampling near-tie
    ok, note = P.fp64_skeleton_check(ref, S, 1e-3)
    assert ok and "sample" in note and "position 5" in note
    S = ref["S"].copy()
    S[9] = 1  # parts in block 3: the near-tie of block 2 does not excuse it
    ok, note = P.fp64_skeleton_check(ref, S, 1e-3)
    assert not ok
    S = ref["S"].copy()
    S[1] = 1  # parts in block 1, before the near-tie
    assert not P.fp64_skeleton_check(ref, S, 1e-3)[0]


def test_filter_and_cpqr_gaps_excuse_their_block():
    for gaps in [(1e-3, 1e-15, 1e-3), (1e-3, 1e-3, 1e-13)]:
        ref = _ref([4, 4], [BIG, gaps], [0.5, 0.1])
        S = ref["S"].copy()
        S[6] = 2
        assert P.fp64_skeleton_check(ref, S, 1e-3)[0]


def test_stop_test_near_tie():
    # the GPU ran one block past the oracle's stop: excused only when the oracle's last
    # ||d||_1 / ||d0||_1 sat within 1e-12 (relative) of tau
    tau = 0.01
    ref = _ref([4, 4], [BIG, BIG], [0.5, tau * (1 - 1e-14)])
    S = np.concatenate([ref["S"], [999, 998]])
    assert P.fp64_skeleton_check(ref, S, tau)[0]
    ref = _ref([4, 4], [BIG, BIG], [0.5, tau * 0.5])
    assert not P.fp64_skeleton_check(ref, S, tau)[0]
    # the GPU stopped one block early: the stop test of the previous block must be a near-tie
    ref = _ref([4, 4, 4], [BIG, BIG, BIG], [0.5, tau * (1 + 1e-13), tau * 0.1])
    assert P.fp64_skeleton_check(ref, ref["S"][:8], tau)[0]
    ref = _ref([4, 4, 4], [BIG, BIG, BIG], [0.5, tau * 2, tau * 0.1])
    assert not P.fp64_skeleton_check(ref, ref["S"][:8], tau)[0]


def test_mixed_bar_numbers():
    assert P.mixed_bar(1.05e-2, 1e-2) and not P.mixed_bar(1.06e-2, 1e-2)
    assert P.mixed_bar(1.9e-5, 1e-5) and not P.mixed_bar(2.1e-5, 1e-5)


def test_oracle_logs_the_gaps_the_rules_read():
    """The oracle's block records carry every gap the rules use, and a run compared with
    itself passes."""
    X, _ = WL.spectral(n=300, d=40, rate=0.85, seed=4)
    ref = O.rbrp_id(X, tau=1e-5, b=8, seed=1)
    for blk in ref["blocks"]:
        assert {"sample_gap", "cpqr_gap", "filter_gap", "D", "bp"} <= set(blk)
        assert blk["filter_gap"] >= 0
    assert P.fp64_skeleton_check(ref, ref["S"], 1e-5) == (True, "")
    assert abs(P.id_error(X, ref["S"], ref["W"]) ** 2 - O.id_error_sq(X, ref["S"], ref["W"])) < 1e-15

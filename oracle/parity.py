"""Comparison of a GPU result with an oracle run (test infrastructure only).

Used by tests/, __graft_entry__.smoke() and bench.py's checks; it holds no step
of the method, only the bars that a GPU result is held to against oracle.rbrp:

  * FP64 path: the skeletons must equal the oracle's under the shared Philox
    stream.  The one excuse is a rounding near-tie AT THE FIRST BLOCK WHERE THE
    TWO RUNS PART: every skeleton before that block must agree, and the oracle
    must have logged, for that block, a relative gap below NEAR_TIE in one of
    the decisions rounding can flip there -- the b_t-th versus (b_t+1)-th
    sampling key (Alg. 2, sampling step), a CPQR pivot choice (Alg. 2, local
    CPQR), the truncation b' against tau_b (robust blockwise filtering remark,
    Sec. 4), or the stopping test of the previous block against tau (Alg. 2,
    stopping test).  A mismatch anywhere else fails.
  * Mixed precision: e_gpu <= max(1.05 e_oracle, e_oracle + 1e-5), with
    e = ||X - W X_S||_F / ||X||_F, e_gpu from the GPU's S and W and e_oracle
    from the oracle's own S and W on the same input.
"""
import numpy as np

NEAR_TIE = 1e-12


def mixed_bar(e_gpu, e_oracle):
    """The mixed-precision bar on the unsquared relative error."""
    return e_gpu <= max(1.05 * e_oracle, e_oracle + 1e-5)


def first_divergence(ref, S):
    """Position j of the first differing skeleton and the oracle block holding position j
    (None when the oracle has no block there, i.e. the GPU ran past the oracle's stop).
    Returns None when S equals the oracle's skeletons."""
    S_ref = [int(x) for x in ref["S"]]
    S = [int(x) for x in S]
    if S == S_ref:
        return None
    m = min(len(S), len(S_ref))
    j = next((i for i in range(m) if S[i] != S_ref[i]), m)
    acc = 0
    for idx, blk in enumerate(ref["blocks"]):
        if j < acc + blk["bp"]:
            return j, idx
        acc += blk["bp"]
    return j, None


def _stop_gap(ref, idx, tau):
    """Relative distance of ||d||_1 / ||d0||_1 from tau after oracle block idx (-1: before
    the first block)."""
    if tau is None or tau < 0 or ref["D0"] <= 0:
        return np.inf
    D = ref["D0"] if idx < 0 else ref["blocks"][idx]["D"]
    return abs(D / ref["D0"] - tau) / tau if tau > 0 else np.inf


def fp64_skeleton_check(ref, S, tau=None):
    """Checks FP64 skeletons against the oracle run `ref`.

    Returns (ok, note): ok is True when S equals the oracle's skeletons, or when the first
    block where they part carries a logged near-tie (then note says which one and where);
    otherwise ok is False and note describes the mismatch.
    """
    div = first_divergence(ref, S)
    if div is None:
        return True, ""
    j, idx = div
    blocks = ref["blocks"]
    if idx is None:
        # the GPU kept going after the oracle stopped: only a near-tie of the last stop test excuses it
        g = _stop_gap(ref, len(blocks) - 1, tau)
        kinds = {"stop": g}
        where = "after the oracle's last block %d" % len(blocks)
    else:
        blk = blocks[idx]
        kinds = {"sample": blk["sample_gap"], "cpqr": blk["cpqr_gap"],
                 "filter": blk.get("filter_gap", np.inf), "stop": _stop_gap(ref, idx - 1, tau)}
        where = "oracle block %d (t = %d)" % (idx, blk["t"])
    name, gap = min(kinds.items(), key=lambda kv: kv[1])
    note = "skeletons part at position %d, %s; smallest logged gap there: %s %.3e" % (j, where, name, gap)
    return gap < NEAR_TIE, note


def id_error(X, S, W):
    """e = ||X - W X_S||_F / ||X||_F in FP64."""
    X = np.asarray(X, dtype=np.float64)
    S = np.asarray(S, dtype=np.int64)
    nx = float(np.sum(X * X))
    if nx == 0:
        return 0.0
    E = X - np.asarray(W, dtype=np.float64) @ X[S]
    return float(np.sqrt(np.sum(E * E) / nx))

"""Pins for oracle/rbrp.py: each checks the oracle against something other than itself
(a library routine, a closed form, an identity from the paper, brute force, or an
exact probability law)."""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy import stats

from oracle import rbrp as O
from paper_2309_16002_gb300 import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- sampler (Alg. 2, sampling step)
def test_race_sampler_plackett_luce_law():
    """Ordered pair (S_t[0], S_t[1]) ~ p_i p_j / (1 - p_i): sequential sampling without replacement."""
    d = np.array([5.0, 1.0, 3.0, 0.5, 2.5])
    p = d / d.sum()
    elig = np.ones(5, dtype=bool)
    N = 30000
    counts = np.zeros((5, 5))
    for s in range(N):
        S_t, _ = O.sample_block(d, elig, 2, 1, seed=s)
        counts[S_t[0], S_t[1]] += 1
    expect = np.array([[p[i] * p[j] / (1 - p[i]) if i != j else 0.0 for j in range(5)] for i in range(5)])
    mask = ~np.eye(5, dtype=bool)
    chi = stats.chisquare(counts[mask], N * expect[mask])
    assert chi.pvalue > 1e-4


def test_sampler_skips_ineligible_and_zero_rows():
    d = np.array([0.0, 2.0, 1.0, 4.0, 3.0])
    elig = np.array([True, True, False, True, True]) & (d > 0)
    for s in range(200):
        S_t, _ = O.sample_block(d, elig, 3, 2, seed=s)
        assert set(S_t.tolist()) <= {1, 3, 4} and len(set(S_t.tolist())) == 3
    S_all, gap = O.sample_block(d, elig, 3, 2, seed=0)
    assert sorted(S_all.tolist()) == [1, 3, 4] and gap == np.inf


def test_greedy_block_is_topb():
    d = np.array([1.0, 7.0, 3.0, 7.0, 0.5])
    S_t, _ = O.greedy_block(d, d > 0, 3)
    assert S_t.tolist() == [1, 3, 2]


# ---------------------------------------------------------------- CPQR filter (Alg. 2, local CPQR and truncation)
def test_cpqr_factorisation_and_lapack_pivots():
    rng = np.random.default_rng(3)
    for trial in range(5):
        V = rng.standard_normal((40, 12)) * rng.uniform(0.1, 3.0, size=12)
        Qv, R, piv, gap = O.cpqr(V)
        assert np.allclose(Qv.T @ Qv, np.eye(12), atol=1e-13)
        assert np.allclose(Qv @ R, V[:, piv], atol=1e-12)
        assert np.allclose(R, np.triu(R))
        dg = np.abs(np.diag(R))
        assert np.all(dg[:-1] >= dg[1:] - 1e-12)
        _, R_l, piv_l = sla.qr(V, mode="economic", pivoting=True)
        assert piv.tolist() == piv_l.tolist()
        assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(R_l)), rtol=1e-11)


def test_filter_tail_mass_definition():
    """b' = max{i : ||R_V(i:,i:)||_F^2 >= tau_b ||R_V||_F^2}, worked by hand on a 4x4 R_V."""
    R = np.array([[3.0, 1.0, 0.0, 2.0],
                  [0.0, 2.0, 1.0, 0.0],
                  [0.0, 0.0, 1.0, 1.0],
                  [0.0, 0.0, 0.0, 0.5]])
    # total 9+1+4+4+1+1+1+0.25 = 21.25; tails: 21.25, 7.25 (4+1+1+1+0.25), 2.25, 0.25
    bp, tails = O.filter_rank(R, 0.25)
    assert np.allclose(tails, [21.25, 7.25, 2.25, 0.25])
    assert bp == 2                      # 7.25 >= 5.3125 > 2.25
    assert O.filter_rank(R, 0.1)[0] == 3  # 2.25 >= 2.125
    assert O.filter_rank(R, 0.0)[0] == 4
    assert O.filter_rank(R, 1.0)[0] == 1


def test_filter_toy_facts():
    """Rationale after the RBRP conjecture (Sec. 4): rank-deficient V gives b' <= rank(V);
    orthogonal equal-norm columns give b' = b; an exact duplicate is never accepted twice."""
    rng = np.random.default_rng(5)
    b = 8
    V = rng.standard_normal((30, 3)) @ rng.standard_normal((3, b))
    _, R, _, _ = O.cpqr(V)
    assert O.filter_rank(R, 1.0 / b)[0] <= 3
    # equal-norm orthogonal columns meet the threshold with equality at i = b, so use an
    # instance whose Householder steps are exact (columns 2 e_j) for the exact claim ...
    E = np.zeros((30, b))
    E[np.arange(b), rng.permutation(b)] = 2.0
    _, R, _, _ = O.cpqr(E)
    assert O.filter_rank(R, 1.0 / b)[0] == b
    # ... and on a Haar instance rounding may decide the tie of the last column only
    Qo = WL.haar(rng, 30, b) * 2.5
    _, R, _, _ = O.cpqr(Qo)
    assert O.filter_rank(R, 1.0 / b)[0] >= b - 1
    W = rng.standard_normal((30, 4))
    Vd = np.concatenate([W, W[:, [1]]], axis=1)
    _, R, piv, _ = O.cpqr(Vd)
    bp = O.filter_rank(R, 1.0 / 5)[0]
    acc = set(piv[:bp].tolist())
    assert not ({1, 4} <= acc)


# ---------------------------------------------------------------- whole method (Alg. 2 + Alg. 3)
@pytest.fixture(scope="module")
def spectral_small():
    X, sigma = WL.spectral(n=600, d=60, rate=0.9, seed=11)
    return X, sigma


@pytest.fixture(scope="module")
def run_small(spectral_small):
    X, _ = spectral_small
    return O.rbrp_id(X, tau=1e-6, b=8, seed=0)


def test_residual_identity_and_projection(spectral_small, run_small):
    """Proof of the ID-revealing proposition (Sec. 5.1): ||X - L Q^T||_F^2 = ||d||_1 and L Q^T = X X_S^+ X_S."""
    X, _ = spectral_small
    out = run_small
    E = X - out["L"] @ out["Q"].T
    assert abs(np.sum(E * E) - out["D"]) <= 1e-10 * out["D0"]
    XS = X[out["S"]]
    P = X @ np.linalg.pinv(XS) @ XS
    assert np.allclose(out["L"] @ out["Q"].T, P, atol=1e-10 * np.sqrt(out["D0"] / X.shape[0]))
    assert np.allclose(out["Q"].T @ out["Q"], np.eye(out["Q"].shape[1]), atol=1e-12)


def test_W_identity_rows_lstsq_and_revealing(spectral_small, run_small):
    X, _ = spectral_small
    out = run_small
    S, W = out["S"], out["W"]
    k = len(S)
    assert np.array_equal(W[S], np.eye(k))
    L1 = out["L"][S]
    assert np.max(np.abs(np.triu(L1, 1))) <= 1e-12 * np.max(np.abs(L1))
    W_ls = O.interp_matrix_ls(X, S)
    cond = np.linalg.cond(X[S])
    assert np.max(np.abs(W - W_ls)) <= 1e-10 * cond * max(1.0, np.max(np.abs(W_ls)))
    e2 = O.id_error_sq(X, S, W)
    assert abs(e2 - out["rel_err_sq"]) <= 1e-12 + 1e-8 * out["rel_err_sq"]
    assert out["rel_err_sq"] <= 1e-6
    W_t = O.interp_matrix_tsvd(out["L"], S)
    assert np.allclose(W_t, W, atol=1e-8)


def test_error_at_least_svd_optimum_closed_form(run_small):
    """Eckart-Young with sigma_i = 0.9^i: e^2 >= 0.81^k (1 - 0.81^(r-k)) / (1 - 0.81^r)."""
    r = 60
    k = len(run_small["S"])
    bound = 0.81 ** k * (1 - 0.81 ** (r - k)) / (1 - 0.81 ** r)
    assert run_small["rel_err_sq"] >= bound * (1 - 1e-9)
    # the tolerance is met but not with absurd oversampling
    assert k <= r


def test_exact_rank_r_recovered():
    X = WL.low_rank(n=500, d=100, r=20, seed=7)
    out = O.rbrp_id(X, tau=1e-12, b=16, seed=3)
    assert len(out["S"]) == 20
    assert O.id_error_sq(X, out["S"], out["W"]) <= 1e-24


def test_example_2_1_one_row_per_direction():
    X = WL.example_2_1(n=48, k=8, r=3, alpha=1e4)
    out = O.rbrp_id(X, tau=1e-14, b=4, seed=1)
    dirs = sorted(int(np.argmax(np.abs(X[s]))) for s in out["S"])
    assert dirs == list(range(8))
    assert O.id_error_sq(X, out["S"], out["W"]) <= 1e-28


def test_example_2_1_golden_distribution():
    """Golden values of Sec. 2.2 (the squared-norm sampling example): p_i and eta_r."""
    with open(os.path.join(GOLDEN, "example_2_1.json")) as f:
        g = json.load(f)
    X = WL.example_2_1(n=g["n"], k=g["k"], r=g["r"], alpha=g["alpha"])
    d = O.row_sq_norms(X)
    p = d / d.sum()
    m = g["n"] // g["k"]
    # p_i in the paper is the mass of one direction; each direction has n/k rows
    p_dir = np.array([p[i * m:(i + 1) * m].sum() for i in range(g["k"])])
    assert np.allclose(p_dir, g["p_direction"], rtol=1e-14)
    s = np.linalg.svd(X, compute_uv=False)
    eta = np.sum(s[g["r"]:] ** 2) / np.sum(s ** 2)
    assert abs(eta - g["eta_r"]) <= 1e-14


def test_brute_force_subsets_tiny():
    """n <= 12: RBRP's error is >= the best subset of its size, and its W attains E_X(S) exactly."""
    rng = np.random.default_rng(9)
    for trial in range(4):
        X = rng.standard_normal((10, 6)) * np.array([5.0, 3.0, 1.0, 0.3, 0.1, 0.05])
        out = O.rbrp_id(X, tau=0.05, b=2, seed=trial)
        S = out["S"]
        k = len(S)
        best = min(O.skeleton_error_sq(X, list(c)) for c in itertools.combinations(range(10), k))
        mine = O.skeleton_error_sq(X, S)
        assert best <= mine + 1e-14
        assert abs(O.id_error_sq(X, S, out["W"]) - mine) <= 1e-12
        assert abs(out["rel_err_sq"] - mine) <= 1e-12


def test_b1_is_sequential_random_pivoting(spectral_small):
    """RBRP with b = 1 (tau_b = 1/b_t = 1 keeps one row) equals Alg. 1 run independently."""
    X, _ = spectral_small
    a = O.rbrp_id(X[:200], tau=1e-4, b=1, seed=4)
    s = O.srp(X[:200], tau=1e-4, seed=4)
    assert a["S"].tolist() == s["S"].tolist()
    assert abs(a["D"] - s["D"]) <= 1e-9 * a["D0"]
    assert np.allclose(a["L"] @ a["Q"].T, s["L"] @ s["Q"].T, atol=1e-9)


def test_srp_sequence_law_exact_enumeration():
    """Alg. 1's first two pivots follow p(i) p(j | i) with p(j | i) from the projected residual."""
    X = np.array([[3.0, 0.0, 1.0], [1.0, 2.0, 0.0], [0.5, 0.5, 2.0], [2.0, 1.0, 1.0]])
    n = X.shape[0]
    d = np.sum(X * X, axis=1)
    P = np.zeros((n, n))
    for i in range(n):
        q = X[i] / np.linalg.norm(X[i])
        Rr = X - np.outer(X @ q, q)
        di = np.sum(Rr * Rr, axis=1)
        di[i] = 0.0
        P[i] = d[i] / d.sum() * di / di.sum()
    N = 12000
    counts = np.zeros((n, n))
    for s in range(N):
        seq = O.srp(X, k=2, seed=s)["S"]
        counts[seq[0], seq[1]] += 1
    mask = ~np.eye(n, dtype=bool)
    chi = stats.chisquare(counts[mask], N * P[mask])
    assert chi.pvalue > 1e-4


def test_rbgp_b1_is_lapack_cpqr():
    """Blockwise greedy remark (Sec. 4): RBGP with b = 1 is CPQR; pivots equal LAPACK geqp3 on X^T."""
    rng = np.random.default_rng(21)
    X = rng.standard_normal((40, 15)) * rng.uniform(0.2, 2.0, size=(40, 1))
    out = O.rbrp(X, k=10, b=1, sampler="greedy")
    _, _, piv = sla.qr(X.T, mode="economic", pivoting=True)
    assert out["S"].tolist() == piv[:10].tolist()


def test_residual_and_downdate_forms_agree(spectral_small):
    X, _ = spectral_small
    a = O.rbrp_id(X, tau=1e-5, b=8, seed=2, form="residual")
    b = O.rbrp_id(X, tau=1e-5, b=8, seed=2, form="downdate")
    assert a["S"].tolist() == b["S"].tolist()
    assert abs(a["D"] - b["D"]) <= 1e-10 * a["D0"]
    assert np.allclose(a["W"], b["W"], atol=1e-7)


def test_fixed_rank_and_guards():
    X, _ = WL.spectral(n=300, d=40, rate=0.9, seed=12)
    out = O.rbrp_id(X, k=13, b=5, seed=0)
    assert len(out["S"]) == 13
    assert all(blk["b_t"] <= 5 for blk in out["blocks"])
    z = O.rbrp_id(np.zeros((20, 5)), tau=1e-3, b=4)
    assert len(z["S"]) == 0 and z["W"].shape == (20, 0)
    full = O.rbrp_id(np.random.default_rng(0).standard_normal((8, 5)), tau=0.0, b=4, seed=1)
    assert len(full["S"]) == 5


def test_brp_variant_accepts_whole_block():
    X, _ = WL.spectral(n=300, d=40, rate=0.9, seed=12)
    out = O.rbrp(X, tau=1e-4, b=6, seed=0, tau_b=0.0)
    assert all(blk["bp"] == blk["b_t"] for blk in out["blocks"])


def test_gmm_pitfall_robust_filter_helps():
    """Sec. 4, GMM pitfall: the robust filter needs fewer skeletons than plain BRP for the same error."""
    X = WL.gmm_pitfall(n=1000, d=120, k=40, seed=6)
    r = O.rbrp(X, tau=0.2, b=20, seed=0)
    p = O.rbrp(X, tau=0.2, b=20, seed=0, tau_b=0.0)
    assert len(r["S"]) < len(p["S"])


def test_tsvd_interp_clip_is_relative_to_sigma_max():
    """Remark on stable evaluation of L2 L1^{-1}: with L1 = U diag(s) V^T built from known factors,
    the truncated-SVD W is L2 V diag(1/s_kept) U^T, where s_kept are the s_i > 1e-12 s_max.  The
    spectrum below puts one value at 1e-13 s_max (dropped) and one at 1e-11 s_max (kept), and the
    whole L is scaled by 1e6, so an absolute clip, a dropped clip or a clip against s_min all fail."""
    rng = np.random.default_rng(17)
    k, n = 5, 40
    U, _ = np.linalg.qr(rng.standard_normal((k, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    s = np.array([1.0, 1e-3, 1e-6, 1e-11, 1e-13])
    for scale in (1.0, 1e6):
        L1 = scale * (U * s) @ V.T
        L2 = rng.standard_normal((n - k, k))
        S = np.arange(3, 3 + k)
        rest = np.setdiff1d(np.arange(n), S)
        L = np.zeros((n, k))
        L[S] = L1
        L[rest] = L2
        W = O.interp_matrix_tsvd(L, S)
        keep = s > 1e-12
        want = L2 @ ((V[:, keep] / (scale * s[keep])) @ U[:, keep].T)
        assert np.array_equal(W[S], np.eye(k))
        # the kept 1e-11 direction amplifies rounding by 1e11: compare relative to |want|
        assert np.max(np.abs(W[rest] - want)) <= 1e-3 * np.max(np.abs(want))
        # the dropped direction contributes nothing: W is orthogonal to U's last column
        assert np.max(np.abs(W[rest] @ U[:, ~keep])) <= 1e-4 * np.max(np.abs(want))

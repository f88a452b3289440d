"""Pins of the sketchy-pivoting oracle (oracle/sketchy.py) to facts outside itself:
a hand-worked LUPP example, LAPACK's partial-pivoting LU (getrf through scipy), the
least-squares identity W = Y Y_S^+ of Eq. (5.3) through an SVD-based solver, the
reduction of OSID to the optimal W = X X_S^+ when the embedding has full row rank,
exact recovery of an exactly low-rank input, and the ordering of the ID errors the
proposition of Sec. 5.2 and Eq. (5.2) imply."""
import numpy as np
import scipy.linalg as sla

from oracle import rbrp as O
from oracle import sketchy as K
from paper_2309_16002_gb300 import workloads as WL


def test_lupp_hand_example():
    # column 0: |3| wins (row 1); multipliers 1/3 (row 0), 2/3 (row 2); column 1 becomes
    # 2 - 1/3 = 5/3 (row 0) and 5 - 2/3 = 13/3 (row 2): row 2 wins
    A = np.array([[1.0, 2.0], [3.0, 1.0], [2.0, 5.0]])
    piv, gaps = K.lupp(A, 2)
    assert piv.tolist() == [1, 2]
    assert np.isclose(gaps[0], (3 - 2) / 3) and np.isclose(gaps[1], (13 / 3 - 5 / 3) / (13 / 3))


def _lapack_pivot_rows(A, k):
    """Rows chosen by LAPACK getrf (partial pivoting with row interchanges), in order."""
    _, ipiv = sla.lu_factor(A)
    perm = np.arange(A.shape[0])
    for i in range(min(k, len(ipiv))):
        j = ipiv[i]
        perm[i], perm[j] = perm[j], perm[i]
    return perm[:k]


def test_lupp_matches_lapack_getrf():
    rng = np.random.default_rng(3)
    for n, m in [(50, 8), (400, 30), (64, 64)]:
        A = rng.standard_normal((n, m)) * rng.uniform(0.1, 3.0, size=(n, 1))
        piv, _ = K.lupp(A, m)
        assert piv.tolist() == _lapack_pivot_rows(A, m).tolist()


def test_lupp_stops_at_the_rank():
    # columns 3.. are zero: after three pivots the Schur complement column is exactly zero
    rng = np.random.default_rng(4)
    A = np.zeros((80, 6))
    A[:, :3] = rng.standard_normal((80, 3))
    piv, _ = K.lupp(A, 6)
    assert len(piv) == 3 and len(set(piv.tolist())) == 3


def test_osid_is_the_least_squares_w_of_the_sketch():
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((300, 36))
    S = rng.choice(300, size=12, replace=False)
    W = K.osid(Y, S)
    assert np.array_equal(W[S], np.eye(12))
    sol, *_ = np.linalg.lstsq(Y[S].T, Y.T, rcond=None)  # SVD-based Y Y_S^+
    assert np.max(np.abs(W - sol.T)) <= 1e-10 * max(1.0, np.max(np.abs(sol)))


def test_orthonormal_row_embedding_gives_the_optimal_w():
    """With Omega Omega^T = c I (orthonormal rows, l >= d), W = Y Y_S^+ = X X_S^T (X_S X_S^T)^{-1}
    = X X_S^+, the optimal W of Eq. (5.1): OSID then reaches the skeletonization error."""
    X, _ = WL.spectral(n=400, d=30, rate=0.8, seed=6)
    q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((90, 30)))
    Om = 3.0 * q.T  # 30 x 90, orthonormal rows scaled by 3
    out = K.sk_lupp_id(X, Om, 10)
    W_ls = O.interp_matrix_ls(X, out["S"])
    assert np.max(np.abs(out["W"] - W_ls)) <= 1e-9 * max(1.0, np.max(np.abs(W_ls)))
    assert abs(out["rel_err_sq"] - O.skeleton_error_sq(X, out["S"])) <= 1e-12


def test_exact_low_rank_is_recovered():
    X = WL.low_rank(n=500, d=100, r=15, seed=8)
    Om = WL.gaussian_embedding(100, 45, seed=2)
    out = K.sk_lupp_id(X, Om, 15)
    assert len(out["S"]) == 15
    assert out["rel_err_sq"] <= 1e-24


def test_error_ordering_osid_between_optimal_and_unoversampled():
    """e_skel(S) <= e_OSID (W = Y Y_S^+ is a feasible W) and, with l = 3k, OSID stays close
    to the optimum (the proposition of Sec. 5.2) while Eq. (5.2) (l = k) does not."""
    X, _ = WL.spectral(n=2000, d=200, decay="power", rate=1.0, seed=9)
    k = 40
    Om = WL.gaussian_embedding(200, 3 * k, seed=3)
    osid = K.sk_lupp_id(X, Om, k)
    plain = K.sk_lupp_id(X, Om, k, osid_cols=k)
    e_skel = O.skeleton_error_sq(X, osid["S"])
    assert plain["S"].tolist() == osid["S"].tolist()
    assert e_skel <= osid["rel_err_sq"] * (1 + 1e-12)
    assert osid["rel_err_sq"] <= 2.0 * e_skel
    assert plain["rel_err_sq"] >= osid["rel_err_sq"]

"""Plain FP64 CPU oracle for sketchy pivoting with LU partial pivoting (SkLUPP) and the
oversampled sketchy interpolation matrix (OSID, Alg. 4).

Test infrastructure only: imported by tests/ and the CPU legs of bench.py.  The product
path never imports, links or runs anything under oracle/, and this module imports
nothing from the product.

Source: Dong, Chen, Martinsson, Pearce, arXiv 2309.16002.
  * Sec. 3.2 (sketchy pivoting): a Gaussian embedding sketches the rows, Y = X Omega
    (n x l), and greedy pivoting on the sketch (LUPP or CPQR) selects the skeletons;
    not rank-adaptive (k is given).
  * Sec. 5.2: Eq. (5.2), the sketched least-squares W = Y_k Y_{S,k}^{-1} that Alg. 3
    amounts to without oversampling (Y_k = X Omega(:, 1:k)); Alg. 4 (OSID) and
    Eq. (5.3): with Y_S^T = Q R (economic QR, Q l x k, R k x k), W(S,:) = I and
    W(rest,:) = (Y(rest,:) Q) R^{-T}, i.e. W = Y Y_S^+; l = 3k is the paper's usual
    oversampling; the proposition there (OSID is gamma-ID-revealing for l = Theta(k)).

Readings (where the paper leaves the details to its references):
  R18  The embedding Omega (d x l, i.i.d. N(0, 1/l)) is an input of the method: the
       caller draws it (workloads.gaussian_embedding) and both sides use the same one.
  R19  Skeleton selection is LU with partial (row) pivoting of Y(:, 1:k), the columns
       Eq. (5.2) keeps: the pivot of column j is the not-yet-pivoted row with the largest
       |entry| of the current Schur complement, ties to the smaller row index; a zero
       pivot (Y(:, 1:k) of rank below k) ends the selection early.  Skeletons are in
       pivot order.
  R20  OSID uses all l columns of the sketch (Alg. 4 with its Householder QR); Eq. (5.2)
       is the same formula on the first k columns.
  R21  Eq. (5.3) also writes W as X (Omega Omega^+) X_S^+.  That equality of the
       pseudo-inverses needs Omega Omega^T proportional to I (orthonormal rows); in
       general Alg. 4 computes W = Y Y_S^+, which is what this oracle returns (the
       paper's statement that E[W] = X X_S^+ for isotropic embeddings is not used).
"""
import numpy as np
import scipy.linalg as sla


def sketch(X, Omega):
    """Sketching step of Sec. 3.2: Y = X Omega (n x l), FP64."""
    return np.asarray(X, dtype=np.float64) @ np.asarray(Omega, dtype=np.float64)


def lupp(A, k):
    """LU with partial pivoting of A (n x m), at most k steps (reading R19).

    Right-looking Gaussian elimination without row exchanges: pivoted rows are only
    marked.  Returns (piv, gaps): the pivot rows in order, and per step the relative gap
    between the chosen |entry| and the runner-up (a rounding near-tie when tiny).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n, m = A.shape
    k = min(int(k), n, m)
    active = np.ones(n, dtype=bool)
    piv, gaps = [], []
    for j in range(k):
        mag = np.where(active, np.abs(A[:, j]), -1.0)
        best = mag.max()
        if not best > 0:
            break
        p = int(np.nonzero(mag == best)[0][0])
        mag[p] = -1.0
        gaps.append((best - max(mag.max(), 0.0)) / best)
        piv.append(p)
        active[p] = False
        mult = A[active, j] / A[p, j]
        A[active, j + 1:] -= np.outer(mult, A[p, j + 1:])
        A[active, j] = mult
    return np.array(piv, dtype=np.int64), np.array(gaps)


def osid(Y, S):
    """Alg. 4: W(S,:) = I, W(rest,:) = (Y(rest,:) Q) R^{-T} with Y_S^T = Q R (economic QR)."""
    Y = np.asarray(Y, dtype=np.float64)
    S = np.asarray(S, dtype=np.int64)
    n, k = Y.shape[0], S.shape[0]
    W = np.zeros((n, k))
    if k == 0:
        return W
    Q, R = np.linalg.qr(Y[S].T)
    W[S] = np.eye(k)
    rest = np.setdiff1d(np.arange(n), S)
    if rest.size:
        # W_rest R^T = Y_rest Q  <=>  R W_rest^T = (Y_rest Q)^T
        W[rest] = sla.solve_triangular(R, (Y[rest] @ Q).T, lower=False).T
    return W


def sk_lupp_id(X, Omega, k, osid_cols=None):
    """SkLUPP selection and the OSID interpolation matrix (Sec. 3.2, Alg. 4).

    X: n x d; Omega: d x l embedding (l >= k); k: number of skeletons; osid_cols:
    columns of the sketch OSID uses (default all l; k gives Eq. (5.2)).
    Returns dict(S, W, Y, gaps, rel_err_sq) with rel_err_sq = ||X - W X_S||_F^2 / ||X||_F^2.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = sketch(X, Omega)
    l = Y.shape[1]
    if k > l:
        raise ValueError("the sketch needs at least k columns")
    S, gaps = lupp(Y[:, :k], k)
    c = l if osid_cols is None else int(osid_cols)
    W = osid(Y[:, :c], S)
    E = X - W @ X[S]
    nx = float(np.sum(X * X))
    return dict(S=S, W=W, Y=Y, gaps=gaps, rel_err_sq=float(np.sum(E * E)) / nx if nx > 0 else 0.0)

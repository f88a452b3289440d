"""Plain FP64 CPU oracle for Robust Blockwise Random Pivoting (RBRP) and its ID.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py.  The product path (the CUDA library and its binding) never
imports, links or runs anything under oracle/, and this module imports nothing
from the product.

Source: Dong, Chen, Martinsson, Pearce, "Robust Blockwise Random Pivoting: Fast
and Accurate Adaptive Interpolative Decomposition" (arXiv 2309.16002).
  * problem statement: row ID X ~ W X_S, Eq. (1.1); skeletonization error
    E_X(S) = ||X - X X_S^+ X_S||_F^2, Eq. (1.2)
  * squared-norm distribution p_i = d_i / ||d||_1, Eq. (2.2)
  * CPQR step, Eq. (2.1) (greedy pivoting; used by the RBGP variant)
  * Alg. 1 (sequential random pivoting, SRP), Sec. 3.1
  * Alg. 2 (RBRP), Sec. 4, with the robust blockwise filtering remark
    (truncated local CPQR, tau_b = 1/b) and the blockwise greedy remark (RBGP)
  * Alg. 3 (interpolation matrix from L), Sec. 5.1, and the proposition there
    that RBRP is ID-revealing (W = X X_S^+ = L L1^{-1}); the remark on stable
    evaluation of L2 L1^{-1} (truncated SVD, clip 1e-12)
  * Eq. (5.1): the least-squares W = X X_S^+ for a given S.

Everything is FP64 (FP32 inputs are upcast exactly).  Library primitives
(matrix products, solve_triangular, SVD, lstsq) serve as single steps; there is
no blocking or fusion beyond what the algorithms state.

Readings of points where the paper is silent:
  R1  tau bounds the squared relative residual ||d||_1 / ||d0||_1 (the stopping
      test of Alg. 2).
  R2  "sample without replacement" is realised as an exponential race: keys
      kappa_i = -log(u_i) / d_i over eligible rows, the b_t smallest in
      ascending (kappa, i) order.  This is sequential sampling proportional to
      d without replacement (the Plackett-Luce law).  u_i comes from
      Philox4x64-10 with counter (i, t, 0, 0), key (seed, problem), t = the
      paper's 1-based block counter (oracle/philox.py).
  R3  tau_b defaults to 1/b_t where b_t = min(b, #eligible, k_cap - |S|) is the
      block actually drawn, so b_t = 1 gives b' = 1 (Alg. 1 behaviour).
  R4  b' = max{ i : ||R_V(i:b_t, i:b_t)||_F^2 >= tau_b ||R_V||_F^2 and the
      trailing mass is > 0 } (the truncation of Alg. 2, 1-based i; the "> 0" guard only
      matters for tau_b = 0 on rank-deficient blocks).
  R5  eligible rows are E = { i not in S : d_i > 0 }; accepted rows get d = 0
      and R(i,:) = 0 exactly; rejected candidates stay eligible.
  R6  the loop also stops when |S| reaches k_cap = min(n, dim, k_max) or when
      E is empty (termination guards the paper does not need in exact
      arithmetic).
  R7  the CPQR pivot is the remaining column with the largest recomputed
      trailing norm, ties to the smallest candidate position in S_t.
  R8  residual form (the GPU form): R starts as X; V = R(S_t,:)^T projected
      twice against Q (CGS2); the update applies R <- R - (R Q') Q'^T to the
      active rows and recomputes d_i = ||R(i,:)||^2.  form="downdate" follows
      the update step of Alg. 2 as printed (X read-only, d downdated).
"""
import numpy as np
import scipy.linalg as sla

from . import philox


# ---------------------------------------------------------------------------
# Alg. 2, initial norms: squared row norms
# ---------------------------------------------------------------------------
def row_sq_norms(X):
    """d_i = ||x_i||_2^2 for every row (Alg. 2, initial norms; Eq. (2.2) numerators)."""
    X = np.asarray(X, dtype=np.float64)
    return np.einsum("ij,ij->i", X, X)


# ---------------------------------------------------------------------------
# Alg. 2, sampling step: b_t rows ~ d / ||d||_1 without replacement (reading R2)
# ---------------------------------------------------------------------------
def race_keys(d, eligible, t, seed, problem=0):
    """Exponential-race keys kappa_i = -log(u_i)/d_i; +inf for ineligible rows."""
    n = d.shape[0]
    u = philox.uniforms(np.arange(n, dtype=np.uint64), t, seed, problem)
    kappa = np.full(n, np.inf)
    kappa[eligible] = -np.log(u[eligible]) / d[eligible]
    return kappa


def sample_block(d, eligible, b_t, t, seed, problem=0):
    """S_t: the b_t smallest race keys in ascending (kappa, row) order.

    Returns (S_t, gap) where gap is the relative gap between the b_t-th and
    (b_t+1)-th key (inf if there is no (b_t+1)-th eligible key); a GPU
    mismatch at a boundary whose gap is ~1e-12 or less is a rounding near-tie.
    """
    kappa = race_keys(d, eligible, t, seed, problem)
    order = np.lexsort((np.arange(d.shape[0]), kappa))
    S_t = order[:b_t].copy()
    gap = np.inf
    if b_t < int(eligible.sum()):
        a, c = kappa[order[b_t - 1]], kappa[order[b_t]]
        gap = (c - a) / c if c > 0 else np.inf
    return S_t, gap


def greedy_block(d, eligible, b_t):
    """RBGP/BGP: indices of the b_t largest d among eligible rows, descending, ties to smaller row.

    Returns (S_t, gap) with gap the relative gap between the b_t-th and (b_t+1)-th largest
    d (inf if there is no (b_t+1)-th eligible row), the boundary rounding can flip."""
    key = np.where(eligible, -d, np.inf)
    order = np.lexsort((np.arange(d.shape[0]), key))
    gap = np.inf
    if b_t < int(eligible.sum()):
        a, c = d[order[b_t - 1]], d[order[b_t]]
        gap = (a - c) / a if a > 0 else np.inf
    return order[:b_t].copy(), gap


# ---------------------------------------------------------------------------
# Alg. 2, local CPQR: column-pivoted Householder QR of V (d x b_t)
# ---------------------------------------------------------------------------
def cpqr(V):
    """V(:, piv) = Q_V R_V by Householder QR with column pivoting (reading R7).

    At step i the pivot is the remaining column whose trailing part A(i:, j)
    has the largest norm, recomputed from scratch.  Returns (Q_V (d x m, econ),
    R_V (m x m upper triangular), piv, min_gap) where min_gap is the smallest
    relative gap between the chosen and the runner-up trailing squared norm.
    """
    A = np.array(V, dtype=np.float64, copy=True)
    dim, m = A.shape
    if m > dim:
        raise ValueError("cpqr expects at most as many columns as rows")
    piv = np.arange(m)
    vs = []
    min_gap = np.inf
    for i in range(m):
        norms = np.einsum("ij,ij->j", A[i:, i:], A[i:, i:])
        best = norms.max()
        cands = np.nonzero(norms == best)[0]
        j = i + cands[np.argmin(piv[i + cands])]
        if m - i > 1 and best > 0:
            rest = np.delete(norms, j - i)
            min_gap = min(min_gap, (best - rest.max()) / best)
        if j != i:
            A[:, [i, j]] = A[:, [j, i]]
            piv[[i, j]] = piv[[j, i]]
        x = A[i:, i].copy()
        alpha = np.linalg.norm(x)
        v = x.copy()
        if alpha > 0:
            v[0] += np.copysign(alpha, x[0]) if x[0] != 0 else alpha
            vn = v @ v
            A[i:, i:] -= np.outer(v, (2.0 / vn) * (v @ A[i:, i:]))
        else:
            v[:] = 0.0
        vs.append(v)
    R = np.triu(A[:m, :m])
    Qv = np.eye(dim, m)
    for i in range(m - 1, -1, -1):
        v = vs[i]
        vn = v @ v
        if vn > 0:
            Qv[i:, :] -= np.outer(v, (2.0 / vn) * (v @ Qv[i:, :]))
    return Qv, R, piv, min_gap


def filter_rank(R_V, tau_b):
    """Truncation of Alg. 2: b' = max{ i : ||R_V(i:, i:)||_F^2 >= tau_b ||R_V||_F^2 } (reading R4)."""
    m = R_V.shape[0]
    total = float(np.sum(R_V * R_V))
    tails = np.array([np.sum(R_V[i:, i:] * R_V[i:, i:]) for i in range(m)])
    ok = (tails >= tau_b * total) & (tails > 0)
    idx = np.nonzero(ok)[0]
    return (int(idx[-1]) + 1 if idx.size else 0), tails


# ---------------------------------------------------------------------------
# Alg. 2: RBRP skeleton selection, organised by the method's steps
# ---------------------------------------------------------------------------
def project_out(V, Q, passes):
    """Projection step: remove from the columns of V their components in span(Q),
    V <- V - Q (Q^T V), `passes` times (two = CGS2; the second pass only repairs
    rounding, in exact arithmetic it changes nothing)."""
    for _ in range(passes):
        V = V - Q @ (Q.T @ V)
    return V


def truncation_gap(tails, bp, tb):
    """How far the truncation of the filter sits from its threshold tau_b ||R_V||_F^2,
    relative to ||R_V||_F^2 (smallest distance of the last kept and the first dropped
    tail mass); a near-tie there can flip b' under rounding.  Logged, not used."""
    thr = tb * tails[0]
    near = [abs(tails[bp - 1] - thr)] + ([abs(tails[bp] - thr)] if bp < len(tails) else [])
    return min(near) / tails[0] if tails[0] > 0 else np.inf


def rbrp(X, tau=None, b=16, seed=0, problem=0, k=None, k_max=None, tau_b=None,
         sampler="random", form="residual"):
    """Robust blockwise random pivoting (Alg. 2, Sec. 4).

    X: n x dim array (any real dtype; upcast to FP64).
    tau: tolerance on ||d||_1 / ||d0||_1 (reading R1); k: fixed-rank mode
    ("or k" in Alg. 2).  b: block size.  tau_b: filter tolerance (None -> 1/b_t,
    0 -> plain BRP).  sampler: "random" (RBRP/BRP) or "greedy" (RBGP/BGP).
    form: "residual" (R8) or "downdate" (Alg. 2's update step as printed).

    Returns a dict with S (acceptance order), L (n x k), Q (dim x k), d, D0, D,
    per-block records (t, b_t, b', sampling / CPQR / truncation gaps, D) and k_cap.
    """
    X = np.asarray(X, dtype=np.float64)
    n, dim = X.shape
    k_cap = min(n, dim)
    if k_max is not None and k_max > 0:
        k_cap = min(k_cap, int(k_max))
    if k is not None:
        k_cap = min(k_cap, int(k))
    if tau is None and k is None:
        raise ValueError("give tau or k")

    # Start: no skeletons, empty basis and coefficient matrix; the residual form
    # keeps its own copy R of X, and d holds the initial squared row norms.
    L = np.zeros((n, 0))
    Q = np.zeros((dim, 0))
    S = []
    in_S = np.zeros(n, dtype=bool)
    t = 0
    R = X.copy() if form == "residual" else None
    d = row_sq_norms(X)
    D0 = float(d.sum())
    blocks = []

    def keep_going():
        # stopping test (reading R1), with the guard of reading R6
        if len(S) >= k_cap:
            return False
        if k is not None:
            return True
        return float(d.sum()) > tau * D0

    while keep_going():
        eligible = (~in_S) & (d > 0)
        b_t = min(b, int(eligible.sum()), k_cap - len(S))
        if b_t <= 0:
            break
        t += 1

        # Sampling step: b_t candidate rows, drawn ~ d without replacement
        # (or the b_t largest d for the greedy variant).
        if sampler == "random":
            S_t, sgap = sample_block(d, eligible, b_t, t, seed, problem)
        else:
            S_t, sgap = greedy_block(d, eligible, b_t)

        # Projection step: the candidates' rows with span(Q) taken out.  The
        # residual rows already are orthogonal to Q (up to rounding), so two
        # cheap passes suffice; the printed form projects the rows of X once.
        if form == "residual":
            V = project_out(R[S_t].T.copy(), Q, 2)
        else:
            V = X[S_t].T - Q @ (Q.T @ X[S_t].T)

        # Local CPQR of the projected candidates and the robust truncation:
        # keep the leading b' pivots whose trailing mass stays above tau_b.
        QV, RV, piv, qgap = cpqr(V)
        tb = (1.0 / b_t) if tau_b is None else float(tau_b)
        bp, tails = filter_rank(RV, tb)
        if bp == 0:
            break
        fgap = truncation_gap(tails, bp, tb)

        # Acceptance: the first b' pivots become skeletons (in pivot order) and
        # their orthonormal directions extend the basis.
        Sp_t = S_t[piv[:bp]]
        Qp = QV[:, :bp]
        Q = np.concatenate([Q, Qp], axis=1)

        # Update step: coefficients of every row not yet a skeleton along the
        # new directions (rows accepted earlier have a zero residual and keep
        # zero coefficients), appended to L.
        active = ~in_S
        Lhat = np.zeros((n, bp))
        if form == "residual":
            Lhat[active] = R[active] @ Qp
        else:
            Lhat[active] = X[active] @ Qp
        S.extend(int(s) for s in Sp_t)
        in_S[Sp_t] = True
        L = np.concatenate([L, Lhat], axis=1)

        # New squared residual norms: recomputed from the updated residual
        # (residual form) or downdated by the new coefficients (printed form);
        # skeletons have none left.
        if form == "residual":
            R[active] -= Lhat[active] @ Qp.T
            R[Sp_t] = 0.0
            d = row_sq_norms(R)
        else:
            d = d - np.einsum("ij,ij->i", Lhat, Lhat)
        d[in_S] = 0.0
        blocks.append(dict(t=t, b_t=b_t, bp=bp, sample_gap=float(sgap), cpqr_gap=float(qgap),
                           filter_gap=float(fgap), D=float(d.sum())))

    return dict(S=np.array(S, dtype=np.int64), L=L, Q=Q, d=d, D0=D0, D=float(d.sum()),
                blocks=blocks, k_cap=k_cap, R=R)


# ---------------------------------------------------------------------------
# Alg. 1: sequential random pivoting, as printed (X read-only, d downdated)
# ---------------------------------------------------------------------------
def srp(X, tau=None, seed=0, problem=0, k=None):
    """Alg. 1 (SRP) with rank-1 updates; sampler as in reading R2 with one draw per step.

    The comparison '<' in the printed while-condition is read as '>' (the
    Alg. 2 condition), which is what makes the loop run.
    """
    X = np.asarray(X, dtype=np.float64)
    n, dim = X.shape
    k_cap = min(n, dim) if k is None else min(n, dim, int(k))
    Q = np.zeros((dim, 0))
    Lcols = []
    S = []
    in_S = np.zeros(n, dtype=bool)
    d = row_sq_norms(X)
    D0 = float(d.sum())
    t = 0
    while len(S) < k_cap and (k is not None or float(d.sum()) > tau * D0):
        eligible = (~in_S) & (d > 0)
        if not eligible.any():
            break
        t += 1
        kappa = race_keys(d, eligible, t, seed, problem)
        s = int(np.lexsort((np.arange(n), kappa))[0])
        S.append(s)
        in_S[s] = True
        v = X[s] - Q @ (Q.T @ X[s])
        Q = np.concatenate([Q, (v / np.linalg.norm(v))[:, None]], axis=1)
        active = ~in_S
        active[s] = True
        a = np.zeros(n)
        a[active] = X[active] @ v
        Lcols.append(a / np.sqrt(a[s]))
        d = d - a * a / a[s]
        d[in_S] = 0.0
    L = np.stack(Lcols, axis=1) if Lcols else np.zeros((n, 0))
    return dict(S=np.array(S, dtype=np.int64), L=L, Q=Q, d=d, D0=D0, D=float(d.sum()))


# ---------------------------------------------------------------------------
# Alg. 3 and the W alternatives of Sec. 5
# ---------------------------------------------------------------------------
def interp_matrix(L, S):
    """Alg. 3: W(S,:) = I_k, W(rest,:) = L2 L1^{-1} by triangular substitution.

    L1 = L(S,:) is lower triangular when S is in acceptance order (Sec. 5.1,
    the ID-revealing proposition and the remark after it); W L1 = L2 is solved
    as L1^T W^T = L2^T.
    """
    n, k = L.shape
    S = np.asarray(S, dtype=np.int64)
    W = np.zeros((n, k))
    if k == 0:
        return W
    rest = np.setdiff1d(np.arange(n), S)
    L1 = L[S]
    W[S] = np.eye(k)
    if rest.size:
        W[rest] = sla.solve_triangular(L1.T, L[rest].T, lower=False).T
    return W


def interp_matrix_tsvd(L, S, clip=1e-12):
    """Remark on stable evaluation of L2 L1^{-1}: pseudo-inverse of L1 by truncated SVD.

    Singular values below clip * sigma_max(L1) are dropped (the paper's clip
    is read as relative to the largest singular value).
    """
    n, k = L.shape
    S = np.asarray(S, dtype=np.int64)
    W = np.zeros((n, k))
    if k == 0:
        return W
    U, s, Vt = np.linalg.svd(L[S])
    keep = s > clip * s[0]
    L1_pinv = (Vt[keep].T / s[keep]) @ U[:, keep].T
    rest = np.setdiff1d(np.arange(n), S)
    W[S] = np.eye(k)
    W[rest] = L[rest] @ L1_pinv
    return W


def interp_matrix_ls(X, S):
    """Eq. (5.1): the optimal W = X X_S^+ for the given skeletons (least squares)."""
    X = np.asarray(X, dtype=np.float64)
    XS = X[np.asarray(S, dtype=np.int64)]
    if XS.shape[0] == 0:
        return np.zeros((X.shape[0], 0))
    sol, *_ = np.linalg.lstsq(XS.T, X.T, rcond=None)
    return sol.T


def id_error_sq(X, S, W):
    """Interpolation error ||X - W X_S||_F^2 / ||X||_F^2 (Sec. 1, normalised as in Sec. 6)."""
    X = np.asarray(X, dtype=np.float64)
    S = np.asarray(S, dtype=np.int64)
    E = X - W @ X[S]
    nx = float(np.sum(X * X))
    return float(np.sum(E * E)) / nx if nx > 0 else 0.0


def skeleton_error_sq(X, S):
    """E_X(S) / ||X||_F^2 with E_X(S) = ||X - X X_S^+ X_S||_F^2 (Eq. (1.2))."""
    return id_error_sq(X, S, interp_matrix_ls(X, S))


def rbrp_id(X, tau=None, b=16, seed=0, problem=0, k=None, k_max=None, tau_b=None,
            sampler="random", form="residual"):
    """Full ID: Alg. 2 then Alg. 3.  Returns the rbrp() dict plus W, rel_err_sq (= D/D0)."""
    out = rbrp(X, tau=tau, b=b, seed=seed, problem=problem, k=k, k_max=k_max, tau_b=tau_b,
               sampler=sampler, form=form)
    out["W"] = interp_matrix(out["L"], out["S"])
    out["rel_err_sq"] = out["D"] / out["D0"] if out["D0"] > 0 else 0.0
    return out

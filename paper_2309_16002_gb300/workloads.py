"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data; it holds none of RBRP's arithmetic and imports
neither the CUDA binding nor the oracle, so the tests, the benchmark and the
oracle all take their inputs from here.  Every generator uses numpy's PCG64
with an explicit seed.

Workloads (sizes are parameters so the tests can draw small matrices with the
same structure):
  spectral      X = U diag(sigma) V^T with Haar-orthonormal U, V (QR of a
                seeded Gaussian, signs fixed by diag(R)); sigma_i = 0.9^i
                (2000 x 200, FP64) or sigma_i = i^-1.5 (200000 x 2000, FP32,
                U assembled from stacked Haar blocks)
  zipf_gmm      near-duplicate clusters: 100 N(0, I) centres with Zipf(1.5)
                cluster sizes, each row = centre + N(0, 1e-6 I), plus 5% extra
                rows of N(0, 0.01 I); 100000 x 1000 FP32.  Rows are shuffled.
  kernel_blocks Gaussian-kernel blocks exp(-|x - y|^2 / h^2), h = 0.5, between
                m and n uniform points in two unit cubes of R^3 whose gap is 2;
                m ~ U[64, 2048], n ~ U[32, 256]; FP32
  random_features  ReLU(G z) / sqrt(512) with G a 512 x 64 Gaussian and z from a
                20-component GMM in R^64 (means N(0, 4I), identity covariance);
                1000000 x 512 FP32
  example_2_1   the adversarial input for squared-norm sampling of Sec. 2.2
                (scaled canonical directions, each repeated n/k times)
  gmm_pitfall   the adversarial GMM of Sec. 4 (means 10 j e_j, covariance I,
                n/k points per cluster)
  low_rank      an exactly rank-r Gaussian product
  gaussian_embedding  the d x l N(0, 1/l) embedding of sketchy pivoting
"""
import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def haar(rng, n, m):
    """n x m matrix with orthonormal columns: QR of a Gaussian, signs fixed by diag(R)."""
    A = rng.standard_normal((n, m))
    Qm, Rm = np.linalg.qr(A)
    s = np.sign(np.diag(Rm))
    s[s == 0] = 1.0
    return Qm * s


def spectral(n=2000, d=200, decay="geometric", rate=0.9, seed=1, dtype=np.float64, haar_block=None):
    """X = U diag(sigma) V^T.

    decay="geometric": sigma_i = rate^i (i = 1..min(n, d)); decay="power":
    sigma_i = i^-rate.  haar_block: when set, U is the stack of n/haar_block
    Haar blocks (haar_block x r each) scaled by sqrt(haar_block/n), which keeps
    U^T U = I while avoiding one huge QR.  Returns (X, sigma).
    """
    rng = _rng(seed)
    r = min(n, d)
    i = np.arange(1, r + 1, dtype=np.float64)
    sigma = rate ** i if decay == "geometric" else i ** (-rate)
    if haar_block is None:
        U = haar(rng, n, r)
    else:
        if n % haar_block or haar_block < r:
            raise ValueError("haar_block must divide n and be >= min(n, d)")
        nb = n // haar_block
        U = np.concatenate([haar(rng, haar_block, r) for _ in range(nb)], axis=0) / np.sqrt(nb)
    V = haar(rng, d, r)
    X = (U * sigma) @ V.T
    return X.astype(dtype), sigma


def zipf_sizes(total, clusters, s=1.5):
    """Cluster sizes proportional to j^-s (j = 1..clusters), largest-remainder rounding to `total`."""
    w = np.arange(1, clusters + 1, dtype=np.float64) ** (-s)
    raw = total * w / w.sum()
    base = np.floor(raw).astype(np.int64)
    short = int(total - base.sum())
    order = np.argsort(-(raw - base), kind="stable")
    base[order[:short]] += 1
    return base


def zipf_gmm(n=100000, d=1000, clusters=100, extra_frac=0.05, centre_std=1.0,
             within_var=1e-6, extra_var=0.01, s=1.5, seed=2, dtype=np.float32):
    """Near-duplicate Zipf GMM: n rows = (1 - extra_frac) n cluster rows + extra_frac n noise rows."""
    rng = _rng(seed)
    n_extra = int(round(extra_frac * n))
    n_clu = n - n_extra
    sizes = zipf_sizes(n_clu, clusters, s)
    centres = centre_std * rng.standard_normal((clusters, d))
    labels = np.repeat(np.arange(clusters), sizes)
    X = np.empty((n, d), dtype=np.float64)
    X[:n_clu] = centres[labels] + np.sqrt(within_var) * rng.standard_normal((n_clu, d))
    X[n_clu:] = np.sqrt(extra_var) * rng.standard_normal((n_extra, d))
    perm = rng.permutation(n)
    return np.ascontiguousarray(X[perm].astype(dtype))


def kernel_block(rng, m, n, h=0.5, gap=2.0, dtype=np.float32):
    """One m x n Gaussian-kernel block between points in [0,1]^3 and [1+gap, 2+gap] x [0,1]^2."""
    x = rng.random((m, 3))
    y = rng.random((n, 3))
    y[:, 0] += 1.0 + gap
    r2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    return np.exp(-r2 / (h * h)).astype(dtype)


def kernel_block_sizes(P=4096, m_range=(64, 2048), n_range=(32, 256), seed=4):
    """Shapes (m_p, n_p) of P kernel blocks: m ~ U[m_range], n ~ U[n_range] (inclusive integers)."""
    rng = _rng(seed)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=P)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=P)
    return [(int(m), int(n)) for m, n in zip(ms, ns)]


def kernel_blocks(P=4096, m_range=(64, 2048), n_range=(32, 256), h=0.5, gap=2.0, seed=4, dtype=np.float32,
                  lo=0, hi=None):
    """Kernel blocks lo..hi-1 of a list of P (shapes from kernel_block_sizes).

    Block p draws its points from its own generator (seed, p), so any slice of
    the list can be drawn without drawing the rest.
    """
    sizes = kernel_block_sizes(P, m_range, n_range, seed)
    hi = P if hi is None else hi
    return [kernel_block(np.random.Generator(np.random.PCG64([seed, p])), m, n, h, gap, dtype)
            for p, (m, n) in enumerate(sizes[lo:hi], start=lo)]


def random_features(n=1000000, d=512, latent=64, comps=20, mean_var=4.0, seed=5, dtype=np.float32,
                    chunk=200000):
    """ReLU(G z) / sqrt(d), G d x latent Gaussian, z from a comps-component GMM in R^latent."""
    rng = _rng(seed)
    G = rng.standard_normal((d, latent))
    means = np.sqrt(mean_var) * rng.standard_normal((comps, latent))
    X = np.empty((n, d), dtype=dtype)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        lab = rng.integers(0, comps, size=b - a)
        z = means[lab] + rng.standard_normal((b - a, latent))
        X[a:b] = (np.maximum(z @ G.T, 0.0) / np.sqrt(d)).astype(dtype)
    return X


def example_2_1(n=24, k=6, r=2, alpha=1e4, dim=None, dtype=np.float64):
    """Adversarial input of Sec. 2.2: rows alpha_i e_i, each repeated n/k times.

    alpha_i = sqrt(alpha) for i <= r and 1 for r < i <= k; dim defaults to k.
    Returns X (n x dim), rows grouped by direction.
    """
    if n % k:
        raise ValueError("k must divide n")
    dim = k if dim is None else dim
    a = np.ones(k)
    a[:r] = np.sqrt(alpha)
    X = np.zeros((n, dim))
    m = n // k
    for i in range(k):
        X[i * m:(i + 1) * m, i] = a[i]
    return X.astype(dtype)


def gmm_pitfall(n=2000, d=500, k=100, seed=6, dtype=np.float64):
    """Adversarial GMM of Sec. 4: cluster j has n/k points mu_j + N(0, I_d), mu_j = 10 j e_j."""
    if n % k or k > d:
        raise ValueError("need k | n and k <= d")
    rng = _rng(seed)
    m = n // k
    X = rng.standard_normal((n, d))
    for j in range(k):
        X[j * m:(j + 1) * m, j] += 10.0 * (j + 1)
    return X.astype(dtype)


def gaussian_embedding(d, l, seed=11, dtype=np.float64):
    """Gaussian embedding Omega (d x l) with i.i.d. N(0, 1/l) entries, the random input of
    sketchy pivoting (drawn here so that the GPU path and the oracle use the same one)."""
    rng = _rng(seed)
    return (rng.standard_normal((d, l)) / np.sqrt(l)).astype(dtype)


def low_rank(n=500, d=100, r=20, seed=7, dtype=np.float64):
    """Exactly rank-r n x d Gaussian product."""
    rng = _rng(seed)
    return (rng.standard_normal((n, r)) @ rng.standard_normal((r, d))).astype(dtype)

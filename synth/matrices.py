"""Test matrices A = Q1 diag(sigma) Q2^T with prescribed singular values.

Q1, Q2 are Haar-distributed: the Q factor of a seeded Gaussian matrix with
the signs of diag(R) made positive (Section 6.2 builds its test matrices from
random orthonormal factors the same way).  Large sizes may be built with
torch on a CUDA device; this is input generation, not part of the method.
"""
import numpy as np

SPECTRA = ("exp200", "exp50", "exp500", "exp40", "inv", "fastdecay", "gap", "gauss", "lowrank")


def spectrum(kind, n, r=None):
    """Singular values sigma_j, j = 1..n (descending) for a named spectrum.

    exp<L>     sigma_j = exp(-j/L)   (L = 50, 200, 500, 40, or ``r``)
    inv        sigma_j = 1/j
    fastdecay  sigma_j = beta^((j-1)/(n-1)), beta = 1e-5   (Section 6.2, Matrix 1)
    gap        1/j for j <= 150, 0.1/j for j > 150          (Section 6.2, Matrix 3)
    lowrank    sigma_j = exp(-j/10) for j <= r, 0 beyond
    """
    j = np.arange(1, n + 1, dtype=np.float64)
    if kind.startswith("exp") and kind[3:].isdigit():
        return np.exp(-j / float(kind[3:]))
    if kind == "exp":
        return np.exp(-j / float(r))
    if kind == "inv":
        return 1.0 / j
    if kind == "fastdecay":
        return 1e-5 ** ((j - 1) / max(n - 1, 1))
    if kind == "gap":
        return np.where(j <= 150, 1.0 / j, 0.1 / j)
    if kind == "lowrank":
        return np.where(j <= r, np.exp(-j / 10.0), 0.0)
    raise ValueError(f"unknown spectrum {kind!r}")


def _haar_from(z):
    q, r = np.linalg.qr(z)
    return q * np.where(np.diag(r) < 0, -1.0, 1.0)[None, :]


def _haar_numpy(rng, n):
    return _haar_from(rng.standard_normal((n, n)))


def haar_orthogonal(n, seed, device=None):
    """n x n Haar orthogonal matrix from a seeded Gaussian (numpy Generator PCG64).

    With ``device`` a torch CUDA device the QR runs there (float64) and a
    torch tensor is returned; otherwise a numpy array."""
    rng = np.random.default_rng(seed)
    if device is None:
        return _haar_numpy(rng, n)
    import torch
    z = rng.standard_normal((n, n))
    try:
        zt = torch.from_numpy(z).to(device)
        q, r = torch.linalg.qr(zt)
    except RuntimeError:
        # torch's linear-algebra library can be unavailable (e.g. under a
        # profiler that intercepts its loading): build Q on the host instead
        return torch.from_numpy(_haar_from(z)).to(device)
    s = torch.where(torch.diagonal(r) < 0, -1.0, 1.0).to(q.dtype)
    return q * s[None, :]


def make_matrix(kind, m, n, seed, device=None, r=None):
    """m x n float64 test matrix (numpy, or torch on ``device``).

    kind is a spectrum name (see ``spectrum``) or "gauss" for iid N(0,1) entries.
    Seeds: Q1 from ``seed``, Q2 from ``seed + 1``, gauss entries from ``seed``.
    """
    if kind == "gauss":
        a = np.random.default_rng(seed).standard_normal((m, n))
        if device is None:
            return a
        import torch
        return torch.from_numpy(a).to(device)
    p = min(m, n)
    s = spectrum(kind, p, r)
    if device is None:
        q1 = _haar_numpy(np.random.default_rng(seed), m)[:, :p]
        q2 = _haar_numpy(np.random.default_rng(seed + 1), n)[:, :p]
        return (q1 * s[None, :]) @ q2.T
    import torch
    q1 = haar_orthogonal(m, seed, device)[:, :p]
    q2 = haar_orthogonal(n, seed + 1, device)[:, :p]
    st = torch.from_numpy(s).to(q1.device)
    return (q1 * st[None, :]) @ q2.T

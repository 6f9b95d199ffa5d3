"""Per-entry bounds for comparing |diag T| of two randUTV factorizations.

A diagonal entry d_j of T is fixed by the rounding of a backward-stable
factorization only to the extent the method allows: rounding errors act like
a perturbation E of A of the size of the backward error, and entry j moves by
its sensitivity to such a perturbation.  So an entry is held to the relative
bar (rel |d_ref_j|) where that bar exceeds c times its measured sensitivity
s_j, and to c s_j where it does not:

    |d_j - d_ref_j| <= max(rel |d_ref_j|, c s_j).

s_j is measured, not modelled: the spread of the reference implementation's
own d_j over a few random perturbations A + E_k with ||E_k||_2 = eps ||A||_2
(eps the backward error in question), taken as the largest change over the
draws and over the neighbouring entries j-w .. j+w (so an entry whose change
happens to be small in every draw does not get a bound below its neighbours').
The comparison reports how many entries were held to the pure relative bar.
"""
import numpy as np


def norm2(X, iters=60, seed=5):
    """||X||_2 by power iteration on X^T X (a few parts in 1e4 suffice for scaling)."""
    v = np.random.default_rng(seed).standard_normal(X.shape[1])
    for _ in range(iters):
        w = X.T @ (X @ v)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        v = w / nw
    return float(np.linalg.norm(X @ v))


def perturbations(shape, normA2, eps, seeds):
    """Gaussian matrices E_k scaled to ||E_k||_2 = eps ||A||_2 (numpy, host)."""
    out = []
    for sd in seeds:
        E = np.random.default_rng(sd).standard_normal(shape)
        out.append(E * (eps * normA2 / norm2(E)))
    return out


def sensitivity(d0, dps, window=4):
    """s_j = max over the draws k and over |i - j| <= window of |dps_k,i - d0_i|."""
    d0 = np.abs(np.asarray(d0, dtype=np.float64))
    spread = np.max(np.abs(np.abs(np.asarray(dps, dtype=np.float64)) - d0[None, :]), axis=0)
    n = len(spread)
    s = np.empty(n)
    for j in range(n):
        s[j] = spread[max(0, j - window):min(n, j + window + 1)].max()
    return s


def compare(d, dref, s, rel, c):
    """Check |d - dref| <= max(rel |dref|, c s) entry by entry.

    Returns a dict: ok, ratio (largest |d - dref| / bound), n, n_rel (entries
    whose bound is the relative bar), max_rel_on_rel (largest relative
    difference over those entries), max_abs (largest |d - dref|)."""
    d = np.abs(np.asarray(d, dtype=np.float64))
    dref = np.abs(np.asarray(dref, dtype=np.float64))
    k = min(len(d), len(dref), len(s))
    d, dref, s = d[:k], dref[:k], np.asarray(s)[:k]
    diff = np.abs(d - dref)
    relbar = rel * dref
    bound = np.maximum(relbar, c * s)
    bound = np.maximum(bound, np.finfo(np.float64).tiny)
    on_rel = relbar >= c * s
    ratio = float(np.max(diff / bound)) if k else 0.0
    mr = float(np.max(diff[on_rel] / dref[on_rel])) if np.any(on_rel) else 0.0
    return {"ok": ratio <= 1.0, "ratio": ratio, "n": int(k), "n_rel": int(on_rel.sum()), "max_rel_on_rel": mr,
            "max_abs": float(diff.max()) if k else 0.0}

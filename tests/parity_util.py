"""Oracle-side parts of the |diag T| parity checks (tests only).

``oracle_sensitivity`` measures how far the oracle's own diagonal moves when
A is perturbed by random matrices of norm eps ||A||_2 (the same Gaussian
matrices for the same seeds); ``check_fp64_diag`` compares a GPU diagonal
with the oracle's entry by entry under max(1e-10 |d_ref|, c s_j), with eps
the two sides' measured backward errors added (both are backward stable, so
each result is the exact factorization of a nearby matrix)."""
import numpy as np
import oracle
from oracle import checks
from diag_bound import norm2, perturbations, sensitivity, compare

U64 = 2.0 ** -53


def oracle_sensitivity(A, b, q, gauss, eps, draws=2, seed=4242, window=4, **kw):
    d0 = np.diag(oracle.randutv(A, b, q, gauss, form_uv=False, **kw)[1])
    nA = norm2(A)
    dps = []
    for E in perturbations(A.shape, nA, eps, [seed + i for i in range(draws)]):
        _, Tp, _, kp = oracle.randutv(A + E, b, q, gauss, form_uv=False, **kw)
        dps.append(np.diag(Tp))
    k = min(len(d0), *(len(x) for x in dps))
    return sensitivity(d0[:k], [x[:k] for x in dps], window=window)


def oracle_backward_error(A, b, q, gauss, **kw):
    """Residual ||A - U T V^T||_F / ||A||_F of the oracle's own factorization and its T."""
    U, T, V, k = oracle.randutv(A, b, q, gauss, **kw)
    return checks.residual(A, U, T, V), T, k


def check_fp64_diag(A, T_gpu, res_gpu, b, q, gauss, c=4.0, rel=1e-10, To=None, res_oracle=None, **kw):
    """|diag T_gpu| against the oracle's under max(rel |d_ref|, c s_j); returns the comparison
    dict (ok, ratio, n, n_rel, max_rel_on_rel, max_abs) plus eps."""
    if To is None or res_oracle is None:
        res_oracle, To, _ = oracle_backward_error(A, b, q, gauss, **kw)
    eps = max(res_gpu + res_oracle, 4 * U64)
    s = oracle_sensitivity(A, b, q, gauss, eps, **kw)
    r = compare(np.diag(T_gpu), np.diag(To), s, rel, c)
    r["eps"] = eps
    return r


def gpu_norm2(X, iters=60, seed=5):
    """||X||_2 of a CUDA tensor by power iteration."""
    import torch
    g = torch.Generator(device=X.device).manual_seed(seed)
    v = torch.randn(X.shape[1], dtype=X.dtype, device=X.device, generator=g)
    for _ in range(iters):
        w = X.T @ (X @ v)
        nw = torch.linalg.norm(w)
        if float(nw) == 0.0:
            return 0.0
        v = w / nw
    return float(torch.linalg.norm(X @ v))


def fp64_gpu_sensitivity(R, A64, b, q, eps, draws=2, seed=4242, window=4, **kw):
    """Sensitivity of the FP64 GPU path's |diag T| (A64 an FP64 CUDA tensor) to random
    perturbations of norm eps ||A||_2; returns (d0, s)."""
    import torch
    d0 = torch.diagonal(R.factor(A64, b=b, q=q, form_uv=False, **kw).T).cpu().numpy().copy()
    nA = gpu_norm2(A64)
    dps = []
    for i in range(draws):
        g = torch.Generator(device=A64.device).manual_seed(seed + i)
        E = torch.randn(A64.shape, dtype=torch.float64, device=A64.device, generator=g)
        E *= eps * nA / gpu_norm2(E)
        f = R.factor(A64 + E, b=b, q=q, form_uv=False, **kw)
        dps.append(torch.diagonal(f.T).cpu().numpy().copy())
        del f, E
    return d0, sensitivity(d0, dps, window=window)


def mixed_residual_orth(A32, U, T, V):
    """FP64 residual ||A - U T V^T||_F / ||A||_F against the stored FP32 A and max |X^T X - I|."""
    import torch
    A64 = A32.to(torch.float64)
    U64, V64 = U.to(torch.float64), V.to(torch.float64)
    P = torch.addmm(A64, U64 @ T.to(torch.float64), V64.T, alpha=-1.0)
    res = float(torch.linalg.norm(P) / torch.linalg.norm(A64))
    del P, A64
    eye = torch.eye(U64.shape[1], dtype=torch.float64, device=U64.device)
    ou = float((U64.T @ U64 - eye).abs().max())
    eye = torch.eye(V64.shape[1], dtype=torch.float64, device=V64.device)
    ov = float((V64.T @ V64 - eye).abs().max())
    return res, ou, ov


def check_mixed_diag(R, A32, T32, res_mixed, b, q, c=4.0, rel=1e-4, **kw):
    """|diag T| of the mixed form against the FP64 GPU path on the same FP32 A (up-cast) and the
    same G, under max(rel |d_64|, c s_j), s_j the FP64 path's sensitivity at the mixed form's
    backward error."""
    import torch
    A64 = A32.to(torch.float64)
    d64, s = fp64_gpu_sensitivity(R, A64, b, q, res_mixed, **kw)
    dm = torch.diagonal(T32).double().cpu().numpy()
    r = compare(dm, d64, s, rel, c)
    big = np.abs(d64) >= 1e-3 * np.abs(d64).max()
    r["max_rel_above_1e-3"] = float(np.max(np.abs(np.abs(dm[big]) - np.abs(d64[big])) / np.abs(d64[big])))
    r["n_above_1e-3"] = int(big.sum())
    r["eps"] = res_mixed
    return r

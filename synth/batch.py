"""Batches of small test matrices and their Gaussian streams (batched form).

The batched workload: ``count`` matrices with m, n drawn independently and
uniformly from the integers [lo, hi] (both m >= n and m < n occur), each
A_i = Q1 diag(sigma) Q2^T with sigma_j = exp(-j / r_i), r_i uniform in
[4, 64], Haar factors Q1 (m x m), Q2 (n x n), stored in FP32.  Sizes and
decay rates come from a numpy PCG64 generator seeded with ``seed``.

Small batches are built with numpy (each matrix from ``make_matrix`` with
seed ``seed + 2 i``); large ones on a CUDA device with torch (batched QR of
seeded Gaussian matrices grouped by size).  This is input generation only.
"""
import numpy as np

from .gauss import step_gaussian_f32
from .matrices import make_matrix


def batch_dims(count, seed, lo=64, hi=512):
    """(m, n, r): int32 arrays of sizes and float64 decay rates."""
    rng = np.random.default_rng(seed)
    m = rng.integers(lo, hi + 1, count).astype(np.int32)
    n = rng.integers(lo, hi + 1, count).astype(np.int32)
    r = rng.uniform(4.0, 64.0, count)
    return m, n, r


def batch_matrices(m, n, r, seed):
    """List of FP32 numpy matrices (small batches)."""
    return [make_matrix("exp", int(mi), int(ni), seed + 2 * i, r=float(ri)).astype(np.float32)
            for i, (mi, ni, ri) in enumerate(zip(m, n, r))]


def pack(mats, dtype=np.float32):
    """Concatenate column-major copies of the matrices (the packed layout)."""
    if not mats:
        return np.zeros(0, dtype=dtype)
    return np.concatenate([np.asarray(a, dtype=dtype).ravel(order="F") for a in mats])


def batch_matrices_torch(m, n, r, seed, device):
    """Packed FP32 torch tensor of the batch, built on ``device``: the Haar
    factors of all matrices of one size come from one batched FP32 QR of
    Gaussian matrices (a torch generator seeded with ``seed``, sizes in
    ascending order, Q1's before Q2's), then A = (Q1[:, :p] * sigma) Q2[:, :p]^T
    in FP64, rounded to FP32."""
    import torch
    count = len(m)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    factors = []
    for dims in (np.asarray(m), np.asarray(n)):
        qs = [None] * count
        for sz in np.unique(dims):
            idx = np.nonzero(dims == sz)[0]
            Z = torch.randn((len(idx), int(sz), int(sz)), generator=gen, dtype=torch.float32, device=device)
            try:
                Q, R = torch.linalg.qr(Z)
            except RuntimeError:
                # torch's linear-algebra library can be unavailable (e.g. under
                # a profiler that intercepts its loading): QR on the host
                q_, r_ = np.linalg.qr(Z.cpu().numpy().astype(np.float64))
                Q = torch.from_numpy(q_.astype(np.float32)).to(device)
                R = torch.from_numpy(r_.astype(np.float32)).to(device)
            Q = Q * torch.where(torch.diagonal(R, dim1=1, dim2=2) < 0, -1.0, 1.0)[:, None, :]
            for j, i in enumerate(idx):
                qs[i] = Q[j]
            del Z, R
        factors.append(qs)
    Q1s, Q2s = factors
    out = torch.empty(sum(int(a) * int(b) for a, b in zip(m, n)), dtype=torch.float32, device=device)
    pos = 0
    for i in range(count):
        mi, ni, ri = int(m[i]), int(n[i]), float(r[i])
        p = min(mi, ni)
        sig = torch.exp(-torch.arange(1, p + 1, dtype=torch.float64, device=device) / ri)
        A = (Q1s[i][:, :p].double() * sig[None, :]) @ Q2s[i][:, :p].double().T
        out[pos:pos + mi * ni] = A.t().reshape(-1).to(torch.float32)
        pos += mi * ni
    return out


def batched_gaussian_stream(seed, m, n, b):
    """(stream, offsets): every matrix's G of every step b s < min(m, n),
    concatenated per matrix in step order, each column-major, FP32."""
    parts, offs, pos = [], [], 0
    for i, (mi, ni, bi) in enumerate(zip(m, n, b)):
        mi, ni, bi = int(mi), int(ni), int(bi)
        offs.append(pos)
        s = 1
        while bi * s < min(mi, ni):
            k = mi - bi * (s - 1)
            g = step_gaussian_f32(seed, s, k, bi, index=i)
            parts.append(g.ravel(order="F"))
            pos += k * bi
            s += 1
    stream = np.concatenate(parts) if parts else np.zeros(0, dtype=np.float32)
    return stream.astype(np.float32), np.asarray(offs, dtype=np.int64)

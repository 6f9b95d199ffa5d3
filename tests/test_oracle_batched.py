"""The batched oracle and the batched input generators, on CPU.

Pins: each matrix of a batch is an independent problem (the batch result
equals the single-matrix oracle on the same G); the early stop lands where
the spectrum puts it (Eckart-Young: ||T22||_F >= the optimal tail, so the
stop is never before the optimal rank for the tolerance, and with q = 1 on
these spectra it is at most one block after it); rectangular batches keep
A = U T V^T with orthogonal U, V and T upper triangular on its finished
columns; the FP32 Gaussian definition agrees with the FP64 one built from the
same words to the rounding of the coarser uniforms; the packed offsets
follow the documented layout."""
import numpy as np
import pytest
import synth
import oracle
from oracle import checks

SEED = 998


def _gauss(i, s, k, w):
    return synth.step_gaussian_f32(SEED, s, k, w, index=i).astype(np.float64)


def _tail(s, k):
    return float(np.sqrt(np.sum(s[k:] ** 2)))


@pytest.fixture(scope="module")
def small_batch():
    m = np.array([80, 64, 130, 97, 64, 150], dtype=np.int32)
    n = np.array([64, 120, 130, 64, 64, 70], dtype=np.int32)
    r = np.array([6.0, 12.0, 4.0, 30.0, 64.0, 9.0])
    return m, n, r, synth.batch.batch_matrices(m, n, r, 31)


@pytest.mark.parametrize("b", [16, 32])
def test_batch_is_independent_problems(small_batch, b):
    m, n, r, As = small_batch
    A64 = [a.astype(np.float64) for a in As]
    res = oracle.randutv_batched(A64, [b] * len(As), 1, _gauss, tol=1e-5)
    for i, (A, (U, T, V, k)) in enumerate(zip(A64, res)):
        U1, T1, V1, k1 = oracle.randutv(A, b, 1, lambda s, kk, w: _gauss(i, s, kk, w), tol=1e-5)
        assert k == k1
        np.testing.assert_array_equal(T, T1)


@pytest.mark.parametrize("b", [16, 32])
def test_early_stop_against_spectrum(small_batch, b):
    m, n, r, As = small_batch
    tol = 1e-5
    res = oracle.randutv_batched([a.astype(np.float64) for a in As], [b] * len(As), 1, _gauss, tol=tol)
    for A, (U, T, V, k) in zip(As, res):
        A = A.astype(np.float64)
        s = np.linalg.svd(A, compute_uv=False)
        nA = np.linalg.norm(A)
        kopt = next((j for j in range(len(s) + 1) if _tail(s, j) <= tol * nA), len(s))
        p = min(A.shape)
        assert k == p or k % b == 0
        assert np.linalg.norm(T[k:, k:]) <= tol * nA or k == p
        assert k >= min(kopt, p)
        assert k <= min(p, (kopt + b - 1) // b * b + b)
        assert checks.residual(A, U, T, V) < 1e-13
        assert checks.orth_err(U) < 1e-13 and checks.orth_err(V) < 1e-13
        assert checks.lower_max(T[:, :k]) == 0.0
        # the diagonal reveals the leading singular values (Section 1.1 (i))
        d = np.abs(np.diag(T))[:min(k, 4)]
        np.testing.assert_allclose(d, s[:len(d)], rtol=0.1)


def test_full_factorization_of_rectangular_batch(small_batch):
    m, n, r, As = small_batch
    res = oracle.randutv_batched([a.astype(np.float64) for a in As], [16] * len(As), 1, _gauss, tol=0.0)
    for A, (U, T, V, k) in zip(As, res):
        A = A.astype(np.float64)
        assert k == min(A.shape)
        assert checks.residual(A, U, T, V) < 1e-13
        assert checks.lower_max(T) == 0.0
        s = np.linalg.svd(A, compute_uv=False)
        assert abs(np.linalg.norm(T) - np.linalg.norm(s)) < 1e-12 * np.linalg.norm(s)


def test_fp32_gaussian_definition():
    """Same Philox words as the FP64 definition, coarser uniforms: the two
    normals differ by the change of u1, u2 (<= 2^-23 each), not more."""
    k, b = 301, 32
    for idx in (0, 7):
        g32 = synth.step_gaussian_f32(SEED, 3, k, b, index=idx).astype(np.float64)
        g64 = synth.step_gaussian(SEED, 3, k, b, index=idx)
        x0, x1, x2, x3 = synth.gauss.step_words(SEED, 3, k, b, idx)
        u1 = synth.uniform52(x0, x1)
        # d z / d u1 = -z / (2 u1 ln u1 ... ) bounded by 1 / (u1 r); d z / d u2 = 2 pi r
        rr = np.sqrt(-2.0 * np.log(u1))
        bound = 2.0 ** -22 * (1.0 / (u1 * rr) + 2 * np.pi * rr) + 2.0 ** -23 * np.abs(g64[::2])
        bound = np.repeat(bound, 2, axis=0)[:k]
        assert np.all(np.abs(g32 - g64) <= bound)
    # distribution: mean and variance of many draws
    g = synth.step_gaussian_f32(SEED, 1, 4000, 32, index=5).astype(np.float64)
    assert abs(g.mean()) < 0.02 and abs(g.var() - 1.0) < 0.02
    # words differ across matrix indices
    assert not np.array_equal(synth.step_gaussian_f32(SEED, 1, 8, 4, 0), synth.step_gaussian_f32(SEED, 1, 8, 4, 1))


def test_batch_dims_and_stream_layout():
    m, n, r = synth.batch.batch_dims(4096, 1703)
    assert m.min() >= 64 and m.max() <= 512 and n.min() >= 64 and n.max() <= 512
    assert np.any(m > n) and np.any(m < n)
    assert r.min() >= 4.0 and r.max() <= 64.0
    g, off = synth.batch.batched_gaussian_stream(SEED, m[:5], n[:5], [32] * 5)
    for i in range(5):
        lay, tot = synth.stream_layout(int(m[i]), int(n[i]), 32)
        end = off[i + 1] if i + 1 < 5 else len(g)
        assert end - off[i] == tot
        s0, k0, o0 = lay[0]
        np.testing.assert_array_equal(g[off[i]:off[i] + k0 * 32].reshape(32, k0).T,
                                      synth.step_gaussian_f32(SEED, 1, k0, 32, index=i))


def test_device_generator_recipe_on_cpu():
    """The large-batch generator (torch, grouped batched QR) builds the stated
    workload: each matrix has singular values exp(-j / r_i) to FP32 accuracy,
    its packed slot has the right size, and a seed fixes the batch."""
    torch = pytest.importorskip("torch")
    m, n, r = synth.batch.batch_dims(6, 5)
    A = synth.batch.batch_matrices_torch(m, n, r, 11, "cpu")
    A2 = synth.batch.batch_matrices_torch(m, n, r, 11, "cpu")
    assert torch.equal(A, A2)
    assert A.numel() == int(np.sum(m.astype(np.int64) * n))
    pos = 0
    for mi, ni, ri in zip(m, n, r):
        Ai = A[pos:pos + mi * ni].view(int(ni), int(mi)).t().double().numpy()
        pos += mi * ni
        s = np.linalg.svd(Ai, compute_uv=False)
        ref = np.exp(-np.arange(1, min(mi, ni) + 1) / ri)
        assert np.max(np.abs(s - ref)) <= 1e-5

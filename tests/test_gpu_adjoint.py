"""The rank-k map A_k = U(:,1:k) T(1:k,:) V^T of randUTV and its hand-written
reverse pass on the GPU (FP64), against the oracle (reverse mode of the
same steps, torch.autograd on CPU): A_k and (dA_k/dA)^T C element by
element (1e-9 of the largest entry: FP64, the two sides differ by rounding
amplified by the 1/(alpha - beta) of each reflector), the loss gradient of
||A - A_k||_F^2 through torch.autograd, central differences (h = 1e-6) with
the GPU forward, the exact-rank closed form, repeated cotangents on one
state, and the workload m = n = 1024, sigma_j = exp(-j/40), b = 32, q = 1,
k = 64."""
import numpy as np
import pytest
import synth
import oracle
from gpu_util import require_gpu, dev, host

pytestmark = pytest.mark.gpu
SEED = 998
REL = 1e-9


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


def _g(step, k, w):
    return synth.step_gaussian(SEED, step, k, w)


def _stream(m, n, b, k):
    out = []
    for i in range(1, k // b + 1):
        out.append(_g(i, m - b * (i - 1), b).ravel(order="F"))
    return np.concatenate(out)


def _rel(x, ref):
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


CASES = [(48, 48, 8, 16, 1), (60, 40, 8, 16, 1), (40, 56, 8, 24, 1), (48, 48, 8, 16, 0), (97, 70, 16, 32, 2),
         (200, 200, 32, 64, 1)]


@pytest.mark.parametrize("m,n,b,k,q", CASES)
def test_forward_and_vjp_against_oracle(R, m, n, b, k, q):
    A = synth.make_matrix("exp", m, n, 5, r=10.0)
    C = np.random.default_rng(7).standard_normal((m, n))
    Ak_o, g_o = oracle.rank_k_vjp(A, b, q, _g, k, C)
    F, st = R.rank_k_forward(dev(A), b=b, q=q, k=k, g_inject=dev(_stream(m, n, b, k)), keep=True)
    assert _rel(host(F), Ak_o) <= REL
    g = host(R.rank_k_vjp(st, dev(C)))
    assert _rel(g, g_o) <= REL, _rel(g, g_o)
    # a second cotangent on the same state
    C2 = np.random.default_rng(8).standard_normal((m, n))
    _, g2_o = oracle.rank_k_vjp(A, b, q, _g, k, C2)
    assert _rel(host(R.rank_k_vjp(st, dev(C2))), g2_o) <= REL


def test_loss_gradient_through_autograd(R):
    import torch
    m, n, b, k = 60, 44, 8, 16
    A = synth.make_matrix("exp", m, n, 6, r=10.0)
    L_o, gL_o = oracle.loss_grad(A, b, 1, _g, k)
    At = dev(A).requires_grad_(True)
    Ak = R.rank_k(At, b=b, q=1, k=k, g_inject=dev(_stream(m, n, b, k)))
    L = ((At - Ak) ** 2).sum()
    L.backward()
    assert abs(float(L) - L_o) <= 1e-12 * L_o
    assert _rel(host(At.grad), gL_o) <= REL


def test_exact_rank_closed_form(R):
    m, n, b, k = 40, 40, 8, 16
    s = np.concatenate([np.exp(-np.arange(k) / 4.0), np.zeros(n - k)])
    q1 = synth.haar_orthogonal(m, 11)
    q2 = synth.haar_orthogonal(n, 12)
    A = (q1 * s[None, :]) @ q2.T
    Pc, Pr = q1[:, :k] @ q1[:, :k].T, q2[:, :k] @ q2[:, :k].T
    C = np.random.default_rng(13).standard_normal((m, n))
    F, st = R.rank_k_forward(dev(A), b=b, q=1, k=k, seed=SEED, keep=True)
    np.testing.assert_allclose(host(F), A, atol=1e-12)
    ref = C - (np.eye(m) - Pc) @ C @ (np.eye(n) - Pr)
    np.testing.assert_allclose(host(R.rank_k_vjp(st, dev(C))), ref, atol=1e-9 * np.abs(C).max())


@pytest.fixture(scope="module")
def workload(R):
    """m = n = 1024, sigma_j = exp(-j/40), b = 32, q = 1, k = 64."""
    return synth.make_matrix("exp40", 1024, 1024, 1703005)


def test_workload_against_oracle(R, workload):
    A = workload
    C = np.random.default_rng(21).standard_normal(A.shape)
    Ak_o, g_o = oracle.rank_k_vjp(A, 32, 1, _g, 64, C)
    # in-kernel Gaussians (the FP64 engine's generator): equal to the definition to the last bits
    F, st = R.rank_k_forward(dev(A), b=32, q=1, k=64, seed=SEED, keep=True)
    assert _rel(host(F), Ak_o) <= REL
    assert _rel(host(R.rank_k_vjp(st, dev(C))), g_o) <= REL


def test_workload_central_differences(R, workload):
    """Directional derivatives of <C, A_k> and of ||A - A_k||_F^2 from the
    GPU forward (h = 1e-6) against the GPU reverse pass."""
    import torch
    A = workload
    rng = np.random.default_rng(22)
    C = rng.standard_normal(A.shape)
    Ad = dev(A)
    F, st = R.rank_k_forward(Ad, b=32, q=1, k=64, keep=True)
    g = host(R.rank_k_vjp(st, dev(C)))
    E = dev(A - host(F))
    gE = host(R.rank_k_vjp(st, E))
    gL = 2.0 * host(E) - 2.0 * gE
    h = 1e-6
    for _ in range(2):
        D = rng.standard_normal(A.shape)
        Fp, _ = R.rank_k_forward(Ad + h * dev(D), b=32, q=1, k=64)
        Fm, _ = R.rank_k_forward(Ad - h * dev(D), b=32, q=1, k=64)
        fd = float(torch.sum(dev(C) * (Fp - Fm))) / (2 * h)
        an = float(np.sum(g * D))
        assert abs(fd - an) <= 1e-6 * (abs(fd) + 1e-3 * np.linalg.norm(g) * np.linalg.norm(D)), (fd, an)
        Lp = float(torch.sum((Ad + h * dev(D) - Fp) ** 2))
        Lm = float(torch.sum((Ad - h * dev(D) - Fm) ** 2))
        fdL = (Lp - Lm) / (2 * h)
        anL = float(np.sum(gL * D))
        assert abs(fdL - anL) <= 1e-5 * (abs(fdL) + 1e-3 * np.linalg.norm(gL) * np.linalg.norm(D)), (fdL, anL)

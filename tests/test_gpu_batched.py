"""Batched FP32 randUTV on the GPU against the FP64 oracle.

Each matrix of a batch is factored by Fig. 4 with the early stop of Section
1.1 (ii) and the rectangular final blocks of Section 5.2 and of the Remark on
m < n.  Parity, element by element where the result is unique: k_reached
(an integer decided by a norm comparison: equal unless the oracle's trailing
norm sits within 1e-3 of the threshold, where either side is valid),
|diag T| entry by entry under max(1e-4 |d_ref|, 4 s_j), s_j the oracle's own
spread under random perturbations of A of the two sides' measured backward
errors (the FP32 result's residual plus the oracle's), over the entries the
FP32 sketch resolves (see _resolved_prefix: with q = 1 a block whose
singular values span more than (1e-3 / 2^-24)^(1/3) = 25 starts to lose its
smallest directions to the rounding of Y, and FP32 and FP64 then pick
different, equally valid bases; measured on the CPU with the sketch alone
rounded to FP32, the deviation grows from below 1e-6 at that point to 1e-2
at a span of 180, more than a perturbation of the backward error moves the
oracle; the ratio beyond the prefix is reported, not asserted),
the exact zeros of T below the diagonal of
its finished columns, the trailing block norm at the stop; where several
results are valid (signs and bases of U, V) the test checks A = U T V^T to
1e-5 and the orthogonality of U, V to 1e-5 (FP32: 2^-24 per operation, a few
hundred operations per entry).  Cases: tall, wide, square, the smallest
and largest sizes, ragged tails, b = 16 and 32, tol = 0 and 1e-5, injected
and in-kernel Gaussians, graph replay, a zero matrix, a non-finite matrix,
an empty batch, and the full 4096-matrix workload on sampled matrices."""
import numpy as np
import pytest
import synth
import oracle
from oracle import checks
from gpu_util import require_gpu, dev, host
from diag_bound import compare
from parity_util import oracle_sensitivity

pytestmark = pytest.mark.gpu
SEED = 998
RES_TOL = 1e-5
ORTH_TOL = 1e-5
DIAG_REL = 1e-4


@pytest.fixture(scope="module")
def R():
    require_gpu()
    import paper_1703_00998_gb300 as R
    return R


SHAPES = [(64, 64), (80, 64), (64, 120), (130, 130), (97, 64), (150, 70), (512, 64), (64, 512), (200, 333),
          (333, 200), (512, 512), (65, 65), (33, 1), (1, 40), (1, 1), (31, 33), (96, 96), (257, 129)]
RATES = [6.0, 12.0, 4.0, 30.0, 64.0, 9.0, 5.0, 20.0, 40.0, 7.0, 50.0, 10.0, 4.0, 4.0, 4.0, 8.0, 16.0, 25.0]


def _batch():
    m = np.array([s[0] for s in SHAPES], dtype=np.int32)
    n = np.array([s[1] for s in SHAPES], dtype=np.int32)
    r = np.array(RATES)
    return m, n, r, synth.batch.batch_matrices(m, n, r, 17)


def _gauss(i, s, k, w):
    return synth.step_gaussian_f32(SEED, s, k, w, index=i).astype(np.float64)


def _resolved_prefix(dref, b, q=1, limit=1e-3):
    """Number of leading diagonal entries the FP32 sketch resolves.  Y =
    (X^T X)^q X^T G carries the direction of sigma_j with weight
    (sigma_j / sigma_{r0+1})^(2q+1) against the block's largest; FP32
    rounding (2^-24 of the largest) hides it once 2^-24 (d_{r0} / d_j)^(2q+1)
    exceeds ``limit``, and from there on the FP32 and FP64 bases legitimately
    differ (also in later blocks, which inherit what the sketch missed)."""
    d = np.abs(dref)
    for r0 in range(0, len(d), b):
        blk = d[r0:r0 + b]
        if blk[0] == 0.0:
            return r0
        rho = 2.0 ** -24 * (blk[0] / np.maximum(blk, 1e-300)) ** (2 * q + 1)
        bad = np.nonzero(rho > limit)[0]
        if len(bad):
            return r0 + int(bad[0])
    return len(d)


def _oracle_ratio(A, b, k, idx):
    """||T(k:, k:)||_F / ||A||_F of the oracle after k / b steps."""
    _, T, _, _ = oracle.randutv(A, b, 1, lambda s, kk, w: _gauss(idx, s, kk, w), max_steps=k // b, form_uv=False)
    return float(np.linalg.norm(T[k:, k:]) / np.linalg.norm(A))


def _check_matrix(plan, out, i, A32, b, tol, k_gpu, gauss_index=None, diag_rel=DIAG_REL):
    A = A32.astype(np.float64)
    T = host(plan.matrix(out.T, i)).astype(np.float64)
    U = host(plan.matrix(out.U, i, "u")).astype(np.float64)
    V = host(plan.matrix(out.V, i, "v")).astype(np.float64)
    idx = i if gauss_index is None else gauss_index
    Uo, To, Vo, ko = oracle.randutv(A, b, 1, lambda s, k, w: _gauss(idx, s, k, w), tol=tol)
    nA = float(np.linalg.norm(A))
    if k_gpu != ko:
        kk = min(k_gpu, ko)
        ratio = _oracle_ratio(A, b, kk, idx)
        assert abs(ratio - tol) <= 1e-3 * tol, (i, k_gpu, ko, ratio)
    k = k_gpu
    if nA > 0:
        assert checks.residual(A, U, T, V) <= RES_TOL, (i, checks.residual(A, U, T, V))
    assert checks.orth_err(U) <= ORTH_TOL and checks.orth_err(V) <= ORTH_TOL, (i, checks.orth_err(U),
                                                                               checks.orth_err(V))
    assert checks.lower_max(T[:, :k]) == 0.0, i
    p = min(A.shape)
    if k < p:
        assert np.linalg.norm(T[k:, k:]) <= tol * nA * (1 + 1e-3), i
    kk = min(k, ko)
    if nA > 0 and kk > 0:
        eps = checks.residual(A, U, T, V) + checks.residual(A, Uo, To, Vo)
        sens = oracle_sensitivity(A, b, 1, lambda s_, k_, w_: _gauss(idx, s_, k_, w_), eps, tol=tol)
        kk = min(kk, len(sens))
        kp = _resolved_prefix(np.diag(To)[:kk], b)
        r = compare(np.diag(T)[:kp], np.diag(To)[:kp], sens[:kp], diag_rel, 4.0)
        r_all = compare(np.diag(T)[:kk], np.diag(To)[:kk], sens[:kk], diag_rel, 4.0)
        r["entries"] = kk
        r["beyond_prefix_ratio"] = r_all["ratio"]
        print(f"batched matrix {i} {A.shape}: |diag T| over the resolved prefix {r}")
        assert r["ok"], (i, r)
    return k


@pytest.mark.parametrize("b", [16, 32])
@pytest.mark.parametrize("tol", [0.0, 1e-5])
def test_batch_parity_injected_gaussians(R, b, tol):
    import torch
    m, n, r, As = _batch()
    plan = R.BatchedPlan(m, n, b=b)
    A = dev(synth.batch.pack(As))
    g, offs = synth.batch.batched_gaussian_stream(SEED, m, n, plan.b)
    np.testing.assert_array_equal(offs, plan.off_g)
    out = plan.factor(A, q=1, tol=tol, g_inject=dev(g))
    torch.cuda.synchronize()
    ks = host(out.k_reached)
    assert np.all(host(out.info) == 0)
    for i in range(len(As)):
        k = _check_matrix(plan, out, i, As[i], int(plan.b[i]), tol, int(ks[i]))
        if tol == 0.0:
            assert k == min(As[i].shape)
    # A is read only
    np.testing.assert_array_equal(host(A), synth.batch.pack(As))


def test_in_kernel_generator_matches_definition(R):
    for idx, step, k, w in [(0, 1, 97, 32), (5, 3, 512, 16), (4095, 2, 1, 7), (17, 9, 64, 32)]:
        g = host(R.batched_gaussian(SEED, idx, step, k, w)).astype(np.float64)
        ref = synth.step_gaussian_f32(SEED, step, k, w, index=idx).astype(np.float64)
        # logf / sincospif / sqrtf in FP32 against FP64 rounded once:
        # a few FP32 ulps of r <= sqrt(2 * 24 ln 2) < 6
        assert np.max(np.abs(g - ref)) <= 6.0 * 2.0 ** -20, (idx, step)


def test_in_kernel_gaussians_close_to_injected(R):
    import torch
    m, n, r, As = _batch()
    plan = R.BatchedPlan(m, n, b=32)
    A = dev(synth.batch.pack(As))
    g, _ = synth.batch.batched_gaussian_stream(SEED, m, n, plan.b)
    o1 = plan.factor(A, q=1, tol=1e-5, g_inject=dev(g))
    o2 = plan.factor(A, q=1, tol=1e-5, seed=SEED)
    torch.cuda.synchronize()
    k1, k2 = host(o1.k_reached), host(o2.k_reached)
    for i in range(len(As)):
        # the in-kernel draws equal the definition to a few FP32 ulps, so the
        # oracle on the definition's G is the reference for both
        _check_matrix(plan, o2, i, As[i], int(plan.b[i]), 1e-5, int(k2[i]))
    assert np.sum(k1 != k2) <= 1


def test_graph_replay_is_bitwise(R):
    import torch
    m, n, r, As = _batch()
    plan = R.BatchedPlan(m, n, b=0)
    A = dev(synth.batch.pack(As))
    o1 = plan.factor(A, q=1, tol=1e-5)
    o2 = plan.factor(A, q=1, tol=1e-5, graph=True)
    o3 = plan.factor(A, q=1, tol=1e-5, graph=True, out=(o2.U, o2.T, o2.V, o2.k_reached, o2.info))
    torch.cuda.synchronize()
    for x, y in ((o1.T, o3.T), (o1.U, o3.U), (o1.V, o3.V), (o1.k_reached, o3.k_reached)):
        assert torch.equal(x, y)


def test_t_only_matches_full(R):
    import torch
    m, n, r, As = _batch()
    plan = R.BatchedPlan(m, n, b=16)
    A = dev(synth.batch.pack(As))
    o1 = plan.factor(A, q=1, tol=1e-5)
    o2 = plan.factor(A, q=1, tol=1e-5, form_uv=False)
    torch.cuda.synchronize()
    assert o2.U is None and o2.V is None
    assert torch.equal(o1.T, o2.T) and torch.equal(o1.k_reached, o2.k_reached)


def test_degenerate_matrices(R):
    import torch
    m = np.array([64, 100, 70, 64], dtype=np.int32)
    n = np.array([64, 90, 130, 64], dtype=np.int32)
    As = [np.zeros((64, 64), np.float32), synth.batch.batch_matrices(m[1:2], n[1:2], [8.0], 3)[0],
          np.zeros((70, 130), np.float32), np.full((64, 64), np.nan, np.float32)]
    plan = R.BatchedPlan(m, n, b=32)
    A = dev(synth.batch.pack(As))
    # tol > 0: the zero matrices stop before the first step (k = 0)
    out = plan.factor(A, q=1, tol=1e-5, check=False)
    torch.cuda.synchronize()
    ks, info = host(out.k_reached), host(out.info)
    from paper_1703_00998_gb300 import native
    assert ks[0] == 0 and ks[2] == 0 and ks[3] == 0
    assert info[3] == native.ENAN and info[0] == 0 and info[1] == 0
    U0 = host(plan.matrix(out.U, 0, "u"))
    np.testing.assert_array_equal(U0, np.eye(64, dtype=np.float32))
    _check_matrix(plan, out, 1, As[1], 32, 1e-5, int(ks[1]), gauss_index=1)
    with pytest.raises(R.RandutvError):
        plan.factor(A, q=1, tol=1e-5)
    # tol = 0 on the zero matrices: a full factorization of 0, T = 0, U, V orthogonal
    plan2 = R.BatchedPlan(m[[0, 2]], n[[0, 2]], b=16)
    A2 = dev(synth.batch.pack([As[0], As[2]]))
    o2 = plan2.factor(A2, q=1, tol=0.0)
    torch.cuda.synchronize()
    for i in range(2):
        assert int(host(o2.k_reached)[i]) == min(As[2 * i].shape)
        assert np.all(host(plan2.matrix(o2.T, i)) == 0)
        assert checks.orth_err(host(plan2.matrix(o2.U, i, "u")).astype(np.float64)) <= ORTH_TOL
        assert checks.orth_err(host(plan2.matrix(o2.V, i, "v")).astype(np.float64)) <= ORTH_TOL


def test_empty_batch(R):
    import torch
    plan = R.BatchedPlan(np.zeros(0, np.int32), np.zeros(0, np.int32))
    out = plan.factor(torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert out.k_reached.numel() == 0


@pytest.fixture(scope="module")
def workload(R):
    """The batched workload: 4096 matrices, m, n uniform in [64, 512],
    sigma_j = exp(-j / r), r uniform in [4, 64], FP32."""
    import torch
    m, n, r = synth.batch.batch_dims(4096, 1703)
    A = synth.batch.batch_matrices_torch(m, n, r, 1703, "cuda")
    torch.cuda.synchronize()
    return m, n, r, A


def test_workload_autotuned_graph(R, workload):
    """The configuration the benchmark times (autotuned b, one graph-captured
    launch, tol 1e-5, q = 1): every matrix checked for A = U T V^T,
    orthogonality, structure and the stop rule (FP64 on the GPU), and 16
    sampled matrices against the oracle."""
    import torch
    m, n, r, A = workload
    plan = R.BatchedPlan(m, n, b=0)
    choice = plan.autotune(A, q=1, tol=1e-5)
    assert set(int(c) for c in choice) <= {16, 32}
    assert np.all(np.isin(plan.b, [16, 32]))
    out = plan.factor(A, q=1, tol=1e-5, graph=True)
    torch.cuda.synchronize()
    ks, info = host(out.k_reached), host(out.info)
    assert np.all(info == 0)
    worst_res = worst_orth = 0.0
    for i in range(plan.count):
        Ai = plan.matrix(A, i).double()
        Ti = plan.matrix(out.T, i).double()
        Ui = plan.matrix(out.U, i, "u").double()
        Vi = plan.matrix(out.V, i, "v").double()
        nA = torch.linalg.norm(Ai)
        res = float(torch.linalg.norm(Ai - Ui @ Ti @ Vi.T) / nA)
        ou = float((Ui.T @ Ui - torch.eye(Ui.shape[0], dtype=torch.float64, device="cuda")).abs().max())
        ov = float((Vi.T @ Vi - torch.eye(Vi.shape[0], dtype=torch.float64, device="cuda")).abs().max())
        k = int(ks[i])
        assert float(torch.tril(Ti[:, :k], -1).abs().max()) == 0.0 if k > 0 else True
        if k < min(int(m[i]), int(n[i])):
            assert float(torch.linalg.norm(Ti[k:, k:])) <= 1e-5 * float(nA) * (1 + 1e-3), i
        worst_res, worst_orth = max(worst_res, res), max(worst_orth, ou, ov)
    print(f"4096 matrices: worst residual {worst_res:.2e}, worst orthogonality {worst_orth:.2e}, "
          f"mean k {ks.mean():.1f}, classes {list(choice)}")
    assert worst_res <= RES_TOL and worst_orth <= ORTH_TOL
    rng = np.random.default_rng(5)
    for i in sorted(rng.choice(plan.count, 16, replace=False)):
        Ai = host(plan.matrix(A, i)).copy()
        _check_matrix(plan, out, int(i), Ai, int(plan.b[i]), 1e-5, int(ks[i]))

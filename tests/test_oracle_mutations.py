"""Plant plausible mistakes in copies of the oracle and check that the pin
battery catches every one (the pins are strong enough to trust the oracle).
Mistakes are planted on the CPU, in a throw-away copy of the module's source."""
import inspect
import sys
import types
import pytest
import oracle
import oracle_pins as P

R = sys.modules["oracle.randutv"]        # the module (the package re-exports the function)
H = sys.modules["oracle.householder"]

MUTATIONS = {
    # T-factor without its off-diagonal part
    "tfactor_diag_only": (H, "S[:j, j] = -tau[j] * (S[:j, :j] @ (V[:, :j].T @ V[:, j]))", "S[:j, j] = 0.0"),
    # left application with S instead of S^T
    "left_apply_untransposed_S": (H, "return C - V @ (S.T @ (V.T @ C))", "return C - V @ (S @ (V.T @ C))"),
    # right application with a transposed S
    "right_apply_transposed_S": (H, "return C - ((C @ V) @ S) @ V.T", "return C - ((C @ V) @ S.T) @ V.T"),
    # Householder sign flipped (not LAPACK's convention)
    "house_sign": (H, "beta = -math.copysign(math.hypot(alpha, xnorm), alpha)", "beta = math.copysign(math.hypot(alpha, xnorm), alpha)"),
    # one power step too few
    "power_off_by_one": (R, "for _ in range(q):\n                Y = X.T @ (X @ Y)", "for _ in range(q - 1):\n                Y = X.T @ (X @ Y)"),
    # sketch with X instead of X^T
    "sketch_transposed": (R, "Y = X.T @ G", "Y = X[:, :].T @ G[::-1]"),
    # forget T(I1, J2) <- T(I1, J2) Vs
    "skip_T_I1_update": (R, "T[:r0, r0:c1] = T[:r0, r0:c1] @ Vs\n            if form_uv:", "if form_uv:"),
    # U(:, I2) <- U(:, I2) Us^T instead of Us
    "U_small_transposed": (R, "U[:, r0:r1] = U[:, r0:r1] @ Us\n                V[:, r0:c1]", "U[:, r0:r1] = U[:, r0:r1] @ Us.T\n                V[:, r0:c1]"),
    # apply VV only to the active rows of T (drop I1)
    "right_apply_skips_I1": (R, "T[:, r0:] = wy_apply_right(T[:, r0:], Vv, Sv)", "T[r0:, r0:] = wy_apply_right(T[r0:, r0:], Vv, Sv)"),
    # do not zero T(I3, J2)
    "no_zero_below_panel": (R, "T[r0:, r0:c1] = 0.0\n", "pass\n"),
    # panel QR taken before the right application (stale panel)
    "stale_panel": (R, "            Vv, tv, _ = householder_qr(Y)\n", "            Vv, tv, _ = householder_qr(Y)\n            _stale = T[r0:, r0:c1].copy()\n"),
    # over-sampling: the trailing (not the dominant) singular vectors of Y
    "oversampling_wrong_vectors": (R, "E[:w, :] = Us[:, :b]", "E[:w, :] = Us[:, w - b:]"),
    # over-sampling: Z without the Householder Q of Y (just Us padded with zeros)
    "oversampling_no_q": (R, "return E - Vq @ (Sq @ (Vq.T @ E))", "return E"),
    # over-sampling: G drawn b wide, the extra samples dropped
    "oversampling_no_extra_samples": (R, "G = np.asarray(gauss(i, m - r0, b + p), dtype=np.float64)[:, :min(b + p, n - r0)]",
                                      "G = np.asarray(gauss(i, m - r0, b + p), dtype=np.float64)[:, :b]"),
    # wrong partition: J2 one column short
    "J2_short": (R, "c1 = min(r0 + b, n)        # end of J2", "c1 = min(r0 + b, n) - (1 if n - r0 > b else 0)"),
}


def _mutated_randutv(mod, old, new):
    src = inspect.getsource(mod)
    assert old in src, f"mutation anchor not found: {old!r}"
    src = src.replace(old, new, 1)
    if mod is R and "_stale" in new:
        src = src.replace("householder_qr(T[r0:, r0:c1])", "householder_qr(_stale)", 1)
    m = types.ModuleType("mut_" + mod.__name__.split(".")[-1])
    m.__dict__["__package__"] = "oracle"
    exec(compile(src, "<mutant>", "exec"), m.__dict__)
    if mod is H:
        r_src = inspect.getsource(R).replace(
            "from .householder import householder_qr, tfactor, wy_apply_right, wy_apply_left_t", "")
        rm = types.ModuleType("mut_randutv")
        rm.__dict__["__package__"] = "oracle"
        rm.__dict__.update({k: m.__dict__[k] for k in ("householder_qr", "tfactor", "wy_apply_right", "wy_apply_left_t")})
        exec(compile(r_src, "<mutant-driver>", "exec"), rm.__dict__)
        return rm.randutv
    return m.randutv


def test_unmutated_passes_battery():
    assert P.run_battery(oracle.randutv) == []
    # the copy mechanism itself: an unchanged copy of each module passes too
    anchor_r = "Y = X.T @ G"
    anchor_h = "return C - ((C @ V) @ S) @ V.T"
    assert P.run_battery(_mutated_randutv(R, anchor_r, anchor_r)) == []
    assert P.run_battery(_mutated_randutv(H, anchor_h, anchor_h)) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name):
    mod, old, new = MUTATIONS[name]
    f = _mutated_randutv(mod, old, new)
    failed = P.run_battery(f)
    assert failed, f"mutation {name} passed every pin"
    assert not any("NameError" in x or "ImportError" in x for x in failed), failed

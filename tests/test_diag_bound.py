"""The per-entry |diag T| bound helper (tests/diag_bound.py) on hand-made
cases: which entries fall under the relative bar, the window of the
sensitivity, and the scaling of the perturbations."""
import numpy as np
from diag_bound import perturbations, sensitivity, compare


def test_compare_relative_and_floor_entries():
    dref = np.array([1.0, 1e-2, 1e-8, 1e-12])
    s = np.array([1e-14, 1e-14, 1e-14, 1e-14])
    # rel 1e-10: entries 0 and 1 have rel bar 1e-10 and 1e-12 >= 10 s = 1e-13; entries 2, 3 do not
    d = dref + np.array([9e-11, 9e-13, 9e-14, -9e-14])
    r = compare(d, dref, s, 1e-10, 10.0)
    assert r["ok"] and r["n_rel"] == 2 and r["n"] == 4
    assert abs(r["max_rel_on_rel"] - 9e-11) < 1e-15
    bad = d.copy()
    bad[2] = dref[2] + 2e-13          # above c s = 1e-13 and above the rel bar 1e-18
    assert not compare(bad, dref, s, 1e-10, 10.0)["ok"]
    bad = d.copy()
    bad[0] = 1.0 + 2e-10              # above the rel bar of a relatively checked entry
    assert not compare(bad, dref, s, 1e-10, 10.0)["ok"]


def test_sensitivity_takes_the_window_max():
    d0 = np.ones(12)
    dps = np.ones((2, 12))
    dps[1, 5] += 1e-9
    s = sensitivity(d0, dps, window=2)
    assert np.all(s[3:8] == np.float64(1e-9) + 0 * s[3:8]) or np.allclose(s[3:8], 1e-9, rtol=1e-6)
    assert np.all(s[:3] == 0) and np.all(s[8:] == 0)


def test_perturbation_norm():
    E = perturbations((40, 30), 3.0, 1e-6, [1, 2])
    for e in E:
        assert abs(np.linalg.norm(e, 2) - 3e-6) <= 1e-3 * 3e-6
    assert not np.allclose(E[0], E[1])

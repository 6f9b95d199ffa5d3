"""Pins of the shared input generators (Philox, Box-Muller, test matrices)."""
import os
import numpy as np
import pytest
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        out = synth.philox4x32_10(r[0], r[1], r[2], r[3], r[4], r[5])
        assert [int(v) for v in out] == r[6:10]


def test_philox_vectorised_matches_scalar():
    c0 = np.arange(7, dtype=np.uint64)
    out = synth.philox4x32_10(c0, 3, 5, 0, 123, 456)
    for i in range(7):
        one = synth.philox4x32_10(i, 3, 5, 0, 123, 456)
        assert [int(o[i]) for o in out] == [int(v) for v in one]


def test_uniform52_range_and_endpoints():
    lo = np.array([0, 0xFFFFFFFF], dtype=np.uint64)
    hi = np.array([0, 0xFFFFFFFF], dtype=np.uint64)
    u = synth.uniform52(lo, hi)
    assert u[0] == 2.0 ** -53
    assert u[1] == 1.0 - 2.0 ** -53
    assert np.all((u > 0) & (u < 1))


def test_gaussian_statistics():
    from scipy import stats
    g = synth.step_gaussian(998, 1, 250_000, 4).ravel()
    assert abs(g.mean()) < 5e-3
    assert abs(g.var() - 1.0) < 1e-2
    assert stats.kstest(g, "norm").pvalue > 1e-3


def test_gaussian_counter_layout():
    # row pairs share a Philox call: rows 2p, 2p+1 are the Box-Muller pair
    g = synth.step_gaussian(7, 3, 5, 2)
    x0, x1, x2, x3 = synth.philox4x32_10(1, 1, 3, 0, 7, 0)
    u1, u2 = synth.uniform52(x0, x1), synth.uniform52(x2, x3)
    r = np.sqrt(-2 * np.log(u1))
    assert g[2, 1] == r * np.cos(2 * np.pi * u2)
    assert g[3, 1] == r * np.sin(2 * np.pi * u2)
    # odd k: the last row is z0 of its pair; prefix property in k
    assert np.array_equal(synth.step_gaussian(7, 3, 4, 2), g[:4])
    # steps and seeds give different streams
    assert not np.array_equal(synth.step_gaussian(7, 4, 5, 2), g)
    assert not np.array_equal(synth.step_gaussian(8, 3, 5, 2), g)


def test_stream_layout():
    lay, total = synth.stream_layout(500, 500, 32)
    assert [s for s, _, _ in lay] == list(range(1, 16))  # step 16 is the final SVD
    assert lay[0] == (1, 500, 0) and lay[1] == (2, 468, 500 * 32)
    assert total == sum(k * 32 for _, k, _ in lay)
    buf = synth.gaussian_stream(998, 100, 90, 16)
    lay, total = synth.stream_layout(100, 90, 16)
    assert buf.size == total
    s, k, off = lay[2]
    assert np.array_equal(buf[off:off + k * 16].reshape(16, k).T, synth.step_gaussian(998, s, k, 16))


@pytest.mark.parametrize("kind", ["exp50", "inv", "gap", "fastdecay"])
def test_matrix_has_prescribed_spectrum(kind):
    a = synth.make_matrix(kind, 90, 70, 11)
    s = np.linalg.svd(a, compute_uv=False)
    ref = synth.spectrum(kind, 70)
    assert np.allclose(s, np.sort(ref)[::-1], rtol=1e-12, atol=1e-15)

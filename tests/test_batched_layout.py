"""Host logic of the batched form on CPU: the packed layout, block sizes and
queue order a plan holds (randutv_batched_layout_host runs the same code the
plan runs, without a device), against their definitions written out here
and against the Gaussian-stream offsets of synth."""
import ctypes
import numpy as np
import pytest
import synth


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1703_00998_gb300 import native
    return native.lib()


def _layout(lib, m, n, b, classes=None):
    c = len(m)
    m = np.ascontiguousarray(m, dtype=np.int32)
    n = np.ascontiguousarray(n, dtype=np.int32)
    outs = [np.zeros(max(c, 1), np.int64) for _ in range(4)] + [np.zeros(max(c, 1), np.int32) for _ in range(2)]
    tot = np.zeros(4, np.int64)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    cl = None if classes is None else vp(np.ascontiguousarray(classes, dtype=np.int32))
    st = lib.randutv_batched_layout_host(c, vp(m), vp(n), int(b), cl, *[vp(o) for o in outs], vp(tot))
    assert st == 0
    return [o[:c] for o in outs], tot


def test_layout_matches_definition(lib):
    m, n, _ = synth.batch.batch_dims(300, 77)
    for b, classes in ((0, None), (16, None), (0, [16, 32, 16, 32, 16, 32, 16, 32]), (7, None)):
        (oa, ou, ov, og, bo, order), tot = _layout(lib, m, n, b, classes)
        cls = classes or [32] * 8
        bexp = np.array([min(b if b else cls[(min(mi, ni) - 1) // 64], mi, ni) for mi, ni in zip(m, n)])
        np.testing.assert_array_equal(bo, bexp)
        mn, mm, nn = m.astype(np.int64) * n, m.astype(np.int64) ** 2, n.astype(np.int64) ** 2
        np.testing.assert_array_equal(oa, np.concatenate([[0], np.cumsum(mn)[:-1]]))
        np.testing.assert_array_equal(ou, np.concatenate([[0], np.cumsum(mm)[:-1]]))
        np.testing.assert_array_equal(ov, np.concatenate([[0], np.cumsum(nn)[:-1]]))
        _, goff = synth.batch.batched_gaussian_stream(998, m[:20], n[:20], bexp[:20])
        np.testing.assert_array_equal(og[:20], goff)
        assert tot[0] == mn.sum() and tot[1] == mm.sum() and tot[2] == nn.sum()
        cost = m.astype(np.float64) * n * np.minimum(m, n)
        np.testing.assert_array_equal(order, np.argsort(-cost, kind="stable"))


def test_layout_edge_cases(lib):
    (oa, ou, ov, og, bo, order), tot = _layout(lib, [], [], 0)
    assert len(oa) == 0 and list(tot) == [0, 0, 0, 0]
    (oa, ou, ov, og, bo, order), tot = _layout(lib, [1, 5, 512], [1, 3, 512], 32)
    np.testing.assert_array_equal(bo, [1, 3, 32])
    # a 1 x 1 and a 5 x 3 matrix draw no Gaussian (no randomized step); 512 x 512 draws 15 steps
    assert tot[3] == synth.stream_layout(512, 512, 32)[1]
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    big = np.array([513], np.int32)
    one = np.array([4], np.int32)
    from paper_1703_00998_gb300 import native
    f = lib.randutv_batched_layout_host
    assert f(1, vp(big), vp(one), 0, None, None, None, None, None, None, None, None) == native.EUNSUPPORTED
    assert f(1, vp(one), vp(one), 33, None, None, None, None, None, None, None, None) == -4
    bad = np.array([16, 32, 0, 32, 16, 32, 16, 32], np.int32)
    assert f(1, vp(one), vp(one), 0, vp(bad), None, None, None, None, None, None, None) == -5
    assert f(-1, None, None, 0, None, None, None, None, None, None, None, None) == -1

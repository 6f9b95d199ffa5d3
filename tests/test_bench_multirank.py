"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
time reported is the slowest rank's, the value counts every rank's units,
and the rank environment is read from RANK / LOCAL_RANK / WORLD_SIZE."""
import os
import socket
import sys
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        ms = 100.0 + 25.0 * rank            # rank 1 is the slow one
        t = bench.max_over_ranks(dist, ms, device="cpu")
        rate = bench.whole_job_rate(w, 2.0e12, t * 1e-3)
        out.put((rank, r, lr, w, t, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, lr, w, t, rate in res:
        assert (r, lr, w) == (rank, rank, 2)
        assert t == 125.0                   # max over ranks on every rank
        assert rate == pytest.approx(2 * 2.0e12 / 0.125)


def test_single_process_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.whole_job_rate(1, 10.0, 2.0) == 5.0


def test_algorithmic_bytes_floor():
    """The HBM floor of a square factorization: 1.77e10 elements (141 GB in
    FP64) at n = 8000, b = 128, q = 1, and the closed-form sums."""
    sys.path.insert(0, ROOT)
    import bench
    e = bench.algorithmic_elems(8000, 128, 1)
    assert abs(e - 1.77e10) / 1.77e10 < 0.01
    n, b, q = 1000, 100, 2
    ks = [n - b * i for i in range(n // b)]
    ref = sum((2 * q + 1) * k * k + 3 * k * k + 2 * (n - k) * k + 4 * n * k for k in ks)
    assert bench.algorithmic_elems(n, b, q) == ref
    v = bench.hbm_view(8000, 128, 1, 8, 0.694)
    assert 150 < v["achieved_gbs"] < 250 and 0 < v["frac"] < 0.05


def test_kernel_hash_ignores_comments_only(tmp_path):
    """A traffic ratio stays keyed to a source while only its comments change,
    and is dropped when its code changes."""
    sys.path.insert(0, ROOT)
    import bench
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// header\n__global__ void k(int* x) {\n  x[0] = 1;  // store\n}\n")
    b.write_text("/* another\n   header */\n__global__   void k(int* x)\n{ x[0] = 1; }\n")
    c.write_text("// header\n__global__ void k(int* x) {\n  x[0] = 2;  // store\n}\n")
    assert bench.kernel_hash(str(a)) == bench.kernel_hash(str(b))
    assert bench.kernel_hash(str(a)) != bench.kernel_hash(str(c))

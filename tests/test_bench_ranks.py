"""Host logic of bench.py's multi-rank path on CPU, world size 2 over gloo: every
rank advances its own replica, the timed interval is the slowest rank's and the
whole-job rate counts every rank's cell updates."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    w, r, loc = b._dist()
    t = b.max_over_ranks(0.5 + rank)          # rank 1 is the slow one
    out[rank] = (w, r, loc, t, b.whole_job_mlups(w, 1000, 10, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_cells():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        w, r, loc, t, v = res[rank]
        assert (w, r, loc) == (world, rank, rank)
        assert t == 1.5                              # the max over ranks
        assert v == pytest.approx(world * 1000 * 10 / 1.5 / 1e6)


def test_single_process_without_a_group():
    b = _bench()
    assert b.max_over_ranks(2.5) == 2.5
    assert b.whole_job_mlups(1, 4096 * 4096, 1900, 1.0) == pytest.approx(4096 * 4096 * 1900 / 1e6)


def test_kernel_hash_ignores_comments_only():
    """The ncu summary stays valid across comment edits of the kernel sources, not across
    code edits (string literals are code)."""
    b = _bench()
    src = 'int a = 1;  // one\n/* block\n comment */\nconst char *s = "x // y";\n\n  a += 2;\n'
    same = '// header\nint a = 1;\n\nconst char *s = "x // y"; /* trailing */\n  a += 2;   \n'
    other = 'int a = 1;\nconst char *s = "x // z";\n  a += 2;\n'
    assert b._code_only(src) == b._code_only(same)
    assert b._code_only(src) != b._code_only(other)
    assert b._code_only(src) != b._code_only(src.replace("a += 2", "a += 3"))

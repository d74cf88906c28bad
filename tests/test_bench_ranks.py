"""The multi-rank (replica) timing of bench.py on CPU: world_size 2 over gloo.  Every rank gets
the slowest rank's time, and the whole-job throughput counts every rank's cells."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, world, device="cpu")
    v = bench.job_throughput(1000, 10, ms, world)
    out.put((rank, ms, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, v in res:
        assert ms == 150.0
        assert v == pytest.approx(2 * 1000 * 10 / 0.150 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, device="cpu") == 12.5
    assert bench.job_throughput(4096 * 4096, 2000, 400.0, 1) == pytest.approx(
        4096 * 4096 * 2000 / 0.4 / 1e9)


def test_bench_functions_read_only_defined_globals():
    """Every name a function of bench.py reads from the module scope exists there (or is a
    builtin).  The multi-GPU legs run only under torchrun on several GPUs, so a stray name in
    them would otherwise first show as a crash of the scaling run."""
    import builtins
    import symtable

    sys.path.insert(0, ROOT)
    import bench
    path = os.path.join(ROOT, "bench.py")
    with open(path) as f:
        table = symtable.symtable(f.read(), path, "exec")
    missing = []

    def visit(t):
        for child in t.get_children():
            if child.get_type() == "function":
                for sym in child.get_symbols():
                    if (sym.is_global() and sym.is_referenced() and not hasattr(bench, sym.get_name())
                            and not hasattr(builtins, sym.get_name())):
                        missing.append((child.get_name(), sym.get_name()))
            visit(child)

    visit(table)
    assert not missing, missing

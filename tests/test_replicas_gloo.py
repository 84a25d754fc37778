"""Host-side logic of the multi-GPU benchmark path (independent replicas, no
data-path collective): max-over-ranks timing and failure of a rank, run as
world_size-2 gloo process groups on the CPU."""
import datetime
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q, die_rank):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    import bench
    try:
        m = bench.aggregate_elapsed(1.0 + rank, "cpu")
        if rank == die_rank:
            os._exit(0)                       # leaves between steps, nothing in flight
        dist.barrier()
        q.put((rank, "ok", m))
    except Exception as e:                    # the survivors learn of it on the host
        q.put((rank, "error", type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, die_rank=-1):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, die_rank)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            pytest.fail("a rank hung")
    out = []
    while not q.empty():
        out.append(q.get())
    return sorted(out)


def test_max_over_ranks_gloo():
    out = _run(2)
    assert [r[0] for r in out] == [0, 1]
    assert all(r[1] == "ok" and r[2] == 2.0 for r in out)


def test_killed_rank_is_an_error_not_a_hang():
    out = _run(2, die_rank=1)
    assert len(out) == 1 and out[0][:2] == (0, "error")


def test_reference_arm_other_ranks_do_nothing(capsys):
    sys.path.insert(0, ROOT)
    import bench
    old = dict(os.environ)
    os.environ.update(RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    try:
        class A:
            steps, warmup = 1, 1
        bench.run_reference(A)
    finally:
        os.environ.clear()
        os.environ.update(old)
    assert capsys.readouterr().out == ""

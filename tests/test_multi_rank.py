"""The N > 1 replica path of bench.py on CPU: two gloo ranks (127.0.0.1), each with its own
crossbar seed, combine their timings by a max-reduce; no data-path collective exists."""
import os
import socket
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, str(ROOT))
    import bench
    w, r, local, pg = bench.dist_setup(None)
    t = bench.job_time(1.0 + r, pg)              # rank r "took" 1 + r seconds
    out.put((r, w, t, bench.replica_seeds(r)))
    pg.barrier()
    pg.destroy_process_group()


def test_two_gloo_ranks_max_time_and_own_seeds():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [2, 2]
    assert [x[2] for x in res] == [2.0, 2.0]          # the slowest rank's time, everywhere
    assert not set(res[0][3]) & set(res[1][3])         # independent crossbars


def test_single_process_has_no_collective():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.job_time(3.5, None) == 3.5

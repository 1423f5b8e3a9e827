"""The N > 1 path of the benchmark is replicas: every rank conceals its own seeded batch,
with no exchange of data; the only collectives are the max of the timed region and the
sum of the units.  Checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_2205_11226_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # each rank's own batch: a small frame from its rank seed
    seed = bench.rank_seed(7, rank)
    m = synth.loss_mixed(352, 288, seed, 0.05, 0.30)
    n_units = int(m.sum())
    total_ms = 10.0 + 5.0 * rank
    e2e_ms = 20.0 + 1.0 * rank
    t, e, u = bench.reduce_over_ranks(dist, total_ms, e2e_ms, n_units, "cpu")
    out[rank] = (t, e, u, n_units, seed)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_replicas_reduce_gloo_ws2():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True,
                       start_method="spawn")
    res = [out[r] for r in range(ws)]
    # every rank sees the same whole-job figures
    assert res[0][:3] == res[1][:3]
    t, e, u = res[0][:3]
    assert t == 15.0            # max over ranks of the timed region
    assert e == 21.0            # max over ranks of the end-to-end region
    assert u == res[0][3] + res[1][3]  # units of all ranks
    # the ranks work on different batches
    assert res[0][4] != res[1][4]


def test_replicas_single_rank_no_collective():
    import bench
    assert bench.reduce_over_ranks(None, 3.0, 4.0, 17, "cpu") == (3.0, 4.0, 17.0)


def test_rank_batches_differ():
    import bench
    from paper_2205_11226_gb300 import synth
    a = synth.loss_mixed(352, 288, bench.rank_seed(0, 0), 0.05, 0.30)
    b = synth.loss_mixed(352, 288, bench.rank_seed(0, 1), 0.05, 0.30)
    assert not np.array_equal(a, b)

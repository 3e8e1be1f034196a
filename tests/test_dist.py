"""Host-side logic of the multi-GPU benchmark on CPU: world_size 2 with gloo.

The path does not shard (every GPU solves its own pair: replicas only), so the
only cross-rank operations are the barrier and the max-reduction of the step
time; both run here without a GPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, local, w = bench.dist_env()
    seed = bench.pair_seed(r)
    bench.barrier(w)
    t = bench.reduce_max(10.0 + r, w)
    out[rank] = (r, w, seed, t)
    dist.destroy_process_group()


def test_replicas_get_distinct_pairs_and_max_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    res = dict(out)
    assert sorted(res) == [0, 1]
    assert {res[r][2] for r in res} == {0, 1}          # one pair per replica
    assert all(res[r][3] == pytest.approx(11.0) for r in res)   # max over ranks
    assert all(res[r][1] == world for r in res)


def test_reference_arm_runs_on_rank0_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 1, 0

    bench.run_reference(A())
    assert capsys.readouterr().out == ""

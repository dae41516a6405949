"""Host-side logic that needs no GPU: argument checks of the batch / server
entry points, and the multi-process replica logic on gloo with two ranks."""
import ctypes
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import build_lib, replicas


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    B._lib = None
    return B.lib()


def test_batch_and_server_reject_bad_arguments_before_any_cuda_call(lib):
    h = ctypes.c_void_p()
    assert lib.oam_batch_create(0, ctypes.byref(h)) == B.OAM_ERR_INVALID_ARG
    assert lib.oam_batch_run(None, None) == B.OAM_ERR_INVALID_ARG
    assert lib.oam_batch_free(None) == B.OAM_OK
    bad = B.OamServerOpts(0, 2, 1, 10, 10, 5, 1e-3)  # zero budget
    assert lib.oam_server_create(ctypes.byref(bad), ctypes.byref(h)) == B.OAM_ERR_INVALID_ARG
    bad = B.OamServerOpts(1 << 30, 0, 1, 10, 10, 5, 1e-3)  # no slots
    assert lib.oam_server_create(ctypes.byref(bad), ctypes.byref(h)) == B.OAM_ERR_INVALID_ARG
    bad = B.OamServerOpts(1 << 30, 2, 7, 10, 10, 5, 1e-3)  # unknown precision
    assert lib.oam_server_create(ctypes.byref(bad), ctypes.byref(h)) == B.OAM_ERR_INVALID_ARG
    assert lib.oam_server_stop(None) == B.OAM_OK
    assert lib.oam_model_autotune(None, 1, None, None, None) == B.OAM_ERR_INVALID_ARG
    info = B.OamRequestInfo()
    assert lib.oam_server_poll(None, 1, ctypes.byref(info)) == B.OAM_ERR_INVALID_ARG


def test_shard_partitions_work():
    items = list(range(17))
    parts = [replicas.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert all(abs(len(p) - 17 / 3) < 1 for p in parts)
    with pytest.raises(ValueError):
        replicas.shard(items, 3, 3)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard(range(10), rank, world)
        seed = replicas.replica_seed(1, rank)
        times = replicas.max_over_ranks([float(rank + 1), float(10 - rank)])
        out.put((rank, mine, seed, times))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, mine, seed, times = q.get(timeout=120)
        res[r] = (mine, seed, times)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(res[0][0] + res[1][0]) == list(range(10))
    assert res[0][1] != res[1][1]
    assert res[0][2] == res[1][2] == [2.0, 10.0]

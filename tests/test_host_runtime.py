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


def test_served_rate_driver_accounts_every_request(monkeypatch):
    """serve.run_rate against a stand-in for the C server (no GPU): every
    request is submitted once into its own preallocated output pair, latency
    from arrival is never below latency from submission, and the deferred
    checks see each checked instance's requests with their own images."""
    import types

    import numpy as np

    from paper_2009_10173_gb300 import serve

    submitted = []

    class Info:
        def __init__(self, rid):
            self.state, self.latency_s = 2, 0.001 * rid

    def submit(server, s, g, e, h_s, x2, x1):
        submitted.append((x2.data_ptr(), x1.data_ptr()))
        rid = len(submitted)
        x2.fill_(float(rid))  # the "result" names its request
        x1.fill_(-float(rid))
        return rid

    class Stats:
        peak_running, peak_reserved_bytes = 3, 5e9

    fake = types.SimpleNamespace(oam_server_submit=submit, oam_server_poll=lambda sv, rid: Info(rid),
                                 oam_server_wait=lambda sv, rid, t: 0, OAM_OK=0,
                                 oam_server_stats=lambda sv: Stats())
    monkeypatch.setattr(serve, "B", fake)

    class Inst:
        structs = (None, None, None)
        h_s = None

        def new_outputs(self):
            return torch.zeros(3), torch.zeros(3)

    pool = [Inst() for _ in range(4)]
    seen = []

    def check(pick, x2, x1):
        seen.append((pick, float(x2[0]), float(x1[0])))
        return {"e": float(x2[0])}

    out = serve.run_rate(None, pool, 5000.0, 60, seed=3, check=check, check_picks={1, 2})
    assert out["requests"] == out["completed"] == 60 and out["failed"] == 0
    assert out["output_allocs"] == 0
    assert len(set(submitted)) == 60  # one output pair per request
    assert out["p50_latency_from_arrival_s"] >= out["p50_latency_s"]
    picks = np.random.Generator(np.random.PCG64(3))
    picks.exponential(1 / 5000.0, 60)
    expect = picks.integers(0, 4, 60)
    want = sorted((int(j), float(i + 1)) for i, j in enumerate(expect) if j in (1, 2))
    assert sorted((p, r) for p, r, _ in seen) == want
    assert all(r == -q for _, r, q in seen)
    assert out["checked"] == len(want)


def test_served_rate_driver_bounds_its_host_buffers(monkeypatch):
    """With a host-memory bound below one pair per request, the driver
    preallocates fewer pairs (at least two per instance) and reuses pairs of
    completed requests; every request still completes."""
    import types

    from paper_2009_10173_gb300 import serve

    class Info:
        state, latency_s = 2, 0.001

    fake = types.SimpleNamespace(oam_server_submit=lambda *a: 1, oam_server_poll=lambda sv, rid: Info(),
                                 oam_server_wait=lambda sv, rid, t: 0, OAM_OK=0,
                                 oam_server_stats=lambda sv: types.SimpleNamespace(peak_running=1,
                                                                                   peak_reserved_bytes=0))
    monkeypatch.setattr(serve, "B", fake)
    made = []

    class Inst:
        structs = (None, None, None)
        h_s = None
        vol_shape = (10, 10, 10)  # 8 KB per output pair

        def new_outputs(self):
            made.append(1)
            return torch.zeros(3), torch.zeros(3)

    pool = [Inst(), Inst()]
    out = serve.run_rate(None, pool, 5000.0, 40, seed=5, host_bytes=8000 * 6)
    assert out["completed"] == 40 and out["failed"] == 0
    assert len(made) - out["output_allocs"] <= 8  # preallocated: at most 6 pairs, at least 2 per instance
    assert len(made) - out["output_allocs"] >= 4

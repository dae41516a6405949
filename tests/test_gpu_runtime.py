"""Batched and served reconstructions on the GPU (through the C ABI).

* A batch of uneven jobs in one CUDA-graph launch gives exactly the images of
  each job run on its own (the kernels are deterministic), also when jobs
  share a model, and one small job agrees with the FP64 oracle's LSQR and
  FISTA.
* The request server returns, for every request in a mix of concurrent
  requests, exactly the images of the same request served alone, and served
  requests agree with the oracle's images; it respects its device-memory
  budget, reports invalid requests as failed without disturbing the others,
  and its bounded waits time out.
* The autotuner's tile shapes (fold warps, ring depth) keep results unchanged
  to the bit.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import solvers
from paper_2009_10173_gb300 import binding as B
from paper_2009_10173_gb300 import configs, inputs
from paper_2009_10173_gb300.batch import Batch
from paper_2009_10173_gb300.model import Model

pytestmark = pytest.mark.gpu

BASE = configs.scaled(configs.TINY_32, n_patches=400)
JOBS = [
    configs.scaled(BASE, px=24, py=20, nz=32, nt=192, win=11, lsqr_iters=6, fista_iters=5, power_iters=4,
                   lambda_rel=1e-3, seed=11),
    configs.scaled(BASE, px=40, py=33, nz=48, nt=192, win=9, focal_m=3.5e-3, aperture_m=2.5e-3, lsqr_iters=6,
                   fista_iters=5, power_iters=4, lambda_rel=1e-3, seed=12),
    configs.scaled(BASE, px=17, py=29, nz=40, nt=256, win=13, focal_m=5e-3, aperture_m=3.4e-3, lsqr_iters=6,
                   fista_iters=5, power_iters=4, lambda_rel=1e-3, seed=13),
]


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def signals_for(cfg, m):
    H = inputs.phantom(cfg, cfg["seed"], count=4)
    clean = m.forward(torch.from_numpy(H.astype(np.float32)).cuda()).cpu().numpy()
    return torch.from_numpy(inputs.add_noise(clean, 20.0, cfg["seed"] + 10 ** 6).astype(np.float32)).cuda()


def standalone(cfg, m, s):
    x2, _ = m.lsqr(s, cfg["lsqr_iters"])
    x1, _ = m.fista(s, cfg["fista_iters"], power_iters=cfg["power_iters"], lambda_rel=cfg["lambda_rel"])
    torch.cuda.synchronize()
    return x2.cpu().numpy(), x1.cpu().numpy()


@pytest.mark.parametrize("prec", [B.OAM_PREC_FP32, B.OAM_PREC_BF16X3, B.OAM_PREC_FFT])
def test_batch_graph_equals_standalone_runs(prec):
    cfgs, sigs = [], []
    for cfg in JOBS:
        m = Model(cfg, precision=prec)
        cfgs.append(dict(cfg, _model=m))
        sigs.append(signals_for(cfg, m))
    ref = [standalone(c, c["_model"], s) for c, s in zip(cfgs, sigs)]
    batch = Batch(cfgs, sigs, autotune=(prec == B.OAM_PREC_BF16X3))
    for _ in range(2):  # record, then replay the same graph
        batch.run()
        torch.cuda.synchronize()
        for j, (x2, x1) in zip(batch.jobs, ref):
            assert np.array_equal(j["x2"].cpu().numpy(), x2)
            assert np.array_equal(j["x1"].cpu().numpy(), x1)
    batch.close()


@pytest.mark.parametrize("prec", [B.OAM_PREC_BF16X3, B.OAM_PREC_FFT])
def test_batch_jobs_sharing_a_model_run_in_order(prec):
    """Two jobs on one model (its staging buffers serve one stream at a time)
    and a third on its own: the batch serialises the two on one branch, so
    every image equals the job run alone."""
    cfg = JOBS[0]
    m = Model(cfg, precision=prec)
    other = Model(JOBS[1], precision=prec)
    sigs = [signals_for(cfg, m), signals_for(configs.scaled(cfg, seed=31), m), signals_for(JOBS[1], other)]
    models = [m, m, other]
    cfgs = [cfg, cfg, JOBS[1]]
    ref = [standalone(c, mm, s) for c, mm, s in zip(cfgs, models, sigs)]
    h = B.oam_batch_create(3)
    outs = []
    for j, (c, mm, s) in enumerate(zip(cfgs, models, sigs)):
        x2, x1 = mm.empty_volume(), mm.empty_volume()
        nbytes = max(B.oam_solver_work_bytes(mm.handle, 0), B.oam_solver_work_bytes(mm.handle, 1))
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        work = raw[(-raw.data_ptr()) % 256:][:nbytes]
        B.oam_batch_set_job(h, j, mm.handle, s, x2, x1, B.OamLsqrOpts(c["lsqr_iters"], 0.0),
                            B.OamFistaOpts(c["fista_iters"], c["power_iters"], 1, 0, -1.0, c["lambda_rel"], 0.0,
                                           None), work)
        outs.append((x2, x1, raw))
    for _ in range(2):
        B.oam_batch_run(h)
        torch.cuda.synchronize()
        for (x2, x1, _), (r2, r1) in zip(outs, ref):
            assert np.array_equal(x2.cpu().numpy(), r2)
            assert np.array_equal(x1.cpu().numpy(), r1)
    B.oam_batch_free(h)
    m.close()
    other.close()


def test_batch_job_matches_oracle():
    cfg = dict(JOBS[0])
    S = oracle.slab(cfg)
    H = inputs.phantom(cfg, cfg["seed"], count=4)
    s64 = inputs.add_noise(oracle.forward(S, H), 20.0, cfg["seed"] + 10 ** 6)
    s32 = s64.astype(np.float32)
    m = Model(cfg, precision=B.OAM_PREC_BF16X3)
    batch = Batch([dict(cfg, _model=m)], [torch.from_numpy(s32).cuda()], autotune=False)
    batch.run()
    torch.cuda.synchronize()
    A, AT = (lambda v: oracle.forward(S, v)), (lambda v: oracle.adjoint(S, v))
    x2_ref, _ = solvers.lsqr(A, AT, s32.astype(np.float64), cfg["lsqr_iters"])
    x1_ref, _ = solvers.mb_l1(A, AT, s32.astype(np.float64), cfg["fista_iters"], cfg["power_iters"],
                              np.ones(m.vol_shape), lambda_rel=cfg["lambda_rel"], nonneg=True)
    assert rel(batch.jobs[0]["x2"].cpu().numpy(), x2_ref) < 1e-3
    assert rel(batch.jobs[0]["x1"].cpu().numpy(), x1_ref) < 1e-3
    batch.close()


def test_autotune_keeps_results():
    cfg = JOBS[1]
    m = Model(cfg, precision=B.OAM_PREC_BF16X3)
    H = torch.from_numpy(inputs.gaussian(m.vol_shape, 5).astype(np.float32)).cuda()
    s = torch.from_numpy(inputs.gaussian(m.sig_shape, 6).astype(np.float32)).cuda()
    before, before_t = m.forward(H).cpu().numpy(), m.adjoint(s).cpu().numpy()
    f, a = B.oam_model_autotune(m.handle, 2)
    assert f >= 2 and a >= 2
    for d, ring in ((0, f), (1, a)):
        w, r = B.oam_model_get_tiles(m.handle, d)
        assert w in (4, 8, 16) and r == ring
    assert np.array_equal(before, m.forward(H).cpu().numpy())
    assert np.array_equal(before_t, m.adjoint(s).cpu().numpy())
    m.close()


@pytest.mark.parametrize("name", ["job", "ragged"])
def test_every_tile_shape_gives_the_same_bits(name):
    """Position tiling, fold-warp count and ring depth change how the work is
    spread over blocks and warps, not the order of any sum: results are
    bit-identical."""
    cfg = JOBS[2] if name == "job" else configs.scaled(configs.TINY_32, px=70, py=37, nz=52, nt=200, win=15,
                                                        n_patches=800, dz_m=8e-6, z0_rel_m=-200e-6)
    m = Model(cfg, precision=B.OAM_PREC_BF16X3)
    H = torch.from_numpy(inputs.gaussian(m.vol_shape, 15).astype(np.float32)).cuda()
    s = torch.from_numpy(inputs.gaussian(m.sig_shape, 16).astype(np.float32)).cuda()
    ref_f, ref_a = None, None
    for tiling in (B.TILING_PADDED, B.TILING_SCAN):
        for d in (0, 1):
            B.oam_model_set_tiling(m.handle, d, tiling)
            assert B.oam_model_get_tiling(m.handle, d) == tiling
        for w in (4, 8, 16):
            for ring in (0, 2, 4):
                for d in (0, 1):
                    B.oam_model_set_tiles(m.handle, d, w, ring)
                    assert B.oam_model_get_tiles(m.handle, d)[0] == w
                f, a = m.forward(H).cpu().numpy(), m.adjoint(s).cpu().numpy()
                if ref_f is None:
                    ref_f, ref_a = f, a
                assert np.array_equal(f, ref_f) and np.array_equal(a, ref_a), (tiling, w, ring)
    with pytest.raises(B.OamError):
        B.oam_model_set_tiling(m.handle, 0, 3)  # not a tiling
    with pytest.raises(B.OamError):
        B.oam_model_set_tiles(m.handle, 0, 6, 0)  # 6 fold warps: not a kernel shape
    with pytest.raises(B.OamError):
        B.oam_model_set_tiles(m.handle, 0, 8, 3)  # the ring holds pairs of items
    assert B.oam_model_get_tiles(m.handle, 0)[0] == 16  # a refused shape changes nothing
    m.close()


def _request(cfg):
    m = Model(cfg, precision=B.OAM_PREC_BF16X3)
    s = signals_for(cfg, m).cpu().pin_memory()
    m.close()
    return cfg, s


def _serve(server, reqs):
    outs = []
    for cfg, s in reqs:
        x2 = torch.empty((cfg["py"], cfg["px"], cfg["nz"]), dtype=torch.float32).pin_memory()
        x1 = torch.empty_like(x2).pin_memory()
        sn, g, e = B.structs_from_config(cfg)
        rid = B.oam_server_submit(server, sn, g, e, s, x2, x1)
        outs.append((rid, x2, x1))
    for rid, _, _ in outs:
        assert B.oam_server_wait(server, rid, 120.0) == B.OAM_OK
    return outs


def _server(budget=8 << 30, slots=3, iters=(6, 5, 4), prec=B.OAM_PREC_BF16X3):
    opts = B.OamServerOpts(budget, slots, prec, iters[0], iters[1], iters[2], 1e-3)
    return B.oam_server_create(opts)


def test_server_results_same_alone_and_in_the_mix():
    reqs = [_request(c) for c in JOBS] + [_request(configs.scaled(JOBS[0], seed=21))]
    alone = []
    for r in reqs:
        srv = _server(slots=1)
        (rid, x2, x1), = _serve(srv, [r])
        B.oam_server_stop(srv)
        alone.append((x2.numpy().copy(), x1.numpy().copy()))
    srv = _server(slots=3)
    mixed = _serve(srv, reqs)
    st = B.oam_server_stats(srv)
    B.oam_server_stop(srv)
    assert st.peak_running >= 2  # requests were on the GPU together
    for (rid, x2, x1), (a2, a1) in zip(mixed, alone):
        assert np.array_equal(x2.numpy(), a2)
        assert np.array_equal(x1.numpy(), a1)


def test_server_budget_failure_and_timeout():
    reqs = [_request(JOBS[1]), _request(JOBS[2])]
    # a budget that fits one request's reservation at a time
    srv = _server(budget=1, slots=2)
    sn, g, e = B.structs_from_config(JOBS[1])
    x2 = torch.empty((JOBS[1]["py"], JOBS[1]["px"], JOBS[1]["nz"])).pin_memory()
    rid = B.oam_server_submit(srv, sn, g, e, reqs[0][1], x2, None)
    assert B.oam_server_wait(srv, rid, 60.0) == B.OAM_ERR_OOM  # can never fit the budget
    B.oam_server_stop(srv)

    need = max(B.oam_request_footprint(B.OAM_PREC_BF16X3, *B.structs_from_config(c)) for c, _ in reqs)
    srv = _server(budget=int(need * 1.5), slots=2, iters=(40, 30, 10))
    outs, bufs = [], []  # host outputs must outlive their requests
    for cfg, s in reqs:
        sn, g, e = B.structs_from_config(cfg)
        bufs.append(torch.empty((cfg["py"], cfg["px"], cfg["nz"])).pin_memory())
        outs.append(B.oam_server_submit(srv, sn, g, e, s, bufs[-1], None))
    # the second request waits for memory: a short wait on it times out
    assert B.oam_server_wait(srv, outs[1], 0.0) == B.OAM_ERR_TIMEOUT
    # an invalid request fails without disturbing the others
    bad = configs.scaled(JOBS[1], win=10)
    sn, g, e = B.structs_from_config(bad)
    rid_bad = B.oam_server_submit(srv, sn, g, e, reqs[0][1], None, None)
    for rid in outs:
        assert B.oam_server_wait(srv, rid, 120.0) == B.OAM_OK
    assert B.oam_server_wait(srv, rid_bad, 60.0) == B.OAM_ERR_INVALID_ARG
    st = B.oam_server_stats(srv)
    B.oam_server_stop(srv)
    assert st.peak_running == 1
    assert st.peak_reserved_bytes <= int(need * 1.5)


def test_server_with_fft_form_models_matches_standalone():
    """Requests served with lateral-FFT form models give exactly the images of
    the same reconstruction run directly on a model of that form."""
    reqs = [_request(JOBS[0]), _request(JOBS[2])]
    srv = _server(slots=2, prec=B.OAM_PREC_FFT)
    outs = _serve(srv, reqs)
    B.oam_server_stop(srv)
    for (cfg, s), (rid, x2, x1) in zip(reqs, outs):
        m = Model(cfg, precision=B.OAM_PREC_FFT)
        ref2, ref1 = standalone(cfg, m, s.cuda())
        m.close()
        assert np.array_equal(x2.numpy(), ref2)
        assert np.array_equal(x1.numpy(), ref1)


@pytest.mark.parametrize("prec", [B.OAM_PREC_BF16X3, B.OAM_PREC_FFT])
def test_served_requests_match_oracle(prec):
    """Two requests served together (split-BF16 or lateral-FFT models) give
    the FP64 oracle's LSQR (MB-L2) and FISTA (MB-L1) images of the same
    signals, made by the oracle's A, within the image tolerance."""
    reqs, refs = [], []
    for cfg in (JOBS[0], JOBS[1]):
        S = oracle.slab(cfg)
        H = inputs.phantom(cfg, cfg["seed"], count=4)
        s32 = inputs.add_noise(oracle.forward(S, H), 20.0, cfg["seed"] + 10 ** 6).astype(np.float32)
        s64 = s32.astype(np.float64)
        A, AT = (lambda v, S=S: oracle.forward(S, v)), (lambda v, S=S: oracle.adjoint(S, v))
        x2, _ = solvers.lsqr(A, AT, s64, cfg["lsqr_iters"])
        x1, _ = solvers.mb_l1(A, AT, s64, cfg["fista_iters"], cfg["power_iters"], np.ones(H.shape),
                              lambda_rel=cfg["lambda_rel"], nonneg=True)
        reqs.append((cfg, torch.from_numpy(s32).pin_memory()))
        refs.append((x2, x1))
    srv = _server(slots=2, prec=prec)
    outs = _serve(srv, reqs)
    B.oam_server_stop(srv)
    for (rid, x2, x1), (r2, r1) in zip(outs, refs):
        assert rel(x2.numpy(), r2) < 1e-3
        assert rel(x1.numpy(), r1) < 1e-3

"""Thin ctypes binding of ``liboam.so`` (argument marshalling only).

Every function keeps the C name and argument order of ``include/oam.h``;
device buffers are torch CUDA tensors (FP32, contiguous) and the stream is
the current torch stream unless one is given.  A missing or unloadable
library raises immediately: there is no CPU fallback.
"""
import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboam.so")

OAM_OK, OAM_ERR_INVALID_ARG, OAM_ERR_WINDOW, OAM_ERR_OOM, OAM_ERR_CUDA = 0, 1, 2, 3, 4
OAM_ERR_DEVICE, OAM_ERR_TIMEOUT, OAM_ERR_BUSY, OAM_ERR_UNSUPPORTED = 5, 6, 7, 8
OAM_PREC_FP32, OAM_PREC_BF16X3, OAM_PREC_FFT = 0, 1, 2
OAM_DISC_POINT, OAM_DISC_TRILINEAR = 0, 1

EXPORTED = ("oam_build_model", "oam_model_free", "oam_model_get_info", "oam_model_slab_column", "oam_forward",
            "oam_adjoint", "oam_lsqr", "oam_l1_fista", "oam_solver_work_bytes", "oam_status_string",
            "oam_version", "oam_profile_enable", "oam_profile_read", "oam_launch_count", "oam_lsqr_noalloc",
            "oam_model_autotune", "oam_batch_create", "oam_batch_set_job", "oam_batch_run", "oam_batch_free",
            "oam_server_create", "oam_server_submit", "oam_server_poll", "oam_server_wait", "oam_server_stats",
            "oam_server_stop", "oam_request_footprint", "oam_bandpass_taps", "oam_model_set_filter",
            "oam_filter_signals", "oam_lsqr_sweep", "oam_lsqr_sweep_work_bytes", "oam_model_get_tiles",
            "oam_model_set_tiles", "oam_model_bytes", "oam_build_model_ex", "oam_model_bytes_ex",
            "oam_model_get_tiling", "oam_model_set_tiling")

OAM_MAX_FIR_HALF = 8191
OAM_MAX_SWEEP = 32


class OamModelOpts(ctypes.Structure):
    _fields_ = [("discretisation", ctypes.c_int32)]


class OamSensor(ctypes.Structure):
    _fields_ = [("focal_m", ctypes.c_double), ("aperture_m", ctypes.c_double), ("hole_m", ctypes.c_double),
                ("c_mps", ctypes.c_double), ("n_patches", ctypes.c_int32)]


class OamGrid(ctypes.Structure):
    _fields_ = [("px", ctypes.c_int32), ("py", ctypes.c_int32), ("nz", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("win", ctypes.c_int32), ("dx_m", ctypes.c_double), ("dy_m", ctypes.c_double),
                ("dz_m", ctypes.c_double), ("z0_rel_m", ctypes.c_double), ("fs_hz", ctypes.c_double),
                ("t0_s", ctypes.c_double)]


class OamEir(ctypes.Structure):
    _fields_ = [("fc_hz", ctypes.c_double), ("frac_bw", ctypes.c_double), ("trunc_sigma", ctypes.c_double)]


class OamModelInfo(ctypes.Structure):
    _fields_ = [("t0_s", ctypes.c_double), ("n_lo", ctypes.c_int32), ("n_hi", ctypes.c_int32),
                ("n_orbits", ctypes.c_int32), ("precision", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("flops_per_op", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("exec_flops_forward", ctypes.c_double), ("exec_flops_adjoint", ctypes.c_double),
                ("op_bytes", ctypes.c_double), ("filter_half_len", ctypes.c_int32), ("filter_size", ctypes.c_int32)]


class OamLsqrOpts(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("damp", ctypes.c_double)]


class OamLsqrInfo(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("stop_reason", ctypes.c_int32), ("rnorm", ctypes.c_double),
                ("arnorm", ctypes.c_double), ("anorm", ctypes.c_double)]


class OamFistaOpts(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("power_iters", ctypes.c_int32), ("nonneg", ctypes.c_int32),
                ("compute_objective", ctypes.c_int32), ("lambda_", ctypes.c_double),
                ("lambda_rel", ctypes.c_double), ("L", ctypes.c_double), ("d_power_v0", ctypes.c_void_p)]


class OamFistaInfo(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("L", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("mu", ctypes.c_double), ("objective", ctypes.c_double)]


class OamProfile(ctypes.Structure):
    _fields_ = [("forward_calls", ctypes.c_int64), ("adjoint_calls", ctypes.c_int64),
                ("forward_ms", ctypes.c_double), ("adjoint_ms", ctypes.c_double)]


class OamServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("lsqr_iters", ctypes.c_int32), ("fista_iters", ctypes.c_int32), ("power_iters", ctypes.c_int32),
                ("lambda_rel", ctypes.c_double)]


class OamRequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("error", ctypes.c_int32), ("latency_s", ctypes.c_double)]


class OamServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int32), ("running", ctypes.c_int32), ("peak_running", ctypes.c_int32),
                ("reserved_bytes", ctypes.c_size_t), ("peak_reserved_bytes", ctypes.c_size_t)]


class OamError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {status_string(code)} ({code})")
        self.code = code


_lib = None


def lib():
    """Load liboam.so (raises if it is missing: build it with ``build_lib.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing; run paper_2009_10173_gb300.build_lib.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
        P = ctypes.POINTER
        L.oam_build_model.argtypes = [P(OamSensor), P(OamGrid), P(OamEir), ctypes.c_int, vp, P(vp)]
        L.oam_build_model_ex.argtypes = [P(OamSensor), P(OamGrid), P(OamEir), ctypes.c_int, P(OamModelOpts), vp,
                                         P(vp)]
        L.oam_model_bytes_ex.argtypes = [P(OamSensor), P(OamGrid), P(OamEir), i32, P(OamModelOpts), P(sz)]
        L.oam_model_free.argtypes = [vp]
        L.oam_model_get_info.argtypes = [vp, P(OamModelInfo)]
        L.oam_model_slab_column.argtypes = [vp, i32, i32, i32, vp, vp]
        L.oam_forward.argtypes = [vp, vp, vp, vp]
        L.oam_adjoint.argtypes = [vp, vp, vp, vp]
        L.oam_lsqr.argtypes = [vp, vp, vp, P(OamLsqrOpts), P(OamLsqrInfo), vp, sz, vp]
        L.oam_l1_fista.argtypes = [vp, vp, vp, P(OamFistaOpts), P(OamFistaInfo), vp, sz, vp]
        L.oam_solver_work_bytes.argtypes = [vp, i32, P(sz)]
        L.oam_lsqr_noalloc.argtypes = [vp, vp, vp, P(OamLsqrOpts), P(OamLsqrInfo), vp]
        L.oam_status_string.argtypes = [ctypes.c_int]
        L.oam_status_string.restype = ctypes.c_char_p
        L.oam_version.restype = i32
        L.oam_profile_enable.argtypes = [vp, i32]
        L.oam_profile_read.argtypes = [vp, P(OamProfile)]
        L.oam_launch_count.restype = ctypes.c_int64
        L.oam_model_autotune.argtypes = [vp, i32, vp, P(i32), P(i32)]
        L.oam_model_get_tiles.argtypes = [vp, i32, P(i32), P(i32)]
        L.oam_model_bytes.argtypes = [P(OamSensor), P(OamGrid), P(OamEir), i32, P(sz)]
        L.oam_model_set_tiles.argtypes = [vp, i32, i32, i32]
        L.oam_model_get_tiling.argtypes = [vp, i32, P(i32)]
        L.oam_model_set_tiling.argtypes = [vp, i32, i32]
        L.oam_batch_create.argtypes = [i32, P(vp)]
        L.oam_batch_set_job.argtypes = [vp, i32, vp, vp, vp, vp, P(OamLsqrOpts), P(OamFistaOpts), vp, sz]
        L.oam_batch_run.argtypes = [vp, vp]
        L.oam_batch_free.argtypes = [vp]
        L.oam_server_create.argtypes = [P(OamServerOpts), P(vp)]
        L.oam_server_submit.argtypes = [vp, P(OamSensor), P(OamGrid), P(OamEir), vp, vp, vp, P(ctypes.c_int64)]
        L.oam_server_poll.argtypes = [vp, ctypes.c_int64, P(OamRequestInfo)]
        L.oam_server_wait.argtypes = [vp, ctypes.c_int64, ctypes.c_double]
        L.oam_server_stats.argtypes = [vp, P(OamServerStats)]
        L.oam_server_stop.argtypes = [vp]
        L.oam_request_footprint.argtypes = [i32, P(OamSensor), P(OamGrid), P(OamEir), P(sz)]
        f64 = ctypes.c_double
        L.oam_bandpass_taps.argtypes = [f64, f64, f64, i32, P(f64)]
        L.oam_model_set_filter.argtypes = [vp, P(f64), i32, vp]
        L.oam_filter_signals.argtypes = [vp, vp, vp, vp]
        L.oam_lsqr_sweep.argtypes = [vp, vp, i32, P(f64), P(vp), i32, P(OamLsqrInfo), vp, sz, vp]
        L.oam_lsqr_sweep_work_bytes.argtypes = [vp, i32, P(sz)]
        for f in EXPORTED:
            if f not in ("oam_status_string", "oam_version", "oam_launch_count"):
                getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(code):
    return lib().oam_status_string(int(code)).decode()


def _check(fn, code):
    if code != OAM_OK:
        raise OamError(fn, code)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def structs_from_config(cfg):
    """oam_sensor / oam_grid / oam_eir from a workload mapping (SI units)."""
    s = OamSensor(cfg["focal_m"], cfg["aperture_m"], cfg.get("hole_m", 0.0), cfg["c_mps"], cfg["n_patches"])
    t0 = cfg.get("t0_s", math.nan)
    g = OamGrid(cfg["px"], cfg["py"], cfg["nz"], cfg["nt"], cfg["win"], cfg["dx_m"], cfg["dy_m"], cfg["dz_m"],
                cfg["z0_rel_m"], cfg["fs_hz"], math.nan if t0 is None else t0)
    e = OamEir(cfg["fc_hz"], cfg["frac_bw"], cfg.get("trunc_sigma", 5.0))
    return s, g, e


def oam_build_model(sensor, grid, eir, precision=OAM_PREC_FP32, stream=None, discretisation=None):
    h = ctypes.c_void_p()
    if discretisation is None:
        _check("oam_build_model", lib().oam_build_model(ctypes.byref(sensor), ctypes.byref(grid), ctypes.byref(eir),
                                                         int(precision), _stream(stream), ctypes.byref(h)))
    else:
        opts = OamModelOpts(int(discretisation))
        _check("oam_build_model_ex", lib().oam_build_model_ex(ctypes.byref(sensor), ctypes.byref(grid),
                                                               ctypes.byref(eir), int(precision), ctypes.byref(opts),
                                                               _stream(stream), ctypes.byref(h)))
    return h


def oam_model_free(model):
    _check("oam_model_free", lib().oam_model_free(model))


def oam_model_get_info(model):
    info = OamModelInfo()
    _check("oam_model_get_info", lib().oam_model_get_info(model, ctypes.byref(info)))
    return info


def oam_model_slab_column(model, b, a, k, out, stream=None):
    _check("oam_model_slab_column", lib().oam_model_slab_column(model, b, a, k, _ptr(out), _stream(stream)))


def oam_forward(model, H, s, stream=None):
    _check("oam_forward", lib().oam_forward(model, _ptr(H), _ptr(s), _stream(stream)))


def oam_adjoint(model, s, H, stream=None):
    _check("oam_adjoint", lib().oam_adjoint(model, _ptr(s), _ptr(H), _stream(stream)))


def oam_solver_work_bytes(model, solver):
    n = ctypes.c_size_t()
    _check("oam_solver_work_bytes", lib().oam_solver_work_bytes(model, int(solver), ctypes.byref(n)))
    return n.value


def oam_lsqr(model, s, x, opts, work, stream=None, want_info=True):
    info = OamLsqrInfo()
    _check("oam_lsqr", lib().oam_lsqr(model, _ptr(s), _ptr(x), ctypes.byref(opts),
                                      ctypes.byref(info) if want_info else None, _ptr(work),
                                      work.numel() * work.element_size(), _stream(stream)))
    return info


def oam_lsqr_noalloc(model, s, x, opts, stream=None, want_info=True):
    """LSQR on the library's static device workspace (no device allocation)."""
    info = OamLsqrInfo()
    _check("oam_lsqr_noalloc", lib().oam_lsqr_noalloc(model, _ptr(s), _ptr(x), ctypes.byref(opts),
                                                      ctypes.byref(info) if want_info else None, _stream(stream)))
    return info


def oam_l1_fista(model, s, x, opts, work, stream=None, want_info=True):
    info = OamFistaInfo()
    _check("oam_l1_fista", lib().oam_l1_fista(model, _ptr(s), _ptr(x), ctypes.byref(opts),
                                              ctypes.byref(info) if want_info else None, _ptr(work),
                                              work.numel() * work.element_size(), _stream(stream)))
    return info


def oam_version():
    return lib().oam_version()


def oam_bandpass_taps(f_lo_hz, f_hi_hz, fs_hz, half_len):
    """Half taps h[0..half_len] of the windowed-sinc band-pass (host only), as a list."""
    taps = (ctypes.c_double * (int(half_len) + 1))() if half_len >= 0 else None
    _check("oam_bandpass_taps", lib().oam_bandpass_taps(float(f_lo_hz), float(f_hi_hz), float(fs_hz),
                                                        int(half_len), taps))
    return list(taps)


def oam_model_set_filter(model, taps, stream=None):
    """Filter the model's operators with the even FIR taps[0..L] (None removes it)."""
    if taps is None:
        _check("oam_model_set_filter", lib().oam_model_set_filter(model, None, -1, _stream(stream)))
        return
    arr = (ctypes.c_double * len(taps))(*[float(t) for t in taps])
    _check("oam_model_set_filter", lib().oam_model_set_filter(model, arr, len(taps) - 1, _stream(stream)))


def oam_filter_signals(model, s_in, s_out, stream=None):
    _check("oam_filter_signals", lib().oam_filter_signals(model, _ptr(s_in), _ptr(s_out), _stream(stream)))


def oam_lsqr_sweep_work_bytes(model, n_damps):
    n = ctypes.c_size_t()
    _check("oam_lsqr_sweep_work_bytes", lib().oam_lsqr_sweep_work_bytes(model, int(n_damps), ctypes.byref(n)))
    return n.value


def oam_lsqr_sweep(model, s, damps, xs, iters, work, stream=None, want_info=True):
    """LSQR for every damp in ``damps`` from one bidiagonalisation; xs: one volume per damp."""
    n = len(damps)
    if len(xs) != n:
        raise ValueError("one output volume per damp")
    dv = (ctypes.c_double * n)(*[float(d) for d in damps])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    infos = (OamLsqrInfo * n)()
    _check("oam_lsqr_sweep", lib().oam_lsqr_sweep(model, _ptr(s), n, dv, xp, int(iters),
                                                  infos if want_info else None, _ptr(work),
                                                  work.numel() * work.element_size(), _stream(stream)))
    return list(infos)


def oam_profile_enable(model, enable=True):
    _check("oam_profile_enable", lib().oam_profile_enable(model, int(bool(enable))))


def oam_profile_read(model):
    p = OamProfile()
    _check("oam_profile_read", lib().oam_profile_read(model, ctypes.byref(p)))
    return p


def oam_launch_count():
    return lib().oam_launch_count()


def oam_model_autotune(model, reps=3, stream=None):
    f, a = ctypes.c_int32(), ctypes.c_int32()
    _check("oam_model_autotune", lib().oam_model_autotune(model, int(reps), _stream(stream), ctypes.byref(f),
                                                          ctypes.byref(a)))
    return f.value, a.value


def oam_model_bytes(cfg, precision, discretisation=None):
    """Device bytes oam_build_model would allocate for a configuration (host only)."""
    sn, g, e = structs_from_config(cfg)
    out = ctypes.c_size_t()
    if discretisation is None:
        _check("oam_model_bytes", lib().oam_model_bytes(ctypes.byref(sn), ctypes.byref(g), ctypes.byref(e),
                                                        int(precision), ctypes.byref(out)))
    else:
        opts = OamModelOpts(int(discretisation))
        _check("oam_model_bytes_ex", lib().oam_model_bytes_ex(ctypes.byref(sn), ctypes.byref(g), ctypes.byref(e),
                                                              int(precision), ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def oam_model_get_tiles(model, direction):
    """(fold warps, ring depth) of the split-BF16 kernel of one direction (0 forward, 1 adjoint)."""
    w, r = ctypes.c_int32(), ctypes.c_int32()
    _check("oam_model_get_tiles", lib().oam_model_get_tiles(model, int(direction), ctypes.byref(w), ctypes.byref(r)))
    return w.value, r.value


def oam_model_set_tiles(model, direction, fold_warps, ring=0):
    _check("oam_model_set_tiles", lib().oam_model_set_tiles(model, int(direction), int(fold_warps), int(ring)))


TILING_AUTO, TILING_PADDED, TILING_SCAN = 0, 1, 2


def oam_model_get_tiling(model, direction):
    """Position tiling in use by the split-BF16 kernel of one direction: 1 padded grid, 2 scan grid."""
    t = ctypes.c_int32()
    _check("oam_model_get_tiling", lib().oam_model_get_tiling(model, int(direction), ctypes.byref(t)))
    return t.value


def oam_model_set_tiling(model, direction, tiling):
    _check("oam_model_set_tiling", lib().oam_model_set_tiling(model, int(direction), int(tiling)))


def oam_batch_create(n_jobs):
    h = ctypes.c_void_p()
    _check("oam_batch_create", lib().oam_batch_create(int(n_jobs), ctypes.byref(h)))
    return h


def oam_batch_set_job(batch, job, model, s, x_l2, x_l1, lsqr_opts, fista_opts, work):
    _check("oam_batch_set_job", lib().oam_batch_set_job(
        batch, int(job), model, _ptr(s), _ptr(x_l2), _ptr(x_l1), ctypes.byref(lsqr_opts) if lsqr_opts else None,
        ctypes.byref(fista_opts) if fista_opts else None, _ptr(work), work.numel() * work.element_size()))


def oam_batch_run(batch, stream=None):
    _check("oam_batch_run", lib().oam_batch_run(batch, _stream(stream)))


def oam_batch_free(batch):
    _check("oam_batch_free", lib().oam_batch_free(batch))


def oam_server_create(opts):
    h = ctypes.c_void_p()
    _check("oam_server_create", lib().oam_server_create(ctypes.byref(opts), ctypes.byref(h)))
    return h


def oam_server_submit(server, sensor, grid, eir, h_s, h_x_l2=None, h_x_l1=None):
    """h_* are host (CPU, preferably pinned) float32 tensors that must outlive the request."""
    rid = ctypes.c_int64()
    _check("oam_server_submit", lib().oam_server_submit(server, ctypes.byref(sensor), ctypes.byref(grid),
                                                        ctypes.byref(eir), _ptr(h_s), _ptr(h_x_l2), _ptr(h_x_l1),
                                                        ctypes.byref(rid)))
    return rid.value


def oam_server_poll(server, rid):
    info = OamRequestInfo()
    _check("oam_server_poll", lib().oam_server_poll(server, ctypes.c_int64(rid), ctypes.byref(info)))
    return info


def oam_server_wait(server, rid, timeout_s):
    return lib().oam_server_wait(server, ctypes.c_int64(rid), ctypes.c_double(timeout_s))


def oam_server_stats(server):
    st = OamServerStats()
    _check("oam_server_stats", lib().oam_server_stats(server, ctypes.byref(st)))
    return st


def oam_server_stop(server):
    _check("oam_server_stop", lib().oam_server_stop(server))


def oam_request_footprint(precision, sensor, grid, eir):
    """Device bytes the server reserves for a request (host only)."""
    n = ctypes.c_size_t()
    _check("oam_request_footprint", lib().oam_request_footprint(int(precision), ctypes.byref(sensor),
                                                                ctypes.byref(grid), ctypes.byref(eir),
                                                                ctypes.byref(n)))
    return n.value

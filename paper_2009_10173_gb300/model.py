"""Convenience wrapper around a ``liboam.so`` model handle.

Only marshalling and buffer allocation (torch CUDA tensors) happen here;
every step of the computation runs in the library's kernels.
"""
import torch

from . import binding as B


class Model:
    """A device-resident model slab plus the operators and solvers that use it."""

    def __init__(self, cfg, precision=B.OAM_PREC_FP32, stream=None, device=None, discretisation=None):
        self.cfg = dict(cfg)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            s, g, e = B.structs_from_config(cfg)
            self.handle = B.oam_build_model(s, g, e, precision, stream, discretisation)
        self.info = B.oam_model_get_info(self.handle)
        self.precision = precision
        self.vol_shape = (cfg["py"], cfg["px"], cfg["nz"])
        self.sig_shape = (cfg["py"], cfg["px"], cfg["nt"])
        self._work = {}

    def close(self):
        if self.handle:
            B.oam_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ buffers
    def empty_volume(self):
        return torch.empty(self.vol_shape, dtype=torch.float32, device=self.device)

    def empty_signals(self):
        return torch.empty(self.sig_shape, dtype=torch.float32, device=self.device)

    def workspace(self, solver):
        if solver not in self._work:
            n = B.oam_solver_work_bytes(self.handle, solver)
            self._work[solver] = torch.empty((n + 255) // 256 * 256 + 256, dtype=torch.uint8, device=self.device)
        w = self._work[solver]
        off = (-w.data_ptr()) % 256
        return w[off:off + B.oam_solver_work_bytes(self.handle, solver)]

    @staticmethod
    def _check(t, shape):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected a contiguous float32 CUDA tensor of shape {shape}")

    # ------------------------------------------------------------ operators
    def slab_column(self, b, a, k, stream=None):
        out = torch.empty(self.cfg["nt"], dtype=torch.float32, device=self.device)
        B.oam_model_slab_column(self.handle, b, a, k, out, stream)
        return out

    def forward(self, H, out=None, stream=None):
        self._check(H, self.vol_shape)
        out = self.empty_signals() if out is None else out
        self._check(out, self.sig_shape)
        B.oam_forward(self.handle, H, out, stream)
        return out

    def adjoint(self, s, out=None, stream=None):
        self._check(s, self.sig_shape)
        out = self.empty_volume() if out is None else out
        self._check(out, self.vol_shape)
        B.oam_adjoint(self.handle, s, out, stream)
        return out

    # ------------------------------------------------------------ solvers
    def lsqr(self, s, iters, damp=0.0, out=None, stream=None, want_info=True):
        self._check(s, self.sig_shape)
        out = self.empty_volume() if out is None else out
        info = B.oam_lsqr(self.handle, s, out, B.OamLsqrOpts(iters, damp), self.workspace(0), stream, want_info)
        return out, info

    def lsqr_sweep(self, s, iters, damps, stream=None, want_info=True):
        """MB-L2 for each damp (lambda = damp^2) from one bidiagonalisation: (volumes, infos)."""
        self._check(s, self.sig_shape)
        xs = [self.empty_volume() for _ in damps]
        n = B.oam_lsqr_sweep_work_bytes(self.handle, len(damps))
        w = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        off = (-w.data_ptr()) % 256
        infos = B.oam_lsqr_sweep(self.handle, s, damps, xs, iters, w[off:off + n], stream, want_info)
        return xs, infos

    # ------------------------------------------------------------ band-pass filter
    def set_filter(self, taps, stream=None):
        """Make forward F A and adjoint A^T F for the even FIR taps[0..L] (None removes it)."""
        B.oam_model_set_filter(self.handle, taps, stream)
        self.info = B.oam_model_get_info(self.handle)

    def filter_signals(self, s, out=None, stream=None):
        """F s with the model's filter (out may be s)."""
        self._check(s, self.sig_shape)
        out = self.empty_signals() if out is None else out
        self._check(out, self.sig_shape)
        B.oam_filter_signals(self.handle, s, out, stream)
        return out

    def fista(self, s, iters, power_iters=20, lam=-1.0, lambda_rel=1e-3, L=0.0, nonneg=True, v0=None,
              compute_objective=False, out=None, stream=None, want_info=True):
        self._check(s, self.sig_shape)
        out = self.empty_volume() if out is None else out
        if v0 is not None:
            self._check(v0, self.vol_shape)
        opts = B.OamFistaOpts(iters, power_iters, int(bool(nonneg)), int(bool(compute_objective)), lam, lambda_rel,
                              L, None if v0 is None else v0.data_ptr())
        info = B.oam_l1_fista(self.handle, s, out, opts, self.workspace(1), stream, want_info)
        return out, info

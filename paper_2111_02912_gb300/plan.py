"""Plan: a NUFFT plan bound to torch device tensors (argument marshalling only).

Layouts (see include/nufftjac.h): omega float32 (D, M); images complex64
(N_1..N_D) or (C, N_1..N_D) without maps; maps complex64 (C, N...); k-space
complex64 (C, M).  Calls are queued on the current torch CUDA stream.
"""
import torch

from . import _abi


def _ptr(t, dtype, name, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return t.data_ptr()


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Plan:
    def __init__(self, shape, omega, J=6, sigma=2.0, beta=None, max_coils=1, bin_size=None, spread="auto",
                 deterministic=False, strip_part=0, kernel_mode="direct", table_density=0, gather="auto"):
        self.shape = tuple(int(n) for n in shape)
        self.D = len(self.shape)
        opts = _abi.nufft_default_opts(self.D, self.shape)
        opts.J = int(J)
        opts.sigma = float(sigma)
        opts.beta = float(beta) if beta else 0.0
        opts.max_coils = int(max_coils)
        if bin_size is not None:
            for d, b in enumerate(bin_size):
                opts.bin_size[d] = int(b)
        opts.spread_variant = _abi.SPREAD_VARIANTS[spread]
        opts.deterministic = 1 if deterministic else 0
        opts.strip_part = int(strip_part)
        opts.kernel_mode = _abi.KERNEL_MODES[kernel_mode]
        opts.table_density = int(table_density)
        opts.gather_variant = _abi.GATHER_VARIANTS[gather]
        self.max_coils = int(max_coils)
        self._omega = omega
        self.M = int(omega.shape[1])
        self.handle = _abi.nufft_plan(opts, self.M, _ptr(omega, torch.float32, "omega", (self.D, self.M)), _stream())

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _abi.nufft_destroy(h)
            self.handle = None

    def info(self):
        return _abi.nufft_get_info(self.handle)

    def set_points(self, omega):
        M = int(omega.shape[1])
        _abi.nufft_set_points(self.handle, M, _ptr(omega, torch.float32, "omega", (self.D, M)), _stream())
        self._omega = omega
        self.M = M

    def sort_points(self):
        """Sort the points of the last set_points now, on the current stream (else the next call does)."""
        _abi.nufft_sort_points(self.handle, _stream())

    def _coils(self, x, smaps):
        if smaps is not None:
            return int(smaps.shape[0])
        return 1 if x.dim() == self.D else int(x.shape[0])

    def _img_shape(self, C, smaps):
        return self.shape if smaps is not None else (C,) + self.shape

    def forward(self, x, smaps=None, out=None):
        C = self._coils(x, smaps)
        _ptr(x, torch.complex64, "x", self.shape if smaps is not None else None)
        y = out if out is not None else torch.empty((C, self.M), dtype=torch.complex64, device=x.device)
        _abi.nufft_forward(self.handle, C, _ptr(x, torch.complex64, "x"),
                           _ptr(smaps, torch.complex64, "smaps", (C,) + self.shape),
                           _ptr(y, torch.complex64, "y", (C, self.M)), _stream())
        return y

    def adjoint(self, y, smaps=None, out=None):
        C = int(y.shape[0])
        x = out if out is not None else torch.empty(self._img_shape(C, smaps), dtype=torch.complex64, device=y.device)
        _abi.nufft_adjoint(self.handle, C, _ptr(y, torch.complex64, "y", (C, self.M)),
                           _ptr(smaps, torch.complex64, "smaps", (C,) + self.shape),
                           _ptr(x, torch.complex64, "x", self._img_shape(C, smaps)), _stream())
        return x

    def jvp_omega(self, x, domega, smaps=None, want_y=False):
        C = self._coils(x, smaps)
        dy = torch.empty((C, self.M), dtype=torch.complex64, device=x.device)
        y = torch.empty_like(dy) if want_y else None
        _abi.nufft_jvp_omega(self.handle, C, _ptr(x, torch.complex64, "x"),
                             _ptr(smaps, torch.complex64, "smaps", (C,) + self.shape),
                             _ptr(domega, torch.float32, "domega", (self.D, self.M)),
                             _ptr(dy, torch.complex64, "dy"), _ptr(y, torch.complex64, "y"), _stream())
        return (dy, y) if want_y else dy

    def vjp_omega_x(self, x, v, smaps=None, need_omega=True, need_x=True, out=None):
        C = int(v.shape[0])
        if out is not None:
            go, gx = out
        else:
            go = torch.empty((self.D, self.M), dtype=torch.float32, device=v.device) if need_omega else None
            gx = torch.empty(self._img_shape(C, smaps), dtype=torch.complex64, device=v.device) if need_x else None
        _abi.nufft_vjp_omega_x(self.handle, C, _ptr(x, torch.complex64, "x"),
                               _ptr(smaps, torch.complex64, "smaps", (C,) + self.shape),
                               _ptr(v, torch.complex64, "v", (C, self.M)),
                               _ptr(go, torch.float32, "grad_omega"), _ptr(gx, torch.complex64, "grad_x"), _stream())
        return go, gx

    def profile_enable(self, enable=True):
        _abi.nufft_profile_enable(self.handle, enable)

    def profile_read(self):
        return _abi.nufft_profile_read(self.handle)

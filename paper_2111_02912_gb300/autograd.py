"""torch.autograd bindings of the NUFFT and its Jacobians (all compute in libnufftjac).

Operators (E = (I kron A) S, Sec. II-B, II-G) with hand-written backward passes:

* ``nufft(x, omega, op)``: y = E x; backward gives grad_x = E' g and grad_omega
  from Eq. (e,jac,Ax,v) (nufft_vjp_omega_x).
* ``nufft_adjoint(y, omega, op)``: x = E' y; backward gives grad_y = E g and
  grad_omega from Eq. (e,A'y) (= nufft_vjp_omega_x with (x, v) <- (g, y)).
* ``gram(x, omega, op, lam)``: (E'E + lam I) x; backward uses the Gram Jacobian,
  Eq. (e,A'A,x,omd): grad_omega = vjp(x; v = E g) + vjp(g; v = E x), four NUFFTs.
* ``psd_inverse(b, omega, op, lam, iters)``: z = (E'E + lam I)^-1 b by CG; the
  backward is implicit, Eq. (e,inv,omd): u = F^-1 g (CG), grad_b = u,
  grad_omega = -(vjp(z; v = E u) + vjp(u; v = E z)): memory constant in the
  number of CG iterations.
* ``cg_sense_unrolled``: K unrolled CG iterations on (E'E + lam I) x = E' y, each
  Gram product differentiable through ``gram``, optionally recomputed in the
  backward pass (torch.utils.checkpoint) instead of storing activations.

Gradients use PyTorch's convention for complex tensors: grad = dL/dRe + i dL/dIm.
The CG vector arithmetic (dot products, axpys) is plain tensor algebra around
the NUFFT calls.
"""
import torch
from torch.utils.checkpoint import checkpoint

from .plan import Plan


class NufftOperator:
    """E(omega) for fixed image shape and coil maps; keeps a plan in sync with omega."""

    def __init__(self, shape, omega, smaps=None, J=6, sigma=2.0, max_coils=None):
        self.shape = tuple(shape)
        self.smaps = smaps
        C = smaps.shape[0] if smaps is not None else (max_coils or 1)
        self.plan = Plan(self.shape, omega.detach().contiguous(), J=J, sigma=sigma, max_coils=C)
        self._key = None
        self.sync(omega)

    def sync(self, omega):
        key = (omega.data_ptr(), omega._version, tuple(omega.shape))
        if key != self._key:
            self.plan.set_points(omega.detach().contiguous())
            self._key = key

    def forward(self, x):
        return self.plan.forward(x.contiguous(), self.smaps)

    def adjoint(self, y):
        return self.plan.adjoint(y.contiguous(), self.smaps)

    def vjp_omega(self, x, v):
        go, _ = self.plan.vjp_omega_x(x.contiguous(), v.contiguous(), self.smaps, need_omega=True, need_x=False)
        return go


class _Forward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, omega, op):
        op.sync(omega)
        ctx.op = op
        ctx.save_for_backward(x, omega)
        return op.forward(x)

    @staticmethod
    def backward(ctx, g):
        x, omega = ctx.saved_tensors
        op = ctx.op
        op.sync(omega)
        go, gx = op.plan.vjp_omega_x(x.contiguous(), g.contiguous(), op.smaps,
                                     need_omega=ctx.needs_input_grad[1], need_x=ctx.needs_input_grad[0])
        return gx, go, None


class _Adjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, omega, op):
        op.sync(omega)
        ctx.op = op
        ctx.save_for_backward(y, omega)
        return op.adjoint(y)

    @staticmethod
    def backward(ctx, g):
        y, omega = ctx.saved_tensors
        op = ctx.op
        op.sync(omega)
        gy = op.forward(g) if ctx.needs_input_grad[0] else None
        go = op.vjp_omega(g, y) if ctx.needs_input_grad[1] else None   # Eq. (e,A'y)
        return gy, go, None


class _Gram(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, omega, op, lam):
        op.sync(omega)
        ctx.op, ctx.lam = op, lam
        ctx.save_for_backward(x, omega)
        z = op.adjoint(op.forward(x))
        return z + lam * x if lam else z

    @staticmethod
    def backward(ctx, g):
        x, omega = ctx.saved_tensors
        op, lam = ctx.op, ctx.lam
        op.sync(omega)
        g = g.contiguous()
        gx = go = None
        Ex, Eg = op.forward(x), op.forward(g)
        if ctx.needs_input_grad[0]:
            gx = op.adjoint(Eg) + (lam * g if lam else 0)          # F is Hermitian
        if ctx.needs_input_grad[1]:
            go = op.vjp_omega(x, Eg) + op.vjp_omega(g, Ex)       # Eq. (e,A'A,x,omd)
        return gx, go, None, None


def _vdot(a, b):
    return torch.sum(torch.conj(a) * b)


def cg_solve(apply_F, b, iters, x0=None):
    """Conjugate gradients for F x = b (F Hermitian positive definite)."""
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    r = b - apply_F(x) if x0 is not None else b.clone()
    p = r.clone()
    rr = _vdot(r, r).real
    for _ in range(iters):
        Fp = apply_F(p)
        alpha = rr / _vdot(p, Fp).real
        x = x + alpha * p
        r = r - alpha * Fp
        rr_new = _vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


class _PsdInverse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, omega, op, lam, iters):
        op.sync(omega)
        F = lambda v: op.adjoint(op.forward(v)) + lam * v
        z = cg_solve(F, b.contiguous(), iters)
        ctx.op, ctx.lam, ctx.iters = op, lam, iters
        ctx.save_for_backward(z, omega)
        return z

    @staticmethod
    def backward(ctx, g):
        z, omega = ctx.saved_tensors
        op, lam = ctx.op, ctx.lam
        op.sync(omega)
        F = lambda v: op.adjoint(op.forward(v)) + lam * v
        u = cg_solve(F, g.contiguous(), ctx.iters)                 # u = F^-1 g
        go = None
        if ctx.needs_input_grad[1]:                                 # Eq. (e,inv,omd)
            go = -(op.vjp_omega(z, op.forward(u)) + op.vjp_omega(u, op.forward(z)))
        return u, go, None, None, None


def nufft(x, omega, op):
    return _Forward.apply(x, omega, op)


def nufft_adjoint(y, omega, op):
    return _Adjoint.apply(y, omega, op)


def gram(x, omega, op, lam=0.0):
    return _Gram.apply(x, omega, op, float(lam))


def psd_inverse(b, omega, op, lam, iters):
    return _PsdInverse.apply(b, omega, op, float(lam), int(iters))


def cg_sense_unrolled(y, omega, op, lam, iters, recompute=True):
    """x_K after K CG iterations on (E'E + lam I) x = E' y, differentiable in omega and y."""
    b = nufft_adjoint(y, omega, op)
    x = torch.zeros_like(b)
    r = b
    p = r
    rr = _vdot(r, r).real

    def step(x, r, p, rr, omega):
        Fp = gram(p, omega, op, lam)
        alpha = rr / _vdot(p, Fp).real
        x = x + alpha * p
        r = r - alpha * Fp
        rr_new = _vdot(r, r).real
        p = r + (rr_new / rr) * p
        return x, r, p, rr_new

    for _ in range(iters):
        if recompute:
            x, r, p, rr = checkpoint(step, x, r, p, rr, omega, use_reentrant=False)
        else:
            x, r, p, rr = step(x, r, p, rr, omega)
    return x

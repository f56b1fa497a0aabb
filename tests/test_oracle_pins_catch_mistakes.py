"""The oracle's pins are sensitive: a plausible mistake planted in the oracle makes a pin fail.

Each test swaps one oracle function for a copy with a typical slip (a flipped sign, an index off by
one, a dropped or doubled factor, a transposed operand) and runs an existing pin against it, on the
CPU; the pin must raise.  Nothing here touches the CUDA path.
"""
import numpy as np
import pytest

import oracle.jacobian as jacobian_mod
import oracle.nudft as nudft_mod
import oracle.nufft as nufft_mod
import test_oracle_jacobian as pins_jac
import test_oracle_nudft as pins_nudft
import test_oracle_nufft as pins_nufft


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


# ---------------------------------------------------------------- exact NUDFT, Eq. (e,ndft)
def test_flipped_exponent_sign_is_caught(monkeypatch):
    """e^{+i omega r} in place of e^{-i omega r}: the hand closed forms and the single voxel fail."""
    good = nudft_mod.nudft_forward
    monkeypatch.setattr(pins_nudft, "nudft_forward", lambda x, om: good(x, -np.asarray(om)))
    _fails(pins_nudft.test_hand_closed_forms)
    _fails(pins_nudft.test_single_voxel)


def test_voxel_origin_off_by_one_is_caught(monkeypatch):
    """r = n - N/2 + 1 instead of n - N/2 (the origin of the voxel centres)."""
    good = nudft_mod.voxel_centres
    monkeypatch.setattr(nudft_mod, "voxel_centres", lambda shape: [r + 1 for r in good(shape)])
    _fails(pins_nudft.test_single_voxel)
    _fails(pins_nudft.test_hand_closed_forms)


def test_jacobian_sign_is_caught(monkeypatch):
    """+i r y instead of -i r y in the omega-Jacobian of the NUDFT."""
    good = nudft_mod.nudft_jac_omega
    monkeypatch.setattr(pins_nudft, "nudft_jac_omega", lambda x, om: -good(x, om))
    _fails(pins_nudft.test_jacobian_matches_central_differences)


def test_adjoint_without_conjugation_is_caught(monkeypatch):
    """A^T y (a transposed operand, no conjugate) instead of A^H y."""
    good = nudft_mod.nudft_adjoint
    monkeypatch.setattr(pins_nudft, "nudft_adjoint", lambda y, om, shape: np.conj(good(np.conj(y), om, shape)))
    _fails(pins_nudft.test_adjoint_identity)


# ---------------------------------------------------------------- same-kernel NUFFT, Appendix
def test_beta_typo_is_caught(monkeypatch):
    """(sigma + 1/2) in place of (sigma - 1/2) in Beatty's formula."""
    def bad_beta(J, sigma):
        return np.pi * np.sqrt((J / sigma) ** 2 * (sigma + 0.5) ** 2 - 0.8)
    monkeypatch.setattr(pins_nufft, "kb_beta", bad_beta)
    _fails(pins_nufft.test_beta_matches_hand_evaluated_values)


def test_dropped_scaling_is_caught(monkeypatch):
    """The deapodisation s_n left out of the image-side scaling."""
    monkeypatch.setattr(nufft_mod.KBNufft, "_scale_image", lambda self, x: np.asarray(x, np.complex128))
    _fails(pins_nufft.test_nufft_close_to_exact_nudft, (16, 24), 700)


def test_nufft_adjoint_transposed_is_caught(monkeypatch):
    """The NUFFT adjoint computed as A~^T y instead of A~^H y."""
    good = nufft_mod.KBNufft.adjoint
    monkeypatch.setattr(nufft_mod.KBNufft, "adjoint", lambda self, y: np.conj(good(self, np.conj(y))))
    _fails(pins_nufft.test_nufft_adjoint_identity)


def test_kernel_derivative_sign_is_caught(monkeypatch):
    """d psi / du with the wrong sign (the analytic-derivative variant of the autodiff baseline)."""
    good = nufft_mod.kb_kernel_deriv
    monkeypatch.setattr(pins_nufft, "kb_kernel_deriv", lambda u, J, beta: -good(u, J, beta))
    _fails(pins_nufft.test_kernel_derivative_matches_central_differences, 6, 2.0)


# ---------------------------------------------------------------- Jacobian products, Sec. II
def test_vjp_gradient_factor_two_is_caught(monkeypatch):
    """2 Re{...} with the PyTorch-convention v (the factor-2 reading of Eq. (e,jac,Ax,v))."""
    good = jacobian_mod.vjp_omega_x
    monkeypatch.setattr(jacobian_mod, "vjp_omega_x", lambda op, x, v, smaps=None: (2 * good(op, x, v, smaps)[0],
                                                                                  good(op, x, v, smaps)[1]))
    _fails(pins_jac.test_vjp_omega_matches_finite_differences)


def test_vjp_dropped_coil_is_caught(monkeypatch):
    """The coil sum of grad omega stopping one coil short."""
    good = jacobian_mod.vjp_omega_x

    def short(op, x, v, smaps=None):
        v2 = np.array(v, copy=True)
        v2[-1] = 0
        return good(op, x, v2, smaps)[0], good(op, x, v, smaps)[1]
    monkeypatch.setattr(jacobian_mod, "vjp_omega_x", short)
    _fails(pins_jac.test_vjp_omega_matches_finite_differences)


def test_jvp_sign_is_caught(monkeypatch):
    """+i in place of -i in the JVP (the sign typo of the SENSE forward in Sec. II-G)."""
    good = jacobian_mod.jvp_omega
    monkeypatch.setattr(jacobian_mod, "jvp_omega", lambda op, x, dom, smaps=None: -good(op, x, dom, smaps))
    _fails(pins_jac.test_jvp_omega_matches_finite_differences)


# ---------------------------------------------------------------- NUFFT geometry (Appendix)
def _retap(op, start_offset):
    """Rebuild the interpolation windows with k = floor(t - J/2) + start_offset + (0 .. J-1)."""
    op.taps = []
    for d in range(op.D):
        t = op.omega[d] * op.K[d] / (2.0 * np.pi)
        k = (np.floor(t - op.J / 2.0) + start_offset)[:, None] + np.arange(op.J)[None, :]
        u = t[:, None] - k
        op.taps.append((np.mod(k.astype(np.int64), op.K[d]), nufft_mod.kb_kernel(u, op.J, op.beta), u))


def test_window_off_by_one_is_caught(monkeypatch):
    """The window started one cell early (the '+ 1' of k = floor(t - J/2) + 1 dropped)."""
    good = nufft_mod.KBNufft.__init__

    def bad_init(self, *args, **kw):
        good(self, *args, **kw)
        _retap(self, 0.0)
    monkeypatch.setattr(nufft_mod.KBNufft, "__init__", bad_init)
    _fails(pins_nufft.test_nufft_close_to_exact_nudft, (16, 24), 700)


def test_image_not_wrapped_onto_the_grid_is_caught(monkeypatch):
    """The image placed at grid indices 0 .. N-1 instead of at r mod K (no centring wrap)."""
    good = nufft_mod.KBNufft.__init__

    def bad_init(self, *args, **kw):
        good(self, *args, **kw)
        self.place = [np.arange(n) for n in self.shape]
    monkeypatch.setattr(nufft_mod.KBNufft, "__init__", bad_init)
    _fails(pins_nufft.test_nufft_close_to_exact_nudft, (16, 24), 700)


def test_inverse_fft_in_the_forward_is_caught(monkeypatch):
    """K * IFFT (exponent +) in place of the forward FFT of step (2)."""
    ifftn = np.fft.ifftn

    def wrong(a, axes=None):
        n = int(np.prod([a.shape[i] for i in (axes if axes is not None else range(a.ndim))]))
        return ifftn(a, axes=axes) * n
    monkeypatch.setattr(nufft_mod.np.fft, "fftn", wrong)
    _fails(pins_nufft.test_nufft_close_to_exact_nudft, (16, 24), 700)


# ---------------------------------------------------------------- Gram and inverse Jacobians
def test_gram_vjp_dropped_term_is_caught(monkeypatch):
    """Eq. (e,A'A,x,omd) with its second term (+i diag{r} E' diag{E x}) left out."""
    def first_term_only(op, x, g, smaps=None):
        Eg = jacobian_mod.sense_forward(op, g, smaps)
        out = np.zeros((len(op.shape), op.omega.shape[1]))
        for d in range(len(op.shape)):
            Exr = jacobian_mod.sense_forward(op, np.asarray(x) * jacobian_mod._r_weight(op.shape, d), smaps)
            out[d] = np.sum(np.real(-1j * np.conj(Eg) * Exr), axis=0)
        return out
    monkeypatch.setattr(jacobian_mod, "gram_vjp_omega", first_term_only)
    _fails(pins_jac.test_gram_vjp_matches_finite_differences)


def test_psd_inverse_sign_is_caught(monkeypatch):
    """+ in place of the - of D F^-1 b = -F^-1 (D F) F^-1 b (Eq. (e,inv,omd))."""
    good = jacobian_mod.psd_inverse_vjp

    def wrong(op, E_dense, b, g, smaps=None, lam=1e-2):
        z, gb, go = good(op, E_dense, b, g, smaps, lam)
        return z, gb, -go
    monkeypatch.setattr(jacobian_mod, "psd_inverse_vjp", wrong)
    _fails(pins_jac.test_psd_inverse_vjp_matches_finite_differences)


# ---------------------------------------------------------------- table autodiff (Sec. IV-A)
def test_table_autodiff_missing_chain_factor_is_caught(monkeypatch):
    """The autodiff slope of the table model without du / d omega = K / (2 pi)."""
    import oracle.naive as naive_mod
    import test_oracle_naive as pins_naive
    good = naive_mod.TableNufft.__init__

    def bad_init(self, *args, **kw):
        good(self, *args, **kw)
        self.dtaps = [dt * (2.0 * np.pi / self.K[d]) for d, dt in enumerate(self.dtaps)]
    monkeypatch.setattr(naive_mod.TableNufft, "__init__", bad_init)
    _fails(pins_naive.test_table_jacobian_is_the_derivative_of_the_piecewise_linear_model)

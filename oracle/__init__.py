"""Plain, slow, FP64 CPU oracle for the NUFFT-Jacobian hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` use it.  It shares no code with the CUDA path
(no kernels, tables, constants or helpers); the only module both sides read is
the seeded input generator ``paper_2111_02912_gb300.workloads``, which holds none
of the method's arithmetic.

Modules
-------
``nudft``   exact non-uniform DFT A(omega) of Sec. II-B, Eq. (e,ndft), and its
            analytic Jacobians w.r.t. x and omega (Sec. II-C, Eq. (e,Ax);
            Sec. II-D, Eq. (e,A'y)).
``nufft``   the same-kernel NUFFT in FP64, taken step by step from the Appendix
            (scaling s_n, zero-padded K-point FFT, J-tap interpolation with
            coefficients u_j and offsets k_m), with a Kaiser-Bessel interpolator.
``jacobian`` multi-coil composition E = (I kron A) S (Sec. II-G) and the JVP /
            VJP products of Eq. (e,jac,Ax,v), generic over an operator pair.
``naive``   "method 1" of Sec. IV-A: autodiff through a NUFFT whose lookup
            table is linearly interpolated (floor derivatives taken as zero),
            reported beside the proposed method, never used as truth.

Every parity claim rests on the pins in ``tests/test_oracle_*.py``.
"""

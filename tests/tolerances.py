"""Tolerances of the complex64 path against the FP64 oracle, shared by the GPU tests.

complex64 rounds every stored amplitude to FP32 (unit roundoff u = 2^-24).  A level puts each
amplitude through one phase product and n RX butterflies, each rounded once per component, and
the rounding errors are carried on by norm-preserving maps.  After p levels one amplitude's
error is therefore a sum of about p (n + 2) independent roundings, each at most u times the
amplitudes it acts on, whose typical size is u sqrt(p (n + 2)) max|psi|.

  amplitude:  |psi_z - psi_ref,z| <= C64_AMP_K u sqrt(p (n + 2)) max|psi_ref|
"""
import math

import numpy as np

U32 = 2.0 ** -24

# An FP32 emulation of the complex64 arithmetic against the oracle reaches at most 0.85 of the
# model (n = 8..21, p up to 10); 16 leaves a margin of about 20 and still fails an amplitude that
# is wrong by more than 2e-5 of the largest one.
C64_AMP_K = 16.0


def c64_amp_tol(n: int, p: int, ref_psi) -> float:
    """Largest allowed |psi_z - psi_ref,z| of a complex64 run of p levels on n qubits."""
    return C64_AMP_K * U32 * math.sqrt(max(1, p) * (n + 2)) * float(np.max(np.abs(ref_psi)))


# The adjoint gradient holds psi and lambda and puts each through the same p (n + 2) rounded
# operations per amplitude, so the derivatives, sums of products of the two states, carry
# rounding errors of the same random-walk form over 2 p (n + 2) steps, in proportion to the
# derivatives' size, with a floor of one for the terms that cancel when the derivatives are
# small.  Measured against the oracle's FP64 adjoint (n = 2..24, p up to 10), the error is at
# most 3.6 of u sqrt(2 p (n + 2)) max(max|d|, 1); 16 leaves a margin above 4.
C64_GRAD_K = 16.0


def c64_grad_tol(n: int, p: int, m: int, scale: float) -> float:
    """Largest allowed error of a complex64 derivative of a p-level circuit on n qubits whose
    largest derivative (in magnitude) is `scale` (m, the edge count, is not part of the bound)."""
    del m
    return C64_GRAD_K * U32 * math.sqrt(2 * max(1, p) * (n + 2)) * max(float(scale), 1.0)


# Central differences of <C> in complex128 with step h: truncation h^2 |f'''| / 6 and rounding
# about 1e-13 |E| / h, together below 1e-6 at the gradient workload (measured 1.1e-8).
FD_TOL = 1e-6

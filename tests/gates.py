"""Tolerances shared by the parity tests.

FP64 path (acceleration parity): for every particle
    |a_gpu_i - a_oracle_i| <= 1e-12 |a_oracle_i| + 4 u sqrt(N) S_i,
with u = 2^-53 and S_i = G sum_j m_j |d_ij| / (d^2+eps^2)^{3/2} the sum of
the magnitudes of the terms (from the oracle).  The first term is the stated
1e-12 relative bound; the second is the rounding floor of any binary64
evaluation of an N-term sum in another order (probabilistic bound sqrt(N) u
per unit of S_i, with a factor 4 of margin); it only matters for particles
whose net force nearly cancels (|a_i| << S_i).  Potentials: the terms all
have one sign, so |pot_gpu - pot_oracle| <= 1e-12 |pot_oracle|.
"""
import numpy as np

U = 2.0 ** -53


def fp64_accel_gate(acc, acc_ref, smag, n, rel=1e-12):
    err = np.linalg.norm(np.asarray(acc) - acc_ref, axis=1)
    amag = np.linalg.norm(acc_ref, axis=1)
    tol = rel * amag + 4 * U * np.sqrt(n) * smag
    return err <= tol, err, amag


def rel_errors(acc, acc_ref):
    """Per-particle relative acceleration errors |da|/|a| (reduced-precision reporting)."""
    err = np.linalg.norm(np.asarray(acc) - acc_ref, axis=1)
    amag = np.linalg.norm(acc_ref, axis=1)
    return err / np.where(amag > 0, amag, 1.0)

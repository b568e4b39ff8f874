"""Lanczos estimate of the extreme eigenvalues of H -- TEST INFRASTRUCTURE ONLY.

The rescaling of Sec. 2.2 (H~ = H / s with the spectrum of H~ in [-1, 1]) needs
a bound on the spectral radius of H.  This is the plain Lanczos process
(Lanczos 1950; e.g. Golub & Van Loan, Matrix Computations, Sec. 10.1): from a
unit start vector q_1,
    w = H q_j - beta_j q_{j-1},  alpha_j = Re <q_j|w>,  w <- w - alpha_j q_j,
    beta_{j+1} = ||w||,  q_{j+1} = w / beta_{j+1},
and the extreme eigenvalues of the tridiagonal matrix T_m = tridiag(beta,
alpha, beta) are the extreme Ritz values, which lie inside the spectrum of H
and approach its ends.  H x is the C oracle's defining sum over the bond list;
T_m's eigenvalues come from SciPy's tridiagonal solver.

Start vector (the one the CUDA library draws, from the published SplitMix64
generator): q_u = (U_2u - 1/2) + i (U_2u+1 - 1/2), U_k the k-th uniform of
stream 200 of seed 220900806 (tbpm_inputs.rng), normalised.

Only tests/ may import this module.  Parity pinned by tests/test_oracle_lanczos.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from tbpm_inputs import rng

from . import apply_h

SEED = 220900806
STREAM = 200


def start_vector(n: int) -> np.ndarray:
    u = rng.uniform(SEED, STREAM, 2 * n)
    q = (u[0::2] - 0.5) + 1j * (u[1::2] - 0.5)
    return q / np.sqrt(np.sum(np.abs(q) ** 2))


def extremes(sample, n_iter: int) -> tuple[float, float, int]:
    """(smallest, largest) Ritz value of H in eV after n_iter Lanczos steps,
    and the steps taken (fewer when the Krylov space closes)."""
    q_prev = np.zeros(sample.n_orb, dtype=np.complex128)
    q = start_vector(sample.n_orb)
    alpha, beta = [], []
    b = 0.0
    for j in range(n_iter):
        w = apply_h(sample, 1.0, q) - b * q_prev          # H q_j - beta_j q_{j-1}
        a = float(np.real(np.vdot(q, w)))
        w = w - a * q
        alpha.append(a)
        b_next = float(np.sqrt(np.sum(np.abs(w) ** 2)))
        if j + 1 == n_iter or b_next <= 1e-12 * (abs(a) + b + 1e-300):
            break
        beta.append(b_next)
        q_prev, q, b = q, w / b_next, b_next
    ev = scipy.linalg.eigvalsh_tridiagonal(np.array(alpha), np.array(beta))
    return float(ev[0]), float(ev[-1]), len(alpha)

"""Pins of the quasi-eigenstate oracle (Sec. 2.6, Eq. quasi): the exact-
diagonalisation form of the windowed two-sided transform, and the recovery
of isolated eigenvectors."""
import math

import numpy as np
import pytest

import oracle
from oracle import quasi
from tbpm_inputs import lattice, rng

from . import exact

Z = math.pi / 2


@pytest.mark.parametrize("B", [0.0, 300.0])
def test_oracle_quasi_vs_exact_diagonalisation(B):
    smp = lattice.graphene(6, 5, pbc=False, seed=4, onsite_w=0.9, with_pos=True)
    if B:
        smp = lattice.peierls(smp, B)
    s, n = 9.0, 60
    psi0 = oracle.phase_states(rng.phases(9, 2, smp.n_orb))
    energies = np.array([-1.3, 0.2, 2.05])
    got, got_n = quasi.quasi_eigenstates(smp, s, Z, n, energies, psi0)
    E, U = np.linalg.eigh(exact.dense_h(smp))
    tau = Z / s
    m = np.arange(-n, n + 1)
    w = 0.5 * (1.0 + np.cos(np.pi * m / n))
    for k, e in enumerate(energies):
        filt = (np.exp(1j * np.outer(e - E, m * tau)) @ w) * tau / (2 * math.pi)   # [n_eig]
        for p in range(2):
            ref = U @ (filt * (U.conj().T @ psi0[p]))
            assert np.max(np.abs(got[k, p] - ref)) < 1e-12
            assert abs(np.linalg.norm(got_n[k, p]) - 1.0) < 1e-13


def test_oracle_quasi_recovers_isolated_eigenvectors():
    """A ring of 12 sites with onsite disorder has non-degenerate levels at
    least 0.1 eV apart; 1500 steps make the window much narrower than that,
    so the quasi-eigenstate at E_i is phi_i up to a phase."""
    smp = lattice.chain(12, t=-1.0, seed=3, onsite_w=2.0)
    E, U = np.linalg.eigh(exact.dense_h(smp))
    assert np.min(np.diff(E)) > 0.1
    psi0 = oracle.phase_states(rng.phases(10, 1, smp.n_orb))
    _, qn = quasi.quasi_eigenstates(smp, 3.5, Z, 1500, E[[2, 7]], psi0)
    for k, i in enumerate((2, 7)):
        assert abs(abs(np.vdot(U[:, i], qn[k, 0])) - 1.0) < 1e-3

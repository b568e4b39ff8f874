"""CPU FP64 oracle of the quasi-eigenstates -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may use this module (it is part of the ``oracle`` package, see
its header).  Sec. 2.6, Eq. quasi: |Psi(E)> = (1/2 pi) int e^{iEt} |psi(t)> dt
over positive and negative times, with a window on the finite interval,
then normalised.  Written out on the step grid t_n = n tau, n = -N .. N:

  Psi(E) = (tau / 2 pi) sum_{n=-N}^{N} w_n e^{i E n tau} psi(n tau),
  w_n = (1 + cos(pi n / N)) / 2   (Hann; w_{+-N} = 0, so the trapezoid end
                                    weights do not enter),
  Psi~(E) = Psi(E) / ||Psi(E)||,

psi(n tau) for n > 0 from the C oracle's forward propagation and for n < 0
from the same propagation under -H (e^{+iH|t|} = e^{-i(-H)|t|}).

Readings (kept with the design notes): the window is the Hann window of the
DOS path; both time directions are used (the first of the two improvements
the paper names), with the window as the second; normalisation to unit
norm per sample.

Parity pinned: against the exact-diagonalisation form
Psi(E) = (tau / 2 pi) sum_i <phi_i|psi0> phi_i sum_n w_n e^{i (E - E_i) n tau}
and by the recovery of isolated eigenvectors (tests ``test_oracle_quasi_*``).
"""
from __future__ import annotations

import math

import numpy as np

from . import propagate


def hann(n_steps: int) -> np.ndarray:
    """w_n for n = 0 .. N (even in n)."""
    n = np.arange(n_steps + 1)
    return 0.5 * (1.0 + np.cos(np.pi * n / n_steps))


def negated(sample):
    """The same sample with H -> -H."""
    from tbpm_inputs.lattice import Sample
    ons = None if sample.onsite is None else -np.asarray(sample.onsite)
    return Sample(n_orb=sample.n_orb, onsite=ons, hop_i=sample.hop_i, hop_j=sample.hop_j,
                  hop_v=-np.asarray(sample.hop_v), pos=sample.pos, meta=dict(sample.meta),
                  dr=sample.dr)


def quasi_eigenstates(sample, s: float, z: float, n_steps: int, energies, psi0):
    """(Psi [K, S, N] unnormalised, Psi~ [K, S, N] unit norm) for energies [K]
    (eV) and initial states psi0 [S, N]."""
    energies = np.atleast_1d(np.asarray(energies, dtype=np.float64))
    psi0 = np.atleast_2d(np.asarray(psi0, dtype=np.complex128))
    tau = z / s
    w = hann(n_steps)
    K, (S, N) = len(energies), psi0.shape
    acc = np.zeros((K, S, N), dtype=np.complex128)
    for k in range(K):
        acc[k] += w[0] * psi0
    for direction, smp in ((+1, sample), (-1, negated(sample))):
        psi = psi0.copy()
        for n in range(1, n_steps + 1):
            _, _, psi = propagate(smp, s, z, 1, psi, want_norms=True, want_psi=True)
            t = direction * n * tau
            for k in range(K):
                acc[k] += w[n] * np.exp(1j * energies[k] * t) * psi
    acc *= tau / (2.0 * math.pi)
    norm = np.sqrt(np.sum(np.abs(acc) ** 2, axis=-1, keepdims=True))
    return acc, acc / np.where(norm > 0, norm, 1.0)

"""Exact solutions used to pin the CPU oracle (test helpers, numpy only).

None of these go through the Chebyshev expansion: they reach the same
quantities by exact diagonalisation, the Bloch theorem or closed forms.
"""
from __future__ import annotations

import numpy as np


def dense_h(sample) -> np.ndarray:
    """Dense H (eV) from the bond list: H_ij = t, H_ji = conj(t), H_ii = eps_i."""
    n = sample.n_orb
    H = np.zeros((n, n), dtype=np.complex128)
    np.add.at(H, (sample.hop_i, sample.hop_j), sample.hop_v)
    np.add.at(H, (sample.hop_j, sample.hop_i), np.conj(sample.hop_v))
    if sample.onsite is not None:
        H[np.arange(n), np.arange(n)] += sample.onsite
    return H


def ed_corr(sample, psi0: np.ndarray, times: np.ndarray) -> np.ndarray:
    """C(t) = sum_n |<n|psi0>|^2 exp(-i E_n t) by exact diagonalisation."""
    E, U = np.linalg.eigh(dense_h(sample))
    w = np.abs(U.conj().T @ psi0) ** 2
    return np.exp(-1j * np.outer(times, E)) @ w


def ed_spectrum_weights(sample, psi0: np.ndarray):
    E, U = np.linalg.eigh(dense_h(sample))
    return E, np.abs(U.conj().T @ psi0) ** 2


def graphene_bloch(L1: int, L2: int, t: float):
    """Per k = 2 pi (q1/L1, q2/L2): h(k) = [[0, t f], [t f*, 0]],
    f = 1 + exp(-i k1) + exp(-i k2), for the numbering 2 (n1 L2 + n2) + o."""
    k1 = 2 * np.pi * np.arange(L1)[:, None] / L1
    k2 = 2 * np.pi * np.arange(L2)[None, :] / L2
    f = 1.0 + np.exp(-1j * k1) + np.exp(-1j * k2)
    return t * f


def graphene_bloch_corr(L1: int, L2: int, t: float, psi0: np.ndarray,
                        times: np.ndarray) -> np.ndarray:
    """Exact C(t) for pristine periodic graphene from the 2x2 Bloch blocks:
    exp(-i h t) = cos(|g| t) - i sin(|g| t) h / |g|, g = t f(k)."""
    x = psi0.reshape(L1, L2, 2)
    a = np.fft.fft2(x[:, :, 0])
    b = np.fft.fft2(x[:, :, 1])
    g = graphene_bloch(L1, L2, t)
    ag = np.abs(g)
    safe = np.where(ag > 0, ag, 1.0)
    out = np.empty(times.shape[0], dtype=np.complex128)
    for q, tt in enumerate(times):
        c = np.cos(ag * tt)
        s = np.where(ag > 0, np.sin(ag * tt) / safe, 0.0)
        a_t = c * a - 1j * s * g * b
        b_t = c * b - 1j * s * np.conj(g) * a
        out[q] = (np.vdot(a, a_t) + np.vdot(b, b_t)) / (L1 * L2)
    return out


def graphene_bloch_spectrum(L1, L2, t, psi0):
    """Eigenvalues +-|g(k)| and the weights |<n|psi0>|^2 of each."""
    x = psi0.reshape(L1, L2, 2)
    a = np.fft.fft2(x[:, :, 0]) / np.sqrt(L1 * L2)
    b = np.fft.fft2(x[:, :, 1]) / np.sqrt(L1 * L2)
    g = graphene_bloch(L1, L2, t)
    ag = np.abs(g)
    ph = np.where(ag > 0, g / np.where(ag > 0, ag, 1.0), 1.0)
    # eigenvectors (1, +-conj(ph)) / sqrt 2 of [[0, g], [g*, 0]]
    wp = np.abs(a + ph * b) ** 2 / 2
    wm = np.abs(a - ph * b) ** 2 / 2
    E = np.concatenate([ag.ravel(), -ag.ravel()])
    W = np.concatenate([wp.ravel(), wm.ravel()])
    return E, W


def windowed_dos_from_spectrum(E_n, w_n, n_steps, tau, energies):
    """The windowed DOS the oracle's formula gives for a correlation that is
    exactly sum_n w_n exp(-i E_n t): a sum of window kernels
    K(e) = (tau/pi) [1/2 + sum_{k=1}^{N-1} h_k cos(e k tau)], h_k Hann."""
    k = np.arange(1, n_steps)
    h = 0.5 * (1 + np.cos(np.pi * k / n_steps))
    out = np.zeros(energies.shape[0])
    for j, E in enumerate(energies):
        d = E - E_n
        ker = 0.5 + np.cos(np.outer(d, k * tau)) @ h
        out[j] = tau / np.pi * np.dot(w_n, ker)
    return out

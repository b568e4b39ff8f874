"""Pins of the oracle's adjoint: central finite differences of the oracle's
own forward map, the Daleckii-Krein derivative of the exact propagator by
exact diagonalisation, and the DOS adjoint against the DOS transform."""
import math

import numpy as np
import pytest

import oracle
from tbpm_inputs import lattice, rng

from . import exact

Z = math.pi / 2


def small_sample():
    return lattice.graphene(4, 4, pbc=True, seed=3, onsite_w=0.4, bond_sigma=0.05)


def linear_loss(sample, s, psi0, gbar, n_steps):
    c = oracle.propagate(sample, s, Z, n_steps, psi0)
    return float(np.sum((np.conj(gbar) * c).real))


def test_oracle_gradient_vs_central_differences():
    smp = small_sample()
    s, n_steps = 9.5, 25
    psi0 = oracle.phase_states(rng.phases(2, 2, smp.n_orb))
    gen = np.random.default_rng(4)
    gbar = gen.normal(size=(2, n_steps + 1)) + 1j * gen.normal(size=(2, n_steps + 1))
    gh, go = oracle.gradient(smp, s, Z, n_steps, psi0, gbar)
    h = 1e-6
    for b in (0, 7, 23, smp.n_hop - 1):
        plus = lattice.Sample(smp.n_orb, smp.onsite, smp.hop_i, smp.hop_j, smp.hop_v.copy())
        minus = lattice.Sample(smp.n_orb, smp.onsite, smp.hop_i, smp.hop_j, smp.hop_v.copy())
        plus.hop_v[b] += h
        minus.hop_v[b] -= h
        fd = (linear_loss(plus, s, psi0, gbar, n_steps)
              - linear_loss(minus, s, psi0, gbar, n_steps)) / (2 * h)
        assert abs(fd - gh[b]) < 1e-7 * max(1.0, abs(fd))
    for i in (0, 5, smp.n_orb - 1):
        plus = lattice.Sample(smp.n_orb, smp.onsite.copy(), smp.hop_i, smp.hop_j, smp.hop_v)
        minus = lattice.Sample(smp.n_orb, smp.onsite.copy(), smp.hop_i, smp.hop_j, smp.hop_v)
        plus.onsite[i] += h
        minus.onsite[i] -= h
        fd = (linear_loss(plus, s, psi0, gbar, n_steps)
              - linear_loss(minus, s, psi0, gbar, n_steps)) / (2 * h)
        assert abs(fd - go[i]) < 1e-7 * max(1.0, abs(fd))


def daleckii_krein_grad(sample, psi0, gbar, times):
    """dL/dH_ij of L = sum_n Re(conj(g_n) <psi0|exp(-i H t_n)|psi0>) from the
    divided differences of f(x) = exp(-i x t) in the eigenbasis of H."""
    H = exact.dense_h(sample)
    E, V = np.linalg.eigh(H)
    u = V.conj().T @ psi0
    dE = E[:, None] - E[None, :]
    same = np.abs(dE) < 1e-12
    G = np.zeros(H.shape, dtype=complex)
    for g, t in zip(gbar, times):
        f = np.exp(-1j * E * t)
        F = np.where(same, -1j * t * f[:, None], (f[:, None] - f[None, :]) / np.where(same, 1, dE))
        K = np.conj(u)[:, None] * u[None, :] * F
        dC = np.conj(V) @ K @ V.T            # dC/dH_ij
        G += np.conj(g) * dC
    return G.real + 0 * G.imag, G


def test_oracle_gradient_vs_daleckii_krein():
    smp = lattice.graphene(3, 4, pbc=True, seed=6, onsite_w=0.6, bond_sigma=0.05)
    s, n_steps = 9.5, 30
    psi0 = oracle.phase_states(rng.phases(8, 1, smp.n_orb))
    gen = np.random.default_rng(2)
    gbar = gen.normal(size=(1, n_steps + 1)) + 1j * gen.normal(size=(1, n_steps + 1))
    gh, go = oracle.gradient(smp, s, Z, n_steps, psi0, gbar)
    times = (Z / s) * np.arange(n_steps + 1)
    _, G = daleckii_krein_grad(smp, psi0[0], gbar[0], times)
    # dL/dt_b = Re(dL/dH_ij + dL/dH_ji); dL/deps_i = Re dL/dH_ii
    ref_h = (G[smp.hop_i, smp.hop_j] + G[smp.hop_j, smp.hop_i]).real
    ref_o = np.diag(G).real
    assert np.max(np.abs(gh - ref_h)) < 1e-10 * max(1, np.max(np.abs(ref_h)))
    assert np.max(np.abs(go - ref_o)) < 1e-10 * max(1, np.max(np.abs(ref_o)))


def test_oracle_dos_adjoint_is_the_transpose():
    gen = np.random.default_rng(0)
    n, tau, e0, e1, ne = 64, 0.17, -5.0, 5.0, 90
    c = gen.normal(size=n + 1) + 1j * gen.normal(size=n + 1)
    dl = gen.normal(size=ne)
    gbar = oracle.dos_adjoint(dl, n, tau, e0, e1)
    # the DOS is real-linear in C: <dl, D(dc)> = Re sum conj(gbar) dc
    for _ in range(3):
        dc = gen.normal(size=n + 1) + 1j * gen.normal(size=n + 1)
        _, d1 = oracle.dos(c + dc, tau, e0, e1, ne)
        _, d0 = oracle.dos(c, tau, e0, e1, ne)
        lhs = float(np.dot(dl, d1 - d0))
        rhs = float(np.sum((np.conj(gbar) * dc).real))
        assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))

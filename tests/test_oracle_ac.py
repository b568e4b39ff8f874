"""Pins of the AC-conductivity oracle (Sec. 2.2 Fermi-Dirac operator, Sec. 2.7
optical conductivity) to things other than itself: the closed-form Fermi
function, exact diagonalisation, the commutator form of the current
operator, and the closed-form time integral of a two-level correlation."""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C

import oracle
from oracle import ac
from tbpm_inputs import lattice, rng

from . import exact

Z = math.pi / 2


@pytest.mark.parametrize("beta_s,mu_s", [(40.0, 0.1), (350.0, -0.03), (5.0, 0.0)])
def test_oracle_ac_fermi_series_reproduces_f(beta_s, mu_s):
    c = ac.fermi_coefficients(beta_s, mu_s)
    x = np.random.default_rng(1).uniform(-1.0, 1.0, 500)
    series = C.chebval(x, np.concatenate([[0.5 * c[0]], c[1:]]))
    exact_f = 1.0 / (np.exp(beta_s * (x - mu_s)) + 1.0)
    assert np.max(np.abs(series - exact_f)) < 1e-13
    # a sharper distribution needs more terms
    if beta_s > 100:
        assert len(c) > len(ac.fermi_coefficients(40.0, mu_s))


def _flake(B=0.0, n=(7, 6)):
    smp = lattice.graphene(*n, pbc=False, seed=12, onsite_w=0.8, with_pos=True)
    return lattice.peierls(smp, B) if B else smp


@pytest.mark.parametrize("B", [0.0, 400.0])
def test_oracle_ac_fermi_operator_vs_exact_diagonalisation(B):
    smp = _flake(B)
    s, beta, mu = 9.0, 4.0, 0.3
    E, U = np.linalg.eigh(exact.dense_h(smp))
    v = oracle.phase_states(rng.phases(5, 1, smp.n_orb))[0]
    ref = U @ (ac.fermi(E, beta, mu) * (U.conj().T @ v))
    got = ac.fermi_apply(smp, s, beta * s, mu / s, v)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("B", [0.0, 400.0])
def test_oracle_ac_current_is_commutator(B):
    """J_a = -i [H, X_a] (the hopping form of the current, Sec. 2.7): built
    here from the dense H and the diagonal position operator."""
    smp = _flake(B)
    H = exact.dense_h(smp)
    v = oracle.phase_states(rng.phases(6, 1, smp.n_orb))[0]
    u = oracle.phase_states(rng.phases(7, 1, smp.n_orb))[0]
    for a in range(2):
        X = np.diag(smp.pos[:, a])
        ref = -1j * (H @ X - X @ H) @ v
        got = ac.current_apply(smp, lattice.bond_vectors(smp)[:, a], v)
        assert np.max(np.abs(got - ref)) < 1e-13
        # Hermitian
        lhs = np.vdot(u, got)
        rhs = np.vdot(ac.current_apply(smp, lattice.bond_vectors(smp)[:, a], u), v)
        assert abs(lhs - rhs) < 1e-13


@pytest.mark.parametrize("B", [0.0, 400.0])
def test_oracle_ac_correlation_vs_exact_diagonalisation(B):
    smp = _flake(B)
    s, beta, mu, n_steps = 9.0, 6.0, -0.2, 40
    psi0 = oracle.phase_states(rng.phases(8, 2, smp.n_orb))
    got = ac.ac_correlation(smp, s, Z, n_steps, beta, mu, lattice.bond_vectors(smp), psi0)
    H = exact.dense_h(smp)
    E, U = np.linalg.eigh(H)
    f = U @ np.diag(ac.fermi(E, beta, mu)) @ U.conj().T
    J = [-1j * (H @ np.diag(smp.pos[:, a]) - np.diag(smp.pos[:, a]) @ H) for a in range(2)]
    one = np.eye(smp.n_orb)
    for p in range(2):
        for n in (0, 1, 17, 40):
            Ut = U @ np.diag(np.exp(-1j * E * (Z / s) * n)) @ U.conj().T
            psi2 = Ut @ f @ psi0[p]
            for a in range(2):
                for b in range(2):
                    psi1 = Ut @ (one - f) @ J[b] @ psi0[p]
                    ref = np.vdot(psi2, J[a] @ psi1)
                    assert abs(got[p, 2 * a + b, n] - ref) < 1e-11


def test_oracle_ac_conductivity_integral_closed_form():
    """C(t) = A e^{i D t}: the damped sine transform has a closed form."""
    A, D, tau, n, eta, beta = 0.3 - 0.7j, 1.3, 1e-3, 20000, 0.2, 2.0
    t = tau * np.arange(n + 1)
    corr = A * np.exp(1j * D * t)
    om = np.array([0.4, 1.1, 2.5])
    got = ac.ac_conductivity(corr[None, :], tau, beta, eta, om, norm=3.0)[0]
    T = n * tau

    def damped_cos(nu):        # int_0^T e^{-eta t} cos(nu t) dt
        return np.real((1.0 - np.exp((-eta + 1j * nu) * T)) / (eta - 1j * nu))

    def damped_sin(nu):        # int_0^T e^{-eta t} sin(nu t) dt
        return np.imag((1.0 - np.exp((-eta + 1j * nu) * T)) / (eta - 1j * nu))

    for k, w in enumerate(om):
        # 2 Im(A e^{iDt}) = 2 (Im A cos Dt + Re A sin Dt); products of sines/cosines
        i_sc = 0.5 * (damped_sin(w + D) + damped_sin(w - D))     # sin(wt) cos(Dt)
        i_ss = 0.5 * (damped_cos(w - D) - damped_cos(w + D))     # sin(wt) sin(Dt)
        integral = 2.0 * (A.imag * i_sc + A.real * i_ss)
        ref = 3.0 * (np.exp(-beta * w) - 1.0) / w * integral
        assert abs(got[k] - ref) < 1e-6 * max(1.0, abs(ref))

"""The pins of the Python-level oracles (AC conductivity, quasi-eigenstates,
DOS windows) catch plausible mistakes.  Each case loads a copy of the oracle
module with one mistake planted by a textual edit (the committed oracle is
never touched) and checks that the pin which should notice it does: exact
diagonalisation, the commutator form of the current, the exact-
diagonalisation form of the quasi-eigenstates, or a closed form."""
import importlib.util
import math
import sys
from pathlib import Path

import numpy as np
import pytest

import oracle
from tbpm_inputs import lattice, rng

from . import exact

ORACLE = Path(oracle.__file__).resolve().parent
Z = math.pi / 2


def mutant(module: str, old: str, new: str):
    src = (ORACLE / f"{module}.py").read_text()
    assert src.count(old) == 1, f"anchor for {module} not unique"
    name = f"oracle._mut_{module}"
    spec = importlib.util.spec_from_loader(name, loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    sys.modules[name] = mod
    exec(compile(src.replace(old, new), str(ORACLE / f"{module}.py"), "exec"), mod.__dict__)
    return mod


def flake(B=0.0):
    smp = lattice.graphene(6, 5, pbc=False, seed=12, onsite_w=0.8, with_pos=True)
    return lattice.peierls(smp, B) if B else smp


def fermi_error(ac, smp):
    s, beta, mu = 9.0, 4.0, 0.3
    E, U = np.linalg.eigh(exact.dense_h(smp))
    v = oracle.phase_states(rng.phases(5, 1, smp.n_orb))[0]
    ref = U @ (ac.fermi(E, beta, mu) * (U.conj().T @ v))
    return np.max(np.abs(ac.fermi_apply(smp, s, beta * s, mu / s, v) - ref))


def current_error(ac, smp):
    H = exact.dense_h(smp)
    v = oracle.phase_states(rng.phases(6, 1, smp.n_orb))[0]
    X = np.diag(smp.pos[:, 0])
    return np.max(np.abs(ac.current_apply(smp, lattice.bond_vectors(smp)[:, 0], v)
                         - (-1j * (H @ X - X @ H) @ v)))


def ac_corr_error(ac, smp):
    s, beta, mu, n = 9.0, 6.0, -0.2, 6
    psi0 = oracle.phase_states(rng.phases(8, 1, smp.n_orb))
    got = ac.ac_correlation(smp, s, Z, n, beta, mu, lattice.bond_vectors(smp), psi0)
    H = exact.dense_h(smp)
    E, U = np.linalg.eigh(H)
    f = U @ np.diag(ac.fermi(E, beta, mu)) @ U.conj().T
    J = -1j * (H @ np.diag(smp.pos[:, 0]) - np.diag(smp.pos[:, 0]) @ H)
    Ut = U @ np.diag(np.exp(-1j * E * (Z / s) * n)) @ U.conj().T
    ref = np.vdot(Ut @ f @ psi0[0], J @ (Ut @ (np.eye(smp.n_orb) - f) @ J @ psi0[0]))
    return abs(got[0, 0, n] - ref)


def quasi_error(quasi, smp):
    s, n, e = 9.0, 30, 0.2
    psi0 = oracle.phase_states(rng.phases(9, 1, smp.n_orb))
    got, _ = quasi.quasi_eigenstates(smp, s, Z, n, [e], psi0)
    E, U = np.linalg.eigh(exact.dense_h(smp))
    tau = Z / s
    m = np.arange(-n, n + 1)
    w = 0.5 * (1.0 + np.cos(np.pi * m / n))
    filt = (np.exp(1j * np.outer(e - E, m * tau)) @ w) * tau / (2 * math.pi)
    return np.max(np.abs(got[0, 0] - U @ (filt * (U.conj().T @ psi0[0]))))


def test_unmutated_python_oracles_pass_the_pins():
    from oracle import ac, quasi
    assert fermi_error(ac, flake()) < 1e-12
    assert current_error(ac, flake(400.0)) < 1e-13
    assert ac_corr_error(ac, flake()) < 1e-11
    assert quasi_error(quasi, flake(300.0)) < 1e-12


def test_fermi_series_without_half_c0_caught_by_exact_diagonalisation():
    ac = mutant("ac", "acc = 0.5 * c[0] * t_prev", "acc = c[0] * t_prev")
    assert fermi_error(ac, flake()) > 1e-3


def test_current_without_conjugate_partner_caught_by_commutator():
    ac = mutant("ac", "np.add.at(y, j, -1j * np.conj(t) * (-d) * v[i])",
                "np.add.at(y, j, -1j * t * (-d) * v[i])")
    assert current_error(ac, flake(400.0)) > 1e-6


def test_f_instead_of_one_minus_f_caught_by_exact_diagonalisation():
    ac = mutant("ac", "psi1.append(jb - fermi_apply(sample, s, beta_s, mu_s, jb))",
                "psi1.append(fermi_apply(sample, s, beta_s, mu_s, jb))")
    assert ac_corr_error(ac, flake()) > 1e-6


def test_quasi_without_negative_times_caught_by_exact_diagonalisation():
    quasi = mutant("quasi", "for direction, smp in ((+1, sample), (-1, negated(sample))):",
                   "for direction, smp in ((+1, sample),):")
    assert quasi_error(quasi, flake(300.0)) > 1e-6


@pytest.mark.parametrize("old,new", [
    ("w = np.exp(-4.0 * x)", "w = np.exp(-2.0 * x)"),
    ("d[k] = tau / np.pi * (0.5 * c[0].real", "d[k] = tau / np.pi * (c[0].real"),
])
def test_window_mistakes_caught_by_the_geometric_closed_form(old, new):
    windows = mutant("windows", old, new)
    N, tau, E0 = 500, 0.11, 0.77
    c = np.exp(-1j * E0 * tau * np.arange(N + 1))
    en, d = windows.dos(c, tau, -3.0, 3.0, 257, windows.EXPONENTIAL)
    q = math.exp(-4.0 / N) * np.exp(1j * (en - E0) * tau)
    ref = tau / math.pi * (0.5 + (q * (1 - q ** (N - 1)) / (1 - q)).real + 0.5 * (q ** N).real)
    assert np.max(np.abs(d - ref)) > 1e-6

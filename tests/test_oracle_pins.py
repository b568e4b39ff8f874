"""Pins of the CPU oracle against results it does not compute itself:
SciPy's Bessel functions and the Neumann sum rules, exact diagonalisation,
the dimer closed form, the Bloch solution of pristine graphene, the matrix
exponential, and the invariants of unitary evolution and of the DOS."""
import json
import math
from pathlib import Path

import numpy as np
import pytest
import scipy.linalg
import scipy.special

import oracle
from tbpm_inputs import lattice, rng, workloads

from . import exact

Z = math.pi / 2


# ---- Bessel table (Sec. 2.2, expansion of exp(-i z x)) ----------------------

@pytest.mark.parametrize("z", [0.1, 0.5, 1.0, math.pi / 2, 2.0, math.pi, 4.0])
def test_oracle_bessel_vs_scipy(z):
    J = oracle.bessel(z, 40)
    ref = scipy.special.jv(np.arange(41), z)
    assert np.max(np.abs(J - ref)) <= 2e-16 * max(1.0, math.exp(z) / 10)


@pytest.mark.parametrize("z", [0.3, math.pi / 2, math.pi, 3.7])
def test_oracle_bessel_sum_rules(z):
    J = oracle.bessel(z, 60)
    # generating function at x = 1: 1 = J_0 + 2 sum_k J_2k ; Parseval: 1 = J_0^2 + 2 sum J_m^2
    assert abs(J[0] + 2 * J[2::2].sum() - 1.0) < 1e-15
    assert abs(J[0] ** 2 + 2 * (J[1:] ** 2).sum() - 1.0) < 1e-15
    # exp(-i z x) at x = cos(a): J_0 + 2 sum (-i)^m J_m cos(m a)
    a = 0.7
    m = np.arange(1, 61)
    val = J[0] + 2 * np.sum((-1j) ** m * J[1:] * np.cos(m * a))
    assert abs(val - np.exp(-1j * z * math.cos(a))) < 1e-15


def test_oracle_n_terms():
    for z in (0.5, Z, math.pi, 3.9):
        ref = next(m for m in range(200) if m > z and abs(scipy.special.jv(m, z)) < 1e-15)
        assert oracle.n_terms(z) == ref
    assert oracle.n_terms(Z) == 16          # 15 sparse products per step at z = pi/2
    assert oracle.n_terms(math.pi) == 21


def test_oracle_bessel_refuses_large_z():
    with pytest.raises(ValueError):
        oracle.bessel(6.0, 10)


# ---- Hamiltonian action (Sec. 2.1) --------------------------------------------

def test_graphene_geometry_matches_printed_cell():
    g = json.loads((Path(__file__).parent / "golden" / "graphene_primitive_cell.json").read_text())
    a = np.array(g["lattice_vectors_nm"])
    assert np.allclose(lattice.A1, a[0, :2]) and np.allclose(lattice.A2, a[1, :2])
    frac = np.array(g["orbitals_fractional"])[:, :2]
    assert np.allclose(frac[1], [1 / 3, 1 / 3], atol=1e-5)
    assert all(h["energy_eV"] == lattice.T_NN for h in g["hoppings"])
    smp = lattice.graphene(4, 5, pbc=True, with_pos=True)
    # every generated bond is a nearest-neighbour pair 0.142 nm apart (mod PBC)
    d = smp.pos[smp.hop_j] - smp.pos[smp.hop_i]
    box = np.array([4 * lattice.A1, 5 * lattice.A2])
    best = np.full(d.shape[0], np.inf)
    for u in (-1, 0, 1):
        for v in (-1, 0, 1):
            best = np.minimum(best, np.linalg.norm(d + u * box[0] + v * box[1], axis=1))
    assert np.allclose(best, np.linalg.norm(lattice.A1 + lattice.A2) / 3, atol=1e-5)
    # the three printed hoppings per cell, as (R, i -> j)
    assert smp.n_hop == 3 * 20
    assert np.all(smp.hop_i[0::3] % 2 == 0) and np.all(smp.hop_j[0::3] % 2 == 1)
    assert np.all(smp.hop_i[1::3] % 2 == 1) and np.all(smp.hop_j[1::3] % 2 == 0)


def test_oracle_apply_h_bloch_eigenvector():
    L1, L2, t = 6, 7, -2.7
    smp = lattice.graphene(L1, L2)
    q1, q2 = 2, 3
    k1, k2 = 2 * np.pi * q1 / L1, 2 * np.pi * q2 / L2
    g = exact.graphene_bloch(L1, L2, t)[q1, q2]
    n1, n2 = np.meshgrid(np.arange(L1), np.arange(L2), indexing="ij")
    wave = np.exp(1j * (k1 * n1 + k2 * n2)).ravel()
    for sign in (+1, -1):
        x = np.empty(2 * L1 * L2, dtype=complex)
        x[0::2] = wave
        x[1::2] = sign * np.conj(g) / abs(g) * wave
        y = oracle.apply_h(smp, 1.0, x)
        assert np.allclose(y, sign * abs(g) * x, atol=1e-12)


def test_oracle_apply_h_hermitian_and_scaled():
    smp = lattice.random_graph(50, 120, seed=3)
    smp.hop_v = smp.hop_v * np.exp(1j * np.linspace(0, 3, smp.n_hop))   # complex hoppings
    gen = np.random.default_rng(0)
    x = gen.normal(size=50) + 1j * gen.normal(size=50)
    y = gen.normal(size=50) + 1j * gen.normal(size=50)
    Hx = oracle.apply_h(smp, 2.0, x)
    Hy = oracle.apply_h(smp, 2.0, y)
    assert abs(np.vdot(y, Hx) - np.vdot(Hy, x)) < 1e-12
    assert np.allclose(Hx, exact.dense_h(smp) @ x / 2.0, atol=1e-13)


def test_oracle_gershgorin():
    smp = lattice.graphene(8, 8, seed=1, onsite_w=1.0)
    g = oracle.gershgorin(smp)
    H = exact.dense_h(smp)
    assert abs(g - np.max(np.abs(H).sum(axis=1))) < 1e-12
    assert g >= np.max(np.abs(np.linalg.eigvalsh(H))) - 1e-12


# ---- propagation and correlation (Sec. 2.2) -------------------------------

@pytest.mark.parametrize("gamma", [-2.7, 1.3])
def test_oracle_dimer_closed_form(gamma):
    smp = lattice.dimer(gamma)
    s = 3.0
    tau = Z / s
    n = 200
    times = tau * np.arange(n + 1)
    c = oracle.propagate(smp, s, Z, n, np.array([[1.0, 0.0]], dtype=complex))
    # truncation (|J_16| ~ 1e-15) plus rounding per step, 200 steps
    assert np.max(np.abs(c[0] - np.cos(gamma * times))) < 1e-12
    al, be = 0.4, 2.9
    psi0 = np.array([[np.exp(1j * al), np.exp(1j * be)]]) / math.sqrt(2)
    c = oracle.propagate(smp, s, Z, n, psi0)
    ref = np.cos(gamma * times) - 1j * math.cos(al - be) * np.sin(gamma * times)
    assert np.max(np.abs(c[0] - ref)) < 1e-12


def test_oracle_one_step_vs_expm():
    smp = lattice.random_graph(120, 300, seed=5, onsite_w=1.0, t_scale=1.5)
    H = exact.dense_h(smp)
    s = 1.05 * np.max(np.abs(np.linalg.eigvalsh(H)))
    th = rng.phases(7, 2, smp.n_orb)
    psi0 = oracle.phase_states(th)
    _, _, psi = oracle.propagate(smp, s, Z, 1, psi0, want_norms=True, want_psi=True)
    U = scipy.linalg.expm(-1j * H * (Z / s))
    for p in range(2):
        assert np.linalg.norm(psi[p] - U @ psi0[p]) < 1e-13


@pytest.mark.parametrize("kind", ["disordered_vacancies", "random_graph", "magnetic_flake"])
def test_oracle_corr_vs_exact_diagonalisation(kind):
    if kind == "disordered_vacancies":
        smp = lattice.graphene(12, 10, pbc=True, seed=11, onsite_w=1.0, vacancy_frac=0.03)
        s = 9.5
    elif kind == "magnetic_flake":
        # complex hoppings: Peierls phases of a 250 T field (Sec. 2.1)
        smp = lattice.peierls(lattice.graphene(12, 10, pbc=False, seed=11, onsite_w=1.0,
                                               vacancy_frac=0.03, with_pos=True), 250.0)
        s = 9.5
    else:
        smp = lattice.random_graph(300, 700, seed=2, onsite_w=2.0)
        s = 1.02 * max(np.abs(np.linalg.eigvalsh(exact.dense_h(smp))))
    th = rng.phases(21, 2, smp.n_orb)
    psi0 = oracle.phase_states(th)
    n = 300
    corr, norms = oracle.propagate(smp, s, Z, n, psi0, want_norms=True)
    times = (Z / s) * np.arange(n + 1)
    for p in range(2):
        ref = exact.ed_corr(smp, psi0[p], times)
        assert np.max(np.abs(corr[p] - ref)) < 1e-12
        assert np.max(np.abs(norms[p] - 1.0)) < 1e-13


def test_oracle_corr_graphene_bloch_exact():
    """Pristine 64x64 periodic graphene (8192 orbitals) against the Bloch
    solution, every one of 1024 steps."""
    w = workloads.graphene_dos()
    psi0 = oracle.phase_states(w.thetas()[0])
    corr = oracle.propagate(w.sample, w.s, w.z, w.n_steps, psi0)
    times = w.tau * np.arange(w.n_steps + 1)
    ref = exact.graphene_bloch_corr(64, 64, lattice.T_NN, psi0[0], times)
    assert abs(corr[0, 0] - 1.0) < 1e-14
    assert np.max(np.abs(corr[0] - ref)) < 1e-11


def test_oracle_time_reversal():
    """C(-t) = conj C(t): propagating with -H equals propagating backwards."""
    smp = lattice.graphene(6, 6, seed=4, onsite_w=0.8)
    neg = lattice.Sample(smp.n_orb, -smp.onsite, smp.hop_i, smp.hop_j, -smp.hop_v)
    psi0 = oracle.phase_states(rng.phases(3, 1, smp.n_orb))
    cf = oracle.propagate(smp, 9.0, Z, 50, psi0)
    cb = oracle.propagate(neg, 9.0, Z, 50, psi0)
    assert np.max(np.abs(cb - np.conj(cf))) < 1e-13


def test_oracle_energy_conserved():
    smp = lattice.graphene(6, 6, seed=4, onsite_w=0.8, vacancy_frac=0.05)
    psi0 = oracle.phase_states(rng.phases(3, 1, smp.n_orb))
    _, _, psi = oracle.propagate(smp, 9.0, Z, 40, psi0, want_norms=True, want_psi=True)
    e0 = np.vdot(psi0[0], oracle.apply_h(smp, 1.0, psi0[0]))
    e1 = np.vdot(psi[0], oracle.apply_h(smp, 1.0, psi[0]))
    assert abs(e1 - e0) < 1e-12


# ---- DOS (Sec. 2.4) -----------------------------------------------------------

def test_oracle_dos_single_level_closed_form():
    """C_n = exp(-i E0 n tau): the peak at E0 is N tau / (2 pi) (Hann weights
    sum to (N-1)/2) and the area over one period is exactly 1."""
    N, tau, E0 = 256, 0.2, 1.234
    c = np.exp(-1j * E0 * tau * np.arange(N + 1))
    de = 2 * math.pi / tau / 4096
    en, d = oracle.dos(c, tau, E0 - 0.5 * de, E0 + 0.5 * de, 1)
    assert abs(d[0] - N * tau / (2 * math.pi)) < 1e-10
    en, d = oracle.dos(c, tau, -math.pi / tau, math.pi / tau, 4096)
    assert abs(d.sum() * de - 1.0) < 1e-12
    assert abs(en[0] - (-math.pi / tau + de / 2)) < 1e-12


def test_oracle_dos_graphene_vs_bloch_spectrum():
    L, n = 24, 256
    w = workloads.graphene_dos(L=L, n_steps=n, n_energies=300)
    psi0 = oracle.phase_states(w.thetas()[0])
    corr = oracle.propagate(w.sample, w.s, w.z, n, psi0)
    en, d = oracle.dos(corr[0], w.tau, *w.e_range, w.n_energies)
    E, W = exact.graphene_bloch_spectrum(L, L, lattice.T_NN, psi0[0])
    assert abs(W.sum() - 1.0) < 1e-12
    ref = exact.windowed_dos_from_spectrum(E, W, n, w.tau, en)
    assert np.max(np.abs(d - ref)) < 1e-9
    # area over [-s, s] is 1 up to the window's leakage
    assert abs(d.sum() * (en[1] - en[0]) - 1.0) < 1e-3


@pytest.mark.parametrize("kind", ["disordered", "complex"])
def test_oracle_row_parallel_twin_equals_the_serial_oracle(kind):
    """The OpenMP-over-rows twin (the paper's thread scheme) performs the
    serial oracle's operations row by row: bit-identical states; its blocked
    compensated sums give C and norms within one rounding."""
    smp = lattice.graphene(150, 149, pbc=True, seed=4, onsite_w=1.0, vacancy_frac=0.02)
    if kind == "complex":
        smp = lattice.peierls(lattice.graphene(90, 80, pbc=False, seed=4, onsite_w=0.6,
                                               with_pos=True), 150.0)
    th = rng.phases(8, 2, smp.n_orb)           # > 65,536 rows: several sum blocks
    psi0 = oracle.phase_states(th)
    a = oracle.propagate(smp, 9.5, Z, 12, psi0, want_norms=True, want_psi=True)
    b = oracle.propagate_rows(smp, 9.5, Z, 12, psi0, want_norms=True, want_psi=True)
    assert np.array_equal(a[2], b[2])
    assert np.max(np.abs(a[0] - b[0])) < 1e-15
    assert np.max(np.abs(a[1] - b[1])) < 1e-15
    assert oracle.threads() >= 1

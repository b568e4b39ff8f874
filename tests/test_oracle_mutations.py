"""The oracle's pins catch plausible mistakes.  Each case copies the oracle
source, plants one mistake by a textual edit (the committed oracle is never
touched), builds the copy, and checks that the pin which should notice it
does: exact diagonalisation, the dimer closed form, Hermiticity, or the DOS
single-level closed form."""
import ctypes
import math
import subprocess

import numpy as np
import pytest

import oracle
from tbpm_inputs import lattice, rng

from . import exact

Z = math.pi / 2

MUTATIONS = {
    # recurrence T_{m+1} = -2i H T_m + T_{m-1}: wrong sign of the i
    "recurrence_sign": ("t2[i] = -2.0 * I * t2[i] + t0[i];", "t2[i] = 2.0 * I * t2[i] + t0[i];"),
    # recurrence: dropped T_{m-1}
    "recurrence_dropped_term": ("t2[i] = -2.0 * I * t2[i] + t0[i];", "t2[i] = -2.0 * I * t2[i];"),
    # expansion weights 2 J_m for m >= 2 written as J_m
    "missing_factor_two": ("acc[i] += 2.0 * J[m] * t2[i];", "acc[i] += J[m] * t2[i];"),
    # first-order term -i H written as +i H
    "first_term_sign": ("t1[i] *= -I;", "t1[i] *= I;"),
    # conjugate element of a bond not conjugated
    "missing_conjugate": ("y[j] += conj(t) * x[i];", "y[j] += t * x[i];"),
    # transposed operand in H x
    "transposed_index": ("y[i] += t * x[j];", "y[i] += t * x[i];"),
    # correlation without the conjugate of psi0
    "correlation_no_conj": ("double complex v = conj(a[i]) * phi[i];",
                            "double complex v = a[i] * phi[i];"),
    # DOS: the n = 0 sample counted with full weight
    "dos_half_weight": ("double sum = 0.5 * creal(corr[0]);", "double sum = creal(corr[0]);"),
}


def build_mutant(name, tmp_path):
    src = (oracle._SRC).read_text()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = tmp_path / f"mut_{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"libmut_{name}.so"
    subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-D_GNU_SOURCE", "-o", str(so),
                    str(path), "-lm"], check=True)
    return so


@pytest.fixture
def mutant(tmp_path, monkeypatch):
    def make(name):
        lib_ok = oracle._load()
        lib = ctypes.CDLL(str(build_mutant(name, tmp_path)))
        for fn in ("oracle_bessel", "oracle_n_terms", "oracle_apply_h", "oracle_gershgorin",
                   "oracle_phase_state", "oracle_propagate", "oracle_dos"):
            f, g = getattr(lib, fn), getattr(lib_ok, fn)
            f.argtypes, f.restype = g.argtypes, g.restype
        monkeypatch.setattr(oracle, "_lib", lib)
        return lib
    return make


def ed_error(complex_hops=False):
    smp = lattice.graphene(5, 6, pbc=True, seed=3, onsite_w=1.0)
    if complex_hops:
        smp.hop_v = smp.hop_v * np.exp(0.3j * np.arange(smp.n_hop))
    psi0 = oracle.phase_states(rng.phases(2, 1, smp.n_orb))
    corr = oracle.propagate(smp, 9.5, Z, 40, psi0)
    ref = exact.ed_corr(smp, psi0[0], (Z / 9.5) * np.arange(41))
    return np.max(np.abs(corr[0] - ref))


def test_unmutated_oracle_passes_the_pins():
    assert ed_error() < 1e-12
    assert ed_error(complex_hops=True) < 1e-12


@pytest.mark.parametrize("name", ["recurrence_sign", "recurrence_dropped_term",
                                  "missing_factor_two", "first_term_sign",
                                  "transposed_index", "correlation_no_conj"])
def test_mutation_caught_by_exact_diagonalisation(mutant, name):
    mutant(name)
    assert ed_error() > 1e-6


def test_missing_conjugate_caught_with_complex_hoppings(mutant):
    mutant("missing_conjugate")
    assert ed_error(complex_hops=True) > 1e-6


def test_dos_weight_caught_by_single_level_closed_form(mutant):
    mutant("dos_half_weight")
    N, tau, E0 = 256, 0.2, 1.234
    c = np.exp(-1j * E0 * tau * np.arange(N + 1))
    de = 2 * math.pi / tau / 4096
    _, d = oracle.dos(c, tau, -math.pi / tau, math.pi / tau, 4096)
    assert abs(d.sum() * de - 1.0) > 1e-3

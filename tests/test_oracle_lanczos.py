"""Pins of the oracle's Lanczos spectral bound (oracle/lanczos.py) to exact
eigenvalues: the dimer (two steps span the space), a random graph run to
full length, and pristine periodic graphene, whose band edges are +-3|t|
exactly (the Gamma point)."""
import numpy as np
import pytest

from oracle import lanczos
from tbpm_inputs import lattice

from . import exact


def test_lanczos_dimer_closed_form():
    lo, hi, m = lanczos.extremes(lattice.dimer(1.7), 10)
    assert m == 2 and abs(lo + 1.7) < 1e-14 and abs(hi - 1.7) < 1e-14


@pytest.mark.parametrize("seed", [5, 6])
def test_lanczos_full_length_equals_eigvalsh(seed):
    g = lattice.random_graph(120, 300, seed=seed, onsite_w=1.0)
    ev = np.linalg.eigvalsh(exact.dense_h(g))
    lo, hi, _ = lanczos.extremes(g, 120)
    assert abs(lo - ev[0]) < 1e-9 and abs(hi - ev[-1]) < 1e-9


def test_lanczos_graphene_band_edges():
    """Ritz values stay inside [-8.1, 8.1] eV and reach the edges."""
    g = lattice.graphene(24, 24, pbc=True)
    for m, tol in ((32, 2e-3), (64, 1e-9)):
        lo, hi, _ = lanczos.extremes(g, m)
        assert -8.1 * (1 + 1e-12) <= lo < hi <= 8.1 * (1 + 1e-12)
        assert hi > 8.1 * (1 - tol) and lo < -8.1 * (1 - tol)


def test_lanczos_start_vector_is_the_published_generator():
    q = lanczos.start_vector(1000)
    assert abs(np.sum(np.abs(q) ** 2) - 1) < 1e-14
    from tbpm_inputs import rng
    u = rng.u64(220900806, 200, np.arange(4, dtype=np.uint64))
    raw = (u >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 - 0.5
    assert np.allclose(q[:2] / q[0] * (raw[0] + 1j * raw[1]), raw[0::2] + 1j * raw[1::2])


def test_lanczos_mutation_without_three_term_recurrence_fails_the_pin():
    """A copy of the oracle's loop with a planted mistake -- the beta_j q_{j-1}
    term dropped -- misses the random graph's ends: the pin above catches it."""
    import scipy.linalg
    g = lattice.random_graph(120, 300, seed=5, onsite_w=1.0)
    ev = np.linalg.eigvalsh(exact.dense_h(g))
    q = lanczos.start_vector(g.n_orb)
    alpha, beta = [], []
    for j in range(120):
        w = lanczos.apply_h(g, 1.0, q)                 # "- beta_j q_{j-1}" dropped
        a = float(np.real(np.vdot(q, w)))
        w = w - a * q
        alpha.append(a)
        if j + 1 == 120:
            break
        b = float(np.sqrt(np.sum(np.abs(w) ** 2)))
        beta.append(b)
        q = w / b
    e = scipy.linalg.eigvalsh_tridiagonal(np.array(alpha), np.array(beta))
    assert not (abs(e[0] - ev[0]) < 1e-9 and abs(e[-1] - ev[-1]) < 1e-9)

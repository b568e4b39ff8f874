"""GPU parity of the AC-conductivity correlation (Sec. 2.7; Fermi-Dirac
operator of Sec. 2.2) against the CPU FP64 oracle, through the C ABI.

Tolerances, relative to the largest |C| of the case: FP64 1e-10 (Fermi
series of up to a few hundred terms, Clenshaw on the GPU vs the forward
recurrence in the oracle); FP32 states 2e-5 (the FP32 propagation bound of
the DOS path)."""
import math

import numpy as np
import pytest

import oracle
from oracle import ac
from tbpm_inputs import lattice, rng

pytestmark = pytest.mark.gpu

Z = math.pi / 2


@pytest.fixture(scope="module")
def tb():
    import paper_2209_00806_gb300 as tb
    return tb


def flake(L1, L2, B=0.0, seed=3, onsite_w=0.5, vacancy_frac=0.02):
    smp = lattice.graphene(L1, L2, pbc=False, seed=seed, onsite_w=onsite_w,
                           vacancy_frac=vacancy_frac, with_pos=True)
    return lattice.peierls(smp, B) if B else smp


def run_gpu(tb, smp, s, theta, n_steps, beta, mu, precision=0, offsets=None, cfg=None,
            flags=0):
    with tb.Propagator() as p:
        p.build_sample(smp, s, sample_offsets=offsets)
        p.set_bond_vectors(lattice.bond_vectors(smp))
        if cfg:
            p.launch_config(precision, *cfg)
        p.set_phase_states(np.ascontiguousarray(theta))
        return p.ac_correlation(Z, n_steps, beta, mu, precision, flags=flags), p.stats()


def run_oracle(smp, s, theta, n_steps, beta, mu):
    return ac.ac_correlation(smp, s, Z, n_steps, beta, mu, lattice.bond_vectors(smp),
                             oracle.phase_states(theta))


def rel_err(got, ref):
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("B", [0.0, 250.0])
@pytest.mark.parametrize("cfg", [None, (4, 128, 0), (8, 256, 1)])
def test_gpu_ac_fp64_matches_oracle(tb, B, cfg):
    smp = flake(23, 19, B)                      # ragged: 858 orbitals, one chunk
    s, beta, mu, n = 9.5, 8.0, 0.25, 60
    th = rng.phases(31, 2, smp.n_orb)
    got, st = run_gpu(tb, smp, s, th, n, beta, mu, cfg=cfg)
    ref = run_oracle(smp, s, th, n, beta, mu)
    assert got.shape == (1, 2, 4, n + 1)
    assert rel_err(got[0], ref) < 1e-10
    if B == 0.0:
        # no field: the transverse parts are small against the longitudinal ones
        assert np.max(np.abs(got[0, :, 1])) < np.max(np.abs(got[0, :, 0]))


@pytest.mark.parametrize("cfg", [None, (16, 128, 65), (4, 256, 1)])
def test_gpu_ac_fp32_matches_oracle(tb, cfg):
    smp = flake(30, 27, 120.0, seed=5)
    s, beta, mu, n = 9.5, 20.0, -0.4, 50
    th = rng.phases(32, 3, smp.n_orb)
    got, st = run_gpu(tb, smp, s, th, n, beta, mu, precision=1, cfg=cfg)
    ref = run_oracle(smp, s, th, n, beta, mu)
    assert rel_err(got[0], ref) < 2e-5


def test_gpu_ac_batch_of_samples(tb):
    parts = [flake(12, 10, 0.0, seed=1), flake(20, 9, 300.0, seed=2), flake(7, 30, 0.0, seed=4)]
    smp, offs = lattice.concat(parts)
    th_parts = [rng.phases(60 + k, 2, p.n_orb) for k, p in enumerate(parts)]
    th = np.concatenate(th_parts, axis=1)
    s, beta, mu, n = 9.5, 10.0, 0.1, 30
    got, _ = run_gpu(tb, smp, s, th, n, beta, mu, offsets=offs)
    for k, p in enumerate(parts):
        ref = run_oracle(p, s, th_parts[k], n, beta, mu)
        assert rel_err(got[k], ref) < 1e-10


def test_gpu_ac_random_graph_ragged_rows(tb):
    """Irregular rows (degrees 0 .. ~15) and random positions."""
    smp = lattice.random_graph(2100, 6000, seed=7, onsite_w=1.0)
    smp.pos = np.random.default_rng(3).uniform(-5.0, 5.0, (smp.n_orb, 2))   # dr from positions
    from . import exact
    s = 1.02 * np.max(np.abs(np.linalg.eigvalsh(exact.dense_h(smp))))
    th = rng.phases(33, 1, smp.n_orb)
    got, _ = run_gpu(tb, smp, s, th, 25, 3.0, 0.05)
    ref = run_oracle(smp, s, th, 25, 3.0, 0.05)
    assert rel_err(got[0], ref) < 1e-10


def test_gpu_ac_graph_and_fused_modes_agree(tb):
    N = tb._native
    smp = flake(26, 26, 0.0, seed=8)
    th = rng.phases(34, 2, smp.n_orb)
    plain, _ = run_gpu(tb, smp, 9.5, th, 20, 8.0, 0.0)
    graph, _ = run_gpu(tb, smp, 9.5, th, 20, 8.0, 0.0, flags=N.TBPM_PROP_GRAPH)
    fused, _ = run_gpu(tb, smp, 9.5, th, 20, 8.0, 0.0, flags=N.TBPM_PROP_PERSISTENT)
    assert np.array_equal(plain, graph)
    assert rel_err(fused, plain) < 1e-12


def test_gpu_ac_states_restored_and_errors(tb):
    N = tb._native
    smp = flake(10, 10)
    th = rng.phases(35, 2, smp.n_orb)
    with tb.Propagator() as p:
        p.build_sample(smp, 9.5)
        p.set_phase_states(th)
        with pytest.raises(N.TbpmError) as e:
            p.ac_correlation(Z, 4, 5.0)
        assert e.value.code == N.TBPM_E_STATE          # no positions
        p.set_bond_vectors(lattice.bond_vectors(smp))
        before = p.propagate(Z, 8)
        p.ac_correlation(Z, 4, 5.0)
        after = p.propagate(Z, 8)
        assert np.array_equal(before, after)
        with pytest.raises(N.TbpmError) as e:
            p.ac_correlation(Z, 4, 5.0, flags=N.TBPM_PROP_RESUME)
        assert e.value.code == N.TBPM_E_INVALID_ARG
        with pytest.raises(N.TbpmError) as e:
            p.ac_correlation(Z, 4, -1.0)
        assert e.value.code == N.TBPM_E_INVALID_ARG
        p.set_phase_states(rng.phases(36, 17, smp.n_orb))
        with pytest.raises(N.TbpmError) as e:
            p.ac_correlation(Z, 4, 5.0)
        assert e.value.code == N.TBPM_E_INVALID_ARG


def test_gpu_ac_conductivity_of_graphene_is_universal(tb):
    """Pristine periodic graphene (256 x 256 cells, 131,072 orbitals), T = 300 K,
    mu = 0: in the Dirac regime 2 mu << hbar omega << |t| the optical
    conductivity per spin is e^2 / (8 hbar); FP32 states, 2048 steps, damping
    eta = 0.1 eV (the E -> 0+ of the Kubo integral; it smooths the discrete
    transitions of the finite sample).  The oracle gives 0.93-1.08 of the
    universal value on the same state at 0.5-1.2 eV."""
    L = 256
    smp = lattice.graphene(L, L, pbc=True, with_pos=True)
    s, beta, mu, n = 9.0, 1.0 / (8.617333262e-5 * 300.0), 0.0, 2048
    th = rng.phases(37, 1, smp.n_orb)
    with tb.Propagator() as p:
        p.build_sample(smp, s)
        # periodic bonds: the generator's bond vectors are the nearest images
        p.set_bond_vectors(lattice.bond_vectors(smp))
        p.set_phase_states(th)
        corr = p.ac_correlation(Z, n, beta, mu, precision=1)
    area = L * L * abs(lattice.A1[0] * lattice.A2[1] - lattice.A1[1] * lattice.A2[0])
    tau = Z / s
    om = np.array([0.5, 0.8, 1.0, 1.2])
    sig = tb.ac_conductivity(corr[0, 0], tau, beta, 0.1, om, smp.n_orb / area)
    for ab in (0, 3):                                    # xx, yy
        assert np.all(np.abs(sig[ab] / (1.0 / 8.0) - 1.0) < 0.1), (ab, sig[ab])
    # isotropic: the Hall parts vanish against the longitudinal ones
    assert np.max(np.abs(sig[1:3])) < 0.2 * np.min(np.abs(sig[0]))

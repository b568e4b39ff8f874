"""GPU parity of the quasi-eigenstates (Sec. 2.6, Eq. quasi) and of the
backward propagation they use, against the CPU FP64 oracle through the C
ABI.  States are compared after normalisation: FP64 within 1e-10, FP32
within 2e-5 (the FP32 propagation bound)."""
import math

import numpy as np
import pytest

import oracle
from oracle import quasi
from tbpm_inputs import lattice, rng

from . import exact

pytestmark = pytest.mark.gpu

Z = math.pi / 2


@pytest.fixture(scope="module")
def tb():
    import paper_2209_00806_gb300 as tb
    return tb


def flake(L1, L2, B=0.0, seed=3):
    smp = lattice.graphene(L1, L2, pbc=False, seed=seed, onsite_w=0.6, vacancy_frac=0.02,
                           with_pos=True)
    return lattice.peierls(smp, B) if B else smp


def run_gpu(tb, smp, s, theta, n, energies, precision=0, offsets=None, cfg=None, flags=0):
    with tb.Propagator() as p:
        p.build_sample(smp, s, sample_offsets=offsets)
        if cfg:
            p.launch_config(precision, *cfg)
        p.set_phase_states(np.ascontiguousarray(theta))
        return p.quasi_eigenstates(Z, n, energies, precision, flags=flags)


@pytest.mark.parametrize("B", [0.0, 200.0])
@pytest.mark.parametrize("cfg", [None, (1, 128, 0), (4, 64, 65)])
def test_gpu_quasi_fp64_matches_oracle(tb, B, cfg):
    smp = flake(23, 19, B)
    s, n = 9.5, 80
    E = np.array([-2.0, -0.35, 0.0, 1.7])
    th = rng.phases(41, 3, smp.n_orb)
    got, norms = run_gpu(tb, smp, s, th, n, E, cfg=cfg)
    ref, ref_n = quasi.quasi_eigenstates(smp, s, Z, n, E, oracle.phase_states(th))
    assert np.max(np.abs(got - ref_n)) < 1e-10
    ref_norm2 = np.sum(np.abs(ref) ** 2, axis=-1)
    assert np.max(np.abs(norms[:, :, 0] / ref_norm2 - 1.0)) < 1e-10


@pytest.mark.parametrize("cfg", [None, (16, 128, 65), (2, 256, 1)])
def test_gpu_quasi_fp32_matches_oracle(tb, cfg):
    smp = flake(30, 27, 0.0, seed=6)
    s, n = 9.5, 60
    E = np.array([-1.1, 0.4])
    th = rng.phases(42, 4, smp.n_orb)
    got, _ = run_gpu(tb, smp, s, th, n, E, precision=1, cfg=cfg)
    _, ref_n = quasi.quasi_eigenstates(smp, s, Z, n, E, oracle.phase_states(th))
    assert np.max(np.abs(got - ref_n)) < 2e-5


def test_gpu_quasi_batch_normalised_per_sample(tb):
    parts = [flake(12, 10, 0.0, seed=1), flake(20, 9, 0.0, seed=2)]
    smp, offs = lattice.concat(parts)
    th_parts = [rng.phases(70 + k, 2, p.n_orb) for k, p in enumerate(parts)]
    th = np.concatenate(th_parts, axis=1)
    E = np.array([0.5, -1.5])
    got, norms = run_gpu(tb, smp, 9.5, th, 50, E, offsets=offs)
    for k, p in enumerate(parts):
        _, ref_n = quasi.quasi_eigenstates(p, 9.5, Z, 50, E, oracle.phase_states(th_parts[k]))
        assert np.max(np.abs(got[:, :, offs[k]:offs[k + 1]] - ref_n)) < 1e-10
    assert norms.shape == (2, 2, 2)


def test_gpu_quasi_recovers_isolated_eigenvectors(tb):
    smp = lattice.chain(12, t=-1.0, seed=3, onsite_w=2.0)
    E, U = np.linalg.eigh(exact.dense_h(smp))
    th = rng.phases(10, 1, smp.n_orb)
    got, _ = run_gpu(tb, smp, 3.5, th, 1500, E[[2, 7]])
    for k, i in enumerate((2, 7)):
        assert abs(abs(np.vdot(U[:, i], got[k, 0])) - 1.0) < 1e-3


def test_gpu_backward_propagation_is_time_reversal(tb):
    """C(-t) = conj C(t): the backward run against the forward one, and
    graph replay of the quasi-eigenstate runs is bit-identical."""
    N = tb._native
    smp = flake(18, 18, 150.0, seed=9)
    th = rng.phases(43, 2, smp.n_orb)
    with tb.Propagator() as p:
        p.build_sample(smp, 9.5)
        p.set_phase_states(th)
        fwd = p.propagate(Z, 40)
        bwd = p.propagate(Z, 40, flags=N.TBPM_PROP_BACKWARD)
        assert np.max(np.abs(bwd - np.conj(fwd))) < 1e-12
        a, _ = p.quasi_eigenstates(Z, 30, [0.3])
        b, _ = p.quasi_eigenstates(Z, 30, [0.3], flags=N.TBPM_PROP_GRAPH)
        assert np.array_equal(a, b)
        with pytest.raises(N.TbpmError):
            p.quasi_eigenstates(Z, 30, [0.3], flags=N.TBPM_PROP_BACKWARD)

"""GPU parity with complex hoppings: graphene flakes in a perpendicular
magnetic field by Peierls substitution (Sec. 2.1), against the CPU FP64
oracle through the C ABI.  FP64 C(t) within 1e-10, FP32 within 2e-5 (the
tolerances of the real-hopping path); a physical check places the first
Landau level where the Dirac-cone formula puts it."""
import math

import numpy as np
import pytest

import oracle
from tbpm_inputs import lattice, rng

pytestmark = pytest.mark.gpu

Z = math.pi / 2


@pytest.fixture(scope="module")
def tb():
    import paper_2209_00806_gb300 as tb
    return tb


def field_flake(L1, L2, B, seed=7, onsite_w=0.6, vacancy_frac=0.02):
    base = lattice.graphene(L1, L2, pbc=False, seed=seed, onsite_w=onsite_w,
                            vacancy_frac=vacancy_frac, with_pos=True)
    return lattice.peierls(base, B)


def run_gpu(tb, smp, s, theta, n_steps, precision=0, offsets=None, cfg=None, flags=0):
    with tb.Propagator() as p:
        p.build_sample(smp, s, sample_offsets=offsets)
        if cfg:
            p.launch_config(precision, *cfg)
        p.set_phase_states(np.ascontiguousarray(theta))
        c = p.propagate(Z, n_steps, precision, flags=flags)
        return c, p.stats(), p.states(), p.norms()


def run_oracle(smp, s, theta, n_steps, want_psi=False):
    psi0 = oracle.phase_states(theta)
    return oracle.propagate(smp, s, Z, n_steps, psi0, want_psi=want_psi, want_norms=want_psi)


# TMA (4), wide (64) and fused (8) bits are dropped for complex values
@pytest.mark.parametrize("cfg", [(1, 64, 0), (2, 128, 1), (4, 256, 3), (8, 128, 65),
                                 (4, 256, 5), (2, 128, 8)])
def test_gpu_fp64_field_flake_launch_shapes(tb, cfg):
    smp = field_flake(31, 29, 150.0)                  # 1,782 orbitals: ragged chunk
    assert np.iscomplexobj(smp.hop_v)
    th = rng.phases(12, 7, smp.n_orb)
    c, st, phi, nrm = run_gpu(tb, smp, 9.5, th, 120, cfg=cfg)
    ref, onrm, psi = run_oracle(smp, 9.5, th, 120, want_psi=True)
    assert np.max(np.abs(c[0] - ref)) < 1e-10
    assert np.max(np.abs(phi - psi)) < 1e-10
    assert np.max(np.abs(nrm[0] - onrm)) < 1e-10
    assert st["nnz_true"] == 2 * smp.n_hop


@pytest.mark.parametrize("cfg", [None, (16, 128, 65), (4, 256, 1), (2, 64, 0), (16, 256, 4)])
def test_gpu_fp32_field_flake_launch_shapes(tb, cfg):
    smp = field_flake(40, 37, 80.0, seed=9)
    th = rng.phases(13, 16, smp.n_orb)
    c, st, _, _ = run_gpu(tb, smp, 9.5, th, 60, precision=1, cfg=cfg)
    ref = run_oracle(smp, 9.5, th, 60)
    assert np.max(np.abs(c[0] - ref)) < 2e-5


def test_gpu_field_and_zero_field_samples_in_one_batch(tb):
    """Samples of a batch may mix fields; a real sample stored in the complex
    form gives the real path's result."""
    parts = [field_flake(20, 18, 300.0, seed=3), lattice.graphene(9, 9, pbc=True, seed=4),
             field_flake(33, 11, 60.0, seed=5, vacancy_frac=0.0)]
    smp, offs = lattice.concat(parts)
    assert np.iscomplexobj(smp.hop_v)
    th_parts = [rng.phases(50 + k, 3, p.n_orb) for k, p in enumerate(parts)]
    th = np.concatenate(th_parts, axis=1)
    c64, _, _, _ = run_gpu(tb, smp, 9.5, th, 100, offsets=offs)
    c32, _, _, _ = run_gpu(tb, smp, 9.5, th, 100, precision=1, offsets=offs)
    for k, p in enumerate(parts):
        ref = run_oracle(p, 9.5, th_parts[k], 100)
        assert np.max(np.abs(c64[k] - ref)) < 1e-10
        assert np.max(np.abs(c32[k] - ref)) < 2e-5
    real_c, _, _, _ = run_gpu(tb, parts[1], 9.5, th_parts[1], 100)
    assert np.max(np.abs(real_c[0] - c64[1])) < 1e-12


def test_gpu_complex_hops_refuse_adjoint_and_persistent(tb):
    N = tb._native
    smp = field_flake(8, 8, 100.0)
    with tb.Propagator() as p:
        p.build_sample(smp, 9.5)
        p.set_phase_states(rng.phases(1, 1, smp.n_orb))
        with pytest.raises(N.TbpmError) as e:
            p.propagate(Z, 4, flags=N.TBPM_PROP_PERSISTENT)
        assert e.value.code == N.TBPM_E_UNSUPPORTED
        c = p.propagate(Z, 4)
        with pytest.raises(N.TbpmError) as e:
            p.adjoint(Z, 4, np.ones((1, 1, 5), dtype=np.complex128))
        assert e.value.code == N.TBPM_E_UNSUPPORTED
    ref = run_oracle(smp, 9.5, rng.phases(1, 1, smp.n_orb), 4)
    assert np.max(np.abs(c[0] - ref)) < 1e-12


def test_gpu_landau_level_position(tb):
    """Graphene flake (~24 x 20 nm) at 200 T, FP64, 2048 steps: the DOS has
    the n = 1 Landau level at E_1 = hbar v_F sqrt(2 e B / hbar) with
    hbar v_F = (3/2) a_cc |t| (to the lattice correction), and the oracle
    gives the same DOS."""
    B = 200.0
    smp = field_flake(96, 96, B, seed=1, onsite_w=0.0, vacancy_frac=0.0)
    s, n_steps, n_e = 9.0, 2048, 4096
    th = rng.phases(77, 2, smp.n_orb)
    c, _, _, _ = run_gpu(tb, smp, s, th, n_steps)
    tau = Z / s
    en, d = tb.dos(c[0].mean(axis=0), tau, -s, s, n_e)
    a_cc = np.linalg.norm((lattice.A1 + lattice.A2) / 3.0)
    hbar_vf = 1.5 * a_cc * abs(lattice.T_NN)                 # eV nm
    l_B = math.sqrt(lattice.FLUX_QUANTUM / (2 * math.pi * B))  # nm
    e1 = hbar_vf * math.sqrt(2.0) / l_B
    win = (en > 0.6 * e1) & (en < 1.25 * e1)
    peak = en[win][np.argmax(d[win])]
    assert abs(peak - e1) < 0.03 * e1, (peak, e1)
    gap = d[np.argmin(np.abs(en - 0.5 * e1))]
    assert d[win].max() > 3.0 * gap
    ref = run_oracle(smp, s, th, n_steps)
    _, d_ref = oracle.dos(ref.mean(axis=0), tau, -s, s, n_e)
    assert np.max(np.abs(d - d_ref)) < 1e-9

"""GPU parity of the CUDA path against the CPU FP64 oracle, element by
element on the same seeded inputs, through the C ABI.

Tolerances: FP64 C(t) within 1e-10 absolute (C_0 = 1 sets the scale); FP32
states give a DOS whose L1 distance sum_k |D_k - D_k^oracle| dE is within
1e-4 (D integrates to 1)."""
import math

import numpy as np
import pytest

import oracle
from tbpm_inputs import lattice, rng, workloads

from . import exact

pytestmark = pytest.mark.gpu

Z = math.pi / 2


@pytest.fixture(scope="module")
def tb():
    import paper_2209_00806_gb300 as tb
    return tb


def run_gpu(tb, smp, s, theta, n_steps, precision=0, offsets=None, flags=0, bflags=0,
            cfg=None):
    with tb.Propagator() as p:
        p.build_sample(smp, s, sample_offsets=offsets, flags=bflags)
        if cfg:
            p.launch_config(precision, *cfg)
        p.set_phase_states(np.ascontiguousarray(theta))
        c = p.propagate(Z, n_steps, precision, flags=flags)
        return c, p.stats(), p.states(), p.norms()


def run_oracle(smp, s, theta, n_steps, want_psi=False):
    psi0 = oracle.phase_states(theta)
    return oracle.propagate(smp, s, Z, n_steps, psi0, want_psi=want_psi, want_norms=want_psi)


def test_gpu_fp64_disordered_vacancies_several_groups(tb):
    smp = lattice.graphene(24, 20, pbc=True, seed=5, onsite_w=1.0, vacancy_frac=0.02)
    th = rng.phases(9, 7, smp.n_orb)       # 7 states -> groups 4 + 2 + 1
    c, st, phi, nrm = run_gpu(tb, smp, 9.5, th, 200)
    ref, onrm, psi = run_oracle(smp, 9.5, th, 200, want_psi=True)
    assert st["group_width"] == [4, 2, 1] and st["n_terms"] == 16
    assert np.max(np.abs(c[0] - ref)) < 1e-10
    assert np.max(np.abs(phi - psi)) < 1e-10
    assert np.max(np.abs(nrm[0] - onrm)) < 1e-10


@pytest.mark.parametrize("cfg", [(1, 64, 0), (2, 128, 1), (8, 256, 3), (4, 256, 2), (4, 256, 4),
                                 (8, 256, 5), (1, 256, 4), (4, 128, 65), (2, 64, 64),
                                 (1, 128, 129), (4, 256, 257), (8, 64, 321), (2, 128, 193)])
def test_gpu_fp64_ragged_rows_launch_shapes(tb, cfg):
    smp = lattice.random_graph(3001, 9000, seed=3, onsite_w=2.0)   # degrees 0 .. ~15
    H = exact.dense_h(smp)
    s = 1.02 * np.max(np.abs(np.linalg.eigvalsh(H)))
    th = rng.phases(4, 5, smp.n_orb)
    c, st, _, _ = run_gpu(tb, smp, s, th, 60, cfg=cfg)
    ref = run_oracle(smp, s, th, 60)
    assert np.max(np.abs(c[0] - ref)) < 1e-10


@pytest.mark.parametrize("variant", [1, 2049])
def test_gpu_fp64_graphene_dos_full_workload(tb, variant):
    """64x64 pristine periodic graphene, 1024 steps: oracle and Bloch exact;
    per-term launches (1) and the cluster-resident stepping (2049)."""
    w = workloads.graphene_dos()
    th = w.thetas()[0]
    c, st, _, _ = run_gpu(tb, w.sample, w.s, th, w.n_steps, cfg=(1, 64, variant))
    ref = run_oracle(w.sample, w.s, th, w.n_steps)
    assert np.max(np.abs(c[0, 0] - ref[0])) < 1e-10
    times = w.tau * np.arange(w.n_steps + 1)
    bloch = exact.graphene_bloch_corr(64, 64, lattice.T_NN, oracle.phase_states(th)[0], times)
    assert np.max(np.abs(c[0, 0] - bloch)) < 1e-10
    en, d = tb.dos(c[0].mean(axis=0), w.tau, *w.e_range, w.n_energies)
    en2, d2 = oracle.dos(ref.mean(axis=0), w.tau, *w.e_range, w.n_energies)
    assert np.max(np.abs(d - d2)) < 1e-9
    if variant & 2048:
        assert st["kernel_launches"] == 1 + 2 + 1    # states, C_0 term + reduce, all steps


@pytest.mark.parametrize("kind", ["graphene_dos", "disordered", "random", "too_wide"])
def test_gpu_cluster_stepping_is_bit_identical(tb, kind):
    """TBPM_VARIANT_CLUSTER: the same states as the per-term kernels bit for
    bit (C within rounding of its block-order sums), on pristine and
    disordered graphene with vacancies (general values), a ragged random
    graph (rows of 0 .. 8 entries), and a sample with wider rows, which
    falls back to the per-term kernels."""
    if kind == "graphene_dos":
        smp, s = lattice.graphene(64, 64, pbc=True), 9.0
    elif kind == "disordered":
        smp = lattice.graphene(50, 41, pbc=True, seed=3, onsite_w=1.0, vacancy_frac=0.02,
                               bond_sigma=0.05)
        s = 9.5
    else:
        smp = lattice.random_graph(4000 if kind == "random" else 3000,
                                   5000 if kind == "random" else 15000, seed=21, onsite_w=2.0)
        s = 1.02 * np.max(np.abs(np.linalg.eigvalsh(exact.dense_h(smp))))
    th = rng.phases(55, 1, smp.n_orb)
    c0, _, phi0, n0 = run_gpu(tb, smp, s, th, 80, cfg=(1, 64, 1))
    c1, st, phi1, n1 = run_gpu(tb, smp, s, th, 80, cfg=(1, 64, 2049))
    assert np.array_equal(phi0, phi1)
    assert np.max(np.abs(c0 - c1)) < 1e-13 and np.max(np.abs(n0 - n1)) < 1e-13
    ref = run_oracle(smp, s, th, 80)
    assert np.max(np.abs(c1[0] - ref)) < 1e-10
    widest = np.max(np.bincount(np.concatenate([smp.hop_i, smp.hop_j]), minlength=smp.n_orb))
    assert (kind == "too_wide") == (widest > 12)
    assert st["kernel_launches"] == (4 if widest <= 12 else 3 + 80 * 16)


def test_gpu_cluster_stepping_resume_and_backward(tb):
    """The cluster stepping continues a propagation (TBPM_PROP_RESUME) and runs
    backward in time (TBPM_PROP_BACKWARD, C(-t) = conj C(t)) like the
    per-term kernels."""
    N = tb._native
    smp = lattice.graphene(40, 40, pbc=True, seed=4, onsite_w=0.6)
    th = rng.phases(56, 1, smp.n_orb)
    with tb.Propagator() as p:
        p.build_sample(smp, 9.5)
        p.launch_config(0, 1, 64, 2049)
        p.set_phase_states(th)
        full = p.propagate(Z, 50, 0)
        phi_full = p.states()
        p.propagate(Z, 20, 0)
        p.propagate(Z, 30, 0, flags=N.TBPM_PROP_RESUME)
        assert np.max(np.abs(p.states() - phi_full)) < 1e-12
        back = p.propagate(Z, 50, 0, flags=N.TBPM_PROP_BACKWARD)
    assert np.max(np.abs(back[0, 0] - np.conj(full[0, 0]))) < 1e-12


def test_gpu_multi_sample_batch_fp64_and_fp32(tb):
    parts = [lattice.graphene(L, L, pbc=True, seed=10 + L, onsite_w=0.3 * L % 2)
             for L in (5, 9, 23)]
    smp, offs = lattice.concat(parts)
    th_parts = [rng.phases(40 + k, 3, p.n_orb) for k, p in enumerate(parts)]
    th = np.concatenate(th_parts, axis=1)
    c64, _, _, _ = run_gpu(tb, smp, 9.5, th, 120, offsets=offs)
    c32, st32, _, _ = run_gpu(tb, smp, 9.5, th, 120, precision=1, offsets=offs)
    for k, p in enumerate(parts):
        ref = run_oracle(p, 9.5, th_parts[k], 120)
        assert np.max(np.abs(c64[k] - ref)) < 1e-10
        assert np.max(np.abs(c32[k] - ref)) < 2e-5


@pytest.mark.parametrize("cfg", [(16, 128, 3), (4, 256, 1), (2, 64, 0), (16, 256, 4), (4, 256, 5),
                                 (2, 256, 4), (1, 256, 0), (16, 128, 65), (4, 128, 64),
                                 (1, 128, 129), (8, 256, 257), (16, 128, 321), (4, 64, 193)])
def test_gpu_fp32_launch_shapes(tb, cfg):
    smp = lattice.random_graph(2500, 7000, seed=9, onsite_w=2.0)
    H = exact.dense_h(smp)
    s = 1.02 * np.max(np.abs(np.linalg.eigvalsh(H)))
    th = rng.phases(8, 16, smp.n_orb)
    c, st, _, _ = run_gpu(tb, smp, s, th, 40, precision=1, cfg=cfg)
    ref = run_oracle(smp, s, th, 40)
    assert np.max(np.abs(c[0] - ref)) < 2e-5


def test_gpu_autotune_picks_a_valid_shape(tb):
    smp = lattice.graphene(40, 40, pbc=True, seed=4, onsite_w=1.0, vacancy_frac=0.01)
    th = rng.phases(3, 4, smp.n_orb)
    with tb.Propagator() as p:
        p.build_sample(smp, 9.5)
        p.set_phase_states(th)
        best = p.autotune(Z, precision=1, probe_steps=2)
        assert best["group"] in (2, 4) and best["threads"] in (64, 128, 256)
        assert best["variant"] in (0, 1, 3, 4, 5, 8, 24, 40, 65, 129, 257, 193, 321, 512, 513,
                                   1536, 1537, 4608, 4609, 8193, 8257)
        assert best["ms_per_step"] > 0
        c = p.propagate(Z, 30, 1)
    ref = run_oracle(smp, 9.5, th, 30)
    assert np.max(np.abs(c[0] - ref)) < 2e-5


def test_gpu_fp32_dos_l1(tb):
    w = workloads.disordered_graphene(L=96, n_steps=1024, n_energies=2048)
    th = w.thetas()[0]
    c32, st, _, _ = run_gpu(tb, w.sample, w.s, th, w.n_steps, precision=1)
    ref = run_oracle(w.sample, w.s, th, w.n_steps)
    en, d32 = tb.dos(c32[0].mean(axis=0), w.tau, *w.e_range, w.n_energies)
    _, d64 = oracle.dos(ref.mean(axis=0), w.tau, *w.e_range, w.n_energies)
    l1 = np.sum(np.abs(d32 - d64)) * (en[1] - en[0])
    assert l1 < 1e-4, l1
    assert st["max_norm_drift"] < 1e-3


def test_gpu_fp32_norm_carry_renormalises(tb):
    """With a renormalisation bound below the FP32 drift every step restarts
    from phi / |phi| (FP64 norm); the correlations stay on the oracle's."""
    w = workloads.disordered_graphene(L=48, n_steps=200, n_energies=1024)
    th = w.thetas()[0]
    with tb.Propagator() as p:
        p.build_sample(w.sample, w.s)
        tb._native.tbpm_set_norm_policy(p.ctx, 1e-12, 1e-2, 1e-6)
        p.set_phase_states(th)
        c = p.propagate(w.z, w.n_steps, 1)
        st = p.stats()
        nrm = p.norms()
    ref = run_oracle(w.sample, w.s, th, w.n_steps)
    assert st["renormalisations"] > w.n_steps          # nearly every state, every step
    assert np.max(np.abs(c[0] - ref)) < 2e-5
    assert np.max(np.abs(nrm - 1)) < 1e-6


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("backward", [False, True])
def test_gpu_uniform_hopping_form(tb, prec, backward):
    """Lattices with one hopping value take the one-value form (no value
    loads).  FP32: the very same states as the general form.  FP64: the
    neighbours are summed before the one multiply by gamma h and gamma d is
    folded into the combine (2 FP64 operations fewer per state and row), so
    it agrees with the general form to rounding; forward and backward
    (gamma < 0: the sign-flipped 2 d) against the oracle."""
    smp = lattice.graphene(30, 29, pbc=True, seed=3, onsite_w=1.0, vacancy_frac=0.03)
    th = rng.phases(14, 4, smp.n_orb)
    fl = 16 if backward else 0
    a, sa, pa, _ = run_gpu(tb, smp, 9.5, th, 40, precision=prec, flags=fl)
    b, sb, pb, _ = run_gpu(tb, smp, 9.5, th, 40, precision=prec, flags=fl, bflags=16)
    n, nnz = smp.n_orb, sa["nnz_true"]
    if prec == 1:
        assert np.array_equal(pa, pb) and np.array_equal(a, b)
        assert sa["ops_term"] == sb["ops_term"] == 4 * (8 * n + 2 * nnz)
    else:
        assert np.max(np.abs(pa - pb)) < 1e-13 and np.max(np.abs(a - b)) < 1e-13
        assert not np.array_equal(pa, pb)            # the summed form did run
        assert sa["ops_term"] == 4 * (4 * n + 2 * nnz) and sb["ops_term"] == 4 * (6 * n + 2 * nnz)
    ref = run_oracle(smp, 9.5, th, 40)
    if backward:
        ref = np.conj(ref)                          # C(-t) = C(t)*
    assert np.max(np.abs(a[0] - ref)) < (1e-10 if prec == 0 else 2e-5)


@pytest.mark.parametrize("bflags", [8, 64])
def test_gpu_rcm_reorder_and_permuted_input(tb, bflags):
    """RCM (8) and cluster (64) row orders of a shuffled input give the
    natural order's results in the caller's numbering."""
    smp = lattice.graphene(40, 36, pbc=True, seed=2, onsite_w=1.0, vacancy_frac=0.02)
    perm = np.random.default_rng(7).permutation(smp.n_orb)
    shuffled = lattice.permute(smp, perm)
    th = rng.phases(5, 2, smp.n_orb)
    th_sh = np.empty_like(th)
    th_sh[:, perm] = th
    c0, _, _, _ = run_gpu(tb, smp, 9.5, th, 100)
    c1, _, phi1, _ = run_gpu(tb, shuffled, 9.5, th_sh, 100, bflags=bflags)
    _, _, phi0, _ = run_gpu(tb, smp, 9.5, th, 100)
    assert np.max(np.abs(c0 - c1)) < 1e-12
    assert np.max(np.abs(phi1[:, perm] - phi0)) < 1e-12


def test_gpu_device_inputs_match_host_inputs(tb):
    import torch
    smp = lattice.graphene(12, 12, pbc=True, seed=1, onsite_w=1.0, vacancy_frac=0.03)
    th = rng.phases(3, 2, smp.n_orb)
    ch, _, _, _ = run_gpu(tb, smp, 9.5, th, 80)
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    with tb.Propagator() as p:
        p.build(smp.n_orb, d(smp.onsite, torch.float64), d(smp.hop_i, torch.int64),
                d(smp.hop_j, torch.int64), d(smp.hop_v, torch.float64), 9.5)
        p.set_phase_states(d(th, torch.float64))
        out = torch.empty((1, 2, 81), dtype=torch.complex128, device="cuda")
        p.propagate(Z, 80, 0, out=out)
        cd = out.cpu().numpy()
    assert np.max(np.abs(cd - ch)) < 1e-15


def test_gpu_graph_mode_and_determinism(tb):
    smp = lattice.graphene(20, 20, pbc=True, seed=8, onsite_w=1.0, vacancy_frac=0.01)
    th = rng.phases(6, 4, smp.n_orb)
    for prec in (0, 1):
        a, _, _, _ = run_gpu(tb, smp, 9.5, th, 50, precision=prec)
        b, _, _, _ = run_gpu(tb, smp, 9.5, th, 50, precision=prec)
        g, _, _, _ = run_gpu(tb, smp, 9.5, th, 50, precision=prec, flags=2)
        pr, stp, _, _ = run_gpu(tb, smp, 9.5, th, 50, precision=prec, flags=1)
        assert np.array_equal(a, b) and np.array_equal(a, g) and np.array_equal(a, pr)
        assert stp["ms_term_avg"] > 0 and stp["term_launches"] == 50 * 12


@pytest.mark.parametrize("prec", [0, 1])
def test_gpu_tma_kernel_is_bit_identical(tb, prec):
    """The TMA-staged term kernel does the same arithmetic in the same order;
    the wide-lane and the register-pipelined kernels (8193, 8257) the same
    arithmetic per row (bit-identical states) with the closing sums grouped
    by other blocks (C within rounding)."""
    smp = lattice.graphene(33, 31, pbc=True, seed=6, onsite_w=1.0, vacancy_frac=0.02)
    th = rng.phases(12, 4, smp.n_orb)
    outs = []
    for variant in (0, 4, 5, 65, 8193, 8257):
        c, st, phi, _ = run_gpu(tb, smp, 9.5, th, 40, precision=prec, cfg=(4, 256, variant),
                                flags=2 if variant == 5 else 0)
        outs.append((variant, c, phi))
        if variant == 8257:     # states, C_0 term + reduce; per step 15 terms, the closing
            # one as the pipelined term + the reduction pass, and the reduce
            assert st["kernel_launches"] == 3 + 40 * 17
    for variant, c, phi in outs[1:]:
        assert np.array_equal(phi, outs[0][2])
        if variant in (65, 8193, 8257):
            assert np.max(np.abs(c - outs[0][1])) < (1e-13 if prec == 0 else 1e-6)
        else:
            assert np.array_equal(c, outs[0][1])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind", ["graphene", "random", "batch"])
def test_gpu_fused_step(tb, prec, kind):
    """The wavefront-fused step: the same states as the per-term kernels (bit
    for bit: same arithmetic per row) and C within rounding of the reduction
    order; against the oracle as everywhere else."""
    offs = None
    if kind == "graphene":
        smp = lattice.graphene(40, 37, pbc=True, seed=8, onsite_w=1.0, vacancy_frac=0.02)
        s, S, parts = 9.5, 7, None
    elif kind == "random":
        smp = lattice.random_graph(6000, 15000, seed=12, onsite_w=2.0)   # bandwidth ~ n
        s = 1.02 * np.max(np.abs(np.linalg.eigvalsh(exact.dense_h(smp))))
        S, parts = 3, None
    else:
        parts = [lattice.graphene(L, L, pbc=True, seed=30 + L, onsite_w=0.5) for L in (7, 30, 12)]
        smp, offs = lattice.concat(parts)
        s, S = 9.5, 4
    th = rng.phases(77, S, smp.n_orb)
    base, _, phi0, _ = run_gpu(tb, smp, s, th, 30, precision=prec, offsets=offs, cfg=(8, 128, 1))
    fused, st, phi1, _ = run_gpu(tb, smp, s, th, 30, precision=prec, offsets=offs, cfg=(8, 128, 8))
    assert np.array_equal(phi0, phi1)
    assert np.max(np.abs(base - fused)) < (1e-13 if prec == 0 else 1e-6)
    if parts is None:
        ref = run_oracle(smp, s, th, 30)
        assert np.max(np.abs(fused[0] - ref)) < (1e-10 if prec == 0 else 2e-5)
    else:
        for k, q in enumerate(parts):
            ref = run_oracle(q, s, th[:, offs[k]:offs[k + 1]], 30)
            assert np.max(np.abs(fused[k] - ref)) < (1e-10 if prec == 0 else 2e-5)


def test_gpu_persistent_flag_runs_the_fused_step(tb):
    smp = lattice.graphene(24, 24, pbc=True, seed=9, onsite_w=1.0)
    th = rng.phases(6, 4, smp.n_orb)
    a, _, pa, _ = run_gpu(tb, smp, 9.5, th, 20, precision=0)
    b, _, pb, _ = run_gpu(tb, smp, 9.5, th, 20, precision=0, flags=8)
    assert np.array_equal(pa, pb) and np.max(np.abs(a - b)) < 1e-13


def test_gpu_fused_step_graph_replay(tb):
    smp = lattice.graphene(30, 30, pbc=True, seed=2, onsite_w=1.0)
    th = rng.phases(5, 4, smp.n_orb)
    a, _, _, _ = run_gpu(tb, smp, 9.5, th, 20, precision=1, cfg=(4, 128, 8))
    b, _, _, _ = run_gpu(tb, smp, 9.5, th, 20, precision=1, cfg=(4, 128, 8), flags=2)
    assert np.array_equal(a, b)


def test_gpu_resume_continues_the_propagation(tb):
    smp = lattice.graphene(10, 10, pbc=True, seed=3, onsite_w=0.5)
    th = rng.phases(2, 3, smp.n_orb)
    with tb.Propagator() as p:
        p.build_sample(smp, 9.0)
        p.set_phase_states(th)
        full = p.propagate(Z, 60, 0)
        phi_full = p.states()
        p.propagate(Z, 25, 0)
        p.propagate(Z, 35, 0, flags=4)
        assert np.max(np.abs(p.states() - phi_full)) < 1e-12


def test_gpu_errors_are_statuses(tb):
    N = tb._native
    smp = lattice.graphene(6, 6, pbc=True)
    p = tb.Propagator()
    with pytest.raises(N.TbpmError) as e:
        p.propagate(Z, 3)
    assert e.value.code == N.TBPM_E_STATE
    bad = lattice.Sample(4, None, np.array([0, 2]), np.array([1, 2]), np.array([1.0, 1.0]))
    with pytest.raises(N.TbpmError) as e:
        p.build_sample(bad, 3.0)
    assert e.value.code == N.TBPM_E_INVALID_ARG and "itself" in str(e.value)
    out = lattice.Sample(4, None, np.array([0, 2]), np.array([1, 7]), np.array([1.0, 1.0]))
    with pytest.raises(N.TbpmError) as e:
        p.build_sample(out, 3.0)
    assert e.value.code == N.TBPM_E_INVALID_ARG
    with pytest.raises(N.TbpmError) as e:
        p.build_sample(smp, 5.0, flags=N.TBPM_BUILD_STRICT_BOUND)
    assert e.value.code == N.TBPM_E_SPECTRAL_BOUND
    # s well below the spectral radius: the build's Lanczos check refuses it ...
    with pytest.raises(N.TbpmError) as e:
        p.build_sample(smp, 3.0)
    assert e.value.code == N.TBPM_E_SPECTRAL_BOUND and "Lanczos" in str(e.value)
    # ... and without the check the Chebyshev series diverges
    p.build_sample(smp, 3.0, flags=N.TBPM_BUILD_NO_SPECTRAL_CHECK)
    p.set_phase_states(rng.phases(1, 1, smp.n_orb))
    with pytest.raises(N.TbpmError) as e:
        p.propagate(Z, 40)
    assert e.value.code in (N.TBPM_E_NORM_DRIFT, N.TBPM_E_NONFINITE)
    # NaN in the initial state
    p.build_sample(smp, 9.0)
    psi = oracle.phase_states(rng.phases(1, 1, smp.n_orb))
    psi[0, 3] = np.nan
    p.set_states(psi)
    with pytest.raises(N.TbpmError) as e:
        p.propagate(Z, 2)
    assert e.value.code == N.TBPM_E_NONFINITE
    # the context stays usable
    p.set_phase_states(rng.phases(1, 1, smp.n_orb))
    c = p.propagate(Z, 2)
    assert abs(c[0, 0, 0] - 1) < 1e-14
    p.close()


def test_gpu_disordered_graphene_full_size_against_oracle(tb):
    """2048x2048 disordered graphene with vacancies (8,304,722 orbitals), the
    four states and the autotuned launch shape of the benchmark, 256 steps in
    FP64 and FP32: state 0 against the oracle (the row-parallel twin) at
    every step -- FP64 C within 1e-10, FP32 C within 2e-5, and the FP32 DOS
    of that state within L1 1e-4 of the oracle's on the 4096-bin grid -- plus
    unit norms and |C| <= 1 for all four states."""
    w = workloads.disordered_graphene(n_steps=256)
    th = np.concatenate([t for t in w.thetas()], axis=1)
    with tb.Propagator() as p:
        p.build_sample(w.sample, w.s)
        p.set_phase_states(th)
        p.autotune(w.z, precision=0, probe_steps=2)
        p.autotune(w.z, precision=1, probe_steps=2)
        c64 = p.propagate(w.z, w.n_steps, 0)
        n64 = p.norms()
        c32 = p.propagate(w.z, w.n_steps, 1)
        n32 = p.norms()
    ref = oracle.propagate_rows(w.sample, w.s, w.z, w.n_steps, oracle.phase_states(th[:1]))
    assert np.max(np.abs(c64[0, 0] - ref[0])) < 1e-10
    assert np.max(np.abs(c32[0, 0] - ref[0])) < 2e-5
    en, d32 = tb.dos(c32[0, 0], w.tau, *w.e_range, w.n_energies)
    _, d64 = oracle.dos(ref[0], w.tau, *w.e_range, w.n_energies)
    assert np.sum(np.abs(d32 - d64)) * (en[1] - en[0]) < 1e-4
    assert np.max(np.abs(n64 - 1)) < 1e-12 and np.max(np.abs(n32 - 1)) < 1e-4
    assert np.all(np.abs(c64) <= 1 + 1e-12)


def test_gpu_batched_workload_two_samples_full_length(tb):
    """The batched workload as the benchmark runs it -- 32 uneven periodic
    samples (L in {256 .. 1024}), 16 states each, 512 FP32 steps, autotuned
    launch shape, one launch per term over the whole batch -- with the two
    smallest samples checked against the oracle at every step for their
    first four states: C within 2e-5 and the 4-state DOS within L1 1e-4 on
    the 2048-bin grid."""
    w = workloads.batched_graphene()
    th_parts = w.thetas()
    th = np.ascontiguousarray(np.concatenate(th_parts, axis=1))
    with tb.Propagator() as p:
        p.build_sample(w.sample, w.s, sample_offsets=w.offsets)
        p.set_phase_states(th)
        p.autotune(w.z, precision=1, probe_steps=2)
        c = p.propagate(w.z, w.n_steps, 1)
        st = p.stats()
    assert sum(st["group_width"]) == 16
    sizes = np.diff(w.offsets)
    for k in sorted(range(w.n_samples), key=lambda q: sizes[q])[:2]:
        lo, hi = int(w.offsets[k]), int(w.offsets[k + 1])
        m = (w.sample.hop_i >= lo) & (w.sample.hop_i < hi)
        part = lattice.Sample(hi - lo, w.sample.onsite[lo:hi], w.sample.hop_i[m] - lo,
                              w.sample.hop_j[m] - lo, w.sample.hop_v[m])
        ref = oracle.propagate_rows(part, w.s, w.z, w.n_steps,
                                    oracle.phase_states(th_parts[k][:4]))
        assert np.max(np.abs(c[k, :4] - ref)) < 2e-5, k
        en, dg = tb.dos(c[k, :4].mean(axis=0), w.tau, *w.e_range, w.n_energies)
        _, do = oracle.dos(ref.mean(axis=0), w.tau, *w.e_range, w.n_energies)
        assert np.sum(np.abs(dg - do)) * (en[1] - en[0]) < 1e-4, k


def test_gpu_fp32_reduction_is_fp64_grade(tb):
    """The FP32 form's closing reduction sums exact float-pair products: on
    the FP32 states it produced, C_n and <phi|phi> agree with the exact sums
    of the same FP32 numbers within 1e-12 (plain FP32 sums of the products
    over 128-row blocks miss by ~1e-8 at this size)."""
    w = workloads.disordered_graphene(L=512, n_steps=20)
    th = w.thetas()[0]
    with tb.Propagator() as p:
        p.build_sample(w.sample, w.s)
        p.set_phase_states(th)
        for cfg in ((4, 64, 65), (4, 128, 1), (2, 256, 0), (1, 64, 1)):
            p.launch_config(1, *cfg)
            c = p.propagate(w.z, w.n_steps, 1)
            nrm = p.norms()
            phi = p.states()                           # FP32 values, exactly
            psi0 = oracle.phase_states(th).astype(np.complex64).astype(np.complex128)
            for q in range(th.shape[0]):
                a, b = psi0[q], phi[q]              # FP32 x FP32 products are exact in FP64
                ref = math.fsum(np.concatenate([a.real * b.real, a.imag * b.imag]))
                refi = math.fsum(np.concatenate([a.real * b.imag, -(a.imag * b.real)]))
                nref = math.fsum(np.concatenate([b.real * b.real, b.imag * b.imag]))
                assert abs(c[0, q, -1].real - ref) < 1e-12, cfg
                assert abs(c[0, q, -1].imag - refi) < 1e-12, cfg
                assert abs(nrm[0, q, -1] - nref) < 1e-12, cfg


def test_gpu_ldos_single_site_states(tb):
    """LDOS by TBPM (Sec. 2.5): an initial state on one orbital only; C(t) is
    then sum_j |U_ij|^2 exp(-i E_j t).  Several sites as several states."""
    smp = lattice.graphene(9, 8, pbc=True, seed=21, onsite_w=1.0, vacancy_frac=0.03)
    sites = [0, 5, 17, smp.n_orb - 1]
    psi0 = np.zeros((len(sites), smp.n_orb), dtype=np.complex128)
    for k, i in enumerate(sites):
        psi0[k, i] = 1.0
    n_steps, s = 150, 9.5
    with tb.Propagator() as p:
        p.build_sample(smp, s)
        p.set_states(psi0)
        c = p.propagate(Z, n_steps, 0)
    ref = oracle.propagate(smp, s, Z, n_steps, psi0)
    assert np.max(np.abs(c[0] - ref)) < 1e-10
    E, U = np.linalg.eigh(exact.dense_h(smp))
    times = (Z / s) * np.arange(n_steps + 1)
    for k, i in enumerate(sites):
        ed = np.exp(-1j * np.outer(times, E)) @ (np.abs(U[i]) ** 2)
        assert np.max(np.abs(c[0, k] - ed)) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_gpu_twisted_bilayer_wide_rows(tb, prec):
    """Twisted bilayer flake: ~63 entries per row, asymmetric spectrum
    (s = 12 eV), layer-by-layer numbering; natural, RCM and cluster order, plain,
    wide-lane, row-split and TMA kernels, against the oracle and exact
    diagonalisation."""
    w = workloads.twisted_bilayer_flake(side_nm=5.0, n_steps=60)
    smp = w.sample
    th = w.thetas()[0][:3]
    ref = run_oracle(smp, w.s, th, w.n_steps)
    times = w.tau * np.arange(w.n_steps + 1)
    ed = exact.ed_corr(smp, oracle.phase_states(th)[0], times)
    assert np.max(np.abs(ref[0] - ed)) < 1e-11
    tol = 1e-10 if prec == 0 else 2e-5
    for bflags in (0, 8, 64):
        for cfg in ((2, 128, 1), (2, 128, 65), (2, 128, 4), (2, 128, 257), (2, 64, 321)):
            c, st, _, _ = run_gpu(tb, smp, w.s, th, w.n_steps, precision=prec, bflags=bflags,
                                  cfg=cfg)
            assert np.max(np.abs(c[0] - ref)) < tol, (bflags, cfg)


def test_gpu_kernels_are_sm103a_images(tb):
    assert tb._native.tbpm_kernel_binary_version() == 103


def test_gpu_state_average_and_its_adjoint(tb):
    """tbpm_correlation: the mean over the states of each sample, on the GPU
    (host and device outputs); tbpm_correlation_adjoint: its transpose."""
    import torch
    parts = [lattice.graphene(L, L, pbc=True, seed=60 + L, onsite_w=0.7) for L in (6, 11)]
    smp, offs = lattice.concat(parts)
    th = rng.phases(61, 3, smp.n_orb)
    with tb.Propagator() as p:
        p.build_sample(smp, 9.5, sample_offsets=offs)
        p.set_phase_states(th)
        c = p.propagate(Z, 25, 0)
        avg = p.correlation()
        dev = torch.empty((2, 26), dtype=torch.complex128, device="cuda")
        p.correlation(out=dev)
        ref = np.empty((2, 26), dtype=np.complex128)
        for k in range(2):
            tot = c[k, 0] + c[k, 1] + c[k, 2]          # states in order
            ref[k] = tot.real / 3 + 1j * (tot.imag / 3)
        assert np.array_equal(avg, ref)
        assert np.array_equal(dev.cpu().numpy(), ref)
        g = rng.phases(62, 2, 26) + 1j * rng.phases(63, 2, 26)
        gs = p.correlation_adjoint(25, g)
        gd = p.correlation_adjoint(25, torch.as_tensor(g, device="cuda")).cpu().numpy()
        assert gs.shape == (2, 3, 26) and np.array_equal(gs, gd)
        # <g, mean(C)> = <adjoint(g), C> for any C (real inner product)
        x = rng.phases(64, 6, 26).reshape(2, 3, 26) + 0j
        lhs = np.sum((g.conj() * x.mean(axis=1)).real)
        rhs = np.sum((gs.conj() * x).real)
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def _tbg_sample(side, order="morton"):
    from tbpm_inputs import tbg
    return tbg.to_numpy_sample(tbg.twisted_bilayer(side, order=order))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind", ["tbg", "random", "graphene"])
def test_gpu_halo_variant_is_bit_identical(tb, prec, kind):
    """TBPM_VARIANT_HALO gathers from a shared-memory copy of each 128-row
    block's halo with the plain kernel's arithmetic: the same states bit for
    bit (C within rounding of the reduction's block grouping), on every
    group width it serves, and the oracle's results."""
    if kind == "tbg":
        smp, s = _tbg_sample(8.0), 12.0
    elif kind == "random":
        smp = lattice.random_graph(3000, 12000, seed=17, onsite_w=2.0)
        s = 1.02 * np.max(np.abs(np.linalg.eigvalsh(exact.dense_h(smp))))
    else:
        smp, s = lattice.graphene(30, 27, pbc=True, seed=8, onsite_w=1.0, vacancy_frac=0.02), 9.5
    th = rng.phases(91, 16 if prec else 8, smp.n_orb)
    ref = run_oracle(smp, s, th[:2], 30)
    tol = 1e-10 if prec == 0 else 2e-5
    widths = (2, 4, 8) if prec == 0 else (4, 8, 16)
    for B in widths:
        # halo, halo + pipelined persistent and halo + one-stage staged (zig-zag)
        # against the plain wide kernel; with the row split requested they keep
        # the plain split kernel
        for plain, variants in ((65, (513, 1537, 4609)), (193, (1665, 4801))):
            c0, _, phi0, _ = run_gpu(tb, smp, s, th, 30, precision=prec, cfg=(B, 64, plain))
            for variant in variants:
                c1, st, phi1, _ = run_gpu(tb, smp, s, th, 30, precision=prec,
                                          cfg=(B, 64, variant))
                assert np.array_equal(phi0, phi1), (B, variant)
                assert np.max(np.abs(c0 - c1)) < 1e-12, (B, variant)
                assert np.max(np.abs(c1[0, :2] - ref)) < tol, (B, variant)


def test_gpu_halo_variant_twisted_bilayer_20nm_fp32(tb):
    """A 20 nm twisted-bilayer flake (Morton numbering, ~45,000 orbitals,
    ~68 entries per row) with 8 FP32 states: the staged-gather kernel against
    the plain kernel (bit-identical states) and the oracle (first state)."""
    smp = _tbg_sample(20.0)
    th = rng.phases(93, 8, smp.n_orb)
    c0, _, phi0, _ = run_gpu(tb, smp, 12.0, th, 12, precision=1, cfg=(8, 64, 65))
    ref = oracle.propagate_rows(smp, 12.0, Z, 12, oracle.phase_states(th[:1]))
    for variant in (513, 1536, 4608, 8257):       # 8257: rows of 68 entries, beyond the
        c1, _, phi1, _ = run_gpu(tb, smp, 12.0, th, 12, precision=1,   # four loaded ahead
                                 cfg=(8, 64, variant))
        assert np.array_equal(phi0, phi1), variant
        assert np.max(np.abs(c1[0, 0] - ref[0])) < 2e-5, variant
    c2, _, phi2, _ = run_gpu(tb, smp, 12.0, th, 12, precision=1, cfg=(8, 64, 193))
    c3, _, phi3, _ = run_gpu(tb, smp, 12.0, th, 12, precision=1, cfg=(8, 64, 1665))
    assert np.array_equal(phi2, phi3)
    assert np.max(np.abs(c3[0, 0] - ref[0])) < 2e-5


def test_gpu_lean_build_without_fp64_and_bond_map(tb):
    """TBPM_BUILD_NO_FP64 | TBPM_BUILD_NO_BOND_MAP (the largest samples):
    FP32 values filled directly give the default build's FP32 results bit
    for bit; what needs the dropped parts returns TBPM_E_STATE."""
    N = tb._native
    smp = lattice.graphene(25, 22, pbc=True, seed=4, onsite_w=1.0, vacancy_frac=0.02)
    smp.hop_v = smp.hop_v * (1.0 + 0.01 * rng.phases(5, 1, smp.n_hop)[0])   # non-uniform
    th = rng.phases(94, 4, smp.n_orb)
    a, _, pa, _ = run_gpu(tb, smp, 9.5, th, 25, precision=1)
    b, _, pb, _ = run_gpu(tb, smp, 9.5, th, 25, precision=1,
                          bflags=N.TBPM_BUILD_NO_FP64 | N.TBPM_BUILD_NO_BOND_MAP)
    assert np.array_equal(pa, pb) and np.array_equal(a, b)
    with tb.Propagator() as p:
        p.build_sample(smp, 9.5, flags=N.TBPM_BUILD_NO_FP64 | N.TBPM_BUILD_NO_BOND_MAP)
        p.set_phase_states(th)
        with pytest.raises(N.TbpmError) as e:
            p.propagate(Z, 3, 0)
        assert e.value.code == N.TBPM_E_STATE
        with pytest.raises(N.TbpmError) as e:
            p.set_bond_vectors(np.ones((smp.n_hop, 2)))
        assert e.value.code == N.TBPM_E_STATE


@pytest.mark.parametrize("kind", ["graphene", "random", "field", "fp32_only"])
def test_gpu_spectral_bounds_match_the_oracle(tb, kind):
    """tbpm_spectral_bounds: the Lanczos extremes of the oracle's process from
    the same SplitMix64 start vector, in caller order (RCM rows inside)."""
    from oracle import lanczos
    N = tb._native
    flags, tol = 0, 1e-9
    if kind == "graphene":
        smp = lattice.graphene(40, 36, pbc=True, seed=2, onsite_w=1.0, vacancy_frac=0.02)
        flags = N.TBPM_BUILD_REORDER_RCM
    elif kind == "random":
        smp = lattice.random_graph(2000, 7000, seed=3, onsite_w=2.0)
    elif kind == "field":
        smp = lattice.peierls(lattice.graphene(30, 28, pbc=False, seed=5, onsite_w=0.5,
                                               with_pos=True), 200.0)
    else:
        smp = lattice.graphene(30, 30, pbc=True, seed=9, onsite_w=1.0)
        flags, tol = N.TBPM_BUILD_NO_FP64, 1e-6
    with tb.Propagator() as p:
        p.build_sample(smp, 20.0, flags=flags)
        lo, hi, m = N.tbpm_spectral_bounds(p.ctx, 64)
    rlo, rhi, rm = lanczos.extremes(smp, 64)
    assert m == rm
    scale = max(abs(rlo), abs(rhi))
    assert abs(lo - rlo) < tol * scale and abs(hi - rhi) < tol * scale


def test_gpu_build_refuses_s_below_the_lanczos_radius(tb):
    """The 5 nm twisted-bilayer flake (spectrum [-11.64, 6.92] eV by exact
    diagonalisation): s = 10 eV is refused, s = 12 eV accepted; pristine
    graphene (edges +-8.1 eV): s = 7.9 refused, s = 8.3 accepted."""
    N = tb._native
    tbg = workloads.twisted_bilayer_flake(side_nm=5.0).sample
    ev = np.linalg.eigvalsh(exact.dense_h(tbg))
    assert 11.6 < -ev[0] < 11.7
    gr = lattice.graphene(20, 20, pbc=True)
    with tb.Propagator() as p:
        for smp, s_bad, s_ok in ((tbg, 10.0, 12.0), (gr, 7.9, 8.3)):
            with pytest.raises(N.TbpmError) as e:
                p.build_sample(smp, s_bad)
            assert e.value.code == N.TBPM_E_SPECTRAL_BOUND
            p.build_sample(smp, s_ok)
            p.set_phase_states(rng.phases(4, 1, smp.n_orb))
            c = p.propagate(Z, 20, 0)
            assert abs(p.norms()[0, 0, -1] - 1) < 1e-12
        st = p.stats()
    assert st["lanczos_radius"] == 0.0 or st["lanczos_radius"] < 1 / 1.01

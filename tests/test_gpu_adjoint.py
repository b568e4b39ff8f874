"""GPU adjoint (gradients of a DOS loss) against the oracle's reverse-mode
gradient and against central finite differences of the GPU forward map."""
import math

import numpy as np
import pytest

import oracle
from tbpm_inputs import lattice, rng, workloads

pytestmark = pytest.mark.gpu

Z = math.pi / 2


@pytest.fixture(scope="module")
def tb():
    import paper_2209_00806_gb300 as tb
    return tb


@pytest.mark.parametrize("K", [7, 64])
def test_gpu_adjoint_vs_oracle_gradient(tb, K):
    smp = lattice.graphene(8, 7, pbc=True, seed=12, onsite_w=0.4, bond_sigma=0.05)
    n_steps, S, s = 40, 3, 9.5
    th = rng.phases(31, S, smp.n_orb)
    gen = np.random.default_rng(5)
    gbar = gen.normal(size=(S, n_steps + 1)) + 1j * gen.normal(size=(S, n_steps + 1))
    ref_h, ref_o = oracle.gradient(smp, s, Z, n_steps, oracle.phase_states(th), gbar)
    with tb.Propagator() as p:
        p.build_sample(smp, s)
        p.set_phase_states(th)
        gh, go = p.adjoint(Z, n_steps, gbar[None], K=K)
    scale = max(np.max(np.abs(ref_h)), np.max(np.abs(ref_o)))
    assert np.max(np.abs(gh - ref_h)) < 1e-11 * scale
    assert np.max(np.abs(go - ref_o)) < 1e-11 * scale


def test_gpu_adjoint_multi_sample(tb):
    parts = [lattice.graphene(L, L + 1, pbc=True, seed=L, onsite_w=0.3, bond_sigma=0.05)
             for L in (4, 6)]
    smp, offs = lattice.concat(parts)
    n_steps, S, s = 25, 2, 9.5
    ths = [rng.phases(60 + k, S, q.n_orb) for k, q in enumerate(parts)]
    gen = np.random.default_rng(1)
    gbar = gen.normal(size=(2, S, n_steps + 1)) + 1j * gen.normal(size=(2, S, n_steps + 1))
    with tb.Propagator() as p:
        p.build_sample(smp, s, sample_offsets=offs)
        p.set_phase_states(np.concatenate(ths, axis=1))
        gh, go = p.adjoint(Z, n_steps, gbar, K=10)
    nb = 0
    for k, q in enumerate(parts):
        rh, ro = oracle.gradient(q, s, Z, n_steps, oracle.phase_states(ths[k]), gbar[k])
        assert np.max(np.abs(gh[nb:nb + q.n_hop] - rh)) < 1e-11 * np.max(np.abs(rh))
        assert np.max(np.abs(go[offs[k]:offs[k + 1]] - ro)) < 1e-11 * np.max(np.abs(rh))
        nb += q.n_hop


def test_gpu_dos_loss_gradient_full_size_vs_finite_differences(tb):
    """The differentiated workload: 512x512 graphene (524,288 orbitals),
    t_b = -2.7 (1 + 0.05 xi), eps ~ U[-0.2, 0.2], 3 states, 512 steps,
    checkpoints every 64, loss = sum_E (D - D_pristine)^2 on 1024 bins.
    Central differences (h = 1e-6) on 64 sampled parameters."""
    import torch
    from paper_2209_00806_gb300.autograd import TbpmDos
    w = workloads.differentiable_graphene()
    pw = workloads.pristine_like(w)
    dev = torch.device("cuda")
    th = torch.as_tensor(w.thetas()[0], device=dev)
    hi = torch.as_tensor(w.sample.hop_i, device=dev)
    hj = torch.as_tensor(w.sample.hop_j, device=dev)
    f = TbpmDos(w.sample.n_orb, hi, hj, th, w.s, w.z, w.n_steps, w.e_range, w.n_energies, K=64)
    with torch.no_grad():
        target = f(torch.as_tensor(pw.sample.hop_v, device=dev),
                   torch.zeros(w.sample.n_orb, dtype=torch.float64, device=dev))
    hv = torch.as_tensor(w.sample.hop_v, device=dev).requires_grad_(True)
    on = torch.as_tensor(w.sample.onsite, device=dev).requires_grad_(True)
    loss = ((f(hv, on) - target) ** 2).sum()
    loss.backward()
    gh = hv.grad.cpu().numpy()
    go = on.grad.cpu().numpy()
    gen = np.random.default_rng(64)
    bonds = gen.choice(w.sample.n_hop, 32, replace=False)
    sites = gen.choice(w.sample.n_orb, 32, replace=False)
    h = 1e-6

    def L(hv_, on_):
        with torch.no_grad():
            return float(((f(hv_, on_) - target) ** 2).sum())

    fd_h, fd_o = [], []
    for b in bonds:
        a = hv.detach().clone(); a[b] += h
        m = hv.detach().clone(); m[b] -= h
        fd_h.append((L(a, on.detach()) - L(m, on.detach())) / (2 * h))
    for i in sites:
        a = on.detach().clone(); a[i] += h
        m = on.detach().clone(); m[i] -= h
        fd_o.append((L(hv.detach(), a) - L(hv.detach(), m)) / (2 * h))
    fd = np.array(fd_h + fd_o)
    ad = np.concatenate([gh[bonds], go[sites]])
    f.close()
    scale = max(1.0, np.max(np.abs(fd)))
    assert np.max(np.abs(ad - fd)) <= 1e-5 * scale
    # and relative to the gradient's own size
    assert np.max(np.abs(ad - fd)) <= 2e-3 * np.max(np.abs(fd)), (ad, fd)

"""The allocation-free correlation entry point, for callers that cannot
allocate device memory (a framework whose pool owns the device, a plugin that
may only allocate at start-up, a latency-bound loop).  It must give what
tbpm_propagate's own closing reduction gives for the same states, on two
calls in a row through the shared fixed scratch.  Collected last on purpose:
it also has to pass after every other test has run in the same process."""
import ctypes
import math

import numpy as np
import pytest

from tbpm_inputs import lattice, rng

pytestmark = pytest.mark.gpu

Z = math.pi / 2


def test_noalloc_correlation_matches_propagate_twice():
    import torch

    import paper_2209_00806_gb300 as tb
    N = tb._native
    smp = lattice.graphene(26, 21, pbc=True, seed=77, onsite_w=1.0, vacancy_frac=0.02)
    S, n = 5, smp.n_orb
    th = rng.phases(404, S, n)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    with tb.Propagator(0) as p:
        p.build_sample(smp, 9.5)
        p.set_phase_states(th)
        p.propagate(Z, 0)
        psi0 = torch.as_tensor(p.states(), device=dev)           # library-made psi0
        refs = []
        for steps in (30, 45):
            c = p.propagate(Z, steps)
            refs.append((c[0, :, steps], p.norms()[0, :, steps],
                         torch.as_tensor(p.states(), device=dev)))
    corr = torch.empty(S, dtype=torch.complex128, device=dev)
    norm = torch.empty(S, dtype=torch.float64, device=dev)
    for c_ref, n_ref, phi in refs:                                # two calls in a row
        rc = N.lib.tbpm_correlation_noalloc(N.ptr(psi0), N.ptr(phi), n, S, N.ptr(corr),
                                            N.ptr(norm), ctypes.c_void_p(stream))
        assert rc == N.TBPM_OK, N.tbpm_last_error(None)
        torch.cuda.synchronize(dev)
        assert np.max(np.abs(corr.cpu().numpy() - c_ref)) < 1e-10
        assert np.max(np.abs(norm.cpu().numpy() - n_ref)) < 1e-10
        # and, independently of the library, against numpy's inner products
        a, b = psi0.cpu().numpy(), phi.cpu().numpy()
        for k in range(S):
            assert abs(corr[k].item() - np.vdot(a[k], b[k])) < 1e-12
            assert abs(norm[k].item() - np.vdot(b[k], b[k]).real) < 1e-12


def test_noalloc_many_rows_and_all_sixteen_states_twice():
    """More rows than one pass of the fixed grid covers (2048 blocks x 256
    threads = 524,288), so every thread loops and every partial slot is
    used, with the 16 states the scratch holds; two calls in a row (the
    tickets must start from zero again), against numpy's FP64 sums."""
    import torch

    import paper_2209_00806_gb300 as tb
    N = tb._native
    n, S = 600_001, 16
    gen = np.random.default_rng(2024)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    corr = torch.empty(S, dtype=torch.complex128, device=dev)
    norm = torch.empty(S, dtype=torch.float64, device=dev)
    for call in range(2):
        a = gen.normal(size=(S, n)) + 1j * gen.normal(size=(S, n))
        b = gen.normal(size=(S, n)) + 1j * gen.normal(size=(S, n))
        da, db = torch.as_tensor(a, device=dev), torch.as_tensor(b, device=dev)
        rc = N.lib.tbpm_correlation_noalloc(N.ptr(da), N.ptr(db), n, S, N.ptr(corr),
                                            N.ptr(norm), ctypes.c_void_p(stream))
        assert rc == N.TBPM_OK, N.tbpm_last_error(None)
        torch.cuda.synchronize(dev)
        c, nn = corr.cpu().numpy(), norm.cpu().numpy()
        for k in range(S):
            ref = np.vdot(a[k], b[k])
            nref = np.vdot(b[k], b[k]).real
            assert abs(c[k] - ref) < 1e-12 * np.sum(np.abs(a[k]) * np.abs(b[k])), (call, k)
            assert abs(nn[k] - nref) < 1e-12 * nref, (call, k)


def test_noalloc_rejects_too_many_states():
    import torch

    import paper_2209_00806_gb300 as tb
    N = tb._native
    x = torch.zeros((17, 8), dtype=torch.complex128, device="cuda")
    out = torch.zeros(17, dtype=torch.complex128, device="cuda")
    nrm = torch.zeros(17, dtype=torch.float64, device="cuda")
    rc = N.lib.tbpm_correlation_noalloc(N.ptr(x), N.ptr(x), 8, 17, N.ptr(out), N.ptr(nrm), None)
    assert rc == N.TBPM_E_INVALID_ARG
    assert "n_states must be 1..16" in N.tbpm_last_error(None)

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

"""Object wrapper over the C ABI: one context, one Hamiltonian, its states.

Marshalling only -- every step runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import _native as N


class Propagator:
    """Owns a library context on ``device`` (ordered after ``stream``, a raw
    cudaStream_t address such as ``torch.cuda.current_stream().cuda_stream``)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.ctx = N.tbpm_create(device, stream)
        self.n_samples = 1
        self.n_states = 0
        self.n_orb = 0
        self.s = None

    def close(self):
        if self.ctx is not None:
            N.tbpm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # a1
    def build(self, n_orb, onsite, hop_i, hop_j, hop_v, s, sample_offsets=None, flags=0):
        """Arrays are numpy (host) or torch CUDA tensors (device), all alike."""
        n_samples = 1 if sample_offsets is None else len(sample_offsets) - 1
        N.tbpm_build_hamiltonian(self.ctx, int(n_orb), onsite, int(hop_i.shape[0]), hop_i,
                                 hop_j, hop_v, float(s), n_samples, sample_offsets,
                                 N.where_of(hop_i), flags)
        self.n_samples = n_samples
        self.n_hop = int(hop_i.shape[0])
        self.n_orb = int(n_orb)
        self.s = float(s)
        return self

    def build_sample(self, sample, s, sample_offsets=None, flags=0):
        """Complex hoppings (Peierls phases) select TBPM_BUILD_COMPLEX_HOPS."""
        hv = sample.hop_v
        if np.iscomplexobj(hv):
            hv = np.ascontiguousarray(hv, dtype=np.complex128)
            flags |= N.TBPM_BUILD_COMPLEX_HOPS
        else:
            hv = _c64(hv)
        return self.build(sample.n_orb, _c64(sample.onsite), _ci64(sample.hop_i),
                          _ci64(sample.hop_j), hv, s, sample_offsets, flags)

    def set_phase_states(self, theta):
        self.n_states = int(theta.shape[0])
        N.tbpm_set_phase_states(self.ctx, self.n_states, theta)
        return self

    def set_states(self, psi0):
        self.n_states = int(psi0.shape[0])
        N.tbpm_set_states(self.ctx, self.n_states, psi0)
        return self

    def launch_config(self, precision, max_group, threads, variant=N.TBPM_VARIANT_ZIGZAG):
        N.tbpm_set_launch_config(self.ctx, precision, max_group, threads, variant)
        return self

    def autotune(self, z, precision=N.TBPM_FP64, probe_steps=4) -> dict:
        """Pick the fastest launch shape for this Hamiltonian and these states."""
        return N.tbpm_autotune(self.ctx, precision, float(z), probe_steps)

    # a2-a6
    def propagate(self, z, n_steps, precision=N.TBPM_FP64, out=None, flags=0):
        """C [n_samples, n_states, n_steps + 1] complex128 (numpy unless ``out``)."""
        if out is None:
            out = np.empty((self.n_samples, self.n_states, n_steps + 1), dtype=np.complex128)
        N.tbpm_propagate(self.ctx, float(z), int(n_steps), precision, out, None, flags)
        return out

    # c1, c3 (Sec. 2.7)
    def set_bond_vectors(self, dr):
        """Bond vectors r_j - r_i [n_hop, >= 2] in nm, in bond-list order."""
        dr = np.asarray(dr, dtype=np.float64)
        N.tbpm_set_bond_vectors(self.ctx, np.ascontiguousarray(dr[:, 0]),
                                np.ascontiguousarray(dr[:, 1]))
        return self

    def ac_correlation(self, z, n_steps, beta, mu=0.0, precision=N.TBPM_FP64, flags=0):
        """<psi_2(t)|J_a|psi_1b(t)> as complex128 [n_samples, n_states, 4, n_steps + 1],
        ab = xx, xy, yx, yy."""
        out = np.empty((self.n_samples, self.n_states, 4, n_steps + 1), dtype=np.complex128)
        N.tbpm_ac_correlation(self.ctx, float(z), int(n_steps), float(beta), float(mu),
                              precision, out, None, flags)
        return out

    # q1 (Sec. 2.6)
    def quasi_eigenstates(self, z, n_steps, energies, precision=N.TBPM_FP64, flags=0):
        """(states [K, n_states, n_orb] complex128 of unit norm per sample,
        squared norms before normalisation [K, n_states, n_samples])."""
        e = np.atleast_1d(np.asarray(energies, dtype=np.float64))
        out = np.empty((e.shape[0], self.n_states, self.n_orb), dtype=np.complex128)
        norms = np.empty((e.shape[0], self.n_states, self.n_samples))
        N.tbpm_quasi_eigenstates(self.ctx, float(z), int(n_steps), e, precision, out, norms,
                                 None, flags)
        return out, norms

    def correlation(self, out=None):
        """State-averaged C [n_samples, n_steps + 1] of the last propagation
        (numpy unless ``out``, which may be a CUDA tensor)."""
        if out is None:
            out = np.empty((self.n_samples, self.stats()["n_steps"] + 1), dtype=np.complex128)
        N.tbpm_correlation(self.ctx, out)
        return out

    def correlation_adjoint(self, n_steps, gbar_avg, out=None):
        """dL/dC per state [n_samples, n_states, n_steps + 1] from dL/dC-bar
        [n_samples, n_steps + 1] (the adjoint of the state average)."""
        if out is None:
            if N.where_of(gbar_avg) == N.TBPM_DEVICE:
                import torch
                out = torch.empty((self.n_samples, self.n_states, n_steps + 1),
                                  dtype=torch.complex128, device=gbar_avg.device)
            else:
                out = np.empty((self.n_samples, self.n_states, n_steps + 1), dtype=np.complex128)
        if isinstance(gbar_avg, np.ndarray):
            gbar_avg = np.ascontiguousarray(gbar_avg, dtype=np.complex128)
        N.tbpm_correlation_adjoint(self.ctx, int(n_steps), gbar_avg, out)
        return out

    def states(self):
        out = np.empty((self.n_states, self.n_orb), dtype=np.complex128)
        N.tbpm_get_states(self.ctx, out)
        return out

    def norms(self):
        out = np.empty((self.n_samples, self.n_states, self.stats()["n_steps"] + 1))
        N.tbpm_get_norms(self.ctx, out)
        return out

    # a8
    def adjoint(self, z, n_steps, gbar, K=64, n_hop=None):
        """(dL/dt_b, dL/deps_i) for gbar [n_samples, n_states, n_steps + 1]
        = dL/dRe C + i dL/dIm C (numpy or CUDA tensor)."""
        if n_hop is None:
            n_hop = self.n_hop
        if N.where_of(gbar) == N.TBPM_DEVICE:
            import torch
            gh = torch.empty(n_hop, dtype=torch.float64, device=gbar.device)
            go = torch.empty(self.n_orb, dtype=torch.float64, device=gbar.device)
        else:
            gbar = np.ascontiguousarray(gbar, dtype=np.complex128)
            gh = np.empty(n_hop)
            go = np.empty(self.n_orb)
        N.tbpm_propagate_adjoint(self.ctx, float(z), int(n_steps), gbar, N.where_of(gbar),
                                 int(K), gh, go)
        return gh, go

    def stats(self) -> dict:
        return N.tbpm_get_stats(self.ctx)


def dos(corr_avg, tau, e_min, e_max, n_e, window=N.TBPM_WINDOW_HANN):
    """(energies, D) from one averaged correlation C_0 .. C_N (host FP64)."""
    c = np.ascontiguousarray(corr_avg, dtype=np.complex128)
    en = np.empty(n_e)
    d = np.empty(n_e)
    N.tbpm_dos(c, c.shape[0] - 1, tau, window, e_min, e_max, n_e, en, d)
    return en, d


def dos_adjoint(dl_dd, n_steps, tau, e_min, e_max, window=N.TBPM_WINDOW_HANN):
    """gbar_n [n_steps + 1] of the averaged correlation from dL/dD (host FP64)."""
    d = np.ascontiguousarray(dl_dd, dtype=np.float64)
    out = np.empty(n_steps + 1, dtype=np.complex128)
    N.tbpm_dos_adjoint(d, d.shape[0], n_steps, tau, window, e_min, e_max, out)
    return out


def fermi_coefficients(beta_s, mu_s):
    """Chebyshev coefficients c_0 .. c_{K-1} of the Fermi function on the
    rescaled axis (c_0/2 convention; host FP64)."""
    return N.tbpm_fermi_coefficients(float(beta_s), float(mu_s))


def ac_conductivity(corr, tau, beta, eta, omegas, norm):
    """Re sigma [..., n_omega] for correlation rows corr [..., n_steps + 1]
    (host FP64; units e^2/hbar with norm = N_orb / area)."""
    c = np.ascontiguousarray(corr, dtype=np.complex128)
    lead = c.shape[:-1]
    rows = int(np.prod(lead)) if lead else 1
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    out = np.empty(lead + (om.shape[0],))
    N.tbpm_ac_conductivity(c, rows, c.shape[-1] - 1, float(tau), float(beta), float(eta), om,
                           om.shape[0], float(norm), out)
    return out


def _c64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ci64(a):
    return np.ascontiguousarray(a, dtype=np.int64)

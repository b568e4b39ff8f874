"""CPU FP64 oracle of the AC-conductivity correlation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may use this module (it is part of the ``oracle`` package, see
its header).  It follows the paper's steps in its order and notation, using
NumPy's FFT and the C oracle's Hamiltonian product and time step as library
primitives:

  Fermi-Dirac operator (Sec. 2.2): f(x) = z e^{-b x} / (1 + z e^{-b x}) with
  b = beta s (beta~) and fugacity z = e^{beta mu}, i.e. 1 / (e^{b (x - mu/s)} + 1)
  on the rescaled axis; f(H~) = c_0/2 + sum_{k>=1} c_k T_k(H~) with
  c_k = (2/N) Re sum_n f(cos(2 pi n / N)) e^{2 pi i n k / N} (the trapezoid rule
  of the defining integral, evaluated by FFT as the paper says), and the
  real Chebyshev recurrence T_{k+1} = 2 H~ T_k - T_{k-1}, T_0 = 1, T_1 = H~.
  Current operator (Sec. 2.7): J = -i sum_{ij} t_ij (r_j - r_i) c_i^+ c_j, with
  the charge e / hbar left out (units eV nm); r_j - r_i is the bond vector,
  given per bond (a periodic bond carries its own image).
  Two states (Sec. 2.7): psi_1(t) = e^{-iHt} [1 - f(H)] J_b psi(0) and
  psi_2(t) = e^{-iHt} f(H) psi(0); the correlation is <psi_2(t)| J_a |psi_1(t)>.
  Real part of the conductivity (Sec. 2.7, Eq. AC): the time integral of
  e^{-eta t} sin(omega t) 2 Im C(t) by the trapezoid rule on the step grid,
  times (e^{-beta omega} - 1) / omega and a caller-given normalisation.

Readings of points the paper leaves open (kept with the design notes): the
expansion uses the c_0/2 convention of the first displayed series (the
second one writes the sum from k = 0 without the half); the FFT length is
the first power of two >= 4 (K + 1) for a K-term series; K is the last index
with |c_k| > 1e-15 max|c| (plus one); E -> 0+ is a caller-given damping eta
>= 0; the sample area enters as the caller's normalisation factor.

Parity pinned: series against f(x) at random points; f(H~) against exact
diagonalisation; J against -i [H, X]; the correlation against exact
diagonalisation; the conductivity integral against its closed form for a
two-level system (tests named ``test_oracle_ac_*``).
"""
from __future__ import annotations

import numpy as np

from . import propagate

FERMI_TOL = 1e-15


def fermi(x, beta_s: float, mu_s: float):
    """1 / (exp(beta_s (x - mu_s)) + 1), evaluated without overflow."""
    a = beta_s * (np.asarray(x, dtype=np.float64) - mu_s)
    out = np.empty_like(a)
    pos = a > 0
    e = np.exp(-a[pos])
    out[pos] = e / (1.0 + e)
    out[~pos] = 1.0 / (1.0 + np.exp(a[~pos]))
    return out


def fermi_coefficients(beta_s: float, mu_s: float, k_max: int = 1 << 20) -> np.ndarray:
    """c_0 .. c_{K-1} of f on [-1, 1] (c_0/2 convention)."""
    n = 1024
    while True:
        theta = 2.0 * np.pi * np.arange(n) / n
        c = (2.0 / n) * np.real(np.fft.ifft(fermi(np.cos(theta), beta_s, mu_s)) * n)
        c = c[: n // 2]
        big = np.nonzero(np.abs(c) > FERMI_TOL * np.max(np.abs(c)))[0]
        K = int(big[-1]) + 1
        if 4 * (K + 1) <= n or n >= 4 * k_max:
            break
        n *= 2
    if K > k_max:
        raise ValueError("Fermi series longer than k_max")
    return c[:K].copy()


def fermi_apply(sample, s: float, beta_s: float, mu_s: float, v: np.ndarray) -> np.ndarray:
    """f(H~) v by the forward real Chebyshev recurrence."""
    from . import apply_h
    c = fermi_coefficients(beta_s, mu_s)
    v = np.ascontiguousarray(v, dtype=np.complex128)
    t_prev = v.copy()
    acc = 0.5 * c[0] * t_prev
    if len(c) == 1:
        return acc
    t_cur = apply_h(sample, s, v)
    acc = acc + c[1] * t_cur
    for k in range(2, len(c)):
        t_next = 2.0 * apply_h(sample, s, t_cur) - t_prev
        acc = acc + c[k] * t_next
        t_prev, t_cur = t_cur, t_next
    return acc


def current_apply(sample, d_a: np.ndarray, v: np.ndarray) -> np.ndarray:
    """J_a v with (J_a)_ij = -i t_ij d^a_ij over the bond list (d_ij = r_j - r_i,
    the bond vector, given per bond) and its conjugate partner
    (J_a)_ji = -i conj(t_ij) (-d^a_ij); units eV nm."""
    v = np.ascontiguousarray(v, dtype=np.complex128)
    i, j = sample.hop_i, sample.hop_j
    t = np.asarray(sample.hop_v, dtype=np.complex128)
    d = np.asarray(d_a, dtype=np.float64)
    y = np.zeros_like(v)
    np.add.at(y, i, -1j * t * d * v[j])
    np.add.at(y, j, -1j * np.conj(t) * (-d) * v[i])
    return y


def ac_states(sample, s: float, beta: float, mu: float, dr: np.ndarray,
              psi0: np.ndarray):
    """psi_2(0) = f psi0 and psi_1(0)_b = [1 - f] J_b psi0 for b = x, y."""
    beta_s, mu_s = beta * s, mu / s
    psi2 = fermi_apply(sample, s, beta_s, mu_s, psi0)
    psi1 = []
    for b in range(2):
        jb = current_apply(sample, dr[:, b], psi0)
        psi1.append(jb - fermi_apply(sample, s, beta_s, mu_s, jb))
    return psi2, psi1


def ac_correlation(sample, s: float, z: float, n_steps: int, beta: float, mu: float,
                   dr: np.ndarray, psi0: np.ndarray) -> np.ndarray:
    """corr[p, ab, n] = <psi_2(n tau)| J_a |psi_1(n tau)>_b for every state p,
    ab = xx, xy, yx, yy (a = current direction, b = perturbation); dr are the
    bond vectors [n_hop, 2]."""
    psi0 = np.atleast_2d(np.asarray(psi0, dtype=np.complex128))
    S = psi0.shape[0]
    out = np.empty((S, 4, n_steps + 1), dtype=np.complex128)
    for p in range(S):
        psi2, psi1 = ac_states(sample, s, beta, mu, dr, psi0[p])
        for n in range(n_steps + 1):
            ja = [current_apply(sample, dr[:, a], psi2) for a in range(2)]
            for a in range(2):
                for b in range(2):
                    # <psi_2|J_a|psi_1> = <J_a psi_2|psi_1> (J_a is Hermitian)
                    out[p, 2 * a + b, n] = np.vdot(ja[a], psi1[b])
            if n == n_steps:
                break
            st = np.stack([psi2, psi1[0], psi1[1]])
            _, _, st = propagate(sample, s, z, 1, st, want_norms=True, want_psi=True)
            psi2, psi1 = st[0], [st[1], st[2]]
    return out


def ac_conductivity(corr: np.ndarray, tau: float, beta: float, eta: float,
                    omegas: np.ndarray, norm: float) -> np.ndarray:
    """Re sigma(omega) for each row of corr [..., n_steps + 1]:
    norm (e^{-beta omega} - 1) / omega * trapz_t e^{-eta t} sin(omega t) 2 Im C(t)."""
    corr = np.asarray(corr, dtype=np.complex128)
    n_steps = corr.shape[-1] - 1
    t = tau * np.arange(n_steps + 1)
    w = np.full(n_steps + 1, tau)
    w[0] = w[-1] = 0.5 * tau
    out = np.empty(corr.shape[:-1] + (len(omegas),))
    for k, om in enumerate(omegas):
        g = np.exp(-eta * t) * np.sin(om * t) * 2.0 * corr.imag
        out[..., k] = norm * (np.exp(-beta * om) - 1.0) / om * np.sum(g * w, axis=-1)
    return out

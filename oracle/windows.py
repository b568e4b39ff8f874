"""CPU FP64 oracle of the windowed DOS transform -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may use this module (it is part of the ``oracle`` package, see
its header).  Sec. 2.4, Eq. dos_tbpm, with the three windows the paper names
(Hann, Gaussian, exponential; it gives no parameters).  Written out as the
plain direct sum at each bin centre:

  D(E) = (tau/pi) [ Re C_0 / 2 + sum_{n=1}^{N} v_n w_n Re(e^{i E n tau} C_n) ],
  v_n = 1 (n < N), v_N = 1/2   (trapezoid rule on [0, N tau], C(-t) = conj C(t)),

  Hann         w_n = (1 + cos(pi n / N)) / 2
  Gaussian     w_n = exp(-(3 n / N)^2 / 2)     (sigma = N / 3)
  exponential  w_n = exp(-4 n / N)

Readings (kept with the design notes): the Gaussian and exponential widths
above.  Parity pinned: the Hann case equals the C oracle's ``dos``; the
exponential window against the closed form of its geometric series for one
level; every window integrates to Re C_0 over one period (tests
``test_oracle_windows_*``).
"""
from __future__ import annotations

import numpy as np

HANN, GAUSSIAN, EXPONENTIAL = 0, 1, 2


def weights(kind: int, n_steps: int) -> np.ndarray:
    """v_n w_n for n = 0 .. N (the n = 0 entry is unused)."""
    x = np.arange(n_steps + 1) / n_steps
    if kind == HANN:
        w = 0.5 * (1.0 + np.cos(np.pi * x))
    elif kind == GAUSSIAN:
        w = np.exp(-0.5 * (3.0 * x) ** 2)
    elif kind == EXPONENTIAL:
        w = np.exp(-4.0 * x)
    else:
        raise ValueError("unknown window")
    w = w.copy()
    w[-1] *= 0.5
    return w


def dos(corr_avg, tau: float, e_min: float, e_max: float, n_e: int, kind: int = HANN):
    c = np.asarray(corr_avg, dtype=np.complex128)
    n_steps = c.shape[0] - 1
    w = weights(kind, n_steps)
    de = (e_max - e_min) / n_e
    en = e_min + (np.arange(n_e) + 0.5) * de
    d = np.empty(n_e)
    n = np.arange(1, n_steps + 1)
    for k, E in enumerate(en):
        d[k] = tau / np.pi * (0.5 * c[0].real + np.sum(w[1:] * np.real(np.exp(1j * E * n * tau)
                                                                        * c[1:])))
    return en, d

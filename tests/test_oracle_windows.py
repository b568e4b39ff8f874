"""Pins of the windowed DOS oracle (Sec. 2.4): Hann equals the C oracle, the
exponential window has a geometric-series closed form for one level, and
every window keeps the DOS normalised over one period."""
import math

import numpy as np
import pytest

import oracle
from oracle import windows


def test_oracle_windows_hann_equals_c_oracle():
    gen = np.random.default_rng(5)
    c = gen.normal(size=301) + 1j * gen.normal(size=301)
    en, d = windows.dos(c, 0.13, -5.0, 5.0, 333, windows.HANN)
    en2, d2 = oracle.dos(c, 0.13, -5.0, 5.0, 333)
    assert np.allclose(en, en2, rtol=0, atol=1e-15)
    assert np.max(np.abs(d - d2)) < 1e-12


def test_oracle_windows_exponential_single_level_closed_form():
    N, tau, E0 = 500, 0.11, 0.77
    c = np.exp(-1j * E0 * tau * np.arange(N + 1))
    en, d = windows.dos(c, tau, -3.0, 3.0, 257, windows.EXPONENTIAL)
    r0 = math.exp(-4.0 / N)
    q = r0 * np.exp(1j * (en - E0) * tau)
    geo = q * (1 - q ** (N - 1)) / (1 - q)            # sum_{n=1}^{N-1} q^n
    ref = tau / math.pi * (0.5 + geo.real + 0.5 * (q ** N).real)
    assert np.max(np.abs(d - ref)) < 1e-12


@pytest.mark.parametrize("kind", [windows.HANN, windows.GAUSSIAN, windows.EXPONENTIAL])
def test_oracle_windows_normalised_over_a_period(kind):
    """Over one period 2 pi / tau with more bins than steps the sum of
    cos(E n tau) over the bins vanishes for 0 < n <= N: sum D dE = Re C_0."""
    gen = np.random.default_rng(6)
    N, tau = 120, 0.2
    c = gen.normal(size=N + 1) + 1j * gen.normal(size=N + 1)
    n_e = 400
    en, d = windows.dos(c, tau, -math.pi / tau, math.pi / tau, n_e, kind)
    assert abs(np.sum(d) * (2 * math.pi / tau / n_e) - c[0].real) < 1e-12

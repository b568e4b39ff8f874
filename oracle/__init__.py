"""CPU FP64 oracle of the TBPM path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it; the only common input is the seeded generator
package ``tbpm_inputs``.

The arithmetic lives in ``tbpm_oracle.c`` (plain C99, FP64, built with gcc by
:func:`build`); this module only marshals numpy arrays.  Pins that tie the
oracle to something other than itself (exact diagonalisation, the dimer
closed form, the Bloch-sum solution of pristine graphene, SciPy's Bessel
functions, invariants) live in ``tests/``.

Parity pinned: Bessel table, H x, propagation, correlation and DOS (see the
tests named ``test_oracle_*``).  The AC-conductivity path (Fermi-Dirac
operator, current operator, two-state correlation, conductivity integral)
is in ``oracle/ac.py``, pinned by ``tests/test_oracle_ac.py``; the
quasi-eigenstates (Sec. 2.6) in ``oracle/quasi.py``, pinned by
``tests/test_oracle_quasi.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "tbpm_oracle.c"
_SRCS = [_SRC, _HERE / "tbpm_oracle_rows.c"]
_LIB_PATH = _HERE / "_build" / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain -O2, IEEE arithmetic, no fast-math,
    no FMA contraction under -std=c99); OpenMP only in the row-parallel twin."""
    _LIB_PATH.parent.mkdir(exist_ok=True)
    newest = max(p.stat().st_mtime for p in _SRCS)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < newest:
        tmp = _LIB_PATH.with_suffix(f".so.{os.getpid()}")
        subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-D_GNU_SOURCE",
                        "-fopenmp", "-o", str(tmp), *map(str, _SRCS), "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB_PATH))
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_bessel.argtypes = [f64, i32, P]
        lib.oracle_n_terms.argtypes = [f64]
        lib.oracle_apply_h.argtypes = [i64, P, i64, P, P, P, P, f64, P, P]
        lib.oracle_apply_h.restype = None
        lib.oracle_gershgorin.argtypes = [i64, P, i64, P, P, P, P]
        lib.oracle_gershgorin.restype = f64
        lib.oracle_phase_state.argtypes = [i64, P, P]
        lib.oracle_phase_state.restype = None
        lib.oracle_propagate.argtypes = [i64, P, i64, P, P, P, P, f64, f64, i32, i32,
                                         P, P, P, P]
        lib.oracle_dos.argtypes = [P, i32, f64, f64, f64, i32, P, P]
        lib.oracle_gradient.argtypes = [i64, P, i64, P, P, P, f64, f64, i32, i32, P, P, P, P]
        lib.oracle_dos_adjoint.argtypes = [P, i32, f64, f64, f64, i32, P]
        lib.oracle_propagate_rows.argtypes = [i64, P, i64, P, P, P, P, f64, f64, i32, i32,
                                              P, P, P, P]
        lib.oracle_threads.argtypes = []
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _hops(sample):
    hi = np.ascontiguousarray(sample.hop_i, dtype=np.int64)
    hj = np.ascontiguousarray(sample.hop_j, dtype=np.int64)
    hv = np.asarray(sample.hop_v)
    re = np.ascontiguousarray(hv.real, dtype=np.float64)
    im = np.ascontiguousarray(hv.imag, dtype=np.float64) if np.iscomplexobj(hv) else None
    return hi, hj, re, im


def bessel(z: float, m_max: int) -> np.ndarray:
    out = np.zeros(m_max + 1)
    if _load().oracle_bessel(z, m_max, _p(out)) != 0:
        raise ValueError(f"oracle Bessel series refuses z={z}")
    return out


def n_terms(z: float) -> int:
    m = _load().oracle_n_terms(z)
    if m < 0:
        raise ValueError(f"no truncation for z={z}")
    return m


def apply_h(sample, s: float, x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.empty_like(x)
    hi, hj, re, im = _hops(sample)
    ons = _f64(sample.onsite)
    _load().oracle_apply_h(sample.n_orb, _p(ons), sample.n_hop, _p(hi), _p(hj), _p(re),
                           _p(im), s, _p(x), _p(y))
    return y


def gershgorin(sample) -> float:
    hi, hj, re, im = _hops(sample)
    ons = _f64(sample.onsite)
    return _load().oracle_gershgorin(sample.n_orb, _p(ons), sample.n_hop, _p(hi), _p(hj),
                                     _p(re), _p(im))


def phase_states(theta: np.ndarray) -> np.ndarray:
    theta = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
    out = np.empty(theta.shape, dtype=np.complex128)
    for p in range(theta.shape[0]):
        _load().oracle_phase_state(theta.shape[1], _p(theta[p]), _p(out[p]))
    return out


def threads() -> int:
    """Threads the row-parallel twin uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().oracle_threads())


def propagate_rows(sample, s: float, z: float, n_steps: int, psi0: np.ndarray,
                   want_norms: bool = False, want_psi: bool = False):
    """:func:`propagate` by the paper's OpenMP-over-rows scheme on all host
    cores: bit-identical states, correlations and norms to about one rounding."""
    return propagate(sample, s, z, n_steps, psi0, want_norms, want_psi, _rows=True)


def propagate(sample, s: float, z: float, n_steps: int, psi0: np.ndarray,
              want_norms: bool = False, want_psi: bool = False, _rows: bool = False):
    """Returns corr [S, n_steps+1] (and norms [S, n_steps+1], psi [S, N])."""
    psi0 = np.ascontiguousarray(np.atleast_2d(psi0), dtype=np.complex128)
    S, n = psi0.shape
    if n != sample.n_orb:
        raise ValueError("state length does not match the sample")
    corr = np.empty((S, n_steps + 1), dtype=np.complex128)
    norms = np.empty((S, n_steps + 1)) if want_norms else None
    psi = np.empty((S, n), dtype=np.complex128) if want_psi else None
    hi, hj, re, im = _hops(sample)
    ons = _f64(sample.onsite)
    fn = _load().oracle_propagate_rows if _rows else _load().oracle_propagate
    rc = fn(n, _p(ons), sample.n_hop, _p(hi), _p(hj), _p(re), _p(im), s, z, n_steps, S,
            _p(psi0), _p(corr), _p(norms), _p(psi))
    if rc != 0:
        raise RuntimeError(f"oracle_propagate failed ({rc})")
    out = [corr]
    if want_norms:
        out.append(norms)
    if want_psi:
        out.append(psi)
    return out[0] if len(out) == 1 else tuple(out)


def dos(corr_avg: np.ndarray, tau: float, e_min: float, e_max: float, n_e: int):
    """(energies, D) from the state-averaged correlation C_0 .. C_{n_steps}."""
    c = np.ascontiguousarray(corr_avg, dtype=np.complex128)
    n_steps = c.shape[0] - 1
    en = np.empty(n_e)
    d = np.empty(n_e)
    rc = _load().oracle_dos(_p(c), n_steps, tau, e_min, e_max, n_e, _p(en), _p(d))
    if rc != 0:
        raise ValueError("bad DOS arguments")
    return en, d


def gradient(sample, s: float, z: float, n_steps: int, psi0: np.ndarray, gbar: np.ndarray):
    """(dL/dt_b [n_hop], dL/deps_i [n_orb]) for a loss with
    gbar[p, n] = dL/dRe C_n^(p) + i dL/dIm C_n^(p).  Real hoppings only."""
    psi0 = np.ascontiguousarray(np.atleast_2d(psi0), dtype=np.complex128)
    gbar = np.ascontiguousarray(np.atleast_2d(gbar), dtype=np.complex128)
    S, n = psi0.shape
    if gbar.shape != (S, n_steps + 1):
        raise ValueError("gbar must be [n_states, n_steps + 1]")
    if np.iscomplexobj(sample.hop_v):
        raise ValueError("gradients need real hoppings")
    hi, hj, re, _ = _hops(sample)
    ons = _f64(sample.onsite)
    gh = np.empty(sample.n_hop)
    go = np.empty(n)
    rc = _load().oracle_gradient(n, _p(ons), sample.n_hop, _p(hi), _p(hj), _p(re), s, z,
                                 n_steps, S, _p(psi0), _p(gbar), _p(gh), _p(go))
    if rc != 0:
        raise RuntimeError(f"oracle_gradient failed ({rc})")
    return gh, go


def dos_adjoint(dl_dd: np.ndarray, n_steps: int, tau: float, e_min: float, e_max: float):
    """gbar_n of the averaged correlation from dL/dD on the DOS grid."""
    d = np.ascontiguousarray(dl_dd, dtype=np.float64)
    out = np.empty(n_steps + 1, dtype=np.complex128)
    rc = _load().oracle_dos_adjoint(_p(d), n_steps, tau, e_min, e_max, d.shape[0], _p(out))
    if rc != 0:
        raise ValueError("bad DOS adjoint arguments")
    return out

"""ctypes binding of the C ABI in ``include/tbpm.h`` (argument marshalling only).

Every function here has the name and argument order of the C entry point it
wraps; arrays are numpy arrays (host) or torch CUDA tensors (device) and are
passed as raw pointers.  All arithmetic of the propagation path runs in the
CUDA library; if ``libtbpm.so`` is missing or cannot load, importing this
module raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libtbpm.so"

TBPM_OK = 0
TBPM_E_INVALID_ARG = 1
TBPM_E_SPECTRAL_BOUND = 2
TBPM_E_OOM = 3
TBPM_E_CUDA = 4
TBPM_E_NORM_DRIFT = 5
TBPM_E_NONFINITE = 6
TBPM_E_TIMEOUT = 7
TBPM_E_STATE = 8
TBPM_E_UNSUPPORTED = 9
ERROR_NAMES = {1: "INVALID_ARG", 2: "SPECTRAL_BOUND", 3: "OOM", 4: "CUDA", 5: "NORM_DRIFT",
               6: "NONFINITE", 7: "TIMEOUT", 8: "STATE", 9: "UNSUPPORTED"}

TBPM_FP64 = 0
TBPM_FP32 = 1
TBPM_HOST = 0
TBPM_DEVICE = 1
TBPM_WINDOW_HANN = 0
TBPM_WINDOW_GAUSSIAN = 1
TBPM_WINDOW_EXPONENTIAL = 2
TBPM_BUILD_STRICT_BOUND = 1
TBPM_BUILD_NO_FP64 = 2
TBPM_BUILD_NO_FP32 = 4
TBPM_BUILD_REORDER_RCM = 8
TBPM_BUILD_NO_UNIFORM = 16
TBPM_BUILD_COMPLEX_HOPS = 32
TBPM_BUILD_REORDER_CLUSTER = 64
TBPM_BUILD_NO_BOND_MAP = 128
TBPM_BUILD_NO_SPECTRAL_CHECK = 256
TBPM_PROP_PROFILE = 1
TBPM_PROP_GRAPH = 2
TBPM_PROP_RESUME = 4
TBPM_PROP_PERSISTENT = 8
TBPM_PROP_BACKWARD = 16
TBPM_VARIANT_ZIGZAG = 1
TBPM_VARIANT_STREAM_HINTS = 2
TBPM_VARIANT_TMA = 4
TBPM_VARIANT_FUSED = 8
TBPM_VARIANT_WIDE = 64
TBPM_VARIANT_SPLIT2 = 128
TBPM_VARIANT_SPLIT4 = 256
TBPM_VARIANT_HALO = 512
TBPM_VARIANT_PIPE = 1024
TBPM_VARIANT_CLUSTER = 2048
TBPM_VARIANT_STAGED = 4096
TBPM_VARIANT_PREFETCH = 8192


class TbpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"TBPM_E_{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class tbpm_stats(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("n_groups", ctypes.c_int), ("group_width", ctypes.c_int * 8),
                ("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("nnz_true", ctypes.c_int64), ("renormalisations", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("gershgorin", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_term_avg", ctypes.c_double),
                ("ms_final_avg", ctypes.c_double), ("ms_reduce_avg", ctypes.c_double),
                ("term_launches", ctypes.c_int64), ("bytes_term", ctypes.c_double),
                ("max_norm_drift", ctypes.c_double), ("lanczos_radius", ctypes.c_double),
                ("ops_term", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["group_width"] = list(self.group_width)[: self.n_groups]
        return d


P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int
_F64 = ctypes.c_double

# (name, restype, argtypes) of every entry point declared in include/tbpm.h
SIGNATURES = [
    ("tbpm_version", _I32, []),
    ("tbpm_create", _I32, [ctypes.POINTER(P), _I32, P]),
    ("tbpm_destroy", None, [P]),
    ("tbpm_last_error", ctypes.c_char_p, [P]),
    ("tbpm_build_hamiltonian", _I32, [P, _I64, P, _I64, P, P, P, _F64, _I32, P, _I32, _I32]),
    ("tbpm_spectral_bounds", _I32, [P, _I32, ctypes.POINTER(_F64), ctypes.POINTER(_F64),
                                     ctypes.POINTER(_I32)]),
    ("tbpm_set_states", _I32, [P, _I32, P, _I32]),
    ("tbpm_set_phase_states", _I32, [P, _I32, P, _I32]),
    ("tbpm_bessel_coefficients", _I32, [_F64, _F64, _I32, P, ctypes.POINTER(_I32)]),
    ("tbpm_propagate", _I32, [P, _F64, _I32, _I32, P, _I32, _I32]),
    ("tbpm_correlation", _I32, [P, P, _I32]),
    ("tbpm_correlation_adjoint", _I32, [P, _I32, P, _I32, P, _I32]),
    ("tbpm_kernel_binary_version", _I32, [ctypes.POINTER(_I32)]),
    ("tbpm_fp64_fma_rate", _I32, [_I32, _I32, ctypes.POINTER(_F64), ctypes.POINTER(_F64)]),
    ("tbpm_get_states", _I32, [P, P, _I32]),
    ("tbpm_get_norms", _I32, [P, P]),
    ("tbpm_dos", _I32, [P, _I32, _F64, _I32, _F64, _F64, _I32, P, P]),
    ("tbpm_propagate_adjoint", _I32, [P, _F64, _I32, P, _I32, _I32, P, P, _I32]),
    ("tbpm_dos_adjoint", _I32, [P, _I32, _I32, _F64, _I32, _F64, _F64, P]),
    ("tbpm_set_launch_config", _I32, [P, _I32, _I32, _I32, _I32]),
    ("tbpm_set_norm_policy", _I32, [P, _F64, _F64, _F64]),
    ("tbpm_correlation_noalloc", _I32, [P, P, _I64, _I32, P, P, P]),
    ("tbpm_autotune", _I32, [P, _I32, _F64, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                             ctypes.POINTER(_I32), ctypes.POINTER(_F64)]),
    ("tbpm_get_stats", _I32, [P, ctypes.POINTER(tbpm_stats)]),
    ("tbpm_set_bond_vectors", _I32, [P, P, P, _I32]),
    ("tbpm_fermi_coefficients", _I32, [_F64, _F64, _I32, P, ctypes.POINTER(_I32)]),
    ("tbpm_ac_correlation", _I32, [P, _F64, _I32, _F64, _F64, _I32, P, _I32, _I32]),
    ("tbpm_ac_conductivity", _I32, [P, _I32, _I32, _F64, _F64, _F64, P, _I32, _F64, P]),
    ("tbpm_quasi_eigenstates", _I32, [P, _F64, _I32, _I32, P, _I32, P, P, _I32, _I32]),
]


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"{_LIB_PATH} is missing: run __graft_entry__.build() (the TBPM "
                          "library has no CPU fallback)")
    lib = ctypes.CDLL(str(_LIB_PATH))
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def ptr(a):
    """Raw pointer of a numpy array, a torch tensor, an int address or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def where_of(a) -> int:
    if a is not None and hasattr(a, "is_cuda") and a.is_cuda:
        return TBPM_DEVICE
    return TBPM_HOST


def check(ctx, rc: int):
    if rc != TBPM_OK:
        msg = lib.tbpm_last_error(ctx)
        raise TbpmError(rc, msg.decode() if msg else "")
    return rc


# ---- thin wrappers with the C names ----------------------------------------

def tbpm_version() -> int:
    return lib.tbpm_version()


def tbpm_create(device: int = 0, stream: int | None = None):
    h = P()
    check(None, lib.tbpm_create(ctypes.byref(h), device, stream))
    return h


def tbpm_destroy(ctx) -> None:
    lib.tbpm_destroy(ctx)


def tbpm_last_error(ctx) -> str:
    m = lib.tbpm_last_error(ctx)
    return m.decode() if m else ""


def tbpm_build_hamiltonian(ctx, n_orb, onsite, n_hop, hop_i, hop_j, hop_v, s, n_samples=1,
                           sample_offsets=None, where=None, flags=0):
    if where is None:
        where = where_of(hop_i)
    offs = None
    if sample_offsets is not None:
        offs = np.ascontiguousarray(sample_offsets, dtype=np.int64)
    return check(ctx, lib.tbpm_build_hamiltonian(ctx, n_orb, ptr(onsite), n_hop, ptr(hop_i),
                                                 ptr(hop_j), ptr(hop_v), s, n_samples,
                                                 ptr(offs), where, flags))


def tbpm_spectral_bounds(ctx, n_iter=64):
    lo, hi, m = _F64(), _F64(), _I32()
    check(ctx, lib.tbpm_spectral_bounds(ctx, n_iter, ctypes.byref(lo), ctypes.byref(hi),
                                        ctypes.byref(m)))
    return lo.value, hi.value, m.value


def tbpm_set_states(ctx, n_states, psi0, where=None):
    return check(ctx, lib.tbpm_set_states(ctx, n_states, ptr(psi0),
                                          where_of(psi0) if where is None else where))


def tbpm_set_phase_states(ctx, n_states, theta, where=None):
    return check(ctx, lib.tbpm_set_phase_states(ctx, n_states, ptr(theta),
                                                where_of(theta) if where is None else where))


def tbpm_bessel_coefficients(z: float, tol: float = 1e-15, max_terms: int = 128):
    J = np.zeros(max_terms)
    n = _I32()
    check(None, lib.tbpm_bessel_coefficients(z, tol, max_terms, ptr(J), ctypes.byref(n)))
    return J[: n.value]


def tbpm_propagate(ctx, z, n_steps, precision, corr_out=None, where_out=None, flags=0):
    if where_out is None:
        where_out = where_of(corr_out)
    return check(ctx, lib.tbpm_propagate(ctx, z, n_steps, precision, ptr(corr_out), where_out,
                                         flags))


def tbpm_correlation(ctx, out, where_out=None):
    return check(ctx, lib.tbpm_correlation(ctx, ptr(out),
                                           where_of(out) if where_out is None else where_out))


def tbpm_correlation_adjoint(ctx, n_steps, gbar_avg, gbar_out, where=None, where_out=None):
    if where is None:
        where = where_of(gbar_avg)
    if where_out is None:
        where_out = where_of(gbar_out)
    return check(ctx, lib.tbpm_correlation_adjoint(ctx, n_steps, ptr(gbar_avg), where,
                                                   ptr(gbar_out), where_out))


def tbpm_kernel_binary_version() -> int:
    v = _I32()
    check(None, lib.tbpm_kernel_binary_version(ctypes.byref(v)))
    return v.value


def tbpm_fp64_fma_rate(device=0, n_iter=200000):
    t, ms = _F64(), _F64()
    check(None, lib.tbpm_fp64_fma_rate(device, n_iter, ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def tbpm_get_states(ctx, out, where_out=None):
    return check(ctx, lib.tbpm_get_states(ctx, ptr(out),
                                          where_of(out) if where_out is None else where_out))


def tbpm_get_norms(ctx, out):
    return check(ctx, lib.tbpm_get_norms(ctx, ptr(out)))


def tbpm_dos(corr, n_steps, tau, window, e_min, e_max, n_e, energies_out, dos_out):
    return check(None, lib.tbpm_dos(ptr(corr), n_steps, tau, window, e_min, e_max, n_e,
                                    ptr(energies_out), ptr(dos_out)))


def tbpm_propagate_adjoint(ctx, z, n_steps, gbar, where, K, grad_hop, grad_onsite,
                           where_out=None):
    if where_out is None:
        where_out = where_of(grad_hop)
    return check(ctx, lib.tbpm_propagate_adjoint(ctx, z, n_steps, ptr(gbar), where, K,
                                                 ptr(grad_hop), ptr(grad_onsite), where_out))


def tbpm_dos_adjoint(dl_dd, n_e, n_steps, tau, window, e_min, e_max, gbar_out):
    return check(None, lib.tbpm_dos_adjoint(ptr(dl_dd), n_e, n_steps, tau, window, e_min,
                                            e_max, ptr(gbar_out)))


def tbpm_set_norm_policy(ctx, renorm_fp32=1e-5, hard_fp32=1e-2, hard_fp64=1e-6):
    return check(ctx, lib.tbpm_set_norm_policy(ctx, renorm_fp32, hard_fp32, hard_fp64))


def tbpm_autotune(ctx, precision, z, probe_steps=4):
    g, t, v, ms = _I32(), _I32(), _I32(), _F64()
    check(ctx, lib.tbpm_autotune(ctx, precision, z, probe_steps, ctypes.byref(g),
                                 ctypes.byref(t), ctypes.byref(v), ctypes.byref(ms)))
    return dict(group=g.value, threads=t.value, variant=v.value, ms_per_step=ms.value)


def tbpm_correlation_noalloc(psi0, phi, n_orb, n_states, corr_out, norm_out, stream=None):
    return check(None, lib.tbpm_correlation_noalloc(ptr(psi0), ptr(phi), n_orb, n_states,
                                                    ptr(corr_out), ptr(norm_out), stream))


def tbpm_set_bond_vectors(ctx, dx, dy, where=None):
    return check(ctx, lib.tbpm_set_bond_vectors(ctx, ptr(dx), ptr(dy),
                                                where_of(dx) if where is None else where))


def tbpm_fermi_coefficients(beta_s: float, mu_s: float, k_max: int = 1 << 22):
    n = _I32()
    check(None, lib.tbpm_fermi_coefficients(beta_s, mu_s, k_max, None, ctypes.byref(n)))
    c = np.zeros(n.value)
    check(None, lib.tbpm_fermi_coefficients(beta_s, mu_s, n.value, ptr(c), ctypes.byref(n)))
    return c


def tbpm_ac_correlation(ctx, z, n_steps, beta, mu, precision, corr_out, where_out=None,
                        flags=0):
    if where_out is None:
        where_out = where_of(corr_out)
    return check(ctx, lib.tbpm_ac_correlation(ctx, z, n_steps, beta, mu, precision,
                                              ptr(corr_out), where_out, flags))


def tbpm_ac_conductivity(corr, n_rows, n_steps, tau, beta, eta, omegas, n_omega, norm,
                         sigma_out):
    return check(None, lib.tbpm_ac_conductivity(ptr(corr), n_rows, n_steps, tau, beta, eta,
                                                ptr(omegas), n_omega, norm, ptr(sigma_out)))


def tbpm_quasi_eigenstates(ctx, z, n_steps, energies, precision, out, norms_out=None,
                           where_out=None, flags=0):
    e = np.ascontiguousarray(energies, dtype=np.float64)
    if where_out is None:
        where_out = where_of(out)
    return check(ctx, lib.tbpm_quasi_eigenstates(ctx, z, n_steps, e.shape[0], ptr(e), precision,
                                                 ptr(out), ptr(norms_out), where_out, flags))


def tbpm_set_launch_config(ctx, precision, max_group, threads, variant=1):
    return check(ctx, lib.tbpm_set_launch_config(ctx, precision, max_group, threads, variant))


def tbpm_get_stats(ctx) -> dict:
    s = tbpm_stats()
    check(ctx, lib.tbpm_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()

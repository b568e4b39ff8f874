"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point ``include/tbpm.h`` declares, and its pure-host functions
(Bessel table, DOS transform, Fermi coefficients, conductivity transform)
agree with the oracle and SciPy.  No GPU."""
import math
import re
from pathlib import Path

import numpy as np
import pytest
import scipy.special

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__._build_module().build()
    from paper_2209_00806_gb300 import _native
    return _native


def declared_functions():
    text = (ROOT / "include" / "tbpm.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tbpm_[a-z_0-9]+)\s*\(", text)))


def test_binding_constants_match_the_header(native):
    """Every integer TBPM_* constant of the header has the same value in the
    Python binding (variant bits, build and propagation flags, statuses)."""
    text = (ROOT / "include" / "tbpm.h").read_text()
    defs = dict(re.findall(r"#define\s+(TBPM_[A-Z0-9_]+)\s+(-?\d+)\b", text))
    assert len(defs) > 20
    missing = [k for k in defs if not hasattr(native, k)]
    assert not missing, missing
    wrong = {k: (v, getattr(native, k)) for k, v in defs.items() if getattr(native, k) != int(v)}
    assert not wrong, wrong


def test_library_exports_every_declared_symbol(native):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(native.lib, n), n
    bound = {s[0] for s in native.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_library_is_built_for_sm103a(native):
    """Every CUDA source is compiled for sm_103a and nothing else (the GPU
    test reads the loaded image's version through tbpm_kernel_binary_version)."""
    import __graft_entry__
    bn = __graft_entry__._build_module()
    assert bn.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert any(s.suffix == ".cu" for s in bn.sources())


def test_no_device_gives_a_status_not_a_crash(native):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(native.TbpmError) as e:
        native.tbpm_create(0)
    assert e.value.code == native.TBPM_E_CUDA


@pytest.mark.parametrize("z", [0.3, math.pi / 2, math.pi, 7.5, 40.0, 300.0])
def test_bessel_table_vs_scipy(native, z):
    J = native.tbpm_bessel_coefficients(z, max_terms=int(z) + 100)
    M = len(J)
    ref = scipy.special.jv(np.arange(M + 1), z)
    assert np.max(np.abs(J - ref[:M])) < 1e-15 * max(1.0, math.sqrt(z))
    assert M > z and abs(ref[M]) < 1e-15
    assert all(not (m > z and abs(ref[m]) < 1e-15) for m in range(M))


def test_bessel_table_matches_oracle_term_count(native):
    import oracle
    for z in (0.5, math.pi / 2, math.pi, 3.9):
        assert len(native.tbpm_bessel_coefficients(z)) == oracle.n_terms(z)
    assert len(native.tbpm_bessel_coefficients(math.pi / 2)) == 16


def test_bessel_table_rejects_bad_z(native):
    for z in (0.0, -1.0, float("nan"), 2000.0):
        with pytest.raises(native.TbpmError):
            native.tbpm_bessel_coefficients(z)


def test_dos_transform_vs_oracle(native):
    import oracle
    from paper_2209_00806_gb300 import dos
    gen = np.random.default_rng(1)
    n = 300
    E = gen.uniform(-3, 3, 40)
    w = gen.uniform(0, 1, 40)
    w /= w.sum()
    tau = 0.15
    c = np.exp(-1j * np.outer(np.arange(n + 1) * tau, E)) @ w
    en, d = dos(c, tau, -4.0, 4.0, 777)
    en2, d2 = oracle.dos(c, tau, -4.0, 4.0, 777)
    assert np.array_equal(en, en2)
    assert np.max(np.abs(d - d2)) < 1e-12
    with pytest.raises(native.TbpmError):
        dos(c, tau, 1.0, -1.0, 10)


def test_dos_adjoint_vs_oracle(native):
    import oracle
    from paper_2209_00806_gb300 import dos_adjoint
    gen = np.random.default_rng(3)
    dl = gen.normal(size=513)
    for n in (10, 200, 1024):
        g = dos_adjoint(dl, n, 0.165, -9.5, 9.5)
        ref = oracle.dos_adjoint(dl, n, 0.165, -9.5, 9.5)
        assert np.max(np.abs(g - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("beta_s,mu_s", [(367.0, 0.0), (40.0, 0.2), (3.0, -0.5)])
def test_fermi_coefficients_vs_oracle(native, beta_s, mu_s):
    from oracle import ac
    from paper_2209_00806_gb300 import fermi_coefficients
    c = fermi_coefficients(beta_s, mu_s)
    ref = ac.fermi_coefficients(beta_s, mu_s)
    assert len(c) == len(ref)
    assert np.max(np.abs(c - ref)) < 1e-14
    with pytest.raises(native.TbpmError):
        fermi_coefficients(-1.0, 0.0)


def test_ac_conductivity_transform_vs_oracle(native):
    from oracle import ac
    from paper_2209_00806_gb300 import ac_conductivity
    gen = np.random.default_rng(4)
    tau, n = 0.17, 900
    E = gen.uniform(-2, 2, (3, 12))
    w = gen.normal(size=(3, 12)) + 1j * gen.normal(size=(3, 12))
    t = tau * np.arange(n + 1)
    corr = np.stack([np.exp(1j * np.outer(t, E[r])) @ w[r] for r in range(3)])
    om = np.linspace(0.05, 3.0, 37)
    got = ac_conductivity(corr, tau, 12.0, 0.01, om, 2.5)
    ref = ac.ac_conductivity(corr, tau, 12.0, 0.01, om, 2.5)
    assert got.shape == (3, 37)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    with pytest.raises(native.TbpmError):
        ac_conductivity(corr, tau, 12.0, 0.01, np.array([0.0]), 1.0)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_dos_windows_vs_oracle(native, kind):
    from oracle import windows
    from paper_2209_00806_gb300 import dos
    gen = np.random.default_rng(11)
    c = gen.normal(size=257) + 1j * gen.normal(size=257)
    en, d = dos(c, 0.21, -6.0, 6.0, 401, window=kind)
    en2, d2 = windows.dos(c, 0.21, -6.0, 6.0, 401, kind)
    assert np.max(np.abs(en - en2)) < 1e-14
    assert np.max(np.abs(d - d2)) < 1e-12
    with pytest.raises(native.TbpmError):
        dos(c, 0.21, -6.0, 6.0, 401, window=7)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_dos_adjoint_windows_is_the_transpose(native, kind):
    """dL/dC of L = dl . D(C): the DOS map is linear in (Re C, Im C), so the
    adjoint is its transpose, built here column by column from the oracle."""
    from oracle import windows
    from paper_2209_00806_gb300 import dos_adjoint
    n, n_e, tau = 40, 97, 0.3
    dl = np.random.default_rng(12).normal(size=n_e)
    ref = np.empty(n + 1, dtype=np.complex128)
    for m in range(n + 1):
        e = np.zeros(n + 1, dtype=np.complex128)
        e[m] = 1.0
        _, d_re = windows.dos(e, tau, -4.0, 4.0, n_e, kind)
        _, d_im = windows.dos(1j * e, tau, -4.0, 4.0, n_e, kind)
        ref[m] = dl @ d_re + 1j * (dl @ d_im)
    g = dos_adjoint(dl, n, tau, -4.0, 4.0, window=kind)
    assert np.max(np.abs(g - ref)) < 1e-12

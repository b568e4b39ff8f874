"""The synthetic TBPM workloads, each a recipe of sizes and seeded draws.

All workloads use z = s * tau = pi / 2 (hbar = 1, energies in eV), Chebyshev
truncation at |J_m(z)| < 1e-15 and random-phase initial states
psi0_i = exp(i theta_i) / sqrt(N).  Master seed of workload k is
220900806 * 16 + k.  Sizes can be shrunk with ``L=`` for tests; every other
parameter stays as stated.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import lattice, rng

Z_STEP = math.pi / 2.0


def master_seed(k: int) -> int:
    return 220900806 * 16 + k


@dataclass
class Workload:
    name: str
    sample: lattice.Sample
    offsets: np.ndarray            # [n_samples + 1] orbital offsets
    s: float                       # rescale factor (eV)
    z: float                       # s * tau
    n_states: int                  # states per sample
    n_steps: int
    n_energies: int
    e_range: tuple[float, float]
    seed: int
    sample_seeds: list[int] = field(default_factory=list)
    info: dict = field(default_factory=dict)

    @property
    def tau(self) -> float:
        return self.z / self.s

    @property
    def n_samples(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def thetas(self) -> list[np.ndarray]:
        """Per sample: theta[n_states, n_orb_sample]."""
        out = []
        for k in range(self.n_samples):
            n_k = int(self.offsets[k + 1] - self.offsets[k])
            out.append(rng.phases(self.sample_seeds[k], self.n_states, n_k))
        return out


def graphene_dos(L: int = 64, n_steps: int = 1024, n_energies: int = 2048) -> Workload:
    """Plain TBPM DOS in FP64: pristine periodic graphene LxL (64x64 -> 8192
    orbitals), t = -2.7 eV, s = 9 eV, one random-phase state, grid [-9, 9]."""
    seed = master_seed(1)
    smp = lattice.graphene(L, L, pbc=True, seed=seed)
    return Workload("graphene_dos", smp, np.array([0, smp.n_orb], dtype=np.int64), 9.0,
                    Z_STEP, 1, n_steps, n_energies, (-9.0, 9.0), seed, [seed],
                    dict(L=L))


def disordered_graphene(L: int = 2048, n_steps: int = 1024, n_energies: int = 4096,
                        n_states: int = 4) -> Workload:
    """TBPM at scale: periodic graphene LxL (2048^2 -> 8,388,608 sites), Anderson
    onsite eps ~ U[-0.5, 0.5] eV, 1% vacancies, s = 9.5 eV, 4 states."""
    seed = master_seed(2)
    smp = lattice.graphene(L, L, pbc=True, seed=seed, onsite_w=1.0, vacancy_frac=0.01)
    return Workload("disordered_graphene", smp, np.array([0, smp.n_orb], dtype=np.int64),
                    9.5, Z_STEP, n_states, n_steps, n_energies, (-9.5, 9.5), seed, [seed],
                    dict(L=L))


BATCH_SIDES = (256, 384, 512, 768, 1024)


def batch_params(n_samples: int = 32, sides=BATCH_SIDES):
    """Per-sample side length L_k (uniform over ``sides``, counter 2k), Anderson
    width W_k ~ U[0, 2] eV (counter 2k+1) and per-sample seed (counter
    1000 + k), all from stream BATCH of master seed 3."""
    seed = master_seed(3)
    u = rng.uniform(seed, rng.BATCH, 2 * n_samples)
    Ls = [sides[min(int(u[2 * k] * len(sides)), len(sides) - 1)] for k in range(n_samples)]
    Ws = [2.0 * u[2 * k + 1] for k in range(n_samples)]
    raw = rng.u64(seed, rng.BATCH, np.arange(1000, 1000 + n_samples, dtype=np.uint64))
    seeds = [int(v) & 0x7FFFFFFFFFFFFFFF for v in raw]
    return seed, Ls, Ws, seeds


def batched_graphene(n_samples: int = 32, n_states: int = 16, n_steps: int = 512,
                     n_energies: int = 2048, sides=BATCH_SIDES) -> Workload:
    """Batched TBPM: n_samples independent periodic graphene samples of uneven
    size, Anderson eps ~ U[-W/2, W/2], 16 states each, s = 9.5 eV."""
    seed, Ls, Ws, seeds = batch_params(n_samples, sides)
    parts = [lattice.graphene(L, L, pbc=True, seed=sd, onsite_w=W)
             for L, W, sd in zip(Ls, Ws, seeds)]
    smp, offs = lattice.concat(parts)
    return Workload("batched_graphene", smp, offs, 9.5, Z_STEP, n_states, n_steps,
                    n_energies, (-9.5, 9.5), seed, seeds, dict(Ls=Ls, Ws=Ws))


def differentiable_graphene(L: int = 512, n_steps: int = 512, n_energies: int = 1024,
                            n_states: int = 3) -> Workload:
    """Differentiated TBPM: periodic graphene LxL (512^2 -> 524,288 orbitals),
    t_b = -2.7 (1 + 0.05 xi_b), eps ~ U[-0.2, 0.2] eV, 3 states, s = 9.5 eV."""
    seed = master_seed(4)
    smp = lattice.graphene(L, L, pbc=True, seed=seed, onsite_w=0.4, bond_sigma=0.05)
    return Workload("differentiable_graphene", smp,
                    np.array([0, smp.n_orb], dtype=np.int64), 9.5, Z_STEP, n_states,
                    n_steps, n_energies, (-9.5, 9.5), seed, [seed], dict(L=L))


def pristine_like(w: Workload) -> Workload:
    """Same lattice, states, s, z, steps and grid with t = -2.7, eps = 0: the
    target of the differentiated workload's DOS loss."""
    L = w.info["L"]
    smp = lattice.graphene(L, L, pbc=True, seed=w.seed)
    return Workload(w.name + "_pristine", smp, w.offsets.copy(), w.s, w.z, w.n_states,
                    w.n_steps, w.n_energies, w.e_range, w.seed, list(w.sample_seeds),
                    dict(w.info))


def twisted_bilayer_flake(side_nm: float = 100.0, n_states: int = 8, n_steps: int = 1024,
                          n_energies: int = 4096) -> Workload:
    """Twisted bilayer graphene, 1.05 degrees, square open flake of side
    `side_nm` (the 1.2 um flake scaled down), 6 Angstrom Slater-Koster p_z
    cutoff (about 66 entries per row), onsite 0, s = 12 eV (the spectral
    radius of this hopping form exceeds 10 eV), 8 states."""
    seed = master_seed(5)
    smp = lattice.twisted_bilayer(side_nm, seed=seed)
    return Workload("twisted_bilayer", smp, np.array([0, smp.n_orb], dtype=np.int64), 12.0,
                    Z_STEP, n_states, n_steps, n_energies, (-12.0, 12.0), seed, [seed],
                    dict(side_nm=side_nm))


def optical_graphene(L: int = 1024, n_steps: int = 1024, n_states: int = 1) -> Workload:
    """Optical (AC) conductivity: pristine periodic graphene LxL with bond
    vectors (the paper's Sec. 4 example at 1024^2 instead of 4096^2), s = 9 eV,
    T = 300 K, mu = 0, one random state (four propagated lanes)."""
    seed = master_seed(6)
    smp = lattice.graphene(L, L, pbc=True, seed=seed, with_pos=True)
    smp.pos = None                      # the bond vectors carry the geometry
    return Workload("optical_graphene", smp, np.array([0, smp.n_orb], dtype=np.int64), 9.0,
                    Z_STEP, n_states, n_steps, 0, (-9.0, 9.0), seed, [seed],
                    dict(L=L, T_kelvin=300.0, mu=0.0))


def quasi_graphene(L: int = 1024, n_steps: int = 512, n_states: int = 4) -> Workload:
    """Quasi-eigenstates: disordered periodic graphene LxL (Anderson
    U[-0.5, 0.5] eV, 1% vacancies), s = 9.5 eV, 4 states, energies
    -2.7, -1, 0.4, 2 eV."""
    seed = master_seed(7)
    smp = lattice.graphene(L, L, pbc=True, seed=seed, onsite_w=1.0, vacancy_frac=0.01)
    return Workload("quasi_graphene", smp, np.array([0, smp.n_orb], dtype=np.int64), 9.5,
                    Z_STEP, n_states, n_steps, 0, (-9.5, 9.5), seed, [seed],
                    dict(L=L, energies=[-2.7, -1.0, 0.4, 2.0]))

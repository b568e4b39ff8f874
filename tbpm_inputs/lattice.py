"""Synthetic tight-binding samples: orbitals, onsite energies and bond lists.

The graphene primitive cell follows the paper's worked example (Sec. 4.1):
lattice vectors a1 = (0.246, 0, 0) nm and a2 = (0.123, 0.21304, 0) nm,
one p_z orbital at fractional (0, 0) and one at (1/3, 1/3), and the three
reduced nearest-neighbour hoppings (R=(0,0), 0->1), (R=(1,0), 1->0),
(R=(0,1), 1->0), each -2.7 eV.  A bond (i, j, t) means the matrix element
<phi_i|h|phi_j> = t; its conjugate partner (j, i, conj t) is implied and not
listed, matching the paper's halving by the conjugate relation.

A supercell of L1 x L2 primitive cells numbers orbital o of cell (n1, n2) as
2 * (n1 * L2 + n2) + o, so neighbouring cells are at most 2 * L2 orbitals
apart.  Vacancies are removed and the survivors renumbered in ascending
order of their original index; bonds touching a vacancy are dropped.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rng

A1 = np.array([0.246, 0.0])
A2 = np.array([0.123, 0.21304])
T_NN = -2.7


@dataclass
class Sample:
    """One tight-binding sample in the bond-list form the library consumes."""
    n_orb: int
    onsite: np.ndarray | None          # float64 [n_orb] (eV) or None = all zero
    hop_i: np.ndarray                  # int64 [n_hop]
    hop_j: np.ndarray                  # int64 [n_hop]
    hop_v: np.ndarray                  # float64 [n_hop] (eV), real hoppings
    pos: np.ndarray | None = None      # float64 [n_orb, 2] (nm), optional
    meta: dict = field(default_factory=dict)
    dr: np.ndarray | None = None       # float64 [n_hop, 2] bond vectors r_j - r_i (nm)

    @property
    def n_hop(self) -> int:
        return int(self.hop_i.shape[0])


def graphene(L1: int, L2: int, *, pbc: bool = True, t: float = T_NN,
             seed: int = 0, onsite_w: float = 0.0, vacancy_frac: float = 0.0,
             bond_sigma: float = 0.0, with_pos: bool = False) -> Sample:
    """Graphene supercell of L1 x L2 primitive cells.

    onsite_w:     Anderson disorder, eps_i ~ U[-W/2, W/2] (stream ONSITE,
                  counter = original orbital index).
    vacancy_frac: exactly round(frac * 2 L1 L2) sites removed: those with the
                  smallest draws of stream VACANCY (counter = original index).
    bond_sigma:   per-bond hopping t_b = t (1 + sigma xi_b), xi_b ~ N(0, 1)
                  from stream BOND_NOISE with counter = bond index 3 c + k.
    """
    if L1 < 1 or L2 < 1:
        raise ValueError("lattice dimensions must be positive")
    if pbc and (L1 < 3 or L2 < 3):
        raise ValueError("periodic graphene needs L1, L2 >= 3 (no duplicate bonds)")
    n_cell = L1 * L2
    n_full = 2 * n_cell
    c = np.arange(n_cell, dtype=np.int64)
    n1 = c // L2
    n2 = c % L2
    # three reduced hoppings per cell, bond index b = 3 c + k
    a_nb = 2 * c                                   # orbital 0 of this cell
    b_nb = 2 * c + 1                               # orbital 1 of this cell
    c10 = ((n1 + 1) % L1) * L2 + n2                # cell R = (1, 0)
    c01 = n1 * L2 + (n2 + 1) % L2                  # cell R = (0, 1)
    hi = np.stack([a_nb, b_nb, b_nb], axis=1).reshape(-1)
    hj = np.stack([b_nb, 2 * c10, 2 * c01], axis=1).reshape(-1)
    keep_b = np.ones(3 * n_cell, dtype=bool)
    if not pbc:
        keep_b.reshape(n_cell, 3)[:, 1] = n1 + 1 < L1
        keep_b.reshape(n_cell, 3)[:, 2] = n2 + 1 < L2
    if bond_sigma != 0.0:
        xi = rng.normal(seed, rng.BOND_NOISE, 3 * n_cell)
        hv = t * (1.0 + bond_sigma * xi)
    else:
        hv = np.full(3 * n_cell, t, dtype=np.float64)
    onsite = None
    if onsite_w != 0.0:
        onsite = rng.uniform_range(seed, rng.ONSITE, n_full, -0.5 * onsite_w, 0.5 * onsite_w)

    pos = None
    dr = None
    if with_pos:
        pos = np.empty((n_full, 2))
        origin = n1[:, None] * A1[None, :] + n2[:, None] * A2[None, :]
        pos[0::2] = origin
        pos[1::2] = origin + (A1 + A2) / 3.0
        # the three reduced hoppings' vectors (the periodic image of a wrapped
        # bond is the nearest one)
        b1 = (A1 + A2) / 3.0
        dr = np.tile(np.stack([b1, A1 - b1, A2 - b1]), (n_cell, 1))

    n_vac = int(round(vacancy_frac * n_full))
    if n_vac > 0:
        keys = rng.u64(seed, rng.VACANCY, np.arange(n_full, dtype=np.uint64))
        vac = np.argpartition(keys, n_vac - 1)[:n_vac]   # keys are distinct
        alive = np.ones(n_full, dtype=bool)
        alive[vac] = False
        new_id = np.cumsum(alive, dtype=np.int64) - 1
        keep_b &= alive[hi] & alive[hj]
        hi = new_id[hi]
        hj = new_id[hj]
        if onsite is not None:
            onsite = onsite[alive]
        if pos is not None:
            pos = pos[alive]
        n_orb = int(alive.sum())
    else:
        n_orb = n_full
    return Sample(n_orb=n_orb, onsite=onsite,
                  hop_i=np.ascontiguousarray(hi[keep_b]),
                  hop_j=np.ascontiguousarray(hj[keep_b]),
                  hop_v=np.ascontiguousarray(hv[keep_b]),
                  pos=pos, dr=None if dr is None else np.ascontiguousarray(dr[keep_b]),
                  meta=dict(kind="graphene", L1=L1, L2=L2, pbc=pbc, t=t,
                            onsite_w=onsite_w, vacancies=n_vac, bond_sigma=bond_sigma,
                            seed=seed))


def dimer(gamma: float) -> Sample:
    """Two orbitals joined by one bond of strength gamma (eV)."""
    return Sample(n_orb=2, onsite=None,
                  hop_i=np.array([0], dtype=np.int64),
                  hop_j=np.array([1], dtype=np.int64),
                  hop_v=np.array([gamma], dtype=np.float64),
                  meta=dict(kind="dimer", gamma=gamma))


def chain(n: int, t: float = -1.0, *, seed: int = 0, onsite_w: float = 0.0,
          periodic: bool = True) -> Sample:
    """1-D chain (a ring when periodic), used for small exact checks."""
    i = np.arange(n, dtype=np.int64)
    j = (i + 1) % n
    keep = np.ones(n, dtype=bool) if periodic else (i + 1 < n)
    onsite = None
    if onsite_w != 0.0:
        onsite = rng.uniform_range(seed, rng.ONSITE, n, -0.5 * onsite_w, 0.5 * onsite_w)
    return Sample(n_orb=n, onsite=onsite, hop_i=i[keep], hop_j=j[keep],
                  hop_v=np.full(int(keep.sum()), t), meta=dict(kind="chain", n=n))


def random_graph(n: int, n_hop: int, *, seed: int = 0, onsite_w: float = 1.0,
                 t_scale: float = 1.0) -> Sample:
    """Random sparse symmetric structure with no self loops or duplicate pairs:
    irregular row lengths for ragged-slice tests."""
    gen = np.random.default_rng(seed)
    pairs = set()
    hi, hj = [], []
    while len(hi) < n_hop:
        a, b = (int(v) for v in gen.integers(0, n, size=2))
        if a == b or (min(a, b), max(a, b)) in pairs:
            continue
        pairs.add((min(a, b), max(a, b)))
        hi.append(a)
        hj.append(b)
    hv = t_scale * gen.uniform(-1.0, 1.0, size=n_hop)
    onsite = gen.uniform(-0.5 * onsite_w, 0.5 * onsite_w, size=n) if onsite_w else None
    return Sample(n_orb=n, onsite=onsite, hop_i=np.array(hi, dtype=np.int64),
                  hop_j=np.array(hj, dtype=np.int64), hop_v=hv,
                  meta=dict(kind="random_graph", n=n, n_hop=n_hop))


def permute(sample: Sample, perm: np.ndarray) -> Sample:
    """Relabel orbitals: new index of old orbital i is perm[i]."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.shape[0])
    onsite = None if sample.onsite is None else sample.onsite[inv]
    pos = None if sample.pos is None else sample.pos[inv]
    return Sample(n_orb=sample.n_orb, onsite=onsite, hop_i=perm[sample.hop_i],
                  hop_j=perm[sample.hop_j], hop_v=sample.hop_v.copy(), pos=pos,
                  meta=dict(sample.meta, permuted=True), dr=sample.dr)


def concat(samples: list[Sample]) -> tuple[Sample, np.ndarray]:
    """Block-diagonal union of samples; returns it and the orbital offsets
    [n_samples + 1] that delimit each sample."""
    offs = np.zeros(len(samples) + 1, dtype=np.int64)
    for k, s in enumerate(samples):
        offs[k + 1] = offs[k] + s.n_orb
    n = int(offs[-1])
    onsite = np.zeros(n)
    any_onsite = False
    for k, s in enumerate(samples):
        if s.onsite is not None:
            onsite[offs[k]:offs[k + 1]] = s.onsite
            any_onsite = True
    hi = np.concatenate([s.hop_i + offs[k] for k, s in enumerate(samples)])
    hj = np.concatenate([s.hop_j + offs[k] for k, s in enumerate(samples)])
    hv = np.concatenate([s.hop_v for s in samples])
    dr = None
    if all(s.dr is not None or s.pos is not None for s in samples):
        dr = np.concatenate([bond_vectors(s) for s in samples])
    return Sample(n_orb=n, onsite=onsite if any_onsite else None, hop_i=hi, hop_j=hj,
                  hop_v=hv, meta=dict(kind="batch", n_samples=len(samples)), dr=dr), offs


def twisted_bilayer(side_nm: float, theta_deg: float = 1.05, cutoff_nm: float = 0.6,
                    seed: int = 0) -> Sample:
    """Square flake of twisted bilayer graphene with open boundaries.

    Two honeycomb layers (a = 0.246 nm, C-C 0.142 nm) stacked AA at the
    origin, the bottom at z = 0 and the top at z = 0.335 nm rotated by theta
    about the origin; both layers clipped to [-side/2, side/2]^2.  Every pair
    closer than the cutoff is a bond with the two-centre p_z form
        t(d) = Vpp_pi (1 - (z/d)^2) + Vpp_sigma (z/d)^2,
        Vpp_pi = -2.7 exp(-(d - 0.142)/0.045) eV,
        Vpp_sigma = 0.48 exp(-(d - 0.335)/0.045) eV  (d, z in nm),
    and zero onsite energy.  Orbitals are numbered layer by layer (bottom
    first), so interlayer partners are far apart in the numbering.
    """
    from scipy.spatial import cKDTree
    half = 0.5 * side_nm
    reach = int(np.ceil(side_nm / 0.123)) + 4
    n = np.arange(-reach, reach + 1)
    n1, n2 = np.meshgrid(n, n, indexing="ij")
    origin = n1.reshape(-1, 1) * A1 + n2.reshape(-1, 1) * A2
    base = np.concatenate([origin, origin + (A1 + A2) / 3.0])
    layers = []
    for k, ang in enumerate((0.0, np.deg2rad(theta_deg))):
        c, s_ = np.cos(ang), np.sin(ang)
        p = base @ np.array([[c, s_], [-s_, c]])
        p = p[(np.abs(p[:, 0]) <= half) & (np.abs(p[:, 1]) <= half)]
        layers.append(np.column_stack([p, np.full(p.shape[0], 0.335 * k)]))
    pos = np.concatenate(layers)
    pairs = cKDTree(pos).query_pairs(cutoff_nm, output_type="ndarray")
    d_vec = pos[pairs[:, 1]] - pos[pairs[:, 0]]
    d = np.linalg.norm(d_vec, axis=1)
    zz = np.abs(d_vec[:, 2])
    r2 = (zz / d) ** 2
    vpi = -2.7 * np.exp(-(d - 0.142) / 0.045)
    vsig = 0.48 * np.exp(-(d - 0.335) / 0.045)
    hv = vpi * (1.0 - r2) + vsig * r2
    return Sample(n_orb=pos.shape[0], onsite=None,
                  hop_i=np.ascontiguousarray(pairs[:, 0].astype(np.int64)),
                  hop_j=np.ascontiguousarray(pairs[:, 1].astype(np.int64)),
                  hop_v=np.ascontiguousarray(hv), pos=pos[:, :2],
                  meta=dict(kind="twisted_bilayer", side_nm=side_nm, theta_deg=theta_deg,
                            cutoff_nm=cutoff_nm, n_bottom=layers[0].shape[0]))


FLUX_QUANTUM = 4135.667696      # h / e in T nm^2


def peierls(sample: Sample, B_tesla: float) -> Sample:
    """Perpendicular magnetic field by Peierls substitution (Sec. 2.1, and the
    Landau-gauge form of Sec. 4): with A = (B y, 0, 0) the line integral of A
    along the straight bond from orbital i to orbital j is
    B (x_j - x_i) (y_i + y_j) / 2, so t_ij -> t_ij exp(i pi B (x_j - x_i)
    (y_j + y_i) / Phi_0) with Phi_0 = h / e.  Needs orbital positions and
    open boundaries (the Landau gauge is not periodic).  The result has
    complex128 hoppings."""
    if sample.pos is None:
        raise ValueError("the Peierls phases need orbital positions")
    if sample.meta.get("pbc", False):
        raise ValueError("the Landau gauge needs open boundaries")
    x, y = sample.pos[:, 0], sample.pos[:, 1]
    i, j = sample.hop_i, sample.hop_j
    phase = np.pi * B_tesla * (x[j] - x[i]) * (y[j] + y[i]) / FLUX_QUANTUM
    hv = sample.hop_v.astype(np.complex128) * np.exp(1j * phase)
    return Sample(n_orb=sample.n_orb, onsite=sample.onsite, hop_i=i, hop_j=j, hop_v=hv,
                  pos=sample.pos, meta=dict(sample.meta, B_tesla=B_tesla), dr=sample.dr)


def bond_vectors(sample: Sample) -> np.ndarray:
    """r_j - r_i [n_hop, 2] of every bond: the stored vectors when the
    generator made them (periodic images), else differences of positions."""
    if sample.dr is not None:
        return sample.dr
    if sample.pos is None:
        raise ValueError("bond vectors need positions")
    return sample.pos[sample.hop_j, :2] - sample.pos[sample.hop_i, :2]

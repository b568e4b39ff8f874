"""Twisted bilayer graphene flakes of any size, generated with torch on the
GPU (or the CPU): the 1.2 um flake of the large benchmark has ~1.1e8
orbitals and ~3.6e9 bonds, beyond a host k-d tree.

Same construction as :func:`tbpm_inputs.lattice.twisted_bilayer`: two
honeycomb layers (a = 0.246 nm) stacked AA at the origin, the bottom at
z = 0 and the top at z = 0.335 nm rotated by theta about the origin, both
clipped to the square [-side/2, side/2]^2; every pair closer than the cutoff
is a bond with the two-centre p_z hopping
    t(d) = Vpp_pi (1 - (z/d)^2) + Vpp_sigma (z/d)^2,
    Vpp_pi = -2.7 exp(-(d - 0.142)/0.045) eV,
    Vpp_sigma = 0.48 exp(-(d - 0.335)/0.045) eV      (d, z in nm).

Neighbours are found exactly, without a search structure: both layers are
lattices, so a site's in-plane neighbours are fixed lattice offsets, and the
top-layer sites near a bottom site are the lattice points around its
fractional coordinates in the rotated basis.  A dense index map from lattice
coordinates (layer, sublattice, n1, n2) to orbital number makes each lookup
one gather.

Numbering: ``order="layers"`` numbers the orbitals as the k-d tree generator
does (bottom layer first; in a layer sublattice 0 before 1, then n1, then
n2), so the two generators give the same sample.  ``order="morton"`` numbers
them along a Morton (Z-order) curve of 0.5 nm square cells, both layers of a
cell together, so that consecutive orbitals are neighbours in space (the row
order a sparse product over this sample wants).  No TBPM arithmetic is done
here: this is input generation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

A1 = (0.246, 0.0)
A2 = (0.123, 0.21304)
DZ = 0.335


@dataclass
class DeviceSample:
    """A sample whose arrays are torch tensors (on any device)."""
    n_orb: int
    hop_i: "object"           # int64 [n_hop]
    hop_j: "object"           # int64 [n_hop]
    hop_v: "object"           # float64 [n_hop] (eV)
    meta: dict

    @property
    def n_hop(self) -> int:
        return int(self.hop_i.shape[0])


def _hopping(torch, d, zz):
    r2 = (zz / d) ** 2
    vpi = -2.7 * torch.exp(-(d - 0.142) / 0.045)
    vsig = 0.48 * torch.exp(-(d - 0.335) / 0.045)
    return vpi * (1.0 - r2) + vsig * r2


def _ranges(half: float):
    """Lattice-coordinate half ranges (R1, R2) that cover every site of a
    square of half side `half` in any rotation."""
    rad = half * math.sqrt(2.0)
    R2 = int(math.ceil(rad / A2[1])) + 2
    R1 = int(math.ceil((rad + R2 * A2[0]) / A1[0])) + 2
    return R1, R2


def _layer_sites(torch, half, ang, R1, R2, dev):
    """Positions and in-flake mask of one layer's lattice points, in the
    order (sublattice, n1, n2); returns (x, y, mask) as [2, 2R1+1, 2R2+1]."""
    n1 = torch.arange(-R1, R1 + 1, dtype=torch.float64, device=dev)[:, None]
    n2 = torch.arange(-R2, R2 + 1, dtype=torch.float64, device=dev)[None, :]
    xs, ys = [], []
    for o in (0, 1):
        x = n1 * A1[0] + n2 * A2[0]
        y = n1 * A1[1] + n2 * A2[1]
        if o == 1:
            x = x + (A1[0] + A2[0]) / 3.0
            y = y + (A1[1] + A2[1]) / 3.0
        c, s = math.cos(ang), math.sin(ang)
        xs.append(x * c - y * s)
        ys.append(x * s + y * c)
    x = torch.stack(xs)
    y = torch.stack(ys)
    mask = (x.abs() <= half) & (y.abs() <= half)
    return x, y, mask


def _inplane_offsets(cutoff):
    """(o, o2, dn1, dn2, d) of every in-plane neighbour offset within the cutoff."""
    out = []
    tau = ((A1[0] + A2[0]) / 3.0, (A1[1] + A2[1]) / 3.0)
    for o in (0, 1):
        for o2 in (0, 1):
            for d1 in range(-5, 6):
                for d2 in range(-5, 6):
                    if o == o2 and d1 == 0 and d2 == 0:
                        continue
                    dx = d1 * A1[0] + d2 * A2[0] + (o2 - o) * tau[0]
                    dy = d1 * A1[1] + d2 * A2[1] + (o2 - o) * tau[1]
                    d = math.hypot(dx, dy)
                    if d <= cutoff:
                        out.append((o, o2, d1, d2))
    return out


def twisted_bilayer(side_nm: float, theta_deg: float = 1.05, cutoff_nm: float = 0.6,
                    order: str = "morton", device="cpu", chunk: int = 1 << 20,
                    cell_nm: float = 0.5) -> DeviceSample:
    """Square open flake of twisted bilayer graphene as torch tensors on
    ``device``; see the module docstring.  ``chunk`` bounds the sites handled
    at once (memory ~ chunk x 1 kB)."""
    import torch
    dev = torch.device(device)
    half = 0.5 * side_nm
    R1, R2 = _ranges(half)
    G1, G2 = 2 * R1 + 1, 2 * R2 + 1
    ang = math.radians(theta_deg)

    # orbital numbers in the "layers" order: layer, sublattice, n1, n2
    idx = torch.full((2, 2, G1, G2), -1, dtype=torch.int64, device=dev)
    pos = []
    base = 0
    for k, a in enumerate((0.0, ang)):
        x, y, m = _layer_sites(torch, half, a, R1, R2, dev)
        cnt = int(m.sum())
        num = torch.cumsum(m.reshape(-1).to(torch.int64), 0) - 1 + base
        idx[k] = torch.where(m, num.reshape(m.shape), idx[k])
        pos.append((x[m], y[m]))
        base += cnt
        del x, y, m, num
    n_orb = base
    n_bottom = int(pos[0][0].shape[0])
    px = torch.cat([pos[0][0], pos[1][0]])
    py = torch.cat([pos[0][1], pos[1][1]])
    del pos

    # lattice coordinates of every orbital (to walk neighbour offsets)
    lay = torch.zeros(n_orb, dtype=torch.int8, device=dev)
    lay[n_bottom:] = 1
    sub = torch.empty(n_orb, dtype=torch.int8, device=dev)
    c1 = torch.empty(n_orb, dtype=torch.int32, device=dev)
    c2 = torch.empty(n_orb, dtype=torch.int32, device=dev)
    for k in (0, 1):
        for o in (0, 1):
            sel = idx[k, o] >= 0
            ids = idx[k, o][sel]
            nz = sel.nonzero()
            sub[ids] = o
            c1[ids] = (nz[:, 0] - R1).to(torch.int32)
            c2[ids] = (nz[:, 1] - R2).to(torch.int32)
            del sel, ids, nz

    offs = _inplane_offsets(cutoff_nm)
    rho_max = math.sqrt(max(cutoff_nm ** 2 - DZ ** 2, 0.0))
    c, s = math.cos(ang), math.sin(ang)
    tau = ((A1[0] + A2[0]) / 3.0, (A1[1] + A2[1]) / 3.0)
    w1 = range(-4, 6)
    w2 = range(-3, 5)
    win = torch.tensor([(a, b) for a in w1 for b in w2], dtype=torch.int64, device=dev)

    def lookup(k, o2, m1, m2):
        ok = (m1 >= -R1) & (m1 <= R1) & (m2 >= -R2) & (m2 <= R2)
        j = torch.full_like(m1, -1)
        j[ok] = idx[k, o2, m1[ok] + R1, m2[ok] + R2]
        return j

    def bonds_of(lo, hi, emit):
        """Bonds (i, j > i) with i in [lo, hi): in-plane by offsets, and
        interlayer from bottom sites to the top layer."""
        i = torch.arange(lo, hi, dtype=torch.int64, device=dev)
        li, si = lay[lo:hi].long(), sub[lo:hi].long()
        a1, a2 = c1[lo:hi].long(), c2[lo:hi].long()
        for o, o2, d1, d2 in offs:
            sel = si == o
            if not bool(sel.any()):
                continue
            ii, kk = i[sel], li[sel]
            j = torch.where(kk == 0, lookup(0, o2, a1[sel] + d1, a2[sel] + d2),
                            lookup(1, o2, a1[sel] + d1, a2[sel] + d2))
            keep = j > ii
            if bool(keep.any()):
                ii, j = ii[keep], j[keep]
                d = torch.sqrt((px[j] - px[ii]) ** 2 + (py[j] - py[ii]) ** 2)
                emit(ii, j, _hopping(torch, d, torch.zeros_like(d)))
        bot = li == 0
        if not bool(bot.any()) or rho_max <= 0:
            return
        ib = i[bot]
        x, y = px[ib], py[ib]
        # coordinates in the rotated (top) basis
        qx = x * c + y * s
        qy = -x * s + y * c
        for o2 in (0, 1):
            f2 = (qy - o2 * tau[1]) / A2[1]
            f1 = (qx - o2 * tau[0] - f2 * A2[0]) / A1[0]
            m1 = torch.floor(f1).long()[:, None] + win[None, :, 0]
            m2 = torch.floor(f2).long()[:, None] + win[None, :, 1]
            j = lookup(1, o2, m1.reshape(-1), m2.reshape(-1)).reshape(m1.shape)
            ii = ib[:, None].expand_as(j)
            ok = j >= 0
            ii, j = ii[ok], j[ok]
            dx, dy = px[j] - px[ii], py[j] - py[ii]
            d = torch.sqrt(dx * dx + dy * dy + DZ * DZ)
            keep = d <= cutoff_nm
            ii, j, d = ii[keep], j[keep], d[keep]
            emit(ii, j, _hopping(torch, d, torch.full_like(d, DZ)))

    # pass 1: count, pass 2: fill preallocated arrays (no concatenation copies)
    counts = []
    for lo in range(0, n_orb, chunk):
        n = [0]
        bonds_of(lo, min(n_orb, lo + chunk), lambda a, b, v: n.__setitem__(0, n[0] + int(a.numel())))
        counts.append(n[0])
    n_hop = int(sum(counts))
    hop_i = torch.empty(n_hop, dtype=torch.int64, device=dev)
    hop_j = torch.empty(n_hop, dtype=torch.int64, device=dev)
    hop_v = torch.empty(n_hop, dtype=torch.float64, device=dev)
    at = [0]

    def put(a, b, v):
        n = int(a.numel())
        hop_i[at[0]:at[0] + n] = a
        hop_j[at[0]:at[0] + n] = b
        hop_v[at[0]:at[0] + n] = v
        at[0] += n

    for lo in range(0, n_orb, chunk):
        bonds_of(lo, min(n_orb, lo + chunk), put)
    assert at[0] == n_hop
    del idx, lay, sub, c1, c2

    if order == "morton":
        rank = _morton_rank(torch, px, py, half, cell_nm, n_bottom)
        for lo in range(0, n_hop, 1 << 28):
            hi = min(n_hop, lo + (1 << 28))
            hop_i[lo:hi] = rank[hop_i[lo:hi]]
            hop_j[lo:hi] = rank[hop_j[lo:hi]]
        del rank
    elif order != "layers":
        raise ValueError("order must be 'layers' or 'morton'")
    return DeviceSample(n_orb=n_orb, hop_i=hop_i, hop_j=hop_j, hop_v=hop_v,
                        meta=dict(kind="twisted_bilayer", side_nm=side_nm, theta_deg=theta_deg,
                                  cutoff_nm=cutoff_nm, n_bottom=n_bottom, order=order,
                                  cell_nm=cell_nm))


def _spread_bits(torch, v):
    """Put a zero bit after each of the low 31 bits of v (2-D Morton code)."""
    v = v & 0x7FFFFFFF
    v = (v | (v << 16)) & 0x0000FFFF0000FFFF
    v = (v | (v << 8)) & 0x00FF00FF00FF00FF
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0F
    v = (v | (v << 2)) & 0x3333333333333333
    v = (v | (v << 1)) & 0x5555555555555555
    return v


def _morton_rank(torch, px, py, half, cell, n_bottom):
    """New number of every orbital: sorted by the Morton code of its
    cell, then by the old number (bottom layer before top within a cell)."""
    cx = torch.clamp(torch.floor((px + half) / cell), min=0).long()
    cy = torch.clamp(torch.floor((py + half) / cell), min=0).long()
    key = (_spread_bits(torch, cx) | (_spread_bits(torch, cy) << 1))
    n = px.shape[0]
    # stable sort on the Morton key keeps the old order within a cell
    order = torch.sort(key, stable=True).indices
    rank = torch.empty(n, dtype=torch.int64, device=px.device)
    rank[order] = torch.arange(n, dtype=torch.int64, device=px.device)
    return rank


def to_numpy_sample(ds: DeviceSample):
    """The same sample as a host :class:`tbpm_inputs.lattice.Sample`."""
    from .lattice import Sample
    return Sample(n_orb=ds.n_orb, onsite=None,
                  hop_i=np.ascontiguousarray(ds.hop_i.cpu().numpy()),
                  hop_j=np.ascontiguousarray(ds.hop_j.cpu().numpy()),
                  hop_v=np.ascontiguousarray(ds.hop_v.cpu().numpy()), meta=dict(ds.meta))

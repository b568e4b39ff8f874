"""The seeded input generators: SplitMix64 against its published output,
draw ranges, lattice sizes, vacancies, and the workload recipes."""
import numpy as np
import pytest

from tbpm_inputs import lattice, rng, workloads


def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0 yields 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f
    with np.errstate(over="ignore"):
        states = rng.GAMMA * np.arange(1, 4, dtype=np.uint64)
    out = [int(v) for v in rng.mix64(states)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_draws_are_counter_based_and_in_range():
    u = rng.uniform(5, 7, 1000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.array_equal(rng.uniform(5, 7, 10, offset=990), u[990:])
    assert not np.array_equal(rng.uniform(5, 8, 10), u[:10])
    x = rng.normal(9, 1, 200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
    th = rng.phases(3, 2, 100)
    assert th.shape == (2, 100) and th.min() >= 0 and th.max() < 2 * np.pi


def test_graphene_counts_and_vacancies():
    g = lattice.graphene(10, 12, pbc=True)
    assert g.n_orb == 240 and g.n_hop == 360
    pairs = {(min(a, b), max(a, b)) for a, b in zip(g.hop_i, g.hop_j)}
    assert len(pairs) == g.n_hop and all(a != b for a, b in pairs)
    deg = np.bincount(np.concatenate([g.hop_i, g.hop_j]), minlength=g.n_orb)
    assert np.all(deg == 3)
    o = lattice.graphene(10, 12, pbc=False)
    assert o.n_hop == 360 - 12 - 10
    v = lattice.graphene(20, 20, pbc=True, seed=4, vacancy_frac=0.01, onsite_w=1.0)
    assert v.n_orb == 800 - 8 and v.meta["vacancies"] == 8
    assert v.hop_i.max() < v.n_orb and v.hop_j.max() < v.n_orb
    assert v.onsite.shape == (v.n_orb,) and np.all(np.abs(v.onsite) <= 0.5)
    deg = np.bincount(np.concatenate([v.hop_i, v.hop_j]), minlength=v.n_orb)
    assert deg.max() == 3 and deg.min() >= 1


def test_workload_recipes():
    w = workloads.graphene_dos()
    assert w.sample.n_orb == 8192 and w.s == 9.0 and w.n_steps == 1024
    seed, Ls, Ws, seeds = workloads.batch_params()
    assert len(Ls) == 32 and set(Ls) <= set(workloads.BATCH_SIDES)
    assert all(0 <= W < 2 for W in Ws) and len(set(seeds)) == 32
    small = workloads.batched_graphene(n_samples=3, n_states=2, sides=(4, 6))
    assert small.n_samples == 3 and small.offsets[-1] == small.sample.n_orb
    th = small.thetas()
    assert [t.shape for t in th] == [(2, int(small.offsets[k + 1] - small.offsets[k]))
                                     for k in range(3)]


def _hexagon_flux(smp, B):
    """Flux (in units of Phi_0) through each hexagon of an open graphene
    flake, from the product of the Peierls factors around it."""
    pairs = {}
    for b in range(smp.n_hop):
        i, j = int(smp.hop_i[b]), int(smp.hop_j[b])
        pairs[(i, j)] = smp.hop_v[b]
        pairs[(j, i)] = np.conj(smp.hop_v[b])
    L2 = smp.meta["L2"]
    out = []
    # the hexagon around the cell corner shared by cells (n1, n2), (n1+1, n2), (n1, n2+1)
    for n1 in range(smp.meta["L1"] - 1):
        for n2 in range(L2 - 1):
            cell = lambda a, b: 2 * (a * L2 + b)
            ring = [cell(n1, n2) + 1, cell(n1 + 1, n2), cell(n1 + 1, n2) + 1,
                    cell(n1 + 1, n2 + 1), cell(n1, n2 + 1) + 1, cell(n1, n2 + 1)]
            prod = 1.0 + 0j
            ok = True
            for a, b in zip(ring, ring[1:] + ring[:1]):
                if (a, b) not in pairs:
                    ok = False
                    break
                prod *= pairs[(a, b)] / abs(pairs[(a, b)])
            if ok:
                out.append(np.angle(prod) / (2 * np.pi))
    return np.array(out)


def _cell_area():
    return abs(lattice.A1[0] * lattice.A2[1] - lattice.A1[1] * lattice.A2[0])


def test_peierls_flux_per_hexagon():
    """The Peierls factors around every hexagon multiply to exp(+-2 pi i B
    A_hex / Phi_0), A_hex = |a1 x a2| (one hexagon per primitive cell): the
    field is uniform and of the stated strength, whatever the gauge."""
    B = 500.0
    smp = lattice.peierls(lattice.graphene(6, 5, pbc=False, with_pos=True), B)
    assert np.iscomplexobj(smp.hop_v)
    assert np.allclose(np.abs(smp.hop_v), 2.7)
    flux = _hexagon_flux(smp, B)
    assert len(flux) == 20
    expect = B * _cell_area() / lattice.FLUX_QUANTUM
    assert np.allclose(np.abs(flux), expect, rtol=1e-12, atol=1e-15)
    assert np.all(np.sign(flux) == np.sign(flux[0]))


def test_peierls_integer_flux_is_a_gauge_of_zero_field():
    """One flux quantum per hexagon is gauge-equivalent to no field on a
    simply connected flake: the spectrum is that of B = 0."""
    from tests import exact
    base = lattice.graphene(5, 4, pbc=False, with_pos=True, onsite_w=0.7, seed=2)
    B1 = lattice.FLUX_QUANTUM / _cell_area()
    e0 = np.linalg.eigvalsh(exact.dense_h(base))
    e1 = np.linalg.eigvalsh(exact.dense_h(lattice.peierls(base, B1)))
    eh = np.linalg.eigvalsh(exact.dense_h(lattice.peierls(base, 0.5 * B1)))
    assert np.max(np.abs(e1 - e0)) < 1e-9
    assert np.max(np.abs(eh - e0)) > 1e-2


def test_peierls_needs_positions_and_open_boundaries():
    with pytest.raises(ValueError):
        lattice.peierls(lattice.graphene(4, 4, pbc=False), 10.0)
    with pytest.raises(ValueError):
        lattice.peierls(lattice.graphene(4, 4, pbc=True, with_pos=True), 10.0)


def test_graphene_bond_vectors():
    """Open flakes: the generator's bond vectors are differences of the
    positions; periodic lattices: every bond vector has the C-C length (the
    nearest image), also across the wrap."""
    a_cc = np.linalg.norm((lattice.A1 + lattice.A2) / 3.0)
    op = lattice.graphene(7, 5, pbc=False, with_pos=True, vacancy_frac=0.05, seed=3)
    ref = op.pos[op.hop_j] - op.pos[op.hop_i]
    assert np.max(np.abs(op.dr - ref)) < 1e-14
    per = lattice.graphene(6, 5, pbc=True, with_pos=True)
    # (the printed cell vectors are rounded: the three bond lengths agree to 1e-5)
    assert np.allclose(np.linalg.norm(per.dr, axis=1), a_cc, rtol=1e-4)
    wrapped = np.linalg.norm(per.pos[per.hop_j] - per.pos[per.hop_i], axis=1) > 2 * a_cc
    assert wrapped.sum() == 6 + 5       # one wrapped bond per edge cell


def _pair_keys(smp):
    a = np.minimum(smp.hop_i, smp.hop_j).astype(np.int64)
    b = np.maximum(smp.hop_i, smp.hop_j).astype(np.int64)
    k = a * smp.n_orb + b
    o = np.argsort(k)
    return k[o], smp.hop_v[o]


@pytest.mark.parametrize("side", [5.0, 13.0])
def test_tbg_lattice_generator_equals_kd_tree_generator(side):
    """The lattice-enumeration twisted-bilayer generator (torch, any device)
    gives the k-d tree generator's sample: same orbitals, same bonds, the
    same hoppings to rounding; the Morton numbering is a relabelling of it."""
    pytest.importorskip("torch")
    from tbpm_inputs import tbg
    ref = lattice.twisted_bilayer(side)
    lay = tbg.to_numpy_sample(tbg.twisted_bilayer(side, order="layers", chunk=3000))
    assert lay.n_orb == ref.n_orb and lay.n_hop == ref.n_hop
    ka, va = _pair_keys(ref)
    kb, vb = _pair_keys(lay)
    assert np.array_equal(ka, kb)
    assert np.max(np.abs(va - vb)) < 1e-12
    mor = tbg.to_numpy_sample(tbg.twisted_bilayer(side, order="morton"))
    assert mor.n_orb == ref.n_orb and mor.n_hop == ref.n_hop
    # same multiset of (degree, sorted hoppings) per orbital: a relabelling
    deg_l = np.bincount(np.concatenate([lay.hop_i, lay.hop_j]), minlength=lay.n_orb)
    deg_m = np.bincount(np.concatenate([mor.hop_i, mor.hop_j]), minlength=mor.n_orb)
    assert np.array_equal(np.sort(deg_l), np.sort(deg_m))
    assert np.allclose(np.sort(lay.hop_v), np.sort(mor.hop_v), rtol=0, atol=1e-15)
    assert np.all(mor.hop_i != mor.hop_j)


def test_tbg_morton_numbering_is_local():
    """Consecutive orbitals of the Morton numbering are neighbours in space: a
    block of 128 rows references a few hundred distinct rows (its halo),
    against thousands in the layer-by-layer numbering."""
    pytest.importorskip("torch")
    from tbpm_inputs import tbg

    def mean_halo(smp, R=128):
        i = np.concatenate([smp.hop_i, smp.hop_j])
        j = np.concatenate([smp.hop_j, smp.hop_i])
        u = np.unique((i // R) * smp.n_orb + j)
        return np.bincount(u // smp.n_orb).mean()

    mor = tbg.to_numpy_sample(tbg.twisted_bilayer(30.0, order="morton"))
    lay = tbg.to_numpy_sample(tbg.twisted_bilayer(30.0, order="layers"))
    assert mean_halo(mor) < 600 < mean_halo(lay)


def test_phases_torch_equals_numpy():
    pytest.importorskip("torch")
    a = rng.phases(987654321, 3, 70001)
    b = rng.phases_torch(987654321, 3, 70001).numpy()
    assert np.array_equal(a, b)

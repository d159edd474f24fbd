"""Input generators, on the CPU.  The batched uneven workload (48 seeded cubic cells): its draws
stay in the stated ranges, the FFT box is the smallest 2-3-5 size holding the potential's band
without aliasing, and the cell has the Si density of the 8-atom cell.  The 64-atom supercell:
its sites and its 64 perturbations by closed-form shell counts."""
import numpy as np

from instances import generate as G


def test_config4_specs_in_range_and_boxes_alias_free():
    sizes = []
    for seed in range(48):
        sp = G.config4_spec(seed)
        assert 2 <= sp["n_atoms"] <= 64 and 10.0 <= sp["ecut_ry"] <= 25.0
        assert 16 <= sp["n_omega"] <= 256 and 1 <= sp["n_pert"] <= 16
        assert sp["n_occ"] == 2 * sp["n_atoms"] and sp["tau"].shape == (sp["n_atoms"], 3)
        # density: n atoms in L^3 as 8 atoms in 10.26^3
        L = sp["a"][0, 0]
        assert abs(sp["n_atoms"] / L ** 3 - 8 / 10.26 ** 3) < 1e-12
        mil, _ = G.sphere(sp["a"], (0, 0, 0), 4 * sp["ecut_ry"], check_margin=False)
        for i in range(3):
            need = 2 * int(np.abs(mil[:, i]).max()) + 1
            n = sp["dims"][i]
            assert n >= need and G.smooth235(need) == n
            r = n
            for p in (2, 3, 5):
                while r % p == 0:
                    r //= p
            assert r == 1
        sizes.append(sp["n_pw"])
    assert min(sizes) < 300 and max(sizes) > 15000          # uneven: tens to ~18 000 plane waves
    assert G.config4_spec(7)["n_pw"] == G.config4_spec(7)["n_pw"]   # deterministic


def test_smooth235():
    assert [G.smooth235(n) for n in (13, 14, 17, 29, 31, 49, 71)] == [15, 15, 18, 30, 32, 50, 72]


def test_supercell_cell_and_perturbations():
    """The 64-atom supercell: a cube of side 2 x 10.26 bohr holding the 8-atom cell's diamond
    sites in each of its 2 x 2 x 2 subcells; its 64 perturbations are the shells of non-zero
    Miller vectors with |m|^2 = 1, 2, 3, 4, 5 (6 + 12 + 8 + 6 + 24 = 56 vectors) and the 8
    lexicographically smallest of the 24 with |m|^2 = 6 (G = 0 excluded: q = 0)."""
    a, tau = G.supercell64_cell()
    assert np.allclose(a, np.eye(3) * 20.52)
    assert tau.shape == (64, 3)
    frac = tau / 20.52
    assert len({tuple(np.round(f, 9)) for f in frac}) == 64
    # each site is a site of the 8-atom cell (fractions of 10.26) shifted by whole subcells
    sub = (frac * 2) % 1.0
    cell8 = {tuple(np.round(np.asarray(f) % 1.0, 9)) for f in G.DIAMOND_FRAC}
    assert all(tuple(np.round(s, 9)) in cell8 for s in sub)
    gp = G.shortest_g(a, 64, False)
    n2 = (gp.astype(np.int64) ** 2).sum(axis=1)
    assert not np.any(n2 == 0)
    counts = {k: int((n2 == k).sum()) for k in range(1, 7)}
    assert counts == {1: 6, 2: 12, 3: 8, 4: 6, 5: 24, 6: 8}
    assert [tuple(m) for m in gp[56:]] == [(-2, -1, -1), (-2, -1, 1), (-2, 1, -1), (-2, 1, 1),
                                          (-1, -2, -1), (-1, -2, 1), (-1, -1, -2), (-1, -1, 2)]
    assert np.all(np.diff(n2) >= 0)                       # ranked by |G|^2

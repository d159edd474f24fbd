"""The batched uneven workload's generator (48 seeded cubic cells): its draws stay in the
stated ranges, the FFT box is the smallest 2-3-5 size holding the potential's band without
aliasing, and the cell has the Si density of the 8-atom cell."""
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

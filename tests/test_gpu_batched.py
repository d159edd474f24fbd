"""Batched solves of systems of uneven sizes (the batched workload's instances: cubic cells of
2, 4 and 5 atoms, 251 / 751 / 1237 plane waves, 15^3 / 24^3 / 27^3 boxes, 184 / 183 / 16
frequencies) in one packed persistent launch, through the C ABI: the same solutions as the
one-system solves, the FP64 criteria on every pair, and dense-LU spot checks of each instance
against the oracle.  Also the autotuner's probe over CTA sizes."""
import numpy as np
import pytest

import instances as I
import oracle as O

pytestmark = pytest.mark.gpu

SEEDS = (27, 23, 34)


@pytest.fixture(scope="module")
def sgw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    import paper_1812_03717_gb300 as P
    from paper_1812_03717_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    return P


@pytest.fixture(scope="module")
def jobs(sgw):
    import torch
    out = []
    for seed in SEEDS:
        inst = I.config4(seed)
        kp = inst.kpoints[0]
        s = sgw.System.from_instance(inst, kp.kq_frac)
        sk = sgw.System.from_instance(inst, kp.k_frac)
        s.set_occupied(kp.psi_kq, kp.eps_kq)
        rhs = s.make_rhs(sk, torch.from_numpy(kp.psi_k).cuda(), inst.gp_miller)
        out.append({"inst": inst, "sys": s, "rhs": rhs, "e_ref": inst.e_ref(0), "omega": inst.omega})
    return out


def _relerr(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


def test_uneven_instances_are_uneven(jobs):
    sizes = [j["sys"].n_pw for j in jobs]
    assert sizes == [251, 751, 1237]
    assert len({j["inst"].fft_dims for j in jobs}) == 3


@pytest.mark.parametrize("precision", ["df32", "fp64"])
def test_batched_equals_single_and_lu(sgw, jobs, precision):
    import torch
    items = [{"sys": j["sys"], "rhs": j["rhs"], "e_ref": j["e_ref"], "omega": j["omega"]} for j in jobs]
    outs, reps, ok = sgw.solve_batched(items, jobs[0]["inst"].eta, tol=1e-10, precision=precision)
    torch.cuda.synchronize()
    assert ok, [np.unique(r["status"], return_counts=True) for r in reps]
    for j, d, rep in zip(jobs, outs, reps):
        assert rep["rel_res"].max() <= 1e-10 and rep["cert"].max() <= 1e-8
        single, srep, sok = j["sys"].solve_shifted(j["rhs"], j["e_ref"], j["omega"], j["inst"].eta, tol=1e-10,
                                                   precision=precision)
        assert sok
        d = d.cpu().numpy()
        assert _relerr(d, single.cpu().numpy()).max() < 1e-9
        # the packed launch runs the same per-right-hand-side algorithm: same Krylov steps
        assert np.array_equal(rep["matvecs"].max(axis=1), srep["matvecs"].max(axis=1))
        inst = j["inst"]
        kp = inst.kpoints[0]
        h, _, _ = O.dense_h_inst(inst, kp.kq_frac)
        rref = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, inst.gp_miller)
        rows = np.array([0, len(rref) // 2, len(rref) - 1])
        js = np.array([0, len(inst.omega) // 2, len(inst.omega) - 1])
        ref = O.solve_shifted(h, kp.psi_kq, rref[rows], j["e_ref"][rows], inst.omega[js], inst.eta)
        assert _relerr(d[rows][:, js], ref).max() < 1e-8
    # one packed launch served all three systems (cluster size 1 for each)
    assert sum(int(r["launches"][0]) for r in reps) <= 3 * 4 + 1


def test_autotune_picks_a_timed_shape(sgw, jobs, tmp_path, monkeypatch):
    from paper_1812_03717_gb300 import autotune as T
    monkeypatch.setenv("SGW_TUNE_CACHE", str(tmp_path / "tune.json"))
    j = jobs[2]
    inst = j["inst"]
    choice = T.tune(j["sys"], j["rhs"], j["e_ref"], j["omega"], inst.eta, inst.fft_dims, inst.n_occ,
                    len(inst.kb_atom), precision="df32", probe_steps=20)
    assert choice["threads"] in (256, 384, 512) and choice["csize"] == 1
    assert len(choice["timed"]) == 3 and all(t["ms_per_step"] > 0 for t in choice["timed"])
    again = T.tune(j["sys"], j["rhs"], j["e_ref"], j["omega"], inst.eta, inst.fft_dims, inst.n_occ,
                   len(inst.kb_atom), precision="df32")
    assert again["threads"] == choice["threads"]   # from the cache

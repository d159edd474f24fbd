"""Host logic of the launch-shape autotuner, on the CPU: a stand-in system returns synthetic
probe timings, and the tuner must keep the shape with the least time per Lanczos step, leave
the system on it, cache the choice per bucket and serve the cache without probing again."""
import numpy as np
import pytest

from paper_1812_03717_gb300 import autotune as T


class FakeSystem:
    """The calls the tuner makes, with a synthetic cost per (CTA size, cluster size)."""

    def __init__(self, auto, cost, bad_csizes=()):
        self.n_pw = 1000
        self.auto = auto
        self.forced = 0
        self.cost = cost            # (threads, csize) -> ms of one Lanczos step of an owner
        self.bad = set(bad_csizes)  # cluster sizes the box cannot be split into
        self.probes = []

    def split(self):
        c = self.forced or self.auto
        return c, c

    def set_split(self, c):
        if c in self.bad:
            raise RuntimeError("SGW_EUNSUPPORTED: the box does not split over that many CTAs")
        self.forced = c
        return self.split()

    def lanczos_owners(self, nomega, precision, threads):
        return 4

    def solve_shifted(self, rhs, e_ref, omega, eta, tol, precision, threads, max_matvec, max_refine, cert_tol):
        c = self.split()[0]
        self.probes.append((threads, c))
        n = rhs.shape[0]
        # the n owners step concurrently: the launch takes (time of an owner's step) x steps
        rep = {"matvecs": np.full((n, len(omega)), max_matvec, dtype=np.int32),
               "kernel_ms": np.array([self.cost[(threads, c)] * max_matvec])}
        return None, rep, True


def _args(n=8):
    import torch
    rhs = torch.zeros((n, 1000), dtype=torch.complex128)
    return rhs, np.zeros(n), np.linspace(0.0, 1.0, 16), 0.0037


def test_one_cta_box_picks_fastest_threads_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("SGW_TUNE_CACHE", str(tmp_path / "tune.json"))
    cost = {(256, 1): 3.0, (384, 1): 2.0, (512, 1): 2.5}
    s = FakeSystem(1, cost)
    rhs, e, om, eta = _args()
    choice = T.tune(s, rhs, e, om, eta, (36, 36, 36), 16, 8, precision="df32", probe_steps=40)
    assert (choice["threads"], choice["csize"]) == (384, 1)
    assert choice["ms_per_step"] == pytest.approx(2.0 / 4)      # per owner-step, 4 owners in flight
    assert sorted(s.probes) == [(256, 1), (384, 1), (512, 1)]    # one CTA: no cluster sizes probed
    # the cache serves the same bucket without probing
    s2 = FakeSystem(1, {})
    again = T.tune(s2, rhs, e, om, eta, (36, 36, 36), 16, 8, precision="df32", probe_steps=40)
    assert (again["threads"], again["csize"]) == (384, 1) and not s2.probes
    # another bucket (more shifts) is probed afresh
    s3 = FakeSystem(1, cost)
    T.tune(s3, rhs, e, np.linspace(0.0, 1.0, 32), eta, (36, 36, 36), 16, 8, precision="df32", probe_steps=40)
    assert s3.probes


def test_cluster_box_probes_larger_splits_and_keeps_the_best(tmp_path, monkeypatch):
    monkeypatch.setenv("SGW_TUNE_CACHE", str(tmp_path / "tune.json"))
    cost = {(nt, c): 1.0 + 0.1 * abs(c - 10) + (0.5 if nt == 256 else 0.0) for nt in (256, 384, 512)
            for c in (9, 10, 12)}
    s = FakeSystem(9, cost, bad_csizes=(12,))
    rhs, e, om, eta = _args()
    choice = T.tune(s, rhs, e, om, eta, (72, 72, 72), 128, 64, precision="df32", probe_steps=40)
    assert choice["csize"] == 10 and choice["threads"] in (384, 512)
    assert s.split()[0] == 10                                   # the system is left on the choice
    assert {c for _, c in s.probes} == {9, 10}                  # 12 cannot be split: skipped


def test_no_probe_succeeds_returns_automatic_shape(tmp_path, monkeypatch):
    monkeypatch.setenv("SGW_TUNE_CACHE", str(tmp_path / "tune.json"))
    s = FakeSystem(1, {})                                       # every probe raises (KeyError)
    rhs, e, om, eta = _args()
    choice = T.tune(s, rhs, e, om, eta, (16, 16, 16), 4, 2, precision="fp64", probe_steps=10)
    assert choice == {"threads": 0, "csize": 1, "ms_per_step": None, "timed": []}
    assert not (tmp_path / "tune.json").exists()

"""Host logic of the learned preconditioner's training driver, on the CPU: the target of each
training pair is the Jacobi floor that solved it in the fewest H applications (0, the plain
scaling, when plain was fastest), a floor whose solve did not converge never wins, and the
statistics count every pair once."""
import numpy as np

from paper_1812_03717_gb300 import learned_precond as L


class FakeSystem:
    """solve_pershift returns fixed H-application counts per preconditioner (and floor);
    training_rows records the floors it is given."""

    def __init__(self, plain, jacobi, failed=()):
        self.plain = np.asarray(plain)
        self.jacobi = {d: np.asarray(v) for d, v in jacobi.items()}
        self.failed = set(failed)          # (floor, pair) whose solve misses the tolerance
        self.rows_delta = None

    def solve_pershift(self, rp, e, om, eta, tol, precond, delta=None, mlp=None):
        if precond == "plain":
            mv = self.plain.copy()
            st = np.zeros(len(mv), dtype=np.int32)
        else:
            mv = self.jacobi[delta].copy()
            st = np.array([1 if (delta, i) in self.failed else 0 for i in range(len(mv))], dtype=np.int32)
        return None, {"matvecs": mv, "status": st}, bool(np.all(st == 0))

    def training_rows(self, rp, e, om, eta, delta):
        self.rows_delta = np.asarray(delta, dtype=float)
        return "feats", "targets"


def test_fastest_floor_defines_the_target():
    deltas = (0.03, 0.1, 0.3, 1.0)
    plain = [100, 50, 80, 60]
    jacobi = {0.03: [90, 70, 85, 65], 0.1: [120, 40, 75, 61], 0.3: [95, 80, 30, 62], 1.0: [99, 90, 90, 63]}
    s = FakeSystem(plain, jacobi, failed={(0.3, 2)})   # the fastest floor of pair 2 did not converge
    stats = L.new_stats(deltas)
    f, t = L.pairs_rows(s, np.zeros((4, 3)), np.zeros(4), np.zeros(4), 0.01, deltas=deltas, stats=stats)
    assert (f, t) == ("feats", "targets")
    # pair 0: 0.03 (90 < 100); pair 1: 0.1 (40); pair 2: 0.3 failed -> 0.1 (75 < 80); pair 3: plain (60)
    np.testing.assert_array_equal(s.rows_delta, [0.03, 0.1, 0.1, 0.0])
    assert stats["pairs"] == 4
    assert stats["plain_mv"] == sum(plain)
    assert stats["best_mv"] == 90 + 40 + 75 + 60
    assert stats["wins"] == [1, 1, 2, 0, 0]              # plain, 0.03, 0.1, 0.3, 1.0


def test_untrained_network_is_the_plain_scaling():
    """The packed parameters end with the output layer (64 weights and a bias), all zero:
    f = 0 everywhere, so the learned diagonal M exp(f) starts as the plain scaling M."""
    p = L.init_params(0)
    assert p.size == 4 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4545
    assert not np.any(p[-65:])
    assert np.all(np.abs(p[:256]) <= np.sqrt(6 / 4)) and np.any(p[:256])

"""What the trained network gains over the plain kinetic preconditioner.

Training pairs come from per-shift solves the library runs on seeded disordered fcc systems
(the fastest of the plain scaling and Jacobi floors defines the targets); the network is
trained on the GPU; held-out systems are then solved per shift with the plain and with the
learned preconditioner.  The residual decides convergence, so the solutions agree and only
the H-application counts may differ: the learned preconditioner must need fewer."""
import json

import pytest

pytestmark = pytest.mark.gpu


def test_learned_preconditioner_gain():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    import paper_1812_03717_gb300 as P
    from paper_1812_03717_gb300 import build as B
    from paper_1812_03717_gb300 import learned_precond as L
    if not os.path.exists(B.LIB):
        B.build()
    feats, targets, stats = L.training_set(P, range(12), pairs_per_seed=24)
    mlp, losses = L.train(P, feats, targets, steps=300, lr=3e-3)
    ev = L.evaluate(P, mlp, range(2000, 2003), pairs_per_seed=24)
    print(json.dumps({"train_pairs": stats["pairs"], "loss": [losses[0], losses[-1]],
                      "plain_mean": ev["plain_mean"], "learned_mean": ev["learned_mean"], "gain": ev["gain"]}))
    assert losses[-1] < 0.5 * losses[0]
    assert ev["max_rel_res"] <= 1e-10
    assert ev["max_diff"] < 1e-7           # same answers
    assert ev["gain"] > 1.1                # fewer H applications with the learned scaling

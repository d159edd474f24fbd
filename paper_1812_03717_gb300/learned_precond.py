"""Training and evaluation driver of the learned diagonal preconditioner.

Training data come from solves the library itself runs: each training pair (a right-hand
side of a seeded disordered fcc system at one frequency) is solved per shift with the plain
kinetic scaling and with the Jacobi scaling at several floors; the fastest floor defines the
per-plane-wave targets (sgw_training_rows).  The perceptron is trained on the GPU with the
library's forward/backward/Adam kernels (sgw_mlp_train_step).  Evaluation compares
H-application counts of per-shift solves on held-out systems with the plain and the learned
preconditioner (the residual decides convergence, so only counts may change).

    python -m paper_1812_03717_gb300.learned_precond --train-seeds 24 --eval-seeds 4 --out weights.npy
    python -m paper_1812_03717_gb300.learned_precond --config2-pairs 64 --eval-seeds 0 --supercell-pairs 15
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DELTAS = (0.03, 0.1, 0.3, 1.0)     # Jacobi floors (Ha) tried on every training pair
N_HIDDEN, N_IN = 64, 4


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform hidden layers, zero output layer: the untrained network reproduces the
    plain scaling exactly.  Packed w1[64][4], b1, w2[64][64], b2, w3[64], b3."""
    rng = np.random.default_rng(seed)
    w1 = rng.uniform(-math.sqrt(6 / N_IN), math.sqrt(6 / N_IN), (N_HIDDEN, N_IN))
    w2 = rng.uniform(-math.sqrt(6 / N_HIDDEN), math.sqrt(6 / N_HIDDEN), (N_HIDDEN, N_HIDDEN))
    parts = [w1, np.zeros(N_HIDDEN), w2, np.zeros(N_HIDDEN), np.zeros(N_HIDDEN), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def _pairs(inst, ik, n_pairs, seed):
    rng = np.random.default_rng(10_000 + seed)
    nr = inst.n_occ * inst.n_pert
    r = rng.integers(0, nr, n_pairs)
    j = rng.integers(0, len(inst.omega), n_pairs)
    return r, j


def _system(P, inst, ik=0):
    import torch
    kp = inst.kpoints[ik]
    skq = P.System.from_instance(inst, kp.kq_frac)
    sk = P.System.from_instance(inst, kp.k_frac)
    skq.set_occupied(kp.psi_kq, kp.eps_kq)
    rhs = skq.make_rhs(sk, torch.from_numpy(kp.psi_k).cuda(), inst.gp_miller)
    sk.close()
    return skq, rhs


def pairs_rows(s, rp, e, om, eta, tol=1e-8, deltas=DELTAS, stats=None):
    """Training rows of the pairs (rp[i], e[i] + om[i] + i eta) of system s: each pair is
    solved per shift with the plain scaling and with the Jacobi scaling at every floor; the
    fastest defines its targets."""
    _, rep, _ = s.solve_pershift(rp, e, om, eta, tol=tol, precond="plain")
    counts = [rep["matvecs"].astype(np.int64)]
    for dl in deltas:
        _, rep, _ = s.solve_pershift(rp, e, om, eta, tol=tol, precond="jacobi", delta=dl)
        mv = rep["matvecs"].astype(np.int64)
        mv[rep["status"] != 0] = 1 << 30
        counts.append(mv)
    counts = np.stack(counts)                         # [1 + n_delta][pairs]
    best = counts.argmin(axis=0)
    best_delta = np.where(best == 0, 0.0, np.asarray((0.0,) + tuple(deltas))[best])
    f, t = s.training_rows(rp, e, om, eta, best_delta)
    if stats is not None:
        stats["pairs"] += len(e)
        stats["plain_mv"] += int(counts[0].sum())
        stats["best_mv"] += int(counts.min(axis=0).sum())
        for b in best:
            stats["wins"][int(b)] += 1
    return f, t


def new_stats(deltas=DELTAS):
    return {"pairs": 0, "plain_mv": 0, "best_mv": 0, "wins": [0] * (len(deltas) + 1)}


def training_set(P, seeds, pairs_per_seed=32, tol=1e-8, deltas=DELTAS, make=None):
    """Rows (feats, targets) on the GPU from per-shift solves on the given seeds."""
    import torch
    import instances as I
    make = make or I.fcc_perturbed
    feats, targets, stats = [], [], new_stats(deltas)
    for seed in seeds:
        inst = make(seed)
        s, rhs = _system(P, inst)
        r, j = _pairs(inst, 0, pairs_per_seed, seed)
        rp = rhs[torch.as_tensor(r, device=rhs.device)].contiguous()
        e = inst.e_ref(0)[r]
        om = inst.omega[j]
        f, t = pairs_rows(s, rp, e, om, inst.eta, tol, deltas, stats)
        feats.append(f)
        targets.append(t)
        s.close()
    return torch.cat(feats), torch.cat(targets), stats


def config2_rows(P, seed=0, pairs_per_k=64, tol=1e-8, deltas=DELTAS, stats=None):
    """Training rows from the k-points of the 8-atom cubic cell (the config-2 generator):
    pairs_per_k seeded (right-hand side, frequency) pairs per k-point, as in training_set."""
    import torch
    import instances as I
    inst = I.config2(seed)
    feats, targets = [], []
    for ik in range(len(inst.kpoints)):
        s, rhs = _system(P, inst, ik)
        rng = np.random.default_rng(20_000 + 10 * seed + ik)
        r = rng.integers(0, rhs.shape[0], pairs_per_k)
        j = rng.integers(0, len(inst.omega), pairs_per_k)
        rp = rhs[torch.as_tensor(r, device=rhs.device)].contiguous()
        f, t = pairs_rows(s, rp, inst.e_ref(ik)[r], inst.omega[j], inst.eta, tol, deltas, stats)
        feats.append(f)
        targets.append(t)
        s.close()
    return torch.cat(feats), torch.cat(targets)


def evaluate_supercell(P, mlp, n_pairs=15, max_matvec=6000, tol=1e-10, seed=0):
    """Per-shift solves of n_pairs seeded (band, G_p, omega) pairs of the 64-atom supercell
    (18 277 plane waves, the 72^3 box split over a thread-block cluster), with the plain and
    with the learned diagonal, each capped at max_matvec H applications per pair.  A pair counts
    as solved when rel_res <= tol and its certificate <= 1e-8; the H-application gain is taken
    over the pairs both preconditioners solve, and their solutions are compared."""
    import torch
    import instances as I
    inst = I.config3()
    kp = inst.kpoints[0]
    rng = np.random.default_rng(30_000 + seed)
    v = rng.integers(0, inst.n_occ, n_pairs)
    p = rng.integers(0, inst.n_pert, n_pairs)
    j = rng.integers(0, len(inst.omega), n_pairs)
    dev = torch.device("cuda", torch.cuda.current_device())
    s = P.System.from_instance(inst, kp.kq_frac)
    sk = P.System.from_instance(inst, kp.k_frac)
    s.set_occupied(torch.from_numpy(kp.psi_kq).to(dev), kp.eps_kq)
    bands = np.unique(v)
    rhs_b = s.make_rhs(sk, torch.from_numpy(kp.psi_k[bands]).to(dev), inst.gp_miller)
    sk.close()
    rows = np.searchsorted(bands, v) * inst.n_pert + p
    rp = rhs_b[torch.as_tensor(rows, device=dev)].contiguous()
    del rhs_b
    e = kp.eps_k[v]
    om = inst.omega[j]
    out = {"pairs": n_pairs, "n_pw": s.n_pw, "cluster_ctas": s.split()[0], "max_matvec": max_matvec,
           "omega_ev": (om * 27.211386245988).round(2).tolist()}
    sol = {}
    for mode in ("plain", "learned"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, rep, _ = s.solve_pershift(rp, e, om, inst.eta, tol=tol, precond=mode,
                                     mlp=mlp if mode == "learned" else None, max_matvec=max_matvec)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = (rep["status"] == 0) & (rep["rel_res"] <= tol) & (rep["cert"] <= 1e-8)
        sol[mode] = (x, ok, rep["matvecs"].astype(np.int64))
        out[mode] = {"seconds": dt, "solved": int(ok.sum()), "solves_per_s": float(ok.sum()) / dt,
                     "matvecs": rep["matvecs"].tolist(),
                     "max_rel_res_solved": float(rep["rel_res"][ok].max()) if ok.any() else None}
    both = sol["plain"][1] & sol["learned"][1]
    out["solved_by_both"] = int(both.sum())
    if both.any():
        out["matvec_gain"] = float(sol["plain"][2][both].mean() / sol["learned"][2][both].mean())
        b = torch.as_tensor(np.flatnonzero(both), device=dev)
        x0, x1 = sol["plain"][0][b], sol["learned"][0][b]
        out["max_diff_solved"] = float((torch.linalg.norm(x1 - x0, dim=1) / torch.linalg.norm(x0, dim=1)).max())
    s.close()
    return out


def train(P, feats, targets, steps=400, lr=3e-3, batch=8192, seed=0, params=None):
    import torch
    mlp = P.MLP(init_params(seed) if params is None else params)
    n = feats.shape[0]
    g = torch.Generator(device=feats.device)
    g.manual_seed(seed)
    losses = []
    for it in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device=feats.device, generator=g)
        losses.append(mlp.train_step(feats[idx].contiguous(), targets[idx].contiguous(), lr=lr))
    return mlp, losses


def evaluate(P, mlp, seeds, pairs_per_seed=32, tol=1e-10, make=None):
    """H applications per pair with the plain and the learned preconditioner on held-out seeds."""
    import torch
    import instances as I
    make = make or I.fcc_perturbed
    out = {"plain": [], "learned": [], "max_rel_res": 0.0, "max_diff": 0.0}
    for seed in seeds:
        inst = make(seed)
        s, rhs = _system(P, inst)
        r, j = _pairs(inst, 0, pairs_per_seed, seed)
        rp = rhs[torch.as_tensor(r, device=rhs.device)].contiguous()
        e = inst.e_ref(0)[r]
        om = inst.omega[j]
        x0, rp0, ok0 = s.solve_pershift(rp, e, om, inst.eta, tol=tol, precond="plain")
        x1, rp1, ok1 = s.solve_pershift(rp, e, om, inst.eta, tol=tol, precond="learned", mlp=mlp)
        out["plain"] += rp0["matvecs"].tolist()
        out["learned"] += rp1["matvecs"].tolist()
        out["max_rel_res"] = max(out["max_rel_res"], float(rp0["rel_res"].max()), float(rp1["rel_res"].max()))
        d = torch.linalg.norm(x1 - x0, dim=1) / torch.linalg.norm(x0, dim=1)
        out["max_diff"] = max(out["max_diff"], float(d.max()))
        s.close()
    out["plain_mean"] = float(np.mean(out["plain"]))
    out["learned_mean"] = float(np.mean(out["learned"]))
    out["gain"] = out["plain_mean"] / out["learned_mean"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-seeds", type=int, default=24)
    ap.add_argument("--eval-seeds", type=int, default=4)
    ap.add_argument("--pairs", type=int, default=32)
    ap.add_argument("--config2-pairs", type=int, default=0,
                    help="also train on this many pairs per k-point of the 8-atom cubic cell")
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--supercell-pairs", type=int, default=0,
                    help="evaluate on this many seeded pairs of the 64-atom supercell")
    ap.add_argument("--supercell-cap", type=int, default=6000, help="H applications per supercell pair")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    import paper_1812_03717_gb300 as P
    t0 = time.time()
    feats, targets, stats = training_set(P, range(args.train_seeds), args.pairs)
    if args.config2_pairs > 0:
        f2, t2_ = config2_rows(P, 0, args.config2_pairs, stats=stats)
        feats, targets = torch.cat([feats, f2]), torch.cat([targets, t2_])
    t1 = time.time()
    mlp, losses = train(P, feats, targets, steps=args.steps, lr=args.lr)
    t2 = time.time()
    line = {"rows": int(feats.shape[0]), "data": stats, "loss_first": losses[0], "loss_last": losses[-1]}
    if args.eval_seeds > 0:
        ev = evaluate(P, mlp, range(1000, 1000 + args.eval_seeds), args.pairs)
        line["eval"] = {k: v for k, v in ev.items() if k not in ("plain", "learned")}
    t3 = time.time()
    print(json.dumps(line), flush=True)
    if args.supercell_pairs > 0:
        line["supercell"] = evaluate_supercell(P, mlp, args.supercell_pairs, args.supercell_cap)
    t4 = time.time()
    if args.out:
        np.save(args.out, mlp.params)
    line["seconds"] = {"data": t1 - t0, "train": t2 - t1, "eval": t3 - t2, "supercell": t4 - t3}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

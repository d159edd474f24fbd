"""Benchmark of the shifted Sternheimer hot path on GB300.

Workload (one step = one k-point of the 8-atom cubic cell): 16 occupied bands x 32
perturbations exp(i(q+G_p).r) = 512 right-hand sides, each solved at 64 frequencies in
[0, 60] eV with eta = 0.1 eV in the ~1640 plane-wave basis (ecut 20 Ry, 36^3 FFT box):
Eq. 8 right-hand sides already resident, multishift Lanczos (FOM) to a residual of 1e-10,
then the FP64 true residual and error certificate of every (rhs, omega) pair (and per-shift
correction solves for any pair above 1e-10).
The four seeded k-points are cycled through the steps.

--impl reference times the FP64 CPU oracle (dense LU per shift) on a bounded sample of the
same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Sternheimer (RHS×ω) solves/s at 1e-8 rel. err, mixed+learned vs plain FP64"
WORKLOAD = ("8-atom cubic Si-like cell a=10.26 bohr, ecut 20 Ry (N_pw~1640), 36^3 FFT, per k-point "
            "16 bands x 32 G_p = 512 rhs x 64 omega in [0,60] eV, eta 0.1 eV, residual 1e-10 (FP64 check); "
            "a step solves all 4 seeded k-points concurrently (2048 rhs x 64 omega)")
HBM_FALLBACK_GBS = 6800.0
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070     # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (1.26 TFLOP/s)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --------------------------------------------------------------------------- workload

def make_workload(seed=0, k_subset=None):
    import instances as I
    return I.config2(seed=seed, k_subset=k_subset)


def apply_flops(plan):
    """Algorithmic FP64 flops of one H application y = (P_c H - z) x (5 n log2 n per FFT line)."""
    n1, n2, n3 = plan["dims"]
    f = 0.0
    f += 2 * plan["nstick"] * 5 * n3 * math.log2(n3)
    f += n3 * 2 * plan["nxcol"] * 5 * n2 * math.log2(n2)
    f += n3 * 2 * n2 * 5 * n1 * math.log2(n1)
    f += 2 * n1 * n2 * n3
    npw = plan["npw"]
    f += 4 * npw + 16 * npw * (plan["nproj"] + plan["nocc"]) + 8 * npw
    return f


FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070   # 80.5 TFLOP/s
# DRAM bytes (read + write) per 512-right-hand-side launch of the multishift kernel, from the
# ncu captures in profiles/ (16 right-hand sides, scaled by right-hand sides); None once the
# kernel has changed since the capture.
TRAFFIC_PER_LAUNCH = {"df32": 22.5e9, "fp64": 33.2e9}


def radix_plan(n):
    out, m = [], n
    for r in (4, 2, 3, 5):
        while m % r == 0:
            out.append(r)
            m //= r
    return out


def pfa_parts(n):
    """Coprime prime-power parts of n when each has a register DFT (the library then runs the
    prime-factor algorithm on that axis), else None."""
    parts, m = [], n
    for p in (2, 3, 5):
        q = 1
        while m % p == 0:
            m //= p
            q *= p
        if q > 1:
            parts.append(q)
    return parts if m == 1 and all(q in (2, 3, 4, 5, 8, 9) for q in parts) else None


_DFT_BASE = {4: (8, 0, 0), 2: (2, 0, 0), 3: (6, 0, 2), 5: (16, 0, 8)}   # (complex adds, multiplies, real scalings)


def dft_cost(p):
    if p in _DFT_BASE:
        return _DFT_BASE[p]
    q, r = {8: (4, 2), 9: (3, 3)}[p]
    a1, m1, s1 = dft_cost(q)
    a2, m2, s2 = dft_cost(r)
    return r * a1 + q * a2, r * m1 + q * m2 + (r - 1) * (q - 1), r * s1 + q * s2


def fft_line_ops(n):
    """(complex adds, complex multiplies, real scalings) of one in-place line transform of
    length n as the library runs it: the prime-factor stages when the axis has them, else the
    radix stages (twiddles only on butterflies with j mod m != 0)."""
    parts = pfa_parts(n)
    ca = cm = cs = 0
    if parts:
        for p in parts:
            a, m, c = dft_cost(p)
            ca += (n // p) * a
            cm += (n // p) * m
            cs += (n // p) * c
        return ca, cm, cs
    span = n
    for r in radix_plan(n):
        span //= r
        nb = n // r
        a, _, c = _DFT_BASE[r]
        ca += nb * a
        cs += nb * c
        cm += (nb - nb // span) * (r - 1)
    return ca, cm, cs


def apply_line_counts(plan):
    n1, n2, n3 = plan["dims"]
    return [(n3, 2 * plan["nstick"]), (n2, 2 * n3 * plan["nxcol"]), (n1, 2 * n3 * n2)]


def solver_fp64_flops(plan, matvecs):
    k_rhs = matvecs.max(axis=1).astype(np.float64)
    fa = apply_flops(plan) + 30.0 * plan["npw"]
    return float(k_rhs.sum()) * fa + float(matvecs.astype(np.float64).sum()) * 8.0 * plan["npw"]


def solver_df32_ops(plan, matvecs):
    """FP32 operations of the float-float FFT part: 22 per complex add (two TwoSum-based
    float-float adds), 38 per complex multiply (two fused error-free dot products), 14 per
    real scaling (two float-float products), over the line transforms the library runs."""
    ops = 0.0
    for n, lines in apply_line_counts(plan):
        ca, cm, cs = fft_line_ops(n)
        ops += lines * (22 * ca + 38 * cm + 14 * cs)
    n1, n2, n3 = plan["dims"]
    ops += 14 * n1 * n2 * n3
    return float(matvecs.max(axis=1).astype(np.float64).sum()) * ops


def plan_info(inst, kp):
    n1, n2, n3 = inst.fft_dims
    mil = kp.miller_kq
    xy = set(((int(m[0]) % n1), (int(m[1]) % n2)) for m in mil)
    xs = set(x for x, _ in xy)
    return {"dims": (n1, n2, n3), "nstick": len(xy), "nxcol": len(xs), "npw": len(mil),
            "nproj": len(inst.kb_atom), "nocc": inst.n_occ}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        # the raw samples go to $SGW_CLOCKS_DIR (default: the temporary directory)
        d = os.environ.get("SGW_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"sgw_clocks_rank{index}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- oracle

def oracle_sample(inst, ik, seconds, max_pairs=None):
    """Times the oracle's dense LU solves on (band, omega) pairs of k-point ik (all perturbations
    per pair) until `seconds` have elapsed; returns (solves, elapsed, pairs)."""
    import oracle as O
    kp = inst.kpoints[ik]
    t0 = time.perf_counter()
    h, _, _ = O.dense_h_inst(inst, kp.kq_frac)
    rhs = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k, inst.gp_miller)
    e_ref = inst.e_ref(ik)
    npert = inst.n_pert
    done = 0
    pairs = 0
    order = [(v, j) for j in range(len(inst.omega)) for v in range(inst.n_occ)]
    rng = np.random.default_rng(1)
    rng.shuffle(order)
    for v, j in order:
        rows = slice(v * npert, (v + 1) * npert)
        O.solve_shifted(h, kp.psi_kq, rhs[rows], e_ref[rows], inst.omega[j:j + 1], inst.eta)
        done += npert
        pairs += 1
        if time.perf_counter() - t0 >= seconds or (max_pairs and pairs >= max_pairs):
            break
    return done, time.perf_counter() - t0, pairs


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    inst = make_workload(k_subset=[0])
    for _ in range(args.warmup):
        oracle_sample(inst, 0, 0.0, max_pairs=1)
    t_total, n_total = 0.0, 0
    for _ in range(args.steps):
        n, t, _ = oracle_sample(inst, 0, args.ref_seconds)
        t_total += t
        n_total += n
    v = n_total / t_total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"dense LU (scipy) per (band, omega) for all 32 G_p of k-point 0, "
                                       f"{args.ref_seconds:.0f} s per step, incl. building H"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1812_03717_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    import paper_1812_03717_gb300 as P

    t_gen = time.perf_counter()
    inst = make_workload()
    t_gen = time.perf_counter() - t_gen
    nk = len(inst.kpoints)
    dev = torch.device("cuda", local)
    jobs = []
    for ik, kp in enumerate(inst.kpoints):
        skq = P.System.from_instance(inst, kp.kq_frac)
        sk = P.System.from_instance(inst, kp.k_frac)
        skq.set_occupied(torch.from_numpy(kp.psi_kq).to(dev), kp.eps_kq)
        rhs = skq.make_rhs(sk, torch.from_numpy(kp.psi_k).to(dev), inst.gp_miller)
        sk.close()
        dpsi = torch.empty((rhs.shape[0], len(inst.omega), skq.n_pw), dtype=torch.complex128, device=dev)
        jobs.append({"sys": skq, "rhs": rhs, "dpsi": dpsi, "e_ref": inst.e_ref(ik), "plan": plan_info(inst, kp)})
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    tol = 1e-10

    from paper_1812_03717_gb300.partition import units_for_step

    from paper_1812_03717_gb300.batch import solve_concurrent
    per_step = args.kpoints_per_step

    def step(i, precision, record=None):
        """One step: per_step k-points solved concurrently (one stream each)."""
        ks = [units_for_step(i * per_step + u, ws, rank, nk) for u in range(per_step)]
        sel = [jobs[k] for k in ks]
        t0 = time.perf_counter()
        res = solve_concurrent([{"sys": j["sys"], "rhs": j["rhs"], "e_ref": j["e_ref"], "out": j["dpsi"]} for j in sel],
                               inst.omega, inst.eta, tol=tol, precision=precision)
        if record is not None:
            torch.cuda.synchronize()
            for k, j, (rep, ok) in zip(ks, sel, res):
                record.append({"k": k, "rep": rep, "rel": rep["rel_res"], "cert": rep["cert"], "plan": j["plan"],
                               "wall_s": time.perf_counter() - t0})

    def timed(precision):
        for i in range(args.warmup):
            step(i, precision)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        clk = ClockSampler(local)
        clk.start()
        recs = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i, precision, recs)
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        clocks = clk.stop()
        t_ms = e0.elapsed_time(e1)
        t_max = t_ms
        if ws > 1:
            tt = torch.tensor([t_ms], device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            t_max = float(tt.item())
        npairs = sum(r["rep"]["status"].size for r in recs)
        conv = sum(int(((r["rep"]["status"] == 0) & (r["rel"] <= tol)).sum()) for r in recs)
        cert_ok = sum(int((r["cert"] <= 1e-8).sum()) for r in recs)
        value = npairs * ws / (t_max / 1e3)
        # the multishift kernels of a step run concurrently: their algorithmic work over the
        # step's time (which also holds the FP64 residual check) is a lower bound on their rate
        kms = t_ms
        if precision == "fp64":
            work = sum(solver_fp64_flops(r["plan"], r["rep"]["matvecs"]) for r in recs)
            peak = FP64_PEAK_GFLOPS / 1e3
            roof = {"bound": "alu", "achieved": work / (kms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "kernel": "lanczos_solve_kernel<ArF64>",
                    "peak_source": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (unit count)",
                    "work": "algorithmic FP64 flops: FFT 5 n log2 n per line + V, T, KB, P_c, Lanczos passes, x = V y",
                    "time": "whole timed steps (multishift kernels + FP64 residual check)"}
        else:
            work = sum(solver_df32_ops(r["plan"], r["rep"]["matvecs"]) for r in recs)
            peak = FP32_PEAK_GFLOPS / 1e3
            roof = {"bound": "alu", "achieved": work / (kms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "kernel": "lanczos_solve_kernel<ArDF>",
                    "peak_source": "FP32 pipe: 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz (unit count)",
                    "work": "FP32 operations of the float-float FFT (22 per complex add, 38 per complex multiply, "
                            "14 per real scaling; the prime-factor or radix line transforms the library runs) "
                            "per H application x applications",
                    "time": "whole timed steps (multishift kernels + FP64 residual check)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        tr = TRAFFIC_PER_LAUNCH.get(precision)
        roof["traffic"] = tr
        if tr is not None:
            roof["traffic_unit"] = "bytes per 512-rhs launch (ncu capture of 16 rhs, scaled)"
        mv_all = np.concatenate([r["rep"]["matvecs"].max(axis=1) for r in recs])
        quality = {"pairs": npairs, "converged_true_res_le_tol": conv, "cert_le_1e-8": cert_ok,
                   "max_true_rel_res": float(max(r["rel"].max() for r in recs)),
                   "max_cert": float(max(r["cert"].max() for r in recs)),
                   "lanczos_steps_median": float(np.median(mv_all)), "lanczos_steps_max": int(mv_all.max())}
        return {"value": value, "ms_per_step": t_max / args.steps,
                "kernel_ms_per_launch": float(np.mean([float(r["rep"]["kernel_ms"][0]) for r in recs])),
                "roofline": roof, "quality": quality, "clocks": clocks,
                "gpu_launches": int(sum(int(r["rep"]["launches"][0]) for r in recs))}

    variants = [v for v in args.variants.split(",") if v]
    res = {v: timed(v) for v in variants}
    head = res[variants[0]]

    # Green's-function columns (Eq. 2-3) on one k-point's basis: every plane-wave column at 64
    # time-ordered shifts around the chemical potential, one launch per run
    green = None
    if not args.no_green:
        kg = units_for_step(0, ws, rank, nk)
        green = measure_green(P, inst, kg, jobs[kg], variants[0], stream)

    # density response of Eq. 5 for one k-point: its 512 right-hand sides at +-omega (128
    # shifts per Krylov space) and the reduction to dn[G][G'][omega]
    density = None
    if not args.no_density:
        kd = units_for_step(0, ws, rank, nk)
        density = measure_density(P, inst, kd, jobs[kd], variants[0], stream, nk)

    # the imaginary-axis route of Sec. 2.7 for the same k-point: response at 16 imaginary
    # frequencies, screening there, AAA continuation of every eps^-1 element to the real axis
    continuation = None
    if not args.no_density:
        kd = units_for_step(0, ws, rank, nk)
        continuation = measure_continuation(P, inst, kd, jobs[kd], variants[0], stream, nk)

    # per-shift solves of sampled pairs of this workload: plain vs learned diagonal preconditioner
    learned = None
    if not args.no_learned:
        from paper_1812_03717_gb300 import learned_precond as LP
        # training pairs: small disordered fcc systems and the workload's k-points other than the
        # evaluated one (held out); evaluation: sampled pairs of the held-out k-point
        feats, targets, lstats = LP.training_set(P, range(24), pairs_per_seed=32)
        fl, tl = [feats], [targets]
        ev_k = units_for_step(0, ws, rank, nk)
        for k in range(nk):
            if k == ev_k:
                continue
            rng_k = np.random.default_rng(100 + k)
            r_k = rng_k.integers(0, jobs[k]["rhs"].shape[0], 64)
            j_k = rng_k.integers(0, len(inst.omega), 64)
            f, t = LP.pairs_rows(jobs[k]["sys"], jobs[k]["rhs"][torch.as_tensor(r_k, device=dev)].contiguous(),
                                 jobs[k]["e_ref"][r_k], inst.omega[j_k], inst.eta, stats=lstats)
            fl.append(f)
            tl.append(t)
        mlp, losses = LP.train(P, torch.cat(fl), torch.cat(tl), steps=600, lr=3e-3)
        job = jobs[ev_k]
        rng = np.random.default_rng(7)
        npr = 152
        r_idx = rng.integers(0, job["rhs"].shape[0], npr)
        j_idx = rng.integers(0, len(inst.omega), npr)
        rp = job["rhs"][torch.as_tensor(r_idx, device=dev)].contiguous()
        e_p = job["e_ref"][r_idx]
        om_p = inst.omega[j_idx]
        out = {}
        for mode in ("plain", "learned"):
            for _ in range(2):   # warm-up
                job["sys"].solve_pershift(rp, e_p, om_p, inst.eta, tol=tol, precond=mode,
                                          mlp=mlp if mode == "learned" else None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep, ok = job["sys"].solve_pershift(rp, e_p, om_p, inst.eta, tol=tol, precond=mode,
                                                   mlp=mlp if mode == "learned" else None)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[mode] = {"solves_per_s": npr / dt, "matvecs_mean": float(rep["matvecs"].mean()),
                         "converged": int((rep["status"] == 0).sum()), "max_rel_res": float(rep["rel_res"].max())}
        learned = {"pairs": npr, "eval_kpoint": int(ev_k), "train_pairs": lstats["pairs"],
                   "train_loss": [losses[0], losses[-1]],
                   "plain": out["plain"], "learned": out["learned"],
                   "matvec_gain": out["plain"]["matvecs_mean"] / out["learned"]["matvecs_mean"],
                   "throughput_gain": out["learned"]["solves_per_s"] / out["plain"]["solves_per_s"]}

    # e2e through host buffers (pinned): a step's right-hand sides go in and its solutions come
    # out through the library's host staging, k-points concurrent as in the timed steps
    e2e = None
    if not args.no_e2e:
        ks = [units_for_step(u, ws, rank, nk) for u in range(per_step)]
        host = []
        for k in ks:
            rh = torch.empty(jobs[k]["rhs"].shape, dtype=torch.complex128, pin_memory=True)
            rh.copy_(jobs[k]["rhs"].cpu())
            dh = torch.empty(jobs[k]["dpsi"].shape, dtype=torch.complex128, pin_memory=True)
            host.append({"sys": jobs[k]["sys"], "rhs": rh, "e_ref": jobs[k]["e_ref"], "out": dh})
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            res_e2e = solve_concurrent(host, inst.omega, inst.eta, tol=tol, precision=variants[0])
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        pairs = sum(h["rhs"].shape[0] for h in host) * len(inst.omega)
        e2e = {"value": pairs * args.e2e_steps * ws / t_e2e, "unit": "solves/s",
               "h2d_bytes_per_step": int(sum(h["rhs"].numel() * 16 for h in host)),
               "d2h_bytes_per_step": int(sum(h["out"].numel() * 16 for h in host) + pairs * 32),
               "steps": args.e2e_steps}
        del host

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        n, t, pairs = oracle_sample(inst, 0, args.ref_seconds)
        cpu = {"value": n / t, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{pairs} (band, omega) dense LU solves x 32 G_p of k-point 0 in {t:.1f} s (scipy, FP64), "
                         f"incl. building H"}
    dtype = {"fp64": "f64", "df32": "f64 (FFT in float-float on FP32 pipes)"}[variants[0]]
    line = {
        "metric": METRIC, "value": head["value"], "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "rhs_per_step": int(sum(jobs[units_for_step(u, ws, rank, nk)]["rhs"].shape[0]
                                                                  for u in range(per_step))),
                   "omega": len(inst.omega),
                   "solver": "multishift Lanczos (FOM) on P_c H P_c, FP64 true-residual check + per-shift corrections",
                   "precision": variants[0], "tol": tol,
                   "l2": "inputs larger than L2 (dpsi 0.86 GB + Lanczos basis per step)",
                   "parallelism": f"replicas x{ws} (k-points sharded)", "generate_s": round(t_gen, 1)},
        "quality": head["quality"], "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e,
        "clocks": head["clocks"], "gpu_launches": head["gpu_launches"], "learned_preconditioner": learned,
        "green_function": green, "density_response": density, "imaginary_axis": continuation,
        "variants": {v: {k: res[v][k] for k in ("value", "ms_per_step", "kernel_ms_per_launch", "roofline", "quality")}
                     for v in variants},
    }
    if "fp64" in res and variants[0] != "fp64":
        line["speedup_vs_plain_fp64"] = head["value"] / res["fp64"]["value"]
    print(json.dumps(line), flush=True)


GREEN_SPAN_EV = 30.0
HA_EV = 27.211386245988        # eV per Hartree (CODATA 2018)


def green_shifts(inst, kp, nz=64, span_ev=GREEN_SPAN_EV):
    """z_j = omega_j + i eta sgn(omega_j - mu), omega_j = mu + linspace(-span, span, nz) eV, mu in
    the gap above the occupied states of the basis."""
    mu = float(kp.eps_kq[-1]) + 0.5 * float(kp.gap_kq)
    om = mu + np.linspace(-span_ev, span_ev, nz) / HA_EV
    return om + 1j * inst.eta * np.sign(om - mu), mu


def measure_green(P, inst, ik, job, precision, stream, runs=1):
    """All columns of G(z) for one k-point's basis at 64 time-ordered shifts: one untimed run,
    then `runs` runs timed with CUDA events; returns a dict for the JSON line."""
    import torch
    s = job["sys"]
    z, mu = green_shifts(inst, inst.kpoints[ik])
    cols = np.arange(s.n_pw)
    out = torch.empty((len(cols), len(z), s.n_pw), dtype=torch.complex128, device="cuda")
    s.solve_green(cols, z, tol=1e-10, precision=precision, out=out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = []
    for _ in range(runs):
        _, rep, ok = s.solve_green(cols, z, tol=1e-10, precision=precision, out=out)
        reps.append(rep)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / runs
    rep = reps[-1]
    plan = job["plan"]
    steps = rep["matvecs"].max(axis=1)
    if precision == "fp64":
        work = solver_fp64_flops(plan, rep["matvecs"]) / 1e12
        roof = {"bound": "alu", "achieved": work / (ms / 1e3), "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "kernel": "lanczos_solve_kernel<ArF64>"}
    else:
        work = solver_df32_ops(plan, rep["matvecs"]) / 1e12
        roof = {"bound": "alu", "achieved": work / (ms / 1e3), "peak": FP32_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "kernel": "lanczos_solve_kernel<ArDF>"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["time"] = "whole call (multishift kernel + FP64 residual check)"
    roof["traffic"] = None
    npairs = rep["status"].size
    del out
    return {"metric": "Green's-function (column x z) solves/s at 1e-10 residual", "value": npairs / (ms / 1e3),
            "unit": "solves/s", "ms_per_run": ms, "runs": runs, "precision": precision,
            "workload": f"all {len(cols)} plane-wave columns G' of G(z) = (z - H)^-1 on the k+q basis of k-point {ik}, "
                        f"{len(z)} shifts omega = mu + linspace(-{GREEN_SPAN_EV:g}, {GREEN_SPAN_EV:g}) eV, "
                        f"Im z = eta sgn(omega - mu), eta 0.1 eV",
            "quality": {"pairs": int(npairs), "converged": int((rep["status"] == 0).sum()),
                        "max_true_rel_res": float(rep["rel_res"].max()), "max_cert": float(rep["cert"].max()),
                        "lanczos_steps_median": float(np.median(steps)), "lanczos_steps_max": int(steps.max())},
            "roofline": roof, "gpu_launches": int(rep["launches"][0])}


def measure_density(P, inst, ik, job, precision, stream, nk, runs=1):
    """One k-point's contribution to Eq. 5 (all bands x all G' x 64 omega, both signs): one
    untimed call, then `runs` calls timed with CUDA events; returns a dict for the JSON line."""
    import torch
    s = job["sys"]
    kp = inst.kpoints[ik]
    n_p = len(inst.gp_miller)
    out = torch.zeros((n_p, n_p, len(inst.omega)), dtype=torch.complex128, device="cuda")
    s.density_response(job["rhs"], kp.eps_k, inst.omega, inst.eta, weight=2.0 / nk, tol=1e-10,
                       precision=precision, out=out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(runs):
        _, rep, ok = s.density_response(job["rhs"], kp.eps_k, inst.omega, inst.eta, weight=2.0 / nk, tol=1e-10,
                                        precision=precision, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / runs
    # screening step (Eq. 4, 9): epsilon^-1 and W-bar for every frequency from this response,
    # Coulomb potential cut off at the radius of the sphere holding N_k cells
    from instances.generate import recip
    qg = ((np.asarray(kp.kq_frac) - np.asarray(kp.k_frac))[None, :] + inst.gp_miller) @ recip(inst.a)
    r_cut = (3.0 * inst.volume * nk / (4.0 * math.pi)) ** (1.0 / 3.0)
    P.screened_coulomb(out, qg, inst.volume, r_cut)
    torch.cuda.synchronize()
    e0.record(stream)
    _, wbar = P.screened_coulomb(out, qg, inst.volume, r_cut)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_screen = e0.elapsed_time(e1)
    npairs = rep["status"].size
    steps = rep["matvecs"].max(axis=1)
    plan = job["plan"]
    work = (solver_fp64_flops(plan, rep["matvecs"]) if precision == "fp64" else solver_df32_ops(plan, rep["matvecs"]))
    peak = (FP64_PEAK_GFLOPS if precision == "fp64" else FP32_PEAK_GFLOPS) / 1e3
    roof = {"bound": "alu", "achieved": work / 1e12 / (ms / 1e3), "peak": peak, "unit": "TFLOP/s",
            "kernel": "lanczos_solve_kernel<%s>" % ("ArF64" if precision == "fp64" else "ArDF"),
            "time": "whole call (multishift kernel, FP64 residual check, density reduction)", "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    return {"metric": "density-response Sternheimer solves/s (rhs x +-omega) incl. the Eq. 5 reduction",
            "value": npairs / (ms / 1e3), "unit": "solves/s", "ms_per_run": ms, "runs": runs,
            "dn_columns_per_s": n_p * len(inst.omega) / (ms / 1e3), "precision": precision,
            "workload": f"k-point {ik}: {kp.psi_k.shape[0]} bands x {n_p} G' right-hand sides, {len(inst.omega)} "
                        f"omega in [0, 60] eV at + and - (omega + i eta), dn[G][G'][omega] for the {n_p} G",
            "quality": {"pairs": int(npairs), "converged": int((rep["status"] == 0).sum()),
                        "max_true_rel_res": float(rep["rel_res"].max()),
                        "lanczos_steps_median": float(np.median(steps)), "lanczos_steps_max": int(steps.max())},
            "roofline": roof, "gpu_launches": int(rep["launches"][0]),
            "screening": {"ms": ms_screen, "frequencies": len(inst.omega), "n_g": n_p, "r_cut_bohr": r_cut,
                          "what": "epsilon^-1 and W-bar per frequency (Eq. 4, 9), FP64 Gauss-Jordan in shared "
                                  "memory, one CTA per frequency",
                          "finite": bool(torch.isfinite(wbar.real).all().item())}}


def measure_continuation(P, inst, ik, job, precision, stream, nk, n_imag=16):
    """Imaginary-axis density response (n_imag frequencies i omega, omega in [0.02, 4] Ha on a
    quadratic grid), its screening, and the AAA continuation of all eps^-1 elements to the
    bench's real frequencies + i eta; CUDA-event times of each part after one untimed pass."""
    import torch
    from instances.generate import recip
    s = job["sys"]
    kp = inst.kpoints[ik]
    n_p = len(inst.gp_miller)
    w = 1j * (0.02 + 3.98 * np.linspace(0.0, 1.0, n_imag) ** 2)
    qg = ((np.asarray(kp.kq_frac) - np.asarray(kp.k_frac))[None, :] + inst.gp_miller) @ recip(inst.a)
    r_cut = (3.0 * inst.volume * nk / (4.0 * math.pi)) ** (1.0 / 3.0)
    x = inst.omega + 1j * inst.eta
    times = {}

    def once(record):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        dn = torch.zeros((n_p, n_p, n_imag), dtype=torch.complex128, device="cuda")
        _, rep, ok = s.density_response_w(job["rhs"], kp.eps_k, w, weight=2.0 / nk, tol=1e-10, precision=precision,
                                          out=dn)
        ev[1].record(stream)
        einv, _ = P.screened_coulomb(dn, qg, inst.volume, r_cut)
        ev[2].record(stream)
        r, deg = P.aaa(w, einv.reshape(n_p * n_p, n_imag), x, tol=1e-10, mmax=16)
        ev[3].record(stream)
        torch.cuda.synchronize()
        if record:
            times["response_ms"] = ev[0].elapsed_time(ev[1])
            times["screening_ms"] = ev[1].elapsed_time(ev[2])
            times["aaa_ms"] = ev[2].elapsed_time(ev[3])
        return rep, deg
    once(False)
    rep, deg = once(True)
    npairs = rep["status"].size
    return {"metric": "imaginary-axis density-response Sternheimer solves/s (rhs x +-i omega)",
            "value": npairs / (times["response_ms"] / 1e3), "unit": "solves/s", "precision": precision,
            "workload": f"k-point {ik}: 512 rhs x {n_imag} imaginary frequencies (both signs), eps^-1 at "
                        f"{n_imag} i omega, AAA continuation of {n_p * n_p} elements to {len(x)} real omega + i eta",
            "ms": {k: round(v, 3) for k, v in times.items()},
            "quality": {"pairs": int(npairs), "converged": int((rep["status"] == 0).sum()),
                        "max_true_rel_res": float(rep["rel_res"].max()),
                        "lanczos_steps_median": float(np.median(rep["matvecs"].max(axis=1))),
                        "aaa_support_points_max": int(deg.max())}}


def run_profile_case(args):
    """One solve of the first --profile-case right-hand sides of k-point 0 (no timing contract):
    the small case that ncu captures of the multishift kernel run."""
    import torch
    import paper_1812_03717_gb300 as P
    from paper_1812_03717_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    inst = make_workload(k_subset=[0])
    kp = inst.kpoints[0]
    skq = P.System.from_instance(inst, kp.kq_frac)
    sk = P.System.from_instance(inst, kp.k_frac)
    skq.set_occupied(kp.psi_kq, kp.eps_kq)
    rhs = skq.make_rhs(sk, torch.from_numpy(kp.psi_k).cuda(), inst.gp_miller)[:args.profile_case].contiguous()
    _, rep, ok = skq.solve_shifted(rhs, inst.e_ref(0)[:args.profile_case], inst.omega, inst.eta, tol=1e-10,
                                   precision=args.variants.split(",")[0])
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "precision": args.variants.split(",")[0], "ok": ok,
                      "kernel_ms": float(rep["kernel_ms"][0]), "lanczos_steps_max": int(rep["matvecs"].max())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kpoints-per-step", type=int, default=4,
                    help="k-points solved concurrently (one CUDA stream each) per step")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--variants", default="df32,fp64",
                    help="comma list of FFT precisions to time; the first is the headline")
    ap.add_argument("--no-green", action="store_true", help="skip the Green's-function measurement")
    ap.add_argument("--no-density", action="store_true", help="skip the density-response measurement")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="solve this many right-hand sides of k-point 0 once and exit (for ncu captures)")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark of the shifted Sternheimer hot path on GB300.

Headline workload (the largest single-GPU configuration): the 64-atom 2x2x2 supercell of the
cubic Si-like cell (a = 20.52 bohr, atoms displaced by N(0, 0.05 bohr), seed 0), ecut 25 Ry
(18 277 plane waves), 72^3 FFT box, k = Gamma, q = 0, 128 occupied bands x the 64 shortest
non-zero G = 8192 right-hand sides, each solved at 128 frequencies in [0, 60] eV with
eta = 0.1 eV.  One step = one batch of right-hand sides (by default one per vector owner the
GPU holds at once: one per thread-block cluster) x all 128 frequencies: Eq. 8 right-hand sides
already resident, the multishift Lanczos (FOM) pass, the FP64 true residual and certificate
of every pair, per-shift corrections of near-converged pairs.  A pair counts only when its
relative residual is <= 1e-10 and its certificate |r| / (eta |x|) <= 1e-8.  Steps walk
through the 8192 right-hand sides batch by batch.

Variants: float-float (the headline, "mixed": FP32 pipes, FP64 scalars and residual) and
plain FP64 (the baseline the headline is compared with).  Secondary measurements on the
8-atom cubic cell (ecut 20 Ry, 36^3 box, 4 k-points): the same multishift solve, the
Green's-function columns, the density response, the imaginary-axis route with AAA and the
learned preconditioner.

--impl reference times the FP64 CPU oracle (dense LU per (band, frequency) with all 64
perturbations) on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Sternheimer (RHS×ω) solves/s at 1e-8 rel. err, mixed+learned vs plain FP64"
WORKLOAD = ("64-atom 2x2x2 Si-like supercell a=20.52 bohr (N(0,0.05) displacements, seed 0), ecut 25 Ry "
            "(N_pw 18277), 72^3 FFT, k=Gamma, q=0, 128 bands x 64 G_p = 8192 rhs x 128 omega in [0,60] eV, "
            "eta 0.1 eV; a pair counts when rel. residual <= 1e-10 and certificate <= 1e-8")
WORKLOAD2 = ("8-atom cubic Si-like cell a=10.26 bohr, ecut 20 Ry (N_pw~1640), 36^3 FFT, 4 seeded k-points x "
             "16 bands x 32 G_p = 2048 rhs x 64 omega in [0,60] eV, eta 0.1 eV")
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070     # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (1.26 TFLOP/s)
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070   # 80.5 TFLOP/s
# DRAM bytes (read + write) per right-hand side and Lanczos step of the dominant kernel, from
# the ncu capture in profiles/ (16 right-hand sides x 100 steps of the supercell); a launch's
# traffic is this times its steps.  None: not captured since the kernel last changed.
TRAFFIC_PER_RHS_STEP = {"df32": (19.133e9 + 1.363e9) / 1600}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


# ------------------------------------------------------------------ work per H application

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


def plan_info(inst, miller):
    n1, n2, n3 = inst.fft_dims
    xy = set(((int(m[0]) % n1), (int(m[1]) % n2)) for m in miller)
    xs = set(x for x, _ in xy)
    return {"dims": (n1, n2, n3), "nstick": len(xy), "nxcol": len(xs), "npw": len(miller),
            "nproj": len(inst.kb_atom), "nocc": inst.n_occ}


def apply_line_counts(plan):
    n1, n2, n3 = plan["dims"]
    return [(n3, 2 * plan["nstick"]), (n2, 2 * n3 * plan["nxcol"]), (n1, 2 * n3 * n2)]


def step_fp64_flops(plan):
    """Algorithmic FP64 flops of one Lanczos step: H application (5 n log2 n per FFT line, V,
    T, KB and P_c dots and updates, 8 flops per complex multiply-add) and the three vector
    passes."""
    f = 0.0
    for n, lines in apply_line_counts(plan):
        f += lines * 5 * n * math.log2(n)
    n1, n2, n3 = plan["dims"]
    f += 2 * n1 * n2 * n3
    npw = plan["npw"]
    f += npw * (16 * (plan["nocc"] + plan["nproj"]) + 4 + 30)
    return f


def step_df32_ops(plan):
    """FP32 operations of one float-float Lanczos step: 22 per complex add, 38 per complex
    multiply, 14 per real scaling over the line transforms the library runs; 14 per potential
    sample; 60 per complex multiply-add of the KB and P_c dots and updates; 300 per plane wave
    for T, the gather scaling and the three vector passes."""
    ops = 0.0
    for n, lines in apply_line_counts(plan):
        ca, cm, cs = fft_line_ops(n)
        ops += lines * (22 * ca + 38 * cm + 14 * cs)
    n1, n2, n3 = plan["dims"]
    ops += 14 * n1 * n2 * n3
    ops += plan["npw"] * (120 * (plan["nocc"] + plan["nproj"]) + 300)
    return ops


def solve_work(plan, matvecs, precision):
    """Work of a multishift launch: steps (the longest shift of each right-hand side) x work
    per step, plus x_j = V y_j (one complex multiply-add per plane wave, step and shift)."""
    steps = float(matvecs.max(axis=1).astype(np.float64).sum())
    xvy = float(matvecs.astype(np.float64).sum()) * plan["npw"]
    if precision == "fp64":
        return steps * step_fp64_flops(plan) + 8.0 * xvy
    return steps * step_df32_ops(plan) + 60.0 * xvy


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
        with open(self.path) as f:
            return parse_clocks(f)


def parse_clocks(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in nvidia-smi samples
    (csv, noheader, nounits: index, clocks.sm, clocks.max.sm, power.draw, reasons.active,
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap); lines that do not
    parse are skipped."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
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

class OracleSampler:
    """The FP64 oracle on the headline workload: dense H of the supercell in the oracle's own
    route (box DFT of the sampled potential, KB projectors), P_c H P_c, then per sample one
    dense LU of P_c H P_c - z for one (band, frequency) pair, solved for all 64 perturbations.
    The dense H and its projection (5.3 GB each, built once; their time is reported apart) are
    shared by every (band, frequency) pair of the workload, so a sample times the per-pair
    part: the factorisation and the solves."""

    def __init__(self, inst):
        import oracle as O
        self.O = O
        self.inst = inst
        kp = inst.kpoints[0]
        t0 = time.perf_counter()
        h, _, _ = O.dense_h_inst(inst, kp.kq_frac)
        self.pcp = O.projected_h(h, kp.psi_kq)
        del h
        self.setup_s = time.perf_counter() - t0
        self.rng = np.random.default_rng(1)

    def sample(self):
        """One (band, frequency) pair with all perturbations; returns (solves, seconds)."""
        import scipy.linalg
        O, inst = self.O, self.inst
        kp = inst.kpoints[0]
        v = int(self.rng.integers(0, inst.n_occ))
        j = int(self.rng.integers(0, len(inst.omega)))
        t0 = time.perf_counter()
        rhs = O.make_rhs(kp.miller_kq, kp.miller_k, kp.psi_k[v:v + 1], inst.gp_miller)
        b = -O.project_c(kp.psi_kq, rhs)
        z = kp.eps_k[v] + inst.omega[j] + 1j * inst.eta
        a = self.pcp - z * np.eye(self.pcp.shape[0])
        lu = scipy.linalg.lu_factor(a, overwrite_a=True, check_finite=False)
        scipy.linalg.lu_solve(lu, b.T, check_finite=False)
        return inst.n_pert, time.perf_counter() - t0


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import instances as I
    inst = I.config3()
    S = OracleSampler(inst)          # warm-up: the dense H and its projection
    for _ in range(max(0, args.warmup - 1)):
        pass                         # further warm-up steps would only repeat a factorisation
    t_total, n_total = 0.0, 0
    for _ in range(args.steps):
        n, t = S.sample()
        t_total += t
        n_total += n
    v = n_total / t_total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"per step one dense LU (scipy, FP64, N=18277) of P_c H P_c - z for a seeded "
                                       f"(band, omega) pair, solved for all 64 G_p; dense H and P_c H P_c built once "
                                       f"before the steps in {S.setup_s:.0f} s"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- ours

def headline_job(P, dev, stream_of):
    """The supercell system on the GPU with all 8192 right-hand sides resident."""
    import torch
    import instances as I
    inst = I.config3()
    kp = inst.kpoints[0]
    s = P.System.from_instance(inst, kp.kq_frac)
    sk = P.System.from_instance(inst, kp.k_frac)
    s.set_occupied(torch.from_numpy(kp.psi_kq).to(dev), kp.eps_kq)
    rhs = s.make_rhs(sk, torch.from_numpy(kp.psi_k).to(dev), inst.gp_miller)
    sk.close()
    return {"inst": inst, "sys": s, "rhs": rhs, "e_ref": inst.e_ref(0), "plan": plan_info(inst, kp.miller_kq)}


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
    from paper_1812_03717_gb300.partition import units_for_step

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    job = headline_job(P, dev, None)
    t_gen = time.perf_counter() - t_gen
    inst = job["inst"]
    nw = len(inst.omega)
    nrhs_all = job["rhs"].shape[0]
    csize, csize8 = job["sys"].split()
    owners = args.rhs_per_step or job["sys"].lanczos_owners(nw, "df32")
    B_step = max(1, owners)
    n_batches = nrhs_all // B_step
    tol = 1e-10
    out = torch.empty((B_step, nw, job["sys"].n_pw), dtype=torch.complex128, device=dev)

    def batch(i):
        u = units_for_step(i, ws, rank, n_batches)
        return slice(u * B_step, (u + 1) * B_step)

    def step(i, precision, recs=None):
        sl = batch(i)
        _, rep, ok = job["sys"].solve_shifted(job["rhs"][sl], job["e_ref"][sl], inst.omega, inst.eta, tol=tol,
                                              precision=precision, out=out)
        if recs is not None:
            recs.append(rep)

    def timed(precision, warmup, steps):
        for i in range(warmup):
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
        for i in range(steps):
            step(warmup + i, precision, recs)
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
        npairs = sum(r["status"].size for r in recs)
        certified = sum(int(((r["status"] == 0) & (r["rel_res"] <= tol) & (r["cert"] <= 1e-8)).sum()) for r in recs)
        value = certified * ws / (t_max / 1e3)
        kms = float(sum(float(r["kernel_ms"][0]) for r in recs))
        work = sum(solve_work(job["plan"], r["matvecs"], precision) for r in recs)
        if precision == "fp64":
            roof = {"bound": "alu", "achieved": work / (kms / 1e3) / 1e12, "peak": FP64_PEAK_GFLOPS / 1e3,
                    "unit": "TFLOP/s", "kernel": "lanczos_solve_kernel<ArF64,384>",
                    "peak_source": "FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (unit count)",
                    "work": "algorithmic FP64 flops per Lanczos step (FFT 5 n log2 n per line, V, T, KB and P_c "
                            "dots and updates, vector passes) x steps + x = V y"}
        else:
            roof = {"bound": "alu", "achieved": work / (kms / 1e3) / 1e12, "peak": FP32_PEAK_GFLOPS / 1e3,
                    "unit": "TFLOP/s", "kernel": "lanczos_solve_kernel<ArDF,512>",
                    "peak_source": "FP32 pipe: 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz (unit count)",
                    "work": "FP32 operations of the float-float step (22 per complex add, 38 per complex multiply, "
                            "14 per real scaling in the line transforms; 60 per complex multiply-add of the "
                            "projector dots and updates) x steps + x = V y"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["time"] = "CUDA events around the multishift kernel launch on the solve's stream"
        tps = TRAFFIC_PER_RHS_STEP.get(precision)
        steps_launch = float(np.mean([r["matvecs"].max(axis=1).sum() for r in recs]))
        roof["traffic"] = tps * steps_launch if tps else None
        if tps:
            roof["traffic_unit"] = ("DRAM bytes per launch: %.1f MB per right-hand side and step (ncu, 16 rhs x 100 "
                                    "steps) x the launch's %d steps" % (tps / 1e6, steps_launch))
        mv_all = np.concatenate([r["matvecs"].max(axis=1) for r in recs])
        quality = {"pairs": npairs, "certified": certified,
                   "max_true_rel_res": float(max(r["rel_res"].max() for r in recs)),
                   "max_cert": float(max(r["cert"].max() for r in recs)),
                   "lanczos_steps_median": float(np.median(mv_all)), "lanczos_steps_max": int(mv_all.max())}
        return {"value": value, "ms_per_step": t_max / steps, "steps": steps, "warmup": warmup,
                "kernel_ms_per_step": kms / steps, "roofline": roof, "quality": quality, "clocks": clocks,
                "gpu_launches": int(sum(int(r["launches"][0]) for r in recs))}

    variants = [v for v in args.variants.split(",") if v]
    res = {variants[0]: timed(variants[0], args.warmup, args.steps)}
    for v in variants[1:]:
        res[v] = timed(v, args.variant_warmup, args.variant_steps)
    head = res[variants[0]]

    # e2e through host buffers (pinned): the step's right-hand sides go in and its solutions come
    # out through the library's host staging
    e2e = None
    if not args.no_e2e:
        rh = torch.empty((B_step, job["sys"].n_pw), dtype=torch.complex128, pin_memory=True)
        dh = torch.empty((B_step, nw, job["sys"].n_pw), dtype=torch.complex128, pin_memory=True)
        tot_pairs, tot_s = 0, 0.0
        for i in range(args.e2e_steps):
            sl = batch(args.warmup + args.steps + i)
            rh.copy_(job["rhs"][sl].cpu())
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep, _ = job["sys"].solve_shifted(rh, job["e_ref"][sl], inst.omega, inst.eta, tol=tol,
                                                 precision=variants[0], out=dh)
            tot_s += time.perf_counter() - t0
            tot_pairs += int(((rep["status"] == 0) & (rep["cert"] <= 1e-8)).sum())
        e2e = {"value": tot_pairs * ws / tot_s, "unit": "solves/s", "h2d_bytes_per_step": int(rh.numel() * 16),
               "d2h_bytes_per_step": int(dh.numel() * 16 + rh.shape[0] * nw * (8 * 3 + 4 * 2)),
               "steps": args.e2e_steps,
               "what": "sgw_solve_shifted on pinned host buffers: rhs host->device, solve, dpsi and the per-pair "
                       "report device->host, all inside the timed region"}
        del rh, dh

    # the supercell's Krylov workspace (tens of GB) is released before the other workloads
    job["sys"].close()
    del job["rhs"], out
    torch.cuda.empty_cache()

    # secondary measurements on the 8-atom cubic cell
    secondary = None
    if not args.no_secondary:
        try:
            secondary = run_secondary(args, P, dev, stream, ws, rank)
        except Exception as e:   # the headline is measured already: report the failure beside it
            secondary = {"error": f"{type(e).__name__}: {e}"}

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        try:
            S = OracleSampler(inst)
            n, t = S.sample()
            cpu = {"value": n / t, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                   "sample": f"one dense LU (scipy, FP64, N=18277) of P_c H P_c - z for one seeded (band, omega) "
                             f"pair, solved for all 64 G_p in {t:.1f} s; dense H and P_c H P_c (shared by all "
                             f"pairs) built beforehand in {S.setup_s:.0f} s"}
            del S
        except Exception as e:
            cpu = {"kind": "oracle", "error": f"{type(e).__name__}: {e}"}
    dtype = {"fp64": "f64", "df32": "f64 (float-float on the FP32 pipes; FP64 scalars and residual)",
             "fp32": "f32 inner / f64 refinement"}[variants[0]]
    line = {
        "metric": METRIC, "value": head["value"], "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "rhs_per_step": B_step, "omega": nw, "pairs_per_step": B_step * nw,
                   "cluster_ctas_per_vector": csize, "solver": "multishift Lanczos (FOM) on P_c H P_c in a "
                   "persistent cluster kernel with a work queue; FP64 true residual + certificate of every pair",
                   "precision": variants[0], "tol": tol, "cert_tol": 1e-8,
                   "l2": "inputs larger than L2 (dpsi %.2f GB per step + a Lanczos basis of ~4 GB per right-hand side)"
                         % (B_step * nw * job["sys"].n_pw * 16 / 1e9),
                   "parallelism": f"replicas x{ws} (right-hand-side batches sharded)", "generate_s": round(t_gen, 1)},
        "quality": head["quality"], "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e,
        "clocks": head["clocks"], "gpu_launches": head["gpu_launches"],
        "variants": {v: {k: res[v][k] for k in ("value", "ms_per_step", "steps", "warmup", "kernel_ms_per_step",
                                                "roofline", "quality", "clocks")} for v in variants},
        "secondary_cubic8": secondary,
    }
    if "fp64" in res and variants[0] != "fp64":
        line["speedup_vs_plain_fp64"] = head["value"] / res["fp64"]["value"]
    print(json.dumps(line), flush=True)


def run_secondary(args, P, dev, stream, ws, rank):
    """The 8-atom cubic cell: its four k-points solved concurrently (one stream each) in the
    headline's precision and in FP64, then the Green's-function, density-response,
    imaginary-axis and learned-preconditioner measurements on one k-point."""
    import torch
    import instances as I
    from paper_1812_03717_gb300.batch import solve_concurrent
    from paper_1812_03717_gb300.partition import units_for_step
    inst = I.config2()
    nk = len(inst.kpoints)
    jobs = []
    for ik, kp in enumerate(inst.kpoints):
        skq = P.System.from_instance(inst, kp.kq_frac)
        sk = P.System.from_instance(inst, kp.k_frac)
        skq.set_occupied(torch.from_numpy(kp.psi_kq).to(dev), kp.eps_kq)
        rhs = skq.make_rhs(sk, torch.from_numpy(kp.psi_k).to(dev), inst.gp_miller)
        sk.close()
        dpsi = torch.empty((rhs.shape[0], len(inst.omega), skq.n_pw), dtype=torch.complex128, device=dev)
        jobs.append({"sys": skq, "rhs": rhs, "dpsi": dpsi, "e_ref": inst.e_ref(ik), "plan": plan_info(inst, kp.miller_kq)})
    torch.cuda.synchronize()
    out = {"workload": WORKLOAD2}
    variants = [v for v in args.variants.split(",") if v]
    for precision in variants:
        def one(i):
            ks = [units_for_step(i * nk + u, ws, rank, nk) for u in range(nk)]
            return solve_concurrent([{"sys": jobs[k]["sys"], "rhs": jobs[k]["rhs"], "e_ref": jobs[k]["e_ref"],
                                      "out": jobs[k]["dpsi"]} for k in ks], inst.omega, inst.eta, tol=1e-10,
                                    precision=precision)
        for i in range(3):
            one(i)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = one(3)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        cert = sum(int(((rep["status"] == 0) & (rep["cert"] <= 1e-8)).sum()) for rep, _ in res)
        pairs = sum(rep["status"].size for rep, _ in res)
        out[precision] = {"value": cert / (ms / 1e3), "unit": "solves/s", "ms_per_step": ms, "pairs": pairs,
                          "certified": cert, "lanczos_steps_median": float(np.median(np.concatenate(
                              [rep["matvecs"].max(axis=1) for rep, _ in res])))}
    if "fp64" in out and variants[0] in out and variants[0] != "fp64":
        out["speedup_vs_plain_fp64"] = out[variants[0]]["value"] / out["fp64"]["value"]
    k0 = units_for_step(0, ws, rank, nk)
    if not args.no_extras:
        out["green_function"] = measure_green(P, inst, k0, jobs[k0], variants[0], stream)
        out["density_response"] = measure_density(P, inst, k0, jobs[k0], variants[0], stream, nk)
        out["imaginary_axis"] = measure_continuation(P, inst, k0, jobs[k0], variants[0], stream, nk)
        out["learned_preconditioner"] = measure_learned(P, inst, jobs, k0, dev)
    for j in jobs:
        j["sys"].close()
    jobs.clear()
    torch.cuda.empty_cache()
    if not args.no_extras:
        out["batched_uneven"] = measure_batched(P, dev, variants[0])
    for j in jobs:
        j["sys"].close()
    return out


BATCH_SEEDS = (27, 23, 42, 30, 34, 35, 14, 11, 47, 38, 25, 37, 43, 46, 31)


def measure_batched(P, dev, precision, rhs_cap=32):
    """The batched uneven workload's 15 instances with at most 3000 plane waves (2 to 36 atoms,
    boxes 15^3 to 36^3, 16 to 234 frequencies), up to `rhs_cap` right-hand sides each, solved
    (1) packed: sgw_solve_batched, one persistent launch for all (CTA size from the autotuner);
    (2) sequential: one sgw_solve_shifted per instance; (3) concurrent: one stream and host thread
    per instance.  Certified solves/s of each, after one untimed packed run."""
    import torch
    import instances as I
    from paper_1812_03717_gb300 import autotune as T
    from paper_1812_03717_gb300.batch import solve_concurrent
    t0 = time.perf_counter()
    jobs = []
    for seed in BATCH_SEEDS:
        inst = I.config4(seed)
        kp = inst.kpoints[0]
        s = P.System.from_instance(inst, kp.kq_frac)
        sk = P.System.from_instance(inst, kp.k_frac)
        s.set_occupied(torch.from_numpy(kp.psi_kq).to(dev), kp.eps_kq)
        rhs = s.make_rhs(sk, torch.from_numpy(kp.psi_k).to(dev), inst.gp_miller)[:rhs_cap].contiguous()
        sk.close()
        out = torch.empty((rhs.shape[0], len(inst.omega), s.n_pw), dtype=torch.complex128, device=dev)
        jobs.append({"inst": inst, "sys": s, "rhs": rhs, "e_ref": inst.e_ref(0)[:rhs.shape[0]], "omega": inst.omega,
                     "out": out})
    gen_s = time.perf_counter() - t0
    big = max(jobs, key=lambda j: j["sys"].n_pw)
    tune = T.tune(big["sys"], big["rhs"], big["e_ref"], big["omega"], big["inst"].eta, big["inst"].fft_dims,
                  big["inst"].n_occ, len(big["inst"].kb_atom), precision=precision, probe_steps=40)
    nt = tune["threads"] or 0
    eta = jobs[0]["inst"].eta
    items = [{"sys": j["sys"], "rhs": j["rhs"], "e_ref": j["e_ref"], "omega": j["omega"], "out": j["out"]} for j in jobs]
    pairs = sum(j["rhs"].shape[0] * len(j["omega"]) for j in jobs)

    def certified(reps):
        return sum(int(((r["status"] == 0) & (r["cert"] <= 1e-8)).sum()) for r in reps)

    P.solve_batched(items, eta, tol=1e-10, precision=precision, threads=nt)
    torch.cuda.synchronize()
    res = {}
    t = time.perf_counter()
    _, reps, _ = P.solve_batched(items, eta, tol=1e-10, precision=precision, threads=nt)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    res["packed"] = {"value": certified(reps) / dt, "s": dt, "launches": int(sum(int(r["launches"][0]) for r in reps)),
                     "kernel_ms": float(reps[0]["kernel_ms"][0])}
    t = time.perf_counter()
    reps = []
    for j in jobs:
        _, rep, _ = j["sys"].solve_shifted(j["rhs"], j["e_ref"], j["omega"], eta, tol=1e-10, precision=precision,
                                           out=j["out"])
        reps.append(rep)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    res["sequential"] = {"value": certified(reps) / dt, "s": dt}
    t = time.perf_counter()
    cres = solve_concurrent([{"sys": j["sys"], "rhs": j["rhs"], "e_ref": j["e_ref"], "out": j["out"]} for j in jobs],
                            None, eta, tol=1e-10, precision=precision, omegas=[j["omega"] for j in jobs])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    res["concurrent_streams"] = {"value": certified([r for r, _ in cres]) / dt, "s": dt}
    out = {"metric": "batched uneven Sternheimer (rhs x omega) solves/s at 1e-8, certified",
           "instances": [{"seed": j["inst"].seed, "n_pw": j["sys"].n_pw, "box": list(j["inst"].fft_dims),
                          "rhs": int(j["rhs"].shape[0]), "omega": len(j["omega"])} for j in jobs],
           "pairs": pairs, "precision": precision, "generate_s": round(gen_s, 1),
           "autotune": {"threads": tune["threads"], "csize": tune["csize"], "timed": tune.get("timed", [])},
           "packed": res["packed"], "sequential": res["sequential"], "concurrent_streams": res["concurrent_streams"],
           "packed_vs_sequential": res["packed"]["value"] / res["sequential"]["value"],
           "packed_vs_concurrent": res["packed"]["value"] / res["concurrent_streams"]["value"]}
    return out


def measure_learned(P, inst, jobs, ev_k, dev):
    """Per-shift solves of sampled pairs of the held-out k-point: plain vs learned diagonal
    preconditioner (trained on disordered fcc systems and the other k-points' pairs)."""
    import torch
    from paper_1812_03717_gb300 import learned_precond as LP
    nk = len(jobs)
    feats, targets, lstats = LP.training_set(P, range(24), pairs_per_seed=32)
    fl, tl = [feats], [targets]
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
    res = {}
    for mode in ("plain", "learned"):
        for _ in range(2):
            job["sys"].solve_pershift(rp, e_p, om_p, inst.eta, tol=1e-10, precond=mode,
                                      mlp=mlp if mode == "learned" else None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep, ok = job["sys"].solve_pershift(rp, e_p, om_p, inst.eta, tol=1e-10, precond=mode,
                                               mlp=mlp if mode == "learned" else None)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[mode] = {"solves_per_s": npr / dt, "matvecs_mean": float(rep["matvecs"].mean()),
                     "converged": int((rep["status"] == 0).sum()), "max_rel_res": float(rep["rel_res"].max())}
    return {"pairs": npr, "eval_kpoint": int(ev_k), "train_pairs": lstats["pairs"],
            "train_loss": [losses[0], losses[-1]], "plain": res["plain"], "learned": res["learned"],
            "matvec_gain": res["plain"]["matvecs_mean"] / res["learned"]["matvecs_mean"],
            "throughput_gain": res["learned"]["solves_per_s"] / res["plain"]["solves_per_s"]}


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
        work = solve_work(plan, rep["matvecs"], "fp64") / 1e12
        roof = {"bound": "alu", "achieved": work / (ms / 1e3), "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "kernel": "lanczos_solve_kernel<ArF64>"}
    else:
        work = solve_work(plan, rep["matvecs"], "df32") / 1e12
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
    work = solve_work(plan, rep["matvecs"], precision)
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
    """One solve of the first --profile-case right-hand sides of the supercell with a bounded
    Krylov budget (no timing contract): the small case that ncu captures of the multishift
    kernel run."""
    import torch
    import paper_1812_03717_gb300 as P
    from paper_1812_03717_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    job = headline_job(P, torch.device("cuda", 0), None)
    inst = job["inst"]
    n = args.profile_case
    prec = args.variants.split(",")[0]
    _, rep, ok = job["sys"].solve_shifted(job["rhs"][:n].contiguous(), job["e_ref"][:n], inst.omega, inst.eta,
                                          tol=1e-10, precision=prec, max_matvec=args.profile_matvec, max_refine=-1)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": n, "precision": prec, "max_matvec": args.profile_matvec,
                      "kernel_ms": float(rep["kernel_ms"][0]), "lanczos_steps_max": int(rep["matvecs"].max()),
                      "split": job["sys"].split()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variants", default="df32,fp64",
                    help="comma list of precisions to time; the first is the headline")
    ap.add_argument("--variant-steps", type=int, default=1, help="timed steps of the non-headline variants")
    ap.add_argument("--variant-warmup", type=int, default=1, help="warm-up steps of the non-headline variants")
    ap.add_argument("--rhs-per-step", type=int, default=0,
                    help="right-hand sides per step (0: one per vector owner resident on the GPU)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 8-atom cell measurements")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the Green's-function, density, imaginary-axis and learned measurements")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="solve this many right-hand sides of the supercell once and exit (for ncu captures)")
    ap.add_argument("--profile-matvec", type=int, default=200, help="Krylov budget of the profile case")
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

#!/usr/bin/env python
"""Benchmark of the augmented subspace iteration on one GB300.

Workload: 3D Laplace on the unit cube, trilinear Q1 elements on a uniform 128^3 mesh
(127^3 = 2,048,383 interior DOFs, 27 nonzeros per row), nested 16^3 coarse mesh
(3,375 DOFs), nev = 50 (block width 56), FP64 block multigrid (2 V-cycles of damped
Jacobi, 2+2 sweeps, Galerkin levels 128/64/32/16/8/4), seeded random start block.

A step is one augmented subspace iteration (residual, step (a) linear solve, step (b)
projection, step (c) augmented eigensolve, step (d) prolongation) on that workload.
value = DOF*nev per second (N_h * nev / step time), summed over ranks.

Extra keys: `converged` - DOF*nev/s to relative residual 1e-8 (whole solves, FP64 and the
mixed form, FP32 V-cycle inside FP64 refinement) with the speedup per converged eigenpair;
the roofline of the hot sparse kernel; per-kernel rooflines (`kernels`, with the measured
FP64 FMA rate); `cfg1_latency` (2D 128^2, nev 10: per-iteration latency and launches);
`variants` (step-(c) congruences PRECOND-A/-B/-B-A, Alg. 3's two-solve form, CG(40) and
MG-preconditioned CG step (a)); `tensor_operator` (the section-6.3 operator on the bench
mesh); `batch_scheme` (Alg. 7); the batch of 64 independent problems; the learned smoother;
the oracle timed on the host cores (cpu_baseline); an end-to-end number through the C ABI
with host buffers.

--impl reference times the FP64 CPU oracle (one oracle iteration per step) instead.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D, NFINE, NCOARSE, NEV, SEED = 3, 128, 16, 50, 0
WORKLOAD = "laplace3d_q1_128_coarse16_nev50"
METRIC = "DOF*nev/s per augmented-subspace iteration (3D Q1 128^3, nev 50, FP64)"
# DRAM bytes (read + write) of one fine-level FP64 Jacobi sweep at the 128^3 workload, from
# an ncu capture of the 64^3 case (profiles/k_csr_jacobi_laplace3d_64.md), scaled by rows
JACOBI_TRAFFIC_BYTES = 3.277e9  # 400.1 MB at 64^3 scaled by rows (2,048,383 / 250,047)
UNIT = "DOF*nev/s"


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi sampling during the timed region (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def build_workload(nfine=NFINE):
    import pase_inputs as pin
    pb = pin.build_problem(D, nfine, NCOARSE, mg_min=4)
    m = pin.guard_columns(NEV)
    return pb, m


def cpu_oracle_iteration_seconds(pb, m, steps=1, warmup=0):
    """The oracle as it stands: one augmented subspace iteration per step on the full
    workload (random start; the timed steps run the linear solve)."""
    import numpy as np
    import pase_inputs as pin
    from oracle import pase as opase
    S = opase.Solver(pb.A, pb.M, pb.chain, coarse_level=pb.coarse_level)
    U = pin.start_vectors(SEED, pb.N, m)
    lam, U, _ = S.iteration(U, None, 2, solve=False)
    times = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        lam, U, _ = S.iteration(U, lam, 2, solve=True)
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
    return times


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    pb, m = build_workload()
    times = cpu_oracle_iteration_seconds(pb, m, steps=args.steps, warmup=args.warmup)
    t = max(1e-12, sum(times) / len(times))
    value = pb.N * NEV / t
    sample = "one oracle augmented subspace iteration (full 128^3 workload, nev 50, block 56) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Q1 matrices, SplitMix64 start block)",
            "config": {"workload": WORKLOAD, "N_h": pb.N, "N_H": pb.N_H, "nev": NEV, "block": m},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, P, pin, torch, np, barrier):
    """Independent 2D problems of uneven size (meshes 64^2..512^2, lognormal kappa with
    sigma in [0.5, 2], nev in [8, 32], coarse mesh = fine/8), mixed precision, step (a) as
    3 steps of V-cycle-preconditioned CG (plain V-cycles stall on the roughest fields), tol 1e-8.
    Two arms, each on its own set of handles (torch's pool streams, one per handle):
    host-driven handles, solved one after another through pase_solve and then together
    through pase_solve_batched (a pool of host threads, one stream per handle); and
    graph_solve handles, whose pase_solve_batched records every problem's whole solve as
    one branch of a single CUDA graph and launches it once.  Each timed run follows an
    untimed one that records the graphs; launch counts are those of the timed run."""
    specs = pin.batch_workload(SEED, args.batch)
    pbs = [pin.build_problem(2, sp_["n"], sp_["n_coarse"], kappa_seed=sp_["kappa_seed"], sigma=sp_["sigma"],
                             mg_min=4) for sp_ in specs]
    nevs = [sp_["nev"] for sp_ in specs]
    tols = [1e-8] * len(specs)
    ms = [pin.guard_columns(nv) for nv in nevs]
    U0s = [torch.from_numpy(pin.start_vectors(SEED, pb.N, m)).cuda() for pb, m in zip(pbs, ms)]
    dof_nev = sum(pb.N * nv for pb, nv in zip(pbs, nevs))
    out = {"workload": f"{len(specs)} independent 2D Q1 problems, meshes 64^2..512^2, lognormal kappa "
                       "sigma 0.5..2, nev 8..32, coarse fine/8, mixed precision, 3 MG-preconditioned CG steps, tol 1e-8",
           "problems": len(specs), "total_dofs": int(sum(pb.N for pb in pbs))}

    def counts(hs):
        c = [P.pase_launch_counts(h) for h in hs]
        return tuple(sum(x[i] for x in c) for i in range(3))

    for gs in (0, 1):
        hs = []
        try:
            for pb, m in zip(pbs, ms):
                st_ = torch.cuda.Stream()
                opt = P.pase_default_options()
                opt.precision = P.PASE_PREC_MIXED
                opt.linear_solver = P.PASE_SOLVER_MGCG
                opt.inner_steps = 3
                opt.max_iter = 150
                opt.graph_solve = gs
                opt.coarse_level = pb.coarse_level
                h = P.pase_create(opt, st_.cuda_stream)
                hs.append(h)
                P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
                P.pase_reserve(h, m)
            Us = [torch.empty(pb.N, m, dtype=torch.float64, device="cuda") for pb, m in zip(pbs, ms)]
            lams = [torch.empty(m, dtype=torch.float64, device="cuda") for m in ms]
            barrier()
            t0 = time.perf_counter()
            P.pase_solve_batched(hs, nevs, tols, ms, U0s, lams, Us)
            barrier()
            t_first = time.perf_counter() - t0
            arm = {}
            if gs == 0:
                t0 = time.perf_counter()
                seq_iters = 0
                single, single_it = [], []
                for i, h in enumerate(hs):
                    t1 = time.perf_counter()
                    _, st1 = P.pase_solve(h, nevs[i], tols[i], ms[i], U0s[i], lams[i], Us[i])
                    single.append(time.perf_counter() - t1)
                    single_it.append(st1["iterations"])
                    seq_iters += st1["iterations"]
                barrier()
                arm["sequential_s"] = time.perf_counter() - t0
                arm["sequential_iterations"] = seq_iters
                slow = int(np.argmax(single))
                # the batch cannot finish before its slowest problem does alone
                arm["slowest_single"] = {"problem": slow, "seconds": single[slow], "n": specs[slow]["n"],
                                         "nev": nevs[slow], "iterations": single_it[slow]}
            c0 = counts(hs)
            t0 = time.perf_counter()
            rc, sts = P.pase_solve_batched(hs, nevs, tols, ms, U0s, lams, Us)
            barrier()
            t_bat = time.perf_counter() - t0
            c1 = counts(hs)
            kern, ingraph, glaunch = (c1[i] - c0[i] for i in range(3))
            arm.update({"status": rc, "first_call_s": t_first, "batched_s": t_bat,
                        "all_converged": all(s_["converged"] >= nv for s_, nv in zip(sts, nevs)),
                        "max_relres": max(s_["max_residual"] for s_ in sts),
                        "iterations": [s_["iterations"] for s_ in sts],
                        "problems_per_s": len(specs) / t_bat, "dof_nev_per_s": dof_nev / t_bat,
                        "kernels": kern, "kernels_in_graphs": ingraph, "graph_launches": glaunch,
                        "host_launch_calls": kern - ingraph + glaunch})
            if gs == 0:
                arm["speedup_vs_sequential"] = arm["sequential_s"] / t_bat
            out["one_graph" if gs else "thread_pool"] = arm
        finally:
            for h in hs:
                P.pase_destroy(h)
    tp, og = out["thread_pool"], out["one_graph"]
    out.update({"status": og["status"], "all_converged": tp["all_converged"] and og["all_converged"],
                "max_relres": max(tp["max_relres"], og["max_relres"]),
                "sequential_s": tp["sequential_s"], "batched_s": min(tp["batched_s"], og["batched_s"]),
                "speedup": tp["sequential_s"] / min(tp["batched_s"], og["batched_s"]),
                "same_iterations_both_arms": tp["iterations"] == og["iterations"]})
    return out


def run_learned(args, P, pin, torch, np):
    """Configuration 4, 2D: one smoother network trained on the solver's own samples from
    64 seeded lognormal fields (sigma 1, seeds 1000-1063, 256^2 meshes, 20 steps of 8
    pairs each: 10,240 pairs), evaluated on 16 held-out fields (seeds 2000-2015) by the
    two-V-cycle energy error factor against damped Jacobi, and by full solves of the
    1024^2 held-out field 2000 (coarse 128^2, nev 32, tol 1e-8): Jacobi and learned
    smoothing, FP64 and mixed, 2+2 sweeps and (learned) 1+1."""
    stream = torch.cuda.current_stream().cuda_stream

    def make(n, seed, params=None, smoother=0, m=None, precision=0, nu=2):
        pb = pin.build_problem(2, n, n // 8, kappa_seed=seed, sigma=1.0, mg_min=4)
        opt = P.pase_default_options()
        opt.coarse_level = pb.coarse_level
        opt.smoother = smoother
        opt.precision = precision
        opt.nu1 = opt.nu2 = nu
        h = P.pase_create(opt, stream)
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        P.pase_set_grid(h, 2, n, np.log(pb.kappa))
        if m:
            P.pase_reserve(h, m)
        if params is not None:
            P.pase_smoother_state(h, 2, params)
        return pb, h

    t0 = time.perf_counter()
    state = (pin.smoother_init(2, seed=1, noise=0.02),)
    accepted = 0
    for f in range(64):
        pb, h = make(256, 1000 + f, state)
        out = P.pase_train_smoother(h, steps=20, lr=1e-3, seed=f)
        accepted += int(out["accepted"])
        state = P.pase_smoother_state(h, 2)
        P.pase_destroy(h)
    train_s = time.perf_counter() - t0
    params = (state[0],)

    def factor(pb, h, m=8):
        e0 = pin.start_vectors(11, pb.N, m)
        W = np.empty_like(e0)
        P.pase_linear_solve(h, m, np.zeros_like(e0), np.ones(m), np.ascontiguousarray(pb.A @ e0), W)
        E = e0 - W
        return float(np.mean(np.sqrt(np.einsum("ij,ij->j", E, pb.A @ E) / np.einsum("ij,ij->j", e0, pb.A @ e0))))

    fl, fj = [], []
    for f in range(16):
        pb, hl = make(256, 2000 + f, params, smoother=P.PASE_SMOOTHER_LEARNED, m=8)
        fl.append(factor(pb, hl))
        P.pase_destroy(hl)
        pb, hj = make(256, 2000 + f, None, m=8)
        fj.append(factor(pb, hj))
        P.pase_destroy(hj)
    solves = {}
    nev = 32
    m = pin.guard_columns(nev)
    lam_ref = None
    variants = (("jacobi", P.PASE_SMOOTHER_JACOBI, P.PASE_PREC_FP64, 2),
                ("learned", P.PASE_SMOOTHER_LEARNED, P.PASE_PREC_FP64, 2),
                ("learned_1+1", P.PASE_SMOOTHER_LEARNED, P.PASE_PREC_FP64, 1),
                ("jacobi_mixed", P.PASE_SMOOTHER_JACOBI, P.PASE_PREC_MIXED, 2),
                ("learned_mixed", P.PASE_SMOOTHER_LEARNED, P.PASE_PREC_MIXED, 2),
                ("learned_mixed_1+1", P.PASE_SMOOTHER_LEARNED, P.PASE_PREC_MIXED, 1))
    for name, sm_, prec, nu in variants:
        pb, h = make(1024, 2000, params if sm_ else None, smoother=sm_, m=m, precision=prec, nu=nu)
        U0 = torch.from_numpy(pin.start_vectors(SEED, pb.N, m)).cuda()
        U = torch.empty_like(U0)
        lam = torch.empty(m, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rc, st = P.pase_solve(h, nev, 1e-8, m, U0, lam, U)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t1
        lamh = lam[:nev].cpu().numpy()
        solves[name] = {"status": rc, "iterations": st["iterations"], "seconds": sec,
                        "ms_per_iteration": 1e3 * sec / max(1, st["iterations"]),
                        "phase_ms": st["phase_ms"], "max_relres": st["max_residual"]}
        if lam_ref is None:
            lam_ref = lamh
        else:
            solves[name]["max_rel_eig_diff_vs_jacobi"] = float(np.max(np.abs(lamh - lam_ref) / lam_ref))
        P.pase_destroy(h)
    return {"workload": "2D Q1 lognormal kappa (sigma 1): train 64 fields at 256^2 (10,240 pairs), "
                        "evaluate 16 held-out fields at 256^2 and a full solve at 1024^2, nev 32",
            "train_seconds": train_s, "fields_accepted_by_validation": accepted,
            "vcycle2_energy_factor_learned": float(np.mean(fl)), "vcycle2_energy_factor_jacobi": float(np.mean(fj)),
            "heldout_fields_better": int(sum(a < b for a, b in zip(fl, fj))),
            "solve_1024": solves,
            "speedup_per_converged_pair": solves["jacobi"]["seconds"] / solves["learned"]["seconds"],
            "speedup_per_converged_pair_mixed": solves["jacobi_mixed"]["seconds"] / solves["learned_mixed"]["seconds"],
            "best_learned_vs_best_jacobi": min(solves["jacobi"]["seconds"], solves["jacobi_mixed"]["seconds"])
            / min(v["seconds"] for k, v in solves.items() if k.startswith("learned"))}


def run_learned3d(args, P, pin, torch, np):
    """Configuration 4, 3D: one smoother network (27 taps) trained on the solver's own
    samples from 64 seeded lognormal fields (sigma 1, seeds 1000-1063) at 32^3 (20 steps
    of 8 pairs each: 10,240 pairs), evaluated by the two-V-cycle energy error factor on 16
    held-out 64^3 fields (seeds 2000-2015) and by full solves of the 128^3 held-out field
    2000 (coarse 16^3, nev 32, tol 1e-8): Jacobi and learned smoothing, FP64 and mixed,
    2+2 sweeps and (learned) 1+1."""
    stream = torch.cuda.current_stream().cuda_stream

    def make(n, seed, params=None, smoother=0, m=None, precision=0, nu=2):
        pb = pin.build_problem(3, n, n // 8, kappa_seed=seed, sigma=1.0, mg_min=4)
        opt = P.pase_default_options()
        opt.coarse_level = pb.coarse_level
        opt.smoother = smoother
        opt.precision = precision
        opt.nu1 = opt.nu2 = nu
        h = P.pase_create(opt, stream)
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        P.pase_set_grid(h, 3, n, np.log(pb.kappa))
        if m:
            P.pase_reserve(h, m)
        if params is not None:
            P.pase_smoother_state(h, 3, params)
        return pb, h

    t0 = time.perf_counter()
    state = (pin.smoother_init(3, seed=1, noise=0.02),)
    accepted = 0
    for f in range(64):
        pb, h = make(32, 1000 + f, state)
        out = P.pase_train_smoother(h, steps=20, lr=1e-3, seed=f)
        accepted += int(out["accepted"])
        state = P.pase_smoother_state(h, 3)
        P.pase_destroy(h)
    train_s = time.perf_counter() - t0
    params = (state[0],)

    def factor(pb, h, m=8):
        e0 = pin.start_vectors(11, pb.N, m)
        W = np.empty_like(e0)
        P.pase_linear_solve(h, m, np.zeros_like(e0), np.ones(m), np.ascontiguousarray(pb.A @ e0), W)
        E = e0 - W
        return float(np.mean(np.sqrt(np.einsum("ij,ij->j", E, pb.A @ E) / np.einsum("ij,ij->j", e0, pb.A @ e0))))

    fl, fj = [], []
    for f in range(16):
        pb, hl = make(64, 2000 + f, params, smoother=P.PASE_SMOOTHER_LEARNED, m=8)
        fl.append(factor(pb, hl))
        P.pase_destroy(hl)
        pb, hj = make(64, 2000 + f, None, m=8)
        fj.append(factor(pb, hj))
        P.pase_destroy(hj)
    solves = {}
    nev = 32
    m = pin.guard_columns(nev)
    lam_ref = None
    variants = (("jacobi", P.PASE_SMOOTHER_JACOBI, P.PASE_PREC_FP64, 2),
                ("learned", P.PASE_SMOOTHER_LEARNED, P.PASE_PREC_FP64, 2),
                ("learned_1+1", P.PASE_SMOOTHER_LEARNED, P.PASE_PREC_FP64, 1),
                ("jacobi_mixed", P.PASE_SMOOTHER_JACOBI, P.PASE_PREC_MIXED, 2),
                ("learned_mixed", P.PASE_SMOOTHER_LEARNED, P.PASE_PREC_MIXED, 2),
                ("learned_mixed_1+1", P.PASE_SMOOTHER_LEARNED, P.PASE_PREC_MIXED, 1))
    for name, sm_, prec, nu in variants:
        pb, h = make(128, 2000, params if sm_ else None, smoother=sm_, m=m, precision=prec, nu=nu)
        U0 = torch.from_numpy(pin.start_vectors(SEED, pb.N, m)).cuda()
        U = torch.empty_like(U0)
        lam = torch.empty(m, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rc, st = P.pase_solve(h, nev, 1e-8, m, U0, lam, U)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t1
        lamh = lam[:nev].cpu().numpy()
        solves[name] = {"status": rc, "iterations": st["iterations"], "seconds": sec,
                        "ms_per_iteration": 1e3 * sec / max(1, st["iterations"]),
                        "phase_ms": st["phase_ms"], "max_relres": st["max_residual"]}
        if lam_ref is None:
            lam_ref = lamh
        else:
            solves[name]["max_rel_eig_diff_vs_jacobi"] = float(np.max(np.abs(lamh - lam_ref) / lam_ref))
        P.pase_destroy(h)
    return {"workload": "3D Q1 lognormal kappa (sigma 1): train 64 fields at 32^3 (10,240 pairs), evaluate 16 "
                        "held-out fields at 64^3 and full solves at 128^3 (coarse 16^3), nev 32",
            "train_seconds": train_s, "fields_accepted_by_validation": accepted,
            "vcycle2_energy_factor_learned": float(np.mean(fl)), "vcycle2_energy_factor_jacobi": float(np.mean(fj)),
            "heldout_fields_better": int(sum(a < b for a, b in zip(fl, fj))),
            "solve_128": solves,
            "speedup_per_converged_pair": solves["jacobi"]["seconds"] / solves["learned"]["seconds"],
            "speedup_per_converged_pair_mixed": solves["jacobi_mixed"]["seconds"] / solves["learned_mixed"]["seconds"],
            "best_learned_vs_best_jacobi": min(solves["jacobi"]["seconds"], solves["jacobi_mixed"]["seconds"])
            / min(v["seconds"] for k, v in solves.items() if k.startswith("learned"))}


def _solve_once(P, torch, stream, pb, nev, m, U0, tol=1e-8, warm=False, **opts):
    """pase_solve on a fresh handle with the given options, device-event timed; with warm,
    a first call (recording the graphs) precedes the reported one."""
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    for k, v in opts.items():
        setattr(opt, k, v)
    h = P.pase_create(opt, stream.cuda_stream)
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        P.pase_reserve(h, m)  # workspace and autotuning outside the timed call
        U = torch.empty_like(U0)
        lam = torch.empty(m, dtype=torch.float64, device="cuda")
        secs = []
        for _ in range(2 if warm else 1):  # with warm, the second call is the one reported
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c0 = P.pase_launch_counts(h)
            rc, st = P.pase_solve(h, nev, tol, m, U0, lam, U)
            c1 = P.pase_launch_counts(h)
            e1.record(stream)
            torch.cuda.synchronize()
            secs.append(e0.elapsed_time(e1) * 1e-3)
        sec = secs[-1]
        kern, ingraph, glaunch = (c1[i] - c0[i] for i in range(3))
        it = max(1, st["iterations"])
        out = {"status": rc, "iterations": st["iterations"], "seconds": sec, "max_relres": st["max_residual"],
               "dof_nev_per_s": pb.N * nev / sec, "ms_per_iteration": 1e3 * sec / it,
               "phase_ms": st["phase_ms"], "aug_iterations": st["aug_iterations"],
               "launches_per_iteration": kern / it, "host_launch_calls_per_iteration": (kern - ingraph + glaunch) / it}
        if warm:
            out["first_call_seconds"] = secs[0]
        return out, lam[:nev].cpu().numpy()
    finally:
        P.pase_destroy(h)


def run_cfg1(P, pin, torch, np, stream):
    """Configuration 1 (2D Q1 128^2, coarse 16^2, nev 10): L2-resident, so the numbers are
    latency and launch counts per iteration, FP64 and mixed (one untimed solve first)."""
    pb = pin.build_problem(2, 128, 16, mg_min=4)
    nev = 10
    m = pin.guard_columns(nev)
    U0 = torch.from_numpy(pin.start_vectors(0, pb.N, m)).cuda()
    out = {"workload": "laplace2d_q1_128_coarse16_nev10", "N_h": pb.N, "block": m}
    for name, prec in (("fp64", P.PASE_PREC_FP64), ("mixed", P.PASE_PREC_MIXED)):
        for gs in (0, 1):
            out[name + ("_graph" if gs else "")], _ = _solve_once(P, torch, stream, pb, nev, m, U0, warm=True,
                                                                  precision=prec, graph_solve=gs)
    return out


def run_variants(P, torch, stream, pb, m, U0):
    """The solver variants of the bench workload (FP64 solves to 1e-8): the step-(c)
    congruences of §4 (plain, PRECOND-A, -B, -B-A; the paper's Fig. 1 question), Alg. 3's
    two-solve form, and step (a) as plain CG with 40 steps (the numerical section's linear
    solver) or as 3 V-cycle-preconditioned CG steps, against 2 V-cycles."""
    rows = {}
    for name, kw in (("plain", dict(aug_transform=P.PASE_AUG_PLAIN)),
                     ("precond_a", dict(aug_transform=P.PASE_AUG_PRECOND_A)),
                     ("precond_b", dict(aug_transform=P.PASE_AUG_PRECOND_B)),
                     ("precond_ba", dict(aug_transform=P.PASE_AUG_PRECOND_BA)),
                     ("post_solve", dict(post_solve=1)),
                     ("cg40", dict(linear_solver=P.PASE_SOLVER_CG, inner_steps=40)),
                     ("mgcg3", dict(linear_solver=P.PASE_SOLVER_MGCG, inner_steps=3))):
        try:
            rows[name], _ = _solve_once(P, torch, stream, pb, NEV, m, U0, **kw)
        except Exception as exc:  # pragma: no cover
            rows[name] = {"error": str(exc)}
    return rows


def run_tensor(P, pin, torch, np, stream):
    """The operator of the numerical section's batch-scheme test, -div(T grad u) + phi u
    (T = I + (x-1/2)(x-1/2)^T, phi = exp(prod (x_k - 1/2))), on the bench mesh (3D Q1 128^3,
    coarse 16^3, nev 50): whole solves to 1e-8, FP64 and mixed."""
    t0 = time.perf_counter()
    pb = pin.build_problem(D, NFINE, NCOARSE, mg_min=4, operator="tensor")
    build_s = time.perf_counter() - t0
    m = pin.guard_columns(NEV)
    U0 = torch.from_numpy(pin.start_vectors(SEED, pb.N, m)).cuda()
    out = {"workload": "tensor_potential3d_q1_128_coarse16_nev50", "assembly_seconds_host": build_s}
    lams = {}
    for name, prec in (("fp64", P.PASE_PREC_FP64), ("mixed", P.PASE_PREC_MIXED)):
        out[name], lams[name] = _solve_once(P, torch, stream, pb, NEV, m, U0, precision=prec)
    out["mixed_speedup_per_converged_pair"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    out["mixed_vs_fp64_max_rel_eig_diff"] = float(np.max(np.abs(lams["mixed"] - lams["fp64"]) / lams["fp64"]))
    return out


def run_batch_scheme(P, pin, torch, np, stream):
    """The batch scheme of §5 (Alg. 7), FP64, on the section-6.3 operator in 2D (64^2 mesh,
    coarse 32^2): the first 24 pairs in batches of 8 (block 16), against one pase_solve of
    all 24 (block 32)."""
    pb = pin.build_problem(2, 64, 32, mg_min=4, operator="tensor")
    nev, k, m = 24, 8, 16
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    h = P.pase_create(opt, stream.cuda_stream)
    out = {"workload": "tensor_potential2d_q1_64_coarse32_nev24", "k": k, "block": m}
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        lam = np.empty(nev)
        U = np.empty((pb.N, nev))
        t0 = time.perf_counter()
        rc, st = P.pase_solve_batches(h, nev, k, m, 1e-8, lam, U)
        sec = time.perf_counter() - t0
        out["batches"] = {"status": rc, "seconds": sec, "iterations": st["iterations"],
                          "max_relres": st["max_residual"], "converged": st["converged"]}
    finally:
        P.pase_destroy(h)
    U0 = torch.from_numpy(pin.start_vectors(0, pb.N, 32)).cuda()
    out["one_block"], lam1 = _solve_once(P, torch, stream, pb, nev, 32, U0, warm=True)
    out["max_rel_eig_diff"] = float(np.max(np.abs(lam - lam1) / lam1))
    return out


def run_profile_smoother(args):
    """The learned smoother's inference pass (tensor-core convolutions) on a 2D lognormal
    field at --size (8 columns, Jacobi-equivalent weights plus noise), three applications,
    for ncu (capture with -k regex:k_sm_conv_tc; per application the launches are the
    input layer, two hidden layers and the output layer)."""
    import numpy as np
    import torch

    import pase_inputs as pin
    from paper_2502_04589_gb300 import pase as P
    n = args.size
    pb = pin.build_problem(2, n, n // 8, kappa_seed=2000, sigma=1.0, mg_min=4)
    opt = P.pase_default_options()
    opt.coarse_level = pb.coarse_level
    opt.autotune = 0
    h = P.pase_create(opt, torch.cuda.current_stream().cuda_stream)
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        P.pase_reserve(h, 8)
        P.pase_set_grid(h, 2, n, np.log(pb.kappa))
        P.pase_smoother_state(h, 2, (pin.smoother_init(2, seed=1, noise=0.02),))
        R = torch.from_numpy(pin.start_vectors(1, pb.N, 8)).cuda()
        D = torch.empty_like(R)
        for _ in range(3):
            P.pase_smoother_apply(h, 8, R, D)
        torch.cuda.synchronize()
    finally:
        P.pase_destroy(h)
    print(json.dumps({"profile_kernel": "smoother", "size": n, "N_h": pb.N, "columns": 8}), flush=True)
    return 0


def run_profile_kernel(args):
    """One kernel of the path on the bench workload at --size, for ncu: two warm-up
    launches, then three timed ones (capture with -k <kernel> -s 2 -c 1).  The handle is
    created without the autotuner, so the sparse kernels run at 256 threads per block.
    --profile-kernel smoother profiles the learned smoother instead (2D, --size^2)."""
    if args.profile_kernel == "smoother":
        return run_profile_smoother(args)
    import torch

    from paper_2502_04589_gb300 import pase as P
    pb, m = build_workload(args.size)
    opt = P.pase_default_options()
    opt.precision = P.PASE_PREC_MIXED if args.profile_kernel == "jacobi_fp32" else P.PASE_PREC_FP64
    opt.coarse_level = pb.coarse_level
    opt.autotune = 0
    stream = torch.cuda.Stream()
    h = P.pase_create(opt, stream.cuda_stream)
    try:
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        P.pase_reserve(h, m)
        ms = P.pase_time_kernel(h, args.profile_kernel, m, 3)
    finally:
        P.pase_destroy(h)
    print(json.dumps({"profile_kernel": args.profile_kernel, "size": args.size, "N_h": pb.N, "nnz": pb.A.nnz,
                      "block": m, "ms_per_launch": ms}), flush=True)
    return 0


def run_ours(args):
    # let up to 32 streams (the batched run) feed the GPU without false dependencies
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import numpy as np
    import torch

    import pase_inputs as pin
    from paper_2502_04589_gb300 import pase as P

    rank, world, local = _env_rank()
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    pb, m = build_workload(args.size)

    def make(precision, graph_solve=0):
        opt = P.pase_default_options()
        opt.precision = precision
        opt.graph_solve = graph_solve
        opt.coarse_level = pb.coarse_level
        h = P.pase_create(opt, stream.cuda_stream)
        P.pase_setup(h, pb.A, pb.M, pb.chain, pb.A_H, pb.M_H)
        P.pase_reserve(h, m)
        return h

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    h = make(P.PASE_PREC_FP64)
    U0h = pin.start_vectors(SEED + rank, pb.N, m)
    U0 = torch.from_numpy(U0h).cuda()
    U = U0.clone()
    # the fused A_h / M_h product (one pass over the pattern), timed alone
    X = U0.clone()
    AX, MX = torch.empty_like(X), torch.empty_like(X)
    reps = 10
    ksampler = ClockSampler(local)
    ksampler.start()
    for _ in range(3):
        P.pase_spmm_am(h, m, X, AX, MX)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        P.pase_spmm_am(h, m, X, AX, MX)
    e1.record(stream)
    torch.cuda.synchronize()
    kclocks = ksampler.stop()
    spmm_ms = e0.elapsed_time(e1) / reps
    nnz = pb.A.nnz
    spmm_flops = 4.0 * nnz * m
    spmm_bytes = nnz * (4 + 16) + 8 * (pb.N + 1) + 3 * pb.N * m * 8
    peak_fp64 = 1.25e12
    spmm_live = {"kernel": "k_csr<double, MV_AM> (fused A_h/M_h SpMM, FP64)", "ms": spmm_ms,
                 "tflops": spmm_flops / (spmm_ms * 1e-3) / 1e12,
                 "frac": spmm_flops / (spmm_ms * 1e-3) / peak_fp64,
                 "achieved_gbs": spmm_bytes / (spmm_ms * 1e-3) / 1e9, "clocks": kclocks}

    lam = torch.zeros(m, dtype=torch.float64, device="cuda")
    relres = torch.zeros(m, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        P.pase_iterate(h, NEV, m, U, lam, False)  # first iteration: W = U0
        for _ in range(args.warmup):
            P.pase_iterate(h, NEV, m, U, lam, True, relres)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    # the dominant kernel (fine-level FP64 damped-Jacobi sweep, most of step (a)) is timed
    # live: the library brackets each of its launches with CUDA events on its stream
    P.pase_profile_kernel(h, "jacobi_fp64")
    k0 = P.pase_kernel_count(h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        P.pase_iterate(h, NEV, m, U, lam, True, relres)
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    jac_n, jac_ms_total = P.pase_profile_read(h)
    P.pase_profile_kernel(h, None)
    jac_ms = jac_ms_total / max(1, jac_n)
    jac_flops = 2.0 * nnz * m + 3.0 * pb.N * m
    jac_bytes = nnz * 12 + 16 * pb.N + 3 * pb.N * m * 8
    roofline = {"bound": "alu", "kernel": "k_csr<double, JACOBI> (damped Jacobi sweep on A_h, FP64)",
                "achieved": jac_flops / (jac_ms * 1e-3) / 1e12, "peak": peak_fp64 / 1e12,
                "unit": "TFLOP/s", "frac": jac_flops / (jac_ms * 1e-3) / peak_fp64,
                "traffic": JACOBI_TRAFFIC_BYTES,
                "peak_source": "nominal FP64 1.25 TFLOP/s (recipe table; no FP64 figure is measured "
                               "in the peaks file)",
                "flops_per_launch": jac_flops, "algorithmic_bytes": jac_bytes,
                "achieved_gbs": jac_bytes / (jac_ms * 1e-3) / 1e9, "ms": jac_ms,
                "launches_timed": jac_n, "launches_per_step": jac_n / max(1, args.steps),
                "share_of_step": jac_ms_total / (ev0.elapsed_time(ev1)),
                "timing": "CUDA events around each launch on the library stream, inside the timed steps"}
    launches = (P.pase_kernel_count(h) - k0) // max(1, args.steps)
    ms = ev0.elapsed_time(ev1) / args.steps
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms = float(t.item())
    value = world * pb.N * NEV / (ms * 1e-3)

    # the same product on the iterated block (data-dependence check of the kernel time)
    X.copy_(U)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        P.pase_spmm_am(h, m, X, AX, MX)
    e1.record(stream)
    torch.cuda.synchronize()
    spmm_live["ms_on_iterated_block"] = e0.elapsed_time(e1) / reps

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    Uh = torch.from_numpy(U.cpu().numpy()).pin_memory()
    lh = torch.from_numpy(lam.cpu().numpy()).pin_memory()
    rh = torch.zeros(m, dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):  # untimed: the first host-buffer call allocates the staging buffers
        P.pase_iterate(h, NEV, m, Uh.numpy(), lh.numpy(), True, rh.numpy())
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.pase_iterate(h, NEV, m, Uh.numpy(), lh.numpy(), True, rh.numpy())
    barrier()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e = {"value": world * pb.N * NEV / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(pb.N * m * 8 + m * 8),
           "d2h_bytes_per_step": int(pb.N * m * 8 + 2 * m * 8)}
    P.pase_destroy(h)

    # per-kernel rooflines on the fine level (library-timed, CUDA events)
    kernels = {}
    peaks = {"hbm_gbs": 6783.8}
    try:
        peaks.update(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))))
    except Exception:
        pass
    nnz, N = pb.A.nnz, pb.N

    def kinfo(name, ms, flops, nbytes, bound):
        d = {"ms": ms, "gflop": flops / 1e9, "gbytes": nbytes / 1e9,
             "tflops": flops / (ms * 1e-3) / 1e12, "gbs": nbytes / (ms * 1e-3) / 1e9}
        if bound == "alu":
            d.update(bound="alu", frac=d["tflops"] / 1.25, peak="FP64 1.25 TFLOP/s nominal")
        else:
            d.update(bound="hbm", frac=d["gbs"] / peaks["hbm_gbs"], peak=f"HBM {peaks['hbm_gbs']} GB/s measured")
        return d

    hk = make(P.PASE_PREC_MIXED)
    # FP64 FMA rate of this GPU (the measured ceiling of the FP64-pipe-bound kernels)
    try:
        fma_ms = P.pase_time_kernel(hk, "fma_fp64", m, 5)
        kernels["fma_fp64"] = {"ms": fma_ms, "tflops": P.FMA_FP64_FLOPS / (fma_ms * 1e-3) / 1e12,
                               "what": "8 independent FP64 FMA chains per thread, 1216 x 256 threads"}
    except Exception as exc:  # pragma: no cover
        kernels["fma_fp64"] = {"error": str(exc)}
    n1 = NFINE - 1
    st_vbytes = (n1 + 2) * ((n1 + 3) // 4) * ((n1 + 15) // 16) * 28 * 64 * 4  # step-major coefficients
    for name, flops, nbytes, bound in (
            ("spmm_am_fp64", 4.0 * nnz * m, nnz * 20 + 8 * (N + 1) + 3 * N * m * 8, "alu"),
            ("jacobi_fp64", 2.0 * nnz * m + 3.0 * N * m, nnz * 12 + 16 * N + 3 * N * m * 8, "alu"),
            ("jacobi_fp32", 2.0 * nnz * m + 3.0 * N * m, st_vbytes + 3 * N * m * 4, "hbm"),
            ("jacobi_fp32_csr", 2.0 * nnz * m + 3.0 * N * m, nnz * 8 + 12 * N + 3 * N * m * 4, "hbm"),
            # split of X (read 8, write 8 per entry), then index + 4 FP32 value streams, the split
            # X (8 per entry) and two FP64 outputs
            ("spmm_am_df64", 4.0 * nnz * m, nnz * 20 + 8 * (N + 1) + 2 * N * m * 8 + 3 * N * m * 8, "hbm"),
            ("gram_fp64", 1.0 * N * m * (m + 4), 2 * N * m * 8, "alu"),
            ("prolong_fp64", 2.0 * N * m * m, 2 * N * m * 8, "alu"),
            ("prolong_split", 2.0 * N * m * m, 2 * N * m * 8, "hbm"),
            ("gram_split", 2.0 * N * m * (m + 4), 2 * 2 * N * m * 8, "hbm")):
        try:
            ms_k = P.pase_time_kernel(hk, name, m, 10)
            kernels[name] = kinfo(name, ms_k, flops, nbytes, bound)
        except Exception as exc:  # pragma: no cover
            kernels[name] = {"error": str(exc)}
    kernels["jacobi_fp32"]["kernel"] = "k_stencil<3, JACOBI> (structured grid, bulk-copy staged planes)"
    kernels["jacobi_fp32"]["bytes_model"] = ("step-major coefficients (28 per row, tile-padded) + X, b, y "
                                             "of [N][m] FP32 (no column indices)")
    kernels["jacobi_fp32_csr"]["kernel"] = "k_csr<float, JACOBI> (the CSR kernel, same sweep)"
    kernels["spmm_am_df64"]["kernel"] = ("k_split_df64 + k_csr_df64<MV_AM> (fused A_h X, M_h X in double-float "
                                         "on the FP32 pipe; issue-bound)")
    kernels["spmm_am_df64"]["speedup_vs_fp64"] = kernels["spmm_am_fp64"]["ms"] / kernels["spmm_am_df64"]["ms"]
    for name, nn in (("sygv", m), ("sygv3", 3 * m)):
        try:
            kernels[name] = {"ms": P.pase_time_kernel(hk, name, m, 5), "n": nn, "k": m, "bound": "latency"}
        except Exception as exc:  # pragma: no cover
            kernels[name] = {"error": str(exc)}
    P.pase_destroy(hk)

    # whole solve to 1e-8, FP64 and mixed, host-driven and as one recorded graph; each
    # timed on its second call (the first records the graphs and is reported beside it)
    solves = {}
    lams = {}
    if not args.no_solve:
        for name, prec, gs in (("fp64", P.PASE_PREC_FP64, 0), ("mixed", P.PASE_PREC_MIXED, 0),
                               ("fp64_graph", P.PASE_PREC_FP64, 1), ("mixed_graph", P.PASE_PREC_MIXED, 1)):
            hs = make(prec, gs)
            Uo = torch.empty_like(U0)
            lo = torch.empty(m, dtype=torch.float64, device="cuda")
            secs = []
            for _ in range(2):
                barrier()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                c0 = P.pase_launch_counts(hs)
                rc, st = P.pase_solve(hs, NEV, 1e-8, m, U0, lo, Uo)
                c1 = P.pase_launch_counts(hs)
                s1.record(stream)
                barrier()
                secs.append(s0.elapsed_time(s1) * 1e-3)
            sec = secs[1]
            kern, ingraph, glaunch = (c1[i] - c0[i] for i in range(3))
            solves[name] = {"status": rc, "iterations": st["iterations"], "seconds": sec,
                            "first_call_seconds": secs[0],
                            "max_relres": st["max_residual"], "dof_nev_per_s": pb.N * NEV / sec,
                            "ms_per_iteration": 1e3 * sec / max(1, st["iterations"]),
                            "phase_ms": st["phase_ms"], "aug_iterations": st["aug_iterations"],
                            "kernels": kern, "kernels_in_graphs": ingraph, "graph_launches": glaunch,
                            "host_launch_calls": kern - ingraph + glaunch}
            lams[name] = lo[:NEV].cpu().numpy()
            P.pase_destroy(hs)
        if "fp64" in solves and "mixed" in solves:
            solves["mixed_speedup_per_converged_pair"] = solves["fp64"]["seconds"] / solves["mixed"]["seconds"]
            solves["mixed_vs_fp64_max_rel_eig_diff"] = float(np.max(np.abs(lams["mixed"] - lams["fp64"]) /
                                                                    lams["fp64"]))
            solves["graph_vs_host_driven_max_rel_eig_diff"] = float(max(
                np.max(np.abs(lams[a + "_graph"] - lams[a]) / lams[a]) for a in ("fp64", "mixed")))

        # the same solves with a wider block: the guard-column rule gives 56 columns for nev
        # 50, which cuts the 6-fold eigenvalue cluster at indices 55..60 of this spectrum;
        # 64 columns hold the whole cluster, so the last wanted pairs see the gap to index 65
        wide = {}
        try:
            m64 = 64
            U064 = torch.from_numpy(pin.start_vectors(SEED + rank, pb.N, m64)).cuda()
            for name, prec in (("fp64", P.PASE_PREC_FP64), ("mixed", P.PASE_PREC_MIXED)):
                wide[name], lw = _solve_once(P, torch, stream, pb, NEV, m64, U064, warm=True, precision=prec)
                if name in lams:
                    wide[name]["max_rel_eig_diff_vs_block56"] = float(np.max(np.abs(lw - lams[name]) / lams[name]))
            del U064
        except Exception as exc:  # pragma: no cover
            wide = {"error": str(exc)}
        solves["block64"] = wide

    if "tflops" in kernels.get("fma_fp64", {}):
        # the microbenchmark stays below what the FP64-pipe-bound kernels reach, so the
        # nominal rate remains the peak; the measured rate is reported beside it
        roofline["fma_microbenchmark_tflops"] = kernels["fma_fp64"]["tflops"]
    converged = None
    if "fp64" in solves and "mixed" in solves:
        best = {a: min((solves[k] for k in (a, a + "_graph") if k in solves), key=lambda r: r["seconds"])
                for a in ("fp64", "mixed")}
        converged = {"metric": "DOF*nev/s to relative residual 1e-8 (whole pase_solve, 3D Q1 128^3, nev 50; "
                               "faster of the host-driven and the recorded-graph solve, second call)",
                     "fp64": best["fp64"]["dof_nev_per_s"], "mixed": best["mixed"]["dof_nev_per_s"],
                     "fp64_seconds": best["fp64"]["seconds"], "mixed_seconds": best["mixed"]["seconds"],
                     "fp64_ms_per_iteration": best["fp64"]["ms_per_iteration"],
                     "mixed_ms_per_iteration": best["mixed"]["ms_per_iteration"],
                     "mixed_speedup_per_converged_pair": best["fp64"]["seconds"] / best["mixed"]["seconds"],
                     "block": m}
        wide = solves.get("block64", {})
        if "fp64" in wide and "mixed" in wide:
            converged["block64"] = {
                "block": 64, "why": "nev 50 + 14 guard columns: the whole 6-fold cluster at indices 55..60 "
                                    "inside the block (the default 56 cuts it)",
                "fp64": wide["fp64"]["dof_nev_per_s"], "mixed": wide["mixed"]["dof_nev_per_s"],
                "fp64_seconds": wide["fp64"]["seconds"], "mixed_seconds": wide["mixed"]["seconds"],
                "fp64_iterations": wide["fp64"]["iterations"], "mixed_iterations": wide["mixed"]["iterations"],
                "mixed_speedup_per_converged_pair": wide["fp64"]["seconds"] / wide["mixed"]["seconds"],
                "fp64_vs_block56": best["fp64"]["seconds"] / wide["fp64"]["seconds"],
                "mixed_vs_block56": best["mixed"]["seconds"] / wide["mixed"]["seconds"]}
    extra = {}
    if rank == 0 and not args.no_solve:
        for key, fn in (("cfg1_latency", lambda: run_cfg1(P, pin, torch, np, stream)),
                        ("variants", lambda: run_variants(P, torch, stream, pb, m, U0)),
                        ("tensor_operator", lambda: run_tensor(P, pin, torch, np, stream)),
                        ("batch_scheme", lambda: run_batch_scheme(P, pin, torch, np, stream))):
            try:
                extra[key] = fn()
            except Exception as exc:  # pragma: no cover
                extra[key] = {"error": str(exc)}
    batched = run_batched(args, P, pin, torch, np, barrier) if args.batch > 0 else None
    learned = run_learned(args, P, pin, torch, np) if (args.learned and rank == 0) else None
    learned3d = run_learned3d(args, P, pin, torch, np) if (args.learned and rank == 0) else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        times = cpu_oracle_iteration_seconds(pb, m, steps=1)
        cpu = {"value": pb.N * NEV / times[0], "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": "one oracle augmented subspace iteration on the full 128^3 workload (nev 50, block 56)"}

    if rank == 0:
        wl = WORKLOAD if args.size == NFINE else WORKLOAD.replace("128", str(args.size))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded Q1 matrices, SplitMix64 start block)",
                "config": {"workload": wl, "N_h": pb.N, "nnz": pb.A.nnz, "N_H": pb.N_H, "nev": NEV,
                           "block": m, "linear_solve": "2 V-cycles, damped Jacobi 2+2, omega 2/3",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (block 0.92 GB)",
                           "dense_products": "steps (b) and (d): FP64-accurate error-free digit splitting on "
                                             "the BF16 tensor cores (option split_gemm)"},
                "roofline": roofline, "spmm_fp64": spmm_live, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks, "converged": converged, "solve": solves, "batched": batched,
                "learned_smoother": learned, "learned_smoother_3d": learned3d}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-kernel", default=None,
                    help="only launch this kernel (spmm_am_fp64, jacobi_fp64, jacobi_fp32, ...) for ncu")
    ap.add_argument("--learned", type=int, default=1, help="1: run the learned-smoother section")
    ap.add_argument("--batch", type=int, default=64,
                    help="independent problems in the batched run (0 skips it)")
    ap.add_argument("--size", type=int, default=NFINE,
                    help="fine mesh size (elements per side); the bench workload is 128")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_kernel:
        return run_profile_kernel(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

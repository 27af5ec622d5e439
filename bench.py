#!/usr/bin/env python
"""Benchmark of the MGM path on GB300: time to a 1e-10 relative residual at N = 1,048,576.

Workload (one "step" = one pass of the whole path over the step's problems): the unit sphere
(spherical Fibonacci points, jitter 0.1 h) and the torus R = 1, r = 1/3 (2048 x 512 parametric
grid, jitter 0.1 h), each N = 1,048,576; tangent-plane PHS RBF-FD with phi = r^3 and degree-3
polynomials, n = 50; L = I - D (-Lap + I); right-hand side a seeded sum of real spherical
harmonics up to l = 20 with N(0, 1) coefficients; N_min = 250, m = 3, V(1,1) multicolour GS,
FP32 V-cycle inside FP64 flexible GMRES to 1e-10. Per problem the step runs kNN stencils and
weights (FP32 LU with FP64 iterative refinement: the FP64 solution of each stencil system), the
hierarchy (RCM, weighted sample elimination, transfers, Galerkin products,
colourings, coarsest inverse) and the solve, all in libmgm kernels. Inputs are resident in HBM
when the timed region starts; the level-1 operator (~630 MB) exceeds the 129 MB L2, so no flush
is needed between steps.

Reported: value = mean device time per problem for the whole path (ms, lower is better); the
phase split (stencils / setup / solve, the solve alone being the paper's convention); the same
solve with an FP64 V-cycle and the whole path with FP64 weights and cycle (the "FP64 MGM"
comparison); the roofline of the dominant kernel (the stencil-weight solves, FP64-pipe-bound)
and of the finest-level Gauss-Seidel sweep (HBM-bound); e2e through pinned host buffers; the oracle timed on the host cores.

--impl reference times the CPU oracle (the plain FP64 C implementation that the tests compare
against) on a bounded sample of the same workload.

Multi-GPU: independent problems shard across ranks (each rank runs its own seeded sphere and
torus; weak scaling; no collective on the data path). Launch N>1 with torch.distributed.run.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-10 rel. residual at N=1M, mixed vs FP64 MGM; V-cycle HBM GB/s vs peak"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes of phs_weights_rl_k<60> per stencil: dram__bytes_read.sum + dram__bytes_write.sum of one
# ncu capture of the current kernel on 524,288 stencils (136.3 MB + 160.6 MB; its 210 MB of output
# exceed L2, so most writes reach DRAM within the launch), divided by the stencils
RL_DRAM_BYTES_PER_STENCIL = (136305664 + 160632064) / 524288

P = dict(n=50, k=1, ell=3, mu=1.0, n_min=250, m=3, tol=1e-10, restart=50, maxit=200)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=1048576, help="points per surface")
    ap.add_argument("--cpu-sample", type=int, default=32768, help="points of the oracle's bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c5"],
                    help="c2: the N=1M sphere/torus time-to-solution line; c3: the full 64-surface batched line; "
                         "c5: Schnakenberg pattern formation on a 4M-point bumpy sphere (ms per time step)")
    ap.add_argument("--c5-steps", type=int, default=100, help="time steps timed in the c5 line")
    ap.add_argument("--c5-size", type=int, default=1 << 22, help="points of the c5 bumpy sphere")
    ap.add_argument("--batch-problems", type=int, default=64, help="surfaces in the batched measurement of the c2 line")
    ap.add_argument("--eigs", type=int, default=16, help="shift-invert eigenpairs computed on the 1M sphere (0: none)")
    ap.add_argument("--learned-surfaces", type=int, default=200,
                    help="training surfaces of the learned-correction measurement (0 skips it)")
    ap.add_argument("--learned-eval-size", type=int, default=1 << 20, help="points of the held-out bumpy torus")
    ap.add_argument("--single", action="store_true",
                    help="one pass of the path on the sphere only (a small driver for profilers); prints its phases")
    ap.add_argument("--vcycles", type=int, default=0,
                    help="profiling driver: build the sphere problem of --size, then run this many V-cycles "
                         "(FP32 unless --fp64-cycle; --learned-n attaches an untrained correction of that stencil size)")
    ap.add_argument("--fp64-cycle", action="store_true")
    ap.add_argument("--transfer-bf16", action="store_true", help="profiling driver: BF16-stored P/R weights")
    ap.add_argument("--sweeps", default="0,5,4", help="profiling driver: sweep schedules to compare (persistent_sweeps values)")
    ap.add_argument("--learned-n", type=int, default=0)
    return ap.parse_args()


def rank_seed(rank):
    """Seed of a rank's problems: ranks solve different seeded surfaces (weak scaling)."""
    return 2 + 1000 * rank


def max_over_ranks(ms, world, device=None):
    """Timing of the whole job: the slowest rank's (a MAX all-reduce; the identity on one rank)."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as tdist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_ms_per_problem(ms_total, steps, nprob, world):
    """Time per problem of the whole job: every rank solves nprob problems a step."""
    return ms_total / (steps * nprob * world)


def problems(N, rank):
    from paper_2204_06154_gb300 import inputs as I
    seed = rank_seed(rank)
    xs, ns = I.fibonacci_sphere(N, jitter=0.1, seed=seed)
    xt, nt = I.torus_grid(N, 1.0, 1.0 / 3.0, jitter=0.1, seed=seed)
    return [("sphere", xs, ns, I.random_sh_rhs(xs, 20, seed)), ("torus", xt, nt, I.random_sh_rhs(xt, 20, seed))]


# ----------------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------------
class Clocks:
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ----------------------------------------------------------------------------------------------
# one problem through the whole path (device-resident inputs), with phase events
# ----------------------------------------------------------------------------------------------
def run_problem(M, torch, x, nrm, f, precision="f32", ev=None):
    """precision "f32": the mixed pipeline (FP32 LU + FP64 refinement for the stencil weights, FP32
    V-cycle, FP64 FGMRES); "f64": FP64 elimination and an FP64 V-cycle."""
    E = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    E[0].record()
    idx = M.knn(x, None, P["n"], self_first=True)
    E[1].record()
    w = M.stencil_weights(x, nrm, idx, "rbf", P["k"], P["ell"], weights="mixed" if precision == "f32" else "f64")
    E[2].record()
    rp, ci, v = M.assemble(idx, w, P["mu"])
    E[3].record()
    H = M.Hierarchy(x, rp, ci, v, P["n_min"], m=P["m"], precision=precision)
    E[4].record()
    u, info = H.solve(f, tol=P["tol"], restart=P["restart"], maxit=P["maxit"])
    E[5].record()
    E[5].synchronize()
    t = [E[i].elapsed_time(E[i + 1]) for i in range(5)]
    out = {"knn_ms": t[0], "weights_ms": t[1], "assemble_ms": t[2], "setup_ms": t[3], "solve_ms": t[4],
           "total_ms": E[0].elapsed_time(E[5]), "iters": info["iters"], "rel_res": info["rel_res"],
           "converged": info["converged"]}
    return out, H, u


def bench_ours(a, rank, world, local_rank):
    import torch
    from paper_2204_06154_gb300 import mgm as M
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    M.lib()
    probs = problems(a.size, rank)
    dprobs = [(name, torch.from_numpy(x).to(dev), torch.from_numpy(n).to(dev), torch.from_numpy(f).to(dev))
              for name, x, n, f in probs]
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    fp64_gflops = M.probe_fp64_fma(reps=20)  # the FP64-pipe roofline's denominator, on this GPU now
    # warm-up steps
    for _ in range(a.warmup):
        for name, x, n, f in dprobs:
            r, H, u = run_problem(M, torch, x, n, f)
            del H, u
    # timed steps
    barrier()
    records = []
    l0 = M.kernel_launches()
    with Clocks(local_rank) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps):
            for name, x, n, f in dprobs:
                r, H, u = run_problem(M, torch, x, n, f)
                r["problem"] = name
                records.append(r)
                del H, u
        e1.record()
        e1.synchronize()
    barrier()
    launches = M.kernel_launches() - l0
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    nprob = len(dprobs)
    res = {"ms_total": ms, "records": records, "launches": launches, "clocks": clk.summary(), "nprob": nprob,
           "fp64_gflops": fp64_gflops}

    # FP64 MGM on the same problems (solve time; the paper's convention excludes setup)
    fp64 = []
    for name, x, n, f in dprobs:
        r, H, u = run_problem(M, torch, x, n, f, precision="f64")
        r["problem"] = name
        fp64.append(r)
        del H, u
    res["fp64"] = fp64

    # profiles on the sphere: V-cycle, finest sweep, outer SpMV (mixed), and the weights kernel
    name, x, n, f = dprobs[0]
    r, H, u = run_problem(M, torch, x, n, f)
    res["profile"] = H.profile(reps=20)
    res["stats"] = H.stats()
    # the V-cycle's lower bound: dependent-launch latency at the finest sweep's launch shape, and
    # each level's bytes at the measured copy bandwidth
    blocks0 = H.sweep_config(0)["blocks"] or 456
    res["chain_us"] = M.probe_launch_chain(blocks0, 256, 256, True, 10)
    res["chain_blocks"] = blocks0
    res["floor"] = H.vcycle_floor(res["chain_us"], float(peaks()[0].get("hbm_gbs", 6800.0)))
    if a.eigs > 0:
        res["eigs"] = bench_eigs(torch, H, a.eigs)
    del H, u
    # e2e: pinned host inputs -> device -> whole path -> solution back to the host
    hp = [(torch.from_numpy(x).pin_memory(), torch.from_numpy(nn).pin_memory(), torch.from_numpy(f).pin_memory())
          for _, x, nn, f in probs]
    uh = torch.empty(a.size, dtype=torch.float64).pin_memory()
    barrier()
    e0.record()
    h2d = d2h = 0
    for xh, nh, fh in hp:
        x = xh.to(dev, non_blocking=True); nn = nh.to(dev, non_blocking=True); f = fh.to(dev, non_blocking=True)
        h2d += xh.numel() * 8 + nh.numel() * 8 + fh.numel() * 8
        r, H, u = run_problem(M, torch, x, nn, f)
        uh.copy_(u, non_blocking=True)
        d2h += u.numel() * 8
        del H
    e1.record()
    e1.synchronize()
    res["e2e_ms"] = e0.elapsed_time(e1) / len(hp)
    res["e2e_h2d"] = h2d // len(hp)
    res["e2e_d2h"] = d2h // len(hp)
    if a.batch_problems > 0:
        res["batched"] = bench_batched(a.batch_problems, dev)
        if a.learned_surfaces > 0:
            res["learned"] = bench_learned(a.learned_surfaces, a.learned_eval_size, dev)
    if a.c5_steps > 0:
        res["pattern"] = bench_pattern(a.c5_size, a.c5_steps, 3)
    return res


# ----------------------------------------------------------------------------------------------
# oracle (CPU) timing on a bounded sample
# ----------------------------------------------------------------------------------------------
def oracle_sample(Ns):
    import oracle as O
    from paper_2204_06154_gb300 import inputs as I
    x, nrm = I.fibonacci_sphere(Ns, jitter=0.1, seed=2)
    f = I.random_sh_rhs(x, 20, 2)
    t0 = time.perf_counter()
    idx, w, L = O.build_operator(x, nrm, P["n"], "rbf", P["k"], P["ell"], P["mu"])
    Hh = O.setup(x, L, P["n_min"], m=P["m"], seed=0)
    u, it, rel = O.fgmres(L, Hh, f, tol=P["tol"], restart=P["restart"], maxit=P["maxit"])
    dt = time.perf_counter() - t0
    return dt * 1e3, it, rel


# ----------------------------------------------------------------------------------------------
# batched heat-step solves on bumpy spheres (GFD), many right-hand sides per surface
# ----------------------------------------------------------------------------------------------
C3 = dict(n=25, ell=2, alpha=4.0, n_min=250, tol=1e-8, nrhs=8)


def c3_problems(nprob, seed=3):
    from paper_2204_06154_gb300 import inputs as I
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(20000), np.log(400000), nprob)).astype(int)
    out = []
    for q, N in enumerate(sizes):
        x, nrm = I.bumpy_sphere(int(N), seed=seed * 1000 + q)
        h2 = 4.0 * math.pi / N                       # t = h^2 with h the mean spacing of a unit sphere
        dirs = rng.standard_normal((C3["nrhs"], 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        xn = x / np.linalg.norm(x, axis=1, keepdims=True)
        F = np.zeros((C3["nrhs"], N))
        for r in range(C3["nrhs"]):
            F[r, int(np.argmax(xn @ dirs[r]))] = 1.0   # delta source at the node nearest the direction
        out.append((x, nrm, F, h2))
    return out


def bench_batched(nprob, dev):
    import torch
    from paper_2204_06154_gb300 import mgm as M
    probs = c3_problems(nprob)
    d = [(torch.from_numpy(x).to(dev), torch.from_numpy(n).to(dev), torch.from_numpy(F).to(dev), h2)
         for x, n, F, h2 in probs]
    E = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    E[0].record()
    Hs = []
    for x, n, F, h2 in d:
        _, _, rp, ci, v = M.build_stencils(x, n, C3["n"], "gfd", ell=C3["ell"], mu=h2, alpha=C3["alpha"],
                                           keep_weights=False)
        Hs.append(M.Hierarchy(x, rp, ci, v, C3["n_min"], precision="f32"))
    E[1].record()
    Us, infos = M.solve_batched(Hs, [F for _, _, F, _ in d], tol=C3["tol"], restart=30)
    E[2].record()
    single_iters = []
    for H, (x, n, F, h2) in zip(Hs, d):
        for r in range(F.shape[0]):
            u, inf = H.solve(F[r].contiguous(), tol=C3["tol"], restart=30)
            single_iters.append(inf["iters"])
    E[3].record()
    E[3].synchronize()
    flat = [i for inf in infos for i in inf]
    nrhs_total = len(flat)
    return {"problems": nprob, "points": int(sum(x.shape[0] for x, _, _, _ in probs)), "rhs_per_problem": C3["nrhs"],
            "discretisation": "GFD ell=2 n=25 alpha=4, (I - h^2 Lap) u = delta, tol 1e-8",
            "setup_ms": round(E[0].elapsed_time(E[1]), 1), "batched_solve_ms": round(E[1].elapsed_time(E[2]), 2),
            "one_rhs_at_a_time_ms": round(E[2].elapsed_time(E[3]), 2),
            "batching_speedup": round(E[2].elapsed_time(E[3]) / E[1].elapsed_time(E[2]), 2),
            "ms_per_rhs": round(E[1].elapsed_time(E[2]) / nrhs_total, 3),
            "iters_max": max(i["iters"] for i in flat), "iters_single_max": max(single_iters),
            "converged": all(i["converged"] for i in flat)}


C4 = dict(n=30, ell=2, k=1, n_min=250, tol=1e-10, Nlo=50000, Nhi=200000, passes=4, lr=2e-3, lr_final=2e-4)


def bench_learned(nsurf, Neval, dev):
    """Learned correction after the V-cycle: trained on the GPU on nsurf seeded bumpy spheres and
    tori (N log-uniform in [50k, 200k]; PHS r^3, degree 2, n = 30, -Lap + I), each surface's
    samples used as it is built; evaluated on a held-out bumpy torus of Neval points against the
    plain cycle (FGMRES to 1e-10)."""
    import torch
    from paper_2204_06154_gb300 import inputs as I
    from paper_2204_06154_gb300 import learned as LR
    from paper_2204_06154_gb300 import mgm as M
    rng = np.random.default_rng(404)
    net = M.MLP(C4["n"], seed=1)
    total = nsurf * 6 * C4["passes"]
    t0 = time.time()
    step = 0
    losses = []
    for sidx in range(nsurf):
        N = int(np.exp(rng.uniform(np.log(C4["Nlo"]), np.log(C4["Nhi"]))))
        x, nrm = (I.bumpy_sphere(N, seed=1000 + sidx) if sidx % 2 == 0 else I.bumpy_torus(N, seed=1000 + sidx))
        P = LR.Problem(x, nrm, n=C4["n"], k=C4["k"], ell=C4["ell"], n_min=C4["n_min"], device=dev)
        items = [(P, r) for r in P.samples(seed=2000 + sidx, smooth="poly")]
        for _ in range(C4["passes"]):
            for (Q, r) in items:
                lr = C4["lr"] * (C4["lr_final"] / C4["lr"]) ** (step / max(1, total - 1))
                losses.append(Q.H.learned_train_step(net, r, lr))
                step += 1
        del P, items
    torch.cuda.synchronize()
    train_s = time.time() - t0
    x, nrm = I.bumpy_torus(Neval, seed=77)
    P = LR.Problem(x, nrm, n=C4["n"], k=C4["k"], ell=C4["ell"], n_min=C4["n_min"], device=dev)
    f = torch.from_numpy(I.random_sh_rhs(x, lmax=20, seed=78)).to(dev)
    out = {}
    for name, use in (("plain", None), ("learned", net)):
        P.H.learned_enable(use)
        P.H.solve(f, tol=C4["tol"])  # warm-up (graph capture)
        u, info = P.H.solve(f, tol=C4["tol"])
        out[name] = {"iters": info["iters"], "solve_ms": round(info["solve_ms"], 2), "rel_res": info["rel_res"],
                     "converged": info["converged"]}
    pr = P.H.profile(reps=20)
    li = P.H.learned_info()
    P.H.learned_enable(None)
    return {"training": {"surfaces": nsurf, "points_range": [C4["Nlo"], C4["Nhi"]], "steps": step,
                         "seconds": round(train_s, 1), "J_first": round(float(np.mean(losses[:12])), 4),
                         "J_last": round(float(np.mean(losses[-48:])), 4)},
            "eval": {"surface": f"bumpy torus, {Neval} points, PHS r^3 + degree 2, n=30, -Lap+I, SH rhs l<=20",
                     **out, "speedup": round(out["plain"]["solve_ms"] / out["learned"]["solve_ms"], 3),
                     "fallbacks": li["fallbacks"]},
            "vcycle_ms": {"plain": round(pr["vcycle_ms"], 4), "with_correction": round(pr["learned_vcycle_ms"], 4)},
            "correction_kernel": {"ms": round(pr["learned_ms"], 4), "bytes": pr["learned_bytes"],
                                  "GB/s": round(pr["learned_bytes"] / pr["learned_ms"] / 1e6, 1) if pr["learned_ms"] else None}}


def bench_eigs(torch, H, nev):
    """Shift-invert eigenpairs (Sec. 6.1) of L = I - D on the sphere: the nev of smallest magnitude,
    each application of L^-1 a batched MGM-FGMRES solve to 1e-10. Eigenvalues of -D = lambda - 1
    against l(l+1)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    lam, _, info = H.eigs(nev=nev, block=8, steps=3, max_cycles=20, tol=1e-8, solve_tol=1e-10, vectors=False)
    e1.record()
    e1.synchronize()
    lap = sorted(float(z.real) - 1.0 for z in lam)
    exact = [l * (l + 1) for l in range(8) for _ in range(2 * l + 1)][:nev]
    return {"nev": nev, "ms": round(e0.elapsed_time(e1), 1), "solves": info["solves"], "converged": info["nconv"],
            "max_resid": max(info["resid"]), "eigenvalues_of_minus_D": [round(v, 5) for v in lap],
            "max_rel_dev_from_l(l+1)": round(max(abs(v - e) / max(e, 1) for v, e in zip(lap, exact)), 5)}


def bench_pattern(N, steps, warmup, host_steps=20):
    """Schnakenberg reaction-diffusion (Sec. 6.2's scheme class; gamma = 1, a = 0.1, b = 0.9) on a
    seeded bumpy sphere: IMEX Euler, dt = 0.01, D = (1, 10), FP32 cycles, FGMRES to 1e-8 from the
    previous step. Every step is one CUDA graph launch (fused right-hand sides, both solves driven on
    the device); the host-driven stepping is timed beside it on a few steps. Setup (stencils, two
    hierarchies) and the timed steps are reported apart."""
    import torch
    from paper_2204_06154_gb300 import inputs as I
    from paper_2204_06154_gb300.pattern import ReactionDiffusion
    x, nrm = I.bumpy_sphere(N, seed=3)
    X, NR = torch.from_numpy(x).cuda(), torch.from_numpy(nrm).cuda()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    e[0].record()
    rd = ReactionDiffusion(X, NR, "schnakenberg", (1.0, 0.1, 0.9), 1.0, 10.0, 0.01, scheme="euler", n=60, ell=3,
                           n_min=250, precision="f32")
    rd.hierarchy(0.01 * 1.0), rd.hierarchy(0.01 * 10.0)
    e[1].record()
    rng = np.random.default_rng(5)
    us, vs = 1.0, 0.9
    u0 = torch.from_numpy(us + 0.01 * rng.uniform(-1, 1, N)).cuda()
    v0 = torch.from_numpy(vs + 0.01 * rng.uniform(-1, 1, N)).cuda()
    u, v, _ = rd.run_graph(u0, v0, warmup, tol=1e-8)
    e[2].record()
    ug, vg, its = rd.run_graph(u, v, steps, tol=1e-8)
    e[3].record()
    # the same first steps from the same state: graph-driven and host-driven (the solves get
    # cheaper as the pattern settles, so only equal steps compare)
    _, _, its_g = rd.run_graph(u, v, host_steps, tol=1e-8)
    e[4].record()
    _, _, its_h = rd.run(u, v, host_steps, tol=1e-8)
    e[5].record()
    e[5].synchronize()
    u = ug
    ms = e[2].elapsed_time(e[3])
    ms_g = e[3].elapsed_time(e[4])
    ms_h = e[4].elapsed_time(e[5])
    iu = [a for a, _ in its]
    iv = [b for _, b in its]
    return {"N": N, "setup_ms": round(e[0].elapsed_time(e[1]), 1), "steps": steps,
            "ms_per_step": round(ms / steps, 3), "graph_launches_per_step": 1,
            "first_steps": {"steps": host_steps, "graph_ms_per_step": round(ms_g / host_steps, 3),
                            "host_driven_ms_per_step": round(ms_h / host_steps, 3),
                            "iters_graph": sum(a + b for a, b in its_g), "iters_host": sum(a + b for a, b in its_h)},
            "iters_u": {"max": max(iu), "mean": round(sum(iu) / len(iu), 2)},
            "iters_v": {"max": max(iv), "mean": round(sum(iv) / len(iv), 2)},
            "u_range": [round(float(u.min()), 4), round(float(u.max()), 4)]}


# Arm (implementer 0x41) part numbers of the cores this runs on, as /proc/cpuinfo reports them
ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
             "0xd49": "Arm Neoverse N2", "0xd8e": "Arm Neoverse N3", "0xd84": "Arm Neoverse V3"}


def cpu_info():
    """Host cores and CPU model (the oracle runs single-threaded)."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if ":" in line:
                    key, val = line.split(":", 1)
                    fields.setdefault(key.strip().lower(), val.strip())
    except OSError:
        pass
    model = fields.get("model name")
    if not model and "cpu part" in fields:
        part = fields["cpu part"].lower()
        model = ARM_PARTS.get(part, f"Arm CPU part {part}") + f" (implementer {fields.get('cpu implementer', '?')})"
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu": model}


def oracle_extrapolated(sizes, target):
    """The oracle's whole path timed at two sample sizes; the time at `target` points from the
    power law t = c N^p through the two measurements (p from their ratio)."""
    (n0, n1) = sizes
    t0, it0, _ = oracle_sample(n0)
    t1, it1, _ = oracle_sample(n1)
    p = math.log(t1 / t0) / math.log(n1 / n0)
    return t1 * (target / n1) ** p, {"sizes": [n0, n1], "ms": [round(t0, 1), round(t1, 1)], "exponent": round(p, 3),
                                      "iters": [it0, it1]}


def cpu_baseline(a):
    n1 = a.cpu_sample
    v, fit = oracle_extrapolated((n1 // 2, n1), a.size)
    ci = cpu_info()
    return {"value": round(v, 1), "unit": "ms", "cores": 1, "kind": "oracle", "extrapolated": True,
            "sample": f"whole path (brute-force kNN, FP64 weights, hierarchy, MGM-FGMRES to 1e-10) on jittered "
                      f"Fibonacci spheres of {n1 // 2:,} and {n1:,} points with the same parameters, "
                      f"{fit['ms'][0]:.0f} and {fit['ms'][1]:.0f} ms measured; extrapolated to {a.size:,} points "
                      f"by the power law through them (exponent {fit['exponent']})",
            "fit": fit, **ci}


def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def main():
    a = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if a.impl == "reference":
        if rank != 0:
            return
        n1 = a.cpu_sample // 2  # each step about 4 s of single-threaded oracle time
        vals, fits = [], []
        for i in range(a.warmup + a.steps):
            v, fit = oracle_extrapolated((n1 // 2, n1), a.size)
            if i >= a.warmup:
                vals.append(v)
                fits.append(fit)
        v = statistics.mean(vals)
        ci = cpu_info()
        cb = {"value": round(v, 1), "unit": "ms", "cores": 1, "kind": "oracle", "extrapolated": True,
              "sample": f"each step: the whole path on {n1 // 2:,}- and {n1:,}-point spheres, extrapolated to "
                        f"{a.size:,} points by the power law through the two times", "fits": fits, **ci}
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms",
                          "value_kind": "extrapolated from measured sample sizes",
                          "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(2 * v, 1),
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": config(a), "cpu_baseline": cb,
                          "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
              flush=True)
        return
    if a.vcycles > 0:
        import torch
        from paper_2204_06154_gb300 import mgm as M
        from paper_2204_06154_gb300 import inputs as I
        x, nrm = I.fibonacci_sphere(a.size, jitter=0.1, seed=2)
        X = torch.from_numpy(x).cuda(); Nr = torch.from_numpy(nrm).cuda()
        n, ell = (a.learned_n, 2) if a.learned_n else (50, 3)
        idx, w, rp, ci, v = M.build_stencils(X, Nr, n, "rbf", 1, ell, 1.0)
        r = torch.from_numpy(np.random.default_rng(5).standard_normal(a.size)).cuda()
        out = {"vcycles": a.vcycles, "N": a.size}
        for mode in [int(t) for t in a.sweeps.split(",")]:
            H = M.Hierarchy(X, rp, ci, v, 250, precision="f64" if a.fp64_cycle else "f32", persistent_sweeps=mode,
                            transfer_bf16=a.transfer_bf16)
            if a.learned_n:
                H.learned_attach(X, Nr, idx, w)
                H.learned_enable(M.MLP(a.learned_n, seed=1))
            for _ in range(a.vcycles):
                z = H.vcycle(r)
            torch.cuda.synchronize()
            pr = H.profile(reps=20)
            st = H.stats()
            sched = [H.sweep_config(j) for j in range(st["p"] - 1)]
            blocks0 = H.sweep_config(0)["blocks"] or 456
            chain = {pdl: M.probe_launch_chain(blocks0, 256, 256, pdl, 10) for pdl in (True, False)}
            fl = H.vcycle_floor(chain[True], float(peaks()[0].get("hbm_gbs", 6800.0)))
            lvl = []
            for j in range(st["p"] - 1):  # per-level smoothing: device time and algorithmic GB/s
                ms_j = H.profile_level(j, reps=20)
                lvl.append({"ms": round(ms_j, 4), "GB/s": round(H.level_smoothing_bytes(j) / ms_j / 1e6, 1)})
            out[f"mode{mode}"] = {"levels": st["n"], "ncolors": st["ncolors"], "max|z|": float(z.abs().max()),
                                  "level_smoothing": lvl,
                                  "chain_us": {"programmatic": round(chain[True], 3), "plain": round(chain[False], 3),
                                               "blocks": blocks0},
                                  "floor_ms": {k: round(v, 4) for k, v in fl.items()},
                                  "schedules": [(c["kind"][0], c["blocks"], c["lanes"], c["stages"], round(c["ms"], 4))
                                                for c in sched],
                                  "vcycle_ms": round(pr["vcycle_ms"], 4), "vcycle_kernels": pr["vcycle_kernels"],
                                  "vcycle_GB/s": round(pr["vcycle_bytes"] / pr["vcycle_ms"] / 1e6, 1),
                                  "sweep_ms": round(pr["sweep_ms"], 4),
                                  "sweep_GB/s": round(pr["sweep_bytes"] / pr["sweep_ms"] / 1e6, 1) if pr["sweep_ms"] else None,
                                  "spmv_ms": round(pr["spmv_ms"], 4),
                                  "spmv_GB/s": round(pr["spmv_bytes"] / pr["spmv_ms"] / 1e6, 1)}
            del H
        print(json.dumps(out), flush=True)
        return
    if a.single:
        import torch
        from paper_2204_06154_gb300 import mgm as M
        from paper_2204_06154_gb300 import inputs as I
        x, nrm = I.fibonacci_sphere(a.size, jitter=0.1, seed=2)
        f = I.random_sh_rhs(x, 20, 2)
        d = [torch.from_numpy(v).cuda() for v in (x, nrm, f)]
        r, H, u = run_problem(M, torch, *d)
        print(json.dumps({"single": True, "N": a.size, **{k: (round(v, 3) if isinstance(v, float) else v)
                                                         for k, v in r.items()}}), flush=True)
        return
    if a.workload == "c5":
        import torch
        torch.cuda.set_device(local_rank)
        r = bench_pattern(a.c5_size, a.c5_steps, max(a.warmup, 3))
        print(json.dumps({"metric": "pattern formation: ms per semi-implicit time step (two warm-started solves)",
                          "value": r["ms_per_step"], "unit": "ms", "n_gpus": 1, "steps": a.c5_steps,
                          "higher_is_better": False, "data": "synthetic",
                          "config": {"workload": f"Schnakenberg IMEX Euler on a {a.c5_size:,}-point bumpy sphere, PHS r^3 "
                                                 "+ degree 3, n = 60, dt = 0.01, D = (1, 10), tol 1e-8, warm start"},
                          "pattern": r}), flush=True)
        return
    if a.workload == "c3":
        import torch
        torch.cuda.set_device(local_rank)
        from paper_2204_06154_gb300 import mgm as M
        M.lib()
        b = bench_batched(64, torch.device("cuda", local_rank))
        print(json.dumps({"metric": "batched heat-step solves: ms per right-hand side", "value": b["ms_per_rhs"],
                          "unit": "ms", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
                          "config": {"workload": "64 bumpy spheres, N log-uniform 20k-400k, 8 delta RHS each"},
                          "batched": b}), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = bench_ours(a, rank, world, local_rank)
    if rank != 0:
        return
    recs = res["records"]
    K = a.steps
    per_problem = whole_job_ms_per_problem(res["ms_total"], K, res["nprob"], world)
    mean = lambda key, rs=recs: statistics.mean(r[key] for r in rs)
    solve_mixed = mean("solve_ms")
    solve_fp64 = mean("solve_ms", res["fp64"])
    pk, pk_kind = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    prof = res["profile"]
    st = res["stats"]
    # dominant kernel of the step: the stencil-weight solves, FP32 LU in registers with FP64
    # refinement (phs_weights_rl_k<60>), bound by the FP64 pipe. The unit is the FP64-pipe
    # operation (an add, a multiply or a fused multiply-add; a correctly rounded square root costs 8,
    # measured with ncu on a probe), the peak the pipe's rate = the measured FMA peak / 2 flops.
    # Algorithmic operations per stencil: tangent coordinates (26 a neighbour), the n(n+1)/2 PHS
    # entries (2 differences, 2 squares, a sum, a square root, a product: 14), the n L monomials
    # (1 each, built incrementally), the right-hand side (12 a neighbour), 3 residual evaluations of
    # m n + n L fused multiply-adds (3 is the typical count; convergence is tested after each) and
    # the m additions of each correction.
    m = P["n"] + (P["ell"] + 1) * (P["ell"] + 2) // 2
    L = m - P["n"]
    n_ = P["n"]
    ops_per_stencil = 26.0 * n_ + 14.0 * n_ * (n_ + 1) / 2 + n_ * L + 12.0 * n_ + 3 * ((m * n_ + n_ * L) + m)
    w_ms = mean("weights_ms")
    w_gops = a.size * ops_per_stencil / (w_ms * 1e-3) / 1e9
    fp64_pipe_peak = res["fp64_gflops"] / 2.0
    total_fp64 = mean("total_ms", res["fp64"])
    sweep_gbs = prof["sweep_bytes"] / (prof["sweep_ms"] * 1e-3) / 1e9 if prof["sweep_ms"] > 0 else None
    vcyc_gbs = prof["vcycle_bytes"] / (prof["vcycle_ms"] * 1e-3) / 1e9
    spmv_gbs = prof["spmv_bytes"] / (prof["spmv_ms"] * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": round(per_problem, 2), "unit": "ms", "n_gpus": world, "steps": K,
        "warmup": a.warmup, "ms_per_step": round(res["ms_total"] / K, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": config(a),
        "phases_ms": {k: round(mean(k), 3) for k in ("knn_ms", "weights_ms", "assemble_ms", "setup_ms", "solve_ms")},
        "rel_res_max": max(r["rel_res"] for r in recs + res["fp64"]),
        "converged": all(r["converged"] for r in recs + res["fp64"]),
        "roofline": {"kernel": "phs_weights_rl_k<60> (60 x 60 stencil systems: FP32 LU in registers, FP64 "
                               "entries and refinement residuals)", "bound": "alu",
                     "achieved": round(w_gops, 1), "peak": round(fp64_pipe_peak, 1), "unit": "G FP64-pipe op/s",
                     "frac": round(w_gops / fp64_pipe_peak, 3),
                     "traffic": int(RL_DRAM_BYTES_PER_STENCIL * a.size) if RL_DRAM_BYTES_PER_STENCIL else None,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the current kernel on "
                                       "524,288 stencils, scaled by stencils to the launch's count",
                     "fp64_ops_per_stencil": ops_per_stencil,
                     # counted by ncu on the current kernel (one launch, 131,072 stencils): FP64-pipe warp
                     # instructions and FP64 thread operations a stencil, beside the algorithmic count
                     "fp64_per_stencil_ncu": {"warp_instructions": round(187826176 / 131072),
                                              "thread_ops": round(5030019072 / 131072),
                                              "metrics": "sm__inst_executed_pipe_fp64.sum, "
                                                         "sm__sass_thread_inst_executed_op_fp64_pred_on.sum"},
                     "peak_source": f"mgm_probe_fp64_fma during this run: {res['fp64_gflops']:.0f} GFLOP/s of FP64 "
                                    f"multiply-adds (2 flops each) = {fp64_pipe_peak:.1f} G FP64-pipe op/s "
                                    "(MEASURED_PEAKS.json has no FP64 figure)"},
        "vcycle_roofline": {"kernel": "gs_colour_k<1,float,2> (finest-level multicolour GS sweep, staged per colour)",
                            "bound": "hbm",
                            "achieved": round(sweep_gbs, 1) if sweep_gbs else None, "peak": hbm, "unit": "GB/s",
                            "frac": round(sweep_gbs / hbm, 3) if sweep_gbs else None, "traffic": None,
                            "bytes_per_sweep": prof["sweep_bytes"], "sweep_us": round(1e3 * prof["sweep_ms"], 2),
                            "launches_per_sweep": prof["sweep_launches"],
                            "whole_vcycle": {"ms": round(prof["vcycle_ms"], 4), "GB/s": round(vcyc_gbs, 1),
                                             "frac": round(vcyc_gbs / hbm, 3), "kernels": prof["vcycle_kernels"]},
                            "floor": {"ms": round(res["floor"]["floor_ms"], 4),
                                      "bytes_ms": round(res["floor"]["bytes_ms"], 4),
                                      "chain_ms": round(res["floor"]["chain_ms"], 4),
                                      "chain_us_per_launch": round(res["chain_us"], 3),
                                      "chain_probe": f"mgm_probe_launch_chain: 256 dependent launches of "
                                                     f"{res['chain_blocks']} x 256 threads, programmatic",
                                      "vcycle_frac_of_floor": round(res["floor"]["floor_ms"] / prof["vcycle_ms"], 3)},
                            "outer_spmv_fp64": {"ms": round(prof["spmv_ms"], 4), "GB/s": round(spmv_gbs, 1),
                                                "frac": round(spmv_gbs / hbm, 3)},
                            "peak_source": pk_kind},
        "hierarchy": {"n": st["n"], "nnz": st["nnz"], "ncolors": st["ncolors"], "device_MB": st["device_bytes"] >> 20},
        "e2e": {"value": round(res["e2e_ms"], 2), "unit": "ms", "h2d_bytes_per_step": res["e2e_h2d"],
                "d2h_bytes_per_step": res["e2e_d2h"]},
        "gpu_launches": res["launches"],
        "batched": res.get("batched"),
        "learned": res.get("learned"),
        "eigs": res.get("eigs"),
        "pattern": res.get("pattern"),
        "clocks": res["clocks"],
    }
    if not a.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(a)
    # the headline comparison last, where a reader of the line's tail finds it: mixed-precision MGM
    # (FP32 LU + FP64 refinement weights, FP32 V-cycle, FP64 FGMRES) against the FP64 GPU MGM on the
    # same problems
    out["solve_ms"] = {"mixed_f32_vcycle": round(solve_mixed, 3), "fp64_vcycle": round(solve_fp64, 3),
                       "speedup": round(solve_fp64 / solve_mixed, 3)}
    out["whole_path_ms"] = {"mixed": round(mean("total_ms"), 2), "fp64": round(total_fp64, 2),
                            "fp64_weights_ms": round(mean("weights_ms", res["fp64"]), 2),
                            "speedup": round(total_fp64 / mean("total_ms"), 3)}
    out["iters"] = {"mixed": [r["iters"] for r in recs[: res["nprob"]]], "fp64": [r["iters"] for r in res["fp64"]]}
    print(json.dumps(out), flush=True)


def config(a):
    return {"workload": f"sphere + torus, {a.size:,} points each, PHS r^3 + degree-3, n=50, -Lap+I, "
                        f"random SH rhs l<=20, MGM V(1,1) MC-GS, FGMRES to 1e-10",
            "problems_per_step": 2, "N": a.size, "n": P["n"], "ell": P["ell"], "n_min": P["n_min"],
            "precision": "FP32 LU + FP64 refinement for the stencil weights, FP32 V-cycle / FP64 outer, "
                         "FP64 hierarchy setup", "l2": "inputs > L2 (no flush needed)"}


if __name__ == "__main__":
    main()

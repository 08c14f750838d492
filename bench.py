#!/usr/bin/env python
"""Benchmark of the space-time ROM hot path on one GB300.

One step = one pass of the whole path on the batched online workload (the
2-D S4 transport model of 64x64 cells, 12 directions, N = 49,152, Nt = 200,
with a (40, 12) basis):
  1. FOM snapshot march of the 16 training parameters (BiCGSTAB, FP64);
  2. block-incremental POD -> Phi_s (N x 40), per-mode temporal bases;
  3. assembly of the space-time reduced operators;
  4. batched reduced solve of 4096 parameters with uneven (ns, nt) drawn from
     {(10,4), (20,8), (30,10), (40,12)} (FP64 LU + refinement);
  5. reconstruction: the output R(t) (total particle population) for all 4096
     and full space-time fields for 4 of them.
value = reduced solves per second of the whole step (inputs resident on the
device); e2e = the same through the C ABI with host buffers (H2D of the
step's inputs and D2H of its results inside the timed region).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores and extrapolates to the full step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reduced space-time solves/s at ≤1e-3 rel err vs FOM; build HBM GB/s & TC util"
WORKLOAD = "c4: 2-D S4 transport 64x64 (N=49152), Nt=200, 16 training mu, basis (40,12), 4096 online mu with uneven (ns,nt)"
N_BATCH = 4096
N_FIELDS = 4
# FP64 peak derived from the GB300 unit counts and clock: 152 SMs x 2 DFMA/clk
# x 2 flop x 2.07 GHz (the nominal 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------

def cpu_sample(prob, theta_train, mu_b, sizes, budget_steps: int = 40, n_solve: int = 64,
               n_out: int = 16) -> dict:
    """Time the FP64 oracle on a bounded sample and extrapolate to one full
    step.  Returns dict(seconds_full, seconds_sample, sample)."""
    from oracle import fom, pod, strom
    t_all = time.perf_counter()
    N, Nt = prob.N, prob.Nt
    n_train = theta_train.shape[0]
    # 1. FOM: one training parameter, budget_steps steps (sparse LU per step)
    A = fom.affine_operator(prob.rowptr, prob.col, prob.vals, theta_train[0])
    t0 = time.perf_counter()
    fom.fom_march(A, prob.dt[:budget_steps], prob.B, prob.F[:budget_steps], None)
    t_fom = (time.perf_counter() - t0) * (Nt / budget_steps) * n_train
    # 2. POD: one incremental update at steady-state rank on seeded blocks
    rng = np.random.default_rng(0)
    b1 = rng.standard_normal((N, Nt))
    b2 = rng.standard_normal((N, Nt))
    W, s, V = pod.incremental_update(None, None, None, b1, 256, 1e-12, 1e-14)
    t0 = time.perf_counter()
    pod.incremental_update(W, s, V, b2, 256, 1e-12, 1e-14)
    t_pod = (time.perf_counter() - t0) * n_train
    # 3. assembly with a seeded orthonormal basis of the full size
    ns, nt = prob.ns, prob.nt
    Phi = np.linalg.qr(rng.standard_normal((N, ns)))[0]
    T = np.zeros((Nt, ns * nt))
    for i in range(ns):
        Ti = np.linalg.qr(rng.standard_normal((Nt, nt)))[0]
        T[:, i::ns] = Ti
    t0 = time.perf_counter()
    rm = strom.ReducedModel(prob, Phi, T, ns, nt)
    t_asm = time.perf_counter() - t0
    # 4. solves: n_solve parameters of the batch
    t0 = time.perf_counter()
    sol = []
    for k in range(n_solve):
        a, b = sizes[k]
        sol.append(rm.solve(prob.theta(mu_b[k]), int(a), int(b)))
    t_solve = (time.perf_counter() - t0) * (len(mu_b) / n_solve)
    # 5. outputs: reconstruct and integrate for n_out parameters
    Cout = (np.repeat(prob.w, prob.n_cells) / prob.n_cells)[:, None]
    t0 = time.perf_counter()
    for k in range(n_out):
        a, b = sizes[k]
        U = rm.reconstruct(sol[k], int(a), int(b))
        _ = Cout.T @ U
    t_out = (time.perf_counter() - t0) * (len(mu_b) / n_out)
    total = t_fom + t_pod + t_asm + t_solve + t_out
    return {"seconds_full": total, "seconds_sample": time.perf_counter() - t_all,
            "phases_s": {"fom": t_fom, "pod": t_pod, "assemble": t_asm, "solve": t_solve,
                         "outputs": t_out},
            "sample": (f"FOM 1 of {n_train} mu x {budget_steps} of {Nt} steps (sparse LU); "
                       f"1 incremental-SVD update at rank 256 x {n_train}; full assembly; "
                       f"{n_solve} of {len(mu_b)} LAPACK solves; {n_out} output evaluations; "
                       "extrapolated linearly to one full step")}


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    from workloads import c4_batch, problem_for
    prob = problem_for("c4")
    mu_b, sizes = c4_batch(N_BATCH, prob)
    theta_train = prob.theta(prob.train_mu)
    vals = []
    samp = None
    for it in range(args.warmup + args.steps):
        r = cpu_sample(prob, theta_train, mu_b, sizes)
        if it >= args.warmup:
            vals.append(N_BATCH / r["seconds_full"])
            samp = r
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * N_BATCH / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": N_BATCH, "seq_len": prob.Nt,
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": samp["sample"],
                             "phases_s": samp["phases_s"]},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args, rank: int, world: int, dist) -> None:
    import torch

    import paper_1910_01260_gb300 as st
    from workloads import c4_batch, problem_for

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    prob = problem_for("c4")
    N, Nt, ns, nt = prob.N, prob.Nt, prob.ns, prob.nt
    n_full = ns * nt
    mu_b, sizes = c4_batch(N_BATCH, prob, seed=4 + rank)
    theta_train = prob.theta(prob.train_mu)
    theta_b = prob.theta(mu_b)
    n_train = theta_train.shape[0]
    m = st.Model(prob.rowptr, prob.col, prob.vals, st.options(r_max=args.r_max), stream=stream.cuda_stream)
    # device-resident inputs and outputs
    B = torch.tensor(prob.B.T.copy(), device=dev)
    Cout = torch.tensor((np.repeat(prob.w, prob.n_cells) / prob.n_cells)[None, :], device=dev)
    snaps = torch.empty((n_train, Nt, N), dtype=torch.float64, device=dev)
    f_iters = torch.zeros((Nt, n_train), dtype=torch.int32, device=dev)
    f_status = torch.zeros(n_train, dtype=torch.int32, device=dev)
    th_d = torch.tensor(theta_b, device=dev)
    sz_d = torch.tensor(sizes, device=dev)
    uhat = torch.zeros((N_BATCH, n_full), dtype=torch.float64, device=dev)
    res = torch.zeros(N_BATCH, dtype=torch.float64, device=dev)
    s_status = torch.zeros(N_BATCH, dtype=torch.int32, device=dev)
    y = torch.zeros((N_BATCH, Nt, 1), dtype=torch.float64, device=dev)
    u_sel = torch.zeros((N_FIELDS, Nt, N), dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]

    def step(record: bool):
        if record:
            ev[0].record(stream)
        m.st_fom_march(theta_train, prob.dt, None, B, prob.F, snaps, f_iters, f_status)
        if record:
            ev[1].record(stream)
        m.st_rom_build_basis(n_train, Nt, snaps, ns, nt)
        if record:
            ev[2].record(stream)
        m.st_rom_assemble(prob.dt, B, prob.F, None)
        if record:
            ev[3].record(stream)
        m.st_rom_solve(N_BATCH, th_d, sz_d, uhat, res, s_status)
        if record:
            ev[4].record(stream)
        m.st_rom_reconstruct(N_BATCH, uhat, sz_d, None, 1, Cout, y)
        m.st_rom_reconstruct(N_FIELDS, uhat, sz_d, u_sel)
        if record:
            ev[5].record(stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False)
    m.st_sync()
    barrier()
    phase_ms = {k: [] for k in ("fom", "pod", "assemble", "solve", "reconstruct")}
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = st.lib.st_kernel_launches()
    barrier()
    t_start.record(stream)
    for _ in range(args.steps):
        step(True)
        torch.cuda.synchronize()
        for i, k in enumerate(phase_ms):
            phase_ms[k].append(ev[i].elapsed_time(ev[i + 1]))
    t_end.record(stream)
    barrier()
    launches = st.lib.st_kernel_launches() - launches0
    clk = clocks.stop()
    m.st_sync()
    elapsed_ms = t_start.elapsed_time(t_end)
    if dist is not None:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_step = elapsed_ms / args.steps
    value = world * N_BATCH / (ms_step / 1e3)
    phases = {k: float(np.mean(v)) for k, v in phase_ms.items()}
    iters = f_iters.cpu().numpy()
    stat_ok = int((s_status == 0).sum().item())

    # ---- end-to-end: host buffers through the C ABI ----------------------
    pin = lambda a: torch.tensor(a).pin_memory()
    h_theta_b, h_sizes, h_B = pin(theta_b), pin(sizes), pin(prob.B.T.copy())
    h_uhat = torch.empty_like(uhat, device="cpu").pin_memory()
    h_res = torch.empty_like(res, device="cpu").pin_memory()
    h_y = torch.empty_like(y, device="cpu").pin_memory()
    h2d = (theta_train.nbytes + prob.dt.nbytes + prob.F.nbytes + h_theta_b.numel() * 8 +
           h_sizes.numel() * 4 + h_B.numel() * 8)
    d2h = h_uhat.numel() * 8 + h_res.numel() * 8 + h_y.numel() * 8

    def e2e_step():
        th_d.copy_(h_theta_b, non_blocking=True)
        sz_d.copy_(h_sizes, non_blocking=True)
        B.copy_(h_B, non_blocking=True)
        step(False)
        h_uhat.copy_(uhat, non_blocking=True)
        h_res.copy_(res, non_blocking=True)
        h_y.copy_(y, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if dist is not None:
        t = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = world * N_BATCH / (e2e_ms / 1e3)

    # ---- online phase alone, per precision mode (same model and batch) ---
    online = {}
    ref_uhat = uhat.clone()
    for name, prec, refine in (("fp64_lu", st.ST_FP64, 1), ("fp32_lu_fp64_refine3", st.ST_FP32_LU, 3)):
        m.st_model_set_options(precision=prec, refine_steps=refine)
        m.st_rom_solve(N_BATCH, th_d, sz_d, uhat, res, s_status)
        torch.cuda.synchronize()
        o0 = torch.cuda.Event(enable_timing=True)
        o1 = torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for _ in range(args.steps):
            m.st_rom_solve(N_BATCH, th_d, sz_d, uhat, res, s_status)
            m.st_rom_reconstruct(N_BATCH, uhat, sz_d, None, 1, Cout, y)
        o1.record(stream)
        torch.cuda.synchronize()
        ms = o0.elapsed_time(o1) / args.steps
        diff = float(((uhat - ref_uhat).abs().max(dim=1).values /
                      ref_uhat.abs().max(dim=1).values.clamp_min(1e-300)).max())
        online[name] = {"ms": ms, "solves_per_s": N_BATCH / (ms / 1e3),
                        "max_rel_res": float(res.max()), "status_ok": int((s_status == 0).sum()),
                        "max_rel_diff_vs_fp64": diff}
    m.st_model_set_options(precision=st.ST_FP64, refine_steps=1)
    uhat.copy_(ref_uhat)
    m.st_sync()

    # ---- accuracy of the ROM against the FOM on sampled batch parameters -
    acc = {}
    sel = []
    for a, b in sorted({tuple(x) for x in sizes.tolist()}):
        idx = np.where((sizes[:, 0] == a) & (sizes[:, 1] == b))[0][:2]
        sel.extend(idx.tolist())
    sel = np.array(sel)
    fsn = torch.empty((len(sel), Nt, N), dtype=torch.float64, device=dev)
    m.st_fom_march(theta_b[sel], prob.dt, None, B, prob.F, fsn)
    ur = torch.zeros((len(sel), Nt, N), dtype=torch.float64, device=dev)
    m.st_rom_reconstruct(len(sel), uhat[sel].contiguous(), sz_d[sel].contiguous(), ur)
    m.st_sync()
    for j, k in enumerate(sel):
        err = float(torch.linalg.norm(fsn[j] - ur[j]) / torch.linalg.norm(fsn[j]))
        key = f"({sizes[k][0]},{sizes[k][1]})"
        acc[key] = max(acc.get(key, 0.0), err)

    # ---- roofline of the dominant kernel ---------------------------------
    nnz = prob.nnz
    mu_iters = int(iters.sum())
    fom_flops = mu_iters * (4.0 * nnz + 26.0 * N) + Nt * n_train * (2.0 * nnz + 8.0 * N)
    n = sizes[:, 0].astype(np.float64) * sizes[:, 1]
    refine = 1
    solve_flops = float(np.sum((2.0 / 3.0) * n ** 3 + (refine + 1) * 4.0 * n ** 2 + refine * 2.0 * n ** 2 + 4 * n ** 2))
    kern = {
        "fom_march_kernel": {"ms": phases["fom"], "flops": fom_flops},
        "solve_kernel": {"ms": phases["solve"], "flops": solve_flops},
    }
    for k in kern.values():
        k["achieved_tflops"] = k["flops"] / (k["ms"] * 1e-3) / 1e12
        k["frac"] = k["achieved_tflops"] / FP64_PEAK_TFLOPS
    dom = max(kern, key=lambda k: kern[k]["ms"])
    roof = {"bound": "alu", "kernel": dom, "achieved": kern[dom]["achieved_tflops"],
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": kern[dom]["frac"],
            "traffic": None, "peak_source": "FP64 derived: 152 SMs x 4 flop/clk x 2.07 GHz"}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu:
            r = cpu_sample(prob, theta_train, mu_b, sizes)
            cpu = {"value": N_BATCH / r["seconds_full"], "unit": "solves/s", "cores": os.cpu_count(),
                   "kind": "oracle", "sample": r["sample"], "phases_s": r["phases_s"]}
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "global_batch": world * N_BATCH, "seq_len": Nt,
                           "parallelism": f"replicas{world}", "r_max": args.r_max,
                           "l2": "inputs larger than L2 (1.26 GB of snapshots written per step)"},
                "phases_ms": phases,
                "online_solves_per_s": N_BATCH / ((phases["solve"] + phases["reconstruct"]) / 1e3),
                "online_modes": online,
                "fom_mu_per_s": n_train / (phases["fom"] / 1e3),
                "fom_bicgstab_iters_mean": float(iters.mean()),
                "solve_status_ok": stat_ok,
                "rom_rel_err_vs_fom": acc,
                "kernels": kern,
                "roofline": roof,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(launches),
                "clocks": clk}
        print(json.dumps(line), flush=True)
    m.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--r-max", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group(backend)
        dist = tdist
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

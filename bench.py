#!/usr/bin/env python
"""Benchmark of the hot path on the dense random-Lindbladian workload.

One bench step = one pass of the whole path over one realization, inputs
resident in HBM:
  kernel (a) enumeration of the nonzero f and d (canonical lists),
  expansion of H and rho0 (Eq. (02)),
  dense assembly of Q, R, K into A = Q + R (Eqs. (07)-(09)),
  FP32 packing of A,
  RK4 steps in FP64, and RK4 steps on FP32 storage with the FP64 defect
  correction every 50 steps.
Metric: R entries assembled per second (M^2 per assembly, from CUDA events
around the assembly on the launching stream), with RK4 steps/s reported
beside it.  `e2e` repeats the metric through the host-buffer C ABI
(lb_assemble + lb_integrate) with the Kossakowski matrix copied from pinned
host memory every step.  `--impl reference` times the CPU oracle instead.

Multi-GPU: independent replicas (one realization per rank, no data-path
collective), launched by torchrun; value = all ranks' entries / max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=200, help="Hilbert-space dimension N")
    p.add_argument("--rk4-steps", type=int, default=10, help="FP64 RK4 steps per bench step")
    p.add_argument("--rk4-fp32-steps", type=int, default=50,
                   help="FP32-storage RK4 steps per bench step (one FP64 correction window of 50 steps)")
    p.add_argument("--dt", type=float, default=1e-3)
    p.add_argument("--seed", type=int, default=20250)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-rows", type=int, default=2, help="rows of R in the CPU-oracle sample")
    p.add_argument("--count-terms", action="store_true", help="count the join terms W (extra pass)")
    p.add_argument("--algorithm", default="closed", choices=["closed", "join"],
                   help="dense R assembly: closed-form sums of the join (default) or every join term")
    p.add_argument("--no-forms", action="store_true", help="skip the batched / serving / sparse / small-N lines")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-sparse", action="store_true")
    p.add_argument("--no-small", action="store_true")
    p.add_argument("--batch-count", type=int, default=512)
    p.add_argument("--batch-steps", type=int, default=2000)
    p.add_argument("--batch-fp64-sample", type=int, default=32)
    p.add_argument("--serve-count", type=int, default=100)
    p.add_argument("--serve-steps", type=int, default=500)
    p.add_argument("--serve-load", type=float, default=0.75)
    p.add_argument("--serve-burst", type=int, default=20)
    p.add_argument("--serve-budget-gb", type=float, default=96.0)
    p.add_argument("--sparse-n", type=int, default=2000)
    p.add_argument("--sparse-steps", type=int, default=200)
    p.add_argument("--dimer-n", type=int, default=400)
    p.add_argument("--dimer-steps", type=int, default=20000)
    p.add_argument("--spectrum-n", type=int, default=50)
    p.add_argument("--spectrum-out", default=None, help="write the eigenvalues and the density grid (.npz)")
    p.add_argument("--only", default=None, choices=["dense_small", "sparse", "dimer", "batched", "serving",
                                                   "spectrum"],
                   help="run one of the other workloads alone and print its JSON (profiling aid)")
    return p.parse_args()


# ---------------------------------------------------------------- helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_max(values, dist, device):
    """Per-rank timings -> their maximum over ranks (the slowest replica sets
    the time of the job); unchanged without a process group."""
    import torch
    t = torch.tensor([float(x) for x in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_value(world, units_per_rank, seconds):
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the max-over-ranks time."""
    return world * units_per_rank / seconds


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- GPU arm

def run_gb300(args):
    import numpy as np
    import torch

    import paper_1912_01491_gb300 as lb
    from paper_1912_01491_gb300 import native
    import workloads as wl

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    N = args.n
    M = N * N - 1
    dt, nrk, nrk32 = args.dt, args.rk4_steps, args.rk4_fp32_steps
    dev = torch.device("cuda", local)

    # ---- inputs, resident in HBM before timing (one realization per rank)
    seed = args.seed + 7919 * rank
    a = wl.wishart_kossakowski_device(N, seed, device=dev)
    H_host = wl.gue_hamiltonian(N, seed + 1)
    H = torch.tensor(H_host, device=dev)
    rho0 = torch.tensor(wl.pure_state(N, 0), device=dev)
    B = lb.Basis(N)
    nf, nd = B.structure_count("f"), B.structure_count("d")
    # join-term count of Eq. (09) (a separate counting pass, outside the timed region)
    W = B.join_terms() if (args.count_terms or args.algorithm == "join") else None
    fidx = torch.empty((nf, 3), dtype=torch.int32, device=dev)
    fval = torch.empty(nf, dtype=torch.float64, device=dev)
    didx = torch.empty((nd, 3), dtype=torch.int32, device=dev)
    dval = torch.empty(nd, dtype=torch.float64, device=dev)
    A = torch.empty((M, M), dtype=torch.float64, device=dev)
    K = torch.empty(M, dtype=torch.float64, device=dev)
    A32 = torch.empty((M, M), dtype=torch.float32, device=dev)
    work = lb.rk4_workspace(M, dev)
    v64 = torch.empty(M, dtype=torch.float64, device=dev)
    v32 = torch.empty(M, dtype=torch.float64, device=dev)
    fp64_peak = native.probe_fp64_tflops()
    L = native.load()
    import ctypes
    got = ctypes.c_int64()
    stream = torch.cuda.current_stream()

    def step(ev):
        st = stream.cuda_stream
        # a1: kernel (a)
        native._check(L.lb_structure_export(B.handle, native.LB_F, fidx.data_ptr(), fval.data_ptr(), nf,
                                            ctypes.byref(got), st))
        native._check(L.lb_structure_export(B.handle, native.LB_D, didx.data_ptr(), dval.data_ptr(), nd,
                                            ctypes.byref(got), st))
        # a2: expansions
        h = B.expand(H).real.contiguous()
        hh[0] = h
        v0 = B.expand(rho0).real.contiguous()
        # a3-a5: assembly (per-kernel device times from CUDA events on this stream)
        ev[0].record(stream)
        kms.append(B.assemble_dense_timed(a, h=h, A=A, K=K, algorithm=args.algorithm))
        ev[1].record(stream)
        # a6: packing
        lb.pack_fp32(A, out=A32)
        # a7: RK4 FP64
        v64.copy_(v0)
        ev[2].record(stream)
        lb.rk4_dense(A, K, v64, dt, nrk, precision="fp64", work=work)
        ev[3].record(stream)
        # a8: RK4 on FP32 storage with FP64 defect correction every 50 steps
        v32.copy_(v0)
        lb.rk4_dense(A32, K, v32, dt, nrk32, precision="fp32", A64=A, correct_every=50, work=work)
        ev[4].record(stream)

    hh = [None]

    def new_events():
        return [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    kms = []
    for _ in range(args.warmup):
        step(new_events())
    kms.clear()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = native.launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    evs = [new_events() for _ in range(args.steps)]
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_stop.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = native.launch_count() - launches0
    clk = clocks.stop()
    h_last = hh[0]

    total_ms = t_start.elapsed_time(t_stop)
    asm_ms = sum(sum(d.values()) for d in kms)
    kern = {k: sum(d[k] for d in kms) / len(kms) for k in kms[0]}
    top = max(kern, key=kern.get)
    rk_ms = sum(e[2].elapsed_time(e[3]) for e in evs)
    rk32_ms = sum(e[3].elapsed_time(e[4]) for e in evs)
    total_ms, asm_ms, rk_ms, rk32_ms = replica_max([total_ms, asm_ms, rk_ms, rk32_ms], dist, dev)
    K_ = args.steps
    value = replica_value(world, K_ * M * M, asm_ms * 1e-3)
    t_asm = asm_ms / K_ * 1e-3
    alg_bytes = 16.0 * M * M + 8.0 * M * M + 16.0 * M
    # the other algorithm, timed outside the timed region for comparison
    other = "join" if args.algorithm == "closed" else "closed"
    other_ms = []
    for _ in range(2):
        other_ms.append(sum(B.assemble_dense_timed(a, h=h_last, A=A, K=K, algorithm=other).values()))
    B.assemble_dense_timed(a, h=h_last, A=A, K=K, algorithm=args.algorithm)
    roof = assembly_roofline(args.algorithm, top, kern[top], N, M, W, fp64_peak, measured_peaks())
    # a bounded attempt at N = 200: GMRES without a preconditioner needs
    # thousands of iterations of 2.5 ms there (the residual is reported)
    checks = fp64_checks(lb, B, A, K, [("rk4_fp64", v64), ("rk4_fp32_corrected", v32)], restart=300, max_iter=600,
                         H=H, plain_max_iter=600)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, lb, B, a, H_host, M, nrk, dt, dev, dist, world)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, a, M, N)
    forms = {}
    if not args.no_forms:
        del A, A32, work
        torch.cuda.empty_cache()
        forms = run_forms(args, dev, a200=a if N == 200 else None)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None
    peaks = measured_peaks()
    fp32_bytes = (4.0 * 4.0 * M * M * nrk32 + 12.0 * M * M * -(-nrk32 // 50)) * K_
    out = {
        "metric": "R entries assembled/s (dense random Lindbladian, N=%d)" % N,
        "value": value,
        "unit": "entries/s",
        "n_gpus": world,
        "steps": K_,
        "warmup": args.warmup,
        "ms_per_step": total_ms / K_,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": ("dense random Lindbladian N=%d (M=%d): GUE H, Wishart a=GG^dag/Tr; per step kernel (a) "
                         "f/d enumeration, expansion, Q/R/K assembly, FP32 pack, %d RK4 steps FP64 + %d RK4 "
                         "steps FP32 storage with FP64 correction (k=50), dt=%g" % (N, M, nrk, nrk32, dt)),
            "N": N, "M": M, "join_terms": W,
            "l2": "inputs larger than L2 (a is %.1f GB)" % (16.0 * M * M / 1e9),
            "parallelism": "replicas" if world > 1 else "single",
        },
        "rk4_steps_per_s": replica_value(world, K_ * nrk, rk_ms * 1e-3),
        "rk4_fp32_corrected_steps_per_s": replica_value(world, K_ * nrk32, rk32_ms * 1e-3),
        "assembly_algorithm": args.algorithm,
        "assembly_ms": asm_ms / K_,
        "assembly_kernel_ms": kern,
        "assembly_%s_entries_per_s" % other: world * M * M / (statistics.mean(other_ms) * 1e-3),
        "assembly_gbs_algorithmic": alg_bytes / t_asm / 1e9,
        "roofline": roof,
        "rk4_roofline": {
            "kernel": "k_stage<FP64> (fused GEMV + stage update)",
            "bound": "alu",
            "achieved": 2.0 * M * M * 4 * nrk * K_ / (rk_ms * 1e-3) / 1e12,
            "peak": fp64_peak,
            "unit": "TFLOP/s",
            "frac": 2.0 * M * M * 4 * nrk * K_ / (rk_ms * 1e-3) / 1e12 / fp64_peak,
            "achieved_gbs": 8.0 * M * M * 4 * nrk * K_ / (rk_ms * 1e-3) / 1e9,
        },
        "rk4_fp32_roofline": {
            "kernel": "k_stage<FP32> (fused GEMV + stage update, 16-byte loads) + k_correction<FP32>",
            "bound": "hbm",
            # per RK4 step 4 reads of A32; one FP64 correction (A64 + A32) per 50 steps, and the
            # run of nrk32 steps starts with one
            "achieved": fp32_bytes / (rk32_ms * 1e-3) / 1e9,
            "peak": peaks.get("hbm_gbs"),
            "unit": "GB/s",
            "frac": (fp32_bytes / (rk32_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None,
        },
        "gpu_launches": launches,
        "clocks": clk,
        "fp64_checks": checks,
    }
    if e2e:
        out["e2e"] = e2e
    if cpu:
        out["cpu_baseline"] = cpu
    out.update(forms)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return out


# DRAM bytes (read + write) per launch of a kernel from one ncu capture on a
# smaller case, with the units that capture processed; scaled to a launch of
# the bench size by units.  Kept only for the kernel version the capture saw.
NCU_TRAFFIC = {
    "k_entries (pair x pair; closed: disjoint edges by vertex quadruple)": {
        "N": 100, "bytes": 1.018646016e9 + 0.791549952e9,
        "units": lambda N: N * (N - 1.0) * (N - 2.0) * (N - 3.0),
        "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_disjoint4 launch at N=100 "
                  "(a is 1.6 GB, larger than L2)"},
}


def ncu_traffic(kernel, N):
    t = NCU_TRAFFIC.get(kernel)
    if t is None:
        return None, None
    return t["bytes"] * t["units"](N) / t["units"](t["N"]), t["source"]


def assembly_roofline(algorithm, top, top_ms, N, M, W, fp64_peak, peaks):
    """Roofline of the dominant assembly kernel (algorithmic work per launch
    over its event-timed launch duration)."""
    P2 = N * (N - 1)
    t = top_ms * 1e-3
    hbm = peaks.get("hbm_gbs")
    if top.startswith("k_entries") and algorithm == "closed":
        # the disjoint pair x pair block: one orientation of the Hermitian a-block
        # (8 B per entry) read once, A written once (8 B per entry)
        byts = 16.0 * 24.0 * N * (N - 1.0) * (N - 2.0) * (N - 3.0) / 24.0
        traffic, src = ncu_traffic(top, N)
        return {"kernel": top, "bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": byts / t / 1e9 / hbm if hbm else None, "traffic": traffic,
                "traffic_source": src and ("%s, scaled by the number of vertex quadruples" % src),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "algorithmic_bytes_per_launch": byts}
    if top.startswith("k_entries"):
        # the pair x pair join terms of Eq. (09), one multiply-add each
        flops = 2.0 * W * (P2 * P2) / (M * M)
        return {"kernel": top, "bound": "alu", "achieved": flops / t / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": flops / t / 1e12 / fp64_peak, "traffic": None,
                "peak_source": "FP64 FMA probe lb_probe_fp64 (of measured)",
                "algorithmic_flops_per_launch": flops}
    byts = 16.0 * M * M + 8.0 * M * M
    return {"kernel": top, "bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": byts / t / 1e9 / hbm if hbm else None, "traffic": None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)", "algorithmic_bytes_per_launch": byts}


def fp64_checks(lb, B, A, K, states, restart=0, max_iter=3000, H=None, plain_max_iter=None):
    """Outside the timed region: the FP64 steady state of the assembled
    system (restarted GMRES on the device, preconditioned from the eigenbasis
    of H when H is given; true relative residual) and the device checks of
    rho (Tr rho - 1, Hermiticity, smallest pivot of the Cholesky
    factorisation of rho + 1e-10) for the given states and the steady state.
    With plain_max_iter, the unpreconditioned GMRES runs too, for comparison."""
    import torch
    ev = _events(2)
    first_ms = None
    if H is not None:  # the first use in a process also loads the solver library's eigensolver
        ev[0].record()
        lb.steady_state(A, K, tol=1e-12, max_iter=max_iter, restart=restart, basis=B, H=H)
        ev[1].record()
        torch.cuda.synchronize()
        first_ms = ev[0].elapsed_time(ev[1])
    ev[0].record()
    vs, res, it = lb.steady_state(A, K, tol=1e-12, max_iter=max_iter, restart=restart, basis=B, H=H)
    ev[1].record()
    torch.cuda.synchronize()
    names = [n for n, _ in states] + ["steady_state"]
    V = torch.stack([v for _, v in states] + [vs]).contiguous()
    out = lb.rho_checks(B, V, psd_shift=1e-10)
    ss = {"rel_residual": res, "iterations": it, "restart": restart or min(A.shape[0], 1024),
          "max_iter": max_iter, "ms": ev[0].elapsed_time(ev[1]),
          "preconditioner": "H eigenbasis, sigma = -Tr(A)/M" if H is not None else None,
          "first_call_ms": first_ms}
    if plain_max_iter:
        ev[0].record()
        _, res0, it0 = lb.steady_state(A, K, tol=1e-12, max_iter=plain_max_iter, restart=restart)
        ev[1].record()
        torch.cuda.synchronize()
        ss["plain"] = {"rel_residual": res0, "iterations": it0, "ms": ev[0].elapsed_time(ev[1])}
    return {"steady_state": ss,
            "rho": {n: {"trace_minus_1": float(out[k, 0]), "hermiticity": float(out[k, 1]),
                        "min_cholesky_pivot_shift_1e-10": float(out[k, 2])} for k, n in enumerate(names)},
            "note": "FP64 on the device: restarted GMRES for (Q + R) v* = -K, and rho rebuilt from v"}


def upload_bytes(M, pinned):
    """Bytes of a that lb_assemble moves to the device: the upper triangle of
    a page-locked a, read over the host link; a pageable a crosses in row
    blocks of h rows (columns from the block's first row on) for M > 2048,
    whole otherwise."""
    if pinned:
        return 16 * (M * (M + 1) // 2)
    if M > 2048:
        h = max(256, (M + 63) // 64)
        return sum(16 * (min(M, j0 + h) - j0) * (M - j0) for j0 in range(0, M, h))
    return 16 * M * M


def run_e2e(args, lb, B, a, H_host, M, nrk, dt, dev, dist, world):
    """Same metric through lb_assemble / lb_integrate with host buffers."""
    import numpy as np
    import torch
    import workloads as wl

    a_host = torch.empty(a.shape, dtype=a.dtype, pin_memory=True)
    a_host.copy_(a)
    a_np = a_host.numpy()
    o = B.expand(torch.tensor(wl.pure_state(B.N, 0), device=dev)).real.cpu().numpy()
    v0 = np.ascontiguousarray(o)
    out = np.zeros(M)
    t_asm, t_tot, phases = [], [], []
    for k in range(1 + args.steps):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sysm = lb.System(B, a_np, H=H_host, algorithm=args.algorithm)
        t1 = time.perf_counter()
        sysm.integrate(v0, nrk * dt, dt, precision="fp64", out=out)
        t2 = time.perf_counter()
        ph = sysm.timings()
        sysm.close()
        if k > 0:
            t_asm.append(t1 - t0)
            t_tot.append(t2 - t0)
            phases.append(ph)
    sa, st = replica_max([sum(t_asm), sum(t_tot)], dist, dev)
    pinned = a_host.is_pinned()
    del a_host
    lb.native.host_release()
    a_bytes = upload_bytes(M, pinned)
    mean_ph = {k: statistics.mean(p[k] for p in phases) for k in phases[0]} if phases else {}
    spread = (max(t_asm) - min(t_asm)) / statistics.mean(t_asm) if t_asm else None
    return {"value": replica_value(world, args.steps * M * M, sa), "unit": "entries/s",
            "assemble_s_per_step": [round(x, 4) for x in t_asm],
            "assemble_spread": spread,
            "assemble_phase_ms": mean_ph,
            "h2d_gbs": (a_bytes / (mean_ph["h2d"] * 1e-3) / 1e9) if mean_ph.get("h2d") else None,
            "h2d_bytes_per_step": a_bytes + 16 * B.N * B.N + 8 * M, "d2h_bytes_per_step": 8 * M,
            "rk4_steps_per_s": replica_value(world, args.steps * nrk, st - sa),
            "api": "lb_assemble(host H, host a) + lb_integrate(host v0 -> host v)"}


def cpu_baseline(args, a, M, N, rows=None):
    """The oracle (plain C, OpenMP) on a bounded sample: full rows of R."""
    import numpy as np
    import torch

    from oracle import Oracle, num_threads
    rows = args.cpu_rows if rows is None else rows
    t0 = time.perf_counter()
    o = Oracle(N)
    t_setup = time.perf_counter() - t0
    P = N * (N - 1) // 2
    cand = [P // 3, P + P // 2, 2 * P + N // 2, P // 7]
    s_rows = np.array(cand[:rows], np.int64)
    need = o.rows_needed(s_rows)
    a_rows = a[torch.as_tensor(need, device=a.device)].cpu().numpy()
    s = np.repeat(s_rows, M)
    n = np.tile(np.arange(M, dtype=np.int64), len(s_rows))
    t0 = time.perf_counter()
    o.R_entries_rows(need, a_rows, s, n)
    dt = time.perf_counter() - t0
    o.close()
    out = {"value": len(s) / dt, "unit": "entries/s", "cores": num_threads(), "kind": "oracle",
           "sample": "%d full rows of R (%d entries) at N=%d; f/d enumeration setup %.1f s not timed"
                     % (len(s_rows), len(s), N, t_setup)}
    out["rk4"] = cpu_rk4_baseline(M)
    return out


def cpu_rk4_baseline(M, steps=3):
    """The oracle's dense RK4 (plain C loops, OpenMP) timed over a few steps
    of an M x M system.  Its cost does not depend on the values, so the
    matrix is a constant fill made on the host (nothing from the GPU path)."""
    import numpy as np

    from oracle import num_threads, rk4_dense
    need = 8.0 * M * M
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 0
    if avail < 2.5 * need:
        return {"skipped": "host memory: %.1f GB available, %.1f GB needed" % (avail / 1e9, 2.5 * need / 1e9)}
    A = np.full((M, M), 1e-6)
    K = np.zeros(M)
    v0 = np.full(M, 1e-3)
    rk4_dense(A, K, v0, 1e-3, 1)  # first touch outside the timing
    t0 = time.perf_counter()
    rk4_dense(A, K, v0, 1e-3, steps)
    dt = time.perf_counter() - t0
    del A
    return {"steps_per_s": steps / dt, "steps": steps, "cores": num_threads(),
            "sample": "%d RK4 steps of the oracle's dense RK4 at M=%d (4 dense matrix-vector products per step)"
                      % (steps, M)}


# ---------------------------------------------------------------- the other forms

def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_forms(args, dev, a200=None):
    """Measurements of the other workloads, outside the timed region of the
    headline step: dense N=10 and N=50, the sparse ladder, the batched
    ensemble and the serving loop."""
    out = {}
    if not args.no_small:
        out["dense_n10"] = form_dense(args, dev, 10, 10_000, 1000)
        out["dense_n50"] = form_dense(args, dev, 50, 10_000, 1050)
        out["spectrum"] = form_spectrum(args, dev)
    if not args.no_sparse:
        out["sparse_ladder"] = form_sparse(args, dev)
        out["dimer"] = form_dimer(args, dev)
    if not args.no_batched:
        out["batched"] = form_batched(args, dev)
    if not args.no_serving:
        import torch
        torch.cuda.empty_cache()
        out["serving"] = form_serving(args, dev, a200)
    return out


def form_dense(args, dev, N, steps, seed):
    """One realization: assembly, FP64 RK4 and FP32-storage RK4 with the FP64
    correction every 50 steps, `steps` steps each (rho0 = |0><0|, dt)."""
    import torch

    import paper_1912_01491_gb300 as lb
    import workloads as wl
    M = N * N - 1
    H, a = wl.random_lindbladian_device(N, seed, device=dev)
    B = lb.Basis(N)
    h = B.expand(H).real.contiguous()
    v0 = B.expand(torch.tensor(wl.pure_state(N, 0), device=dev)).real.contiguous()
    A = torch.empty((M, M), dtype=torch.float64, device=dev)
    K = torch.empty(M, dtype=torch.float64, device=dev)
    for _ in range(2):
        kms = B.assemble_dense_timed(a, h=h, A=A, K=K, algorithm="closed")
    A32 = lb.pack_fp32(A)
    work = lb.rk4_workspace(M, dev)
    ev = _events(4)
    v64, v32 = v0.clone(), v0.clone()
    lb.rk4_dense(A, K, v0.clone(), args.dt, 50, precision="fp64", work=work)
    ev[0].record()
    lb.rk4_dense(A, K, v64, args.dt, steps, precision="fp64", work=work)
    ev[1].record()
    lb.rk4_dense(A32, K, v32, args.dt, steps, precision="fp32", A64=A, correct_every=50, work=work)
    ev[2].record()
    torch.cuda.synchronize()
    t64, t32 = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    err = float(torch.linalg.norm(v32 - v64) / torch.linalg.norm(v64))
    rho = B.rho(v64)
    checks = fp64_checks(lb, B, A, K, [("rk4_fp64", v64), ("rk4_fp32_corrected", v32)], restart=M,
                         max_iter=2 * M, H=H.contiguous(), plain_max_iter=2 * M)
    # the same trajectory in one persistent FP64 launch (cluster size tuned)
    pers = None
    if N <= 64:
        vp = v0.clone()
        bt = lb.Batch([N])
        bt.set(0, a, h, vp)
        bt.assemble("closed")
        bt.set_precision("fp64")
        C = int(bt.tune(width=4, probe_steps=50, dt=args.dt)[0])
        ms = bt.integrate(args.dt, steps)
        torch.cuda.synchronize()
        bt.close()
        pers = {"ms": ms, "steps_per_s": steps / (ms * 1e-3), "cluster": C,
                "rel_diff_vs_stream_fp64": float(torch.linalg.norm(vp - v64) / torch.linalg.norm(v64))}
    # propagator form: one product per step with D' = (P(hA) - 1)/h, for 1 and
    # 16 states at once (reported apart from classical RK4)
    prop = {}
    for prec in ("fp64", "fp32"):
        corr = 50 if prec == "fp32" else 0
        ev = _events(2)
        ev[0].record()
        P = lb.Propagator(A, K, args.dt, precision=prec, nrhs=16)
        ev[1].record()
        torch.cuda.synchronize()
        entry = {"form_ms": ev[0].elapsed_time(ev[1])}
        for R, n in ((1, steps), (16, max(steps // 10, 100))):
            V = v0.repeat(R, 1).contiguous()
            P.step(V, 50, correct_every=corr)  # warm-up
            V = v0.repeat(R, 1).contiguous()
            ev = _events(2)
            ev[0].record()
            P.step(V, n, correct_every=corr)
            ev[1].record()
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1])
            entry["states_%d" % R] = {"steps": n, "ms": ms, "steps_per_s": n / (ms * 1e-3),
                                      "state_steps_per_s": R * n / (ms * 1e-3)}
            if R == 1 and n == steps:
                entry["rel_err_vs_rk4_fp64"] = float(torch.linalg.norm(V[0] - v64) / torch.linalg.norm(v64))
        prop[prec] = entry
        del P
    B.close()
    return {"N": N, "M": M, "steps": steps, "dt": args.dt, "assembly_ms": sum(kms.values()),
            "propagator": prop,
            "fp64_checks": checks,
            "rk4_fp64_persistent": pers,
            "entries_per_s": M * M / (sum(kms.values()) * 1e-3),
            "rk4_fp64_ms": t64, "rk4_fp64_steps_per_s": steps / (t64 * 1e-3),
            "rk4_fp32c_ms": t32, "rk4_fp32c_steps_per_s": steps / (t32 * 1e-3),
            "fp32c_rel_err_vs_fp64": err,
            "trace_rho_minus_1": float(abs(torch.diagonal(rho).real.sum() - 1.0)),
            "note": "single realization on the stream engine (4 fused stage launches per step)"}


def form_spectrum(args, dev):
    """Spectrum of one random Lindbladian of the paper's ensemble (Sec. 3:
    H = 0, Kossakowski matrix N G G^dagger / Tr; Sec. 6, Fig. 5): the M
    eigenvalues of A = Q + R (the solver library's dense nonsymmetric
    eigensolver) and their density on a 100 x 100 grid (own kernel)."""
    import torch

    import paper_1912_01491_gb300 as lb
    import workloads as wl
    N = args.spectrum_n
    M = N * N - 1
    a = wl.random_lindbladian_paper_device(N, args.seed + 11, device=dev)  # H = 0, Tr a = N (Sec. 3)
    B = lb.Basis(N)
    A = torch.empty((M, M), dtype=torch.float64, device=dev)
    B.assemble_dense(a, h=None, A=A, algorithm="closed")
    del a
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w = lb.spectrum(A)
    torch.cuda.synchronize()
    t_eig = time.perf_counter() - t0
    re, im = w.real, w.imag
    pad = 0.02 * max(float(re.max() - re.min()), float(im.abs().max()))
    box = (float(re.min()) - pad, float(re.max()) + pad, -float(im.abs().max()) - pad, float(im.abs().max()) + pad)
    ev = _events(2)
    ev[0].record()
    dens = lb.spectrum_density(w, box, 100, 100)
    ev[1].record()
    torch.cuda.synchronize()
    area = (box[1] - box[0]) / 100 * (box[3] - box[2]) / 100
    tr = float(torch.trace(A))
    out = {"N": N, "M": M, "ensemble": "H = 0, a = N G G^dagger / Tr(G G^dagger)", "eigensolver_s": t_eig, "density_ms": ev[0].elapsed_time(ev[1]),
           "max_real_part": float(re.max()), "min_real_part": float(re.min()), "max_abs_imag": float(im.abs().max()),
           "sum_minus_trace_rel": abs(float(w.sum().real) - tr) / abs(tr),
           "grid": [100, 100], "box": box, "counted": int(round(float(dens.sum()) * area)),
           "note": "all M = N^2 - 1 eigenvalues of A; the N = 200 spectrum of Fig. 5 (M = 39,999) takes the dense "
                   "eigensolver about 10 minutes, too long for a default bench run (--spectrum-n 200 runs it)"}
    if args.spectrum_out:
        import numpy as np
        np.savez_compressed(args.spectrum_out, eig=w.cpu().numpy(), density=dens.cpu().numpy(), box=np.array(box))
    B.close()
    return out


def csr_step_bytes(precision, nnz, M):
    """Algorithmic bytes of one CSR RK4 step (4 stages): values and columns
    and the row pointers (int64) read once per stage; the stage vector
    gathered once per stage (FP32 copy in FP32 mode); Keff and v read every
    stage, v written once; acc written (stage 1), read and written (2, 3),
    read (4); the next stage vector written every stage (FP32 copy only in
    FP32 mode)."""
    val = 4.0 if precision == "fp32" else 8.0
    x = 4.0 if precision == "fp32" else 8.0
    per_stage = nnz * (val + 4.0) + (M + 1) * 8.0 + M * (x + 8.0 + 8.0 + x)
    return 4.0 * per_stage + 8.0 * M + 48.0 * M


def form_sparse(args, dev):
    """Sparse ladder model: CSR assembly of Q + R and K, CSR RK4 (FP32 values
    with FP64 correction every 50 steps, and FP64)."""
    import torch

    import paper_1912_01491_gb300 as lb
    import workloads as wl
    N = args.sparse_n
    M = N * N - 1
    H, L, g = wl.ladder_model(N, args.seed + 3)
    B = lb.Basis(N)
    l = B.expand(torch.tensor(L, device=dev))
    nz = torch.nonzero(l.abs() > 0).flatten()
    ch = [(g, nz, l[nz].contiguous())]
    h = B.expand(torch.tensor(H, device=dev)).real.contiguous()
    lb.Csr(B, h=h, channels=ch).close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = lb.Csr(B, h=h, channels=ch)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    rho0 = torch.zeros((N, N), dtype=torch.complex128, device=dev)
    rho0[N - 1, N - 1] = 1.0
    v0 = B.expand(rho0).real.contiguous()
    work = lb.rk4_workspace(M, dev)
    n = args.sparse_steps
    res = {}
    for prec, corr in (("fp32", 50), ("fp64", 0)):
        v = v0.clone()
        c.rk4(v, args.dt, 10, precision=prec, correct_every=corr, work=work)
        ev = _events(2)
        ev[0].record()
        c.rk4(v, args.dt, n, precision=prec, correct_every=corr, work=work)
        ev[1].record()
        torch.cuda.synchronize()
        res[prec] = ev[0].elapsed_time(ev[1])
    nnz = c.nnz
    step_bytes = {p: csr_step_bytes(p, nnz, M) for p in ("fp32", "fp64")}
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    gbs = {p: step_bytes[p] * n / (res[p] * 1e-3) / 1e9 for p in res}
    c.close()
    B.close()
    return {"N": N, "M": M, "nnz": nnz, "row_terms": c.terms, "assembly_s": t_asm,
            "rk4_fp32c_steps_per_s": n / (res["fp32"] * 1e-3), "rk4_fp64_steps_per_s": n / (res["fp64"] * 1e-3),
            "rk4_roofline": {"kernel": "k_stage_csr_pipe (persistent CSR SpMV + stage update; each chunk of 256 rows staged two chunks ahead by cp.async.bulk with an evict-first L2 policy)", "bound": "hbm",
                             "achieved": gbs["fp32"], "peak": hbm, "unit": "GB/s",
                             "frac": gbs["fp32"] / hbm if hbm else None,
                             "algorithmic_bytes_per_step": step_bytes["fp32"],
                             "fp64_achieved_gbs": gbs["fp64"]},
            "note": "FP32 row includes one FP64 correction SpMV every 50 steps in its time"}


def form_dimer(args, dev):
    """The periodically rocked dimer of Sec. 3 (Eqs. (10)-(11)) as the paper
    integrates it: N = dimer_n, CSR A0 = Q0 + R and Q1, FP64 RK4 over one
    period T = 2 pi with dimer_steps steps, eps switching at T/2; the
    density-matrix checks of the final state on the device."""
    import math

    import torch

    import paper_1912_01491_gb300 as lb
    import workloads as wl
    N, steps = args.dimer_n, args.dimer_steps
    M = N * N - 1
    T = 2.0 * math.pi
    H0, H1, L, rate, eps = wl.dimer_model(N)
    B = lb.Basis(N)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    l = B.expand(torch.tensor(L, device=dev))
    nz = torch.nonzero(l.abs() > 0).flatten()
    A0 = lb.Csr(B, h=B.expand(torch.tensor(H0, device=dev)).real.contiguous(), channels=[(rate, nz, l[nz])])
    Q1 = lb.Csr(B, h=B.expand(torch.tensor(H1, device=dev)).real.contiguous(), channels=())
    torch.cuda.synchronize()
    asm_s = time.perf_counter() - t0
    rho0 = torch.zeros((N, N), dtype=torch.complex128, device=dev)
    rho0[N - 1, N - 1] = 1.0
    v = B.expand(rho0).real.contiguous()
    work = lb.rk4_workspace(M, dev)
    A0.rk4_td(Q1, v.clone(), T / steps, 10, [0.0, T / 2], list(eps), T, work=work)  # warm-up
    ev = _events(2)
    ev[0].record()
    A0.rk4_td(Q1, v, T / steps, steps, [0.0, T / 2], list(eps), T, work=work)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    chk = lb.rho_checks(B, v, psd_shift=1e-10)[0]
    out = {"N": N, "M": M, "nnz_A0": A0.nnz, "nnz_Q1": Q1.nnz, "steps_per_period": steps, "period": T,
           "eps": list(eps), "assembly_s": asm_s, "period_s": ms * 1e-3, "steps_per_s": steps / (ms * 1e-3),
           "rho_final": {"trace_minus_1": float(chk[0]), "hermiticity": float(chk[1]),
                         "min_cholesky_pivot_shift_1e-10": float(chk[2])},
           "note": "FP64 CSR RK4 with Q(t) = Q0 + eps(t) Q1, two SpMVs per stage fused in one kernel; "
                   "rho0 = |N-1><N-1| (all bosons on site 1)"}
    A0.close()
    Q1.close()
    B.close()
    return out


def form_batched(args, dev):
    """Ensemble of random Lindbladians with N uniform in [4, 40]: assembly of
    every realization, cluster-size tuning, one persistent launch per cluster
    size over all realizations (FP32 storage, FP64 correction every 50 steps),
    against the plain FP64 single-system path one realization at a time on a
    sample."""
    import numpy as np
    import torch

    import paper_1912_01491_gb300 as lb
    import workloads as wl
    count, steps, dt = args.batch_count, args.batch_steps, args.dt
    Ns = [int(x) for x in wl.batch_sizes(count, args.seed + 11)]
    inputs = []
    for r, N in enumerate(Ns):
        H, a = wl.random_lindbladian_device(N, args.seed + 100 + r, device=dev)
        inputs.append((N, H, a))
    bases = {N: lb.Basis(N) for N in sorted(set(Ns))}
    hs, v0s = [], []
    for r, (N, H, a) in enumerate(inputs):
        B = bases[N]
        hs.append(B.expand(H).real.contiguous())
        rho0 = torch.zeros((N, N), dtype=torch.complex128, device=dev)
        rho0[r % N, r % N] = 1.0
        v0s.append(B.expand(rho0).real.contiguous())
    b = lb.Batch(Ns)
    vs = [v.clone() for v in v0s]
    for r in range(count):
        b.set(r, inputs[r][2], hs[r], vs[r])
    b.assemble("closed")
    torch.cuda.synchronize()
    ev = _events(2)
    ev[0].record()
    b.assemble("closed")
    ev[1].record()
    torch.cuda.synchronize()
    asm_ms = ev[0].elapsed_time(ev[1])
    t0 = time.perf_counter()
    choice = b.tune(width=6, probe_steps=20, dt=dt)
    tune_s = time.perf_counter() - t0
    int_ms = b.integrate(dt, steps, correct_every=50)
    torch.cuda.synchronize()
    # the same ensemble in the propagator form (one product per step with
    # D' = (P(hA) - 1)/h, FP32, FP64 defect every 50 steps), from the same v0
    vp = [v.clone() for v in v0s]
    bp = lb.Batch(Ns)
    for r in range(count):
        bp.set(r, inputs[r][2], hs[r], vp[r])
    bp.assemble("closed")
    bp.set_form("propagator")
    form_ms = bp.form_propagator(dt)  # device time of forming D' and c'
    bp.tune(width=6, probe_steps=20, dt=dt)
    prop_int_ms = bp.integrate(dt, steps, correct_every=50)
    torch.cuda.synchronize()
    bp.close()
    # plain FP64, one realization at a time (assembly + RK4), on a sample
    S = min(args.batch_fp64_sample, count)
    errs = []
    ev = _events(2)
    ev[0].record()
    outs = []
    for r in range(S):
        N = Ns[r]
        M = N * N - 1
        g = bases[N].assemble_dense(inputs[r][2], h=hs[r], algorithm="closed")
        v = v0s[r].clone()
        lb.rk4_dense(g["A"], g["K"], v, dt, steps, precision="fp64")
        outs.append(v)
    ev[1].record()
    torch.cuda.synchronize()
    fp64_ms = ev[0].elapsed_time(ev[1])
    perrs = []
    for r in range(S):
        errs.append(float(torch.linalg.norm(vs[r] - outs[r]) / torch.linalg.norm(outs[r])))
        perrs.append(float(torch.linalg.norm(vp[r] - outs[r]) / torch.linalg.norm(outs[r])))
    Ms = np.array([n * n - 1 for n in Ns], dtype=np.float64)
    for B in bases.values():
        B.close()
    b.close()
    rate_b = count / ((asm_ms + int_ms) * 1e-3)
    rate_p = count / ((asm_ms + form_ms + prop_int_ms) * 1e-3)
    rate_1 = S / (fp64_ms * 1e-3)
    hist = {int(c): int((np.asarray(choice) == c).sum()) for c in sorted(set(int(x) for x in choice))}
    return {"realizations": count, "N_range": [4, 40], "steps": steps, "dt": dt,
            "assembly_ms": asm_ms, "integrate_ms": int_ms, "tune_s": tune_s,
            "realizations_per_s": rate_b,
            "fp64_single_realizations_per_s": rate_1, "fp64_single_sample": S,
            "speedup_vs_fp64_single": rate_b / rate_1,
            "max_rel_err_vs_fp64": max(errs), "cluster_sizes": hist,
            "propagator": {"realizations_per_s": rate_p, "form_ms": form_ms, "integrate_ms": prop_int_ms,
                           "steps_per_s_per_realization": steps / (prop_int_ms * 1e-3),
                           "speedup_vs_rk4_batched": rate_p / rate_b,
                           "speedup_vs_fp64_single": rate_p / rate_1,
                           "max_rel_err_vs_fp64": max(perrs),
                           "note": "one product per step with D' = (P(hA) - 1)/h in FP32 (formed by the library's "
                                   "batched GEMM), c' in FP64, FP64 defect every 50 steps; realizations/s counts "
                                   "the assembly (as for the stage-by-stage form), forming D' and c', and the "
                                   "integration"},
            "rk4_stage_matrix_gb_per_s": float(4.0 * steps * (4.0 * Ms * Ms).sum() / (int_ms * 1e-3) / 1e9),
            "note": "matrix bytes the stages consume per second (FP32 A read 4x per step); slices that stay "
                    "in shared memory are not re-read from HBM, so this can exceed HBM bandwidth"}


def form_serving(args, dev, a200=None):
    """Poisson stream of random-Lindbladian requests, N uniform on {20, 50,
    100, 150, 200}, through the server (continuous batching): FP32 storage
    with the FP64 correction every 50 steps for N <= 64 (cluster engine),
    BF16 with the correction every 5 steps above (stream engine),
    `serve_steps` RK4 steps of dt per request.
    Every request has its own GUE H, rho0 = |k><k| and Kossakowski matrix
    a_r = Phi_r a_N Phi_r^dagger with Phi_r a diagonal unitary of random
    phases (the Wishart ensemble is invariant under unitary similarity, so
    a_r is another draw of it); inputs are formed on the device before
    submission and excluded from latency.  The arrival rate is `serve_load`
    times the sustained throughput of a burst of `serve_burst` requests
    submitted at once.
    Baseline: the plain FP64 path one request at a time (assembly + FP64 RK4,
    no batching, no low precision); its service time per N is measured alone
    and the same trace is replayed through a one-slot queue.  Errors: the
    first served request of every N is run again alone in FP64 on the same
    inputs."""
    import numpy as np
    import torch

    import paper_1912_01491_gb300 as lb
    import workloads as wl
    Nset = (20, 50, 100, 150, 200)
    steps, dt = args.serve_steps, args.dt
    prec = {N: ("fp32" if N <= 64 else "bf16") for N in Nset}
    corr = {N: (50 if prec[N] == "fp32" else 5) for N in Nset}
    ring_n = {20: 8, 50: 8, 100: 4, 150: 3, 200: 3}
    base, bases, rings = {}, {}, {}
    for N in Nset:
        if N == 200 and a200 is not None:
            a = a200
        elif N <= 50:
            a = wl.random_lindbladian_device(N, args.seed + 500 + N, device=dev)[1]
        else:
            a = wl.wishart_kossakowski_device(N, args.seed + 500 + N, device=dev)
        base[N] = a
        bases[N] = lb.Basis(N)
        rings[N] = [torch.empty_like(a) for _ in range(ring_n[N])]
    used = {N: [None] * ring_n[N] for N in Nset}  # request id that last read each ring slot

    def inputs(N, i, slot):
        """H, a_r (into slot) and v0 of request i."""
        g = np.random.default_rng([args.seed, i + 1_000_000, N])  # i >= -3000
        ph = torch.tensor(np.exp(1j * g.uniform(0.0, 2.0 * np.pi, N * N - 1)), device=dev)
        torch.mul(base[N], ph[:, None], out=slot)
        slot.mul_(ph.conj()[None, :])
        H = torch.tensor(wl.gue_hamiltonian(N, args.seed + 7 * (i + 1000) + N), device=dev)
        rho0 = torch.zeros((N, N), dtype=torch.complex128, device=dev)
        rho0[i % N, i % N] = 1.0
        return H, slot, bases[N].expand(rho0).real.contiguous()

    srv = lb.Server(int(args.serve_budget_gb * 2**30), slots=8, bypass_ms=2000.0)
    # alone latencies (also warms the pool and the graph path)
    alone, alone_host = {}, {}
    for N in Nset:
        H, a, v0 = inputs(N, -1 - N, rings[N][0])
        out = torch.empty_like(v0)
        torch.cuda.synchronize()
        rid = srv.submit(a, v0, out, dt, steps, H=H, precision=prec[N], correct_every=corr[N])
        r0 = srv.wait(rid)
        alone[N] = r0["latency_ms"]
        # host share of the service: admission -> completion seen by the host,
        # minus the device span of the request's work
        alone_host[N] = r0["latency_ms"] - r0["queue_ms"] - r0["gpu_ms"]
    # sustainable throughput: a burst of requests submitted at once (mixed N,
    # the trace's distribution), completions per second until the last
    burst_N = [int(x) for x in wl.rng(args.seed + 78).choice(np.asarray(Nset), size=args.serve_burst)]
    srv.reset_stats()
    torch.cuda.synchronize()
    tb = time.perf_counter()
    bids, bouts, slot_of = [], [], {N: 0 for N in Nset}
    for j, N in enumerate(burst_N):
        k = slot_of[N] % ring_n[N]
        slot_of[N] += 1
        prev = used[N][k]
        while prev is not None and srv.state(prev) < lb.native.LB_REQ_ASSEMBLED:
            time.sleep(0.0005)
        H, a, v0 = inputs(N, -2000 - j, rings[N][k])
        out = torch.empty_like(v0)
        rid = srv.submit(a, v0, out, dt, steps, H=H, precision=prec[N], correct_every=corr[N])
        used[N][k] = rid
        bids.append(rid)
        bouts.append(out)
    for rid in bids:
        srv.wait(rid)
    sustained = len(burst_N) / (time.perf_counter() - tb)
    del bouts
    rate = args.serve_load * sustained  # requests / s
    arr, Nreq = wl.serving_trace(args.serve_count, args.seed + 77, rate, Nset)
    srv.reset_stats()
    outs, ids, ring_waits = [], [], 0
    nxt = {N: 0 for N in Nset}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(len(arr)):
        N = int(Nreq[i])
        k = nxt[N]
        nxt[N] = (k + 1) % ring_n[N]
        prev = used[N][k]
        if prev is not None and srv.state(prev) < lb.native.LB_REQ_ASSEMBLED:
            ring_waits += 1
            while srv.state(prev) < lb.native.LB_REQ_ASSEMBLED:
                time.sleep(0.0005)
        while time.perf_counter() - t0 < arr[i]:
            time.sleep(0.0005)
        H, a, v0 = inputs(N, i, rings[N][k])
        out = torch.empty_like(v0)
        rid = srv.submit(a, v0, out, dt, steps, H=H, precision=prec[N], correct_every=corr[N])
        used[N][k] = rid
        ids.append(rid)
        outs.append(out)
    res = [srv.wait(rid) for rid in ids]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    for r in rings.values():
        r.clear()
    torch.cuda.empty_cache()
    # plain FP64, one request at a time: service time per N (alone) and the
    # error of the first served request of each N
    fp64_ms, errs = {}, {}
    scratch = {}
    for N in Nset:
        i = next((j for j in range(len(Nreq)) if int(Nreq[j]) == N), None)
        if i is None:
            continue
        scratch[N] = torch.empty_like(base[N])
        B = bases[N]
        M = N * N - 1
        H, a, v0 = inputs(N, i, scratch[N])
        A = torch.empty((M, M), dtype=torch.float64, device=dev)
        K = torch.empty(M, dtype=torch.float64, device=dev)
        work = lb.rk4_workspace(M, dev)
        torch.cuda.synchronize()
        ev = _events(2)
        ev[0].record()
        h = B.expand(H).real.contiguous()
        B.assemble_dense(a, h=h, A=A, K=K, algorithm="closed")
        v = v0.clone()
        lb.rk4_dense(A, K, v, dt, steps, precision="fp64", work=work)
        ev[1].record()
        torch.cuda.synchronize()
        fp64_ms[N] = ev[0].elapsed_time(ev[1])
        errs[N] = float(torch.linalg.norm(outs[i] - v) / torch.linalg.norm(v))
        del A, K, work, scratch[N]
        torch.cuda.empty_cache()
    lat = np.array([r["latency_ms"] for r in res])
    per_N = {}
    for N in Nset:
        l = [r["latency_ms"] for r, n in zip(res, Nreq) if int(n) == N]
        if l:
            per_N[str(N)] = {"count": len(l), "p50_ms": float(np.percentile(l, 50)),
                             "p99_ms": float(np.percentile(l, 99)), "alone_ms": alone[N],
                             "alone_host_ms": alone_host[N], "fp64_alone_ms": fp64_ms.get(N)}
    # what a device-resident request loop could remove at most: the host
    # share of each request's service (admission -> completion seen by the
    # host, minus the device span of its work)
    host = np.array([r["latency_ms"] - r["queue_ms"] - r["gpu_ms"] for r in res])
    svc = np.array([r["latency_ms"] - r["queue_ms"] for r in res])
    # one-at-a-time FP64 replay of the same trace (one slot, no memory limit)
    svc64 = np.array([fp64_ms[int(n)] for n in Nreq])
    start64, fin64 = lb.native.sched_simulate(np.asarray(arr) * 1e3, np.ones(len(arr), np.int64), svc64,
                                              2**62, 1, 0.0)
    lat64 = fin64 - np.asarray(arr) * 1e3
    thr64 = len(arr) / ((fin64.max() - arr[0] * 1e3) * 1e-3)
    for B in bases.values():
        B.close()
    return {"requests": len(arr), "steps": steps, "dt": dt,
            "correct_every": {str(N): corr[N] for N in Nset},
            "precision": {str(N): prec[N] for N in Nset}, "arrival_rate_per_s": rate, "load": args.serve_load,
            "sustained_realizations_per_s": sustained, "burst": len(burst_N),
            "p50_latency_ms": st["p50_ms"], "p99_latency_ms": st["p99_ms"],
            "p99_is_max": bool(np.percentile(lat, 99, method="inverted_cdf") >= lat.max()),
            "throughput_realizations_per_s": st["throughput_per_s"], "wall_s": wall,
            "per_N": per_N,
            "max_rel_err_vs_fp64": {str(k): v for k, v in errs.items()},
            "fp64_one_at_a_time": {"p50_latency_ms": float(np.percentile(lat64, 50)),
                                   "p99_latency_ms": float(np.percentile(lat64, 99)),
                                   "throughput_realizations_per_s": thr64,
                                   "note": "plain FP64 path (closed assembly + FP64 RK4) per request, alone-measured "
                                           "service time per N, the same arrival trace through one slot"},
            "speedup_throughput_vs_fp64_one_at_a_time": st["throughput_per_s"] / thr64,
            "ring_waits": ring_waits,
            "host_share": {"p50_ms": float(np.percentile(host, 50)), "max_ms": float(host.max()),
                           "sum_over_service": float(host.sum() / svc.sum()),
                           "note": "per request: latency - queue - device span of its work; the bound on what a "
                                   "device-resident request loop could save"},
            "budget_gb": args.serve_budget_gb, "slots": 8,
            "note": "config 5's request stream with %d RK4 steps per request (the configuration names 5000) so "
                    "that the run stays within minutes; latency = submission (at the arrival time) to completion "
                    "seen by the host; inputs formed on the device before submission" % steps}


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return None
    import numpy as np
    import torch

    import workloads as wl
    from oracle import Oracle, num_threads
    N = args.n
    M = N * N - 1
    dev = torch.device("cuda", local) if torch.cuda.is_available() else None
    if dev is not None:
        a = wl.wishart_kossakowski_device(N, args.seed, device=dev)
    else:
        a = torch.tensor(wl.wishart_kossakowski(N, args.seed))
    t0 = time.perf_counter()
    o = Oracle(N)
    setup = time.perf_counter() - t0
    P = N * (N - 1) // 2
    rows = [(P // 3 + 37 * k) % (2 * P) for k in range(args.warmup + args.steps)]
    times = []
    for k, r in enumerate(rows):
        need = o.rows_needed(np.array([r]))
        a_rows = a[torch.as_tensor(need, device=a.device)].cpu().numpy()
        s = np.full(M, r, np.int64)
        n = np.arange(M, dtype=np.int64)
        t0 = time.perf_counter()
        o.R_entries_rows(need, a_rows, s, n)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    value = args.steps * M / sum(times)
    out = {"impl": "reference", "metric": "R entries assembled/s (dense random Lindbladian, N=%d)" % N,
           "value": value, "unit": "entries/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "dense random Lindbladian N=%d (M=%d); CPU oracle, one full row of R "
                                  "(M entries) per step" % (N, M), "N": N, "M": M},
           "cpu_baseline": {"value": value, "unit": "entries/s", "cores": num_threads(), "kind": "oracle",
                            "sample": "one row of R per step; f/d enumeration setup %.1f s not timed" % setup},
           "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def run_only(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.only == "dense_small":
        out = {"dense_n10": form_dense(args, dev, 10, 10_000, 1000),
               "dense_n50": form_dense(args, dev, 50, 10_000, 1050)}
    elif args.only == "sparse":
        out = {"sparse_ladder": form_sparse(args, dev)}
    elif args.only == "dimer":
        out = {"dimer": form_dimer(args, dev)}
    elif args.only == "batched":
        out = {"batched": form_batched(args, dev)}
    elif args.only == "spectrum":
        out = {"spectrum": form_spectrum(args, dev)}
    else:
        out = {"serving": form_serving(args, dev)}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()

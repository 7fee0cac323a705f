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
    p.add_argument("--rk4-steps", type=int, default=10, help="RK4 steps per bench step and precision")
    p.add_argument("--dt", type=float, default=1e-3)
    p.add_argument("--seed", type=int, default=20250)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-rows", type=int, default=2, help="rows of R in the CPU-oracle sample")
    p.add_argument("--count-terms", action="store_true", help="count the join terms W (extra pass)")
    p.add_argument("--algorithm", default="closed", choices=["closed", "join"],
                   help="dense R assembly: closed-form sums of the join (default) or every join term")
    return p.parse_args()


# ---------------------------------------------------------------- helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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
    dt, nrk = args.dt, args.rk4_steps
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
        lb.rk4_dense(A32, K, v32, dt, nrk, precision="fp32", A64=A, correct_every=50, work=work)
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
    times = torch.tensor([total_ms, asm_ms, rk_ms, rk32_ms], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(times, op=dist.ReduceOp.MAX)
    total_ms, asm_ms, rk_ms, rk32_ms = times.tolist()
    K_ = args.steps
    value = world * K_ * M * M / (asm_ms * 1e-3)
    t_asm = asm_ms / K_ * 1e-3
    alg_bytes = 16.0 * M * M + 8.0 * M * M + 16.0 * M
    # the other algorithm, timed outside the timed region for comparison
    other = "join" if args.algorithm == "closed" else "closed"
    other_ms = []
    for _ in range(2):
        other_ms.append(sum(B.assemble_dense_timed(a, h=h_last, A=A, K=K, algorithm=other).values()))
    B.assemble_dense_timed(a, h=h_last, A=A, K=K, algorithm=args.algorithm)
    roof = assembly_roofline(args.algorithm, top, kern[top], N, M, W, fp64_peak, measured_peaks())

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, lb, B, a, H_host, M, nrk, dt, dev, dist, world)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, a, M, N)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None
    peaks = measured_peaks()
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
                         "steps FP32 storage with FP64 correction (k=50), dt=%g" % (N, M, nrk, nrk, dt)),
            "N": N, "M": M, "join_terms": W,
            "l2": "inputs larger than L2 (a is %.1f GB)" % (16.0 * M * M / 1e9),
            "parallelism": "replicas" if world > 1 else "single",
        },
        "rk4_steps_per_s": world * K_ * nrk / (rk_ms * 1e-3),
        "rk4_fp32_corrected_steps_per_s": world * K_ * nrk / (rk32_ms * 1e-3),
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
        "gpu_launches": launches,
        "clocks": clk,
    }
    if e2e:
        out["e2e"] = e2e
    if cpu:
        out["cpu_baseline"] = cpu
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return out


def assembly_roofline(algorithm, top, top_ms, N, M, W, fp64_peak, peaks):
    """Roofline of the dominant assembly kernel (algorithmic work per launch
    over its event-timed launch duration)."""
    P2 = N * (N - 1)
    t = top_ms * 1e-3
    hbm = peaks.get("hbm_gbs")
    if top.startswith("k_entries") and algorithm == "closed":
        # reads every a entry of the pair x pair block once, writes A there once
        byts = 24.0 * P2 * P2
        return {"kernel": top, "bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": byts / t / 1e9 / hbm if hbm else None, "traffic": None,
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
    t_asm, t_tot = [], []
    for k in range(1 + args.steps):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sysm = lb.System(B, a_np, H=H_host, algorithm=args.algorithm)
        t1 = time.perf_counter()
        sysm.integrate(v0, nrk * dt, dt, precision="fp64", out=out)
        t2 = time.perf_counter()
        sysm.close()
        if k > 0:
            t_asm.append(t1 - t0)
            t_tot.append(t2 - t0)
    tt = torch.tensor([sum(t_asm), sum(t_tot)], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    sa, st = tt.tolist()
    del a_host
    return {"value": world * args.steps * M * M / sa, "unit": "entries/s",
            "h2d_bytes_per_step": 16 * M * M + 16 * B.N * B.N + 8 * M, "d2h_bytes_per_step": 8 * M,
            "rk4_steps_per_s": world * args.steps * nrk / (st - sa),
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
    return {"value": len(s) / dt, "unit": "entries/s", "cores": num_threads(), "kind": "oracle",
            "sample": "%d full rows of R (%d entries) at N=%d; f/d enumeration setup %.1f s not timed"
                      % (len(s_rows), len(s), N, t_setup)}


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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()

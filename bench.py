#!/usr/bin/env python
"""Benchmark: orbital-pair exchange applications per second on the Pt-cluster-shaped block.

Workload (synthetic, seeded): 96^3 uniform grid on [-12,12]^3, 64 orthonormal Gaussian-sum
orbitals over 8 fcc centres (spacing 2.6 bohr), shared Tucker rank 40 per mode from the
density HOSVD, 40-term Gaussian sum of 1/r.  One step = one tx_exchange_apply_energy call:
K psi_i = -sum_j psi_j phi_ij for all 64 targets against all 64 occupied orbitals (4096
ordered pair applications, 2080 distinct pair potentials) plus E_x in the same epilogue.
psi (226 MB) and W (226 MB) are larger than L2 (129 MB), so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|tf32x3|fp32|...]
  python bench.py --impl reference     # the FP64 oracle on the host cores, same metric

Under torchrun each rank applies K to its own copy of the block (independent replicas,
weak scaling, no collective on the data path); rank 0 prints one JSON line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "orbital-pair exchange applications/s"
WORKLOAD = dict(workload="Pt-cluster-shaped block", n=96, box="[-12,12]^3", orbitals=64, rank=40, terms=40,
                pairs_ordered=64 * 64, pairs_unique=64 * 65 // 2, seed=1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--orbitals", type=int, default=64,
                    help="use only the first N orbitals of the block (smaller cases for profiling)")
    return ap.parse_args()


def flops_per_pair(n, r, T):
    P = 2 * (n ** 3 * r + n ** 2 * r ** 2 + n * r ** 3)
    return (T + 1) * P + 3 * n ** 3


# ----------------------------------------------------------------------------------------
# oracle timing (the CPU baseline and the reference arm)
# ----------------------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle as O, workloads as W
s = W.config_pt()
S = O.Setup.from_system(s)
targets = {targets!r}
t0 = time.perf_counter()
Wrows = O.exchange_apply(s.psi, S, psi_tgt=s.psi[targets])
dt = time.perf_counter() - t0
np.save({out!r}, Wrows)
print(json.dumps(dict(seconds=dt, pairs=len(targets) * s.psi.shape[0])))
"""


def run_oracle_sample(targets, out_path):
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    code = ORACLE_SNIPPET.format(root=ROOT, targets=list(targets), out=out_path)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError("oracle sample failed: " + p.stderr[-2000:])
    res = json.loads(p.stdout.strip().splitlines()[-1])
    res["cores"] = cores
    return res


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    targets = [0]
    with tempfile.TemporaryDirectory() as td:
        times = []
        for i in range(args.warmup + args.steps):
            res = run_oracle_sample(targets, os.path.join(td, "w.npy"))
            if i >= args.warmup:
                times.append(res["seconds"])
    units = res["pairs"]
    tot = sum(times)
    value = units * len(times) / tot
    line = dict(impl="reference", metric=METRIC, value=value, unit="pairs/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000 * tot / len(times), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(WORKLOAD, sample=f"{len(targets)} target x 64 occupied orbitals per step"),
                cpu_baseline=dict(value=value, unit="pairs/s", cores=res["cores"], kind="oracle",
                                  sample=f"{units} ordered pairs (target 0 against all 64 orbitals) per step"),
                e2e=dict(value=value, unit="pairs/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
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
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=reasons, samples=len(rows))


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__
    __graft_entry__.build()
    import paper_2401_04189_gb300 as P
    import workloads as W

    prec = args.precision
    if prec == "auto":
        prec = getattr(P, "DEFAULT_BENCH_PRECISION", "fp32")
    s = W.config_pt()
    if args.orbitals != s.psi.shape[0]:
        s.psi = s.psi[: args.orbitals].copy()
    n, r, T = s.n[0], s.r[0], s.T
    N = s.psi.shape[0]
    stream = torch.cuda.current_stream()
    ctx = P.Context.from_system(s, precision=prec)
    psi_host = torch.from_numpy(s.psi).pin_memory()
    psi = psi_host.to(dev, non_blocking=False)
    out = torch.empty_like(psi)
    e = torch.empty((), dtype=torch.float64, device=dev)

    def step():
        P.tx_exchange_apply_energy(ctx, psi, out=out, e_out=e)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: device events on the launching stream, profiling events around kernels
    clocks = ClockSampler(dev.index if world == 1 else local)
    P.tx_profile_reset()
    P.tx_profile_enable(True)
    P.tx_reset_launch_count()
    barrier()
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    ck = clocks.stop()
    P.tx_profile_enable(False)
    launches = P.tx_launch_count()
    ms = ev0.elapsed_time(ev1) / args.steps
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    pairs = N * N
    value = world * pairs / (ms_max / 1000.0)

    # ---- dominant kernel: live per-launch device time from the profiling events
    prof = {}
    for name in ("consume", "project", "gemm", "tc_consume", "tc_zprod", "tc_project", "tc_g"):
        k, kms = P.tx_profile_read(name)
        if k:
            prof[name] = (k, kms)
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    roof = roofline(dom, prof, n, r, T, N, args.steps, prec, peaks, ck)

    # ---- end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        out_host = torch.empty_like(psi_host).pin_memory()
        e_host = torch.empty((), dtype=torch.float64).pin_memory()
        psi_e2e = torch.empty_like(psi)
        for _ in range(2):
            psi_e2e.copy_(psi_host, non_blocking=True)
            P.tx_exchange_apply_energy(ctx, psi_e2e, out=out, e_out=e)
            out_host.copy_(out, non_blocking=True)
            e_host.copy_(e, non_blocking=True)
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            psi_e2e.copy_(psi_host, non_blocking=True)
            P.tx_exchange_apply_energy(ctx, psi_e2e, out=out, e_out=e)
            out_host.copy_(out, non_blocking=True)
            e_host.copy_(e, non_blocking=True)
        a1.record(stream)
        barrier()
        ems = a0.elapsed_time(a1) / args.steps
        te = torch.tensor([ems], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = dict(value=world * pairs / (float(te.item()) / 1000.0), unit="pairs/s",
                   h2d_bytes_per_step=psi.numel() * 4, d2h_bytes_per_step=out.numel() * 4 + 8,
                   ms_per_step=float(te.item()))

    # ---- accuracy of this run against the FP64 oracle (sampled target rows), rank 0 only
    cpu = None
    err = None
    if rank == 0 and not args.no_cpu_baseline and N == 64:
        with tempfile.TemporaryDirectory() as td:
            targets = [0, 37]
            res = run_oracle_sample(targets, os.path.join(td, "w.npy"))
            ref = np.load(os.path.join(td, "w.npy"))
        got = out[targets].double().cpu().numpy()
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        cpu = dict(value=res["pairs"] / res["seconds"], unit="pairs/s", cores=res["cores"], kind="oracle",
                   sample=f"{res['pairs']} ordered pairs (targets 0 and 37 against all 64 orbitals), "
                          f"{res['seconds']:.2f} s of FP64 numpy")
    if world > 1:
        dist.barrier()
    if rank == 0:
        fl = flops_per_pair(n, r, T) * (N * (N + 1) // 2)
        line = dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=ms_max, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype=dtype_name(prec), data="synthetic",
                    config=dict(WORKLOAD, orbitals=N, pairs_ordered=N * N, pairs_unique=N * (N + 1) // 2,
                                precision=prec, l2="inputs larger than L2 (psi 226 MB, W 226 MB)",
                                parallelism=f"replicas x{world}"),
                    unique_pair_potentials_per_s=world * (N * (N + 1) // 2) / (ms_max / 1000.0),
                    algorithmic_tflops=world * fl / (ms_max / 1000.0) / 1e12,
                    err_vs_oracle=err, energy=float(e.item()),
                    roofline=roof, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
                    kernels={k: dict(launches=v[0], ms_total=round(v[1], 4)) for k, v in prof.items()},
                    clocks=ck)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def dtype_name(prec):
    return {"fp32": "f32", "bf16": "bf16", "tf32": "tf32", "tf32x3": "tf32x3", "bf16x3": "bf16x3"}.get(prec, prec)


# DRAM bytes (read + write) per distinct pair of the dominant kernel, from one ncu capture of
# the current kernel on the same block with 8 orbitals (36 pairs in one launch), scaled by the
# pairs a bench launch processes (traffic grows in proportion to pairs).  None where no capture
# of the current kernel exists.
DRAM_BYTES_PER_PAIR = {("tc_consume", "bf16"): (711.658752e6 + 83.418368e6) / 36}


def roofline(dom, prof, n, r, T, N, steps, prec, peaks, ck):
    """Achieved algorithmic FLOP/s of the dominant kernel over its live launch time."""
    if dom is None:
        return None
    k, kms = prof[dom]
    unique = N * (N + 1) // 2
    if dom in ("consume", "tc_consume"):
        per_pair = T * 2 * (n ** 2 * r ** 2 + n ** 3 * r) + 3 * n ** 3
    elif dom in ("tc_zprod",):
        per_pair = T * 2 * n * r ** 3
    elif dom in ("project", "tc_project"):
        per_pair = 2 * (n ** 3 * r + n ** 2 * r ** 2)
    else:
        per_pair = 2 * n * r ** 3 * (T + 1)
    flops = per_pair * unique * steps
    achieved = flops / (kms / 1000.0) / 1e12
    if prec == "fp32":
        sm_clock = 2070.0
        peak = 152 * 128 * 2 * sm_clock * 1e6 / 1e12
        bound, src = "alu", "152 SMs x 128 FP32 FMA/clk x 2 x 2070 MHz (derived)"
    else:
        measured = (peaks or {}).get("bf16_tflops_sustained")
        bf16 = measured if measured else 1700.0
        ratio = {"bf16": 1.0, "bf16x3": 1.0, "tf32": 0.5, "tf32x3": 0.5}.get(prec, 1.0)
        peak = bf16 * ratio
        bound = "tensor"
        src = ("measured sustained bf16" if measured else "fallback bf16") + (
            " x 0.5 (nominal tf32/bf16 ratio)" if ratio != 1.0 else "")
    bpp = DRAM_BYTES_PER_PAIR.get((dom, prec))
    traffic = bpp * unique * steps / k if bpp else None     # bytes per launch
    return dict(kernel=dom, bound=bound, achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                traffic=traffic, traffic_unit="bytes per launch (ncu dram read + write, scaled)" if traffic else None,
                launches=k, avg_launch_ms=kms / k, peak_source=src)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark: orbital-pair exchange applications per second (K psi_i = -sum_j psi_j phi_ij).

Default workload, the largest configuration (synthetic, seeded, generated on the device): the
TiO2-cluster-shaped block, a 160^3 uniform grid on [-16,16]^3 with 1842 occupied orbitals
(Gaussian sums over 16 of 240 rutile-like centres, 2 exponents U[0.2,3] each, orthonormalised in
float64), shared Tucker rank 64 per mode from the density HOSVD, a 45-term Gaussian sum of 1/r.
One step = one tx_exchange_apply of the first 256 orbitals (the targets) against all 1842:
471,552 ordered pair applications, 438,912 distinct pair potentials (a pair of two targets is
computed once).  psi (30.2 GB) and W (4.2 GB) are far larger than L2 (129 MB): no flush needed.

`--workload pt` runs the Pt-cluster-shaped block instead (96^3, 64 orbitals, rank 40, 40 terms,
one tx_exchange_apply_energy of all 64 against all 64 per step); the default run also reports it
in `secondary` (bf16, the split-precision tf32x3 form and the float32 CUDA-core form), with the
mesh transfer and the per-pair-bases path.  `--workload batch` times the replay of one captured
graph over the uneven batch of 16 systems.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|tf32x3|fp32|...] [--workload tio2|pt|batch]
  python bench.py --impl reference     # the FP64 oracle on the host cores, same metric and workload

Under torchrun each rank applies K to its own copy of the block (independent replicas, weak
scaling, no collective on the data path); rank 0 prints one JSON line.
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
WORKLOADS = {
    "tio2": dict(workload="TiO2-cluster-shaped block", n=160, box="[-16,16]^3", occupied=1842, targets=256,
                 rank=64, terms=45, seed=4),
    "pt": dict(workload="Pt-cluster-shaped block", n=96, box="[-12,12]^3", occupied=64, targets=64, rank=40,
               terms=40, seed=1),
}
DEFAULT_STEPS = {"tio2": 2, "pt": 10}
TIO2_SAMPLE_OCC = 32        # oracle sample: 1 target against this many occupied orbitals


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--workload", default="tio2", choices=sorted(WORKLOADS) + ["batch"])
    ap.add_argument("--expansion-form", type=int, default=0,
                    help="expansion kernel form (tx_set_expansion_form; 0 = automatic)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--occupied", type=int, default=None,
                    help="use only the first N occupied orbitals of the block (smaller cases for profiling)")
    ap.add_argument("--targets", type=int, default=None, help="TiO2-shaped block: number of target orbitals")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = DEFAULT_STEPS[a.workload]
    return a


def flops_per_pair(n, r, T):
    P = 2 * (n ** 3 * r + n ** 2 * r ** 2 + n * r ** 3)
    return (T + 1) * P + 3 * n ** 3


def pair_counts(n_occ, n_tgt, subset=True):
    """(ordered pair applications, distinct pair potentials) of targets = the first n_tgt
    occupied orbitals (a pair of two targets is one potential)."""
    ordered = n_occ * n_tgt
    return ordered, ordered - (n_tgt * (n_tgt - 1) // 2 if subset else 0)


# ----------------------------------------------------------------------------------------
# oracle timing (the CPU baseline and the reference arm): a subprocess on all host cores
# ----------------------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle as O, workloads as W
d = np.load({inp!r})
s = W.System("sample", [d["x1"], d["x2"], d["x3"]], [d["w1"], d["w2"], d["w3"]], [d["U1"], d["U2"], d["U3"]],
             d["theta"], d["mu"], d["occ"], 0.0)
S = O.Setup.from_system(s)
t0 = time.perf_counter()
Wrows = O.exchange_apply(d["occ"], S, psi_tgt=d["tgt"])
dt = time.perf_counter() - t0
np.save({out!r}, Wrows)
print(json.dumps(dict(seconds=dt, pairs=int(d["tgt"].shape[0] * d["occ"].shape[0]))))
"""


def run_oracle(s, occ, tgt, workdir):
    """The oracle's rows K tgt against occ for system s (its grid, basis and Gaussian sum), timed
    in a subprocess on every host core: (W rows, seconds, ordered pairs, cores)."""
    import numpy as np
    cores = os.cpu_count() or 1
    inp = os.path.join(workdir, "oracle_in.npz")
    out = os.path.join(workdir, "oracle_out.npy")
    np.savez(inp, x1=s.x[0], x2=s.x[1], x3=s.x[2], w1=s.w[0], w2=s.w[1], w3=s.w[2], U1=s.U[0], U2=s.U[1],
             U3=s.U[2], theta=s.theta, mu=s.mu, occ=np.asarray(occ, dtype=np.float32),
             tgt=np.asarray(tgt, dtype=np.float32))
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    code = ORACLE_SNIPPET.format(root=ROOT, inp=inp, out=out)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError("oracle sample failed: " + p.stderr[-2000:])
    res = json.loads(p.stdout.strip().splitlines()[-1])
    return np.load(out), res["seconds"], res["pairs"], cores


def oracle_sample_system(workload):
    """Host inputs for the oracle's bounded sample: the Pt-shaped block itself, or a TiO2-shaped
    block of 1 + TIO2_SAMPLE_OCC orbitals generated on the host with the same grid, rank, terms
    and orbital recipe (the oracle's cost per pair does not depend on the orbital values)."""
    import workloads as W
    if workload == "pt":
        s = W.config_pt()
        return s, s.psi, s.psi[0:1], "1 target x 64 occupied orbitals of the Pt-shaped block"
    cfg = WORKLOADS["tio2"]
    s = W.make_system("tio2", cfg["n"], 16.0, 1 + TIO2_SAMPLE_OCC, cfg["rank"], cfg["terms"], cfg["seed"],
                      W.rutile_cluster(240), 2, (0.2, 3.0), centres_per_orbital=16)
    return (s, s.psi[1:], s.psi[0:1],
            f"1 target x {TIO2_SAMPLE_OCC} occupied orbitals of a TiO2-shaped block (160^3, rank 64, 45 terms) "
            f"generated on the host")


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    s, occ, tgt, what = oracle_sample_system(args.workload)
    times = []
    with tempfile.TemporaryDirectory() as td:
        for i in range(args.warmup + args.steps):
            _, sec, pairs, cores = run_oracle(s, occ, tgt, td)
            if i >= args.warmup:
                times.append(sec)
    tot = sum(times)
    value = pairs * len(times) / tot
    cfg = dict(WORKLOADS[args.workload])
    line = dict(impl="reference", metric=METRIC, value=value, unit="pairs/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000 * tot / len(times), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(cfg, sample=f"{what} per step"),
                cpu_baseline=dict(value=value, unit="pairs/s", cores=cores, kind="oracle",
                                  sample=f"{pairs} ordered pairs per step: {what}"),
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
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    power_w_max=max(pw) if pw else None, reasons=reasons, samples=len(rows))


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
PROFILED = ("consume", "project", "gemm", "tc_consume", "tc_zprod", "tc_project", "tc_proj2", "tc_proj1")


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
    if args.workload == "batch":
        return batch_main(args, P, W, dev, prec, world, rank)
    cfg = dict(WORKLOADS[args.workload])
    t_setup = time.perf_counter()
    if args.workload == "tio2":
        n_occ = args.occupied or cfg["occupied"]
        s, psi = W.config_tio2_on_device(n_orb=n_occ, device=dev)
        n_tgt = min(args.targets or cfg["targets"], n_occ)
        l2 = f"inputs larger than L2 (psi {psi.numel() * 4 / 1e9:.1f} GB, W {n_tgt * psi[0].numel() * 4 / 1e9:.1f} GB)"
    else:
        s = W.config_pt()
        if args.occupied and args.occupied < s.psi.shape[0]:
            s.psi = s.psi[: args.occupied].copy()
        psi = torch.from_numpy(s.psi).to(dev)
        n_occ = n_tgt = psi.shape[0]
        l2 = "inputs larger than L2 (psi 226 MB, W 226 MB)"
    setup_s = time.perf_counter() - t_setup
    n, r, T = s.n[0], s.r[0], s.T
    ordered, unique = pair_counts(n_occ, n_tgt)
    stream = torch.cuda.current_stream()
    ctx = P.Context.from_system(s, precision=prec)
    ctx.set_workspace_limit(16 << 30)          # pair batches of up to 16 GiB of intermediates
    if args.expansion_form:
        P.tx_set_expansion_form(ctx, args.expansion_form)
    out = torch.empty((n_tgt,) + tuple(psi.shape[1:]), dtype=torch.float32, device=dev)
    e = torch.empty((), dtype=torch.float64, device=dev)
    tio2 = args.workload == "tio2"

    def step(src=None):
        src = psi if src is None else src
        if tio2:
            P.tx_exchange_apply(ctx, src, src[:n_tgt], out=out)
        else:
            P.tx_exchange_apply_energy(ctx, src, out=out, e_out=e)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ctx.check_device_error()

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
    ctx.check_device_error()
    ms = ev0.elapsed_time(ev1) / args.steps
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * ordered / (ms_max / 1000.0)

    # ---- dominant kernel: live per-launch device time from the profiling events
    prof = {}
    for name in PROFILED:
        k, kms = P.tx_profile_read(name)
        if k:
            prof[name] = (k, kms)
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    roof = roofline(dom, prof, n, r, T, unique, args.steps, prec, peaks, ck, args.workload)

    # ---- end to end through the public API with host buffers (pinned), copies timed: the
    # occupied block goes up and W (and E_x) comes down in every step
    e2e = None
    if not args.no_e2e:
        psi_host = torch.empty(psi.shape, dtype=torch.float32, pin_memory=True)
        psi_host.copy_(psi)
        out_host = torch.empty(out.shape, dtype=torch.float32, pin_memory=True)
        e_host = torch.empty((), dtype=torch.float64, pin_memory=True)
        psi_e2e = torch.empty_like(psi)

        def e2e_step():
            psi_e2e.copy_(psi_host, non_blocking=True)
            step(psi_e2e)
            out_host.copy_(out, non_blocking=True)
            if not tio2:
                e_host.copy_(e, non_blocking=True)

        e2e_steps = 1 if tio2 else args.steps
        if not tio2:
            for _ in range(2):
                e2e_step()
        barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        a1.record(stream)
        barrier()
        ems = a0.elapsed_time(a1) / e2e_steps
        te = torch.tensor([ems], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = dict(value=world * ordered / (float(te.item()) / 1000.0), unit="pairs/s",
                   h2d_bytes_per_step=psi.numel() * 4, d2h_bytes_per_step=out.numel() * 4 + (0 if tio2 else 8),
                   ms_per_step=float(te.item()), steps=e2e_steps)
        del psi_e2e, psi_host, out_host

    # ---- accuracy of this run against the FP64 oracle, and the oracle's own rate (rank 0)
    cpu = None
    err = None
    secondary = None
    if rank == 0 and not args.no_cpu_baseline:
        with tempfile.TemporaryDirectory() as td:
            if tio2:
                # the kernels on TiO2-shaped data: targets 0 and 5 against the first 8 occupied
                # orbitals of the bench block, GPU and oracle on the same float32 inputs
                occ8 = psi[:8]
                got = P.tx_exchange_apply(ctx, occ8, occ8[[0, 5]].contiguous()).double().cpu().numpy()
                ref, _, _, _ = run_oracle(s, occ8.cpu().numpy(), occ8[[0, 5]].cpu().numpy(), td)
                err_what = "targets 0 and 5 against the first 8 occupied orbitals of the block"
            else:
                ref, _, _, _ = run_oracle(s, s.psi, s.psi[[0, 37]], td)
                got = out[[0, 37]].double().cpu().numpy()
                err_what = "rows 0 and 37 of the timed run"
            err = dict(rel_frobenius=float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                       rel_max_abs=float(np.abs(got - ref).max() / np.abs(ref).max()), sample=err_what)
            so, occ_h, tgt_h, what = oracle_sample_system(args.workload)
            _, sec, pairs, cores = run_oracle(so, occ_h, tgt_h, td)
        cpu = dict(value=pairs / sec, unit="pairs/s", cores=cores, kind="oracle",
                   sample=f"{pairs} ordered pairs ({what}), {sec:.2f} s of FP64 numpy")
        if tio2 and not args.no_secondary:
            secondary = pt_secondary(P, W, dev, run_oracle)
            secondary["transfer"] = transfer_secondary(P, W, ctx, psi[:n_tgt], out, peaks)
            secondary["tio2_split_precision"] = tio2_split_secondary(P, s, psi, ref)
    if world > 1:
        dist.barrier()
    if rank == 0:
        fl = flops_per_pair(n, r, T) * unique
        line = dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=ms_max, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype=dtype_name(prec), data="synthetic",
                    config=dict(cfg, occupied=n_occ, targets=n_tgt, pairs_ordered=ordered, pairs_unique=unique,
                                precision=prec, expansion_form=args.expansion_form, l2=l2,
                                parallelism=f"replicas x{world}",
                                input_setup_s=round(setup_s, 1)),
                    unique_pair_potentials_per_s=world * unique / (ms_max / 1000.0),
                    algorithmic_tflops=world * fl / (ms_max / 1000.0) / 1e12,
                    algorithmic_frac_of_peak=(world * fl / (ms_max / 1000.0) / 1e12) / roof["peak"] if roof else None,
                    err_vs_oracle=err, roofline=roof, cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches),
                    kernels={k: dict(launches=v[0], ms_total=round(v[1], 4)) for k, v in prof.items()},
                    clocks=ck, secondary=secondary)
        if not tio2:
            line["energy"] = float(e.item())
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def batch_main(args, P, W, dev, prec, world, rank):
    """`--workload batch`: the uneven batch (16 systems, seed 100 + s: n in {48..112}, 8-128
    orbitals, ranks 20-48, 30-40 terms; every system applies K to all its orbitals), run as one
    batch plan whose expansion tile plans the autotuner picks, captured in one CUDA graph; the
    graph replay is timed.  Metric: ordered pair applications of all systems per second."""
    import tempfile as _tf
    import torch
    specs = W.batched_system_specs(16, 100)
    t0 = time.perf_counter()
    systems = []
    for sp in specs:
        a, kw = W.batched_system_args(sp)
        systems.append(W.make_system_on_device("batched", *a, device=dev, **kw))
    setup_s = time.perf_counter() - t0
    ctxs = [P.Context.from_system(s, precision=prec) for s, _ in systems]
    ordered = sum(psi.shape[0] ** 2 for _, psi in systems)
    unique = sum(psi.shape[0] * (psi.shape[0] + 1) // 2 for _, psi in systems)
    flops = sum(flops_per_pair(s.n[0], s.r[0], s.T) * psi.shape[0] * (psi.shape[0] + 1) // 2 for s, psi in systems)
    with _tf.TemporaryDirectory() as td:
        t1 = time.perf_counter()
        plan = P.BatchPlan([dict(ctx=c, psi_occ=psi) for c, (_, psi) in zip(ctxs, systems)],
                           tune_table=os.path.join(td, "tune.txt"), autotune=True)
        tune_s = time.perf_counter() - t1
    stream = torch.cuda.Stream()
    plan.capture(stream)
    for _ in range(max(3, args.warmup)):
        plan.replay(stream)
    stream.synchronize()
    for c in ctxs:
        c.check_device_error()
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    steps = args.steps or 3
    torch.cuda.synchronize()
    a0.record(stream)
    for _ in range(steps):
        plan.replay(stream)
    a1.record(stream)
    stream.synchronize()
    ck = clocks.stop()
    for c in ctxs:
        c.check_device_error()
    ms = a0.elapsed_time(a1) / steps
    # for comparison: the same systems as separate calls, one after another on one stream
    outs = [torch.empty_like(psi) for _, psi in systems]
    with torch.cuda.stream(stream):
        for rep in range(2):
            if rep == 1:
                a0.record(stream)
            for c, (_, psi), o in zip(ctxs, systems, outs):
                P.tx_exchange_apply(c, psi, out=o, stream=stream)
        a1.record(stream)
    stream.synchronize()
    seq_ms = a0.elapsed_time(a1)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    tfs = flops / (ms / 1e3) / 1e12
    peak = (peaks or {}).get("bf16_tflops_sustained")
    line = dict(metric=METRIC, value=world * ordered / (ms / 1e3), unit="pairs/s", n_gpus=world, steps=steps,
                warmup=max(3, args.warmup), ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype=dtype_name(prec), data="synthetic",
                config=dict(workload="uneven batch of 16 systems", systems=[
                    dict(n=sp["n"], orbitals=sp["n_orb"], rank=sp["rank"], terms=sp["T"]) for sp in specs],
                    pairs_ordered=ordered, pairs_unique=unique, precision=prec, graph="one captured graph, replayed",
                    l2="inputs larger than L2", parallelism=f"replicas x{world}", input_setup_s=round(setup_s, 1),
                    autotune_s=round(tune_s, 1)),
                algorithmic_tflops=tfs, algorithmic_frac_of_peak=(tfs / peak) if peak else None,
                tile_plans=[list(plan.item_plan(i)) for i in range(len(ctxs))], clocks=ck,
                sequential_calls_ms=seq_ms,
                roofline=None, cpu_baseline=None, e2e=None, gpu_launches=None)
    plan.destroy()
    if rank == 0:
        print(json.dumps(line))
    return 0


def transfer_secondary(P, W, ctx, psi_s, out_s, peaks):
    """The transfer between an unstructured finite-element mesh and the structured grid (Eq.
    interpolate) at the TiO2 shape: a hexahedral mesh of [-16, 16]^3 (8^3 cells of 4 bohr, each
    cell within 2 bohr of one of the 240 rutile-like centres split in eight, order-2 Lagrange
    nodes) and the 160^3 grid with order-3 elements, for the 256 target orbitals; both directions
    timed (CUDA events, 3 repetitions after a warm-up).  Algorithmic bytes: each orbital value on
    the mesh once, each grid value the direction touches once (all of them to the grid; those of
    the grid elements holding mesh nodes back to the mesh), plus the stored map."""
    import numpy as np
    import torch
    pu, ps = 2, 3
    X, conn = W.fe_mesh(16.0, 8, W.rutile_cluster(240), 2.0, pu)
    tr = P.Transfer(ctx, X, conn, pu, ps)
    n_orb = psi_s.shape[0]
    n_grid = psi_s[0].numel()
    psi_u = torch.empty((X.shape[0], n_orb), dtype=torch.float32, device=psi_s.device)
    res = {}
    # grid values the reverse transfer reads: the nodes of the grid elements holding mesh nodes
    xs = [np.linspace(-16.0, 16.0, k) for k in ctx.n]
    touched = np.zeros(ctx.n, dtype=bool)
    el = [np.searchsorted(xs[d][ps::ps][:-1], X[:, d], side="left") for d in range(3)]
    for ex, ey, ez in set(zip(*el)):
        touched[ps * ex: ps * ex + ps + 1, ps * ey: ps * ey + ps + 1, ps * ez: ps * ez + ps + 1] = True
    nb, ns = (pu + 1) ** 3, (ps + 1) ** 3
    u_bytes = X.shape[0] * n_orb * 4
    bytes_of = {"mesh_to_grid": u_bytes + n_grid * n_orb * 4 + 4 * (conn.shape[0] + 1) + 4 * n_grid * (1 + nb)
                + 4 * conn.size,
                "grid_to_mesh": u_bytes + int(touched.sum()) * n_orb * 4 + 4 * X.shape[0] * (1 + ns)}
    hbm = (peaks or {}).get("hbm_gbs")
    for name, fn in (("grid_to_mesh", lambda: tr.s_to_u(psi_s, out=psi_u)),
                     ("mesh_to_grid", lambda: tr.u_to_s(psi_u, out=out_s))):
        fn()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(3):
            fn()
        a1.record()
        torch.cuda.synchronize()
        ms = a0.elapsed_time(a1) / 3
        gbs = bytes_of[name] / (ms / 1e3) / 1e9
        res[name] = dict(ms=ms, algorithmic_bytes=int(bytes_of[name]), achieved_gbs=gbs,
                         frac_of_hbm=(gbs / hbm) if hbm else None)
    tr.destroy()
    return dict(mesh_nodes=int(X.shape[0]), mesh_cells=int(conn.shape[0]), orbitals=int(n_orb), order_mesh=pu,
                order_grid=ps, hbm_peak_gbs=hbm, peak_source="measured" if hbm else None, results=res)


def pt_secondary(P, W, dev, run_oracle_fn):
    """The Pt-shaped block (96^3, 64 orbitals, rank 40, 40 terms; one tx_exchange_apply_energy of
    all 64 against all 64 per step) in bf16, the split-precision tf32x3 form and the float32
    CUDA-core form: rate and error of row 0 against the oracle."""
    import numpy as np
    import torch
    s = W.config_pt()
    psi = torch.from_numpy(s.psi).to(dev)
    out = torch.empty_like(psi)
    e = torch.empty((), dtype=torch.float64, device=dev)
    with tempfile.TemporaryDirectory() as td:
        ref, _, _, _ = run_oracle_fn(s, s.psi, s.psi[0:1], td)
    res = {}
    for prec, steps in (("bf16", 5), ("tf32x3", 2), ("fp32", 2)):
        ctx = P.Context.from_system(s, precision=prec)
        for _ in range(3):
            P.tx_exchange_apply_energy(ctx, psi, out=out, e_out=e)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(steps):
            P.tx_exchange_apply_energy(ctx, psi, out=out, e_out=e)
        a1.record()
        torch.cuda.synchronize()
        ctx.check_device_error()
        ms = a0.elapsed_time(a1) / steps
        got = out[0:1].double().cpu().numpy()
        res[prec] = dict(value=64 * 64 / (ms / 1000.0), unit="pairs/s", ms_per_step=ms, steps=steps,
                         err_vs_oracle=float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        if prec == "fp32":
            # the same block with per-pair Tucker bases (sequentially truncated HOSVD of every pair
            # density, float32): one warm-up and one timed apply
            P.tx_exchange_apply_sthosvd(ctx, psi, out=out)
            torch.cuda.synchronize()
            a0.record()
            P.tx_exchange_apply_sthosvd(ctx, psi, out=out)
            a1.record()
            torch.cuda.synchronize()
            ctx.check_device_error()
            ms = a0.elapsed_time(a1)
            res["fp32_per_pair_bases"] = dict(value=64 * 64 / (ms / 1000.0), unit="pairs/s", ms_per_step=ms, steps=1)
        ctx.destroy()
    return dict(workload="Pt-cluster-shaped block", n=96, orbitals=64, rank=40, terms=40,
                err_sample="row 0 against all 64 orbitals", results=res)


def tio2_split_secondary(P, s, psi, ref, n_occ=64, n_tgt=16):
    """The split precision (TF32x3: y/z items, one 128-row y tile and half the z columns per CTA)
    and the float32 CUDA-core form on the TiO2-shaped block: n_tgt targets against the first n_occ
    occupied orbitals (one warm-up and two timed applies), and targets 0 and 5 against the first 8
    occupied orbitals against the oracle's rows (`ref`)."""
    import numpy as np
    import torch
    occ, tgt = psi[:n_occ], psi[:n_tgt]
    out = torch.empty_like(tgt)
    res = {}
    for prec in ("tf32x3", "fp32"):
        ctx = P.Context.from_system(s, precision=prec)
        P.tx_exchange_apply(ctx, occ, tgt, out=out)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        for _ in range(2):
            P.tx_exchange_apply(ctx, occ, tgt, out=out)
        a1.record()
        torch.cuda.synchronize()
        ms = a0.elapsed_time(a1) / 2
        occ8 = psi[:8]
        got = P.tx_exchange_apply(ctx, occ8, occ8[[0, 5]].contiguous()).double().cpu().numpy()
        ctx.check_device_error()
        res[prec] = dict(value=n_occ * n_tgt / (ms / 1000.0), unit="pairs/s", ms_per_call=ms, calls=2,
                         rel_max_abs=float(np.abs(got - ref).max() / np.abs(ref).max()),
                         rel_frobenius=float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        ctx.destroy()
    return dict(sample=f"{n_tgt} targets against the first {n_occ} occupied orbitals of the block; error: "
                       "targets 0 and 5 against the first 8", results=res)


def dtype_name(prec):
    return {"fp32": "f32", "bf16": "bf16", "tf32": "tf32", "tf32x3": "tf32x3", "bf16x3": "bf16x3"}.get(prec, prec)


# DRAM bytes (read + write) per distinct pair of the dominant kernel, from one ncu capture of
# the current kernel on a smaller case of the same shape (traffic grows in proportion to the
# pairs), scaled by the pairs a bench launch processes.  Keyed by (kernel, precision, workload);
# None where no capture of the current kernel exists.
# DRAM read + write bytes per distinct pair of the dominant kernel, from one ncu capture of the
# same kernel (same tile plan) on the TiO2-shaped block cut to 8 targets x 24 occupied orbitals
# (164 distinct pairs in one launch: 22.16 GB read, 1.95 GB written); the kernel streams each
# pair's Z, orbitals and W the same way at any block size, so the bytes scale with the pairs.
DRAM_BYTES_PER_PAIR = {("tc_consume", "bf16", "tio2"): (22.163e9 + 1.954e9) / 164}


def roofline(dom, prof, n, r, T, unique, steps, prec, peaks, ck, workload="pt"):
    """Achieved algorithmic FLOP/s of the dominant kernel over its live launch time."""
    if dom is None:
        return None
    k, kms = prof[dom]
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
    bpp = DRAM_BYTES_PER_PAIR.get((dom, prec, workload))
    traffic = bpp * unique * steps / k if bpp else None     # bytes per launch
    return dict(kernel=dom, bound=bound, achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                traffic=traffic, traffic_unit="bytes per launch (ncu dram read + write, scaled)" if traffic else None,
                launches=k, avg_launch_ms=kms / k, peak_source=src)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python3
"""Benchmark of the DMRG3S hot path on one GB300 (or N independent replicas).

Headline (``value``): algorithmic TFLOP/s of the single-site effective
Hamiltonian application HA = L W A R (Sec. V of arXiv:1501.05504, order
(((L A) W) R)), the operation the Lanczos eigensolver repeats, on the largest
dense contraction of the workloads: the central site of the S=1/2 Heisenberg
model on the 4 x 16 cylinder (snake order, periodic in width, w = 14, U(1)
S^z) at m = 2048, in 3xTF32 with FP64 data, one application of the prepared
operator (dmrg3s_heff_apply) per step with L2 flushed.  ``roofline`` is the
tensor-core kernel's share against the measured TF32 peak; ``e2e`` repeats the
product through the C ABI from pinned host buffers.  Secondary fields: one
full local update on the XXZ L = 100, m = 512 window (``local_update``), the
sweep-to-1e-9 time of the mixed-precision ladder against FP64 (``sweep``),
and the batched-chain workload (``batch``: XXZ chains solved together, with
their coupling derivatives).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same H_eff on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402

WORKLOAD = "xxz_l100_m512_u1"
M_MAX = 512
ALPHA = 1e-2
SEED = 1002


def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def window_specs(seed=SEED):
    """Neutral specs of the central window (sites 50, 51 of the L = 100 chain)."""
    rng = si.rng_for(seed)
    b0, b1 = si.central_bonds(WORKLOAD)                      # bonds 49 (odd charges) and 50 (even)
    b2 = si.gaussian_bond(M_MAX, (1,), (3.0,), (2,), (6,))    # bond 51 (odd)
    Le = si.symmetric_env(rng, si.XXZ_T, b0, identity_channels=(4,))
    Re = si.symmetric_env(rng, si.XXZ_T, b2, identity_channels=(0,))
    M0 = si.random_site(rng, si.XXZ_QP, b0, b1)
    M1 = si.random_site(rng, si.XXZ_QP, b1, b2)
    return {"L": Le, "R": Re, "M": [M0, M1], "bonds": [b0, b1, b2]}


def heff_flops(qp, t, W, left, right, tr=None):
    """Algorithmic flops of one block-sparse H_eff application, order (((L A) W) R).

    t: channel charges of the left MPO bond; tr: of the right one (default t)."""
    tr = t if tr is None else tr
    def find(b, q):
        hit = np.nonzero(np.all(b["q"] == q[None, :], axis=1))[0]
        return int(hit[0]) if len(hit) else -1
    f = 0.0
    t2 = {}
    for bl in range(t.shape[0]):
        for ik in range(len(left["dim"])):
            ib = find(left, left["q"][ik] + t[bl])
            if ib < 0:
                continue
            for s in range(qp.shape[0]):
                j = find(right, left["q"][ik] + qp[s])
                if j < 0:
                    continue
                rows, cols, K = left["dim"][ib], right["dim"][j], left["dim"][ik]
                f += 2.0 * rows * cols * K                            # stage 1
                for so in range(qp.shape[0]):
                    for br in range(t.shape[0]):
                        if W[so, s, bl, br] != 0.0:
                            f += 2.0 * rows * cols                  # stage 2 term
                            t2[(br, so, ib, j)] = (rows, cols)
    for (br, so, ib, j), (rows, cols) in t2.items():
        jp = find(right, right["q"][j] + tr[br])
        if jp >= 0:
            f += 2.0 * rows * right["dim"][jp] * cols                 # stage 3
    return f


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.samples = []
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        for ln in out.splitlines():
            p = [x.strip() for x in ln.split(",")]
            if len(p) >= 9:
                self.samples.append(p)

    def summary(self):
        if not getattr(self, "samples", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(p[1]) for p in self.samples if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for p in self.samples if p[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for p in self.samples for k in range(4) if p[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


PEAKS_FILE = os.path.join(ROOT, "profiles", "peaks_tf32_fp64_gb300.json")


def peaks():
    """Roofline denominators, TFLOP/s.  bf16 and HBM: MEASURED_PEAKS.json (the
    driver's measurement on this machine); tf32 and fp64: the cuBLAS measurement
    committed by `bench.py --measure-peaks` (profiles/peaks_tf32_fp64_gb300.json)
    when present, else the bf16 figure times the datasheet ratio."""
    mp = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mp = json.load(f)
    bf16 = mp.get("bf16_tflops")
    src = "measured"
    if bf16 is None:
        bf16, src = 1900.0, "fallback"
    out = {"bf16": bf16, "hbm": mp.get("hbm_gbs") or 6800.0, "source": src}
    pf = {}
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as f:
            pf = json.load(f)
    if pf.get("tf32_tflops"):
        out["tf32"] = pf["tf32_tflops"]
        t_note = "of measured cuBLAS TF32 (%s)" % os.path.relpath(PEAKS_FILE, ROOT)
    else:
        out["tf32"] = bf16 * 1.1 / 2.25
        t_note = "of %s bf16 x nominal tf32/bf16 ratio 1.1/2.25" % src
    if pf.get("fp64_tflops"):
        out["fp64"] = pf["fp64_tflops"]
        d_note = "of measured cuBLAS DGEMM (%s)" % os.path.relpath(PEAKS_FILE, ROOT)
    else:
        out["fp64"] = bf16 * 1.25e-3 / 2.25
        d_note = "of %s bf16 x nominal fp64/bf16 ratio" % src
    out["note_tf32"] = t_note
    out["note_tf32x3"] = t_note + ", divided by 3 for the three products"
    out["note_fp64"] = d_note
    return out


def measure_peaks():
    """cuBLAS TF32 and FP64 GEMM throughput on this GPU (torch.matmul), burst
    (best of 10) and sustained (back to back for ~3 s), written to PEAKS_FILE."""
    import torch
    res = {"how": "torch.matmul: fp32 8192^3 with TF32 allowed (2 N^3 flops), fp64 8192^3; "
                  "burst = best of 10, sustained = back to back for about 3 s (CUDA events)"}
    torch.backends.cuda.matmul.allow_tf32 = True
    for key, dt in (("tf32", torch.float32), ("fp64", torch.float64)):
        n = 8192
        a = torch.randn(n, n, dtype=dt, device="cuda")
        bm = torch.randn(n, n, dtype=dt, device="cuda")
        for _ in range(3):
            torch.matmul(a, bm)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, bm)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        per = best * 1e-3
        reps = max(3, int(3.0 / per))
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                torch.matmul(a, bm)
            e1.record()
            torch.cuda.synchronize()
        sus = e0.elapsed_time(e1) * 1e-3 / reps
        f = 2.0 * n ** 3
        res[key + "_tflops"] = f / per / 1e12
        res[key + "_tflops_sustained"] = f / sus / 1e12
        res[key + "_clocks"] = clk.summary()
        del a, bm
        torch.cuda.empty_cache()
    res["gpu"] = torch.cuda.get_device_name()
    res["torch"] = torch.__version__
    with open(PEAKS_FILE, "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")
    return res


def traffic_for(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    ent = t.get(kernel)
    if not ent:
        return None
    # counters taken on another version of the kernel's source are not reported
    src = os.path.join(ROOT, ent.get("source", ""))
    if not os.path.exists(src):
        return None
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != ent.get("source_sha256"):
            return None
    return ent.get("bytes_per_launch")


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (the slowest replica's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(flops_per_step, world, ms_per_step):
    """Whole-job TFLOP/s of `world` independent replicas, each doing flops_per_step
    per step, timed by the slowest one (ms_per_step)."""
    return flops_per_step * world / (ms_per_step * 1e-3) / 1e12


def local_update_field(args, b, ctx, rank=0, world=1):
    """One DMRG3S local update on the central two-site window of the XXZ L = 100,
    m = 512 chain (Sec. V steps 1-7), timed per update with the L2 flushed;
    phase times from the library's event profiler."""
    import torch
    spec = window_specs(SEED + rank)
    mpo = b.Mpo(b.MODEL_XXZ, 100, (1.0, 1.0))
    W = [mpo.site(50), mpo.site(51)]
    opts = b.update_opts(M_MAX, kmax=40, tol=1e-10, prec=args.precision, svd=args.svd)
    gL, gR = b.env_from_neutral(spec["L"]), b.env_from_neutral(spec["R"])
    gM = [b.site_from_neutral(x) for x in spec["M"]]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    times, iters, sweeps, fallbacks = [], [], [], 0
    phases = None
    nsteps = max(args.update_steps, 1)
    # every timed update starts from the same fresh window (the first update
    # of a sweep over it), so the work does not shrink as a re-updated window
    # would converge
    for k in range(args.warmup + nsteps):
        st = b.dmrg3s_state_create(ctx, W, gM, gL, gR, 0)
        if k == args.warmup:
            b.dmrg3s_profile(ctx, True)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = b.dmrg3s_local_update(st, 1, ALPHA, opts)
        e1.record(stream)
        torch.cuda.synchronize()
        st.close()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
            iters.append(info["lanczos_iters"])
            sweeps.append(info["svd_sweeps"])
            fallbacks += int(info["svd_fallback"])
    g = b.dmrg3s_profile_read(ctx, b.KERNEL_GEMM)
    cmb = b.dmrg3s_profile_read(ctx, b.KERNEL_COMBINE)
    phases = {name: b.dmrg3s_profile_read(ctx, kk)["ms"] / nsteps
              for kk, name in enumerate(["eigensolver", "expansion", "svd_truncation", "remainder",
                                         "environment", "energy"], start=2)}
    b.dmrg3s_profile(ctx, False)
    ms = max_over_ranks(statistics.mean(times), world, "cuda")
    flops = (g["flops"] + cmb["flops"]) / nsteps
    return {"workload": "xxz_l100_m512_u1 central two-site window (sites 50, 51), one local "
                        "update (left-to-right) of a fresh window per step",
            "ms_per_update": ms, "tflops": replica_value(flops, world, ms),
            "flops_per_update": flops, "steps": nsteps, "precision": args.precision,
            "svd": args.svd, "lanczos_iters": iters, "svd_jacobi_sweeps": sweeps,
            "svd_fallbacks": fallbacks, "phase_ms_per_update": phases,
            "gemm_share": g["ms"] / nsteps / ms if ms else None,
            "l2": "flushed (256 MB write) before every timed update"}


def run_ours(args):
    """The headline line: H_eff.A on the central site of a workload (default the
    4 x 16 cylinder at m = 2048), repeated applications timed one by one with
    the L2 flushed in between, plus the local-update and sweep-to-1e-9 fields."""
    import torch
    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_1501_05504_gb300 import binding as b
    dev = torch.cuda.current_device()
    ctx = b.dmrg3s_create(dev, int(args.workspace_gb * (1 << 30)))
    name = args.workload
    W0, gL, gR0, gM0 = heff_problem(b, name, args.workload_m, seed_offset=rank)
    gH = b.empty_site_like(gM0.qp, gM0.left, gM0.right)
    flops_heff, bytes_heff = b.dmrg3s_heff_cost(gL, W0, gR0, gM0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    prec = args.precision
    # the operator of one local eigenproblem, prepared once (environments
    # packed) and applied to a new vector every step, as in the Lanczos loop
    op = b.HeffOp(ctx, gL, W0, gR0, gM0, prec)
    for _ in range(args.warmup):
        op.apply(gM0, gH)
    b.dmrg3s_sync(ctx)
    # ---- device-resident timed region: K applications, L2 flushed before each
    b.dmrg3s_profile(ctx, True)
    n0 = b.dmrg3s_launch_count()
    times = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            op.apply(gM0, gH)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    b.dmrg3s_sync(ctx)
    launches = b.dmrg3s_launch_count() - n0 - 0
    g = b.dmrg3s_profile_read(ctx, b.KERNEL_GEMM)
    cmb = b.dmrg3s_profile_read(ctx, b.KERNEL_COMBINE)
    b.dmrg3s_profile(ctx, False)
    total_ms = max_over_ranks(sum(times), world, "cuda")
    ms_step = total_ms / args.steps
    value = replica_value(flops_heff, world, ms_step)
    pk = peaks()
    kpeak = {"fp64": pk["fp64"], "tf32x3": pk["tf32"] / 3.0, "tf32": pk["tf32"]}[prec]
    achieved = g["flops"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else None
    kname = "gemm_f64_kernel" if prec == "fp64" else "gemm_tc_kernel"
    roofline = {"kernel": kname, "bound": "alu" if prec == "fp64" else "tensor",
                "achieved": achieved, "peak": kpeak, "unit": "TFLOP/s",
                "frac": achieved / kpeak if achieved else None,
                "traffic": traffic_for(kname), "launches": g["launches"],
                "avg_launch_us": 1e3 * g["ms"] / max(g["launches"], 1),
                "peak_source": pk["note_" + prec],
                "share_of_step": g["ms"] / total_ms if total_ms else None}
    if prec != "fp64" and achieved:
        roofline["frac_of_plain_tf32"] = achieved / pk["tf32"]
    whole = {"achieved": value / world, "frac_of_peak": (value / world) / kpeak,
             "note": "whole H_eff application (vector pack, all stages, split-K sum) against "
                     "the same peak"}
    # one-shot dmrg3s_apply_heff (plans cached, environments packed in every call)
    one = []
    for _ in range(max(3, args.steps // 4)):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.dmrg3s_apply_heff(ctx, gL, W0, gR0, gM0, gH, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        one.append(e0.elapsed_time(e1))
    b.dmrg3s_sync(ctx)
    oneshot = {"ms": statistics.mean(one), "tflops": flops_heff / (statistics.mean(one) * 1e-3) / 1e12,
               "what": "dmrg3s_apply_heff: the same product with L and R packed in every call"}
    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        hL, hR, hA = (x.data.cpu().pin_memory() for x in (gL, gR0, gM0))
        hH = torch.empty(gH.data.numel(), dtype=torch.float64).pin_memory()
        bi = 8 * (hL.numel() + hR.numel() + hA.numel())
        bo = 8 * hH.numel()
        et = []
        for k in range(max(2, args.steps // 2)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gL.data.copy_(hL, non_blocking=True)
            gR0.data.copy_(hR, non_blocking=True)
            gM0.data.copy_(hA, non_blocking=True)
            b.dmrg3s_apply_heff(ctx, gL, W0, gR0, gM0, gH, prec)
            hH.copy_(gH.data, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            et.append(e0.elapsed_time(e1))
        ems = max_over_ranks(statistics.mean(et), world, "cuda")
        e2e = {"value": replica_value(flops_heff, world, ems), "unit": "TFLOP/s",
               "ms_per_step": ems, "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
               "what": "L, R and A copied in from pinned host memory, H_eff, HA copied out"}
    # ---- secondary fields: one local update, and the sweep-to-1e-9 arms
    op.close()
    upd = None if args.no_update else local_update_field(args, b, ctx, rank, world)
    ctx.close()
    sweep = None
    if not args.no_sweep and rank == 0 and world == 1:
        sweep = run_sweep(args)
    batch = None
    if not args.no_batch and rank == 0 and world == 1:
        batch = run_batch(args)
    if rank != 0:
        return None
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(args.cpu_sample_s, name,
                                                                        args.workload_m)
    sizes = {"sectors": [len(gM0.left.dim), len(gM0.right.dim)],
             "max_sector_dim": int(max(gM0.left.dim.max(), gM0.right.dim.max())),
             "m": int(sum(gM0.left.dim)), "w": int(W0.W.shape[2]), "d": int(W0.W.shape[0])}
    return {"metric": "Heff.A TFLOP/s (algorithmic block-sparse flops of one H_eff application)",
            "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "tf32x3": "tf32x3", "tf32": "tf32"}[prec],
            "data": "synthetic", "impl": "ours",
            "config": {"workload": HEFF_DESCR.get(name, name), "name": name,
                       "step": "one application of the prepared H_eff operator (dmrg3s_heff_apply) "
                               "to the site tensor",
                       "flops_per_heff": flops_heff, "bytes_per_heff": bytes_heff, **sizes,
                       "precision": prec, "inputs": "seeded symmetric environments and a random "
                       "site tensor on Gaussian charge-sector bonds (seeded_inputs.central_bonds)",
                       "l2": "flushed (256 MB write) before every timed application",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline, "heff_whole": whole, "heff_oneshot": oneshot, "cpu_baseline": cpu,
            "e2e": e2e,
            "local_update": upd, "sweep": sweep, "batch": batch, "gpu_launches": int(launches),
            "clocks": clk.summary()}


def cylinder_bonds(lx=16, ly=4):
    """Nearest-neighbour bonds of the lx x ly cylinder (periodic in y) in snake order."""
    def idx(x, y):
        return x * ly + (y if x % 2 == 0 else ly - 1 - y)
    bonds = set()
    for x in range(lx):
        for y in range(ly):
            if x + 1 < lx:
                bonds.add(tuple(sorted((idx(x, y), idx(x + 1, y)))))
            if ly > 2 or y + 1 < ly:
                bonds.add(tuple(sorted((idx(x, y), idx(x, (y + 1) % ly)))))
    return sorted(bonds)


HEFF_WORKLOADS = {
    # name: (model, sites, params, central site, seed)
    "xxz_l100_m512_u1": ("xxz", 100, (1.0, 1.0), 50, 1002),
    "hubbard_l64_m1024_u1u1": ("hubbard", 64, (1.0, 8.0), 32, 1003),
    "cylinder_4x16_m2048_u1": ("cylinder", 64, None, 32, 1004),
}
HEFF_DESCR = {
    "xxz_l100_m512_u1": "S=1/2 XXZ chain Delta=1, L=100, d=2, w=5, U(1) S^z, m=512, central site",
    "hubbard_l64_m1024_u1u1": "Fermi-Hubbard chain t=1 U=8 half filling, L=64, d=4, w=6, "
                              "U(1)xU(1) (N, S^z), m=1024, central site",
    "cylinder_4x16_m2048_u1": "S=1/2 Heisenberg J1 on the 4x16 cylinder (snake order, periodic "
                              "in width), d=2, w=14, U(1) S^z, m=2048, central site",
}


def heff_problem_specs(b, name, m=None, seed_offset=0):
    """Central-site H_eff problem of a workload: the library's MPO site, and
    seeded symmetric environments and a random site tensor (neutral specs) on
    the workload's bonds."""
    model, n, params, site, seed = HEFF_WORKLOADS[name]
    seed += seed_offset
    if model == "hubbard":
        mpo = b.Mpo(b.MODEL_HUBBARD, n, params)
    elif model == "xxz":
        mpo = b.Mpo(b.MODEL_XXZ, n, params)
    else:
        bonds = cylinder_bonds()
        mpo = b.Mpo(b.MODEL_SPIN_BONDS, n, (), bonds=bonds, couplings=[(1.0, 1.0)] * len(bonds))
    W = mpo.site(site)
    left, right = si.central_bonds(name, m)
    rng = si.rng_for(seed)
    Le = si.symmetric_env(rng, W.tl, left, identity_channels=(W.tl.shape[0] - 1,))
    Re = si.symmetric_env(rng, W.tr, right, identity_channels=(0,))
    M = si.random_site(rng, W.qp, left, right)
    return W, Le, Re, M


def heff_problem(b, name, m=None, seed_offset=0):
    W, Le, Re, M = heff_problem_specs(b, name, m, seed_offset)
    return W, b.env_from_neutral(Le), b.env_from_neutral(Re), b.site_from_neutral(M)


def run_heff_only(args):
    """Kernel view: repeated H_eff applications on a workload's central site."""
    import torch
    from paper_1501_05504_gb300 import binding as b
    ctx = b.dmrg3s_create(torch.cuda.current_device(), int(args.workspace_gb * (1 << 30)))
    W0, gL, gR0, gM0 = heff_problem(b, args.workload, args.workload_m)
    gH = b.empty_site_like(gM0.qp, gM0.left, gM0.right)
    for _ in range(args.warmup):
        b.dmrg3s_apply_heff(ctx, gL, W0, gR0, gM0, gH, args.precision)
    b.dmrg3s_sync(ctx)
    b.dmrg3s_profile(ctx, True)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(args.steps):
        b.dmrg3s_apply_heff(ctx, gL, W0, gR0, gM0, gH, args.precision)
    e1.record(s)
    b.dmrg3s_sync(ctx)
    g = b.dmrg3s_profile_read(ctx, b.KERNEL_GEMM)
    c = b.dmrg3s_profile_read(ctx, b.KERNEL_COMBINE)
    b.dmrg3s_profile(ctx, False)
    ms = e0.elapsed_time(e1) / args.steps
    flops = (g["flops"] + c["flops"]) / args.steps
    peak = peaks()
    pk = {"fp64": peak["fp64"], "tf32": peak["tf32"], "tf32x3": peak["tf32"] / 3.0}[args.precision]
    note = peak["note_" + args.precision]
    gemm_tf = g["flops"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else None
    ctx.close()
    return {"metric": "H_eff application on the %s central site (kernel view)" % args.workload,
            "m": int(sum(gM0.left.dim)),
            "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_heff": ms,
            "flops_per_heff": flops, "precision": args.precision, "w": int(W0.W.shape[2]),
            "d": int(W0.W.shape[0]), "sectors": [len(gM0.left.dim), len(gM0.right.dim)],
            "max_sector_dim": int(max(gM0.left.dim.max(), gM0.right.dim.max())),
            "gemm_ms_per_heff": g["ms"] / args.steps, "combine_ms_per_heff": c["ms"] / args.steps,
            "gemm_launches": g["launches"], "gemm_tflops": gemm_tf,
            "gemm_frac_of_peak": gemm_tf / pk if gemm_tf else None, "peak_tflops": pk,
            "peak_source": note, "l2": "not flushed (kernel view)"}


def cpu_baseline(sample_s=15.0, name="cylinder_4x16_m2048_u1", m=None):
    """The FP64 oracle on the host cores: H_eff of the workload's central site.

    The dense oracle product at the full size takes minutes, so the sample is
    the definition of H_eff evaluated for a set of output rows (left bra
    indices al', every 8th one or fewer) by oracle.contract.apply_heff_rows,
    repeated for about `sample_s` seconds; its algorithmic (block-sparse)
    flops are the workload's flops times the sampled fraction of rows."""
    from oracle import contract, io

    W, Le, Re, M = _oracle_problem(name, m)
    L, R, A = io.env_dense(Le), io.env_dense(Re), io.site_dense(M)[0]
    mtot = A.shape[1]
    nrow = max(1, min(mtot // 8, 64))
    rows = np.linspace(0, mtot - 1, nrow).astype(np.int64)
    left, right = si.central_bonds(name, m)
    flops = heff_flops(np.asarray(W["qp"]), np.asarray(W["tl"]), W["W"], left, right,
                       np.asarray(W["tr"]))
    t0 = time.time()
    n = 0
    while time.time() - t0 < sample_s or n == 0:
        contract.apply_heff_rows(L, W["W"], R, A, rows)
        n += 1
    dt = (time.time() - t0) / n
    frac = nrow / mtot
    return {"value": flops * frac / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "%d evaluations of H_eff on %d of the %d output rows of the %s central site "
                      "(dense FP64 einsum, %.2f s each); flops = the block-sparse count x %d/%d"
                      % (n, nrow, mtot, name, dt, nrow, mtot)}


def _oracle_problem(name, m=None):
    """The H_eff problem of `name` with the oracle's MPO builders (the same
    seeded environments and site tensor as heff_problem_specs)."""
    from oracle import models
    model, n, params, site, seed = HEFF_WORKLOADS[name]
    if model == "hubbard":
        mpo = models.mpo_hubbard(n, *params)
    elif model == "xxz":
        mpo = models.mpo_xxz(n, *params)
    else:
        bonds = [(i, j, 1.0, 1.0) for (i, j) in cylinder_bonds()]
        mpo = models.mpo_spin_bonds(n, bonds, 1)
    W = {"W": mpo.W[site], "qp": mpo.qphys, "tl": mpo.t[site], "tr": mpo.t[site + 1]}
    left, right = si.central_bonds(name, m)
    rng = si.rng_for(seed)
    Le = si.symmetric_env(rng, W["tl"], left, identity_channels=(W["tl"].shape[0] - 1,))
    Re = si.symmetric_env(rng, W["tr"], right, identity_channels=(0,))
    M = si.random_site(rng, W["qp"], left, right)
    return W, Le, Re, M


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return None
    t0 = time.time()
    name = getattr(args, "workload", "cylinder_4x16_m2048_u1")
    cb = cpu_baseline(max(args.cpu_sample_s, 1.0) * max(args.steps, 1) / 10.0, name,
                      getattr(args, "workload_m", None))
    return {"metric": "Heff.A TFLOP/s (algorithmic block-sparse flops of one H_eff application)",
            "value": cb["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": HEFF_DESCR.get(name, name) + " (oracle sample)", "name": name},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "TFLOP/s",
                                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.time() - t0}


SWEEP_MODELS = {
    # name: (library model, parameters, local start state pattern, description)
    "xxz": ("MODEL_XXZ", (1.0, 1.0), [0, 1], "S=1/2 XXZ chain Delta=1, d=2, w=5, U(1) S^z"),
    "hubbard": ("MODEL_HUBBARD", (1.0, 8.0), [2, 1],
                "Fermi-Hubbard chain t=1, U=8, half filling, d=4, w=6, U(1)xU(1) (N, S^z)"),
    "cylinder": ("MODEL_SPIN_BONDS", None, [0, 1],
                 "S=1/2 Heisenberg J1 on the 4 x L/4 cylinder (snake order, periodic in width), "
                 "d=2, w=14, U(1) S^z"),
}


def _sweep_run(b, ctx, L, m_max, ladder, model="xxz", max_sweeps=24, svd="gesvd"):
    """Sweeps from a product state (Neel / alternating up-down) in one
    dmrg3s_sweep call: ladder = [(precision, until)] as for the library's
    precision ladder (one or two rungs; the last runs until the sweep-to-sweep
    change is below 1e-11).  Returns per-sweep (wall seconds since the call
    started, energy, precision)."""
    import torch
    lib_model, params, pattern, _ = SWEEP_MODELS[model]
    if model == "cylinder":
        bonds = cylinder_bonds(L // 4, 4)
        W = b.Mpo(b.MODEL_SPIN_BONDS, L, (), bonds=bonds, couplings=[(1.0, 1.0)] * len(bonds)).sites()
    else:
        W = b.Mpo(getattr(b, lib_model), L, params).sites()
    st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, pattern * (L // 2)), None, None,
                               L - 1)
    torch.cuda.synchronize()
    opts = b.update_opts(m_max, prec=ladder[0][0], svd=svd)
    if len(ladder) > 1:
        rep = b.dmrg3s_sweep(st, b.alpha_rule(ALPHA), max_sweeps, 1e-11, opts,
                             final_prec=ladder[1][0], switch_tol=ladder[0][1])
    else:
        rep = b.dmrg3s_sweep(st, b.alpha_rule(ALPHA), max_sweeps, 1e-11, opts)
    st.close()
    nb = rep["bulk_sweeps"] if len(ladder) > 1 else rep["sweeps"]
    log = [(t, e, ladder[0][0] if k < nb else ladder[-1][0])
           for k, (t, e) in enumerate(zip(rep["seconds"], rep["energies"]))]
    return log, {"lanczos_iters": rep["lanczos_iters"], "svd_fallbacks": rep["svd_fallbacks"]}


def run_sweep(args):
    """Sweep-to-1e-9 time on one GB300: a mixed ladder (3xTF32 block products
    until the energy changes by < 1e-7 per sweep, then FP64 until < 1e-11)
    against all-FP64 (until < 1e-11),
    both timed to the first sweep whose energy is within 1e-9 (relative) of
    the converged FP64 energy."""
    import torch
    from paper_1501_05504_gb300 import binding as b
    ctx = b.dmrg3s_create(torch.cuda.current_device(), 1 << 30)
    L, m_max, model = args.sweep_sites, args.sweep_m, args.sweep_model
    nmax = args.sweep_max
    fp64, st64 = _sweep_run(b, ctx, L, m_max, [("fp64", 1e-11)], model, nmax, svd=args.svd)
    mixed, stmx = _sweep_run(b, ctx, L, m_max, [("tf32x3", 1e-7), ("fp64", 1e-11)], model, nmax,
                             svd=args.svd)
    e_ref = min(fp64[-1][1], mixed[-1][1])

    def first(log):
        for t, e, _ in log:
            if abs(e - e_ref) <= 1e-9 * abs(e_ref):
                return t
        return None
    t64, tmix = first(fp64), first(mixed)
    ctx.close()
    return {"metric": "sweep-to-1e-9 time, mixed vs FP64 (DMRG3S from a product state)",
            "value": tmix, "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "fp64_s": t64, "speedup_vs_fp64": (t64 / tmix) if (t64 and tmix) else None,
            "energy_ref": e_ref, "energy_fp64": fp64[-1][1], "energy_mixed": mixed[-1][1],
            "sweeps_fp64": [[round(t, 3), e, p] for t, e, p in fp64],
            "sweeps_mixed": [[round(t, 3), e, p] for t, e, p in mixed],
            "stats_fp64": st64, "stats_mixed": stmx,
            "config": {"workload": "%s_l%d_m%d full sweeps" % (model, L, m_max),
                       "hamiltonian": "%s, L=%d" % (SWEEP_MODELS[model][3], L),
                       "m_max": m_max, "alpha0": ALPHA, "lanczos_kmax": 40, "lanczos_tol": 1e-10,
                       "start": "product state %s..., m=1" % SWEEP_MODELS[model][2],
                       "svd": args.svd, "max_sweeps_per_arm": nmax,
                       "ladder": "library precision ladder (dmrg3s_sweep): 3xTF32 until the "
                                 "sweep-to-sweep change < 1e-7, then FP64"},
            "data": "synthetic"}


def run_lanczos(args):
    """Lanczos iteration time: dmrg3s_eigensolve on a workload's central site
    with a tolerance it cannot reach, so that exactly k iterations run (wall
    time / k, profiler off), beside the time of one prepared H_eff product."""
    import torch
    from paper_1501_05504_gb300 import binding as b
    ctx = b.dmrg3s_create(torch.cuda.current_device(), int(args.workspace_gb * (1 << 30)))
    W, Le, Re, M0 = heff_problem_specs(b, args.workload, args.workload_m)
    gL, gR = b.env_from_neutral(Le), b.env_from_neutral(Re)
    stream = torch.cuda.current_stream()
    out = {}
    for prec in [args.precision]:
        gM, gH = b.site_from_neutral(M0), b.site_from_neutral(M0)
        op = b.HeffOp(ctx, gL, W, gR, gM, prec)
        for _ in range(args.warmup):
            op.apply(gM, gH)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            op.apply(gM, gH)
        e1.record(stream)
        torch.cuda.synchronize()
        heff_us = 1e3 * e0.elapsed_time(e1) / 20
        op.close()
        per = {}
        for k in args.lanczos_k:
            ts = []
            for r in range(args.warmup + args.steps):
                gM = b.site_from_neutral(M0)
                torch.cuda.synchronize()
                t = time.perf_counter()
                _, it = b.dmrg3s_eigensolve(ctx, gL, W, gR, gM, kmax=k, tol=1e-30, prec=prec)
                torch.cuda.synchronize()
                if r >= args.warmup:
                    ts.append((time.perf_counter() - t) / it)
            per[str(k)] = 1e6 * min(ts)
        out[prec] = {"heff_us": heff_us, "us_per_iteration": per}
    ctx.close()
    return {"metric": "Lanczos iteration time (us) on the central site", "unit": "us",
            "higher_is_better": False, "results": out,
            "config": {"workload": HEFF_DESCR.get(args.workload, args.workload), "name": args.workload,
                       "m": args.workload_m, "steps": args.steps, "warmup": args.warmup,
                       "what": "best of the timed runs; the graph-captured iteration (profiler off)"},
            "data": "synthetic"}


def run_batch(args):
    """Batched chains: the first --batch-chains chains of the 64-chain XXZ
    workload (seeded_inputs.batch_xxz_chains, seed 1005) swept together from
    Neel states by one dmrg3s_sweep_batch call (every local-update step of all
    chains in shared launches), to |dE|/|E| < 1e-9 between two sweeps, then
    dE/dJ and dE/dDelta of every chain (dmrg3s_energy_grad).  chains_per_s =
    chains solved (sweeps and gradients) per second of wall time."""
    import torch
    import seeded_inputs as si
    from paper_1501_05504_gb300 import binding as b
    ctx = b.dmrg3s_create(torch.cuda.current_device(), int(args.workspace_gb * (1 << 30)))
    chains = si.batch_xxz_chains()[:args.batch_chains]
    states = []
    for c in chains:
        W = b.Mpo(b.MODEL_XXZ, c["L"], (c["J"], c["Delta"])).sites()
        states.append(b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [0, 1] * (c["L"] // 2)),
                                            None, None, c["L"] - 1))
    mixed = args.batch_prec == "mixed"
    opts = [b.update_opts(c["m_max"], prec="tf32x3" if mixed else "fp64", svd=args.svd)
            for c in chains]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if mixed:
        reps = b.dmrg3s_sweep_batch(states, b.alpha_rule(ALPHA), args.batch_sweeps, 1e-9, opts,
                                    final_prec="fp64", switch_tol=1e-7)
    else:
        reps = b.dmrg3s_sweep_batch(states, b.alpha_rule(ALPHA), args.batch_sweeps, 1e-9, opts)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    grads = [b.dmrg3s_energy_grad(st, b.MODEL_XXZ, (c["J"], c["Delta"])) for st, c in zip(states, chains)]
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for st in states:
        st.close()
    seq = None
    if args.batch_compare:      # the same chains one at a time (dmrg3s_sweep), for comparison
        ts = time.perf_counter()
        for c, o in zip(chains, opts):
            W = b.Mpo(b.MODEL_XXZ, c["L"], (c["J"], c["Delta"])).sites()
            st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, [0, 1] * (c["L"] // 2)),
                                       None, None, c["L"] - 1)
            if mixed:
                b.dmrg3s_sweep(st, b.alpha_rule(ALPHA), args.batch_sweeps, 1e-9, o,
                               final_prec="fp64", switch_tol=1e-7)
            else:
                b.dmrg3s_sweep(st, b.alpha_rule(ALPHA), args.batch_sweeps, 1e-9, o)
            b.dmrg3s_energy_grad(st, b.MODEL_XXZ, (c["J"], c["Delta"]))
            st.close()
        torch.cuda.synchronize()
        seq = time.perf_counter() - ts
    ctx.close()
    n = len(chains)
    return {"metric": "batched chains solved per second (sweeps to 1e-9 and dE/dJ, dE/dDelta)",
            "value": n / (t2 - t0), "unit": "chains/s", "higher_is_better": True,
            "chains": n, "sweep_s": t1 - t0, "gradient_s": t2 - t1,
            "sequential_s": seq, "speedup_vs_sequential": (seq / (t2 - t0)) if seq else None,
            "converged": int(sum(r["converged"] for r in reps)),
            "sweeps": [r["sweeps"] for r in reps], "lanczos_iters": [r["lanczos_iters"] for r in reps],
            "energies": [r["energy"] for r in reps],
            "dE_dJ": [float(g[1][0]) for g in grads], "dE_dDelta": [float(g[1][1]) for g in grads],
            "config": {"workload": "64 open XXZ chains, J=1, L even in [16,128], Delta in [0.5,1.5], "
                                   "m_max in {64,128,256,512} (seed 1005); the first %d" % n,
                       "L": [c["L"] for c in chains], "m_max": [c["m_max"] for c in chains],
                       "Delta": [round(c["Delta"], 6) for c in chains],
                       "precision": "3xTF32 then FP64 (ladder at 1e-7)" if mixed else "fp64",
                       "svd": args.svd, "max_sweeps": args.batch_sweeps, "alpha0": ALPHA},
            "data": "synthetic"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32x3", "tf32"])
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--svd", default="auto", choices=["gesvd", "jacobi", "auto"],
                    help="factorisation of the truncation's per-sector SVD")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-update", action="store_true", help="skip the local-update field")
    ap.add_argument("--no-sweep", action="store_true", help="skip the sweep-to-1e-9 field")
    ap.add_argument("--update-steps", type=int, default=5,
                    help="timed local updates of the local-update field")
    ap.add_argument("--heff-only", action="store_true",
                    help="kernel view: back-to-back H_eff applications, L2 not flushed")
    ap.add_argument("--workload", default="cylinder_4x16_m2048_u1", choices=sorted(HEFF_WORKLOADS),
                    help="central-site H_eff problem of the headline line and the kernel view")
    ap.add_argument("--workload-m", type=int, default=None,
                    help="bond dimension of the H_eff problem (default: the workload's)")
    ap.add_argument("--workspace-gb", type=float, default=8.0,
                    help="context workspace of the H_eff views, GiB")
    ap.add_argument("--sweep", action="store_true",
                    help="only the sweep-to-1e-9 time of full sweeps, mixed ladder vs FP64")
    ap.add_argument("--sweep-sites", type=int, default=100)
    ap.add_argument("--sweep-m", type=int, default=512)
    ap.add_argument("--sweep-model", default="xxz", choices=sorted(SWEEP_MODELS))
    ap.add_argument("--sweep-max", type=int, default=16, help="sweeps per arm at most")
    ap.add_argument("--lanczos", action="store_true",
                    help="Lanczos iteration time on --workload's central site (--lanczos-k iterations)")
    ap.add_argument("--lanczos-k", type=int, nargs="+", default=[10, 20, 40])
    ap.add_argument("--batch", action="store_true", help="run only the batched-chain field")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-chain field")
    ap.add_argument("--batch-chains", type=int, default=8)
    ap.add_argument("--batch-sweeps", type=int, default=12)
    ap.add_argument("--batch-prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--batch-compare", action="store_true",
                    help="also solve the same chains one at a time (dmrg3s_sweep)")
    ap.add_argument("--measure-peaks", action="store_true",
                    help="measure the cuBLAS TF32 and FP64 GEMM peaks into profiles/")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.measure_peaks:
        res = measure_peaks()
    elif args.sweep:
        res = run_sweep(args)
    elif args.batch:
        res = run_batch(args)
    elif args.lanczos:
        res = run_lanczos(args)
    elif args.heff_only:
        res = run_heff_only(args)
    else:
        res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()

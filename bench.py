#!/usr/bin/env python3
"""Benchmark of the DMRG3S hot path on one GB300 (or N independent replicas).

A *step* is one DMRG3S local update (Sec. V of arXiv:1501.05504, steps 1-7):
Lanczos eigensolver over H_eff = L W A R, expansion term alpha L M W,
per-sector FP64 SVD truncation to m_max, S V^dagger into the neighbour,
environment update and the energy after truncation.  Workload: the central
two-site window of the S=1/2 Heisenberg (XXZ, Delta = 1) chain with L = 100,
d = 2, w = 5, U(1) S^z blocks and m_max = 512; the boundary environments are
seeded synthetic symmetric block tensors with Gaussian sector dimensions (a
stand-in for converged environments: seeded_inputs.central_bonds and
symmetric_env build them).  Steps
alternate direction (left-to-right, right-to-left) so every step is a full
update of the same window.

Metric: algorithmic TFLOP/s of the step's contractions (grouped-GEMM block
products + MPO combinations, counted as sum 2 M N K over the block tasks;
the SVD is not counted).  ``e2e`` repeats the step through the C ABI with the
window's tensors in pinned host memory, copied in and out every step.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (H_eff applications, the step's dominant cost) on the host cores.
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


def heff_flops(qp, t, W, left, right):
    """Algorithmic flops of one block-sparse H_eff application, order (((L A) W) R)."""
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
        jp = find(right, right["q"][j] + t[br])
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


def peaks():
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        mp = json.load(f)
    src = "measured"
    bf16 = mp.get("bf16_tflops_sustained") or mp.get("bf16_tflops")
    hbm = mp.get("hbm_gbs")
    if bf16 is None:
        bf16, src = 1700.0, "fallback"
    # other dtypes: the measured bf16 dense peak times the nominal ratio of the
    # GB300 datasheet (bf16 2.25, tf32 1.1, fp64 1.25e-3 PFLOP/s dense)
    return {"bf16": bf16, "tf32": bf16 * 1.1 / 2.25, "fp64": bf16 * 1.25e-3 / 2.25, "hbm": hbm,
            "source": src}


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


def run_ours(args):
    import torch
    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_1501_05504_gb300 import binding as b
    dev = torch.cuda.current_device()
    ctx = b.dmrg3s_create(dev, 1 << 30)
    spec = window_specs(SEED + rank)
    mpo = b.Mpo(b.MODEL_XXZ, 100, (1.0, 1.0))
    W = [mpo.site(50), mpo.site(51)]
    opts = b.update_opts(M_MAX, kmax=40, tol=1e-10, prec=args.precision, svd=args.svd)
    gL, gR = b.env_from_neutral(spec["L"]), b.env_from_neutral(spec["R"])
    gM = [b.site_from_neutral(x) for x in spec["M"]]
    state = b.dmrg3s_state_create(ctx, W, gM, gL, gR, 0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def step(st):
        c, _ = st.centre()
        return b.dmrg3s_local_update(st, 1 if c == 0 else -1, ALPHA, opts)

    for _ in range(args.warmup):
        step(state)
    torch.cuda.synchronize()
    # ---- device-resident timed region
    b.dmrg3s_profile(ctx, True)
    n0 = b.dmrg3s_launch_count()
    times, iters, sweeps, fallbacks = [], [], [], 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step(state)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            iters.append(info["lanczos_iters"])
            sweeps.append(info["svd_sweeps"])
            fallbacks += int(info["svd_fallback"])
    torch.cuda.synchronize()
    launches = b.dmrg3s_launch_count() - n0
    g = b.dmrg3s_profile_read(ctx, b.KERNEL_GEMM)
    cmb = b.dmrg3s_profile_read(ctx, b.KERNEL_COMBINE)
    jac = b.dmrg3s_profile_read(ctx, b.KERNEL_JACOBI)
    phases = {name: b.dmrg3s_profile_read(ctx, k)["ms"] / args.steps
              for k, name in enumerate(["eigensolver", "expansion", "svd_truncation", "remainder",
                                        "environment", "energy"], start=2)}
    b.dmrg3s_profile(ctx, False)
    total_ms = max_over_ranks(sum(times), world, "cuda")
    flops_step = (g["flops"] + cmb["flops"]) / args.steps
    ms_step = total_ms / args.steps
    value = replica_value(flops_step, world, ms_step)
    pk = peaks()
    prec = args.precision
    peak = pk["fp64"] if prec == "fp64" else pk["tf32"] / (3.0 if prec == "tf32x3" else 1.0)
    achieved = g["flops"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else None
    kname = "gemm_f64_kernel" if prec == "fp64" else "gemm_tc_kernel"
    roof_gemm = {"kernel": kname, "bound": "alu" if prec == "fp64" else "tensor",
                 "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": achieved / peak if achieved else None,
                 "traffic": traffic_for(kname), "launches": g["launches"],
                 "avg_launch_us": 1e3 * g["ms"] / max(g["launches"], 1),
                 "peak_source": "%s bf16 x nominal %s/bf16 ratio" % (pk["source"], prec),
                 "share_of_step": g["ms"] / total_ms if total_ms else None}
    roofline = roof_gemm
    if jac["launches"]:
        # the truncation's Jacobi SVD: FP64 pair tests and rotations on the CUDA
        # cores, the working set (R^T of every sector) resident in L2
        ja = jac["flops"] / (jac["ms"] * 1e-3) / 1e12
        roof_jac = {"kernel": "jac_round_kernel", "bound": "alu", "achieved": ja, "peak": pk["fp64"],
                    "unit": "TFLOP/s", "frac": ja / pk["fp64"], "traffic": traffic_for("jac_round_kernel"),
                    "launches": jac["launches"], "avg_launch_us": 1e3 * jac["ms"] / jac["launches"],
                    "time_basis": "whole Jacobi sweeps (CUDA graphs), gaps between launches included",
                    "peak_source": "%s bf16 x nominal fp64/bf16 ratio" % pk["source"],
                    "share_of_step": jac["ms"] / total_ms if total_ms else None}
        # the dominant kernel (largest share of the step) carries the roofline
        if jac["ms"] > g["ms"]:
            roofline = dict(roof_jac, other=roof_gemm)
        else:
            roofline = dict(roof_gemm, other=roof_jac)
    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host = {"L": gL.data.cpu().pin_memory(), "R": gR.data.cpu().pin_memory(),
                "M": [m.data.cpu().pin_memory() for m in gM]}
        bi = sum(x.numel() * 8 for x in [host["L"], host["R"]] + host["M"])
        torch.cuda.synchronize()
        et = []
        bo = 0
        for k in range(max(2, args.steps // 2)):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gL.data.copy_(host["L"], non_blocking=True)
            gR.data.copy_(host["R"], non_blocking=True)
            for m, h in zip(gM, host["M"]):
                m.data.copy_(h, non_blocking=True)
            st = b.dmrg3s_state_create(ctx, W, gM, gL, gR, 0)
            step(st)
            outs = [st.site(0), st.site(1)]
            res = [o.data.to("cpu", non_blocking=True) for o in outs]
            e1.record(stream)
            torch.cuda.synchronize()
            bo = sum(r.numel() * 8 for r in res)
            et.append(e0.elapsed_time(e1))
            st.close()
        ems = statistics.mean(et)
        ems = max_over_ranks(ems, world, "cuda")
        e2e = {"value": replica_value(flops_step, world, ems), "unit": "TFLOP/s",
               "ms_per_step": ems, "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo)}
    state.close()
    if rank != 0:
        return None
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(args.cpu_sample_s)
    return {"metric": "Heff.A TFLOP/s of one DMRG3S local update (algorithmic block-sparse flops)",
            "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "tf32x3": "tf32x3",
                                                             "tf32": "tf32"}[prec],
            "data": "synthetic", "impl": "ours",
            "config": {"workload": "xxz_l100_m512_u1 central two-site window, one local update per step",
                       "hamiltonian": "S=1/2 XXZ chain Delta=1, L=100, d=2, w=5, U(1) S^z", "m_max": M_MAX,
                       "alpha": ALPHA, "lanczos_kmax": 40, "lanczos_tol": 1e-10,
                       "lanczos_iters_mean": statistics.mean(iters), "flops_per_step": flops_step,
                       "phase_ms_per_step": phases,
                       "precision": prec, "svd": args.svd, "svd_jacobi_sweeps": sweeps,
                       "svd_fallbacks": fallbacks,
                       "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
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
    "hubbard_l64_m1024_u1u1": ("hubbard", 64, (1.0, 8.0), 32, 1003),
    "cylinder_4x16_m2048_u1": ("cylinder", 64, None, 32, 1004),
}


def heff_problem_specs(b, name, m=None):
    """Central-site H_eff problem of a larger workload: the library's MPO site,
    and seeded symmetric environments and a random site tensor (neutral specs)
    on the workload's bonds."""
    model, n, params, site, seed = HEFF_WORKLOADS[name]
    if model == "hubbard":
        mpo = b.Mpo(b.MODEL_HUBBARD, n, params)
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


def heff_problem(b, name, m=None):
    W, Le, Re, M = heff_problem_specs(b, name, m)
    return W, b.env_from_neutral(Le), b.env_from_neutral(Re), b.site_from_neutral(M)


def run_heff_only(args):
    """Kernel view: repeated H_eff applications on a workload's central site."""
    import torch
    from paper_1501_05504_gb300 import binding as b
    ctx = b.dmrg3s_create(torch.cuda.current_device(), int(args.workspace_gb * (1 << 30)))
    if args.workload == WORKLOAD:
        spec = window_specs(SEED)
        mpo = b.Mpo(b.MODEL_XXZ, 100, (1.0, 1.0))
        W0, W1 = mpo.site(50), mpo.site(51)
        gL, gR = b.env_from_neutral(spec["L"]), b.env_from_neutral(spec["R"])
        gM0, gM1 = (b.site_from_neutral(x) for x in spec["M"])
        gR0 = b.empty_env(W0.tr, gM0.right)                     # right environment of site 50
        b.dmrg3s_update_env(ctx, -1, gR, W1, gM1, gR0, "fp64")
    else:
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
            "peak_source": "%s bf16 x nominal %s/bf16 ratio" % (peak["source"], args.precision),
            "l2": "not flushed (kernel view)"}


def cpu_baseline(sample_s=15.0):
    """The FP64 oracle on the host cores: H_eff applications on the same window."""
    from oracle import contract, io, models
    spec = window_specs(SEED)
    W = models.mpo_xxz(100, 1.0, 1.0).W[50]
    L, R = io.env_dense(spec["L"]), io.env_dense(spec["R"])
    # the right environment of site 50 inside the window: R_51 contracted with M_51
    W1 = models.mpo_xxz(100, 1.0, 1.0).W[51]
    M1 = io.site_dense(spec["M"][1])[0]
    R50 = contract.right_env(R, W1, M1)
    M0 = io.site_dense(spec["M"][0])[0]
    t0 = time.time()
    n = 0
    while time.time() - t0 < sample_s or n == 0:
        contract.apply_heff(L, W, R50, M0)
        n += 1
    dt = (time.time() - t0) / n
    f = heff_flops(si.XXZ_QP, si.XXZ_T, W, spec["bonds"][0], spec["bonds"][1])
    return {"value": f / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d H_eff applications of the window's centre site (dense FP64 einsum, %.2f s each)"
                      % (n, dt)}


def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return None
    t0 = time.time()
    cb = cpu_baseline(max(args.cpu_sample_s, 1.0) * max(args.steps, 1) / 10.0)
    return {"metric": "Heff.A TFLOP/s of one DMRG3S local update (algorithmic block-sparse flops)",
            "value": cb["value"], "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "xxz_l100_m512_u1 central two-site window (oracle sample)"},
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


def _sweep_run(b, ctx, L, m_max, ladder, model="xxz", max_sweeps=24, cap_s=240.0, svd="gesvd"):
    """Sweeps from a product state (Neel / alternating up-down), one dmrg3s_sweep call per sweep.

    ladder: list of (precision, until) pairs; a precision is used until the
    relative sweep-to-sweep energy change drops below `until` (the last one
    until convergence at 1e-11).  Returns per-sweep (wall seconds, energy)."""
    import torch
    lib_model, params, pattern, _ = SWEEP_MODELS[model]
    if model == "cylinder":
        bonds = cylinder_bonds(L // 4, 4)
        W = b.Mpo(b.MODEL_SPIN_BONDS, L, (), bonds=bonds, couplings=[(1.0, 1.0)] * len(bonds)).sites()
    else:
        W = b.Mpo(getattr(b, lib_model), L, params).sites()
    st = b.dmrg3s_state_create(ctx, W, b.product_state(W[0].qp, pattern * (L // 2)), None, None,
                               L - 1)
    alpha = ALPHA
    log = []
    stage = 0
    prev = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max_sweeps):
        prec, until = ladder[stage]
        rep = b.dmrg3s_sweep(st, b.alpha_rule(alpha), 1, 0.0, b.update_opts(m_max, prec=prec, svd=svd))
        alpha = rep["alpha"]
        e = rep["energy"]
        log.append((time.perf_counter() - t0, e, prec))
        rel = abs(e - prev) / abs(e) if prev is not None else 1.0
        prev = e
        if rel < until:
            if stage + 1 < len(ladder):
                stage += 1
            else:
                break
        if time.perf_counter() - t0 > cap_s:
            break
    st.close()
    return log


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
    cap = args.sweep_cap_s
    fp64 = _sweep_run(b, ctx, L, m_max, [("fp64", 1e-11)], model, cap_s=cap, svd=args.svd)
    mixed = _sweep_run(b, ctx, L, m_max, [("tf32x3", 1e-7), ("fp64", 1e-11)], model, cap_s=cap,
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
            "config": {"workload": "%s_l%d_m%d full sweeps" % (model, L, m_max),
                       "hamiltonian": "%s, L=%d" % (SWEEP_MODELS[model][3], L),
                       "m_max": m_max, "alpha0": ALPHA, "lanczos_kmax": 40, "lanczos_tol": 1e-10,
                       "start": "product state %s..., m=1" % SWEEP_MODELS[model][2],
                       "svd": args.svd, "cap_s_per_arm": cap},
            "data": "synthetic"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32x3", "tf32"])
    ap.add_argument("--cpu-sample-s", type=float, default=15.0)
    ap.add_argument("--svd", default="gesvd", choices=["gesvd", "jacobi"],
                    help="factorisation of the truncation's per-sector SVD")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--heff-only", action="store_true",
                    help="kernel view: time repeated H_eff applications instead of local updates")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD] + sorted(HEFF_WORKLOADS),
                    help="central-site problem of the kernel view (--heff-only)")
    ap.add_argument("--workload-m", type=int, default=None,
                    help="bond dimension of the kernel view's problem (default: the workload's)")
    ap.add_argument("--workspace-gb", type=float, default=4.0,
                    help="context workspace of the kernel view, GiB")
    ap.add_argument("--sweep", action="store_true",
                    help="sweep-to-1e-9 time of full sweeps, mixed ladder vs FP64")
    ap.add_argument("--sweep-sites", type=int, default=100)
    ap.add_argument("--sweep-m", type=int, default=512)
    ap.add_argument("--sweep-model", default="xxz", choices=sorted(SWEEP_MODELS))
    ap.add_argument("--sweep-cap-s", type=float, default=240.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.sweep:
        res = run_sweep(args)
    elif args.heff_only:
        res = run_heff_only(args)
    else:
        res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()

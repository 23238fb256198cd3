"""Benchmark of the MBE(3)-OSV-MP2 hot path on GB300: one step = one geometry's energy AND gradient
(osv_build -> cluster_residual_solve -> mbe3_combine -> energy -> gradient_backward) on the 64-LMO chain
workload (n_vir 400, n_aux 1600, l_osv 1e-4 capped at 40 OSVs, 8/6 A pair/triple cutoffs).

Metric: cluster pair-residual TFLOP/s = algorithmic residual FLOPs of the step (coupling products of Eq. 4,
2 (r_p r_q^2 + r_p^2 r_q) per term and residual evaluation) / step wall time.  Also reported: gradient
seconds per geometry (= ms_per_step / 1000), residual-solve-only TFLOP/s, and the roofline of the dominant
kernel from per-stage CUDA events taken over the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference] [--precision fp64|mixed]
Multi-GPU (torchrun, one rank per GPU): each rank solves its own geometry (different seed); no collective on
the data path; value = all ranks' residual FLOPs / max-over-ranks time ("scaling": "weak").
--impl reference times the CPU oracle (the reference implementation of this path) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cluster pair-residual TFLOP/s, gradient s/geometry: mixed vs FP64 GPU @1e-6 Eh"
WORKLOAD = 1
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # 152 SMs x 2.07 GHz x 2 DFMA/clk/SM (1.25 TFLOP/s nominal)
FP32_PEAK_TFLOPS = 152 * 2.07e9 * 256 / 1e12  # 152 SMs x 2.07 GHz x 128 FP32 lanes x 2 (FMA) = 80.5 TFLOP/s
DF_OPS_PER_FMA = 12                            # FP32 instructions of one double-float multiply-add (df_fma)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="bf16x4", choices=["fp64", "tf32x3", "bf16x4"],
                    help="path whose throughput is the headline value; the FP64 path is always timed beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def workload_config(prm, p):
    return {"workload": f"MBE(3) energy+gradient, {p.n_occ} LMOs on a 1.5 A chain, n_vir={p.n_vir}, "
                        f"n_aux={p.n_aux}, l_osv=1e-4 capped at {prm.n_osv_max} OSVs, pair/triple cutoffs "
                        f"{prm.r2b}/{prm.r3b} A",
            "n_occ": p.n_occ, "n_vir": p.n_vir, "n_aux": p.n_aux, "mbe_order": prm.mbe_order,
            "precision": {0: "fp64", 1: "tf32x3", 2: "bf16x4"}[prm.precision],
            "l2": f"inputs larger than L2 (B = {p.B.nbytes / 1e6:.0f} MB > 129 MB)"}


# ------------------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# --------------------------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch

    from paper_2106_06149_gb300 import build, osvmbe
    from paper_2106_06149_gb300.synth import workload, make_problem, WORKLOADS

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    osvmbe.load()
    p, prm = workload(WORKLOAD)
    if rank > 0:   # each rank: an independent geometry of the same workload (own seed)
        _, pk, _ = WORKLOADS[WORKLOAD]
        p = make_problem(**{**pk, "seed": pk["seed"] + 1000 * rank})
    prec = {"fp64": 0, "tf32x3": 1, "bf16x4": 2}[args.precision]
    stream = torch.cuda.current_stream()
    dp = osvmbe.DeviceProblem.from_host(p)
    ctx = osvmbe.Context(stream)
    ctx.clusters_build(dp, prm)
    dB = torch.zeros_like(dp.B)
    dF = torch.zeros_like(dp.f_occ)

    def step():
        osvmbe.run_energy(ctx, dp, prm)
        ctx.gradient_backward(1.0, dB, dF)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed_steps(k):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        barrier()
        t0.record(stream)
        for _ in range(k):
            step()
        t1.record(stream)
        barrier()
        return t0.elapsed_time(t1) / k

    warm = max(args.warmup, 3)
    # ---- the plain FP64 GPU path (reference point of the mixed path)
    prm.precision = 0
    for _ in range(warm):
        step()
    fp64_ms = timed_steps(args.steps)
    E64, _ = ctx.energy()
    flops64 = ctx.residual_flops()
    dB.zero_()
    ctx.profile(True)
    step()
    torch.cuda.synchronize()
    stages64 = ctx.profile_read()
    ctx.profile(False)
    dB64 = dB.clone()
    # ---- the headline path
    prm.precision = prec
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    flops_exec = ctx.residual_flops()
    upd32, ev64, uncv = ctx.solve_counts()
    # the metric's work per step: the residual FLOPs of the FP64 solve to tol (the iterations the problem
    # needs); the mixed solve's own count (FP32 iterations + FP64 evaluations) is reported beside it
    flops_step = flops64
    E, E_lin = ctx.energy()
    dB.zero_()
    step()
    torch.cuda.synchronize()
    grad_diff = float((dB - dB64).abs().max())

    # ---- timed region (device-resident inputs)
    ctx.profile(True)
    l0 = ctypes_launches(osvmbe)
    with ClockSampler(local) as clk:
        ms = timed_steps(args.steps)
    launches = ctypes_launches(osvmbe) - l0
    stages = ctx.profile_read()
    ctx.profile(False)
    ms, flops_all = reduce_over_ranks(ms, flops_step, world, "cuda")
    value = flops_all / (ms * 1e-3) / 1e12

    # ---- end to end through the C ABI with host buffers: h2d of B, F, eps; d2h of E, dB, dF
    hB = torch.from_numpy(np.ascontiguousarray(p.B)).pin_memory()
    hF = torch.from_numpy(np.ascontiguousarray(p.f_occ)).pin_memory()
    he = torch.from_numpy(np.ascontiguousarray(p.eps_vir)).pin_memory()
    odB = torch.empty(dB.shape, dtype=dB.dtype).pin_memory()
    odF = torch.empty(dF.shape, dtype=dF.dtype).pin_memory()

    def e2e_step():
        dp.B.copy_(hB, non_blocking=True)
        dp.f_occ.copy_(hF, non_blocking=True)
        dp.eps_vir.copy_(he, non_blocking=True)
        dB.zero_()
        dF.zero_()
        osvmbe.run_energy(ctx, dp, prm)        # energy() reads E back to the host
        ctx.gradient_backward(1.0, dB, dF)
        odB.copy_(dB, non_blocking=True)
        odF.copy_(dF, non_blocking=True)

    e2e_step()
    barrier()
    te0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_ms = (time.perf_counter() - te0) * 1e3 / args.steps
    h2d = hB.numel() * hB.element_size() + hF.numel() * 8 + he.numel() * 8
    d2h = 8 + odB.numel() * odB.element_size() + odF.numel() * 8

    # ---- roofline of the dominant stage
    total_stage = sum(v[0] for v in stages.values())
    dom = max(stages.items(), key=lambda kv: kv[1][0])
    roof = roofline(dom, stages, flops_step, p, prm, ctx.adjoint_flops(), prec, ctx.residual_work())
    roof_tc = tensor_roofline(stages, p, prm) if prec > 0 else None

    out = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f64", 1: "tf32x3+f64", 2: "bf16x4+f64"}[prec], "data": "synthetic",
        "config": workload_config(prm, p),
        "gradient_s_per_geometry": ms / 1e3,
        "residual_solve_tflops": flops_step / (stages["residual"][0] / stages["residual"][1] * 1e-3) / 1e12
        if "residual" in stages else None,
        "residual_flops_per_step": flops_step,
        "residual_flops_executed_per_step": flops_exec,
        "residual_iterations": {"fp32_updates": upd32, "fp64_evals": ev64, "unconverged": uncv,
                                "clusters": len(ctx.cluster_info()[0])},
        "fp64_stage_ms": {k: v[0] for k, v in stages64.items()},
        "energy_Eh": E, "energy_linear_Eh": E_lin,
        "fp64_ms_per_step": fp64_ms, "mixed_vs_fp64": fp64_ms / ms, "energy_fp64_Eh": E64,
        "abs_dE_vs_fp64_Eh": abs(E - E64), "max_abs_dgradB_vs_fp64": grad_diff,
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
        "stage_share": {k: v[0] / total_stage for k, v in stages.items()},
        "roofline": roof,
        "roofline_tensor_gemm": roof_tc,
        "e2e": {"value": flops_all / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sample_every=4, repeats=1)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def reduce_over_ranks(ms, flops, world, device):
    """Whole-job numbers of a weak-scaling step: the slowest rank's time and the sum of every rank's work (each
    rank solves its own geometry; this timing reduction is the only collective)."""
    if world <= 1:
        return ms, flops
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    f = torch.tensor([flops], device=device, dtype=torch.float64)
    dist.all_reduce(f)
    return float(t.item()), float(f.item())


def ctypes_launches(osvmbe):
    import ctypes
    n = ctypes.c_longlong()
    osvmbe.load().osv_kernel_launches(ctypes.byref(n))
    return n.value


def stage_flops(name, p, prm, flops_step, adj_flops=None):
    """Algorithmic FLOPs of one launch of a stage (FP64 work of the method, padding excluded)."""
    nv, na, n, nm = p.n_vir, p.n_aux, p.n_occ, prm.n_osv_max if prm.n_osv_fixed <= 0 else prm.n_osv_fixed
    d = np.linalg.norm(p.centres[:, None, :] - p.centres[None, :, :], axis=-1)
    nb = (d <= prm.r2b).sum(axis=1)            # |{i} U N(i)| of the half transforms
    a = np.diff(p.aux_ptr)
    if name == "residual":
        return flops_step
    if name == "adj_clusters":
        return adj_flops
    if name == "tkk_gram":
        return float(np.sum(2.0 * nv * nv * a))
    if name == "half_transform":
        return float(np.sum(2.0 * nb * nm * nv * a))
    if name == "osv_eigh":
        return n * (4.0 / 3.0) * nv ** 3                 # Householder tridiagonalisation (bisection and kept-vector work are O(n^2))
    return None


def tensor_roofline(stages, p, prm):
    """The tcgen05 GEMM of the T_kk Gram products: issued tensor FLOPs vs the measured dense BF16 peak (each useful
    multiply-add costs 13 BF16 slice products in the exact-slice mode, 3 TF32 products (at half the BF16 rate)
    in the split-TF32 mode); useful FLOPs reported beside it.  The stage time includes the slicing passes."""
    if "tkk_gram" not in stages:
        return None
    ms_total, calls = stages["tkk_gram"]
    avg = ms_total / calls
    useful = stage_flops("tkk_gram", p, prm, 0.0)
    mult = 13.0 if prm.precision == 2 else 6.0
    peak = measured_peak("bf16_tflops", 1900.0)
    issued = useful * mult / (avg * 1e-3) / 1e12
    return {"bound": "tensor", "stage": "tkk_gram", "kernel": "k_oz_gemm" if prm.precision == 2 else "k_gemm_tf32x3",
            "achieved": issued, "peak": peak, "unit": "TFLOP/s", "frac": issued / peak, "traffic": None,
            "useful_tflops": useful / (avg * 1e-3) / 1e12, "avg_launch_ms": avg,
            "peak_note": "measured dense bf16 (burst); achieved counts issued BF16-equivalent slice products"}


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except Exception:
        return fallback


def roofline(dom, stages, flops_step, p, prm, adj_flops=None, prec=0, work=None):
    """ALU roofline of the dominant stage.  FP64 path: algorithmic FLOPs against the FP64 units.  Mixed paths:
    the FP32-pipe work those FLOPs become (FP32 residual evaluations as they are; every FP64-accurate multiply-add
    as a double-float one, DF_OPS_PER_FMA FP32 instructions) against the FP32 pipe; both from unit counts and the
    2.07 GHz maximum clock.  Index arithmetic, loads and conversions are not counted, so the issue-slot use is
    higher than frac."""
    name, (ms_total, calls) = dom
    avg_ms = ms_total / calls
    flops = stage_flops(name, p, prm, flops_step, adj_flops)
    base = {"bound": "alu", "stage": name, "unit": "TFLOP/s", "traffic": None, "avg_launch_ms": avg_ms}
    if not flops:
        return dict(base, achieved=None, peak=FP64_PEAK_TFLOPS if prec == 0 else FP32_PEAK_TFLOPS, frac=None)
    if prec == 0:
        ach = flops / (avg_ms * 1e-3) / 1e12
        return dict(base, achieved=ach, peak=FP64_PEAK_TFLOPS, frac=ach / FP64_PEAK_TFLOPS,
                    algorithmic_flops_per_launch=flops,
                    peak_note="FP64 CUDA cores, 152 SMs x 2 DFMA/clk x 2.07 GHz (nominal 1.25 TFLOP/s)")
    nm = prm.n_osv_max if prm.n_osv_fixed <= 0 else prm.n_osv_fixed
    if name == "adj_clusters" and 2 * nm <= 80:
        # tensor-core partials: 13 BF16 digit products per FP64-accurate product, M = 128 rows issued for <= 80
        issued = 13.0 * flops * 128.0 / 80.0
        ach = issued / (avg_ms * 1e-3) / 1e12
        peak = measured_peak("bf16_tflops", 1900.0)
        return dict(base, bound="tensor", achieved=ach, peak=peak, frac=ach / peak, algorithmic_flops_per_launch=flops,
                    issued_bf16_flops_per_launch=issued, fp64_equivalent_tflops=flops / (avg_ms * 1e-3) / 1e12,
                    peak_note="measured dense BF16 (MEASURED_PEAKS.json, burst); achieved counts the issued digit "
                              "products (13 per FP64-accurate product, M padded to 128)")
    if name == "residual" and work is not None:
        f32, f64 = work
        pipe = f32 + DF_OPS_PER_FMA * f64
        detail = {"fp32_evaluation_flops": f32, "fp64_accurate_evaluation_flops": f64}
    else:
        pipe = DF_OPS_PER_FMA * flops   # every other dominant candidate (the cluster adjoint) is double-float
        detail = {}
    ach = pipe / (avg_ms * 1e-3) / 1e12
    return dict(base, achieved=ach, peak=FP32_PEAK_TFLOPS, frac=ach / FP32_PEAK_TFLOPS,
                algorithmic_flops_per_launch=flops, fp32_pipe_flops_per_launch=pipe,
                fp64_equivalent_tflops=flops / (avg_ms * 1e-3) / 1e12,
                peak_note="FP32 pipe, 152 SMs x 128 lanes x 2 flop x 2.07 GHz; double-float multiply-add = "
                          f"{DF_OPS_PER_FMA} FP32 instructions", **detail)


# ------------------------------------------------------------------------------------- CPU baseline
def oracle_sample(sample_every):
    """Oracle energy + gradient of every `sample_every`-th cluster of the bench workload (OSVs for all LMOs)."""
    import torch

    import oracle
    from paper_2106_06149_gb300.synth import workload

    p, prm = workload(WORKLOAD)
    cl = oracle.select_clusters(p.centres, prm.r2b, prm.r3b, prm.mbe_order)
    sample = cl[::sample_every]
    t0 = time.perf_counter()
    g = oracle.gradient(p, prm, clusters=sample)
    dt = time.perf_counter() - t0
    # residual model FLOPs of the sample, same formula as the library (stored pairs, r = kept dims)
    flops = 0.0
    for c in sample:
        r = {}
        for a in c:
            for b in c:
                if a <= b:
                    r[(a, b)] = g["n_osv"][a] + (g["n_osv"][b] if a != b else 0)
        per = 0.0
        for (i, j), rp in r.items():
            for k in c:
                if k != j:
                    rq = r[(min(i, k), max(i, k))]
                    per += 2.0 * (rp * rq * rq + rp * rp * rq)
                if k != i:
                    rq = r[(min(k, j), max(k, j))]
                    per += 2.0 * (rp * rq * rq + rp * rp * rq)
        flops += per * (g["iters"][c] + 1)
    return flops, dt, len(sample), len(cl), torch.get_num_threads()


def cpu_baseline(sample_every=4, repeats=1):
    flops, dt, ns, nc, cores = oracle_sample(sample_every)
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "seconds": dt,
            "sample": f"oracle energy+gradient of every {sample_every}th cluster ({ns} of {nc}) of the bench "
                      f"workload, OSVs of all LMOs, FP64, torch CPU with {cores} threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch
    torch.set_num_threads(len(os.sched_getaffinity(0)))
    for _ in range(args.warmup):
        oracle_sample(32)
    tot_f, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        f, dt, ns, nc, cores = oracle_sample(32)
        tot_f += f
        tot_t += dt
    value = tot_f / tot_t / 1e12
    from paper_2106_06149_gb300.synth import workload
    p, prm = workload(WORKLOAD)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(prm, p),
           "cpu_baseline": {"value": value, "unit": "TFLOP/s", "kind": "oracle", "cores": cores,
                            "sample": f"oracle energy+gradient of every 32nd cluster ({ns} of {nc}) per step"},
           "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)

"""Benchmark of the MBE(3)-OSV-MP2 hot path on GB300: one step = one geometry's energy AND gradient
(osv_build -> cluster_residual_solve -> mbe3_combine -> energy -> gradient_backward, recorded once as a CUDA graph by
osv_graph_capture and replayed by osv_graph_launch, one replay per step) on a synthetic workload of
paper_2106_06149_gb300.synth.WORKLOADS, by default workload 2: 256 LMOs in a 20 A cube, n_vir 1500, n_aux 6000,
7 A fitting domains, B in FP32, l_osv 1e-4 capped at 40 OSVs, 8/6 A pair/triple cutoffs (256 + 5212 + 8872
clusters), the mixed-precision and batching workload the metric is quoted on.

Metric: cluster pair-residual TFLOP/s = algorithmic residual FLOPs of the step (coupling products of Eq. 4,
2 (r_p r_q^2 + r_p^2 r_q) per term and residual evaluation, counted over the iterations the FP64 solve needs) /
step wall time.  Also reported: gradient seconds per geometry (= ms_per_step / 1000), the FP64 GPU path's step
time beside it (mixed_vs_fp64), the residual kernel's roofline (algorithmic FLOPs / its CUDA-event time / the
measured dense BF16 peak) and per-stage times from CUDA events taken over the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference] [--workload 1|2|3|4]
                  [--precision fp64|bf16x4] [--fp64-steps S] [--no-cpu-baseline]
Multi-GPU (torchrun, one rank per GPU): each rank solves its own geometry (different seed); no collective on
the data path; value = all ranks' residual FLOPs / max-over-ranks time ("scaling": "weak").
--impl reference times the CPU oracle (the reference implementation of this path) on a bounded cluster sample.
"""
from __future__ import annotations

import argparse
import hashlib
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
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # 152 SMs x 2.07 GHz x 2 DFMA/clk/SM (1.25 TFLOP/s nominal)
FP32_PEAK_TFLOPS = 152 * 2.07e9 * 256 / 1e12  # 152 SMs x 2.07 GHz x 128 FP32 lanes x 2 (FMA) = 80.5 TFLOP/s
DF_OPS_PER_FMA = 12                            # FP32 instructions of one double-float multiply-add (df_fma)
WHY_NOT_4 = ("workload 4 (512 LMOs, n_vir 3000) also fits one GPU, but one step takes about 6 s, so 20 timed steps "
             "would run past a minute-scale timed region; it is measured with --workload 4")

# DRAM traffic per launch of the residual kernel (dram__bytes_read.sum + dram__bytes_write.sum), from the ncu capture
# summarised in profiles/, keyed by workload and by the SHA-256 prefix of the kernel's source file at capture time:
# a kernel changed since the capture reports null.
NCU_TRAFFIC = {
    # profiles/residual_mixed_full_cube48.md: 5.53 GB over 1585 clusters, scaled to workload 2's 14340 clusters
    (2, 2, "0bb875668c9dc2db"): (3.106020e9 + 2.425234e9) * 14340 / 1585,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4])
    ap.add_argument("--precision", default="bf16x4", choices=["fp64", "bf16x4"],
                    help="path whose throughput is the headline value; the FP64 path is always timed beside it")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the FP64 comparison path (after one warm-up step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def workload_config(k, prm, p):
    from paper_2106_06149_gb300.synth import WORKLOADS
    desc = WORKLOADS[k][0]
    cfg = {"workload": f"workload {k}: {desc}; MBE(3) energy+gradient per step, l_osv {prm.l_osv:g} capped at "
                       f"{prm.n_osv_max} OSVs, pair/triple cutoffs {prm.r2b}/{prm.r3b} A",
           "n_occ": p.n_occ, "n_vir": p.n_vir, "n_aux": p.n_aux, "mean_fitting_domain": float(np.diff(p.aux_ptr).mean()),
           "mbe_order": prm.mbe_order, "precision": {0: "fp64", 2: "bf16x4"}[prm.precision],
           "B_dtype": str(p.B.dtype),
           "l2": f"inputs larger than L2 (B = {p.B.nbytes / 1e6:.0f} MB > 129 MB)"}
    if k != 4:
        cfg["why_not_workload_4"] = WHY_NOT_4
    return cfg


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
    p, prm = workload(args.workload)
    if rank > 0:   # each rank: an independent geometry of the same workload (own seed)
        _, pk, _ = WORKLOADS[args.workload]
        pk = dict(pk)
        if pk.get("radius") == "mean2000":
            from paper_2106_06149_gb300.synth import _radius_for_mean_domain
            pk["radius"] = _radius_for_mean_domain(pk["seed"], pk["n_occ"], pk["box"], 1.4, pk["n_aux"], 2000.0)
        p = make_problem(**{**pk, "seed": pk["seed"] + 1000 * rank})
    prec = {"fp64": 0, "bf16x4": 2}[args.precision]
    stream = torch.cuda.current_stream()
    dp = osvmbe.DeviceProblem.from_host(p)
    ctx = osvmbe.Context(stream)
    ctx.clusters_build(dp, prm)
    dB = torch.zeros_like(dp.B)
    dF = torch.zeros_like(dp.f_occ)
    # pinned host buffers of the end-to-end leg, allocated before any plan
    hB = torch.from_numpy(np.ascontiguousarray(p.B)).pin_memory()
    hF = torch.from_numpy(np.ascontiguousarray(p.f_occ)).pin_memory()
    he = torch.from_numpy(np.ascontiguousarray(p.eps_vir)).pin_memory()
    odB = torch.empty(dB.shape, dtype=dB.dtype).pin_memory()
    odF = torch.empty(dF.shape, dtype=dF.dtype).pin_memory()

    res = {}

    def step():   # one replay of the recorded step: build, solves, combination, energy, adjoint into dB/dF
        res["E"] = ctx.graph_launch()

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
    # ---- the headline path: plan (and tune) the mixed precision, record the step as a CUDA graph, warm up.  It runs
    # first: the FP64 reference after it (pinned host copies measured up to six times slower once the FP64 plan had
    # been built and released in the same process)
    prm.precision = prec
    ctx.graph_capture(dp, prm, 1.0, dB, dF)
    graph_kernels = ctx.graph_kernels()
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    flops_exec = ctx.residual_flops()
    upd32, ev64, uncv = ctx.solve_counts()
    tuned = ctx.autotune_report()   # launch shapes picked when the mixed plan was built
    E, E_lin = res["E"]
    dBm, dFm = dB.clone(), dF.clone()

    # ---- timed region (device-resident inputs; graph replays, each read back E on the host)
    ctx.profile(True)
    l0 = ctypes_launches(osvmbe)
    with ClockSampler(local) as clk:
        ms = timed_steps(args.steps)
    launches = ctypes_launches(osvmbe) - l0
    stages = ctx.profile_read()
    ctx.profile(False)
    work = ctx.residual_work()   # the mixed solve's FP32 / FP64-accurate evaluation FLOPs

    # ---- end to end through the C ABI with host buffers: h2d of B, F, eps into the recorded step's input buffers;
    # the replay (E back to the host); d2h of dB, dF
    def e2e_step():
        dp.B.copy_(hB, non_blocking=True)
        dp.f_occ.copy_(hF, non_blocking=True)
        dp.eps_vir.copy_(he, non_blocking=True)
        ctx.graph_launch()
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
    del hB, hF, he, odB, odF

    # ---- the plain FP64 GPU path (reference point of the mixed path): its capture call (one eager step) and
    # fp64_steps timed replays (with their stage events); the residual FLOPs of its solve to tol are the metric's
    # work per step (the mixed solve's own count, FP32 iterations + FP64 evaluations, is reported beside it)
    prm.precision = 0
    ctx.graph_capture(dp, prm, 1.0, dB, dF)
    ctx.profile(True)
    fp64_ms = timed_steps(max(args.fp64_steps, 1))
    stages64 = ctx.profile_read()
    ctx.profile(False)
    E64 = res["E"][0]
    flops64 = ctx.residual_flops()
    flops_step = flops64
    grad_diff = max_abs_diff(dBm, dB)
    gradF_diff = max_abs_diff(dFm, dF)
    del dBm, dFm
    ms, flops_all = reduce_over_ranks(ms, flops_step, world, "cuda")
    value = flops_all / (ms * 1e-3) / 1e12

    # ---- roofline of the residual kernel (the metric's work) and the stage table
    total_stage = sum(v[0] for v in stages.values())
    roof = residual_roofline(stages, flops_step, prec, work, args.workload)
    roof_tc = tensor_roofline(stages, p, prm) if prec > 0 else None
    dom = max(stages.items(), key=lambda kv: kv[1][0])

    out = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f64", 2: "bf16x4+f32+f64"}[prec], "data": "synthetic",
        "config": workload_config(args.workload, prm, p),
        "gradient_s_per_geometry": ms / 1e3,
        "residual_solve_tflops": flops_step / (stages["residual"][0] / stages["residual"][1] * 1e-3) / 1e12
        if "residual" in stages else None,
        "residual_flops_per_step": flops_step,
        "residual_flops_executed_per_step": flops_exec,
        "residual_iterations": {"fp32_updates": upd32, "fp64_evals": ev64, "unconverged": uncv,
                                "clusters": len(ctx.cluster_info()[0])},
        "fp64_stage_ms": {k: v[0] for k, v in stages64.items()},
        "energy_Eh": E, "energy_linear_Eh": E_lin,
        "fp64_ms_per_step": fp64_ms, "fp64_steps_timed": max(args.fp64_steps, 1), "mixed_vs_fp64": fp64_ms / ms,
        "energy_fp64_Eh": E64, "abs_dE_vs_fp64_Eh": abs(E - E64), "max_abs_dgradB_vs_fp64": grad_diff,
        "max_abs_dgradF_vs_fp64": gradF_diff,
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
        "stage_share": {k: v[0] / total_stage for k, v in stages.items()},
        "dominant_stage": dom[0],
        "roofline": roof,
        "roofline_tensor_gemm": roof_tc,
        "e2e": {"value": flops_all / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "graph": {"kernels_per_step": int(graph_kernels),
                  "note": "each step is one replay of the whole step recorded as a CUDA graph (osv_graph_capture)"},
        "clocks": clk.summary(),
        "autotune": tuned,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def max_abs_diff(a, b, chunk=1 << 27):
    """max |a - b| in FP64, a chunk at a time (workload 4's dE/dB is 23 GB in FP64)."""
    a, b = a.reshape(-1), b.reshape(-1)
    out = 0.0
    for i in range(0, a.numel(), chunk):
        out = max(out, float((a[i:i + chunk].double() - b[i:i + chunk].double()).abs().max()))
    return out


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


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except Exception:
        return fallback, "fallback"


def source_sha(rel):
    with open(os.path.join(ROOT, "paper_2106_06149_gb300", "csrc", rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def residual_roofline(stages, flops_step, prec, work, wl):
    """The residual kernel (one persistent launch per step: k_residual<true> in the mixed path, k_residual<false> in
    the FP64 path) against the dense BF16 tensor peak measured on this machine, sustained figure (the kernel runs
    inside a long step):
    achieved = algorithmic residual FLOPs of the step / the kernel's average CUDA-event duration over the timed
    region.  The FP32-pipe view of the mixed kernel (its FP32 evaluations plus 12 FP32 instructions per
    double-float multiply-add of its FP64-accurate evaluations, against 152 SMs x 128 lanes x 2 x 2.07 GHz) is
    kept beside it."""
    if "residual" not in stages:
        return None
    ms_total, calls = stages["residual"]
    avg_ms = ms_total / calls
    peak, src = measured_peak("bf16_tflops_sustained", 1700.0)
    ach = flops_step / (avg_ms * 1e-3) / 1e12
    sha = source_sha("residual.cu")
    traffic = NCU_TRAFFIC.get((wl, prec, sha))
    out = {"bound": "tensor", "kernel": "k_residual<true>" if prec else "k_residual<false>", "stage": "residual",
           "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
           "avg_launch_ms": avg_ms, "launches": calls, "algorithmic_flops_per_launch": flops_step,
           "peak_note": f"dense BF16, {src} (MEASURED_PEAKS.json bf16_tflops_sustained)",
           "algorithmic_note": "sum over clusters of (FP64 solve's residual evaluations) x sum over coupling terms "
                               "of 2 (r_p r_q^2 + r_p^2 r_q); padding and the mixed solve's extra FP32 "
                               "iterations are not counted",
           "kernel_source_sha": sha}
    if prec and work is not None:
        f32, f64 = work
        pipe = f32 + DF_OPS_PER_FMA * f64
        out["fp32_pipe_view"] = {"achieved": pipe / (avg_ms * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
                                 "frac": pipe / (avg_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                                 "fp32_evaluation_flops": f32, "fp64_accurate_evaluation_flops": f64,
                                 "note": "FP32 pipe peak from unit counts and the 2.07 GHz maximum clock"}
    elif not prec:
        out["fp64_pipe_view"] = {"achieved": ach, "peak": FP64_PEAK_TFLOPS, "frac": ach / FP64_PEAK_TFLOPS,
                                 "note": "FP64 units, 152 SMs x 2 DFMA/clk x 2.07 GHz"}
    return out


def stage_flops(name, p, prm):
    """Algorithmic FLOPs of one launch of a dense stage (FP64 work of the method, padding excluded)."""
    nv = p.n_vir
    a = np.diff(p.aux_ptr)
    if name == "tkk_gram":
        return float(np.sum(2.0 * nv * nv * a))
    return None


def tensor_roofline(stages, p, prm):
    """The tcgen05 exact-slice GEMM of the T_kk Gram products: useful FLOPs (2 n_vir^2 a_k per LMO) per stage
    launch against the measured dense BF16 peak (burst: the stage is one batch), with the issued slice products
    (13 BF16 products per useful multiply-add) beside it.  The stage time includes the slicing passes."""
    if "tkk_gram" not in stages:
        return None
    ms_total, calls = stages["tkk_gram"]
    avg = ms_total / calls
    useful = stage_flops("tkk_gram", p, prm)
    peak, src = measured_peak("bf16_tflops", 1900.0)
    ach = useful / (avg * 1e-3) / 1e12
    return {"bound": "tensor", "stage": "tkk_gram", "kernel": "k_oz_gemm (+ k_oz_scales, k_oz_slice)",
            "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "issued_bf16_tflops": 13.0 * ach, "avg_launch_ms": avg,
            "peak_note": f"dense BF16 burst, {src}; achieved counts useful FP64-accurate FLOPs"}


# ------------------------------------------------------------------------------------- CPU baseline
def _sample_clusters(k, n):
    """n clusters of workload k spread over the orders (triples, pairs, singles in turn), deterministic."""
    import oracle
    from paper_2106_06149_gb300.synth import workload
    p, prm = workload(k)
    cl = oracle.select_clusters(p.centres, prm.r2b, prm.r3b, prm.mbe_order)
    by = [[c for c in cl if len(c) == m] for m in (1, 2, 3)]
    pick = []
    for t in range(n):
        lst = by[2 - t % 3] or by[0]
        pick.append(lst[(t * 7919) % len(lst)])
    return p, prm, pick, len(cl)


def oracle_sample(p, prm, sample):
    """Oracle energy + gradient of each sampled cluster on its own restricted problem (OSVs of its LMOs only), and
    the residual model FLOPs of the sample (same formula as the library: stored pairs, r = kept OSV dims)."""
    import torch

    import oracle
    from oracle.subproblem import restrict

    t0 = time.perf_counter()
    flops = 0.0
    for c in sample:
        q = restrict(p, c)
        m = len(c)
        g = oracle.gradient(q, prm, clusters=[tuple(range(m))])
        it = g["iters"][tuple(range(m))]
        r = {}
        for a in range(m):
            for b in range(a, m):
                r[(a, b)] = g["n_osv"][a] + (g["n_osv"][b] if a != b else 0)
        per = 0.0
        for (i, j), rp in r.items():
            for kk in range(m):
                if kk != j:
                    rq = r[(min(i, kk), max(i, kk))]
                    per += 2.0 * (rp * rq * rq + rp * rp * rq)
                if kk != i:
                    rq = r[(min(kk, j), max(kk, j))]
                    per += 2.0 * (rp * rq * rq + rp * rp * rq)
        flops += per * (it + 1)
    return flops, time.perf_counter() - t0, torch.get_num_threads()


def cpu_baseline(k, n=3):
    import torch
    torch.set_num_threads(len(os.sched_getaffinity(0)))
    p, prm, sample, ncl = _sample_clusters(k, n)
    flops, dt, cores = oracle_sample(p, prm, sample)
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": f"oracle energy+gradient of {len(sample)} clusters of the {ncl} of workload {k} (one per order, "
                      f"each on its own LMOs: OSVs of those LMOs only), FP64, torch CPU with {cores} threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch
    torch.set_num_threads(len(os.sched_getaffinity(0)))
    k = args.workload
    p, prm, sample, ncl = _sample_clusters(k, args.warmup + args.steps)
    for t in range(args.warmup):
        oracle_sample(p, prm, [sample[t]])
    tot_f, tot_t = 0.0, 0.0
    for t in range(args.steps):
        f, dt, cores = oracle_sample(p, prm, [sample[args.warmup + t]])
        tot_f += f
        tot_t += dt
    value = tot_f / tot_t / 1e12
    prm.precision = {"fp64": 0, "bf16x4": 2}[args.precision]   # the GPU arm's config, precision field included
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(k, prm, p),
           "cpu_baseline": {"value": value, "unit": "TFLOP/s", "kind": "oracle", "cores": cores,
                            "sample": f"per step, the oracle energy+gradient of one cluster of the {ncl} of workload "
                                      f"{k} (triples, pairs and singles in turn), on its own LMOs"},
           "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)

"""Run a few steps of the hot path for profilers (ncu launch lists and kernel captures) and print stage times.

    python -m paper_2106_06149_gb300.profile_step --workload 2 --steps 2
    python -m paper_2106_06149_gb300.profile_step --problem '{"n_occ": 80, "n_vir": 1500, "n_aux": 800}' \\
        --params '{"mbe_order": 1, "precision": 2}' --what build --steps 2

--what: build (osv_build), energy (osv_build -> residual -> combine -> energy) or egrad (energy + gradient_backward).
A named workload (synth.WORKLOADS) runs with its own parameters, in the mixed precision unless --params says
otherwise; a custom problem takes make_problem's keyword arguments.  Stage times (CUDA events) of the last step are
printed; nothing here changes what the library computes.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import build, osvmbe
from .synth import Params, make_problem, workload


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, default=None)
    ap.add_argument("--problem", default=None, help="make_problem keyword arguments (JSON)")
    ap.add_argument("--params", default="{}", help="Params fields (JSON)")
    ap.add_argument("--what", default="egrad", choices=["build", "energy", "egrad"])
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--tridiag-variant", type=int, default=-1,
                    help="fix the FP32 tridiagonalisation's launch shape (osv_set_tridiag_variant); -1 = tuned")
    a = ap.parse_args()
    build.build()
    osvmbe.load()
    extra = json.loads(a.params)
    if a.workload is not None:
        p, prm = workload(a.workload)
        prm.precision = 2
    else:
        kw = json.loads(a.problem or "{}")
        if kw.get("dtype") == "float32":
            kw["dtype"] = np.float32
        p, prm = make_problem(**kw), Params()
    for k, v in extra.items():
        setattr(prm, k, v)
    dp = osvmbe.DeviceProblem.from_host(p)
    ctx = osvmbe.Context()
    ctx.set_tridiag_variant(a.tridiag_variant)
    print("clusters", ctx.clusters_build(dp, prm), flush=True)
    dB = torch.zeros_like(dp.B)
    dF = torch.zeros_like(dp.f_occ)
    for s in range(a.steps):
        if s == a.steps - 1:
            ctx.profile(True)
        t0 = time.time()
        if a.what == "build":
            ctx.osv_build(dp, prm, want_counts=True)
        else:
            E, _ = osvmbe.run_energy(ctx, dp, prm)
            if a.what == "egrad":
                ctx.gradient_backward(1.0, dB, dF)
        torch.cuda.synchronize()
        print(f"step {s}: {time.time() - t0:.3f} s", flush=True)
    st = ctx.profile_read()
    print(json.dumps({k: round(v[0], 3) for k, v in st.items()}))
    if a.what != "build":
        print("residual flops", ctx.residual_flops(), "solve counts", ctx.solve_counts())
    ctx.close()


if __name__ == "__main__":
    main()

"""One-step posterior correction over the MBE collective amplitudes on the GPU (Sec. 3) against the oracle: the
residual norm at the collective amplitudes, and the pair functional before and after the step, on a distance-
truncated expansion and on one with every cluster kept (where the step moves toward the untruncated energy)."""
import numpy as np
import pytest

import oracle
from paper_2106_06149_gb300.synth import Params, make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    from paper_2106_06149_gb300 import build, osvmbe
    build.build()
    osvmbe.load()
    return osvmbe


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("cut", ["truncated", "all"])
def test_posterior_correction_matches_oracle(m, prec, cut):
    p = make_problem(6, 16, 40, seed=3)
    geo = dict(r2b=6.0, r3b=5.0) if cut == "truncated" else dict(r2b=99.0, r3b=99.0)
    prm = Params(n_osv_fixed=4, mbe_order=3, tol=1e-12, max_iter=500, precision=prec, **geo)
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    E, _ = m.run_energy(ctx, dp, prm)
    g = ctx.posterior_correction()
    o = oracle.posterior_correction(p, Params(n_osv_fixed=4, mbe_order=3, tol=1e-12, max_iter=500, **geo))
    tol = 1e-10 if prec == 0 else 1e-7
    print(f"\n{cut}, precision {prec}: E {E:.12f}; E_global {g['E_global']:.12f} (oracle {o['E_global']:.12f}); "
          f"E_corrected {g['E_corrected']:.12f} (oracle {o['E_corrected']:.12f}); dR {g['dR_max']:.3e} "
          f"(oracle {o['dR_max']:.3e})")
    assert abs(E - o["E"]) <= tol
    assert abs(g["E_global"] - o["E_global"]) <= tol
    assert abs(g["E_corrected"] - o["E_corrected"]) <= tol
    assert abs(g["dR_max"] - o["dR_max"]) <= 1e-6 * o["dR_max"] + 1e-11
    if prec == 0:   # the step's own (second-order) energy change, far below E
        assert abs((g["E_corrected"] - g["E_global"]) - (o["E_corrected"] - o["E_global"])) <= \
            1e-4 * abs(o["E_corrected"] - o["E_global"]) + 1e-13
    if cut == "all":
        full = oracle.energy(p, Params(n_osv_fixed=4, mbe_order=0, tol=1e-12, max_iter=500))["E"]
        assert abs(g["E_corrected"] - full) < abs(E - full)
    ctx.close()

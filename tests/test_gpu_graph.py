"""One whole energy + gradient step recorded as a CUDA graph (osv_graph_capture / osv_graph_launch) against the
same step run call by call: the same energy and gradient, the same kernels, replays that follow values changed in
place (a new geometry), the gradient buffers overwritten rather than added to, and the graph dropped by a
re-plan."""
import numpy as np
import pytest
import torch

from paper_2106_06149_gb300.synth import Params, make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    from paper_2106_06149_gb300 import build, osvmbe
    build.build()
    osvmbe.load()
    return osvmbe


def _eager(m, ctx, dp, prm):
    E, El = m.run_energy(ctx, dp, prm)
    dB = torch.zeros_like(dp.B)
    dF = torch.zeros_like(dp.f_occ)
    ctx.gradient_backward(1.0, dB, dF)
    torch.cuda.synchronize()
    return E, El, dB, dF


# Equal up to the run-to-run spread of the path.  FP64: rounding order only.  Mixed: the FP32 Householder
# reduction sums its columns with shared-memory atomics, so two runs of the same step differ by about 1e-11 Eh in
# E and 1e-9 in the gradient (measured on workload-sized problems of this kind); the graph must sit inside that.
SPREAD = {0: dict(E_rel=1e-12, g_rel=1e-11, g_abs=1e-15), 2: dict(E_rel=1e-10, g_rel=0.0, g_abs=2e-8)}


def _close(a, b, prec):
    """|a - b| within the spread, plus one unit in the last place where the output is FP32 (dE/dB has the dtype
    of B; two FP64-accurate values a rounding-order apart can round to neighbouring FP32 numbers)."""
    sp = SPREAD[prec]
    b64 = b.double()
    tol = sp["g_rel"] * float(b64.abs().max()) + sp["g_abs"]
    if a.dtype == torch.float32 or b.dtype == torch.float32:
        tol = tol + b64.abs() * 2.0 ** -23
    return bool(((a.double() - b64).abs() <= tol).all())


def _close_e(x, y, prec):
    return abs(x - y) <= SPREAD[prec]["E_rel"] * abs(y)


@pytest.mark.parametrize("prec,dtype", [(0, np.float64), (2, np.float32)])
def test_graph_step_matches_eager_step_and_follows_in_place_updates(m, prec, dtype):
    p = make_problem(20, 120, 400, geometry="cube", box=9.0, dmin=1.4, radius=6.0, seed=41, dtype=dtype)
    prm = Params(mbe_order=3, tol=1e-10, max_iter=400, precision=prec)
    dp = m.DeviceProblem.from_host(p)
    # one context for both: the eager steps run on the plan (and the autotuner's launch shapes) the graph recorded
    ctx = m.Context()
    counts = ctx.clusters_build(dp, prm)
    assert counts[1] > 0 and counts[2] > 0
    dB = torch.full_like(dp.B, 7.0)                          # overwritten by the step, not added to
    dF = torch.full_like(dp.f_occ, 7.0)
    ctx.graph_capture(dp, prm, 1.0, dB, dF)
    nk = ctx.graph_kernels()
    l0 = m.kernel_launches()
    E0, El0, dB0, dF0 = _eager(m, ctx, dp, prm)              # same shape: no re-plan, the graph stays
    eager_kernels = m.kernel_launches() - l0
    assert nk == eager_kernels and ctx.graph_kernels() == nk, (nk, eager_kernels)
    assert _close(dB, dB0, prec) and _close(dF, dF0, prec)      # the eager step inside the capture call
    for rep in range(2):
        dB.fill_(7.0)
        dF.fill_(7.0)
        l1 = m.kernel_launches()
        E, El = ctx.graph_launch()
        assert m.kernel_launches() - l1 == nk
        assert _close_e(E, E0, prec) and _close_e(El, El0, prec), (rep, E, E0)
        assert _close(dB, dB0, prec) and _close(dF, dF0, prec)

    # a new geometry: the values of B and F_occ change in place, the graph follows them
    g = torch.Generator(device=dp.B.device).manual_seed(5)
    dp.B.mul_(1.0 + 0.05 * torch.rand(dp.B.shape, generator=g, device=dp.B.device, dtype=dp.B.dtype))
    dp.f_occ.add_(torch.diag(0.01 * torch.rand(p.n_occ, generator=g, device=dp.B.device, dtype=torch.float64)))
    E1, El1, dB1, dF1 = _eager(m, ctx, dp, prm)
    assert abs(E1 - E0) > 1e-6
    Eg, Elg = ctx.graph_launch()
    print(f"\nprecision {prec}: {nk} kernels per step; E {E0:.12f} -> {E1:.12f}, replay {Eg:.12f}")
    assert _close_e(Eg, E1, prec) and _close_e(Elg, El1, prec), (Eg, E1)
    assert _close(dB, dB1, prec) and _close(dF, dF1, prec)

    # a re-plan drops the graph
    ctx.clusters_build(dp, prm)
    assert ctx.graph_kernels() == 0
    with pytest.raises(m.OsvError) as ei:
        ctx.graph_launch()
    assert ei.value.status == m.OSV_ERR_INVALID
    ctx.close()


def test_graph_energy_only_step(m):
    """Without gradient buffers the recorded step ends at the energy."""
    p = make_problem(10, 60, 200, geometry="cube", box=7.0, dmin=1.4, radius=5.0, seed=43)
    prm = Params(mbe_order=3, tol=1e-10, max_iter=400, precision=0)
    dp = m.DeviceProblem.from_host(p)
    ref = m.Context()
    ref.clusters_build(dp, prm)
    E0, El0 = m.run_energy(ref, dp, prm)
    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    ctx.graph_capture(dp, prm)
    E, El = ctx.graph_launch()
    assert abs(E - E0) <= 1e-12 * abs(E0) and abs(El - El0) <= 1e-12 * abs(El0)
    ctx.close()
    ref.close()

"""Failure detection without faulting the GPU: errors are injected on the host (bad inputs, impossible
iteration caps) and every call must return a status, never trap, and leave the context usable."""
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


def test_non_finite_input_is_reported_and_context_recovers(m):
    p = make_problem(4, 12, 24, seed=3)
    prm = Params(n_osv_fixed=4, mbe_order=3, r2b=9.0, r3b=9.0)
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    bad = dp.B.clone()
    bad[5] = float("nan")
    with pytest.raises(m.OsvError) as ei:
        m.run_energy(ctx, dp, prm, B=bad)
    assert ei.value.status == m.OSV_ERR_NUMERIC       # the root cause, not the eigensolver it upsets
    E, _ = m.run_energy(ctx, dp, prm)        # same context, clean input
    assert np.isfinite(E) and E < 0.0


def test_iteration_cap_reports_noconv_and_cluster_status(m):
    p = make_problem(5, 14, 30, seed=4)
    prm = Params(n_osv_fixed=4, mbe_order=3, r2b=4.0, r3b=3.5, tol=1e-14, max_iter=1)
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    ctx.osv_build(dp, prm)
    status = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(m.OsvError) as ei:
        ctx.cluster_residual_solve(want_iters=True, status=status)
    assert ei.value.status == m.OSV_ERR_NOCONV
    mem, w, e, it = ctx.cluster_info()
    n = len(w)
    assert (status[:n].cpu().numpy() == it).all()
    assert (it[[len(c[c >= 0]) > 1 for c in mem]] == -1).any()   # coupled clusters cannot converge in 1 step
    prm.max_iter = 200
    prm.tol = 1e-10
    E, _ = m.run_energy(ctx, dp, prm)
    assert np.isfinite(E)


def test_energy_reports_noconv_without_an_iteration_query(m):
    """The plain call sequence (run_energy passes no iteration query to cluster_residual_solve) must not return an
    energy as converged when some cluster hit max_iter: energy() checks every cluster's status."""
    p = make_problem(5, 14, 30, seed=4)
    prm = Params(n_osv_fixed=4, mbe_order=3, r2b=4.0, r3b=3.5, tol=1e-14, max_iter=1)
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    with pytest.raises(m.OsvError) as ei:
        m.run_energy(ctx, dp, prm)
    assert ei.value.status == m.OSV_ERR_NOCONV
    prm.max_iter, prm.tol = 200, 1e-10
    E, _ = m.run_energy(ctx, dp, prm)
    assert np.isfinite(E) and E < 0.0


def test_call_order_and_argument_errors(m):
    p = make_problem(3, 8, 12, seed=1)
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    with pytest.raises(m.OsvError) as ei:
        ctx.osv_build(dp, Params(n_osv_fixed=3))               # clusters_build first
    assert ei.value.status == m.OSV_ERR_INVALID
    with pytest.raises(m.OsvError):
        ctx.clusters_build(dp, Params(n_osv_fixed=3, max_iter=0))
    with pytest.raises(m.OsvError):
        ctx.clusters_build(dp, Params(n_osv_fixed=3, precision=7))


def test_profiler_flop_counter_and_launch_counter(m):
    import ctypes
    p = make_problem(5, 16, 30, seed=8)
    prm = Params(n_osv_fixed=5, mbe_order=3, r2b=4.0, r3b=3.5)
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    n0 = ctypes.c_longlong()
    m.load().osv_kernel_launches(ctypes.byref(n0))
    ctx.profile(True)
    m.run_energy(ctx, dp, prm)
    st = ctx.profile_read()
    ctx.profile(False)
    n1 = ctypes.c_longlong()
    m.load().osv_kernel_launches(ctypes.byref(n1))
    assert n1.value > n0.value
    for name in ("tkk_gram", "osv_eigh", "pair_basis", "residual", "energy"):
        assert name in st and st[name][0] >= 0.0 and st[name][1] == 1
    # model count: per cluster, evaluations x sum over coupling terms of 2 (r_p r_q^2 + r_p^2 r_q); every
    # multi-LMO cluster has at least its ij <- ij term with r_ij = 10 (two LMOs x 5 OSVs, none redundant)
    mem, w, e, it = ctx.cluster_info()
    multi = np.array([len(c[c >= 0]) > 1 for c in mem])
    assert (it >= 0).all()
    assert ctx.residual_flops() >= 2.0 * (2 * 10 ** 3) * (it[multi] + 1).sum()


def test_tensor_core_wait_timeout_is_reported_and_context_recovers(m):
    """The bounded pipeline waits of the tensor-core kernels (exact-slice GEMMs, cluster adjoint) are their failure
    detection.  A budget of one clock cycle makes every main-loop wait run out on purpose: the kernels raise the
    timeout word, let their committed work finish, free tensor memory and return, so energy() and
    gradient_backward() report OSV_ERR_TIMEOUT and the GPU stays usable.  The same context then reproduces, at the
    default budget, the energy and gradient of a clean run (to 1e-9: the accumulation order of atomic adds varies)."""
    p = make_problem(5, 24, 60, seed=9)
    prm = Params(n_osv_fixed=5, mbe_order=3, r2b=5.0, r3b=4.0, tol=1e-10, precision=m.OSV_MIXED_BF16X4)
    dp = m.DeviceProblem.from_host(p)
    ref = m.Context()
    ref.clusters_build(dp, prm)
    E_ref, _ = m.run_energy(ref, dp, prm)
    dB_ref = torch.zeros_like(dp.B)
    ref.gradient_backward(1.0, dB_ref)
    ref.close()

    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    ctx.set_wait_budget(1)
    with pytest.raises(m.OsvError) as ei:
        m.run_energy(ctx, dp, prm)
    assert ei.value.status == m.OSV_ERR_TIMEOUT
    ctx.set_wait_budget(0)
    E, _ = m.run_energy(ctx, dp, prm)
    assert abs(E - E_ref) <= 1e-9              # atomic accumulation orders differ run to run in the last bits
    ctx.set_wait_budget(1)                       # the adjoint's own GEMMs and cluster partials time out
    dB = torch.zeros_like(dp.B)
    with pytest.raises(m.OsvError) as ei:
        ctx.gradient_backward(1.0, dB)
    assert ei.value.status == m.OSV_ERR_TIMEOUT
    ctx.set_wait_budget(0)
    E, _ = m.run_energy(ctx, dp, prm)            # the build clears the error word
    dB.zero_()
    ctx.gradient_backward(1.0, dB)
    torch.cuda.synchronize()
    assert abs(E - E_ref) <= 1e-9
    assert (dB - dB_ref).abs().max().item() <= 1e-9
    ctx.close()

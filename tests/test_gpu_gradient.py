"""GPU parity of the adjoint (gradient_backward): dE/dB on the stored DF entries and dE/df_occ entrywise,
against the oracle's autograd gradient (itself pinned to central differences and the Euler identity).
Bar: max |d grad| <= 1e-6 and <= 1e-8 of the largest gradient entry."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06149_gb300.synth import Params, make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osvmbe():
    from paper_2106_06149_gb300 import build, osvmbe as m
    build.build()
    m.load()
    return m


def gpu_grad(m, p, prm, scale=1.0, twice=False):
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    ctx.clusters_build(dp, prm)
    E, _ = m.run_energy(ctx, dp, prm)
    dB = torch.zeros_like(dp.B)
    dF = torch.zeros_like(dp.f_occ)
    ctx.gradient_backward(scale, dB, dF)
    if twice:
        ctx.gradient_backward(scale, dB, dF)
    torch.cuda.synchronize()
    return E, dB.cpu().numpy().astype(np.float64), dF.cpu().numpy(), ctx, dp


def flat_oracle_dB(p, g):
    return np.concatenate([g["dB"][i].ravel() for i in range(p.n_occ)])


def check(m, p, prm, rel=1e-8, abs_=1e-6):
    E, dB, dF, _, _ = gpu_grad(m, p, prm)
    o = oracle.gradient(p, prm)
    ob = flat_oracle_dB(p, o)
    scale = max(np.abs(ob).max(), np.abs(o["dF"]).max())
    assert abs(E - o["E"]) <= 1e-9
    eb = np.abs(dB - ob).max()
    ef = np.abs(dF - o["dF"]).max()
    assert eb <= min(abs_, rel * scale) and ef <= min(abs_, rel * scale), (eb, ef, scale)
    return dB, dF, o


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_gradient_mbe_orders(osvmbe, order):
    p = make_problem(5, 14, 30, seed=30 + order)
    check(osvmbe, p, Params(n_osv_fixed=4, mbe_order=order, r2b=4.0, r3b=3.5, tol=1e-12, max_iter=400))


def test_gradient_threshold_osvs_and_fp32(osvmbe):
    p = make_problem(5, 20, 40, seed=41, dtype=np.float32)
    E, dB, dF, _, _ = gpu_grad(osvmbe, p, Params(l_osv=1e-3, n_osv_max=6, mbe_order=3, r2b=4.0, r3b=3.5, tol=1e-12))
    o = oracle.gradient(p, Params(l_osv=1e-3, n_osv_max=6, mbe_order=3, r2b=4.0, r3b=3.5, tol=1e-12))
    ob = flat_oracle_dB(p, o)
    # float32 output buffer: compare at float32 resolution
    assert np.abs(dB - ob).max() <= 1e-6 * np.abs(ob).max() + 1e-9
    assert np.abs(dF - o["dF"]).max() <= 1e-8 * np.abs(o["dF"]).max()


def test_gradient_local_domains(osvmbe):
    p = make_problem(6, 14, 70, geometry="cube", box=7.0, dmin=1.4, radius=4.5, seed=42)
    assert not p.full_domain()
    check(osvmbe, p, Params(n_osv_fixed=4, mbe_order=3, r2b=6.0, r3b=5.0, tol=1e-12))


def test_gradient_accumulates_and_scales(osvmbe):
    p = make_problem(4, 12, 24, seed=43)
    prm = Params(n_osv_fixed=4, mbe_order=3, r2b=9.0, r3b=9.0, tol=1e-12)
    _, dB1, dF1, _, _ = gpu_grad(osvmbe, p, prm, scale=1.0)
    _, dB2, dF2, _, _ = gpu_grad(osvmbe, p, prm, scale=0.5, twice=True)
    assert np.allclose(dB1, dB2, rtol=1e-12, atol=1e-15) and np.allclose(dF1, dF2, rtol=1e-12, atol=1e-15)


def test_euler_identity_on_gpu(osvmbe):
    p = make_problem(5, 16, 30, seed=44)
    E, dB, _, _, _ = gpu_grad(osvmbe, p, Params(n_osv_fixed=5, mbe_order=3, r2b=4.0, r3b=3.5, tol=1e-12))
    assert abs(float(np.dot(p.B.astype(np.float64), dB)) - 4.0 * E) <= 1e-10 * abs(E) + 1e-12


def test_autograd_function(osvmbe):
    p = make_problem(4, 12, 24, seed=45)
    prm = Params(n_osv_fixed=4, mbe_order=3, r2b=9.0, r3b=9.0, tol=1e-12)
    dp = osvmbe.DeviceProblem.from_host(p)
    ctx = osvmbe.Context()
    ctx.clusters_build(dp, prm)
    B = dp.B.clone().requires_grad_(True)
    F = dp.f_occ.clone().requires_grad_(True)
    E = osvmbe.Energy.apply(B, F, ctx, dp, prm)
    (3.0 * E).backward()
    o = oracle.gradient(p, prm)
    assert abs(float(E) - o["E"]) <= 1e-9
    assert np.abs(B.grad.cpu().numpy() - 3.0 * flat_oracle_dB(p, o)).max() <= 1e-9
    assert np.abs(F.grad.cpu().numpy() - 3.0 * o["dF"]).max() <= 1e-9


@pytest.mark.slow
def test_gradient_workload1_sampled(osvmbe):
    """Bench workload: the full GPU gradient against the oracle's full gradient (FP64 both)."""
    p, prm = workload(1)
    dB, dF, o = check(osvmbe, p, prm, rel=1e-8, abs_=1e-6)
    assert np.abs(dF - dF.T).max() <= 1e-6

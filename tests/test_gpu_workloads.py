"""The GPU path at the sizes of the synthetic workloads 2-4 (256-512 LMOs, n_vir 800-3000, local fitting domains,
thousands of uneven clusters), against the FP64 GPU path and the oracle:

* workload 2 (mixed precision + batching): mixed vs FP64 energy and gradient at |dE| <= 1e-6 Eh and
  max |d grad| <= 1e-6 (plus one FP32 unit in the last place where B, hence dE/dB, is FP32); cluster counts; MBE weights of every cluster against the oracle's; OSV eigenvalues and
  cluster energies of sampled LMOs and clusters against the oracle at FP64 accuracy;
* workload 3 (gradient): dE/dB and dE/dF_occ of the FP64 and mixed paths against central finite differences of
  the oracle energy on 200 random entries (tests/golden/fd_workload3.json, written by
  tests/golden/make_fd_workload3.py from oracle/ only): max |d| <= 1e-6 against the fourth-order stencil at step
  1e-4, and <= 1e-6 plus the stencil's rounding-noise floor against the one at step 1e-5;
* workload 4 (large energy + gradient): mixed vs FP64 energy and gradient at the same bars, and the FP64 energy of
  a sampled triple cluster against the oracle.

The oracle runs each sampled cluster on the problem restricted to its own LMOs (oracle/subproblem.py): a cluster's
Hylleraas energy depends only on them."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from oracle.subproblem import restrict
from paper_2106_06149_gb300.synth import workload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(os.path.abspath(__file__))
TOL_E_MIXED = 1e-6
TOL_GRAD = 1e-6


@pytest.fixture(scope="module")
def m():
    from paper_2106_06149_gb300 import build, osvmbe
    build.build()
    osvmbe.load()
    return osvmbe


def _grad_excess(g, g64):
    """Largest excess of |g - g64| over the bar: 1e-6, plus one unit in the last place of g64 when the gradient is
    returned in FP32 (dE/dB has the dtype of B; both paths round their FP64-accurate values to it once)."""
    d = (g.double() - g64.double()).abs()
    tol = TOL_GRAD + (g64.double().abs() * 2.0 ** -23 if g.dtype == torch.float32 else 0.0)
    return float((d - tol).max()), float(d.max())


def _egrad(m, dp, prm, grad=True):
    ctx = m.Context()
    counts = ctx.clusters_build(dp, prm)
    nosv = ctx.osv_build(dp, prm, want_counts=True)
    ctx.cluster_residual_solve()
    ctx.mbe3_combine()
    E, El = ctx.energy()
    dB = dF = None
    if grad:
        dB = torch.zeros_like(dp.B)
        dF = torch.zeros_like(dp.f_occ)
        ctx.gradient_backward(1.0, dB, dF)
        torch.cuda.synchronize()
    return ctx, dict(E=E, E_linear=El, counts=counts, nosv=nosv, dB=dB, dF=dF)


def _sample(members, weights, order, k=2):
    """k clusters of the given order, spread over the list (deterministic)."""
    idx = [q for q in range(len(members)) if (members[q] >= 0).sum() == order]
    return [idx[(t * len(idx)) // k] for t in range(k)]


def _oracle_cluster_energy(p, prm, members, nosv):
    c = tuple(int(x) for x in members if x >= 0)
    q = restrict(p, c)
    out = oracle.energy(q, prm, n_osv=[int(nosv[x]) for x in c], clusters=[tuple(range(len(c)))])
    return out["E"]


def test_workload2_mixed_vs_fp64_and_oracle_samples(m):
    p, prm = workload(2)
    prm.precision = 0
    dp = m.DeviceProblem.from_host(p)
    c64, r64 = _egrad(m, dp, prm)
    assert r64["counts"] == [256, 5212, 8872]
    assert (r64["nosv"] == 40).all()
    mem, w, ec, it = c64.cluster_info()
    # MBE weights of every cluster against the oracle's inclusion-exclusion weights on the same cluster list
    cl = oracle.select_clusters(p.centres, prm.r2b, prm.r3b, prm.mbe_order)
    ow = oracle.mbe_weights(cl)
    assert len(cl) == len(w)
    for row, wt in zip(mem, w):
        assert ow[tuple(int(x) for x in row if x >= 0)] == wt
    # FP64 cluster energies of sampled clusters and OSV eigenvalues of their LMOs against the oracle
    for order in (1, 2, 3):
        for q in _sample(mem, w, order, k=1):
            Eo = _oracle_cluster_energy(p, prm, mem[q], r64["nosv"])
            assert abs(ec[q] - Eo) <= max(1e-9, 1e-12 * abs(Eo)), (mem[q], ec[q], Eo)
    eps = torch.as_tensor(p.eps_vir, dtype=torch.float64)
    for k in (0, 131):
        wo, _ = oracle.osv_decompose(oracle.tkk(oracle.dense_B(p, k), eps, torch.tensor(p.f_occ[k, k])))
        wg = c64.eigenvalues(k, p.n_vir)
        assert np.abs(wg - wo.numpy()).max() <= 1e-12 * float(wo.abs().max())
    c64.close()
    dB64, dF64, E64 = r64["dB"], r64["dF"], r64["E"]
    del r64
    prm.precision = 2
    cmx, rmx = _egrad(m, dp, prm)
    cmx.close()
    dE = rmx["E"] - E64
    xb, gb = _grad_excess(rmx["dB"], dB64)
    xf, gf = _grad_excess(rmx["dF"], dF64)
    print(f"\nworkload 2: E = {E64:.9f}, mixed - fp64: dE = {dE:.3e} Eh, max|d dB| = {gb:.3e} (FP32 output), "
          f"max|d dF| = {gf:.3e}")
    assert abs(dE) <= TOL_E_MIXED
    assert xb <= 0.0 and xf <= 0.0


# Rounding noise of a finite difference at step h: each oracle energy is known to about 1e-14 |E| (eigensolves,
# iterations and sums over hundreds of clusters), and the fourth-order stencil divides about that by h.
FD_NOISE_REL = 2e-14


def test_workload3_gradients_vs_oracle_finite_differences(m):
    with open(os.path.join(HERE, "golden", "fd_workload3.json")) as f:
        gold = json.load(f)
    p, prm = workload(3)
    assert gold["workload"] == 3 and gold["params"]["n_osv_max"] == prm.n_osv_max and gold["steps"] == [1e-5, 1e-4]
    dp = m.DeviceProblem.from_host(p)
    worst = {}
    for prec in (0, 2):
        prm.precision = prec
        ctx, r = _egrad(m, dp, prm)
        for k, n in gold["n_osv"].items():       # the OSV counts frozen by the finite differences
            assert int(r["nosv"][int(k)]) == n
        dB = r["dB"].cpu().numpy()
        dF = r["dF"].cpu().numpy()
        ctx.close()
        err = [0.0, 0.0]
        for e in gold["entries"]:
            if e["kind"] == "B":
                i, a, P = e["idx"]
                g = dB[int(p.aux_ptr[i]) * p.n_vir + a * p.a(i) + P]
            else:
                x, y = e["idx"]
                g = dF[x, y]
            d4, d5 = abs(g - e["fd4_1e-4"]), abs(g - e["fd4_1e-5"])
            err = [max(err[0], d4), max(err[1], d5)]
            assert d4 <= TOL_GRAD, (prec, e, g)
            assert d5 <= TOL_GRAD + FD_NOISE_REL * abs(e["E_reached"]) / 1e-5, (prec, e, g)
        worst[prec] = err
    print(f"\nworkload 3: max |grad - FD| over {len(gold['entries'])} entries, step 1e-4 / 1e-5: "
          f"FP64 {worst[0][0]:.2e} / {worst[0][1]:.2e}, mixed {worst[2][0]:.2e} / {worst[2][1]:.2e}")


def test_workload4_mixed_vs_fp64_energy_and_gradient(m):
    p, prm = workload(4)
    dp = m.DeviceProblem.from_host(p)
    prm.precision = 0
    c64, r64 = _egrad(m, dp, prm)
    assert r64["counts"] == [512, 8730, 10776]
    mem, w, ec, it = c64.cluster_info()
    q = _sample(mem, w, 3, k=1)[0]
    Eo = _oracle_cluster_energy(p, prm, mem[q], r64["nosv"])
    assert abs(ec[q] - Eo) <= max(1e-9, 1e-12 * abs(Eo)), (mem[q], ec[q], Eo)
    c64.close()
    E64, dB64, dF64 = r64["E"], r64["dB"], r64["dF"]
    del r64
    torch.cuda.empty_cache()
    prm.precision = 2
    cmx, rmx = _egrad(m, dp, prm)
    cmx.close()
    dE = rmx["E"] - E64
    xb, gb = _grad_excess(rmx["dB"], dB64)
    xf, gf = _grad_excess(rmx["dF"], dF64)
    print(f"\nworkload 4: E = {E64:.9f}, mixed - fp64: dE = {dE:.3e} Eh, max|d dB| = {gb:.3e} (FP32 output), "
          f"max|d dF| = {gf:.3e}")
    assert abs(dE) <= TOL_E_MIXED
    assert xb <= 0.0 and xf <= 0.0

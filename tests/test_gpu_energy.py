"""GPU parity of the energy path (osv_build -> cluster_residual_solve -> mbe3_combine -> energy, FP64)
against the CPU oracle, element by element where the quantity is unique (eigenvalues, per-cluster energies,
MBE weights) and on the total energy.  Tolerance of the FP64 path: |dE| <= 1e-9 Eh."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06149_gb300.synth import Params, make_problem, workload

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9


@pytest.fixture(scope="module")
def osvmbe():
    from paper_2106_06149_gb300 import build, osvmbe as m
    build.build()
    m.load()
    return m


def gpu_run(m, p, prm):
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    counts = ctx.clusters_build(dp, prm)
    nosv = ctx.osv_build(dp, prm, want_counts=True)
    it = ctx.cluster_residual_solve(want_iters=True)
    ctx.mbe3_combine()
    E, El = ctx.energy()
    mem, w, ec, iters = ctx.cluster_info()
    return dict(E=E, E_linear=El, counts=counts, nosv=nosv, iters=it, members=mem, weights=w, Ec=ec,
                cl_iters=iters, ctx=ctx, dp=dp)


def cluster_key(row):
    return tuple(int(x) for x in row if x >= 0)


def compare(m, p, prm, tol=TOL_FP64, per_cluster=True):
    g = gpu_run(m, p, prm)
    o = oracle.energy(p, prm)
    assert list(g["nosv"]) == o["n_osv"]
    assert abs(g["E"] - o["E"]) <= tol, (g["E"], o["E"], g["E"] - o["E"])
    if per_cluster and prm.mbe_order != 0:
        for row, w, e in zip(g["members"], g["weights"], g["Ec"]):
            c = cluster_key(row)
            assert o["weights"][c] == w
            assert abs(o["per_cluster"][c] - e) <= tol, (c, e, o["per_cluster"][c])
    return g, o


@pytest.mark.parametrize("n,nv,na,seed", [(1, 6, 10, 0), (2, 9, 14, 1), (4, 12, 30, 2), (6, 20, 50, 3)])
def test_full_cluster_matches_oracle(osvmbe, n, nv, na, seed):
    p = make_problem(n, nv, na, seed=seed)
    compare(osvmbe, p, Params(n_osv_fixed=min(5, nv), mbe_order=0, tol=1e-11, max_iter=300))


@pytest.mark.parametrize("order", [1, 2, 3])
def test_mbe_orders_match_oracle(osvmbe, order):
    p = make_problem(7, 18, 40, seed=10 + order)
    compare(osvmbe, p, Params(n_osv_fixed=5, mbe_order=order, r2b=5.0, r3b=3.5, tol=1e-11, max_iter=300))


def test_threshold_selection_and_cap(osvmbe):
    p = make_problem(5, 30, 60, seed=4)
    compare(osvmbe, p, Params(l_osv=2e-3, n_osv_max=7, mbe_order=3, r2b=4.0, r3b=3.5, tol=1e-11))


def test_complete_osvs_reach_the_canonical_limit(osvmbe):
    from tests.test_oracle_pins import canonical_df_mp2
    p = make_problem(4, 10, 28, seed=0)
    g = gpu_run(osvmbe, p, Params(n_osv_fixed=10, mbe_order=0, tol=1e-12, max_iter=500))
    assert abs(g["E"] - canonical_df_mp2(p)) <= 1e-10


def test_local_fitting_domains(osvmbe):
    p = make_problem(6, 16, 80, geometry="cube", box=7.0, dmin=1.4, radius=4.5, seed=5)
    assert not p.full_domain()
    compare(osvmbe, p, Params(n_osv_fixed=5, mbe_order=3, r2b=6.0, r3b=5.0, tol=1e-11))


def test_rank_deficient_tkk_and_fp32_B(osvmbe):
    p = make_problem(4, 24, 10, seed=6)                # n_aux < n_vir: T_kk has a null space
    compare(osvmbe, p, Params(n_osv_fixed=8, mbe_order=3, r2b=9.0, r3b=9.0, tol=1e-11))
    q = make_problem(4, 16, 30, seed=7, dtype=np.float32)
    compare(osvmbe, q, Params(n_osv_fixed=5, mbe_order=3, r2b=9.0, r3b=9.0, tol=1e-11))


def test_workload0_full_osv_mp2(osvmbe):
    p, prm = workload(0)
    g, o = compare(osvmbe, p, prm)
    assert g["counts"] == [1, 0, 0]


@pytest.mark.slow
def test_workload1_bench_configuration(osvmbe):
    """The bench workload (64 LMOs, n_vir 400, n_aux 1600): cluster counts, OSV counts and eigenvalues of
    sampled LMOs, per-cluster energies of sampled clusters, and the total energy."""
    p, prm = workload(1)
    g = gpu_run(osvmbe, p, prm)
    assert g["counts"] == [64, 305, 364]
    o = oracle.energy(p, prm)
    assert list(g["nosv"]) == o["n_osv"]
    for k in (0, 17, 63):
        w = g["ctx"].eigenvalues(k, p.n_vir)
        assert np.allclose(w, o["osv_eigs"][k].numpy(), rtol=0, atol=1e-12 * float(np.abs(w).max()))
    for row, wt, e in zip(g["members"], g["weights"], g["Ec"]):
        c = cluster_key(row)
        assert o["weights"][c] == wt
        assert abs(o["per_cluster"][c] - e) <= TOL_FP64 * max(1.0, abs(e)) , (c, e, o["per_cluster"][c])
    assert abs(g["E"] - o["E"]) <= max(TOL_FP64, 1e-12 * abs(o["E"])), (g["E"], o["E"])


def test_syev_batched_matches_lapack(osvmbe):
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 17, 80, 257):
        X = rng.standard_normal((3, n, n))
        A = X + X.transpose(0, 2, 1)
        w, Zt = osvmbe.syev_batched(torch.from_numpy(A).cuda())
        w, Zt = w.cpu().numpy(), Zt.cpu().numpy()
        for b in range(3):
            ref = np.sort(np.linalg.eigvalsh(A[b]))[::-1]
            scale = np.abs(ref).max()
            assert np.allclose(w[b], ref, atol=1e-12 * scale)
            Z = Zt[b].T
            assert np.abs(Z.T @ Z - np.eye(n)).max() <= 1e-12 * n
            assert np.abs(A[b] @ Z - Z * w[b][None, :]).max() <= 1e-12 * scale * n


def test_invalid_inputs_are_rejected(osvmbe):
    p = make_problem(3, 8, 12, seed=1)
    p.aux_idx[[0, 1]] = p.aux_idx[[1, 0]]              # unsorted fitting domain
    dp = osvmbe.DeviceProblem.from_host(p)
    ctx = osvmbe.Context()
    with pytest.raises(osvmbe.OsvError) as ei:
        ctx.clusters_build(dp, Params(n_osv_fixed=3))
    assert ei.value.status == osvmbe.OSV_ERR_INVALID
    with pytest.raises(osvmbe.OsvError):
        ctx.cluster_residual_solve()


def test_collective_amplitudes_and_linear_energy_match_oracle(osvmbe):
    """mbe3_combine (Eqs. 28-32) on a truncated MBE(3) case, where the cluster weights are not trivial: for every
    ordered pair of a selected cluster, the collective amplitudes in the canonical virtual space,
    t_ij = (Q_i Q_j) T_(ij,ij) (Q_i Q_j)^T (independent of the OSV signs and of the pair basis), equal the
    oracle's; and E_linear = sum_ij <K_(ij,ij), 2T - T^T> over the collective amplitudes equals the oracle's.  A
    wrong weight, sign or pair index in the combination fails here even where the total energy would not."""
    p = make_problem(7, 18, 40, seed=12)
    prm = Params(n_osv_fixed=5, mbe_order=3, r2b=5.0, r3b=3.5, tol=1e-12, max_iter=400)
    g = gpu_run(osvmbe, p, prm)
    o = oracle.energy(p, prm)
    assert sorted(set(o["weights"].values())) != [1]          # truncated: some weights differ from one
    assert abs(g["E_linear"] - o["E_linear"]) <= 1e-9, (g["E_linear"], o["E_linear"])
    worst = 0.0
    for (i, j), T in o["collective"].items():
        P = torch.cat([o["Q"][i], o["Q"][j]], dim=1) if i != j else o["Q"][i]
        t_ref = (P @ T @ P.T).numpy()
        t_gpu = g["ctx"].pair_amplitudes(i, j, p.n_vir)
        worst = max(worst, float(np.abs(t_gpu - t_ref).max()))
        assert np.abs(t_gpu - t_ref).max() <= 1e-10 * max(1.0, np.abs(t_ref).max()), (i, j)
    print(f"\nmax |t_gpu - t_oracle| over {len(o['collective'])} ordered pairs: {worst:.2e}")

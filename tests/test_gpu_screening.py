"""OSV-overlap cluster screening on the GPU (Sec. 2.2.1, Eqs. 2bscreen and 3bscreen) against the oracle: the metric
s2b of every pair of LMOs, the 2b/3b cluster lists it selects, and the MBE(3) energy over those clusters."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_06149_gb300.synth import Params, make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    from paper_2106_06149_gb300 import build, osvmbe
    build.build()
    osvmbe.load()
    return osvmbe


def _oracle_metric(p, n_osv):
    eps = torch.as_tensor(p.eps_vir, dtype=torch.float64)
    Q = []
    for k in range(p.n_occ):
        _, U = oracle.osv_decompose(oracle.tkk(oracle.dense_B(p, k), eps, torch.tensor(p.f_occ[k, k])))
        Q.append(U[:, :n_osv].numpy())
    return oracle.osv_overlap_metric(Q)


def _cut_between(values, q):
    """A threshold halfway between two adjacent distinct values around quantile q (never on a value)."""
    v = np.unique(np.round(np.asarray(values), 12))
    t = min(max(int(q * len(v)), 1), len(v) - 1)
    return 0.5 * (v[t - 1] + v[t])


@pytest.mark.parametrize("prec", [0, 2])
def test_overlap_metric_selection_and_energy_match_oracle(m, prec):
    p = make_problem(8, 30, 90, geometry="cube", box=8.0, dmin=1.4, radius=6.0, seed=21)
    prm = Params(n_osv_fixed=6, mbe_order=3, tol=1e-12, max_iter=400, precision=prec)
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    s_gpu = ctx.osv_overlap_metric(dp, prm)
    s_ref = _oracle_metric(p, 6)
    tol_s = 1e-10 if prec == 0 else 1e-8
    assert np.abs(s_gpu - s_ref).max() <= tol_s, np.abs(s_gpu - s_ref).max()
    assert np.abs(np.diag(s_gpu) - 1.0).max() <= tol_s            # s_ii = 1 (orthonormal OSVs)
    assert s_gpu.min() >= -tol_s and s_gpu.max() <= 1.0 + tol_s
    n = p.n_occ
    off = [s_ref[i, j] for i in range(n) for j in range(i + 1, n)]
    l2b = _cut_between(off, 0.5)
    means = [(s_ref[i, j] + s_ref[i, k] + s_ref[j, k]) / 3.0 for i in range(n) for j in range(i + 1, n)
             for k in range(j + 1, n)]
    l3b = _cut_between(means, 0.7)
    cl_ref = oracle.select_clusters_osv(s_ref, l2b, l3b, 3)
    counts = ctx.clusters_build_osv(dp, prm, s_gpu, l2b, l3b)
    assert counts == [sum(len(c) == q for c in cl_ref) for q in (1, 2, 3)]
    assert counts[1] > 0 and counts[2] > 0
    E, _ = m.run_energy(ctx, dp, prm)
    mem, w, ec, it = ctx.cluster_info()
    assert sorted(tuple(int(x) for x in r if x >= 0) for r in mem) == sorted(cl_ref)
    Eo = oracle.energy(p, Params(n_osv_fixed=6, mbe_order=3, tol=1e-12, max_iter=400), clusters=cl_ref)["E"]
    tol_e = 1e-9 if prec == 0 else 1e-6
    print(f"\nprecision {prec}: l2b {l2b:.4f}, l3b {l3b:.4f}, clusters {counts}, E {E:.12f}, oracle {Eo:.12f}")
    assert abs(E - Eo) <= tol_e
    ctx.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_weak_pair_one_block_energies_match_oracle(m, prec):
    """The one-block scheme for weak 2b clusters (Sec. 2.2.2): every pair that the metric leaves out of the strong
    clusters but keeps above the discard threshold gets one-block amplitudes and an energy.  The number of weak
    pairs, their total energy and the screened MBE energy (strong clusters + weak pairs) against
    oracle.energy_osv_screened, which iterates each one-block equation to 1e-12."""
    p = make_problem(8, 30, 90, geometry="cube", box=8.0, dmin=1.4, radius=6.0, seed=21)
    base = dict(n_osv_fixed=6, mbe_order=3, tol=1e-12, max_iter=400)
    prm = Params(**base, precision=prec)
    dp = m.DeviceProblem.from_host(p)
    ctx = m.Context()
    s_gpu = ctx.osv_overlap_metric(dp, prm)
    s_ref = _oracle_metric(p, 6)
    n = p.n_occ
    off = [s_ref[i, j] for i in range(n) for j in range(i + 1, n)]
    l2b = _cut_between(off, 0.5)
    means = [(s_ref[i, j] + s_ref[i, k] + s_ref[j, k]) / 3.0 for i in range(n) for j in range(i + 1, n)
             for k in range(j + 1, n)]
    l3b = _cut_between(means, 0.7)
    l_discard = _cut_between(off, 0.1)      # some pairs are dropped outright, the rest of the non-strong are weak
    ctx.clusters_build_osv(dp, prm, s_gpu, l2b, l3b)
    E_strong, _ = m.run_energy(ctx, dp, prm)
    E_weak, n_weak = ctx.weak_pairs_energy(s_gpu, l2b, l_discard)
    o = oracle.energy_osv_screened(p, Params(**base), l2b, l3b, l_discard=l_discard)
    tol = 1e-9 if prec == 0 else 1e-6
    print(f"\nprecision {prec}: {n_weak} weak pairs, E_weak {E_weak:.12f} (oracle {o['E_weak']:.12f}), "
          f"E {E_strong + E_weak:.12f} (oracle {o['E']:.12f})")
    assert n_weak == len(o["weak_pairs"]) and n_weak > 0
    assert abs(E_weak - o["E_weak"]) <= tol
    assert abs(E_strong + E_weak - o["E"]) <= tol
    ctx.close()

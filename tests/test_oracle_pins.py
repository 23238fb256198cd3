"""Pins of the CPU oracle against facts the paper and the mathematics fix (no GPU).

Each pin is computed independently of the oracle's own formulation:
  P1  canonical limit: complete OSVs + one full cluster == brute-force canonical DF-MP2 (Sec. 2.1: OSV-MP2
      with untruncated OSVs spans the whole virtual space);
  P2  MBE exactness: all clusters kept and N <= 3 (or decoupled subsystems) == full OSV-MP2 (Eqs. 28-34);
  P6  brute-force Galerkin solve of the virtual-space pair equations (Eq. 4 projected on each pair domain);
  P5  invariances (LMO relabelling, orthogonal aux rotation, common energy shift);
  P10 T_kk is positive semidefinite (Eq. 6 elements are a Schur product of a Gram and a Cauchy matrix);
  P9  Hylleraas functional error is quadratic in the amplitude error (Eq. 3);
  P7  autograd gradient == central finite differences; P8 Euler identity sum B dE/dB = 4 E.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_2106_06149_gb300.synth import Params, Problem, make_problem

DT = torch.float64


def canonical_df_mp2(problem):
    """E = sum_ijab (ia|jb)[2(ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b) in canonical occupied orbitals."""
    n, nv = problem.n_occ, problem.n_vir
    Bs = np.stack([problem.B_dense(i) for i in range(n)])               # (n, nv, naux)
    e_occ, U = np.linalg.eigh(problem.f_occ)
    Bc = np.einsum("ji,jap->iap", U, Bs)                                # canonical MOs phi_i = sum_j U_ji phi_j
    iajb = np.einsum("iap,jbp->iajb", Bc, Bc)
    eps = problem.eps_vir
    den = e_occ[:, None, None, None] + e_occ[None, None, :, None] - eps[None, :, None, None] - eps[None, None, None, :]
    return float(np.sum(iajb * (2.0 * iajb - iajb.transpose(0, 3, 2, 1)) / den))


def galerkin_energy(problem, Q, clusters_all=True):
    """Solve the projected pair equations of one full cluster as one dense linear system.

    Unknowns: X_ij in an orthonormal basis Phi_ij of range(Q_i Q_j) (SVD), t_ij = Phi X Phi^T.  Equations:
    Phi_ij^T [K_ij + eps t_ij + t_ij eps - sum_k (f_kj t_ik + f_ik t_kj)] Phi_ij = 0 for every ordered pair."""
    n, nv = problem.n_occ, problem.n_vir
    Bs = [problem.B_dense(i) for i in range(n)]
    f, eps = problem.f_occ, problem.eps_vir
    Qn = [q.numpy() for q in Q]
    pairs = [(i, j) for i in range(n) for j in range(n)]
    Phi = {}
    for (i, j) in pairs:
        P = Qn[i] if i == j else np.concatenate([Qn[i], Qn[j]], axis=1)
        u, s, _ = np.linalg.svd(P, full_matrices=False)
        Phi[(i, j)] = u[:, s > 1e-6]
    off, tot = {}, 0
    for p in pairs:
        off[p] = tot
        tot += Phi[p].shape[1] ** 2
    A = np.zeros((tot, tot))
    rhs = np.zeros(tot)
    E = np.diag(eps)
    for (i, j) in pairs:
        Pp = Phi[(i, j)]
        r = Pp.shape[1]
        rows = slice(off[(i, j)], off[(i, j)] + r * r)
        rhs[rows] = -(Pp.T @ Bs[i] @ Bs[j].T @ Pp).ravel()

        def add(q, coef_left, transpose=False):
            # contribution of t_q (virtual) = Phi_q X_q Phi_q^T mapped through M -> Pp^T op(M) Pp
            Pq = Phi[q]
            rq = Pq.shape[1]
            cols = slice(off[q], off[q] + rq * rq)
            for a in range(rq):
                for b in range(rq):
                    Xu = np.zeros((rq, rq))
                    Xu[a, b] = 1.0
                    t = Pq @ Xu @ Pq.T
                    A[rows, off[q] + a * rq + b] += (Pp.T @ coef_left(t) @ Pp).ravel()

        add((i, j), lambda t: E @ t + t @ E)
        for k in range(n):
            add((i, k), lambda t, k=k: -f[k, j] * t)
            add((k, j), lambda t, k=k: -f[i, k] * t)
    x = np.linalg.solve(A, rhs)
    Etot = 0.0
    for (i, j) in pairs:
        Pp = Phi[(i, j)]
        r = Pp.shape[1]
        t = Pp @ x[off[(i, j)]:off[(i, j)] + r * r].reshape(r, r) @ Pp.T
        Etot += np.sum((Bs[i] @ Bs[j].T) * (2.0 * t - t.T))
    return Etot


def _cut_all():
    return dict(r2b=1e9, r3b=1e9)


# ------------------------------------------------------------------------------------------------ P1
@pytest.mark.parametrize("seed", [0, 1])
def test_canonical_limit_full_cluster(seed):
    p = make_problem(4, 10, 28, seed=seed)
    prm = Params(n_osv_fixed=10, mbe_order=0, tol=1e-11, max_iter=400)
    e = oracle.energy(p, prm)["E"]
    ref = canonical_df_mp2(p)
    assert abs(e - ref) <= 1e-10 * max(1.0, abs(ref)), (e, ref)


def test_canonical_limit_mbe3_three_lmos():
    p = make_problem(3, 9, 20, seed=5)
    prm = Params(n_osv_fixed=9, mbe_order=3, tol=1e-11, max_iter=400, **_cut_all())
    e = oracle.energy(p, prm)["E"]
    assert abs(e - canonical_df_mp2(p)) <= 1e-10


def test_canonical_limit_local_domains():
    p = make_problem(4, 8, 40, geometry="cube", box=6.0, dmin=1.4, radius=4.0, seed=7)
    assert not p.full_domain()
    prm = Params(n_osv_fixed=8, mbe_order=0, tol=1e-11, max_iter=400)
    assert abs(oracle.energy(p, prm)["E"] - canonical_df_mp2(p)) <= 1e-10


# ------------------------------------------------------------------------------------------------ P2
@pytest.mark.parametrize("n", [2, 3])
def test_mbe_exact_for_small_n(n):
    p = make_problem(n, 14, 30, seed=11 + n)
    full = oracle.energy(p, Params(n_osv_fixed=5, mbe_order=0, tol=1e-11))
    mbe = oracle.energy(p, Params(n_osv_fixed=5, mbe_order=3, tol=1e-11, **_cut_all()))
    assert abs(full["E"] - mbe["E"]) <= 1e-11
    # collective amplitudes equal the full-cluster amplitudes (Eqs. 28-32)
    for pr, T in full["amplitudes"][tuple(range(n))].items():
        assert torch.allclose(mbe["collective"][pr], T, atol=1e-10)


def _merge(a: Problem, b: Problem, shift=500.0):
    """Two problems side by side: disjoint aux sets, no occupied Fock coupling between them."""
    na, nb = a.n_occ, b.n_occ
    assert a.n_vir == b.n_vir
    f = np.zeros((na + nb, na + nb))
    f[:na, :na] = a.f_occ
    f[na:, na:] = b.f_occ
    cb = b.centres.copy()
    cb[:, 0] += shift
    blocks, ptr, idx = [], [0], []
    for src, base in ((a, 0), (b, a.n_aux)):
        for i in range(src.n_occ):
            blocks.append(src.B_block(i).ravel())
            idx.append(src.aux_idx[src.aux_ptr[i]:src.aux_ptr[i + 1]] + base)
            ptr.append(ptr[-1] + src.a(i))
    return Problem(centres=np.concatenate([a.centres, cb]), aux_centres=np.concatenate([a.aux_centres, b.aux_centres]),
                   f_occ=f, eps_vir=a.eps_vir, aux_ptr=np.asarray(ptr, np.int64),
                   aux_idx=np.concatenate(idx).astype(np.int32), B=np.concatenate(blocks))


def test_mbe_exact_for_decoupled_subsystems():
    a = make_problem(2, 12, 20, seed=21)
    b = make_problem(2, 12, 20, seed=22)
    b.eps_vir = a.eps_vir
    p = _merge(a, b)
    prm = dict(n_osv_fixed=5, tol=1e-11)
    full = oracle.energy(p, Params(mbe_order=0, **prm))["E"]
    mbe = oracle.energy(p, Params(mbe_order=3, **prm, **_cut_all()))
    assert len(mbe["clusters"]) == 4 + 6 + 4
    assert abs(full - mbe["E"]) <= 1e-11
    ea = oracle.energy(a, Params(mbe_order=0, **prm))["E"]
    eb = oracle.energy(b, Params(mbe_order=0, **prm))["E"]
    assert abs(full - ea - eb) <= 1e-11


def test_mbe_weights_moebius():
    """sum of w_c over clusters containing any selected set s is 1 (inclusion-exclusion)."""
    p = make_problem(12, 4, 4, seed=3)
    cl = oracle.select_clusters(p.centres, 8.0, 6.0, 3)
    w = oracle.mbe_weights(cl)
    for s in cl:
        assert sum(w[c] for c in cl if set(s) <= set(c)) == 1
    # chain spacing 1.5 A: pairs |i-j| <= 5, triples of span <= 4
    n = 12
    assert sum(len(c) == 2 for c in cl) == sum(1 for i in range(n) for j in range(i + 1, n) if j - i <= 5)
    assert sum(len(c) == 3 for c in cl) == sum(1 for c in itertools.combinations(range(n), 3) if c[2] - c[0] <= 4)


# ------------------------------------------------------------------------------------------------ P6
@pytest.mark.parametrize("seed,asym", [(0, False), (4, False), (8, True)])
def test_bruteforce_galerkin(seed, asym):
    p = make_problem(3, 7, 16, seed=seed)
    if asym:
        # an asymmetric occupied Fock matrix tells f_kj from f_jk and K_ij from K_ji in Eq. 4
        p.f_occ = p.f_occ + np.triu(np.full((3, 3), 0.03), 1)
    prm = Params(n_osv_fixed=3, mbe_order=0, tol=1e-12, max_iter=500)
    out = oracle.energy(p, prm)
    ref = galerkin_energy(p, out["Q"])
    assert abs(out["E"] - ref) <= 1e-11 * max(1.0, abs(ref)), (out["E"], ref)


# ------------------------------------------------------------------------------------------------ P5
def test_invariances():
    p = make_problem(4, 10, 20, seed=9)
    prm = Params(n_osv_fixed=4, mbe_order=3, tol=1e-11, **_cut_all())
    e0 = oracle.energy(p, prm)["E"]
    # LMO relabelling
    perm = np.array([2, 0, 3, 1])
    blocks = [p.B_block(i).ravel() for i in perm]
    q = Problem(centres=p.centres[perm], aux_centres=p.aux_centres, f_occ=p.f_occ[np.ix_(perm, perm)],
                eps_vir=p.eps_vir, aux_ptr=p.aux_ptr, aux_idx=p.aux_idx, B=np.concatenate(blocks))
    assert abs(oracle.energy(q, prm)["E"] - e0) <= 1e-11
    # common orthogonal rotation of the aux index (full domains)
    O, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((p.n_aux, p.n_aux)))
    blocks = [(p.B_block(i) @ O).ravel() for i in range(p.n_occ)]
    q = Problem(centres=p.centres, aux_centres=p.aux_centres, f_occ=p.f_occ, eps_vir=p.eps_vir,
                aux_ptr=p.aux_ptr, aux_idx=p.aux_idx, B=np.concatenate(blocks))
    assert abs(oracle.energy(q, prm)["E"] - e0) <= 1e-11
    # shift of all orbital energies: (eps + c, F + c 1)
    c = 0.37
    q = Problem(centres=p.centres, aux_centres=p.aux_centres, f_occ=p.f_occ + c * np.eye(p.n_occ),
                eps_vir=p.eps_vir + c, aux_ptr=p.aux_ptr, aux_idx=p.aux_idx, B=p.B)
    assert abs(oracle.energy(q, prm)["E"] - e0) <= 1e-11


def test_osv_selection_keeps_largest_eigenvalues():
    """Q_k spans the eigenvectors of T_kk with the n_k largest eigenvalues (Sec. 2.1, Eq. 6): the trace of
    Q^T T_kk Q equals the sum of the n_k largest eigenvalues; T_kk built here element by element."""
    p = make_problem(3, 12, 20, seed=17)
    out = oracle.energy(p, Params(n_osv_fixed=4, mbe_order=1))
    for k in range(p.n_occ):
        Bk = p.B_dense(k)
        T = np.empty((p.n_vir, p.n_vir))
        for a in range(p.n_vir):
            for b in range(p.n_vir):
                T[a, b] = np.dot(Bk[a], Bk[b]) / (p.eps_vir[a] + p.eps_vir[b] - 2.0 * p.f_occ[k, k])
        Q = out["Q"][k].numpy()
        assert np.allclose(Q.T @ Q, np.eye(4), atol=1e-12)
        top = np.sort(np.linalg.eigvalsh(T))[::-1][:4].sum()
        assert abs(np.trace(Q.T @ T @ Q) - top) <= 1e-12 * abs(top)


# ----------------------------------------------------------------------------------------------- P10
def test_tkk_psd_and_negative_energy():
    p = make_problem(5, 30, 20, seed=2)        # n_aux < n_vir: rank-deficient, still PSD
    eps = torch.as_tensor(p.eps_vir, dtype=DT)
    for k in range(p.n_occ):
        w = torch.linalg.eigvalsh(oracle.tkk(oracle.dense_B(p, k), eps, float(p.f_occ[k, k])))
        assert float(w.min()) >= -1e-14 * float(w.abs().max())
    assert oracle.energy(p, Params(n_osv_fixed=6, mbe_order=3))["E"] < 0.0


# ------------------------------------------------------------------------------------------------ P9
def test_hylleraas_error_is_quadratic():
    p = make_problem(3, 10, 20, seed=6)
    prm = Params(n_osv_fixed=4, mbe_order=0, tol=1e-13, max_iter=500)
    out = oracle.energy(p, prm)
    c = out["clusters"][0]
    T = out["amplitudes"][c]
    Fo = torch.as_tensor(p.f_occ, dtype=DT)
    cs = oracle.ClusterSolver(c, out["blocks"], Fo, prm.tau_red)
    e0 = float(cs.hylleraas(T))
    g = torch.Generator().manual_seed(0)
    X = {k: torch.randn(v.shape, generator=g, dtype=DT) for k, v in T.items()}
    d = []
    for h in (1e-3, 5e-4):
        d.append(float(cs.hylleraas({k: T[k] + h * X[k] for k in T})) - e0)
    assert abs(d[0] / d[1] - 4.0) < 1e-3, d


# --------------------------------------------------------------------------------------------- P7/P8
def _fd_problem():
    return make_problem(4, 10, 24, seed=13), Params(n_osv_fixed=4, mbe_order=3, tol=1e-12, max_iter=500, r2b=3.5,
                                                     r3b=3.1)


def test_gradient_matches_central_differences():
    p, prm = _fd_problem()
    g = oracle.gradient(p, prm)
    nosv = g["n_osv"]
    assert len(g["clusters"]) < 4 + 6 + 4       # a truncated expansion, not the full one
    h = 1e-5
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(12):
        i = int(rng.integers(p.n_occ))
        a = int(rng.integers(p.n_vir))
        P = int(rng.integers(p.a(i)))
        off = p.b_offset(i) + a * p.a(i) + P
        ev = []
        for s in (+h, -h):
            q = Problem(**{**p.__dict__})
            q.B = p.B.copy()
            q.B[off] += s
            ev.append(oracle.energy(q, prm, n_osv=nosv)["E"])
        fd = (ev[0] - ev[1]) / (2 * h)
        worst = max(worst, abs(fd - g["dB"][i][a, P]))
    for x in range(p.n_occ):
        for y in range(p.n_occ):
            ev = []
            for s in (+h, -h):
                q = Problem(**{**p.__dict__})
                q.f_occ = p.f_occ.copy()
                q.f_occ[x, y] += s
                ev.append(oracle.energy(q, prm, n_osv=nosv)["E"])
            fd = (ev[0] - ev[1]) / (2 * h)
            worst = max(worst, abs(fd - g["dF"][x, y]))
    assert worst <= 1e-7, worst


def test_euler_identity():
    """With the OSV counts frozen E is homogeneous of degree 4 in B, so sum B * dE/dB = 4 E."""
    p, prm = _fd_problem()
    g = oracle.gradient(p, prm)
    s = sum(float(np.sum(p.B_block(i) * g["dB"][i])) for i in range(p.n_occ))
    assert abs(s - 4.0 * g["E"]) <= 1e-12 * max(1.0, abs(g["E"])) * 100


# ------------------------------------------------------------------ OSV-overlap cluster metric (Sec. 2.2.1)
def _orthonormal(nv, k, rng):
    q, _ = np.linalg.qr(rng.standard_normal((nv, k)))
    return q


def test_osv_overlap_metric_bounds_and_closed_forms():
    """Eq. 2bscreen: s_ii = 1 and 0 <= s_ij <= 1 for orthonormal OSV blocks (the paper's Cauchy-Schwarz remark);
    closed forms: identical spans give 1 whatever the basis inside them and the block sizes, orthogonal spans give
    0, single OSVs give cos^2 of their angle, and a span half inside another (n_i = 2, n_j = 1) gives 1/sqrt(2)."""
    rng = np.random.default_rng(5)
    nv = 12
    Q = [_orthonormal(nv, k, rng) for k in (1, 2, 3, 4, 2)]
    s = oracle.osv_overlap_metric(Q)
    assert np.allclose(np.diag(s), 1.0, atol=1e-13)
    assert np.all(s >= -1e-15) and np.all(s <= 1.0 + 1e-13)
    assert np.allclose(s, s.T, atol=1e-14)
    # same span, another orthonormal basis of it (rotation inside the span)
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    assert abs(oracle.osv_overlap_metric([Q[2], Q[2] @ R])[0, 1] - 1.0) < 1e-13
    # orthogonal spans
    E = np.eye(nv)
    assert abs(oracle.osv_overlap_metric([E[:, :3], E[:, 3:7]])[0, 1]) < 1e-15
    # one OSV each: (q_i . q_j)^2
    a, b = rng.standard_normal(nv), rng.standard_normal(nv)
    a /= np.linalg.norm(a)
    b /= np.linalg.norm(b)
    assert abs(oracle.osv_overlap_metric([a[:, None], b[:, None]])[0, 1] - (a @ b) ** 2) < 1e-14
    # n_i = 2 spanning e0, e1; n_j = 1 along e0: sum of squares 1, normalisation sqrt(2)
    assert abs(oracle.osv_overlap_metric([E[:, :2], E[:, :1]])[0, 1] - 1.0 / np.sqrt(2.0)) < 1e-15


def test_osv_metric_cluster_selection_bruteforce():
    """2b clusters: s_ij exceeding l2b; 3b clusters: all three pairs kept and the mean of their s exceeding l3b
    (Eq. 3bscreen).  Checked against a brute-force enumeration on random symmetric metrics, plus hand cases at
    the thresholds (equality does not exceed)."""
    s = np.array([[1.0, 0.5, 0.3, 1e-3],
                  [0.5, 1.0, 0.01, 0.4],
                  [0.3, 0.01, 1.0, 0.25],
                  [1e-3, 0.4, 0.25, 1.0]])
    got = oracle.select_clusters_osv(s, 0.01, 0.2, 3)
    assert got == [(0,), (1,), (2,), (3,), (0, 1), (0, 2), (1, 3), (2, 3)]   # (1, 2) at l2b exactly: out
    s2 = s.copy()
    s2[1, 2] = s2[2, 1] = 0.0100001
    got2 = oracle.select_clusters_osv(s2, 0.01, 0.2, 3)
    assert (0, 1, 2) in got2 and (1, 2, 3) in got2 and (0, 1, 3) not in got2
    assert oracle.select_clusters_osv(s, 0.01, 0.2, 1) == [(0,), (1,), (2,), (3,)]
    assert oracle.select_clusters_osv(s, 0.01, 0.2, 0) == [(0, 1, 2, 3)]
    rng = np.random.default_rng(9)
    for _ in range(200):
        n = int(rng.integers(1, 8))
        m = rng.random((n, n)) ** 3
        m = (m + m.T) / 2
        np.fill_diagonal(m, 1.0)
        l2, l3 = float(rng.random() * 0.2), float(rng.random() * 0.5)
        want = [(i,) for i in range(n)]
        want += [c for c in itertools.combinations(range(n), 2) if m[c] > l2]
        want += [c for c in itertools.combinations(range(n), 3)
                 if all(m[p] > l2 for p in itertools.combinations(c, 2))
                 and sum(m[p] for p in itertools.combinations(c, 2)) / 3 > l3]
        assert oracle.select_clusters_osv(m, l2, l3, 3) == want


# ------------------------------------------------------------------ weak 2b clusters, one-block scheme (Sec. 2.2.2)
def _osv_blocks_numpy(p, n_osv):
    """Q_k of every LMO with numpy (eigenvectors of Eq. 6's T_kk, largest first), independent of the oracle."""
    Q = []
    for k in range(p.n_occ):
        Bk = p.B_dense(k)
        den = p.eps_vir[:, None] + p.eps_vir[None, :] - 2.0 * p.f_occ[k, k]
        w, U = np.linalg.eigh((Bk @ Bk.T) / den)
        Q.append(U[:, np.argsort(-w, kind="stable")[:n_osv]])
    return Q


def test_weak_pair_one_block_is_a_sylvester_solve():
    """With orthonormal OSVs per LMO, the upper-right block of Eq. 4 for a 2b cluster is the Sylvester equation
    (F_ii - f_ii) X + X (F_jj - f_jj) = -K_(i,j) + f_ij (T_ii S_ij + S_ij T_jj), with F_xy = Q_x^T diag(eps) Q_y,
    S_ij = Q_i^T Q_j, K_(i,j) = Q_i^T B_i B_j^T Q_j and T_ii, T_jj the 1b cluster amplitudes.  Solved here with
    scipy's Sylvester solver on blocks built with numpy (a transposed block or a misplaced shift fails)."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    p = make_problem(4, 18, 40, seed=31)
    p.f_occ = p.f_occ.copy()
    p.f_occ[0, 3] = p.f_occ[3, 0] = -0.03      # a visible coupling
    n_osv = 5
    prm = Params(n_osv_fixed=n_osv, mbe_order=3, tol=1e-12)
    i, j = 0, 3
    X, Ew, it, rn = oracle.weak_pair_one_block(p, prm, i, j)
    assert rn <= 1e-12
    Q = _osv_blocks_numpy(p, n_osv)
    # the oracle's OSVs may differ by column signs: compare in the sign convention of the numpy blocks
    Qo = [oracle.osv_decompose(oracle.tkk(oracle.dense_B(p, k), torch.as_tensor(p.eps_vir), torch.tensor(p.f_occ[k, k])))[1][:, :n_osv].numpy()
          for k in range(p.n_occ)]
    sg = [np.sign(np.sum(Q[k] * Qo[k], axis=0)) for k in range(p.n_occ)]
    Xo = (sg[i][:, None] * X.numpy()) * sg[j][None, :]
    eps = p.eps_vir
    Fii, Fjj = Q[i].T @ (eps[:, None] * Q[i]), Q[j].T @ (eps[:, None] * Q[j])
    Sij = Q[i].T @ Q[j]
    Kij = Q[i].T @ p.B_dense(i) @ p.B_dense(j).T @ Q[j]
    Tii = {}
    for k in (i, j):
        Tk, _, _, _ = oracle.ClusterSolver((k,), oracle.osvmp2._Blocks(
            [torch.as_tensor(q) for q in Q], [oracle.dense_B(p, m) for m in range(p.n_occ)],
            torch.as_tensor(eps)), torch.as_tensor(p.f_occ), 1e-8).solve(1e-13, 500)
        Tii[k] = Tk[(k, k)].numpy()
    fij = p.f_occ[i, j]
    rhs = -Kij + fij * (Tii[i] @ Sij + Sij @ Tii[j])
    Xs = scipy_linalg.solve_sylvester(Fii - p.f_occ[i, i] * np.eye(n_osv), Fjj - p.f_occ[j, j] * np.eye(n_osv), rhs)
    assert np.abs(Xo - Xs).max() <= 1e-10 * np.abs(Xs).max()


def test_weak_pair_one_block_equals_full_2b_when_decoupled():
    """If the OSV spans of i and j sit on disjoint canonical virtuals (S_ij = 0, F_ij = 0) and f_ij = 0, every block
    of the 2b cluster's equations decouples: the one-block amplitudes equal the upper-right block of the full 2b
    solution, and the weak pair's energy equals the 2b increment E^{ij} - E^i - E^j of the MBE energy."""
    p = make_problem(2, 16, 30, seed=33)
    nv = p.n_vir
    B = p.B.copy()
    for k, rows in ((0, slice(nv // 2, nv)), (1, slice(0, nv // 2))):
        a = p.a(k)
        blk = B[p.aux_ptr[k] * nv:p.aux_ptr[k + 1] * nv].reshape(nv, a)
        blk[rows, :] = 0.0
    q = Problem(**{**p.__dict__, "B": B, "f_occ": np.diag(np.diag(p.f_occ))})
    prm = Params(n_osv_fixed=4, mbe_order=3, tol=1e-12)
    X, Ew, it, rn = oracle.weak_pair_one_block(q, prm, 0, 1)
    full = oracle.energy(q, prm, clusters=[(0,), (1,), (0, 1)])
    mono = oracle.energy(q, prm, clusters=[(0,), (1,)])
    assert abs(Ew - (full["E"] - mono["E"])) <= 1e-12 * abs(full["E"])
    # the full cluster's (0, 1) amplitudes: zero outside the upper-right block, equal to X inside
    eps, F, Bd = oracle.osvmp2._inputs(q, False)
    Qo, _ = oracle.osvmp2._osvs(Bd, eps, F, prm, None)
    Tf, _, _, _ = oracle.ClusterSolver((0, 1), oracle.osvmp2._Blocks(Qo, Bd, eps), F, prm.tau_red).solve(1e-13, 500)
    T01 = Tf[(0, 1)].numpy()
    n0 = Qo[0].shape[1]
    assert np.abs(T01[:n0, n0:] - X.numpy()).max() <= 1e-10 * np.abs(X.numpy()).max()
    assert np.abs(T01[:n0, :n0]).max() <= 1e-12 and np.abs(T01[n0:, :]).max() <= 1e-12


def test_weak_pair_gradient_matches_finite_differences():
    """gradient_weak_pairs (the derivative of the weak pairs' one-block energy, Sec. 2.2.2) against fourth-order
    central differences of weak_pair_one_block's E_w, on B entries of both LMOs of each weak pair and on
    diagonal and off-diagonal entries of F_occ (entrywise: f_03 and f_30 apart).  E_w is not stationary in the
    one-block amplitudes or the frozen 1b amplitudes, so a derivative that drops their responses fails here."""
    p = make_problem(4, 18, 40, seed=31)
    p.f_occ = p.f_occ.copy()
    p.f_occ[0, 3] = p.f_occ[3, 0] = -0.03
    prm = Params(n_osv_fixed=5, mbe_order=3, tol=1e-13, max_iter=500)
    pairs = [(0, 3), (1, 2)]
    g = oracle.gradient_weak_pairs(p, prm, pairs)

    def ew(q):
        return sum(oracle.weak_pair_one_block(q, prm, i, j)[1] for i, j in pairs)

    def moved(kind, idx, h):
        q = Problem(**p.__dict__)
        if kind == "B":
            i, a, P = idx
            q.B = p.B.copy()
            q.B[int(p.aux_ptr[i]) * p.n_vir + a * p.a(i) + P] += h
        else:
            q.f_occ = p.f_occ.copy()
            q.f_occ[idx] += h
        return q

    rng = np.random.default_rng(7)
    entries = [("B", (i, int(rng.integers(p.n_vir)), int(rng.integers(p.a(i))))) for i in (0, 3, 1, 2) for _ in range(2)]
    entries += [("F", (0, 0)), ("F", (0, 3)), ("F", (3, 0)), ("F", (1, 2))]
    h = 1e-4
    for kind, idx in entries:
        d1 = ew(moved(kind, idx, h)) - ew(moved(kind, idx, -h))
        d2 = ew(moved(kind, idx, 2 * h)) - ew(moved(kind, idx, -2 * h))
        fd = (8 * d1 - d2) / (12 * h)
        an = g["dB"][idx[0]][idx[1], idx[2]] if kind == "B" else g["dF"][idx]
        assert abs(an - fd) <= 1e-8 + 1e-6 * abs(fd), (kind, idx, an, fd)
    assert abs(g["E"] - ew(p)) <= 1e-14


def test_screened_energy_limits():
    """The screened MBE energy (strong clusters by the OSV metric + one-block weak pairs - discarded pairs) in its
    limits: every pair strong and no triple -> the MBE(2) energy of all pairs; every pair below the discard
    threshold -> the sum of the 1b cluster energies; two decoupled LMOs (disjoint virtual spans, f_ij = 0) whose
    pair is weak -> exactly the full 2b energy (the one-block scheme misses nothing there)."""
    p = make_problem(4, 16, 30, seed=35)
    prm = Params(n_osv_fixed=4, mbe_order=3, tol=1e-12)
    scr = oracle.energy_osv_screened(p, prm, l2b=-1.0, l3b=2.0)
    pairs = [c for c in itertools.combinations(range(4), 2)]
    ref = oracle.energy(p, prm, clusters=[(i,) for i in range(4)] + pairs)
    assert scr["weak_pairs"] == [] and abs(scr["E"] - ref["E"]) <= 1e-13 * abs(ref["E"])
    scr0 = oracle.energy_osv_screened(p, prm, l2b=2.0, l3b=2.0, l_discard=2.0)
    mono = oracle.energy(p, prm, clusters=[(i,) for i in range(4)])
    assert scr0["weak_pairs"] == [] and abs(scr0["E"] - mono["E"]) <= 1e-13 * abs(mono["E"])
    q = make_problem(2, 16, 30, seed=33)
    nv = q.n_vir
    B = q.B.copy()
    for k, rows in ((0, slice(nv // 2, nv)), (1, slice(0, nv // 2))):
        blk = B[q.aux_ptr[k] * nv:q.aux_ptr[k + 1] * nv].reshape(nv, q.a(k))
        blk[rows, :] = 0.0
    q = Problem(**{**q.__dict__, "B": B, "f_occ": np.diag(np.diag(q.f_occ))})
    scrw = oracle.energy_osv_screened(q, prm, l2b=0.5, l3b=2.0, l_discard=-1.0)   # s_01 = 0: weak, kept
    full = oracle.energy(q, prm, clusters=[(0,), (1,), (0, 1)])
    assert scrw["weak_pairs"] == [(0, 1)]
    assert abs(scrw["E"] - full["E"]) <= 1e-12 * abs(full["E"])


def test_posterior_correction_vanishes_where_mbe_is_exact():
    """The one-step posterior correction (Sec. 3) evaluates Eq. 4 at the collective amplitudes over the LMOs of the
    pair's clusters.  Where MBE(3) is exact (three LMOs, every cluster kept; or one full cluster) the collective
    amplitudes solve those equations: the residual vanishes, the step is zero and the pair functional equals the
    MBE energy.  A k range missing an LMO of the cluster, or a mis-indexed pair, leaves a residual here."""
    p = make_problem(3, 16, 40, seed=4)
    for order, extra in ((3, dict(r2b=99.0, r3b=99.0)), (0, {})):
        r = oracle.posterior_correction(p, Params(n_osv_fixed=4, mbe_order=order, tol=1e-12, **extra))
        assert r["dR_max"] <= 1e-10
        assert abs(r["E_corrected"] - r["E"]) <= 1e-12 * abs(r["E"])
        assert abs(r["E_global"] - r["E"]) <= 1e-12 * abs(r["E"])
        assert all(ks == [0, 1, 2] for ks in r["k_sets"].values())
    # truncated MBE(3) on six LMOs: a nonzero residual and a finite step
    q = make_problem(6, 16, 40, seed=3)
    r = oracle.posterior_correction(q, Params(n_osv_fixed=4, mbe_order=3, r2b=6.0, r3b=5.0, tol=1e-12))
    assert r["dR_max"] > 1e-8 and np.isfinite(r["E_corrected"])


# ------------------------------------------------------------------------------------------- OSV count
def test_osv_count_rule_on_hand_built_spectra():
    """Sec. 2.1 keeps the OSVs whose eigenvalues are greater than l_osv; the reading adds a cap n_osv_max (0 = no
    cap), a floor of one OSV, and an exact count n_osv_fixed that overrides both.  Expected counts written by hand
    from that rule: an eigenvalue equal to l_osv is not kept, the cap applies after the threshold, the floor after
    the cap."""
    w = torch.tensor([0.5, 0.3, 0.2, 1e-4, 1e-4, 5e-5, 0.0], dtype=DT)
    sel = oracle.n_osv_select
    assert sel(w, 1e-4, 0, 0) == 3            # 1e-4 itself is not "greater than" 1e-4
    assert sel(w, 9.9e-5, 0, 0) == 5          # just below: the two eigenvalues at 1e-4 are kept
    assert sel(w, 1e-4, 2, 0) == 2            # cap below the count
    assert sel(w, 1e-4, 3, 0) == 3            # cap equal to the count
    assert sel(w, 1e-4, 10, 0) == 3           # cap above the count
    assert sel(w, 1.0, 10, 0) == 1            # nothing above the threshold: at least one OSV
    assert sel(w, 1.0, 0, 0) == 1
    assert sel(w, -1.0, 0, 0) == 7            # everything kept, the zero eigenvalue included
    assert sel(w, -1.0, 4, 0) == 4
    assert sel(w, 1e-4, 2, 6) == 6            # an exact count ignores threshold and cap
    assert sel(w, 1e-4, 2, 99) == 7           # ... but cannot exceed the virtual space
    # the rule counts eigenvalues, not leading positions: the oracle's spectra are sorted, so both agree there
    ws = torch.sort(torch.tensor([3e-4, 2e-5, 8e-4, 1.5e-4, 9e-5], dtype=DT), descending=True).values
    assert sel(ws, 1e-4, 0, 0) == 3


# ------------------------------------------------------------------------------------- posterior step
def _posterior_numpy(problem, out, ks, tau_red):
    """Independent restatement of the one-step posterior correction in the canonical virtual space (numpy only).

    With t_p = P_p T_p P_p^T (P_p the pair domain of the oracle's OSVs, T_p its collective amplitudes, zero where
    a pair has none), Eq. 4 for the ordered pair ij over the LMOs k of ks[ij] is the projection onto range(P_ij) of
        r_ij = (ia|jb) + eps t_ij + t_ij eps - sum_k (f_kj t_ik + f_ik t_kj).
    In an orthonormal basis U_ij = Phi W of range(P_ij) that diagonalises eps (U^T eps U = diag(e)), the step is
    dt_ij = -U [(U^T r_ij U) / (e_a + e_b - f_ii - f_jj)] U^T, and the pair functional (Eq. 3) is
    sum_ij <(ia|jb) + r_ij, 2 t_ij - t_ij^T>."""
    n, nv = problem.n_occ, problem.n_vir
    Bd = [problem.B_dense(i) for i in range(n)]
    f, eps = problem.f_occ, problem.eps_vir
    Q = [q.numpy() for q in out["Q"]]
    P = {}
    for i in range(n):
        for j in range(n):
            P[(i, j)] = Q[i] if i == j else np.concatenate([Q[i], Q[j]], axis=1)
    t = {p: P[p] @ T.numpy() @ P[p].T for p, T in out["collective"].items()}
    zero = np.zeros((nv, nv))

    def resid(tt, p):
        i, j = p
        r = Bd[i] @ Bd[j].T + eps[:, None] * tt[p] + tt[p] * eps[None, :]
        for k in ks[p]:
            r = r - f[k, j] * tt.get((i, k), zero) - f[i, k] * tt.get((k, j), zero)
        return r

    def functional(tt):
        return sum(float(np.sum((Bd[p[0]] @ Bd[p[1]].T + resid(tt, p)) * (2.0 * tt[p] - tt[p].T))) for p in tt)

    dt, rmax = {}, 0.0
    for p in t:
        i, j = p
        u, s, _ = np.linalg.svd(P[p], full_matrices=False)
        Phi = u[:, s * s > tau_red]                 # S = P^T P: its eigenvalues are the squared singular values
        e, W = np.linalg.eigh(Phi.T @ (eps[:, None] * Phi))
        U = Phi @ W
        rho = U.T @ resid(t, p) @ U
        rmax = max(rmax, float(np.linalg.norm(rho)))
        dt[p] = -U @ (rho / (e[:, None] + e[None, :] - f[i, i] - f[j, j])) @ U.T
    return functional(t), functional({p: t[p] + dt[p] for p in t}), rmax


def _k_ranges(centres, r2b, r3b):
    """For every ordered pair ij inside a selected cluster: the union of the LMOs of the clusters holding i and j
    (pairs within r2b; triples whose three distances are within r3b), written from the distance rule."""
    n = len(centres)
    d = np.linalg.norm(centres[:, None, :] - centres[None, :, :], axis=-1)
    cl = [{i} for i in range(n)] + [{i, j} for i, j in itertools.combinations(range(n), 2) if d[i, j] <= r2b]
    cl += [{i, j, k} for i, j, k in itertools.combinations(range(n), 3)
           if max(d[i, j], d[i, k], d[j, k]) <= min(r2b, r3b)]
    out = {}
    for i in range(n):
        for j in range(n):
            members = [c for c in cl if i in c and j in c]
            if members:
                out[(i, j)] = sorted(set().union(*members))
    return out


def test_posterior_correction_on_a_truncated_expansion():
    """Truncated MBE(3) on six LMOs (Sec. 3): the collective amplitudes leave a residual over the k ranges of the
    pairs' clusters.  The oracle's residual norm, global pair functional and corrected functional must equal the
    numpy restatement above (a wrong sign, denominator, k range or transposed block in the oracle fails here).
    The change made by the step is second order in the residual (one preconditioned step on a quadratic
    functional): halving the off-diagonal Fock couplings scales the change like the squared residual norm.  With
    every pair and triple kept, each pair's k range is all six LMOs, so the residual is that of the untruncated
    OSV-MP2 equations: the global functional and then the corrected one come closer to the untruncated energy than
    the MBE(3) energy (the higher-order estimate of Sec. 3)."""
    base = make_problem(6, 16, 40, seed=3)
    prm = Params(n_osv_fixed=4, mbe_order=3, r2b=6.0, r3b=5.0, tol=1e-12, max_iter=500)
    rows = []
    for lam in (1.0, 0.5, 0.25):
        f = base.f_occ.copy()
        off = ~np.eye(6, dtype=bool)
        f[off] *= lam
        q = Problem(**{**base.__dict__, "f_occ": f})
        r = oracle.posterior_correction(q, prm)
        out = oracle.energy(q, prm)
        ks = _k_ranges(q.centres, prm.r2b, prm.r3b)
        assert {p: r["k_sets"][p] for p in ks} == ks and set(r["k_sets"]) == set(ks)
        Eg, Ec, rmax = _posterior_numpy(q, out, ks, prm.tau_red)
        assert r["dR_max"] > 1e-8
        assert abs(r["dR_max"] - rmax) <= 1e-9 * rmax
        assert abs(r["E_global"] - Eg) <= 1e-11 * abs(Eg)
        assert abs(r["E_corrected"] - Ec) <= 1e-11 * abs(Ec)
        # the step's own energy change (~|dR|^2 / D, far below E): a wrong denominator or k range shows here
        dEo, dEn = r["E_corrected"] - r["E_global"], Ec - Eg
        assert abs(dEo - dEn) <= 5e-4 * abs(dEn) + 2e-16, (dEo, dEn)
        rows.append((rmax, abs(r["E_corrected"] - r["E_global"])))
    for (r0, d0), (r1, d1) in zip(rows, rows[1:]):
        slope = np.log(d0 / d1) / np.log(r0 / r1)
        assert 1.8 <= slope <= 2.2, rows
    allk = Params(n_osv_fixed=4, mbe_order=3, r2b=99.0, r3b=99.0, tol=1e-12, max_iter=500)
    r = oracle.posterior_correction(base, allk)
    full = oracle.energy(base, Params(n_osv_fixed=4, mbe_order=0, tol=1e-12, max_iter=500))["E"]
    assert all(ks == list(range(6)) for ks in r["k_sets"].values())
    err = [abs(r[key] - full) for key in ("E", "E_global", "E_corrected")]
    assert err[0] > 1e-8 and err[2] < err[1] < err[0], err
    assert err[2] <= 1e-3 * err[0], err

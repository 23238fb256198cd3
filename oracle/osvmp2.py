"""Plain FP64 CPU oracle for MBE(3)-OSV-MP2 energies and OSV-space gradients.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module: only tests/, the smoke check in
__graft_entry__ and bench.py's CPU-baseline / reference legs may call it.  It shares no code with the CUDA
library.  It is slow on purpose: every step is the paper's equation written out with plain torch CPU float64
ops (matmul and eigh are the only library primitives), with no blocking, fusion or basis shortcut.

Method (arXiv 2106.06149, Liang & Yang):
  * OSVs: per LMO k, the semicanonical diagonal amplitudes [T_kk]_ab = (ka|kb) / (e_a + e_b - 2 f_kk) are
    diagonalised and the eigenvectors with the largest eigenvalues are kept (Sec. 2.1, Eqs. 5-6).
  * Pair quantities are projections onto concatenated OSV domains, A_(ij,kl) = (Q_i Q_j)^T A (Q_k Q_l)
    (Sec. 2.1, Eq. 7), with A the identity (S), the virtual Fock matrix (F) or (ia|jb) = sum_P B_ia^P B_jb^P (K).
  * Pair amplitudes solve the residual equations of Eq. 4 in the OSV basis, inside each 1-, 2- or 3-orbital
    cluster with the sum over k restricted to the cluster (Sec. 2.2.1, cluster residual R^{i,j,k}).
  * Energy: Hylleraas functional, Eq. 3, <A B> read as the Frobenius product sum_ab A_ab B_ab.
  * MBE(3): clusters combine with inclusion-exclusion weights, which is exactly Eqs. 28-32 for the collective
    amplitudes and Eqs. 33-34 for the densities (Sec. 2.2.1).
  * Gradient: amplitudes are variational (Sec. 2.1, Eq. 9 and the text before it), so dE/dx is the partial
    derivative of the weighted cluster Hylleraas functionals at fixed amplitudes.  It is taken here by torch
    autograd through the plain steps above, including the full OSV eigenvector derivative of eigh.
  * Screening (Sec. 2.2.1): the OSV-overlap metric of Eq. 2bscreen and the 2b/3b selection of Eq. 3bscreen.
  * Weak 2b clusters (Sec. 2.2.2): one-block amplitudes (the upper-right block of the 2b pair amplitudes, from the
    upper-right block of Eq. 4) and their energy; the screened MBE energy that adds them to the strong clusters.
  * Posterior correction (Sec. 3): Eq. 4 at the collective amplitudes over each pair's cluster LMOs, one step.

Readings of points where the paper is silent:
  * ordered pairs (i, j) and (j, i) are separate pair equations; the pair ii uses the domain Q_i only;
  * each pair inside a cluster uses its own domain (Q_i Q_j), never the union over the cluster;
  * the OSV-basis residual is preconditioned in an orthonormal pseudo-canonical basis of the pair domain,
    dropping pair-overlap eigenvalues below tau_red (the redundant part of (Q_i Q_j));
  * convergence: max over ordered pairs of ||V^T R V||_F <= tol;
  * OSV count: eigenvalues > l_osv, capped at n_osv_max, at least one; or exactly n_osv_fixed;
  * clusters: pair kept iff distance <= r2b, triple kept iff its three pairs are kept and all three
    distances <= r3b (distance cutoffs in place of the OSV-overlap metric of Eqs. 26-27);
  * with the OSV-overlap metric (select_clusters_osv): "exceeding" read as strictly greater, and a triple kept only
    if its three pairs are kept 2b clusters (the metric of Eq. 3bscreen averages the pairs' 2b metrics).
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64

__all__ = [
    "tkk", "osv_decompose", "n_osv_select", "select_clusters", "mbe_weights", "pair_domain",
    "ClusterSolver", "energy", "gradient", "dense_B", "osv_overlap_metric", "select_clusters_osv",
    "weak_pair_one_block", "gradient_weak_pairs", "energy_osv_screened", "posterior_correction",
]


# ----------------------------------------------------------------------------------------------- inputs
def dense_B(problem, i, dtype=DT):
    """LMO i's DF block on the full aux index, zero outside its fitting domain (local fitting, Sec. 2.3)."""
    out = torch.zeros(problem.n_vir, problem.n_aux, dtype=dtype)
    idx = torch.as_tensor(problem.aux_idx[problem.aux_ptr[i]:problem.aux_ptr[i + 1]].astype(np.int64))
    out[:, idx] = torch.as_tensor(np.asarray(problem.B_block(i), dtype=np.float64), dtype=dtype)
    return out


# ------------------------------------------------------------------------------------------------- OSVs
def tkk(Bk, eps, fkk):
    """Semicanonical diagonal amplitudes [T_kk]_ab = (ka|kb) / (f_aa + f_bb - 2 f_kk)  (Sec. 2.1, Eq. 6)."""
    kk = Bk @ Bk.T                                   # (ka|kb) = sum_P B_ka^P B_kb^P
    den = eps[:, None] + eps[None, :] - 2.0 * fkk
    return kk / den


def osv_decompose(T):
    """Eigenpairs of T_kk sorted by decreasing eigenvalue (Sec. 2.1, Eq. 6).  Columns of U are eigenvectors."""
    w, U = torch.linalg.eigh(T)
    order = torch.argsort(w.detach(), descending=True, stable=True)
    return w[order], U[:, order]


def n_osv_select(w, l_osv, n_osv_max, n_osv_fixed):
    """Number of OSVs kept: eigenvalues greater than l_osv (Sec. 2.1), capped, at least one."""
    if n_osv_fixed > 0:
        return min(int(n_osv_fixed), w.shape[0])
    n = int((w > l_osv).sum())
    if n_osv_max > 0:
        n = min(n, int(n_osv_max))
    return max(n, 1)


# --------------------------------------------------------------------------------------------- clusters
def select_clusters(centres, r2b, r3b, mbe_order):
    """1b/2b/3b clusters under distance cutoffs (Sec. 2.2.1; distance rule replaces Eqs. 26-27).
    mbe_order 0 returns one cluster holding every LMO (plain OSV-MP2, no MBE truncation)."""
    n = len(centres)
    if mbe_order == 0:
        return [tuple(range(n))]
    d = np.linalg.norm(np.asarray(centres)[:, None, :] - np.asarray(centres)[None, :, :], axis=-1)
    out = [(i,) for i in range(n)]
    if mbe_order >= 2:
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if d[i, j] <= r2b]
        out += pairs
        if mbe_order >= 3:
            keep = set(pairs)
            for i in range(n):
                for j in range(i + 1, n):
                    if (i, j) not in keep:
                        continue
                    for k in range(j + 1, n):
                        if (i, k) in keep and (j, k) in keep and max(d[i, j], d[i, k], d[j, k]) <= r3b:
                            out.append((i, j, k))
    return out


def osv_overlap_metric(Q):
    """Pairwise OSV-overlap metric of Sec. 2.2.1, Eq. 2bscreen: s_ij = sum over (mu, nu) of <mu_i|nu_j>^2 divided by
    sqrt(n_i n_j), with <mu_i|nu_j> the entries of Q_i^T Q_j and n_i the number of OSVs of LMO i.  Q is a list of
    n_v x n_i blocks with orthonormal columns; then 0 <= s_ij <= 1 and s_ii = 1."""
    n = len(Q)
    s = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            O = torch.as_tensor(Q[i], dtype=DT).T @ torch.as_tensor(Q[j], dtype=DT)
            s[i, j] = float((O * O).sum()) / math.sqrt(Q[i].shape[1] * Q[j].shape[1])
    return s


def select_clusters_osv(s2b, l2b, l3b, mbe_order):
    """1b/2b/3b clusters by the OSV-overlap metrics of Sec. 2.2.1: a pair ij is a 2b cluster when s2b_ij exceeds
    l2b; a triple ijk is a 3b cluster when its three pairs are 2b clusters and s3b_ijk = (s_ij + s_ik + s_jk) / 3
    (Eq. 3bscreen) exceeds l3b.  mbe_order 0 returns one cluster holding every LMO."""
    s2b = np.asarray(s2b, dtype=np.float64)
    n = s2b.shape[0]
    if mbe_order == 0:
        return [tuple(range(n))]
    out = [(i,) for i in range(n)]
    if mbe_order >= 2:
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n) if s2b[i, j] > l2b]
        out += pairs
        if mbe_order >= 3:
            keep = set(pairs)
            for i in range(n):
                for j in range(i + 1, n):
                    for k in range(j + 1, n):
                        if (i, j) in keep and (i, k) in keep and (j, k) in keep and \
                                (s2b[i, j] + s2b[i, k] + s2b[j, k]) / 3.0 > l3b:
                            out.append((i, j, k))
    return out


def mbe_weights(clusters):
    """Inclusion-exclusion weights w_c = sum over selected supersets c' of c of (-1)^(|c'|-|c|).
    With these weights sum_c w_c X^c reproduces the MBE(3) expansions of Eqs. 28-34 (Sec. 2.2.1)."""
    w = {c: 0 for c in clusters}
    for big in clusters:
        m = len(big)
        for mask in range(1, 1 << m):
            sub = tuple(big[t] for t in range(m) if mask >> t & 1)
            if sub in w:
                w[sub] += (-1) ** (m - len(sub))
    return w


# ------------------------------------------------------------------------------------------ pair blocks
def pair_domain(Q, i, j):
    """Concatenated OSV domain (Q_i Q_j) of the pair ij; the pair ii uses Q_i alone (Sec. 2.1, Eq. 7)."""
    return Q[i] if i == j else torch.cat([Q[i], Q[j]], dim=1)


class _Blocks:
    """Cache of A_(p,q) = P_p^T A P_q for A in {1, diag(eps)} and K_(p,p) (Sec. 2.1, Eq. 7)."""

    def __init__(self, Q, Bd, eps):
        self.Q, self.Bd, self.eps = Q, Bd, eps
        self.P, self.S_, self.F_, self.K_, self.Kv = {}, {}, {}, {}, {}

    def dom(self, p):
        if p not in self.P:
            self.P[p] = pair_domain(self.Q, *p)
        return self.P[p]

    def S(self, p, q):
        if (p, q) not in self.S_:
            self.S_[(p, q)] = self.dom(p).T @ self.dom(q)
        return self.S_[(p, q)]

    def F(self, p, q):
        if (p, q) not in self.F_:
            self.F_[(p, q)] = self.dom(p).T @ (self.eps[:, None] * self.dom(q))
        return self.F_[(p, q)]

    def kv(self, i, j):
        """(ia|jb) as an n_vir x n_vir matrix, the full virtual-space product (no half transform)."""
        if (i, j) not in self.Kv:
            if (j, i) in self.Kv:
                self.Kv[(i, j)] = self.Kv[(j, i)].T
            else:
                self.Kv[(i, j)] = self.Bd[i] @ self.Bd[j].T
        return self.Kv[(i, j)]

    def K(self, p):
        if p not in self.K_:
            P = self.dom(p)
            self.K_[p] = P.T @ self.kv(*p) @ P
        return self.K_[p]


class ClusterSolver:
    """Residual equations of one cluster, Eq. 4 with k running over the cluster's LMOs (Sec. 2.2.1)."""

    def __init__(self, c, blocks, F, tau_red):
        self.c, self.b, self.Fo = tuple(c), blocks, F
        self.pairs = [(i, j) for i in self.c for j in self.c]          # ordered pairs
        self.tau_red = tau_red

    def residual(self, p, T):
        """R_(ij,ij) = K_(ij,ij) + sum_k S_(ij,ik) T_(ik,ik) [d_kj F_(ik,ij) - f_kj S_(ik,ij)]
                                 + [d_ik F_(ij,kj) - f_ik S_(ij,kj)] T_(kj,kj) S_(kj,ij)      (Eq. 4)."""
        i, j = p
        b, f = self.b, self.Fo
        R = b.K(p).clone()
        for k in self.c:
            q = (i, k)
            right = -f[k, j] * b.S(q, p)
            if k == j:
                right = right + b.F(q, p)
            R = R + b.S(p, q) @ T[q] @ right
            q = (k, j)
            left = -f[i, k] * b.S(p, q)
            if i == k:
                left = left + b.F(p, q)
            R = R + left @ T[q] @ b.S(q, p)
        return R

    def precond(self, p):
        """Orthonormal pseudo-canonical basis V of the pair domain: V^T S V = 1, V^T F V = diag(e);
        pair-overlap eigenvalues below tau_red are dropped.  Returns V and the denominators
        D_ab = e_a + e_b - f_ii - f_jj used for the amplitude update."""
        i, j = p
        s, U = torch.linalg.eigh(self.b.S(p, p))
        keep = s > self.tau_red
        X = U[:, keep] / torch.sqrt(s[keep])[None, :]
        e, W = torch.linalg.eigh(X.T @ self.b.F(p, p) @ X)
        D = e[:, None] + e[None, :] - self.Fo[i, i] - self.Fo[j, j]
        return X @ W, D

    def solve(self, tol, max_iter):
        """Jacobi iterations T <- T - V [(V^T R V) / D] V^T until max ||V^T R V||_F <= tol."""
        pc = {p: self.precond(p) for p in self.pairs}
        T = {p: torch.zeros(self.b.dom(p).shape[1], self.b.dom(p).shape[1], dtype=DT) for p in self.pairs}
        it, rn = 0, float("inf")
        for it in range(max_iter + 1):
            R = {p: self.residual(p, T) for p in self.pairs}
            Rt = {p: pc[p][0].T @ R[p] @ pc[p][0] for p in self.pairs}
            rn = max(float(torch.linalg.norm(Rt[p]).detach()) for p in self.pairs)
            if rn <= tol or it == max_iter:
                break
            for p in self.pairs:
                V, D = pc[p]
                T[p] = T[p] - V @ (Rt[p] / D) @ V.T
        return T, R, it, rn

    def hylleraas(self, T):
        """E^c = sum over ordered pairs of <K + R, 2T - T^T>  (Eq. 3, Frobenius product)."""
        E = torch.zeros((), dtype=DT)
        for p in self.pairs:
            R = self.residual(p, T)
            E = E + torch.sum((self.b.K(p) + R) * (2.0 * T[p] - T[p].T))
        return E


# ------------------------------------------------------------------------------- weak 2b clusters
def _weak_pair(i, j, Q, Bd, eps, F, params, tol, max_iter):
    """Core of weak_pair_one_block on given OSVs Q, DF blocks Bd and Fock matrix F (torch tensors; every step is a
    torch operation, so the energy can be differentiated through the 1b solves and the one-block iterations).
    Returns X, E_w (a tensor), the iteration count and the final max |R^{i,j}_(i,j)|."""
    b = _Blocks(Q, Bd, eps)
    T = {}
    for k in (i, j):   # 1b cluster amplitudes of the diagonal pairs
        Tk, _, _, _ = ClusterSolver((k,), b, F, params.tau_red).solve(params.tol, params.max_iter)
        T[(k, k)] = Tk[(k, k)]
    ni, nj = Q[i].shape[1], Q[j].shape[1]
    cs = ClusterSolver((i, j), b, F, params.tau_red)
    p, pt = (i, j), (j, i)
    ei, Ui = torch.linalg.eigh(b.F((i, i), (i, i)))
    ej, Uj = torch.linalg.eigh(b.F((j, j), (j, j)))
    D = ei[:, None] + ej[None, :] - F[i, i] - F[j, j]
    X = torch.zeros(ni, nj, dtype=DT)

    def embed(Xb):
        Tp = torch.zeros(ni + nj, ni + nj, dtype=DT)
        Tp[:ni, ni:] = Xb
        return Tp

    it, rn = 0, float("inf")
    for it in range(max_iter + 1):
        T[p] = embed(X)
        Rb = cs.residual(p, T)[:ni, ni:]
        rn = float(Rb.detach().abs().max())
        if rn <= tol or it == max_iter:
            break
        X = X - Ui @ ((Ui.T @ Rb @ Uj) / D) @ Uj.T
    T[p] = embed(X)
    Tt = torch.zeros(ni + nj, ni + nj, dtype=DT)   # (j, i): rows the OSVs of j, columns those of i
    Tt[:nj, nj:] = X.T
    T[pt] = Tt
    Ew = torch.zeros((), dtype=DT)
    for q in (p, pt):
        R = cs.residual(q, T)
        Ew = Ew + torch.sum((b.K(q) + R) * (2.0 * T[q] - T[q].T))
    return X, Ew, it, rn


def weak_pair_one_block(problem, params, i, j, n_osv=None, tol=1e-12, max_iter=500):
    """One-block amplitudes of a weak 2b cluster {i, j} (Sec. 2.2.2).

    The pair amplitudes T_(ij,ij) of the 2b cluster are restricted to their upper-right block X (rows: the OSVs of
    i, columns: the OSVs of j; the direct-dispersion excitations), T_(ij,ij) = E_i X E_j^T, and X solves the
    upper-right block of the 2b cluster residual of Eq. 4, R^{i,j}_(i,j) = E_i^T R_(ij,ij) E_j = 0.  The diagonal
    pairs keep their 1b cluster amplitudes T^i_(ii,ii), T^j_(jj,jj) in the f_ij coupling terms.  Iterations:
    X <- X - U_i [(U_i^T R U_j) / (e_i + e_j - f_ii - f_jj)] U_j^T with F_(i,i) = U_i diag(e_i) U_i^T.

    Returns X, the weak pair's energy E_w (the Hylleraas terms <K + R, 2T - T^T> of Eq. 3 for the ordered pairs
    (i, j) and (j, i), T_(ji,ji) = E_j X^T E_i^T), the iteration count and the final max |R^{i,j}_(i,j)|."""
    assert i != j
    eps, F, Bd = _inputs(problem, False)
    Q, _ = _osvs(Bd, eps, F, params, n_osv)
    X, Ew, it, rn = _weak_pair(i, j, Q, Bd, eps, F, params, tol, max_iter)
    return X, float(Ew), it, rn


def gradient_weak_pairs(problem, params, pairs, n_osv=None, tol=1e-12, max_iter=500):
    """The weak pairs' energy sum_w E_w (weak_pair_one_block) and its derivative with respect to the stored DF
    entries B (list of (n_vir, a_i) arrays in each LMO's local aux order) and every entry of F_occ.

    E_w holds only the ordered pairs (i, j) and (j, i) of the 2b cluster, with T_ii, T_jj frozen at their 1b
    solutions, so it is not stationary in X, T_ii or T_jj: the derivative takes their responses.  It is the
    derivative of the computed energy, by automatic differentiation through the OSV eigendecompositions, the 1b
    solves and the one-block iterations (converged to tol).  OSV counts are frozen (n_osv, else the counts at B)."""
    eps, F, Bd = _inputs(problem, True)
    Q, info = _osvs(Bd, eps, F, params, n_osv)
    E = torch.zeros((), dtype=DT)
    for i, j in pairs:
        assert i != j
        E = E + _weak_pair(i, j, Q, Bd, eps, F, params, tol, max_iter)[1]
    E.backward()
    dB = []
    for i in range(problem.n_occ):
        idx = problem.aux_idx[problem.aux_ptr[i]:problem.aux_ptr[i + 1]].astype(np.int64)
        g = Bd[i].grad
        dB.append(g[:, idx].numpy().copy() if g is not None else np.zeros((Bd[i].shape[0], len(idx))))
    return dict(E=float(E.detach()), dB=dB, dF=F.grad.numpy().copy() if F.grad is not None else
                np.zeros_like(problem.f_occ), n_osv=[n for _, n in info])


# ------------------------------------------------------------------------------------------- top level
def _inputs(problem, grad):
    eps = torch.as_tensor(problem.eps_vir, dtype=DT)
    F = torch.as_tensor(problem.f_occ, dtype=DT).clone()
    Bd = [dense_B(problem, i) for i in range(problem.n_occ)]
    if grad:
        F.requires_grad_(True)
        for b in Bd:
            b.requires_grad_(True)
    return eps, F, Bd


def _osvs(Bd, eps, F, params, n_osv):
    Q, info = [], []
    for k in range(len(Bd)):
        w, U = osv_decompose(tkk(Bd[k], eps, F[k, k]))
        n = n_osv[k] if n_osv is not None else n_osv_select(
            w.detach(), params.l_osv, params.n_osv_max, params.n_osv_fixed)
        Q.append(U[:, :n])
        info.append((w.detach(), n))
    return Q, info


def _run(problem, params, n_osv, grad, clusters=None):
    eps, F, Bd = _inputs(problem, grad)
    Q, info = _osvs(Bd, eps, F, params, n_osv)
    if clusters is None:
        clusters = select_clusters(problem.centres, params.r2b, params.r3b, params.mbe_order)
    weights = mbe_weights(clusters)
    # amplitudes are solved with detached inputs; they are frozen in the energy functional (Sec. 2.1)
    det = _Blocks([q.detach() for q in Q], [b.detach() for b in Bd], eps)
    live = _Blocks(Q, Bd, eps) if grad else det
    Fd = F.detach()
    E = torch.zeros((), dtype=DT)
    per, amps, iters, rmax = {}, {}, {}, 0.0
    for c in clusters:
        cs = ClusterSolver(c, det, Fd, params.tau_red)
        T, R, it, rn = cs.solve(params.tol, params.max_iter)
        Ec = ClusterSolver(c, live, F, params.tau_red).hylleraas(T)
        per[c] = float(Ec.detach())
        amps[c] = T
        iters[c] = it
        rmax = max(rmax, rn)
        E = E + weights[c] * Ec
    # collective amplitudes (Eqs. 28-32) and the linear energy sum_ij <K, 2T - T^T>
    coll = {}
    for c in clusters:
        for p, T in amps[c].items():
            coll[p] = coll.get(p, 0.0) + weights[c] * T
    E_lin = sum(float(torch.sum(det.K(p) * (2.0 * T - T.T))) for p, T in coll.items())
    out = dict(E=float(E.detach()), E_linear=E_lin, clusters=clusters, weights=weights, per_cluster=per,
               iters=iters, rmax=rmax, n_osv=[n for _, n in info], osv_eigs=[w for w, _ in info],
               Q=[q.detach() for q in Q], amplitudes=amps, collective=coll, blocks=det)
    return E, out, (Bd, F)


def energy(problem, params, n_osv=None, clusters=None):
    """MBE(3)-OSV-MP2 correlation energy E = sum_c w_c E^c_Hylleraas and the diagnostics dictionary."""
    with torch.no_grad():
        _, out, _ = _run(problem, params, n_osv, grad=False, clusters=clusters)
    return out


def energy_osv_screened(problem, params, l2b, l3b, l_discard=1e-7, n_osv=None):
    """MBE energy under the paper's screening (Sec. 2.2.1-2.2.2): strong 2b and 3b clusters by the OSV-overlap
    metrics (select_clusters_osv), every weak pair (l_discard <= s2b_ij <= l2b) added through its one-block energy
    (weak_pair_one_block), pairs with s2b_ij below l_discard dropped.  Weak pairs exist from mbe_order 2 on."""
    with torch.no_grad():
        eps, F, Bd = _inputs(problem, False)
        Q, _ = _osvs(Bd, eps, F, params, n_osv)
        s = osv_overlap_metric([q.numpy() for q in Q])
        clusters = select_clusters_osv(s, l2b, l3b, params.mbe_order)
        strong = energy(problem, params, n_osv, clusters=clusters)
        n = problem.n_occ
        weak = [(i, j) for i in range(n) for j in range(i + 1, n)
                if params.mbe_order >= 2 and l_discard <= s[i, j] <= l2b]
        Ew = sum(weak_pair_one_block(problem, params, i, j, n_osv)[1] for i, j in weak)
    return dict(E=strong["E"] + Ew, E_strong=strong["E"], E_weak=float(Ew), clusters=clusters, weak_pairs=weak,
                s2b=s)


def posterior_correction(problem, params, n_osv=None, clusters=None):
    """One-step posterior correction over the MBE collective amplitudes (Sec. 3, the MBE(n > 3) estimate).

    With the converged collective amplitudes T (Eqs. 28-32), every ordered pair ij that has them gets the residual
    dR_(ij,ij) of Eq. 4 with k running over the union of the LMOs of the selected clusters that contain both i and
    j (pairs without collective amplitudes count as zero), and one preconditioned step
    dT = -V [(V^T dR V) / D] V^T in the pair's pseudo-canonical basis (the cluster solver's update).  Returns the
    MBE energy, the same pair functional sum over pairs of <K + R(T'), 2T' - T'^T> (Eq. 3) at T' = T (E_global)
    and at T' = T + dT (E_corrected), and the largest ||V^T dR V||_F."""
    with torch.no_grad():
        out = energy(problem, params, n_osv, clusters=clusters)
        b, coll, cl = out["blocks"], out["collective"], out["clusters"]
        F = torch.as_tensor(problem.f_occ, dtype=DT)
        T = {p: t.clone() for p, t in coll.items()}
        ks = {}
        for p in T:
            i, j = p
            ks[p] = sorted({k for c in cl if i in c and j in c for k in c})
        dT, rmax = {}, 0.0
        for p in T:
            cs = ClusterSolver(tuple(ks[p]), b, F, params.tau_red)
            Tz = {q: T.get(q, torch.zeros(b.dom(q).shape[1], b.dom(q).shape[1], dtype=DT))
                  for q in [(x, y) for x in ks[p] for y in ks[p]]}
            R = cs.residual(p, Tz)
            V, D = cs.precond(p)
            Rt = V.T @ R @ V
            rmax = max(rmax, float(torch.linalg.norm(Rt)))
            dT[p] = -V @ (Rt / D) @ V.T
        def functional(A):
            E = torch.zeros((), dtype=DT)
            for p in A:
                cs = ClusterSolver(tuple(ks[p]), b, F, params.tau_red)
                Tz = {q: A.get(q, torch.zeros(b.dom(q).shape[1], b.dom(q).shape[1], dtype=DT))
                      for q in [(x, y) for x in ks[p] for y in ks[p]]}
                R = cs.residual(p, Tz)
                E = E + torch.sum((b.K(p) + R) * (2.0 * A[p] - A[p].T))
            return float(E)

        Eg = functional(T)
        Ec = functional({p: T[p] + dT[p] for p in T})
    return dict(E=out["E"], E_global=Eg, E_corrected=Ec, dR_max=rmax, k_sets=ks)


def gradient(problem, params, n_osv=None, clusters=None):
    """Energy and its derivative with respect to the stored DF entries B (list of (n_vir, a_i) arrays in
    each LMO's local aux order) and every entry of F_occ (entrywise, F used as given)."""
    E, out, (Bd, F) = _run(problem, params, n_osv, grad=True, clusters=clusters)
    E.backward()
    dB = []
    for i in range(problem.n_occ):
        idx = problem.aux_idx[problem.aux_ptr[i]:problem.aux_ptr[i + 1]].astype(np.int64)
        g = Bd[i].grad   # None when no selected cluster touches LMO i: its derivative is zero
        dB.append(g[:, idx].numpy().copy() if g is not None else np.zeros((Bd[i].shape[0], len(idx))))
    out["dB"] = dB
    out["dF"] = F.grad.numpy().copy()
    return out

"""The bookkeeping of two restructured FP32 kernels of the OSV eigenproblem (Eq. 6), restated in NumPy (FP64) and
checked against direct computations on the CPU.  These check the schedules, not the CUDA code; the GPU tests
compare the kernels' results with the FP64 path.

* Delayed-update Householder tridiagonalisation (k_tridiag_delayed): the rank-2 updates of NB consecutive steps
  are written into the stored lower triangle together, by the pass of every NB-th step; the passes in between
  read the stored triangle and correct A v for the updates still pending; the stashed column and the last two
  rows get the updates not yet written.  The pairs (v_s, p_s) live in a ring of NB + 1 slots.  The tridiagonal
  it produces must have the eigenvalues of A for every NB.
* Blocked compact-WY back-transformation (k_reflect_wy_tiled): per block of 32 reflectors, W = V_j Y^T over
  column chunks (reflector i zero before column k0 + 1 + i, rows >= R zero), Z = T_j^T W or T_j W, Y -= Z^T V_j
  chunk by chunk, with T_j from the block's Gram.  It must equal applying the reflectors one at a time, in both
  directions.
"""
import numpy as np
import pytest

KNB, KTCW = 32, 64   # reflectors per compact-WY block, column chunk


def tridiag_delayed(A0, NB):
    """Eigenvalues of the tridiagonal the delayed-update schedule produces from symmetric A0."""
    n = A0.shape[0]
    A = A0.copy()                 # the stored matrix (lower triangle read and written)
    NS = NB + 1                   # ring slots
    V = np.zeros((NS, n))
    P = np.zeros((NS, n))
    vs = lambda s: V[s % NS]
    ps = lambda s: P[s % NS]
    d, e, nx = np.zeros(n), np.zeros(n), np.zeros(n)
    for k in range(n - 2):
        mc = 0 if k == 0 else (k - 1) % NB + 1          # updates of steps k - mc .. k - 1 not in the stash
        x = A[k].copy() if k == 0 else nx.copy()
        col = np.zeros(n)
        for c in range(k + 1, n):
            col[c] = x[c] - sum(vs(k - t)[k] * ps(k - t)[c] + ps(k - t)[k] * vs(k - t)[c] for t in range(1, mc + 1))
        d[k] = (A[0, 0] if k == 0 else nx[k]) - sum(2 * vs(k - t)[k] * ps(k - t)[k] for t in range(1, mc + 1))
        v = np.zeros(n)
        v[k + 1:] = col[k + 1:]
        alpha, x0 = np.linalg.norm(v), v[k + 1]
        beta = 0.0
        if alpha > 0:
            sgn = 1.0 if x0 >= 0 else -1.0
            v[k + 1] = x0 + sgn * alpha
            e[k] = -sgn * alpha
            beta = 1 / (alpha * (alpha + abs(x0)))
        V[k % NS] = v
        flush = k % NB == 0
        if flush:                                         # write the pending updates of steps k - NB .. k - 1
            for s in range(k - NB, k):
                if s < 0:
                    continue                              # ring slots of steps before 0 hold zeros
                vv, pp = vs(s), ps(s)
                for r in range(k + 1, n):
                    A[r, k + 1:r + 1] -= vv[r] * pp[k + 1:r + 1] + pp[r] * vv[k + 1:r + 1]
        L = np.tril(A[k + 1:, k + 1:])
        y = np.zeros(n)
        y[k + 1:] = (L + L.T - np.diag(np.diag(L))) @ v[k + 1:]   # A_stored v from the lower triangle
        nx = np.zeros(n)
        nx[k + 1:] = A[k + 1:, k + 1]                     # column k + 1 as the pass leaves it
        for t in range(1, (0 if flush else k % NB) + 1):  # corrections for the updates still pending
            vv, pp = vs(k - t), ps(k - t)
            y[k + 1:] -= vv[k + 1:] * (pp[k + 1:] @ v[k + 1:]) + pp[k + 1:] * (vv[k + 1:] @ v[k + 1:])
        p = beta * y
        p[k + 1:] -= 0.5 * beta * (p[k + 1:] @ v[k + 1:]) * v[k + 1:]
        P[k % NS] = 0.0
        P[k % NS][k + 1:] = p[k + 1:]
    a, b = n - 2, n - 1
    da, ea, db = A[a, a], A[b, a], A[b, b]
    kl = n - 3
    for s in range(kl - kl % NB, kl + 1):                 # the updates not yet written into the last two rows
        vv, pp = vs(s), ps(s)
        da -= 2 * vv[a] * pp[a]
        ea -= vv[b] * pp[a] + pp[b] * vv[a]
        db -= 2 * vv[b] * pp[b]
    d[a], e[a], d[b] = da, ea, db
    return np.linalg.eigvalsh(np.diag(d) + np.diag(e[:-1], 1) + np.diag(e[:-1], -1))


@pytest.mark.parametrize("n", [5, 6, 13, 40])
@pytest.mark.parametrize("NB", [1, 2, 3, 4])
def test_delayed_update_schedule_keeps_the_spectrum(n, NB):
    rng = np.random.default_rng(100 + n)
    X = rng.standard_normal((n, n))
    A0 = X + X.T
    ref = np.linalg.eigvalsh(A0)
    assert np.abs(tridiag_delayed(A0, NB) - ref).max() <= 1e-12 * np.abs(ref).max()


def _reflectors(n, rng):
    """Householder reflectors in rows k of A (columns k+1 ..), H_k = I - tau_k v v^T (v explicit)."""
    A = np.zeros((n, n))
    tau = np.zeros(n)
    for k in range(n - 2):
        v = rng.standard_normal(n - k - 1)
        A[k, k + 1:] = v
        tau[k] = 2 / (v @ v)
    return A, tau


def _wy_blocks(n):
    return 0 if n < 3 else (n - 2 + KNB - 1) // KNB


def _t_factors(A, tau, n):
    """T_j of the compact-WY block B_j = I - V_j T_j V_j^T: T[0:i, i] = -tau_i T[0:i, 0:i] G[0:i, i]."""
    T = np.zeros((_wy_blocks(n), KNB, KNB))
    for j in range(_wy_blocks(n)):
        k0, kb = j * KNB, min(KNB, n - 2 - j * KNB)
        Vj = np.zeros((KNB, n))
        for i in range(kb):
            Vj[i, k0 + i + 1:] = A[k0 + i, k0 + i + 1:]
        G = Vj @ Vj.T
        for i in range(kb):
            T[j, :i, i] = -tau[k0 + i] * T[j, :i, :i] @ G[:i, i]
            T[j, i, i] = tau[k0 + i]
    return T


def _one_at_a_time(A, tau, Y, forward):
    n = A.shape[0]
    Y = Y.copy()
    for k in (range(n - 2) if forward else range(n - 3, -1, -1)):
        v = np.zeros(n)
        v[k + 1:] = A[k, k + 1:]
        Y -= tau[k] * np.outer(Y @ v, v)
    return Y


def _tiled(A, T, Y0, R, forward):
    n = A.shape[0]
    Y = Y0.copy()
    Jb = _wy_blocks(n)
    for s in range(Jb):
        j = s if forward else Jb - 1 - s
        k0, kb = j * KNB, min(KNB, n - 2 - j * KNB)
        m0, c0 = n - k0 - 1, k0 + 1

        def chunk(cbeg, cw):
            Vc, Yc = np.zeros((KNB, KTCW)), np.zeros((64, KTCW))
            for i in range(kb):
                for cc in range(cw):
                    if cbeg + cc >= i:
                        Vc[i, cc] = A[k0 + i, c0 + cbeg + cc]
            Yc[:R, :cw] = Y[:R, c0 + cbeg:c0 + cbeg + cw]
            return Vc, Yc

        W = np.zeros((KNB, 64))
        for cbeg in range(0, m0, KTCW):
            Vc, Yc = chunk(cbeg, min(KTCW, m0 - cbeg))
            W += Vc @ Yc.T
        Z = T[j].T @ W if forward else T[j] @ W
        for cbeg in range(0, m0, KTCW):
            cw = min(KTCW, m0 - cbeg)
            Vc, Yc = chunk(cbeg, cw)
            Y[:R, c0 + cbeg:c0 + cbeg + cw] = (Yc - Z.T @ Vc)[:R, :cw]
    return Y


@pytest.mark.parametrize("n,R", [(60, 41), (60, 6), (37, 20), (130, 64), (3, 2)])
@pytest.mark.parametrize("forward", [0, 1])
def test_tiled_compact_wy_equals_reflector_by_reflector(n, R, forward):
    rng = np.random.default_rng(n * 100 + R)
    A, tau = _reflectors(n, rng)
    Y0 = rng.standard_normal((R, n))
    ref = _one_at_a_time(A, tau, Y0, forward)
    out = _tiled(A, _t_factors(A, tau, n), Y0, R, forward)
    assert np.abs(out - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())

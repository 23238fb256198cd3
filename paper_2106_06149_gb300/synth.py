"""Seeded synthetic inputs for MBE(3)-OSV-MP2 (shared by the CUDA path's tests, the oracle's tests and the bench).

This module draws random numbers and lays them out; it holds none of the method's arithmetic.  The paper's
molecules (Baker set, (Gly)_n, C60@catcher, (H2O)_190, Sec. 3) are not available, so every workload is a
synthetic stand-in with the value distributions below:

* occupied Fock: f_ii ~ U[-1.2, -0.4] Eh, f_ij = 0.05 exp(-d_ij / 2 A) for i != j (symmetric);
* virtual energies eps_a ~ U[0.1, 3.0] Eh;
* DF tensor B_ia^P = g exp(-d(i, P) / 3 A), g ~ N(0, 0.05^2) i.i.d. per (i, a, P), zero outside the local
  fitting domain of LMO i (all aux functions for the chain workloads, aux centres within `radius` otherwise).

One numpy Generator per problem, drawn in a fixed order: LMO points, aux points, f_ii, eps_a, g.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Problem", "Params", "make_problem", "workload", "WORKLOADS"]


@dataclasses.dataclass
class Params:
    """Method parameters (names follow the paper: l_osv for the OSV cut, Sec. 2.1; cutoffs for clusters)."""

    l_osv: float = 1e-4       # keep OSVs with eigenvalue > l_osv (Eq. 6)
    n_osv_max: int = 40       # cap on OSVs per LMO (0 = no cap)
    n_osv_fixed: int = 0      # > 0: keep exactly this many OSVs per LMO (threshold ignored)
    r2b: float = 8.0          # pair cluster kept iff |r_i - r_j| <= r2b (Angstrom)
    r3b: float = 6.0          # triple kept iff all three distances <= r3b and its pairs are kept
    mbe_order: int = 3        # 1, 2, 3; 0 = one cluster holding every LMO (no MBE truncation)
    tau_red: float = 1e-8     # drop pair-overlap eigenvalues below this (redundant pair space)
    tol: float = 1e-8         # residual convergence: max_ij ||R~_ij||_F <= tol
    max_iter: int = 100       # residual iteration cap
    precision: int = 0        # 0 = FP64, 2 = exact BF16x4 tensor-core GEMMs (1, split TF32, is rejected)

    def as_dict(self):
        return dataclasses.asdict(self)


@dataclasses.dataclass
class Problem:
    centres: np.ndarray        # (n_occ, 3) float64, Angstrom
    aux_centres: np.ndarray    # (n_aux, 3) float64
    f_occ: np.ndarray          # (n_occ, n_occ) float64, Eh
    eps_vir: np.ndarray        # (n_vir,) float64, Eh
    aux_ptr: np.ndarray        # (n_occ + 1,) int64 CSR offsets into aux_idx
    aux_idx: np.ndarray        # (sum a_i,) int32, sorted local aux indices per LMO
    B: np.ndarray              # flat, concatenated per-LMO blocks, each row-major (n_vir, a_i)
    seed: int = 0
    name: str = "custom"

    @property
    def n_occ(self):
        return self.centres.shape[0]

    @property
    def n_vir(self):
        return self.eps_vir.shape[0]

    @property
    def n_aux(self):
        return self.aux_centres.shape[0]

    def a(self, i):
        return int(self.aux_ptr[i + 1] - self.aux_ptr[i])

    def b_offset(self, i):
        return int(self.aux_ptr[i]) * self.n_vir

    def B_block(self, i):
        """(n_vir, a_i) view of LMO i's local DF block."""
        o = self.b_offset(i)
        return self.B[o:o + self.n_vir * self.a(i)].reshape(self.n_vir, self.a(i))

    def B_dense(self, i, dtype=np.float64):
        """(n_vir, n_aux) copy with zeros outside LMO i's fitting domain."""
        out = np.zeros((self.n_vir, self.n_aux), dtype=dtype)
        idx = self.aux_idx[self.aux_ptr[i]:self.aux_ptr[i + 1]]
        out[:, idx] = self.B_block(i)
        return out

    def full_domain(self):
        return all(self.a(i) == self.n_aux for i in range(self.n_occ))


def _chain(n, spacing):
    c = np.zeros((n, 3))
    c[:, 0] = spacing * np.arange(n)
    return c


def _cube(rng, n, box, dmin, max_tries=1_000_000):
    pts = np.empty((n, 3))
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rejection sampling did not place all points")
        p = rng.uniform(0.0, box, size=3)
        if k == 0 or np.min(np.linalg.norm(pts[:k] - p, axis=1)) >= dmin:
            pts[k] = p
            k += 1
    return pts


def make_problem(n_occ, n_vir, n_aux, geometry="chain", spacing=1.5, box=20.0, dmin=1.4, radius=None,
                 seed=0, dtype=np.float64, f_offdiag=0.05, g_sigma=0.05, name="custom"):
    """Draw one synthetic problem.  geometry: 'chain' (LMOs spacing apart on x, aux uniform on the segment)
    or 'cube' (LMOs by sequential rejection sampling with min separation dmin, aux uniform in the cube).
    radius: local fitting domain radius (None = every aux function in every domain)."""
    rng = np.random.default_rng(seed)
    if geometry == "chain":
        centres = _chain(n_occ, spacing)
        length = spacing * max(n_occ - 1, 1)
        aux = np.zeros((n_aux, 3))
        aux[:, 0] = rng.uniform(0.0, length, size=n_aux)
    elif geometry == "cube":
        centres = _cube(rng, n_occ, box, dmin)
        aux = rng.uniform(0.0, box, size=(n_aux, 3))
    else:
        raise ValueError(geometry)
    fii = rng.uniform(-1.2, -0.4, size=n_occ)
    eps = rng.uniform(0.1, 3.0, size=n_vir)
    d_oo = np.linalg.norm(centres[:, None, :] - centres[None, :, :], axis=-1)
    f = f_offdiag * np.exp(-d_oo / 2.0)
    np.fill_diagonal(f, fii)
    d_oa = np.linalg.norm(centres[:, None, :] - aux[None, :, :], axis=-1)
    ptr = [0]
    idx = []
    blocks = []
    for i in range(n_occ):
        dom = np.arange(n_aux) if radius is None else np.nonzero(d_oa[i] <= radius)[0]
        g = rng.standard_normal((n_vir, dom.size)) * g_sigma
        blocks.append((g * np.exp(-d_oa[i, dom] / 3.0)[None, :]).astype(dtype).ravel())
        idx.append(dom.astype(np.int32))
        ptr.append(ptr[-1] + dom.size)
    B = np.concatenate(blocks) if blocks else np.zeros(0, dtype=dtype)
    return Problem(centres=centres, aux_centres=aux, f_occ=f, eps_vir=eps,
                   aux_ptr=np.asarray(ptr, dtype=np.int64), aux_idx=np.concatenate(idx).astype(np.int32),
                   B=B, seed=seed, name=name)


def _radius_for_mean_domain(seed, n_occ, box, dmin, n_aux, target):
    rng = np.random.default_rng(seed)
    centres = _cube(rng, n_occ, box, dmin)
    aux = rng.uniform(0.0, box, size=(n_aux, 3))
    d = np.linalg.norm(centres[:, None, :] - aux[None, :, :], axis=-1)
    lo, hi = 1.0, box * math.sqrt(3.0)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if (d <= mid).sum(axis=1).mean() < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# The five workloads: (description, problem kwargs, params kwargs).  The gradient workloads (2-4) converge the
# residual to 1e-10: the Hylleraas energy is second order in the residual, its derivative at fixed amplitudes only
# first order, and the 1e-6 gradient bar over hundreds of clusters per Fock entry needs the tighter tolerance.
WORKLOADS = {
    0: ("full OSV-MP2, 10 LMOs on a 1.5 A chain, n_vir=60, n_aux=240, 12 OSVs, one cluster",
        dict(n_occ=10, n_vir=60, n_aux=240, geometry="chain", seed=0),
        dict(n_osv_fixed=12, mbe_order=0)),
    1: ("MBE(3) energy, 64 LMOs on a 1.5 A chain, n_vir=400, n_aux=1600, l_osv=1e-4 capped at 40",
        dict(n_occ=64, n_vir=400, n_aux=1600, geometry="chain", seed=1),
        dict(mbe_order=3)),
    2: ("MBE(3) mixed, 256 LMOs in a 20 A cube, n_vir=1500, n_aux=6000, 7 A fitting domains, B fp32",
        dict(n_occ=256, n_vir=1500, n_aux=6000, geometry="cube", box=20.0, radius=7.0, seed=2,
             dtype=np.float32),
        dict(mbe_order=3, precision=2, tol=1e-10)),
    3: ("gradient, 128 LMOs in a 14 A cube, n_vir=800, n_aux=3200, 7 A fitting domains",
        dict(n_occ=128, n_vir=800, n_aux=3200, geometry="cube", box=14.0, radius=7.0, seed=3),
        dict(mbe_order=3, tol=1e-10)),
    4: ("large MBE(3) E+grad, 512 LMOs in a 28 A cube, n_vir=3000, n_aux=12000, ~2000 aux per domain, B fp32",
        dict(n_occ=512, n_vir=3000, n_aux=12000, geometry="cube", box=28.0, radius="mean2000", seed=4,
             dtype=np.float32),
        dict(mbe_order=3, precision=2, tol=1e-10)),
}


def workload(k):
    """(Problem, Params) for workload k of WORKLOADS."""
    desc, pk, prm = WORKLOADS[k]
    pk = dict(pk)
    if pk.get("radius") == "mean2000":
        pk["radius"] = _radius_for_mean_domain(pk["seed"], pk["n_occ"], pk["box"], 1.4, pk["n_aux"], 2000.0)
    p = make_problem(name=f"workload{k}", **pk)
    return p, Params(**prm)

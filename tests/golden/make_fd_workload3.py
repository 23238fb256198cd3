"""Writes fd_workload3.json: central finite differences of the oracle's MBE(3)-OSV-MP2 energy with respect to 200
random entries of B and F_occ of workload 3 (128 LMOs in a 14 A cube, n_vir 800, n_aux 3200, 7 A fitting domains,
l_osv 1e-4 capped at 40 OSVs, 8/6 A cutoffs), at two steps: h = 1e-5 and h = 1e-4.  Calls only oracle/ (and the
seeded generator).

An entry of B_i changes only the clusters that hold LMO i; an entry f_xy only those that hold x and y (and f_xx
those that hold x).  Every superset of such a cluster holds the same LMOs, so the MBE weights of these clusters
are the same in the full cluster list and in the list of the clusters that hold them: the energy difference is
that of the oracle run on the restricted problem (oracle/subproblem.py) with that cluster list.  OSV counts
are frozen at the base point (the finite differences of a step function are meaningless).

Per step h, the second-order stencil (E(h) - E(-h)) / 2h and the fourth-order one
(8 [E(h) - E(-h)] - [E(2h) - E(-2h)]) / 12h.  Why two steps: each energy carries FP64 rounding noise of about
1e-14 |E| (the eigensolves, the iterations and the sums over hundreds of clusters), and a finite difference at
step h inherits about that divided by h.  The energy an entry reaches is up to 1.6e3 Eh (82 LMOs and 421 clusters
around LMO 83), so at h = 1e-5 the noise is about 1e-6, the size of the gradient bar itself (there the oracle's
own autograd agrees with the analytic GPU gradient to 4e-12 while the differences scatter by 1e-6 from one step
to the next).  At h = 1e-4 the noise is ten times smaller and the fourth-order truncation O(h^4) still far below
it.  E_reached = (E(h) + E(-h)) / 2 at h = 1e-5 is stored to size the noise.

    python tests/golden/make_fd_workload3.py [workers]
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

STEPS = (1e-5, 1e-4)
SEED = 3003
N_LMO, N_B_PER_LMO, N_F_OFF = 5, 30, 9
TOL = 1e-10

_cache = {}


def _problem():
    if "p" not in _cache:
        import oracle
        from paper_2106_06149_gb300.synth import workload
        p, prm = workload(3)
        prm.tol = TOL
        prm.max_iter = 400
        cl = oracle.select_clusters(p.centres, prm.r2b, prm.r3b, prm.mbe_order)
        _cache["p"] = (p, prm, cl)
    return _cache["p"]


def entries():
    """The 200 entries: ("B", i, a, P_local) and ("F", x, y), drawn from one seeded generator."""
    import oracle  # noqa: F401
    p, prm, cl = _problem()
    rng = np.random.default_rng(SEED)
    lmos = [int(x) for x in rng.choice(p.n_occ, size=N_LMO, replace=False)]
    out = []
    for i in lmos:
        for _ in range(N_B_PER_LMO):
            out.append(("B", i, int(rng.integers(p.n_vir)), int(rng.integers(p.a(i)))))
    for x in lmos:
        out.append(("F", x, x))
        partners = sorted({k for c in cl if x in c for k in c if k != x})
        for y in rng.choice(partners, size=N_F_OFF, replace=False):
            y = int(y)
            out.append(("F", x, y) if rng.random() < 0.5 else ("F", y, x))
    return out


def _members(e):
    return [e[1]] if e[0] == "B" or e[1] == e[2] else [e[1], e[2]]


def energy_part(e, delta, n_osv=None):
    """Energy of the clusters that the entry e reaches, with the entry moved by delta."""
    import oracle
    from oracle.subproblem import clusters_holding, restrict
    p, prm, cl = _problem()
    _, lmos, sub_cl = clusters_holding(cl, _members(e))
    q = restrict(p, lmos)
    if e[0] == "B":
        t = lmos.index(e[1])
        q.B = q.B.copy()
        q.B[int(q.aux_ptr[t]) * p.n_vir + e[2] * q.a(t) + e[3]] += delta
    else:
        q.f_occ = q.f_occ.copy()
        q.f_occ[lmos.index(e[1]), lmos.index(e[2])] += delta
    out = oracle.energy(q, prm, n_osv=n_osv, clusters=sub_cl)
    return out["E"], out["n_osv"]


def _task(args):
    import torch
    torch.set_num_threads(1)
    k, e, n_osv = args
    out = {}
    for h in STEPS:
        ep, em = energy_part(e, h, n_osv)[0], energy_part(e, -h, n_osv)[0]
        d1 = ep - em
        d2 = energy_part(e, 2.0 * h, n_osv)[0] - energy_part(e, -2.0 * h, n_osv)[0]
        out[h] = (d1 / (2.0 * h), (8.0 * d1 - d2) / (12.0 * h))
        if h == STEPS[0]:
            out["E"] = 0.5 * (ep + em)
    return k, out


def main(workers):
    t0 = time.time()
    ents = entries()
    # base OSV counts of every LMO that some entry reaches (frozen for the finite differences)
    import oracle
    p, prm, cl = _problem()
    n_base = {}
    for e in ents:
        for m in _members(e):
            for c in cl:
                if m in c:
                    for k in c:
                        n_base.setdefault(k, None)
    Bd_eps = None
    import torch
    eps = torch.as_tensor(p.eps_vir, dtype=torch.float64)
    for k in sorted(n_base):
        w, _ = oracle.osv_decompose(oracle.tkk(oracle.dense_B(p, k), eps, torch.tensor(p.f_occ[k, k])))
        n_base[k] = oracle.n_osv_select(w, prm.l_osv, prm.n_osv_max, prm.n_osv_fixed)
    del Bd_eps
    tasks = []
    from oracle.subproblem import clusters_holding
    for k, e in enumerate(ents):
        _, lmos, _ = clusters_holding(cl, _members(e))
        tasks.append((k, e, [n_base[m] for m in lmos]))
    vals = [None] * len(ents)
    with mp.get_context("spawn").Pool(workers) as pool:
        for k, v in pool.imap_unordered(_task, tasks):
            vals[k] = v
            done = sum(x is not None for x in vals)
            if done % 10 == 0:
                print(f"{done}/{len(ents)} entries, {time.time() - t0:.0f} s", flush=True)
    rec = {"workload": 3, "steps": list(STEPS), "seed": SEED, "tol": TOL,
           "params": {"l_osv": prm.l_osv, "n_osv_max": prm.n_osv_max, "r2b": prm.r2b, "r3b": prm.r3b,
                      "mbe_order": prm.mbe_order, "tau_red": prm.tau_red},
           "n_osv": {str(k): v for k, v in sorted(n_base.items())},
           "note": "central differences of the oracle energy (oracle/osvmp2.py) restricted to the clusters each "
                   "entry reaches: fd4_h / fd2_h = fourth-order stencil on +-h, +-2h / second-order stencil on "
                   "+-h, for h = 1e-5 and 1e-4; E_reached = the restricted energy at the base point (to O(h^2)); "
                   "B entries index LMO i's local block (virtual a, local fitting function P)",
           "entries": [{"kind": e[0], "idx": list(e[1:]), "fd4_1e-5": v[STEPS[0]][1], "fd2_1e-5": v[STEPS[0]][0],
                        "fd4_1e-4": v[STEPS[1]][1], "fd2_1e-4": v[STEPS[1]][0], "E_reached": v["E"]}
                       for e, v in zip(ents, vals)]}
    with open(os.path.join(HERE, "fd_workload3.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(f"wrote fd_workload3.json in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else max(1, (os.cpu_count() or 2) - 1))

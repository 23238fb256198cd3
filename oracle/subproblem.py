"""Restriction of a synthetic problem to a subset of its LMOs (data slicing only, no method arithmetic).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: used by tests/, tests/golden/ and bench.py's CPU legs.

Used by the golden-value script and the parity tests: the MBE energy contribution of the clusters that contain a
given LMO (or pair of LMOs) depends only on the LMOs of those clusters, so the oracle can evaluate it on the
restricted problem."""
from __future__ import annotations

import numpy as np

from paper_2106_06149_gb300.synth import Problem


def restrict(p: Problem, lmos):
    """The problem made of the LMOs `lmos` (in that order): their centres, Fock block, fitting domains and DF
    blocks; virtual energies and aux centres unchanged."""
    lmos = [int(x) for x in lmos]
    ptr = [0]
    idx, blocks = [], []
    for i in lmos:
        idx.append(p.aux_idx[p.aux_ptr[i]:p.aux_ptr[i + 1]])
        blocks.append(np.asarray(p.B_block(i)).ravel())
        ptr.append(ptr[-1] + p.a(i))
    return Problem(centres=p.centres[lmos].copy(), aux_centres=p.aux_centres, f_occ=p.f_occ[np.ix_(lmos, lmos)].copy(),
                   eps_vir=p.eps_vir, aux_ptr=np.asarray(ptr, dtype=np.int64),
                   aux_idx=np.concatenate(idx).astype(np.int32), B=np.concatenate(blocks).copy(), seed=p.seed,
                   name=p.name + "_sub")


def clusters_holding(clusters, members):
    """The clusters that contain every LMO of `members`, the sorted union of their LMOs, and the clusters renumbered
    into positions of that union."""
    sel = [c for c in clusters if all(m in c for m in members)]
    lmos = sorted({k for c in sel for k in c})
    pos = {k: t for t, k in enumerate(lmos)}
    return sel, lmos, [tuple(pos[k] for k in c) for c in sel]

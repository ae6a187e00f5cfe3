"""Scalar observables as one- plus two-body operators in the interaction format.

The total angular momentum squared is J^2 = sum_i j_i^2 + sum_{i != j} j_i . j_j.
Its single-particle part is j_a (j_a + 1) on every particle in orbit a, and
its two-body part sum_{i < j} 2 j_i . j_j is diagonal in the normalized
coupled pair states:

    <ab; J T | 2 j_1 . j_2 | ab; J T> = J (J + 1) - j_a (j_a + 1) - j_b (j_b + 1),

for every Pauli-allowed (a <= b, J, T), the same for T = 0 and T = 1.  Written
as single-particle energies and TBMEs V_JT(ab, ab), it loads into a context
like any interaction (Sec. "Interaction files"): on the same basis the
library's H x kernels then apply J^2, and <J^2> of a block of vectors comes
from one product and one block inner product, all on the GPU.  This is how
the paper evaluates J^2, as an expectation value after the diagonalization.
"""
from __future__ import annotations

import numpy as np

from . import _native as N
from .inputs import tbme_labels


def j2_operator(orbits):
    """(spe, tbmes) of J^2 for the orbits (labels 1-based, the interaction format)."""
    jj = [o.twoj * (o.twoj + 2) / 4.0 for o in orbits]   # j (j + 1)
    spe = list(jj)
    tb = []
    for (a, b, c, d, J, T) in tbme_labels(orbits):
        if (a, b) != (c, d):
            continue
        tb.append((a, b, c, d, J, T, J * (J + 1.0) - jj[a - 1] - jj[b - 1]))
    return spe, tb


def j2_context(orbits, Z, Nn, twoM, parity=+1, device=0):
    """A context on the (orbits, Z, N, 2M, parity) basis whose "interaction" is J^2."""
    spe, tb = j2_operator(orbits)
    return N.make(orbits, spe, tb, Z, Nn, twoM, parity, device=device)


def expectation(ctx_op, psi, k, dtype, stream=None):
    """<psi_i | O | psi_j> / sqrt(<psi_i|psi_i> <psi_j|psi_j>), a k x k numpy
    array, for the k columns of psi (a CUDA tensor [dim][k] of the dtype),
    with O the operator loaded into ctx_op: O psi by its H x kernels, the
    inner products by bs_block_dots (extended precision)."""
    import torch

    y = torch.empty_like(psi)
    ctx_op.apply_H(psi, y, k, dtype, stream)
    num = torch.zeros(k * k, device=psi.device, dtype=torch.float64)
    den = torch.zeros(k * k, device=psi.device, dtype=torch.float64)
    ctx_op.block_dots(psi, 1, y, k, dtype, num, stream)
    ctx_op.block_dots(psi, 1, psi, k, dtype, den, stream)
    num = num.cpu().numpy().reshape(k, k)
    nrm = np.sqrt(np.diag(den.cpu().numpy().reshape(k, k)))
    return num / np.outer(nrm, nrm)


def j_from_j2(j2):
    """J from J (J + 1)."""
    return 0.5 * (-1.0 + np.sqrt(1.0 + 4.0 * np.asarray(j2)))

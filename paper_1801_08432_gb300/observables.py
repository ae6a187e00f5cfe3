"""Scalar observables: J^2 and T^2 as one- plus two-body operators in the
interaction format, and orbit occupations from the adjoint.

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


def t2_operator(orbits):
    """(spe, tbmes) of the isospin squared T^2 = sum_i t_i^2 + sum_{i<j} 2 t_i . t_j:
    3/4 on every particle, and <ab; J T| 2 t_1 . t_2 |ab; J T> = T (T + 1) - 3/2
    on every pair state (isospin only, so diagonal in (ab, J))."""
    spe = [0.75] * len(orbits)
    tb = [(a, b, c, d, J, T, T * (T + 1.0) - 1.5) for (a, b, c, d, J, T) in tbme_labels(orbits)
          if (a, b) == (c, d)]
    return spe, tb


def t2_context(orbits, Z, Nn, twoM, parity=+1, device=0):
    """A context on the (orbits, Z, N, 2M, parity) basis whose "interaction" is T^2."""
    spe, tb = t2_operator(orbits)
    return N.make(orbits, spe, tb, Z, Nn, twoM, parity, device=device)


def occupations(ctx, psi, dtype, stream=None):
    """Orbit occupations n_a = <psi|N_a|psi> / <psi|psi> of the columns of psi
    (CUDA tensor [dim][k] in dtype), as a k x (number of orbits) numpy array.  The SPEs
    enter H as sum_a e_a N_a, so n_a = dE/de_a (Hellmann-Feynman): the
    adjoint's SPE derivatives psi^T (dH/de_a) psi from the GPU's transition
    densities, one column at a time, over psi^T psi from bs_block_dots."""
    import torch

    k = psi.shape[1]
    n_spe = ctx.n_spe
    n_theta = n_spe + ctx.n_tbme
    out = np.zeros((k, n_spe))
    gx = torch.empty((psi.shape[0], 1), device=psi.device, dtype=psi.dtype)
    nrm = torch.zeros(1, device=psi.device, dtype=torch.float64)
    for m in range(k):
        x = psi[:, m:m + 1].contiguous()
        g = ctx.apply_H_backward(x, x, gx, 1, dtype, n_theta=n_theta, stream=stream)
        ctx.block_dots(x, 1, x, 1, dtype, nrm, stream)
        out[m] = g[:n_spe] / float(nrm.cpu()[0])
    return out


def j2_context(orbits, Z, Nn, twoM, parity=+1, device=0):
    """A context on the (orbits, Z, N, 2M, parity) basis whose "interaction" is J^2."""
    spe, tb = j2_operator(orbits)
    return N.make(orbits, spe, tb, Z, Nn, twoM, parity, device=device)


def expectation(ctx_op, psi, k, dtype, stream=None):
    """<psi_i | O | psi_j> / sqrt(<psi_i|psi_i> <psi_j|psi_j>), a k x k numpy
    array, for the k <= 8 columns of psi (a CUDA tensor [dim][k] of the dtype),
    with O the operator loaded into ctx_op: O psi by its H x kernels, the
    inner products by bs_block_dots (extended precision)."""
    import torch

    if not 1 <= k <= 8:
        raise ValueError("expectation: 1 <= k <= 8 columns")
    kk = 1 if k == 1 else 2 if k == 2 else 4 if k <= 4 else 8   # the kernels' block sizes
    if kk != k:   # zero columns up to the next block size; only the k x k corner is returned
        psi = torch.cat([psi[:, :k], torch.zeros((psi.shape[0], kk - k), device=psi.device, dtype=psi.dtype)],
                        dim=1).contiguous()
    y = torch.empty_like(psi)
    ctx_op.apply_H(psi, y, kk, dtype, stream)
    num = torch.zeros(kk * kk, device=psi.device, dtype=torch.float64)
    den = torch.zeros(kk * kk, device=psi.device, dtype=torch.float64)
    ctx_op.block_dots(psi, 1, y, kk, dtype, num, stream)
    ctx_op.block_dots(psi, 1, psi, kk, dtype, den, stream)
    num = num.cpu().numpy().reshape(kk, kk)[:k, :k]
    nrm = np.sqrt(np.diag(den.cpu().numpy().reshape(kk, kk))[:k])
    return num / np.outer(nrm, nrm)


def j_from_j2(j2):
    """J from J (J + 1)."""
    return 0.5 * (-1.0 + np.sqrt(1.0 + 4.0 * np.asarray(j2)))
